"""The seeded synthetic inputs: basis sizes, knot structure, k-points.

These are the shapes the benchmark and the parity tests run on (the cells
that stand in for the paper's C(001) slab, graphene and k-point scans); the
counts of plane waves come from the oracle's own cutoff sphere (Eq. 6), so a
change to the recipe or to the cutoff rule shows up here first."""
import math

import numpy as np
import pytest

from oracle import hamiltonian as Hm
from paper_1406_4960_gb300 import workloads as W


def _spheres(w):
    """(nb, [G index array of every k-point]) from one oracle model, its
    cutoff sphere re-evaluated at each k (the z basis does not depend on k)."""
    m = Hm.Model(w.a1, w.a2, w.kpts[0], w.ecut, w.breaks, w.order, [], w.grid, w.nquad)
    out = []
    for ik in range(w.nk):
        m.k = np.asarray(w.kpts[ik], dtype=np.float64)
        m._sphere()
        out.append(m.gidx.copy())
    return m.nb, out


# name: (k-points, G per k (min, max), B-splines, intervals, grid, atoms, projectors, bands)
SIZES = {
    "tiny": (1, (45, 45), 40, 37, (16, 16), 2, 0, 8),
    "slab": (4, (179, 179), 120, 117, (32, 16), 12, 48, 32),
    "graphene": (1, (1417, 1417), 80, 77, (64, 64), 32, 128, 80),
    "kbatch": (64, (352, 361), 100, 97, (32, 32), 8, 32, 24),
}


@pytest.mark.parametrize("name", list(SIZES))
def test_workload_sizes(name):
    nk, (gmin, gmax), nb, n_int, grid, natoms, nproj, nbands = SIZES[name]
    w = W.BY_NAME[name]()
    assert (w.nk, w.n_int, w.nb_retained, tuple(w.grid), len(w.atoms), w.nbands) == (nk, n_int, nb, grid, natoms, nbands)
    assert sum(a.nproj for a in w.atoms) == nproj
    assert (w.order, w.nquad) == (6, 6)
    mnb, gidx = _spheres(w)
    assert mnb == nb
    ngs = [len(g) for g in gidx]
    assert gmin == min(ngs) and max(ngs) == gmax
    for g in gidx:
        # the FFT grid holds the whole disc of G indices without overlap
        span = g.max(axis=0) - g.min(axis=0) + 1
        assert span[0] <= grid[0] and span[1] <= grid[1]


def test_slab_knots_are_uniform_inside_and_geometric_outside():
    z = W.slab().breaks
    h = np.diff(z)
    assert z[0] == pytest.approx(-15.0) and z[-1] == pytest.approx(15.0)
    assert np.all(h > 0)
    inner = (z[:-1] >= -6.0 - 1e-9) & (z[1:] <= 6.0 + 1e-9)
    h0 = h[inner]
    assert np.ptp(h0) < 1e-12 * h0[0]                      # one spacing across the slab
    right = h[z[:-1] >= 6.0 - 1e-9]
    ratios = right[1:-1] / right[:-2]                     # the last interval is clipped at the box edge
    assert np.allclose(ratios, 1.15, rtol=1e-12)
    assert right[0] == pytest.approx(1.15 * h0[0], rel=1e-12)
    assert np.allclose(h, h[::-1], rtol=1e-12)            # symmetric about z = 0


def test_kbatch_kpoints_lie_in_the_first_zone_and_are_distinct():
    w = W.kbatch()
    b1, b2 = W.reciprocal(w.a1, w.a2)
    shells = [i * b1 + j * b2 for i in range(-2, 3) for j in range(-2, 3) if (i, j) != (0, 0)]
    for k in w.kpts:
        for G in shells:                                  # nearer to Gamma than to any other lattice point
            assert np.linalg.norm(k) <= np.linalg.norm(k - G) + 1e-12
    d = np.linalg.norm(w.kpts[:, None, :] - w.kpts[None, :, :], axis=-1)
    assert np.min(d + np.eye(w.nk)) > 1e-9
    assert np.array_equal(w.kpts, W.kbatch().kpts)        # seeded


def test_random_blocks_are_seeded_and_shaped():
    a = W.random_block(3, 10, 7, seed=5, ld=8)
    b = W.random_block(3, 10, 7, seed=5, ld=8)
    c = W.random_block(3, 10, 7, seed=6, ld=8)
    assert a.shape == (3, 10, 8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.all(a[:, :, 7:] == 0)                       # padding beyond the disc is zero
    assert math.isfinite(float(np.abs(a).max()))
