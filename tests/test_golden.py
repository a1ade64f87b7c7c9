"""The stored reference eigenvalues under tests/golden/ (each written by a
committed script that calls only oracle/): shapes, ordering, the symmetry the
physics fixes, and -- for the slab -- agreement of two independent oracle
routes: the Lanczos-Krylov iteration (slab_eigs.txt) and the dense
Cholesky-reduced generalized problem solved by LAPACK (slab_eigs_dense.txt)."""
import os

import numpy as np

from paper_1406_4960_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    return [l.split() for l in open(os.path.join(GOLD, name)) if l.strip() and not l.startswith("#")]


def test_slab_golden_shape_and_time_reversal_pairs():
    """The 2x2 Monkhorst-Pack k-points pair up as k3 = -k0 and k2 = -k1, and
    time reversal gives each pair one spectrum."""
    w = W.slab()
    ev = np.array(_rows("slab_eigs.txt"), dtype=float)
    assert ev.shape == (w.nk, w.nbands)
    assert np.all(np.diff(ev, axis=1) >= 0)
    assert np.allclose(w.kpts[3], -w.kpts[0]) and np.allclose(w.kpts[2], -w.kpts[1])
    assert np.abs(ev[0] - ev[3]).max() < 1e-12
    assert np.abs(ev[1] - ev[2]).max() < 1e-12


def test_slab_golden_two_independent_routes_agree():
    """Dense definition (LAPACK on the Cholesky-reduced matrix) vs the
    oracle's Lanczos-Krylov iteration: 1e-9 Ha."""
    lk = np.array(_rows("slab_eigs.txt"), dtype=float)
    dense = _rows("slab_eigs_dense.txt")
    assert len(dense) == 2
    for r in dense:
        ik = int(r[0])
        d = np.array(r[1:], dtype=float)
        assert d.shape == lk[ik].shape
        assert np.abs(d - lk[ik]).max() < 1e-9, (ik, np.abs(d - lk[ik]).max())


def test_kbatch_golden_shape():
    w = W.kbatch()
    rows = _rows("kbatch_eigs.txt")
    assert sorted(int(r[0]) for r in rows) == [0, 3, 23, 40]
    for r in rows:
        ev = np.array(r[1:], dtype=float)
        assert ev.shape == (w.nbands,)
        assert np.all(np.diff(ev) >= 0)


def test_graphene_golden_shape():
    w = W.graphene()
    rows = _rows("graphene_eigs.txt")
    assert len(rows) == 1
    ev = np.array(rows[0], dtype=float)
    assert ev.shape == (w.nbands,)
    assert np.all(np.diff(ev) >= 0)
