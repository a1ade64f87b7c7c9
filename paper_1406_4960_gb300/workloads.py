"""Seeded synthetic workloads for the mixed-basis slab problem.

This module only *describes inputs*: in-plane cells, atom positions and
pseudopotential parameters, knot breakpoints along z, k-points, cutoffs,
grid shapes and seeded random trial blocks.  It holds none of the method's
arithmetic (no B-splines, no quadrature, no matrix elements), so both the
CPU oracle and the CUDA library can be fed from it without sharing code.

The five workloads stand in for the paper's physical systems (§III:
C(001)-(2x1) slab, graphene and delta-doped graphene), whose pseudopotential
files and relaxed geometries are not available:

* ``tiny``      Gamma point, square cell a=4.7 bohr, Ecut 12 Ha, 16x16 grid,
                40 order-6 B-splines on [-10, 10], two Gaussian wells
                (depth 2 Ha, width 1 bohr) at z=+-1.5, no projectors, 8 bands.
* ``slab``      C(001)-(2x1)-like slab: rectangular 9.5x4.75 bohr cell,
                12 pseudo-atoms in 6 layers 1.7 bohr apart, Ecut 25 Ha,
                32x16 grid, 120 B-splines dense in the slab and geometric
                (ratio 1.15) into +-15 bohr of vacuum, KB s+p projectors,
                2x2 Monkhorst-Pack k-points, 32 bands.
* ``graphene``  4x4 graphene supercell (a=4.65 bohr, 32 atoms), Ecut 30 Ha,
                64x64 grid, 80 B-splines on [-12, 12], Gamma, 80 bands.
* ``kbatch``    2x2 graphene cell, Ecut 30 Ha, 32x32 grid, 100 B-splines on
                [-12, 12], 64 seeded k-points in the irreducible wedge, 24 bands.
* ``serve``     a Poisson stream of requests drawn from the first three.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Project defaults for the synthetic pseudo-atoms (the paper prints no
# parameters for them): local Gaussian amplitude/width and KB strengths.
LOCAL_A_TINY = -2.0        # Ha
LOCAL_A_ATOM = -3.0        # Ha
LOCAL_W = 1.0              # bohr
KB_RC = 1.2                # bohr (alpha = 1/(2 rc^2))
KB_E = (1.0, -0.5, -0.5, -0.5)   # Ha: s, px, py, pz


@dataclasses.dataclass
class Atom:
    pos: Tuple[float, float, float]      # cartesian, bohr
    A: float                             # local Gaussian amplitude, Ha
    w: float                             # local Gaussian width, bohr
    nproj: int = 0                       # 0, 4 (1s, px, py, pz) or 5 (+ 2s)
    E: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)
    rc: float = 1.0                      # KB Gaussian radius, bohr
    e2s: float = 0.0                     # E of the second s channel (nproj == 5), Ha
    e12: float = 0.0                     # 1s-2s coupling E_{12} = E_{21} (nproj == 5), Ha
    Z: float = 0.0                       # core term -Z erf(r/Rcore)/r (0: none)
    Rcore: float = 0.0                   # its radius, bohr
    q: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)   # ultrasoft q of 1s, p_x, p_y, p_z
    q2s: float = 0.0                     # q of the 2s channel (nproj == 5)
    q12: float = 0.0                     # 1s-2s q (nproj == 5)
    rQ: float = 0.0                      # radius of the augmentation Gaussian, bohr


@dataclasses.dataclass
class Workload:
    name: str
    a1: Tuple[float, float]
    a2: Tuple[float, float]
    kpts: np.ndarray                     # (nk, 2) cartesian, 1/bohr
    ecut: float                          # Ha, on |k+G|^2/2
    breaks: np.ndarray                   # strictly increasing z breakpoints, bohr
    order: int                           # B-spline order kappa
    nquad: int                           # Gauss points per knot interval
    grid: Tuple[int, int]                # in-plane FFT grid (n1, n2)
    atoms: List[Atom]
    nbands: int

    @property
    def nk(self) -> int:
        return int(self.kpts.shape[0])

    @property
    def n_int(self) -> int:
        return int(len(self.breaks) - 1)

    @property
    def nb_retained(self) -> int:
        """B-splines kept after the two end splines are dropped."""
        return self.n_int + self.order - 3


def reciprocal(a1, a2):
    """b_i with a_i . b_j = 2 pi delta_ij (a plain lattice fact, used to place k-points)."""
    A = np.array([a1, a2], dtype=np.float64)
    B = 2.0 * np.pi * np.linalg.inv(A).T
    return B[0], B[1]


def uniform_breaks(z0: float, z1: float, n_int: int) -> np.ndarray:
    return np.linspace(z0, z1, n_int + 1)


def slab_geometric_breaks(n_int: int = 117, slab_half: float = 6.0,
                          z_max: float = 15.0, ratio: float = 1.15) -> np.ndarray:
    """Uniform breakpoints over [-slab_half, slab_half], then intervals growing by
    `ratio` outward on both sides, the outermost clipped to end at +-z_max.

    The uniform spacing h0 = 2*slab_half/n_s is chosen by scanning odd n_s until
    the total interval count equals `n_int`.
    """
    for n_s in range(1, 4 * n_int):
        h0 = 2.0 * slab_half / n_s
        outer = []
        z = slab_half
        m = 1
        while z < z_max - 1e-12:
            h = h0 * ratio ** m
            outer.append(min(h, z_max - z))
            z += h
            m += 1
        if outer and outer[-1] < 0.5 * h0 * ratio ** (len(outer) - 1) and len(outer) > 1:
            # a sliver at the end: merge it into its neighbour
            last = outer.pop()
            outer[-1] += last
        if n_s + 2 * len(outer) == n_int:
            inner = np.linspace(-slab_half, slab_half, n_s + 1)
            right = slab_half + np.cumsum(outer)
            right[-1] = z_max
            left = -right[::-1]
            return np.concatenate([left, inner, right])
    raise ValueError("no uniform slab spacing gives %d intervals" % n_int)


def monkhorst_pack(a1, a2, q1: int, q2: int) -> np.ndarray:
    b1, b2 = reciprocal(a1, a2)
    us = [(2 * r - q1 - 1) / (2.0 * q1) for r in range(1, q1 + 1)]
    vs = [(2 * r - q2 - 1) / (2.0 * q2) for r in range(1, q2 + 1)]
    return np.array([u * b1 + v * b2 for u in us for v in vs])


def _hex(a: float):
    return (a, 0.0), (0.5 * a, 0.5 * math.sqrt(3.0) * a)


def _graphene_atoms(a: float, n: int) -> List[Atom]:
    p1, p2 = np.array(_hex(a)[0]), np.array(_hex(a)[1])
    atoms = []
    for i in range(n):
        for j in range(n):
            for f in (1.0 / 3.0, 2.0 / 3.0):
                r = (i + f) * p1 + (j + f) * p2
                atoms.append(Atom((float(r[0]), float(r[1]), 0.0), LOCAL_A_ATOM, LOCAL_W,
                                  4, KB_E, KB_RC))
    return atoms


def tiny() -> Workload:
    rng = np.random.default_rng(0)
    a = 4.7
    a1, a2 = (a, 0.0), (0.0, a)
    atoms = []
    for z in (-1.5, 1.5):
        f = rng.random(2)
        atoms.append(Atom((float(f[0] * a), float(f[1] * a), z), LOCAL_A_TINY, LOCAL_W))
    return Workload("tiny", a1, a2, np.zeros((1, 2)), 12.0,
                    uniform_breaks(-10.0, 10.0, 37), 6, 6, (16, 16), atoms, 8)


def slab() -> Workload:
    rng = np.random.default_rng(1)
    a1, a2 = (9.5, 0.0), (0.0, 4.75)
    atoms = []
    for l in range(6):
        z = -4.25 + 1.7 * l
        for _ in range(2):
            f = rng.random(2)
            atoms.append(Atom((float(f[0] * 9.5), float(f[1] * 4.75), z), LOCAL_A_ATOM,
                              LOCAL_W, 4, KB_E, KB_RC))
    return Workload("slab", a1, a2, monkhorst_pack(a1, a2, 2, 2), 25.0,
                    slab_geometric_breaks(117), 6, 6, (32, 16), atoms, 32)


def graphene() -> Workload:
    a = 4.65
    p1, p2 = _hex(a)
    a1 = (4 * p1[0], 4 * p1[1])
    a2 = (4 * p2[0], 4 * p2[1])
    return Workload("graphene", a1, a2, np.zeros((1, 2)), 30.0,
                    uniform_breaks(-12.0, 12.0, 77), 6, 6, (64, 64),
                    _graphene_atoms(a, 4), 80)


def wedge_kpoints(a1, a2, nk: int, seed: int) -> np.ndarray:
    """Seeded points in the triangle Gamma-M-K of a hexagonal cell."""
    b1, b2 = reciprocal(a1, a2)
    G = np.zeros(2)
    M = 0.5 * b1
    K = (2.0 * b1 + b2) / 3.0
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nk):
        u, v = rng.random(2)
        if u + v > 1.0:
            u, v = 1.0 - u, 1.0 - v
        out.append(G + u * (M - G) + v * (K - G))
    return np.array(out)


def kbatch(nk: int = 64) -> Workload:
    a = 4.65
    p1, p2 = _hex(a)
    a1 = (2 * p1[0], 2 * p1[1])
    a2 = (2 * p2[0], 2 * p2[1])
    return Workload("kbatch", a1, a2, wedge_kpoints(a1, a2, nk, 3), 30.0,
                    uniform_breaks(-12.0, 12.0, 97), 6, 6, (32, 32),
                    _graphene_atoms(a, 2), 24)


def scaled(w: Workload, *, ecut: Optional[float] = None, n_int: Optional[int] = None,
           nbands: Optional[int] = None, kpts: Optional[np.ndarray] = None,
           grid: Optional[Tuple[int, int]] = None, name: Optional[str] = None) -> Workload:
    """A smaller copy of `w` (fewer plane waves / B-splines / bands) for fast tests."""
    breaks = w.breaks
    if n_int is not None and n_int != w.n_int:
        breaks = uniform_breaks(float(w.breaks[0]), float(w.breaks[-1]), n_int)
    return dataclasses.replace(
        w, name=name or (w.name + "-small"),
        ecut=w.ecut if ecut is None else ecut,
        breaks=breaks,
        nbands=w.nbands if nbands is None else nbands,
        kpts=w.kpts if kpts is None else np.asarray(kpts, dtype=np.float64),
        grid=w.grid if grid is None else grid,
        atoms=list(w.atoms))


def with_core(w: Workload, Z: float, Rcore: float, name: Optional[str] = None) -> Workload:
    """A copy of `w` whose atoms also carry the core term -Z erf(r/Rcore)/r."""
    return dataclasses.replace(w, name=name or (w.name + "-core"),
                               atoms=[dataclasses.replace(a, Z=float(Z), Rcore=float(Rcore)) for a in w.atoms])


def with_uspp(w: Workload, q: Tuple[float, float, float, float], rQ: float, q2s: float = 0.0, q12: float = 0.0,
              name: Optional[str] = None) -> Workload:
    """A copy of `w` whose projectors carry ultrasoft augmentation q (the
    overlap S = S_0 + sum q |beta><beta|) with Gaussian charges of radius rQ."""
    return dataclasses.replace(w, name=name or (w.name + "-uspp"),
                               atoms=[dataclasses.replace(a, q=tuple(float(x) for x in q), q2s=float(q2s),
                                                          q12=float(q12), rQ=float(rQ)) for a in w.atoms])


def random_block(nbands: int, nb: int, ng: int, seed: int, ld: Optional[int] = None) -> np.ndarray:
    """Seeded complex trial block X[band][j][G] (unit-variance normal entries).

    Padding columns G >= ng (when ld > ng) are zero.
    """
    ld = ng if ld is None else ld
    rng = np.random.default_rng(seed)
    x = np.zeros((nbands, nb, ld), dtype=np.complex128)
    x[:, :, :ng] = rng.standard_normal((nbands, nb, ng)) + 1j * rng.standard_normal((nbands, nb, ng))
    return x


@dataclasses.dataclass
class Request:
    arrival_s: float
    base: str
    n_int: int
    nbands: int
    nk: int
    seed: int


def serve_stream(n: int = 256, rate_hz: float = 50.0, seed: int = 4) -> List[Request]:
    """Poisson arrivals; each request draws a base workload, a z resolution,
    a band count and a k-point count uniformly."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    bases = ("tiny", "slab", "graphene")
    for i in range(n):
        t += rng.exponential(1.0 / rate_hz)
        base = bases[int(rng.integers(0, 3))]
        nz = int(rng.integers(40, 161))    # retained B-splines
        m = int(rng.integers(8, 81))
        nk = int(rng.integers(1, 9))
        out.append(Request(t, base, nz, m, nk, 1000 + i))
    return out


def random_kpoints(a1, a2, nk: int, seed: int) -> np.ndarray:
    """Seeded k-points uniform in the first cell of the reciprocal lattice."""
    b1, b2 = reciprocal(a1, a2)
    rng = np.random.default_rng(seed)
    u = rng.random((nk, 2)) - 0.5
    return u[:, :1] * b1[None, :] + u[:, 1:] * b2[None, :]


def request_workload(r: Request) -> Workload:
    """The slab problem of a served request: its base workload with the
    request's z resolution (Nz retained B-splines), band count and k-points."""
    base = BY_NAME[r.base]()
    nb = max(r.n_int, base.order + 1)
    n_int = nb - base.order + 3
    if r.base == "slab":
        try:
            breaks = slab_geometric_breaks(n_int)
        except ValueError:
            breaks = uniform_breaks(-15.0, 15.0, n_int)
    else:
        breaks = uniform_breaks(float(base.breaks[0]), float(base.breaks[-1]), n_int)
    return dataclasses.replace(base, name="req-%s" % r.base, breaks=breaks, nbands=r.nbands,
                               kpts=random_kpoints(base.a1, base.a2, r.nk, r.seed))


BY_NAME = {"tiny": tiny, "slab": slab, "graphene": graphene, "kbatch": kbatch}
