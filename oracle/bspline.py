"""B-spline basis along z (§II.A, Eqs. (1)-(3)).  FP64, plain loops.

Readings (the paper is silent on these):
* the knot sequence is *clamped*: the first and last breakpoints carry
  multiplicity kappa, interior breakpoints multiplicity one;
* the indicator of Eq. (2) is half-open [tau_i, tau_{i+1}), except that the
  last non-empty interval is also closed on the right;
* Eqs. (1)-(2) write ``x`` where they mean ``z`` (a typo);
* zero boundary values: the first and the last B-spline of the clamped basis
  (the only ones non-zero at the ends) are dropped, so "N B-splines" counts the
  retained ones and N = n_int + kappa - 3;
* integrals along z use Gauss-Legendre with ``nquad`` points on every knot
  interval (default nquad = kappa, which integrates B_i B_i' and B_i' B_i'
  exactly).
"""
from __future__ import annotations

import numpy as np


def clamped_knots(breaks, order):
    """Full knot sequence tau: end breakpoints repeated `order` times."""
    b = np.asarray(breaks, dtype=np.float64)
    return np.concatenate([np.full(order - 1, b[0]), b, np.full(order - 1, b[-1])])


def _order1(tau, z):
    """Eq. (2): B_{i,1}(z) = 1 on [tau_i, tau_{i+1}), else 0 (last non-empty
    interval closed on the right)."""
    n = len(tau) - 1
    out = np.zeros(n)
    last = max(i for i in range(n) if tau[i + 1] > tau[i])
    for i in range(n):
        if tau[i] <= z < tau[i + 1]:
            out[i] = 1.0
        elif i == last and z == tau[i + 1]:
            out[i] = 1.0
    return out


def _ratio(num, den):
    return 0.0 if den == 0.0 else num / den


def bsplines_all_orders(tau, order, z):
    """List [B_{.,1}(z), ..., B_{.,order}(z)] by the recursion of Eq. (1).

    Entry m-1 has len(tau) - m values (one per B-spline of order m)."""
    levels = [_order1(tau, z)]
    for m in range(2, order + 1):
        prev = levels[-1]
        n = len(tau) - m
        cur = np.zeros(n)
        for i in range(n):
            left = _ratio(z - tau[i], tau[i + m - 1] - tau[i]) * prev[i]
            right = _ratio(tau[i + m] - z, tau[i + m] - tau[i + 1]) * prev[i + 1]
            cur[i] = left + right
        levels.append(cur)
    return levels


def bsplines(tau, order, z):
    """B_{i,kappa}(z) for every i of the full clamped basis (Eq. (1))."""
    return bsplines_all_orders(tau, order, z)[-1]


def bspline_derivs(tau, order, z):
    """dB_{i,kappa}/dz for every i (Eq. (3))."""
    lower = bsplines_all_orders(tau, order, z)[-2]
    n = len(tau) - order
    d = np.zeros(n)
    k = order
    for i in range(n):
        d[i] = (k - 1) * (_ratio(lower[i], tau[i + k - 1] - tau[i])
                          - _ratio(lower[i + 1], tau[i + k] - tau[i + 1]))
    return d


def quadrature(breaks, nquad):
    """Gauss-Legendre nodes and weights, `nquad` per knot interval.

    Returns (zq, wq) ordered interval by interval."""
    x, w = np.polynomial.legendre.leggauss(nquad)
    b = np.asarray(breaks, dtype=np.float64)
    zs, ws = [], []
    for t in range(len(b) - 1):
        h = b[t + 1] - b[t]
        zs.append(b[t] + 0.5 * h * (x + 1.0))
        ws.append(0.5 * h * w)
    return np.concatenate(zs), np.concatenate(ws)


class ZBasis:
    """Retained B-splines B_j (j = 0..N-1, the full basis minus its two end
    splines), tabulated with their derivatives on the quadrature planes."""

    def __init__(self, breaks, order, nquad=None):
        self.breaks = np.asarray(breaks, dtype=np.float64)
        self.order = int(order)
        self.nquad = int(order if nquad is None else nquad)
        self.tau = clamped_knots(self.breaks, self.order)
        self.n_full = len(self.tau) - self.order
        self.nb = self.n_full - 2
        self.zq, self.wq = quadrature(self.breaks, self.nquad)
        nq = len(self.zq)
        self.B = np.zeros((nq, self.nb))     # B[q][j]
        self.dB = np.zeros((nq, self.nb))
        for q in range(nq):
            self.B[q] = bsplines(self.tau, self.order, self.zq[q])[1:-1]
            self.dB[q] = bspline_derivs(self.tau, self.order, self.zq[q])[1:-1]

    def values(self, z):
        return bsplines(self.tau, self.order, z)[1:-1]

    def overlap(self):
        """S_z[i][i'] = <B_i|B_i'> (Eq. (8)) by the quadrature."""
        return np.einsum("q,qi,qj->ij", self.wq, self.B, self.B)

    def stiffness(self):
        """D_z[i][i'] = <B'_i|B'_i'> (Eq. (9), first term after integration by parts)."""
        return np.einsum("q,qi,qj->ij", self.wq, self.dB, self.dB)

    def weighted(self, f):
        """Sum_q w_q B_i(z_q) B_i'(z_q) f(z_q) for a function f on the planes."""
        fq = np.asarray(f, dtype=np.float64)
        return np.einsum("q,qi,qj->ij", self.wq * fq, self.B, self.B)
