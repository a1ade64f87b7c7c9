"""Pins for the oracle's B-spline basis (§II.A, Eqs. (1)-(3)) and z quadrature.

Every check here is fixed by mathematics outside the oracle: textbook values
of uniform B-splines, partition of unity, Marsden's identity, the integral
identity int B_i = (tau_{i+k} - tau_i)/k, finite differences, and exactness of
Gauss-Legendre for polynomials."""
import numpy as np
import pytest

from oracle import bspline as bs
from paper_1406_4960_gb300 import workloads as W


def _uniform_tau(n, h=1.0):
    # non-clamped uniform knots: every B-spline is a translate of the cardinal one
    return np.arange(n, dtype=np.float64) * h


@pytest.mark.parametrize("order,expected", [
    (2, [1.0]),
    (3, [0.5, 0.5]),
    (4, [1 / 6, 4 / 6, 1 / 6]),
    (6, [1 / 120, 26 / 120, 66 / 120, 26 / 120, 1 / 120]),
])
def test_cardinal_values_at_knots(order, expected):
    """Uniform B-splines at an interior knot take the textbook (Euler-number) values."""
    tau = _uniform_tau(3 * order)
    z = tau[order + 2]
    vals = bs.bsplines(tau, order, z)
    nz = vals[vals > 1e-14]
    assert np.allclose(nz, expected, atol=1e-15, rtol=0)


def test_cardinal_value_mid_interval_cubic():
    """Cubic cardinal B-spline at the middle of its first interval: (1/2)^3/6."""
    tau = _uniform_tau(10)
    vals = bs.bsplines(tau, 4, 0.5)
    assert abs(vals[0] - 0.5 ** 3 / 6) < 1e-15


@pytest.mark.parametrize("breaks", [
    W.uniform_breaks(-10, 10, 37),
    W.slab_geometric_breaks(117),
])
def test_partition_of_unity_and_marsden(breaks):
    order = 6
    tau = bs.clamped_knots(breaks, order)
    greville = np.array([np.mean(tau[i + 1:i + order]) for i in range(len(tau) - order)])
    zs = np.concatenate([breaks, np.linspace(breaks[0], breaks[-1], 97)])
    for z in zs:
        v = bs.bsplines(tau, order, z)
        assert abs(v.sum() - 1.0) < 1e-13
        assert np.all(v >= -1e-15)
        assert abs(greville @ v - z) < 1e-12 * max(1.0, abs(z))


def test_support_and_count():
    breaks = W.uniform_breaks(-3, 3, 7)
    order = 5
    tau = bs.clamped_knots(breaks, order)
    assert len(tau) - order == 7 + order - 1
    for z in np.linspace(-3, 3, 41):
        v = bs.bsplines(tau, order, z)
        assert np.count_nonzero(np.abs(v) > 0) <= order
        for i in np.nonzero(v)[0]:
            assert tau[i] <= z <= tau[i + order]


def test_derivative_matches_finite_differences():
    breaks = W.slab_geometric_breaks(117)
    order = 6
    tau = bs.clamped_knots(breaks, order)
    h = 1e-6
    rng = np.random.default_rng(3)
    for z in rng.uniform(breaks[0] + 0.01, breaks[-1] - 0.01, 25):
        d = bs.bspline_derivs(tau, order, z)
        fd = (bs.bsplines(tau, order, z + h) - bs.bsplines(tau, order, z - h)) / (2 * h)
        scale = max(1.0, np.abs(d).max())
        assert np.abs(d - fd).max() < 2e-6 * scale


def test_derivatives_sum_to_zero():
    tau = bs.clamped_knots(W.uniform_breaks(0, 5, 9), 6)
    for z in np.linspace(0.05, 4.95, 17):
        assert abs(bs.bspline_derivs(tau, 6, z).sum()) < 1e-11


def test_integral_identity_and_quadrature_exactness():
    """int B_i dz = (tau_{i+k} - tau_i)/k (de Boor); Gauss with p=k points per
    interval integrates products of two splines exactly."""
    breaks = W.slab_geometric_breaks(117)
    order = 6
    zb = bs.ZBasis(breaks, order)
    tau = zb.tau
    expect = np.array([(tau[i + order] - tau[i]) / order for i in range(len(tau) - order)])[1:-1]
    integral = zb.wq @ zb.B
    assert np.allclose(integral, expect, rtol=1e-13, atol=1e-15)
    zb2 = bs.ZBasis(breaks, order, nquad=order + 4)
    S1, S2 = zb.overlap(), zb2.overlap()
    D1, D2 = zb.stiffness(), zb2.stiffness()
    assert np.abs(S1 - S2).max() < 1e-14 * np.abs(S1).max()
    assert np.abs(D1 - D2).max() < 1e-12 * np.abs(D1).max()


def test_gauss_legendre_rule():
    zq, wq = bs.quadrature(np.array([0.0, 1.0, 3.0]), 4)
    # int_0^3 z^7 dz = 3^8/8 (degree 7 = 2p-1 is exact)
    assert abs(wq @ zq ** 7 - 3 ** 8 / 8) < 1e-10
    assert abs(wq.sum() - 3.0) < 1e-14


def test_overlap_spd_banded_rowsums():
    breaks = W.uniform_breaks(-10, 10, 37)
    order = 6
    zb = bs.ZBasis(breaks, order)
    S, D = zb.overlap(), zb.stiffness()
    assert np.abs(S - S.T).max() < 1e-16
    assert np.linalg.eigvalsh(S).min() > 0
    assert np.linalg.eigvalsh(D).min() > 0       # end splines dropped: D is SPD
    n = S.shape[0]
    for i in range(n):
        for j in range(n):
            if abs(i - j) >= order:
                assert S[i, j] == 0.0 and D[i, j] == 0.0
    assert np.count_nonzero(S[0, :order]) == order
    # full basis: sum_i' S_ii' = int B_i, sum_i' D_ii' = 0
    tau = zb.tau
    Bfull = np.array([bs.bsplines(tau, order, z) for z in zb.zq])
    dfull = np.array([bs.bspline_derivs(tau, order, z) for z in zb.zq])
    Sf = np.einsum("q,qi,qj->ij", zb.wq, Bfull, Bfull)
    Df = np.einsum("q,qi,qj->ij", zb.wq, dfull, dfull)
    ints = np.array([(tau[i + order] - tau[i]) / order for i in range(len(tau) - order)])
    assert np.allclose(Sf.sum(axis=1), ints, atol=1e-14)
    assert np.abs(Df.sum(axis=1)).max() < 1e-12
