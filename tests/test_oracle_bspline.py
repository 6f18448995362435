"""Pins of the oracle's B-spline evaluation (Sec. 2.1 of the paper).

Checked against scipy's independent B-spline routines, the partition of unity,
the clamped end values and the Greville identity that makes X and Y linear.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline, NdBSpline

from paper_2302_12031_gb300 import workloads as W


@pytest.mark.parametrize("n,p", [(7, 3), (15, 3), (5, 2), (9, 5), (3, 3), (31, 3)])
def test_knot_vector_is_clamped_and_equispaced(oracle, n, p):
    U = oracle.knots(n, p)
    assert len(U) == n + p + 2
    assert np.all(U[:p + 1] == 0.0) and np.all(U[-(p + 1):] == 1.0)
    interior = U[p:n + 2]
    assert np.allclose(np.diff(interior), 1.0 / (n - p + 1), atol=1e-15)


@pytest.mark.parametrize("n,p", [(7, 3), (15, 3), (5, 2), (9, 5), (3, 3), (23, 3)])
def test_basis_matches_scipy(oracle, n, p):
    U = oracle.knots(n, p)
    us = np.concatenate([np.linspace(0.0, 1.0, 97), U[p:n + 2], [1e-12, 1.0 - 1e-12]])
    for u in us:
        N, dN = oracle.basis(n, p, u)
        ref = np.array([BSpline(U, np.eye(n + 1)[i], p)(u) for i in range(n + 1)])
        dref = np.array([BSpline(U, np.eye(n + 1)[i], p).derivative()(u) for i in range(n + 1)])
        assert np.allclose(N, ref, atol=1e-14), u
        assert np.allclose(dN, dref, atol=1e-11 * max(1.0, np.abs(dref).max())), u


@pytest.mark.parametrize("n,p", [(7, 3), (12, 4), (9, 5)])
def test_partition_of_unity_and_clamped_ends(oracle, n, p):
    for u in np.linspace(0.0, 1.0, 201):
        N, dN = oracle.basis(n, p, u)
        assert abs(N.sum() - 1.0) < 1e-14
        assert abs(dN.sum()) < 1e-10
        assert np.all(N >= -1e-15)
        assert np.count_nonzero(N > 1e-15) <= p + 1
    N0, _ = oracle.basis(n, p, 0.0)
    N1, _ = oracle.basis(n, p, 1.0)
    assert N0[0] == 1.0 and np.all(N0[1:] == 0.0)
    assert N1[n] == 1.0 and np.all(N1[:n] == 0.0)


@pytest.mark.parametrize("n,p", [(7, 3), (15, 3), (9, 5)])
def test_greville_abscissae_make_X_linear(oracle, n, p):
    U = oracle.knots(n, p)
    g = np.array([U[i + 1:i + p + 1].mean() for i in range(n + 1)])
    rx = 0.37
    for u in np.linspace(0.0, 1.0, 101):
        N, _ = oracle.basis(n, p, u)
        assert abs(np.dot((2.0 * g - 1.0) * rx, N) - (2.0 * u - 1.0) * rx) < 1e-14


def _wl(n_ctrl, p=3, seed=11):
    wl = W.collimated("t", 8, n_ctrl, 8, seed, seed)
    wl["lens"]["p"] = wl["lens"]["q"] = p
    return wl


@pytest.mark.parametrize("n_ctrl,p", [(8, 3), (16, 3), (6, 2), (10, 5)])
def test_surface_and_derivatives_match_scipy_tensor_product(oracle, n_ctrl, p):
    wl = _wl(n_ctrl, p)
    P = wl["lens"]["P"]
    n = n_ctrl - 1
    U = oracle.knots(n, p)
    spl = NdBSpline((U, U), P, p)
    rng = np.random.default_rng(0)
    pts = np.vstack([rng.uniform(0, 1, size=(40, 2)), [[0.0, 0.0], [1.0, 1.0], [0.5, 1.0]]])
    for u, v in pts:
        Z, Zu, Zv, Zuu, Zuv, Zvv = oracle.surface(wl, u, v)
        ref = [spl([[u, v]], nu=nu)[0] for nu in [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]]
        got = [Z, Zu, Zv, Zuu, Zuv, Zvv]
        for k in range(6):
            assert abs(got[k] - ref[k]) < 1e-10 * max(1.0, abs(ref[k])), (k, u, v)


def test_convex_hull_bounds_Z(oracle):
    wl = _wl(12)
    P = wl["lens"]["P"]
    rng = np.random.default_rng(1)
    for u, v in rng.uniform(0, 1, size=(200, 2)):
        Z = oracle.surface(wl, u, v)[0]
        assert P.min() - 1e-15 <= Z <= P.max() + 1e-15
