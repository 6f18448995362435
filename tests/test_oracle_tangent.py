"""Pins of the oracle's forward-mode irradiance derivative (dE/dP^z) dP, the
derivative maps of Sec. 3.1.

* FP64 central finite differences of the oracle's forward pass along random
  directions, on tiny problems whose rays change no discrete state inside the
  step, to 1e-6 of the map's largest value;
* the duality <g, (dE/dP) dP> = <(dE/dP)^T g, dP> with the reverse-mode gradient;
* the paper's conservation statement (Sec. 3.1): on a flat lens under collimated
  light the map of one control point sums to zero;
* several directions at once equal the directions one by one.
"""
import numpy as np
import pytest

from paper_2302_12031_gb300 import workloads as W
from tests.test_oracle_gradient import _events


def _fd_map(oracle, wl, dP, h):
    P0 = wl["lens"]["P"]
    Ep, _ = oracle.trace_forward(wl, P=P0 + h * dP)
    Em, _ = oracle.trace_forward(wl, P=P0 - h * dP)
    return (Ep - Em) / (2 * h)


def _check_fd(oracle, wl, seed, n_dirs=8, h=3e-7, tol=1e-6):
    rng = np.random.default_rng(seed)
    P0 = wl["lens"]["P"]
    ev0 = _events(oracle, wl, P0)
    checked = 0
    for _ in range(n_dirs):
        dP = rng.normal(size=P0.shape)
        if not (np.array_equal(_events(oracle, wl, P0 + h * dP), ev0)
                and np.array_equal(_events(oracle, wl, P0 - h * dP), ev0)):
            continue
        t = oracle.trace_tangent(wl, dP)
        fd = _fd_map(oracle, wl, dP, h)
        assert np.abs(t).max() > 0
        assert np.abs(fd - t).max() <= tol * np.abs(t).max()
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("n_ctrl", [6, 9])
def test_collimated_tangent_matches_central_differences(oracle, n_ctrl):
    wl = W.collimated("c", 20, n_ctrl, 8, 1, 2)
    wl["lens"]["P"] = W.control_heights(n_ctrl, n_ctrl, 0.02, 20 + n_ctrl)
    _check_fd(oracle, wl, seed=n_ctrl)


@pytest.mark.parametrize("p,q", [(5, 3), (2, 4)])
def test_other_degree_tangent_matches_central_differences(oracle, p, q):
    # Sec. 3.1 shows derivative maps of a degree (5, 3) net beside (3, 3)
    wl = W.collimated("c", 20, 9, 8, 1, 2)
    wl["lens"]["p"], wl["lens"]["q"] = p, q
    wl["lens"]["P"] = W.control_heights(9, 9, 0.02, 40 + p)
    _check_fd(oracle, wl, seed=p)


def test_jittered_collimated_tangent_matches_central_differences(oracle):
    wl = W.collimated("c", 24, 6, 10, 3, 4, jitter=1)
    wl["lens"]["P"] = W.control_heights(6, 6, 0.03, 98)
    _check_fd(oracle, wl, seed=3)


@pytest.mark.parametrize("grid", [(1, 1), (2, 2)])
def test_point_source_tangent_matches_central_differences(oracle, grid):
    wl = W.point("p", 1200, 6, 8, 3, 5, 6, grid=grid, grid_size=(0.1, 0.1), sigma=0.02)
    _check_fd(oracle, wl, seed=4)


def test_tangent_is_the_transpose_of_the_gradient(oracle):
    wl = W.point("p", 3000, 7, 12, 3, 5, 6, sigma=0.02)
    rng = np.random.default_rng(8)
    dP = rng.normal(size=wl["lens"]["P"].shape)
    gbar = rng.normal(size=(14, 14))
    lhs = np.sum(gbar * oracle.trace_tangent(wl, dP))
    rhs = np.sum(oracle.trace_gradient(wl, gbar) * dP)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs), 1.0)


def test_flat_lens_control_point_map_sums_to_zero(oracle):
    wl = W.collimated("c", 48, 8, 12, 1, 2)
    wl["lens"]["P"][:] = 0.0
    for k in ((3, 3), (2, 5), (0, 4)):
        dP = np.zeros_like(wl["lens"]["P"])
        dP[k] = 1.0
        t = oracle.trace_tangent(wl, dP)
        assert np.abs(t).max() > 1.0
        assert abs(t.sum()) < 1e-12 * np.abs(t).max()


def test_several_directions_at_once(oracle):
    wl = W.collimated("c", 16, 6, 8, 1, 2, jitter=1)
    rng = np.random.default_rng(9)
    dPs = rng.normal(size=(3,) + wl["lens"]["P"].shape)
    dPs[1] = 0.0
    dPs[1][2, 3] = 1.0
    many = oracle.trace_tangent(wl, dPs)
    for q in range(3):
        assert np.allclose(many[q], oracle.trace_tangent(wl, dPs[q]), rtol=0, atol=1e-12)
    assert np.allclose(oracle.trace_tangent(wl, 2.0 * dPs[0] - dPs[2]), 2.0 * many[0] - many[2], rtol=0,
                       atol=1e-10)
