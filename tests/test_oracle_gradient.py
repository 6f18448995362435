"""Pins of the oracle's gradient dL/dP^z.

* FP64 central finite differences of the oracle's own forward pass, on tiny
  problems where no ray crosses a footprint, screen or TIR event inside the
  step, to 1e-6 relative;
* the paper's conservation statement (Sec. 3.1): on a flat lens under collimated
  light, raising a control point leaves the total irradiance unchanged
  (Schlick's slope is zero at normal incidence), so sum_ij dE_ij/dP = 0;
* the "mountain with a surrounding valley" shape of dE/dP for one control point.
"""
import numpy as np
import pytest

from paper_2302_12031_gb300 import workloads as W


def _events(oracle, wl, P):
    """Per-ray status and centre pixel: the discrete state of every ray."""
    rec = oracle.trace_records(wl, P=P)
    t = wl["target"]
    wx, wy = 2 * t["Rx"] / t["nx"], 2 * t["Ry"] / t["ny"]
    ix = np.floor((rec["X"] + t["Rx"]) / wx)
    iy = np.floor((rec["Y"] + t["Ry"]) / wy)
    # footprint edges: a pixel enters or leaves where |X - c| = nu w / 2
    fx = np.floor((rec["X"] + t["Rx"]) / wx + 0.5)
    fy = np.floor((rec["Y"] + t["Ry"]) / wy + 0.5)
    return np.stack([rec["status"], ix, iy, fx, fy])


def _fd_check(oracle, wl, n_check, seed, h=1e-6, tol=1e-6):
    P0 = wl["lens"]["P"].copy()
    E0, _ = oracle.trace_forward(wl)
    L0, dLdE = oracle.loss_l2(wl, E0)
    g = oracle.trace_gradient(wl, dLdE)
    rng = np.random.default_rng(seed)
    idx = rng.choice(P0.size, size=min(n_check, P0.size), replace=False)
    ev0 = _events(oracle, wl, P0)
    gmax = np.abs(g).max()
    assert gmax > 0
    checked = 0
    for k in idx:
        Pp, Pm = P0.copy().ravel(), P0.copy().ravel()
        Pp[k] += h
        Pm[k] -= h
        Pp, Pm = Pp.reshape(P0.shape), Pm.reshape(P0.shape)
        if not (np.array_equal(_events(oracle, wl, Pp), ev0) and np.array_equal(_events(oracle, wl, Pm), ev0)):
            continue                                    # a ray changes state inside the step
        Lp = oracle.loss_l2(wl, oracle.trace_forward(wl, P=Pp)[0])[0]
        Lm = oracle.loss_l2(wl, oracle.trace_forward(wl, P=Pm)[0])[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g.ravel()[k]) <= tol * gmax, (k, fd, g.ravel()[k])
        checked += 1
    assert checked >= n_check // 2
    return checked


@pytest.mark.parametrize("n_ctrl,p", [(6, 3), (8, 3), (6, 2), (8, 5)])
def test_collimated_gradient_matches_central_differences(oracle, n_ctrl, p):
    wl = W.collimated("c", 20, n_ctrl, 8, 1, 2)
    wl["lens"]["p"] = wl["lens"]["q"] = p
    wl["lens"]["P"] = W.control_heights(n_ctrl, n_ctrl, 0.02, 10 + n_ctrl)
    _fd_check(oracle, wl, 16, seed=n_ctrl)


def test_collimated_jitter_gradient_matches_central_differences(oracle):
    wl = W.collimated("c", 24, 6, 10, 3, 4, jitter=1)
    wl["lens"]["P"] = W.control_heights(6, 6, 0.03, 99)
    _fd_check(oracle, wl, 12, seed=1)


@pytest.mark.parametrize("grid", [(1, 1), (2, 2)])
def test_point_source_gradient_matches_central_differences(oracle, grid):
    wl = W.point("p", 1200, 6, 8, 3, 5, 6, grid=grid, grid_size=(0.1, 0.1), sigma=0.02)
    wl["target"]["Rx"] = wl["target"]["Ry"] = 3.5
    _fd_check(oracle, wl, 16, seed=2)


def test_flat_lens_conserves_total_irradiance(oracle):
    wl = W.collimated("c", 48, 8, 12, 1, 2)
    wl["lens"]["P"][:] = 0.0
    E, counts = oracle.trace_forward(wl)
    assert counts[0] == wl["n_rays"]
    ones = np.ones_like(E)
    g_total = oracle.trace_gradient(wl, ones)
    # scale: the derivative of one central pixel
    onehot = np.zeros_like(E)
    onehot[E.shape[0] // 2, E.shape[1] // 2] = 1.0
    g_pix = oracle.trace_gradient(wl, onehot)
    assert np.abs(g_pix).max() > 1.0
    assert np.abs(g_total).max() < 1e-12 * np.abs(g_pix).max()


def test_control_point_derivative_is_a_mountain_with_a_valley(oracle):
    # Flat lens, collimated light: raising a central control point focuses
    # light into the pixels above it and takes it from a ring around them.
    wl = W.collimated("c", 96, 8, 24, 1, 2)
    wl["lens"]["P"][:] = 0.0
    k = (3, 3)
    h = 1e-6
    Pp = wl["lens"]["P"].copy(); Pp[k] += h
    Pm = wl["lens"]["P"].copy(); Pm[k] -= h
    dE = (oracle.trace_forward(wl, P=Pp)[0] - oracle.trace_forward(wl, P=Pm)[0]) / (2 * h)
    assert abs(dE.sum()) < 1e-6 * np.abs(dE).max()
    # the control point's Greville location on the screen (flat lens: X = x)
    U = oracle.knots(7, 3)
    gx = U[k[0] + 1:k[0] + 4].mean()
    x = (2 * gx - 1) * 0.5
    w = 2.0 / 24
    c = int(np.floor((x + 1.0) / w)) + 1          # extended index of the pixel below it
    assert dE[c, c] > 0.0                            # mountain
    ring = [dE[c + a, c + b] for a in (-4, 4) for b in (-4, 0, 4)] + [dE[c, c - 4], dE[c, c + 4]]
    assert min(ring) < 0.0                           # valley
    # the oracle's reverse-mode pixel gradient agrees with this forward difference
    onehot = np.zeros_like(dE)
    onehot[c, c] = 1.0
    g = oracle.trace_gradient(wl, onehot)
    assert abs(g[k] - dE[c, c]) < 1e-6 * abs(dE[c, c])
