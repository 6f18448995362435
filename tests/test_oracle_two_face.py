"""Pins of the oracle's lens with a freeform entry face (both faces as
B-splines, the extension the paper's conclusion proposes, Sec. 4).

* a flat entry net (all heights z_in) reproduces the flat-face trace;
* Snell's law holds at both faces: the tangential part of n times the
  direction is conserved across each, with each face's own normal;
* a tilted plate (two parallel planar faces) leaves the direction unchanged;
* the gradient with respect to both nets matches central differences;
* forward-mode derivatives are the transpose of the gradient.
"""
import numpy as np
import pytest

from paper_2302_12031_gb300 import workloads as W


def _planar_net(oracle, n, rx, ry, c, a, b):
    """Heights of the plane z = c + a x + b y on an n x n net (Greville-linear)."""
    g = oracle.greville(n - 1, 3)
    X, Y = np.meshgrid((2 * g - 1) * rx, (2 * g - 1) * ry, indexing="ij")
    return c + a * X + b * Y


@pytest.mark.parametrize("kind", ["collimated", "point"])
def test_flat_entry_net_reproduces_the_flat_face(oracle, kind):
    if kind == "collimated":
        wl = W.collimated("c", 24, 7, 12, 1, 2, jitter=1, sigma=0.02)
    else:
        wl = W.point("p", 800, 7, 12, 3, 5, 6, sigma=0.02)
    flat = oracle.trace_records(wl)
    wl2 = W.with_entry_face(wl, 5, 0.0, 1)          # every entry height = z_in
    two = oracle.trace_records(wl2)
    assert np.array_equal(flat["status"], two["status"])
    ok = flat["status"] == 0
    assert ok.sum() > 100
    for f in ("u", "v", "x", "y", "z", "dx", "dy", "dz", "tx", "ty", "tz", "X", "Y", "w"):
        assert np.abs(flat[f][ok] - two[f][ok]).max() < 1e-11, f
    E1, _ = oracle.trace_forward(wl)
    E2, _ = oracle.trace_forward(wl2)
    assert np.abs(E1 - E2).max() < 1e-9 * np.abs(E1).max()


def test_tilted_plate_keeps_the_direction(oracle):
    wl = W.collimated("c", 16, 6, 12, 1, 2)
    lens = wl["lens"]
    wl["lens"]["P"] = _planar_net(oracle, 6, 0.5, 0.5, 0.05, 0.15, -0.1)
    wl = W.with_entry_face(wl, 5, 0.0, 1)
    wl["lens"]["P_in"] = _planar_net(oracle, 5, 0.5, 0.5, -0.1, 0.15, -0.1)
    rec = oracle.trace_records(wl)
    ok = rec["status"] == 0
    assert ok.sum() > 200
    assert np.abs(rec["tx"][ok]).max() < 1e-12 and np.abs(rec["ty"][ok]).max() < 1e-12
    # Schlick at both faces, at the plate's incidence angle
    n = lens["n_glass"]
    m = np.array([-0.15, 0.1, 1.0]) / np.linalg.norm([-0.15, 0.1, 1.0])
    ci = m[2]
    ct = np.sqrt(1 - (1 - ci ** 2) / n ** 2)
    R0 = ((n - 1) / (n + 1)) ** 2
    T1 = 1 - (R0 + (1 - R0) * (1 - ci) ** 5)          # incident cosine in air
    T2 = 1 - (R0 + (1 - R0) * (1 - ci) ** 5)          # leaving: the cosine in air is again ci
    w0 = 1.0 / wl["n_rays"]
    assert np.allclose(rec["w"][ok], w0 * T1 * T2, rtol=1e-12, atol=0)
    # inside the plate the ray makes the refracted angle with the normal
    dm = rec["dx"][ok] * m[0] + rec["dy"][ok] * m[1] + rec["dz"][ok] * m[2]
    assert np.abs(dm - ct).max() < 1e-12


@pytest.mark.parametrize("kind", ["collimated", "point"])
def test_snell_invariants_at_both_faces(oracle, kind):
    if kind == "collimated":
        wl = W.collimated("c", 20, 6, 12, 1, 2, sigma=0.02)
    else:
        wl = W.point("p", 600, 6, 12, 3, 5, 6, sigma=0.02)
    wl = W.with_entry_face(wl, 5, 0.02, 9)
    entry_as_exit = dict(wl, lens=dict(wl["lens"], P=wl["lens"]["P_in"], n1=4, n2=4))
    rec = oracle.trace_records(wl)
    ok = np.nonzero(rec["status"] == 0)[0]
    assert len(ok) > 100
    n = wl["lens"]["n_glass"]
    rx, ry = wl["lens"]["rx"], wl["lens"]["ry"]

    def normal(w, u, v):
        S = oracle.surface(w, u, v)
        m = np.array([-S[1] / (2 * rx), -S[2] / (2 * ry), 1.0])
        return m / np.linalg.norm(m)

    for r in ok[:40]:
        d = np.array([rec["dx"][r], rec["dy"][r], rec["dz"][r]])
        t = np.array([rec["tx"][r], rec["ty"][r], rec["tz"][r]])
        assert abs(np.linalg.norm(d) - 1) < 1e-12 and abs(np.linalg.norm(t) - 1) < 1e-12
        # exit face: n d x m = t x m with the exit normal at the hit
        m = normal(wl, rec["u"][r], rec["v"][r])
        assert np.abs(n * np.cross(d, m) - np.cross(t, m)).max() < 1e-11
        if kind == "collimated":
            # entry face, at the ray's grid cell centre: d0 x m_in = n d x m_in
            cols = wl["source"]["cols"]
            u0, v0 = (r % cols + 0.5) / cols, (r // cols + 0.5) / cols
            m_in = normal(entry_as_exit, u0, v0)
            assert np.abs(np.cross([0.0, 0.0, 1.0], m_in) - n * np.cross(d, m_in)).max() < 1e-11
            # and the in-glass ray from the entry point reaches the exit hit
            o = np.array([(2 * u0 - 1) * rx, (2 * v0 - 1) * ry, oracle.surface(entry_as_exit, u0, v0)[0]])
            x = np.array([rec["x"][r], rec["y"][r], rec["z"][r]])
            assert np.linalg.norm(np.cross(x - o, d)) < 1e-11


def _fd_two_face(oracle, wl, n_check, seed, h=1e-6, tol=1e-6):
    E0, _ = oracle.trace_forward(wl)
    rng = np.random.default_rng(seed)
    gbar = rng.normal(size=E0.shape)
    g_out, g_in = oracle.trace_gradient(wl, gbar)
    P, Pin = wl["lens"]["P"], wl["lens"]["P_in"]
    scale = max(np.abs(g_out).max(), np.abs(g_in).max())
    rec0 = oracle.trace_records(wl)["status"]
    checked = 0
    for face, arr, g in (("out", P, g_out), ("in", Pin, g_in)):
        for k in rng.choice(arr.size, size=n_check, replace=False):
            dp = np.zeros(arr.size)
            dp[k] = h
            dp = dp.reshape(arr.shape)
            kw_p = {"P": P + dp} if face == "out" else {"P_in": Pin + dp}
            kw_m = {"P": P - dp} if face == "out" else {"P_in": Pin - dp}
            if not (np.array_equal(oracle.trace_records(wl, **kw_p)["status"], rec0)
                    and np.array_equal(oracle.trace_records(wl, **kw_m)["status"], rec0)):
                continue
            fd = (np.sum(gbar * oracle.trace_forward(wl, **kw_p)[0])
                  - np.sum(gbar * oracle.trace_forward(wl, **kw_m)[0])) / (2 * h)
            assert abs(fd - g.ravel()[k]) <= tol * scale, (face, k, fd, g.ravel()[k])
            checked += 1
    assert checked >= n_check


@pytest.mark.parametrize("kind", ["collimated", "point"])
def test_two_face_gradient_matches_central_differences(oracle, kind):
    if kind == "collimated":
        wl = W.collimated("c", 20, 6, 8, 1, 2, jitter=1, sigma=0.02)
    else:
        wl = W.point("p", 1000, 6, 8, 3, 5, 6, sigma=0.02)
    wl = W.with_entry_face(wl, 5, 0.02, 9)
    _fd_two_face(oracle, wl, 8, seed=3)


def test_two_face_tangent_is_the_transpose_of_the_gradient(oracle):
    wl = W.with_entry_face(W.point("p", 1500, 7, 10, 3, 5, 6, sigma=0.02), 6, 0.02, 4)
    rng = np.random.default_rng(2)
    n = wl["lens"]["P"].size + wl["lens"]["P_in"].size
    dP = rng.normal(size=n)
    gbar = rng.normal(size=(12, 12))
    lhs = np.sum(gbar * oracle.trace_tangent(wl, dP))
    g_out, g_in = oracle.trace_gradient(wl, gbar)
    rhs = np.sum(np.concatenate([g_out.ravel(), g_in.ravel()]) * dP)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs), 1.0)
