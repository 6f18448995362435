"""End-to-end pins of the oracle's trace (Secs. 2.2-2.3 of the paper).

Each check compares the oracle with something other than itself: closed forms
for flat, tilted and quadratic freeforms and for a flat plate under a point
source, energy bookkeeping, numpy's histogram for the box-filter limit, the
paper's scale invariance, and a brute-force scan of the root with scipy's
tensor-product B-spline.
"""
import copy
import math

import numpy as np
import pytest
from scipy.interpolate import NdBSpline

from paper_2302_12031_gb300 import workloads as W

N_GLASS = 1.5
R0 = ((N_GLASS - 1.0) / (N_GLASS + 1.0)) ** 2   # Fresnel reflectance at normal incidence


def _collimated(n_side=64, n_ctrl=8, bins=16, R=1.0):
    wl = W.collimated("t", n_side, n_ctrl, bins, 7, 7, with_target=False)
    wl["target"]["Rx"] = wl["target"]["Ry"] = R
    return wl


def _greville(oracle, n, p):
    U = oracle.knots(n, p)
    return U, np.array([U[i + 1:i + p + 1].mean() for i in range(n + 1)])


def test_flat_lens_gives_uniform_irradiance_T_phi_over_A(oracle):
    wl = _collimated()
    wl["lens"]["P"][:] = 0.013
    E, counts = oracle.trace_forward(wl)
    assert counts[0] == wl["n_rays"]
    # the lit region is [-0.5,0.5]^2 = interior pixels 4..11; one filter
    # radius in from its edge the irradiance is uniform
    h = 1
    inner = E[h + 5:h + 11, h + 5:h + 11]
    expect = (1.0 - R0) ** 2 * 1.0 / (2 * 0.5) ** 2
    assert np.allclose(inner, expect, rtol=1e-12, atol=0)


def test_tilted_plane_compresses_and_deflects(oracle):
    a, b = 0.0, 0.3
    wl = _collimated(bins=16, R=2.0)
    lens = wl["lens"]
    wl["source"]["cols"], wl["source"]["rows"] = 2048, 64
    wl["n_rays"] = 2048 * 64
    _, g = _greville(oracle, lens["n1"], lens["p"])
    P = a + b * (2.0 * g - 1.0) * lens["rx"]
    lens["P"] = np.repeat(P[:, None], lens["n2"] + 1, axis=1)       # Z = a + b x exactly
    beta = math.atan(b)
    theta_t = math.asin(N_GLASS * math.sin(beta))
    dev = theta_t - beta
    kappa = 1.0 - b * math.tan(dev)                                  # dX/dx
    shift = (wl["target"]["z_screen"] - a) * math.tan(dev)
    T = (1.0 - R0) * oracle.schlick_transmission(1.0, N_GLASS, math.cos(theta_t))
    rec = oracle.trace_records(wl, count=4096)
    ok = rec["status"] == 0
    assert ok.all()
    assert np.allclose(rec["X"], kappa * rec["x"] + shift, atol=1e-12)
    assert np.allclose(rec["tx"], math.sin(dev), atol=1e-14)
    assert np.allclose(rec["w"], T / wl["n_rays"], rtol=1e-13)
    E, counts = oracle.trace_forward(wl)
    w = 4.0 / 16
    lo, hi = -0.5 * kappa + shift, 0.5 * kappa + shift
    cols = [i for i in range(16) if lo + 1.5 * w < (i + 0.5) * w - 2.0 < hi - 1.5 * w]
    assert len(cols) >= 1
    # rows: the lit band |y| < 0.5 is interior pixels 6..9; one filter radius in: 7, 8
    inner = E[8:10, [c + 1 for c in cols]]
    assert np.allclose(inner, T / (1.0 * kappa), rtol=1e-4)


def _blossom_quadratic_net(oracle, n, p, r, c):
    """Control points reproducing c*x^2 with x = (2u-1) r (blossoming)."""
    U, g = _greville(oracle, n, p)
    sq = []
    for i in range(n + 1):
        t = U[i + 1:i + p + 1]
        pairs = [t[k] * t[l] for k in range(p) for l in range(k + 1, p)]
        sq.append(np.mean(pairs))                                   # polar form of u^2
    sq = np.array(sq)
    return c * r * r * (4.0 * sq - 4.0 * g + 1.0)


def test_quadratic_freeform_normals_and_hits(oracle):
    c, z0 = 0.15, 0.02
    wl = _collimated(n_side=32, n_ctrl=8, bins=16, R=2.0)
    lens = wl["lens"]
    qx = _blossom_quadratic_net(oracle, lens["n1"], lens["p"], lens["rx"], c)
    qy = _blossom_quadratic_net(oracle, lens["n2"], lens["q"], lens["ry"], c)
    lens["P"] = z0 + qx[:, None] + qy[None, :]
    rng = np.random.default_rng(5)
    for u, v in rng.uniform(0, 1, size=(50, 2)):
        x, y = (2 * u - 1) * lens["rx"], (2 * v - 1) * lens["ry"]
        Z, Zu, Zv = oracle.surface(wl, u, v)[:3]
        assert abs(Z - (z0 + c * (x * x + y * y))) < 1e-14
        assert abs(Zu - 2 * c * x * 2 * lens["rx"]) < 1e-13
        assert abs(Zv - 2 * c * y * 2 * lens["ry"]) < 1e-13
    rec = oracle.trace_records(wl)
    ok = rec["status"] == 0
    assert ok.sum() > 0.9 * len(rec)
    for r in rec[ok]:
        x, y = r["x"], r["y"]
        assert abs(r["z"] - (z0 + c * (x * x + y * y))) < 1e-14
        n = np.array([-2 * c * x, -2 * c * y, 1.0])
        n /= np.linalg.norm(n)
        d = np.array([0.0, 0.0, 1.0])
        t = np.array([r["tx"], r["ty"], r["tz"]])
        assert abs(np.linalg.norm(t) - 1) < 1e-14
        assert np.allclose(N_GLASS * np.cross(d, n), np.cross(t, n), atol=1e-14)
        lam = (wl["target"]["z_screen"] - r["z"]) / t[2]
        assert abs(r["X"] - (x + lam * t[0])) < 1e-12 and abs(r["Y"] - (y + lam * t[1])) < 1e-12


def test_point_source_through_flat_plate(oracle):
    wl = W.point("p", 3000, 8, 32, 1, 11, 1, with_target=False)
    lens = wl["lens"]
    thick = 0.2
    lens["P"][:] = lens["z_in"] + thick
    rec = oracle.trace_records(wl)
    S = np.array(wl["source"]["pos"])
    zs = wl["target"]["z_screen"]
    n_ok = 0
    for rid, r in enumerate(rec):
        if r["status"] != 0:
            continue
        n_ok += 1
        st, o, dg, T1 = oracle.point_ray(wl, rid)
        d0 = (o - S) / np.linalg.norm(o - S)
        # parallel faces: leaves with its incident direction, shifted inside the plate
        sin0 = math.hypot(d0[0], d0[1])
        sing = sin0 / N_GLASS
        tan0, tang = sin0 / d0[2], sing / math.sqrt(1 - sing * sing)
        ax, ay = (d0[0] / sin0, d0[1] / sin0) if sin0 > 0 else (0.0, 0.0)
        rad = tan0 * (lens["z_in"] - S[2]) + tang * thick + tan0 * (zs - lens["z_in"] - thick)
        assert abs(r["X"] - (S[0] + ax * rad)) < 1e-12
        assert abs(r["Y"] - (S[1] + ay * rad)) < 1e-12
        assert abs(r["t"] - thick / math.sqrt(1 - sing * sing)) < 1e-12
        # reciprocal faces: the exit angle in air equals the entry angle
        Ta = oracle.schlick_transmission(1.0, N_GLASS, d0[2])
        assert abs(r["w"] - Ta * Ta / wl["n_rays"]) < 1e-15
    assert n_ok > 2000


@pytest.mark.parametrize("kind", ["collimated", "point"])
def test_energy_bookkeeping(oracle, kind):
    if kind == "collimated":
        wl = W.collimated("c", 128, 8, 32, 1, 2, with_target=False)
        wl["lens"]["P"] = W.control_heights(8, 8, 0.05, 3)
    else:
        wl = W.point("p", 6000, 8, 32, 1, 3, 1, with_target=False)
    E, counts = oracle.trace_forward(wl)
    rec = oracle.trace_records(wl)
    assert counts.sum() == wl["n_rays"]
    for s in range(6):
        assert counts[s] == np.count_nonzero(rec["status"] == s)
    tgt = wl["target"]
    A = (2 * tgt["Rx"] / tgt["nx"]) * (2 * tgt["Ry"] / tgt["ny"])
    on = rec["status"] == 0
    assert abs(E.sum() * A - rec["w"][on].sum()) < 1e-12 * rec["w"][on].sum()
    assert counts[1:].sum() > 0 if kind == "point" else True


def test_box_limit_matches_numpy_histogram(oracle):
    wl = W.collimated("c", 96, 8, 12, 1, 2, with_target=False)
    wl["lens"]["P"] = W.control_heights(8, 8, 0.05, 4)
    wl["target"]["nu_x"] = wl["target"]["nu_y"] = 1
    E, _ = oracle.trace_forward(wl)
    rec = oracle.trace_records(wl)
    on = rec["status"] == 0
    R, n = 1.0, 12
    H, _, _ = np.histogram2d(rec["Y"][on], rec["X"][on], bins=[np.linspace(-R, R, n + 1)] * 2,
                             weights=rec["w"][on])
    A = (2 * R / n) ** 2
    assert np.allclose(E * A, H, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("kind", ["collimated", "point"])
def test_linear_in_flux_and_scale_invariant(oracle, kind):
    if kind == "collimated":
        wl = W.collimated("c", 64, 8, 16, 1, 2, with_target=False)
        wl["lens"]["P"] = W.control_heights(8, 8, 0.03, 5)
    else:
        wl = W.point("p", 3000, 8, 16, 1, 3, 1, with_target=False)
    E, _ = oracle.trace_forward(wl)
    wl2 = copy.deepcopy(wl)
    wl2["source"]["flux"] = 2.5
    E2, _ = oracle.trace_forward(wl2)
    assert np.allclose(E2, 2.5 * E, rtol=1e-13, atol=0)
    s = 2.5
    wl3 = copy.deepcopy(wl)
    for key in ("rx", "ry", "z_in"):
        wl3["lens"][key] *= s
    wl3["lens"]["P"] = wl["lens"]["P"] * s
    for key in ("z_screen", "Rx", "Ry"):
        wl3["target"][key] *= s
    if kind == "point":
        wl3["source"]["pos"] = tuple(s * c for c in wl["source"]["pos"])
    E3, _ = oracle.trace_forward(wl3)
    assert np.allclose(E3 * s * s, E, rtol=1e-11, atol=1e-12 * E.max())


def test_root_is_the_smallest_positive_root(oracle):
    wl = W.point("p", 400, 12, 16, 8, 9, 1, sigma=0.03, with_target=False)
    lens = wl["lens"]
    rec = oracle.trace_records(wl)
    U = oracle.knots(lens["n1"], lens["p"])
    V = oracle.knots(lens["n2"], lens["q"])
    spl = NdBSpline((U, V), lens["P"], 3)
    checked = 0
    for rid in range(0, 400, 7):
        r = rec[rid]
        if r["status"] not in (0, 3, 4):
            continue
        st, o, d, _ = oracle.point_ray(wl, rid)
        ts = np.linspace(0.0, r["t"], 100001)
        u = np.clip((o[0] + d[0] * ts) / (2 * lens["rx"]) + 0.5, 0, 1)
        v = np.clip((o[1] + d[1] * ts) / (2 * lens["ry"]) + 0.5, 0, 1)
        f = spl(np.stack([u, v], axis=1)) - (o[2] + d[2] * ts)
        assert abs(f[-1]) < 1e-12
        assert np.all(f[:-100] > 0.0)             # no earlier crossing
        checked += 1
    assert checked > 20


def _crossings(spl, lens, o, d, t_end, n=20001):
    """f(t) = Z - z on a dense grid of [0, t_end] (scipy's B-spline, not the oracle's)."""
    ts = np.linspace(0.0, t_end, n)
    u = np.clip((o[0] + d[0] * ts) / (2 * lens["rx"]) + 0.5, 0, 1)
    v = np.clip((o[1] + d[1] * ts) / (2 * lens["ry"]) + 0.5, 0, 1)
    return ts, spl(np.stack([u, v], axis=1)) - (o[2] + d[2] * ts)


def test_root_is_the_first_of_several_on_a_wall_lens(oracle):
    # A lens with a wall steeper than the rays: many rays cross the low part,
    # pass under the wall and cross it again. The hit is the first crossing.
    wl = W.wall_lens("wall", 1024)
    lens = wl["lens"]
    rec = oracle.trace_records(wl)
    spl = NdBSpline((oracle.knots(lens["n1"], 3), oracle.knots(lens["n2"], 3)), lens["P"], 3)
    zmax = lens["P"].max()
    several = 0
    for rid in range(1024):
        r = rec[rid]
        st, o, d, _ = oracle.point_ray(wl, rid)
        if st != 0 or r["status"] not in (0, 3, 4):
            continue
        ts, f = _crossings(spl, lens, o, d, (zmax - o[2]) / d[2] * 1.001)
        first = np.argmax(f <= 0.0)
        assert f[first] <= 0.0 and np.all(f[:first] > 0.0)
        assert ts[first - 1] <= r["t"] <= ts[first] + 1e-12       # the first sign change holds the root
        if np.count_nonzero(np.diff(np.sign(f[first:])) != 0) > 0:
            several += 1
    assert several > 50
