"""Pins of the oracle's triangle-mesh intersection (Sec. 2.2.2).

* a planar freeform is its own mesh: every record equals the exact B-spline
  intersection's to FP64 rounding;
* an independent restatement in numpy: mesh heights by barycentric
  interpolation of surface values at the nodes, a dense scan of the ray and
  bisection give the same ray parameter;
* the mesh converges to the B-spline at second order in the cell size;
* the gradient in mesh mode matches central differences.
"""
import numpy as np
import pytest

from paper_2302_12031_gb300 import workloads as W
from tests.test_oracle_gradient import _fd_check


def _point(n_rays=600, n_ctrl=6, sigma=0.02, mesh=(2, 2), seed=3):
    wl = W.point("p", n_rays, n_ctrl, 16, seed, 5, 6, sigma=sigma)
    wl["mesh"] = mesh
    return wl


def test_planar_freeform_mesh_is_exact(oracle):
    wl = _point(n_ctrl=7, mesh=(1, 1))
    n = wl["lens"]["n1"]
    g = oracle.greville(n, 3)
    x = (2 * g - 1) * wl["lens"]["rx"]
    y = (2 * g - 1) * wl["lens"]["ry"]
    X, Y = np.meshgrid(x, y, indexing="ij")
    P = 0.21 + 0.03 * X - 0.02 * Y            # Greville-linear heights: Z is this plane
    exact = dict(wl, mesh=(0, 0))
    for mesh in ((1, 1), (3, 2)):
        m = oracle.trace_records(dict(wl, mesh=mesh), P=P)
        e = oracle.trace_records(exact, P=P)
        assert np.array_equal(m["status"], e["status"])
        ok = e["status"] == 0
        assert ok.sum() > 100
        for f in ("u", "v", "x", "y", "z", "X", "Y", "w", "t"):
            assert np.abs(m[f][ok] - e[f][ok]).max() < 1e-11, f


def _mesh_height_numpy(oracle, wl, NU, NV, u, v):
    K = min(NU - 1, max(0, int(np.floor(u * NU))))
    L = min(NV - 1, max(0, int(np.floor(v * NV))))
    a, b = u * NU - K, v * NV - L
    z = {(c, d): oracle.surface(wl, (K + c) / NU, (L + d) / NV)[0] for c in (0, 1) for d in (0, 1)}
    if a + b < 1:
        return z[0, 0] + (z[1, 0] - z[0, 0]) * a + (z[0, 1] - z[0, 0]) * b
    return z[1, 1] + (z[1, 1] - z[0, 1]) * (a - 1) + (z[1, 1] - z[1, 0]) * (b - 1)


def test_mesh_root_matches_an_independent_scan(oracle):
    wl = _point(n_rays=60, n_ctrl=6, sigma=0.03, mesh=(2, 3))
    NU, NV = 3 * 2, 3 * 3
    rec = oracle.trace_records(wl)
    rx, ry = wl["lens"]["rx"], wl["lens"]["ry"]
    checked = 0
    for rid in np.nonzero(rec["status"] == 0)[0][:25]:
        st, o, d, _ = oracle.point_ray(wl, int(rid))
        assert st == 0
        u = lambda t: (o[0] + d[0] * t) / (2 * rx) + 0.5
        v = lambda t: (o[1] + d[1] * t) / (2 * ry) + 0.5
        f = lambda t: _mesh_height_numpy(oracle, wl, NU, NV, u(t), v(t)) - (o[2] + d[2] * t)
        ts = np.linspace(0.0, 0.5, 2001)
        fs = np.array([f(t) for t in ts])
        k = int(np.argmax(fs <= 0))
        assert fs[k] <= 0 and k > 0
        a, b = ts[k - 1], ts[k]
        for _ in range(60):
            m = 0.5 * (a + b)
            if f(m) > 0:
                a = m
            else:
                b = m
        assert abs(0.5 * (a + b) - rec["t"][rid]) < 1e-12
        checked += 1
    assert checked >= 20


def test_mesh_converges_at_second_order(oracle):
    wl = _point(n_rays=400, n_ctrl=6, sigma=0.03)
    exact = oracle.trace_records(dict(wl, mesh=(0, 0)))
    errs = []
    for n in (2, 4, 8, 16):
        m = oracle.trace_records(dict(wl, mesh=(n, n)))
        ok = (m["status"] == 0) & (exact["status"] == 0)
        errs.append(np.abs(m["z"][ok] - exact["z"][ok]).max())
    ratios = [errs[k] / errs[k + 1] for k in range(3)]
    assert all(3.0 < r < 5.5 for r in ratios), (errs, ratios)


@pytest.mark.parametrize("mesh", [(1, 1), (3, 2)])
def test_mesh_gradient_matches_central_differences(oracle, mesh):
    wl = _point(n_rays=1200, n_ctrl=6, sigma=0.02, mesh=mesh)
    _fd_check(oracle, wl, 16, seed=5)


def test_mesh_tangent_is_the_transpose_of_the_gradient(oracle):
    wl = _point(n_rays=2000, n_ctrl=7, sigma=0.02, mesh=(2, 2))
    rng = np.random.default_rng(1)
    dP = rng.normal(size=wl["lens"]["P"].shape)
    gbar = rng.normal(size=(18, 18))
    lhs = np.sum(gbar * oracle.trace_tangent(wl, dP))
    rhs = np.sum(oracle.trace_gradient(wl, gbar) * dP)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs), 1.0)
