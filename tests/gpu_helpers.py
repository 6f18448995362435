"""Shared helpers of the GPU parity tests (comparison against the FP64 oracle).

Tolerances (from the measurement plan): per-ray hit points 1e-5 relative,
irradiance 1e-4 relative L2, control-point gradients 1e-3 relative L2.
Relative errors of positions are taken against the larger of the value and the
geometric scale (lens half-width on the freeform, screen half-width on the
screen), because a coordinate near 0 has no relative precision.
"""
import numpy as np
import torch

from oracle import oracle as O
from paper_2302_12031_gb300 import api

TOL_HIT = 1e-5
TOL_E = 1e-4
TOL_GRAD = 1e-3


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def options_for(wl, **kw):
    """fr_options matching the workload's intersection (wl["mesh"] for the oracle)."""
    return api.make_options(mesh=tuple(wl.get("mesh", (0, 0))), **kw)


def compare_records(wl, begin, count, min_agree=0.999):
    """GPU debug records vs oracle records on rays [begin, begin+count)."""
    pb = api.Problem(wl)
    g = pb.debug(begin, count, options=options_for(wl))
    o = O.trace_records(wl, begin=begin, count=count)
    agree = g["status"] == o["status"]
    assert agree.mean() >= min_agree, (agree.mean(), np.unique(g["status"][~agree]), np.unique(o["status"][~agree]))
    ok = agree & (o["status"] == 0)
    assert ok.sum() > 0
    lens, tgt = wl["lens"], wl["target"]
    scale_hit = max(lens["rx"], lens["ry"])
    R = max(tgt["Rx"], tgt["Ry"])
    worst = {}
    for f, scale in (("x", scale_hit), ("y", scale_hit), ("z", scale_hit), ("X", R), ("Y", R),
                     ("u", 1.0), ("v", 1.0)):
        d = np.abs(g[f][ok].astype(np.float64) - o[f][ok]) / np.maximum(np.abs(o[f][ok]), scale)
        worst[f] = float(d.max())
        assert worst[f] < TOL_HIT, (f, worst[f])
    for f in ("tx", "ty", "tz", "dx", "dy", "dz"):
        d = np.abs(g[f][ok].astype(np.float64) - o[f][ok])
        worst[f] = float(d.max())
        assert worst[f] < TOL_HIT, (f, worst[f])
    dw = np.abs(g["w"][ok].astype(np.float64) - o["w"][ok]) / o["w"][ok]
    worst["w"] = float(dw.max())
    assert worst["w"] < TOL_HIT, worst["w"]
    # the knot span of every on-screen hit is the oracle's, except on a knot
    span_ok = (g["span_i"][ok] == o["span_i"][ok]) & (g["span_j"][ok] == o["span_j"][ok])
    assert span_ok.mean() > 0.999
    return worst, g, o


def forward_both(wl, begin=0, count=None, options=None):
    """GPU and oracle irradiance (and ray counts) over rays [begin, begin+count).

    With nu = 1 the filter is the box indicator and E jumps where a ray crosses
    a pixel edge; there the contributions of ambiguous rays (see ambiguous_rays)
    are taken out of both sides. For nu >= 3, E is continuous and nothing is."""
    pb = api.Problem(wl)
    stats = api.new_stats()
    if count is None:
        count = wl["n_rays"] - begin
    if options is None:
        options = options_for(wl)
    E = pb.forward(options, ray_begin=begin, ray_count=count, stats=stats).cpu().numpy().astype(np.float64)
    E_or, counts = O.trace_forward(wl, begin=begin, count=count)
    if wl["target"]["nu_x"] == 1 and count > 0:
        for rid in ambiguous_rays(wl, begin, count):
            E -= pb.forward(options, ray_begin=int(rid), ray_count=1).cpu().numpy()
            E_or -= O.trace_forward(wl, begin=int(rid), count=1)[0]
    return E, E_or, stats.cpu().numpy(), counts


def ambiguous_rays(wl, begin, count, eps_px=1e-4):
    """Rays whose discrete state FP32 and FP64 may decide differently.

    The irradiance is continuous where a ray's footprint moves to the next pixel
    or the ray crosses the edge of the screen, but its derivative jumps there
    (the filter is only C0 at its support edge). For a ray within rounding of
    such an edge the gradient has two valid one-sided values, so gradient parity
    is checked on the other rays: those whose status differs between the two
    sides, or whose hit lies within eps_px pixels of a pixel edge.
    """
    g = api.Problem(wl).debug(begin, count, options=options_for(wl))
    o = O.trace_records(wl, begin=begin, count=count)
    t = wl["target"]
    wx, wy = 2 * t["Rx"] / t["nx"], 2 * t["Ry"] / t["ny"]
    hx, hy = (t["nu_x"] - 1) / 2, (t["nu_y"] - 1) / 2
    fx = (o["X"] + t["Rx"] + hx * wx) / wx
    fy = (o["Y"] + t["Ry"] + hy * wy) / wy
    near = lambda f: np.minimum(f - np.floor(f), np.ceil(f) - f) < eps_px
    amb = (g["status"] != o["status"]) | ((o["status"] == 0) & (near(fx) | near(fy)))
    mesh = wl.get("mesh", (0, 0))
    if mesh[0] > 0 and wl["source"]["kind"] == "point":
        # on the triangle mesh t*(P) has a kink on every triangle edge
        lens = wl["lens"]
        NU, NV = (lens["n1"] - 2) * mesh[0], (lens["n2"] - 2) * mesh[1]
        a, b = o["u"] * NU, o["v"] * NV
        a, b = a - np.floor(a), b - np.floor(b)
        edge = np.minimum.reduce([a, 1 - a, b, 1 - b, np.abs(a + b - 1)]) < 1e-4
        amb |= (o["status"] == 0) & edge
    return begin + np.nonzero(amb)[0]


def adjoint_both(wl, dLdE, begin=0, count=None, options=None, exclude_ambiguous=True):
    """GPU and oracle dL/dP over rays [begin, begin+count), without the
    contributions of ambiguous rays (see ambiguous_rays) on either side."""
    pb = api.Problem(wl)
    if count is None:
        count = wl["n_rays"] - begin
    if options is None:
        options = options_for(wl)
    d = torch.as_tensor(dLdE, dtype=torch.float32, device="cuda")
    g = pb.adjoint(d, options, ray_begin=begin, ray_count=count).cpu().numpy().astype(np.float64)
    g_or = O.trace_gradient(wl, dLdE, begin=begin, count=count)
    if exclude_ambiguous:
        amb = ambiguous_rays(wl, begin, count)
        assert len(amb) <= max(3, 2e-3 * count), len(amb)
        for rid in amb:
            g -= pb.adjoint(d, options, ray_begin=int(rid), ray_count=1).cpu().numpy()
            g_or -= O.trace_gradient(wl, dLdE, begin=int(rid), count=1)
    return g, g_or


def oracle_dLdE(wl, begin=0, count=None):
    """dL/dE of the squared-L2 loss at the oracle's own irradiance."""
    E_or, _ = O.trace_forward(wl, begin=begin, count=count)
    _, d = O.loss_l2(wl, E_or)
    return d


def random_dLdE(wl, seed):
    """A seeded dL/dE on the extended grid with zero ghost pixels."""
    t = wl["target"]
    ny, nx, hx, hy = t["ny"], t["nx"], (t["nu_x"] - 1) // 2, (t["nu_y"] - 1) // 2
    rng = np.random.default_rng(seed)
    d = np.zeros((ny + 2 * hy, nx + 2 * hx))
    d[hy:hy + ny, hx:hx + nx] = rng.normal(size=(ny, nx))
    return d
