"""Forward-mode irradiance derivatives (fr_trace_tangent, the derivative maps of
Sec. 3.1) against the oracle's, element by element on the extended grid.

Tolerance: relative L2 1e-3, the gradient tolerance of the path. As for the
gradient, a ray within rounding of a pixel edge (where the filter's derivative
jumps) or whose status FP32 and FP64 decide differently has two valid one-sided
derivatives; its contribution is taken out of both sides (ambiguous_rays).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2302_12031_gb300 import api
from paper_2302_12031_gb300 import workloads as W
from tests.gpu_helpers import TOL_GRAD, ambiguous_rays, options_for, random_dLdE, rel_l2

pytestmark = pytest.mark.gpu


def tangent_both(wl, dP, begin=0, count=None):
    pb = api.Problem(wl)
    if count is None:
        count = wl["n_rays"] - begin
    opt = options_for(wl)
    g = pb.tangent(dP, opt, ray_begin=begin, ray_count=count).cpu().numpy().astype(np.float64)
    o = O.trace_tangent(wl, dP, begin=begin, count=count)
    amb = ambiguous_rays(wl, begin, count)
    assert len(amb) <= max(3, 2e-3 * count), len(amb)
    for rid in amb:
        g -= pb.tangent(dP, opt, ray_begin=int(rid), ray_count=1).cpu().numpy()
        o -= O.trace_tangent(wl, dP, begin=int(rid), count=1)
    return g, o


def _unit(wl, k, l):
    d = np.zeros_like(wl["lens"]["P"])
    d[k, l] = 1.0
    return d


@pytest.mark.parametrize("kind", ["single", "dense", "three"])
def test_collimated_tangent_matches_oracle(kind):
    wl = W.config(1, with_target=False)
    rng = np.random.default_rng(1)
    shape = wl["lens"]["P"].shape
    if kind == "single":
        dP = _unit(wl, 3, 4)
    elif kind == "dense":
        dP = rng.normal(size=shape)
    else:
        dP = np.stack([_unit(wl, 0, 0), rng.normal(size=shape), _unit(wl, 7, 2)])
    g, o = tangent_both(wl, dP)
    if dP.ndim == 2:
        g, o = g[None], o[None]
    for q in range(g.shape[0]):
        assert np.abs(o[q]).max() > 0
        assert rel_l2(g[q], o[q]) < TOL_GRAD, (q, rel_l2(g[q], o[q]))


@pytest.mark.parametrize("nu", [1, 5])
def test_collimated_tangent_filter_sizes(nu):
    wl = W.collimated("c", 192, 9, 24, 1, 2, with_target=False, jitter=1)
    wl["target"]["nu_x"] = wl["target"]["nu_y"] = nu
    dP = np.random.default_rng(nu).normal(size=wl["lens"]["P"].shape)
    g, o = tangent_both(wl, dP)
    assert rel_l2(g, o) < TOL_GRAD


@pytest.mark.parametrize("grid", [(1, 1), (3, 3)])
def test_point_source_tangent_matches_oracle(grid):
    n = (1 << 16) if grid == (1, 1) else 9 << 13      # a multiple of the number of sources
    wl = W.point("p", n, 12, 32, 3, 4, 5, grid=grid, grid_size=(0.2, 0.2), with_target=False)
    rng = np.random.default_rng(2)
    dP = np.stack([rng.normal(size=wl["lens"]["P"].shape), _unit(wl, 5, 6)])
    g, o = tangent_both(wl, dP)
    for q in range(2):
        assert rel_l2(g[q], o[q]) < TOL_GRAD, (q, rel_l2(g[q], o[q]))


def test_full_size_subrange_matches_oracle():
    wl = W.config(2, with_target=False)
    dP = _unit(wl, 7, 8)
    begin = 1 << 21                                   # rows through the middle of the aperture
    g, o = tangent_both(wl, dP, begin=begin, count=1 << 18)
    assert np.abs(o).max() > 0
    assert rel_l2(g, o) < TOL_GRAD


def test_tangent_is_the_transpose_of_the_adjoint():
    wl = W.config(1, with_target=False)
    pb = api.Problem(wl)
    rng = np.random.default_rng(3)
    dP = rng.normal(size=wl["lens"]["P"].shape)
    gbar = random_dLdE(wl, 4)
    lhs = float(np.sum(gbar * pb.tangent(dP).cpu().numpy()))
    G = pb.adjoint(torch.as_tensor(gbar, dtype=torch.float32, device="cuda")).cpu().numpy()
    rhs = float(np.sum(G * dP))
    assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), abs(rhs))


def test_flat_lens_control_point_map_sums_to_zero():
    wl = W.collimated("c", 1024, 12, 64, 1, 2, with_target=False)
    wl["lens"]["P"][:] = 0.0
    pb = api.Problem(wl)
    stats = api.new_stats()
    t = pb.tangent(_unit(wl, 5, 6), stats=stats).double()
    assert int(stats.cpu()[0]) == wl["n_rays"]          # every ray on the screen
    # the map's total is zero (Sec. 3.1) up to FP32 rounding of its terms
    assert abs(float(t.sum())) < 1e-5 * float(t.abs().sum())
    o = O.trace_tangent(wl, _unit(wl, 5, 6))
    assert rel_l2(t.cpu().numpy(), o) < TOL_GRAD


def test_tangent_argument_errors():
    wl = W.config(1, with_target=False)
    pb = api.Problem(wl)
    h = api.default_handle()
    dP = torch.zeros((33,) + pb.ctrl_shape, device="cuda")
    dE = torch.zeros((33,) + pb.ext_shape, device="cuda")
    for n in (0, 33):
        with pytest.raises(api.FreerayError):
            api.fr_trace_tangent(h, pb.lens, pb.source, pb.target, pb.n_rays, pb.seed, 0, api.ALL_RAYS, None, dP, n,
                                 dE)
    # a direction that moves nothing gives a zero map
    assert float(pb.tangent(dP[0]).abs().max()) == 0.0


@pytest.mark.parametrize("nu", [7, 11])
def test_wide_filter_maps_match_oracle(nu):
    # Sec. 3.1 shows maps with filter sizes 3 and 11: wide filters for the maps
    wl = W.collimated("c", 192, 9, 24, 1, 2, with_target=False, jitter=1)
    wl["target"]["nu_x"] = wl["target"]["nu_y"] = nu
    dP = np.stack([np.random.default_rng(nu).normal(size=wl["lens"]["P"].shape), _unit(wl, 4, 4)])
    g, o = tangent_both(wl, dP)
    for q in range(2):
        assert rel_l2(g[q], o[q]) < TOL_GRAD, (q, rel_l2(g[q], o[q]))


def test_flat_lens_maps_sum_to_zero_for_both_filter_sizes():
    for nu in (3, 11):
        wl = W.collimated("c", 512, 8, 48, 1, 2, with_target=False)
        wl["lens"]["P"][:] = 0.0
        wl["target"]["nu_x"] = wl["target"]["nu_y"] = nu
        t = api.Problem(wl).tangent(_unit(wl, 3, 4)).double()
        # zero up to FP32 rounding of the float-atomic sums: the map's terms
        # cancel to ~1e-5 of their absolute sum
        assert abs(float(t.sum())) < 5e-5 * float(t.abs().sum())


@pytest.mark.parametrize("p,q,nu", [(5, 3, 3), (5, 3, 11), (2, 4, 1), (3, 5, 5)])
def test_other_degree_maps_match_oracle(p, q, nu):
    # Sec. 3.1 shows derivative maps of a degree (5, 3) net beside (3, 3): the
    # general-degree kernel against the oracle's maps (which take any degree)
    wl = W.collimated("c", 192, 9, 24, 1, 2, with_target=False, jitter=1 if q == 5 else 0)
    wl["lens"]["p"], wl["lens"]["q"] = p, q
    wl["target"]["nu_x"] = wl["target"]["nu_y"] = nu
    rng = np.random.default_rng(p * 10 + q)
    dP = np.stack([rng.normal(size=wl["lens"]["P"].shape), _unit(wl, 4, 3), _unit(wl, 0, 8)])
    pb = api.Problem(wl)
    g = pb.tangent(dP).cpu().numpy().astype(np.float64)
    o = O.trace_tangent(wl, dP)
    # the rays within rounding of a pixel edge or of the screen's edge (the
    # debug kernel behind ambiguous_rays takes degree 3 only), out of both sides
    rec = O.trace_records(wl)
    t = wl["target"]
    wx, wy = 2 * t["Rx"] / t["nx"], 2 * t["Ry"] / t["ny"]
    fx = (rec["X"] + t["Rx"] + (nu - 1) / 2 * wx) / wx
    fy = (rec["Y"] + t["Ry"] + (nu - 1) / 2 * wy) / wy
    near = lambda f: np.minimum(f - np.floor(f), np.ceil(f) - f) < 1e-4
    rim = (np.abs(np.abs(rec["X"]) - t["Rx"]) < 1e-4 * wx) | (np.abs(np.abs(rec["Y"]) - t["Ry"]) < 1e-4 * wy)
    amb = np.nonzero(((rec["status"] == 0) & (near(fx) | near(fy))) | rim)[0]
    assert len(amb) <= max(3, 2e-3 * wl["n_rays"]), len(amb)
    for rid in amb:
        g -= pb.tangent(dP, ray_begin=int(rid), ray_count=1).cpu().numpy()
        o -= O.trace_tangent(wl, dP, begin=int(rid), count=1)
    for k in range(3):
        assert rel_l2(g[k], o[k]) < TOL_GRAD, (k, rel_l2(g[k], o[k]))
