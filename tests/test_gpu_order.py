"""The coherent ray order of point sources (fr_ray_order, fr_options.ray_order).

The order is a permutation of the ray ids: the H rays that meet the aperture
first, grouped by source and sorted by entry-plane cell, then the misses.
Tracing in it sums over the same rays, so deterministic mode gives
bit-identical irradiance, gradients and counts (float mode agrees to FP32
summation order), and neighbouring positions are neighbouring rays.
"""
import numpy as np
import pytest
import torch

from paper_2302_12031_gb300 import api, step
from paper_2302_12031_gb300 import workloads as W
from tests.gpu_helpers import TOL_E, TOL_GRAD, forward_both, random_dLdE, rel_l2

pytestmark = pytest.mark.gpu


def _wl(n_rays=9 * 12000, grid=(1, 1), bins=64, mesh=None):
    wl = W.point("o", n_rays, 12, bins, 4, 9, 6, grid=grid, grid_size=(0.2, 0.2), sigma=0.02)
    if mesh:
        wl["mesh"] = mesh
    return wl


def _opts(wl, order=None, **kw):
    return api.make_options(mesh=tuple(wl.get("mesh", (0, 0))), ray_order=order, **kw)


@pytest.mark.parametrize("n_rays,grid", [(100003, (1, 1)), (9 * 12000, (3, 3)), (1 << 20, (1, 1)), (7, (1, 1))])
def test_order_is_a_permutation(n_rays, grid):
    wl = _wl(n_rays, grid)
    pb = api.Problem(wl)
    full = pb.ray_order().cpu().numpy().astype(np.int64)
    order, H = full[:n_rays], int(full[n_rays])
    assert np.array_equal(np.sort(order), np.arange(n_rays))
    assert 0 <= H <= n_rays
    if grid != (1, 1):          # the hits grouped by source: source index never decreases
        assert np.all(np.diff(order[:H] // (n_rays // (grid[0] * grid[1]))) >= 0)
    if n_rays <= 1 << 17:       # the rays placed last miss the aperture; nearly all others meet it
        rec = pb.debug(0, n_rays)
        assert np.all(rec["status"][order[H:]] == 1)
        assert np.mean(rec["status"][order[:H]] == 1) < 1e-3


def test_order_is_coherent():
    wl = _wl(1 << 17)
    pb = api.Problem(wl)
    order = pb.ray_order().cpu().numpy().astype(np.int64)[:wl["n_rays"]]
    rec = pb.debug(0, wl["n_rays"])
    ok = rec["status"] == 0
    span = rec["span_i"] * 64 + rec["span_j"]
    # neighbouring positions of the order share the knot span far more often than neighbouring ids
    so, sid = span[order], span
    oko, okid = ok[order], ok
    same_order = np.mean((so[1:] == so[:-1])[oko[1:] & oko[:-1]])
    same_id = np.mean((sid[1:] == sid[:-1])[okid[1:] & okid[:-1]])
    assert same_order > 0.8 and same_id < 0.1, (same_order, same_id)
    # and the entry points run in cells: the hits of a run of 64 positions are close together
    x, y = rec["x"][order], rec["y"][order]
    d = np.hypot(x[64:] - x[:-64], y[64:] - y[:-64])[oko[64:] & oko[:-64]]
    assert np.median(d) < 0.05


@pytest.mark.parametrize("grid,mesh", [((1, 1), None), ((3, 3), None), ((1, 1), (2, 2))])
def test_deterministic_results_do_not_depend_on_the_order(grid, mesh):
    wl = _wl(9 * 12000, grid, mesh=mesh)
    pb = api.Problem(wl)
    order = pb.ray_order()
    d = torch.as_tensor(random_dLdE(wl, 5), dtype=torch.float32, device="cuda")
    s0, s1 = api.new_stats(), api.new_stats()
    E0 = pb.forward(_opts(wl, deterministic=True), stats=s0)
    E1 = pb.forward(_opts(wl, order, deterministic=True), stats=s1)
    assert torch.equal(E0, E1) and torch.equal(s0, s1)
    g0 = pb.adjoint(d, _opts(wl, deterministic=True))
    g1 = pb.adjoint(d, _opts(wl, order, deterministic=True))
    assert torch.equal(g0, g1)


def test_float_results_in_order_match_the_oracle():
    wl = _wl(9 * 20000, (3, 3))
    pb = api.Problem(wl)
    order = pb.ray_order()
    E, E_or, st, counts = forward_both(wl, options=_opts(wl, order))
    assert rel_l2(E, E_or) < TOL_E
    E_id = pb.forward(_opts(wl)).double().cpu().numpy()
    assert rel_l2(E, E_id) < 1e-5
    d = torch.as_tensor(random_dLdE(wl, 2), dtype=torch.float32, device="cuda")
    g = pb.adjoint(d, _opts(wl, order)).double().cpu().numpy()
    g_id = pb.adjoint(d, _opts(wl)).double().cpu().numpy()
    assert rel_l2(g, g_id) < 1e-5
    from oracle import oracle as O
    assert rel_l2(g, O.trace_gradient(wl, d.double().cpu().numpy())) < TOL_GRAD


def test_derivative_maps_in_order():
    wl = _wl(60000)
    pb = api.Problem(wl)
    order = pb.ray_order()
    dP = torch.randn((2,) + pb.ctrl_shape, generator=torch.Generator().manual_seed(3)).cuda()
    a = pb.tangent(dP, options=_opts(wl, order)).double().cpu().numpy()
    b = pb.tangent(dP, options=_opts(wl)).double().cpu().numpy()
    assert rel_l2(a, b) < 1e-5


def test_order_refusals():
    wl = _wl(9000)
    pb = api.Problem(wl)
    order = pb.ray_order()
    with pytest.raises(api.FreerayError):
        pb.forward(_opts(wl, order), ray_begin=10, ray_count=100)          # not all rays
    wc = W.collimated("c", 64, 8, 16, 1, 2)
    pc = api.Problem(wc)
    with pytest.raises(api.FreerayError):
        pc.forward(_opts(wc, torch.zeros(64 * 64 + 1, dtype=torch.int32, device="cuda")))
    with pytest.raises(api.FreerayError):
        pc.ray_order()


def test_step_in_order_matches_id_order():
    wl = _wl(9 * 12000, (3, 3))
    wl["E_ref"] = W.gaussian_mixture_target(64, 64, wl["target"]["Rx"], wl["target"]["Ry"], 6, 0.3)
    kw = dict(lr=1e-3, options=api.make_options(deterministic=True))
    a = step.OptimStep(wl, ray_order=True, **kw)
    b = step.OptimStep(wl, ray_order=False, **kw)
    assert a.order is not None and b.order is None
    for _ in range(3):
        a.step()
        b.step()
    torch.cuda.synchronize()
    assert torch.equal(a.P, b.P) and torch.equal(torch.stack(a.loss), torch.stack(b.loss))


def test_batch_with_orders_and_windows():
    # a batch of point lenses (ordered, grids too large for shared memory: windows)
    # and a collimated lens: deterministic results equal the unordered ones bit
    # for bit; float results (windows, orders) agree with them and the oracle
    wls = [_wl(9 * 6000, (3, 3), bins=200), _wl(40000, bins=150), W.collimated("c", 200, 9, 180, 5, 6)]
    pbs = [api.Problem(w) for w in wls]
    orders = [pbs[0].ray_order(), pbs[1].ray_order(), None]
    h = api.default_handle()
    Es = {}
    for label, det, use in (("det", True, False), ("det_order", True, True), ("float", False, True)):
        E = [torch.zeros(pb.ext_shape, device="cuda") for pb in pbs]
        items = [pb.batch_item(E=e, ray_order=o if use else None) for pb, e, o in zip(pbs, E, orders)]
        api.fr_trace_batch_forward(h, items, api.make_options(deterministic=det))
        Es[label] = [e.double().cpu().numpy() for e in E]
    for a, b in zip(Es["det"], Es["det_order"]):
        assert np.array_equal(a, b)
    for a, b in zip(Es["float"], Es["det"]):
        assert rel_l2(a, b) < 1e-5
    from oracle import oracle as O
    for w, e in zip(wls, Es["float"]):
        assert rel_l2(e, O.trace_forward(w)[0]) < TOL_E
    ds = [torch.as_tensor(random_dLdE(w, 4), dtype=torch.float32, device="cuda") for w in wls]
    gs = {}
    for label, det, use in (("det", True, False), ("det_order", True, True), ("float", False, True)):
        G = [torch.zeros(pb.ctrl_shape, device="cuda") for pb in pbs]
        items = [pb.batch_item(dLdE=d, dLdP=g, ray_order=o if use else None) for pb, d, g, o in zip(pbs, ds, G, orders)]
        api.fr_trace_batch_adjoint(h, items, api.make_options(deterministic=det))
        gs[label] = [g.double().cpu().numpy() for g in G]
    for a, b in zip(gs["det"], gs["det_order"]):
        assert np.array_equal(a, b)
    for a, b in zip(gs["float"], gs["det"]):
        assert rel_l2(a, b) < 1e-5


def test_two_face_point_lens_in_order():
    # a freeform entry face: every position is traced (H = n_rays), the entry
    # face decides the aperture; deterministic results equal the id order's
    wl = W.with_entry_face(_wl(9 * 8000, (3, 3)), 8, 0.01, 5)
    pb = api.Problem(wl)
    full = pb.ray_order()
    assert int(full[-1]) == wl["n_rays"]
    assert np.array_equal(np.sort(full[:-1].cpu().numpy()), np.arange(wl["n_rays"]))
    order = full
    s0, s1 = api.new_stats(), api.new_stats()
    E0 = pb.forward(_opts(wl, deterministic=True), stats=s0)
    E1 = pb.forward(_opts(wl, order, deterministic=True), stats=s1)
    assert torch.equal(E0, E1) and torch.equal(s0, s1)
    d = torch.as_tensor(random_dLdE(wl, 7), dtype=torch.float32, device="cuda")
    g0 = pb.adjoint(d, _opts(wl, deterministic=True))
    g1 = pb.adjoint(d, _opts(wl, order, deterministic=True))
    for a, b in zip(g0, g1):
        assert torch.equal(a, b)
    E2 = pb.forward(_opts(wl, order)).double().cpu().numpy()
    assert rel_l2(E2, E0.double().cpu().numpy()) < 1e-5


@pytest.mark.parametrize("nu", [1, 5])
def test_order_with_other_filter_sizes(nu):
    wl = _wl(9 * 10000, (3, 3))
    wl["target"]["nu_x"] = wl["target"]["nu_y"] = nu
    pb = api.Problem(wl)
    order = pb.ray_order()
    E0 = pb.forward(_opts(wl, deterministic=True))
    E1 = pb.forward(_opts(wl, order, deterministic=True))
    assert torch.equal(E0, E1)
    d = torch.as_tensor(random_dLdE(wl, 3), dtype=torch.float32, device="cuda")
    assert torch.equal(pb.adjoint(d, _opts(wl, deterministic=True)), pb.adjoint(d, _opts(wl, order, deterministic=True)))
    E2 = pb.forward(_opts(wl, order)).double().cpu().numpy()
    assert rel_l2(E2, E0.double().cpu().numpy()) < 1e-5


def test_full_size_point_workload_in_order():
    # the 16M-ray point source as the optimisation step traces it (window form,
    # ray order) against the deterministic id-order traces
    wl = W.config(3)
    pb = api.Problem(wl)
    order = pb.ray_order()
    s0, s1 = api.new_stats(), api.new_stats()
    E_det = pb.forward(api.make_options(deterministic=True), stats=s0).double().cpu().numpy()
    E_ord = pb.forward(api.make_options(ray_order=order), stats=s1).double().cpu().numpy()
    assert torch.equal(s0, s1)
    assert rel_l2(E_ord, E_det) < 1e-5
    d = torch.as_tensor(random_dLdE(wl, 9), dtype=torch.float32, device="cuda")
    g_det = pb.adjoint(d, api.make_options(deterministic=True)).double().cpu().numpy()
    g_ord = pb.adjoint(d, api.make_options(ray_order=order)).double().cpu().numpy()
    assert rel_l2(g_ord, g_det) < 1e-5


def test_full_size_grid_of_sources_float_matches_deterministic():
    # the 64M-ray 8 x 8 grid of point sources as the optimisation step traces
    # it (window form with u32 fixed point in shared memory, ray order) against
    # the deterministic traces: the u32 quantum grows with the rays per CTA,
    # and this is the largest single-lens workload
    wl = W.config(4)
    pb = api.Problem(wl)
    order = pb.ray_order()
    s0, s1 = api.new_stats(), api.new_stats()
    E_det = pb.forward(api.make_options(deterministic=True), stats=s0).double().cpu().numpy()
    E_ord = pb.forward(api.make_options(ray_order=order), stats=s1).double().cpu().numpy()
    assert torch.equal(s0, s1)
    assert rel_l2(E_ord, E_det) < 1e-5
    d = torch.as_tensor(random_dLdE(wl, 11), dtype=torch.float32, device="cuda")
    g_det = pb.adjoint(d, api.make_options(deterministic=True)).double().cpu().numpy()
    g_ord = pb.adjoint(d, api.make_options(ray_order=order)).double().cpu().numpy()
    assert rel_l2(g_ord, g_det) < 1e-5
