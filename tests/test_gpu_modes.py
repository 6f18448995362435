"""Modes and interfaces of the CUDA path: deterministic fixed point, finite
differences, autograd, the batched launch, the graph-captured Adam step, and the
error codes of the C ABI."""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2302_12031_gb300 import api, autograd, step
from paper_2302_12031_gb300 import workloads as W
from tests.gpu_helpers import TOL_E, TOL_GRAD, forward_both, random_dLdE, rel_l2

pytestmark = pytest.mark.gpu


def _det(**kw):
    return api.make_options(deterministic=True, **kw)


@pytest.mark.parametrize("k", [2, 3])
def test_deterministic_mode_is_bit_exact_across_runs_and_schedules(k):
    wl = W.config(k, with_target=False)
    if k == 3:
        wl["n_rays"] = 1 << 21                    # same source, fewer rays
    pb = api.Problem(wl)
    d = torch.as_tensor(random_dLdE(wl, 1), dtype=torch.float32, device="cuda")
    schedules = [_det(), _det(), _det(warps_per_cta=4, rays_per_lane=5, ctas_per_sm=1, hist_mode=1),
                 _det(warps_per_cta=2, rays_per_lane=16, hist_mode=2)]
    Es = [pb.forward(o).clone() for o in schedules]
    Gs = [pb.adjoint(d, o).clone() for o in schedules]
    for E in Es[1:]:
        assert torch.equal(E, Es[0])
    for G in Gs[1:]:
        assert torch.equal(G, Gs[0])
    Ef = pb.forward(api.make_options())
    Gf = pb.adjoint(d, api.make_options())
    assert rel_l2(Ef.cpu().numpy(), Es[0].cpu().numpy()) < 1e-5
    assert rel_l2(Gf.cpu().numpy(), Gs[0].cpu().numpy()) < 1e-4


def test_deterministic_mode_matches_oracle():
    wl = W.config(1)
    E, E_or, _, _ = forward_both(wl, options=_det())
    assert rel_l2(E, E_or) < TOL_E
    d = random_dLdE(wl, 4)
    g = api.Problem(wl).adjoint(torch.as_tensor(d, dtype=torch.float32, device="cuda"), _det()).cpu().numpy()
    assert rel_l2(g, O.trace_gradient(wl, d)) < TOL_GRAD


def test_finite_differences_on_16_control_points_workload2():
    # Workload 2 in deterministic mode, central differences on 16 random control
    # heights. At h = 1e-4 the rays move about half a pixel, so the difference
    # quotient carries an O(h^2) truncation error of about 1%; at h = 3e-6 it
    # must agree to 3e-3.
    wl = W.config(2)
    pb = api.Problem(wl)
    E_ref = torch.as_tensor(wl["E_ref"], dtype=torch.float32, device="cuda")
    opt = _det()
    h = api.default_handle()

    def loss(P):
        pb.set_ctrl(P)
        E = pb.forward(opt)
        L = torch.zeros((), dtype=torch.float64, device="cuda")
        d = torch.empty_like(E)
        api.fr_loss_l2(h, E, E_ref, pb.nx, pb.ny, pb.nu_x, pb.nu_y, L, d)
        return float(L), d

    P0 = pb.ctrl_z.clone()
    L0, d0 = loss(P0)
    pb.set_ctrl(P0)
    g = pb.adjoint(d0, opt).cpu().numpy().ravel()
    idx = np.random.default_rng(3).choice(P0.numel(), 16, replace=False)
    for step_h, tol in ((1e-4, 2.5e-2), (3e-6, 3e-3)):
        fd = []
        for k in idx:
            Pp, Pm = P0.clone().view(-1), P0.clone().view(-1)
            Pp[k] += step_h
            Pm[k] -= step_h
            width = float(Pp[k] - Pm[k])          # the step as rounded in FP32
            fd.append((loss(Pp.view(P0.shape))[0] - loss(Pm.view(P0.shape))[0]) / width)
        err = rel_l2(g[idx], np.array(fd))
        assert err < tol, (step_h, err)


def test_autograd_function_matches_adjoint():
    wl = W.config(1)
    pb = api.Problem(wl)
    P = pb.ctrl_z.clone().requires_grad_(True)
    E_ref = torch.as_tensor(wl["E_ref"], dtype=torch.float32, device="cuda")
    E = autograd.trace(P, pb)
    L = autograd.loss_l2(E, E_ref, pb)
    L.backward()
    E_or, _ = O.trace_forward(wl)
    L_or, d_or = O.loss_l2(wl, E_or)
    assert abs(float(L) - L_or) < 1e-3 * L_or
    assert rel_l2(P.grad.cpu().numpy(), O.trace_gradient(wl, d_or)) < TOL_GRAD


def test_batched_launch_equals_single_calls():
    wls = [W.collimated("a", 160, 8, 24, 1, 2), W.point("b", 8 * 1024, 12, 32, 3, 4, 5),
           W.point("c", 9 * 1000, 16, 48, 6, 7, 8, grid=(3, 3), grid_size=(0.2, 0.2)),
           W.collimated("d", 96, 32, 16, 9, 10, jitter=1)]
    pbs = [api.Problem(w) for w in wls]
    h = api.default_handle()
    for opt in (api.make_options(), _det()):
        Es = [torch.zeros(pb.ext_shape, device="cuda") for pb in pbs]
        api.fr_trace_batch_forward(h, [pb.batch_item(E=E) for pb, E in zip(pbs, Es)], opt)
        ds = [torch.as_tensor(random_dLdE(w, i), dtype=torch.float32, device="cuda") for i, w in enumerate(wls)]
        Gs = [torch.zeros(pb.ctrl_shape, device="cuda") for pb in pbs]
        api.fr_trace_batch_adjoint(h, [pb.batch_item(dLdE=d, dLdP=g) for pb, d, g in zip(pbs, ds, Gs)], opt)
        for pb, E, d, G in zip(pbs, Es, ds, Gs):
            E1 = pb.forward(opt)
            G1 = pb.adjoint(d, opt)
            if opt.deterministic:
                assert torch.equal(E, E1) and torch.equal(G, G1)
            else:
                assert rel_l2(E.cpu().numpy(), E1.cpu().numpy()) < 1e-6
                assert rel_l2(G.cpu().numpy(), G1.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("batched", [False, True])
def test_graph_step_matches_eager_and_oracle_adam(batched):
    wls = [W.config(1)] if not batched else [W.config(1), W.point("p", 4 * 4096, 12, 32, 3, 4, 5)]
    sg = step.OptimStep(wls if batched else wls[0], lr=1e-3, graph=True)
    se = step.OptimStep(wls if batched else wls[0], lr=1e-3, graph=False)
    P0 = sg.P.clone()
    for _ in range(3):
        sg.step()
        se.step()
    torch.cuda.synchronize()
    assert int(sg.step_count) == 3 and int(se.step_count) == 3
    assert torch.allclose(sg.P, se.P, rtol=0, atol=1e-6)
    # one step by hand: oracle Adam on the GPU gradient from the same start
    s1 = step.OptimStep(wls if batched else wls[0], lr=1e-3, graph=False)
    s1._forward(); s1._loss(); s1._adjoint()
    g = s1.g.double().cpu().numpy()
    theta = P0.double().cpu().numpy().copy()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    O.adam_step(theta, m, v, g, lr=1e-3, step=1)
    s1._adam()
    assert np.allclose(s1.P.double().cpu().numpy(), theta, rtol=0, atol=1e-6)


def test_loss_matches_oracle():
    wl = W.config(1)
    pb = api.Problem(wl)
    E = pb.forward()
    L = torch.zeros((), dtype=torch.float64, device="cuda")
    d = torch.empty_like(E)
    api.fr_loss_l2(api.default_handle(), E, torch.as_tensor(wl["E_ref"], dtype=torch.float32, device="cuda"),
                   pb.nx, pb.ny, pb.nu_x, pb.nu_y, L, d)
    L_or, d_or = O.loss_l2(wl, E.double().cpu().numpy())
    assert abs(float(L) - L_or) <= 1e-6 * L_or
    assert np.allclose(d.cpu().numpy(), d_or, rtol=1e-6, atol=1e-6)


def test_invalid_arguments_return_error_codes():
    h = api.default_handle()
    wl = W.config(1)
    pb = api.Problem(wl)
    E = torch.zeros(pb.ext_shape, device="cuda")
    L = api.lib()

    def fwd(lens=None, src=None, tgt=None, n=None, begin=0, count=api.ALL_RAYS, E_ptr=True):
        return L.fr_trace_forward(h.ptr, C.byref(lens or pb.lens), C.byref(src or pb.source),
                                  C.byref(tgt or pb.target), pb.n_rays if n is None else n, 1, begin, count, None,
                                  C.c_void_p(E.data_ptr()) if E_ptr else None, None, None)

    assert fwd() == api.FR_OK
    bad = api.LensDesc.from_buffer_copy(pb.lens); bad.p = 6
    assert fwd(lens=bad) == api.FR_ERR_UNSUPPORTED
    bad = api.LensDesc.from_buffer_copy(pb.lens); bad.n1 = 40
    assert fwd(lens=bad) == api.FR_ERR_UNSUPPORTED
    bad = api.LensDesc.from_buffer_copy(pb.lens); bad.ctrl_z = None
    assert fwd(lens=bad) == api.FR_ERR_INVALID_ARG
    bad = api.LensDesc.from_buffer_copy(pb.lens); bad.rx = float("nan")
    assert fwd(lens=bad) == api.FR_ERR_INVALID_ARG
    assert fwd(n=pb.n_rays + 1) == api.FR_ERR_INVALID_ARG               # not cols*rows
    assert fwd(begin=pb.n_rays + 1) == api.FR_ERR_INVALID_ARG
    assert fwd(begin=10, count=pb.n_rays) == api.FR_ERR_INVALID_ARG
    assert fwd(E_ptr=False) == api.FR_ERR_INVALID_ARG
    bt = api.TargetDesc.from_buffer_copy(pb.target); bt.nu_x = bt.nu_y = 13
    assert fwd(tgt=bt) == api.FR_ERR_UNSUPPORTED
    bt = api.TargetDesc.from_buffer_copy(pb.target); bt.nx = 0
    assert fwd(tgt=bt) == api.FR_ERR_INVALID_ARG
    bs = api.SourceDesc.from_buffer_copy(pb.source); bs.kind = 7
    assert fwd(src=bs) == api.FR_ERR_INVALID_ARG
    pw = api.Problem(W.point("p", 1000, 8, 16, 1, 2, 3, grid=(3, 3)))
    assert L.fr_trace_forward(h.ptr, C.byref(pw.lens), C.byref(pw.source), C.byref(pw.target), 1000, 1, 0,
                              api.ALL_RAYS, None, C.c_void_p(E.data_ptr()), None, None) == api.FR_ERR_INVALID_ARG
    assert b"multiple" in L.fr_last_error(h.ptr)
    assert L.fr_trace_batch_forward(h.ptr, None, 0, None, None) == api.FR_ERR_INVALID_ARG
    one = torch.zeros(1, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert L.fr_adam_step(h.ptr, C.c_void_p(one.data_ptr()), C.c_void_p(one.data_ptr()),
                          C.c_void_p(one.data_ptr()), C.c_void_p(one.data_ptr()), 1, 1e-3, 1.5, 0.999, 1e-8,
                          C.c_void_p(st.data_ptr()), None) == api.FR_ERR_INVALID_ARG
    torch.cuda.synchronize()


def test_workspace_growth_is_refused_during_capture():
    h = api.Handle()                            # a fresh handle: no scratch memory yet
    pb = api.Problem(W.config(1))
    E = torch.zeros(pb.ext_shape, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    try:
        with torch.cuda.graph(g, stream=s):
            status = api.lib().fr_trace_forward(h.ptr, C.byref(pb.lens), C.byref(pb.source), C.byref(pb.target),
                                                pb.n_rays, 1, 0, api.ALL_RAYS, None, C.c_void_p(E.data_ptr()),
                                                None, C.c_void_p(s.cuda_stream))
    except RuntimeError:
        pass                                    # an empty capture may be rejected by torch
    assert status == api.FR_ERR_WORKSPACE
    assert b"capturing" in api.lib().fr_last_error(h.ptr)
    h.close()
    torch.cuda.synchronize()


def test_stream_wait_times_out_and_completes():
    h = api.default_handle()
    api.fr_stream_wait(h, 1000)
    torch.cuda.synchronize()


def test_programmatic_launch_gives_the_same_step():
    wl = W.config(1)
    det = api.make_options(deterministic=True)
    a = step.OptimStep(wl, lr=1e-3, graph=True, options=det, pdl=True)
    b = step.OptimStep(wl, lr=1e-3, graph=True, options=det, pdl=False)
    for _ in range(4):
        a.step()
        b.step()
    torch.cuda.synchronize()
    assert torch.equal(a.P, b.P) and torch.equal(a.losses(), b.losses())
    h = api.default_handle()
    assert api.lib().fr_set_programmatic_launch(h.ptr, 3) == api.FR_ERR_INVALID_ARG
    api.fr_set_programmatic_launch(h, 0)


def test_checkpoint_resume_is_bit_exact(tmp_path):
    wl = W.config(1)
    det = api.make_options(deterministic=True)
    a = step.OptimStep(wl, lr=1e-3, graph=True, options=det)
    for _ in range(3):
        a.step()
    a.save(str(tmp_path / "ckpt.pt"))
    for _ in range(3):
        a.step()
    b = step.OptimStep(wl, lr=1e-3, graph=True, options=det)
    b.load(str(tmp_path / "ckpt.pt"))
    for _ in range(3):
        b.step()
    torch.cuda.synchronize()
    assert torch.equal(a.P, b.P) and torch.equal(a.m, b.m) and torch.equal(a.v, b.v)
    assert int(a.step_count) == int(b.step_count) == 6
    other = W.config(1)
    other["seed"] = 99
    c = step.OptimStep(other, lr=1e-3, graph=False, options=det)
    with pytest.raises(ValueError):
        c.load(str(tmp_path / "ckpt.pt"))


def test_non_finite_control_heights_lose_rays_not_the_image():
    # a NaN height: the rays over its patches are culled (and counted), E stays finite
    for wl in (W.config(1, with_target=False), W.point("p", 1 << 15, 8, 16, 3, 4, 5, with_target=False)):
        wl["lens"]["P"][3, 4] = float("nan")
        pb = api.Problem(wl)
        stats = api.new_stats()
        E = pb.forward(stats=stats)
        counts = stats.cpu().numpy()
        assert torch.isfinite(E).all()
        assert counts.sum() == wl["n_rays"] and counts[0] < wl["n_rays"]
        g = pb.adjoint(torch.ones(pb.ext_shape, device="cuda"))
        assert torch.isfinite(g).all()


def test_lens_below_its_entry_face_is_counted_invalid():
    wl = W.point("p", 1 << 14, 8, 16, 3, 4, 5, with_target=False)
    wl["lens"]["P"][:] = wl["lens"]["z_in"] - 0.05          # the freeform below the flat entry face
    pb = api.Problem(wl)
    stats = api.new_stats()
    E = pb.forward(stats=stats)
    counts = stats.cpu().numpy()
    assert float(E.abs().sum()) == 0.0
    assert counts[5] > 0 and counts[0] == 0                # FR_RAY_INVALID


def test_zero_list_clears_exactly_its_buffers():
    h = api.default_handle()
    big = torch.full((4096,), 7.0, device="cuda")
    views = [big[1:2], big[3:70], big[101:1100], big[2000:2003], big[3000:3000]]   # 4-byte offsets, odd lengths, empty
    api.fr_zero_list(h, views)
    torch.cuda.synchronize()
    want = torch.full((4096,), 7.0)
    for a, b in ((1, 2), (3, 70), (101, 1100), (2000, 2003)):
        want[a:b] = 0.0
    assert torch.equal(big.cpu(), want)
    api.fr_zero_list(h, [])
    with pytest.raises(api.FreerayError):
        api.fr_zero_list(h, [big] * 81)
