"""The paper's loss and parametrisation on the GPU against the oracle: the
normalised Frobenius loss (Sec. 2.5), the tanh reparametrisation with its
adjoint, the spherical offsets (Sec. 2.4.2, Table magndata), the fused Adam
step on the unconstrained variables, and the optimisation step built from them.

Tolerances: the loss kernel reads the same float32 images as the oracle; per
pixel it works in FP32 with E/S carried as a pair of floats (about 2^-44
relative), each thread sums at most a few dozen FP32 terms and FP64 adds the
partial sums, so the loss agrees to 1e-6 relative; dL/dE is formed in FP32 from
FP32-rounded factors (1e-5 of its largest value). The maps are written in FP32
(1e-6 relative). Adam in FP32 against FP64 over a few steps: 1e-5 absolute on
the unconstrained variables.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2302_12031_gb300 import api, autograd, step
from paper_2302_12031_gb300 import workloads as W
from tests.gpu_helpers import TOL_E, TOL_GRAD, rel_l2

pytestmark = pytest.mark.gpu


def _frob_gpu(E, Eref, nx, ny, nu):
    L = torch.zeros((), dtype=torch.float64, device="cuda")
    d = torch.full(E.shape, 7.0, device="cuda")           # ghost pixels must be overwritten with 0
    api.fr_loss_frobenius(api.default_handle(), E, Eref, nx, ny, nu, nu, L, d)
    return float(L), d.cpu().numpy()


def _wl(nx, ny, nu, Eref):
    return {"target": {"nx": nx, "ny": ny, "nu_x": nu, "nu_y": nu}, "E_ref": Eref}


@pytest.mark.parametrize("nx,ny,nu", [(32, 32, 3), (128, 128, 3), (256, 256, 3), (97, 61, 5), (7, 3, 1), (1, 1, 1)])
def test_frobenius_loss_matches_oracle(nx, ny, nu):
    g = torch.Generator(device="cpu").manual_seed(nx * 1000 + ny)
    Eref = torch.rand(ny, nx, generator=g)
    E = torch.zeros(ny + nu - 1, nx + nu - 1)
    h = (nu - 1) // 2
    E[h:h + ny, h:h + nx] = torch.rand(ny, nx, generator=g)
    if nu > 1:
        E[0, :] += 3.0                                     # ghost values never enter the loss
    L, d = _frob_gpu(E.cuda(), Eref.cuda(), nx, ny, nu)
    L_or, d_or = O.loss_frobenius(_wl(nx, ny, nu, Eref.double().numpy()), E.double().numpy())
    if nx * ny == 1:
        # one pixel: both normalised images are 1 (the kernel's to about 2^-44)
        assert L_or == 0.0 and L < 1e-12 and np.abs(d).max() < 1e-10 / float(E.sum())
        return
    assert abs(L - L_or) <= 1e-6 * L_or
    assert np.max(np.abs(d - d_or)) <= 1e-5 * np.max(np.abs(d_or))
    # the reduction order is fixed: bit-identical on a second call
    L2, d2 = _frob_gpu(E.cuda(), Eref.cuda(), nx, ny, nu)
    assert L2 == L and np.array_equal(d2, d)


def test_frobenius_loss_degenerate_cases():
    nx = ny = 16
    Eref = torch.rand(ny, nx, device="cuda")
    E = torch.zeros(ny + 2, nx + 2, device="cuda")
    L, d = _frob_gpu(E, Eref, nx, ny, 3)                  # no light on the screen
    assert np.isnan(L) and np.all(d == 0)
    E[1:-1, 1:-1] = 4.0 * Eref                            # equal up to a power-of-two scale
    L, d = _frob_gpu(E, Eref, nx, ny, 3)
    assert L == 0.0 and np.all(d == 0)


def test_frobenius_loss_on_traced_image_and_its_gradient():
    wl = W.config(1)
    pb = api.Problem(wl)
    E = pb.forward()
    Eref = torch.as_tensor(wl["E_ref"], dtype=torch.float32, device="cuda")
    L, d = _frob_gpu(E, Eref, pb.nx, pb.ny, pb.nu_x)
    E_or, _ = O.trace_forward(wl)
    L_or, d_or = O.loss_frobenius(wl, E_or)
    assert abs(L - L_or) <= TOL_E * L_or
    assert rel_l2(d, d_or) < TOL_E * 10
    # the whole chain: dL/dP through the Frobenius loss and the adjoint
    g = pb.adjoint(torch.as_tensor(d, device="cuda")).cpu().numpy()
    g_or = O.trace_gradient(wl, d_or)
    assert rel_l2(g, g_or) < TOL_GRAD


def test_reparam_tanh_and_adjoint_match_oracle():
    h = api.default_handle()
    n = 33 * 33
    gen = torch.Generator(device="cpu").manual_seed(7)
    theta = (torch.randn(n, generator=gen) * 2).cuda()
    off = (torch.randn(n, generator=gen) * 0.1).cuda()
    dLdP = torch.randn(n, generator=gen).cuda()
    zmin, zmax = -0.05, 0.15
    P = torch.empty(n, device="cuda")
    api.fr_reparam_tanh(h, theta, off, n, zmin, zmax, P)
    P_or = O.reparam_tanh(theta.double().cpu().numpy(), np.float32(zmin), np.float32(zmax),
                          off.double().cpu().numpy())
    assert np.max(np.abs(P.cpu().numpy() - P_or)) < 1e-6
    api.fr_reparam_tanh(h, theta, None, n, zmin, zmax, P)
    P_or0 = O.reparam_tanh(theta.double().cpu().numpy(), np.float32(zmin), np.float32(zmax))
    assert np.max(np.abs(P.cpu().numpy() - P_or0)) < 1e-6
    G = torch.empty(n, device="cuda")
    api.fr_reparam_tanh_adjoint(h, theta, dLdP, n, zmin, zmax, G)
    G_or = O.reparam_tanh_adjoint(theta.double().cpu().numpy(), dLdP.double().cpu().numpy(), np.float32(zmin),
                                  np.float32(zmax))
    assert np.max(np.abs(G.cpu().numpy() - G_or)) <= 1e-6 * np.max(np.abs(G_or))
    # autograd: the same adjoint
    t = theta.clone().requires_grad_(True)
    autograd.reparam_tanh(t, zmin, zmax, off).backward(dLdP)
    assert torch.equal(t.grad, G)


@pytest.mark.parametrize("n", [3, 7, 23, 31])
@pytest.mark.parametrize("c,R", [(0.5, 0.0), (0.5, 8.0), (0.5, 4.0), (0.1, -4.0)])
def test_offset_spherical_matches_oracle(n, c, R):
    wl = W.collimated("c", 8, n + 1, 8, 1, 2, with_target=False)
    pb = api.Problem(wl)
    out = torch.empty(pb.ctrl_shape, device="cuda")
    api.fr_offset_spherical(api.default_handle(), pb.lens, c, R, out)
    lens = wl["lens"]
    ref = O.offset_spherical(n, n, 3, 3, np.float32(lens["rx"]), np.float32(lens["ry"]), np.float32(c),
                             np.float32(R))
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-6


def test_offset_spherical_rejects_a_sphere_too_small():
    wl = W.collimated("c", 8, 8, 8, 1, 2, with_target=False)
    pb = api.Problem(wl)
    out = torch.empty(pb.ctrl_shape, device="cuda")
    with pytest.raises(api.FreerayError):
        api.fr_offset_spherical(api.default_handle(), pb.lens, 0.5, 0.6, out)
    st = api.lib().fr_reparam_tanh(api.default_handle().ptr, api._ptr(out), None, out.numel(), 0.2, 0.1,
                                   api._ptr(out), None)
    assert st == api.FR_ERR_INVALID_ARG


def test_fused_tanh_adam_matches_oracle_steps():
    h = api.default_handle()
    n = 24 * 24
    gen = torch.Generator(device="cpu").manual_seed(11)
    theta0 = torch.randn(n, generator=gen) * 0.5
    off = torch.randn(n, generator=gen) * 0.05
    zmin, zmax = -0.1, 0.3
    theta, m, v = theta0.clone().cuda(), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    P = torch.empty(n, device="cuda")
    stepc = torch.zeros(1, dtype=torch.int32, device="cuda")
    th_o, m_o, v_o = theta0.double().numpy().copy(), np.zeros(n), np.zeros(n)
    for k in range(1, 6):
        dLdP = torch.randn(n, generator=gen) * 10.0 ** (k - 3)
        api.fr_adam_step_tanh(h, theta, m, v, dLdP.cuda(), off.cuda(), n, 1e-2, 0.9, 0.999, 1e-8, zmin, zmax,
                              stepc, P)
        g_th = O.reparam_tanh_adjoint(th_o, dLdP.double().numpy(), np.float32(zmin), np.float32(zmax))
        O.adam_step(th_o, m_o, v_o, g_th, lr=1e-2, step=k)
    assert int(stepc) == 5
    assert np.max(np.abs(theta.double().cpu().numpy() - th_o)) < 1e-5
    P_o = O.reparam_tanh(th_o, np.float32(zmin), np.float32(zmax), off.double().numpy())
    assert np.max(np.abs(P.double().cpu().numpy() - P_o)) < 1e-5


def test_step_with_frobenius_loss_and_reparametrisation():
    wl = W.config(1)
    rp = dict(z_min=-0.05, z_max=0.05, offset=("sphere", 0.0, 8.0))
    kw = dict(lr=1e-2, loss="frobenius", reparam=rp, options=api.make_options(deterministic=True))
    sg = step.OptimStep(wl, graph=True, **kw)
    se = step.OptimStep(wl, graph=False, **kw)
    assert torch.equal(sg.P, se.P) and torch.equal(sg.theta, se.theta)
    # the starting heights are the reparametrised ones
    lens = wl["lens"]
    off = O.offset_spherical(lens["n1"], lens["n2"], 3, 3, np.float32(lens["rx"]), np.float32(lens["ry"]), 0.0, 8.0)
    P0 = O.reparam_tanh(sg.theta.double().cpu().numpy(), np.float32(-0.05), np.float32(0.05), off.reshape(-1))
    assert np.max(np.abs(sg.P.double().cpu().numpy() - P0)) < 1e-6
    # one step by hand against the oracle, from the GPU gradient
    theta0 = sg.theta.double().cpu().numpy().copy()
    wl0 = dict(wl)
    wl0["lens"] = dict(lens, P=sg.P.double().cpu().numpy().reshape(lens["n1"] + 1, lens["n2"] + 1))
    E_or, _ = O.trace_forward(wl0)
    L_or, d_or = O.loss_frobenius(wl0, E_or)
    g_or = O.trace_gradient(wl0, d_or)
    losses = []
    for k in range(20):
        sg.step()
        se.step()
        losses.append(float(sg.losses()[0]))
        if k == 0:
            assert abs(losses[0] - L_or) <= TOL_E * L_or
            assert rel_l2(sg.g.cpu().numpy(), g_or.reshape(-1)) < TOL_GRAD
            th_o, m_o, v_o = theta0.copy(), np.zeros_like(theta0), np.zeros_like(theta0)
            O.adam_step(th_o, m_o, v_o, O.reparam_tanh_adjoint(theta0, sg.g.double().cpu().numpy(),
                                                               np.float32(-0.05), np.float32(0.05)),
                        lr=1e-2, step=1)
            assert np.max(np.abs(sg.theta.double().cpu().numpy() - th_o)) < 1e-5
    torch.cuda.synchronize()
    assert torch.equal(sg.P, se.P) and torch.equal(sg.theta, se.theta)   # graph replay = eager, bit for bit
    assert losses[-1] < losses[0]
