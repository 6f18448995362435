"""Lenses with a freeform entry face (both faces as B-splines, the extension
the paper's conclusion proposes) on the GPU against the oracle: per-ray
records, irradiance, and the gradient with respect to both nets. Tolerances as
for the single-face path; ambiguous rays (gpu_helpers.ambiguous_rays) are
taken out of both sides of the gradient."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2302_12031_gb300 import api, step
from paper_2302_12031_gb300 import workloads as W
from tests.gpu_helpers import (TOL_E, TOL_GRAD, ambiguous_rays, compare_records, forward_both, random_dLdE,
                               rel_l2)

pytestmark = pytest.mark.gpu


def _wl(kind, n_entry=6):
    if kind == "collimated":
        wl = W.collimated("c", 256, 8, 32, 1, 2, sigma=0.01)
    elif kind == "jitter":
        wl = W.collimated("c", 256, 8, 32, 1, 2, sigma=0.01, jitter=1)
    else:
        wl = W.point("p", 1 << 16, 12, 32, 3, 4, 5, sigma=0.01)
    return W.with_entry_face(wl, n_entry, 0.01, 9)


def _cat(g):
    return np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in g])


@pytest.mark.parametrize("kind", ["collimated", "jitter", "point"])
def test_two_face_records_match_oracle(kind):
    wl = _wl(kind)
    worst, g, o = compare_records(wl, 0, 1 << 14)
    ok = (g["status"] == 0) & (o["status"] == 0)
    assert ok.sum() > 3000


@pytest.mark.parametrize("kind", ["collimated", "point"])
def test_two_face_irradiance_matches_oracle(kind):
    wl = _wl(kind)
    E, E_or, stats, counts = forward_both(wl)
    assert rel_l2(E, E_or) < TOL_E
    assert np.array_equal(stats, counts)


@pytest.mark.parametrize("kind", ["collimated", "jitter", "point"])
def test_two_face_gradient_matches_oracle(kind):
    wl = _wl(kind)
    pb = api.Problem(wl)
    dLdE = random_dLdE(wl, 7)
    d = torch.as_tensor(dLdE, dtype=torch.float32, device="cuda")
    g = _cat(t.cpu().numpy() for t in pb.adjoint(d))
    g_or = _cat(O.trace_gradient(wl, dLdE))
    n = wl["n_rays"]
    amb = ambiguous_rays(wl, 0, n)
    assert len(amb) <= max(3, 2e-3 * n), len(amb)
    for rid in amb:
        g -= _cat(t.cpu().numpy() for t in pb.adjoint(d, ray_begin=int(rid), ray_count=1))
        g_or -= _cat(O.trace_gradient(wl, dLdE, begin=int(rid), count=1))
    n_out = wl["lens"]["P"].size
    assert rel_l2(g[:n_out], g_or[:n_out]) < TOL_GRAD
    assert rel_l2(g[n_out:], g_or[n_out:]) < TOL_GRAD
    assert np.abs(g_or[n_out:]).max() > 0


def test_flat_entry_net_equals_the_flat_face():
    wl = W.point("p", 1 << 16, 12, 32, 3, 4, 5, sigma=0.01)
    two = W.with_entry_face(wl, 6, 0.0, 9)
    E1 = api.Problem(wl).forward().cpu().numpy()
    E2 = api.Problem(two).forward().cpu().numpy()
    assert rel_l2(E2, E1) < 1e-5
    wc = W.collimated("c", 256, 8, 32, 1, 2, sigma=0.01)
    E1 = api.Problem(wc).forward().cpu().numpy()
    E2 = api.Problem(W.with_entry_face(wc, 6, 0.0, 9)).forward().cpu().numpy()
    assert rel_l2(E2, E1) < 1e-5


@pytest.mark.parametrize("kind", ["collimated", "point"])
def test_two_face_deterministic_is_bit_exact_across_schedules(kind):
    wl = _wl(kind)
    pb = api.Problem(wl)
    d = torch.as_tensor(random_dLdE(wl, 3), dtype=torch.float32, device="cuda")
    ops = [api.make_options(deterministic=True), api.make_options(deterministic=True, warps_per_cta=4,
                                                                  rays_per_lane=3, ctas_per_sm=1, hist_mode=1)]
    Es = [pb.forward(o).clone() for o in ops]
    Gs = [torch.cat([t.reshape(-1) for t in pb.adjoint(d, o)]).clone() for o in ops]
    assert torch.equal(Es[0], Es[1]) and torch.equal(Gs[0], Gs[1])


def test_two_face_unsupported_combinations_are_refused():
    wl = _wl("point")
    pb = api.Problem(wl)
    with pytest.raises(api.FreerayError):
        pb.forward(api.make_options(mesh=(2, 2)))
    with pytest.raises(api.FreerayError):
        pb.tangent(torch.zeros(pb.n_params(), device="cuda").reshape(1, -1)[:, :pb.ctrl_shape[0] * pb.ctrl_shape[1]]
                   .reshape(1, *pb.ctrl_shape))
    E = torch.zeros(pb.ext_shape, device="cuda")
    with pytest.raises(api.FreerayError):
        api.fr_trace_batch_forward(api.default_handle(), [pb.batch_item(E=E), pb.batch_item(E=E)])


def test_two_face_optimisation_step():
    wl = _wl("collimated")
    wl["E_ref"] = W.gaussian_mixture_target(32, 32, 1.0, 1.0, 2, 0.9216)
    sg = step.OptimStep(wl, lr=1e-3, graph=True, options=api.make_options(deterministic=True))
    se = step.OptimStep(wl, lr=1e-3, graph=False, options=api.make_options(deterministic=True))
    n_out, n_in = wl["lens"]["P"].size, wl["lens"]["P_in"].size
    assert sg.n_params == n_out + n_in
    P0 = sg.P.double().cpu().numpy().copy()
    sg.step()
    se.step()
    torch.cuda.synchronize()
    # the first step's gradient over both nets against the oracle's
    E_or, _ = O.trace_forward(wl)
    _, d_or = O.loss_l2(wl, E_or)
    g_or = _cat(O.trace_gradient(wl, d_or))
    assert rel_l2(sg.g.cpu().numpy(), g_or) < TOL_GRAD
    for _ in range(3):
        sg.step()
        se.step()
    torch.cuda.synchronize()
    assert torch.equal(sg.P, se.P)                       # graph replay = eager, bit for bit
    moved = np.abs(sg.P.double().cpu().numpy() - P0)
    assert moved[:n_out].max() > 0 and moved[n_out:].max() > 0   # both faces are optimised
