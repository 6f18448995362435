"""The triangle-mesh intersection (Sec. 2.2.2) on the GPU against the oracle's:
per-ray records, irradiance, gradient and derivative maps, for point sources
with several mesh resolutions. Tolerances as for the Newton path; rays within
rounding of a triangle edge (where the hit's derivative has a kink) or of a
pixel edge are ambiguous for the gradient (gpu_helpers.ambiguous_rays)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2302_12031_gb300 import api
from paper_2302_12031_gb300 import workloads as W
from tests.gpu_helpers import (TOL_E, TOL_GRAD, adjoint_both, compare_records, forward_both, oracle_dLdE,
                               options_for, rel_l2)
from tests.test_gpu_tangent import tangent_both

pytestmark = pytest.mark.gpu


def _wl(mesh, n_rays=1 << 16, grid=(1, 1), n_ctrl=12, bins=32):
    wl = W.point("p", n_rays, n_ctrl, bins, 3, 4, 5, grid=grid, grid_size=(0.2, 0.2), sigma=0.01)
    wl["mesh"] = mesh
    return wl


@pytest.mark.parametrize("mesh", [(1, 1), (2, 3), (4, 4), (16, 16)])
def test_mesh_records_match_oracle(mesh):
    wl = _wl(mesh)
    worst, g, o = compare_records(wl, 0, 1 << 14)
    ok = (g["status"] == 0) & (o["status"] == 0)
    assert ok.sum() > 3000
    assert np.abs(g["t"][ok] - o["t"][ok]).max() < 1e-5


@pytest.mark.parametrize("mesh", [(2, 2), (4, 4)])
def test_mesh_irradiance_matches_oracle(mesh):
    wl = _wl(mesh)
    E, E_or, stats, counts = forward_both(wl)
    assert rel_l2(E, E_or) < TOL_E
    assert np.array_equal(stats, counts)


@pytest.mark.parametrize("mesh,grid", [((2, 2), (1, 1)), ((4, 3), (3, 3))])
def test_mesh_gradient_matches_oracle(mesh, grid):
    n = (1 << 16) if grid == (1, 1) else 9 << 13
    wl = _wl(mesh, n_rays=n, grid=grid)
    wl["E_ref"] = W.gaussian_mixture_target(32, 32, W.POINT_SCREEN_R, W.POINT_SCREEN_R, 5, 0.3)
    g, g_or = adjoint_both(wl, oracle_dLdE(wl))
    assert rel_l2(g, g_or) < TOL_GRAD


def test_mesh_deterministic_gradient_matches_float():
    wl = _wl((4, 4))
    pb = api.Problem(wl)
    d = torch.randn(pb.ext_shape, device="cuda")
    gf = pb.adjoint(d, options_for(wl)).cpu().numpy()
    gd = pb.adjoint(d, options_for(wl, deterministic=True)).cpu().numpy()
    assert rel_l2(gf, gd) < 1e-4


def test_mesh_tangent_matches_oracle():
    wl = _wl((3, 3))
    rng = np.random.default_rng(4)
    one = np.zeros_like(wl["lens"]["P"])
    one[6, 5] = 1.0
    dP = np.stack([rng.normal(size=one.shape), one])
    g, o = tangent_both(wl, dP)
    for q in range(2):
        assert rel_l2(g[q], o[q]) < TOL_GRAD, (q, rel_l2(g[q], o[q]))


def test_fine_mesh_approaches_newton():
    # the mesh converges to the B-spline: hits of a fine mesh agree with Newton's
    wl = _wl((0, 0), n_rays=1 << 15)
    pb = api.Problem(wl)
    newton = pb.debug(0, 1 << 15)
    errs = []
    for n in (2, 8, 32):
        m = pb.debug(0, 1 << 15, options=api.make_options(mesh=(n, n)))
        ok = (m["status"] == 0) & (newton["status"] == 0)
        errs.append(float(np.abs(m["z"][ok] - newton["z"][ok]).max()))
    # second order: 16x per 4x finer cells, down to the FP32 floor
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[2] > 50, errs


def test_mesh_options_are_checked():
    wl = _wl((0, 0), n_rays=1024)
    pb = api.Problem(wl)
    for mesh in ((1, 0), (0, 2), (65, 1), (-1, -1)):
        with pytest.raises(api.FreerayError):
            pb.forward(api.make_options(mesh=mesh))
