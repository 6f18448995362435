"""fr_trace_forward_static: the forward trace for callers that cannot allocate
device memory (its scratch is a static device array inside the library).

Checked through the C ABI against fr_trace_forward on two calls in a row, in
float mode (within the irradiance tolerance of the parity tests) and in
deterministic mode (bit for bit), for flat and freeform entry faces and for a
point-source grid beyond shared memory (the window form), and for the
rejection of a problem larger than the static array. This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2302_12031_gb300 import api
from paper_2302_12031_gb300 import workloads as W
from tests.gpu_helpers import TOL_E, rel_l2

pytestmark = pytest.mark.gpu


def _static_call(pb, options, E, stats=None, begin=0, count=api.ALL_RAYS):
    return api.lib().fr_trace_forward_static(
        C.byref(pb.lens), C.byref(pb.source), C.byref(pb.target), pb.n_rays, pb.seed, begin, count,
        C.byref(options), C.c_void_p(E.data_ptr()), None if stats is None else C.c_void_p(stats.data_ptr()),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _workload(which):
    if which == "collimated":
        return W.config(1)
    if which == "point":
        return W.point("p", 6 * 4096, 24, 96, 4, 4, 4)
    if which == "point-256":        # grid beyond shared memory: the window form in float mode
        return W.point("p", 1 << 16, 24, 256, 4, 4, 4)
    if which == "two-face-collimated":
        return W.with_entry_face(W.collimated("c", 256, 8, 32, 1, 2), 6, 0.01, 9)
    return W.with_entry_face(W.point("p", 1 << 15, 12, 32, 3, 4, 5), 6, 0.01, 9)


@pytest.mark.parametrize("deterministic", [False, True])
@pytest.mark.parametrize("which", ["collimated", "point", "point-256", "two-face-collimated", "two-face-point"])
def test_static_forward_matches_handle_forward_twice(deterministic, which):
    wl = _workload(which)
    pb = api.Problem(wl)
    opt = api.make_options(deterministic=deterministic)
    ref_stats = api.new_stats()
    E_ref = pb.forward(opt, stats=ref_stats)
    for _ in range(2):                                   # two calls in a row share the static array
        E = torch.full(pb.ext_shape, float("nan"), device="cuda")
        stats = api.new_stats()
        assert _static_call(pb, opt, E, stats) == api.FR_OK
        torch.cuda.synchronize()
        assert torch.isfinite(E).all()
        if deterministic:
            assert torch.equal(E, E_ref)
        else:
            assert rel_l2(E.cpu().numpy(), E_ref.cpu().numpy()) < TOL_E
        assert torch.equal(stats, ref_stats)


def test_static_forward_rejects_grids_beyond_its_array():
    wl = W.collimated("big", 64, 8, 400, 1, 2, with_target=False)   # 402 x 402 extended cells
    pb = api.Problem(wl)
    E = torch.zeros(pb.ext_shape, device="cuda")
    st = _static_call(pb, api.make_options(deterministic=True), E)
    assert st == api.FR_ERR_WORKSPACE
    assert b"122000" in api.lib().fr_last_error(None)
    # the float mode needs no accumulator and runs at that size
    E_ref = pb.forward(api.make_options())
    assert _static_call(pb, api.make_options(), E) == api.FR_OK
    torch.cuda.synchronize()
    assert rel_l2(E.cpu().numpy(), E_ref.cpu().numpy()) < TOL_E
