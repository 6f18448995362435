"""The autotuner: cache keys, candidate choice and the JSON cache (CPU), and a
tuned schedule that gives the default's results (GPU)."""
import pytest
import torch

from paper_2302_12031_gb300 import api, autotune
from paper_2302_12031_gb300 import workloads as W


def test_pick_best_skips_refused_candidates_and_keeps_ties_first():
    a, b, c = dict(x=1), dict(x=2), dict(x=3)
    assert autotune.pick_best([(a, None), (b, 2.0), (c, 2.0)]) == (b, 2.0)
    assert autotune.pick_best([(a, 1.5), (b, 2.0)]) == (a, 1.5)
    assert autotune.pick_best([(a, None)]) is None


def test_cache_round_trip(tmp_path):
    c = autotune.Cache(str(tmp_path / "t.json"))
    assert c.get("k") is None
    c.put("k", {"warps_per_cta": 8, "ms": 0.1})
    assert autotune.Cache(str(tmp_path / "t.json")).get("k")["warps_per_cta"] == 8


def test_batch_candidates_start_with_the_default():
    cands = autotune.batch_candidates()
    assert cands[0] == dict(warps_per_cta=0, rays_per_lane=0, ctas_per_sm=0, batch_waves=0)
    assert all(set(c) == set(autotune.BATCH_FIELDS) for c in cands)
    assert len({tuple(sorted(c.items())) for c in cands}) == len(cands)      # no candidate twice


def test_candidates_start_with_the_default():
    for kind in ("forward", "adjoint"):
        for src in (api.FR_SOURCE_COLLIMATED, api.FR_SOURCE_POINT):
            cands = autotune.candidates(kind, src)
            assert cands[0] == dict(warps_per_cta=0, rays_per_lane=0, ctas_per_sm=0, hist_mode=0)
            assert all(set(c) == set(autotune.OPTION_FIELDS) for c in cands)


@pytest.mark.gpu
def test_tuned_schedule_gives_the_same_results(tmp_path):
    wl = W.config(1)
    pb = api.Problem(wl)
    cache = autotune.Cache(str(tmp_path / "tune.json"))
    det = api.make_options(deterministic=True)
    E0 = pb.forward(det)
    of = autotune.tune(pb, "forward", deterministic=True, cache=cache, reps=3)
    oa = autotune.tune(pb, "adjoint", deterministic=True, cache=cache, reps=3)
    assert len(cache.data) == 2
    assert torch.equal(pb.forward(of), E0)                  # fixed point: bit-identical
    d = torch.randn(pb.ext_shape, device="cuda")
    assert torch.equal(pb.adjoint(d, oa), pb.adjoint(d, det))
    # a second call is served from the cache
    of2 = autotune.tune(pb, "forward", deterministic=True, cache=cache, reps=3)
    assert all(getattr(of, f) == getattr(of2, f) for f in autotune.OPTION_FIELDS)
