"""Autotuner of the trace kernels' schedule.

For one problem it times a set of candidate schedules (warps per CTA, minimum
rays per lane, CTAs per SM, histogram placement) of the forward and the adjoint
trace kernels, each replayed from a CUDA graph with the kernel bracketed by the
library's own events, and keeps the fastest; for a batch of lenses traced in
one launch (tune_batch), the waves of CTAs the launch holds, warps per CTA,
rays per lane and CTAs per SM. Choices are cached in a JSON file keyed by the
device name and the problems' shapes, so a problem of the same shape is not
tuned twice.
"""
import hashlib
import json
import os
import statistics

import torch

from . import api

_DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")

OPTION_FIELDS = ("warps_per_cta", "rays_per_lane", "ctas_per_sm", "hist_mode")
BATCH_FIELDS = ("warps_per_cta", "rays_per_lane", "ctas_per_sm", "batch_waves")


def problem_key(pb, kind, deterministic, device_name):
    """Cache key: device, direction, mode and the shape of the problem."""
    src = "collimated" if pb.source.kind == api.FR_SOURCE_COLLIMATED else "point"
    rays = pb.n_rays
    bucket = 1 << max(0, rays.bit_length() - 1)          # ray count to a power of two
    return "|".join(str(x) for x in (device_name, kind, int(deterministic), src, pb.source.jitter,
                                     pb.ctrl_shape[0], pb.ctrl_shape[1], pb.nx, pb.ny, pb.nu_x, bucket))


def candidates(kind, source_kind):
    """Schedules worth trying; the first is the library default."""
    out = [dict(warps_per_cta=0, rays_per_lane=0, ctas_per_sm=0, hist_mode=0)]
    # warps per CTA within each kernel's launch bounds (larger requests are capped): the
    # collimated forward takes up to 12, the collimated adjoint 10, the point-source
    # forward's window form 20 (one CTA per SM), other variants 8
    collimated = source_kind == api.FR_SOURCE_COLLIMATED
    if kind == "forward":
        warps = (8, 10, 12) if collimated else (8, 16, 20)
    else:
        warps = (8, 10) if collimated else (4, 8)
    for w in warps:
        for rpl in (2, 8, 32):
            for cps in (0, 1):
                out.append(dict(warps_per_cta=w, rays_per_lane=rpl, ctas_per_sm=cps, hist_mode=0))
    if kind == "forward":
        out.append(dict(warps_per_cta=0, rays_per_lane=0, ctas_per_sm=0, hist_mode=1))
    return out


def pick_best(timings):
    """The candidate with the smallest median time; ties keep the earlier one."""
    best = None
    for cand, t in timings:
        if t is None:
            continue
        if best is None or t < best[1]:
            best = (cand, t)
    return best


class Cache:
    def __init__(self, path=None):
        self.path = path or _DEFAULT_CACHE
        self.data = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}

    def get(self, key):
        return self.data.get(key)

    def put(self, key, value):
        self.data[key] = value
        tmp = self.path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def _time_kernel(call, events, reps, flush):
    """Median kernel time (ms) of `call` replayed from a graph."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        call()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        call()
    g.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush()
        g.replay()
        torch.cuda.synchronize()
        ts.append(events[0].elapsed_time(events[1]))
    return statistics.median(ts)


def tune(pb, kind="forward", deterministic=False, reps=7, cache=None, flush=None, h=None):
    """Best fr_options for `pb` (an api.Problem) and `kind` ("forward"/"adjoint")."""
    h = h or api.default_handle()
    cache = cache if cache is not None else Cache()
    name = torch.cuda.get_device_name()
    key = problem_key(pb, kind, deterministic, name)
    hit = cache.get(key)
    if hit is not None:
        return api.make_options(deterministic=deterministic, **{k: hit[k] for k in OPTION_FIELDS})
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for e in ev:
        e.record()
    E = torch.zeros(pb.ext_shape, dtype=torch.float32, device=pb.device)
    dLdE = torch.randn(pb.ext_shape, dtype=torch.float32, device=pb.device)
    G = torch.zeros(pb.ctrl_shape, dtype=torch.float32, device=pb.device)
    timings = []
    for cand in candidates(kind, pb.source.kind):
        opt = api.make_options(deterministic=deterministic, events=ev, **cand)
        if kind == "forward":
            call = lambda: api.fr_trace_forward(h, pb.lens, pb.source, pb.target, pb.n_rays, pb.seed, 0,
                                                api.ALL_RAYS, opt, E)
        else:
            call = lambda: api.fr_trace_adjoint(h, pb.lens, pb.source, pb.target, pb.n_rays, pb.seed, 0,
                                                api.ALL_RAYS, opt, dLdE, G)
        try:
            t = _time_kernel(call, ev, reps, flush)
        except api.FreerayError:
            t = None                              # a schedule the library refuses (e.g. does not fit)
        timings.append((cand, t))
    best, t = pick_best(timings)
    cache.put(key, dict(best, ms=t))
    return api.make_options(deterministic=deterministic, **best)


def batch_key(problems, kind, deterministic, device_name):
    """Cache key of a batch: the hash of its problems' keys, in order."""
    joined = "/".join(problem_key(pb, kind, deterministic, device_name) for pb in problems)
    return "batch|%s|%s|%d|%s" % (device_name, kind, int(deterministic), hashlib.sha1(joined.encode()).hexdigest())


def batch_candidates():
    """Schedules of a batched launch worth trying; the first is the library default
    (eight waves of CTAs, 8 warps, the kernels' occupancy)."""
    out = [dict(warps_per_cta=0, rays_per_lane=0, ctas_per_sm=0, batch_waves=0)]
    for waves in (4, 8, 16, 32):
        for warps in (4, 8):
            for rpl in (0, 16):
                out.append(dict(warps_per_cta=warps, rays_per_lane=rpl, ctas_per_sm=0, batch_waves=waves))
    return out


def tune_batch(problems, kind="forward", orders=None, deterministic=False, reps=5, cache=None, flush=None, h=None):
    """Best fr_options for tracing `problems` (api.Problem list) in one batched launch;
    `orders`: their ray orders (None entries for id order), as the optimisation step traces them."""
    h = h or api.default_handle()
    cache = cache if cache is not None else Cache()
    name = torch.cuda.get_device_name()
    key = batch_key(problems, kind, deterministic, name)
    hit = cache.get(key)
    if hit is not None:
        return api.make_options(deterministic=deterministic, **{k: hit[k] for k in BATCH_FIELDS})
    orders = orders if orders is not None else [None] * len(problems)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for e in ev:
        e.record()
    bufs = []
    for pb in problems:
        if kind == "forward":
            bufs.append(dict(E=torch.zeros(pb.ext_shape, dtype=torch.float32, device=pb.device)))
        else:
            bufs.append(dict(dLdE=torch.randn(pb.ext_shape, dtype=torch.float32, device=pb.device),
                             dLdP=torch.zeros(pb.n_params(), dtype=torch.float32, device=pb.device)))
    items = [pb.batch_item(ray_order=o, **b) for pb, o, b in zip(problems, orders, bufs)]
    timings = []
    for cand in batch_candidates():
        opt = api.make_options(deterministic=deterministic, events=ev, **cand)
        fn = api.fr_trace_batch_forward if kind == "forward" else api.fr_trace_batch_adjoint
        call = lambda: fn(h, items, opt)
        try:
            t = _time_kernel(call, ev, reps, flush)
        except api.FreerayError:
            t = None
        timings.append((cand, t))
    best, t = pick_best(timings)
    default_ms = timings[0][1]
    cache.put(key, dict(best, ms=t, default_ms=default_ms))
    return api.make_options(deterministic=deterministic, **best)
