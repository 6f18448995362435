"""Benchmark of the differentiable freeform-lens trace on GB300.

Default workload (N = 1): collimated beam, 2048 x 2048 rays (4.2M), bicubic
16 x 16 control net, 128 x 128 bins over a 2 x 2 screen. One step is the whole
hot path: forward trace, squared-L2 loss and dL/dE, recompute adjoint to the
control heights, Adam, replayed from a CUDA graph. The headline `value` is
forward+adjoint rays per second over all GPUs; the forward-only rays/s, the
roofline of the dominant kernel (timed live with CUDA events on its stream),
an end-to-end figure through the public API with host buffers, the oracle on
the host cores, and secondary workloads (point source, batched graph steps)
are reported beside it on the same JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 it runs under torchrun, one rank per GPU; every rank traces its own
replica (the path has no exchange step), and the timing is the max over ranks.
`--impl reference` times the FP64 oracle on the host cores instead (the paper
publishes no code to run).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/s per forward+adjoint step vs forward-only at stated error; % roofline"
L2_FLUSH_BYTES = 256 << 20          # larger than the 129 MB L2

# Algorithmic FP32 work per collimated ray, counted from the formulas the
# kernels evaluate (FMA = 2 flops; +, -, *, exp2, rsqrt, reciprocal = 1):
# forward = trace 62 + filter 46 + deposit 26; adjoint = trace 62 + filter 46
# + reverse pass 161 + gradient moments 21.
FLOPS_FWD_COLLIMATED = 134
FLOPS_ADJ_COLLIMATED = 290
# DRAM bytes (read + write) per launch of each trace kernel on this workload,
# from one ncu capture of the collimated 2048x2048 workload (dram__bytes_read.sum +
# dram__bytes_write.sum of each trace kernel launch).
# Set to None whenever the kernel changes after that capture.
PROFILED_DRAM_BYTES = {"forward": 115712, "adjoint": 136960}


# Per-ray work of each trace kernel on the cases of counting_cases(), from one
# `ncu --metrics` capture of `python bench.py --counts` (the counts per launch divided by
# the case's rays):
#   warp: warp instructions issued; fp32: FP32 flops executed (FFMA 2, FADD and FMUL 1,
#   their packed pairs twice that); xu: thread operations on the XU pipe (MUFU and
#   conversions); satom: shared-memory atomic warp instructions. None where the kernels
#   changed after that capture.
COUNTS_PER_RAY = {
    "collimated_2048x2048": {
        "forward": {"warp": 8.543, "fp32": 139.2, "xu": 19.87, "satom": 0.257},
        "adjoint": {"warp": 13.948, "fp32": 289.1, "xu": 17.86, "satom": 0.154},
    },
    "plain_256x256": {
        "forward": {"warp": 10.229, "fp32": 147.6, "xu": 22.45, "satom": 0.244},
        "adjoint": {"warp": 21.341, "fp32": 334.2, "xu": 19.53, "satom": 1.014},
    },
    "point_4M": {
        "forward": {"warp": 24.746, "fp32": 402.8, "xu": 37.83, "satom": 0.235},
        "adjoint": {"warp": 32.935, "fp32": 719.4, "xu": 39.15, "satom": 0.304},
    },
    "grid_8x8_4M": {
        "forward": {"warp": 27.175, "fp32": 401.4, "xu": 43.85, "satom": 0.236},
        "adjoint": {"warp": 39.513, "fp32": 718.8, "xu": 43.52, "satom": 1.041},
    },
    "sweep_32_lenses_scaled": {
        "forward": {"warp": 24.821, "fp32": 350.5, "xu": 35.16, "satom": 0.233},
        "adjoint": {"warp": 29.767, "fp32": 612.8, "xu": 33.12, "satom": 0.369},
    },
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-extra", action="store_true", help="skip the secondary workloads")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--table", action="store_true",
                   help="also time the oracle on a sample of each of the five workloads (about a minute)")
    p.add_argument("--tune", action="store_true", help="autotune the trace kernels' schedule first")
    p.add_argument("--point-kernels", action="store_true",
                   help="time only the point-source trace kernels (16M rays), in id order and in the ray order")
    p.add_argument("--counts", action="store_true",
                   help="launch each trace kernel of the roofline table once on its counting case (run under "
                        "ncu --metrics to take the per-ray instruction counts of COUNTS_PER_RAY)")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_count, mhz):
    """FP32 FMA peak: SMs x 128 FP32 lanes x 2 flops x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


PROBES = (  # fr_probe kinds: name, kind, iterations per thread
    ("fp32_fma", 0, 4096), ("fp32_fma2", 1, 4096), ("xu_ex2", 2, 1024), ("xu_rsqrt", 3, 1024),
    ("xu_cvt", 4, 1024), ("shared_atom_u32", 5, 256), ("shared_atom_f32", 6, 256), ("global_red_v4", 7, 64))


def measure_ceilings(sm_count, repeats=5):
    """Throughput of each fr_probe kernel (operations per second, best of `repeats` launches timed
    by CUDA events on the launching stream): the measured ceilings of the trace kernels' roofline."""
    import torch
    from paper_2302_12031_gb300 import api
    h = api.default_handle()
    buf = torch.zeros(4 << 20, dtype=torch.float32, device="cuda")
    blocks, threads = sm_count * 8, 256
    out = {}
    for name, kind, iters in PROBES:
        best = 0.0
        for _ in range(repeats + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ops = api.fr_probe(h, kind, blocks, threads, iters, buf)
            b.record()
            b.synchronize()
            best = max(best, ops / (a.elapsed_time(b) * 1e-3))
        out[name] = best
    return out


def kernel_roofline(counts, n_rays, ms, sm_count, mhz, ceil):
    """Fractions of each ceiling one trace kernel reaches: per-ray counts x rays / kernel time
    against the issue rate (4 warp instructions per SM per clock), the FP32 FMA rate (128 lanes x 2
    flops per SM per clock), and the measured XU (MUFU ex2) and shared-atomic probe rates. The
    binding ceiling is the one with the largest fraction: no schedule can run the kernel faster
    than that resource allows."""
    if counts is None:
        return None
    t = ms * 1e-3
    issue_peak = sm_count * 4 * mhz * 1e6
    fp32_peak = sm_count * 128 * 2 * mhz * 1e6
    rows = {"issue": (counts["warp"] * n_rays / t, issue_peak, "warp inst/s"),
            "fp32": (counts["fp32"] * n_rays / t, fp32_peak, "flop/s"),
            "xu": (counts["xu"] * n_rays / t, ceil["xu_ex2"], "ops/s"),
            "shared_atomics": (counts["satom"] * n_rays / t, ceil["shared_atom_u32"] / 32.0, "warp inst/s")}
    out = {k: {"achieved": a, "peak": p, "unit": u, "frac": a / p} for k, (a, p, u) in rows.items()}
    binding = max(out, key=lambda k: out[k]["frac"])
    return {"binding": binding, "frac": out[binding]["frac"], "kernel_ms": ms, "ceilings": out}


def time_steps(fn, steps, warmup, flush):
    """Per-step device time (ms) of fn() with an L2 flush before every step."""
    import torch
    for _ in range(warmup):
        flush()
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        flush()
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def graphed(fn):
    """fn captured into a CUDA graph (after one eager run); returns its replay."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g.replay


def oracle_rays_per_s(wl, n_sample, begin):
    """The FP64 oracle (forward + gradient) on rays [begin, begin+n_sample)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    E, _ = O.trace_forward(wl, begin=begin, count=n_sample)
    _, d = O.loss_l2(wl, E)
    O.trace_gradient(wl, d, begin=begin, count=n_sample)
    dt = time.perf_counter() - t0
    return n_sample / dt, dt


def oracle_table():
    """The FP64 oracle (forward + gradient, all host cores) on a sample of each of the five
    workloads: all of the 256x256 grid; 2^20 consecutive rays from the middle of the 2048x2048
    grid; 2^14 consecutive ids from the middle of the point-source workloads (the oracle's
    first-root scan of the whole slab makes a point ray about a millisecond of one core);
    2^10 ids from the middle of each lens of the sweep."""
    from oracle import oracle as O
    from paper_2302_12031_gb300 import workloads as W
    out = {}
    for k in range(1, 6):
        wls = W.config(k)
        wls = wls if isinstance(wls, list) else [wls]
        if k == 1:
            samples, desc = [(wls[0], 0, wls[0]["n_rays"])], "all rays"
        elif k == 2:
            n = 1 << 20
            samples, desc = [(wls[0], wls[0]["n_rays"] // 2 - n // 2, n)], "2^20 consecutive rays, middle of the grid"
        elif k == 5:
            n = 1 << 10
            samples = [(w, w["n_rays"] // 2 - n // 2, n) for w in wls]
            desc = "2^10 consecutive ids from the middle of each of the 32 lenses"
        else:
            n = 1 << 14
            samples, desc = [(wls[0], wls[0]["n_rays"] // 2 - n // 2, n)], "2^14 consecutive ids, middle of the ids"
        rays = sum(c for _, _, c in samples)
        dt = sum(oracle_rays_per_s(w, c, b)[1] for w, b, c in samples)
        out["config_%d" % k] = {"rays_per_s": rays / dt, "rays": rays, "seconds": dt,
                                "cores": O.default_threads(), "sample": desc}
    return out


def run_reference(args, rank, world):
    """The oracle as the reference arm, on the host cores."""
    if rank != 0:
        return
    from paper_2302_12031_gb300 import workloads as W
    from oracle import oracle as O
    wl = W.config(2)
    n_sample = 1 << 16
    mid = wl["n_rays"] // 2
    for _ in range(max(1, args.warmup)):
        oracle_rays_per_s(wl, n_sample // 8, mid)
    times = []
    for k in range(args.steps):
        v, dt = oracle_rays_per_s(wl, n_sample, mid + (k % 4) * n_sample)
        times.append(dt)
    value = args.steps * n_sample / sum(times)
    line = {"metric": METRIC, "value": value, "unit": "rays/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "rays": wl["n_rays"], "sample_rays_per_step": n_sample},
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": O.default_threads(), "kind": "oracle",
                             "sample": "%d consecutive rays per step from the middle of the 2048x2048 grid, "
                                       "forward + gradient" % n_sample},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch
    from paper_2302_12031_gb300 import api, step
    from paper_2302_12031_gb300 import dist as D
    from paper_2302_12031_gb300 import workloads as W

    torch.cuda.set_device(local)
    D.init("nccl")
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    flush_buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def flush():
        flush_buf.zero_()

    wl = W.config(2)
    n_rays = wl["n_rays"]
    ev_f = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev_a = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for e in ev_f + ev_a:
        e.record()                      # materialise the events before handing out their handles
    torch.cuda.synchronize()
    sched_f, sched_a = {}, {}
    if args.tune:
        from paper_2302_12031_gb300 import autotune
        pb = api.Problem(wl)
        pick = lambda o: {k: getattr(o, k) for k in autotune.OPTION_FIELDS}
        sched_f = pick(autotune.tune(pb, "forward", flush=flush))
        sched_a = pick(autotune.tune(pb, "adjoint", flush=flush))
        del pb
    st = step.OptimStep(wl, lr=1e-3, graph=True, options=api.make_options(**sched_f),
                        adj_options=api.make_options(**sched_a))
    # The same step with event-record nodes around the two trace kernels, for
    # their durations: those nodes cost ~15 us per replay, so the headline
    # step is timed on the graph without them and the kernels on this one.
    st_ev = step.OptimStep(wl, lr=1e-3, graph=True, options=api.make_options(events=ev_f, **sched_f),
                           adj_options=api.make_options(events=ev_a, **sched_a))

    # --- headline: forward + loss + adjoint + Adam, one graph replay per step
    for _ in range(args.warmup):
        flush()
        st.step()
        flush()
        st_ev.step()
    D.barrier(dev)
    step_ms, fwd_kernel_ms, adj_kernel_ms, inst_step_ms = [], [], [], []
    with ClockSampler(local) as clocks:
        D.barrier(dev)
        for _ in range(args.steps):
            flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            st.step()
            b.record()
            b.synchronize()
            step_ms.append(a.elapsed_time(b))
        D.barrier(dev)
        for _ in range(args.steps):
            flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            st_ev.step()
            b.record()
            b.synchronize()
            inst_step_ms.append(a.elapsed_time(b))
            fwd_kernel_ms.append(ev_f[0].elapsed_time(ev_f[1]))
            adj_kernel_ms.append(ev_a[0].elapsed_time(ev_a[1]))
        D.barrier(dev)
    value, t_max = D.replica_throughput(n_rays * args.steps, sum(step_ms) * 1e-3, dev)
    ms_per_step = 1e3 * t_max / args.steps

    # --- forward only (prep + trace kernel through the C ABI)
    pb = st.problems[0]
    E = torch.empty(pb.ext_shape, dtype=torch.float32, device=dev)
    h = api.default_handle()

    def fwd():
        api.fr_trace_forward(h, pb.lens, pb.source, pb.target, pb.n_rays, pb.seed, 0, api.ALL_RAYS, None, E)

    f_ms = time_steps(graphed(fwd), args.steps, args.warmup, flush)
    fwd_value, _ = D.replica_throughput(n_rays, statistics.mean(f_ms) * 1e-3, dev)
    # rays by fate, outside the timed region
    stats = api.new_stats(dev)
    pb.forward(stats=stats)
    causes = ("on_screen", "aperture_miss", "out_of_domain", "tir", "off_screen", "invalid", "newton_fail", "other")
    by_cause = dict(zip(causes, (int(c) for c in stats.cpu().tolist())))

    # --- end to end through the public API: pinned host heights in, loss out
    # (the step's graph copies the heights in and the loss out: one launch and
    # one synchronisation per step)
    P_host = torch.as_tensor(wl["lens"]["P"], dtype=torch.float32).reshape(-1).pin_memory()
    loss_host = torch.zeros(1, dtype=torch.float64).pin_memory()
    st.attach_host_io(P_host, loss_host)
    e2e_ms, e2e_losses = [], []
    for k in range(args.warmup + args.steps):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st.step()
        torch.cuda.current_stream().synchronize()
        e2e_losses.append(float(loss_host[0]))
        if k >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    st.attach_host_io(None, None)
    e2e_value, _ = D.replica_throughput(n_rays, statistics.mean(e2e_ms) * 1e-3, dev)

    # --- roofline of the trace kernels, timed live: every ceiling they share
    # (issue slots, FP32, the XU pipe, shared-memory atomics) as a fraction of
    # its peak (the FP32 and issue peaks from the clock, the XU and atomic peaks
    # measured by the fr_probe kernels); the binding one is the largest
    pk, pk_kind = peaks()
    mhz = pk.get("sm_max_mhz", 2070.0)
    ceil = measure_ceilings(sm_count)
    fwd_k = statistics.mean(fwd_kernel_ms)
    adj_k = statistics.mean(adj_kernel_ms)
    dominant = "adjoint" if adj_k >= fwd_k else "forward"
    counts = COUNTS_PER_RAY.get("collimated_2048x2048") if COUNTS_PER_RAY else None
    per_kernel = {}
    for name, ms, fl in (("forward", fwd_k, FLOPS_FWD_COLLIMATED), ("adjoint", adj_k, FLOPS_ADJ_COLLIMATED)):
        rl = kernel_roofline(counts[name] if counts else None, n_rays, ms, sm_count, mhz, ceil) or {"kernel_ms": ms}
        alg = n_rays * fl / (ms * 1e-3) / 1e12
        rl["fp32_algorithmic"] = {"flops_per_ray": fl, "achieved": alg,
                                  "frac": alg / fp32_peak_tflops(sm_count, mhz), "unit": "TFLOP/s"}
        rl["traffic"] = PROFILED_DRAM_BYTES.get(name)
        per_kernel[name] = rl
    dom = per_kernel[dominant]
    if "ceilings" in dom:
        c = dom["ceilings"][dom["binding"]]
        roofline = {"bound": "alu", "binding": dom["binding"], "kernel": "k_%s (trace)" % dominant,
                    "achieved": c["achieved"], "peak": c["peak"], "unit": c["unit"], "frac": c["frac"]}
    else:
        fa = dom["fp32_algorithmic"]
        roofline = {"bound": "alu", "binding": "fp32", "kernel": "k_%s (trace)" % dominant, "achieved": fa["achieved"],
                    "peak": fp32_peak_tflops(sm_count, mhz), "unit": "TFLOP/s", "frac": fa["frac"]}
    roofline.update({
        "traffic": PROFILED_DRAM_BYTES.get(dominant),
        "traffic_unit": "bytes per launch (ncu dram__bytes_read+write)",
        "peak_note": "issue: %d SMs x 4 warp instructions x %.0f MHz; FP32: %d SMs x 128 lanes x 2 flops x %.0f MHz "
                     "(max SM clock of the %s peaks file); XU and shared atomics: fr_probe kernels, this run"
                     % (sm_count, mhz, sm_count, mhz, pk_kind),
        "counts_per_ray": "ncu instruction counts per ray of `bench.py --counts`" if counts else None,
        "probes": {k: v / 1e12 for k, v in ceil.items()}, "probe_unit": "T ops/s (FP32: TFLOP/s)",
        "per_kernel": per_kernel,
        "kernel_timing": "library events around each trace kernel in a second graph of the same step "
                         "(%.1f us per step with those event nodes, %.1f us without), same timed loop"
                         % (1e3 * statistics.mean(inst_step_ms), 1e3 * statistics.mean(step_ms))})

    line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["name"], "rays": n_rays, "control_net": "16x16", "bins": "128x128",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed between steps (256 MiB write)",
                       "step": "graph: clear, forward, loss, adjoint, Adam",
                       "schedule": {"forward": sched_f or "default", "adjoint": sched_a or "default"}},
            "forward_rays_per_s": fwd_value,
            "rays_by_cause": by_cause,
            "forward_ms": statistics.mean(f_ms),
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": "rays/s", "h2d_bytes_per_step": P_host.numel() * 4,
                    "d2h_bytes_per_step": 8},
            "gpu_launches": (st.launches_per_step() + st_ev.launches_per_step()) * args.steps,
            "clocks": clocks.summary()}

    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import oracle as O
        n_sample = 1 << 20
        v, dt = oracle_rays_per_s(wl, n_sample, n_rays // 2 - n_sample // 2)
        line["cpu_baseline"] = {"value": v, "unit": "rays/s", "cores": O.default_threads(), "kind": "oracle",
                                "sample": "%d consecutive rays from the middle of the grid, forward + gradient, "
                                          "%.1f s" % (n_sample, dt)}

    if not args.no_extra:
        line["extra"] = extra_workloads(args, flush, world, (sm_count, mhz, ceil))
    if rank == 0 and world == 1 and args.table:
        line["oracle_by_config"] = oracle_table()

    if rank == 0:
        print(json.dumps(line), flush=True)
    D.barrier(dev)
    if world > 1:
        torch.distributed.destroy_process_group()


def extra_workloads(args, flush, world, roof):
    """The 256x256-ray collimated lens, the point source (16M rays) and the batched graph steps,
    fewer steps each; for these four, the trace kernels' durations (library events in a second
    graph of the same step), forward-only rays/s from the forward kernel and each kernel's
    roofline (`roof`: SMs, clock, measured ceilings); then the mesh, two-face, loss and
    derivative-map variants."""
    import torch
    from paper_2302_12031_gb300 import api, step
    from paper_2302_12031_gb300 import dist as D
    from paper_2302_12031_gb300 import workloads as W
    out = {}
    k = max(3, args.steps // 4)
    autotune_fields = ("warps_per_cta", "rays_per_lane", "ctas_per_sm", "batch_waves")
    for name, wls in (("plain_256x256", W.config(1)), ("point_16M", W.config(3)),
                      ("grid_8x8_64M_batched_graph", W.config(4)), ("sweep_32_lenses_batched_graph", W.config(5))):
        opts = {}
        if name.startswith("sweep"):
            # the batch's schedule (waves of CTAs, warps, rays per lane) from the autotuner,
            # on the ray orders the step traces the point sources in
            from paper_2302_12031_gb300 import autotune
            pbs = [api.Problem(w) for w in wls]
            orders = [pb.ray_order() if pb.source.kind == api.FR_SOURCE_POINT else None for pb in pbs]
            cache = autotune.Cache()
            sched = {}
            for kind in ("forward", "adjoint"):
                o = autotune.tune_batch(pbs, kind, orders, cache=cache, flush=flush)
                opts[kind] = o
                hit = cache.get(autotune.batch_key(pbs, kind, False, torch.cuda.get_device_name()))
                sched[kind] = dict(hit)
            del pbs, orders
            torch.cuda.empty_cache()
        st = step.OptimStep(wls, lr=1e-3, graph=True, options=opts.get("forward"),
                            adj_options=opts.get("adjoint"))   # point sources: traced in the coherent ray order
        order_ms = None
        if any(o is not None for o in st.orders):
            # the orders depend on the sources and apertures only: built once per problem (time of the
            # builds alone, outside the step)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for pb, o in zip(st.problems, st.orders):
                if o is not None:
                    pb.ray_order()
            torch.cuda.synchronize()
            order_ms = 1e3 * (time.perf_counter() - t1)
        ms = time_steps(st.step, k, 2, flush)
        rays = st.n_rays
        rays_per_s, t = D.replica_throughput(rays, statistics.mean(ms) * 1e-3)
        out[name] = {"rays_per_step": rays, "ms_per_step": 1e3 * t, "rays_per_s": rays_per_s,
                     "steps_per_s": 1.0 / t, "lenses": len(st.problems)}
        if opts:
            out[name]["schedule"] = sched
        del st
        # the trace kernels of the same step, timed by library events in a second graph
        ev_f = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev_a = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        for e in ev_f + ev_a:
            e.record()
        torch.cuda.synchronize()
        def with_events(o, ev):
            e = api.make_options(events=ev)
            if o is not None:
                for f in autotune_fields:
                    setattr(e, f, getattr(o, f))
            return e
        st = step.OptimStep(wls, lr=1e-3, graph=True, options=with_events(opts.get("forward"), ev_f),
                            adj_options=with_events(opts.get("adjoint"), ev_a))
        f_ms, a_ms = [], []
        for _ in range(k + 2):
            flush()
            st.step()
            torch.cuda.synchronize()
            f_ms.append(ev_f[0].elapsed_time(ev_f[1]))
            a_ms.append(ev_a[0].elapsed_time(ev_a[1]))
        f_k, a_k = statistics.mean(f_ms[2:]), statistics.mean(a_ms[2:])
        case = COUNTED_AS.get(name)
        counts = COUNTS_PER_RAY.get(case) if COUNTS_PER_RAY and case else None
        sm_count, mhz, ceil = roof
        out[name]["forward_kernel_ms"] = f_k
        out[name]["adjoint_kernel_ms"] = a_k
        out[name]["forward_rays_per_s"] = rays / (f_k * 1e-3)
        out[name]["roofline"] = {
            kind: kernel_roofline(counts[kind] if counts else None, rays, kms, sm_count, mhz, ceil) or {"kernel_ms": kms}
            for kind, kms in (("forward", f_k), ("adjoint", a_k))}
        del st
        if order_ms is not None:
            st = step.OptimStep(wls, lr=1e-3, graph=True, ray_order=False)
            ms = time_steps(st.step, k, 2, flush)
            out[name]["ray_order_build_ms"] = order_ms
            out[name]["ms_per_step_in_id_order"] = statistics.mean(ms)
            del st
        torch.cuda.empty_cache()
    # triangle mesh (Sec. 2.2.2) against Newton on the 16M-ray point source:
    # step time, and the freeform hits' distance to Newton's on 2^16 rays
    wl3 = W.config(3)
    pb3 = api.Problem(wl3)
    newton = pb3.debug(0, 1 << 16)
    mesh_out = {}
    for n in (1, 2, 4, 8):
        opt = api.make_options(mesh=(n, n))
        st = step.OptimStep(wl3, lr=1e-3, graph=True, options=opt)
        ms = time_steps(st.step, k, 2, flush)
        rays_per_s, t = D.replica_throughput(st.n_rays, statistics.mean(ms) * 1e-3)
        m = pb3.debug(0, 1 << 16, options=opt)
        ok = (m["status"] == 0) & (newton["status"] == 0)
        dz = abs(m["z"][ok].astype("float64") - newton["z"][ok])
        mesh_out["%dx%d" % (n, n)] = {"ms_per_step": 1e3 * t, "rays_per_s": rays_per_s,
                                      "hit_dz_max": float(dz.max()), "hit_dz_rms": float((dz ** 2).mean() ** 0.5),
                                      "status_agree": float((m["status"] == newton["status"]).mean())}
        del st
    out["point_16M_triangle_mesh"] = mesh_out
    # both lens faces as freeforms (the paper's proposed extension): the step
    # optimises both nets (16x16 entry net for the collimated beam, 24x24 for
    # the point source)
    for name, wl2 in (("two_face_collimated_2048x2048", W.with_entry_face(W.config(2), 16, 0.01, 7)),
                      ("two_face_point_16M", W.with_entry_face(W.config(3), 24, 0.01, 8))):
        st = step.OptimStep(wl2, lr=1e-3, graph=True)
        ms = time_steps(st.step, k, 2, flush)
        rays_per_s, t = D.replica_throughput(st.n_rays, statistics.mean(ms) * 1e-3)
        out[name] = {"rays_per_step": st.n_rays, "ms_per_step": 1e3 * t, "rays_per_s": rays_per_s,
                     "parameters": st.n_params}
        del st
    # the paper's objective: normalised Frobenius loss, tanh-reparametrised heights
    # over a spherical offset (Table magndata, magnification 3)
    wl = W.config(2)
    st = step.OptimStep(wl, lr=1e-3, graph=True, loss="frobenius",
                        reparam=dict(z_min=-0.05, z_max=0.05, offset=("sphere", 0.0, 8.0)))
    ms = time_steps(st.step, k, 2, flush)
    rays_per_s, t = D.replica_throughput(st.n_rays, statistics.mean(ms) * 1e-3)
    out["frobenius_tanh_step_2048x2048"] = {"rays_per_step": st.n_rays, "ms_per_step": 1e3 * t,
                                            "rays_per_s": rays_per_s}
    pb = st.problems[0]
    h = api.default_handle()
    E = st.E[0]
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    dLdE = torch.empty_like(E)
    Eref = st.E_ref[0]
    for name, fn in (("l2", api.fr_loss_l2), ("frobenius", api.fr_loss_frobenius)):
        call = graphed(lambda: fn(h, E, Eref, pb.nx, pb.ny, pb.nu_x, pb.nu_y, loss, dLdE))
        out.setdefault("loss_kernel_us_128x128", {})[name] = 1e3 * statistics.mean(time_steps(call, k, 2, flush))
    del st
    # derivative maps (Sec. 3.1): flat lens, collimated 2048^2 rays, 16x16 net
    wl["lens"]["P"][:] = 0.0
    pb = api.Problem(wl)
    ncu_, ncv_ = pb.ctrl_shape
    one = torch.zeros((1, ncu_, ncv_), device="cuda")
    one[0, ncu_ // 2, ncv_ // 2] = 1.0
    dense = torch.randn((4, ncu_, ncv_), generator=torch.Generator(device="cpu").manual_seed(1)).cuda()
    for name, dP in (("derivative_map_1_control_point", one), ("derivative_maps_4_dense_directions", dense)):
        dE = torch.empty((dP.shape[0],) + pb.ext_shape, device="cuda")
        call = graphed(lambda: api.fr_trace_tangent(h, pb.lens, pb.source, pb.target, pb.n_rays, pb.seed, 0,
                                                    api.ALL_RAYS, None, dP, dP.shape[0], dE))
        ms = time_steps(call, k, 2, flush)
        rays_per_s, t = D.replica_throughput(pb.n_rays, statistics.mean(ms) * 1e-3)
        out[name] = {"rays": pb.n_rays, "directions": dP.shape[0], "ms": 1e3 * t, "rays_per_s": rays_per_s}
    return out


def run_point_kernels(args):
    """The point-source forward and adjoint trace kernels alone (16M rays, 24x24 net, 256^2 bins), each
    step launching the forward and the adjoint in ray-id order and then in the coherent ray order, every
    launch timed by CUDA events with an L2 flush before it. One JSON line of mean kernel times (us). Under
    ncu, the launches of step k are the (4 k)-th to (4 k + 3)-th trace kernels."""
    import torch
    from paper_2302_12031_gb300 import api
    from paper_2302_12031_gb300 import workloads as W
    wl = W.config(3, with_target=False)
    pb = api.Problem(wl)
    h = api.default_handle()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    order = pb.ray_order()
    torch.cuda.synchronize()
    build_ms = 1e3 * (time.perf_counter() - t0)
    E = torch.empty(pb.ext_shape, device="cuda")
    d = torch.randn(pb.ext_shape, generator=torch.Generator(device="cpu").manual_seed(1)).cuda()
    G = torch.empty(pb.ctrl_shape, device="cuda")
    scratch = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    opts = {"id": api.make_options(), "ray_order": api.make_options(ray_order=order)}
    calls = []
    for name in ("id", "ray_order"):
        calls.append(("forward", name, lambda o=opts[name]: api.fr_trace_forward(
            h, pb.lens, pb.source, pb.target, pb.n_rays, pb.seed, 0, api.ALL_RAYS, o, E)))
    for name in ("id", "ray_order"):
        calls.append(("adjoint", name, lambda o=opts[name]: api.fr_trace_adjoint(
            h, pb.lens, pb.source, pb.target, pb.n_rays, pb.seed, 0, api.ALL_RAYS, o, d, G)))
    times = {}
    for step_no in range(args.warmup + args.steps):
        for kind, name, fn in calls:
            scratch.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            if step_no >= args.warmup:
                times.setdefault(kind, {}).setdefault(name, []).append(1e3 * a.elapsed_time(b))
    out = {"workload": wl["name"], "rays": pb.n_rays, "ray_order_build_ms": build_ms,
           "kernel_us": {k: {n: statistics.mean(v) for n, v in d_.items()} for k, d_ in times.items()}}
    print(json.dumps(out), flush=True)


# The counting case whose per-ray counts stand for each secondary workload.
COUNTED_AS = {"plain_256x256": "plain_256x256", "point_16M": "point_4M", "grid_8x8_64M_batched_graph": "grid_8x8_4M",
              "sweep_32_lenses_batched_graph": "sweep_32_lenses_scaled"}


def counting_cases():
    """The cases whose trace kernels the per-ray counts are taken on: the headline collimated
    workload, the 256x256-ray one, and the point-source, grid-of-sources and sweep workloads
    with fewer rays (the same lenses, screens and schedules; the counts are per ray). Each
    entry: (name, workloads, ray-order flag)."""
    from paper_2302_12031_gb300 import workloads as W
    w3 = W.config(3)
    w3["n_rays"] = 1 << 22
    w4 = W.config(4)
    w4["n_rays"] = 64 << 16
    sweep = W.design_sweep(32, seed=6, min_rays=1 << 16, max_rays=1 << 20)
    return [("collimated_2048x2048", [W.config(2)], False), ("plain_256x256", [W.config(1)], False),
            ("point_4M", [w3], True),
            ("grid_8x8_4M", [w4], True), ("sweep_32_lenses_scaled", sweep, True)]


def run_counts(args):
    """Each counting case: one forward and one adjoint launch of its step's trace kernels, in
    the order of counting_cases()."""
    import torch
    from paper_2302_12031_gb300 import step
    for name, wls, order in counting_cases():
        st = step.OptimStep(wls, lr=1e-3, graph=False, ray_order=order)
        torch.cuda.synchronize()
        st._clear()
        st._forward()
        st._loss()
        st._adjoint()
        torch.cuda.synchronize()
        print(json.dumps({"case": name, "rays": st.n_rays}), flush=True)
        del st
        torch.cuda.empty_cache()


def main():
    args = parse()
    from paper_2302_12031_gb300 import dist as D
    rank, world, local = D.env()
    if args.counts:
        run_counts(args)
    elif args.point_kernels:
        run_point_kernels(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
