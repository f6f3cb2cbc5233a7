"""Benchmark of the sky cross-match hot path (one JSON line on stdout).

A step is one pass of the whole path over one synthetic workload: build the
index of catalogue B (ingest, radix sort on (zone, RA), bucket tables, cell
offsets), match catalogue A against it with both selections (all pairs and
best pair), and build the "1 or 2" join rows. Default workload: the
clump-vs-compact-source case of the paper's §3 use, A = 200,000 per-source
ellipses against B = 5,000,000 point sources in galactic coordinates.

value      A sources per second over K timed steps, inputs resident in HBM,
           float32 path with float64 recheck; L2 flushed before every step.
e2e        the same step through the C ABI with pinned host buffers, the
           host->device copies of the catalogues and the device->host copy of
           the join rows and best pairs inside the timed region.
fp64_path  the same step on the all-float64 path.
roofline   the dominant kernel, timed with CUDA events on its stream during
           the timed steps, against the measured HBM copy bandwidth.
cpu_baseline  the FP64 CPU oracle on a bounded sample of the same workload.

--impl reference times that oracle as the reference arm. Under torchrun
(N > 1) each rank runs its own copy of the workload (weak scaling, no
data-path collective); rank 0 prints the line with the max time over ranks.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "A-sources cross-matched/sec, FP32+FP64-recheck vs FP64 path; serving p99 ms"
UNIT = "A-sources/s"
KERNELS_FOR_ROOFLINE = ("k_scan_fp32_count", "k_digit_scatter", "k_scan_fp32_emit", "k_gather_b")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--zone-height", type=float, default=0.0, help="arcsec; 0 = tuned default")
    p.add_argument("--cpu-sample", type=int, default=0, help="A sources in the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--serve-seconds", type=float, default=60.0,
                   help="serving window after a warm-up of 1/6 of it; 0 skips the serving leg")
    p.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrivals per second")
    p.add_argument("--serve-b", type=int, default=300_000_000, help="resident B sources")
    p.add_argument("--serve-pool", type=int, default=256, help="distinct request payloads")
    p.add_argument("--serve-slots", type=int, default=3)
    p.add_argument("--c3-scale", type=float, default=1.0, help="0 skips the all-sky C3 leg")
    p.add_argument("--c4-requests", type=int, default=4096, help="0 skips the batched C4 leg")
    p.add_argument("--c4-b", type=int, default=100_000_000, help="resident B of the C4 leg")
    p.add_argument("--values-scale", type=float, default=1.0,
                   help="0 skips the Exact Value leg (A 5e7 x B 2e8 int64 keys at 1)")
    return p.parse_args()


def max_over_ranks(local_ms, world, device):
    """The slowest rank's time (every rank gets it): the job's time."""
    if world <= 1:
        return local_ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def weak_scaling_value(units_per_rank, steps, world, job_ms):
    """Whole-job throughput: every rank processed its own units each step."""
    return world * units_per_rank * steps / (job_ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(seed_offset=0, scale=1.0):
    """The C2 workload of one rank: ranks draw different catalogues of the
    same shape (seed 1002 + rank)."""
    from paper_1611_08494_gb300 import synth

    d = synth.c2(seed=1002 + seed_offset, scale=scale)
    d["desc"] = ("c2 clump-vs-compact-source: A=200000 per-source ellipses (a 5-60 arcsec "
                 "log-uniform, b/a 0.3-1, PA 0-180), B=5000000, galactic l 0-60 |b|<=1 "
                 "density exp(-|b|/0.3deg)")
    return d


# ------------------------------------------------------------------- oracle

def oracle_sample(d, n_sample, nthreads):
    """Times the oracle (as it stands) on the first n_sample A sources against
    all of B: its voxel indexing of B, the pair tests and best selection."""
    import oracle

    sub = np.arange(n_sample, dtype=np.int64)
    t = time.perf_counter()
    r = oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], a_frame=d["a_frame"],
                     b_frame=d["b_frame"], subset=sub, nthreads=nthreads, **d["region"])
    oracle.best(r, d["a_lon"].size)
    return time.perf_counter() - t


def cpu_baseline(d, n_sample=0):
    nthreads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    if not n_sample:
        # size the sample so the run takes ~10-20 s of CPU work: the time of
        # a sample is a fixed part (the oracle's grid over all of B) plus a
        # part per A source, estimated from two small samples
        t1 = oracle_sample(d, 2000, nthreads)
        t2 = oracle_sample(d, 12000, nthreads)
        per_a = max((t2 - t1) / 10000, 1e-9)
        fixed = max(t1 - 2000 * per_a, 0.0)
        n_sample = int(min(d["a_lon"].size, max(2000, (12.0 - fixed) / per_a)))
    dt = oracle_sample(d, n_sample, nthreads)
    return {"value": n_sample / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"first {n_sample} of {d['a_lon'].size} A sources against all "
                      f"{d['b_lon'].size} B (voxel grid over B, pair tests, best), "
                      f"{dt:.2f} s on {nthreads} threads"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    d = workload()
    nthreads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    # each step is a bounded sample, sized so the K steps take about a minute
    dt = oracle_sample(d, 2000, nthreads)
    per_step_s = 60.0 / max(args.steps, 1)
    n_s = args.cpu_sample or int(min(d["a_lon"].size, max(200, 2000 * per_step_s / max(dt, 1e-3))))
    cb = {"kind": "oracle", "cores": nthreads, "unit": UNIT,
          "sample": f"first {n_s} of {d['a_lon'].size} A sources per step against all "
                    f"{d['b_lon'].size} B (voxel grid over B, pair tests, best), "
                    f"{nthreads} threads"}
    times = []
    for _ in range(args.warmup):
        oracle_sample(d, min(n_s, 2000), nthreads)
    for _ in range(args.steps):
        times.append(oracle_sample(d, n_s, nthreads))
    tot = sum(times)
    v = n_s * len(times) / tot
    cb = dict(cb, value=v)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": d["desc"], "sample_a": n_s},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- GPU arm

class Clocks:
    """nvidia-smi sampling of the SM clock and throttle reasons. The sampler
    is started, its first sample awaited, then the timed region runs; only
    samples taken between mark_start() and mark_end() are summarised."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.p = None
        self.lines = []
        self.t0 = self.t1 = None

    def _reader(self):
        for ln in self.p.stdout:
            self.lines.append((time.monotonic(), ln))

    def __enter__(self):
        import threading

        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
            return self
        self.th = threading.Thread(target=self._reader, daemon=True)
        self.th.start()
        t_end = time.monotonic() + 5.0
        while not self.lines and time.monotonic() < t_end:
            time.sleep(0.02)
        return self

    def mark_start(self):
        self.t0 = time.monotonic()

    def mark_end(self):
        self.t1 = time.monotonic()

    def __exit__(self, *exc):
        if self.p:
            time.sleep(0.15)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
            self.th.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0 = self.t0 if self.t0 is not None else -1e30
        t1 = (self.t1 if self.t1 is not None else 1e30) + 0.1
        for t, ln in self.lines:
            if not (t0 <= t <= t1):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def nvtx_push(name):
    """Marks the timed region for profilers (ncu --nvtx-include)."""
    try:
        import torch

        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch

        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


# Source files each profiled kernel is built from: a DRAM-traffic record from
# ncu is used only while these files are unchanged.
KERNEL_SOURCES = {
    "k_onesweep": ("xm_sort.cu", "xm_internal.cuh"),
    "k_scan_fp32_count": ("xm_scan.cuh", "xm_internal.cuh"),
    "k_gather_b": ("xm_index.cu", "xm_internal.cuh"),
    "k_ingest_b": ("xm_index.cu", "xm_internal.cuh"),
}


def source_hash(kernel):
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_1611_08494_gb300", "csrc")
    for f in KERNEL_SOURCES.get(kernel, sorted(os.listdir(cs))):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(cs, f), "rb").read())
    return h.hexdigest()[:16]


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1611_08494_gb300 import xm

    d = workload(seed_offset=rank)
    n_a, n_b = d["a_lon"].size, d["b_lon"].size
    cu = lambda x: torch.as_tensor(np.ascontiguousarray(x), device="cuda")  # noqa: E731
    dev = {k: cu(d[k]) for k in ("a_lon", "a_lat", "b_lon", "b_lat")}
    reg_dev = {k: (cu(v) if isinstance(v, np.ndarray) else v) for k, v in d["region"].items()}
    zone_h = args.zone_height or 12.0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    host_out = {}

    def step(prec, fp64_index, cols=None, reg=None, copy_out=False, out_slot=0, idx=None):
        cols = cols or dev
        reg = reg or reg_dev
        # the build's input check is read at the match's synchronisation
        if idx is None:
            idx = xm.Index(cols["b_lon"], cols["b_lat"], frame=d["b_frame"],
                           zone_height_arcsec=zone_h, build_fp64=fp64_index, deferred_check=True)
        res = xm.Result(idx, cols["a_lon"], cols["a_lat"], frame=d["a_frame"], precision=prec,
                        selection=xm.SEL_ALL | xm.SEL_BEST, **reg)
        rows = res.join("or")
        out = None
        if copy_out:
            # results to pinned host buffers (allocated once, the sizes repeat)
            srcs = [rows.a_row, rows.b_row, rows.sep, res.best_b, res.best_sep]
            key = (out_slot,) + tuple(t.numel() for t in srcs)
            slot = host_out.setdefault(out_slot, {})
            if slot.get("key") != key:
                slot["key"] = key
                slot["bufs"] = [torch.empty(t.numel(), dtype=t.dtype).pin_memory() for t in srcs]
            out = slot["bufs"]
            for dst, src in zip(out, srcs):
                dst.copy_(src, non_blocking=True)
        return idx, res, rows, out

    def timed(prec, fp64_index, steps, warmup, cols=None, reg=None, copy_out=False,
              profile=False, clocks=None):
        for _ in range(warmup):
            step(prec, fp64_index, cols, reg, copy_out)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        xm.reset_stats()
        if profile:
            xm.prof_enable(True)
        if clocks:
            clocks.mark_start()
            nvtx_push("xm_timed")
        ms, bytes_out = [], 0
        for _ in range(steps):
            flush.zero_()  # evict the inputs from L2 between steps
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, res, rows, out = step(prec, fp64_index, cols, reg, copy_out)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            if out is not None:
                bytes_out = sum(t.numel() * t.element_size() for t in out)
        torch.cuda.synchronize()
        if clocks:
            nvtx_pop()
            clocks.mark_end()
        prof = xm.prof_all() if profile else {}
        if profile:
            xm.prof_enable(False)
        st = xm.stats()
        if world > 1:
            dist.barrier()
        return ms, st, prof, res, rows, bytes_out

    # float32 + float64 recheck (the product path), uninstrumented
    with Clocks(local) as clk:
        ms, st, _, res, rows, _ = timed(xm.PREC_FP32, False, args.steps, args.warmup, clocks=clk)
    total_ms = max_over_ranks(sum(ms), world, "cuda")
    value = weak_scaling_value(n_a, args.steps, world, total_ms)
    launches = st["kernel_launches"]

    # the same steps again with an event pair around every launch: per-kernel
    # times for the shares and the roofline (the events cost a little time,
    # so these steps are not the ones the value comes from)
    prof_steps = max(10, args.steps // 4)
    ms_p, st_p, prof, _, _, _ = timed(xm.PREC_FP32, False, prof_steps, 1, profile=True)

    # all-float64 path
    ms64, _, _, _, _, _ = timed(xm.PREC_FP64, True, max(3, args.steps // 2), 1)
    v64 = n_a * len(ms64) / (sum(ms64) / 1e3)

    # end to end through the C ABI from pinned host memory
    host = {k: torch.as_tensor(d[k]).pin_memory() for k in ("a_lon", "a_lat", "b_lon", "b_lat")}
    reg_host = {k: (torch.as_tensor(v).pin_memory() if isinstance(v, np.ndarray) else v)
                for k, v in d["region"].items()}
    ms_e2e, _, _, _, _, d2h = timed(xm.PREC_FP32, False, max(3, args.steps // 2), 1, cols=host,
                                    reg=reg_host, copy_out=True)
    h2d = sum(t.numel() * t.element_size() for t in host.values()) + \
        sum(t.numel() * t.element_size() for t in reg_host.values() if hasattr(t, "numel"))
    v_e2e = n_a * len(ms_e2e) / (sum(ms_e2e) / 1e3)

    # the same, pipelined as a throughput-bound user would run it: steps go
    # to two streams in turn, and each step's index build (with its input
    # copy) is issued before the previous step's match, whose pair count
    # holds the host; so one step's input copy and build overlap the
    # previous step's match, and its result copy the next step's work (each
    # step still copies all of its inputs in and its result out; the clock
    # covers the whole run)
    def e2e_pipelined(n_steps, warmup):
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        in_flight = [None, None]

        def build(k):
            with torch.cuda.stream(streams[k % 2]):
                flush.zero_()
                return xm.Index(host["b_lon"], host["b_lat"], frame=d["b_frame"],
                                zone_height_arcsec=zone_h, deferred_check=True)

        def finish(k, idx):
            with torch.cuda.stream(streams[k % 2]):
                in_flight[k % 2] = step(xm.PREC_FP32, False, host, reg_host, True,
                                        out_slot=k % 2, idx=idx)

        def run(n):
            nxt = build(0)
            for k in range(n):
                idx, nxt = nxt, (build(k + 1) if k + 1 < n else None)
                finish(k, idx)

        run(warmup)
        torch.cuda.synchronize()
        cur = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for st in streams:
            st.wait_event(e0)
        run(n_steps)
        for st in streams:
            cur.wait_stream(st)
        e1.record(cur)
        e1.synchronize()
        in_flight[0] = in_flight[1] = None
        return e0.elapsed_time(e1)

    n_pipe = max(3, args.steps // 2)
    ms_pipe = e2e_pipelined(n_pipe, 2)
    v_e2e_pipe = n_a * n_pipe / (ms_pipe / 1e3)

    # roofline of the dominant kernel
    roof = roofline(prof, st_p, prof_steps, n_a, n_b, zone_h, sum(ms_p))

    # further readings of "best pairs" over the C2 pair list (index resident)
    picks = pick_leg(xm, torch, step, stream)

    if rank != 0:
        return
    peaks = load_peaks()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": d["desc"], "n_a": n_a, "n_b": n_b,
                   "step": "build B index + match (all and best pairs) + join '1 or 2'",
                   "precision": "float32 tests, float64 recheck in the guard band",
                   "zone_height_arcsec": zone_h, "l2": "flushed (256 MiB write) before each step",
                   "index_check": "deferred to the match's synchronisation",
                   "pairs": int(res.n_pairs), "join_rows": int(rows.n)},
        "e2e": {"value": v_e2e_pipe, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "mode": "two streams in turn, each step's index build (and input copy) issued "
                        "before the previous step's match: copies overlap the neighbouring "
                        "steps' work; L2 flushed before each step",
                "serial_value": v_e2e,
                "serial_mode": "one step at a time, events around each step"},
        "fp64_path": {"value": v64, "unit": UNIT, "ms_per_step": statistics.mean(ms64)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": clk.summary(),
        "picks": picks,
        "kernels_ms_per_step": {k: round(v[0] / prof_steps, 4) for k, v in
                                sorted(prof.items(), key=lambda kv: -kv[1][0])[:16]},
        "profiled_ms_per_step": sum(ms_p) / prof_steps,
        "stats_per_step": {k: v // args.steps for k, v in st.items()},
        "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "source": peaks.get("_source")},
    }
    if world == 1 and args.c3_scale > 0:
        line["c3"] = c3_leg(args, xm, torch)
    if world == 1 and args.c4_requests > 0:
        line["c4"] = c4_leg(args, xm, torch)
    if world == 1 and args.values_scale > 0:
        line["exact_value"] = values_leg(args, xm, torch)
    if world == 1 and args.serve_seconds > 0:
        line["serving"] = serving_leg(args, xm, torch)
    elif world > 1:
        line["serving"] = {"skipped": "the serving leg runs at N = 1 only"}
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(d, args.cpu_sample)
    print(json.dumps(line), flush=True)


def pick_leg(xm, torch, step, stream):
    """Best pair per B source and mutual best pairs over one C2 result:
    device time of xm_pick_pairs (median of 10) and pairs per second; the
    same for the normalised distances and concentric levels."""
    idx, res, _, _ = step(xm.PREC_FP32, False)
    out = {"pairs_in": int(res.n_pairs)}
    for kind in ("best_b", "mutual"):
        ms = []
        for k in range(11):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rows = res.pick(kind)
            e1.record(stream)
            e1.synchronize()
            if k:
                ms.append(e0.elapsed_time(e1))
        out[kind] = {"ms": statistics.median(ms), "rows": int(rows.n),
                     "pairs_per_s": res.n_pairs / (statistics.median(ms) / 1e3)}
    # normalised distance of every pair, best pair by it, and three concentric
    # copies of each ellipse (xm_levels_compute)
    ms = []
    for k in range(11):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lv = res.levels([0.25, 0.5, 0.75])
        e1.record(stream)
        e1.synchronize()
        if k:
            ms.append(e0.elapsed_time(e1))
        del lv
    out["levels"] = {"scales": [0.25, 0.5, 0.75], "ms": statistics.median(ms),
                     "pairs_per_s": res.n_pairs / (statistics.median(ms) / 1e3)}
    return out


# ------------------------------------------------------- all-sky C3 leg

def c3_leg(args, xm, torch):
    """The all-sky circle workload at full size (A = 5e7, B = 2e8 by
    default): index build, then match with both selections, FP32 + recheck
    and all-FP64; the scan's count pass against the HBM roofline."""
    from paper_1611_08494_gb300 import synth_gpu

    d = synth_gpu.c3(scale=args.c3_scale)
    n_a, n_b = d["a_lon"].numel(), d["b_lon"].numel()
    stream = torch.cuda.current_stream()
    out = {"workload": f"c3 all-sky circle r=2 arcsec: A={n_a}, B={n_b}, density 1+9exp(-|b|/10deg), "
                       "poles and 0/360 seam, int64 ids, galactic", "steps": 3}
    peak = load_peaks().get("hbm_gbs", 6800.0)
    for prec, fp64_index, name in ((xm.PREC_FP32, False, "fp32_recheck"), (xm.PREC_FP64, True, "fp64")):
        t_build, t_match = [], []
        for k in range(5):  # a warm-up, three timed passes, one profiled
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            if k == 4:
                xm.reset_stats()
                xm.prof_enable(True)
                nvtx_push(f"c3_{name}")
            e0.record(stream)
            idx = xm.Index(d["b_lon"], d["b_lat"], frame=d["b_frame"], ids=d["b_id"],
                           zone_height_arcsec=12.0, build_fp64=fp64_index)
            e1.record(stream)
            res = xm.Result(idx, d["a_lon"], d["a_lat"], frame=d["a_frame"], precision=prec,
                            selection=xm.SEL_ALL | xm.SEL_BEST, **d["region"])
            e2.record(stream)
            e2.synchronize()
            if k == 4:
                nvtx_pop()
            if 1 <= k <= 3:
                t_build.append(e0.elapsed_time(e1))
                t_match.append(e1.elapsed_time(e2))
            pairs = int(res.n_pairs)
            del res, idx
        prof = xm.prof_all()
        xm.prof_enable(False)
        st = xm.stats()
        scan = prof.get("k_scan_fp32_count" if prec == xm.PREC_FP32 else "k_scan_fp64_count")
        entry = {"a_per_s_match": n_a / (statistics.median(t_match) / 1e3),
                 "a_per_s_step": n_a / ((statistics.median(t_match) + statistics.median(t_build)) / 1e3),
                 "index_build_ms": statistics.median(t_build), "match_ms": statistics.median(t_match),
                 "pairs": pairs, "candidates": int(st["candidates"]),
                 "kernels_ms": {k: round(v[0], 3) for k, v in
                                sorted(prof.items(), key=lambda kv: -kv[1][0])[:8]}}
        if scan:
            alg = n_a * (16 + 24 + 16) + st["candidates"] * 12
            ach = alg / (scan[0] / scan[1] * 1e-3) / 1e9
            entry["scan_roofline"] = {"kernel": "k_scan count pass", "bound": "hbm",
                                      "algorithmic_bytes": alg, "ms": scan[0] / scan[1],
                                      "achieved": ach, "peak": peak, "unit": "GB/s",
                                      "frac": ach / peak, "peak_source": "of measured"}
        out[name] = entry
    del d
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------- Exact Value case leg

def values_leg(args, xm, torch):
    """The Exact Value functional case: int64 keys, A = 5e7 and B = 2e8 at
    scale 1 (repeats on the B side). A step sorts B's keys, finds every A key
    and writes all pairs and the best pairs; the dominant kernel (the sort
    pass) against the HBM roofline."""
    from paper_1611_08494_gb300 import synth_gpu

    n_a, n_b = int(5e7 * args.values_scale), int(2e8 * args.values_scale)
    d = synth_gpu.values(n_a=n_a, n_b=n_b)
    stream = torch.cuda.current_stream()
    ms = []
    for k in range(5):  # a warm-up, three timed passes, one profiled
        if k == 4:
            xm.reset_stats()
            xm.prof_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = xm.ValueResult(d["a_keys"], d["b_keys"], selection=xm.SEL_ALL | xm.SEL_BEST)
        e1.record(stream)
        e1.synchronize()
        if 1 <= k <= 3:
            ms.append(e0.elapsed_time(e1))
        pairs = int(res.n_pairs)
        del res
    prof = xm.prof_all()
    xm.prof_enable(False)
    peak = load_peaks().get("hbm_gbs", 6800.0)
    out = {"workload": f"exact value: int64 keys, A={n_a} (60 % present in B), B={n_b} "
                       "(10 % repeats)", "pairs": pairs, "ms": statistics.median(ms),
           "a_per_s": n_a / (statistics.median(ms) / 1e3),
           "kernels_ms": {k: round(v[0], 3) for k, v in
                          sorted(prof.items(), key=lambda kv: -kv[1][0])[:6]}}
    sw = prof.get("k_onesweep")
    if sw:
        alg = 24.0 * xm.stats()["sort_key_passes"] / sw[1]  # key and row, read and written
        ach = alg / (sw[0] / sw[1] * 1e-3) / 1e9
        out["roofline"] = {"kernel": "k_onesweep", "bound": "hbm", "algorithmic_bytes": alg,
                           "ms_per_launch": sw[0] / sw[1], "achieved": ach, "peak": peak,
                           "unit": "GB/s", "frac": ach / peak, "peak_source": "of measured"}
    del d
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------- batched C4 leg

def c4_leg(args, xm, torch):
    """Batched jobs (C4): thousands of uneven requests against one resident
    B index, matched by one persistent scan launched as a CUDA graph; the
    zone height and grid come from the autotuner on a sample of the
    requests. Times the whole batch pass (device events around the graph
    launch and its arenas) and reports A sources per second."""
    from paper_1611_08494_gb300 import synth_gpu

    t0 = time.perf_counter()
    d = synth_gpu.c4(n_b=args.c4_b, n_req=args.c4_requests)
    reqs = [dict(lon=q["lon"], lat=q["lat"], selection=q["selection"], join=q["join"],
                 join_selection=q["join_selection"], **q["region"]) for q in d["requests"]]
    total_a = sum(q["lon"].numel() for q in d["requests"])
    sample = reqs[:: max(1, len(reqs) // 64)]
    tuned = xm.autotune(d["b_lon"], d["b_lat"], sample, frame=d["b_frame"],
                        zone_heights=(10.0, 20.0, 40.0), blocks_per_sm=(2, 4, 8))
    idx = xm.Index(d["b_lon"], d["b_lat"], frame=d["b_frame"],
                   zone_height_arcsec=tuned["zone_height_arcsec"])
    setup_s = time.perf_counter() - t0
    ms = []
    for k in range(4):
        b = xm.Batch(idx, reqs, use_graph=True, persistent_blocks=tuned["persistent_blocks"])
        info = b.info()
        if k:
            ms.append(info["device_ms"])
        del b
    out = {"workload": f"c4 batched: {len(reqs)} requests (n_A log-uniform 1e2-1e6, caps 0.1-10 deg, "
                       f"mixed shapes/sizes/joins) against B={args.c4_b} uniform all-sky",
           "requests": len(reqs), "total_a": int(total_a), "pairs": int(info["total_pairs"]),
           "batch_ms": statistics.median(ms), "a_per_s": total_a / (statistics.median(ms) / 1e3),
           "launch": "one persistent scan in one CUDA graph per batch pass",
           "zone_height_arcsec": tuned["zone_height_arcsec"],
           "persistent_blocks": tuned["persistent_blocks"], "tune_trials": tuned["trials"],
           "setup_s": setup_s}
    del d, reqs, idx
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------- serving leg

def serving_leg(args, xm, torch):
    """Poisson arrivals against a resident B index through the library's
    serving loop (continuous batching, admission by free device memory).
    Requests take their payloads from a pool of pre-generated device
    requests; latency is submit -> results complete on the device."""
    import threading

    from paper_1611_08494_gb300 import synth_gpu

    t_setup = time.perf_counter()
    b = synth_gpu.c5_catalogue(n_b=args.serve_b)
    pool = synth_gpu.c5_requests(b, n_pool=args.serve_pool)
    sample = [dict(q, lon=q["lon"], lat=q["lat"], **q["region"]) for q in pool[:6]]
    for q in sample:
        q.pop("region")
    tuned = xm.autotune(b["b_lon"], b["b_lat"], sample, frame=b["b_frame"],
                        zone_heights=(10.0, 20.0, 40.0), blocks_per_sm=(2, 4))
    idx = xm.Index(b["b_lon"], b["b_lat"], frame=b["b_frame"], ids=b["b_id"],
                   zone_height_arcsec=tuned["zone_height_arcsec"])
    del b
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    setup_s = time.perf_counter() - t_setup

    warm = args.serve_seconds / 6.0
    times, h = synth_gpu.poisson_arrivals(args.serve_rate, warm + args.serve_seconds)
    which = h.integers(0, len(pool), len(times))
    srv = xm.Server(idx, slots=args.serve_slots, precision=xm.PREC_FP32, use_graph=True,
                    persistent_blocks=tuned["persistent_blocks"])
    tickets = []
    done = threading.Event()
    lock = threading.Lock()

    def complete():
        k = 0
        while True:
            with lock:
                t = tickets[k] if k < len(tickets) else None
            if t is None:
                if done.is_set():
                    with lock:
                        if k >= len(tickets):
                            return
                    continue
                time.sleep(0.0005)
                continue
            try:
                t.wait(600_000)
            except xm.XMError:
                pass
            t.release()
            k += 1

    th = threading.Thread(target=complete, daemon=True)
    th.start()
    offered_a = 0
    t0 = time.perf_counter()
    reset_done = False
    for t_arr, w in zip(times, which):
        now = time.perf_counter() - t0
        if t_arr > now:
            time.sleep(t_arr - now)
        if not reset_done and t_arr >= warm:
            srv.reset_stats()
            t_win = time.perf_counter()
            reset_done = True
        q = pool[w]
        tk = srv.submit(q["lon"], q["lat"], frame=q["frame"], selection=q["selection"],
                        join=q["join"], join_selection=q["join_selection"], **q["region"])
        with lock:
            tickets.append(tk)
        if reset_done:
            offered_a += q["lon"].numel()
    done.set()
    th.join()
    t_end = time.perf_counter()
    st = srv.stats()
    srv.close()
    window = t_end - t_win if reset_done else float("nan")
    out = {"workload": f"c5 serving: B={args.serve_b} resident (C3 latitude profile, galactic, "
                       f"int64 ids), Poisson {args.serve_rate:g} req/s, n_A log-uniform 1e3-1e7, "
                       "mixed shapes/joins/frames, admission by free HBM",
           "window_s": args.serve_seconds, "warmup_s": warm, "requests": int(st["completed"]),
           "failed": int(st["failed"]), "refused": int(st["refused"]),
           "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
           "sustained_a_per_s": st["a_sources"] / window,
           "offered_a_per_s": offered_a / args.serve_seconds,
           "drain_s": window - args.serve_seconds, "batches": int(st["batches"]),
           "busy_s": st["busy_s"], "slots": args.serve_slots, "pool": len(pool),
           "zone_height_arcsec": tuned["zone_height_arcsec"],
           "persistent_blocks": tuned["persistent_blocks"], "setup_s": setup_s}
    del pool, idx
    torch.cuda.empty_cache()
    return out


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "_source": "fallback"}


def algorithmic_bytes(kernel, st, steps, launches, n_a, n_b, zone_h):
    """Bytes the method must move per launch of a kernel (averaged over the
    launches, so achieved = all bytes / all kernel time):
    k_onesweep   per key and pass 8 B key + 4 B row, read and written, over
                 the passes that ran (the library counts keys x passes; an
                 index sort planned to fewer passes launches the rest empty);
    k_scan_fp32_count  per A 16 B position + 24 B region columns + 16 B best
                 row, per candidate 12 B (offsets + RA key);
    k_gather_b   per B 16 B position read + 16 B record + 16 B position
                 written."""
    if kernel == "k_onesweep":
        return 24.0 * st["sort_key_passes"] / launches
    if kernel == "k_scan_fp32_count":
        return n_a * (16 + 24 + 16) + st["candidates"] / steps * 12
    if kernel == "k_gather_b":
        return n_b * (16 + 16 + 16)
    return None


def roofline(prof, st, steps, n_a, n_b, zone_h, total_ms):
    if not prof:
        return None
    peaks = load_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    name, (tot_ms, launches) = max(prof.items(), key=lambda kv: kv[1][0])
    per_launch_ms = tot_ms / launches
    alg = algorithmic_bytes(name, st, steps, launches, n_a, n_b, zone_h)
    out = {"kernel": name, "bound": "hbm", "peak": peak, "unit": "GB/s", "ms_per_launch": per_launch_ms,
           "launches_per_step": launches / steps, "share_of_step": tot_ms / total_ms,
           "achieved": None, "frac": None, "traffic": None,
           "peak_source": "of measured" if peaks.get("_source") == "measured" else "of fallback"}
    if alg is None:
        return out
    achieved = alg / (per_launch_ms * 1e-3) / 1e9
    out.update(achieved=achieved, frac=achieved / peak, algorithmic_bytes=alg,
               traffic=traffic_record(name))
    return out


def traffic_record(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else null)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(kernel)
    if not rec or rec.get("source_hash") != source_hash(kernel):
        return None
    return rec.get("dram_bytes_per_launch")


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
