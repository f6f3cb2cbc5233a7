"""Benchmark of the sky cross-match hot path (one JSON line on stdout).

A step is one pass of the whole path over one synthetic workload: build the
index of catalogue B (ingest, radix sort on (zone, RA), bucket tables, cell
offsets), match catalogue A against it with both selections (all pairs and
best pair), and build the "1 or 2" join rows. The workload is the largest
single-GPU configuration: the all-sky circle cross-match, A = 5e7 against
B = 2e8 (int64 ids), r = 2 arcsec, density 1 + 9 exp(-|b|/10 deg) in
galactic latitude, both poles and the 0/360 seam included.

value      A sources per second over K timed steps, inputs resident in HBM
           (4 GB of input, far beyond L2; L2 also flushed before every step),
           float32 tests with float64 recheck in the guard band.
e2e        the same step through the C ABI with pinned host buffers: the
           host->device copies of both catalogues (and B's ids) and the
           device->host copy of the join rows and best pairs in the timed
           region.
fp64_path  the same step on the all-float64 path.
roofline   the dominant kernel, timed with CUDA events on its stream during
           profiled steps, against the measured HBM copy bandwidth; and the
           scan's count pass against the same peak (scan_roofline).
peaks      measured float32 / float64 FMA rates and read-only HBM bandwidth
           of this GPU (xm_measure_peak).
cpu_baseline  the FP64 CPU oracle on a bounded sample of the same workload:
           every A source in 16 seeded caps, against every B source they can
           reach.
Legs (N = 1): c2 (the clump-vs-compact-source ellipses, 2e5 x 5e6, with the
count pass against the measured float32 FMA peak), c4 (4096 batched
requests, one graph launch), exact_value, serving (C5).

--impl reference times that oracle as the reference arm on the same sample.
Under torchrun (N > 1) each rank runs its own copy of the workload (weak
scaling, no data-path collective); rank 0 prints the line with the max time
over ranks.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
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


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--scale", type=float, default=1.0,
                   help="size of the all-sky workload (1 = A 5e7 x B 2e8)")
    p.add_argument("--zone-height", type=float, default=0.0, help="arcsec; 0 = tuned default")
    p.add_argument("--cpu-sample", type=int, default=0, help="A sources in the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--serve-seconds", type=float, default=60.0,
                   help="serving window after a warm-up of 1/6 of it; 0 skips the serving leg")
    p.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrivals per second")
    p.add_argument("--serve-b", type=int, default=300_000_000, help="resident B sources")
    p.add_argument("--serve-pool", type=int, default=256, help="distinct request payloads")
    p.add_argument("--serve-slots", type=int, default=3)
    p.add_argument("--c1-leg", type=int, default=1, help="0 skips the small C1 leg")
    p.add_argument("--c2-leg", type=int, default=1, help="0 skips the C2 ellipse leg")
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


def workload(seed_offset=0, scale=1.0, device="cuda"):
    """The all-sky workload of one rank, on the device: ranks draw different
    catalogues of the same shape (seed 1003 + rank)."""
    from paper_1611_08494_gb300 import synth_gpu

    d = synth_gpu.c3(seed=1003 + seed_offset, scale=scale, device=device)
    n_a, n_b = d["a_lon"].numel(), d["b_lon"].numel()
    d["desc"] = (f"c3 all-sky circle cross-match: A={n_a}, B={n_b} (int64 ids), r=2 arcsec, "
                 "density 1+9exp(-|b|/10deg) in galactic latitude, both poles and the 0/360 seam, "
                 "60% of A with a counterpart (sigma 0.5 arcsec)")
    return d


# ------------------------------------------------------------------- oracle

def cap_sample(d, n_target, seed=2003, n_caps=16):
    """A bounded sample of the all-sky workload for the oracle: every A source
    within n_caps caps of equal radius at seeded centres uniform on the
    sphere (sized so the caps hold about n_target of A), and every B source
    within that radius plus twice the region radius (all B that can be a
    member of a sampled A). Host arrays, rows in catalogue order."""
    import torch

    n_a = d["a_lon"].numel()
    f = min(1.0, n_target / max(n_a, 1))
    cos_r = max(-1.0, 1.0 - 2.0 * f / n_caps)  # n_caps x 2 pi (1 - cos r) = 4 pi f
    rad = math.degrees(math.acos(cos_r))
    margin = 2.0 * d["region"]["a"] / 3600.0
    h = np.random.Generator(np.random.Philox(key=seed))
    centres = [(h.uniform(0.0, 360.0), math.degrees(math.asin(h.uniform(-1.0, 1.0))))
               for _ in range(n_caps)]

    def unit(lon, lat):
        lr, br = torch.deg2rad(lon), torch.deg2rad(lat)
        return torch.cos(br) * torch.cos(lr), torch.cos(br) * torch.sin(lr), torch.sin(br)

    def in_caps(lon, lat, r_deg):
        x, y, z = unit(lon, lat)
        m = torch.zeros(lon.numel(), dtype=torch.bool, device=lon.device)
        for cl, cb in centres:
            c = (math.cos(math.radians(cb)) * math.cos(math.radians(cl)),
                 math.cos(math.radians(cb)) * math.sin(math.radians(cl)), math.sin(math.radians(cb)))
            m |= x * c[0] + y * c[1] + z * c[2] >= math.cos(math.radians(r_deg))
        return torch.nonzero(m).flatten()

    a_rows = in_caps(d["a_lon"], d["a_lat"], rad)
    b_rows = in_caps(d["b_lon"], d["b_lat"], min(180.0, rad + margin))
    return {"a_lon": d["a_lon"][a_rows].cpu().numpy(), "a_lat": d["a_lat"][a_rows].cpu().numpy(),
            "b_lon": d["b_lon"][b_rows].cpu().numpy(), "b_lat": d["b_lat"][b_rows].cpu().numpy(),
            "a_frame": d["a_frame"], "b_frame": d["b_frame"], "region": dict(d["region"]),
            "desc": f"every A source within {n_caps} caps of radius {rad:.3f} deg at seeded "
                    f"centres ({a_rows.numel()} of {n_a} A) against the {b_rows.numel()} B within "
                    f"{rad:.3f} deg + {margin * 3600:.0f} arcsec"}


def oracle_time(smp, nthreads):
    """Seconds the oracle (as it stands) takes on a sample: its voxel grid
    over the sample's B, the pair tests and best selection."""
    import oracle

    t = time.perf_counter()
    r = oracle.match(smp["a_lon"], smp["a_lat"], smp["b_lon"], smp["b_lat"], a_frame=smp["a_frame"],
                     b_frame=smp["b_frame"], nthreads=nthreads, **smp["region"])
    oracle.best(r, smp["a_lon"].size)
    return time.perf_counter() - t


def pin_to_gpu_local_cpus(device):
    """Restricts this process to the CPU cores the GPU is attached to (its
    PCI device's local_cpulist), when that is known and overlaps the cores
    the process may use, so pinned host memory allocated afterwards lies on
    the GPU's own memory node. Returns a one-line account of what was done."""
    import torch

    try:
        uuid = str(torch.cuda.get_device_properties(device).uuid)
        out = subprocess.run(["nvidia-smi", "--query-gpu=uuid,pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout
        bus = None
        for line in out.splitlines():
            u, b = [x.strip() for x in line.split(",")]
            if u.lower().endswith(uuid.lower().replace("gpu-", "")) or len(out.splitlines()) == 1:
                bus = b
        if not bus:
            return "unchanged: the GPU's PCI address is unknown"
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest.lower()}/local_cpulist"
        cpus = set()
        for part in open(path).read().strip().split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        allowed = os.sched_getaffinity(0)
        use = cpus & allowed
        if not use:
            return f"unchanged: no allowed core is local to the GPU ({path})"
        os.sched_setaffinity(0, use)
        return f"{len(use)} of {len(allowed)} allowed cores, local to the GPU ({bus})"
    except Exception as e:  # (no nvidia-smi, no sysfs entry: leave the affinity)
        return f"unchanged: {type(e).__name__}"


def host_threads():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def cpu_baseline(smp):
    nthreads = host_threads()
    dt = oracle_time(smp, nthreads)
    n = smp["a_lon"].size
    return {"value": n / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"{smp['desc']}; {dt:.2f} s on {nthreads} threads"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import torch

    d = workload(scale=args.scale)
    # each step is the oracle on a bounded sample, sized so the K + W steps
    # take a minute or two
    smp = cap_sample(d, args.cpu_sample or 400_000)
    desc = d["desc"]
    del d
    torch.cuda.empty_cache()
    nthreads = host_threads()
    for _ in range(args.warmup):
        oracle_time(smp, nthreads)
    times = [oracle_time(smp, nthreads) for _ in range(args.steps)]
    tot = sum(times)
    n_s = smp["a_lon"].size
    v = n_s * len(times) / tot
    cb = {"kind": "oracle", "cores": nthreads, "unit": UNIT, "value": v,
          "sample": f"{smp['desc']}, per step, {nthreads} threads"}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "sample_a": n_s},
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
    "k_scan_src": ("xm_scan.cuh", "xm_internal.cuh"),
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
    # pinned host buffers (the end-to-end legs) on the GPU's own memory node
    affinity = pin_to_gpu_local_cpus(local)
    from paper_1611_08494_gb300 import xm

    measured = xm.measure_peaks()  # this GPU's float32 / float64 FMA and read rates
    d = workload(seed_offset=rank, scale=args.scale)
    n_a, n_b = d["a_lon"].numel(), d["b_lon"].numel()
    # the oracle's sample is cut now (small host arrays), timed at the end
    smp = cap_sample(d, args.cpu_sample or 1_500_000) if (rank == 0 and world == 1
                                                          and not args.no_cpu_baseline) else None
    dev = {k: d[k] for k in ("a_lon", "a_lat", "b_lon", "b_lat", "b_id")}
    zone_h = args.zone_height or 24.0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    host_out = {}

    def step(prec, fp64_index, cols=None, copy_out=False, out_slot=0, idx=None):
        cols = cols or dev
        # the build's input check is read at the match's synchronisation
        if idx is None:
            idx = xm.Index(cols["b_lon"], cols["b_lat"], frame=d["b_frame"], ids=cols["b_id"],
                           zone_height_arcsec=zone_h, build_fp64=fp64_index, deferred_check=True)
        res = xm.Result(idx, cols["a_lon"], cols["a_lat"], frame=d["a_frame"], precision=prec,
                        selection=xm.SEL_ALL | xm.SEL_BEST, **d["region"])
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

    def timed(prec, fp64_index, steps, warmup, cols=None, copy_out=False, profile=False,
              clocks=None):
        for _ in range(warmup):
            step(prec, fp64_index, cols, copy_out)
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
            flush.zero_()  # evict what the previous step left in L2
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, res, rows, out = step(prec, fp64_index, cols, copy_out)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            if out is not None:
                bytes_out = sum(t.numel() * t.element_size() for t in out)
            del res, rows
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
        return ms, st, prof, bytes_out

    # float32 + float64 recheck (the product path), uninstrumented
    with Clocks(local) as clk:
        ms, st, _, _ = timed(xm.PREC_FP32, False, args.steps, args.warmup, clocks=clk)
    total_ms = max_over_ranks(sum(ms), world, "cuda")
    value = weak_scaling_value(n_a, args.steps, world, total_ms)
    launches = st["kernel_launches"]
    _, res, rows, _ = step(xm.PREC_FP32, False)
    n_pairs, n_rows = int(res.n_pairs), int(rows.n)
    del res, rows

    # the same steps again with an event pair around every launch: per-kernel
    # times for the shares and the roofline (the events cost a little time,
    # so these steps are not the ones the value comes from)
    prof_steps = max(5, args.steps // 4)
    ms_p, st_p, prof, _ = timed(xm.PREC_FP32, False, prof_steps, 1, profile=True)

    # all-float64 path
    ms64, _, _, _ = timed(xm.PREC_FP64, True, max(3, args.steps // 2), 1)
    v64 = n_a * len(ms64) / (sum(ms64) / 1e3)

    e2e = None
    if not args.no_e2e:
        e2e = e2e_legs(args, xm, torch, d, step, flush, zone_h, n_a)

    roof = roofline(prof, st_p, prof_steps, n_a, n_b, sum(ms_p), d["region"])
    # the count pass: its sparse form (one lane per source) where it ran
    scan_roof = kernel_roofline(count_kernel(prof), prof, st_p, prof_steps, n_a, n_b, d["region"])
    del dev, d
    torch.cuda.empty_cache()
    xm.free_cached()  # and the blocks the library kept for reuse

    if rank != 0:
        return
    peaks = load_peaks()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64-recheck", "data": "synthetic",
        "config": {"workload": workload_desc(n_a, n_b), "n_a": n_a, "n_b": n_b,
                   "step": "build B index (with int64 ids) + match (all and best pairs) + "
                           "join '1 or 2'",
                   "precision": "float32 tests, float64 recheck in the guard band",
                   "zone_height_arcsec": zone_h,
                   "l2": "inputs 4 GB, larger than L2; L2 also flushed (256 MiB write) before "
                         "each step",
                   "index_check": "deferred to the match's synchronisation",
                   "pairs": n_pairs, "join_rows": n_rows},
        "e2e": e2e and dict(e2e, host_cpus=affinity),
        "fp64_path": {"value": v64, "unit": UNIT, "ms_per_step": statistics.mean(ms64),
                      "fp32_recheck_speedup": v64 and value / world / v64},
        "gpu_launches": int(launches),
        "roofline": roof,
        "scan_roofline": scan_roof,
        "clocks": clk.summary(),
        "kernels_ms_per_step": {k: round(v[0] / prof_steps, 4) for k, v in
                                sorted(prof.items(), key=lambda kv: -kv[1][0])[:16]},
        "profiled_ms_per_step": sum(ms_p) / prof_steps,
        "stats_per_step": {k: v // args.steps for k, v in st.items()},
        "peaks": {"hbm_copy_gbs": peaks.get("hbm_gbs"), "hbm_copy_source": peaks.get("_source"),
                  "hbm_read_gbs": measured["hbm_read_gbs"],
                  "fp32_fma_tflops": measured["fp32_fma_tflops"],
                  "fp64_fma_tflops": measured["fp64_fma_tflops"],
                  "measured_by": "xm_measure_peak on this GPU, best of 5 launches"},
    }
    if world == 1 and args.c1_leg:
        line["c1"] = c1_leg(args, xm, torch)
    if world == 1 and args.c2_leg:
        line["c2"] = c2_leg(args, xm, torch, measured)
    if world == 1 and args.c4_requests > 0:
        line["c4"] = c4_leg(args, xm, torch, measured)
    if world == 1 and args.values_scale > 0:
        line["exact_value"] = values_leg(args, xm, torch)
    if world == 1 and args.serve_seconds > 0:
        line["serving"] = serving_leg(args, xm, torch)
    elif world > 1:
        line["serving"] = {"skipped": "the serving leg runs at N = 1 only"}
    if smp is not None:
        line["cpu_baseline"] = cpu_baseline(smp)
    print(json.dumps(line), flush=True)


def workload_desc(n_a, n_b):
    return (f"c3 all-sky circle cross-match: A={n_a}, B={n_b} (int64 ids), r=2 arcsec, "
            "density 1+9exp(-|b|/10deg) in galactic latitude, both poles and the 0/360 seam, "
            "60% of A with a counterpart (sigma 0.5 arcsec)")


def e2e_legs(args, xm, torch, d, step, flush, zone_h, n_a):
    """The step through the C ABI from pinned host memory: inputs copied in
    and the join rows and best pairs copied out inside the timed region."""
    host = {k: d[k].cpu().pin_memory() for k in ("a_lon", "a_lat", "b_lon", "b_lat", "b_id")}
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    stream = torch.cuda.current_stream()
    n_ser = max(3, args.steps // 4)
    for _ in range(1):
        step(xm.PREC_FP32, False, host, True)
    torch.cuda.synchronize()
    ms_ser, d2h = [], 0
    for _ in range(n_ser):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, res, rows, out = step(xm.PREC_FP32, False, host, True)
        e1.record(stream)
        e1.synchronize()
        ms_ser.append(e0.elapsed_time(e1))
        d2h = sum(t.numel() * t.element_size() for t in out)
        del res, rows
    v_ser = n_a * n_ser / (sum(ms_ser) / 1e3)

    # pipelined as a throughput-bound user would run it, through the same
    # calls with host buffers: step k's match is queued first (xm_match_async:
    # its copy of A goes ahead on the copy queue, which runs host copies of
    # all streams in the order they were queued), then the index build of
    # step k + 2 (which copies B in) on a low-priority stream, then step k's
    # wait for its pair count and its join on a high-priority stream that
    # waited for step k's build, and its result copy on a further stream: B
    # copies in, results out and the builds of later steps fill the time the
    # match and join of the current one leave, and never delay them (the GPU
    # schedules the high-priority stream's blocks first). A step's objects
    # live until its copy out has run (their memory is released in their
    # streams' order after a wait on it). Every step still copies all of its
    # inputs in and its result out; the clock covers the whole run.
    lo_pri, hi_pri = torch.cuda.Stream.priority_range()
    bstreams = [torch.cuda.Stream(priority=lo_pri) for _ in range(3)]
    mstreams = [torch.cuda.Stream(priority=hi_pri) for _ in range(3)]
    out_stream = torch.cuda.Stream(priority=hi_pri)
    streams = bstreams + mstreams
    keep = {}
    out_bufs = {}

    def build(k):
        bs = bstreams[k % 3]
        with torch.cuda.stream(bs):
            idx = xm.Index(host["b_lon"], host["b_lat"], frame=d["b_frame"], ids=host["b_id"],
                           zone_height_arcsec=zone_h, deferred_check=True)
            built = torch.cuda.Event()
            built.record(bs)
        return idx, built

    def start(k, ahead_k):
        idx, built = ahead_k
        ms = mstreams[k % 3]
        ms.wait_event(built)
        with torch.cuda.stream(ms):
            return xm.Pending(idx, host["a_lon"], host["a_lat"], frame=d["a_frame"],
                              precision=xm.PREC_FP32, selection=xm.SEL_ALL | xm.SEL_BEST,
                              **d["region"])

    def finish(k, pending):
        ms = mstreams[k % 3]
        with torch.cuda.stream(ms):
            res = pending.wait()
            idx = pending.index
            rows = res.join("or")
            srcs = [rows.a_row, rows.b_row, rows.sep, res.best_b, res.best_sep]
            done = torch.cuda.Event()
            done.record(ms)
        out_stream.wait_event(done)
        slot = k % 3
        key = tuple(t.numel() for t in srcs)
        if out_bufs.get(slot, (None,))[0] != key:
            out_bufs[slot] = (key, [torch.empty(t.numel(), dtype=t.dtype).pin_memory() for t in srcs])
        with torch.cuda.stream(out_stream):
            for dst, src in zip(out_bufs[slot][1], srcs):
                dst.copy_(src, non_blocking=True)
            copied = torch.cuda.Event()
            copied.record(out_stream)
        keep[k] = (idx, res, rows, srcs, copied, (bstreams[k % 3], ms))
        old = keep.pop(k - 2, None)
        if old is not None:  # its memory is released in its streams after its copy out
            for st in old[5]:
                st.wait_event(old[4])
            del old

    def run(n):
        ahead = {0: build(0), 1: build(1) if n > 1 else None}
        for k in range(n):
            pending = start(k, ahead.pop(k))
            if k + 2 < n:
                ahead[k + 2] = build(k + 2)
            finish(k, pending)
        for k in sorted(keep):
            for st in keep[k][5]:
                st.wait_event(keep[k][4])
        keep.clear()

    run(3)
    torch.cuda.synchronize()
    n_pipe = max(6, args.steps)
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for st in streams + [out_stream]:
        st.wait_event(e0)
    run(n_pipe)
    for st in streams + [out_stream]:
        cur.wait_stream(st)
    e1.record(cur)
    e1.synchronize()
    ms_pipe = e0.elapsed_time(e1)
    copies = copy_rates(torch, h2d, d2h, n_a)
    del host
    return {"value": n_a * n_pipe / (ms_pipe / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h),
            "mode": "each step's index build (and B copy in) issued two steps ahead on a "
                    "low-priority stream, after the current step's match is queued "
                    "(xm_match_async, so A's copy goes first); its wait and join on a "
                    "high-priority stream that waits for the build, result copies out on another "
                    "stream: copies in, compute and copies out of neighbouring steps overlap",
            "serial_value": v_ser, "serial_mode": "one step at a time, events around each step",
            "steps": n_pipe, "copies": copies}


def copy_rates(torch, h2d_bytes, d2h_bytes, n_a):
    """This machine's host <-> device copy rates between pinned host memory and
    the device (1 GiB each way, best of three; each way alone and both at
    once on two streams), and the end-to-end floor they set: a step's copies
    in and out at the rates of both at once."""
    nb = 1 << 30
    dev = torch.empty(nb, dtype=torch.uint8, device="cuda")
    dev2 = torch.empty(nb, dtype=torch.uint8, device="cuda")
    hin = torch.empty(nb, dtype=torch.uint8).pin_memory()
    hout = torch.empty(nb, dtype=torch.uint8).pin_memory()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn_in, fn_out):
        best_in = best_out = 0.0
        for _ in range(3):
            torch.cuda.synchronize()
            evs = {}
            for name, st, fn in (("in", s_in, fn_in), ("out", s_out, fn_out)):
                if fn is None:
                    continue
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(st):
                    a.record(st)
                    fn()
                    b.record(st)
                evs[name] = (a, b)
            torch.cuda.synchronize()
            if "in" in evs:
                best_in = max(best_in, nb / (evs["in"][0].elapsed_time(evs["in"][1]) * 1e-3) / 1e9)
            if "out" in evs:
                best_out = max(best_out, nb / (evs["out"][0].elapsed_time(evs["out"][1]) * 1e-3) / 1e9)
        return best_in, best_out

    cin = lambda: dev.copy_(hin, non_blocking=True)  # noqa: E731
    cout = lambda: hout.copy_(dev2, non_blocking=True)  # noqa: E731
    h2d_alone, _ = timed(cin, None)
    _, d2h_alone = timed(None, cout)
    h2d_both, d2h_both = timed(cin, cout)
    floor_s = max(h2d_bytes / (h2d_both * 1e9), d2h_bytes / (d2h_both * 1e9))
    del dev, dev2, hin, hout
    return {"h2d_gbs": h2d_alone, "d2h_gbs": d2h_alone, "both_gbs": [h2d_both, d2h_both],
            "floor_value": n_a / floor_s,
            "floor": "a step's copies in and out at the rates of both at once, all compute hidden"}


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


# --------------------------------------------------------- C2 ellipse leg

def c1_leg(args, xm, torch):
    """The plain circle cross-match (A = B = 1e4 in a 1 x 1 deg box, r = 1
    arcsec, float64 throughout): a latency-bound case whose step is a dozen
    small launches. The step (build + match all and best + join "1 or 2")
    from device-resident columns, the same from pinned host columns with the
    join rows copied back (the whole call as a user makes it), and the oracle
    on the whole workload on the host cores."""
    from paper_1611_08494_gb300 import synth

    d = synth.c1()
    n_a = d["a_lon"].size
    host = {k: torch.as_tensor(d[k]).pin_memory() for k in ("a_lon", "a_lat", "b_lon", "b_lat")}
    dev = {k: v.cuda() for k, v in host.items()}
    stream = torch.cuda.current_stream()

    def step(cols, copy_out):
        idx = xm.Index(cols["b_lon"], cols["b_lat"], frame=d["b_frame"], build_fp64=True)
        res = xm.Result(idx, cols["a_lon"], cols["a_lat"], frame=d["a_frame"],
                        precision=xm.PREC_FP64, selection=xm.SEL_ALL | xm.SEL_BEST, **d["region"])
        rows = res.join("or")
        if copy_out:
            return [t.to("cpu", non_blocking=True) for t in (rows.a_row, rows.b_row, rows.sep,
                                                               res.best_b, res.best_sep)]
        return rows

    def timed(cols, copy_out, n):
        for _ in range(5):
            step(cols, copy_out)
        torch.cuda.synchronize()
        ms = []
        for _ in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(cols, copy_out)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    xm.reset_stats()
    ms_dev = timed(dev, False, 200)
    launches = xm.stats()["kernel_launches"] / 205
    ms_e2e = timed(host, True, 200)
    smp = dict(d, desc=f"the whole workload ({n_a} A x {d['b_lon'].size} B)")
    out = {"workload": "c1 plain circle cross-match: A=10000, B=10000 (70% offset copies, "
                       "sigma 0.3 arcsec), RA 150-151 Dec 2-3, r=1 arcsec, float64 throughout",
           "ms_per_step": ms_dev, "a_per_s": n_a / (ms_dev / 1e3), "launches_per_step": launches,
           "e2e_ms_per_step": ms_e2e, "e2e_a_per_s": n_a / (ms_e2e / 1e3),
           "e2e": "pinned host columns in, join rows and best pairs copied back, per step",
           "cpu_baseline": cpu_baseline(smp)}
    del dev, host
    return out


def oracle_requests(reqs, b_lon, b_lat, b_frame, n_pick, seed, max_a):
    """The oracle timed request by request (the cpu_baseline of a batched or
    served workload): n_pick seeded requests of at most max_a A sources, each
    matched alone (all pairs, best pairs) against the B sources of its cap
    widened by its offsets and largest region, on the host cores."""
    import torch

    import oracle

    h = np.random.Generator(np.random.Philox(key=seed))
    ok = [r for r, q in enumerate(reqs) if q["lon"].numel() <= max_a]
    pick = sorted(h.choice(ok, min(n_pick, len(ok)), replace=False).tolist())
    nthreads = host_threads()
    tot_a, tot_b, tot_s = 0, 0, 0.0
    for r in pick:
        q = reqs[r]
        c_lon, c_lat, rad = q["cap"]
        if q.get("frame", b_frame) != b_frame:  # the cap centre in B's frame
            if b_frame == oracle.GAL:
                gl, gb = oracle.from_equatorial([c_lon], [c_lat], oracle.GAL)
            else:
                gl, gb = oracle.to_equatorial([c_lon], [c_lat], oracle.GAL)
            c_lon, c_lat = float(gl[0]), float(gb[0])
        reach = rad + (8.0 * q["offset_sigma"] + 1.5 * q["max_size"]) / 3600.0
        cl, cb = math.radians(c_lon), math.radians(c_lat)
        lr, br = torch.deg2rad(b_lon), torch.deg2rad(b_lat)
        dot = (torch.cos(br) * torch.cos(lr) * (math.cos(cb) * math.cos(cl)) +
               torch.cos(br) * torch.sin(lr) * (math.cos(cb) * math.sin(cl)) +
               torch.sin(br) * math.sin(cb))
        rows = torch.nonzero(dot >= math.cos(math.radians(min(180.0, reach)))).flatten()
        bl, bb = b_lon[rows].cpu().numpy(), b_lat[rows].cpu().numpy()
        al, ab = q["lon"].cpu().numpy(), q["lat"].cpu().numpy()
        reg = {k: (v.cpu().numpy() if hasattr(v, "numel") else v) for k, v in q["region"].items()}
        t = time.perf_counter()
        m = oracle.match(al, ab, bl, bb, a_frame=q.get("frame", b_frame), b_frame=b_frame,
                         nthreads=nthreads, **reg)
        oracle.best(m, al.size)
        tot_s += time.perf_counter() - t
        tot_a += al.size
        tot_b += bl.size
    return {"value": tot_a / tot_s if tot_s else None, "unit": UNIT, "cores": nthreads,
            "kind": "oracle", "requests": len(pick), "a_sources": tot_a, "b_in_caps": tot_b,
            "seconds": tot_s,
            "sample": f"{len(pick)} seeded requests of at most {max_a} A, each alone against "
                      f"the B of its cap ({tot_a} A, {tot_b} B), all and best pairs, "
                      f"{tot_s:.2f} s on {nthreads} threads"}


def c2_leg(args, xm, torch, measured):
    """The clump-vs-compact-source case: A = 2e5 per-source ellipses against
    B = 5e6 in the galactic plane. The same step (build + match all and best
    + join "1 or 2") on both paths, the count pass against the measured
    float32 FMA peak (12 float32 operations per candidate), the index sort
    against the HBM peak, and the further readings of "best pairs" over its
    pair list."""
    from paper_1611_08494_gb300 import synth

    d = synth.c2()
    n_a, n_b = d["a_lon"].size, d["b_lon"].size
    cu = lambda x: torch.as_tensor(np.ascontiguousarray(x), device="cuda")  # noqa: E731
    cols = {k: cu(d[k]) for k in ("a_lon", "a_lat", "b_lon", "b_lat")}
    reg = {k: (cu(v) if isinstance(v, np.ndarray) else v) for k, v in d["region"].items()}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(prec, fp64_index=False):
        idx = xm.Index(cols["b_lon"], cols["b_lat"], frame=d["b_frame"], zone_height_arcsec=12.0,
                       build_fp64=fp64_index, deferred_check=True)
        res = xm.Result(idx, cols["a_lon"], cols["a_lat"], frame=d["a_frame"], precision=prec,
                        selection=xm.SEL_ALL | xm.SEL_BEST, **reg)
        rows = res.join("or")
        return idx, res, rows, None

    def timed(prec, fp64_index, steps, profile=False):
        for _ in range(3):
            step(prec, fp64_index)
        torch.cuda.synchronize()
        xm.reset_stats()
        if profile:
            xm.prof_enable(True)
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(prec, fp64_index)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        prof = xm.prof_all() if profile else {}
        if profile:
            xm.prof_enable(False)
        return ms, xm.stats(), prof

    k = max(10, args.steps)
    ms32, _, _ = timed(xm.PREC_FP32, False, k)
    ms64, _, _ = timed(xm.PREC_FP64, True, max(5, k // 2))
    ms_p, st_p, prof = timed(xm.PREC_FP32, False, 10, profile=True)
    out = {"workload": "c2 clump-vs-compact-source: A=200000 per-source ellipses (a 5-60 arcsec "
                       "log-uniform, b/a 0.3-1, PA 0-180), B=5000000, galactic l 0-60 |b|<=1 "
                       "density exp(-|b|/0.3deg)",
           "ms_per_step": statistics.median(ms32), "a_per_s": n_a / (statistics.median(ms32) / 1e3),
           "fp64_ms_per_step": statistics.median(ms64),
           "fp64_a_per_s": n_a / (statistics.median(ms64) / 1e3),
           "kernels_ms_per_step": {kk: round(v[0] / 10, 4) for kk, v in
                                   sorted(prof.items(), key=lambda kv: -kv[1][0])[:10]}}
    scan = prof.get(count_kernel(prof))
    if scan:
        cand = st_p["candidates"] / 10
        t = scan[0] / scan[1] * 1e-3
        flops = 12.0 * cand
        out["count_pass_fp32"] = {"kernel": "k_scan count pass", "bound": "fp32",
                                  "candidates": int(cand), "flops_per_candidate": 12,
                                  "ms": t * 1e3, "achieved_tflops": flops / t / 1e12,
                                  "peak_tflops": measured["fp32_fma_tflops"],
                                  "frac": flops / t / 1e12 / measured["fp32_fma_tflops"],
                                  "peak_source": "of measured (xm_measure_peak)"}
        out["count_pass_hbm"] = kernel_roofline(count_kernel(prof), prof, st_p, 10, n_a, n_b, reg)
    out["sort_roofline"] = kernel_roofline("k_onesweep", prof, st_p, 10, n_a, n_b, reg)
    out["picks"] = pick_leg(xm, torch, step, stream)
    del cols, reg
    torch.cuda.empty_cache()
    xm.free_cached()  # and the blocks the library kept for reuse
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
    xm.free_cached()  # and the blocks the library kept for reuse
    return out


# ------------------------------------------------------- batched C4 leg

def c4_leg(args, xm, torch, measured):
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
    # one more pass launched kernel by kernel, an event pair around each
    # launch: the persistent count pass against HBM (per A 16 B position +
    # 8 B per per-source region column + 16 B best pair, per candidate 12 B)
    # and against the float32 FMA peak (12 operations per candidate)
    xm.reset_stats()
    xm.prof_enable(True)
    b = xm.Batch(idx, reqs, use_graph=False, persistent_blocks=tuned["persistent_blocks"])
    torch.cuda.synchronize()
    prof = xm.prof_all()
    xm.prof_enable(False)
    st = xm.stats()
    del b
    scan = None
    if "k_scan_fp32_count" in prof:
        t_ms, nl = prof["k_scan_fp32_count"]
        cols = sum(q["lon"].numel() * sum(1 for v in q["region"].values() if hasattr(v, "numel"))
                   for q in d["requests"])
        alg = total_a * 32 + 8 * cols + 12 * st["candidates"]
        peaks = load_peaks()
        fp32 = measured["fp32_fma_tflops"]
        achieved = alg / (t_ms * 1e-3) / 1e9
        scan = {"kernel": "k_scan_fp32_count", "launches": nl, "ms": t_ms,
                "candidates": int(st["candidates"]), "algorithmic_bytes": alg,
                "achieved": achieved, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                "frac": achieved / peaks.get("hbm_gbs", 6800.0),
                "peak_source": "of measured" if peaks.get("_source") == "measured" else "of fallback",
                "fp32_tflops": 12.0 * st["candidates"] / (t_ms * 1e-3) / 1e12,
                "fp32_frac": 12.0 * st["candidates"] / (t_ms * 1e-3) / 1e12 / fp32,
                "fp32_peak_source": "of measured (xm_measure_peak)",
                "kernels_ms": {k: round(v[0], 3) for k, v in
                               sorted(prof.items(), key=lambda kv: -kv[1][0])[:8]}}
    base = oracle_requests(d["requests"], d["b_lon"], d["b_lat"], d["b_frame"], 12, 4141, 200_000)
    out = {"workload": f"c4 batched: {len(reqs)} requests (n_A log-uniform 1e2-1e6, caps 0.1-10 deg, "
                       f"mixed shapes/sizes/joins) against B={args.c4_b} uniform all-sky",
           "requests": len(reqs), "total_a": int(total_a), "pairs": int(info["total_pairs"]),
           "batch_ms": statistics.median(ms), "a_per_s": total_a / (statistics.median(ms) / 1e3),
           "launch": "one persistent scan in one CUDA graph per batch pass",
           "zone_height_arcsec": tuned["zone_height_arcsec"],
           "persistent_blocks": tuned["persistent_blocks"], "tune_trials": tuned["trials"],
           "setup_s": setup_s, "scan_roofline": scan, "cpu_baseline": base}
    del d, reqs, idx
    torch.cuda.empty_cache()
    xm.free_cached()  # and the blocks the library kept for reuse
    return out


# ----------------------------------------------------------- serving leg

def serving_leg(args, xm, torch):
    """Poisson arrivals against a resident B index through the library's
    serving loop (continuous batching, admission by free device memory).
    Requests take their payloads from a pool of pre-generated requests;
    latency runs from the call that submits a request (its columns are
    copied inside it) to its results complete on the device. Three windows:
    requests submitted from pinned host columns (the headline), the same
    from device-resident columns, and host submission under a small memory
    budget (admission refuses requests that can never fit and queues the
    ones that do not fit yet)."""
    from paper_1611_08494_gb300 import synth_gpu

    t_setup = time.perf_counter()
    b = synth_gpu.c5_catalogue(n_b=args.serve_b)
    pool = synth_gpu.c5_requests(b, n_pool=args.serve_pool)
    sample = [dict(lon=q["lon"], lat=q["lat"], frame=q["frame"], selection=q["selection"],
                   join=q["join"], join_selection=q["join_selection"], **q["region"])
              for q in pool[:6]]
    tuned = xm.autotune(b["b_lon"], b["b_lat"], sample, frame=b["b_frame"],
                        zone_heights=(10.0, 20.0, 40.0), blocks_per_sm=(2, 4))
    idx = xm.Index(b["b_lon"], b["b_lat"], frame=b["b_frame"], ids=b["b_id"],
                   zone_height_arcsec=tuned["zone_height_arcsec"])
    base = oracle_requests(pool, b["b_lon"], b["b_lat"], b["b_frame"], 12, 5151, 200_000)
    del b
    pinned = lambda t: t.cpu().pin_memory()  # noqa: E731
    host_pool = []
    for q in pool:
        reg = {k: (pinned(v) if hasattr(v, "numel") else v) for k, v in q["region"].items()}
        host_pool.append(dict(q, lon=pinned(q["lon"]), lat=pinned(q["lat"]), region=reg))
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    xm.free_cached()  # and the blocks the library kept for reuse
    setup_s = time.perf_counter() - t_setup
    common = dict(slots=args.serve_slots, pool=len(pool),
                  zone_height_arcsec=tuned["zone_height_arcsec"],
                  persistent_blocks=tuned["persistent_blocks"], setup_s=setup_s)
    out = {"workload": f"c5 serving: B={args.serve_b} resident (C3 latitude profile, galactic, "
                       f"int64 ids), Poisson {args.serve_rate:g} req/s, n_A log-uniform 1e3-1e7, "
                       "mixed shapes/joins/frames, admission by free HBM",
           "latency": "from the submitting call (input copy included) to results complete on "
                      "the device"}
    host = serve_window(args, xm, idx, host_pool, args.serve_seconds, 0, tuned, 0)
    out.update(host, input="pinned host columns, copied by the submitting call", **common)
    out["cpu_baseline"] = base
    short = max(5.0, args.serve_seconds / 3.0)
    out["device_inputs"] = dict(serve_window(args, xm, idx, pool, short, 1, tuned, 0),
                                input="device-resident columns (device-to-device copy)")
    budget = 2 << 30
    out["memory_pressure"] = dict(serve_window(args, xm, idx, host_pool, short, 2, tuned, budget),
                                  input="pinned host columns", mem_budget_bytes=budget)
    del pool, host_pool, idx
    torch.cuda.empty_cache()
    xm.free_cached()  # and the blocks the library kept for reuse
    return out


def serve_window(args, xm, idx, pool, seconds, seed_offset, tuned, budget):
    """One serving window: Poisson arrivals for seconds (after a sixth of it
    of warm-up) drawing payloads from pool; a completion thread waits for and
    releases every ticket. Returns the server's statistics for the window."""
    import threading

    from paper_1611_08494_gb300 import synth_gpu

    warm = seconds / 6.0
    times, h = synth_gpu.poisson_arrivals(args.serve_rate, warm + seconds, seed=1007 + seed_offset)
    which = h.integers(0, len(pool), len(times))
    srv = xm.Server(idx, slots=args.serve_slots, precision=xm.PREC_FP32, use_graph=True,
                    persistent_blocks=tuned["persistent_blocks"], mem_budget_bytes=budget)
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
    refused_submit = 0
    t0 = time.perf_counter()
    reset_done = False
    t_win = t0
    for t_arr, w in zip(times, which):
        now = time.perf_counter() - t0
        if t_arr > now:
            time.sleep(t_arr - now)
        if not reset_done and t_arr >= warm:
            srv.reset_stats()
            t_win = time.perf_counter()
            reset_done = True
        q = pool[w]
        try:
            tk = srv.submit(q["lon"], q["lat"], frame=q["frame"], selection=q["selection"],
                            join=q["join"], join_selection=q["join_selection"], **q["region"])
        except xm.XMError as ex:
            if ex.status != "XM_EBUSY":
                raise
            refused_submit += reset_done
            continue
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
    return {"window_s": seconds, "warmup_s": warm, "requests": int(st["completed"]),
            "failed": int(st["failed"]), "refused": int(st["refused"]),
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
            "sustained_a_per_s": st["a_sources"] / window,
            "offered_a_per_s": offered_a / seconds,
            "drain_s": window - seconds, "batches": int(st["batches"]), "busy_s": st["busy_s"]}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "_source": "fallback"}


def algorithmic_bytes(kernel, st, steps, launches, n_a, n_b, region):
    """Bytes the method must move per launch of a kernel (averaged over the
    launches, so achieved = all bytes / all kernel time):
    k_onesweep   per key and pass 8 B key + 4 B row, read and written, over
                 the passes that ran (the library counts keys x passes; an
                 index sort planned to fewer passes launches the rest empty),
                 and 8 B more each way for keys that carry a payload (the
                 index sort carries each record's float32 offsets);
    k_scan_fp32_count, k_scan_src (the count pass, warp-cooperative or one
                 lane per source)  per A 16 B position + 8 B per region column given per
                 source + 16 B best pair, per candidate 12 B (offsets + RA
                 key);
    k_prep_a     per A 16 B position (+ region columns) read, 88 B of
                 prepared record written;
    k_gather_b   per B 8 B key + 4 B row + 8 B offsets read, 16 B record
                 written."""
    cols = sum(1 for k in ("a_col", "b_col", "pa_col") if region.get(k) is not None)
    if kernel == "k_onesweep":
        return (24.0 * st["sort_key_passes"] + 16.0 * st.get("sort_pay_passes", 0)) / launches
    if kernel in ("k_scan_fp32_count", "k_scan_fp64_count", "k_scan_src"):
        return (n_a * (16 + 8 * cols + 16) + st["candidates"] / steps * 12) * steps / launches
    if kernel == "k_prep_a":
        return n_a * (16 + 8 * cols + 88) * steps / launches
    if kernel == "k_gather_b":
        return n_b * (8 + 4 + 8 + 16) * steps / launches
    return None


def count_kernel(prof):
    """The count pass's kernel: the sparse form where the library ran it
    (the warp-cooperative pass then only takes the sources it left)."""
    return "k_scan_src" if "k_scan_src" in prof else "k_scan_fp32_count"


def kernel_roofline(name, prof, st, steps, n_a, n_b, region):
    """achieved = algorithmic bytes per launch / average launch time, against
    the measured HBM copy bandwidth."""
    if name not in prof:
        return None
    peaks = load_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    tot_ms, launches = prof[name]
    per_launch_ms = tot_ms / launches
    out = {"kernel": name, "bound": "hbm", "peak": peak, "unit": "GB/s",
           "ms_per_launch": per_launch_ms, "launches_per_step": launches / steps,
           "achieved": None, "frac": None, "traffic": None,
           "peak_source": "of measured" if peaks.get("_source") == "measured" else "of fallback"}
    alg = algorithmic_bytes(name, st, steps, launches, n_a, n_b, region)
    if alg is not None:
        achieved = alg / (per_launch_ms * 1e-3) / 1e9
        out.update(achieved=achieved, frac=achieved / peak, algorithmic_bytes=alg,
                   traffic=traffic_record(name))
    return out


def roofline(prof, st, steps, n_a, n_b, total_ms, region):
    """The dominant kernel of the step (largest share of the profiled time)."""
    if not prof:
        return None
    name, (tot_ms, _) = max(prof.items(), key=lambda kv: kv[1][0])
    out = kernel_roofline(name, prof, st, steps, n_a, n_b, region)
    out["share_of_step"] = tot_ms / total_ms
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
