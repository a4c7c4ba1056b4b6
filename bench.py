#!/usr/bin/env python
"""Benchmark of the local noise filter path (arXiv 1807.03119) on GB300.

Workload (one "step"): the 512^3 uint16 insect-like phantom (12-bit, thin
shells, tubes, cavities, Gaussian noise sigma 150, 1% salt-and-pepper), all
five filters at radius 2 (mean, sigma, entropy, Okada, the paper's filter),
with the image entropy of the input and of each output -- statistics pass,
device parameter derivation, five filter kernels and the entropy reduction.

Prints ONE JSON line (rank 0).  `value` = filtered output voxels per second
over the whole job (5 x 512^3 per step and GPU), device-timed with CUDA events
with the input resident in HBM; `e2e` = the same metric through the
host-buffer entry point (lnf_filter_multi_host), with the host->device copy
of the input and the device->host copies of the five outputs and six
entropies inside the timed region.  `roofline` is for the kernel with the
largest device time in the step, from CUDA events recorded around each launch
on the launching stream during the timed region.

`--impl reference` times the CPU oracle (plain C + exact Python integer
derivations) on bounded samples of the same workload on the host cores.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FILTER_NAMES = ["mean", "sigma", "entropy", "okada", "ours"]
DIMS = (512, 512, 512)
RADIUS = 2
N_VOX = DIMS[0] * DIMS[1] * DIMS[2]
ES = 2  # uint16
METRIC = "GVoxel/s and HBM GB/s vs peak at 512^3 uint16 r=2"
UNIT = "GVoxel/s"
WORKLOAD = "512x512x512 uint16 insect-like phantom, five filters at r=2, entropy of input and each output"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "sm_max_mhz": d.get("sm_max_mhz", 2070.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def max_over_ranks(value, world, device):
    """The slowest rank's figure, which is the job's: a MAX all-reduce over the
    ranks of the process group (replicas; no data-path collective)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# plain integer ALU peak: 152 SMs x 128 INT32 lanes x max SM clock
def alu_peak_tops(sm_mhz):
    return 152 * 128 * sm_mhz * 1e6 / 1e12


# algorithmic work per launch of each kernel kind on this workload
def algorithmic(kind, n_pass, hbm_gbs, alu_tops):
    """(bound, work) of one launch: HBM bytes, or integer ALU operations where
    those take longer at peak.  Sigma and Okada test every tap of a voxel whose
    own value passes the gate (P0 >= T) -- four operations per tap: subtract,
    compare, add value, add count -- and nothing for the others, whose output is
    0 whatever their band: their ALU work is 4 x taps x n_pass."""
    M3 = (2 * RADIUS + 1) ** 3
    if kind == "stats":
        return "hbm", N_VOX * ES
    if kind == "filter:gate":     # the five filters: read once, five outputs written
        return "hbm", N_VOX * ES * 6
    if kind.startswith("gate:"):      # one filter through the gate-first kernel: read once, write once
        return "hbm", N_VOX * ES * 2
    if kind.startswith("filter:"):
        f = kind.split(":")[1]
        hbm = N_VOX * ES * 2   # read the input once, write the output once
        if f in ("sigma", "okada"):
            alu = 4 * (M3 if f == "sigma" else 6 * RADIUS + 1) * n_pass
            if alu / (alu_tops * 1e12) > hbm / (hbm_gbs * 1e9):
                return "alu", alu
        return "hbm", hbm
    return None, None


# the kernel sources behind each kind of launch (a recorded traffic figure is
# void once any of them changes)
KIND_SOURCES = {
    "stats": ["stats.cu"],
    "params": ["stats.cu"],
    "entropy": ["stats.cu"],
    "filter:ours": ["fast.cu"],
    "filter:mean": ["fast2.cuh", "fast2_box.cu"],
    "filter:entropy": ["fast2.cuh", "fast2_box.cu"],
    "filter:sigma": ["fast2.cuh", "fast2_tap.cu"],
    "filter:okada": ["fast2.cuh", "fast2_tap.cu"],
    "filter:gate": ["gate.cuh", "gate_u16.cu"],
    "gate:ours": ["gate.cuh", "gate_u16.cu"],
    "gate:cube": ["gate.cuh", "gate_u16.cu"],
}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_512cubed_u16_r2.txt")


def source_digest(kind):
    h = hashlib.sha256()
    cdir = os.path.join(ROOT, "paper_1807_03119_gb300", "csrc")
    for fn in KIND_SOURCES.get(kind, []) + ["lnf_internal.cuh", "lnf_ctx.h"]:
        with open(os.path.join(cdir, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kind):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current sources of that kernel (else None)."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    dig = source_digest(kind)
    with open(TRAFFIC_FILE) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kind and parts[2] == dig:
                return int(parts[1])
    return None


def kind_of_kernel(name):
    """Bench kind of an ncu kernel name (None for launches that are not ours)."""
    import re
    m = re.search(r"k_fast2<[^,]+, \d+, (\d+)", name)
    if m:
        return "filter:" + {0: "mean", 1: "sigma", 2: "entropy", 3: "okada"}[int(m.group(1))]
    m = re.search(r"k_gate<[^,]+, \d+, (\d+)>", name)
    if m:   # the filter set: 3 all five (a multi-filter call), 1 the paper's filter alone, 2 comparison filters
        return {3: "filter:gate", 1: "gate:ours", 2: "gate:cube"}[int(m.group(1))]
    if "k_ours_fast" in name:
        return "filter:ours"
    for k, kind in (("k_stats_batched", None), ("k_stats<", "stats"), ("k_params", "params"),
                    ("k_entropy_pack", "entropy")):
        if k in name:
            return kind
    return None


def record_traffic(csv_path, scale):
    """Write the traffic file from an ncu CSV log (metrics dram__bytes_read.sum and
    dram__bytes_write.sum per launch, e.g. of `bench.py --dims 384 384 512`):
    mean bytes per launch of each kind, times `scale` (the voxel ratio to the
    512^3 workload), tagged with the digest of that kind's sources."""
    import csv
    rows = {}
    with open(csv_path) as f:
        lines = [l for l in f if l.startswith('"')]
    for r in csv.DictReader(lines):
        key = (r["ID"], r["Kernel Name"])
        rows.setdefault(key, {})[r["Metric Name"]] = float(r["Metric Value"].replace(",", ""))
    acc = {}
    for (_, name), m in rows.items():
        kind = kind_of_kernel(name)
        if kind is None or "dram__bytes_read.sum" not in m:
            continue
        a = acc.setdefault(kind, [0, 0.0])
        a[0] += 1
        a[1] += m["dram__bytes_read.sum"] + m.get("dram__bytes_write.sum", 0.0)
    with open(TRAFFIC_FILE, "w") as f:
        for kind in sorted(acc):
            n, b = acc[kind]
            if b / n < 1e6 and kind.startswith("filter:"):
                continue   # launches that returned at once (another kernel did the work)
            f.write(f"{kind} {int(round(b / n * scale))} {source_digest(kind)}\n")
    print(f"wrote {TRAFFIC_FILE}: {sorted(acc)}")


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path=None):
        self.index = index
        self.proc = None
        # the samples go to `path` when given (kept as evidence), else to a temporary file
        self.path = path or os.path.join(tempfile.gettempdir(), f"lnf_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


# ----------------------------------------------------------------------------- CPU oracle

def oracle_step_sample(vol, planes, threads):
    """Time the oracle on a bounded sample of one step: statistics and parameter
    derivation of the whole volume, then each filter on `planes` z-planes of the
    full 512x512 cross-section, split over `threads` threads (the C oracle
    releases the GIL).  Returns a dict: `sample_s` the wall time measured,
    `projected_s` the full step (filter time scaled by nz / planes), `desc`."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    st = oracle.stats(vol)
    t_stats = time.perf_counter() - t0
    t0 = time.perf_counter()
    prm = oracle.derive_params(st, RADIUS)
    t_params = time.perf_counter() - t0
    nz, ny, nx = vol.shape
    z0 = nz // 2 - planes // 2
    per = max(1, planes // threads)
    slabs = [(z, min(per, z0 + planes - z)) for z in range(z0, z0 + planes, per)]
    t_filters = 0.0
    for f in range(5):
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda s: oracle.filter_volume(vol, f, RADIUS, params=prm,
                                                       roi=(0, 0, s[0], nx, ny, s[1])), slabs))
        t_filters += time.perf_counter() - t0
    desc = (f"oracle (plain C per-voxel enumeration + exact Python parameters): statistics and parameters "
            f"of the whole {nx}x{ny}x{nz} volume, each filter on {planes} z-planes x {nx}x{ny} "
            f"({planes * nx * ny} voxels) over {threads} threads; the full step projects the filter time "
            f"by {nz}/{planes}")
    return {"sample_s": t_stats + t_params + t_filters,
            "projected_s": t_stats + t_params + t_filters * (nz / planes),
            "stats_params_s": t_stats + t_params, "filter_sample_s": t_filters, "desc": desc}


def oracle_single_thread(vol, planes=2):
    """The oracle's filters on one thread: `planes` z-planes of the volume per
    filter at the bench radius (parameters derived beforehand, not timed).
    Returns the filter throughput in GVoxel/s (five filters' voxels) and a
    description."""
    import oracle
    st = oracle.stats(vol)
    prm = oracle.derive_params(st, RADIUS)
    nz, ny, nx = vol.shape
    z0 = nz // 2 - planes // 2
    t0 = time.perf_counter()
    for f in range(5):
        oracle.filter_volume(vol, f, RADIUS, params=prm, roi=(0, 0, z0, nx, ny, planes))
    dt = time.perf_counter() - t0
    return 5 * planes * nx * ny / dt / 1e9, (f"one thread, each filter on {planes} z-planes x {nx}x{ny} "
                                             f"({planes * nx * ny} voxels), statistics and parameters not timed")


def cpu_baseline_entry(vol, threads, sample):
    """The cpu_baseline object from one step sample (see oracle_step_sample)."""
    st_value, st_desc = oracle_single_thread(vol)
    return {"value": 5 * N_VOX / sample["projected_s"] / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": sample["desc"], "sample_ms": sample["sample_s"] * 1e3,
            "projected_step_ms": sample["projected_s"] * 1e3,
            "single_thread": {"value": st_value, "unit": UNIT, "sample": st_desc}}


def run_reference(args):
    import numpy as np  # noqa: F401
    import oracle
    import phantoms
    oracle.build()
    vol = phantoms.P2()
    threads = os.cpu_count() or 1
    planes = max(threads, 4)
    for _ in range(args.warmup):
        oracle_step_sample(vol, planes, threads)
    samples = [oracle_step_sample(vol, planes, threads) for _ in range(args.steps)]
    mean = {k: sum(s[k] for s in samples) / len(samples) for k in ("sample_s", "projected_s")}
    mean["desc"] = samples[-1]["desc"]
    cpu = cpu_baseline_entry(vol, threads, mean)
    value = cpu["value"]
    # ms_per_step: what one step of this run timed (the bounded sample); the metric's
    # value: the full 512^3 step projected from it (projected_step_ms)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean["sample_s"] * 1e3,
            "projected_step_ms": mean["projected_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "radius": RADIUS, "filters": FILTER_NAMES,
                       "sample": "each step: the oracle on a bounded sample of the step (cpu_baseline.sample)"},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------- extra configurations

def ctx_kwargs(args):
    """lnf.Context keyword arguments from the configuration flags, and the
    non-default ones (for the line's config)."""
    kw = {"threshold_mode": args.threshold_mode, "threshold_value": args.threshold_value, "sigma_k": args.sigma_k,
          "okada_td": args.okada_td, "entropy_te": args.entropy_te, "entropy_local_te": args.entropy_local_te,
          "cluster_offset": args.cluster_offset, "autotune": args.autotune}
    defaults = {"threshold_mode": 0, "threshold_value": 0, "sigma_k": 2, "okada_td": -1, "entropy_te": -2,
                "entropy_local_te": -2, "cluster_offset": 1, "autotune": False}
    return kw, {k: v for k, v in kw.items() if v != defaults[k]}


def start_generation():
    """Draw the extra workloads' volumes (the 1024^3 uint8 phantom, the 64^3
    phantom, the served and the batched volumes) in a spawn process pool started
    before any CUDA call, while the GPU runs the main step."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import phantoms
    ex = ProcessPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)), mp_context=mp.get_context("spawn"))
    specs = phantoms.batch_volume_specs(64)
    sizes = served_sizes()
    futs = {"P3": ex.submit(phantoms.P3), "P1": ex.submit(phantoms.P1),
            "served": [ex.submit(phantoms.insect_phantom, (n, n, n), 2000 + i, "u16") for i, n in enumerate(sizes)],
            "batch": [ex.submit(phantoms.batch_volume, sp) for sp in specs]}
    return ex, futs, specs, sizes


def finish_generation(gen):
    ex, futs, specs, sizes = gen
    out = {"P3": futs["P3"].result(), "P1": futs["P1"].result(), "served": [f.result() for f in futs["served"]],
           "batch": [f.result() for f in futs["batch"]], "specs": specs, "sizes": sizes}
    ex.shutdown()
    return out


def timed_calls(ctx, fn, torch, warmup, steps):
    """CUDA-event ms per call of `fn` on torch's current stream, and the mean ms
    per call of each kernel kind the library's profiler bracketed."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ctx.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    kern, _ = ctx.profile_read()
    ctx.profile(False)
    return e0.elapsed_time(e1) / steps, {k: v[1] / steps for k, v in kern.items()}


def ours_kernel(kern):
    """The kernel that did the paper's filter's work in a single-filter call: the
    gate-first kernel or the ring kernel (the other returns at once).  The call's
    "filter:ours" bracket holds both launches, "gate:ours" the gate-first one:
    when that holds most of the call's time, the gate-first kernel did the work."""
    ring = kern.get("filter:ours", 0.0)
    gate = kern.get("gate:ours", 0.0)
    if gate > 0.5 * ring:
        return "gate:ours", gate
    return "filter:ours", ring


def extra_configs(lnf, torch, gen, t_p2, hbm_gbs, warmup, steps):
    """The workloads beside the main step, each on its own inputs (all larger
    than L2 except the 64^3 latency case, which flushes L2 between calls)."""
    import numpy as np
    res = {}
    # (a) the paper's filter on a dense volume: the 512^3 phantom with no noise
    # threshold, so every voxel passes the gate and the ring kernel does the work
    ctx = lnf.Context(threshold_mode=lnf.THRESH_NONE)
    out = torch.empty_like(t_p2)
    call_ms, kern = timed_calls(ctx, lambda: ctx.filter_volume(t_p2, lnf.OURS, RADIUS, out=out), torch, warmup, steps)
    kind, kms = ours_kernel(kern)
    n = t_p2.numel()
    res["ours_dense_512_u16"] = {
        "workload": "512^3 uint16 phantom, paper's filter r=2, no noise threshold (every voxel passes)",
        "call_ms": call_ms, "kernel": kind, "kernel_ms": kms, "gvox_s": n / call_ms / 1e6,
        "hbm_frac": 2 * n * 2 / (kms / 1e3) / 1e9 / hbm_gbs}
    ctx.close()
    del out
    # (b) the 1024^3 uint8 phantom, the paper's filter at r = 1..4
    t3 = torch.from_numpy(gen["P3"]).cuda()
    o3 = torch.empty_like(t3)
    n3 = t3.numel()
    ctx = lnf.Context()
    sweep = {}
    for r in (1, 2, 3, 4):
        call_ms, kern = timed_calls(ctx, lambda: ctx.filter_volume(t3, lnf.OURS, r, out=o3), torch, warmup, steps)
        kind, kms = ours_kernel(kern)
        sweep[str(r)] = {"call_ms": call_ms, "gvox_s": n3 / call_ms / 1e6, "kernel": kind, "kernel_ms": kms,
                         "kernel_gvox_s": n3 / kms / 1e6, "hbm_frac": 2 * n3 / (kms / 1e3) / 1e9 / hbm_gbs}
    T = ctx.params()["threshold"]
    res["radius_sweep_1024_u8"] = {
        "workload": "1024^3 uint8 insect-like phantom, paper's filter r = 1..4 (call: statistics, parameters, "
                    "filter; kernel: the filter kernel alone, 2 bytes per voxel)",
        "pass_fraction": float(np.count_nonzero(gen["P3"] >= T)) / n3, "radii": sweep}
    ctx.close()
    del t3, o3
    # (c) latency of one call on the 64^3 uint8 phantom: the paper's filter at r=1
    # and the entropy of input and output, L2 flushed (a 256 MB write) before each
    t1 = torch.from_numpy(gen["P1"]).cuda()
    o1 = torch.empty_like(t1)
    H1 = torch.zeros(2, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")
    ctx = lnf.Context()
    for _ in range(warmup):
        ctx.filter_multi(t1, [lnf.OURS], 1, outs=[o1], H=H1)
    dev_ms, host_ms = [], []
    for _ in range(50):
        flush.add_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        h0 = time.perf_counter()
        e0.record()
        ctx.filter_multi(t1, [lnf.OURS], 1, outs=[o1], H=H1)
        e1.record()
        torch.cuda.synchronize()
        host_ms.append((time.perf_counter() - h0) * 1e3)
        dev_ms.append(e0.elapsed_time(e1))
    res["p1_latency_64_u8"] = {
        "workload": "64^3 uint8 ellipsoid phantom, paper's filter r=1 with input and output entropy, "
                    "one call, L2 flushed before each",
        "device_ms_p50": float(np.percentile(dev_ms, 50)), "device_ms_p99": float(np.percentile(dev_ms, 99)),
        "host_ms_p50": float(np.percentile(host_ms, 50)), "calls": len(dev_ms)}
    ctx.close()
    del t1, o1, flush
    torch.cuda.empty_cache()
    # (d) batched and (e) served
    b = batched_result(lnf, torch, gen["batch"], gen["specs"], warmup, steps)
    res["batched"] = {k: b[k] for k in ("workload", "voxels_per_batch", "batched", "per_volume_loop", "speedup",
                                        "autotune")}
    torch.cuda.empty_cache()
    res["served"] = served_result(lnf, torch, gen["served"], gen["sizes"], 200.0, 5.0)
    torch.cuda.empty_cache()
    return res


# ----------------------------------------------------------------------------- GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lnf", choices=["lnf", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="plain",
                    choices=["plain", "ours", "batched", "served", "render", "variants", "spacing"],
                    help="plain: the 512^3 five-filter step (default); batched / served: the delivery forms")
    ap.add_argument("--duration", type=float, default=10.0, help="served: seconds of Poisson arrivals")
    ap.add_argument("--rate", type=float, default=200.0, help="served: requests per second")
    ap.add_argument("--dims", type=int, nargs=3, default=None,
                    help="profiling: a smaller phantom of the same workload (nx ny nz); not a bench line")
    ap.add_argument("--no-e2e", action="store_true", help="profiling: skip the host-buffer leg")
    # the library's configuration (lnf_config), for the main step and --mode ours
    ap.add_argument("--threshold-mode", type=int, default=0, choices=[0, 1, 2],
                    help="noise threshold: 0 Otsu (Eq. 1), 1 fixed (--threshold-value), 2 none")
    ap.add_argument("--threshold-value", type=int, default=0)
    ap.add_argument("--sigma-k", type=int, default=2, help="sigma band half-width in units of sigma (Eq. 5: 2)")
    ap.add_argument("--okada-td", type=int, default=-1, help="Okada T_d (Eq. 6), -1 automatic")
    ap.add_argument("--entropy-te", type=int, default=-2, help="entropy filter T_e in weight units, -2 auto, -1 all")
    ap.add_argument("--entropy-local-te", type=int, default=-2,
                    help="local entropy filter theta in 2^-22 bits, -2 auto (log2(m)/2), -1 all")
    ap.add_argument("--cluster-offset", type=int, default=1, help="d of the diagonal clusters (paper: 1)")
    ap.add_argument("--autotune", action="store_true", help="lnf_config.autotune (batched calls)")
    ap.add_argument("--dense", action="store_true",
                    help="--mode ours: no noise threshold, so every voxel passes and the ring kernel does the work")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra configurations (radius sweep, dense, latency, batched, served)")
    ap.add_argument("--clocks-csv", default=None, help="keep the nvidia-smi clock samples in this file")
    ap.add_argument("--record-traffic", default=None, metavar="NCU_CSV",
                    help="write the per-kind DRAM traffic file from an ncu CSV log and exit")
    ap.add_argument("--traffic-scale", type=float, default=1.0,
                    help="with --record-traffic: voxels of the 512^3 workload / voxels of the captured case")
    args = ap.parse_args()
    if args.record_traffic:
        return record_traffic(args.record_traffic, args.traffic_scale)
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    if args.mode == "ours":
        return run_ours(args)
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "served":
        return run_served(args)
    if args.mode == "render":
        return run_render(args)
    if args.mode == "variants":
        return run_variants(args)
    if args.mode == "spacing":
        return run_spacing(args)

    # the extra workloads' volumes are drawn meanwhile, in processes started before CUDA
    gen = None
    if world == 1 and not args.dims and not args.no_extras:
        gen = start_generation()

    import numpy as np
    import torch
    import phantoms
    import paper_1807_03119_gb300 as lnf
    from paper_1807_03119_gb300 import builder

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(lnf.LIB_PATH):
        builder.build()
    if world > 1:
        dist.barrier()
    lnf.load()

    global N_VOX
    if args.dims:
        vol = phantoms.P2(seed=2 + rank, dims=tuple(args.dims))
        N_VOX = int(vol.size)
    else:
        vol = phantoms.P2(seed=2 + rank)   # each rank filters its own volume (weak scaling)
    t = torch.from_numpy(vol).cuda()
    filters = [lnf.MEAN, lnf.SIGMA, lnf.ENTROPY, lnf.OKADA, lnf.OURS]
    outs = [torch.empty_like(t) for _ in filters]
    H = torch.zeros(len(filters) + 1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ckw, cfg_set = ctx_kwargs(args)
    ctx = lnf.Context(**ckw)

    def step():
        ctx.filter_multi(t, filters, RADIUS, outs=outs, H=H)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local, args.clocks_csv)
    sampler.start()
    ctx.profile(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    kern, launches = ctx.profile_read()
    ctx.profile(False)
    ms = max_over_ranks(ms, world, "cuda")
    value = world * 5 * N_VOX / (ms / 1e3) / 1e9

    # the host legs below (end to end, the oracle) run with the generator pool done
    gen_data = finish_generation(gen) if gen else None
    if args.no_e2e:
        args.e2e_steps = 0
    # end to end through the host-buffer entry point, from pinned host memory
    pin_in = torch.from_numpy(vol).pin_memory()
    pin_outs = [torch.empty(vol.shape, dtype=torch.uint16).pin_memory() for _ in filters]
    in_np = pin_in.numpy()
    outs_np = [o.numpy() for o in pin_outs]
    if args.e2e_steps > 0:
        ctx.filter_multi_host(in_np, filters, RADIUS, outs=outs_np)   # staging allocation
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ctx.filter_multi_host(in_np, filters, RADIUS, outs=outs_np)
    e2e_s = (time.perf_counter() - t0) / max(1, args.e2e_steps) if args.e2e_steps > 0 else float("nan")
    e2e_s = max_over_ranks(e2e_s, world, "cuda")
    e2e = None
    if args.e2e_steps > 0:
        e2e = {"value": world * 5 * N_VOX / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": N_VOX * ES, "d2h_bytes_per_step": 5 * N_VOX * ES + 8 * 6,
               "ms_per_step": e2e_s * 1e3}

    if rank != 0:
        ctx.close()
        if world > 1:
            dist.destroy_process_group()
        return

    pk = peaks()
    sm_mhz = pk["sm_max_mhz"]
    # voxels whose own value passes the gate: the ones sigma and Okada evaluate
    T = ctx.params()["threshold"]
    n_pass = int(np.count_nonzero(vol >= T))
    rooflines = {}
    # while the gate-first kernel does the five filters, their ring kernels return at once
    five = ("filter:mean", "filter:sigma", "filter:entropy", "filter:okada", "filter:ours")
    gate_worked = "filter:gate" in kern and all(k not in kern or kern[k][1] < 0.1 * kern["filter:gate"][1]
                                                for k in five)
    for kind, (n, tot) in kern.items():
        if gate_worked and kind in five:
            continue
        bound, work = algorithmic(kind, n_pass, pk["hbm_gbs"], alu_peak_tops(sm_mhz))
        if bound is None or n == 0:
            continue
        avg_s = tot / n / 1e3
        if bound == "hbm":
            ach = work / avg_s / 1e9
            rooflines[kind] = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                               "frac": ach / pk["hbm_gbs"], "avg_ms": tot / n,
                               "traffic": recorded_traffic(kind)}
        else:
            peak = alu_peak_tops(sm_mhz)
            ach = work / avg_s / 1e12
            rooflines[kind] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Tops/s",
                               "frac": ach / peak, "avg_ms": tot / n, "traffic": recorded_traffic(kind),
                               "hbm_gbs": N_VOX * ES * 2 / avg_s / 1e9}
        if kind in ("filter:sigma", "filter:okada"):
            rooflines[kind]["gated_voxels"] = n_pass
    dom = max((k for k in rooflines), key=lambda k: kern[k][1]) if rooflines else None
    roof = dict(rooflines[dom], kernel=dom) if dom else None
    if roof:
        roof["peak_source"] = f"{pk['source']} ({'HBM copy' if roof['bound'] == 'hbm' else 'units x max clock'})"

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        cpu = cpu_baseline_entry(vol, threads, oracle_step_sample(vol, max(threads, 4), threads))

    extras = None
    if gen_data is not None:
        sampler = ClockSampler(local, None)
        sampler.start()
        extras = extra_configs(lnf, torch, gen_data, t, pk["hbm_gbs"], args.warmup, 10)
        extras["clocks"] = sampler.stop()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u16", "data": "synthetic",
        "config": dict({"workload": WORKLOAD, "radius": RADIUS, "filters": FILTER_NAMES,
                        "l2": "inputs larger than L2 (268 MB per volume, 1.6 GB touched per step)",
                        "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
                       **({"lnf_config": cfg_set} if cfg_set else {})),
        "e2e": e2e, "gpu_launches": launches, "roofline": roof, "rooflines": rooflines,
        "kernel_ms": {k: v[1] / args.steps for k, v in kern.items()},
        "hbm_gbs_step": (N_VOX * ES + 5 * N_VOX * ES * 2) / (ms / 1e3) / 1e9,
        "cpu_baseline": cpu, "clocks": clocks,
        "entropy": [float(x) for x in H.cpu().numpy()],
    }
    if extras is not None:
        line["extra"] = extras
    print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- delivery forms

def served_sizes():
    """Side lengths of the eight resident volumes of the served workload."""
    import numpy as np
    return [int(np.random.default_rng(2000 + i).integers(128, 769)) for i in range(8)]


def batched_result(lnf, torch, host_vols, specs, warmup, steps):
    """64 uneven volumes, the paper's filter at each spec's radius: one
    persistent graph-captured launch (lnf_filter_batch) against the per-volume
    launch loop (lnf_filter_volume per volume); CUDA-event ms per batch."""
    vols = [torch.from_numpy(v).cuda() for v in host_vols]
    outs = [torch.empty_like(v) for v in vols]
    nvox = sum(v.numel() for v in vols)
    ctx = lnf.Context(autotune=True)
    jobs = [{"in": v, "out": o, "filter": lnf.OURS, "radius": s["radius"]} for v, o, s in zip(vols, outs, specs)]

    def batched():
        ctx.filter_batch(jobs)

    def loop():
        for v, o, s in zip(vols, outs, specs):
            ctx.filter_volume(v, lnf.OURS, s["radius"], out=o)

    res = {}
    for name, fn in (("batched", batched), ("per_volume_loop", loop)):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[name] = {"ms_per_batch": ms, "gvox_s": nvox / (ms / 1e3) / 1e9}
    res["autotune"] = ctx.tuning()
    ctx.close()
    res["speedup"] = res["per_volume_loop"]["ms_per_batch"] / res["batched"]["ms_per_batch"]
    res["voxels_per_batch"] = nvox
    res["workload"] = "64 uneven volumes 96..384 per axis, half uint8 half uint16, paper's filter r in {1,2}"
    return res


def run_batched(args):
    """The batched workload on its own line."""
    import torch
    import phantoms
    import paper_1807_03119_gb300 as lnf
    from paper_1807_03119_gb300 import builder
    builder.build()
    lnf.load()
    specs = phantoms.batch_volume_specs(64)
    res = batched_result(lnf, torch, [phantoms.batch_volume(s) for s in specs], specs, args.warmup, args.steps)
    line = {"metric": "batched vs per-volume loop, GVoxel/s", "mode": "batched",
            "value": res["batched"]["gvox_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "u8+u16", "data": "synthetic",
            "config": {"workload": res["workload"], "voxels_per_batch": res["voxels_per_batch"]},
            "batched": res["batched"], "per_volume_loop": res["per_volume_loop"], "speedup": res["speedup"],
            "autotune": res["autotune"]}
    print(json.dumps(line))


def served_result(lnf, torch, host_vols, sizes, rate, duration):
    """8 resident uint16 volumes, a Poisson request stream (`rate` per second for
    `duration` s) of full-volume or ROI requests with random filter and r in
    {1,2,3}, admitted under a 40 GiB budget: p50/p99 latency at that load, the
    capacity with every request queued at once, and serial plain calls on the
    same requests."""
    import numpy as np
    rng = np.random.default_rng(42)
    n_req = int(rate * duration)
    gaps = rng.exponential(1.0 / rate, n_req)
    reqs = []
    for k in range(n_req):
        vi = int(rng.integers(0, 8))
        n = sizes[vi]
        f = int(rng.integers(0, 5))
        r = int(rng.integers(1, 4))
        if rng.random() < 0.5:
            reqs.append((vi, f, r, None))
        else:
            d = [int(rng.integers(32, min(256, n) + 1)) for _ in range(3)]
            o = [int(rng.integers(0, n - d[a] + 1)) for a in range(3)]
            reqs.append((vi, f, r, (o, d)))
    ctx = lnf.Context(hbm_budget_bytes=40 << 30, max_inflight=64)
    ids = [ctx.register_volume(torch.from_numpy(v).cuda()) for v in host_vols]
    now = ctx.lib.lnf_now
    # warm-up: one request per filter
    for f in range(5):
        t = ctx.submit(ids[0], f, 1)
        ctx.wait(t)
        ctx.release(t)

    def voxels(req):
        vi, f, r, roi = req
        return int(np.prod(roi[1])) if roi else sizes[vi] ** 3

    def submit(k, arr):
        vi, f, r, roi = reqs[k]
        if roi:
            return ctx.submit(ids[vi], f, r, roi_origin=roi[0], roi_dims=roi[1], arrival_time=arr)
        return ctx.submit(ids[vi], f, r, arrival_time=arr)

    def drain(pending, lat, block):
        """Release finished requests (oldest first), as a client consuming its
        results would; returns the latest finish time seen."""
        t_last = 0.0
        while pending:
            tk, arr = pending[0]
            res = ctx.wait(tk, 600.0) if block else ctx.poll(tk)
            if res is None:
                break
            pending.pop(0)
            lat.append(res.t_finish - arr)
            t_last = max(t_last, res.t_finish)
            ctx.release(tk)
        return t_last

    # (1) latency at the stated load: Poisson arrivals at `rate` per second
    pending, lat = [], []
    t0 = now()
    t_next = t0
    t_last = 0.0
    for k in range(n_req):
        t_next += gaps[k]
        while now() < t_next:
            t_last = max(t_last, drain(pending, lat, False))
        arr = now()
        pending.append((submit(k, arr), arr))
    t_last = max(t_last, drain(pending, lat, True))
    vox = sum(voxels(q) for q in reqs)
    lat = np.array(lat) * 1e3
    load_s = t_last - t0
    # (2) capacity: every request queued at once, against serial plain calls
    pending, lat_sat = [], []
    t1 = now()
    for k in range(n_req):
        pending.append((submit(k, t1), t1))
    served_s = drain(pending, lat_sat, True) - t1
    # serial plain calls on the same requests (device buffers, one sync per request)
    dvols = [torch.from_numpy(v).cuda() for v in host_vols]
    torch.cuda.synchronize()
    ts = time.perf_counter()
    for vi, f, r, roi in reqs:
        if roi:
            o = ctx.filter_roi(dvols[vi], f, r, tuple(roi[0]), tuple(roi[1]))
        else:
            o = ctx.filter_volume(dvols[vi], f, r)
        torch.cuda.synchronize()
        del o
    serial_s = time.perf_counter() - ts
    ctx.close()
    return {"workload": "8 resident uint16 volumes 128..768 per side, Poisson arrivals, half full-volume half "
                        "ROI 32..256, random filter, r in {1,2,3}, 40 GiB budget",
            "rate_per_s": rate, "duration_s": duration, "requests": n_req, "sizes": sizes,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max()), "at_rate_per_s": rate, "seconds_to_last_result": load_s},
            "served": {"seconds": served_s, "gvox_s": vox / served_s / 1e9,
                       "note": "all requests queued at once (capacity)"},
            "serial_plain": {"seconds": serial_s, "gvox_s": vox / serial_s / 1e9},
            "offered_gvox_s": vox / duration / 1e9}


def run_served(args):
    """The served workload on its own line."""
    import torch
    import phantoms
    import paper_1807_03119_gb300 as lnf
    from paper_1807_03119_gb300 import builder
    builder.build()
    lnf.load()
    sizes = served_sizes()
    vols = [phantoms.insect_phantom((n, n, n), 2000 + i, "u16") for i, n in enumerate(sizes)]
    res = served_result(lnf, torch, vols, sizes, args.rate, args.duration)
    line = {"metric": "served p50/p99 ms and GVoxel/s vs serial plain calls", "mode": "served",
            "value": res["served"]["gvox_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "u16", "data": "synthetic",
            "config": {"workload": res["workload"], "rate_per_s": args.rate, "duration_s": args.duration,
                       "requests": res["requests"], "sizes": sizes},
            "latency_ms": res["latency_ms"], "served": res["served"], "serial_plain": res["serial_plain"],
            "offered_gvox_s": res["offered_gvox_s"]}
    print(json.dumps(line))


def run_ours(args):
    """The paper's filter alone on the 512^3 uint16 phantom at r = 2 through
    lnf_filter_volume (statistics, parameters, the filter and its output
    histogram): device ms per call, and the roofline of the kernel that did the
    filter's work (2 bytes read and 2 written per voxel)."""
    import torch
    import phantoms
    import paper_1807_03119_gb300 as lnf
    from paper_1807_03119_gb300 import builder
    builder.build()
    lnf.load()
    vol = phantoms.P2()
    t = torch.from_numpy(vol).cuda()
    out = torch.empty_like(t)
    ckw, cfg_set = ctx_kwargs(args)
    if args.dense:
        ckw["threshold_mode"] = lnf.THRESH_NONE
    ctx = lnf.Context(**ckw)
    sampler = ClockSampler(0, args.clocks_csv)
    sampler.start()
    call_ms, kern = timed_calls(ctx, lambda: ctx.filter_volume(t, lnf.OURS, RADIUS, out=out), torch, args.warmup,
                                args.steps)
    clocks = sampler.stop()
    kind, kms = ours_kernel(kern)
    pk = peaks()
    ach = N_VOX * ES * 2 / (kms / 1e3) / 1e9
    line = {"metric": "paper's filter alone, 512^3 uint16 r=2, GVoxel/s", "mode": "ours_dense" if args.dense else "ours",
            "value": N_VOX / call_ms / 1e6, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_call": call_ms, "higher_is_better": True, "dtype": "u16", "data": "synthetic",
            "config": dict({"workload": "512x512x512 uint16 insect-like phantom, the paper's filter at r=2 with "
                                        "its output histogram" +
                                        (", no noise threshold (every voxel passes)" if args.dense else ""),
                            "l2": "inputs larger than L2"}, **({"lnf_config": cfg_set} if cfg_set else {})),
            "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / pk["hbm_gbs"], "avg_ms": kms, "kernel": kind, "traffic": recorded_traffic(kind)},
            "kernel_ms": kern, "clocks": clocks}
    print(json.dumps(line))
    ctx.close()


def run_render(args):
    """The paper's use of its filter: ray-cast the 512^3 uint16 phantom along +z
    (512 x 512 rays) with each filter at r = 2 deciding at the candidate surface
    points.  Per filter: ms per frame for the whole lnf_render call (statistics,
    parameters, rays) and for the ray kernel alone, with the oracle's renderer
    timed on a bounded sample of the rays beside it."""
    import numpy as np
    import torch
    import oracle
    import phantoms
    import paper_1807_03119_gb300 as lnf
    from paper_1807_03119_gb300 import builder
    builder.build()
    lnf.load()
    vol = phantoms.P2()
    t = torch.from_numpy(vol).cuda()
    ctx = lnf.Context()
    rows = 8   # oracle sample: the rays of the first `rows` image rows
    st = oracle.stats(vol)
    res = {}
    for name in FILTER_NAMES:
        f = lnf.FILTERS[name]
        for _ in range(args.warmup):
            ctx.render(t, f, RADIUS, 4, with_depth=False, with_value=False)
        torch.cuda.synchronize()
        ctx.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            im, _, _ = ctx.render(t, f, RADIUS, 4, with_depth=False, with_value=False)
        e1.record()
        torch.cuda.synchronize()
        kern, _ = ctx.profile_read()
        ctx.profile(False)
        ms = e0.elapsed_time(e1) / args.steps
        rk = kern.get("render", (1, float("nan")))
        hit = float((im > 0).float().mean())
        prm = oracle.derive_params(st, RADIUS)
        c0 = time.perf_counter()
        oracle.render(np.ascontiguousarray(vol[:, :rows, :]), f, RADIUS, 4, params=prm)
        cpu_ms = (time.perf_counter() - c0) * 1e3 * (vol.shape[1] / rows)
        res[name] = {"ms_per_frame": ms, "ray_kernel_ms": rk[1] / rk[0], "rays_per_s": 512 * 512 / (ms / 1e3),
                     "hit_fraction": hit, "oracle_ms_per_frame": cpu_ms}
    line = {"metric": "render ms per frame: 512x512 rays along +z through 512^3 uint16, r=2",
            "mode": "render", "value": sum(v["ms_per_frame"] for v in res.values()) / len(res), "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "dtype": "u16", "data": "synthetic",
            "config": {"workload": "512x512x512 uint16 insect-like phantom, orthographic rays along +z",
                       "radius": RADIUS, "oracle_sample": f"the rays of {rows} image rows, scaled to 512 rows, "
                                                          "1 host thread"},
            "filters": res}
    print(json.dumps(line))
    ctx.close()


def run_variants(args):
    """The variants beside the filters they vary, on the 512^3 uint16 phantom at
    r = 2: the cluster-layout variants of the paper's filter (axis-cross and cube
    clusters), the sigma filter with the local sigma of its cube and the entropy
    filter with the grey-level probabilities of its cube; device ms per launch
    (the variants run on the generic kernel, the paper's filter and the sigma
    filter on their specialised ones)."""
    import torch
    import phantoms
    import paper_1807_03119_gb300 as lnf
    from paper_1807_03119_gb300 import builder
    builder.build()
    lnf.load()
    vol = phantoms.P2()
    t = torch.from_numpy(vol).cuda()
    out = torch.empty_like(t)
    ctx = lnf.Context()
    res = {}
    for name in ("ours", "ours_cross", "ours_cube", "sigma", "sigma_local", "entropy_local"):
        f = lnf.FILTERS[name]
        for _ in range(args.warmup):
            ctx.filter_volume(t, f, RADIUS, out=out)
        torch.cuda.synchronize()
        ctx.profile(True)
        for _ in range(args.steps):
            ctx.filter_volume(t, f, RADIUS, out=out)
        torch.cuda.synchronize()
        kern, _ = ctx.profile_read()
        ctx.profile(False)
        # the paper's filter: the kernel that did the work (gate-first or ring)
        kind = ours_kernel({k: v[1] for k, v in kern.items()})[0] if name == "ours" else "filter:" + name
        n, tot = kern[kind]
        ms = tot / n
        res[name] = {"ms_per_launch": ms, "gvox_s": N_VOX / (ms / 1e3) / 1e9,
                     "hbm_frac": N_VOX * ES * 2 / (ms / 1e3) / 1e9 / peaks()["hbm_gbs"]}
    # the gate-first kernels against the plane-ring kernels alone on a sparse
    # volume: 12-bit background noise (400, sigma 30) with 0.1% salt, so about
    # 0.1% of the voxels pass the gate; the paper's filter alone and the five
    # filters of one multi-filter call
    import numpy as np
    rng = np.random.default_rng(9)
    sv = np.clip(np.rint(rng.normal(400.0, 30.0, vol.shape).astype(np.float32)), 0, 4095).astype(np.uint16)
    sv.reshape(-1)[rng.integers(0, sv.size, sv.size // 1000)] = 4095
    ts = torch.from_numpy(sv).cuda()
    os.environ["LNF_NO_GATE"] = "1"
    ring_ctx = lnf.Context()
    del os.environ["LNF_NO_GATE"]
    five = [lnf.FILTERS[n] for n in FILTER_NAMES]
    outs = [torch.empty_like(ts) for _ in five]
    calls = {"ours": lambda c: c.filter_volume(ts, lnf.OURS, RADIUS, out=out),
             "five_filters": lambda c: c.filter_multi(ts, five, RADIUS, outs=outs)}
    sparse = {}
    for name, call in calls.items():
        row = {}
        for label, c in (("gate", ctx), ("ring", ring_ctx)):
            for _ in range(args.warmup):
                call(c)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                call(c)
            e1.record()
            torch.cuda.synchronize()
            row[label + "_ms_per_call"] = e0.elapsed_time(e1) / args.steps
        sparse[name] = row
    sparse["passing_fraction"] = float(np.count_nonzero(sv >= ctx.params()["threshold"]) / sv.size)
    del sv
    ring_ctx.close()
    line = {"metric": "filter variants (cluster layouts, local sigma, local entropy), 512^3 uint16, r=2",
            "mode": "variants",
            "value": res["ours_cube"]["gvox_s"], "unit": UNIT, "higher_is_better": True, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "dtype": "u16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "radius": RADIUS,
                       "sparse_workload": "512^3 uint16, noise 400 +- 30 with 0.1% salt at 4095"},
            "filters": res, "sparse_gate_vs_ring": sparse}
    print(json.dumps(line))
    ctx.close()


def run_spacing(args):
    """Anisotropic voxel spacing and float32 volumes on the 512^3 phantom.
    (a) The uint16 phantom read as a grid of spacing (1, 1, 2) (slices twice as
    thick as the in-plane pixels): each filter at the radii of a 2-voxel extent,
    (2, 2, 1), through lnf_filter_volume_aniso.  (b) The phantom as float32
    values (v / 4 - 1000, exact in float32): the paper's filter at r = 2 through
    lnf_filter_volume_f32.  Device ms per call (events around the whole call:
    statistics, parameters, every kernel) and per kernel (the library's
    profile), GVoxel/s and HBM fractions; the oracle timed beside each on a
    bounded sample (2 of the 512 planes, scaled; float32: its whole-volume
    quantisation, statistics and parameters plus the sampled filter)."""
    import numpy as np
    import torch
    import oracle
    import phantoms
    import paper_1807_03119_gb300 as lnf
    from paper_1807_03119_gb300 import builder
    builder.build()
    lnf.load()
    vol = phantoms.P2()
    t = torch.from_numpy(vol).cuda()
    out = torch.empty_like(t)
    ctx = lnf.Context()
    hbm = peaks()["hbm_gbs"]
    radii = lnf.spacing_radii(2.0, (1.0, 1.0, 2.0))
    sample = 2
    st = oracle.stats(vol)

    def timed(call):
        for _ in range(args.warmup):
            call()
        torch.cuda.synchronize()
        ctx.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            call()
        e1.record()
        torch.cuda.synchronize()
        kern, _ = ctx.profile_read()
        ctx.profile(False)
        return e0.elapsed_time(e1) / args.steps, {k: v[1] / v[0] for k, v in kern.items()}

    aniso = {}
    for name in FILTER_NAMES:
        f = lnf.FILTERS[name]
        ms, kern = timed(lambda: ctx.filter_volume_aniso(t, f, radii, out=out))
        kms = kern["filter:" + name]
        prm = oracle.derive_params(st, radii)
        c0 = time.perf_counter()
        oracle.filter_volume(vol, f, radii, params=prm, roi=(0, 0, 0, DIMS[0], DIMS[1], sample))
        cpu_ms = (time.perf_counter() - c0) * 1e3 * DIMS[2] / sample
        aniso[name] = {"ms_per_call": ms, "filter_kernel_ms": kms, "gvox_s": N_VOX / (ms / 1e3) / 1e9,
                       "filter_hbm_frac": N_VOX * ES * 2 / (kms / 1e3) / 1e9 / hbm,
                       "oracle_ms": cpu_ms}
    vf = (vol.astype(np.float32) / np.float32(4.0) - np.float32(1000.0)).astype(np.float32)
    tf = torch.from_numpy(vf).cuda()
    of = torch.empty_like(tf)
    ms, kern = timed(lambda: ctx.filter_volume_f32(tf, lnf.OURS, RADIUS, out=of))
    per_kernel = {}
    for k, b in (("f32_range", 4), ("f32_quantize", 6), ("f32_dequantize", 6), ("filter:ours", 4)):
        if k in kern:
            per_kernel[k] = {"ms": kern[k], "gb_s": N_VOX * b / (kern[k] / 1e3) / 1e9,
                             "hbm_frac": N_VOX * b / (kern[k] / 1e3) / 1e9 / hbm, "bytes_per_voxel": b}
    c0 = time.perf_counter()
    q, lo, hi = oracle.quantize_f32(vf)
    prm = oracle.derive_params(oracle.stats(q), RADIUS)
    lv = oracle.filter_volume(q, oracle.OURS, RADIUS, params=prm, roi=(0, 0, 0, DIMS[0], DIMS[1], sample))
    oracle.dequantize_f32(lv, lo, hi)
    c1 = time.perf_counter()
    oracle.filter_volume(q, oracle.OURS, RADIUS, params=prm, roi=(0, 0, 0, DIMS[0], DIMS[1], sample))
    filt_s = time.perf_counter() - c1
    cpu_ms = ((c1 - c0) - filt_s + filt_s * DIMS[2] / sample) * 1e3
    f32 = {"ms_per_call": ms, "gvox_s": N_VOX / (ms / 1e3) / 1e9,
           "ideal_bytes_per_voxel": 8, "ideal_hbm_frac": N_VOX * 8 / (ms / 1e3) / 1e9 / hbm,
           "kernels": per_kernel, "oracle_ms": cpu_ms}
    line = {"metric": "anisotropic spacing (5 filters) and float32 (paper's filter), 512^3, GVoxel/s",
            "mode": "spacing", "value": f32["gvox_s"], "unit": UNIT, "higher_is_better": True, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "dtype": "u16 / f32", "data": "synthetic",
            "config": {"workload": "512x512x512 insect-like phantom: uint16 on a (1, 1, 2) grid at the radii "
                                   "of a 2-voxel extent; float32 copy v / 4 - 1000, paper's filter r = 2",
                       "radii": list(radii), "oracle_sample": f"{sample} of {DIMS[2]} planes, scaled, 1 host thread"},
            "aniso": aniso, "f32": f32}
    print(json.dumps(line))
    ctx.close()


if __name__ == "__main__":
    main()
