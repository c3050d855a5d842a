"""Throughput of the coherent F-statistic on GB300: template.SFT pairs per second.

Default workload (one step = one full pass of the path over one workunit):
2 detectors x 1200 gapped SFTs (T = 1800 s), 1 Hz band at 100 Hz with 8
injected signals, templates 10 000 sky x 1800 f x 10 fdot (1.8e8 templates,
4.32e11 pairs), D = 8, top-1000.  Each step runs the FP64 timing / antenna /
basis kernel, the Dirichlet kernel with fused 2F, and the toplist selection.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form c64|f16|bf16]
  python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)
  python bench.py --config batch | semicoherent | proposal   (other workloads)
  python bench.py --coverage F | --noise-floor W | --algo ...   (variants)

The JSON line's `roofline` is the Dirichlet kernel's ALU bound (100 flop per
pair of the direct sum, peak from the queried SM count), with the DRAM traffic
and, for the table forms, the shared-memory bound (`roofline.shared_memory`)
taken from the committed ncu summary while it matches the kernel source.
`plain_fp32` times the plain FP32 form (direct Dirichlet sum) on the same
workunit; `twoF_error` gives max and p99 |GPU 2F - oracle 2F| of both forms
on the CPU baseline's sample (16 sky points x 1800 f x 10 fdot x 2400 SFTs,
signals added by the FP64 oracle), which the plain-C FP64 oracle times on
every host core (`cpu_baseline`, also one core); `--impl reference` times the
same oracle on the same sample per step.

Multi-GPU (torchrun, one process per GPU): sky points are sharded, each rank
runs a full workunit-sized step on its shard (weak scaling) and the local
toplists are merged on rank 0 through one all-gather.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOP_PER_PAIR = 100.0          # direct-sum FP32 work of one template.SFT pair: 16 bins x (4 + 1) + 20 per-pair constants
FP32_LANES = 128
METRIC = "template·SFT pairs/s (2F) on 1 GB300, chosen vs plain FP32 form at stated 2F error"
KERNEL_SOURCES = {"direct": ["fstat_internal.cuh", "dirichlet.cuh", "dirichlet_c64.cu", "dirichlet_f16.cu",
                             "dirichlet_bf16.cu"],
                  "farpoly": ["fstat_internal.cuh", "dirichlet.cuh", "dirichlet_far.cu"],
                  "sincpoly": ["fstat_internal.cuh", "dirichlet.cuh", "dirichlet_far.cu"],
                  "sincrows": ["fstat_internal.cuh", "dirichlet.cuh", "dirichlet_far.cu"],
                  "sincpairs": ["fstat_internal.cuh", "dirichlet.cuh", "dirichlet_far.cu"]}
KERNEL_NAMES = {"direct": "dirichlet_kernel", "farpoly": "dirichlet_far_kernel",
                "sincpoly": "dirichlet_far_ring_kernel", "sincrows": "dirichlet_rows_kernel",
                "sincpairs": "dirichlet_ring2_kernel"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="c64", choices=["c64", "f16", "bf16"])
    ap.add_argument("--n-sky", type=int, default=10000)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare-forms", action="store_true", help="also time the other storage forms")
    ap.add_argument("--n-seg", type=int, default=8, help="time segments (semicoherent mode)")
    ap.add_argument("--coverage", type=float, default=0.0,
                    help="per-SFT frequency coverage: this fraction of the SFTs covers a random contiguous run of "
                         "50-100 %% of the band, the rest all of it (0 = off); pairs count covered pairs only")
    ap.add_argument("--config", default="workunit", choices=["workunit", "batch", "proposal", "semicoherent"],
                    help="workunit: one workunit-sized bank (default); batch: 64 heterogeneous workunits")
    ap.add_argument("--n-wu", type=int, default=64, help="workunits in the batch mode")
    ap.add_argument("--n-train", type=int, default=512, help="training workunits (proposal mode)")
    ap.add_argument("--n-test", type=int, default=128, help="held-out workunits (proposal mode)")
    ap.add_argument("--n-refine", type=int, default=8, help="patches refined per workunit (proposal mode)")
    ap.add_argument("--train-steps", type=int, default=6000, help="Adam steps (proposal mode)")
    ap.add_argument("--proposal-sft", type=int, default=800, help="SFTs per detector (proposal mode)")
    ap.add_argument("--proposal-lines", type=int, default=3,
                    help="detector lines per workunit, at most (proposal mode: training and the second held-out set)")
    ap.add_argument("--algo", default="auto", choices=["auto", "direct", "farpoly", "sincpoly", "sincrows", "sincpairs"],
                    help="evaluation of the D-term kernel sum")
    ap.add_argument("--noise-floor", type=int, default=0,
                    help="running-median half window of the noise-floor normalisation (0 = off)")
    ap.add_argument("--tile-m", type=int, default=0, help="templates per thread (0 = planner)")
    ap.add_argument("--tile-warps", type=int, default=0, help="warps per block (0 = planner)")
    ap.add_argument("--sft-chunk", type=int, default=0, help="SFTs per staging round (0 = planner)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def workload(rank: int, world: int, n_sky: int):
    from workload import config1, fibonacci_sky
    sky_all = fibonacci_sky(n_sky * world)
    return config1(sky=sky_all[rank * n_sky:(rank + 1) * n_sky])


def algo_of(variant: int) -> str:
    """Form of a plan's kernel variant id (include/fstat.h, fstat_get_plan)."""
    if variant < 100:
        return "direct"
    if variant in (127, 128):
        return "sincpairs"
    if 120 <= variant <= 126:
        return "sincrows"
    if variant in (117, 132):   # far field with coverage; blocks of 4 sky points
        return "farpoly"
    return "sincpoly" if variant in (112, 113, 114, 115, 116, 118, 119) or variant >= 129 else "farpoly"


def kernel_hash(algo: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[algo]:
        with open(os.path.join(ROOT, "paper_0904_1826_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_entry(form: str, algo: str):
    """The committed ncu summary of the Dirichlet kernel, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "dirichlet_counters.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    e = d.get(f"{algo}/{form}")
    if not e or e.get("kernel_hash") != kernel_hash(algo):
        return None
    return e


def ncu_traffic(form: str, algo: str):
    """DRAM bytes per launch of the Dirichlet kernel (ncu, current source) or None."""
    e = ncu_entry(form, algo)
    return e.get("dram_bytes_per_full_launch") if e else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        os.unlink(self.out.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


N_SAMPLE_SKY = 16


def baseline_sample(w):
    """The bounded sample of the workunit that the CPU oracle times and that
    the GPU's 2F error is measured on: the 8 sky points of the lattice
    nearest to the 8 signals, then the first sky points, up to 16; every
    frequency, spindown and SFT of each (16 x 1800 x 10 x 2400 = 6.9e8 pairs).
    Signals are added to the SFTs by the FP64 oracle."""
    from oracle import fstat_oracle as O
    from workload import DetectorData, TemplateBank
    sky = w.bank.sky
    n = np.stack([np.cos(sky[:, 1]) * np.cos(sky[:, 0]), np.cos(sky[:, 1]) * np.sin(sky[:, 0]), np.sin(sky[:, 1])], 1)
    pick = []
    for inj in w.injections:
        v = np.array([math.cos(inj.delta) * math.cos(inj.alpha), math.cos(inj.delta) * math.sin(inj.alpha),
                      math.sin(inj.delta)])
        i = int(np.argmax(n @ v))
        if i not in pick:
            pick.append(i)
    i = 0
    while len(pick) < N_SAMPLE_SKY:
        if i not in pick:
            pick.append(i)
        i += 1
    pick = sorted(pick)
    bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
    dets = [DetectorData(d.lat, d.lon, d.az, d.t_start, b) for d, b in zip(w.detectors, bins)]
    sub = TemplateBank(sky[pick], w.bank.f0, w.bank.df, w.bank.n_f, w.bank.fdot, w.bank.t_ref)
    return pick, dets, bins, sub


def cpu_oracle_run(w, dets, sub, threads: int, n_sky: int | None = None):
    """The plain-C FP64 oracle as it stands over the sample's first n_sky sky
    points (all by default) on `threads` host threads: (pairs/s, pairs,
    seconds, 2F [n_sky][n_fdot][n_f])."""
    from oracle import c_oracle as CO
    sel = range(sub.n_sky if n_sky is None else n_sky)
    t0 = time.perf_counter()
    out = CO.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, sub, sky_indices=sel, threads=threads)
    dt = time.perf_counter() - t0
    pairs = len(sel) * sub.n_f * sub.n_fdot * w.n_sft_total
    return pairs / dt, pairs, dt, out


def cpu_baseline(w, gpu_error=None):
    """The oracle on the host cores: all cores on the 16-sky sample, one core
    on one sky point of it (the plain-C oracle), and the numpy oracle on one
    sky point x 2 spindowns; the numbers the 2F error is measured against come
    from the all-core run.  gpu_error(pick, bins, sub, ref) -> dict, if given,
    measures the GPU's 2F on the same sample against the oracle's."""
    from oracle import fstat_oracle as O
    from workload import TemplateBank
    nproc = os.cpu_count() or 1
    pick, dets, bins, sub = baseline_sample(w)
    v_all, p_all, t_all, ref = cpu_oracle_run(w, dets, sub, nproc)
    v_one, p_one, t_one, _ = cpu_oracle_run(w, dets, sub, 1, n_sky=1)
    one = TemplateBank(sub.sky[:1], sub.f0, sub.df, sub.n_f, sub.fdot[:2], sub.t_ref)
    t0 = time.perf_counter()
    O.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, one)
    t_np = time.perf_counter() - t0
    p_np = one.n_f * one.n_fdot * w.n_sft_total
    out = {"value": v_all, "unit": "pairs/s", "cores": min(nproc, sub.n_sky), "kind": "oracle",
           "sample": f"{sub.n_sky} sky (lattice points nearest the 8 signals, then the first) x {sub.n_f} f x "
                     f"{sub.n_fdot} fdot x {w.n_sft_total} SFT = {p_all:.3g} pairs, plain-C FP64 oracle on "
                     f"{min(nproc, sub.n_sky)} threads, {t_all:.1f} s",
           "nproc": nproc, "cpu_model": cpu_model(),
           "single_core": {"value": v_one, "unit": "pairs/s", "sample": f"1 sky x {sub.n_f} f x {sub.n_fdot} fdot "
                                                                        f"x {w.n_sft_total} SFT, {t_one:.1f} s"},
           "numpy_single_core": {"value": p_np / t_np, "unit": "pairs/s",
                                 "sample": f"1 sky x {one.n_f} f x {one.n_fdot} fdot x {w.n_sft_total} SFT, "
                                           f"{t_np:.1f} s"}}
    if gpu_error is not None:
        out["gpu_2F_error"] = gpu_error(pick, bins, sub, ref)
    return out


def twoF_error_stats(got, ref) -> dict:
    """max and p99 of |GPU 2F - oracle 2F| and the largest ratio to the
    tolerance 1e-4 2F + 1e-3, over every template of the sample."""
    got = np.asarray(got, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    err = np.abs(got - ref)
    return {"max_abs": float(err.max()), "p99_abs": float(np.percentile(err, 99)),
            "max_over_tol": float(np.max(err / (1e-4 * ref + 1e-3))), "templates": int(ref.size),
            "max_2F": float(ref.max())}


def shared_config(args) -> dict:
    """The workload description both arms print."""
    return {"workload": "plain workunit: 2 det x 1200 gapped SFT (T=1800 s), 1 Hz band at 100 Hz, "
                        "8 injected signals; 10000 sky x 1800 f x 10 fdot, D=8, top-1000",
            "form": args.form, "pairs_per_step_per_gpu": 432000000000,
            "l2": "per-step working set ~5 GB (bases, 2F array) > 129 MB L2; L2 flushed before timing"}


def run_reference(args):
    """The FP64 oracle on the host cores: each step is the plain-C oracle on
    the 16-sky sample of the workunit (6.9e8 pairs), every core."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    w = workload(0, 1, args.n_sky)
    nproc = os.cpu_count() or 1
    _, dets, _, sub = baseline_sample(w)
    for _ in range(args.warmup):
        cpu_oracle_run(w, dets, sub, nproc)
    tot_pairs, tot_t = 0, 0.0
    for _ in range(args.steps):
        _, p, t, _ = cpu_oracle_run(w, dets, sub, nproc)
        tot_pairs += p
        tot_t += t
    v = tot_pairs / tot_t
    sample = (f"{sub.n_sky} sky (lattice points nearest the 8 signals, then the first) x {sub.n_f} f x "
              f"{sub.n_fdot} fdot x {w.n_sft_total} SFT per step, plain-C FP64 oracle")
    line = {"metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": shared_config(args),
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": min(nproc, sub.n_sky), "kind": "oracle",
                             "sample": sample, "nproc": nproc, "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_semicoherent(args):
    """Semicoherent search over the workunit: its SFTs split into time
    segments, each segment's coherent 2F at the segment's midpoint (bands
    padded for the slide), then the stack-slide sum over segments and the
    top-K of the sum, every step."""
    import torch
    import paper_0904_1826_gb300 as fs
    from workload import TemplateBank, DetectorData, Workload
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    w = workload(rank, world, args.n_sky)
    # signals added to the whole data set on the GPU (model-exact), read back
    full = fs.FStat(local_rank, topk=10, algo=args.algo)
    full.load_workload(w)
    full.inject(w.injections, w.bank.t_ref)
    bins = [fs.fstat_get_bins(full.ctx, i, d.n_sft, w.n_bins) for i, d in enumerate(w.detectors)]
    full.close()
    t_all = np.concatenate([d.t_start for d in w.detectors])
    t0, t1 = float(t_all.min()), float(t_all.max()) + w.T
    edges = t0 + (t1 - t0) * np.arange(args.n_seg + 1) / args.n_seg
    edges[-1] += 1.0
    bank, pad = w.bank, 8
    segs, seg_pairs, seg_bytes = [], 0, 0
    for s in range(args.n_seg):
        dets = []
        for i, d in enumerate(w.detectors):
            sel = (d.t_start >= edges[s]) & (d.t_start < edges[s + 1])
            dets.append(DetectorData(d.lat, d.lon, d.az, d.t_start[sel], bins[i][sel]))
        bs = TemplateBank(sky=bank.sky, f0=bank.f0 - pad * bank.df, df=bank.df, n_f=bank.n_f + 2 * pad,
                          fdot=bank.fdot, t_ref=0.5 * (edges[s] + edges[s + 1]))
        g = fs.FStat(local_rank, topk=10, algo=args.algo)
        g.load_workload(Workload(w.name, w.T, w.k_lo, w.n_bins, w.dterms, 10, dets, bs))
        segs.append(g)
        seg_pairs += bs.n_sky * bs.n_fdot * bs.n_f * sum(d.n_sft for d in dets)
        seg_bytes += 4 * bs.n_sky * bs.n_fdot * bs.n_f
    n_t = bank.n_sky * bank.n_fdot * bank.n_f
    out = torch.empty(n_t, dtype=torch.float32, device="cuda")
    k = w.topk
    idx = torch.empty(k, dtype=torch.int64, device="cuda")
    val = torch.empty(k, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    ctxs = [g.ctx for g in segs]
    ss = []

    def step(timed):
        for g in segs:
            g.compute(stream)
        if timed:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        fs.fstat_stackslide(ctxs, bank.f0, bank.df, bank.n_f, bank.t_ref, out, stream, want_outside=False)
        if timed:
            b.record(stream)
            ss.append((a, b))
        fs.fstat_toplist_noalloc(out, k, idx, val, stream)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    for g in segs:
        g.take_kernel_time()
    junk = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    junk.fill_(1)
    del junk
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    ss_ms = sum(a.elapsed_time(b) for a, b in ss) / args.steps
    k_dir = sum(g.take_kernel_time()[0] for g in segs)   # per step: each is a per-compute average
    n_outside = fs.fstat_stackslide(ctxs, bank.f0, bank.df, bank.n_f, bank.t_ref, out, stream)
    torch.cuda.synchronize()
    top_i, top_v = int(idx[0].item()), float(val[0].item())
    ss_bytes = seg_bytes + 4 * n_t
    peak_gbs = 6797.9
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak_gbs = float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        pass
    achieved = FLOP_PER_PAIR * seg_pairs / (k_dir / 1e3) / 1e12
    n_sm = int(torch.cuda.get_device_properties(local_rank).multi_processor_count)
    peak = n_sm * FP32_LANES * 2 * 2070.0 * 1e6 / 1e12
    line = {"metric": METRIC, "value": seg_pairs * args.steps / (ms / 1e3), "unit": "pairs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"semicoherent: the workunit's 2 det x 1200 SFTs in {args.n_seg} time segments, "
                                   f"coherent 2F per segment ({bank.n_sky} sky x {bank.n_f + 2 * pad} f x "
                                   f"{bank.n_fdot} fdot at the segment midpoint), stack-slide sum over segments, "
                                   f"top-{k} of the sum",
                       "n_seg": args.n_seg, "coherent_pairs_per_step": seg_pairs,
                       "semicoherent_templates": n_t},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "dirichlet (all segments)",
                         "dirichlet_ms": k_dir},
            "stackslide": {"ms_per_step": ss_ms, "bytes_per_step": ss_bytes,
                           "roofline": {"bound": "hbm", "achieved": ss_bytes / (ss_ms / 1e3) / 1e9,
                                        "peak": peak_gbs, "unit": "GB/s",
                                        "frac": ss_bytes / (ss_ms / 1e3) / 1e9 / peak_gbs, "traffic": None,
                                        "kernel": "stackslide_kernel"},
                           "n_outside": n_outside},
            "clocks": clocks, "top": {"sum_2F": top_v, "idx": top_i}}
    print(json.dumps(line))
    for g in segs:
        g.close()


def run_batch(args):
    """64 heterogeneous workunits (SFT counts 200-2400 over 1-2 detectors,
    bands 0.1-2 Hz, 100-20 000 sky points, 1-20 spindowns, 0-4 signals) in
    one persistent, CUDA-graph-captured launch, against one launch per
    workunit on the same data."""
    import torch
    import paper_0904_1826_gb300 as fs
    from workload import config3_specs, config3_workunit
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    specs = config3_specs(args.n_wu)
    ctx = fs.fstat_create(local_rank, dterms=8, topk=100, algo=args.algo)
    pairs = []
    t0 = time.perf_counter()
    for sp in specs:
        w = config3_workunit(sp)
        wid = fs.fstat_batch_add(ctx, w)
        if w.injections:
            fs.fstat_batch_inject(ctx, wid, w.injections, w.bank.t_ref)
        pairs.append(w.n_pairs)
        del w
    setup_s = time.perf_counter() - t0
    tuned = fs.fstat_autotune(ctx)
    stream = torch.cuda.Stream()
    for _ in range(max(args.warmup, 1)):
        fs.fstat_batch_compute(ctx, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        fs.fstat_batch_compute(ctx, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    done, total = fs.fstat_batch_get_times(ctx, len(specs))
    # one ordinary launch per workunit
    seq = []
    for i in range(len(specs)):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fs.fstat_batch_compute_one(ctx, i, stream)
        b.record(stream)
        torch.cuda.synchronize()
        seq.append(a.elapsed_time(b))
    total_pairs = float(sum(pairs))
    plans = [fs.fstat_batch_get_plan(ctx, i) for i in range(len(specs))]
    per_wu = [{"wu": i, "pairs": int(pairs[i]), "ms": float(seq[i]), "pairs_per_s": float(pairs[i] / (seq[i] / 1e3)),
               "n_sft": int(sp["n_sft_total"]), "n_det": int(sp["n_det"]), "n_f": max(1, int(round(sp["band"] * 1800))),
               "n_sky": int(sp["n_sky"]), "n_fdot": int(sp["n_fdot"]), "plan": plans[i]}
              for i, sp in enumerate(specs)]
    value = total_pairs * args.steps / (ms / 1e3)
    seq_value = total_pairs / (sum(seq) / 1e3)
    seq_cum = np.cumsum(seq)
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch of {len(specs)} heterogeneous workunits in one persistent "
                                   "CUDA-graph launch (SFTs 200-2400 over 1-2 det, bands 0.1-2 Hz, "
                                   "100-20000 sky, 1-20 fdot, 0-4 signals), D=8, top-100 each",
                       "pairs_per_step": total_pairs, "autotuned": tuned, "setup_s": setup_s},
            "one_launch_per_workunit": {"value": seq_value, "unit": "pairs/s", "ms_total": float(sum(seq)),
                                        "ms_per_wu_median": float(np.median(seq)), "ms_per_wu_max": float(max(seq))},
            "batch_latency_ms": {"median_wu_done": float(np.median(done)), "max_wu_done": float(max(done)),
                                 "graph_total": total},
            "sequential_latency_ms": {"median_wu_done": float(np.median(seq_cum)), "max_wu_done": float(seq_cum[-1])},
            "speedup_vs_one_launch_per_workunit": value / seq_value,
            "per_workunit": per_wu,
            "clocks": clocks}
    fs.fstat_destroy(ctx)
    print(json.dumps(line))


def run_proposal(args):
    """Learned proposal: coarse 2F maps of 2 det x 800 SFT workunits (64 x 32
    sky x 900 f), a 8192-256-256-1 network trained on the GPU on windows of
    the training maps (signals, and detector lines in the data), then two
    held-out sets of the same workunits -- without and with detector lines --
    where the network's best patches are refined on the 8x finer grid: recall
    against the exhaustive fine grid at refinement budgets of 1-16 patches for
    the network, the coarse-max ranking and random patches, and end-to-end
    device time against the exhaustive grid."""
    import torch
    from paper_0904_1826_gb300 import proposal as PR
    from workload import config4_workunit
    torch.cuda.set_device(0)
    search = PR.ProposalSearch(0, hidden=256, max_batch=1024)
    rng = np.random.default_rng(11)
    t0 = time.perf_counter()
    train = (config4_workunit(i, True, n_sft=args.proposal_sft, n_signals=8, n_lines=args.proposal_lines)
             for i in range(args.n_train))
    X, y = search.training_set(train, rng, 16, 256)
    t_set = time.perf_counter() - t0
    search.init_params(np.random.default_rng(1))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    hist = search.train(X, y, steps=args.train_steps, batch=256, lr=1e-4, pos_frac=0.25, seed=2)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    n_rows, n_pos = int(X.shape[0]), int(y.sum())
    del X
    sampler = ClockSampler(0)
    sampler.start()
    t1 = time.perf_counter()
    res = {}
    for name, nl in (("clean", 0), ("lines", args.proposal_lines)):
        test = [config4_workunit(i, False, n_sft=args.proposal_sft, n_lines=nl) for i in range(args.n_test)]
        res[name] = PR.evaluate(search, test, n_refine=args.n_refine, noise_patches_per_wu=24)
    t_eval = time.perf_counter() - t1
    test = [config4_workunit(i, False, n_sft=args.proposal_sft) for i in range(2)]
    ex_ms = [PR.exhaustive_ms(search, w) for w in test]
    clocks = sampler.stop()
    search.close()
    r0 = res["clean"]
    ms_learned = r0["ms_per_wu_learned"]
    ms_exh = float(np.mean(ex_ms))
    keys = ("recall_nn", "recall_coarse_max", "recall_random", "n_signal", "n_detected_exhaustive", "threshold",
            "n_noise_patches", "budgets", "curve", "n_low_rho", "curve_low_rho", "low_rho", "line_patches_in_top")
    line = {"metric": "learned-proposal device time per workunit vs exhaustive fine grid, at stated recall",
            "value": ms_exh / ms_learned, "unit": "x (speedup)", "n_gpus": 1, "steps": args.n_test, "warmup": 0,
            "ms_per_step": ms_learned, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 2F, bf16 network (fp32 accumulate)", "data": "synthetic",
            "config": {"workload": f"learned proposal: 2 det x {args.proposal_sft} SFTs, coarse 64x32 sky x 900 f "
                                   f"(0.5 Hz at 1/T), patches 16x16x32, fine grid 4x2 sky x 8 f per patch; "
                                   f"{args.n_train} training WUs (8 signals each or noise, 1-{args.proposal_lines} "
                                   f"detector lines), {args.n_test} held-out WUs (1 signal or noise) without and "
                                   f"with 1-{args.proposal_lines} detector lines, rho log-uniform 4-40, "
                                   f"{args.n_refine} of {r0['n_patches']} patches refined",
                       "network": "8192-256-256-1 ReLU, BF16 weights/activations, FP32 accumulate, Adam lr 1e-4, "
                                  f"batch 256, {args.train_steps} steps"},
            "recall": {k: r0[k] for k in keys},
            "recall_with_lines": {k: res["lines"][k] for k in keys},
            "ms_per_wu": {"learned_total": ms_learned, "coarse": r0["ms_coarse"], "network": r0["ms_mlp"],
                          "refine": r0["ms_refine"], "exhaustive_measured": ms_exh,
                          "exhaustive_from_patch_time": r0["ms_per_wu_exhaustive"]},
            "train": {"rows": n_rows, "positives": n_pos, "device_ms": train_ms, "loss_first": hist[0],
                      "loss_last": hist[-1], "set_s": t_set},
            "eval_wall_s": t_eval, "clocks": clocks}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config == "proposal":
        run_proposal(args)
        return
    if args.config == "batch":
        run_batch(args)
        return
    if args.config == "semicoherent":
        run_semicoherent(args)
        return
    import torch
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import paper_0904_1826_gb300 as fs
    from paper_0904_1826_gb300.multi import merge_toplists

    w = workload(rank, world, args.n_sky)
    n_pairs = w.n_pairs
    cov = None
    if args.coverage > 0:
        # a seeded fraction of the SFTs covers a random contiguous run of
        # 50-100 % of the frequencies; the others cover all of them
        rng = np.random.default_rng(4242 + rank)
        n_f = w.bank.n_f
        ragged = rng.random(w.n_sft_total) < args.coverage
        width = np.where(ragged, rng.integers(n_f // 2, n_f + 1, w.n_sft_total), n_f)
        lo = (rng.random(w.n_sft_total) * (n_f - width + 1)).astype(np.int64)
        cov = (lo.astype(np.int32), (lo + width).astype(np.int32))
        n_pairs = w.bank.n_sky * w.bank.n_fdot * int(width.sum())
    stream = torch.cuda.Stream()

    def make(form, kahan=False, algo=None, tiles=True):
        g = fs.FStat(local_rank, dterms=w.dterms, topk=w.topk, bins_form=form, kahan=kahan,
                     tile_m=args.tile_m if tiles else 0, tile_warps=args.tile_warps if tiles else 0,
                     sft_chunk=args.sft_chunk if tiles else 0, algo=args.algo if algo is None else algo)
        g.load_workload(w)
        g.inject(w.injections, w.bank.t_ref)
        if args.noise_floor:
            fs.fstat_set_noise_floor(g.ctx, args.noise_floor)
        if cov is not None:
            fs.fstat_set_coverage(g.ctx, *cov)
        return g

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    per_step = []   # per-step event times of the latest timed run (ms)

    def timed_run(g, steps, warmup, launch_mark=None):
        for _ in range(warmup):
            g.compute(stream)
        torch.cuda.synchronize()
        g.take_kernel_time()
        # flush L2 once before the timed region (each step then streams ~5 GB
        # of bases and 2F through it)
        junk = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        junk.fill_(1)
        del junk
        barrier()
        torch.cuda.synchronize()
        if launch_mark is not None:
            launch_mark[0] = g.launch_count()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for i in range(steps):
            g.compute(stream)
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = ev[0].elapsed_time(ev[-1])
        per_step.clear()
        per_step.extend(ev[i].elapsed_time(ev[i + 1]) for i in range(steps))
        kd, kt, nk = g.take_kernel_time()
        return ms, kd, kt, nk

    g = make(args.form)
    plan = g.plan()
    sampler = ClockSampler(local_rank)
    sampler.start()
    n_launch0 = [0]

    ms, k_dir, k_step, n_k = timed_run(g, args.steps, args.warmup, n_launch0)
    steps_ms = sorted(per_step)
    clocks = sampler.stop()
    launches = g.launch_count() - n_launch0[0]
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    # the exchange step: merge the local toplists
    idx, val = g.toplist(w.topk)
    if world > 1:
        sky_off = rank * args.n_sky * w.bank.n_fdot * w.bank.n_f
        local = torch.tensor(np.stack([idx + sky_off, val.view(np.int32).astype(np.int64)], 1), device="cuda")
        gathered = [torch.empty_like(local) for _ in range(world)]
        torch.distributed.all_gather(gathered, local)
        lists = [(x[:, 0].cpu().numpy(), x[:, 1].cpu().numpy().astype(np.int32).view(np.float32)) for x in gathered]
        idx, val = merge_toplists(lists, w.topk)
    value = n_pairs * world * args.steps / (ms / 1e3)

    # end to end through the public API with host buffers (pinned), per step:
    # SFT and template upload, compute, toplist download
    pinned = []
    for d in w.detectors:
        p = torch.empty((d.n_sft, w.n_bins, 2), dtype=torch.float32, pin_memory=True)
        p.numpy()[:] = d.bins.view(np.float32).reshape(d.n_sft, w.n_bins, 2)
        pinned.append(p)
    h2d = sum(p.numel() * 4 for p in pinned) + sum(d.n_sft * 8 for d in w.detectors) + \
        w.bank.sky.size * 8 + w.bank.fdot.size * 8
    d2h = w.topk * 12
    e2e_ms = []
    for it in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for i, d in enumerate(w.detectors):
            fs.fstat_set_sfts(g.ctx, i, d.lat, d.lon, d.az, w.T, w.k_lo, d.t_start,
                              pinned[i].numpy().view(np.complex64).reshape(d.n_sft, w.n_bins))
        if cov is not None:
            fs.fstat_set_coverage(g.ctx, *cov)
        g.set_bank(w.bank)
        g.compute(stream)
        g.toplist(w.topk)
        barrier()
        if it > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_ms_max = max(e2e_ms) if e2e_ms else float("nan")
    if world > 1 and e2e_ms:
        t = torch.tensor([e2e_ms_max], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms_max = float(t.item())
    e2e_value = n_pairs * world / (e2e_ms_max / 1e3) if e2e_ms else None

    forms = {}
    if args.compare_forms and rank == 0:
        for f, kahan, algo in (("c64", False, "auto"), ("c64", False, "farpoly"), ("c64", False, "direct"),
                               ("f16", False, "auto"),
                               ("bf16", False, "auto"), ("c64", True, "direct"), ("f16", True, "direct"),
                               ("bf16", True, "direct")):
            if (f, kahan, algo) == (args.form, False, args.algo):
                continue
            g2 = make(f, kahan, algo)
            ms2, kd2, _, _ = timed_run(g2, args.steps, 1)
            name = f + ("+kahan" if kahan else "") + ("" if kahan or algo == "auto" else "/" + algo)
            forms[name] = {"value": n_pairs * args.steps / (ms2 / 1e3), "dirichlet_ms": kd2,
                           "algo": algo_of(g2.plan()["variant"])}
            g2.close()

    # the plain FP32 form (direct Dirichlet sum, FP32 bins) on the same workunit
    plain = None
    if rank == 0 and world == 1 and algo_of(plan.get("variant", 0)) != "direct":
        g2 = make("c64", False, "direct", tiles=False)   # the planner's own tiles for the plain form
        ms2, kd2, _, _ = timed_run(g2, 2, 1)
        plain = {"value": n_pairs * 2 / (ms2 / 1e3), "unit": "pairs/s", "ms_per_step": ms2 / 2,
                 "dirichlet_ms": kd2, "algo": "direct", "steps": 2, "warmup": 1}
        g2.close()

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    props = torch.cuda.get_device_properties(local_rank)
    n_sm = int(props.multi_processor_count)
    clock_mhz = float(clocks["sm_max_mhz"]) if clocks and clocks.get("sm_max_mhz") else 2070.0
    peak = n_sm * FP32_LANES * 2 * clock_mhz * 1e6 / 1e12       # TFLOP/s, recipe unit counts, max clock
    achieved = FLOP_PER_PAIR * n_pairs / (k_dir / 1e3) / 1e12
    vid = plan.get("variant", 0)
    algo_used = algo_of(vid)
    kernel_name = KERNEL_NAMES[algo_used] if (vid < 107 or vid >= 120) else "dirichlet_far_ring_kernel"
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": ncu_traffic(args.form, algo_used), "kernel": kernel_name,
                "dirichlet_ms": k_dir, "step_ms_device": k_step,
                "peak_note": f"{n_sm} SM (queried) x {FP32_LANES} FP32 lanes x 2 flop x {clock_mhz:.0f} MHz "
                             "(maximum SM clock)"}
    if clocks and clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (n_sm * FP32_LANES * 2 * clocks["sm_mhz"] * 1e6 / 1e12)
    # the table forms are bound by shared-memory loads: that bound too, from the
    # ncu wavefront count per pair (128 B each) against 128 B per SM and clock
    ent = ncu_entry(args.form, algo_used)
    if ent and ent.get("smem_wavefronts_per_pair"):
        smem_b = ent["smem_wavefronts_per_pair"] * 128.0 * n_pairs
        smem_peak = n_sm * 128.0 * clock_mhz * 1e6 / 1e12       # TB/s
        roofline["shared_memory"] = {"achieved": smem_b / (k_dir / 1e3) / 1e12, "peak": smem_peak, "unit": "TB/s",
                                     "frac": smem_b / (k_dir / 1e3) / 1e12 / smem_peak,
                                     "bytes_per_pair": ent["smem_wavefronts_per_pair"] * 128.0}
    config = shared_config(args)
    config["pairs_per_step_per_gpu"] = n_pairs
    if args.noise_floor:
        config["noise_floor_half_window"] = args.noise_floor
    if args.coverage:
        config["coverage"] = args.coverage
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "step_ms": {"best": steps_ms[0], "median": steps_ms[len(steps_ms) // 2]} if steps_ms else None,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"c64": "f32", "f16": "f16-storage/f32", "bf16": "bf16-storage/f32"}[args.form],
            "data": "synthetic",
            "config": config,
            "kernel": {"algo": algo_used, "plan": plan},
            "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms_max},
            "roofline": roofline,
            "gpu_launches": launches,
            "clocks": clocks,
            "top": {"2F": float(val[0]), "idx": int(idx[0])}}
    if plain:
        plain["chosen_over_plain"] = value / plain["value"]
        line["plain_fp32"] = plain
    if forms:
        line["other_forms"] = forms

    def gpu_error(pick, bins, sub, ref):
        """The GPU's 2F on the CPU baseline's sample (the same bins, signals
        added by the oracle), chosen form and plain FP32 form, against the
        oracle's all-core run."""
        import dataclasses
        wl = dataclasses.replace(w, bank=sub)
        out = {}
        for name, form, algo, tiles in (("chosen", args.form, args.algo, True), ("plain_fp32", "c64", "direct", False)):
            g3 = fs.FStat(local_rank, dterms=w.dterms, topk=10, bins_form=form, algo=algo,
                          tile_m=args.tile_m if tiles else 0, tile_warps=args.tile_warps if tiles else 0,
                          sft_chunk=args.sft_chunk if tiles else 0)
            try:
                g3.load_workload(wl, bins_override=bins)
                g3.compute(stream)
                got = g3.twoF()
                st = twoF_error_stats(got, ref)
                st["variant"] = g3.plan()["variant"]
                out[name] = st
            finally:
                g3.close()
        return out

    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, gpu_error if not (args.coverage or args.noise_floor) else None)
        if "gpu_2F_error" in line["cpu_baseline"]:
            line["twoF_error"] = line["cpu_baseline"]["gpu_2F_error"]
    g.close()
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
