"""Write the FP64 oracle's results for the whole workunit-sized case.

The case: 2 detectors x 1200 gapped SFTs, 1 Hz band at 100 Hz with 8 signals
added by the FP64 oracle (model-exact injection), templates 10 000 Fibonacci
sky points x 1800 frequencies x 10 spindowns, Dterms = 8 (the seeded
``workload.config1()``).  Every one of the 1.8e8 templates is computed by the
plain-C FP64 oracle (the loop nest of Listing 1, Section "Einstein@Home"),
sky points spread over the host's threads.  Nothing here touches the GPU
library.

Outputs (text, next to this script):
  * ``config1_top.txt``: the first 1200 templates in (2F descending, template
    index ascending) order, each re-computed by the numpy oracle as a
    cross-check (the two FP64 oracles must agree to 1e-6 relative);
  * ``config1_sky_max.txt``: the maximum 2F of each sky point (10 000 lines);
  * the header of ``config1_top.txt`` also holds the number of templates
    above fixed 2F thresholds and the FP64 mean of 2F over the whole bank.

Usage: python tests/golden/make_config1_toplist.py [--threads N] [--checkpoint PATH]
(about 4 s of one core per sky point: 1-3 hours on a few cores).
"""
from __future__ import annotations

import argparse
import dataclasses
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import c_oracle as CO  # noqa: E402
from oracle import fstat_oracle as O  # noqa: E402
from workload import TemplateBank, config1  # noqa: E402

N_KEEP = 1200
THRESHOLDS = (8.0, 12.0, 16.0, 20.0, 25.0, 30.0, 40.0, 60.0, 100.0, 200.0, 400.0)


def _merge(cur_idx, cur_val, idx, val, n):
    i = np.concatenate([cur_idx, idx])
    v = np.concatenate([cur_val, val])
    o = np.lexsort((i, -v))[:n]
    return i[o], v[o]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--chunk", type=int, default=56, help="sky points per batch of work")
    ap.add_argument("--checkpoint", default=None, help="npz file to resume from / save to")
    args = ap.parse_args()

    w = config1()
    bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
    dets = [dataclasses.replace(d, bins=b) for d, b in zip(w.detectors, bins)]
    b = w.bank
    per_sky = b.n_fdot * b.n_f

    top_idx = np.zeros(0, np.int64)
    top_val = np.zeros(0, np.float64)
    sky_max = np.full(b.n_sky, np.nan)
    counts = np.zeros(len(THRESHOLDS), np.int64)
    total = 0.0
    start = 0
    if args.checkpoint and os.path.exists(args.checkpoint):
        z = np.load(args.checkpoint)
        top_idx, top_val, sky_max = z["top_idx"], z["top_val"], z["sky_max"]
        counts, total, start = z["counts"], float(z["total"]), int(z["next"])
        print(f"resuming at sky point {start}", flush=True)

    t0 = time.time()
    for s0 in range(start, b.n_sky, args.chunk):
        s1 = min(b.n_sky, s0 + args.chunk)
        r = CO.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, b, sky_indices=range(s0, s1),
                                       threads=args.threads)
        flat = r.reshape(s1 - s0, per_sky)
        sky_max[s0:s1] = flat.max(axis=1)
        v = flat.ravel()
        counts += np.array([(v > t).sum() for t in THRESHOLDS], dtype=np.int64)
        total += float(v.sum())
        cand = np.argpartition(-v, min(N_KEEP, v.size - 1))[:N_KEEP]
        top_idx, top_val = _merge(top_idx, top_val, cand.astype(np.int64) + s0 * per_sky, v[cand], N_KEEP)
        if args.checkpoint:
            np.savez(args.checkpoint, top_idx=top_idx, top_val=top_val, sky_max=sky_max, counts=counts,
                     total=total, next=s1)
        el = time.time() - t0
        done = s1 - start
        print(f"sky {s1}/{b.n_sky}  {el:.0f} s  eta {el / done * (b.n_sky - s1):.0f} s  "
              f"top {top_val[0]:.2f} k-th {top_val[min(999, top_val.size - 1)]:.3f}", flush=True)

    # cross-check the kept templates with the numpy oracle
    ref = O.compute_fstat_templates(dets, w.T, w.k_lo, w.dterms, b, top_idx)
    rel = np.max(np.abs(ref - top_val) / np.maximum(np.abs(ref), 1.0))
    print(f"numpy oracle vs C oracle on the kept templates: max rel {rel:.3e}", flush=True)
    if rel > 1e-6:
        raise SystemExit("the two FP64 oracles disagree")

    n_t = b.n_sky * per_sky
    with open(os.path.join(HERE, "config1_top.txt"), "w") as fh:
        fh.write("# FP64 oracle (plain C, loop nest of Listing 1, Section \"Einstein@Home\"), whole bank of\n")
        fh.write("# workload.config1(): 2 det x 1200 SFT, 10000 sky x 1800 f x 10 fdot, Dterms 8, signals\n")
        fh.write("# injected by oracle.fstat_oracle.inject.  Written by tests/golden/make_config1_toplist.py.\n")
        fh.write(f"# n_templates {n_t}\n")
        fh.write(f"# mean_2F {total / n_t:.12e}\n")
        fh.write("# count_above " + " ".join(f"{t:g}:{c}" for t, c in zip(THRESHOLDS, counts)) + "\n")
        fh.write(f"# numpy_vs_c_max_rel {rel:.3e}\n")
        fh.write("# rank template_index 2F  (2F descending, index ascending)\n")
        for k, (i, v) in enumerate(zip(top_idx, top_val)):
            fh.write(f"{k} {int(i)} {v:.10e}\n")
    with open(os.path.join(HERE, "config1_sky_max.txt"), "w") as fh:
        fh.write("# maximum 2F over 1800 f x 10 fdot of each sky point of workload.config1(), FP64 oracle;\n")
        fh.write("# written by tests/golden/make_config1_toplist.py\n")
        for v in sky_max:
            fh.write(f"{v:.7e}\n")
    print("done", time.time() - t0, flush=True)


if __name__ == "__main__":
    main()
