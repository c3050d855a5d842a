"""Write the FP64 oracle's top templates of whole workunits of the
heterogeneous batch (``workload.config3_specs(64)``), for the batch parity
test.  Each listed workunit is generated at full size, its signals added by
the FP64 oracle (model-exact injection), and every template computed by the
plain-C FP64 oracle (the loop nest of Listing 1, Section "Einstein@Home").
Nothing here touches the GPU library.

Output: ``batch_wu<i>_top.txt`` next to this script, the first 120 templates
in (2F descending, template index ascending) order, with the number of
templates, the FP64 mean of 2F and each sky point's maximum 2F in the header
lines (the maxima as one line of numbers).

Usage: python tests/golden/make_batch_toplists.py [--threads N] [--wu 33 31 14]
"""
from __future__ import annotations

import argparse
import dataclasses
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import c_oracle as CO  # noqa: E402
from oracle import fstat_oracle as O  # noqa: E402
from workload import config3_specs, config3_workunit  # noqa: E402

N_KEEP = 120


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--wu", type=int, nargs="+", default=[33, 31, 14])
    args = ap.parse_args()
    specs = config3_specs(64)
    for i in args.wu:
        t0 = time.time()
        w = config3_workunit(specs[i])
        bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
        dets = [dataclasses.replace(d, bins=b) for d, b in zip(w.detectors, bins)]
        b = w.bank
        r = CO.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, b, threads=args.threads)
        flat = r.reshape(b.n_sky, -1)
        v = flat.ravel()
        cand = np.argpartition(-v, min(N_KEEP, v.size - 1))[:N_KEEP]
        o = np.lexsort((cand, -v[cand]))
        top_i, top_v = cand[o].astype(np.int64), v[cand[o]]
        ref = O.compute_fstat_templates(dets, w.T, w.k_lo, w.dterms, b, top_i)
        rel = float(np.max(np.abs(ref - top_v) / np.maximum(np.abs(ref), 1.0)))
        if rel > 1e-6:
            raise SystemExit(f"workunit {i}: the two FP64 oracles disagree ({rel:.3e})")
        with open(os.path.join(HERE, f"batch_wu{i}_top.txt"), "w") as fh:
            fh.write(f"# FP64 oracle (plain C), whole workunit {i} of workload.config3_specs(64): "
                     f"{w.n_sft_total} SFT over {len(w.detectors)} det, {b.n_sky} sky x {b.n_f} f x {b.n_fdot} fdot,\n")
            fh.write("# signals injected by oracle.fstat_oracle.inject.  Written by tests/golden/make_batch_toplists.py.\n")
            fh.write(f"# n_templates {v.size}\n")
            fh.write(f"# mean_2F {float(v.mean()):.12e}\n")
            fh.write(f"# numpy_vs_c_max_rel {rel:.3e}\n")
            fh.write("# sky_max " + " ".join(f"{x:.7e}" for x in flat.max(axis=1)) + "\n")
            fh.write("# rank template_index 2F  (2F descending, index ascending)\n")
            for k, (ii, vv) in enumerate(zip(top_i, top_v)):
                fh.write(f"{k} {int(ii)} {vv:.10e}\n")
        print(f"workunit {i}: {w.n_pairs:.3e} pairs in {time.time() - t0:.0f} s, top {top_v[0]:.2f}", flush=True)


if __name__ == "__main__":
    main()
