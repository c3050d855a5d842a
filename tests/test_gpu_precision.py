"""Precision forms on workunit-sized data: 2 detectors x 1200 gapped SFTs,
1816 bins at 100 Hz with 8 signals, templates 1800 f x 10 fdot at the sky
positions of four of the signals (72 000 templates, 1.7e8 pairs).  Every form
is compared with the FP64 oracle template by template: max and 99th
percentile of |d2F|, the share within the FP32 tolerance, and the overlap of
its top-1000 with the oracle's top-1000.  The FP32 forms must meet the
element-wise tolerance; the 16-bit forms must stay at their format's level.
Set FSTAT_PRECISION_OUT to a path to keep the table as JSON."""
import dataclasses
import json
import multiprocessing as mp
import os

import numpy as np
import pytest

from workload import TemplateBank, config1

pytestmark = pytest.mark.gpu

REL, ABS = 1e-4, 1e-3
N_SKY = 4


def _oracle_sky(args):
    """FP64 2F of one sky point's 10 x 1800 templates (run in a spawned worker)."""
    from oracle import fstat_oracle as O
    dets, T, k_lo, dterms, bank = args
    return O.compute_fstat_freq_band(dets, T, k_lo, dterms, bank, [0])[0]


@pytest.fixture(scope="module")
def case():
    from oracle import fstat_oracle as O
    w = config1()
    bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
    dets = [dataclasses.replace(d, bins=b) for d, b in zip(w.detectors, bins)]
    sky = np.array([[inj.alpha, inj.delta] for inj in w.injections[:N_SKY]])
    bank = TemplateBank(sky=sky, f0=w.bank.f0, df=w.bank.df, n_f=w.bank.n_f, fdot=w.bank.fdot, t_ref=w.bank.t_ref)
    jobs = [(dets, w.T, w.k_lo, w.dterms, dataclasses.replace(bank, sky=sky[i:i + 1])) for i in range(N_SKY)]
    with mp.get_context("spawn").Pool(N_SKY) as pool:
        ref = np.stack(pool.map(_oracle_sky, jobs))       # [sky][fdot][f]
    w = dataclasses.replace(w, bank=bank)
    return w, bins, ref.ravel()


FORMS = [("c64", False, "sincpoly"), ("c64", False, "farpoly"), ("c64", False, "direct"), ("c64", True, "direct"),
         ("f16", False, "sincpoly"), ("f16", False, "farpoly"), ("f16", True, "direct"),
         ("bf16", False, "sincpoly"), ("bf16", False, "farpoly"), ("bf16", True, "direct")]


def test_precision_forms_on_workunit_data(lib, case):
    w, bins, ref = case
    top_ref = set(np.lexsort((np.arange(ref.size), -ref))[:1000].tolist())
    rows = []
    for form, kahan, algo in FORMS:
        g = lib.FStat(0, dterms=w.dterms, topk=1000, bins_form=form, kahan=kahan, algo=algo)
        try:
            g.load_workload(w, bins_override=bins)
            g.compute()
            got = g.twoF().astype(np.float64)
            assert g.error_flags() == 0
        finally:
            g.close()
        err = np.abs(got - ref)
        top = set(np.lexsort((np.arange(got.size), -got))[:1000].tolist())
        rows.append(dict(form=form, kahan=kahan, algo=algo, max_abs=float(err.max()),
                         p99_abs=float(np.percentile(err, 99)),
                         max_rel=float(np.max(err / (ref + 1.0))),
                         within_tol=float(np.mean(err <= REL * ref + ABS)),
                         top1000_overlap=len(top & top_ref)))
    out = os.environ.get("FSTAT_PRECISION_OUT")
    if out:
        with open(out, "w") as fh:
            json.dump(dict(templates=int(ref.size), pairs=int(ref.size) * w.n_sft_total, max_2F=float(ref.max()),
                           forms=rows), fh, indent=1)
    for r in rows:
        if r["form"] == "c64":
            assert r["within_tol"] == 1.0, r
            assert r["top1000_overlap"] >= 990, r
        elif r["form"] == "f16":
            assert r["max_rel"] < 5e-3 and r["top1000_overlap"] >= 990, r
        else:
            assert r["max_rel"] < 4e-2 and r["top1000_overlap"] >= 980, r


def test_precision_forms_on_the_whole_workunit(lib):
    """Every form on the whole workunit (1.8e8 templates, the bench's bank),
    against the FP64 oracle's run over all of it (tests/golden/): overlap of
    the form's top-1000 with the oracle's top-1000, and |d2F| at the oracle's
    first 1200 templates and at every sky point's maximum.  The FP32 form
    keeps the toplist up to near-ties; the 16-bit forms stay at their
    format's level."""
    from tests.test_gpu_fullsize import _read_golden
    from oracle import fstat_oracle as O
    head, g_idx, g_val, sky_max = _read_golden()
    w = config1()
    bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
    top_ref = set(g_idx[:1000].tolist())
    rows = []
    for form, kahan, algo in (("c64", False, "auto"), ("c64", True, "direct"), ("f16", False, "auto"),
                              ("bf16", False, "auto")):
        g = lib.FStat(0, dterms=w.dterms, topk=1000, bins_form=form, kahan=kahan, algo=algo)
        try:
            g.load_workload(w, bins_override=bins)
            g.compute()
            assert g.error_flags() == 0
            idx, _ = g.toplist(1000)
            allv = g.twoF()
        finally:
            g.close()
        e_top = np.abs(allv[g_idx].astype(np.float64) - g_val)
        smax = allv.reshape(w.bank.n_sky, -1).max(axis=1).astype(np.float64)
        e_sky = np.abs(smax - sky_max)
        rows.append(dict(form=form, kahan=kahan, algo=algo, top1000_overlap=len(set(idx.tolist()) & top_ref),
                         max_abs_top=float(e_top.max()), p99_abs_top=float(np.percentile(e_top, 99)),
                         max_rel_top=float(np.max(e_top / (g_val + 1.0))), max_abs_skymax=float(e_sky.max()),
                         p99_abs_skymax=float(np.percentile(e_sky, 99))))
    out = os.environ.get("FSTAT_PRECISION_OUT")
    if out:
        with open(out.replace(".json", "_whole.json"), "w") as fh:
            json.dump(dict(templates=int(head["n_templates"]), forms=rows), fh, indent=1)
    for r in rows:
        print(r)
        if r["form"] == "c64":
            assert r["top1000_overlap"] >= 990 and r["max_abs_top"] <= REL * g_val.max() + ABS, r
        elif r["form"] == "f16":
            assert r["top1000_overlap"] >= 950 and r["max_rel_top"] < 5e-3, r
        else:
            assert r["top1000_overlap"] >= 800 and r["max_rel_top"] < 4e-2, r
