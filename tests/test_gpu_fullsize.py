"""The full workunit in the bench's launch configuration (10 000 sky x 1800 f
x 10 fdot x 2400 SFTs, default form and tiles) against the FP64 oracle on
sampled templates, computed one by one: random templates over the whole
bank, the last frequency column (ragged tile tail), the last sky points, and
the top of the toplist.  The toplist must also be ordered and exact on the
GPU's own values.  With coverage the same sampling applies."""
import dataclasses
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import fstat_oracle as O
from workload import TemplateBank, config1

pytestmark = pytest.mark.gpu

REL, ABS = 1e-4, 1e-3


_W = {}   # the workload held by each oracle worker (sent once, at start-up)


def _init(dets, T, k_lo, dterms):
    _W.update(dets=dets, T=T, k_lo=k_lo, dterms=dterms)


def _plain_job(args):
    from oracle import fstat_oracle as O_
    bank, idx = args
    return O_.compute_fstat_templates(_W["dets"], _W["T"], _W["k_lo"], _W["dterms"], bank, idx)


def _coverage_job(args):
    from oracle import coverage_oracle as CO_
    one, lo, hi = args
    return CO_.compute_fstat_coverage(_W["dets"], _W["T"], _W["k_lo"], _W["dterms"], one, lo, hi)[0, 0, 0]


def _pool_map(fn, jobs, w, dets):
    n = min(len(jobs), os.cpu_count() or 4)
    with mp.get_context("spawn").Pool(n, initializer=_init, initargs=(dets, w.T, w.k_lo, w.dterms)) as pool:
        return pool.map(fn, jobs)


@pytest.fixture(scope="module")
def full():
    w = config1()
    bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
    dets = [dataclasses.replace(d, bins=b) for d, b in zip(w.detectors, bins)]
    return w, bins, dets


def _samples(w, top_idx, rng):
    b = w.bank
    n = b.n_sky * b.n_fdot * b.n_f
    rand = rng.integers(0, n, 120)
    last_col = ((rng.integers(0, b.n_sky, 20) * b.n_fdot + rng.integers(0, b.n_fdot, 20)) * b.n_f
                + rng.integers(b.n_f - 40, b.n_f, 20))
    last_sky = ((b.n_sky - 1 - rng.integers(0, 3, 20)) * b.n_fdot + rng.integers(0, b.n_fdot, 20)) * b.n_f \
        + rng.integers(0, b.n_f, 20)
    return np.unique(np.concatenate([rand, last_col, last_sky, top_idx[:20]]))


def test_full_workunit_sampled_against_oracle(lib, full):
    w, bins, dets = full
    g = lib.FStat(0, topk=w.topk)
    try:
        g.load_workload(w, bins_override=bins)
        g.compute()
        assert g.error_flags() == 0
        assert g.plan()["variant"] == 112            # the default sinc ring kernel, as benched
        idx, val = g.toplist(w.topk)
        assert np.all(np.diff(val) <= 0)
        sel = _samples(w, idx, np.random.default_rng(5))
        got = np.concatenate([g.twoF(int(i), 1) for i in sel]).astype(np.float64)
        # toplist values are the 2F array's own
        np.testing.assert_array_equal(np.concatenate([g.twoF(int(i), 1) for i in idx[:20]]), val[:20])
    finally:
        g.close()
    chunks = np.array_split(sel, min(len(sel), os.cpu_count() or 4))
    ref = np.concatenate(_pool_map(_plain_job, [(w.bank, c) for c in chunks], w, dets))
    assert np.all(np.abs(got - ref) <= REL * ref + ABS), np.max(np.abs(got - ref) - REL * ref)
    assert ref.max() > 30          # the sample holds the injected signals' peaks


def test_full_workunit_sampled_with_coverage(lib, full):
    w, bins, dets = full
    rng = np.random.default_rng(9)
    n = w.n_sft_total
    ragged = rng.random(n) < 0.1
    width = np.where(ragged, rng.integers(w.bank.n_f // 2, w.bank.n_f + 1, n), w.bank.n_f)
    lo = (rng.random(n) * (w.bank.n_f - width + 1)).astype(np.int32)
    hi = (lo + width).astype(np.int32)
    g = lib.FStat(0, topk=w.topk)
    try:
        g.load_workload(w, bins_override=bins)
        lib.fstat_set_coverage(g.ctx, lo, hi)
        g.compute()
        assert g.error_flags() == 0
        idx, _ = g.toplist(w.topk)
        sel = _samples(w, idx, np.random.default_rng(6))[:96]
        got = np.concatenate([g.twoF(int(i), 1) for i in sel]).astype(np.float64)
    finally:
        g.close()
    # the oracle template by template: a one-template bank at the sampled
    # frequency, its coverage shifted to that frequency index
    b = w.bank
    jobs = []
    for t in sel:
        s, rem = divmod(int(t), b.n_fdot * b.n_f)
        m, j = divmod(rem, b.n_f)
        one = TemplateBank(sky=b.sky[s:s + 1], f0=b.f0 + j * b.df, df=b.df, n_f=1, fdot=b.fdot[m:m + 1],
                           t_ref=b.t_ref)
        jobs.append((one, lo - j, hi - j))
    ref = np.array(_pool_map(_coverage_job, jobs, w, dets))
    assert np.all(np.abs(got - ref) <= REL * ref + ABS), np.max(np.abs(got - ref) - REL * ref)
