"""Sky sharding and the toplist merge through the library, on one GPU.

Two gloo ranks (processes) each compute their shard_range of the sky points
with libfstat on device 0 -- independent launches, no rank ever waits on
another's kernels -- all-gather their local toplists over gloo and merge
them with multi.merge_toplists, as bench.py's multi-GPU path does over NCCL.
The merged list must equal the single-process GPU toplist bit for bit and
pass the toplist check against the FP64 oracle.  Templates are independent
(Section "Implementation on the Cell": frequencies split equally over the
processing elements), so the shards' 2F equal the unsharded 2F exactly."""
import os
import socket

import numpy as np
import pytest

from oracle import fstat_oracle as O
from paper_0904_1826_gb300.multi import merge_toplists, shard_range

pytestmark = pytest.mark.gpu

K = 60


def _workload():
    from workload import config_mid
    w = config_mid(seed=505, n_sky=7, n_f=200, n_fdot=3)
    bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
    return w, bins


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import dataclasses
    import torch
    import torch.distributed as dist
    import paper_0904_1826_gb300 as fs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, bins = _workload()
        lo, hi = shard_range(w.bank.n_sky, rank, world)
        per_sky = w.bank.n_fdot * w.bank.n_f
        shard = dataclasses.replace(w, bank=dataclasses.replace(w.bank, sky=w.bank.sky[lo:hi]))
        g = fs.FStat(0, dterms=w.dterms, topk=K)
        try:
            g.load_workload(shard, bins_override=bins)
            g.compute()
            idx, val = g.toplist(K)
            plan = g.plan()["variant"]
        finally:
            g.close()
        local = torch.tensor(np.stack([idx + lo * per_sky, val.view(np.int32).astype(np.int64)], 1))
        got = [torch.empty_like(local) for _ in range(world)]
        dist.all_gather(got, local)
        lists = [(x[:, 0].numpy(), x[:, 1].numpy().astype(np.int32).view(np.float32)) for x in got]
        m_idx, m_val = merge_toplists(lists, K)
        if rank == 0:
            q.put((m_idx.tolist(), m_val.tolist(), plan))
    finally:
        dist.destroy_process_group()


def test_two_rank_sky_shards_merge_to_the_single_gpu_toplist(lib):
    import multiprocessing as mp
    from tests.test_gpu_parity import _check_toplist
    w, bins = _workload()
    g = lib.FStat(0, dterms=w.dterms, topk=K)
    try:
        g.load_workload(w, bins_override=bins)
        g.compute()
        s_idx, s_val = g.toplist(K)
        allv = g.twoF()
        plan = g.plan()["variant"]
    finally:
        g.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    m_idx, m_val, m_plan = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert m_plan == plan
    np.testing.assert_array_equal(np.array(m_idx, np.int64), s_idx)
    np.testing.assert_array_equal(np.array(m_val, np.float32), s_val)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    _check_toplist((s_idx, s_val), allv, ref, K)


def _dets(w, bins):
    from workload import DetectorData
    return [DetectorData(d.lat, d.lon, d.az, d.t_start, b) for d, b in zip(w.detectors, bins)]
