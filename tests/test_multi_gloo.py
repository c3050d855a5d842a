"""Multi-GPU host logic on CPU: sky sharding and the toplist exchange, with
two gloo ranks standing in for two GPUs (the per-rank 2F comes from the
oracle here; on GPUs each rank runs the library on its shard)."""
import os
import socket

import numpy as np
import pytest

from paper_0904_1826_gb300.multi import merge_toplists, shard_range


def test_shard_range_partitions():
    for n in (1, 7, 10, 10000):
        for w in (1, 2, 3, 8):
            parts = [shard_range(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(w - 1))
            assert max(b - a for a, b in parts) - min(b - a for a, b in parts) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from oracle import fstat_oracle as O
    from workload import config_mid
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = config_mid(n_sky=5, n_f=40, n_fdot=2)
    lo, hi = shard_range(w.bank.n_sky, rank, world)
    per_sky = w.bank.n_fdot * w.bank.n_f
    twoF = O.compute_fstat_freq_band(w.detectors, w.T, w.k_lo, w.dterms, w.bank, range(lo, hi)).ravel()
    idx, val = O.toplist(twoF, 25)
    local = torch.tensor(np.stack([idx + lo * per_sky, val.astype(np.float32).view(np.int32).astype(np.int64)], 1))
    got = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(got, local)
    lists = [(x[:, 0].numpy(), x[:, 1].numpy().astype(np.int32).view(np.float32)) for x in got]
    m_idx, m_val = merge_toplists(lists, 25)
    if rank == 0:
        full = O.compute_fstat_freq_band(w.detectors, w.T, w.k_lo, w.dterms, w.bank).ravel().astype(np.float32)
        r_idx, r_val = O.toplist(full, 25)
        q.put((m_idx.tolist(), r_idx.tolist(), m_val.tolist(), r_val.tolist()))
    dist.destroy_process_group()


@pytest.mark.slow
def test_two_rank_toplist_exchange_matches_single_process():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    m_idx, r_idx, m_val, r_val = res
    assert m_idx == r_idx
    assert np.allclose(m_val, r_val)
