"""The toplist call without device allocation (include/fstat_noalloc.h)
against the context's toplist on the same 2F map, two calls in a row.  The
file name sorts last so that the call also runs after every other test has
used the library in the same process."""
import numpy as np
import pytest

from workload import config_mid

pytestmark = pytest.mark.gpu


def _context_toplist(lib, k):
    w = config_mid(seed=71, n_bins=360, n_sky=40, n_f=300, n_fdot=3)
    g = lib.FStat(0, topk=k)
    g.load_workload(w)
    g.compute()
    idx, val = g.toplist(k)
    twoF = g.twoF()
    g.close()
    return twoF, idx, val


def test_noalloc_toplist_matches_context_toplist_twice(lib):
    import torch
    k = 1000
    twoF, idx, val = _context_toplist(lib, k)
    v = torch.from_numpy(twoF).cuda()
    s = torch.cuda.Stream()
    for _ in range(2):
        io = torch.full((k,), -1, dtype=torch.int64, device="cuda")
        vo = torch.full((k,), -1.0, dtype=torch.float32, device="cuda")
        lib.fstat_toplist_noalloc(v, k, io, vo, stream=s)
        s.synchronize()
        np.testing.assert_array_equal(io.cpu().numpy(), idx)
        np.testing.assert_array_equal(vo.cpu().numpy(), val)


def test_noalloc_toplist_ties_and_limits(lib):
    import torch
    rng = np.random.default_rng(8)
    x = rng.integers(0, 50, 300_001).astype(np.float32)     # many equal values
    v = torch.from_numpy(x).cuda()
    k = lib.NOALLOC_MAX_K
    io = torch.empty(k, dtype=torch.int64, device="cuda")
    vo = torch.empty(k, dtype=torch.float32, device="cuda")
    order = np.lexsort((np.arange(x.size), -x))[:k]
    for _ in range(2):
        lib.fstat_toplist_noalloc(v, k, io, vo)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(io.cpu().numpy(), order)
        np.testing.assert_array_equal(vo.cpu().numpy(), x[order])
    with pytest.raises(lib.FstatError, match="ERANGE.*static scratch limit"):
        lib.fstat_toplist_noalloc(v, k + 1, io, vo)
    with pytest.raises(lib.FstatError, match="EINVAL"):
        lib.fstat_toplist_noalloc(v[:5], 6, io, vo)


def test_noalloc_toplist_on_views_at_any_offset(lib):
    """v may be a view starting at any element: the first values before the
    16-byte boundary are ranked like the rest."""
    import torch
    rng = np.random.default_rng(12)
    base = rng.random(200_003).astype(np.float32) * 100.0
    vb = torch.from_numpy(base).cuda()
    for off in (1, 2, 3, 5):
        for n in (1, 2, 3, 7, 4099, base.size - off):
            x = base[off:off + n]
            k = min(n, 50)
            io = torch.empty(k, dtype=torch.int64, device="cuda")
            vo = torch.empty(k, dtype=torch.float32, device="cuda")
            lib.fstat_toplist_noalloc(vb[off:off + n], k, io, vo)
            torch.cuda.synchronize()
            order = np.lexsort((np.arange(n), -x))[:k]
            np.testing.assert_array_equal(io.cpu().numpy(), order)
            np.testing.assert_array_equal(vo.cpu().numpy(), x[order])


def test_noalloc_toplist_negative_zero_ranks_as_zero(lib):
    import torch
    x = np.zeros(4096, dtype=np.float32)
    x[::3] = -0.0
    x[100] = 2.0
    x[7] = 1.0
    v = torch.from_numpy(x).cuda()
    k = 10
    io = torch.empty(k, dtype=torch.int64, device="cuda")
    vo = torch.empty(k, dtype=torch.float32, device="cuda")
    lib.fstat_toplist_noalloc(v, k, io, vo)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(io.cpu().numpy(), [100, 7, 0, 1, 2, 3, 4, 5, 6, 8])
    got = vo.cpu().numpy()
    np.testing.assert_array_equal(got, [2.0, 1.0] + [0.0] * 8)
    assert not np.any(np.signbit(got))


def test_noalloc_toplist_refuses_misaligned_outputs(lib):
    """Refused on the host, before any launch."""
    import torch
    v = torch.rand(1000, device="cuda")
    k = 10
    raw = torch.empty(8 * k + 16, dtype=torch.uint8, device="cuda")
    vo = torch.empty(k, dtype=torch.float32, device="cuda")
    io = torch.empty(k, dtype=torch.int64, device="cuda")
    with pytest.raises(lib.FstatError, match="EINVAL.*misaligned"):
        lib.fstat_toplist_noalloc(v, k, raw[4:], vo)
    with pytest.raises(lib.FstatError, match="EINVAL.*misaligned"):
        lib.fstat_toplist_noalloc(v, k, io, raw[2:])
