"""Python binding of libfstat, the GB300 coherent F-statistic library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libfstat.so (built in-tree by ``build.py``).  Importing this
module fails loudly if the library has not been built; there is no CPU
fallback.  Functions carry the names of the C calls in include/fstat.h.

Host arrays are numpy arrays; device arrays may be passed as torch CUDA
tensors (their data pointer is handed to the library with FSTAT_MEM_DEVICE).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfstat.so")

FSTAT_OK, FSTAT_EINVAL, FSTAT_ENOMEM, FSTAT_ECUDA, FSTAT_ESTATE, FSTAT_ERANGE, FSTAT_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
FSTAT_BINS_C64, FSTAT_BINS_F16, FSTAT_BINS_BF16 = 0, 1, 2
FSTAT_MEM_HOST, FSTAT_MEM_DEVICE = 0, 1
FORMS = {"c64": FSTAT_BINS_C64, "f16": FSTAT_BINS_F16, "bf16": FSTAT_BINS_BF16}
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ESTATE", -5: "ERANGE", -6: "ETIMEOUT"}


class FstatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class fstat_opts(ctypes.Structure):
    _fields_ = [("dterms", ctypes.c_int32), ("bins_form", ctypes.c_int32), ("topk", ctypes.c_int32),
                ("kahan", ctypes.c_int32), ("tile_m", ctypes.c_int32), ("tile_warps", ctypes.c_int32),
                ("sft_chunk", ctypes.c_int32), ("algo", ctypes.c_int32)]


class fstat_detector(ctypes.Structure):
    _fields_ = [("lat_rad", ctypes.c_double), ("lon_rad", ctypes.c_double), ("xarm_az_rad", ctypes.c_double)]


class fstat_signal(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("alpha", "delta", "psi", "cosi", "phi0", "f", "fdot", "rho")]


class fstat_workunit(ctypes.Structure):
    _fields_ = [("n_det", ctypes.c_int32), ("det", ctypes.POINTER(fstat_detector)),
                ("n_sft", ctypes.POINTER(ctypes.c_int32)), ("t_start", ctypes.POINTER(ctypes.c_void_p)),
                ("bins", ctypes.POINTER(ctypes.c_void_p)), ("Tsft", ctypes.c_double), ("k_lo", ctypes.c_int64),
                ("n_bins", ctypes.c_int32), ("sky", ctypes.c_void_p), ("n_sky", ctypes.c_int32),
                ("f0", ctypes.c_double), ("df", ctypes.c_double), ("n_f", ctypes.c_int32),
                ("fdot", ctypes.c_void_p), ("n_fdot", ctypes.c_int32), ("t_ref", ctypes.c_double)]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double

# name -> (restype, argtypes); the full C ABI of include/fstat.h
SIGNATURES = {
    "fstat_version": (ctypes.c_char_p, []),
    "fstat_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(fstat_opts)]),
    "fstat_destroy": (None, [_P]),
    "fstat_last_error": (ctypes.c_char_p, [_P]),
    "fstat_set_sfts": (ctypes.c_int, [_P, _I32, ctypes.POINTER(fstat_detector), _D, _I64, _I32, _I32, _P, _P, _I32]),
    "fstat_set_templates": (ctypes.c_int, [_P, _P, _I32, _D, _D, _I32, _P, _I32, _D]),
    "fstat_compute": (ctypes.c_int, [_P, _P]),
    "fstat_get_2f": (ctypes.c_int, [_P, _P, _I64, _I64, _I32]),
    "fstat_get_toplist": (ctypes.c_int, [_P, _I32, _P, _P]),
    "fstat_get_abcd": (ctypes.c_int, [_P, _P]),
    "fstat_get_sft_timing": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P]),
    "fstat_inject": (ctypes.c_int, [_P, ctypes.POINTER(fstat_signal), _I32, _D]),
    "fstat_get_bins": (ctypes.c_int, [_P, _I32, _P, _I32]),
    "fstat_get_error_flags": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "fstat_get_plan": (ctypes.c_int, [_P, _P]),
    "fstat_test_ring_stall": (ctypes.c_int, [_P, _I32]),
    "fstat_set_noise_floor": (ctypes.c_int, [_P, _I32]),
    "fstat_set_coverage": (ctypes.c_int, [_P, _P, _P, _I32]),
    "fstat_get_noise": (ctypes.c_int, [_P, _P, _P, _I32]),
    "fstat_get_launch_count": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "fstat_take_kernel_time": (ctypes.c_int, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I32)]),
    "fstat_autotune": (ctypes.c_int, [_P, _P, _P]),
    "fstat_batch_add": (ctypes.c_int, [_P, ctypes.POINTER(fstat_workunit), ctypes.POINTER(_I32)]),
    "fstat_batch_inject": (ctypes.c_int, [_P, _I32, ctypes.POINTER(fstat_signal), _I32, _D]),
    "fstat_batch_clear": (ctypes.c_int, [_P]),
    "fstat_batch_size": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "fstat_batch_compute": (ctypes.c_int, [_P, _P]),
    "fstat_batch_compute_one": (ctypes.c_int, [_P, _I32, _P]),
    "fstat_batch_get_toplist": (ctypes.c_int, [_P, _I32, _I32, _P, _P]),
    "fstat_batch_get_2f": (ctypes.c_int, [_P, _I32, _P, _I64, _I64, _I32]),
    "fstat_batch_get_times": (ctypes.c_int, [_P, _P, ctypes.POINTER(_D)]),
    "fstat_batch_get_plan": (ctypes.c_int, [_P, _I32, _P]),
    "fstat_extract_patches": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _I32, _P, _I32, ctypes.c_float,
                                             ctypes.c_float, _P]),
    "fstat_extract_windows": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _I32, _P, _I32, ctypes.c_float,
                                             ctypes.c_float, _P]),
    # include/fstat_semi.h
    "fstat_stackslide": (ctypes.c_int, [ctypes.POINTER(_P), _I32, _D, _D, _I32, _D, _P, ctypes.POINTER(_I64), _P]),
    # include/fstat_noalloc.h
    "fstat_toplist_noalloc": (ctypes.c_int, [ctypes.c_int, _P, _I64, _I32, _P, _P, _P, ctypes.c_char_p, _I32]),
    # include/fstat_mlp.h
    "fstat_mlp_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _I32, _I32, _I32]),
    "fstat_mlp_destroy": (None, [_P]),
    "fstat_mlp_last_error": (ctypes.c_char_p, [_P]),
    "fstat_mlp_set_params": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "fstat_mlp_get_params": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "fstat_mlp_forward": (ctypes.c_int, [_P, _P, _I32, _P, _I32, _P]),
    "fstat_mlp_train_step": (ctypes.c_int, [_P, _P, _P, _I32, ctypes.c_float, ctypes.c_float, _P, _I32, _P]),
    "fstat_mlp_get_grads": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run __graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def _check(ctx, rc: int):
    if rc != FSTAT_OK:
        msg = _lib.fstat_last_error(ctx) if ctx else b""
        raise FstatError(rc, (msg or b"").decode())


def _host_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


# ---------------------------------------------------------------- C calls

def fstat_version() -> str:
    return _lib.fstat_version().decode()


ALGOS = {"auto": 0, "direct": 1, "farpoly": 2, "sincpoly": 3, "sincrows": 4, "sincpairs": 5}


def fstat_create(device: int = 0, dterms: int = 8, bins_form="c64", topk: int = 1000, kahan: bool = False,
                 tile_m: int = 0, tile_warps: int = 0, sft_chunk: int = 0, algo="auto"):
    form = FORMS[bins_form] if isinstance(bins_form, str) else int(bins_form)
    al = ALGOS[algo] if isinstance(algo, str) else int(algo)
    o = fstat_opts(dterms, form, topk, int(bool(kahan)), tile_m, tile_warps, sft_chunk, al)
    ctx = _P()
    _check(None, _lib.fstat_create(ctypes.byref(ctx), device, ctypes.byref(o)))
    return ctx


def fstat_destroy(ctx) -> None:
    _lib.fstat_destroy(ctx)


def fstat_last_error(ctx) -> str:
    return (_lib.fstat_last_error(ctx) or b"").decode()


def fstat_set_sfts(ctx, det_index: int, lat: float, lon: float, az: float, Tsft: float, k_lo: int,
                   t_start, bins) -> None:
    """bins: complex64 [n_sft, n_bins] numpy array, or a torch CUDA tensor of
    shape [n_sft, n_bins, 2] float32 (or complex64) on the context's device."""
    t = np.ascontiguousarray(t_start, dtype=np.float64)
    det = fstat_detector(lat, lon, az)
    if _is_cuda_tensor(bins):
        if not bins.is_contiguous():
            raise ValueError("device bins must be contiguous")
        n_sft, n_bins = int(bins.shape[0]), int(bins.shape[1])
        ptr, mem = ctypes.c_void_p(bins.data_ptr()), FSTAT_MEM_DEVICE
    else:
        b = np.ascontiguousarray(bins, dtype=np.complex64)
        n_sft, n_bins = b.shape
        ptr, mem = _host_ptr(b), FSTAT_MEM_HOST
    if t.shape[0] != n_sft:
        raise ValueError("t_start and bins disagree on n_sft")
    _check(ctx, _lib.fstat_set_sfts(ctx, det_index, ctypes.byref(det), Tsft, int(k_lo), n_bins, n_sft,
                                    _host_ptr(t), ptr, mem))


def fstat_set_templates(ctx, sky, f0: float, df: float, n_f: int, fdot, t_ref: float) -> None:
    s = np.ascontiguousarray(sky, dtype=np.float64).reshape(-1, 2)
    fd = np.ascontiguousarray(fdot, dtype=np.float64).ravel()
    _check(ctx, _lib.fstat_set_templates(ctx, _host_ptr(s), s.shape[0], f0, df, n_f, _host_ptr(fd), fd.shape[0], t_ref))


def fstat_compute(ctx, stream=None) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    if stream is None:
        h = None
    elif hasattr(stream, "cuda_stream"):
        h = stream.cuda_stream
    else:
        h = int(stream)
    _check(ctx, _lib.fstat_compute(ctx, ctypes.c_void_p(h) if h else None))


def fstat_get_2f(ctx, offset: int, count: int, out=None):
    """Returns a float32 numpy array (or fills `out`, a numpy array or torch CUDA tensor)."""
    if out is None:
        out = np.empty(count, dtype=np.float32)
    if _is_cuda_tensor(out):
        _check(ctx, _lib.fstat_get_2f(ctx, ctypes.c_void_p(out.data_ptr()), offset, count, FSTAT_MEM_DEVICE))
    else:
        _check(ctx, _lib.fstat_get_2f(ctx, _host_ptr(out), offset, count, FSTAT_MEM_HOST))
    return out


def fstat_get_toplist(ctx, k: int):
    idx = np.empty(k, dtype=np.int64)
    val = np.empty(k, dtype=np.float32)
    _check(ctx, _lib.fstat_get_toplist(ctx, k, _host_ptr(idx), _host_ptr(val)))
    return idx, val


def fstat_get_abcd(ctx, n_sky: int):
    out = np.empty((n_sky, 4), dtype=np.float64)
    _check(ctx, _lib.fstat_get_abcd(ctx, _host_ptr(out)))
    return out


def fstat_get_sft_timing(ctx, sky: int, n_sft: int):
    arr = [np.empty(n_sft, dtype=np.float64) for _ in range(4)]
    _check(ctx, _lib.fstat_get_sft_timing(ctx, sky, *[_host_ptr(a) for a in arr]))
    return tuple(arr)


def fstat_inject(ctx, signals, t_ref: float) -> None:
    """signals: iterable of objects with alpha, delta, psi, cosi, phi0, f, fdot, rho."""
    sig = list(signals)
    arr = (fstat_signal * max(len(sig), 1))()
    for i, s in enumerate(sig):
        arr[i] = fstat_signal(s.alpha, s.delta, s.psi, s.cosi, s.phi0, s.f, s.fdot, s.rho)
    _check(ctx, _lib.fstat_inject(ctx, arr, len(sig), t_ref))


def fstat_get_bins(ctx, det_index: int, n_sft: int, n_bins: int):
    out = np.empty((n_sft, n_bins), dtype=np.complex64)
    _check(ctx, _lib.fstat_get_bins(ctx, det_index, _host_ptr(out), FSTAT_MEM_HOST))
    return out


def fstat_get_error_flags(ctx) -> int:
    v = _I32()
    _check(ctx, _lib.fstat_get_error_flags(ctx, ctypes.byref(v)))
    return int(v.value)


def fstat_set_noise_floor(ctx, half_window: int) -> None:
    _check(ctx, _lib.fstat_set_noise_floor(ctx, int(half_window)))


def fstat_set_coverage(ctx, j_lo=None, j_hi=None) -> None:
    """Per-SFT frequency-index ranges [j_lo, j_hi) in SFT load order
    (include/fstat.h); None, None switches coverage off."""
    if j_lo is None and j_hi is None:
        _check(ctx, _lib.fstat_set_coverage(ctx, None, None, 0))
        return
    lo = np.ascontiguousarray(j_lo, dtype=np.int32)
    hi = np.ascontiguousarray(j_hi, dtype=np.int32)
    if lo.shape != hi.shape or lo.ndim != 1:
        raise ValueError("j_lo and j_hi must be equal-length 1-D arrays")
    _check(ctx, _lib.fstat_set_coverage(ctx, _host_ptr(lo), _host_ptr(hi), int(lo.shape[0])))


def fstat_get_noise(ctx, n_sft: int, n_bins: int):
    """(floor [n_sft, n_bins] float32, weights [n_sft] float64) of the last compute."""
    fl = np.empty((n_sft, n_bins), dtype=np.float32)
    w = np.empty(n_sft, dtype=np.float64)
    _check(ctx, _lib.fstat_get_noise(ctx, _host_ptr(fl), _host_ptr(w), FSTAT_MEM_HOST))
    return fl, w


def fstat_test_ring_stall(ctx, after_sft: int) -> None:
    _check(ctx, _lib.fstat_test_ring_stall(ctx, int(after_sft)))


def fstat_get_plan(ctx) -> dict:
    out = np.zeros(8, dtype=np.int32)
    _check(ctx, _lib.fstat_get_plan(ctx, _host_ptr(out)))
    keys = ("P", "L", "M", "warps", "sft_chunk", "lg_row", "w_pairs", "variant")
    return {k: int(v) for k, v in zip(keys, out)}


def fstat_get_launch_count(ctx) -> int:
    n = _I64()
    _check(ctx, _lib.fstat_get_launch_count(ctx, ctypes.byref(n)))
    return int(n.value)


def _stream_handle(stream):
    if stream is None:
        return None
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return ctypes.c_void_p(h) if h else None


def fstat_autotune(ctx, stream=None) -> dict:
    out = np.zeros(4, dtype=np.int32)
    _check(ctx, _lib.fstat_autotune(ctx, _stream_handle(stream), _host_ptr(out)))
    return {"M": int(out[0]), "sft_chunk": int(out[1]), "warps": int(out[2]), "slice_us": int(out[3])}


def fstat_batch_add(ctx, w, bins_override=None) -> int:
    """Add a workload.generate.Workload (its detectors' SFTs and bank) to the batch."""
    dets = w.detectors
    n = len(dets)
    keep = []
    det_arr = (fstat_detector * n)(*[fstat_detector(d.lat, d.lon, d.az) for d in dets])
    n_sft = (ctypes.c_int32 * n)(*[d.n_sft for d in dets])
    tps, bps = (ctypes.c_void_p * n)(), (ctypes.c_void_p * n)()
    for i, d in enumerate(dets):
        t = np.ascontiguousarray(d.t_start, dtype=np.float64)
        b = np.ascontiguousarray(d.bins if bins_override is None else bins_override[i], dtype=np.complex64)
        keep += [t, b]
        tps[i] = t.ctypes.data
        bps[i] = b.ctypes.data
    sky = np.ascontiguousarray(w.bank.sky, dtype=np.float64)
    fd = np.ascontiguousarray(w.bank.fdot, dtype=np.float64)
    wu = fstat_workunit(n, det_arr, n_sft, tps, bps, w.T, int(w.k_lo), int(w.n_bins), sky.ctypes.data,
                        w.bank.n_sky, w.bank.f0, w.bank.df, w.bank.n_f, fd.ctypes.data, w.bank.n_fdot,
                        w.bank.t_ref)
    wid = _I32()
    _check(ctx, _lib.fstat_batch_add(ctx, ctypes.byref(wu), ctypes.byref(wid)))
    del keep
    return int(wid.value)


def fstat_batch_inject(ctx, wu: int, signals, t_ref: float) -> None:
    sig = list(signals)
    arr = (fstat_signal * max(len(sig), 1))()
    for i, s in enumerate(sig):
        arr[i] = fstat_signal(s.alpha, s.delta, s.psi, s.cosi, s.phi0, s.f, s.fdot, s.rho)
    _check(ctx, _lib.fstat_batch_inject(ctx, wu, arr, len(sig), t_ref))


def fstat_batch_clear(ctx) -> None:
    _check(ctx, _lib.fstat_batch_clear(ctx))


def fstat_batch_size(ctx) -> int:
    n = _I32()
    _check(ctx, _lib.fstat_batch_size(ctx, ctypes.byref(n)))
    return int(n.value)


def fstat_batch_compute(ctx, stream=None) -> None:
    _check(ctx, _lib.fstat_batch_compute(ctx, _stream_handle(stream)))


def fstat_batch_compute_one(ctx, wu: int, stream=None) -> None:
    _check(ctx, _lib.fstat_batch_compute_one(ctx, wu, _stream_handle(stream)))


def fstat_batch_get_toplist(ctx, wu: int, k: int):
    idx = np.empty(k, dtype=np.int64)
    val = np.empty(k, dtype=np.float32)
    _check(ctx, _lib.fstat_batch_get_toplist(ctx, wu, k, _host_ptr(idx), _host_ptr(val)))
    return idx, val


def fstat_batch_get_2f(ctx, wu: int, offset: int, count: int):
    out = np.empty(count, dtype=np.float32)
    _check(ctx, _lib.fstat_batch_get_2f(ctx, wu, _host_ptr(out), offset, count, FSTAT_MEM_HOST))
    return out


def fstat_batch_get_plan(ctx, wu: int) -> dict:
    out = np.zeros(8, dtype=np.int32)
    _check(ctx, _lib.fstat_batch_get_plan(ctx, wu, _host_ptr(out)))
    keys = ("P", "L", "M", "warps", "sft_chunk", "lg_row", "w_pairs", "variant")
    return {k: int(v) for k, v in zip(keys, out)}


def fstat_batch_get_times(ctx, n_wu: int):
    done = np.zeros(n_wu, dtype=np.float64)
    tot = _D()
    _check(ctx, _lib.fstat_batch_get_times(ctx, _host_ptr(done), ctypes.byref(tot)))
    return done, float(tot.value)


def fstat_extract_patches(ctx, n_a: int, n_d: int, s_a: int, s_d: int, n_fp: int, f_start, shift: float,
                          scale: float, out) -> None:
    """out: torch CUDA tensor (int16/uint16/bfloat16) of [n_patches, s_a*s_d*n_fp] elements."""
    fst = np.ascontiguousarray(f_start, dtype=np.int32)
    _check(ctx, _lib.fstat_extract_patches(ctx, n_a, n_d, s_a, s_d, n_fp, _host_ptr(fst), fst.size, shift, scale,
                                           ctypes.c_void_p(out.data_ptr())))


def fstat_extract_windows(ctx, n_a: int, n_d: int, s_a: int, s_d: int, n_fp: int, origin, shift: float,
                          scale: float, out) -> None:
    """origin: int array [n_w, 3] of (a0, d0, f0); out: torch CUDA tensor (16-bit) of
    [n_w, s_a*s_d*n_fp] elements."""
    org = np.ascontiguousarray(origin, dtype=np.int32).reshape(-1, 3)
    _check(ctx, _lib.fstat_extract_windows(ctx, n_a, n_d, s_a, s_d, n_fp, _host_ptr(org), org.shape[0], shift, scale,
                                           ctypes.c_void_p(out.data_ptr())))


NOALLOC_MAX_K = 16384


def fstat_toplist_noalloc(v, k: int, idx_out, val_out, stream=None) -> None:
    """Top-k of a CUDA FP32 tensor v into caller-owned CUDA tensors idx_out
    (int64 [k]) and val_out (float32 [k]) without any device allocation by the
    library (include/fstat_noalloc.h); asynchronous on `stream`."""
    msg = ctypes.create_string_buffer(256)
    rc = _lib.fstat_toplist_noalloc(v.device.index, ctypes.c_void_p(v.data_ptr()), int(v.numel()), int(k),
                                    ctypes.c_void_p(idx_out.data_ptr()), ctypes.c_void_p(val_out.data_ptr()),
                                    _stream_handle(stream), msg, len(msg))
    if rc != FSTAT_OK:
        raise FstatError(rc, msg.value.decode())


def fstat_stackslide(segs, f0: float, df: float, n_f: int, t_ref: float, out, stream=None,
                     want_outside: bool = True):
    """Semicoherent stack-slide (include/fstat_semi.h) of the computed
    segment contexts `segs` into the caller's CUDA FP32 tensor `out`
    ([n_sky * n_fdot * n_f]); returns the out-of-band lookup count (or None,
    asynchronous, when want_outside is False)."""
    arr = (_P * len(segs))(*[ctypes.c_void_p(c) if isinstance(c, int) else c for c in segs])
    n_out = _I64(0)
    rc = _lib.fstat_stackslide(arr, len(segs), f0, df, int(n_f), t_ref, ctypes.c_void_p(out.data_ptr()),
                               ctypes.byref(n_out) if want_outside else None, _stream_handle(stream))
    _check(segs[0], rc)
    return int(n_out.value) if want_outside else None


MLP_NAMES = ("W1", "b1", "W2", "b2", "w3", "b3")


def _mlp_check(m, rc):
    if rc != FSTAT_OK:
        raise FstatError(rc, (_lib.fstat_mlp_last_error(m) or b"").decode())


class MLP:
    """The patch-scoring network (include/fstat_mlp.h)."""

    def __init__(self, n_in: int, n_hidden: int, max_batch: int, device: int = 0):
        self.n_in, self.H, self.max_batch = n_in, n_hidden, max_batch
        h = _P()
        _check(None, _lib.fstat_mlp_create(ctypes.byref(h), device, n_in, n_hidden, max_batch))
        self.h = h

    def close(self):
        if self.h:
            _lib.fstat_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shapes(self):
        I, H = self.n_in, self.H
        return {"W1": (I, H), "b1": (H,), "W2": (H, H), "b2": (H,), "w3": (H,), "b3": (1,)}

    def set_params(self, p: dict) -> None:
        arrs = [np.ascontiguousarray(np.asarray(p[k], dtype=np.float32).reshape(self._shapes()[k])) for k in MLP_NAMES]
        _mlp_check(self.h, _lib.fstat_mlp_set_params(self.h, *[_host_ptr(a) for a in arrs]))

    def get_params(self) -> dict:
        out = {k: np.empty(s, dtype=np.float32) for k, s in self._shapes().items()}
        _mlp_check(self.h, _lib.fstat_mlp_get_params(self.h, *[_host_ptr(out[k]) for k in MLP_NAMES]))
        return out

    def get_grads(self) -> dict:
        out = {k: np.empty(s, dtype=np.float32) for k, s in self._shapes().items()}
        _mlp_check(self.h, _lib.fstat_mlp_get_grads(self.h, *[_host_ptr(out[k]) for k in MLP_NAMES]))
        return out

    def forward(self, X, stream=None):
        """X: numpy uint16 (BF16 bits) [B, n_in] or a torch CUDA tensor (16-bit) -> logits."""
        if _is_cuda_tensor(X):
            import torch
            B = int(X.shape[0])
            out = torch.empty(B, dtype=torch.float32, device=X.device)
            _mlp_check(self.h, _lib.fstat_mlp_forward(self.h, ctypes.c_void_p(X.data_ptr()), B,
                                                      ctypes.c_void_p(out.data_ptr()), FSTAT_MEM_DEVICE,
                                                      _stream_handle(stream)))
            return out
        Xh = np.ascontiguousarray(X, dtype=np.uint16)
        out = np.empty(Xh.shape[0], dtype=np.float32)
        _mlp_check(self.h, _lib.fstat_mlp_forward(self.h, _host_ptr(Xh), Xh.shape[0], _host_ptr(out),
                                                  FSTAT_MEM_HOST, _stream_handle(stream)))
        return out

    def train_step(self, X, y, pos_weight: float, lr: float, stream=None, want_loss: bool = True):
        lv = ctypes.c_float()
        lp = ctypes.byref(lv) if want_loss else None
        if _is_cuda_tensor(X):
            _mlp_check(self.h, _lib.fstat_mlp_train_step(self.h, ctypes.c_void_p(X.data_ptr()),
                                                         ctypes.c_void_p(y.data_ptr()), int(X.shape[0]),
                                                         pos_weight, lr, lp, FSTAT_MEM_DEVICE,
                                                         _stream_handle(stream)))
        else:
            Xh = np.ascontiguousarray(X, dtype=np.uint16)
            yh = np.ascontiguousarray(y, dtype=np.float32)
            _mlp_check(self.h, _lib.fstat_mlp_train_step(self.h, _host_ptr(Xh), _host_ptr(yh), Xh.shape[0],
                                                         pos_weight, lr, lp, FSTAT_MEM_HOST, _stream_handle(stream)))
        return float(lv.value) if want_loss else None


def fstat_take_kernel_time(ctx):
    mb, mt, n = _D(), _D(), _I32()
    _check(ctx, _lib.fstat_take_kernel_time(ctx, ctypes.byref(mb), ctypes.byref(mt), ctypes.byref(n)))
    return float(mb.value), float(mt.value), int(n.value)


# ---------------------------------------------------------------- convenience

class FStat:
    """Owns one context; methods forward to the C calls above."""

    def __init__(self, device: int = 0, **opts):
        self.ctx = fstat_create(device, **opts)
        self.n_sky = self.n_f = self.n_fdot = 0
        self.n_sft = 0

    def close(self):
        if self.ctx:
            fstat_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_workload(self, w, bins_override=None):
        """Load a workload.generate.Workload's detectors (optionally with
        replacement bin arrays, e.g. with signals added) and its template bank."""
        self.n_sft = 0
        for i, d in enumerate(w.detectors):
            b = d.bins if bins_override is None else bins_override[i]
            fstat_set_sfts(self.ctx, i, d.lat, d.lon, d.az, w.T, w.k_lo, d.t_start, b)
            self.n_sft += d.n_sft
        self.set_bank(w.bank)

    def set_bank(self, bank):
        fstat_set_templates(self.ctx, bank.sky, bank.f0, bank.df, bank.n_f, bank.fdot, bank.t_ref)
        self.n_sky, self.n_f, self.n_fdot = bank.n_sky, bank.n_f, bank.n_fdot

    @property
    def n_templates(self) -> int:
        return self.n_sky * self.n_f * self.n_fdot

    def compute(self, stream=None):
        fstat_compute(self.ctx, stream)

    def twoF(self, offset: int = 0, count: int | None = None):
        count = self.n_templates - offset if count is None else count
        return fstat_get_2f(self.ctx, offset, count)

    def toplist(self, k: int):
        return fstat_get_toplist(self.ctx, k)

    def abcd(self):
        return fstat_get_abcd(self.ctx, self.n_sky)

    def sft_timing(self, sky: int):
        return fstat_get_sft_timing(self.ctx, sky, self.n_sft)

    def inject(self, signals, t_ref: float):
        fstat_inject(self.ctx, signals, t_ref)

    def error_flags(self) -> int:
        return fstat_get_error_flags(self.ctx)

    def plan(self) -> dict:
        return fstat_get_plan(self.ctx)

    def take_kernel_time(self):
        return fstat_take_kernel_time(self.ctx)

    def launch_count(self) -> int:
        return fstat_get_launch_count(self.ctx)

    def autotune(self, stream=None) -> dict:
        return fstat_autotune(self.ctx, stream)
