"""Loader of the plain-C FP64 oracle (``oracle/fstat_oracle.c``).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  It
compiles the C file with the host's gcc (IEEE FP64, no fast-math) into
``oracle/_build/`` on first use, or when the source is newer than the built
library, and calls it through ctypes.  The C calls release the GIL, so a
thread pool spreads sky points over the host cores.

The arithmetic is that of ``fstat_oracle.py`` (Listing 1's loop nest of the
paper, the Dirichlet-kernel SFT demodulation and the A, B, C, D combine),
written as plain loops; ``tests/test_oracle_c.py`` pins it against the numpy
oracle and against the noise-free closed form.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fstat_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfstat_oracle.so")
_lock = threading.Lock()
_lib = None


def compile_c(src: str, out: str) -> str:
    """gcc -O2, IEEE FP64 (no fast-math, no contraction into fused multiply-adds)."""
    tmp = out + f".{os.getpid()}.tmp"
    cmd = [os.environ.get("CC", "gcc"), "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", src, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed on the C oracle:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the C oracle if the library is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    return compile_c(SRC, LIB)


def open_library(path: str) -> ctypes.CDLL:
    """Load a compiled C oracle and declare its two entry points."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.oracle_fstat_band.argtypes = [i32, P, P, P, P, f64, i64, i32, i32, P, i32, i32,
                                      f64, f64, i32, P, i32, f64, P]
    lib.oracle_fstat_band.restype = i32
    lib.oracle_fstat_templates.argtypes = [i32, P, P, P, P, f64, i64, i32, i32, P,
                                           f64, f64, i32, P, i32, f64, P, i64, P]
    lib.oracle_fstat_templates.restype = i32
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = open_library(build())
    return _lib


class _Data:
    """The detectors' arrays in the flat layout the C oracle reads (kept alive
    for the calls)."""

    def __init__(self, dets, n_bins: int):
        self.n_det = len(dets)
        self.n_sft = np.array([d.n_sft for d in dets], dtype=np.int32)
        self.geom = np.array([[d.lat, d.lon, d.az] for d in dets], dtype=np.float64)
        self.t = np.ascontiguousarray(np.concatenate([np.asarray(d.t_start, np.float64) for d in dets]))
        self.bins = np.ascontiguousarray(np.concatenate(
            [np.asarray(d.bins, dtype=np.complex64).reshape(d.n_sft, n_bins) for d in dets]).view(np.float32))

    def args(self):
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        return [self.n_det, p(self.n_sft), p(self.geom), p(self.t), p(self.bins)]


def _threads(n: int | None) -> int:
    return max(1, n if n else (os.cpu_count() or 1))


def compute_fstat_freq_band(dets, T: float, k_lo: int, dterms: int, bank, sky_indices=None,
                            threads: int | None = None, lib=None):
    """2F over the bank's band, [n_sky_sel, n_fdot, n_f] float64, at the
    selected sky points (all by default); sky points run in parallel."""
    lib = lib or _load()
    n_bins = int(np.asarray(dets[0].bins).shape[1])
    data = _Data(dets, n_bins)
    sky = np.ascontiguousarray(bank.sky, dtype=np.float64)
    fdot = np.ascontiguousarray(bank.fdot, dtype=np.float64)
    sel = np.arange(bank.n_sky) if sky_indices is None else np.asarray(list(sky_indices), dtype=np.int64)
    out = np.empty((len(sel), bank.n_fdot, bank.n_f), dtype=np.float64)

    def one(i):
        s = int(sel[i])
        rc = lib.oracle_fstat_band(*data.args(), float(T), int(k_lo), n_bins, int(dterms),
                                   sky.ctypes.data_as(ctypes.c_void_p), s, s + 1, float(bank.f0), float(bank.df),
                                   int(bank.n_f), fdot.ctypes.data_as(ctypes.c_void_p), int(bank.n_fdot),
                                   float(bank.t_ref), out[i].ctypes.data_as(ctypes.c_void_p))
        if rc != 0:
            raise RuntimeError(f"C oracle failed ({rc})")

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(len(sel))))
    return out


def compute_fstat_templates(dets, T: float, k_lo: int, dterms: int, bank, indices,
                            threads: int | None = None, lib=None):
    """2F of flat template indices ((sky * n_fdot) + fdot) * n_f + f, in the
    order given; groups of one sky point run in parallel."""
    lib = lib or _load()
    n_bins = int(np.asarray(dets[0].bins).shape[1])
    data = _Data(dets, n_bins)
    sky = np.ascontiguousarray(bank.sky, dtype=np.float64)
    fdot = np.ascontiguousarray(bank.fdot, dtype=np.float64)
    indices = np.asarray(indices, dtype=np.int64)
    order = np.argsort(indices // (bank.n_fdot * bank.n_f), kind="stable")
    srt = np.ascontiguousarray(indices[order])
    res = np.empty(srt.shape[0], dtype=np.float64)
    sky_of = srt // (bank.n_fdot * bank.n_f)
    cuts = np.concatenate([[0], np.nonzero(np.diff(sky_of))[0] + 1, [srt.shape[0]]]) if srt.size else [0]

    def one(g):
        a, b = int(cuts[g]), int(cuts[g + 1])
        rc = lib.oracle_fstat_templates(*data.args(), float(T), int(k_lo), n_bins, int(dterms),
                                        sky.ctypes.data_as(ctypes.c_void_p), float(bank.f0), float(bank.df),
                                        int(bank.n_f), fdot.ctypes.data_as(ctypes.c_void_p), int(bank.n_fdot),
                                        float(bank.t_ref), srt[a:].ctypes.data_as(ctypes.c_void_p), b - a,
                                        res[a:].ctypes.data_as(ctypes.c_void_p))
        if rc != 0:
            raise RuntimeError(f"C oracle failed ({rc})")

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(len(cuts) - 1)))
    out = np.empty_like(res)
    out[order] = res
    return out
