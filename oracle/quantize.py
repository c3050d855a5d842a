"""Oracle of the 16-bit SFT storage forms (TEST INFRASTRUCTURE).

Each SFT row is scaled by s = m / 2^14, m = max over its bins of max(|Re|, |Im|)
(FP32), so the stored values stay below 2^14 (head-room under FP16's 65504).
The stored value of a component x is round-to-nearest-even of the FP32
quotient x / s to FP16 or to BF16; the value it stands for is q * s.
An all-zero row gets s = 1.
"""
from __future__ import annotations

import numpy as np

FORMS = ("f16", "bf16")


def row_scales(bins_c64: np.ndarray) -> np.ndarray:
    """Per-SFT scale s (float32), [n_sft]."""
    re = np.abs(bins_c64.real.astype(np.float32))
    im = np.abs(bins_c64.imag.astype(np.float32))
    m = np.maximum(re.max(axis=-1), im.max(axis=-1)).astype(np.float32)
    s = (m * np.float32(2.0 ** -14)).astype(np.float32)
    return np.where(m > 0, s, np.float32(1.0)).astype(np.float32)


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even of float32 to bfloat16 (finite inputs), uint16 bits."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    return ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def quantize(bins_c64: np.ndarray, form: str):
    """Return (bits_re, bits_im, scale): uint16 [n_sft, n_bins] codes of the
    scaled components and the float32 per-SFT scale."""
    if form not in FORMS:
        raise ValueError(form)
    s = row_scales(bins_c64)
    re = (bins_c64.real.astype(np.float32) / s[:, None]).astype(np.float32)
    im = (bins_c64.imag.astype(np.float32) / s[:, None]).astype(np.float32)
    if form == "f16":
        return re.astype(np.float16).view(np.uint16), im.astype(np.float16).view(np.uint16), s
    return f32_to_bf16_bits(re), f32_to_bf16_bits(im), s


def dequantize(bits_re: np.ndarray, bits_im: np.ndarray, scale: np.ndarray, form: str) -> np.ndarray:
    """The complex128 values the codes stand for, q * s (exact in FP64)."""
    if form == "f16":
        re = bits_re.view(np.float16).astype(np.float64)
        im = bits_im.view(np.float16).astype(np.float64)
    else:
        re = bf16_bits_to_f32(bits_re).astype(np.float64)
        im = bf16_bits_to_f32(bits_im).astype(np.float64)
    s = scale.astype(np.float64)[:, None]
    return re * s + 1j * (im * s)
