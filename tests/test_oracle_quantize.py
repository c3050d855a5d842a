"""Pins of the 16-bit storage oracle: exact values, round-to-nearest-even ties,
range, and the error bound of each format (CPU only)."""
import numpy as np
import pytest

from oracle import quantize as Q


def test_bf16_rounding_ties_to_even():
    one = 1.0
    x = np.array([one, one + 2 ** -8, one + 3 * 2 ** -8, one + 2 ** -7, -(one + 2 ** -8),
                  one + 2 ** -8 + 2 ** -20, 3.0, 2.0 ** -100], dtype=np.float32)
    got = Q.bf16_bits_to_f32(Q.f32_to_bf16_bits(x))
    want = np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, -1.0, 1.0 + 2 ** -7, 3.0, 2.0 ** -100],
                    dtype=np.float32)
    np.testing.assert_array_equal(got, want)


def test_scale_and_exact_round_trip():
    # values that are exact multiples of s with few significant bits survive exactly
    m = np.float32(3.0)
    s = m * np.float32(2 ** -14)
    vals = np.array([3.0, -3.0, 1.5, 0.75, 0.0, -0.375], dtype=np.float32)
    row = (vals + 1j * vals[::-1]).astype(np.complex64)[None, :]
    assert Q.row_scales(row)[0] == s
    for form in Q.FORMS:
        br, bi, sc = Q.quantize(row, form)
        back = Q.dequantize(br, bi, sc, form)
        np.testing.assert_array_equal(back, row.astype(np.complex128))
        # the largest component maps to exactly 2^14
        if form == "f16":
            assert np.max(np.abs(br.view(np.float16).astype(np.float32))) == 2 ** 14


@pytest.mark.parametrize("form,rel", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_error_bound(form, rel):
    """|q s - x| <= 2^-(p+1) |x| for a p-bit significand, plus FP16's
    subnormal spacing 2^-24 (times s) near zero."""
    rng = np.random.default_rng(0)
    x = (rng.standard_normal((20, 300)) + 1j * rng.standard_normal((20, 300))).astype(np.complex64)
    x[3] = 0
    br, bi, sc = Q.quantize(x, form)
    back = Q.dequantize(br, bi, sc, form)
    assert sc[3] == 1.0 and np.all(back[3] == 0)
    floor = sc[:, None].astype(np.float64) * (2.0 ** -25 if form == "f16" else 0.0)
    for got, ref in ((back.real, x.real), (back.imag, x.imag)):
        ref = ref.astype(np.float64)
        assert np.all(np.abs(got - ref) <= rel * np.abs(ref) * (1 + 1e-6) + floor)
