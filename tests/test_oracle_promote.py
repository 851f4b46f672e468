"""Pins of the oracle's promotion rule of the mixed path's delta codes (the dtype
counterpart of the paper's per-vertex choice of storage against eps_mf, Sect. 5).

A row is promoted when half a unit of the 16-bit format relative to its scale s
exceeds 2^-8 of the reconstructed diagonal |A_vv|: s > 2 |A_vv| for bf16, s > 16 |A_vv|
for fp16.  Promoted rows store the FP32 bit pattern of delta_k / s (high half in the
code plane, low half in a second plane) and the flag as the sign of the scale word.
The expected bit patterns below are worked out by hand from the IEEE 754 layouts.
"""
import numpy as np
import pytest

from oracle import codec

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _row(center, other):
    """A 9-entry row (offsets -1..1 lexicographic, centre index 4)."""
    r = np.full(9, other, dtype=np.float64)
    r[4] = center
    return r


def test_hand_worked_bit_patterns_and_threshold():
    # scale s = max |delta| = 2 (exact in FP32); the other entries are 2 (1 - 2^-12),
    # so delta_k / s = 1 - 2^-12 = 0.999755859375:
    #   FP32: exponent -1 -> biased 126, fraction (2 (1 - 2^-12) - 1) 2^23 = 2^23 - 2^12
    #         bits = 126 << 23 | 0x7FF000 = 0x3F7FF000 -> high 0x3F7F, low 0xF000
    #   BF16 (8 significant bits): quantum 2^-8 on [1/2, 1); 1 - 2^-12 rounds to 1.0 = 0x3F80
    #   FP16 (11 significant bits): quantum 2^-11 on [1/2, 1); 1 - 2^-12 is a tie between
    #         1 - 2^-11 (odd last bit) and 1.0 (even) -> 1.0 = 0x3C00
    # the centre entry -2 gives delta / s = -1: BF16 0xBF80, FP16 0xBC00, FP32 0xBF800000
    other = 2.0 * (1.0 - 2.0 ** -12)
    d = np.stack([_row(-2.0, other)] * 4)
    # bf16 threshold s > 2 |A_vv|: |A_vv| = 0.999 promotes, 1.0 does not (equality),
    # 1 - 2^-30 promotes, 0.5 promotes
    diag = np.array([0.999, 1.0, 1.0 - 2.0 ** -30, 0.5])
    codes, lo, scale = codec.encode_promoting(d, diag, "bf16")
    flags = np.signbit(scale)
    assert flags.tolist() == [True, False, True, True]
    assert np.all(np.abs(scale) == 2.0)
    for i in range(4):
        if flags[i]:
            assert codes[i, 0] == 0x3F7F and lo[i, 0] == 0xF000
            assert codes[i, 4] == 0xBF80 and lo[i, 4] == 0x0000
        else:
            assert codes[i, 0] == 0x3F80 and lo[i, 0] == 0
            assert codes[i, 4] == 0xBF80
    # fp16 threshold s > 16 |A_vv|: 0.124 promotes, 0.125 does not
    codes, lo, scale = codec.encode_promoting(d[:2], np.array([0.124, 0.125]), "fp16")
    assert np.signbit(scale).tolist() == [True, False]
    assert codes[0, 0] == 0x3F7F and lo[0, 0] == 0xF000  # promoted: FP32 halves
    assert codes[1, 0] == 0x3C00 and lo[1, 0] == 0  # FP16 code
    assert codes[1, 4] == 0xBC00
    # decoding: promoted rows give the FP32 value times s, the others the 16-bit one
    codes, lo, scale = codec.encode_promoting(d[:2], np.array([0.5, 1.0]), "bf16")
    dec = codec.decode_promoting(codes, lo, scale, "bf16")
    assert dec[0, 0] == np.float32(other) and dec[0, 4] == np.float32(-2.0)
    assert dec[1, 0] == np.float32(2.0) and dec[1, 4] == np.float32(-2.0)


def test_zero_rows_and_rows_without_cancellation_are_not_promoted():
    rng = np.random.default_rng(3)
    d = rng.standard_normal((50, 9))
    d[7] = 0.0
    diag = 10.0 * np.abs(d).max(axis=1) + 1.0  # no cancellation anywhere
    codes, lo, scale = codec.encode_promoting(d, diag, "bf16")
    plain_codes, plain_scale = codec.encode(d, "bf16")
    assert not np.signbit(scale).any()
    assert np.array_equal(codes, plain_codes) and np.array_equal(scale, plain_scale) and not lo.any()
    # the all-zero row: s = 0 and never promoted, even against a zero diagonal
    codes, lo, scale = codec.encode_promoting(d[7:8], np.zeros(1), "bf16")
    assert scale[0] == 0.0 and not np.signbit(scale[0]) and not codes.any()


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_rule_bounds_the_diagonal_error_of_every_stored_row(fmt):
    # the promise of the rule: after decoding, every row's reconstructed diagonal
    # A_redisc + decoded delta is within 2^-8 |A_vv| (+ the FP32 product's rounding);
    # promoted rows are within FP32 rounding of each entry
    rng = np.random.default_rng(5)
    n = 4000
    d = rng.standard_normal((n, 9)) * np.exp(rng.uniform(-5, 5, (n, 1)))
    smax = np.abs(d).max(axis=1)
    diag = smax * np.exp(rng.uniform(-12, 4, n))  # from heavy cancellation to none
    diag *= np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    codes, lo, scale = codec.encode_promoting(d, diag, fmt)
    dec = codec.decode_promoting(codes, lo, scale, fmt).astype(np.float64)
    flags = np.signbit(scale)
    assert 0 < flags.sum() < n
    s = np.abs(scale).astype(np.float64)
    err = np.abs(dec - d)
    ok = ~flags
    assert np.all(err[ok, 4] <= codec.PROMOTE_REL * np.abs(diag[ok]) + 2.0 ** -24 * s[ok])
    assert np.all(err[flags] <= 2.0 ** -23 * np.abs(d[flags]) + 2.0 ** -149)
    # and exactly the rows whose 16-bit error bound could exceed 2^-8 |A_vv| are promoted
    assert np.array_equal(flags, s * codec.HALF_UNIT[fmt] > codec.PROMOTE_REL * np.abs(diag))
