"""Pins of the oracle's bpa codec (Sect. 5: f_bpa = m 2^e, per-operator bpa chosen
against eps_mf) against hand-worked values, exactness and error bounds, and the
paper's statement that operators which reduce to rediscretisation / d-linear
transfer cost no storage at all."""
import numpy as np
import pytest

from oracle import bpa, multigrid
from oracle import spacetree as stt
import synthetic as syn


def test_worked_entries_by_hand():
    # bpa = 2: one exponent byte, one byte of m (sign bit + 7 magnitude bits)
    # 0.75 = 0.75 * 2^0 -> e = 0 - 7 = -7, m = 0.75 * 128 = 96
    assert bpa.entry_bytes(0.75, 2) == bytes([0xF9, 0x60])
    assert bpa.entry_bytes(-0.75, 2) == bytes([0xF9, 0xE0])
    # 1/3 = (2/3) 2^-1 -> e = -8, m = rint(256 / 3) = 85, error 1/768
    e, s, m = bpa.encode_entry(1.0 / 3.0, 2)
    assert (e, s, m) == (-8, 0, 85)
    assert bpa.entry_error(1.0 / 3.0, 2) == pytest.approx(1.0 / 768.0, rel=1e-12)
    # 0.998 * 128 = 127.744 rounds to 128 = 2^7: carry to e = -6, m = 64 (value 1.0)
    assert bpa.encode_entry(0.998, 2) == (-6, 0, 64)
    # bpa = 3: 15 magnitude bits; 1/3 -> e = -16, m = rint(65536 / 3) = 21845
    assert bpa.encode_entry(1.0 / 3.0, 3) == (-16, 0, 21845)
    assert bpa.entry_bytes(1.0 / 3.0, 3) == bytes([0xF0, 0x55, 0x55])
    assert bpa.encode_entry(0.0, 5) == (0, 0, 0)
    # the magnitude bits per bpa: 8 (bpa - 1) - 1
    assert [bpa.mantissa_bits(b) for b in range(2, 9)] == [7, 15, 23, 31, 39, 47, 55]


def test_bpa8_is_lossless_and_bytes_roundtrip():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(400) * np.exp2(rng.integers(-70, 100, 400))
    for v in x:
        assert bpa.entry_error(v, 8) == 0.0
        raw = bpa.entry_bytes(v, 8)
        e = raw[0] - 256 if raw[0] >= 128 else raw[0]
        word = int.from_bytes(raw[1:], "little")
        assert bpa.decode_entry(e, word >> 55, word & ((1 << 55) - 1)) == v


def test_relative_error_bound_per_bpa():
    # |f_bpa(x) - x| <= |x| 2^-M with M magnitude bits (half a unit of m, m >= 2^(M-1))
    rng = np.random.default_rng(2)
    x = rng.standard_normal(300) * np.exp2(rng.integers(-40, 40, 300))
    for b in range(2, 9):
        M = bpa.mantissa_bits(b)
        errs = np.array([bpa.entry_error(v, b) for v in x])
        assert np.all(errs <= np.abs(x) * 2.0 ** -M)
        # and not much better: the bound is reached within a factor 4 somewhere
        if M < 50:
            assert np.max(errs / np.abs(x)) > 2.0 ** -M / 4


def test_exponent_clamp():
    # 2^-140 at bpa = 2 would need e = -140 - 7 + 1: clamped to -128, m = rint(2^-12) = 0
    assert bpa.encode_entry(2.0 ** -140, 2) == (-128, 0, 0)
    assert bpa.entry_error(2.0 ** -140, 2) == 2.0 ** -140
    # beyond the largest exponent no bpa can store the value
    assert bpa.encode_entry(2.0 ** 200, 8) is None
    with pytest.raises(ValueError):
        bpa.choose_bpa(np.array([2.0 ** 200]), 1e-8)


def test_choice_is_smallest_within_tolerance():
    rng = np.random.default_rng(3)
    for eps_mf in (1e-2, 1e-4, 1e-8):
        for _ in range(60):
            row = rng.standard_normal(9) * 10.0 ** rng.uniform(-10, 1)
            b = bpa.choose_bpa(row, eps_mf)
            assert all(bpa.entry_error(v, b) <= eps_mf for v in row)
            prev = bpa.BPA_CHOICES[bpa.BPA_CHOICES.index(b) - 1] if b else None
            if prev is not None:
                assert any(bpa.entry_error(v, prev) > eps_mf for v in row)
    assert bpa.choose_bpa(np.zeros(25), 1e-8) == 0
    assert bpa.choose_bpa(np.full(9, 0.5e-2), 1e-2) == 0
    assert bpa.choose_bpa(np.full(9, 2e-2), 1e-2) == 2


def test_rows_roundtrip_and_layout():
    rng = np.random.default_rng(4)
    rows = rng.standard_normal((50, 9)) * 10.0 ** rng.uniform(-12, 0, (50, 1))
    rows[7] = 0.0
    for eps_mf in (1e-2, 1e-4, 1e-8):
        b, off, stream = bpa.encode_rows(rows, eps_mf)
        assert b[7] == 0
        assert len(stream) == int(np.sum(b * 9))
        assert np.array_equal(off[1:], np.cumsum(b * 9)[:-1])
        dec = bpa.decode_rows(b, off, stream, 9)
        assert np.all(np.abs(dec - rows) <= eps_mf)
        rec = bpa.records(b, off)
        assert np.array_equal(rec & np.uint64(15), b.astype(np.uint64))
        assert np.array_equal(rec >> np.uint64(4), off.astype(np.uint64))


@pytest.mark.parametrize("dim,L", [(2, 4), (3, 3)])
def test_constant_coefficient_operators_store_nothing(dim, L):
    # Sect. 5: with constant eps the Galerkin operators equal rediscretisation and BoxMG
    # equals d-linear transfer, so every vertex is marked and no byte is stored
    tree = stt.Spacetree(dim, L)
    H = multigrid.Hierarchy(tree, {L: syn.constant_eps(L, dim)})
    for lv in range(1, L):
        for rows in (H.ops[lv].a_hat, H.ops[lv + 1].p_hat):
            for eps_mf in (1e-2, 1e-4, 1e-8):
                b, _, stream = bpa.encode_rows(rows, eps_mf)
                assert not b.any() and len(stream) == 0


def test_rough_coefficient_operators_need_bytes():
    # a log-normal coefficient makes both deltas non-zero; a tighter eps_mf never
    # needs fewer bytes, and bpa = 0 survives only where the deltas are small
    tree = stt.Spacetree(2, 4)
    H = multigrid.Hierarchy(tree, {4: syn.lognormal_grf_eps(4, 2, sigma=2.0, seed=5)})
    for rows in (H.ops[3].a_hat, H.ops[4].p_hat):
        sizes = [bpa.encode_rows(rows, eps_mf)[0].sum() for eps_mf in (1e-2, 1e-4, 1e-8)]
        assert 0 < sizes[0] <= sizes[1] <= sizes[2]
        b, _, _ = bpa.encode_rows(rows, 1e-8)
        assert np.all(np.abs(rows[b == 0]) <= 1e-8)
