"""Pins of the BFP codec oracle (Section III-C-3) against facts the section fixes.

The expected words below were derived by hand from the section's definitions
(shown in each comment), not by running the oracle; the other checks use
properties that hold independently of how the oracle is written: brute force over
every coefficient, the exponent definition by integer search, the half-quantum
error bound, ties-to-even, and exact round trips of values on the grid.
"""
import numpy as np
import pytest

from oracle.bfp import RATES, bfp_decode, bfp_decode_block, bfp_encode, bfp_encode_block, bfp_layout, bfp_stream_bytes

F32_MAX = float(np.finfo(np.float32).max)


def test_layout_rates():
    # n_bits = 16, 12, 10 -> v_bits = 14, 10, 8; one uint64, three uint16, five uint8 per block
    assert [bfp_layout(n) for n in RATES] == [(14, 8), (10, 6), (8, 5)]
    assert bfp_stream_bytes(0, 16) == 0
    assert bfp_stream_bytes(9, 12) == 3 * 6
    with pytest.raises(ValueError):
        bfp_layout(8)


def test_hand_derived_words():
    # 16 bits: max 1.0 -> e_max = 1 (2^0 <= 1 < 2^1), e = 128 = 0x80; scale 2^(13-1):
    # q = 4096, -2048, 1024, 0 -> fields 0x1000, 0x3800 (2^14 - 2048), 0x0400, 0;
    # word = 0x80 + 0x1000 2^8 + 0x3800 2^22 + 0x400 2^36 = 0x0000400E00100080
    assert bfp_encode_block([1.0, -0.5, 0.25, 0.0], 16) == bytes.fromhex("800010000e400000")
    # 10 bits: max 3 -> e_max = 2, e = 0x81; scale 2^(7-2) = 32: q = 96, -96, 24, round(-0.25) = 0
    # -> bytes 0x81, 0x60, 0xA0 (256 - 96), 0x18, 0x00
    assert bfp_encode_block([3.0, -3.0, 0.75, -0.0078125], 10) == bytes.fromhex("8160a01800")
    # 12 bits: max 6.5 -> e_max = 3, e = 0x82; scale 2^(9-3) = 64: q = -416, round(6.4000001) = 6,
    # 128, 320 -> fields 608, 6, 128, 320; word = 0x82 + 608 2^8 + 6 2^18 + 128 2^28 + 320 2^38
    # = 0x5008001A6082
    assert bfp_encode_block([-6.5, np.float32(0.1), 2.0, 5.0], 12) == bytes.fromhex("82601a000850")
    np.testing.assert_array_equal(bfp_decode_block(bytes.fromhex("82601a000850"), 12),
                                  np.float32([-6.5, 0.09375, 2.0, 5.0]))


def test_brute_force_every_coefficient_v8():
    # e_max = 0 forced by a companion value 0.5 (2^-1 <= max < 1); every q in [-127, 127]
    for q in range(-127, 128):
        x = np.float32([q / 128.0, 0.5, 0.0, 0.0])
        b = bfp_encode_block(x, 10)
        assert b[0] == 127                      # e = e_max + 127
        assert b[1] == (q & 0xFF)               # low 8 bits, two's complement
        assert b[2] == 64 and b[3] == 0 and b[4] == 0
        np.testing.assert_array_equal(bfp_decode_block(b, 10), x)


def _integer_emax(m: float) -> int:
    e = -200
    while not m < 2.0 ** e:
        e += 1
    return e


def _blocks(rng, nblk):
    """Random float32 blocks: block scales from 2^-140 to 2^126, spreads up to 2^20 inside."""
    scale = 2.0 ** rng.uniform(-140, 126, size=(nblk, 1))
    spread = 2.0 ** rng.uniform(-20, 0, size=(nblk, 4))
    sign = rng.choice([-1.0, 1.0], size=(nblk, 4))
    return np.float32(scale * spread * sign)


@pytest.mark.parametrize("nbits", RATES)
def test_exponent_definition_and_error_bound(nbits):
    v, nbytes = bfp_layout(nbits)
    rng = np.random.default_rng(11 + nbits)
    xs = _blocks(rng, 600)
    for x in xs:
        b = bfp_encode_block(x, nbits)
        e = b[0]
        m = float(np.max(np.abs(x.astype(np.float64))))
        emax = _integer_emax(m)                 # smallest E with m < 2^E
        if m >= 2.0 ** -126:
            assert 2.0 ** (emax - 1) <= m < 2.0 ** emax
            assert e == emax + 127
        else:
            assert e == 1                       # subnormal block: e_max = -126
            emax = -126
        y = bfp_decode_block(b, nbits).astype(np.float64)
        quantum = 2.0 ** (emax - v + 1)
        err = np.abs(y - x.astype(np.float64))
        clamped = np.abs(x.astype(np.float64)) / quantum > 2 ** (v - 1) - 1
        assert np.all(err[~clamped] <= quantum / 2)
        assert np.all(err[clamped] <= quantum)


def test_ties_to_even():
    # e_max = 1 (block max 1.0), v = 14: quantum 2^-12
    h = 2.0 ** -12
    x = np.float32([1.0, 2.5 * h, 3.5 * h, -2.5 * h])
    np.testing.assert_array_equal(bfp_decode_block(bfp_encode_block(x, 16), 16), np.float32([1.0, 2 * h, 4 * h, -2 * h]))
    x = np.float32([1.0, 0.5 * h, -1.5 * h, 1.5 * h])
    np.testing.assert_array_equal(bfp_decode_block(bfp_encode_block(x, 16), 16), np.float32([1.0, 0.0, -2 * h, 2 * h]))


def test_upper_clamp_and_lower_bound():
    # largest float below 1: e_max = 0, 2^13 (1 - 2^-24) rounds to 8192 -> clamped to 8191
    x = np.float32([np.nextafter(np.float32(1), np.float32(0)), -0.75, 0, 0])
    y = bfp_decode_block(bfp_encode_block(x, 16), 16)
    assert y[0] == np.float32(8191 * 2.0 ** -13) and y[1] == -0.75
    # -(1 - 2^-24) rounds to -8192 = -2^(v-1): inside the range, no clamp, decodes to -1
    x = np.float32([-np.nextafter(np.float32(1), np.float32(0)), 0.75, 0, 0])
    assert bfp_decode_block(bfp_encode_block(x, 16), 16)[0] == -1.0


def test_zero_subnormal_and_largest_blocks():
    for nbits in RATES:
        _, nbytes = bfp_layout(nbits)
        assert bfp_encode_block([0.0, -0.0, 0.0, 0.0], nbits) == bytes(nbytes)
        np.testing.assert_array_equal(bfp_decode_block(bytes(nbytes), nbits), np.zeros(4, np.float32))
    # subnormal block, v = 14: e = 1 (e_max = -126), quantum 2^-139; multiples of it round-trip
    x = np.float32([5 * 2.0 ** -139, -3 * 2.0 ** -139, 2.0 ** -130, 0.0])
    b = bfp_encode_block(x, 16)
    assert b[0] == 1
    np.testing.assert_array_equal(bfp_decode_block(b, 16), x)
    # top exponent: e = 255; +max clamps to 2^128 - 2^115, -max to its negative (finite)
    b = bfp_encode_block([F32_MAX, -F32_MAX, 1.0, 0.0], 16)
    assert b[0] == 255
    y = bfp_decode_block(b, 16)
    assert np.all(np.isfinite(y))
    assert float(y[0]) == 2.0 ** 128 - 2.0 ** 115 and float(y[1]) == -(2.0 ** 128 - 2.0 ** 115)


@pytest.mark.parametrize("nbits", RATES)
def test_grid_values_round_trip(nbits):
    v, _ = bfp_layout(nbits)
    rng = np.random.default_rng(nbits)
    for emax in (-125, -40, 0, 1, 17, 127):
        q = rng.integers(-(2 ** (v - 1)), 2 ** (v - 1), size=(50, 4))
        q[:, 0] = rng.choice([-1, 1], size=50) * rng.integers(2 ** (v - 2), 2 ** (v - 1), size=50)  # fixes e_max
        x = np.float32(q * 2.0 ** (emax - v + 1))
        y = bfp_decode(bfp_encode(x.ravel(), nbits), x.size, nbits)
        np.testing.assert_array_equal(y, x.ravel())


def test_ragged_stream_pads_with_zeros():
    rng = np.random.default_rng(3)
    x = np.float32(rng.standard_normal(11))
    for nbits in RATES:
        s = bfp_encode(x, nbits)
        assert s.size == bfp_stream_bytes(11, nbits)
        padded = np.concatenate([x, np.zeros(1, np.float32)])
        np.testing.assert_array_equal(s, bfp_encode(padded, nbits))
        y = bfp_decode(s, 11, nbits)
        assert y.shape == (11,)
        np.testing.assert_array_equal(y, bfp_decode(bfp_encode(padded, nbits), 12, nbits)[:11])
    assert bfp_encode(np.zeros(0, np.float32), 16).size == 0
    assert bfp_decode(np.zeros(0, np.uint8), 0, 16).size == 0


def test_sixteen_bit_rate_beats_bfloat16_near_the_block_max():
    # values within a factor of two of the block maximum keep 13 fraction bits (bfloat16: 7)
    rng = np.random.default_rng(5)
    x = np.float32(rng.uniform(1.0, 2.0, size=4000) * rng.choice([-1, 1], size=4000))
    y = bfp_decode(bfp_encode(x, 16), x.size, 16)
    rel = np.abs(y.astype(np.float64) - x) / np.abs(x.astype(np.float64))
    assert rel.max() <= 2.0 ** -13
