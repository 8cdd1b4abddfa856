"""Block floating-point (BFP) codec of Section III-C-3 (TEST INFRASTRUCTURE ONLY).

Four FP32 values form a block of N_bits = 4 n_bits bits.  The low 8 bits hold a
shared biased exponent e = e_max + 127, with e_max the integer such that
2^(e_max - 1) <= max_i |x_i| < 2^e_max; e = 0 marks a block whose four values are
all zero.  The remaining N_bits - 8 bits hold four signed coefficients of
v_bits = n_bits - 2 bits each (two's complement, the dropped high bits being
copies of the sign bit):

    q_i = round(x_i * 2^(v_bits - 1 - e_max)),  clamped above at 2^(v_bits - 1) - 1,
    decoded value  x~_i = q_i * 2^(e_max - v_bits + 1).

n_bits = 16, 12, 10 give v_bits = 14, 10, 8 and blocks of 8, 6 and 5 bytes.

Readings where the section is silent (each listed in the design notes):
- round(): to nearest, ties to even;
- coefficient i (i = 0..3, in the order of the values) occupies bits
  [8 + i v_bits, 8 + (i + 1) v_bits) of the block word, and the word is stored
  little-endian in N_bits / 8 consecutive bytes; block b starts at byte b N_bits / 8;
- a block whose largest magnitude is subnormal (below 2^-126) uses e_max = -126,
  the smallest exponent whose biased value (1) differs from the zero-block mark;
- n values with n not a multiple of four: the last block is completed with zeros,
  and decoding returns the first n values;
- in the top exponent (e_max = 128) the coefficient -2^(v_bits - 1) would decode to
  -2^128, which FP32 cannot hold; there q is also clamped below, at
  -(2^(v_bits - 1) - 1), so that every decoded value is finite (elsewhere the range
  is the section's, [-2^(v_bits - 1), 2^(v_bits - 1) - 1]);
- inputs are finite: the section defines no code for Inf or NaN.

Every value is handled in float64 here, where float32 inputs, the scaling by a
power of two and the decoded values are all exact; only round() rounds.

Parity: pinned in tests/test_oracle_bfp.py by hand-derived words at each rate, by
brute force over every coefficient at v_bits = 8, by the exponent definition
checked with an integer search, by the half-quantum error bound, by ties-to-even
cases, by exact round trips of values on the quantisation grid, and by the
zero-block, subnormal-block and largest-float cases.
"""
from __future__ import annotations

import math

import numpy as np

RATES = (16, 12, 10)


def bfp_layout(nbits: int):
    """(v_bits, bytes per four-value block) for the rate n_bits."""
    if nbits not in RATES:
        raise ValueError(f"n_bits must be one of {RATES}")
    return nbits - 2, (4 * nbits) // 8


def bfp_stream_bytes(n: int, nbits: int) -> int:
    """Bytes of the compressed stream of n values."""
    _, nbytes = bfp_layout(nbits)
    return ((n + 3) // 4) * nbytes


def shared_exponent(m: float) -> int:
    """e_max with 2^(e_max - 1) <= m < 2^e_max for m > 0, at least -126."""
    _, ex = math.frexp(m)          # m = f 2^ex with 1/2 <= f < 1
    return max(ex, -126)


def bfp_encode_block(x4, nbits: int) -> bytes:
    """Encode four float32 values into one block (N_bits / 8 bytes)."""
    v, nbytes = bfp_layout(nbits)
    x = [float(np.float32(t)) for t in x4]
    m = max(abs(t) for t in x)
    if m == 0.0:
        return bytes(nbytes)
    emax = shared_exponent(m)
    qmax = 2 ** (v - 1) - 1
    word = emax + 127
    for i, t in enumerate(x):
        q = int(np.rint(t * 2.0 ** (v - 1 - emax)))   # exact scaling, round half to even
        q = min(q, qmax)
        if emax == 128:
            q = max(q, -qmax)
        word |= (q % (1 << v)) << (8 + i * v)         # low v bits, two's complement
    return word.to_bytes(nbytes, "little")


def bfp_decode_block(block: bytes, nbits: int) -> np.ndarray:
    """Decode one block into four float32 values."""
    v, nbytes = bfp_layout(nbits)
    if len(block) != nbytes:
        raise ValueError("block has the wrong size")
    word = int.from_bytes(bytes(block), "little")
    e = word & 0xFF
    out = np.zeros(4, dtype=np.float32)
    if e == 0:
        return out
    emax = e - 127
    for i in range(4):
        field = (word >> (8 + i * v)) & ((1 << v) - 1)
        q = field - (1 << v) if field >= (1 << (v - 1)) else field   # restore the sign bits
        out[i] = np.float32(q * 2.0 ** (emax - v + 1))
    return out


def bfp_encode(x, nbits: int) -> np.ndarray:
    """Encode a float32 vector into the compressed byte stream (uint8 array)."""
    x = np.asarray(x, dtype=np.float32).ravel()
    _, nbytes = bfp_layout(nbits)
    nblk = (x.size + 3) // 4
    out = np.zeros(nblk * nbytes, dtype=np.uint8)
    for b in range(nblk):
        blk = np.zeros(4, dtype=np.float32)
        part = x[4 * b:4 * b + 4]
        blk[:part.size] = part
        out[b * nbytes:(b + 1) * nbytes] = np.frombuffer(bfp_encode_block(blk, nbits), dtype=np.uint8)
    return out


def bfp_decode(stream, n: int, nbits: int) -> np.ndarray:
    """Decode the first n values of a compressed byte stream."""
    s = np.asarray(stream, dtype=np.uint8).ravel()
    _, nbytes = bfp_layout(nbits)
    nblk = (n + 3) // 4
    if s.size < nblk * nbytes:
        raise ValueError("stream too short")
    out = np.zeros(nblk * 4, dtype=np.float32)
    for b in range(nblk):
        out[4 * b:4 * b + 4] = bfp_decode_block(s[b * nbytes:(b + 1) * nbytes].tobytes(), nbits)
    return out[:n]
