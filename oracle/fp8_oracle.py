"""FP64 CPU oracle of the FP8 copy of X: OCP FP8 E4M3 codes with one E8M0 (power-of-two) scale per
32 x 32 tile of X, and the monitor sums taken against the dequantised copy.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product path.

The paper works in double precision throughout; the reduced-precision copy of X is a systems
choice on top of the method (the sketch and compression contractions read X only). Definitions:

  E4M3 code    s eeee mmm: exponent bias 7; e = 0 encodes subnormals m/8 * 2^-6; e = 1..15
               encode (1 + m/8) * 2^(e - 7), except s 1111 111 (NaN); no infinities. Largest
               finite magnitude 448 (1111 110), smallest subnormal 2^-9.
  encode(v)    the finite E4M3 value nearest to v, ties to the code with an even mantissa (the
               last mantissa bit 0); magnitudes above 448 saturate to 448 (never reached below);
               the sign bit of v is kept, also when the magnitude rounds to zero.
  tile scale   for the 32 x 32 tile T (edge tiles cover what is left), amax = max |x| over T;
               2^k with k the smallest integer such that amax / 2^k <= 448 (amax = f 2^e with
               f in [0.5, 1): k = e - 9 if f <= 0.875, else e - 8), clamped to the E8M0 range
               [-127, 127] (codes then saturate); k = 0 for an all-zero tile. Stored as the
               E8M0 byte k + 127.
  X_q          encode(x / 2^k) * 2^k entry by entry.
  sums         ||X||^2 and <X - X_q, X> (the BF16 path's monitor correction, with X_q the FP8 copy).

Pins (tests/test_oracle_pins.py): the decode table against values the format definition states
(1.0, 448, 2^-6, 2^-9, NaN), monotonicity of the 127 non-negative finite codes, ties at chosen
midpoints, the scale rule's minimality, and the relative error bound 2^-4 of normal values.
"""
from __future__ import annotations

import numpy as np

__all__ = ["e4m3_decode", "e4m3_encode", "e8m0_tile_exponents", "fp8_quantize", "fp8_dequantize",
           "fp8_layout", "E4M3_MAX"]

E4M3_MAX = 448.0
TILE = 32


def e4m3_decode(codes):
    """Value of each E4M3 code (uint8 array) as float64; NaN for s 1111 111."""
    c = np.asarray(codes, dtype=np.uint8).astype(np.int64)
    s = (c >> 7) & 1
    e = (c >> 3) & 0xF
    m = c & 0x7
    mag = np.where(e == 0, (m / 8.0) * 2.0 ** -6, (1.0 + m / 8.0) * 2.0 ** (e - 7))
    val = np.where(s == 1, -mag, mag)
    return np.where((e == 15) & (m == 7), np.nan, val)


def _positive_table():
    codes = np.arange(0, 127, dtype=np.uint8)          # 0 000 000 .. 0 1111 110
    return codes, e4m3_decode(codes)


def e4m3_encode(v):
    """Nearest E4M3 code to each value of v (float64), ties to an even mantissa, saturating at
    448 in magnitude. Brute force over the 127 non-negative finite codes."""
    v = np.asarray(v, dtype=np.float64)
    codes, vals = _positive_table()
    a = np.minimum(np.abs(v), E4M3_MAX)
    hi = np.clip(np.searchsorted(vals, a, side="left"), 0, len(vals) - 1)   # first vals >= a
    lo = np.clip(hi - 1, 0, len(vals) - 1)
    d_lo = a - vals[lo]
    d_hi = vals[hi] - a
    pick_hi = (d_hi < d_lo) | ((d_hi == d_lo) & ((codes[hi] & 1) == 0) & (hi != lo))
    c = np.where(pick_hi, codes[hi], codes[lo]).astype(np.uint8)
    # the sign bit is kept, also for values that round to zero (and for -0)
    return np.where(np.signbit(v), c | 0x80, c).astype(np.uint8)


def e8m0_tile_exponents(X):
    """k for every 32 x 32 tile of X (ceil(m/32) x ceil(n/32) int array), the scale rule above."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    tm, tn = -(-m // TILE), -(-n // TILE)
    k = np.zeros((tm, tn), dtype=np.int64)
    for a in range(tm):
        for b in range(tn):
            amax = np.max(np.abs(X[a * TILE:(a + 1) * TILE, b * TILE:(b + 1) * TILE]))
            if amax == 0.0:
                continue
            f, e = np.frexp(amax)
            k[a, b] = min(127, max(-127, (e - 9) if f <= 0.875 else (e - 8)))
    return k


def fp8_quantize(X):
    """(codes m x n uint8, k tile exponents) of the definitions above."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    k = e8m0_tile_exponents(X)
    kk = np.repeat(np.repeat(k, TILE, axis=0), TILE, axis=1)[:m, :n]
    codes = e4m3_encode(X * 2.0 ** (-kk))
    return codes, k


def fp8_dequantize(codes, k):
    m, n = codes.shape
    kk = np.repeat(np.repeat(np.asarray(k), TILE, axis=0), TILE, axis=1)[:m, :n]
    return e4m3_decode(codes) * 2.0 ** kk


def fp8_layout(m, n):
    """Byte layout of the library's FP8 copy: (row pitch, offset of the scale bytes, total bytes).
    Rows are padded to a multiple of 16 bytes (zero codes); the E8M0 bytes follow at a 256-byte
    boundary, ceil(m/32) rows of ceil(n/32)."""
    ldq = -(-n // 16) * 16
    off = -(-(m * ldq) // 256) * 256
    return ldq, off, off + (-(-m // TILE)) * (-(-n // TILE))
