"""Reduced-precision storage formats of the predictor matrix X.

Test infrastructure only (see ``oracle/__init__.py``).  The paper computes in
FP32 (Sec. 3.1); the BF16 and per-column-scaled FP8 E4M3 storage of X are the
precision variants of the benchmark workloads.  Defined here from the formats
themselves, with no GPU conversion routine involved:

* BF16: the top 16 bits of the IEEE binary32 pattern after round-to-nearest-
  even on the 16 dropped bits.
* FP8 E4M3 (OCP 8-bit floating point): 1 sign, 4 exponent (bias 7) and 3
  mantissa bits, subnormals at exponent field 0, no infinities, S.1111.111 is
  NaN, largest finite 448.  Per column j the scale is s_j = max_i |x_ij| / 448
  in FP32 (s_j = 1 for an all-zero column); x_ij / s_j (FP32 division) is
  rounded to nearest, ties to even mantissa, saturating at +-448.
  Then X B = X_q (diag(s) B) and X^T R = diag(s) X_q^T R.
"""
import numpy as np

FP8_MAX = 448.0


def bf16_bits(x):
    """uint16 BF16 patterns of float32 values (round to nearest even; finite inputs)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bias = np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))
    return ((b + bias) >> np.uint64(16)).astype(np.uint16)


def bf16_decode(bits):
    """float32 values of uint16 BF16 patterns."""
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def bf16_round(x):
    """x rounded to BF16, returned as float32."""
    return bf16_decode(bf16_bits(x))


def e4m3_table():
    """float64 value of every one of the 256 E4M3 codes (NaN for the two NaN codes)."""
    vals = np.empty(256)
    for code in range(256):
        sign = -1.0 if code & 0x80 else 1.0
        e = (code >> 3) & 0xF
        m = code & 0x7
        if e == 0xF and m == 0x7:
            vals[code] = np.nan
        elif e == 0:
            vals[code] = sign * (m / 8.0) * 2.0 ** (-6)
        else:
            vals[code] = sign * (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return vals


def e4m3_encode(v):
    """uint8 codes of float32 values: nearest E4M3 value, ties to the even
    (low mantissa bit 0) code, saturating to +-448.  E4M3 is sign-magnitude
    with a negative zero (code 0x80); as in IEEE 754 conversions, a result
    that rounds to zero keeps the operand's sign."""
    v = np.asarray(v, dtype=np.float64)
    table = e4m3_table()
    pos_codes = np.arange(0, 0x7F)                       # 0x00..0x7E: +0 .. +448
    pos_vals = table[pos_codes]
    a = np.minimum(np.abs(v), FP8_MAX)
    idx = np.searchsorted(pos_vals, a, side="left")      # pos_vals[idx-1] < a <= pos_vals[idx]
    idx = np.clip(idx, 1, len(pos_vals) - 1)
    lo, hi = pos_vals[idx - 1], pos_vals[idx]
    take_hi = (a - lo) > (hi - a)
    tie = (a - lo) == (hi - a)
    hi_even = (pos_codes[idx] & 1) == 0
    take_hi = take_hi | (tie & hi_even)
    code = np.where(take_hi, pos_codes[idx], pos_codes[idx - 1])
    code = np.where(a == 0.0, 0, code)
    sign = np.signbit(v).astype(np.int64) << 7
    return (code | sign).astype(np.uint8)


def e4m3_decode(codes):
    return e4m3_table()[np.asarray(codes, dtype=np.uint8)]


def fp8_column_scales(X):
    """s_j = max_i |x_ij| / 448 in FP32, 1 for an all-zero column (or n = 0)."""
    X = np.asarray(X, dtype=np.float32)
    if X.shape[0] == 0:
        return np.ones(X.shape[1], dtype=np.float32)
    amax = np.abs(X).max(axis=0).astype(np.float32)
    s = (amax / np.float32(FP8_MAX)).astype(np.float32)
    return np.where(amax == 0.0, np.float32(1.0), s).astype(np.float32)


def fp8_quantize(X):
    """(codes uint8 n x p, scales float32 p) of a float32 matrix."""
    X = np.asarray(X, dtype=np.float32)
    s = fp8_column_scales(X)
    v = (X / s[None, :]).astype(np.float32)
    return e4m3_encode(v), s


def fp8_dequantize(codes, scales):
    """float64 matrix X_q diag(s) that the FP8 storage stands for."""
    return e4m3_decode(codes) * np.asarray(scales, dtype=np.float64)[None, :]
