"""Low-precision storage of hierarchical deltas (oracle; test infrastructure only).

Sect. 5 of the paper stores the deltas A_hat, P_hat compressed per vertex (the
bpa codec, exponent byte + integer mantissa, chosen against a threshold).  The
build turns that idea into a dtype: per vertex and operator one FP32 scale
s = fl32(max_k |delta_k|) and codes q_k = RNE_{bf16|fp16}(delta_k / s), the
quotient formed in FP64 and rounded once to the 16-bit format.  Decoding is
fl32(float(q_k) * s) in FP32 arithmetic.  A vertex whose deltas are all zero
gets s = 0 and zero codes ("marked, nothing stored" in the paper's words).

Promotion (the dtype counterpart of the paper's per-vertex choice of bpa against
eps_mf, Sect. 5): reconstructing A = A_redisc + A_hat cancels where the delta is as
large as the operator itself.  A vertex whose row's worst 16-bit rounding, half a
unit of the format relative to the scale (h_fmt s: 2^-9 s for bf16, 2^-12 s for
fp16), could exceed 2^-8 of the reconstructed diagonal |A_vv| keeps FP32 codes
instead: each entry's fl32(delta_k / s) split into its high and low 16 bits (the
code plane and a second plane), and the sign bit of the stored scale set as the
flag.  The comparison h_fmt s > 2^-8 |A_vv| is exact in FP64 (products by powers
of two), i.e. s > 2 |A_vv| (bf16), s > 16 |A_vv| (fp16).

The rounding below is written from the IEEE 754 definition of the two formats:
bf16 = 1 sign, 8 exponent, 7 fraction bits (min normal exponent -126);
fp16 = 1 sign, 5 exponent, 10 fraction bits (min normal exponent -14).
"""
from __future__ import annotations

import numpy as np

_FORMATS = {
    "bf16": dict(frac=7, emin=-126),
    "fp16": dict(frac=10, emin=-14),
}


def round_to_format(t: np.ndarray, fmt: str) -> np.ndarray:
    """Round FP64 values to the nearest (ties to even) value of the 16-bit format, returned as FP64."""
    p = _FORMATS[fmt]
    t = np.asarray(t, dtype=np.float64)
    _, e = np.frexp(t)  # t = f * 2^e, f in [0.5, 1)
    E = np.maximum(e - 1, p["emin"])
    quantum = np.ldexp(1.0, E - p["frac"])
    out = np.rint(t / quantum) * quantum
    return np.where(t == 0.0, 0.0, out)


def to_bits(x: np.ndarray, fmt: str) -> np.ndarray:
    """Bit patterns (uint16) of values already representable in the format."""
    x = np.asarray(x, dtype=np.float64)
    if fmt == "bf16":
        return (x.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    return x.astype(np.float16).view(np.uint16)


def from_bits(b: np.ndarray, fmt: str) -> np.ndarray:
    b = np.asarray(b, dtype=np.uint16)
    if fmt == "bf16":
        return (b.astype(np.uint32) << 16).view(np.float32)
    return b.view(np.float16).astype(np.float32)


def encode(delta: np.ndarray, fmt: str = "bf16"):
    """delta (n, K) FP64 -> (codes (n, K) uint16, scale (n,) float32)."""
    delta = np.asarray(delta, dtype=np.float64)
    m = np.abs(delta).max(axis=1)
    s = m.astype(np.float32)
    sd = s.astype(np.float64)
    safe = np.where(sd > 0.0, sd, 1.0)
    t = np.where(sd[:, None] > 0.0, delta / safe[:, None], 0.0)
    q = round_to_format(t, fmt)
    return to_bits(q, fmt), s


def decode(codes: np.ndarray, scale: np.ndarray, fmt: str = "bf16") -> np.ndarray:
    """FP32 deltas: fl32(float(q) * s)."""
    return (from_bits(codes, fmt) * scale.astype(np.float32)[:, None]).astype(np.float32)


# half a unit of the format relative to the scale: the largest rounding error of a
# code, |decoded - delta| <= HALF_UNIT[fmt] * s, for every entry of a row
HALF_UNIT = {"bf16": 2.0 ** -9, "fp16": 2.0 ** -12}
# a vertex is promoted when that error could exceed this fraction of |A_vv|
PROMOTE_REL = 2.0 ** -8


def promoted(scale: np.ndarray, diag: np.ndarray, fmt: str = "bf16") -> np.ndarray:
    """Promotion flag per row: h_fmt * s > 2^-8 * |A_vv| (s the FP32 scale, A_vv FP64)."""
    s = np.abs(np.asarray(scale, dtype=np.float32).astype(np.float64))
    return s * HALF_UNIT[fmt] > PROMOTE_REL * np.abs(np.asarray(diag, dtype=np.float64))


def encode_promoting(delta: np.ndarray, diag: np.ndarray, fmt: str = "bf16"):
    """delta (n, K) FP64 and the reconstructed diagonals A_vv (n,) FP64 ->
    (codes (n, K) uint16, lo (n, K) uint16, scale (n,) float32 with the flag as its sign).

    Rows that are not promoted get the plain encoding (lo = 0, scale = +s); promoted rows
    get the FP32 bit pattern of fl32(delta_k / s) (quotient in FP64, rounded once to
    nearest even FP32) as high half in codes and low half in lo, and scale = -s."""
    delta = np.asarray(delta, dtype=np.float64)
    codes, s = encode(delta, fmt)
    p = promoted(s, diag, fmt)
    lo = np.zeros_like(codes)
    if p.any():
        sd = s[p].astype(np.float64)
        t = delta[p] / sd[:, None]
        bits = t.astype(np.float32).view(np.uint32)
        codes = codes.copy()
        codes[p] = (bits >> 16).astype(np.uint16)
        lo[p] = (bits & 0xFFFF).astype(np.uint16)
    scale = np.where(p, -s, s).astype(np.float32)
    return codes, lo, scale


def decode_promoting(codes: np.ndarray, lo: np.ndarray, scale: np.ndarray, fmt: str = "bf16") -> np.ndarray:
    """FP32 deltas of encode_promoting: fl32(value(codes[, lo]) * |scale|), the value read
    as FP32 from (codes << 16 | lo) on rows whose scale has its sign bit set."""
    scale = np.asarray(scale, dtype=np.float32)
    flag = np.signbit(scale)
    s = np.abs(scale)
    out = decode(codes, s, fmt)
    if flag.any():
        full = ((codes[flag].astype(np.uint32) << 16) | lo[flag].astype(np.uint32)).view(np.float32)
        out[flag] = (full * s[flag][:, None]).astype(np.float32)
    return out

