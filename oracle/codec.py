"""Low-precision storage of hierarchical deltas (oracle; test infrastructure only).

Sect. 5 of the paper stores the deltas A_hat, P_hat compressed per vertex (the
bpa codec, exponent byte + integer mantissa, chosen against a threshold).  The
build turns that idea into a dtype: per vertex and operator one FP32 scale
s = fl32(max_k |delta_k|) and codes q_k = RNE_{bf16|fp16}(delta_k / s), the
quotient formed in FP64 and rounded once to the 16-bit format.  Decoding is
fl32(float(q_k) * s) in FP32 arithmetic.  A vertex whose deltas are all zero
gets s = 0 and zero codes ("marked, nothing stored" in the paper's words).

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
