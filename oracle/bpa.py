"""The paper's byte-per-attribute (bpa) codec of the hierarchical deltas (oracle; test
infrastructure only).

Sect. 5 stores each operator of a vertex (A_hat with 3^d entries, P_hat = R_hat with
5^d entries) either not at all (bpa = 0: every entry is dropped to zero) or entry by
entry as f_bpa = m * 2^e: one exponent byte e (a C ``char``) followed by an integer m
in bpa - 1 bytes.  Per operator the smallest bpa in {0, 2, 3, ..., 8} is chosen for
which every entry x satisfies |f_bpa(x) - x| <= eps_mf.

Readings where the paper is silent (each also listed with the design notes):

* The sign of m: the paper has m a natural number; the entries of a delta take both
  signs, so m is stored sign-magnitude: the top bit of its bpa - 1 bytes is the sign,
  the other M = 8 (bpa - 1) - 1 bits hold |m|.
* The choice of e for one entry: the smallest exponent whose |m| = round(|x| 2^-e)
  (round half to even) fits in M bits, i.e. e = E - M with |x| = f 2^E, f in [0.5, 1);
  a rounding that carries to 2^M takes e + 1 and 2^(M-1).  x = 0 is stored as e = 0,
  m = 0.  An exponent below -128 is clamped to -128 (m then holds what is left, maybe
  0); an exponent above 127 cannot be stored and fails that bpa.
* The byte layout: e first, then m little-endian; the entries of one operator are
  consecutive, the operators of consecutive vertices follow each other (one byte
  stream per operator kind and level), and a per-vertex record holds bpa and the
  stream offset.  The tolerance test is the FP64 expression |ldexp(m, e) - |x|| <=
  eps_mf (decoded magnitude against |x|, the sign being exact).

With M = 55 bits at bpa = 8 every double is stored exactly (barring the exponent clamp
far below any delta), so a choice always exists for finite entries.
"""
from __future__ import annotations

import numpy as np

BPA_CHOICES = (0, 2, 3, 4, 5, 6, 7, 8)


def mantissa_bits(bpa: int) -> int:
    """Magnitude bits M of the integer part at a given bpa (one bit of bpa-1 bytes is the sign)."""
    return 8 * (bpa - 1) - 1


def encode_entry(x: float, bpa: int):
    """(e, sign, |m|) of one entry at bpa >= 2, or None if its exponent does not fit a byte."""
    x = float(x)
    if x == 0.0:
        return 0, 0, 0
    M = mantissa_bits(bpa)
    a = abs(x)
    _, E = np.frexp(a)  # a = f 2^E, f in [0.5, 1)
    e = int(E) - M
    m = int(np.rint(np.ldexp(a, -e)))
    if m == (1 << M):  # rounding carried into the next power of two
        m >>= 1
        e += 1
    if e < -128:
        e = -128
        m = int(np.rint(np.ldexp(a, 128)))
    if e > 127:
        return None
    return e, 1 if x < 0.0 else 0, m


def decode_entry(e: int, sign: int, m: int) -> float:
    """f_bpa = (-1)^sign m 2^e in FP64 (exact: m has at most 53 significant bits)."""
    v = float(np.ldexp(float(m), e))
    return -v if sign else v


def entry_error(x: float, bpa: int) -> float:
    """|f_bpa(x) - x| as the FP64 expression of the tolerance test (inf if unrepresentable)."""
    if bpa == 0:
        return abs(float(x))
    enc = encode_entry(x, bpa)
    if enc is None:
        return float("inf")
    e, _, m = enc
    return abs(float(np.ldexp(float(m), e)) - abs(float(x)))


def choose_bpa(row: np.ndarray, eps_mf: float) -> int:
    """Smallest bpa of {0, 2, ..., 8} that stores every entry of the operator within eps_mf."""
    row = np.asarray(row, dtype=np.float64)
    if not np.all(np.isfinite(row)):
        raise ValueError("non-finite delta")
    for bpa in BPA_CHOICES:
        if all(entry_error(x, bpa) <= eps_mf for x in row):
            return bpa
    raise ValueError("delta not representable in the bpa format")


def entry_bytes(x: float, bpa: int) -> bytes:
    """The bpa bytes of one entry: e (two's complement), then sign-magnitude m little-endian."""
    e, sign, m = encode_entry(x, bpa)
    word = m | (sign << mantissa_bits(bpa))
    return bytes([e & 0xFF]) + word.to_bytes(bpa - 1, "little")


def encode_rows(rows: np.ndarray, eps_mf: float):
    """Operators (n, K) FP64 -> (bpa (n,) int, offset (n,) int, stream bytes).

    The stream holds the operators of rows 0, 1, ... one after the other; row i occupies
    bpa_i * K bytes starting at offset_i (the exclusive prefix sum of those sizes)."""
    rows = np.asarray(rows, dtype=np.float64)
    n, K = rows.shape
    bpa = np.zeros(n, dtype=np.int64)
    chunks = []
    for i in range(n):
        b = choose_bpa(rows[i], eps_mf)
        bpa[i] = b
        if b:
            chunks.append(b"".join(entry_bytes(x, b) for x in rows[i]))
    sizes = bpa * K
    offset = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    return bpa, offset, b"".join(chunks)


def decode_rows(bpa: np.ndarray, offset: np.ndarray, stream: bytes, K: int) -> np.ndarray:
    """Inverse of ``encode_rows`` in FP64 (rows with bpa = 0 decode to zero)."""
    n = len(bpa)
    out = np.zeros((n, K), dtype=np.float64)
    for i in range(n):
        b = int(bpa[i])
        if b == 0:
            continue
        M = mantissa_bits(b)
        for k in range(K):
            at = int(offset[i]) + k * b
            e = stream[at] - 256 if stream[at] >= 128 else stream[at]
            word = int.from_bytes(stream[at + 1:at + b], "little")
            out[i, k] = decode_entry(e, word >> M, word & ((1 << M) - 1))
    return out


def records(bpa: np.ndarray, offset: np.ndarray) -> np.ndarray:
    """Per-vertex records as 64-bit words: bpa in bits 0-3, the byte offset above."""
    return (np.asarray(offset, dtype=np.uint64) << np.uint64(4)) | np.asarray(bpa, dtype=np.uint64)
