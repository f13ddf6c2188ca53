"""Oracle for reduced-precision storage of the split matrices (BF16 / FP16 with per-row scales).

The paper fixes no precision. This storage rule is a design choice of the
library; the oracle states it independently.

Storage of one split matrix B (A1 or A2), row by row:
- scale: s_i = fl32(max_j |b_ij|), the FP32 rounding of the row maximum. An
  all-zero row gets s_i = 0 and codes 0.
- codes: q_ij = rne_t(fl32(b_ij) / s_i). The division is an IEEE FP32
  division, rounded to nearest. rne_t rounds the FP32 quotient to nearest
  even in the target format t (bfloat16: 8 significant bits; binary16:
  11 significant bits).
- dequantised matrix: B^_ij = s_i q_ij. It is exact in FP64, because the
  product of a 24-bit and an 11-bit significand fits in 53 bits.

The solve on stored values is then SART on B^: R and C come from |B^| in FP64
(see ``oracle.sart``).

This module is test infrastructure: see the package docstring.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def round_bf16(x32: np.ndarray) -> np.ndarray:
    """Round FP32 values to bfloat16, nearest even. Returns the value as FP32.

    bfloat16 keeps the upper 16 bits of the FP32 encoding. Round to nearest even
    adds 0x7FFF plus the lowest kept bit, then truncates. Inputs here are finite.
    """
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def round_f16(x32: np.ndarray) -> np.ndarray:
    """Round FP32 values to IEEE binary16, nearest even. Returns the value as FP32."""
    return np.asarray(x32, dtype=np.float32).astype(np.float16).astype(np.float32)


def quantise_rows(B, fmt: str):
    """Return (scales float32[rows], codes CSR float64, B_hat CSR float64) for B.

    B is an (M/2) x (N/2) split matrix; ``fmt`` is 'bf16' or 'f16'. The CSR
    outputs keep B's stored pattern.
    """
    if fmt not in ("bf16", "f16"):
        raise ValueError(fmt)
    rnd = round_bf16 if fmt == "bf16" else round_f16
    B = sp.csr_matrix(B, dtype=float)
    B.sort_indices()
    rows = B.shape[0]
    scales = np.zeros(rows, dtype=np.float32)
    codes = np.zeros(B.nnz, dtype=np.float64)
    for i in range(rows):
        a, b = B.indptr[i], B.indptr[i + 1]
        if a == b:
            continue
        v32 = B.data[a:b].astype(np.float32)
        s = np.float32(np.max(np.abs(B.data[a:b])))
        scales[i] = s
        if s == 0:
            continue
        q = (v32 / s).astype(np.float32)  # IEEE FP32 division, round to nearest
        codes[a:b] = rnd(q).astype(np.float64)
    C = sp.csr_matrix((codes, B.indices.copy(), B.indptr.copy()), shape=B.shape)
    Bhat = sp.csr_matrix((codes * np.repeat(scales.astype(np.float64), np.diff(B.indptr)),
                          B.indices.copy(), B.indptr.copy()), shape=B.shape)
    return scales, C, Bhat
