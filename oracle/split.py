"""Oracle for the split and the recombination (FP64).

- ``fold_matrix``: the fold formulas after Eq. (4), written out literally on
  the full matrix A (M x N):
      w1_ij = w_ij - w_{M-i+1,j},  w2_ij = w_ij + w_{M-i+1,j},  i <= M/2, j <= N/2.
- ``fold_rhs``: the matching fold of p:
      p1_i = p_i - p_{M-i+1},  p2_i = p_i + p_{M-i+1}.
- ``recombine``: Theorem 1, Eq. (5):
      f_j = (f2_j + f1_j)/2,  f_{N-j+1} = (f2_j - f1_j)/2.
- ``fold_image``: the vectors of the proof of Theorem 1:
      f1_j = f_j - f_{N-j+1},  f2_j = f_j + f_{N-j+1},
  restricted to j <= N/2.
- ``min_norm``: the normal pseudo-solution used in Theorem 2. It is the
  minimum-norm least-squares solution, computed through the Moore-Penrose
  pseudo-inverse.

Everything uses 0-based indices. The paper's i <-> M-i+1 becomes
i <-> M-1-i, and j <-> N-j+1 becomes j <-> N-1-j.

This module is test infrastructure: see the package docstring.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _check_even(M: int, N: int) -> None:
    if M % 2 or N % 2:
        raise ValueError("M and N must be even (Section 2)")


def fold_matrix(A):
    """Return (A1, A2), each M/2 x N/2, from the full A by the fold formulas after Eq. (4).

    The output type follows A: dense in gives dense out, sparse in gives CSR.
    """
    M, N = A.shape
    _check_even(M, N)
    Mh, Nh = M // 2, N // 2
    mirror_rows = M - 1 - np.arange(Mh)  # row M-i+1 for i = 1..M/2
    if sp.issparse(A):
        A = sp.csr_matrix(A)
        top = A[:Mh][:, :Nh]
        bot = A[mirror_rows][:, :Nh]
        return sp.csr_matrix(top - bot), sp.csr_matrix(top + bot)
    A = np.asarray(A, dtype=float)
    top = A[:Mh, :Nh]
    bot = A[mirror_rows, :Nh]
    return top - bot, top + bot


def folded_pattern_size(A) -> int:
    """Return the number of (i, j), i < M/2 and j < N/2, where w_ij or w_{M-1-i,j} is stored.

    This is the size of the union pattern of A1 and A2.
    """
    A = sp.csr_matrix(A)
    M, N = A.shape
    Mh, Nh = M // 2, N // 2
    top = A[:Mh][:, :Nh].copy()
    bot = A[M - 1 - np.arange(Mh)][:, :Nh].copy()
    top.data[:] = 1.0
    bot.data[:] = 1.0
    return int((top + bot).nnz)


def fold_rhs(p):
    """Return (p1, p2), each of length M/2, from the fold formulas after Eq. (4)."""
    p = np.asarray(p, dtype=float)
    M = p.shape[0]
    if M % 2:
        raise ValueError("M must be even (Section 2)")
    Mh = M // 2
    mirror = p[M - 1 - np.arange(Mh)]
    return p[:Mh] - mirror, p[:Mh] + mirror


def recombine(f1, f2):
    """Apply Theorem 1, Eq. (5): rebuild f[N] from f1, f2 of length N/2."""
    f1 = np.asarray(f1, dtype=float)
    f2 = np.asarray(f2, dtype=float)
    Nh = f1.shape[0]
    N = 2 * Nh
    f = np.empty(N)
    j = np.arange(Nh)
    f[j] = (f2 + f1) / 2.0
    f[N - 1 - j] = (f2 - f1) / 2.0
    return f


def fold_image(f):
    """Fold an image as in the proof of Theorem 1.

    Returns (f1, f2) with f1_j = f_j - f_{N-1-j} and f2_j = f_j + f_{N-1-j}, for
    j < N/2.
    """
    f = np.asarray(f, dtype=float)
    N = f.shape[0]
    if N % 2:
        raise ValueError("N must be even (Section 2)")
    Nh = N // 2
    mirror = f[N - 1 - np.arange(Nh)]
    return f[:Nh] - mirror, f[:Nh] + mirror


def min_norm(A, p):
    """Return the normal pseudo-solution: the minimum-norm least-squares solution of A f = p (Theorem 2)."""
    A = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=float)
    return np.linalg.pinv(A) @ np.asarray(p, dtype=float)


def relative_residual(A, f, p) -> float:
    """Return ||A f - p||_2 / ||p||_2 for the full system (Eq. 1)."""
    p = np.asarray(p, dtype=float)
    r = A @ np.asarray(f, dtype=float) - p
    return float(np.linalg.norm(r) / np.linalg.norm(p))
