"""Oracle for least-squares solves of the split systems through their normal matrices (FP64).

The paper notes (after Eq. 18) that the normal matrix of each split system is
the fold of the full normal matrix: with B = A^T A, the folds of B are
B1 = A1^T A1 and B2 = A2^T A2. Two solvers use it:

- ``cgls``: conjugate gradients on the normal equations A_s^T A_s f = A_s^T p_s,
  run without forming B_s (CGLS, the Hestenes-Stiefel iteration as written
  for least squares). For each system s, from x^0 (zero by default):
      r^0 = p - A x^0,   s^0 = A^T r^0,   d^0 = s^0,   gamma_0 = ||s^0||^2
      for k = 0, 1, ...:
          q^k = A d^k
          alpha_k = gamma_k / ||q^k||^2            (0 when ||q^k|| = 0)
          x^{k+1} = x^k + alpha_k d^k
          r^{k+1} = r^k - alpha_k q^k
          s^{k+1} = A^T r^{k+1}
          gamma_{k+1} = ||s^{k+1}||^2
          beta_k = gamma_{k+1} / gamma_k           (0 when gamma_k = 0)
          d^{k+1} = s^{k+1} + beta_k d^k
  The two systems iterate independently (Theorem 1) under the joint stopping
  rule of the SART solver: rho_k = sqrt(||r1^k||^2 + ||r2^k||^2) / ||p||,
  tested before step k; the solve returns x^k at the first k with
  rho_k <= tol, or at k = max_iters. From x^0 = 0 every iterate lies in the
  row space of A_s, so on a consistent system CGLS tends to the normal
  pseudo-solution of Theorem 2.

- ``direct_solve``: the direct method of Example 2 (Table 1), read as the
  Cholesky factorisation of the normal matrix A^T A followed by two
  triangular solves. ``split_direct_solve`` applies it to A1 and A2 and
  recombines by Theorem 1 (Eq. 5).

This module is test infrastructure: see the package docstring.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import split


def cgls(A1, A2, p1, p2, max_iters: int, tol: float = 0.0, check_every: int = 1, f1_0=None, f2_0=None,
         record: bool = False):
    """CGLS on both split systems with the joint stopping rule.

    Returns a dict with keys f1, f2, iters, rho and, if ``record`` is set,
    rho_hist (rho of every tested iterate).
    """
    mats = [sp.csr_matrix(A1, dtype=float), sp.csr_matrix(A2, dtype=float)]
    qs = [np.asarray(p1, dtype=float), np.asarray(p2, dtype=float)]
    x = [np.zeros(m.shape[1]) if f0 is None else np.array(f0, dtype=float) for m, f0 in zip(mats, (f1_0, f2_0))]
    r = [q - m @ xs for m, q, xs in zip(mats, qs, x)]
    s = [m.T @ rs for m, rs in zip(mats, r)]
    d = [ss.copy() for ss in s]
    gamma = [float(ss @ ss) for ss in s]
    pnorm = np.sqrt(sum(float(q @ q) for q in qs))
    hist = []
    k = 0
    rho = None
    while True:
        if k % check_every == 0 or k == max_iters:
            rho = np.sqrt(sum(float(rs @ rs) for rs in r)) / pnorm if pnorm > 0 else 0.0
            hist.append(rho)
            if rho <= tol or k == max_iters:
                break
        for t in range(2):
            qk = mats[t] @ d[t]
            qq = float(qk @ qk)
            alpha = gamma[t] / qq if qq > 0 else 0.0
            x[t] = x[t] + alpha * d[t]
            r[t] = r[t] - alpha * qk
            s_new = mats[t].T @ r[t]
            g_new = float(s_new @ s_new)
            beta = g_new / gamma[t] if gamma[t] > 0 else 0.0
            d[t] = s_new + beta * d[t]
            gamma[t] = g_new
        k += 1
    out = {"f1": x[0], "f2": x[1], "iters": k, "rho": rho}
    if record:
        out["rho_hist"] = np.array(hist)
    return out


def normal_matrix(A) -> np.ndarray:
    """Return B = A^T A as a dense FP64 array."""
    A = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=float)
    return A.T @ A


def direct_solve(A, p) -> np.ndarray:
    """Least-squares solution of A f = p by the Cholesky factor of A^T A (A of full column rank)."""
    B = normal_matrix(A)
    L = np.linalg.cholesky(B)
    rhs = (A.T @ np.asarray(p, dtype=float)) if not sp.issparse(A) else A.T @ np.asarray(p, dtype=float)
    y = sla.solve_triangular(L, rhs, lower=True)
    return sla.solve_triangular(L.T, y, lower=False)


def split_direct_solve(A, p) -> np.ndarray:
    """Fold A and p (after Eq. 4), solve both systems directly, recombine by Theorem 1 (Eq. 5)."""
    A1, A2 = split.fold_matrix(A)
    p1, p2 = split.fold_rhs(p)
    return split.recombine(direct_solve(A1, p1), direct_solve(A2, p2))
