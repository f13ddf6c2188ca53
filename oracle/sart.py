"""Oracle SART-type iteration on the two split systems (FP64).

The paper names SART as the accepted iterative method (Section 1, reference
[001], Andersen and Kak). It does not state the update rule. This oracle uses
the simultaneous form: every ray of a system contributes to one update per
iteration. The sums use absolute values, because the split matrix A1 has
negative entries.

For one system B f = q (either (A1, p1) or (A2, p2)):

    R_i = sum_j |b_ij|,   C_j = sum_i |b_ij|
    1/R_i := 0 if R_i = 0,   1/C_j := 0 if C_j = 0
    r^k = q - B f^k
    u^k_i = r^k_i / R_i
    f^{k+1}_j = f^k_j + lambda (sum_i b_ij u^k_i) / C_j

The two systems iterate independently (Theorem 1). One joint stopping test
couples them:

    rho_k = sqrt(||r1^k||^2 + ||r2^k||^2) / sqrt(||p1||^2 + ||p2||^2)

Because ||r1||^2 + ||r2||^2 = 2 ||A f - p||^2 for the recombined f (Eq. 5),
rho_k equals the full system's relative residual ||A f^k - p|| / ||p||.

For k = 0, 1, ..., max_iters the oracle computes r^k. It stops at the first k
with rho_k <= tol, or at k = max_iters, and returns f^k with iterations = k.
The update is skipped on the stopping pass. The iteration is linear, so no
clipping is applied.

Two independent implementations are provided: ``split_sart`` (SciPy sparse)
and ``split_sart_dense`` (dense NumPy). They must agree to rounding.

This module is test infrastructure: see the package docstring.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def normalisers(B):
    """Return the absolute row sums R and column sums C of B (FP64)."""
    Babs = abs(sp.csr_matrix(B, dtype=float))
    R = np.asarray(Babs.sum(axis=1)).ravel()
    C = np.asarray(Babs.sum(axis=0)).ravel()
    return R, C


def _safe_inv(x):
    out = np.zeros_like(x)
    nz = x != 0
    out[nz] = 1.0 / x[nz]
    return out


def split_sart(A1, A2, p1, p2, lam: float, max_iters: int, tol: float = 0.0,
               f1_0=None, f2_0=None, record: bool = False):
    """Run SART on both split systems with the joint stopping rule.

    Returns a dict with keys f1, f2, iters, rho and, if ``record`` is set,
    rho_hist.
    """
    A1 = sp.csr_matrix(A1, dtype=float)
    A2 = sp.csr_matrix(A2, dtype=float)
    p1 = np.asarray(p1, dtype=float)
    p2 = np.asarray(p2, dtype=float)
    R1, C1 = normalisers(A1)
    R2, C2 = normalisers(A2)
    iR1, iC1, iR2, iC2 = _safe_inv(R1), _safe_inv(C1), _safe_inv(R2), _safe_inv(C2)
    A1t = A1.T.tocsr()
    A2t = A2.T.tocsr()
    f1 = np.zeros(A1.shape[1]) if f1_0 is None else np.array(f1_0, dtype=float)
    f2 = np.zeros(A2.shape[1]) if f2_0 is None else np.array(f2_0, dtype=float)
    pnorm = np.sqrt(p1 @ p1 + p2 @ p2)
    hist = []
    k = 0
    while True:
        r1 = p1 - A1 @ f1
        r2 = p2 - A2 @ f2
        rho = np.sqrt(r1 @ r1 + r2 @ r2) / pnorm if pnorm > 0 else 0.0
        hist.append(rho)
        if rho <= tol or k == max_iters:
            break
        f1 = f1 + lam * (A1t @ (r1 * iR1)) * iC1
        f2 = f2 + lam * (A2t @ (r2 * iR2)) * iC2
        k += 1
    out = {"f1": f1, "f2": f2, "iters": k, "rho": rho}
    if record:
        out["rho_hist"] = np.array(hist)
    return out


def sart_fixed(B, q, lam: float, iters: int, f0=None):
    """SART on one split system for a fixed number of iterations (no stop test).

    This is one of the two independent solves that the method runs in parallel
    (Section 2): with tol = 0 the joint stopping rule never fires, so split_sart
    is exactly this function applied to (A1, p1) and to (A2, p2).
    """
    B = sp.csr_matrix(B, dtype=float)
    q = np.asarray(q, dtype=float)
    R, C = normalisers(B)
    iR, iC = _safe_inv(R), _safe_inv(C)
    Bt = B.T.tocsr()
    f = np.zeros(B.shape[1]) if f0 is None else np.array(f0, dtype=float)
    for _ in range(iters):
        f = f + lam * (Bt @ ((q - B @ f) * iR)) * iC
    return f


def split_sart_dense(A1, A2, p1, p2, lam: float, max_iters: int, tol: float = 0.0,
                     f1_0=None, f2_0=None):
    """Dense matrix form of ``split_sart``, written independently as a cross-check.

    Each system is iterated as f <- f + lam diag(1/C) B^T diag(1/R) (q - B f).
    """
    def prep(B):
        B = B.toarray() if sp.issparse(B) else np.asarray(B, dtype=float)
        R = np.abs(B).sum(axis=1)
        C = np.abs(B).sum(axis=0)
        DR = np.diag([0.0 if x == 0 else 1.0 / x for x in R])
        DC = np.diag([0.0 if x == 0 else 1.0 / x for x in C])
        return B, DC @ B.T @ DR

    B1, G1 = prep(A1)
    B2, G2 = prep(A2)
    q1 = np.asarray(p1, dtype=float)
    q2 = np.asarray(p2, dtype=float)
    x1 = np.zeros(B1.shape[1]) if f1_0 is None else np.array(f1_0, dtype=float)
    x2 = np.zeros(B2.shape[1]) if f2_0 is None else np.array(f2_0, dtype=float)
    den = np.linalg.norm(np.concatenate([q1, q2]))
    for k in range(max_iters + 1):
        e1 = q1 - B1 @ x1
        e2 = q2 - B2 @ x2
        rho = np.linalg.norm(np.concatenate([e1, e2])) / den if den > 0 else 0.0
        if rho <= tol or k == max_iters:
            return {"f1": x1, "f2": x2, "iters": k, "rho": rho}
        x1 = x1 + lam * (G1 @ e1)
        x2 = x2 + lam * (G2 @ e2)
    raise AssertionError("unreachable")


def sart_limit(B, q):
    """Return the limit of SART from f0 = 0 for 0 < lambda < 2.

    With g = C^{1/2} f, the iteration is Landweber's on
    (R^{-1/2} B C^{-1/2}) g = R^{-1/2} q, whose operator norm is at most 1 by
    the Schur test. From g0 = 0, Landweber converges to the minimum-norm
    least-squares solution. So the SART limit is
    f* = C^{-1/2} pinv(R^{-1/2} B C^{-1/2}) R^{-1/2} q.
    """
    B = B.toarray() if sp.issparse(B) else np.asarray(B, dtype=float)
    R = np.abs(B).sum(axis=1)
    C = np.abs(B).sum(axis=0)
    rh = np.array([0.0 if x == 0 else 1.0 / np.sqrt(x) for x in R])
    ch = np.array([0.0 if x == 0 else 1.0 / np.sqrt(x) for x in C])
    Bt = rh[:, None] * B * ch[None, :]
    return ch * (np.linalg.pinv(Bt) @ (rh * np.asarray(q, dtype=float)))


def scaled_operator_norm(B, iters: int = 200, seed: int = 0) -> float:
    """Return ||R^{-1/2} B C^{-1/2}||_2, estimated by power iteration.

    The Schur test bounds it by 1, which is what makes 0 < lambda < 2 converge.
    """
    B = sp.csr_matrix(B, dtype=float)
    R, C = normalisers(B)
    rh = np.where(R > 0, 1.0 / np.sqrt(np.where(R > 0, R, 1.0)), 0.0)
    ch = np.where(C > 0, 1.0 / np.sqrt(np.where(C > 0, C, 1.0)), 0.0)
    x = np.random.default_rng(seed).standard_normal(B.shape[1])
    s = 0.0
    for _ in range(iters):
        y = rh * (B @ (ch * x))
        x = ch * (B.T @ (rh * y))
        s = np.linalg.norm(x)
        if s == 0:
            return 0.0
        x /= s
    return float(np.sqrt(s))
