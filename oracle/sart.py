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

The ordered-subsets form (``os_sart``, with its dense cross-check
``os_sart_dense``) and the projection onto the non-negativity cone
(``cone_project``) follow at the end of the module, with their own notes.

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


# ---------------------------------------------------------------------------
# Ordered subsets and the non-negativity cone.
#
# Andersen and Kak's SART (Section 1, reference [001]) updates the image once
# per projection view. The ordered-subsets form (OS-SART) takes the rows of
# one split system in T disjoint subsets I_0, ..., I_{T-1} and, within one
# iteration, applies for t = 0, 1, ..., T-1 in turn:
#
#     r_t   = q_t - B_t f                      (rows of subset t only)
#     C_t,j = sum_{i in I_t} |b_ij|            (column sums over the subset)
#     f_j  <- f_j + lambda (sum_{i in I_t} b_ij r_i / R_i) / C_t,j
#
# with 1/0 := 0 as before. With one subset holding every row this is exactly
# the simultaneous SART above. For the folded system of a slice, subset t is
# folded view t: rows t nb .. t nb + nb - 1, which carry the rays of sources t
# and K-1-t (a mirror pair of views).
#
# Non-negativity. The image f >= 0 holds iff every voxel pair (j, N-1-j) has
# f_j = (f2_j + f1_j)/2 >= 0 and f_{N-1-j} = (f2_j - f1_j)/2 >= 0 (Eq. 5),
# that is f2_j >= |f1_j|: a cone in the (f1_j, f2_j) plane. The fold
# (a, b) -> (a - b, a + b) is sqrt(2) times a rotation, so the Euclidean
# projection onto that cone is: recombine, clip each of f_j and f_{N-1-j}
# at zero, fold again. It acts on each voxel pair alone.
#
# Stopping: rho_k = ||A f^k - p|| / ||p|| of the iterate after k full sweeps,
# tested when k is a multiple of check_every or k = max_iters, before the
# sweep; the sweep is skipped on the stopping pass. With the cone, the
# projection follows every subset update, and the start itself is projected.
# ---------------------------------------------------------------------------

def cone_project(f1, f2):
    """Project each voxel pair (f1_j, f2_j) onto the cone f2 >= |f1| (image values >= 0, Eq. 5)."""
    f1 = np.asarray(f1, dtype=float)
    f2 = np.asarray(f2, dtype=float)
    a = np.maximum(0.5 * (f2 + f1), 0.0)  # f_j, clipped
    b = np.maximum(0.5 * (f2 - f1), 0.0)  # f_{N-1-j}, clipped
    return a - b, a + b


def view_subsets(Mh: int, rows_per_subset: int):
    """Consecutive row blocks [t r, (t+1) r) of the folded system (the last may be shorter)."""
    return [np.arange(a, min(a + rows_per_subset, Mh)) for a in range(0, Mh, rows_per_subset)]


def os_sart(A1, A2, p1, p2, subsets, lam: float, max_iters: int, tol: float = 0.0, check_every: int = 1,
            cone: bool = False, f1_0=None, f2_0=None, record: bool = False):
    """OS-SART on both split systems with the joint stopping rule (and optionally the cone).

    ``subsets`` is a list of row-index arrays that partition the rows. Returns a
    dict with keys f1, f2, iters, rho and, if ``record`` is set, rho_hist (the
    tested values).
    """
    systems = []
    for B, q in ((A1, p1), (A2, p2)):
        B = sp.csr_matrix(B, dtype=float)
        R, _ = normalisers(B)
        iR = _safe_inv(R)
        parts = []
        for I in subsets:
            Bt = B[I]
            _, Ct = normalisers(Bt)
            parts.append((Bt, Bt.T.tocsr(), np.asarray(q, dtype=float)[I], iR[I], _safe_inv(Ct)))
        systems.append((B, np.asarray(q, dtype=float), parts))
    f = [np.zeros(A1.shape[1]) if f1_0 is None else np.array(f1_0, dtype=float),
         np.zeros(A2.shape[1]) if f2_0 is None else np.array(f2_0, dtype=float)]
    if cone:
        f = list(cone_project(f[0], f[1]))
    pnorm = np.sqrt(sum(q @ q for _, q, _ in systems))
    hist = []
    k = 0
    rho = None
    while True:
        if k % check_every == 0 or k == max_iters:
            rr = 0.0
            for s, (B, q, _) in enumerate(systems):
                r = q - B @ f[s]
                rr += r @ r
            rho = np.sqrt(rr) / pnorm if pnorm > 0 else 0.0
            hist.append(rho)
            if rho <= tol or k == max_iters:
                break
        for t in range(len(subsets)):
            for s, (_, _, parts) in enumerate(systems):
                Bt, BtT, qt, iRt, iCt = parts[t]
                f[s] = f[s] + lam * (BtT @ ((qt - Bt @ f[s]) * iRt)) * iCt
            if cone:
                f = list(cone_project(f[0], f[1]))
        k += 1
    out = {"f1": f[0], "f2": f[1], "iters": k, "rho": rho}
    if record:
        out["rho_hist"] = np.array(hist)
    return out


def os_sart_dense(A1, A2, p1, p2, subsets, lam: float, iters: int, cone: bool = False):
    """Dense form of ``os_sart`` for a fixed number of sweeps, written independently as a cross-check.

    Subset t of system s is the matrix G_t = diag(1/C_t) B_t^T diag(1/R_t) applied to q_t - B_t f.
    The cone is applied as an explicit min over the image coordinates.
    """
    def mats(B):
        B = B.toarray() if sp.issparse(B) else np.asarray(B, dtype=float)
        R = np.abs(B).sum(axis=1)
        out = []
        for I in subsets:
            Bt = B[I, :]
            Ct = np.abs(Bt).sum(axis=0)
            DR = np.diag([0.0 if x == 0 else 1.0 / x for x in R[I]])
            DC = np.diag([0.0 if x == 0 else 1.0 / x for x in Ct])
            out.append((Bt, DC @ Bt.T @ DR, I))
        return out

    M1, M2 = mats(A1), mats(A2)
    q1, q2 = np.asarray(p1, dtype=float), np.asarray(p2, dtype=float)
    x1 = np.zeros(np.shape(A1)[1])
    x2 = np.zeros(np.shape(A2)[1])
    for _ in range(iters):
        for (B1t, G1t, I), (B2t, G2t, _) in zip(M1, M2):
            x1 = x1 + lam * (G1t @ (q1[I] - B1t @ x1))
            x2 = x2 + lam * (G2t @ (q2[I] - B2t @ x2))
            if cone:
                img_a = [min(0.0, v) for v in 0.5 * (x2 + x1)]
                img_b = [min(0.0, v) for v in 0.5 * (x2 - x1)]
                a = 0.5 * (x2 + x1) - np.array(img_a)
                b = 0.5 * (x2 - x1) - np.array(img_b)
                x1, x2 = a - b, a + b
    return x1, x2
