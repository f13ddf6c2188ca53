"""Pins for the oracle's normal-matrix solvers (CGLS and the direct method).

- CGLS after n steps on an n-column full-rank system is the least-squares
  solution (conjugate gradients end in at most n steps in exact arithmetic),
  checked against numpy.linalg.lstsq.
- With all singular values equal, CGLS ends in one step.
- From zero on a rank-deficient consistent symmetric system, CGLS on A1 and A2
  recombines to the full system's normal pseudo-solution (Theorem 2), checked
  against numpy.linalg.pinv; on Example 1 it reproduces the printed normal
  pseudo-solutions.
- The direct method equals lstsq on full-rank systems, and the split direct
  solve equals the full one (Theorem 1).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import normal
from oracle import split
from tests.golden.loader import load

EX1 = load("example1.txt")


def random_symmetric(rng, M, N, density=1.0):
    top = rng.standard_normal((M // 2, N))
    if density < 1.0:
        top *= rng.random((M // 2, N)) < density
    return np.vstack([top, top[::-1, ::-1]])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cgls_is_least_squares_after_n_steps(seed):
    rng = np.random.default_rng(seed)
    B1, B2 = rng.standard_normal((30, 8)), rng.standard_normal((24, 8))
    q1, q2 = rng.standard_normal(30), rng.standard_normal(24)
    out = normal.cgls(B1, B2, q1, q2, 8)
    assert out["iters"] == 8
    ref1 = np.linalg.lstsq(B1, q1, rcond=None)[0]
    ref2 = np.linalg.lstsq(B2, q2, rcond=None)[0]
    assert np.allclose(out["f1"], ref1, rtol=0, atol=1e-9 * np.abs(ref1).max())
    assert np.allclose(out["f2"], ref2, rtol=0, atol=1e-9 * np.abs(ref2).max())
    r = np.concatenate([q1 - B1 @ ref1, q2 - B2 @ ref2])
    assert out["rho"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(np.concatenate([q1, q2])), rel=1e-9)


def test_cgls_one_step_with_equal_singular_values():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 5)))
    B = 2.5 * Q
    q = rng.standard_normal(12)
    out = normal.cgls(B, -B, q, q, 1)
    ref = np.linalg.lstsq(B, q, rcond=None)[0]
    assert np.allclose(out["f1"], ref, atol=1e-13) and np.allclose(out["f2"], -ref, atol=1e-13)


@pytest.mark.parametrize("seed", [4, 5])
def test_cgls_split_recombines_to_the_normal_pseudo_solution(seed):
    """Theorem 2: rank-deficient, consistent; CGLS from zero on each split system, then Eq. (5)."""
    rng = np.random.default_rng(seed)
    A = random_symmetric(rng, 12, 16)  # 12 x 16: rank at most 12 < 16 columns
    f_any = rng.standard_normal(16)
    p = A @ f_any
    A1, A2 = split.fold_matrix(A)
    p1, p2 = split.fold_rhs(p)
    out = normal.cgls(A1, A2, p1, p2, 200, tol=1e-15)
    f = split.recombine(out["f1"], out["f2"])
    ref = np.linalg.pinv(A) @ p
    assert np.allclose(f, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    assert np.linalg.norm(f) ** 2 == pytest.approx(0.5 * (out["f1"] @ out["f1"] + out["f2"] @ out["f2"]), rel=1e-12)


def test_cgls_on_example1_reaches_the_printed_pseudo_solutions():
    out = normal.cgls(EX1["A1"], EX1["A2"], EX1["p1"], EX1["p2"], 50, tol=1e-14)
    assert np.allclose(out["f1"], EX1["f1_min"], atol=5e-5)
    assert np.allclose(out["f2"], EX1["f2_min"], atol=5e-5)
    assert np.allclose(split.recombine(out["f1"], out["f2"]), EX1["f_min"], atol=5e-5)
    assert np.linalg.norm(out["f1"]) == pytest.approx(EX1["f1_min_norm"][0], abs=5e-5)
    assert np.linalg.norm(out["f2"]) == pytest.approx(EX1["f2_min_norm"][0], abs=5e-5)


def test_cgls_stopping_rule():
    rng = np.random.default_rng(6)
    A = random_symmetric(rng, 40, 20, density=0.4)
    p = A @ rng.standard_normal(20)
    A1, A2 = split.fold_matrix(A)
    p1, p2 = split.fold_rhs(p)
    hist = normal.cgls(A1, A2, p1, p2, 8, record=True)["rho_hist"]
    assert len(hist) == 9 and np.all(np.diff(hist) < 0)  # the residual of CGLS never grows
    tol = 0.5 * (hist[4] + hist[5])
    out = normal.cgls(A1, A2, p1, p2, 8, tol=tol)
    assert out["iters"] == 5 and out["rho"] <= tol
    assert normal.cgls(A1, A2, p1, p2, 8, tol=tol, check_every=3)["iters"] == 6
    # rho is the full system's relative residual of the recombined iterate.
    f = split.recombine(out["f1"], out["f2"])
    assert out["rho"] == pytest.approx(split.relative_residual(A, f, p), rel=1e-10)


@pytest.mark.parametrize("seed", [7, 8])
def test_direct_solve_is_least_squares_and_splits(seed):
    rng = np.random.default_rng(seed)
    A = random_symmetric(rng, 40, 12)
    p = rng.standard_normal(40)
    ref = np.linalg.lstsq(A, p, rcond=None)[0]
    got = normal.direct_solve(A, p)
    assert np.allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    assert np.allclose(normal.direct_solve(sp.csr_matrix(A), p), ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    # Theorem 1: the split direct solve gives the full system's solution.
    assert np.allclose(normal.split_direct_solve(A, p), ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    # The normal matrices of the split systems are the folds of B (text after Eq. 18).
    B1, B2 = split.fold_matrix(normal.normal_matrix(A))
    A1, A2 = split.fold_matrix(A)
    assert np.allclose(normal.normal_matrix(A1), B1, atol=1e-12)
    assert np.allclose(normal.normal_matrix(A2), B2, atol=1e-12)
