"""Pins for the oracle's split-SART.

- Closed forms for diagonal and single-row systems.
- The Landweber limit, computed through a pseudo-inverse.
- The residual identity, checked against the full system.
- Agreement of the oracle's two implementations.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import geometry as geo
from oracle import sart, split
from paper_1902_10559_gb300.synthetic import TINY, random_phantom


def test_diagonal_system_closed_form():
    """For B = diag(d) the update is f <- f + lam (q/d - f).

    So f_k = (1 - (1-lam)^k) q/d, and a negative d must still converge to q/d.
    """
    d = np.array([2.0, -3.0, 0.5, -0.25])
    q = np.array([1.0, 2.0, -1.0, 4.0])
    lam = 0.7
    for k in (1, 2, 5, 13):
        out = sart.split_sart(np.diag(d), np.diag(d), q, q, lam, k)
        assert out["iters"] == k
        assert np.allclose(out["f1"], (1 - (1 - lam) ** k) * q / d, rtol=1e-14)


def test_single_row_first_step_closed_form():
    """For one row a, the first step from zero is f_j = lam sign(a_j) q / sum|a|."""
    a = np.array([[1.5, -2.0, 0.0, 4.0]])
    q = np.array([3.0])
    lam = 1.3
    out = sart.split_sart(a, a, q, q, lam, 1)
    expect = lam * np.sign(a[0]) * q[0] / np.abs(a).sum()
    expect[2] = 0.0  # an empty column keeps f0
    assert np.allclose(out["f1"], expect, rtol=1e-15)


def test_zero_rows_and_columns_stay_put():
    B = np.array([[1.0, 0.0, 2.0], [0.0, 0.0, 0.0]])
    q = np.array([1.0, 5.0])
    f0 = np.array([0.1, 0.2, 0.3])
    out = sart.split_sart(B, B, q, q, 1.0, 3, f1_0=f0, f2_0=f0)
    assert out["f1"][1] == 0.2


@pytest.mark.parametrize("seed", range(3))
def test_limit_is_weighted_min_norm_solution(seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((5, 8)) * (rng.random((5, 8)) < 0.7)
    q = rng.standard_normal(5)
    out = sart.split_sart(B, B, q, q, 1.0, 20000)
    assert np.allclose(out["f1"], sart.sart_limit(B, q), atol=1e-8)


def test_sparse_and_dense_implementations_agree():
    rng = np.random.default_rng(11)
    B1 = rng.standard_normal((9, 7)) * (rng.random((9, 7)) < 0.5)
    B2 = rng.standard_normal((9, 7)) * (rng.random((9, 7)) < 0.5)
    q1, q2 = rng.standard_normal(9), rng.standard_normal(9)
    a = sart.split_sart(B1, B2, q1, q2, 0.9, 37)
    b = sart.split_sart_dense(B1, B2, q1, q2, 0.9, 37)
    assert a["iters"] == b["iters"] == 37
    assert np.allclose(a["f1"], b["f1"], rtol=1e-13, atol=1e-14)
    assert np.allclose(a["f2"], b["f2"], rtol=1e-13, atol=1e-14)
    assert np.isclose(a["rho"], b["rho"], rtol=1e-13)


def test_row_and_column_permutation_equivariance():
    rng = np.random.default_rng(12)
    B = rng.standard_normal((8, 6)) * (rng.random((8, 6)) < 0.6)
    q = rng.standard_normal(8)
    pr, pc = rng.permutation(8), rng.permutation(6)
    a = sart.split_sart(B, B, q, q, 0.8, 25)
    b = sart.split_sart(B[pr][:, pc], B[pr][:, pc], q[pr], q[pr], 0.8, 25)
    assert np.allclose(b["f1"], a["f1"][pc], rtol=1e-13, atol=1e-15)


@pytest.fixture(scope="module")
def tiny_system():
    g = TINY
    A = geo.mirrored_system_matrix(g)
    f_true = geo.image_to_snake(g, random_phantom(g, 1, 8))
    p = A @ f_true
    return g, A, f_true, p


def test_split_residual_equals_full_residual(tiny_system):
    """rho from the split residuals equals ||A f - p|| / ||p|| for the recombined f."""
    g, A, f_true, p = tiny_system
    A1, A2 = split.fold_matrix(A)
    p1, p2 = split.fold_rhs(p)
    for iters in (0, 1, 7, 40):
        out = sart.split_sart(A1, A2, p1, p2, 1.0, iters)
        f = split.recombine(out["f1"], out["f2"])
        assert np.isclose(out["rho"], split.relative_residual(A, f, p), rtol=1e-10)


def test_residual_decreases_on_consistent_data(tiny_system):
    g, A, f_true, p = tiny_system
    A1, A2 = split.fold_matrix(A)
    p1, p2 = split.fold_rhs(p)
    out = sart.split_sart(A1, A2, p1, p2, 1.0, 100, record=True)
    h = out["rho_hist"]
    assert h[0] == pytest.approx(1.0)
    assert h[-1] < 0.05
    assert np.all(np.diff(h) <= 1e-12)


def test_stopping_rule(tiny_system):
    g, A, f_true, p = tiny_system
    A1, A2 = split.fold_matrix(A)
    p1, p2 = split.fold_rhs(p)
    full = sart.split_sart(A1, A2, p1, p2, 1.0, 60, record=True)
    h = full["rho_hist"]
    tol = 0.5 * (h[10] + h[11])  # strictly between rho_10 and rho_11
    out = sart.split_sart(A1, A2, p1, p2, 1.0, 60, tol=tol)
    assert out["iters"] == 11
    assert out["rho"] == pytest.approx(h[11], rel=1e-12)


def test_schur_bound_on_split_systems(tiny_system):
    """||R^-1/2 A_s C^-1/2||_2 <= 1, so 0 < lambda < 2 converges for A1 (mixed signs) and A2."""
    g, A, f_true, p = tiny_system
    A1, A2 = split.fold_matrix(A)
    for B in (A1, A2):
        s = sart.scaled_operator_norm(B, iters=300)
        assert 0.5 < s <= 1.0 + 1e-9


def test_split_and_full_matrix_sizes(tiny_system):
    g, A, f_true, p = tiny_system
    A1, A2 = split.fold_matrix(A)
    assert A1.shape == A2.shape == (g.M // 2, g.N // 2)
    S = split.folded_pattern_size(A)
    assert A.nnz / 2 * 0.5 <= S <= A.nnz / 2
    assert sp.csr_matrix(A1).nnz <= S


def test_fixed_iterations_per_system_equal_the_joint_solve():
    """Section 2's independence: without a stop test the two systems do not interact."""
    rng = np.random.default_rng(7)
    A1, A2 = rng.standard_normal((3, 4)), np.abs(rng.standard_normal((3, 4)))
    p1, p2 = rng.standard_normal(3), rng.standard_normal(3)
    ref = sart.split_sart(A1, A2, p1, p2, 0.9, 37)
    assert np.array_equal(sart.sart_fixed(A1, p1, 0.9, 37), ref["f1"])
    assert np.array_equal(sart.sart_fixed(A2, p2, 0.9, 37), ref["f2"])
