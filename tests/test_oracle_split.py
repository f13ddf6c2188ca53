"""Pins for the oracle's fold and recombination.

The references here are the paper's printed Example 1 and its theorems, checked
by brute force with library linear algebra.
"""
import numpy as np
import pytest

from oracle import split
from tests.golden.loader import load

EX1 = load("example1.txt")


def random_symmetric(rng, M, N, density=1.0):
    """A random M x N matrix with w[i,j] = w[M-1-i, N-1-j] (Eq. 2).

    The rows M/2.. are mirrors of the rows ..M/2.
    """
    top = rng.standard_normal((M // 2, N))
    if density < 1.0:
        top *= rng.random((M // 2, N)) < density
    return np.vstack([top, top[::-1, ::-1]])


def test_example1_is_symmetric():
    A = EX1["A"]
    assert np.array_equal(A, A[::-1, ::-1])


def test_example1_fold_matches_printed_split_systems():
    A1, A2 = split.fold_matrix(EX1["A"])
    assert np.array_equal(A1, EX1["A1"])
    assert np.array_equal(A2, EX1["A2"])
    p1, p2 = split.fold_rhs(EX1["p"])
    assert np.array_equal(p1, EX1["p1"])
    assert np.array_equal(p2, EX1["p2"])


@pytest.mark.parametrize("x,y", [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (0.37, -2.5), (-3.0, 7.0)])
def test_example1_recombination_of_general_solutions(x, y):
    """Theorem 1 applied to the printed general solutions must give the printed general solution of Eq. (13)."""
    f1 = EX1["f1_general"] @ np.array([1.0, x])
    f2 = EX1["f2_general"] @ np.array([1.0, y])
    f = split.recombine(f1, f2)
    assert np.allclose(f, EX1["f_general"] @ np.array([1.0, x, y]), rtol=0, atol=1e-12)
    # The recombined general solution solves the full system exactly.
    assert np.allclose(EX1["A"] @ f, EX1["p"], atol=1e-10)


def test_example1_normal_pseudo_solutions():
    f1 = split.min_norm(EX1["A1"], EX1["p1"])
    f2 = split.min_norm(EX1["A2"], EX1["p2"])
    assert np.allclose(f1, EX1["f1_min"], atol=5e-5)
    assert np.allclose(f2, EX1["f2_min"], atol=5e-5)
    assert abs(np.linalg.norm(f1) - EX1["f1_min_norm"][0]) < 5e-5
    assert abs(np.linalg.norm(f2) - EX1["f2_min_norm"][0]) < 5e-5
    f = split.recombine(f1, f2)
    assert np.allclose(f, EX1["f_min"], atol=5e-5)
    assert abs(np.linalg.norm(f) - EX1["f_min_norm"][0]) < 5e-5
    # Theorem 2: the full system's own normal pseudo-solution is the same vector.
    assert np.allclose(split.min_norm(EX1["A"], EX1["p"]), f, atol=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_theorem1_full_rank_least_squares(seed):
    rng = np.random.default_rng(seed)
    M, N = 14, 8
    A = random_symmetric(rng, M, N)
    p = A @ rng.standard_normal(N)
    f_full = np.linalg.lstsq(A, p, rcond=None)[0]
    A1, A2 = split.fold_matrix(A)
    p1, p2 = split.fold_rhs(p)
    f1 = np.linalg.lstsq(A1, p1, rcond=None)[0]
    f2 = np.linalg.lstsq(A2, p2, rcond=None)[0]
    assert np.allclose(split.recombine(f1, f2), f_full, atol=1e-10)


@pytest.mark.parametrize("seed", range(5))
def test_theorem2_rank_deficient(seed):
    rng = np.random.default_rng(100 + seed)
    M, N = 6, 12  # wide: infinitely many solutions, pinv picks the minimum norm
    A = random_symmetric(rng, M, N)
    p = rng.standard_normal(M)
    A1, A2 = split.fold_matrix(A)
    p1, p2 = split.fold_rhs(p)
    f1 = np.linalg.pinv(A1) @ p1
    f2 = np.linalg.pinv(A2) @ p2
    f = split.recombine(f1, f2)
    assert np.allclose(f, np.linalg.pinv(A) @ p, atol=1e-10)
    assert np.isclose(f @ f, 0.5 * (f1 @ f1) + 0.5 * (f2 @ f2), rtol=1e-12)


@pytest.mark.parametrize("n", [2, 4, 6, 10])
def test_determinant_identity(n):
    """The determinant identity after Example 1 (Eq. 18), for square symmetric A."""
    rng = np.random.default_rng(n)
    A = random_symmetric(rng, n, n)
    A1, A2 = split.fold_matrix(A)
    d = np.linalg.det(A)
    assert np.isclose(d, np.linalg.det(A1) * np.linalg.det(A2), rtol=1e-10, atol=0)


def test_normal_matrix_identity():
    """B = A^T A satisfies Eq. (2), and its fold is (A1^T A1, A2^T A2)."""
    rng = np.random.default_rng(7)
    A = random_symmetric(rng, 10, 8)
    B = A.T @ A
    assert np.allclose(B, B[::-1, ::-1], atol=1e-12)
    B1, B2 = split.fold_matrix(B)
    A1, A2 = split.fold_matrix(A)
    assert np.allclose(B1, A1.T @ A1, atol=1e-12)
    assert np.allclose(B2, A2.T @ A2, atol=1e-12)


def test_fold_commutes_with_projection():
    """Folding the image then applying A_s equals folding the projection A f."""
    rng = np.random.default_rng(3)
    A = random_symmetric(rng, 20, 16, density=0.4)
    f = rng.standard_normal(16)
    A1, A2 = split.fold_matrix(A)
    f1, f2 = split.fold_image(f)
    q1, q2 = split.fold_rhs(A @ f)
    assert np.allclose(A1 @ f1, q1, atol=1e-12)
    assert np.allclose(A2 @ f2, q2, atol=1e-12)


def test_recombine_inverts_image_fold():
    rng = np.random.default_rng(4)
    f = rng.standard_normal(18)
    assert np.allclose(split.recombine(*split.fold_image(f)), f, atol=1e-15)


def test_sparse_and_dense_fold_agree():
    import scipy.sparse as sp
    rng = np.random.default_rng(5)
    A = random_symmetric(rng, 12, 10, density=0.3)
    d1, d2 = split.fold_matrix(A)
    s1, s2 = split.fold_matrix(sp.csr_matrix(A))
    assert np.array_equal(s1.toarray(), d1)
    assert np.array_equal(s2.toarray(), d2)


def test_odd_sizes_rejected():
    with pytest.raises(ValueError):
        split.fold_matrix(np.zeros((3, 4)))
    with pytest.raises(ValueError):
        split.fold_rhs(np.zeros(5))


def test_folded_pattern_size_example1_keeps_the_cancelled_zero():
    """Example 1: all 2 x 3 folded positions are stored, including A1[0, 0] = 1 - 1 = 0.

    The union pattern counts a position when w_ij or w_{M-1-i,j} is stored, so the
    zero that cancellation makes in the printed A1 (Eq. 14) still counts: S = 6.
    """
    import scipy.sparse as sp
    A = sp.csr_matrix(EX1["A"])
    assert split.folded_pattern_size(A) == 6
    assert EX1["A1"][0, 0] == 0.0  # the printed zero is a cancellation, not a missing entry


@pytest.mark.parametrize("rows,expect", [
    # One stored pair per row that cancels in A1: kept (1 position), the other half of the row is empty.
    ([[1.0, 0.0, 0.0, 1.0]], 1),
    # Entries only in the right half: their reflections land in distinct folded columns.
    ([[0.0, 0.0, 2.0, 3.0]], 2),
    # A left entry and the reflection of a right entry in the same folded column count once.
    ([[5.0, 0.0, 0.0, 7.0]], 1),
    # Two rows of a 4 x 4 matrix: row 0 fills both folded columns, row 1 only the reflected column 0.
    ([[1.0, 2.0, 0.0, 0.0], [0.0, 0.0, 0.0, 4.0]], 3),
    # An empty folded row contributes nothing.
    ([[0.0, 0.0, 0.0, 0.0], [0.0, 1.0, 1.0, 0.0]], 1),
])
def test_folded_pattern_size_hand_counts(rows, expect):
    """Hand-counted union patterns of small matrices that satisfy Eq. (2).

    Each top row i is given; row M-1-i is its reflection w[M-1-i, N-1-j] = w[i, j].
    Position (i, j), j < N/2, is stored when w[i, j] != 0 or w[i, N-1-j] != 0.
    """
    import scipy.sparse as sp
    top = np.array(rows, dtype=float)
    A = np.vstack([top, top[::-1, ::-1]])
    assert np.array_equal(A, A[::-1, ::-1])
    assert split.folded_pattern_size(sp.csr_matrix(A)) == expect
    # The count is a property of the stored pattern, not of the values: scaling cannot change it.
    assert split.folded_pattern_size(sp.csr_matrix(-3.0 * A)) == expect
