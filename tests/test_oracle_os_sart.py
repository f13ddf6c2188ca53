"""Pins for the oracle's ordered-subsets SART and the non-negativity cone.

OS-SART updates with the rows of one subset at a time (Section 1, reference
[001]: SART's per-view form). The pins:
- one subset holding every row is the simultaneous SART of ``split_sart``;
- a diagonal system has a closed form (each subset moves only its own columns);
- one sweep of a 2 x 2 system with two one-row subsets, by hand;
- the cone projection: feasibility, idempotence, and the variational
  inequality that characterises a Euclidean projection onto a convex set;
- a hand example in which projecting after every subset (the reading taken)
  and projecting once per sweep give different results;
- the sparse and dense implementations agree;
- on a consistent tiny slice the residual falls, and with the cone the
  recombined image stays non-negative.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import geometry as ogeo
from oracle import sart
from oracle import split
from paper_1902_10559_gb300.synthetic import TINY, random_phantom


@pytest.fixture(scope="module")
def tiny():
    A = ogeo.mirrored_system_matrix(TINY)
    f_true = ogeo.image_to_snake(TINY, random_phantom(TINY, 1, 8))
    A1, A2 = split.fold_matrix(A)
    p1, p2 = split.fold_rhs(A @ f_true)
    return A, f_true, A1, A2, p1, p2


def test_one_subset_is_simultaneous_sart(tiny):
    A, f_true, A1, A2, p1, p2 = tiny
    ref = sart.split_sart(A1, A2, p1, p2, 0.9, 30)
    got = sart.os_sart(A1, A2, p1, p2, [np.arange(A1.shape[0])], 0.9, 30)
    assert got["iters"] == 30
    assert np.allclose(got["f1"], ref["f1"], rtol=0, atol=1e-14 * np.abs(ref["f1"]).max())
    assert np.allclose(got["f2"], ref["f2"], rtol=0, atol=1e-14 * np.abs(ref["f2"]).max())
    assert got["rho"] == pytest.approx(ref["rho"], rel=1e-13)


@pytest.mark.parametrize("lam,k", [(1.0, 1), (0.5, 3), (1.5, 7)])
def test_diagonal_system_closed_form(lam, k):
    """B = diag(d): subset t moves only its own columns, f_j = (1 - (1 - lam)^k) q_j / d_j after k sweeps."""
    d = np.array([2.0, -0.5, 3.0, 1.0, -4.0, 0.25])
    q = np.array([1.0, 2.0, -1.0, 0.5, 3.0, -2.0])
    B = sp.diags(d).tocsr()
    subsets = [np.array([0, 1]), np.array([2, 3, 4]), np.array([5])]
    got = sart.os_sart(B, B, q, -q, subsets, lam, k)
    expect = (1.0 - (1.0 - lam) ** k) * q / d
    assert np.allclose(got["f1"], expect, rtol=1e-14, atol=0)
    assert np.allclose(got["f2"], -expect, rtol=1e-14, atol=0)


def test_two_subsets_one_sweep_by_hand():
    """B = [[2, 1], [0, 3]], q = (5, 6), subsets {row 0}, {row 1}, lambda = 1, f0 = 0.

    R = (3, 3). Subset 0: C_0 = (2, 1), u = 5/3, f = (2 (5/3)/2, 1 (5/3)/1) = (5/3, 5/3).
    Subset 1: C_1 = (0, 3), r = 6 - 3 (5/3) = 1, u = 1/3; column 0 has C = 0 and keeps
    5/3, column 1 gains 3 (1/3)/3 = 1/3. Result (5/3, 2). Column sums over all rows
    (C = (2, 4)) or the reverse order of subsets would give other values.
    """
    B = np.array([[2.0, 1.0], [0.0, 3.0]])
    q = np.array([5.0, 6.0])
    got = sart.os_sart(B, B, q, q, [np.array([0]), np.array([1])], 1.0, 1)
    assert np.allclose(got["f1"], [5 / 3, 2.0], rtol=1e-15) and np.allclose(got["f2"], [5 / 3, 2.0], rtol=1e-15)
    assert got["iters"] == 1


def test_cone_projection_properties():
    rng = np.random.default_rng(5)
    x1, x2 = rng.standard_normal(2000) * 3, rng.standard_normal(2000) * 3
    y1, y2 = sart.cone_project(x1, x2)
    assert np.all(y2 >= np.abs(y1))  # feasible: the recombined pair is >= 0
    # Idempotent, and the identity inside the cone, up to the rounding of one fold and recombination.
    eps = 4e-15 * np.abs(np.concatenate([x1, x2])).max()
    z1, z2 = sart.cone_project(y1, y2)
    assert np.allclose(z1, y1, rtol=0, atol=eps) and np.allclose(z2, y2, rtol=0, atol=eps)
    inside = x2 >= np.abs(x1)
    assert inside.sum() > 100
    assert np.allclose(y1[inside], x1[inside], rtol=0, atol=eps) and np.allclose(y2[inside], x2[inside], rtol=0, atol=eps)
    # Euclidean projection onto a convex set: (x - P x) . (v - P x) <= 0 for every feasible v.
    for _ in range(20):
        v2 = np.abs(rng.standard_normal(2000)) * 3
        v1 = (2 * rng.random(2000) - 1) * v2
        dot = (x1 - y1) * (v1 - y1) + (x2 - y2) * (v2 - y2)
        assert np.all(dot <= 1e-12)
    # It is the non-negativity of the image: recombine, clip, fold (Eq. 5 and the proof of Theorem 1).
    f = split.recombine(x1, x2)
    c1, c2 = split.fold_image(np.maximum(f, 0.0))
    assert np.allclose(c1, y1, atol=1e-14) and np.allclose(c2, y2, atol=1e-14)


def test_cone_after_every_subset_by_hand():
    """Two 2 x 1 systems B = [[1], [1]], q1 = (-3, -2), q2 = (-3, 3), lambda = 1/2, subsets {0}, {1}.

    Subset 0: (f1, f2) = (-3/2, -3/2); the image pair is (-3/2, 0), clipped to (0, 0): (f1, f2) = (0, 0).
    Subset 1: (f1, f2) = (-1, 3/2); the image pair (1/4, 5/4) is feasible, so the sweep ends at (-1, 3/2).
    Projecting only once per sweep would give (-5/4, 5/4) instead.
    """
    B = np.array([[1.0], [1.0]])
    got = sart.os_sart(B, B, np.array([-3.0, -2.0]), np.array([-3.0, 3.0]), [np.array([0]), np.array([1])], 0.5, 1,
                       cone=True)
    assert got["f1"][0] == float(Fraction(-1)) and got["f2"][0] == float(Fraction(3, 2))


@pytest.mark.parametrize("cone", [False, True])
def test_sparse_and_dense_agree(tiny, cone):
    A, f_true, A1, A2, p1, p2 = tiny
    subsets = sart.view_subsets(A1.shape[0], TINY.nb)
    assert len(subsets) == TINY.K // 2
    got = sart.os_sart(A1, A2, p1, p2, subsets, 0.8, 6, cone=cone)
    d1, d2 = sart.os_sart_dense(A1, A2, p1, p2, subsets, 0.8, 6, cone=cone)
    assert np.allclose(got["f1"], d1, rtol=0, atol=1e-12 * np.abs(d1).max())
    assert np.allclose(got["f2"], d2, rtol=0, atol=1e-12 * np.abs(d2).max())


@pytest.mark.parametrize("cone", [False, True])
def test_consistent_slice_converges(tiny, cone):
    A, f_true, A1, A2, p1, p2 = tiny
    subsets = sart.view_subsets(A1.shape[0], TINY.nb)
    out = sart.os_sart(A1, A2, p1, p2, subsets, 1.0, 200, check_every=50, cone=cone, record=True)
    hist = out["rho_hist"]
    assert len(hist) == 5 and np.all(np.diff(hist) < 0) and hist[-1] < 0.02
    f = split.recombine(out["f1"], out["f2"])
    assert out["rho"] == pytest.approx(split.relative_residual(A, f, A @ f_true), rel=1e-12)
    if cone:
        assert f.min() >= -1e-12
    # Ordered subsets reach a lower residual than the same number of simultaneous sweeps.
    plain = sart.split_sart(A1, A2, p1, p2, 1.0, 200)
    assert out["rho"] < plain["rho"]


def test_stopping_rule(tiny):
    A, f_true, A1, A2, p1, p2 = tiny
    subsets = sart.view_subsets(A1.shape[0], TINY.nb)
    hist = sart.os_sart(A1, A2, p1, p2, subsets, 1.0, 40, record=True)["rho_hist"]
    tol = 0.5 * (hist[10] + hist[11])
    out = sart.os_sart(A1, A2, p1, p2, subsets, 1.0, 40, tol=tol)
    assert out["iters"] == 11 and out["rho"] <= tol
    out4 = sart.os_sart(A1, A2, p1, p2, subsets, 1.0, 40, tol=tol, check_every=4)
    assert out4["iters"] == 12
