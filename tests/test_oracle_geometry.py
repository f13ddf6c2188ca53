"""Pins for the oracle's geometry.

- Snake numbering: by its defining properties.
- Siddon lengths: by closed forms, by brute-force sampling, and by independently
  traced mirror rays (Eq. 2).
"""
import math

import numpy as np
import pytest

from oracle import geometry as geo
from paper_1902_10559_gb300.synthetic import TINY, Geometry


def test_snake_consecutive_cells_are_adjacent():
    """In the vertical snake, index j+1 is always a neighbour of j.

    Within a column the step is vertical. At a column change the step is
    horizontal, in the same row.
    """
    g = TINY
    c, r = geo.snake_cell(g, np.arange(g.N))
    dc = np.abs(np.diff(c))
    dr = np.abs(np.diff(r))
    assert np.all(dc + dr == 1)
    assert np.all((dc == 0) | (dr == 0))
    # Columns are contiguous index ranges of length nz (vertical numbering).
    assert np.array_equal(c, np.repeat(np.arange(g.nx), g.nz))
    # Column 0 runs bottom -> top.
    assert r[0] == 0 and r[g.nz - 1] == g.nz - 1


@pytest.mark.parametrize("nx,nz", [(2, 1), (4, 3), (32, 16), (6, 5)])
def test_snake_mirror_is_index_reversal(nx, nz):
    g = Geometry(nx=nx, nz=nz, W=1.0, H=1.0, z0=1.0, K=2, gamma_deg=10, R=10, nb=2, D=4)
    c, r = geo.snake_cell(g, np.arange(g.N))
    jm = geo.snake_index(g, nx - 1 - c, r)  # mirror of each cell about OZ
    assert np.array_equal(jm, g.N - 1 - np.arange(g.N))


def test_snake_mirror_fails_for_odd_nx():
    g = Geometry(nx=3, nz=2, W=1.0, H=1.0, z0=1.0, K=2, gamma_deg=10, R=10, nb=2, D=4)
    c, r = geo.snake_cell(g, np.arange(g.N))
    jm = geo.snake_index(g, g.nx - 1 - c, r)
    assert not np.array_equal(jm, g.N - 1 - np.arange(g.N))
    with pytest.raises(ValueError):
        geo.check_params(g)


def test_image_snake_roundtrip():
    g = TINY
    img = np.arange(g.N, dtype=float).reshape(g.nz, g.nx)
    assert np.array_equal(geo.snake_to_image(g, geo.image_to_snake(g, img)), img)


def test_sources_and_bins_mirror_exactly():
    g = TINY
    s = geo.source_positions(g)
    assert np.array_equal(s[::-1, 0], -s[:, 0])
    assert np.array_equal(s[::-1, 1], s[:, 1])
    assert np.allclose(np.hypot(s[:, 0], s[:, 1]), g.R, rtol=1e-15)
    ang = np.degrees(np.arctan2(s[:, 0], s[:, 1]))
    assert np.isclose(ang[0], -g.gamma_deg) and np.isclose(ang[-1], g.gamma_deg)
    assert np.allclose(np.diff(ang), 2 * g.gamma_deg / (g.K - 1))
    u = geo.detector_centres(g)
    assert np.array_equal(u[::-1], -u)
    assert np.allclose(np.diff(u), g.D / g.nb)


def test_vertical_ray_inside_a_column():
    g = TINY
    dx, dz = g.W / g.nx, g.H / g.nz
    c = 5
    x = -g.W / 2 + (c + 0.3) * dx
    j, w = geo.siddon_ray(g, np.array([x, 700.0]), np.array([x, 0.0]))
    assert np.array_equal(np.sort(j), np.sort(geo.snake_index(g, np.full(g.nz, c), np.arange(g.nz))))
    assert np.allclose(w, dz, rtol=1e-13)


def test_vertical_ray_on_a_cell_boundary_splits_half_half():
    g = TINY
    dz = g.H / g.nz
    c = 7  # boundary between columns 6 and 7
    x = (2.0 * c - g.nx) * g.W / (2.0 * g.nx)
    j, w = geo.siddon_ray(g, np.array([x, 700.0]), np.array([x, 0.0]))
    cols, _ = geo.snake_cell(g, j)
    assert sorted(set(cols.tolist())) == [6, 7]
    assert np.allclose(w, 0.5 * dz, rtol=1e-13)
    # On the outer boundary, the half that falls outside the grid is dropped.
    j, w = geo.siddon_ray(g, np.array([-g.W / 2, 700.0]), np.array([-g.W / 2, 0.0]))
    cols, _ = geo.snake_cell(g, j)
    assert set(cols.tolist()) == {0} and np.allclose(w, 0.5 * dz)


def test_diagonal_ray_through_square_cells():
    g = Geometry(nx=8, nz=8, W=8.0, H=8.0, z0=2.0, K=2, gamma_deg=10, R=50, nb=2, D=10)
    # From beyond the top-left corner to beyond the bottom-right corner, at 45 degrees.
    S = np.array([-4.0 - 3.0, 2.0 + 8.0 + 3.0])
    T = np.array([4.0 + 2.0, 2.0 - 2.0])
    j, w = geo.siddon_ray(g, S, T)
    c, r = geo.snake_cell(g, j)
    assert sorted(zip(c.tolist(), r.tolist())) == [(k, 7 - k) for k in range(8)]
    assert np.allclose(w, math.sqrt(2.0), rtol=1e-13)


def test_row_sum_equals_chord_for_rays_through_top_and_bottom():
    """If a ray crosses the top and the bottom faces, its total length is H / cos(phi)."""
    g = TINY
    A = geo.system_matrix(g)
    src = geo.source_positions(g)
    det = geo.detector_centres(g)
    n_checked = 0
    for i in range(g.M):
        k, b = divmod(i, g.nb)
        S, T = src[k], np.array([det[b], 0.0])
        x_at = lambda z: S[0] + (T[0] - S[0]) * (z - S[1]) / (T[1] - S[1])
        xt, xb = x_at(g.z0 + g.H), x_at(g.z0)
        if abs(xt) < g.W / 2 - 1e-9 and abs(xb) < g.W / 2 - 1e-9:
            chord = g.H * math.hypot(T[0] - S[0], T[1] - S[1]) / abs(T[1] - S[1])
            assert math.isclose(A[i].sum(), chord, rel_tol=1e-12)
            n_checked += 1
    assert n_checked > 100


@pytest.mark.parametrize("i", [3, 77, 150, 333, 611])
def test_siddon_against_brute_force_sampling(i):
    g = TINY
    S, T = geo.ray_endpoints(g, i)
    j, w = geo.siddon_ray(g, S, T)
    n = 400_000
    t = (np.arange(n) + 0.5) / n
    P = S[None, :] + t[:, None] * (T - S)[None, :]
    inside = (np.abs(P[:, 0]) < g.W / 2) & (P[:, 1] > g.z0) & (P[:, 1] < g.z0 + g.H)
    c = np.floor((P[inside, 0] + g.W / 2) / (g.W / g.nx)).astype(int)
    r = np.floor((P[inside, 1] - g.z0) / (g.H / g.nz)).astype(int)
    jj = geo.snake_index(g, c, r)
    step = np.linalg.norm(T - S) / n
    brute = np.bincount(jj, minlength=g.N) * step
    dense = np.zeros(g.N)
    dense[j] = w
    assert np.abs(dense - brute).max() <= 2.5 * step


def test_independently_traced_mirror_rays_agree():
    g = TINY
    A = geo.system_matrix(g)
    scale = abs(A).max()
    assert geo.symmetry_defect(A) <= 1e-12 * scale
    Am = geo.mirrored_system_matrix(g)
    assert abs(A - Am).max() <= 1e-12 * scale
    assert geo.symmetry_defect(Am) == 0.0


def test_tiny_workload_shape():
    g = TINY
    A = geo.system_matrix(g)
    assert A.shape == (640, 512)
    hits = np.diff(A.indptr) > 0
    assert 0.3 < hits.mean() <= 1.0
