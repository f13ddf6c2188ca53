"""Oracle geometry: symmetric sources, vertical-snake voxels and Siddon weights (FP64).

Paper reference: Section 2 (Methods).
- Sources sit at positions pairwise symmetric about the axis OZ.
- Voxels follow the vertical "snake" rule (Fig. 1, missing from the source).
- Under these two conditions the system matrix satisfies Eq. (2):
  w_{i,j} = w_{M-i+1,N-j+1}.
- The paper says only that the passage of each beam through the voxels is
  modelled (Example 2). The weight w_ij is taken as Siddon's exact intersection
  length of ray i with cell j, in mm.

Readings, with 0-based indices throughout:
- Source k sits at angle theta_k = gamma (2k + 1 - K) / (K - 1). Its position
  is (R sin theta_k, R cos theta_k) in the (x, z) plane. The mirror source
  K-1-k is set to exactly (-x, z).
- Detector bin b is centred at u_b = D (2b + 1 - nb) / (2 nb), on z = 0.
- Ray i = k nb + b runs from source k to the centre of bin b. Its mirror ray is
  M-1-i.
- Cell (c, r): column c counts x-cells from the left and row r counts z-cells
  from the bottom. Snake index j = c nz + (r if c is even else nz-1-r).
  When nx is even, the mirror of cell j about OZ is cell N-1-j.
- A ray lying exactly on a vertical cell boundary gives half its length to each
  of the two cells that share that boundary. A cell outside the grid drops its
  half.

This module is test infrastructure: see the package docstring.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def source_positions(g) -> np.ndarray:
    """Return the K source positions (x, z), with mirror pairs made exact (Section 2)."""
    K = g.K
    gam = math.radians(g.gamma_deg)
    pos = np.empty((K, 2))
    for k in range(K):
        if 2 * k + 1 > K:  # second half: exact mirror of source K-1-k
            continue
        th = gam * (2 * k + 1 - K) / (K - 1)
        pos[k] = (g.R * math.sin(th), g.R * math.cos(th))
        pos[K - 1 - k] = (-pos[k, 0], pos[k, 1])
    return pos


def detector_centres(g) -> np.ndarray:
    """Return the centres of the nb detector bins along x on z = 0."""
    b = np.arange(g.nb)
    return g.D * (2 * b + 1 - g.nb) / (2 * g.nb)


def ray_endpoints(g, i: int):
    """Return (S, T) for ray i = k nb + b: source k and the centre of bin b."""
    k, b = divmod(i, g.nb)
    S = source_positions(g)[k]
    T = np.array([detector_centres(g)[b], 0.0])
    return S, T


def snake_index(g, c, r):
    """Return the vertical-snake index of cell (c, r) (Section 2, Fig. 1)."""
    c = np.asarray(c)
    r = np.asarray(r)
    return c * g.nz + np.where(c % 2 == 0, r, g.nz - 1 - r)


def snake_cell(g, j):
    """Invert the snake numbering: return the (c, r) of snake index j."""
    j = np.asarray(j)
    c = j // g.nz
    q = j % g.nz
    return c, np.where(c % 2 == 0, q, g.nz - 1 - q)


def image_to_snake(g, img: np.ndarray) -> np.ndarray:
    """Reorder a [nz][nx] image into the snake-ordered vector f[N]."""
    f = np.empty(g.nx * g.nz, dtype=img.dtype)
    for c in range(g.nx):
        for r in range(g.nz):
            f[snake_index(g, c, r)] = img[r, c]
    return f


def snake_to_image(g, f: np.ndarray) -> np.ndarray:
    """Reorder a snake-ordered vector f[N] into a [nz][nx] image."""
    img = np.empty((g.nz, g.nx), dtype=f.dtype)
    for j in range(g.nx * g.nz):
        c, r = snake_cell(g, j)
        img[r, c] = f[j]
    return img


def _planes(g):
    """Return the x and z positions of the cell boundaries.

    x is computed symmetrically, so that x_{nx-c} = -x_c exactly.
    """
    xs = (2.0 * np.arange(g.nx + 1) - g.nx) * g.W / (2.0 * g.nx)
    zs = g.z0 + np.arange(g.nz + 1) * (g.H / g.nz)
    return xs, zs


def siddon_ray(g, S, T):
    """Exact intersection lengths of segment S->T with the cells.

    This is Siddon's method. The segment is parametrised as S + a (T - S), with
    a in [0, 1]. The breakpoints are the parameters of every cell boundary
    crossed inside the box, plus the entry and exit. Each piece between two
    breakpoints belongs to the cell that contains its midpoint.

    Returns (j, length) arrays, sorted by snake index j.
    """
    xs, zs = _planes(g)
    dxr = T[0] - S[0]
    dzr = T[1] - S[1]
    L = math.hypot(dxr, dzr)
    xlo, xhi, zlo, zhi = xs[0], xs[-1], zs[0], zs[-1]
    ddx = g.W / g.nx
    ddz = g.H / g.nz

    if dxr == 0.0:
        # Vertical ray.
        x = S[0]
        if x < xlo or x > xhi:
            return np.zeros(0, dtype=np.int64), np.zeros(0)
        amin = max(0.0, min((zlo - S[1]) / dzr, (zhi - S[1]) / dzr))
        amax = min(1.0, max((zlo - S[1]) / dzr, (zhi - S[1]) / dzr))
        if amax <= amin:
            return np.zeros(0, dtype=np.int64), np.zeros(0)
        az = (zs - S[1]) / dzr
        a = np.unique(np.concatenate([[amin, amax], az[(az > amin) & (az < amax)]]))
        da = np.diff(a)
        mid = 0.5 * (a[1:] + a[:-1])
        zm = S[1] + mid * dzr
        r = np.clip(np.floor((zm - zlo) / ddz).astype(np.int64), 0, g.nz - 1)
        on_plane = np.nonzero(xs == x)[0]
        out = {}
        if on_plane.size:  # exactly on a boundary: half to each side
            cb = int(on_plane[0])
            cols, share = [cb - 1, cb], 0.5
        else:
            cols, share = [min(int(math.floor((x - xlo) / ddx)), g.nx - 1)], 1.0
        for c in cols:
            if 0 <= c < g.nx:
                for rr, d in zip(r, da):
                    if d > 0:
                        jj = int(snake_index(g, c, rr))
                        out[jj] = out.get(jj, 0.0) + share * d * L
        jj = np.array(sorted(out), dtype=np.int64)
        return jj, np.array([out[k] for k in jj])

    ax = (xs - S[0]) / dxr
    az = (zs - S[1]) / dzr
    amin = max(0.0, min(ax[0], ax[-1]), min(az[0], az[-1]))
    amax = min(1.0, max(ax[0], ax[-1]), max(az[0], az[-1]))
    if amax <= amin:
        return np.zeros(0, dtype=np.int64), np.zeros(0)
    inner = np.concatenate([ax[(ax > amin) & (ax < amax)], az[(az > amin) & (az < amax)]])
    a = np.unique(np.concatenate([[amin, amax], inner]))
    da = np.diff(a)
    keep = da > 0
    mid = 0.5 * (a[1:] + a[:-1])
    xm = S[0] + mid * dxr
    zm = S[1] + mid * dzr
    c = np.clip(np.floor((xm - xlo) / ddx).astype(np.int64), 0, g.nx - 1)
    r = np.clip(np.floor((zm - zlo) / ddz).astype(np.int64), 0, g.nz - 1)
    j = snake_index(g, c[keep], r[keep])
    w = da[keep] * L
    order = np.argsort(j, kind="stable")
    j, w = j[order], w[order]
    # A straight segment visits each cell at most once, so j has no repeats.
    # Merge anyway, to be safe.
    uj, inv = np.unique(j, return_inverse=True)
    return uj.astype(np.int64), np.bincount(inv, weights=w, minlength=uj.size)


def check_params(g) -> None:
    """Check the parity conditions the split needs.

    - nx must be even, so that mirror(j) = N-1-j holds.
    - M = K nb must be even, so that no ray is its own mirror (Section 2: N and
      M even).
    """
    if g.nx % 2 != 0:
        raise ValueError("nx must be even for the vertical-snake mirror j <-> N-1-j")
    if (g.K * g.nb) % 2 != 0:
        raise ValueError("M = K nb must be even")
    if g.K < 2:
        raise ValueError("K >= 2 symmetric source positions are required")


def system_matrix(g, rows=None) -> sp.csr_matrix:
    """Trace every ray independently and return A as an M x N CSR (FP64).

    ``rows`` restricts tracing to the given ray indices. The other rows are
    then left empty.
    """
    check_params(g)
    M, N = g.K * g.nb, g.nx * g.nz
    src = source_positions(g)
    det = detector_centres(g)
    indptr = [0]
    indices = []
    data = []
    rows = range(M) if rows is None else set(rows)
    for i in range(M):
        if i in rows:
            k, b = divmod(i, g.nb)
            j, w = siddon_ray(g, src[k], np.array([det[b], 0.0]))
            indices.append(j)
            data.append(w)
            indptr.append(indptr[-1] + j.size)
        else:
            indptr.append(indptr[-1])
    ind = np.concatenate(indices) if indices else np.zeros(0, dtype=np.int64)
    dat = np.concatenate(data) if data else np.zeros(0)
    return sp.csr_matrix((dat, ind, np.array(indptr)), shape=(M, N))


def mirrored_system_matrix(g) -> sp.csr_matrix:
    """Build A by tracing the first M/2 rays and mirroring the rest.

    Eq. (2) gives w[M-1-i, N-1-j] := w[i, j] for the mirrored rows. The result
    satisfies the symmetry exactly by construction.
    """
    check_params(g)
    M, N = g.K * g.nb, g.nx * g.nz
    Mh = M // 2
    top = system_matrix(g, rows=range(Mh))[:Mh].tocoo()
    r = np.concatenate([top.row, M - 1 - top.row])
    c = np.concatenate([top.col, N - 1 - top.col])
    v = np.concatenate([top.data, top.data])
    return sp.csr_matrix((v, (r, c)), shape=(M, N))


def symmetry_defect(A) -> float:
    """Return the largest |w_{i,j} - w_{M-1-i,N-1-j}| over the matrix (Eq. 2)."""
    A = sp.csr_matrix(A)
    Ar = A[::-1, ::-1]
    d = (A - Ar)
    return float(abs(d).max()) if d.nnz else 0.0
