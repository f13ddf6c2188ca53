"""Seeded synthetic inputs: acquisition presets, random-ellipse phantoms, noise draws.

This module holds input generation only, none of the reconstruction arithmetic.
The CUDA path and the CPU oracle both take their inputs from here. Neither side
imports the other.

The paper reconstructs a Shepp-Logan phantom in a tomosynthesis geometry
(Section 2, Example 2). Its figures and phantom table are not available, so the
workloads use seeded random ellipses instead. Densities are drawn from U[0, 1].
Images are returned as [nz][nx] arrays. Row r counts z-cells from the bottom of
the object, column c counts x-cells from the left.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1902_10559


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Parameters of one symmetric 2D acquisition.

    Lengths are in mm and gamma_deg is in degrees.

    - Object: x in [-W/2, W/2], z in [z0, z0+H], split into nx by nz cells.
    - Sources: K point sources on an arc of radius R about the detector
      centre, at angles spread evenly over [-gamma, +gamma].
    - Detector: flat at z = 0, with nb bins spanning [-D/2, D/2].
    """

    nx: int
    nz: int
    W: float
    H: float
    z0: float
    K: int
    gamma_deg: float
    R: float
    nb: int
    D: float

    @property
    def N(self) -> int:
        return self.nx * self.nz

    @property
    def M(self) -> int:
        return self.K * self.nb


# Tiny parity slice: 32 x 16 voxels, 10 sources on +/-20 deg at 600 mm,
# 64 detector bins (M = 640, N = 512).
TINY = Geometry(nx=32, nz=16, W=128.0, H=64.0, z0=50.0, K=10, gamma_deg=20.0,
                R=600.0, nb=64, D=280.0)

# Realistic slice: 512 x 128 voxels, 26 sources on +/-25 deg at 600 mm,
# 1024 detector bins (M = 26624, N = 65536).
REALISTIC = Geometry(nx=512, nz=128, W=256.0, H=128.0, z0=50.0, K=26,
                     gamma_deg=25.0, R=600.0, nb=1024, D=640.0)


def rng_for(config_id: int, stream: int = 0) -> np.random.Generator:
    """The seeded generator for one workload.

    ``stream`` selects independent draws (0 = phantom, 1 = noise, ...).
    """
    return np.random.default_rng([SEED_BASE + config_id, stream])


def ellipse_params(rng: np.random.Generator, g: Geometry, n_ellipses: int) -> np.ndarray:
    """Draw random ellipses.

    Returns an array of rows (cx, cz, ax, az, angle, density).
    - The centre lies in x U[-0.4W, 0.4W] and z z0 + U[0.1H, 0.9H].
    - The semi-axes are U[0.05, 0.3] times (W, H).
    - The angle is U[0, pi) and the density U[0, 1].
    """
    e = np.empty((n_ellipses, 6))
    e[:, 0] = rng.uniform(-0.4 * g.W, 0.4 * g.W, n_ellipses)
    e[:, 1] = g.z0 + rng.uniform(0.1 * g.H, 0.9 * g.H, n_ellipses)
    e[:, 2] = rng.uniform(0.05, 0.3, n_ellipses) * g.W
    e[:, 3] = rng.uniform(0.05, 0.3, n_ellipses) * g.H
    e[:, 4] = rng.uniform(0.0, math.pi, n_ellipses)
    e[:, 5] = rng.uniform(0.0, 1.0, n_ellipses)
    return e


def phantom_image(g: Geometry, ellipses: np.ndarray) -> np.ndarray:
    """Sum the ellipse densities, point-sampled at the cell centres.

    Returns float64 [nz][nx].
    """
    dx = g.W / g.nx
    dz = g.H / g.nz
    xc = -0.5 * g.W + (np.arange(g.nx) + 0.5) * dx
    zc = g.z0 + (np.arange(g.nz) + 0.5) * dz
    X, Z = np.meshgrid(xc, zc)  # [nz][nx]
    img = np.zeros((g.nz, g.nx))
    for cx, cz, ax, az, ang, dens in ellipses:
        ca, sa = math.cos(ang), math.sin(ang)
        xr = (X - cx) * ca + (Z - cz) * sa
        zr = -(X - cx) * sa + (Z - cz) * ca
        img += np.where((xr / ax) ** 2 + (zr / az) ** 2 <= 1.0, dens, 0.0)
    return img


def random_phantom(g: Geometry, config_id: int, n_ellipses: int, stream: int = 0) -> np.ndarray:
    """Draw a seeded random-ellipse phantom [nz][nx] (float64)."""
    return phantom_image(g, ellipse_params(rng_for(config_id, stream), g, n_ellipses))


def noise_draws(M: int, config_id: int, stream: int = 1) -> np.ndarray:
    """Draw M standard-normal values for multiplicative projection noise.

    The noisy projection is p_i (1 + sigma eps_i). A ray that misses the object
    then keeps p_i = 0.
    """
    return rng_for(config_id, stream).standard_normal(M)


def apply_noise(p: np.ndarray, eps: np.ndarray, sigma: float) -> np.ndarray:
    """Apply the multiplicative noise: p (1 + sigma eps)."""
    return p * (1.0 + sigma * eps)


def covering_detector_width(nx: int, nz: int, W: float, H: float, z0: float, K: int, gamma_deg: float,
                            R: float, margin: float = 1.02) -> float:
    """Return the smallest detector width D that covers the object's shadow from every source, times ``margin``.

    The sources sit on the arc of the acquisition.
    """
    gam = math.radians(gamma_deg)
    far = 0.0
    for k in range(K):
        th = gam * (2 * k + 1 - K) / (K - 1)
        sx, sz = R * math.sin(th), R * math.cos(th)
        for cx in (-W / 2, W / 2):
            for cz in (z0, z0 + H):
                far = max(far, abs(sx + (cx - sx) * sz / (sz - cz)))
    return 2.0 * far * margin


def table1_geometries() -> list:
    """The three sizes of Example 2 (Table 1): 32x32, 64x64 and 128x128 voxels with 24, 48 and 96 positions.

    Table 1 prints A's sizes as 1024 x 2280, 4096 x 9120 and 16384 x 36480
    (N x M), so each source has M / K = 95, 190 and 380 detector bins. The other
    parameters are not in the paper. A 128 mm square object (voxels of 4, 2
    and 1 mm) 50 mm above the detector, sources on a +/-20 deg arc at 600 mm
    and a detector covering the object's shadow give systems of full column
    rank (condition numbers of A about 4e3, 2e4 and 6e4); a 256 mm object at
    128 x 128 does not (its detector, 1068 mm wide, has bins coarser than the
    voxels).
    """
    out = []
    for n, K, nb in ((32, 24, 95), (64, 48, 190), (128, 96, 380)):
        W = H = 128.0
        D = covering_detector_width(n, n, W, H, 50.0, K, 20.0, 600.0)
        out.append(Geometry(nx=n, nz=n, W=W, H=H, z0=50.0, K=K, gamma_deg=20.0, R=600.0, nb=nb, D=D))
    return out


def batch_geometries(n_slices: int = 256, seed: int = 3, nx_choices=(256, 512, 768, 1024), nz_range=(64, 256),
                     K_range=(16, 32)) -> list:
    """Draw a batch of uneven slices with seeded sizes.

    Each slice has:
    - nx uniform in ``nx_choices``, nz uniform in ``nz_range`` and K uniform in
      ``K_range`` (both integer and inclusive);
    - nb = 2 nx detector bins;
    - cells of 0.5 mm in x and 1 mm in z, so W = nx/2 mm and H = nz mm;
    - z0 = 50 mm, sources on +/-25 deg at 600 mm;
    - the smallest covering detector width.
    """
    rng = rng_for(seed, 0)
    out = []
    for _ in range(n_slices):
        nx = int(rng.choice(nx_choices))
        nz = int(rng.integers(nz_range[0], nz_range[1] + 1))
        K = int(rng.integers(K_range[0], K_range[1] + 1))
        W, H = 0.5 * nx, 1.0 * nz
        D = covering_detector_width(nx, nz, W, H, 50.0, K, 25.0, 600.0)
        out.append(Geometry(nx=nx, nz=nz, W=W, H=H, z0=50.0, K=K, gamma_deg=25.0, R=600.0, nb=2 * nx, D=D))
    return out


def cnn_initial_params(seed: int = 5, channels: int = 32, out_scale: float = 0.1) -> np.ndarray:
    """Seeded initial parameters of the warm-start network (flat float32 vector).

    - The order is W1, b1, W2, b2, W3, b3, W4, b4, with weights [out][in][3][3].
    - Weights are He-normal: N(0, 2 / fan_in).
    - The last layer is scaled by ``out_scale``, so the untrained network is
      close to the identity through its residual path.
    - Biases start at zero.
    """
    rng = rng_for(seed, 7)
    C = channels
    parts = []
    for cin, cout, scale in ((1, C, 1.0), (C, C, 1.0), (C, C, 1.0), (C, 1, out_scale)):
        fan_in = cin * 9
        parts.append(rng.standard_normal(cout * cin * 9) * math.sqrt(2.0 / fan_in) * scale)
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float32)
