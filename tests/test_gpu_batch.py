"""Batches of independent slices in one persistent launch, on the GPU.

- Each slice of a batch must reproduce the single-slice solve of that slice
  and the FP64 oracle.
- Stopping is per slice: every slice stops at its own first k with
  rho_k <= tol.
"""
import numpy as np
import pytest

from oracle import geometry as ogeo
from oracle import sart as osart
from oracle import split as osplit
from paper_1902_10559_gb300.synthetic import TINY, Geometry, batch_geometries, covering_detector_width, random_phantom
from tests.parity import close, close_scalar

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ss():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_10559_gb300 import build, splitsart
    build.build()
    splitsart.lib()
    return splitsart


def small_geometry(nx, nz, K, nb):
    W, H = 4.0 * nx, 4.0 * nz
    D = covering_detector_width(nx, nz, W, H, 50.0, K, 20.0, 600.0)
    return Geometry(nx=nx, nz=nz, W=W, H=H, z0=50.0, K=K, gamma_deg=20.0, R=600.0, nb=nb, D=D)


SMALL = [TINY, small_geometry(8, 6, 4, 20), small_geometry(16, 10, 6, 34), small_geometry(24, 8, 8, 50),
         small_geometry(10, 12, 5, 26)]


def oracle_case(g, seed):
    A = ogeo.mirrored_system_matrix(g)
    f = ogeo.image_to_snake(g, random_phantom(g, 30 + seed, 6))
    p = A @ f
    A1, A2 = osplit.fold_matrix(A)
    p1, p2 = osplit.fold_rhs(p)
    return A, p, A1, A2, p1, p2


def batch_inputs(ss, geoms, dt):
    cases = [oracle_case(g, k) for k, g in enumerate(geoms)]
    vt = torch.float64 if dt == ss.F64 else torch.float32
    p = torch.as_tensor(np.concatenate([c[1] for c in cases]), dtype=vt, device="cuda")
    return cases, p


def solve(ss, system, p, iters, lam, tol=0.0, kernel=0):
    vt = system.vec_dtype
    p12 = torch.empty(system.Mh, 2, dtype=vt, device="cuda")
    f12 = torch.zeros(system.Nh, 2, dtype=vt, device="cuda")
    f = torch.empty(system.N, dtype=vt, device="cuda")
    ss.fold_rhs(system, p, p12)
    ss.solve(system, p12, f12, ss.solve_opts(iters, lam, tol, kernel=kernel))
    infos = ss.solve_result_slices(system)
    ss.recombine(system, f12, f)
    return infos, f.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dt,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_batch_matches_single_slices_and_oracle(ss, dt, tol):
    dtc = ss.DTYPE_NAMES[dt]
    geoms = [ss.make_geometry(g) for g in SMALL]
    batch = ss.fold_batch(geoms, dtc)
    assert batch.info()["nslices"] == len(SMALL)
    off = ss.system_slices(batch)
    cases, p = batch_inputs(ss, SMALL, dtc)
    infos, f = solve(ss, batch, p, 40, 0.9)
    for k, (g, geo, c) in enumerate(zip(SMALL, geoms, cases)):
        A, pk, A1, A2, p1, p2 = c
        ref = osart.split_sart(A1, A2, p1, p2, 0.9, 40)
        fk = f[off["N"][k]:off["N"][k + 1]]
        assert infos[k]["iters"] == 40 and infos[k]["status"] == 0
        close(fk, osplit.recombine(ref["f1"], ref["f2"]), tol, f"slice {k} ({dt})")
        close_scalar(infos[k]["rho"], ref["rho"], tol, f"rho of slice {k}")
        single = ss.fold_system(geo, dtc)
        _, fs = solve(ss, single, torch.as_tensor(pk, dtype=batch.vec_dtype, device="cuda"), 40, 0.9, kernel=1)
        # Two kernels with different summation orders: equal up to rounding (FP32: a few ulps per iteration).
        close(fk, fs, 1e-13 if dt == "f64" else 1e-5, f"slice {k} in the batch vs alone")


def test_batch_stops_each_slice_on_its_own(ss):
    geoms = [ss.make_geometry(g) for g in SMALL]
    batch = ss.fold_batch(geoms, ss.F64)
    cases, p = batch_inputs(ss, SMALL, ss.F64)
    hists = [osart.split_sart(c[2], c[3], c[4], c[5], 1.0, 60, record=True)["rho_hist"] for c in cases]
    tol = float(np.median([h[25] for h in hists]))
    expect = [next((k for k, r in enumerate(h) if r <= tol), 60) for h in hists]
    assert len(set(expect)) > 1  # the slices really stop at different iterations
    infos, f = solve(ss, batch, p, 60, 1.0, tol=tol)
    off = ss.system_slices(batch)
    for k, c in enumerate(cases):
        assert infos[k]["iters"] == expect[k], (k, infos[k], expect[k])
        ref = osart.split_sart(c[2], c[3], c[4], c[5], 1.0, 60, tol=tol)
        close(f[off["N"][k]:off["N"][k + 1]], osplit.recombine(ref["f1"], ref["f2"]), 1e-10, f"slice {k} at its stop")


def test_batch_layouts_and_projection(ss):
    geoms = [ss.make_geometry(g) for g in SMALL]
    batch = ss.fold_batch(geoms, ss.F64)
    off = ss.system_slices(batch)
    imgs = [random_phantom(g, 50 + k, 5) for k, g in enumerate(SMALL)]
    f_img = torch.as_tensor(np.concatenate([im.reshape(-1) for im in imgs]), device="cuda")
    p = torch.empty(batch.M, dtype=torch.float64, device="cuda")
    ss.project(batch, f_img, p, layout=ss.LAYOUT_IMAGE)
    for k, g in enumerate(SMALL):
        A = ogeo.mirrored_system_matrix(g)
        pk = p[off["M"][k]:off["M"][k + 1]].cpu().numpy()
        close(pk, A @ ogeo.image_to_snake(g, imgs[k]), 1e-12, f"p of slice {k}")
    # fold_image then recombine(image layout) is the identity (up to one rounding).
    f12 = torch.empty(batch.Nh, 2, dtype=torch.float64, device="cuda")
    ss.fold_image(batch, f_img, f12, layout=ss.LAYOUT_IMAGE)
    back = torch.empty_like(f_img)
    ss.recombine(batch, f12, back, layout=ss.LAYOUT_IMAGE)
    assert torch.allclose(back, f_img, rtol=0, atol=1e-14)


@pytest.mark.slow
def test_full_batch_sampled_slices(ss):
    """The 256-slice workload (nx in {256..1024}, nz in [64, 256], K in [16, 32], nb = 2 nx), 20 iterations, FP32.

    The smallest slice, the largest and 4 seeded random others are checked
    against the oracle, element by element at 1e-4. Their projections are the
    oracle's (FP64 A f of its own Siddon matrix, rounded to FP32 for the
    device); the other slices take device projections, which only fill the
    batch. The largest slices are where the row-streaming kernel's chunking
    and the per-slice stop tests are stressed.
    """
    gs = batch_geometries()
    geoms = ss.make_geometries_device(gs)
    batch = ss.fold_batch(geoms, ss.F32)
    off = ss.system_slices(batch)
    imgs = [random_phantom(g, 3, 12, stream=k) for k, g in enumerate(gs)]
    f_img = torch.cat([torch.as_tensor(im.reshape(-1), dtype=torch.float32) for im in imgs]).cuda()
    p = torch.empty(batch.M, device="cuda")
    ss.project(batch, f_img, p, layout=ss.LAYOUT_IMAGE)
    sizes = [g.N for g in gs]
    first, last = int(np.argmin(sizes)), int(np.argmax(sizes))
    rng = np.random.default_rng(1902_10559)
    others = [k for k in range(len(gs)) if k not in (first, last)]
    picks = [first, last] + sorted(int(k) for k in rng.choice(others, 4, replace=False))
    cases = {}
    for k in picks:
        g = gs[k]
        A = ogeo.mirrored_system_matrix(g)
        pk = (A @ ogeo.image_to_snake(g, imgs[k])).astype(np.float32)
        p[off["M"][k]:off["M"][k + 1]] = torch.as_tensor(pk, device="cuda")
        cases[k] = (A, pk.astype(np.float64))
    infos, f = solve(ss, batch, p, 20, 0.8)
    assert all(i["iters"] == 20 and i["status"] == 0 for i in infos)
    for k in picks:
        A, pk = cases[k]
        A1, A2 = osplit.fold_matrix(A)
        p1, p2 = osplit.fold_rhs(pk)
        ref = osart.split_sart(A1, A2, p1, p2, 0.8, 20)
        close(f[off["N"][k]:off["N"][k + 1]], osplit.recombine(ref["f1"], ref["f2"]), 1e-4,
              f"batch slice {k} (N = {gs[k].N})")
        close_scalar(infos[k]["rho"], ref["rho"], 1e-4, f"rho of slice {k}")
