"""Kernels 7 and 8 on the GPU: the compacted streaming solve fed by a producer warp through a shared-memory ring.

Kernels 7 (explicit fold) and 8 (implicit fold) run the iteration of kernels
5 and 6 (Eqs. 3, 4 on both split systems) with the same per-row and
per-column summation order, so they must return those kernels' iterates
bit for bit at equal lanes per column, whatever the chunk size. Pins:
- against the oracle, element by element (1e-10 FP64, 1e-4 FP32), on a slice
  and on a batch with the per-slice stopping rule, with the whole warp on a row
  and with 8 or 16 lanes per row (another fixed summation order);
- bitwise against kernels 5 and 6 on a batch large enough that every CTA
  takes many chunks (the producer's bound loads cross several groups of 32
  and the ring wraps), in FP64, FP32, BF16 and FP16, at several chunk sizes;
- rows longer than the chunk target (empty chunks in the plan), a chunk too
  large for the ring (refused before the launch), a barrier that times out.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import geometry as ogeo
from oracle import sart as osart
from oracle import split as osplit
from paper_1902_10559_gb300.synthetic import TINY, batch_geometries, random_phantom
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


def solve(ss, system, p, iters, lam, tol=0.0, **kw):
    vt = system.vec_dtype
    p12 = torch.empty(system.Mh, 2, dtype=vt, device="cuda")
    f12 = torch.zeros(system.Nh, 2, dtype=vt, device="cuda")
    ss.fold_rhs(system, torch.as_tensor(p, dtype=vt, device="cuda"), p12)
    ss.solve(system, p12, f12, ss.solve_opts(iters, lam, tol, **kw))
    infos = ss.solve_result_slices(system)
    f = torch.empty(system.N, dtype=vt, device="cuda")
    ss.recombine(system, f12, f)
    return infos, f12.cpu().numpy().astype(np.float64), f.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def tiny():
    A = ogeo.mirrored_system_matrix(TINY)
    p = A @ ogeo.image_to_snake(TINY, random_phantom(TINY, 1, 8))
    A1, A2 = osplit.fold_matrix(A)
    p1, p2 = osplit.fold_rhs(p)
    return A, p, A1, A2, p1, p2


@pytest.mark.parametrize("kernel", [7, 8])
@pytest.mark.parametrize("dt,tol", [("f64", 1e-10), ("f32", 1e-4)])
@pytest.mark.parametrize("tile", [0, 1024])
def test_tiny_matches_oracle(ss, tiny, kernel, dt, tol, tile):
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.DTYPE_NAMES[dt])
    ref = osart.split_sart(A1, A2, p1, p2, 1.0, 60)
    infos, f12, f = solve(ss, sysm, p, 60, 1.0, kernel=kernel, tile_entries=tile)
    assert infos[0]["iters"] == 60 and infos[0]["status"] == 0
    close(f, osplit.recombine(ref["f1"], ref["f2"]), tol, f"kernel {kernel} ({dt}, tile {tile})")
    close_scalar(infos[0]["rho"], ref["rho"], tol, "rho")


@pytest.mark.parametrize("kernel", [7, 8])
@pytest.mark.parametrize("dt,tol", [("f64", 1e-10), ("f32", 1e-4)])
@pytest.mark.parametrize("lpr", [8, 16])
def test_lanes_per_row_match_oracle(ss, tiny, kernel, dt, tol, lpr):
    """Fewer lanes per row sum a row in another fixed order: the oracle judges them at the stated tolerance."""
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.DTYPE_NAMES[dt])
    ref = osart.split_sart(A1, A2, p1, p2, 1.0, 60)
    infos, f12, f = solve(ss, sysm, p, 60, 1.0, kernel=kernel, lanes_per_row=lpr, tile_entries=1024)
    assert infos[0]["iters"] == 60 and infos[0]["status"] == 0
    close(f, osplit.recombine(ref["f1"], ref["f2"]), tol, f"kernel {kernel} ({dt}, {lpr} lanes per row)")
    close_scalar(infos[0]["rho"], ref["rho"], tol, "rho")
    _, f12b, _ = solve(ss, sysm, p, 60, 1.0, kernel=kernel, lanes_per_row=lpr, tile_entries=4096)
    assert np.array_equal(f12, f12b)  # the order is fixed: the chunk size does not change it


@pytest.mark.parametrize("kernel", [7, 8])
def test_stopping_rule(ss, tiny, kernel):
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.F64)
    hist = osart.split_sart(A1, A2, p1, p2, 1.0, 80, record=True)["rho_hist"]
    tol = 0.5 * (hist[20] + hist[21])
    infos, f12, f = solve(ss, sysm, p, 80, 1.0, tol=tol, kernel=kernel)
    assert infos[0]["iters"] == 21
    ref = osart.split_sart(A1, A2, p1, p2, 1.0, 80, tol=tol)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-10, "f at the stop")
    infos, _, _ = solve(ss, sysm, p, 0, 1.0, kernel=kernel)
    assert infos[0]["iters"] == 0


@pytest.mark.parametrize("kernel,lpr", [(7, 32), (8, 32), (7, 8), (8, 16)])
def test_batch_matches_oracle_and_stops_per_slice(ss, kernel, lpr):
    from tests.test_gpu_batch import SMALL
    batch = ss.fold_batch([ss.make_geometry(g) for g in SMALL], ss.F64)
    off = ss.system_slices(batch)
    cases = []
    for k, g in enumerate(SMALL):
        A = ogeo.mirrored_system_matrix(g)
        pk = A @ ogeo.image_to_snake(g, random_phantom(g, 30 + k, 6))
        A1, A2 = osplit.fold_matrix(A)
        p1, p2 = osplit.fold_rhs(pk)
        cases.append((pk, A1, A2, p1, p2))
    p = np.concatenate([c[0] for c in cases])
    hists = [osart.split_sart(c[1], c[2], c[3], c[4], 1.0, 60, record=True)["rho_hist"] for c in cases]
    tol = float(np.median([h[25] for h in hists]))
    infos, f12, f = solve(ss, batch, p, 60, 1.0, tol=tol, kernel=kernel, tile_entries=1024, lanes_per_row=lpr)
    for k, c in enumerate(cases):
        ref = osart.split_sart(c[1], c[2], c[3], c[4], 1.0, 60, tol=tol)
        assert infos[k]["iters"] == ref["iters"], (k, infos[k], ref["iters"])
        close(f[off["N"][k]:off["N"][k + 1]], osplit.recombine(ref["f1"], ref["f2"]), 1e-10, f"slice {k}")


@pytest.fixture(scope="module")
def big_batch(ss):
    """Eight slices of the batch workload (about 15 million folded entries): at 1024 entries per chunk
    every CTA takes about a hundred chunks per pass."""
    gs = batch_geometries()[:8]
    geoms = ss.make_geometries_device(gs)
    imgs = [random_phantom(g, 3, 12, stream=k) for k, g in enumerate(gs)]
    return gs, geoms, imgs


def batch_rhs(ss, system, imgs):
    f_img = torch.cat([torch.as_tensor(im.reshape(-1), dtype=system.vec_dtype) for im in imgs]).cuda()
    p = torch.empty(system.M, dtype=system.vec_dtype, device="cuda")
    ss.project(system, f_img, p, layout=ss.LAYOUT_IMAGE)
    return p.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16", "f16"])
def test_ring_equals_row_streaming_bitwise(ss, big_batch, dt):
    gs, geoms, imgs = big_batch
    batch = ss.fold_batch(geoms, ss.DTYPE_NAMES[dt])
    assert batch.info()["S"] > 152 * 32 * 1024  # more than 32 chunks of 1024 entries per CTA
    p = batch_rhs(ss, batch, imgs)
    pairs = [(5, 7)] + ([(6, 8)] if dt in ("f64", "f32") else [])
    for lpc in (4, 8):
        for k_rows, k_ring in pairs:
            _, f_rows, _ = solve(ss, batch, p, 6, 0.8, kernel=k_rows, lanes_per_col=lpc)
            for tile in (1024, 4096):
                infos, f_ring, _ = solve(ss, batch, p, 6, 0.8, kernel=k_ring, lanes_per_col=lpc, tile_entries=tile)
                assert all(i["status"] == 0 and i["iters"] == 6 for i in infos)
                assert np.array_equal(f_rows, f_ring), (dt, lpc, k_ring, tile, np.abs(f_rows - f_ring).max())


def long_row_system(M_half, N, long_len, seed=5):
    """Half rows of a system satisfying Eq. (2): short random rows and one row of long_len entries
    in distinct folded columns."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(M_half):
        if i == M_half // 2:
            js = rng.choice(N // 2, long_len, replace=False)
            js = np.where(rng.random(long_len) < 0.5, js, N - 1 - js)
        else:
            js = rng.choice(N, 6, replace=False)
        rows += [i] * len(js)
        cols += list(js)
        vals += list(rng.random(len(js)) + 0.1)
    return sp.csr_matrix((vals, (rows, cols)), shape=(M_half, N))


def test_rows_longer_than_a_chunk(ss):
    """A folded row of 3000 entries against chunks of 1024: the plan has empty chunks, and both
    kernels still match kernels 5 and 6 bitwise and the oracle."""
    half = long_row_system(400, 8000, 3000)
    A = np.vstack([half.toarray(), half.toarray()[::-1, ::-1]])
    geom = ss.make_geometry_from_csr(A.shape[0], A.shape[1], half.indptr, half.indices, half.data)
    sysm = ss.fold_system(geom, ss.F64)
    p = A @ np.random.default_rng(6).random(A.shape[1])
    _, f5, _ = solve(ss, sysm, p, 20, 1.0, kernel=5)
    _, f7, f = solve(ss, sysm, p, 20, 1.0, kernel=7, tile_entries=1024)
    assert np.array_equal(f5, f7)
    _, f6, _ = solve(ss, sysm, p, 20, 1.0, kernel=6)
    _, f8, _ = solve(ss, sysm, p, 20, 1.0, kernel=8, tile_entries=1024)
    assert np.array_equal(f6, f8)
    A1, A2 = osplit.fold_matrix(A)
    p1, p2 = osplit.fold_rhs(p)
    ref = osart.split_sart(A1, A2, p1, p2, 1.0, 20)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-10, "long rows against the oracle")


def test_chunk_larger_than_the_ring_is_refused(ss):
    half = long_row_system(4, 140000, 60000)
    geom = ss.make_geometry_from_csr(8, 140000, half.indptr, half.indices, half.data)
    sysm = ss.fold_system(geom, ss.F32)
    p12 = torch.zeros(sysm.Mh, 2, device="cuda")
    f12 = torch.zeros(sysm.Nh, 2, device="cuda")
    with pytest.raises(ss.SplitSartError) as e:
        ss.solve(sysm, p12, f12, ss.solve_opts(3, 1.0, kernel=7, tile_entries=16384))
    assert e.value.code == ss.ERR_ARG and "ring" in str(e.value)
    ss.solve(sysm, p12, f12, ss.solve_opts(3, 1.0, kernel=5))  # the row-streaming kernel takes it
    assert ss.solve_result(sysm)["status"] == 0
    with pytest.raises(ss.SplitSartError) as e:
        ss.solve(sysm, p12, f12, ss.solve_opts(3, 1.0, kernel=7, lanes_per_row=4))
    assert e.value.code == ss.ERR_ARG


@pytest.mark.parametrize("kernel", [7, 8])
def test_barrier_timeout_is_reported_and_context_survives(ss, tiny, kernel):
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.F32)
    p12 = torch.zeros(sysm.Mh, 2, device="cuda")
    f12 = torch.zeros(sysm.Nh, 2, device="cuda")
    ss.solve(sysm, p12, f12, ss.solve_opts(10, 1.0, kernel=kernel, timeout_ms=50.0, inject_barrier_fault=True))
    res = ss.solve_result(sysm, raise_on_error=False)
    assert res["status"] == ss.ERR_TIMEOUT and res["iters"] == -1
    infos, _, f = solve(ss, sysm, p, 10, 1.0, kernel=kernel)
    assert infos[0]["status"] == 0
    ref = osart.split_sart(A1, A2, p1, p2, 1.0, 10)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-4, "f after a timed-out launch")
