"""The compacted streaming kernels on the GPU: kernel 5 (explicit fold) and kernel 6 (implicit fold).

The implicit fold stores each entry of A's half rows once: its folded column
with A1's sign in bit 31 and its length w, so a1 = +-w and a2 = w (Eq. 2 and
the fold formulas after Eq. 4). Pins:
- both kernels against the oracle, element by element (1e-10 FP64, 1e-4 FP32),
  on single slices and on batches, with the per-slice stopping rule;
- on a system without ray/mirror twins (no folded cell gets both w_ij and
  w_{i,N-1-j}), the implicit and explicit folds hold the same entries in the
  same order with the same products, so kernels 5 and 6 return bitwise the
  same iterates, in FP64 and FP32. Where twins exist, the explicit fold
  subtracts the two lengths first and the implicit one multiplies them
  separately, so the two differ by rounding only.
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


def solve(ss, system, p, iters, lam, tol=0.0, f0=None, **kw):
    vt = system.vec_dtype
    p12 = torch.empty(system.Mh, 2, dtype=vt, device="cuda")
    f12 = torch.zeros(system.Nh, 2, dtype=vt, device="cuda")
    if f0 is not None:
        ss.fold_image(system, torch.as_tensor(f0, dtype=vt, device="cuda"), f12)
    ss.fold_rhs(system, torch.as_tensor(p, dtype=vt, device="cuda"), p12)
    ss.solve(system, p12, f12, ss.solve_opts(iters, lam, tol, **kw))
    infos = ss.solve_result_slices(system)
    f = torch.empty(system.N, dtype=vt, device="cuda")
    ss.recombine(system, f12, f)
    return infos, f12.cpu().numpy().astype(np.float64), f.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def tiny():
    A = ogeo.mirrored_system_matrix(TINY)
    f_true = ogeo.image_to_snake(TINY, random_phantom(TINY, 1, 8))
    p = A @ f_true
    A1, A2 = osplit.fold_matrix(A)
    p1, p2 = osplit.fold_rhs(p)
    return A, p, A1, A2, p1, p2


@pytest.mark.parametrize("kernel", [5, 6])
@pytest.mark.parametrize("dt,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_tiny_matches_oracle(ss, tiny, kernel, dt, tol):
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.DTYPE_NAMES[dt])
    ref = osart.split_sart(A1, A2, p1, p2, 1.0, 60)
    infos, f12, f = solve(ss, sysm, p, 60, 1.0, kernel=kernel)
    assert infos[0]["iters"] == 60 and infos[0]["status"] == 0
    close(f, osplit.recombine(ref["f1"], ref["f2"]), tol, f"kernel {kernel} ({dt})")
    close_scalar(infos[0]["rho"], ref["rho"], tol, "rho")


@pytest.mark.parametrize("kernel", [5, 6])
def test_stopping_rule_warm_start_and_zero_iterations(ss, tiny, kernel):
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.F64)
    hist = osart.split_sart(A1, A2, p1, p2, 1.0, 80, record=True)["rho_hist"]
    tol = 0.5 * (hist[20] + hist[21])
    infos, f12, f = solve(ss, sysm, p, 80, 1.0, tol=tol, kernel=kernel)
    assert infos[0]["iters"] == 21
    ref = osart.split_sart(A1, A2, p1, p2, 1.0, 80, tol=tol)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-10, "f at the stop")
    infos4, _, _ = solve(ss, sysm, p, 80, 1.0, tol=tol, check_every=4, kernel=kernel)
    assert infos4[0]["iters"] == 24
    f0 = 0.5 * ogeo.image_to_snake(TINY, random_phantom(TINY, 1, 8)) + 0.1
    f10, f20 = osplit.fold_image(f0)
    ref = osart.split_sart(A1, A2, p1, p2, 0.7, 25, f1_0=f10, f2_0=f20)
    infos, f12, f = solve(ss, sysm, p, 25, 0.7, f0=f0, kernel=kernel)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-10, "f from a warm start")
    infos, f12, f = solve(ss, sysm, p, 0, 1.0, f0=f0, kernel=kernel)
    assert infos[0]["iters"] == 0
    close(f, f0, 1e-14, "max_iters = 0 returns the start")


def twin_free(seed=3, M=60, N=40, density=0.3):
    """A sparse matrix satisfying Eq. (2) whose half rows never hold both j and N-1-j."""
    rng = np.random.default_rng(seed)
    top = np.zeros((M // 2, N))
    for i in range(M // 2):
        for j in range(N // 2):
            if rng.random() < density:
                c = j if rng.random() < 0.5 else N - 1 - j
                top[i, c] = rng.random() + 0.1
    return np.vstack([top, top[::-1, ::-1]])


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_implicit_equals_explicit_bitwise_without_twins(ss, dt):
    A = twin_free()
    half = sp.csr_matrix(A[: A.shape[0] // 2])
    geom = ss.make_geometry_from_csr(A.shape[0], A.shape[1], half.indptr, half.indices, half.data)
    sysm = ss.fold_system(geom, ss.DTYPE_NAMES[dt])
    assert sysm.info()["S"] == half.nnz  # no folded cell holds two lengths
    p = A @ np.random.default_rng(4).random(A.shape[1])
    for lpc in (4, 8):
        _, f5, _ = solve(ss, sysm, p, 50, 0.9, kernel=5, lanes_per_col=lpc)
        _, f6, _ = solve(ss, sysm, p, 50, 0.9, kernel=6, lanes_per_col=lpc)
        assert np.array_equal(f5, f6), (dt, lpc, np.abs(f5 - f6).max())
    A1, A2 = osplit.fold_matrix(A)
    p1, p2 = osplit.fold_rhs(p)
    ref = osart.split_sart(A1, A2, p1, p2, 0.9, 50)
    close(f6[:, 0], ref["f1"], 1e-10 if dt == "f64" else 1e-4, "f1 against the oracle")
    close(f6[:, 1], ref["f2"], 1e-10 if dt == "f64" else 1e-4, "f2 against the oracle")


def test_twins_change_only_the_rounding(ss, tiny):
    """On the tiny slice (21 twins) the implicit and explicit folds agree to FP64 rounding."""
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.F64)
    assert sysm.info()["S"] < ss.make_geometry(TINY).nnz_half
    _, f5, _ = solve(ss, sysm, p, 100, 1.0, kernel=5)
    _, f6, _ = solve(ss, sysm, p, 100, 1.0, kernel=6)
    close(f6, f5, 1e-13, "implicit vs explicit fold, FP64")


@pytest.mark.parametrize("kernel", [5, 6])
def test_launch_shapes_agree(ss, tiny, kernel):
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.F64)
    base = solve(ss, sysm, p, 30, 1.0, kernel=kernel, lanes_per_col=4, block_threads=512)[1]
    same = solve(ss, sysm, p, 30, 1.0, kernel=kernel, lanes_per_col=4, block_threads=128)[1]
    assert np.array_equal(base, same)  # per-row and per-column sums do not depend on the grid
    other = solve(ss, sysm, p, 30, 1.0, kernel=kernel, lanes_per_col=8)[1]
    close(other, base, 1e-13, "lanes per column 8 vs 4")


@pytest.mark.parametrize("kernel", [5, 6])
def test_batch_matches_oracle_and_stops_per_slice(ss, kernel):
    from tests.test_gpu_batch import SMALL
    geoms = [ss.make_geometry(g) for g in SMALL]
    batch = ss.fold_batch(geoms, ss.F64)
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
    infos, f12, f = solve(ss, batch, p, 60, 1.0, tol=tol, kernel=kernel)
    for k, c in enumerate(cases):
        ref = osart.split_sart(c[1], c[2], c[3], c[4], 1.0, 60, tol=tol)
        assert infos[k]["iters"] == ref["iters"], (k, infos[k], ref["iters"])
        close(f[off["N"][k]:off["N"][k + 1]], osplit.recombine(ref["f1"], ref["f2"]), 1e-10, f"slice {k}")


@pytest.mark.slow
def test_full_batch_implicit_sampled_slices(ss):
    """The 256-slice batch, FP32, 20 iterations, implicit fold: 4 slices against the oracle at 1e-4."""
    gs = batch_geometries()
    batch = ss.fold_batch(ss.make_geometries_device(gs), ss.F32)
    off = ss.system_slices(batch)
    imgs = [random_phantom(g, 3, 12, stream=k) for k, g in enumerate(gs)]
    f_img = torch.cat([torch.as_tensor(im.reshape(-1), dtype=torch.float32) for im in imgs]).cuda()
    p = torch.empty(batch.M, device="cuda")
    ss.project(batch, f_img, p, layout=ss.LAYOUT_IMAGE)
    sizes = [g.N for g in gs]
    picks = [int(np.argmin(sizes)), int(np.argmax(sizes)), 40, 201]
    cases = {}
    for k in picks:
        A = ogeo.mirrored_system_matrix(gs[k])
        pk = (A @ ogeo.image_to_snake(gs[k], imgs[k])).astype(np.float32)
        p[off["M"][k]:off["M"][k + 1]] = torch.as_tensor(pk, device="cuda")
        cases[k] = (A, pk.astype(np.float64))
    infos, f12, f = solve(ss, batch, p.cpu().numpy(), 20, 0.8, kernel=6)
    assert all(i["iters"] == 20 for i in infos)
    for k in picks:
        A, pk = cases[k]
        A1, A2 = osplit.fold_matrix(A)
        p1, p2 = osplit.fold_rhs(pk)
        ref = osart.split_sart(A1, A2, p1, p2, 0.8, 20)
        close(f[off["N"][k]:off["N"][k + 1]], osplit.recombine(ref["f1"], ref["f2"]), 1e-4,
              f"batch slice {k}, implicit fold")


def test_rejected_shapes(ss, tiny):
    geom = ss.make_geometry(TINY)
    sysm = ss.fold_system(geom, ss.BF16)
    p12 = torch.zeros(sysm.Mh, 2, device="cuda")
    f12 = torch.zeros(sysm.Nh, 2, device="cuda")
    with pytest.raises(ss.SplitSartError) as e:
        ss.solve(sysm, p12, f12, ss.solve_opts(5, 1.0, kernel=6))
    assert e.value.code == ss.ERR_ARG
    s32 = ss.fold_system(geom, ss.F32)
    with pytest.raises(ss.SplitSartError) as e:
        ss.solve(s32, p12, f12, ss.solve_opts(5, 1.0, kernel=5, lanes_per_col=2))
    assert e.value.code == ss.ERR_ARG


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_reduced_precision_codes_on_kernel_5(ss, tiny, fmt):
    """BF16/FP16 codes with per-row scales on the compacted kernel, against the oracle on the stored values."""
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.DTYPE_NAMES[fmt])
    out = sysm.export()
    shape = (TINY.M // 2, TINY.N // 2)
    H1 = sp.csr_matrix((out["a1"], out["col"], out["row_ptr"]), shape=shape)
    H2 = sp.csr_matrix((out["a2"], out["col"], out["row_ptr"]), shape=shape)
    ref = osart.split_sart(H1, H2, p1, p2, 1.0, 200)
    infos, f12, f = solve(ss, sysm, p, 200, 1.0, kernel=5)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-4, f"{fmt} codes, kernel 5")
    close_scalar(infos[0]["rho"], ref["rho"], 1e-4, "rho")
    # The row-streaming kernel on the same codes: the same arithmetic, the same f up to FP32 rounding.
    _, f12_3, _ = solve(ss, sysm, p, 200, 1.0, kernel=3)
    close(f12, f12_3, 1e-5, f"{fmt}: kernel 5 vs kernel 3")
