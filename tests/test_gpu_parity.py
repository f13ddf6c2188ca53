"""GPU parity of the CUDA path against the CPU FP64 oracle, through the C ABI.

Tolerances, element by element (tests/parity.py: relative where the oracle's
value is at least a tenth of its largest, absolute at that level elsewhere):
- FP64 iterates: 1e-10.
- FP32 iterates: 1e-4.
- Index work (patterns, CSC order, iteration counts): exact.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import geometry as ogeo
from oracle import sart as osart
from oracle import split as osplit
from paper_1902_10559_gb300.synthetic import REALISTIC, TINY, apply_noise, noise_draws, random_phantom
from tests.golden.loader import load
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


DEV = "cuda"


class Case:
    def __init__(self, g, config_id, n_ell, noise=0.0):
        self.g = g
        self.A = ogeo.mirrored_system_matrix(g)
        self.f_true = ogeo.image_to_snake(g, random_phantom(g, config_id, n_ell))
        p = self.A @ self.f_true
        if noise:
            p = apply_noise(p, noise_draws(g.M, config_id), noise)
        self.p = p
        self.A1, self.A2 = osplit.fold_matrix(self.A)
        self.p1, self.p2 = osplit.fold_rhs(p)


@pytest.fixture(scope="module")
def tiny():
    return Case(TINY, 1, 8)


@pytest.fixture(scope="module")
def realistic():
    return Case(REALISTIC, 2, 20, noise=0.01)


def run_solve(ss, system, p, iters, lam, tol=0.0, f0=None, **kw):
    vt = system.vec_dtype
    p_d = torch.as_tensor(p, dtype=vt, device=DEV)
    p12 = torch.empty(system.Mh, 2, dtype=vt, device=DEV)
    f12 = torch.zeros(system.Nh, 2, dtype=vt, device=DEV)
    if f0 is not None:
        ss.fold_image(system, torch.as_tensor(f0, dtype=vt, device=DEV), f12)
    ss.fold_rhs(system, p_d, p12)
    ss.solve(system, p12, f12, ss.solve_opts(iters, lam, tol, **kw))
    info = ss.solve_result(system)
    f = torch.empty(system.N, dtype=vt, device=DEV)
    ss.recombine(system, f12, f)
    return info, f12.cpu().numpy().astype(np.float64), f.cpu().numpy().astype(np.float64)


def test_example1_fold_on_gpu_matches_printed_systems(ss):
    ex = load("example1.txt")
    A = ex["A"]
    half = sp.csr_matrix(A[:2])
    geom = ss.make_geometry_from_csr(4, 6, half.indptr, half.indices, half.data)
    sysm = ss.fold_system(geom, ss.F64)
    out = sysm.export()
    dense1 = sp.csr_matrix((out["a1"], out["col"], out["row_ptr"]), shape=(2, 3)).toarray()
    dense2 = sp.csr_matrix((out["a2"], out["col"], out["row_ptr"]), shape=(2, 3)).toarray()
    assert np.array_equal(dense1, ex["A1"])
    assert np.array_equal(dense2, ex["A2"])
    # The union pattern keeps all 6 positions, with A1[0, 0] = 1 - 1 = 0 by cancellation.
    info = sysm.info()
    assert info["S"] == 6 == osplit.folded_pattern_size(sp.csr_matrix(A)) and info["exact_zeros"] == 1
    p = torch.tensor(ex["p"], dtype=torch.float64, device=DEV)
    p12 = torch.empty(2, 2, dtype=torch.float64, device=DEV)
    ss.fold_rhs(sysm, p, p12)
    got = p12.cpu().numpy()
    assert np.array_equal(got[:, 0], ex["p1"]) and np.array_equal(got[:, 1], ex["p2"])
    # Recombination of the printed normal pseudo-solutions (Theorem 2).
    f12 = torch.tensor(np.stack([ex["f1_min"], ex["f2_min"]], 1), dtype=torch.float64, device=DEV)
    f = torch.empty(6, dtype=torch.float64, device=DEV)
    ss.recombine(sysm, f12, f)
    assert np.allclose(f.cpu().numpy(), ex["f_min"], atol=1e-4)


def test_fold_csc_and_normalisers_match_oracle_fp64(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F64)
    info = sysm.info()
    out = sysm.export(normalisers=True)
    S = info["S"]
    assert S == osplit.folded_pattern_size(tiny.A)
    Mh, Nh = tiny.g.M // 2, tiny.g.N // 2
    G1 = sp.csr_matrix((out["a1"], out["col"], out["row_ptr"]), shape=(Mh, Nh))
    G2 = sp.csr_matrix((out["a2"], out["col"], out["row_ptr"]), shape=(Mh, Nh))
    scale = abs(tiny.A).max()
    assert abs(G1 - tiny.A1).max() <= 1e-12 * scale
    assert abs(G2 - tiny.A2).max() <= 1e-12 * scale
    # Columns ascending within each row.
    for i in range(Mh):
        c = out["col"][out["row_ptr"][i]:out["row_ptr"][i + 1]]
        assert np.all(np.diff(c) > 0)
    csc = sysm.export_csc()
    T1 = sp.csc_matrix((csc["a1"], csc["row"], csc["col_ptr"]), shape=(Mh, Nh))
    assert abs(T1 - G1).max() == 0.0
    for j in range(Nh):
        r = csc["row"][csc["col_ptr"][j]:csc["col_ptr"][j + 1]]
        assert np.all(np.diff(r) > 0)
    R1, C1 = osart.normalisers(tiny.A1)
    R2, C2 = osart.normalisers(tiny.A2)
    assert np.allclose(out["R"][:, 0], R1, rtol=1e-12) and np.allclose(out["R"][:, 1], R2, rtol=1e-12)
    assert np.allclose(out["C"][:, 0], C1, rtol=1e-12) and np.allclose(out["C"][:, 1], C2, rtol=1e-12)
    assert info["empty_rows"] == int(np.sum(np.diff(out["row_ptr"]) == 0))


def test_tiny_fp64_solve_matches_oracle(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F64)
    ref = osart.split_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, 1.0, 100)
    info, f12, f = run_solve(ss, sysm, tiny.p, 100, 1.0)
    assert info["iters"] == 100 and info["status"] == 0
    close(f12[:, 0], ref["f1"], 1e-10, "f1")
    close(f12[:, 1], ref["f2"], 1e-10, "f2")
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-10, "f")
    assert abs(info["rho"] - ref["rho"]) <= 1e-10 * ref["rho"]
    # rho equals the full-system relative residual of the recombined image.
    assert abs(info["rho"] - osplit.relative_residual(tiny.A, f, tiny.p)) <= 1e-9 * info["rho"]


@pytest.mark.parametrize("lpc,threads", [(1, 256), (4, 128), (16, 64), (32, 256)])
def test_launch_shapes_agree(ss, tiny, lpc, threads):
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F64)
    ref = osart.split_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, 1.0, 30)
    info, f12, f = run_solve(ss, sysm, tiny.p, 30, 1.0, lanes_per_col=lpc, block_threads=threads)
    close(f12[:, 0], ref["f1"], 1e-10, "f1")
    close(f12[:, 1], ref["f2"], 1e-10, "f2")


def test_solve_is_bitwise_reproducible(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F32)
    a = run_solve(ss, sysm, tiny.p, 50, 1.0)
    b = run_solve(ss, sysm, tiny.p, 50, 1.0)
    assert np.array_equal(a[1], b[1]) and a[0]["rho"] == b[0]["rho"]


def test_tiny_fp32_solve_matches_oracle(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F32)
    ref = osart.split_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, 1.0, 100)
    info, f12, f = run_solve(ss, sysm, tiny.p, 100, 1.0)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-4, "f (FP32)")
    close_scalar(info["rho"], ref["rho"], 1e-4, "rho")


def test_stopping_rule_matches_oracle(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F64)
    hist = osart.split_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, 1.0, 80, record=True)["rho_hist"]
    tol = 0.5 * (hist[20] + hist[21])
    ref = osart.split_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, 1.0, 80, tol=tol)
    info, f12, f = run_solve(ss, sysm, tiny.p, 80, 1.0, tol=tol)
    assert info["iters"] == ref["iters"] == 21
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-10, "f at the stop")
    # Checking every 4th iteration stops at the first multiple of 4 past the crossing.
    info4, _, _ = run_solve(ss, sysm, tiny.p, 80, 1.0, tol=tol, check_every=4)
    assert info4["iters"] == 24


def test_warm_start_matches_oracle(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F64)
    f0 = 0.5 * tiny.f_true + 0.1
    f10, f20 = osplit.fold_image(f0)
    ref = osart.split_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, 0.7, 25, f1_0=f10, f2_0=f20)
    info, f12, f = run_solve(ss, sysm, tiny.p, 25, 0.7, f0=f0)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-10, "f from a warm start")


def test_zero_iterations_returns_f0_and_initial_residual(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F64)
    info, f12, f = run_solve(ss, sysm, tiny.p, 0, 1.0)
    assert info["iters"] == 0 and np.all(f == 0) and info["rho"] == pytest.approx(1.0, rel=1e-14)


@pytest.mark.parametrize("kernel", [1, 2, 3, 4])
def test_start_that_meets_tol_stops_at_zero(ss, tiny, kernel):
    """A start that already meets tol returns unchanged with iters = 0, whatever the kernel."""
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F64)
    ref = osart.split_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, 1.0, 300)
    f0 = osplit.recombine(ref["f1"], ref["f2"])
    info, f12, f = run_solve(ss, sysm, tiny.p, 1000, 1.0, tol=1.5 * ref["rho"], f0=f0, kernel=kernel)
    assert info["iters"] == 0 and info["status"] == 0
    assert info["rho"] <= 1.5 * ref["rho"]
    close(f, f0, 1e-14, "returned start")


def test_project_matches_oracle(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    for dt, tol in ((ss.F64, 1e-12), (ss.F32, 1e-6)):
        sysm = ss.fold_system(geom, dt)
        f = torch.as_tensor(tiny.f_true, dtype=sysm.vec_dtype, device=DEV)
        p = torch.empty(tiny.g.M, dtype=sysm.vec_dtype, device=DEV)
        ss.project(sysm, f, p)
        close(p.cpu().numpy(), tiny.A @ tiny.f_true, tol, "p = A f")
        img = torch.as_tensor(ogeo.snake_to_image(tiny.g, tiny.f_true), dtype=sysm.vec_dtype, device=DEV)
        ss.project(sysm, img.reshape(-1), p, layout=ss.LAYOUT_IMAGE)
        close(p.cpu().numpy(), tiny.A @ tiny.f_true, tol, "p = A f (image layout)")


def test_image_layout_recombine(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F64)
    f1, f2 = osplit.fold_image(tiny.f_true)
    f12 = torch.tensor(np.stack([f1, f2], 1), device=DEV)
    out = torch.empty(tiny.g.N, dtype=torch.float64, device=DEV)
    ss.recombine(sysm, f12, out, layout=ss.LAYOUT_IMAGE)
    # (f2 + f1)/2 reproduces f_j up to one rounding of the fold.
    got = out.cpu().numpy().reshape(tiny.g.nz, tiny.g.nx)
    assert np.allclose(got, ogeo.snake_to_image(tiny.g, tiny.f_true), rtol=0, atol=4e-16 * np.abs(tiny.f_true).max())


def test_empty_system_and_zero_rhs(ss):
    # Rows with no entries: nothing moves, and rho stays 1.
    geom = ss.make_geometry_from_csr(8, 6, np.zeros(5, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0))
    sysm = ss.fold_system(geom, ss.F64)
    assert sysm.info()["S"] == 0 and sysm.info()["empty_rows"] == 4
    info, f12, f = run_solve(ss, sysm, np.arange(8.0) + 1, 5, 1.0)
    assert info["iters"] == 5 and np.all(f == 0) and info["rho"] == pytest.approx(1.0)
    # p = 0: rho is defined as 0, so the solve stops at k = 0.
    ex = load("example1.txt")
    half = sp.csr_matrix(ex["A"][:2])
    s2 = ss.fold_system(ss.make_geometry_from_csr(4, 6, half.indptr, half.indices, half.data), ss.F64)
    info, f12, f = run_solve(ss, s2, np.zeros(4), 10, 1.0, tol=1e-3)
    assert info["iters"] == 0 and info["rho"] == 0.0


def test_example1_solve_converges_to_weighted_min_norm(ss):
    ex = load("example1.txt")
    half = sp.csr_matrix(ex["A"][:2])
    sysm = ss.fold_system(ss.make_geometry_from_csr(4, 6, half.indptr, half.indices, half.data), ss.F64)
    ref = osart.split_sart(ex["A1"], ex["A2"], ex["p1"], ex["p2"], 1.0, 3000)
    info, f12, f = run_solve(ss, sysm, ex["p"], 3000, 1.0)
    close(f12[:, 0], ref["f1"], 1e-10, "f1")
    close(f12[:, 1], ref["f2"], 1e-10, "f2")
    assert np.allclose(ex["A"] @ f, ex["p"], atol=1e-8)  # consistent system: residual -> 0


def test_barrier_timeout_is_reported_and_context_survives(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F32)
    vt = sysm.vec_dtype
    p12 = torch.zeros(sysm.Mh, 2, dtype=vt, device=DEV)
    f12 = torch.zeros(sysm.Nh, 2, dtype=vt, device=DEV)
    ss.solve(sysm, p12, f12, ss.solve_opts(10, 1.0, timeout_ms=50.0, inject_barrier_fault=True))
    res = ss.solve_result(sysm, raise_on_error=False)
    assert res["status"] == ss.ERR_TIMEOUT and res["iters"] == -1
    # The context is still usable.
    ref = osart.split_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, 1.0, 10)
    info, f12b, f = run_solve(ss, sysm, tiny.p, 10, 1.0)
    assert info["status"] == 0
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-4, "f after a timed-out launch")


def test_bad_solve_arguments(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.F32)
    p12 = torch.zeros(sysm.Mh, 2, device=DEV)
    f12 = torch.zeros(sysm.Nh, 2, device=DEV)
    for kw in ({"lam": 0.0}, {"lam": 1.0, "tol": -1.0}, {"lam": 1.0, "lanes_per_col": 3},
               {"lam": 1.0, "block_threads": 48}, {"lam": 1.0, "row_weight": -1}):
        lam = kw.pop("lam")
        with pytest.raises(ss.SplitSartError) as e:
            ss.solve(sysm, p12, f12, ss.solve_opts(5, lam, **kw))
        assert e.value.code == ss.ERR_ARG
    with pytest.raises(ValueError):
        ss.solve(sysm, p12[:-1], f12, ss.solve_opts(5, 1.0))


@pytest.mark.slow
def test_realistic_fp32_solve_matches_oracle(ss, realistic):
    """512 x 128 voxels, 26 sources, 1024 bins, 1% noise, 200 iterations, lambda = 0.8, FP32 vs FP64 oracle."""
    c = realistic
    geom = ss.make_geometry(c.g)
    sysm = ss.fold_system(geom, ss.F32)
    assert sysm.info()["S"] == osplit.folded_pattern_size(c.A)
    ref = osart.split_sart(c.A1, c.A2, c.p1, c.p2, 0.8, 200)
    info, f12, f = run_solve(ss, sysm, c.p, 200, 0.8)
    assert info["iters"] == 200
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-4, "realistic f (FP32)")
    close_scalar(info["rho"], ref["rho"], 1e-4, "rho")


@pytest.mark.parametrize("dt,tol", [("f64", 1e-10), ("f32", 1e-4), ("bf16", 1e-4)])
def test_resident_and_streaming_kernels_agree_with_oracle(ss, tiny, dt, tol):
    """Both solve kernels (matrix kept in shared memory; matrix streamed) reproduce the oracle on stored values."""
    geom = ss.make_geometry(tiny.g)
    sysm = ss.fold_system(geom, ss.DTYPE_NAMES[dt])
    out = sysm.export()
    Mh, Nh = tiny.g.M // 2, tiny.g.N // 2
    H1 = sp.csr_matrix((out["a1"], out["col"], out["row_ptr"]), shape=(Mh, Nh))
    H2 = sp.csr_matrix((out["a2"], out["col"], out["row_ptr"]), shape=(Mh, Nh))
    ref = osart.split_sart(H1, H2, tiny.p1, tiny.p2, 1.0, 60)
    f_ref = osplit.recombine(ref["f1"], ref["f2"])
    for kernel in (1, 2, 3, 4):
        info, f12, f = run_solve(ss, sysm, tiny.p, 60, 1.0, kernel=kernel)
        assert info["iters"] == 60
        close(f, f_ref, tol, f"kernel {kernel}, {dt}")
        close_scalar(info["rho"], ref["rho"], tol, f"rho, kernel {kernel}")


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_resident_row_plans_give_the_same_f(ss, realistic, dt):
    """The row weight only changes which CTA holds a row; each row's sum keeps its order, so f is bitwise equal."""
    c = realistic
    sysm = ss.fold_system(ss.make_geometry(c.g), ss.DTYPE_NAMES[dt])
    runs = [run_solve(ss, sysm, c.p, 40, 0.8, kernel=2, lanes_per_col=4, row_weight=w) for w in (1, 160, 320)]
    for info, f12, _ in runs[1:]:
        assert info["iters"] == 40 and np.array_equal(f12, runs[0][1])
        assert abs(info["rho"] - runs[0][0]["rho"]) <= 1e-6 * runs[0][0]["rho"]  # norm groups follow the plan


@pytest.mark.slow
def test_realistic_kernels_agree(ss, realistic):
    c = realistic
    sysm = ss.fold_system(ss.make_geometry(c.g), ss.F32)
    a = run_solve(ss, sysm, c.p, 50, 0.8, kernel=1)
    b = run_solve(ss, sysm, c.p, 50, 0.8, kernel=2)
    close(a[2], b[2], 1e-5, "kernel 1 vs 2")
    close_scalar(a[0]["rho"], b[0]["rho"], 1e-5, "rho, kernel 1 vs 2")
    for kernel in (3, 4):
        d = run_solve(ss, sysm, c.p, 50, 0.8, kernel=kernel)
        close(d[2], b[2], 1e-5, f"kernel {kernel} vs 2")
        close_scalar(d[0]["rho"], b[0]["rho"], 1e-5, f"rho, kernel {kernel} vs 2")
