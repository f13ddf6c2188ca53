"""CGLS on the split systems, on the GPU, against the oracle.

Tolerances, element by element (tests/parity.py): 1e-10 for FP64 iterates,
1e-4 for FP32. Iteration counts of the stopping rule are exact.

Conjugate gradients amplify rounding on rank-deficient systems. The tiny
slice's A1 has rank 188 of 256 columns, and the oracle itself disagrees with
a copy of itself whose rows are permuted (another summation order) by 7e-15
after 10 steps, 1e-10 after 15 and 2e-4 after 25. Iterates on the tomography
slices are therefore compared over their first 10 steps (FP64) or 5 (FP32).
Longer runs are compared on a well-conditioned system given as a CSR, where
both sides also reach the least-squares solution.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import geometry as ogeo
from oracle import normal as onormal
from oracle import split as osplit
from paper_1902_10559_gb300.synthetic import REALISTIC, TINY, random_phantom
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


@pytest.fixture(scope="module")
def tiny():
    A = ogeo.mirrored_system_matrix(TINY)
    f_true = ogeo.image_to_snake(TINY, random_phantom(TINY, 1, 8))
    p = A @ f_true
    A1, A2 = osplit.fold_matrix(A)
    p1, p2 = osplit.fold_rhs(p)
    return A, p, A1, A2, p1, p2


def run_cgls(ss, system, p, iters, tol=0.0, f0=None, **kw):
    vt = system.vec_dtype
    p12 = torch.empty(system.Mh, 2, dtype=vt, device="cuda")
    f12 = torch.zeros(system.Nh, 2, dtype=vt, device="cuda")
    if f0 is not None:
        ss.fold_image(system, torch.as_tensor(f0, dtype=vt, device="cuda"), f12)
    ss.fold_rhs(system, torch.as_tensor(p, dtype=vt, device="cuda"), p12)
    ss.solve_cgls(system, p12, f12, ss.solve_opts(iters, 1.0, tol, **kw))
    info = ss.solve_result(system)
    f12 = f12.cpu().numpy().astype(np.float64)
    return info, f12, osplit.recombine(f12[:, 0], f12[:, 1])


def test_tiny_fp64_matches_oracle(ss, tiny):
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.F64)
    ref = onormal.cgls(A1, A2, p1, p2, 10)
    info, f12, f = run_cgls(ss, sysm, p, 10)
    assert info["iters"] == 10 and info["status"] == 0
    close(f12[:, 0], ref["f1"], 1e-10, "f1")
    close(f12[:, 1], ref["f2"], 1e-10, "f2")
    close_scalar(info["rho"], ref["rho"], 1e-10, "rho")
    close_scalar(info["rho"], osplit.relative_residual(A, f, p), 1e-9, "rho vs the full residual")


def test_tiny_fp32_matches_oracle(ss, tiny):
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.F32)
    ref = onormal.cgls(A1, A2, p1, p2, 5)
    info, f12, f = run_cgls(ss, sysm, p, 5)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-4, "f (FP32, 5 steps)")
    close_scalar(info["rho"], ref["rho"], 1e-4, "rho")


def test_warm_start_and_launch_shapes(ss, tiny):
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.F64)
    f0 = np.linspace(0.0, 1.0, TINY.N)
    f10, f20 = osplit.fold_image(f0)
    ref = onormal.cgls(A1, A2, p1, p2, 10, f1_0=f10, f2_0=f20)
    for lpc, threads in ((1, 128), (8, 512), (32, 256)):
        info, f12, f = run_cgls(ss, sysm, p, 10, f0=f0, lanes_per_col=lpc, block_threads=threads)
        close(f12[:, 0], ref["f1"], 1e-10, f"f1 from a warm start, LPC {lpc}")
        close(f12[:, 1], ref["f2"], 1e-10, f"f2 from a warm start, LPC {lpc}")


def test_stopping_rule_matches_oracle(ss, tiny):
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.F64)
    hist = onormal.cgls(A1, A2, p1, p2, 40, record=True)["rho_hist"]
    tol = 0.5 * (hist[6] + hist[7])
    for every in (1, 4):
        ref = onormal.cgls(A1, A2, p1, p2, 40, tol=tol, check_every=every)
        info, f12, f = run_cgls(ss, sysm, p, 40, tol=tol, check_every=every)
        assert info["iters"] == ref["iters"], (every, info, ref["iters"])
        close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-10, f"f at the stop (check every {every})")


def well_conditioned(seed=11, M=80, N=24, density=0.6):
    """A random sparse M x N matrix satisfying Eq. (2), with full-column-rank split systems."""
    rng = np.random.default_rng(seed)
    top = rng.standard_normal((M // 2, N)) * (rng.random((M // 2, N)) < density)
    A = np.vstack([top, top[::-1, ::-1]])
    return A


@pytest.mark.parametrize("consistent", [True, False])
def test_well_conditioned_system_long_run(ss, consistent):
    """40 steps on a well-conditioned 80 x 24 system: the iterates match, and both reach lstsq."""
    A = well_conditioned()
    rng = np.random.default_rng(12)
    p = A @ rng.standard_normal(24) if consistent else rng.standard_normal(80)
    half = sp.csr_matrix(A[:40])
    sysm = ss.fold_system(ss.make_geometry_from_csr(80, 24, half.indptr, half.indices, half.data), ss.F64)
    A1, A2 = osplit.fold_matrix(A)
    p1, p2 = osplit.fold_rhs(p)
    for s_ in (A1, A2):
        sv = np.linalg.svd(s_, compute_uv=False)
        assert sv[-1] > 0.05 * sv[0]  # well conditioned
    ref = onormal.cgls(A1, A2, p1, p2, 40)
    info, f12, f = run_cgls(ss, sysm, p, 40)
    close(f12[:, 0], ref["f1"], 1e-10, "f1 after 40 steps")
    close(f12[:, 1], ref["f2"], 1e-10, "f2 after 40 steps")
    close(f, np.linalg.lstsq(A, p, rcond=None)[0], 1e-10, "f against lstsq of the full system (Theorem 1)")


def test_repeatable_bitwise(ss, tiny):
    A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(TINY), ss.F32)
    a = run_cgls(ss, sysm, p, 30)
    b = run_cgls(ss, sysm, p, 30)
    assert np.array_equal(a[1], b[1]) and a[0]["rho"] == b[0]["rho"]


def test_example1_reaches_the_printed_pseudo_solutions(ss):
    """Example 1 from zero: CGLS tends to the normal pseudo-solutions printed before Eq. (18) (Theorem 2)."""
    ex = load("example1.txt")
    half = sp.csr_matrix(ex["A"][:2])
    sysm = ss.fold_system(ss.make_geometry_from_csr(4, 6, half.indptr, half.indices, half.data), ss.F64)
    info, f12, f = run_cgls(ss, sysm, ex["p"], 50, tol=1e-14)
    assert np.allclose(f12[:, 0], ex["f1_min"], atol=5e-5) and np.allclose(f12[:, 1], ex["f2_min"], atol=5e-5)
    assert np.allclose(f, ex["f_min"], atol=5e-5)
    ref = onormal.cgls(ex["A1"], ex["A2"], ex["p1"], ex["p2"], 50, tol=1e-14)
    assert info["iters"] == ref["iters"]


@pytest.mark.slow
def test_realistic_fp32_matches_oracle(ss):
    g = REALISTIC
    A = ogeo.mirrored_system_matrix(g)
    p = A @ ogeo.image_to_snake(g, random_phantom(g, 2, 20))
    A1, A2 = osplit.fold_matrix(A)
    p1, p2 = osplit.fold_rhs(p)
    sysm = ss.fold_system(ss.make_geometry(g), ss.F32)
    ref = onormal.cgls(A1, A2, p1, p2, 8)
    info, f12, f = run_cgls(ss, sysm, p, 8)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-4, "realistic CGLS, 8 steps (FP32)")
    close_scalar(info["rho"], ref["rho"], 1e-4, "rho")


def test_rejected_systems(ss):
    geom = ss.make_geometry(TINY)
    for sysm in (ss.fold_batch([geom, geom], ss.F32), ss.fold_system(geom, ss.F16)):
        p12 = torch.zeros(sysm.Mh, 2, device="cuda")
        f12 = torch.zeros(sysm.Nh, 2, device="cuda")
        with pytest.raises(ss.SplitSartError) as e:
            ss.solve_cgls(sysm, p12, f12, ss.solve_opts(5, 1.0))
        assert e.value.code == ss.ERR_ARG
