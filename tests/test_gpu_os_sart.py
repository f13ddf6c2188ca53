"""Ordered-subsets SART and the non-negativity cone on the GPU, against the oracle.

Subsets are folded view pairs (nb consecutive folded rows) unless stated.
Tolerances, element by element (tests/parity.py): 1e-10 for FP64, 1e-4 for
FP32. Iteration counts of the stopping rule are exact.
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


class Case:
    def __init__(self, g, config_id, n_ell, noise=0.0):
        self.g = g
        self.A = ogeo.mirrored_system_matrix(g)
        f_true = ogeo.image_to_snake(g, random_phantom(g, config_id, n_ell))
        p = self.A @ f_true
        if noise:
            p = apply_noise(p, noise_draws(g.M, config_id), noise)
        self.p = p
        self.A1, self.A2 = osplit.fold_matrix(self.A)
        self.p1, self.p2 = osplit.fold_rhs(p)


@pytest.fixture(scope="module")
def tiny():
    return Case(TINY, 1, 8)


def run_os(ss, system, p, iters, lam, tol=0.0, subset_rows=0, cone=False, f0=None, **kw):
    vt = system.vec_dtype
    p12 = torch.empty(system.Mh, 2, dtype=vt, device="cuda")
    f12 = torch.zeros(system.Nh, 2, dtype=vt, device="cuda")
    if f0 is not None:
        ss.fold_image(system, torch.as_tensor(f0, dtype=vt, device="cuda"), f12)
    ss.fold_rhs(system, torch.as_tensor(p, dtype=vt, device="cuda"), p12)
    ss.solve_os(system, p12, f12, ss.solve_opts(iters, lam, tol, **kw), subset_rows=subset_rows, cone=cone)
    info = ss.solve_result(system)
    f12 = f12.cpu().numpy().astype(np.float64)
    return info, f12, osplit.recombine(f12[:, 0], f12[:, 1])


@pytest.mark.parametrize("cone", [False, True])
def test_tiny_fp64_matches_oracle(ss, tiny, cone):
    sysm = ss.fold_system(ss.make_geometry(tiny.g), ss.F64)
    subsets = osart.view_subsets(tiny.g.M // 2, tiny.g.nb)
    ref = osart.os_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, subsets, 0.9, 30, cone=cone)
    info, f12, f = run_os(ss, sysm, tiny.p, 30, 0.9, cone=cone)
    assert info["iters"] == 30 and info["status"] == 0
    close(f12[:, 0], ref["f1"], 1e-10, f"f1 (cone={cone})")
    close(f12[:, 1], ref["f2"], 1e-10, f"f2 (cone={cone})")
    close_scalar(info["rho"], ref["rho"], 1e-10, "rho")
    if cone:
        assert f.min() >= -1e-12 * np.abs(f).max()


@pytest.mark.parametrize("cone", [False, True])
def test_tiny_fp32_matches_oracle(ss, tiny, cone):
    sysm = ss.fold_system(ss.make_geometry(tiny.g), ss.F32)
    subsets = osart.view_subsets(tiny.g.M // 2, tiny.g.nb)
    ref = osart.os_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, subsets, 1.0, 60, cone=cone)
    info, f12, f = run_os(ss, sysm, tiny.p, 60, 1.0, cone=cone)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-4, f"f (FP32, cone={cone})")
    close_scalar(info["rho"], ref["rho"], 1e-4, "rho")


@pytest.mark.parametrize("rows", [100, 7, 320])
def test_custom_subset_sizes_and_a_ragged_last_subset(ss, tiny, rows):
    """Subsets of 100 rows (a ragged last one of 20), 7 rows (46 subsets), and one subset of all 320 rows."""
    sysm = ss.fold_system(ss.make_geometry(tiny.g), ss.F64)
    subsets = osart.view_subsets(tiny.g.M // 2, rows)
    ref = osart.os_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, subsets, 0.7, 12, cone=True)
    info, f12, f = run_os(ss, sysm, tiny.p, 12, 0.7, subset_rows=rows, cone=True)
    close(f12[:, 0], ref["f1"], 1e-10, f"f1 ({rows} rows per subset)")
    close(f12[:, 1], ref["f2"], 1e-10, f"f2 ({rows} rows per subset)")


def test_one_subset_without_cone_is_the_simultaneous_solve(ss, tiny):
    sysm = ss.fold_system(ss.make_geometry(tiny.g), ss.F64)
    ref = osart.split_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, 1.0, 40)
    info, f12, f = run_os(ss, sysm, tiny.p, 40, 1.0, subset_rows=tiny.g.M // 2)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-10, "one subset vs SART")
    close_scalar(info["rho"], ref["rho"], 1e-10, "rho")


@pytest.mark.parametrize("lpc,threads", [(1, 128), (8, 512), (32, 256)])
def test_launch_shapes_agree(ss, tiny, lpc, threads):
    sysm = ss.fold_system(ss.make_geometry(tiny.g), ss.F64)
    subsets = osart.view_subsets(tiny.g.M // 2, tiny.g.nb)
    ref = osart.os_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, subsets, 1.0, 10, cone=True)
    info, f12, f = run_os(ss, sysm, tiny.p, 10, 1.0, cone=True, lanes_per_col=lpc, block_threads=threads)
    close(f12[:, 0], ref["f1"], 1e-10, f"f1, {lpc} lanes per column, {threads} threads")
    close(f12[:, 1], ref["f2"], 1e-10, f"f2, {lpc} lanes per column, {threads} threads")


@pytest.mark.parametrize("cone", [False, True])
def test_stopping_rule_matches_oracle(ss, tiny, cone):
    sysm = ss.fold_system(ss.make_geometry(tiny.g), ss.F64)
    subsets = osart.view_subsets(tiny.g.M // 2, tiny.g.nb)
    hist = osart.os_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, subsets, 1.0, 60, cone=cone, record=True)["rho_hist"]
    tol = 0.5 * (hist[17] + hist[18])
    for every, expect in ((1, 18), (5, 20)):
        ref = osart.os_sart(tiny.A1, tiny.A2, tiny.p1, tiny.p2, subsets, 1.0, 60, tol=tol, check_every=every,
                            cone=cone)
        assert ref["iters"] == expect
        info, f12, f = run_os(ss, sysm, tiny.p, 60, 1.0, tol=tol, cone=cone, check_every=every)
        assert info["iters"] == expect, (every, info)
        close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-10, f"f at the stop (check every {every})")


def test_fewer_iterations_than_simultaneous_sart(ss, tiny):
    """On the noiseless tiny slice, ordered subsets reach rho <= 1e-2 in fewer iterations than SART."""
    sysm = ss.fold_system(ss.make_geometry(tiny.g), ss.F32)
    os_info, _, _ = run_os(ss, sysm, tiny.p, 5000, 1.0, tol=1e-2, cone=True)
    vt = sysm.vec_dtype
    p12 = torch.empty(sysm.Mh, 2, dtype=vt, device="cuda")
    f12 = torch.zeros(sysm.Nh, 2, dtype=vt, device="cuda")
    ss.fold_rhs(sysm, torch.as_tensor(tiny.p, dtype=vt, device="cuda"), p12)
    ss.solve(sysm, p12, f12, ss.solve_opts(5000, 1.0, 1e-2))
    plain = ss.solve_result(sysm)
    print(f"iterations to rho <= 1e-2: OS-SART with the cone {os_info['iters']}, SART {plain['iters']}")
    assert os_info["rho"] <= 1e-2 and plain["rho"] <= 1e-2
    assert os_info["iters"] < plain["iters"]


@pytest.mark.slow
def test_realistic_fp32_matches_oracle(ss):
    c = Case(REALISTIC, 2, 20, noise=0.01)
    sysm = ss.fold_system(ss.make_geometry(c.g), ss.F32)
    subsets = osart.view_subsets(c.g.M // 2, c.g.nb)
    ref = osart.os_sart(c.A1, c.A2, c.p1, c.p2, subsets, 0.8, 20, cone=True)
    info, f12, f = run_os(ss, sysm, c.p, 20, 0.8, cone=True)
    close(f, osplit.recombine(ref["f1"], ref["f2"]), 1e-4, "realistic OS-SART with the cone (FP32)")
    close_scalar(info["rho"], ref["rho"], 1e-4, "rho")


def test_rejected_systems(ss, tiny):
    geom = ss.make_geometry(tiny.g)
    p12 = torch.zeros(tiny.g.M // 2, 2, device="cuda")
    f12 = torch.zeros(tiny.g.N // 2, 2, device="cuda")
    for make in (lambda: ss.fold_batch([geom, geom], ss.F32), lambda: ss.fold_system(geom, ss.BF16)):
        sysm = make()
        pp = torch.zeros(sysm.Mh, 2, device="cuda")
        ff = torch.zeros(sysm.Nh, 2, device="cuda")
        with pytest.raises(ss.SplitSartError) as e:
            ss.solve_os(sysm, pp, ff, ss.solve_opts(5, 1.0))
        assert e.value.code == ss.ERR_ARG
    ex = load("example1.txt")
    half = sp.csr_matrix(ex["A"][:2])
    csr_sys = ss.fold_system(ss.make_geometry_from_csr(4, 6, half.indptr, half.indices, half.data), ss.F64)
    p = torch.zeros(2, 2, dtype=torch.float64, device="cuda")
    f = torch.zeros(3, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(ss.SplitSartError) as e:
        ss.solve_os(csr_sys, p, f, ss.solve_opts(5, 1.0))  # no geometry: the subset size must be given
    assert e.value.code == ss.ERR_ARG
    ss.solve_os(csr_sys, p, f, ss.solve_opts(5, 1.0), subset_rows=1)
    assert ss.solve_result(csr_sys)["iters"] == 0  # p = 0: rho = 0 stops at once


def test_example1_os_sart_with_the_cone_matches_oracle(ss):
    ex = load("example1.txt")
    half = sp.csr_matrix(ex["A"][:2])
    sysm = ss.fold_system(ss.make_geometry_from_csr(4, 6, half.indptr, half.indices, half.data), ss.F64)
    ref = osart.os_sart(ex["A1"], ex["A2"], ex["p1"], ex["p2"], [np.array([0]), np.array([1])], 1.0, 200, cone=True)
    info, f12, f = run_os(ss, sysm, ex["p"], 200, 1.0, subset_rows=1, cone=True)
    close(f12[:, 0], ref["f1"], 1e-10, "Example 1 f1")
    close(f12[:, 1], ref["f2"], 1e-10, "Example 1 f2")
    assert f.min() >= -1e-12
