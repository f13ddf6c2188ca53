"""Many right-hand sides on one system (SpMM form), on the GPU.

64 right-hand sides share the tiny slice's geometry. Every right-hand side
must match the FP64 oracle and stop on its own.
"""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import geometry as ogeo
from oracle import sart as osart
from oracle import split as osplit
from paper_1902_10559_gb300.synthetic import TINY, random_phantom
from tests.parity import close, close_norm

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
def case():
    g = TINY
    A = ogeo.mirrored_system_matrix(g)
    A1, A2 = osplit.fold_matrix(A)
    fs = [ogeo.image_to_snake(g, random_phantom(g, 40, 8, stream=r)) for r in range(64)]
    ps = [A @ f for f in fs]
    return g, A1, A2, ps


def run(ss, system, ps, iters, lam, tol=0.0, rc=0, lpr=0):
    vt = system.vec_dtype
    n = len(ps)
    p = torch.as_tensor(np.stack(ps), dtype=vt, device="cuda")
    p12 = torch.empty(n, system.Mh, 2, dtype=vt, device="cuda")
    for r in range(n):
        ss.fold_rhs(system, p[r].contiguous(), p12[r])
    f12 = torch.zeros(n, system.Nh, 2, dtype=vt, device="cuda")
    info = torch.zeros(n * ctypes.sizeof(ss.SolveInfo), dtype=torch.uint8, device="cuda")
    ss.solve_multi(system, p12, f12, ss.solve_opts(iters, lam, tol, lanes_per_row=lpr), info, rhs_per_cta=rc)
    torch.cuda.synchronize()
    return ss.read_infos(info, n), f12.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dt,tol,rc,lpr", [("f64", 1e-10, 4, 0), ("f64", 1e-10, 1, 8), ("f32", 1e-4, 1, 0),
                                           ("f32", 1e-4, 1, 4), ("f32", 1e-4, 8, 4), ("f32", 1e-4, 2, 8),
                                           ("bf16", 1e-4, 16, 0)])
def test_multi_rhs_matches_oracle(ss, case, dt, tol, rc, lpr):
    """Each right-hand side against the oracle, element by element.

    For BF16 values the oracle runs on the stored (dequantised) matrix, which
    isolates the kernel's FP32 arithmetic; the storage format's own error
    against the exact matrix is bounded norm-wise at 2e-3.
    """
    g, A1, A2, ps = case
    system = ss.fold_system(ss.make_geometry(g), ss.DTYPE_NAMES[dt])
    B1, B2 = A1, A2
    if dt == "bf16":
        out = system.export()
        shape = (g.M // 2, g.N // 2)
        B1 = sp.csr_matrix((out["a1"], out["col"], out["row_ptr"]), shape=shape)
        B2 = sp.csr_matrix((out["a2"], out["col"], out["row_ptr"]), shape=shape)
    infos, f12 = run(ss, system, ps, 100, 1.0, rc=rc, lpr=lpr)
    for r in (0, 1, 17, 63):
        p1, p2 = osplit.fold_rhs(ps[r])
        ref = osart.split_sart(B1, B2, p1, p2, 1.0, 100)
        f_ref = osplit.recombine(ref["f1"], ref["f2"])
        f = osplit.recombine(f12[r, :, 0], f12[r, :, 1])
        assert infos[r]["iters"] == 100 and infos[r]["status"] == 0
        close(f, f_ref, tol, f"right-hand side {r} ({dt}, {rc} per CTA, {lpr or 2} lanes per row)")
        if dt == "bf16":
            exact = osart.split_sart(A1, A2, p1, p2, 1.0, 100)
            close_norm(f, osplit.recombine(exact["f1"], exact["f2"]), 2e-3, f"right-hand side {r}: BF16 storage")


def test_multi_rhs_rejects_too_many_lanes(ss, case):
    g, A1, A2, ps = case
    system = ss.fold_system(ss.make_geometry(g), ss.F32)
    with pytest.raises(ss.SplitSartError) as e:
        run(ss, system, ps[:4], 5, 1.0, rc=8, lpr=8)  # 8 x 8 lanes exceed a warp
    assert e.value.code == ss.ERR_ARG


def test_multi_rhs_stop_individually(ss, case):
    g, A1, A2, ps = case
    system = ss.fold_system(ss.make_geometry(g), ss.F64)
    hists = []
    for r in range(8):
        p1, p2 = osplit.fold_rhs(ps[r])
        hists.append(osart.split_sart(A1, A2, p1, p2, 1.0, 80, record=True)["rho_hist"])
    tol = float(np.median([h[30] for h in hists]))
    expect = [next((k for k, x in enumerate(h) if x <= tol), 80) for h in hists]
    assert len(set(expect)) > 1
    infos, f12 = run(ss, system, ps[:8], 80, 1.0, tol=tol, rc=4)
    assert [i["iters"] for i in infos] == expect


def test_multi_rhs_queue_refills_slots(ss):
    """More right-hand sides than resident slots: stopped slots are refilled from the queue.

    Every right-hand side still stops at the oracle's iteration and returns the oracle's f.
    """
    g = TINY
    A = ogeo.mirrored_system_matrix(g)
    A1, A2 = osplit.fold_matrix(A)
    n = 700
    ps = [A @ ogeo.image_to_snake(g, random_phantom(g, 41, 8, stream=r)) for r in range(n)]
    system = ss.fold_system(ss.make_geometry(g), ss.F64)
    sample = [0, 1, 151, 152, 303, 304, 455, 699]
    hists = {}
    for r in sample:
        p1, p2 = osplit.fold_rhs(ps[r])
        hists[r] = osart.split_sart(A1, A2, p1, p2, 1.0, 120, record=True)["rho_hist"]
    tol = float(np.median([h[40] for h in hists.values()]))
    infos, f12 = run(ss, system, ps, 120, 1.0, tol=tol, rc=1)
    assert all(i["status"] == 0 for i in infos)
    iters = [i["iters"] for i in infos]
    assert len(set(iters)) > 1
    for r in sample:
        p1, p2 = osplit.fold_rhs(ps[r])
        ref = osart.split_sart(A1, A2, p1, p2, 1.0, 120, tol=tol)
        assert iters[r] == ref["iters"], r
        f = osplit.recombine(f12[r, :, 0], f12[r, :, 1])
        f_ref = osplit.recombine(ref["f1"], ref["f2"])
        close(f, f_ref, 1e-10, f"right-hand side {r} after refills")


@pytest.mark.parametrize("n,rc", [(13, 4), (1, 2), (61, 4)])
def test_multi_rhs_ragged_counts(ss, case, n, rc):
    """Right-hand-side counts that leave slots empty in the last CTA."""
    g, A1, A2, ps = case
    system = ss.fold_system(ss.make_geometry(g), ss.F64)
    infos, f12 = run(ss, system, ps[:n], 40, 1.0, rc=rc)
    for r in sorted({0, n // 2, n - 1}):
        p1, p2 = osplit.fold_rhs(ps[r])
        ref = osart.split_sart(A1, A2, p1, p2, 1.0, 40)
        assert infos[r]["iters"] == 40
        f = osplit.recombine(f12[r, :, 0], f12[r, :, 1])
        f_ref = osplit.recombine(ref["f1"], ref["f2"])
        close(f, f_ref, 1e-10, f"right-hand side {r} of {n}")


def test_multi_rhs_already_converged_start_stops_at_zero(ss, case):
    """A right-hand side whose start already meets tol stops at k = 0 and returns its start unchanged."""
    g, A1, A2, ps = case
    system = ss.fold_system(ss.make_geometry(g), ss.F64)
    p1, p2 = osplit.fold_rhs(ps[3])
    ref = osart.split_sart(A1, A2, p1, p2, 1.0, 400)
    tol = ref["rho"] * 1.5  # the 400-iteration iterate meets it
    vt = system.vec_dtype
    p12 = torch.empty(2, system.Mh, 2, dtype=vt, device="cuda")
    for k in range(2):
        ss.fold_rhs(system, torch.as_tensor(ps[3], dtype=vt, device="cuda"), p12[k])
    f12 = torch.zeros(2, system.Nh, 2, dtype=vt, device="cuda")
    f12[0, :, 0] = torch.as_tensor(ref["f1"], dtype=vt)
    f12[0, :, 1] = torch.as_tensor(ref["f2"], dtype=vt)
    start = f12[0].clone()
    info = torch.zeros(2 * ctypes.sizeof(ss.SolveInfo), dtype=torch.uint8, device="cuda")
    ss.solve_multi(system, p12, f12, ss.solve_opts(1000, 1.0, tol), info, rhs_per_cta=1)
    infos = ss.read_infos(info, 2)
    assert infos[0]["iters"] == 0 and torch.equal(f12[0], start)
    assert infos[1]["iters"] > 0 and infos[1]["rho"] <= tol


@pytest.mark.parametrize("rc", [1, 4])
def test_queue_order_changes_nothing_but_the_schedule(ss, case, rc):
    """splitsart_solve_multi_ordered: each right-hand side's arithmetic does not depend on its slot,
    so any queue order returns bitwise the same f and the same iteration counts."""
    g, A1, A2, ps = case
    system = ss.fold_system(ss.make_geometry(g), ss.F32)
    n = 40
    vt = system.vec_dtype
    p = torch.as_tensor(np.stack(ps[:n]), dtype=vt, device="cuda")
    p12 = torch.empty(n, system.Mh, 2, dtype=vt, device="cuda")
    for r in range(n):
        ss.fold_rhs(system, p[r].contiguous(), p12[r])
    outs = []
    for order in (None, torch.arange(n - 1, -1, -1, dtype=torch.int32, device="cuda"),
                  torch.as_tensor(np.random.default_rng(3).permutation(n).astype(np.int32), device="cuda")):
        f12 = torch.zeros(n, system.Nh, 2, dtype=vt, device="cuda")
        info = torch.zeros(n * ctypes.sizeof(ss.SolveInfo), dtype=torch.uint8, device="cuda")
        ss.solve_multi(system, p12, f12, ss.solve_opts(300, 1.0, 2e-2), info, rhs_per_cta=rc, order=order)
        outs.append((f12.cpu().numpy(), [i["iters"] for i in ss.read_infos(info, n)]))
    assert len(set(outs[0][1])) > 1  # the right-hand sides stop at different iterations
    for f, its in outs[1:]:
        assert np.array_equal(f, outs[0][0]) and its == outs[0][1]
