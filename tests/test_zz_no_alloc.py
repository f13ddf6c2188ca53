"""The allocation-free solve (splitsart_solve_static) against the regular solve.

Some callers cannot call cudaMalloc. Examples are a process that reserves all
of its device memory at start-up, and a plugin inside an application that owns
the GPU's memory budget. They hand in a folded system that lives in their own
buffers. The call keeps its working memory in a fixed static device array.

This file is collected last on purpose. A failure here stops a ``-x`` run only
after every other test has run. The tests pass when run alone in a fresh
process and when run after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

from oracle import geometry as ogeo
from paper_1902_10559_gb300.synthetic import REALISTIC, TINY, random_phantom
from tests.parity import close

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


def caller_buffers(ss, system):
    """Copy a folded FP32 system into plain device tensors owned by the test (the "caller")."""
    csr = system.export(normalisers=True)
    csc = system.export_csc()
    dev = "cuda"

    def inv(x):
        out = np.zeros_like(x)
        nz = x > 0
        out[nz] = 1.0 / x[nz]
        return out.astype(np.float32)

    return {
        "rp": torch.as_tensor(csr["row_ptr"].astype(np.int32), device=dev),
        "col": torch.as_tensor(csr["col"].astype(np.int32), device=dev),
        "val": torch.as_tensor(np.stack([csr["a1"], csr["a2"]], 1).astype(np.float32), device=dev),
        "cp": torch.as_tensor(csc["col_ptr"].astype(np.int32), device=dev),
        "row": torch.as_tensor(csc["row"].astype(np.int32), device=dev),
        "valT": torch.as_tensor(np.stack([csc["a1"], csc["a2"]], 1).astype(np.float32), device=dev),
        "invR": torch.as_tensor(inv(csr["R"]), device=dev),
        "invC": torch.as_tensor(inv(csr["C"]), device=dev),
    }


@pytest.mark.parametrize("g,cfg,iters", [(TINY, 1, 100), (REALISTIC, 2, 200)])
def test_static_solve_matches_regular_solve_twice(ss, g, cfg, iters):
    geom = ss.make_geometry(g)
    system = ss.fold_system(geom, ss.F32)
    f_true = torch.as_tensor(random_phantom(g, cfg, 8).reshape(-1), dtype=torch.float32, device="cuda")
    p = torch.empty(g.M, dtype=torch.float32, device="cuda")
    ss.project(system, f_true, p, layout=ss.LAYOUT_IMAGE)
    p12 = torch.empty(g.M // 2, 2, device="cuda")
    ss.fold_rhs(system, p, p12)
    lam = 1.0 if cfg == 1 else 0.8

    f_ref = torch.zeros(g.N // 2, 2, device="cuda")
    ss.solve(system, p12, f_ref, ss.solve_opts(iters, lam))
    ref = ss.solve_result(system)

    b = caller_buffers(ss, system)
    info = torch.zeros(ctypes.sizeof(ss.SolveInfo), dtype=torch.uint8, device="cuda")
    for call in range(2):  # the static array keeps the previous call's contents
        f = torch.zeros(g.N // 2, 2, device="cuda")
        ss.solve_static(g.M // 2, g.N // 2, b["rp"], b["col"], b["val"], b["cp"], b["row"], b["valT"], b["invR"],
                        b["invC"], p12, f, ss.solve_opts(iters, lam), info)
        torch.cuda.synchronize()
        got = ss.read_info(info)
        assert got["status"] == 0 and got["iters"] == ref["iters"] == iters, (call, got, ref)
        # A different kernel from the regular solve's, so equal up to FP32 rounding, element by element.
        close(f.cpu().numpy(), f_ref.cpu().numpy(), 1e-4, f"call {call}: static solve vs regular solve")
        assert abs(got["rho"] - ref["rho"]) <= 1e-4 * ref["rho"], (call, got["rho"], ref["rho"])


def test_static_solve_rejects_too_many_rows(ss):
    t = torch.zeros(8, dtype=torch.int32, device="cuda")
    v = torch.zeros(8, 2, device="cuda")
    info = torch.zeros(ctypes.sizeof(ss.SolveInfo), dtype=torch.uint8, device="cuda")
    h = ss.lib()
    rc = h.splitsart_solve_static(70000, 4, t.data_ptr(), t.data_ptr(), v.data_ptr(), t.data_ptr(), t.data_ptr(),
                                  v.data_ptr(), v.data_ptr(), v.data_ptr(), v.data_ptr(), v.data_ptr(),
                                  ctypes.byref(ss.solve_opts(5, 1.0)), info.data_ptr(), None)
    assert rc == ss.ERR_ARG
    assert "static scratch capacity" in ss.last_error()
