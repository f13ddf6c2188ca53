"""The autotuner on the GPU: every launch shape it may choose gives the same result.

The tuner chooses among launch shapes of one arithmetic (kernel, lanes per
column, threads, tile size, row weight), so every candidate must return f
within rounding of the library's default shape: 1e-12 element by element
in FP64 on the tiny slice, 1e-5 in FP32 on a 3-slice batch. A second tune
call of the same problem class reads the cache instead of timing again.
"""
import ctypes

import numpy as np
import pytest

from paper_1902_10559_gb300.synthetic import TINY, batch_geometries, random_phantom
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


def inputs(ss, system, gs):
    vt = system.vec_dtype
    img = torch.cat([torch.as_tensor(random_phantom(g, 7, 6, stream=k).reshape(-1), dtype=vt)
                     for k, g in enumerate(gs)]).cuda()
    p = torch.empty(system.M, dtype=vt, device="cuda")
    ss.project(system, img, p, layout=ss.LAYOUT_IMAGE)
    p12 = torch.empty(system.Mh, 2, dtype=vt, device="cuda")
    ss.fold_rhs(system, p, p12)
    return p12


def solve_with(ss, system, p12, iters, **shape):
    f12 = torch.zeros(system.Nh, 2, dtype=system.vec_dtype, device="cuda")
    ss.solve(system, p12, f12, ss.solve_opts(iters, 0.9, **shape))
    info = ss.solve_result(system)
    assert info["iters"] == iters and info["status"] == 0, (shape, info)
    return f12.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", ["tiny_f64", "batch3_f32"])
def test_every_candidate_gives_the_default_result(ss, case):
    from paper_1902_10559_gb300 import autotune
    if case == "tiny_f64":
        gs, dt, tol = [TINY], ss.F64, 1e-12
        system = ss.fold_system(ss.make_geometry(TINY), dt)
    else:
        gs, dt, tol = batch_geometries()[:3], ss.F32, 1e-5
        system = ss.fold_batch(ss.make_geometries_device(gs), dt)
    p12 = inputs(ss, system, gs)
    ref = solve_with(ss, system, p12, 20)
    ran = 0
    for c in autotune.solve_candidates(system):
        try:
            got = solve_with(ss, system, p12, 20, **c)
        except ss.SplitSartError as e:
            assert e.code == ss.ERR_ARG, (c, e)  # a shape this system cannot take is refused, not run
            continue
        close(got, ref, tol, f"{case} {c}")
        ran += 1
    assert ran >= 10


def test_second_tune_reads_the_cache(ss, tmp_path, monkeypatch):
    from paper_1902_10559_gb300 import autotune
    monkeypatch.setenv("SPLITSART_TUNE_CACHE", str(tmp_path / "tune.json"))
    system = ss.fold_system(ss.make_geometry(TINY), ss.F32)
    p12 = inputs(ss, system, [TINY])
    f12 = torch.zeros(system.Nh, 2, device="cuda")
    first = autotune.tune_solve(system, p12, f12, iters=3)
    assert torch.count_nonzero(f12).item() == 0  # the tuner restores f12
    monkeypatch.setattr(autotune, "_time_solve", lambda *a, **k: pytest.fail("timed a cached class"))
    assert autotune.tune_solve(system, p12, f12, iters=3) == first

    nrhs = 8
    pm = torch.stack([p12] * nrhs)
    fm = torch.zeros(nrhs, system.Nh, 2, device="cuda")
    m1 = autotune.tune_multi(system, pm, fm, iters=3)
    calls = []
    orig = ss.solve_multi
    monkeypatch.setattr(ss, "solve_multi", lambda *a, **k: calls.append(1) or orig(*a, **k))
    assert autotune.tune_multi(system, pm, fm, iters=3) == m1 and not calls
