"""CUDA-graph capture of a whole reconstruction (fold p, persistent solve, recombine).

The graph is replayed on new projections and checked against direct calls.
"""
import numpy as np
import pytest

from paper_1902_10559_gb300.synthetic import TINY, Geometry, batch_geometries, random_phantom

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


@pytest.mark.parametrize("batch", [False, True])
def test_graph_replay_matches_direct_calls(ss, batch):
    if batch:
        gs = batch_geometries(n_slices=6, nx_choices=(16, 32), nz_range=(8, 16), K_range=(4, 8))
        system = ss.fold_batch([ss.make_geometry(g) for g in gs], ss.F32)
        imgs = [random_phantom(g, 60, 5, stream=k) for k, g in enumerate(gs)]
    else:
        gs = [TINY]
        system = ss.fold_system(ss.make_geometry(TINY), ss.F32)
        imgs = [random_phantom(TINY, 61, 8)]
    dev = "cuda"
    f_true = torch.as_tensor(np.concatenate([im.reshape(-1) for im in imgs]), dtype=torch.float32, device=dev)
    p = torch.empty(system.M, device=dev)
    ss.project(system, f_true, p, layout=ss.LAYOUT_IMAGE)
    p12 = torch.empty(system.Mh, 2, device=dev)
    f12 = torch.zeros(system.Nh, 2, device=dev)
    f = torch.empty(system.N, device=dev)
    opts = ss.solve_opts(50, 1.0)

    def reconstruct():
        ss.fold_rhs(system, p, p12)
        f12.zero_()
        ss.solve(system, p12, f12, opts)
        ss.recombine(system, f12, f, layout=ss.LAYOUT_IMAGE)

    reconstruct()  # warm-up outside capture (reads the fold statistics once)
    torch.cuda.synchronize()
    direct = f.clone()

    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            reconstruct()
    torch.cuda.current_stream().wait_stream(s)
    f.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(f, direct)
    # New data, same buffers: replay equals a direct run on the new data.
    p.mul_(0.5)
    graph.replay()
    torch.cuda.synchronize()
    replayed = f.clone()
    reconstruct()
    torch.cuda.synchronize()
    assert torch.equal(replayed, f)
