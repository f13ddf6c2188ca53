"""The learned warm start, end to end on the GPU (reduced training set).

The network is trained on 5-iteration -> 500-iteration image pairs made by the
library's own solver. On held-out phantoms:
- it must bring the 5-iteration image closer to the 500-iteration one;
- at the metric's tolerance, rho <= 1e-3, a warm-started solve of 512 held-out
  phantoms must take fewer iterations than plain split-SART from zero, and
  less wall time (median of three launches each; the continuation takes its
  right-hand sides longest first).
The oracle's FP64 residual judges the warm-started result.
"""
import numpy as np
import pytest

from oracle import geometry as ogeo
from oracle import split as osplit
from paper_1902_10559_gb300.synthetic import TINY

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_10559_gb300 import build, splitsart
    build.build()
    splitsart.lib()
    from paper_1902_10559_gb300.warmstart import WarmStart
    return WarmStart(chunk=256, max_batch=64)


def test_training_data_and_warm_start_gain(ws):
    x, t = ws.make_pairs(range(6000))
    assert x.shape == (6000, 16, 32) and torch.isfinite(t).all()
    hist = ws.train(x, t, epochs=8, batch=64, lr=1e-3)
    assert hist[-1] < 0.8 * hist[0], hist
    held = range(10**6, 10**6 + 128)
    xe, te = ws.make_pairs(held)
    guess = ws.predict(xe)
    # In image space the network brings the 5-iteration image closer to the 500-iteration image.
    assert (guess - te).norm() < 0.85 * (xe - te).norm()
    tol = 1e-3
    held = range(10**6, 10**6 + 512)
    runs = [ws.compare(held, tol=tol, max_iters=40000) for _ in range(3)]
    res = runs[0]
    assert np.all(res["rho_plain"] <= tol) and np.all(res["rho_warm"] <= tol)
    ms_plain = float(np.median([r["ms_plain"] for r in runs]))
    ms_warm = float(np.median([r["ms_warm"] for r in runs]))
    print(f"to rho <= {tol}: iterations plain {res['iters_plain'].mean():.0f}, warm {res['iters_warm'].mean():.0f}; "
          f"time plain {ms_plain:.1f} ms, warm {ms_warm:.1f} ms; warm kept {res['warm_kept']:.2f}")
    # Gain at the metric's tolerance: fewer iterations on average and for most phantoms, and less time.
    assert res["iters_warm"].mean() < 0.97 * res["iters_plain"].mean(), (res["iters_warm"].mean(),
                                                                        res["iters_plain"].mean())
    assert np.mean(res["iters_warm"] < res["iters_plain"]) > 0.6
    assert ms_warm < ms_plain, (ms_warm, ms_plain)


def test_oracle_judges_warm_start_residual(ws):
    """The oracle's FP64 residual ||A f - p|| / ||p|| of a warm-started image is within the tolerance."""
    import ctypes
    from paper_1902_10559_gb300 import splitsart as ss
    seeds = range(2 * 10**6, 2 * 10**6 + 4)
    truth = ws.phantoms(seeds)
    p = ws.project(truth)
    p12 = ws.fold_rhs(p)
    f12 = torch.zeros(4, TINY.N // 2, 2, device="cuda")
    ws.solve(p12, f12, 5)
    guess = ws.fold_image(ws.predict(ws.recombine(f12)))
    info = ws.solve(p12, guess, 20000, tol=2e-3)
    img = ws.recombine(guess).cpu().numpy().astype(np.float64)
    A = ogeo.mirrored_system_matrix(TINY)
    for r in range(4):
        f = ogeo.image_to_snake(TINY, img[r])
        rho = osplit.relative_residual(A, f, p[r].double().cpu().numpy())
        assert rho <= 2e-3 * 1.01, (r, rho)


@pytest.mark.gpu
def test_training_checkpoint_resumes_exactly(tmp_path):
    """Per-epoch checkpoints (weights, Adam moments, step): a resumed run continues bit for bit."""
    from paper_1902_10559_gb300.warmstart import WarmStart
    a = WarmStart(chunk=64, max_batch=32)
    x, t = a.make_pairs(np.arange(128))
    ck = tmp_path / "ws.npz"
    a.train(x, t, epochs=1, batch=32, seed=1, checkpoint=str(ck))
    b = WarmStart(chunk=64, max_batch=32)
    b.load(str(ck))
    assert b.steps == a.steps == 4
    a.train(x, t, epochs=1, batch=32, seed=2)
    b.train(x, t, epochs=1, batch=32, seed=2)
    assert np.array_equal(a.cnn.params(), b.cnn.params())
