"""The warm-start network on the GPU against the FP64 oracle.

- FP32 CUDA-core path: forward, gradients and Adam at 1e-4.
- BF16 tensor-core path: forward and gradients at 2e-2 (5e-2 ... 1e-1 for the
  learned part and per-block gradients), on the tiny image and on other sizes.
"""
import numpy as np
import pytest

from oracle import cnn as ocnn
from paper_1902_10559_gb300.synthetic import cnn_initial_params

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


def case(B=6, seed=0):
    rng = np.random.default_rng(seed)
    th = cnn_initial_params(seed=11, out_scale=1.0).astype(np.float64)
    p = ocnn.unpack(th)
    for k in ("b1", "b2", "b3", "b4"):  # non-zero biases exercise the bias paths
        p[k] = rng.standard_normal(p[k].shape) * 0.1
    th = ocnn.pack(p)
    x = rng.uniform(0, 1.5, (B, 16, 32))
    t = x + 0.2 * rng.standard_normal((B, 16, 32))
    return th, x, t


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def dev(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32), device="cuda").contiguous()


@pytest.mark.parametrize("mode,tol", [(0, 1e-5), (1, 2e-2)])
def test_forward_matches_oracle(ss, mode, tol):
    th, x, t = case()
    net = ss.Cnn(16, 32, 8, th)
    if mode:
        net.set_mode(1)
    y = torch.empty(6, 16, 32, device="cuda")
    net.forward(dev(x), y)
    ref, _ = ocnn.forward(th, x)
    assert rel(y.cpu().numpy(), ref) <= tol
    assert rel(y.cpu().numpy() - x, ref - x) <= 5 * tol  # the learned part alone


@pytest.mark.parametrize("mode,tol", [(0, 1e-4), (1, 2e-2)])
def test_gradients_match_oracle(ss, mode, tol):
    th, x, t = case(seed=1)
    net = ss.Cnn(16, 32, 8, th)
    if mode:
        net.set_mode(1)
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(ss.CNN_PARAMS, device="cuda")
    net.loss_grad(dev(x), dev(t), loss, grad)
    ref_loss, ref_g = ocnn.loss_and_grad(th, x, t)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - ref_loss) <= tol * ref_loss
    # Each parameter block separately, so that small blocks are checked too.
    k = 0
    for name, shape in ocnn.SHAPES:
        n = int(np.prod(shape))
        assert rel(g[k:k + n], ref_g[k:k + n]) <= (tol if mode == 0 else 5 * tol), name
        k += n


@pytest.mark.parametrize("nz,nx,B", [(7, 20, 6), (16, 48, 3), (5, 3, 2)])
def test_tensor_core_layers_any_image_size(ss, nz, nx, B):
    """The tcgen05 layers tile 128 consecutive pixels of the batch, so any image size works; a ragged last tile
    (7 x 20 x 6 = 840 pixels; 5 x 3 x 2 = 30) is padded. Forward and gradients against the oracle."""
    rng = np.random.default_rng(nz * nx)
    th = cnn_initial_params(seed=11, out_scale=1.0).astype(np.float64)
    p = ocnn.unpack(th)
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = rng.standard_normal(p[k].shape) * 0.1
    th = ocnn.pack(p)
    x = rng.uniform(0, 1.5, (B, nz, nx))
    t = x + 0.2 * rng.standard_normal((B, nz, nx))
    net = ss.Cnn(nz, nx, B, th)
    net.set_mode(1)
    y = torch.empty(B, nz, nx, device="cuda")
    net.forward(dev(x), y)
    ref, _ = ocnn.forward(th, x)
    assert rel(y.cpu().numpy(), ref) <= 2e-2
    assert rel(y.cpu().numpy() - x, ref - x) <= 1e-1
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(ss.CNN_PARAMS, device="cuda")
    net.loss_grad(dev(x), dev(t), loss, grad)
    ref_loss, ref_g = ocnn.loss_and_grad(th, x, t)
    assert abs(loss.item() - ref_loss) <= 2e-2 * ref_loss
    g = grad.cpu().numpy().astype(np.float64)
    k = 0
    for name, shape in ocnn.SHAPES:
        n = int(np.prod(shape))
        assert rel(g[k:k + n], ref_g[k:k + n]) <= 1e-1, name
        k += n


def test_adam_step_matches_oracle(ss):
    th, x, t = case(seed=2)
    net = ss.Cnn(16, 32, 8, th)
    _, g = ocnn.loss_and_grad(th, x, t)
    lr = 1e-3
    ref, m, v = ocnn.adam_step(th, np.zeros_like(th), np.zeros_like(th), g, 1, lr=lr)
    net.train_step(dev(x), dev(t), lr=lr)
    got, gm, gv = net.params(moments=True)
    clear = np.abs(g) > 1e-3 * np.abs(g).max()  # the first step is lr * sign(g) where g is clearly non-zero
    assert np.allclose(got[clear], ref[clear], rtol=0, atol=1e-6)
    assert np.all(np.abs(got - th) <= lr * (1 + 1e-3))
    assert rel(gm, m) <= 1e-4
    # Second step from the device state agrees with the oracle fed the same state.
    th1 = got.astype(np.float64)
    _, g1 = ocnn.loss_and_grad(th1, x, t)
    ref2, _, _ = ocnn.adam_step(th1, gm.astype(np.float64), gv.astype(np.float64), g1, 2, lr=lr)
    net.train_step(dev(x), dev(t), lr=lr)
    got2 = net.params()
    clear = np.abs(g1) > 1e-3 * np.abs(g1).max()
    assert np.allclose(got2[clear], ref2[clear], rtol=0, atol=2e-6)


def test_checkpoint_roundtrip(ss):
    th, x, t = case(seed=3)
    a = ss.Cnn(16, 32, 8, th)
    for _ in range(3):
        a.train_step(dev(x), dev(t))
    p, m, v = a.params(moments=True)
    b = ss.Cnn(16, 32, 8, np.zeros(ss.CNN_PARAMS, np.float32))
    b.set_params(p, m, v, step=3)
    a.train_step(dev(x), dev(t))
    b.train_step(dev(x), dev(t))
    assert np.array_equal(a.params(), b.params())


def test_training_reduces_loss(ss):
    th, x, t = case(B=8, seed=4)
    net = ss.Cnn(16, 32, 8, th)
    loss = torch.zeros(1, device="cuda")
    first = None
    for k in range(60):
        net.train_step(dev(x), dev(t), lr=2e-3, loss=loss)
        if k == 0:
            first = loss.item()
    assert loss.item() < 0.5 * first
