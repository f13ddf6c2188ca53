"""Reduced-precision storage on the GPU (tiny slice, 500 iterations, lambda = 1).

The folded values are stored as BF16 or FP16 codes with per-row FP32 scales,
with FP32 accumulation. The normalisers and the residual test are FP64.

- Codes: bit-exact against the oracle's quantiser. Both divide in FP32 and
  round to nearest even.
- Kernel parity: the GPU solve on the stored values against the oracle's FP64
  SART on the same dequantised matrix, at 1e-4 (FP32 accumulation), element
  by element.
- Total error: against the FP64 oracle on the exact matrix, at 2e-3
  norm-wise. This is the storage format's error (BF16 keeps 8 mantissa bits),
  not the kernel's; its worst element is printed beside it.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import geometry as ogeo
from oracle import quant as oquant
from oracle import sart as osart
from oracle import split as osplit
from paper_1902_10559_gb300.synthetic import TINY, random_phantom
from tests.parity import close, close_norm, close_scalar

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
    g = TINY
    A = ogeo.mirrored_system_matrix(g)
    f_true = ogeo.image_to_snake(g, random_phantom(g, 4, 8))
    p = A @ f_true
    A1, A2 = osplit.fold_matrix(A)
    p1, p2 = osplit.fold_rhs(p)
    return g, A, p, A1, A2, p1, p2


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_codes_match_oracle_quantiser(ss, tiny, fmt):
    g, A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(g), ss.DTYPE_NAMES[fmt])
    out = sysm.export(normalisers=True)
    Mh, Nh = g.M // 2, g.N // 2
    G1 = sp.csr_matrix((out["a1"], out["col"], out["row_ptr"]), shape=(Mh, Nh))
    G2 = sp.csr_matrix((out["a2"], out["col"], out["row_ptr"]), shape=(Mh, Nh))
    # The oracle quantises its literal fold on the union pattern (explicit zeros kept).
    pat = sp.csr_matrix((np.ones_like(out["a1"]), out["col"], out["row_ptr"]), shape=(Mh, Nh))
    for G, Aref in ((G1, A1), (G2, A2)):
        Af = sp.csr_matrix(Aref).multiply(pat.astype(bool)).tocsr()
        _, _, Bhat = oquant.quantise_rows(Af, fmt)
        assert abs(G - Bhat).max() == 0.0
    R1, C1 = osart.normalisers(G1)
    assert np.allclose(out["R"][:, 0], R1, rtol=1e-13) and np.allclose(out["C"][:, 0], C1, rtol=1e-13)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_reduced_precision_solve(ss, tiny, fmt):
    g, A, p, A1, A2, p1, p2 = tiny
    sysm = ss.fold_system(ss.make_geometry(g), ss.DTYPE_NAMES[fmt])
    out = sysm.export()
    Mh, Nh = g.M // 2, g.N // 2
    H1 = sp.csr_matrix((out["a1"], out["col"], out["row_ptr"]), shape=(Mh, Nh))
    H2 = sp.csr_matrix((out["a2"], out["col"], out["row_ptr"]), shape=(Mh, Nh))
    iters = 500
    ref_hat = osart.split_sart(H1, H2, p1, p2, 1.0, iters)
    ref_exact = osart.split_sart(A1, A2, p1, p2, 1.0, iters)
    p_d = torch.as_tensor(p, dtype=torch.float32, device="cuda")
    p12 = torch.empty(Mh, 2, device="cuda")
    f12 = torch.zeros(Nh, 2, device="cuda")
    f = torch.empty(g.N, device="cuda")
    ss.fold_rhs(sysm, p_d, p12)
    ss.solve(sysm, p12, f12, ss.solve_opts(iters, 1.0))
    info = ss.solve_result(sysm)
    ss.recombine(sysm, f12, f)
    fg = f.cpu().numpy().astype(np.float64)
    f_hat = osplit.recombine(ref_hat["f1"], ref_hat["f2"])
    f_exact = osplit.recombine(ref_exact["f1"], ref_exact["f2"])
    print(f"{fmt}: rho {info['rho']:.6e} (oracle on stored {ref_hat['rho']:.6e}, exact {ref_exact['rho']:.6e})")
    assert info["iters"] == iters
    close(fg, f_hat, 1e-4, f"{fmt}: kernel error vs oracle on the stored values")
    close_norm(fg, f_exact, 2e-3, f"{fmt}: total error vs exact FP64 (storage format)")
    close_scalar(info["rho"], ref_hat["rho"], 1e-4, "rho vs oracle on the stored values")
