"""Pins for the oracle's BF16/FP16 row quantisation.

The references are library rounding routines (torch's bfloat16 cast, NumPy's
float16 cast), explicit ties-to-even cases, and the format error bounds.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import quant


def test_bf16_rounding_matches_torch_cast():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000), rng.uniform(-1, 1, 20000),
                        np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** -130])]).astype(np.float32)
    ours = quant.round_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours, ref)


def test_bf16_ties_go_to_even():
    one = np.float32(1.0)
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: the even neighbour is 1.
    assert quant.round_bf16(np.array([one + np.float32(2.0 ** -8)]))[0] == 1.0
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6: the even neighbour is 1 + 2^-6.
    assert quant.round_bf16(np.array([one + np.float32(3 * 2.0 ** -8)]))[0] == np.float32(1 + 2.0 ** -6)
    # Just above the tie rounds up.
    assert quant.round_bf16(np.array([one + np.float32(2.0 ** -8 + 2.0 ** -20)]))[0] == np.float32(1 + 2.0 ** -7)


def test_f16_ties_go_to_even():
    one = np.float32(1.0)
    assert quant.round_f16(np.array([one + np.float32(2.0 ** -11)]))[0] == 1.0
    assert quant.round_f16(np.array([one + np.float32(3 * 2.0 ** -11)]))[0] == np.float32(1 + 2.0 ** -9)


@pytest.mark.parametrize("fmt,bits", [("bf16", 8), ("f16", 11)])
def test_quantise_rows_error_bound_and_scale(fmt, bits):
    rng = np.random.default_rng(1)
    B = sp.random(40, 30, density=0.3, random_state=2, data_rvs=lambda n: rng.standard_normal(n) * 5).tocsr()
    B[3, :] = 0.0
    B.eliminate_zeros()
    scales, C, Bhat = quant.quantise_rows(B, fmt)
    Bd = B.toarray()
    for i in range(B.shape[0]):
        m = np.abs(Bd[i]).max()
        assert scales[i] == np.float32(m)
    assert np.all(np.abs(C.data) <= 1.0)
    # Relative error of each code is at most half a unit in the last place.
    nz = Bd != 0
    rel = np.abs(Bhat.toarray()[nz] - Bd[nz]) / np.abs(Bd[nz])
    assert rel.max() <= 2.0 ** -bits * 1.0001 + 2.0 ** -23
    # The largest entry of each row is coded exactly as +/-1.
    for i in range(B.shape[0]):
        a, b = B.indptr[i], B.indptr[i + 1]
        if b > a:
            k = np.argmax(np.abs(B.data[a:b]))
            assert abs(C.data[a + k]) == 1.0


def test_exact_values_survive():
    B = sp.csr_matrix(np.array([[4.0, -2.0, 1.0, 0.5], [0.0, 3.0, -1.5, 0.75]]))
    for fmt in ("bf16", "f16"):
        _, _, Bhat = quant.quantise_rows(B, fmt)
        assert np.array_equal(Bhat.toarray(), B.toarray())
