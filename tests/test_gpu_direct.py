"""The direct method of Example 2 (Table 1) on the GPU, against the oracle.

The normal-equation solve (B = A^T A, Cholesky, two triangular solves) is
compared with the oracle's (oracle.normal.direct_solve, SciPy/NumPy)
element by element. Its sensitivity to rounding is kappa(B) eps =
kappa(A)^2 eps, so the tolerance is derived per system: 1e-10 on
well-conditioned random systems, and 200 kappa(A)^2 eps on the Table 1
slices, with kappa(A) computed here by SVD. The split solve (Theorem 1) and
the full solve are both checked, and a rank-deficient system reports
SPLITSART_ERR_NOT_SPD.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import geometry as ogeo
from oracle import normal as onormal
from oracle import split as osplit
from paper_1902_10559_gb300.synthetic import table1_geometries, random_phantom
from tests.parity import close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def ss():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_10559_gb300 import build, splitsart
    build.build()
    splitsart.lib()
    return splitsart


def device_csr_csc(A):
    A = sp.csr_matrix(A)
    A.sort_indices()
    T = sp.csc_matrix(A)
    T.sort_indices()
    dev = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x).astype(dt), device="cuda")
    return ((dev(A.indptr, np.int32), dev(A.indices, np.int32), dev(A.data, np.float64)),
            (dev(T.indptr, np.int32), dev(T.indices, np.int32), dev(T.data, np.float64)))


def gpu_normal_solve(ss, A, b):
    m, n = A.shape
    csr, csc = device_csr_csc(A)
    solver = ss.DenseSolver(n)
    bd = torch.as_tensor(b, dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    ss.normal_solve(solver, m, n, csr, csc, bd, x)
    return solver.result(), x.cpu().numpy()


@pytest.mark.parametrize("m,n,density,seed", [(200, 70, 0.3, 0), (300, 130, 0.2, 1), (150, 64, 0.5, 2), (40, 9, 1.0, 3)])
def test_random_systems_match_oracle_and_lstsq(ss, m, n, density, seed):
    """Ragged block counts (70, 130, 9 unknowns) and an exact multiple of the block size (64)."""
    rng = np.random.default_rng(seed)
    A = sp.random(m, n, density=density, random_state=rng, data_rvs=rng.standard_normal).toarray()
    A += np.eye(m, n) * 3.0  # full column rank, well conditioned
    b = rng.standard_normal(m)
    status, x = gpu_normal_solve(ss, A, b)
    assert status == ss.OK
    close(x, onormal.direct_solve(A, b), 1e-10, f"{m} x {n} against the oracle")
    close(x, np.linalg.lstsq(A, b, rcond=None)[0], 1e-10, f"{m} x {n} against lstsq")


def test_a_voxel_no_ray_crosses_reports_not_spd(ss):
    """A zero column (a voxel that no ray crosses) makes B's pivot exactly 0: SPLITSART_ERR_NOT_SPD."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((50, 20))
    A[:, 7] = 0.0
    status, _ = gpu_normal_solve(ss, A, rng.standard_normal(50))
    assert status == ss.ERR_NOT_SPD


def test_arguments_are_checked(ss):
    h = ss.lib()
    t = torch.zeros(8, dtype=torch.int32, device="cuda")
    v = torch.zeros(8, dtype=torch.float64, device="cuda")
    w = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    rc = h.splitsart_normal_solve(4, 2, t.data_ptr(), t.data_ptr(), v.data_ptr(), t.data_ptr(), t.data_ptr(), None, 1,
                                  v.data_ptr(), 1, v.data_ptr(), 1, w.data_ptr(), t.data_ptr(), None)
    assert rc == ss.ERR_ARG
    rc = h.splitsart_normal_solve(4, 2, t.data_ptr(), t.data_ptr(), v.data_ptr(), t.data_ptr(), t.data_ptr(),
                                  v.data_ptr(), 0, v.data_ptr(), 1, v.data_ptr(), 1, w.data_ptr(), t.data_ptr(), None)
    assert rc == ss.ERR_ARG


@pytest.mark.parametrize("size", [0, 1])
def test_table1_split_and_full_match_oracle(ss, size):
    """Table 1's 32x32 (24 positions, 95 bins) and 64x64 (48, 190) slices, consistent data p = A f_true."""
    g = table1_geometries()[size]
    A = ogeo.mirrored_system_matrix(g)
    f_true = ogeo.image_to_snake(g, random_phantom(g, 7, 10))
    p = A @ f_true
    A1, A2 = osplit.fold_matrix(A)
    Ad, A1d, A2d = A.toarray(), A1.toarray(), A2.toarray()
    kappa = np.linalg.cond(Ad)
    kappa_s = max(np.linalg.cond(A1d), np.linalg.cond(A2d))
    print(f"{g.nx}x{g.nz}: cond(A) {kappa:.3e}, max cond(A_s) {kappa_s:.3e}")
    geom = ss.make_geometry(g)
    # Split: fold, two normal-equation solves, Theorem 1.
    sysm = ss.fold_system(geom, ss.F64)
    solver = ss.DenseSolver(g.N // 2)
    pd = torch.as_tensor(p, device="cuda")
    f = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    ss.direct_split(sysm, solver, pd, f)
    assert solver.result() == ss.OK
    f_split = f.cpu().numpy()
    ref_split = onormal.split_direct_solve(Ad, p)
    close(f_split, ref_split, 200 * kappa_s ** 2 * EPS, "split direct solve against the oracle")
    # Full: the mirrored full matrix (Eq. 2), one normal-equation solve.
    rp, col, val = ss.full_csr(geom)
    status, f_full = gpu_normal_solve(ss, sp.csr_matrix((val, col, rp), shape=(g.M, g.N)), p)
    assert status == ss.OK
    close(f_full, onormal.direct_solve(Ad, p), 200 * kappa ** 2 * EPS, "full direct solve against the oracle")
    err_split = np.linalg.norm(f_split - f_true) / np.linalg.norm(f_true)
    err_full = np.linalg.norm(f_full - f_true) / np.linalg.norm(f_true)
    print(f"error against f_true: split {err_split:.3e}, full {err_full:.3e}")
    assert err_split <= 200 * kappa_s ** 2 * EPS and err_full <= 200 * kappa ** 2 * EPS
