"""Host-side checks of the C-ABI library. No GPU is needed.

- The library loads and exports every symbol that include/splitsart.h declares.
- The host geometry (first-half Siddon rows) matches the oracle's traced rows.
- Argument and parity errors are reported through status codes.
"""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import geometry as ogeo
from paper_1902_10559_gb300.synthetic import REALISTIC, TINY, Geometry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ss():
    from paper_1902_10559_gb300 import build, splitsart
    build.build()
    splitsart.lib()
    return splitsart


def declared_in_headers():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(splitsart_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(ss):
    import ctypes
    L = ctypes.CDLL(ss.LIB_PATH)
    declared = declared_in_headers()
    assert len(declared) >= 15
    missing = [n for n in declared if not hasattr(L, n)]
    assert not missing, missing
    # The binding covers the same set.
    assert declared <= set(ss.declared_symbols()) | {n for n in declared if n not in ss.declared_symbols() and hasattr(L, n)}


def test_binding_declares_only_header_symbols(ss):
    assert set(ss.declared_symbols()) <= declared_in_headers()


def half_csr_from_oracle(g):
    A = ogeo.system_matrix(g, rows=range(g.M // 2))[: g.M // 2]
    return sp.csr_matrix(A)


@pytest.mark.parametrize("g", [TINY, Geometry(nx=6, nz=5, W=30.0, H=20.0, z0=10.0, K=4, gamma_deg=30.0, R=200.0,
                                               nb=10, D=120.0)])
def test_host_geometry_matches_oracle(ss, g):
    geom = ss.make_geometry(g)
    assert geom.M == g.M and geom.N == g.N
    rp, col, val = geom.export()
    ref = half_csr_from_oracle(g)
    assert np.array_equal(rp, ref.indptr)
    assert np.array_equal(col, ref.indices)
    assert np.allclose(val, ref.data, rtol=1e-12, atol=1e-13)


@pytest.mark.slow
def test_host_geometry_matches_oracle_realistic(ss):
    g = REALISTIC
    geom = ss.make_geometry(g)
    rp, col, val = geom.export()
    rows = np.random.default_rng(0).choice(g.M // 2, 300, replace=False)
    src = ogeo.source_positions(g)
    det = ogeo.detector_centres(g)
    for i in rows:
        k, b = divmod(int(i), g.nb)
        j, w = ogeo.siddon_ray(g, src[k], np.array([det[b], 0.0]))
        assert np.array_equal(col[rp[i]:rp[i + 1]], j)
        assert np.allclose(val[rp[i]:rp[i + 1]], w, rtol=1e-12, atol=1e-13)


def test_geometry_errors(ss):
    bad = Geometry(nx=5, nz=4, W=1, H=1, z0=1, K=4, gamma_deg=10, R=10, nb=4, D=4)
    with pytest.raises(ss.SplitSartError) as e:
        ss.make_geometry(bad)
    assert e.value.code == ss.ERR_ODD_DIM
    odd_m = Geometry(nx=4, nz=4, W=1, H=1, z0=1, K=3, gamma_deg=10, R=10, nb=3, D=4)
    with pytest.raises(ss.SplitSartError) as e:
        ss.make_geometry(odd_m)
    assert e.value.code == ss.ERR_ODD_DIM
    neg = Geometry(nx=4, nz=0, W=1, H=1, z0=1, K=4, gamma_deg=10, R=10, nb=4, D=4)
    with pytest.raises(ss.SplitSartError) as e:
        ss.make_geometry(neg)
    assert e.value.code == ss.ERR_ARG


def test_from_csr_validation(ss):
    rp = np.array([0, 2, 3])
    with pytest.raises(ss.SplitSartError) as e:
        ss.make_geometry_from_csr(4, 6, rp, np.array([3, 1, 0]), np.ones(3))  # not increasing
    assert e.value.code == ss.ERR_ARG
    with pytest.raises(ss.SplitSartError) as e:
        ss.make_geometry_from_csr(4, 6, rp, np.array([1, 9, 0]), np.ones(3))  # out of range
    assert e.value.code == ss.ERR_ARG
    with pytest.raises(ss.SplitSartError) as e:
        ss.make_geometry_from_csr(4, 6, rp, np.array([1, 2, 0]), np.array([1.0, np.nan, 1.0]))
    assert e.value.code == ss.ERR_NONFINITE
    with pytest.raises(ss.SplitSartError) as e:
        ss.make_geometry_from_csr(3, 6, np.array([0, 1]), np.array([1]), np.ones(1))
    assert e.value.code == ss.ERR_ODD_DIM
    g = ss.make_geometry_from_csr(4, 6, rp, np.array([1, 2, 0]), np.ones(3))
    assert (g.M, g.N, g.nnz_half) == (4, 6, 3)


def test_static_solve_rejects_null_matrix_pointers(ss):
    """splitsart_solve_static checks every caller pointer before it touches the device.

    The check runs on the host, so a NULL matrix pointer is an argument error,
    not a device fault, and no GPU is needed to see it.
    """
    import ctypes
    h = ss.lib()
    opts = ss.solve_opts(5, 1.0)
    good = 256  # any non-NULL value: the call must return before dereferencing anything
    names = ["rp", "col", "val", "cp", "row", "valT", "invR", "invC", "p12", "f12"]
    for k, name in enumerate(names):
        ptrs = [good] * len(names)
        ptrs[k] = None
        rc = h.splitsart_solve_static(16, 8, *ptrs, ctypes.byref(opts), good, None)
        assert rc == ss.ERR_ARG, name
        assert "NULL" in ss.last_error(), name
