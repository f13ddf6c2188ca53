"""Device tracer (splitsart_make_geometries_device) against the oracle and the host tracer.

- Against the oracle's Siddon tracer (oracle.geometry, written separately in
  NumPy): the same cells in the same order, lengths within 1e-12 relative,
  on every ray of the tiny slice, of a skewed slice and of a slice with a
  vertical ray on a cell boundary, and on 300 sampled
  rays of the realistic slice and of three batch slices.
- Against the library's host tracer: the two trace the same rays with the
  same FP64 expressions (Section 2 geometry, Siddon lengths), so the rows
  must be equal bit for bit: the same row pointers, columns and lengths.
"""
import numpy as np
import pytest

from oracle import geometry as ogeo
from paper_1902_10559_gb300.synthetic import REALISTIC, TINY, Geometry, batch_geometries

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


# A vertical ray on the centre plane: with K = 2 and gamma = 0 source 0 sits on
# x = 0, and with nb odd the middle bin's centre is x = 0, so that ray lies on
# the boundary between the two middle cell columns.
ON_PLANE = Geometry(nx=8, nz=6, W=40.0, H=30.0, z0=10.0, K=2, gamma_deg=0.0, R=300.0, nb=7, D=100.0)
SKEW = Geometry(nx=6, nz=5, W=30.0, H=20.0, z0=10.0, K=4, gamma_deg=30.0, R=200.0, nb=10, D=120.0)


def assert_same_rows(a, b):
    ra, ca, va = a.export()
    rb, cb, vb = b.export()
    assert a.M == b.M and a.N == b.N
    assert np.array_equal(ra, rb)
    assert np.array_equal(ca, cb)
    assert np.array_equal(va.view(np.uint64), vb.view(np.uint64))  # bit for bit


def assert_rows_match_oracle(dev, g, rows):
    """Rows of a device-traced geometry against oracle.geometry.siddon_ray, traced ray by ray."""
    rp, col, val = dev.export()
    assert dev.M == g.M and dev.N == g.N and len(rp) == g.M // 2 + 1
    src = ogeo.source_positions(g)
    det = ogeo.detector_centres(g)
    for i in rows:
        k, b = divmod(int(i), g.nb)
        j, w = ogeo.siddon_ray(g, src[k], np.array([det[b], 0.0]))
        got_j, got_w = col[rp[i]:rp[i + 1]], val[rp[i]:rp[i + 1]]
        assert np.array_equal(got_j, j), (g, i)
        assert np.all(np.abs(got_w - w) <= 1e-12 * np.maximum(np.abs(w), 1.0)), (g, i, np.abs(got_w - w).max())


@pytest.mark.parametrize("g", [TINY, SKEW, ON_PLANE], ids=["tiny", "skew", "on_plane"])
def test_device_tracer_matches_oracle_every_ray(ss, g):
    (dev,) = ss.make_geometries_device([g])
    assert_rows_match_oracle(dev, g, range(g.M // 2))


def test_device_tracer_matches_oracle_sampled_rays(ss):
    """300 seeded rays of the realistic slice and of three batch slices (smallest, largest, one other)."""
    bg = batch_geometries()
    sizes = [x.N for x in bg]
    gs = [REALISTIC, bg[int(np.argmin(sizes))], bg[int(np.argmax(sizes))], bg[17]]
    devs = ss.make_geometries_device(gs)
    rng = np.random.default_rng(2)
    for g, d in zip(gs, devs):
        assert_rows_match_oracle(d, g, rng.choice(g.M // 2, 300, replace=False))


@pytest.mark.parametrize("g", [TINY, SKEW, ON_PLANE, REALISTIC], ids=["tiny", "skew", "on_plane", "realistic"])
def test_device_tracer_equals_host_tracer(ss, g):
    (dev,) = ss.make_geometries_device([g])
    assert_same_rows(dev, ss.make_geometry(g))


def test_on_plane_ray_splits_its_length(ss):
    """The vertical ray gives half of each piece to each of the two middle columns."""
    (dev,) = ss.make_geometries_device([ON_PLANE])
    rp, col, val = dev.export()
    i = ON_PLANE.nb // 2  # source 0, middle bin
    c = col[rp[i]:rp[i + 1]] // ON_PLANE.nz
    assert set(c.tolist()) == {ON_PLANE.nx // 2 - 1, ON_PLANE.nx // 2}
    assert np.isclose(val[rp[i]:rp[i + 1]].sum(), ON_PLANE.H)  # the ray crosses the whole grid height


def test_device_tracer_batch_equals_host_per_slice(ss):
    gs = batch_geometries()[:12] + [TINY, SKEW]
    devs = ss.make_geometries_device(gs)
    assert len(devs) == len(gs)
    for g, d in zip(gs, devs):
        assert_same_rows(d, ss.make_geometry(g))


def test_device_tracer_feeds_the_fold(ss):
    """A system folded from device-traced rows equals one folded from host-traced rows."""
    gs = batch_geometries()[:3]
    a = ss.fold_batch(ss.make_geometries_device(gs), ss.F64)
    b = ss.fold_batch([ss.make_geometry(g) for g in gs], ss.F64)
    ea, eb = a.export(), b.export()
    for k in ("row_ptr", "col", "a1", "a2"):
        assert np.array_equal(ea[k], eb[k]), k


def test_device_tracer_errors(ss):
    odd = Geometry(nx=5, nz=4, W=1, H=1, z0=1, K=4, gamma_deg=10, R=10, nb=4, D=4)
    with pytest.raises(ss.SplitSartError) as e:
        ss.make_geometries_device([TINY, odd])
    assert e.value.code == ss.ERR_ODD_DIM
    with pytest.raises(ss.SplitSartError) as e:
        ss.make_geometries_device([])
    assert e.value.code == ss.ERR_ARG


def test_system_outlives_device_geometries(ss):
    """The fold copies the device rows: the system stays valid after its geometries are freed."""
    import gc
    gs = batch_geometries()[:2]
    geoms = ss.make_geometries_device(gs)
    sysm = ss.fold_batch(geoms, ss.F64)
    del geoms
    gc.collect()
    ref = ss.fold_batch([ss.make_geometry(g) for g in gs], ss.F64)
    p = torch.rand(sysm.M, dtype=torch.float64, device="cuda")
    out = []
    for s_ in (sysm, ref):
        p12 = torch.empty(s_.Mh, 2, dtype=torch.float64, device="cuda")
        f12 = torch.zeros(s_.Nh, 2, dtype=torch.float64, device="cuda")
        ss.fold_rhs(s_, p, p12)
        ss.solve(s_, p12, f12, ss.solve_opts(20, 1.0))
        out.append(f12.cpu().numpy())
    assert np.array_equal(out[0], out[1])
