"""Thin Python binding over libsplitsart.so, the C ABI declared in include/splitsart.h.

This module only marshals arguments. Every step of the method runs in the
library's CUDA kernels. Device buffers are torch CUDA tensors, passed by
pointer, and streams are torch streams. If the library has not been built, the
first call raises. There is no fallback.

The names follow the C ABI without the ``splitsart_`` prefix.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsplitsart.so")

F64, F32, BF16, F16 = 0, 1, 2, 3
LAYOUT_SNAKE, LAYOUT_IMAGE = 0, 1
DTYPE_NAMES = {"f64": F64, "f32": F32, "bf16": BF16, "f16": F16}

OK = 0
ERR_ARG, ERR_ODD_DIM, ERR_ASYMMETRIC, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM, ERR_STATE, ERR_NONFINITE, ERR_NOT_SPD = range(
    -1, -10, -1)


class GeometryParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("nz", ctypes.c_int32), ("W", ctypes.c_double), ("H", ctypes.c_double),
                ("z0", ctypes.c_double), ("K", ctypes.c_int32), ("gamma_deg", ctypes.c_double),
                ("R", ctypes.c_double), ("nb", ctypes.c_int32), ("D", ctypes.c_double)]


class SystemInfo(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("N", ctypes.c_int64), ("Mh", ctypes.c_int64), ("Nh", ctypes.c_int64),
                ("nnz_half", ctypes.c_int64), ("S", ctypes.c_int64), ("empty_rows", ctypes.c_int64),
                ("exact_zeros", ctypes.c_int64), ("dtype", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("device_bytes", ctypes.c_int64), ("nslices", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int32), ("lambda_", ctypes.c_double), ("tol", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("lanes_per_col", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("timeout_ms", ctypes.c_double),
                ("inject_barrier_fault", ctypes.c_int32), ("tile_entries", ctypes.c_int32),
                ("row_weight", ctypes.c_int32), ("lanes_per_row", ctypes.c_int32)]


class OsOpts(ctypes.Structure):
    _fields_ = [("subset_rows", ctypes.c_int32), ("cone", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("rho", ctypes.c_double),
                ("rr", ctypes.c_double), ("pp", ctypes.c_double)]


class SplitSartError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"splitsart error {code}: {msg}")
        self.code = code


_lib = None

# Every symbol the header declares, with its argument and result types.
_P = ctypes.c_void_p
_SIGS = {
    "splitsart_make_geometry": ([ctypes.POINTER(GeometryParams), ctypes.POINTER(_P)], ctypes.c_int),
    "splitsart_make_geometry_from_csr": ([ctypes.c_int64, ctypes.c_int64, _P, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "splitsart_make_geometries_device": ([ctypes.POINTER(GeometryParams), ctypes.c_int, _P, ctypes.POINTER(_P)],
                                         ctypes.c_int),
    "splitsart_geometry_info": ([_P, _P, _P, _P], ctypes.c_int),
    "splitsart_geometry_export": ([_P, _P, _P, _P], ctypes.c_int),
    "splitsart_geometry_destroy": ([_P], None),
    "splitsart_fold_system": ([_P, ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "splitsart_fold_batch": ([ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "splitsart_system_slices": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "splitsart_solve_result_slices": ([_P, ctypes.POINTER(SolveInfo), ctypes.c_int], ctypes.c_int),
    "splitsart_solve_multi": ([_P, ctypes.c_int, _P, _P, ctypes.POINTER(SolveOpts), ctypes.c_int, _P, _P], ctypes.c_int),
    "splitsart_solve_multi_ordered": ([_P, ctypes.c_int, _P, _P, ctypes.POINTER(SolveOpts), ctypes.c_int, _P, _P, _P],
                                      ctypes.c_int),
    "splitsart_pick_start": ([_P, ctypes.c_int, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "splitsart_refold": ([_P, _P], ctypes.c_int),
    "splitsart_system_info_get": ([_P, ctypes.POINTER(SystemInfo)], ctypes.c_int),
    "splitsart_system_export": ([_P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "splitsart_system_export_csc": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "splitsart_system_destroy": ([_P], None),
    "splitsart_fold_rhs": ([_P, _P, _P, _P], ctypes.c_int),
    "splitsart_fold_image": ([_P, _P, ctypes.c_int, _P, _P], ctypes.c_int),
    "splitsart_recombine": ([_P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "splitsart_project": ([_P, _P, ctypes.c_int, _P, _P], ctypes.c_int),
    "splitsart_solve": ([_P, _P, _P, ctypes.POINTER(SolveOpts), _P], ctypes.c_int),
    "splitsart_solve_result": ([_P, ctypes.POINTER(SolveInfo)], ctypes.c_int),
    "splitsart_solve_os": ([_P, _P, _P, ctypes.POINTER(SolveOpts), ctypes.POINTER(OsOpts), _P], ctypes.c_int),
    "splitsart_solve_cgls": ([_P, _P, _P, ctypes.POINTER(SolveOpts), _P], ctypes.c_int),
    "splitsart_normal_solve_bytes": ([ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "splitsart_normal_solve": ([ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, _P, _P, ctypes.c_int32, _P,
                                ctypes.c_int32, _P, ctypes.c_int32, _P, _P, _P], ctypes.c_int),
    "splitsart_direct_split": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "splitsart_solve_static": ([ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                ctypes.POINTER(SolveOpts), _P, _P], ctypes.c_int),
    "splitsart_cnn_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "splitsart_cnn_destroy": ([_P], None),
    "splitsart_cnn_set_mode": ([_P, ctypes.c_int], ctypes.c_int),
    "splitsart_cnn_params": ([_P, _P, _P], ctypes.c_int),
    "splitsart_cnn_set_params": ([_P, _P, _P, ctypes.c_int], ctypes.c_int),
    "splitsart_cnn_forward": ([_P, _P, ctypes.c_int, _P, _P], ctypes.c_int),
    "splitsart_cnn_loss_grad": ([_P, _P, _P, ctypes.c_int, _P, _P, _P], ctypes.c_int),
    "splitsart_cnn_train_step": ([_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, _P, _P], ctypes.c_int),
    "splitsart_last_error": ([ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
    "splitsart_version": ([], ctypes.c_char_p),
}


def lib() -> ctypes.CDLL:
    """Load libsplitsart.so (built by ``paper_1902_10559_gb300.build``). Raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def declared_symbols() -> list[str]:
    return list(_SIGS)


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().splitsart_last_error(buf, 1024)
    return buf.value.decode()


def _check(rc: int) -> None:
    if rc != OK:
        raise SplitSartError(rc, last_error())


def _stream_ptr(stream) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _vec_dtype(dtype: int):
    import torch
    return torch.float64 if dtype == F64 else torch.float32


def _dev_ptr(t, numel: int, dtype, name: str) -> int:
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    return t.data_ptr()


class Geometry:
    """The first M/2 rows of A, on the host. Wraps a ``splitsart_geometry`` handle."""

    def __init__(self, handle: int, params=None):
        self._h = ctypes.c_void_p(handle)
        self.params = params
        M, N, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().splitsart_geometry_info(self._h, ctypes.byref(M), ctypes.byref(N), ctypes.byref(nnz)))
        self.M, self.N, self.nnz_half = M.value, N.value, nnz.value

    def export(self):
        """Return (row_ptr int64[Mh+1], col int32[nnz], val float64[nnz])."""
        rp = np.zeros(self.M // 2 + 1, dtype=np.int64)
        col = np.zeros(max(self.nnz_half, 1), dtype=np.int32)
        val = np.zeros(max(self.nnz_half, 1), dtype=np.float64)
        _check(lib().splitsart_geometry_export(self._h, rp.ctypes.data, col.ctypes.data, val.ctypes.data))
        return rp, col[: self.nnz_half], val[: self.nnz_half]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.splitsart_geometry_destroy(self._h)
            self._h = None


def make_geometry(g) -> Geometry:
    """Build the geometry from an object with nx, nz, W, H, z0, K, gamma_deg, R, nb, D."""
    p = GeometryParams(g.nx, g.nz, g.W, g.H, g.z0, g.K, g.gamma_deg, g.R, g.nb, g.D)
    h = ctypes.c_void_p()
    _check(lib().splitsart_make_geometry(ctypes.byref(p), ctypes.byref(h)))
    return Geometry(h.value, g)


def make_geometries_device(gs, stream=None) -> list:
    """Trace the geometries of several slices on the GPU (same rows as ``make_geometry``, bit for bit)."""
    gs = list(gs)
    params = (GeometryParams * len(gs))(*[GeometryParams(g.nx, g.nz, g.W, g.H, g.z0, g.K, g.gamma_deg, g.R, g.nb, g.D)
                                          for g in gs])
    out = (_P * len(gs))()
    _check(lib().splitsart_make_geometries_device(params, len(gs), _stream_ptr(stream), out))
    return [Geometry(out[k], g) for k, g in enumerate(gs)]


def make_geometry_from_csr(M: int, N: int, row_ptr, col, val) -> Geometry:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib().splitsart_make_geometry_from_csr(M, N, rp.ctypes.data, c.ctypes.data, v.ctypes.data, ctypes.byref(h)))
    return Geometry(h.value)


class System:
    """Folded A1/A2 on the device, for one slice or a batch. Wraps a ``splitsart_system`` handle."""

    def __init__(self, handle: int, dtype: int, geometry, geometries=None):
        self._h = ctypes.c_void_p(handle)
        self.dtype = dtype
        self.geometry = geometry
        self.geometries = geometries if geometries is not None else [geometry]
        self.nslices = len(self.geometries)
        self.M = sum(g.M for g in self.geometries)
        self.N = sum(g.N for g in self.geometries)
        self.Mh, self.Nh = self.M // 2, self.N // 2

    @property
    def handle(self):
        return self._h

    @property
    def vec_dtype(self):
        return _vec_dtype(self.dtype)

    def info(self) -> dict:
        i = SystemInfo()
        _check(lib().splitsart_system_info_get(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in SystemInfo._fields_}

    def export(self, normalisers: bool = False):
        """Return the folded CSR on the host: row_ptr, col, a1, a2 and, if asked, R[Mh,2] and C[Nh,2]."""
        S = self.info()["S"]
        rp = np.zeros(self.Mh + 1, dtype=np.int64)
        col = np.zeros(max(S, 1), dtype=np.int32)
        a1 = np.zeros(max(S, 1))
        a2 = np.zeros(max(S, 1))
        R = np.zeros((max(self.Mh, 1), 2)) if normalisers else None
        C = np.zeros((max(self.Nh, 1), 2)) if normalisers else None
        _check(lib().splitsart_system_export(self._h, rp.ctypes.data, col.ctypes.data, a1.ctypes.data, a2.ctypes.data,
                                             R.ctypes.data if normalisers else None,
                                             C.ctypes.data if normalisers else None))
        out = {"row_ptr": rp, "col": col[:S], "a1": a1[:S], "a2": a2[:S]}
        if normalisers:
            out["R"], out["C"] = R[: self.Mh], C[: self.Nh]
        return out

    def export_csc(self):
        S = self.info()["S"]
        cp = np.zeros(self.Nh + 1, dtype=np.int64)
        row = np.zeros(max(S, 1), dtype=np.int32)
        a1 = np.zeros(max(S, 1))
        a2 = np.zeros(max(S, 1))
        _check(lib().splitsart_system_export_csc(self._h, cp.ctypes.data, row.ctypes.data, a1.ctypes.data,
                                                 a2.ctypes.data))
        return {"col_ptr": cp, "row": row[:S], "a1": a1[:S], "a2": a2[:S]}

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.splitsart_system_destroy(self._h)
            self._h = None


def fold_system(geometry: Geometry, dtype: int = F32, stream=None) -> System:
    h = ctypes.c_void_p()
    _check(lib().splitsart_fold_system(geometry._h, dtype, _stream_ptr(stream), ctypes.byref(h)))
    return System(h.value, dtype, geometry)


def fold_batch(geometries, dtype: int = F32, stream=None) -> System:
    """Fold several independent slices into one block-diagonal batch system."""
    arr = (_P * len(geometries))(*[g._h.value for g in geometries])
    h = ctypes.c_void_p()
    _check(lib().splitsart_fold_batch(arr, len(geometries), dtype, _stream_ptr(stream), ctypes.byref(h)))
    return System(h.value, dtype, geometries[0], list(geometries))


def system_slices(system: System) -> dict:
    """Slice offsets (arrays of nslices + 1) in the full and folded index spaces."""
    n = system.nslices + 1
    out = {k: np.zeros(n, dtype=np.int64) for k in ("M", "N", "Mh", "Nh")}
    _check(lib().splitsart_system_slices(system.handle, out["M"].ctypes.data, out["N"].ctypes.data,
                                         out["Mh"].ctypes.data, out["Nh"].ctypes.data))
    return out


def solve_result_slices(system: System) -> list:
    infos = (SolveInfo * system.nslices)()
    _check(lib().splitsart_solve_result_slices(system.handle, infos, system.nslices))
    return [{"iters": i.iters, "status": i.status, "rho": i.rho, "rr": i.rr, "pp": i.pp} for i in infos]


def refold(system: System, stream=None) -> None:
    _check(lib().splitsart_refold(system.handle, _stream_ptr(stream)))


def fold_rhs(system: System, p, p12, stream=None) -> None:
    """p: vec[M] -> p12: vec[Mh, 2] (pairs (p1_i, p2_i))."""
    vt = system.vec_dtype
    _check(lib().splitsart_fold_rhs(system.handle, _dev_ptr(p, system.M, vt, "p"),
                                    _dev_ptr(p12, 2 * system.Mh, vt, "p12"), _stream_ptr(stream)))


def fold_image(system: System, f, f12, layout: int = LAYOUT_SNAKE, stream=None) -> None:
    vt = system.vec_dtype
    _check(lib().splitsart_fold_image(system.handle, _dev_ptr(f, system.N, vt, "f"), layout,
                                      _dev_ptr(f12, 2 * system.Nh, vt, "f12"), _stream_ptr(stream)))


def recombine(system: System, f12, f, layout: int = LAYOUT_SNAKE, stream=None) -> None:
    vt = system.vec_dtype
    _check(lib().splitsart_recombine(system.handle, _dev_ptr(f12, 2 * system.Nh, vt, "f12"),
                                     _dev_ptr(f, system.N, vt, "f"), layout, _stream_ptr(stream)))


def project(system: System, f, p, layout: int = LAYOUT_SNAKE, stream=None) -> None:
    vt = system.vec_dtype
    _check(lib().splitsart_project(system.handle, _dev_ptr(f, system.N, vt, "f"), layout,
                                   _dev_ptr(p, system.M, vt, "p"), _stream_ptr(stream)))


def solve_opts(max_iters: int, lam: float, tol: float = 0.0, check_every: int = 1, block_threads: int = 0,
               ctas_per_sm: int = 0, lanes_per_col: int = 0, timeout_ms: float = 0.0,
               inject_barrier_fault: bool = False, kernel: int = 0, tile_entries: int = 0,
               row_weight: int = 0, lanes_per_row: int = 0) -> SolveOpts:
    """Solve options (splitsart_solve_opts). kernel: 0 = library choice, 1 = CTA-wide tiles,
    2 = shared-memory resident, 3 = row streaming, 4 = per-warp bulk copies, 5/6 = row streaming in
    compacted order (explicit/implicit fold), 7/8 = the same fed by a producer warp through a
    shared-memory ring (explicit/implicit fold)."""
    return SolveOpts(max_iters, lam, tol, check_every, block_threads, ctas_per_sm, lanes_per_col, kernel, timeout_ms,
                     int(inject_barrier_fault), tile_entries, row_weight, lanes_per_row)


def solve(system: System, p12, f12, opts: SolveOpts, stream=None) -> None:
    """Enqueue the persistent split-SART solve. f12 holds f^0 on entry and the result on exit."""
    vt = system.vec_dtype
    _check(lib().splitsart_solve(system.handle, _dev_ptr(p12, 2 * system.Mh, vt, "p12"),
                                 _dev_ptr(f12, 2 * system.Nh, vt, "f12"), ctypes.byref(opts), _stream_ptr(stream)))


def solve_os(system: System, p12, f12, opts: SolveOpts, subset_rows: int = 0, cone: bool = False,
             stream=None) -> None:
    """Enqueue ordered-subsets SART (splitsart_solve_os); read the result with solve_result.

    subset_rows = 0 takes one folded view pair per subset. cone keeps the image non-negative.
    """
    vt = system.vec_dtype
    os_opts = OsOpts(int(subset_rows), int(bool(cone)))
    _check(lib().splitsart_solve_os(system.handle, _dev_ptr(p12, 2 * system.Mh, vt, "p12"),
                                    _dev_ptr(f12, 2 * system.Nh, vt, "f12"), ctypes.byref(opts),
                                    ctypes.byref(os_opts), _stream_ptr(stream)))


def solve_cgls(system: System, p12, f12, opts: SolveOpts, stream=None) -> None:
    """Enqueue CGLS on both split systems (splitsart_solve_cgls); read the result with solve_result."""
    vt = system.vec_dtype
    _check(lib().splitsart_solve_cgls(system.handle, _dev_ptr(p12, 2 * system.Mh, vt, "p12"),
                                      _dev_ptr(f12, 2 * system.Nh, vt, "f12"), ctypes.byref(opts),
                                      _stream_ptr(stream)))


def normal_solve_bytes(n: int) -> int:
    out = ctypes.c_int64()
    _check(lib().splitsart_normal_solve_bytes(int(n), ctypes.byref(out)))
    return out.value


class DenseSolver:
    """Device work buffer and status word of the direct method (splitsart_normal_solve / splitsart_direct_split)."""

    def __init__(self, n: int, device="cuda"):
        import torch
        self.n = int(n)
        self.work = torch.empty(normal_solve_bytes(n), dtype=torch.uint8, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)

    def result(self) -> int:
        """Synchronise and return the status word: OK or ERR_NOT_SPD."""
        return int(self.status.item())


def normal_solve(solver: DenseSolver, m: int, n: int, csr, csc, b, x, val_stride: int = 1, b_stride: int = 1,
                 x_stride: int = 1, stream=None) -> None:
    """Enqueue the normal-equation solve of an m x n matrix given as device (rp, col, val) CSR and (cp, row, valT) CSC."""
    rp, col, val = csr
    cp, row, valT = csc
    _check(lib().splitsart_normal_solve(int(m), int(n), rp.data_ptr(), col.data_ptr(), val.data_ptr(), cp.data_ptr(),
                                        row.data_ptr(), valT.data_ptr(), val_stride, b.data_ptr(), b_stride,
                                        x.data_ptr(), x_stride, solver.work.data_ptr(), solver.status.data_ptr(),
                                        _stream_ptr(stream)))


def direct_split(system: System, solver: DenseSolver, p, f, stream=None) -> None:
    """Enqueue the split direct method on an FP64 system: p[M] in, f[N] (snake order) out."""
    _check(lib().splitsart_direct_split(system.handle, _dev_ptr(p, system.M, system.vec_dtype, "p"),
                                        _dev_ptr(f, system.N, system.vec_dtype, "f"), solver.work.data_ptr(),
                                        solver.status.data_ptr(), _stream_ptr(stream)))


def full_csr(geometry: Geometry):
    """Host CSR (row_ptr, col, val) of the full M x N matrix, from the stored half rows and Eq. (2).

    Row M-1-i is the reflection of row i: w_{M-1-i, N-1-j} = w_{i,j}.
    """
    rp, col, val = geometry.export()
    M, N, Mh = geometry.M, geometry.N, geometry.M // 2
    lens = np.diff(rp)
    full_rp = np.zeros(M + 1, dtype=np.int64)
    full_rp[1:Mh + 1] = np.cumsum(lens)
    full_rp[Mh + 1:] = full_rp[Mh] + np.cumsum(lens[::-1])
    cols = [col]
    vals = [val]
    for i in range(Mh - 1, -1, -1):  # rows Mh .. M-1 mirror rows Mh-1 .. 0
        cols.append((N - 1 - col[rp[i]:rp[i + 1]])[::-1])
        vals.append(val[rp[i]:rp[i + 1]][::-1])
    return full_rp, np.concatenate(cols).astype(np.int32), np.concatenate(vals)


def solve_result(system: System, raise_on_error: bool = True) -> dict:
    info = SolveInfo()
    rc = lib().splitsart_solve_result(system.handle, ctypes.byref(info))
    if rc != OK and raise_on_error:
        raise SplitSartError(rc, last_error())
    return {"iters": info.iters, "status": info.status, "rho": info.rho, "rr": info.rr, "pp": info.pp}


def solve_static(Mh: int, Nh: int, rp, col, val, cp, row, valT, invR, invC, p12, f12, opts: SolveOpts, info,
                 stream=None) -> None:
    """Allocation-free solve on caller-owned buffers (see splitsart_solve_static in the header).

    All arrays are CUDA tensors: rp/cp int32, col/row int32, and val/valT/invR/
    invC/p12/f12 float32 pairs shaped [n, 2]. ``info`` is a CUDA uint8 tensor of
    at least ``ctypes.sizeof(SolveInfo)`` bytes. Use ``read_info`` to decode it.
    """
    import torch
    S = col.numel()
    i32, f32 = torch.int32, torch.float32
    if info.dtype != torch.uint8 or info.numel() < ctypes.sizeof(SolveInfo) or not info.is_cuda:
        raise ValueError("info: expected a CUDA uint8 tensor of sizeof(SolveInfo) bytes")
    _check(lib().splitsart_solve_static(
        Mh, Nh, _dev_ptr(rp, Mh + 1, i32, "rp"), _dev_ptr(col, S, i32, "col"), _dev_ptr(val, 2 * S, f32, "val"),
        _dev_ptr(cp, Nh + 1, i32, "cp"), _dev_ptr(row, S, i32, "row"), _dev_ptr(valT, 2 * S, f32, "valT"),
        _dev_ptr(invR, 2 * Mh, f32, "invR"), _dev_ptr(invC, 2 * Nh, f32, "invC"),
        _dev_ptr(p12, 2 * Mh, f32, "p12"), _dev_ptr(f12, 2 * Nh, f32, "f12"), ctypes.byref(opts), info.data_ptr(),
        _stream_ptr(stream)))


def solve_multi(system: System, p12, f12, opts: SolveOpts, info, rhs_per_cta: int = 0, stream=None,
                order=None) -> None:
    """Solve nrhs right-hand sides at once. p12: [nrhs, Mh, 2], f12: [nrhs, Nh, 2] (in: f0, out: results).

    ``info`` is a CUDA uint8 tensor of nrhs * sizeof(SolveInfo) bytes; decode it with ``read_infos``.
    ``order`` (optional CUDA int32 [nrhs], a permutation) is the order in which the launch takes them.
    """
    import torch
    vt = system.vec_dtype
    nrhs = p12.shape[0]
    if info.dtype != torch.uint8 or not info.is_cuda or info.numel() < nrhs * ctypes.sizeof(SolveInfo):
        raise ValueError("info: expected a CUDA uint8 tensor of nrhs * sizeof(SolveInfo) bytes")
    if order is not None and (order.dtype != torch.int32 or not order.is_cuda or order.numel() != nrhs):
        raise ValueError("order: expected a CUDA int32 tensor of nrhs entries")
    _check(lib().splitsart_solve_multi_ordered(system.handle, nrhs, _dev_ptr(p12, 2 * system.Mh * nrhs, vt, "p12"),
                                               _dev_ptr(f12, 2 * system.Nh * nrhs, vt, "f12"), ctypes.byref(opts),
                                               rhs_per_cta, None if order is None else order.data_ptr(),
                                               info.data_ptr(), _stream_ptr(stream)))


def pick_start(system: System, f12_warm, info_warm, info_base, f12, picked=None, stream=None) -> None:
    """Keep, per right-hand side, the warm start where its rho is lower than the base start's."""
    nrhs = f12.shape[0]
    vt = system.vec_dtype
    _check(lib().splitsart_pick_start(system.handle, nrhs, _dev_ptr(f12_warm, 2 * system.Nh * nrhs, vt, "f12_warm"),
                                      info_warm.data_ptr(), info_base.data_ptr(),
                                      _dev_ptr(f12, 2 * system.Nh * nrhs, vt, "f12"),
                                      None if picked is None else picked.data_ptr(), _stream_ptr(stream)))


def read_infos(info, n: int) -> list:
    raw = bytes(info[: n * ctypes.sizeof(SolveInfo)].cpu().numpy().tobytes())
    arr = (SolveInfo * n).from_buffer_copy(raw)
    return [{"iters": s.iters, "status": s.status, "rho": s.rho, "rr": s.rr, "pp": s.pp} for s in arr]


def read_info(info) -> dict:
    """Decode a device splitsart_solve_info written by solve_static."""
    raw = bytes(info[: ctypes.sizeof(SolveInfo)].cpu().numpy().tobytes())
    s = SolveInfo.from_buffer_copy(raw)
    return {"iters": s.iters, "status": s.status, "rho": s.rho, "rr": s.rr, "pp": s.pp}


CNN_PARAMS = 19105


class Cnn:
    """The warm-start network. Wraps a ``splitsart_cnn`` handle; images are CUDA float32 [B, nz, nx]."""

    def __init__(self, nz: int, nx: int, max_batch: int, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != CNN_PARAMS:
            raise ValueError(f"expected {CNN_PARAMS} parameters")
        h = ctypes.c_void_p()
        _check(lib().splitsart_cnn_create(nz, nx, max_batch, p.ctypes.data, ctypes.byref(h)))
        self._h = h
        self.nz, self.nx, self.max_batch = nz, nx, max_batch

    def _img(self, t, B, name):
        import torch
        return _dev_ptr(t, B * self.nz * self.nx, torch.float32, name)

    def set_mode(self, mode: int) -> None:
        _check(lib().splitsart_cnn_set_mode(self._h, mode))

    def params(self, moments: bool = False):
        p = np.zeros(CNN_PARAMS, dtype=np.float32)
        mv = np.zeros(2 * CNN_PARAMS, dtype=np.float32) if moments else None
        _check(lib().splitsart_cnn_params(self._h, p.ctypes.data, mv.ctypes.data if moments else None))
        return (p, mv[:CNN_PARAMS], mv[CNN_PARAMS:]) if moments else p

    def set_params(self, params, m=None, v=None, step: int = 0) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        mv = None if m is None else np.ascontiguousarray(np.concatenate([m, v]), dtype=np.float32)
        _check(lib().splitsart_cnn_set_params(self._h, p.ctypes.data, None if mv is None else mv.ctypes.data, step))

    def forward(self, x, y, stream=None) -> None:
        B = x.shape[0]
        _check(lib().splitsart_cnn_forward(self._h, self._img(x, B, "x"), B, self._img(y, B, "y"), _stream_ptr(stream)))

    def loss_grad(self, x, t, loss=None, grad=None, stream=None) -> None:
        B = x.shape[0]
        _check(lib().splitsart_cnn_loss_grad(self._h, self._img(x, B, "x"), self._img(t, B, "t"), B,
                                             None if loss is None else loss.data_ptr(),
                                             None if grad is None else grad.data_ptr(), _stream_ptr(stream)))

    def train_step(self, x, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, loss=None, stream=None) -> None:
        B = x.shape[0]
        _check(lib().splitsart_cnn_train_step(self._h, self._img(x, B, "x"), self._img(t, B, "t"), B, lr, beta1,
                                              beta2, eps, None if loss is None else loss.data_ptr(),
                                              _stream_ptr(stream)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.splitsart_cnn_destroy(self._h)
            self._h = None


def version() -> str:
    return lib().splitsart_version().decode()
