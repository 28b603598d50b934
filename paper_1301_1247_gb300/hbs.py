"""Thin ctypes binding of libhbsqp.so (include/hbsqp.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays,
torch CUDA tensors and integers into the plain pointers and sizes of the C ABI.
Loading fails loudly if the library has not been built (there is no CPU path).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhbsqp.so")

HBS_OK = 0
HBS_ERR_INVALID_ARG = 1
HBS_ERR_OOM = 2
HBS_ERR_CUDA = 3
HBS_ERR_RANK = 4
HBS_WARN_ILLCOND = 5
HBS_ERR_TIMEOUT = 6
HBS_ERR_IO = 7
HBS_ERR_INTERNAL = 8
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "RANK", 5: "WARN_ILLCOND",
                6: "TIMEOUT", 7: "IO", 8: "INTERNAL"}

# Every entry point declared in include/hbsqp.h.
EXPORTED = ("hbs_default_options", "hbs_build", "hbs_build_batch", "hbs_solve", "hbs_solve_plain", "hbs_solve_proxy",
            "hbs_bragg_amplitudes",
            "hbs_result_angle_info", "hbs_info", "hbs_save", "hbs_load", "hbs_apply_inverse",
            "hbs_kernel_block", "hbs_kernel_block_transmission", "hbs_row_id", "hbs_batched_inverse", "hbs_zgemm",
            "hbs_row_id_static",
            "hbs_profile_enable", "hbs_profile_reset", "hbs_profile_get", "hbs_launch_count",
            "hbs_server_create", "hbs_server_add", "hbs_server_remove", "hbs_server_submit", "hbs_server_wait",
            "hbs_server_stats", "hbs_server_free", "hbs_fault_inject", "hbs_barrier_selftest",
            "hbs_free", "hbs_result_free", "hbs_last_error")


class Geometry(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_double), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("dx", ctypes.c_void_p), ("dy", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("n_proxy_min", ctypes.c_int), ("proxy_rho", ctypes.c_double),
                ("nb_radius", ctypes.c_double), ("nb_proxies", ctypes.c_int), ("m", ctypes.c_int),
                ("contour_h", ctypes.c_double), ("contour_c", ctypes.c_double), ("contour_w", ctypes.c_double),
                ("contour_k", ctypes.c_double), ("wood_shift", ctypes.c_double),
                ("n_bragg_samples", ctypes.c_int), ("y0", ctypes.c_double), ("precision", ctypes.c_int),
                ("index", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("levels", ctypes.c_int), ("max_rank", ctypes.c_int),
                ("nb_rank", ctypes.c_int), ("m", ctypes.c_int), ("n_contours", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("build_seconds", ctypes.c_double),
                ("factor_bytes", ctypes.c_double), ("apply_flops_per_rhs", ctypes.c_double),
                ("contour_h", ctypes.c_double), ("contour_c", ctypes.c_double), ("contour_w", ctypes.c_double),
                ("wood_t0", ctypes.c_double), ("n_bragg_samples", ctypes.c_int), ("y0", ctypes.c_double),
                ("nb_radius", ctypes.c_double), ("nb_proxies", ctypes.c_int), ("pid_col_rank", ctypes.c_int),
                ("pid_row_rank", ctypes.c_int), ("pid_residual", ctypes.c_double),
                ("nb_residual", ctypes.c_double), ("unknowns", ctypes.c_int64), ("index", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("mean_batch", ctypes.c_double), ("p50_latency_s", ctypes.c_double),
                ("p99_latency_s", ctypes.c_double), ("max_latency_s", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("resident_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 80), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


_lib = None


def lib():
    """Load libhbsqp.so (raises if it is missing: build it with paper_1301_1247_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_1301_1247_gb300.build` first")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    L.hbs_default_options.argtypes = [ctypes.POINTER(Options)]
    L.hbs_default_options.restype = None
    L.hbs_build.argtypes = [ctypes.POINTER(Geometry), dbl, dbl, ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]
    L.hbs_server_create.argtypes = [ctypes.c_size_t, ci, ci, ctypes.POINTER(vp)]
    L.hbs_server_create.restype = ctypes.c_int
    L.hbs_server_add.argtypes = [vp, vp, ctypes.POINTER(i64)]
    L.hbs_server_add.restype = ctypes.c_int
    L.hbs_server_remove.argtypes = [vp, i64]
    L.hbs_server_remove.restype = ctypes.c_int
    L.hbs_server_submit.argtypes = [vp, i64, dbl, ctypes.POINTER(i64)]
    L.hbs_server_submit.restype = ctypes.c_int
    L.hbs_server_wait.argtypes = [vp, i64, dbl, ctypes.POINTER(vp)]
    L.hbs_server_wait.restype = ctypes.c_int
    L.hbs_server_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.hbs_server_stats.restype = ctypes.c_int
    L.hbs_server_free.argtypes = [vp]
    L.hbs_server_free.restype = None
    L.hbs_build_batch.argtypes = [ctypes.POINTER(Geometry), ctypes.POINTER(dbl), i64, dbl, ctypes.POINTER(Options),
                                  vp, ctypes.POINTER(vp)]
    L.hbs_build_batch.restype = ctypes.c_int
    L.hbs_solve.argtypes = [vp, ctypes.POINTER(dbl), i64, vp, ctypes.POINTER(vp)]
    L.hbs_solve_plain.argtypes = [vp, ctypes.POINTER(dbl), i64, vp, ctypes.POINTER(vp)]
    L.hbs_solve_proxy.argtypes = [vp, ctypes.POINTER(dbl), i64, vp, ctypes.POINTER(vp)]
    L.hbs_bragg_amplitudes.argtypes = [vp, i64, ctypes.POINTER(ci), ctypes.POINTER(ci), vp, vp,
                                       ctypes.POINTER(dbl)]
    L.hbs_result_angle_info.argtypes = [vp, i64, ctypes.POINTER(ci), ctypes.POINTER(dbl)]
    L.hbs_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.hbs_save.argtypes = [vp, ctypes.c_char_p, vp]
    L.hbs_save.restype = ctypes.c_int
    L.hbs_load.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
    L.hbs_load.restype = ctypes.c_int
    L.hbs_apply_inverse.argtypes = [vp, vp, vp, i64, vp]
    L.hbs_kernel_block.argtypes = [ctypes.POINTER(Geometry), dbl, ci, dbl, vp, i64, vp, i64, vp, vp]
    L.hbs_kernel_block_transmission.argtypes = [ctypes.POINTER(Geometry), dbl, dbl, ci, dbl, vp, i64, vp, i64, vp,
                                                vp]
    L.hbs_row_id.argtypes = [vp, i64, i64, dbl, ctypes.POINTER(ci), vp, vp, vp]
    L.hbs_row_id_static.argtypes = [vp, i64, i64, dbl, ctypes.POINTER(ci), vp, vp, vp]
    L.hbs_zgemm.argtypes = [i64, i64, i64, ctypes.POINTER(dbl), vp, i64, ci, vp, i64, ctypes.POINTER(dbl), vp, i64,
                            ci, vp]
    L.hbs_zgemm.restype = ci
    L.hbs_batched_inverse.argtypes = [vp, i64, i64, ci, vp]
    L.hbs_batched_inverse.restype = ci
    L.hbs_fault_inject.argtypes = [ci, i64]
    L.hbs_fault_inject.restype = ci
    L.hbs_barrier_selftest.argtypes = [ci, ci, dbl, ctypes.POINTER(ci), vp]
    L.hbs_barrier_selftest.restype = ci
    L.hbs_profile_enable.argtypes = [ci]
    L.hbs_profile_enable.restype = None
    L.hbs_profile_reset.argtypes = []
    L.hbs_profile_reset.restype = None
    L.hbs_profile_get.argtypes = [ctypes.POINTER(KernelStat), ci]
    L.hbs_profile_get.restype = ci
    L.hbs_launch_count.argtypes = []
    L.hbs_launch_count.restype = i64
    L.hbs_free.argtypes = [vp]
    L.hbs_free.restype = None
    L.hbs_result_free.argtypes = [vp]
    L.hbs_result_free.restype = None
    L.hbs_last_error.argtypes = []
    L.hbs_last_error.restype = ctypes.c_char_p
    for name in ("hbs_build", "hbs_solve", "hbs_solve_plain", "hbs_solve_proxy", "hbs_bragg_amplitudes",
                 "hbs_result_angle_info",
                 "hbs_info", "hbs_apply_inverse", "hbs_kernel_block", "hbs_kernel_block_transmission", "hbs_row_id",
                 "hbs_row_id_static"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class HbsError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().hbs_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st, where, allow_warn=False):
    if st == HBS_OK or (allow_warn and st == HBS_WARN_ILLCOND):
        return st
    raise HbsError(st, where)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(a):
    """Device pointer of a torch tensor, or host pointer of a contiguous numpy array."""
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] and not a.flags["F_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    return ctypes.c_void_p(int(a))


def default_options(**kw) -> Options:
    o = Options()
    lib().hbs_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Result:
    def __init__(self, ptr, n):
        self._p = ptr
        self.n = n

    def __del__(self):
        if getattr(self, "_p", None):
            lib().hbs_result_free(self._p)
            self._p = None

    def bragg(self, i):
        """(orders, c_n, d_n, flux_error) of angle i."""
        nmin, nmax = ctypes.c_int(), ctypes.c_int()
        _check(lib().hbs_bragg_amplitudes(self._p, i, ctypes.byref(nmin), ctypes.byref(nmax), None, None, None),
               "hbs_bragg_amplitudes")
        no = nmax.value - nmin.value + 1
        c = np.zeros(no, dtype=np.complex128)
        d = np.zeros(no, dtype=np.complex128)
        fe = ctypes.c_double()
        _check(lib().hbs_bragg_amplitudes(self._p, i, ctypes.byref(nmin), ctypes.byref(nmax),
                                          c.ctypes.data_as(ctypes.c_void_p), d.ctypes.data_as(ctypes.c_void_p),
                                          ctypes.byref(fe)), "hbs_bragg_amplitudes")
        return np.arange(nmin.value, nmax.value + 1), c, d, fe.value

    def angle_info(self, i):
        nw, t0 = ctypes.c_int(), ctypes.c_double()
        _check(lib().hbs_result_angle_info(self._p, i, ctypes.byref(nw), ctypes.byref(t0)), "hbs_result_angle_info")
        return nw.value, t0.value


class Handle:
    """A built solver (hbs_build)."""

    def __init__(self, x, y, dx, dy, d, omega, tol, opts: Options | None = None, stream=None):
        """Geometry arrays are host numpy arrays, or float64 CUDA tensors (device-resident input)."""
        if hasattr(x, "data_ptr"):
            arrs = [x, y, dx, dy]
            self._keep = arrs
            g = Geometry(int(x.numel()), float(d), *[a.data_ptr() for a in arrs], 1)
            n = int(x.numel())
        else:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, dx, dy)]
            self._keep = arrs
            g = Geometry(len(arrs[0]), float(d), *[a.ctypes.data for a in arrs], 0)
            n = len(arrs[0])
        out = ctypes.c_void_p()
        st = lib().hbs_build(ctypes.byref(g), float(omega), float(tol),
                             ctypes.byref(opts) if opts is not None else None, _stream(stream), ctypes.byref(out))
        _check(st, "hbs_build")
        self._p = out
        self.n = n
        self.unknowns = self.info()["unknowns"]  # n, or 2 n for the transmission problem

    @classmethod
    def load(cls, path, stream=None) -> "Handle":
        """A solver written by save() (hbs_load)."""
        out = ctypes.c_void_p()
        _check(lib().hbs_load(str(path).encode(), _stream(stream), ctypes.byref(out)), "hbs_load")
        h = cls.__new__(cls)
        h._p = out
        h._keep = []
        h.n = h.info()["n"]
        h.unknowns = h.info()["unknowns"]
        return h

    def save(self, path, stream=None):
        """Write the built solver to `path` (hbs_save)."""
        _check(lib().hbs_save(self._p, str(path).encode(), _stream(stream)), "hbs_save")

    def __del__(self):
        if getattr(self, "_p", None):
            lib().hbs_free(self._p)
            self._p = None

    def info(self) -> dict:
        inf = Info()
        _check(lib().hbs_info(self._p, ctypes.byref(inf)), "hbs_info")
        return inf.as_dict()

    def _solve(self, fn, thetas, stream):
        th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).ravel())
        out = ctypes.c_void_p()
        st = fn(self._p, th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(th), _stream(stream),
                ctypes.byref(out))
        _check(st, fn.__name__, allow_warn=True)
        r = Result(out, len(th))
        r.status = st
        return r

    def solve(self, thetas, stream=None) -> Result:
        return self._solve(lib().hbs_solve, thetas, stream)

    def solve_plain(self, thetas, stream=None) -> Result:
        return self._solve(lib().hbs_solve_plain, thetas, stream)

    def solve_proxy(self, thetas, stream=None) -> Result:
        """hbs_solve_proxy: the same amplitudes with the proxy-point / wall-discrepancy periodizer."""
        return self._solve(lib().hbs_solve_proxy, thetas, stream)

    def apply_inverse(self, b, x, nrhs, stream=None):
        """x = A^{-1} b for device complex128 tensors (N x nrhs, column-major, i.e. torch shape (nrhs, N))."""
        _check(lib().hbs_apply_inverse(self._p, _ptr(b), _ptr(x), int(nrhs), _stream(stream)), "hbs_apply_inverse")


class Server:
    """Request loop over resident solvers (hbs_server_*): submit single angles from any
    thread, wait for their Bragg amplitudes."""

    def __init__(self, hbm_budget_bytes: int = 0, slots: int = 2, max_batch: int = 256):
        out = ctypes.c_void_p()
        _check(lib().hbs_server_create(int(hbm_budget_bytes), int(slots), int(max_batch), ctypes.byref(out)),
               "hbs_server_create")
        self._p = out
        self._handles = {}

    def add(self, handle: "Handle") -> int:
        gid = ctypes.c_int64()
        _check(lib().hbs_server_add(self._p, handle._p, ctypes.byref(gid)), "hbs_server_add")
        self._handles[gid.value] = handle
        return gid.value

    def remove(self, gid: int):
        _check(lib().hbs_server_remove(self._p, int(gid)), "hbs_server_remove")
        self._handles.pop(gid, None)

    def submit(self, gid: int, theta: float) -> int:
        rid = ctypes.c_int64()
        _check(lib().hbs_server_submit(self._p, int(gid), float(theta), ctypes.byref(rid)), "hbs_server_submit")
        return rid.value

    def wait(self, rid: int, timeout_s: float = 60.0):
        """(orders, c, d, flux_error) of one request."""
        out = ctypes.c_void_p()
        st = lib().hbs_server_wait(self._p, int(rid), float(timeout_s), ctypes.byref(out))
        _check(st, "hbs_server_wait", allow_warn=True)
        r = Result(out, 1)
        r.status = st
        return r.bragg(0)

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().hbs_server_stats(self._p, ctypes.byref(s)), "hbs_server_stats")
        return s.as_dict()

    def close(self):
        if getattr(self, "_p", None):
            lib().hbs_server_free(self._p)
            self._p = None

    def __del__(self):
        self.close()


def build_batch(geometries, omegas, d, tol, opts: Options | None = None, stream=None) -> list:
    """Several solvers built level-synchronously (hbs_build_batch).  `geometries` is a list
    of host (x, y, dx, dy) tuples; returns one Handle per geometry."""
    cnt = len(geometries)
    keep = []
    garr = (Geometry * cnt)()
    for i, (x, y, dx, dy) in enumerate(geometries):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, dx, dy)]
        keep.append(arrs)
        garr[i] = Geometry(len(arrs[0]), float(d), *[a.ctypes.data for a in arrs], 0)
    om = np.ascontiguousarray(np.asarray(omegas, dtype=np.float64))
    outs = (ctypes.c_void_p * cnt)()
    _check(lib().hbs_build_batch(garr, om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cnt, float(tol),
                                 ctypes.byref(opts) if opts is not None else None, _stream(stream), outs),
           "hbs_build_batch")
    res = []
    for i in range(cnt):
        h = Handle.__new__(Handle)
        h._p = ctypes.c_void_p(outs[i])
        h._keep = keep[i]
        h.n = len(keep[i][0])
        h.unknowns = h.info()["unknowns"]
        res.append(h)
    return res


def kernel_block(x, y, dx, dy, omega, kind, shift_x, rows, cols, out, stream=None):
    """Device-side fill of Nystrom entries (kind 0: A with I/2 and KR6; kind 1: image shifted by shift_x)."""
    g = Geometry(int(x.numel()), 1.0, _ptr(x).value, _ptr(y).value, _ptr(dx).value, _ptr(dy).value, 1)
    _check(lib().hbs_kernel_block(ctypes.byref(g), float(omega), int(kind), float(shift_x), _ptr(rows),
                                  int(rows.numel()), _ptr(cols), int(cols.numel()), _ptr(out), _stream(stream)),
           "hbs_kernel_block")


def kernel_block_transmission(x, y, dx, dy, omega, index, kind, shift_x, rows, cols, out, stream=None):
    """Device-side fill of the transmission operator's entries (Sec. 5) on the interlaced
    unknowns (kind 0: A; kind 1: the pair's image shifted by shift_x)."""
    g = Geometry(int(x.numel()), 1.0, _ptr(x).value, _ptr(y).value, _ptr(dx).value, _ptr(dy).value, 1)
    _check(lib().hbs_kernel_block_transmission(ctypes.byref(g), float(omega), float(index), int(kind),
                                               float(shift_x), _ptr(rows), int(rows.numel()), _ptr(cols),
                                               int(cols.numel()), _ptr(out), _stream(stream)),
           "hbs_kernel_block_transmission")


def row_id(mt, m, n, tol, perm, t, stream=None) -> int:
    """Interpolative decomposition of M = Mt^T (device, m x n column-major, overwritten)."""
    rank = ctypes.c_int()
    _check(lib().hbs_row_id(_ptr(mt), int(m), int(n), float(tol), ctypes.byref(rank), _ptr(perm), _ptr(t),
                            _stream(stream)), "hbs_row_id")
    return rank.value


PRECISION_FP64, PRECISION_DOUBLE_FLOAT, PRECISION_TENSOR = 0, 1, 2


def zgemm(m, n, k, alpha, a, lda, trans_a, b, ldb, beta, c, ldc, precision=PRECISION_FP64, stream=None):
    """hbs_zgemm: C = alpha op(A) B + beta C on device complex128 arrays (column-major)."""
    al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    be = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
    _check(lib().hbs_zgemm(int(m), int(n), int(k), al, _ptr(a), int(lda), int(trans_a), _ptr(b), int(ldb), be, _ptr(c),
                           int(ldc), int(precision), _stream(stream)), "hbs_zgemm")


def batched_inverse(a, n, count, precision=0, stream=None):
    """hbs_batched_inverse: `count` device n x n complex128 blocks (column-major, back to
    back) inverted in place.  Returns the status (HBS_OK or HBS_WARN_ILLCOND); raises on errors."""
    st = lib().hbs_batched_inverse(_ptr(a), int(n), int(count), int(precision), _stream(stream))
    _check(st, "hbs_batched_inverse", allow_warn=True)
    return st


INJECT_CLEAR, INJECT_ALLOC_FAILURE, INJECT_RANK_CAP = 0, 1, 2


def fault_inject(kind, value=0):
    """hbs_fault_inject: arm a host-side fault (allocation failure, rank cap) or clear them."""
    _check(lib().hbs_fault_inject(int(kind), int(value)), "hbs_fault_inject")


def barrier_selftest(ctas, absent_cta, limit_s, stream=None):
    """hbs_barrier_selftest: (status, CTAs that passed all barriers)."""
    passed = ctypes.c_int()
    st = lib().hbs_barrier_selftest(int(ctas), int(absent_cta), float(limit_s), ctypes.byref(passed),
                                    _stream(stream))
    return st, passed.value


ROW_ID_STATIC_MAX_N = 262144


def row_id_static(mt, m, n, tol, perm, t, stream=None) -> int:
    """hbs_row_id_static: the same decomposition as row_id with no device allocation during the
    call (its working arrays sit in a fixed array the library reserves per GPU); n is limited
    to ROW_ID_STATIC_MAX_N and overlapping calls must not run concurrently."""
    rank = ctypes.c_int()
    _check(lib().hbs_row_id_static(_ptr(mt), int(m), int(n), float(tol), ctypes.byref(rank), _ptr(perm), _ptr(t),
                                   _stream(stream)), "hbs_row_id_static")
    return rank.value


def profile_enable(on: bool = True):
    lib().hbs_profile_enable(1 if on else 0)


def profile_reset():
    lib().hbs_profile_reset()


def profile_get() -> dict:
    """Per-kernel records {name: dict(launches, ms, flops, bytes)} (host phases are 'phase:...')."""
    n = lib().hbs_profile_get(None, 0)
    arr = (KernelStat * max(n, 1))()
    n = lib().hbs_profile_get(arr, n)
    return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms, flops=arr[i].flops,
                                        bytes=arr[i].bytes) for i in range(n)}


def launch_count() -> int:
    return int(lib().hbs_launch_count())
