"""Python binding of libwfq (include/wfq.h): argument marshalling only.

Every computation runs inside libwfq.so.  Arrays may be numpy arrays (host) or
torch CUDA tensors (device); the library tells host and device pointers apart.
There is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

WFQ_OK = 0
STATUS = {0: "WFQ_OK", -1: "WFQ_EINVAL", -2: "WFQ_ESINGULAR", -3: "WFQ_ENOMEM", -4: "WFQ_ENOCONV",
          -5: "WFQ_EBREAKDOWN", -6: "WFQ_ETIMEOUT", -7: "WFQ_ECUDA", -8: "WFQ_EUNSUPPORTED"}
STORE_FP64, STORE_BF16X2, STORE_F32X2, STORE_F32X2_SYM = 1, 2, 4, 8
PREC_FP64, PREC_MIXED, PREC_DF, PREC_FMM = 0, 1, 2, 3

# every symbol include/wfq.h declares
EXPORTS = ["wfq_create", "wfq_destroy", "wfq_last_error", "wfq_kernel_launches", "wfq_build_geometry",
           "wfq_build_bem_geometry", "wfq_free_geometry",
           "wfq_geometry_info", "wfq_apply", "wfq_rhs", "wfq_solve_gmres", "wfq_solve_gmres_shifted", "wfq_solve_qmr",
           "wfq_polarizability", "wfq_profile", "wfq_profile_read", "wfq_apply_mixed_noalloc",
           "wfq_server_create", "wfq_server_submit", "wfq_server_poll", "wfq_server_destroy",
           "wfq_memory_stats", "wfq_cross_section", "wfq_fmm_build", "wfq_fmm_info"]
KT_GEMM_MIXED, KT_DAPPLY_FP64, KT_SPARSE, KT_ORTHO, KT_RESIDUAL, KT_DGEMV_DF, KT_FMM = 0, 1, 2, 3, 4, 5, 6


class WfqError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("eta", "d_fermi", "s_fermi", "r0", "area", "n0", "tau", "cutoff_eps")]

    @classmethod
    def from_dict(cls, p):
        return cls(*[float(p[k]) for k, _ in cls._fields_])


class BemParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("eps_out", "eps_inf", "omega_p", "gamma")]

    @classmethod
    def from_dict(cls, p):
        return cls(*[float(p[k]) for k, _ in cls._fields_])


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("status", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("rmse", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p


def load(path: str | None = None):
    """Load libwfq.so (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build()
    L = ctypes.CDLL(path)
    I64, D, INT = ctypes.c_int64, ctypes.c_double, ctypes.c_int
    L.wfq_create.argtypes = [ctypes.POINTER(_P), INT]
    L.wfq_destroy.argtypes = [_P]
    L.wfq_last_error.restype = ctypes.c_char_p
    L.wfq_kernel_launches.restype = ctypes.c_int64
    L.wfq_build_geometry.argtypes = [_P, I64, _P, _P, ctypes.POINTER(Params), ctypes.c_uint32,
                                     ctypes.POINTER(_P)]
    L.wfq_build_bem_geometry.argtypes = [_P, I64, _P, _P, _P, _P, ctypes.POINTER(BemParams), ctypes.c_uint32,
                                         ctypes.POINTER(_P)]
    L.wfq_free_geometry.argtypes = [_P]
    L.wfq_geometry_info.argtypes = [_P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    L.wfq_apply.argtypes = [_P, I64, _P, _P, _P, INT, _P]
    L.wfq_rhs.argtypes = [_P, INT, _P, D, _P, _P]
    L.wfq_solve_gmres.argtypes = [_P, I64, _P, INT, _P, D, INT, D, INT, INT, _P, _P, _P]
    L.wfq_solve_qmr.argtypes = [_P, I64, _P, INT, _P, D, D, INT, INT, INT, _P, _P, _P]
    L.wfq_solve_gmres_shifted.argtypes = [_P, I64, _P, INT, _P, D, INT, D, INT, INT, _P, _P, _P]
    L.wfq_polarizability.argtypes = [_P, I64, _P, D, _P, _P]
    L.wfq_apply_mixed_noalloc.argtypes = [_P, I64, _P, _P, _P, _P]
    L.wfq_server_create.argtypes = [_P, INT, I64, INT, ctypes.POINTER(_P)]
    L.wfq_server_submit.argtypes = [_P, _P, I64, _P, INT, _P, D, INT, D, INT, _P, _P, ctypes.POINTER(I64)]
    L.wfq_server_poll.argtypes = [_P, I64, INT, ctypes.POINTER(INT), ctypes.POINTER(INT), ctypes.POINTER(D),
                                  ctypes.POINTER(D), ctypes.POINTER(INT)]
    L.wfq_server_destroy.argtypes = [_P]
    L.wfq_profile.argtypes = [_P, INT]
    L.wfq_memory_stats.argtypes = [_P, _P]
    L.wfq_fmm_build.argtypes = [_P, INT]
    L.wfq_fmm_info.argtypes = [_P, _P]
    L.wfq_cross_section.argtypes = [_P, I64, _P, INT, _P, D, _P, _P, _P, _P]
    L.wfq_profile_read.argtypes = [_P, INT, ctypes.POINTER(I64), ctypes.POINTER(D), ctypes.POINTER(D)]
    for name in EXPORTS:
        if name not in ("wfq_last_error", "wfq_kernel_launches"):
            getattr(L, name).restype = INT
    _lib = L
    return L


def kernel_launches() -> int:
    """Kernels launched by libwfq in this process so far."""
    return int(load().wfq_kernel_launches())


def _check(rc, allow=()):
    if rc != WFQ_OK and rc not in allow:
        msg = _lib.wfq_last_error().decode(errors="replace")
        raise WfqError(rc, msg)
    return rc


def _ptr(a):
    """Data pointer of a numpy array or a torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _host_f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _buf(a, dtype, rows, size, out, name):
    """(array, pointer) of a caller buffer the library reads (out=False) or writes
    (out=True): C-contiguous, element type `dtype`, `size` elements, first axis `rows`.
    A numpy input of another type or layout is copied into that form; outputs and torch
    tensors must already have it (the library would otherwise read or write the wrong
    elements)."""
    dtype = np.dtype(dtype)
    if hasattr(a, "data_ptr"):   # torch tensor
        import torch
        want = {np.dtype(np.complex128): torch.complex128, np.dtype(np.complex64): torch.complex64,
                np.dtype(np.float64): torch.float64}[dtype]
        if a.dtype != want or a.numel() != size or not a.is_contiguous() or (a.dim() and a.shape[0] != rows):
            raise ValueError(f"{name}: need a contiguous {want} tensor of {size} elements ({rows} rows); got "
                             f"{a.dtype} {tuple(a.shape)}, contiguous={a.is_contiguous()}")
        return a, a.data_ptr()
    if out:
        if (not isinstance(a, np.ndarray) or a.dtype != dtype or a.size != size or not a.flags.c_contiguous
                or not a.flags.writeable or (a.ndim and a.shape[0] != rows)):
            raise ValueError(f"{name}: need a writable C-contiguous {dtype} array of {size} elements ({rows} rows)")
        return a, a.ctypes.data
    arr = np.ascontiguousarray(a, dtype=dtype)
    if arr.size != size or (arr.ndim and arr.shape[0] != rows):
        raise ValueError(f"{name}: need {size} elements ({rows} rows), got shape {arr.shape}")
    return arr, arr.ctypes.data


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Context:
    def __init__(self, device: int = 0):
        L = load()
        h = _P()
        _check(L.wfq_create(ctypes.byref(h), int(device)))
        self.h = h
        self.device = device

    def profile(self, enable: bool):
        """Start (reset) or stop the library's kernel timers."""
        _check(_lib.wfq_profile(self.h, 1 if enable else 0))

    def profile_read(self, kind: int):
        """(launches, total device ms, total work) of a kernel class since profile(True)."""
        n, ms, wk = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _check(_lib.wfq_profile_read(self.h, int(kind), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(wk)))
        return n.value, ms.value, wk.value

    def memory_stats(self):
        """{allocs, pool_reserved, pool_used, pool_used_high}: device allocations the library
        has requested so far (process-wide) and the context pool's byte counts."""
        out = np.zeros(4, dtype=np.int64)
        _check(_lib.wfq_memory_stats(self.h, out.ctypes.data))
        return dict(zip(("allocs", "pool_reserved", "pool_used", "pool_used_high"), (int(v) for v in out)))

    def close(self):
        if self.h:
            _check(_lib.wfq_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Geometry:
    """One structure on the device (wfq_build_geometry)."""

    def __init__(self, ctx: Context, xyz, params: dict, eta=None, store: int = STORE_FP64):
        xyz = _host_f64(xyz)
        if xyz.ndim != 2 or xyz.shape[1] != 3:
            raise ValueError("xyz must be (n, 3)")
        self.ctx = ctx
        self.n = len(xyz)
        self.params = dict(params)
        self._xyz = xyz
        eta_a = None if eta is None else _host_f64(eta)
        p = Params.from_dict(params)
        h = _P()
        _check(_lib.wfq_build_geometry(ctx.h, self.n, _ptr(xyz), _ptr(eta_a), ctypes.byref(p), int(store),
                                       ctypes.byref(h)))
        self.h = h

    def fmm_build(self, order: int = 6):
        """Tree and operators of the fast-multipole D product (wfq_apply with PREC_FMM)."""
        _check(_lib.wfq_fmm_build(self.h, int(order)))

    def fmm_info(self):
        out = np.zeros(7, dtype=np.int64)
        _check(_lib.wfq_fmm_info(self.h, out.ctypes.data))
        return dict(zip(("dim", "depth", "order", "leaves", "boxes", "interactions", "near"), (int(v) for v in out)))

    def info(self):
        n, nnz, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.wfq_geometry_info(self.h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(b)))
        return {"n": n.value, "nnz": nnz.value, "device_bytes": b.value}

    def close(self):
        if self.h:
            _check(_lib.wfq_free_geometry(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- calls

    def apply(self, omega, x, y, prec: int = PREC_FP64, stream=None):
        """y = (A - z(omega_c) I) x; x, y: (n, ncplx) complex128 (FP64, DF) / complex64 (MIXED, FMM)."""
        om = _host_f64(np.atleast_1d(omega))
        dt = np.complex64 if prec in (PREC_MIXED, PREC_FMM) else np.complex128
        x, px = _buf(x, dt, self.n, self.n * len(om), False, "x")
        y, py = _buf(y, dt, self.n, self.n * len(om), True, "y")
        _check(_lib.wfq_apply(self.h, len(om), _ptr(om), px, py, int(prec), _stream_handle(stream)))
        return y

    def apply_mixed_noalloc(self, omega, x, y, stream=None):
        """wfq_apply_mixed_noalloc: the mixed apply with the library's static scratch
        array instead of any allocation; x, y must be device (torch CUDA) complex64."""
        om = _host_f64(np.atleast_1d(omega))
        x, px = _buf(x, np.complex64, self.n, self.n * len(om), False, "x")
        y, py = _buf(y, np.complex64, self.n, self.n * len(om), True, "y")
        _check(_lib.wfq_apply_mixed_noalloc(self.h, len(om), _ptr(om), px, py, _stream_handle(stream)))
        return y

    def rhs(self, dirs, E0=1.0, out=None, stream=None):
        d = _host_f64(np.atleast_2d(dirs))
        if out is None:
            out = np.empty((self.n, len(d)), dtype=np.float64)
        out, po = _buf(out, np.float64, self.n, self.n * len(d), True, "out")
        _check(_lib.wfq_rhs(self.h, len(d), _ptr(d), float(E0), po, _stream_handle(stream)))
        return out

    def _solve(self, kind, omega, dirs, E0, m, rel_tol, max_iter, prec, refine_every, out, stream):
        om = _host_f64(np.atleast_1d(omega))
        d = _host_f64(np.atleast_2d(dirs))
        ncols = len(om) * len(d)
        if out is None:
            out = np.empty((self.n, ncols), dtype=np.complex128)
        out, pq = _buf(out, np.complex128, self.n, self.n * ncols, True, "out")
        stats = (Stats * ncols)()
        if kind == "shifted":
            rc = _lib.wfq_solve_gmres_shifted(self.h, len(om), _ptr(om), len(d), _ptr(d), float(E0), int(m),
                                              float(rel_tol), int(max_iter), int(prec), pq,
                                              ctypes.cast(stats, _P), _stream_handle(stream))
        elif kind == "qmr":
            rc = _lib.wfq_solve_qmr(self.h, len(om), _ptr(om), len(d), _ptr(d), float(E0), float(rel_tol),
                                    int(max_iter), int(prec), int(refine_every), pq,
                                    ctypes.cast(stats, _P), _stream_handle(stream))
        else:
            rc = _lib.wfq_solve_gmres(self.h, len(om), _ptr(om), len(d), _ptr(d), float(E0), int(m),
                                      float(rel_tol), int(max_iter), int(prec), pq,
                                      ctypes.cast(stats, _P), _stream_handle(stream))
        _check(rc, allow=(-4, -5))
        st = [{"iters": s.iters, "restarts": s.restarts, "refinements": s.refinements,
               "status": STATUS.get(s.status, s.status), "rel_residual": s.rel_residual, "rmse": s.rmse}
              for s in stats]
        return out, st, STATUS[rc]

    def solve_gmres(self, omega, dirs, E0=1.0, m=0, rel_tol=1e-8, max_iter=1000, prec=PREC_FP64,
                    out=None, stream=None):
        """q (n, nfreq*ndir) complex128, per-column stats, overall status name."""
        return self._solve("gmres", omega, dirs, E0, m, rel_tol, max_iter, prec, 0, out, stream)

    def solve_gmres_shifted(self, omega, dirs, E0=1.0, m_max=0, rel_tol=1e-8, max_iter=4000, prec=PREC_MIXED,
                            out=None, stream=None):
        """Shifted GMRES: one real Arnoldi per direction for all frequencies (wfq_solve_gmres_shifted)."""
        return self._solve("shifted", omega, dirs, E0, m_max, rel_tol, max_iter, prec, 0, out, stream)

    def solve_qmr(self, omega, dirs, E0=1.0, rel_tol=1e-8, max_iter=1000, prec=PREC_FP64, refine_every=0,
                  out=None, stream=None):
        return self._solve("qmr", omega, dirs, E0, 0, rel_tol, max_iter, prec, refine_every, out, stream)

    def polarizability(self, q, E0=1.0, stream=None):
        """alpha (ncols, 3) complex128 from q (n, ncols) complex128 (host or device)."""
        ncols = q.shape[1] if q.ndim == 2 else 1
        q, pq = _buf(q, np.complex128, self.n, self.n * ncols, False, "q")
        out = np.empty((ncols, 3), dtype=np.complex128)
        _check(_lib.wfq_polarizability(self.h, ncols, pq, float(E0), _ptr(out), _stream_handle(stream)))
        return out

    def cross_section(self, omega, dirs, q, E0=1.0, stream=None):
        """(sigma (nfreq, ndir), sigma_iso (nfreq,)) from q (n, nfreq * ndir) complex128
        solved for these frequencies and directions (Eq. 28 per column; Eq. 29's mean over
        the directions)."""
        om = _host_f64(np.atleast_1d(omega))
        dirs = _host_f64(np.atleast_2d(dirs))
        nf, nd = len(om), len(dirs)
        q, pq = _buf(q, np.complex128, self.n, self.n * nf * nd, False, "q")
        sig = np.empty((nf, nd), dtype=np.float64)
        iso = np.empty(nf, dtype=np.float64)
        _check(_lib.wfq_cross_section(self.h, nf, om.ctypes.data, nd, dirs.ctypes.data, float(E0), pq,
                                      sig.ctypes.data, iso.ctypes.data, _stream_handle(stream)))
        return sig, iso



class BemGeometry(Geometry):
    """A surface for the continuum BEM operator (wfq_build_bem_geometry): collocation
    points, outward unit normals, element areas and mean curvatures (None: flat
    elements), and the Drude parameters (eps_out, eps_inf, omega_p, gamma).  Every
    Geometry call applies; solve_qmr is not available."""

    def __init__(self, ctx: Context, xyz, normal, area, curvature, bem: dict, store: int = STORE_FP64):
        xyz = _host_f64(xyz)
        if xyz.ndim != 2 or xyz.shape[1] != 3:
            raise ValueError("xyz must be (n, 3)")
        n = len(xyz)
        normal = _host_f64(normal)
        area = _host_f64(area)
        if normal.shape != (n, 3) or area.shape != (n,):
            raise ValueError("normal must be (n, 3) and area (n,)")
        curv = None
        if curvature is not None:
            curv = _host_f64(curvature)
            if curv.shape != (n,):
                raise ValueError("curvature must be (n,)")
        self.ctx = ctx
        self.n = n
        self.params = dict(bem)
        self._xyz = xyz
        p = BemParams.from_dict(bem)
        h = _P()
        self.h = None
        _check(_lib.wfq_build_bem_geometry(ctx.h, n, _ptr(xyz), _ptr(normal), _ptr(area), _ptr(curv),
                                           ctypes.byref(p), int(store), ctypes.byref(h)))
        self.h = h


class Server:
    """wfq_server_*: continuous-batching request server over resident geometries."""

    def __init__(self, ctx: Context, nworkers: int = 3, budget_bytes: int = 64 << 30, max_columns: int = 384):
        h = _P()
        _check(_lib.wfq_server_create(ctx.h, int(nworkers), int(budget_bytes), int(max_columns), ctypes.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, geom: Geometry, omega, dirs, E0=1.0, m=50, rel_tol=1e-8, max_iter=4000):
        """Queue a request; returns its id.  The result arrays live until poll() returns them."""
        om = _host_f64(np.atleast_1d(omega))
        d = _host_f64(np.atleast_2d(dirs))
        ncols = len(om) * len(d)
        q = np.empty((geom.n, ncols), dtype=np.complex128)
        stats = (Stats * ncols)()
        rid = ctypes.c_int64()
        _check(_lib.wfq_server_submit(self.h, geom.h, len(om), _ptr(om), len(d), _ptr(d), float(E0), int(m),
                                      float(rel_tol), int(max_iter), _ptr(q), ctypes.cast(stats, _P),
                                      ctypes.byref(rid)))
        self._keep[rid.value] = (q, stats, om, d)
        return rid.value

    def poll(self, rid: int, wait: bool = True):
        """None while running; else dict(status, latency_s, queue_s, batch_columns, q, stats)."""
        done, st, lat, qs, bc = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        _check(_lib.wfq_server_poll(self.h, int(rid), 1 if wait else 0, ctypes.byref(done), ctypes.byref(st),
                                    ctypes.byref(lat), ctypes.byref(qs), ctypes.byref(bc)))
        if not done.value:
            return None
        q, stats, _, _ = self._keep.pop(rid)
        return {"status": STATUS.get(st.value, st.value), "latency_s": lat.value, "queue_s": qs.value,
                "batch_columns": bc.value, "q": q,
                "stats": [{"iters": s.iters, "rel_residual": s.rel_residual,
                           "status": STATUS.get(s.status, s.status)} for s in stats]}

    def close(self):
        if self.h:
            _check(_lib.wfq_server_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
