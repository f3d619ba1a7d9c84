"""ctypes front end of the FP64 CPU oracle (oracle/wfq_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the CPU
legs of bench.py, never by the product package.  Every function here marshals
numpy arrays into the C routines, which follow the paper's equations (the
equation each one implements is named in the C source and repeated below).

Complex vectors are numpy complex128 arrays (interleaved re/im in memory).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_INT = ctypes.c_int

OP_DENSE_A, OP_STORED_D, OP_OTF_D = 0, 1, 2


def lib():
    """The oracle library built from oracle/wfq_oracle.c (built on first use)."""
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


def load(path):
    """Load and bind a build of the oracle's C source at `path` (tests compile copies of
    the source with a planted mistake to show that a pin catches it)."""
    L = ctypes.CDLL(path)
    L.orc_widths.argtypes = [_I64, _P, _P]
    L.orc_d_entry.argtypes = [_P, _P, _I64, _I64]
    L.orc_d_entry.restype = _D
    L.orc_d_matrix.argtypes = [_I64, _P, _P, _P]
    L.orc_fermi.argtypes = [_D, _D, _D, _D]
    L.orc_fermi.restype = _D
    L.orc_kbar_entry.argtypes = [_D, _D, _D, _D, _D]
    L.orc_kbar_entry.restype = _D
    L.orc_kbar_matrix.argtypes = [_I64, _P, _D, _D, _D, _D, _P]
    L.orc_kbar_csr.argtypes = [_I64, _P, _D, _D, _D, _D, _D, _P, _P, _P]
    L.orc_kbar_csr.restype = _I64
    L.orc_z.argtypes = [_D, _D, _D, _P, _P]
    L.orc_rhs_csr.argtypes = [_I64, _P, _P, _P, _P, _P, _D, _P]
    L.orc_rhs_dense.argtypes = [_I64, _P, _P, _P, _D, _P]
    L.orc_a_matrix.argtypes = [_I64, _P, _P, _P]
    L.orc_apply.argtypes = [_INT, _I64, _P, _P, _P, _P, _P, _P, _P, _D, _D, _P, _P]
    L.orc_d_matvec.argtypes = [_INT, _I64, _P, _P, _P, _P, _P]
    L.orc_lu_solve.argtypes = [_I64, _P, _D, _D, _P, _P]
    L.orc_lu_solve.restype = _INT
    L.orc_gmres.argtypes = [_INT, _I64, _P, _P, _P, _P, _P, _P, _P, _D, _D, _P, _INT, _D,
                            _INT, _P, _P]
    L.orc_gmres.restype = _INT
    L.orc_qmr.argtypes = [_INT, _I64, _P, _P, _P, _P, _P, _P, _D, _D, _P, _D, _INT, _P, _P]
    L.orc_qmr.restype = _INT
    L.orc_alpha.argtypes = [_I64, _P, _P, _D, _P]
    L.orc_residual_norm.argtypes = [_INT, _I64, _P, _P, _P, _P, _P, _P, _P, _D, _D, _P, _P]
    L.orc_residual_norm.restype = _D
    L.orc_vdot.argtypes = [_I64, _P, _P, _P]
    L.orc_apply_rows.argtypes = [_I64, _P, _P, _D, _D, _D, _D, _D, _D, _D, _P, _I64, _P, _P, _P]
    L.orc_rhs_rows.argtypes = [_I64, _P, _D, _D, _D, _D, _D, _P, _D, _I64, _P, _P]
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _eta_vec(n, eta):
    eta = np.asarray(eta, dtype=np.float64)
    if eta.ndim == 0:
        eta = np.full(n, float(eta))
    return _f64(eta)


# ---------------------------------------------------------------- assembly

def widths(eta):
    """Eq. 4: Gaussian widths w_i = sqrt(2/pi)/eta_i."""
    eta = _f64(np.atleast_1d(eta))
    w = np.empty_like(eta)
    lib().orc_widths(len(eta), _ptr(eta), _ptr(w))
    return w


def d_matrix(xyz, eta):
    """Eq. 3: dense D, n x n."""
    xyz = _f64(xyz)
    n = len(xyz)
    eta = _eta_vec(n, eta)
    D = np.empty((n, n))
    lib().orc_d_matrix(n, _ptr(xyz), _ptr(eta), _ptr(D))
    return D


def fermi(r, p):
    """Eq. 6: f(r) for the damping parameters in p."""
    return lib().orc_fermi(float(r), p["r0"], p["d_fermi"], p["s_fermi"])


def kbar_entry(r, p):
    """Eq. 9: one off-diagonal Kbar entry."""
    return lib().orc_kbar_entry(float(r), p["r0"], p["d_fermi"], p["s_fermi"], p["area"])


def kbar_matrix(xyz, p):
    """Eq. 9: dense Kbar, every pair kept, zero diagonal."""
    xyz = _f64(xyz)
    n = len(xyz)
    K = np.empty((n, n))
    lib().orc_kbar_matrix(n, _ptr(xyz), p["r0"], p["d_fermi"], p["s_fermi"], p["area"], _ptr(K))
    return K


def kbar_csr(xyz, p, cutoff_eps=None):
    """Eq. 9 as CSR (brute-force pair scan), pairs with 1 - f >= cutoff_eps."""
    xyz = _f64(xyz)
    n = len(xyz)
    eps = p["cutoff_eps"] if cutoff_eps is None else cutoff_eps
    rowptr = np.zeros(n + 1, dtype=np.int64)
    L = lib()
    nnz = L.orc_kbar_csr(n, _ptr(xyz), p["r0"], p["d_fermi"], p["s_fermi"], p["area"], eps,
                         _ptr(rowptr), None, None)
    col = np.empty(max(nnz, 1), dtype=np.int64)
    val = np.empty(max(nnz, 1), dtype=np.float64)
    L.orc_kbar_csr(n, _ptr(xyz), p["r0"], p["d_fermi"], p["s_fermi"], p["area"], eps,
                   _ptr(rowptr), _ptr(col), _ptr(val))
    return rowptr, col[:nnz], val[:nnz]


def z_of_omega(omega, p):
    """Eq. 12: complex shift z(omega)."""
    zr, zi = _D(), _D()
    lib().orc_z(float(omega), p["n0"], p["tau"], ctypes.byref(zr), ctypes.byref(zi))
    return complex(zr.value, zi.value)


def rhs_dense(xyz, K, kdir, E0=1.0):
    """Eq. 2 + Eq. 13 with a dense Kbar; returns a real vector."""
    xyz = _f64(xyz)
    K = _f64(K)
    kd = _f64(kdir)
    R = np.empty(len(xyz))
    lib().orc_rhs_dense(len(xyz), _ptr(xyz), _ptr(K), _ptr(kd), float(E0), _ptr(R))
    return R


def rhs_csr(xyz, csr, kdir, E0=1.0):
    """Eq. 2 + Eq. 13 with a CSR Kbar; returns a real vector."""
    xyz = _f64(xyz)
    rowptr, col, val = csr
    kd = _f64(kdir)
    R = np.empty(len(xyz))
    lib().orc_rhs_csr(len(xyz), _ptr(xyz), _ptr(rowptr), _ptr(col), _ptr(val), _ptr(kd),
                      float(E0), _ptr(R))
    return R


def a_matrix(D, K):
    """Eq. 11, literal triple loop: A_ij = sum_k Kbar_ik (D_kj - D_ij)."""
    D = _f64(D)
    K = _f64(K)
    n = len(D)
    A = np.empty((n, n))
    lib().orc_a_matrix(n, _ptr(D), _ptr(K), _ptr(A))
    return A


# ---------------------------------------------------------------- operators


class Operator:
    """(A - zI) in one of three representations:

    * dense A (Eq. 11)                        -> Operator.dense(A)
    * stored D + CSR Kbar (Eq. 17)            -> Operator.stored(D, csr)
    * D recomputed from Eq. 3 + CSR (Eq. 17)  -> Operator.on_the_fly(xyz, eta, csr)
    """

    def __init__(self, kind, n, A=None, D=None, xyz=None, eta=None, csr=None):
        self.kind, self.n = kind, n
        self.A = None if A is None else _f64(A)
        self.D = None if D is None else _f64(D)
        self.xyz = None if xyz is None else _f64(xyz)
        self.eta = None if eta is None else _eta_vec(n, eta)
        if csr is None:
            self.rowptr = self.col = self.val = None
        else:
            self.rowptr = np.ascontiguousarray(csr[0], dtype=np.int64)
            self.col = np.ascontiguousarray(csr[1], dtype=np.int64)
            self.val = _f64(csr[2])

    @classmethod
    def dense(cls, A):
        return cls(OP_DENSE_A, len(A), A=A)

    @classmethod
    def stored(cls, D, csr):
        return cls(OP_STORED_D, len(D), D=D, csr=csr)

    @classmethod
    def on_the_fly(cls, xyz, eta, csr):
        return cls(OP_OTF_D, len(xyz), xyz=xyz, eta=eta, csr=csr)

    def _args(self):
        return (self.kind, self.n, _ptr(self.A), _ptr(self.D), _ptr(self.xyz), _ptr(self.eta),
                _ptr(self.rowptr), _ptr(self.col), _ptr(self.val))

    def apply(self, z, x):
        """y = (A - zI) x for one complex vector x."""
        x = _c128(x)
        y = np.empty_like(x)
        lib().orc_apply(*self._args(), z.real, z.imag, _ptr(x), _ptr(y))
        return y

    def d_matvec(self, x):
        """u = D x (stored or recomputed kinds)."""
        x = _c128(x)
        u = np.empty_like(x)
        lib().orc_d_matvec(self.kind, self.n, _ptr(self.D), _ptr(self.xyz), _ptr(self.eta),
                           _ptr(x), _ptr(u))
        return u

    def residual_norm(self, z, R, q):
        """Eq. 27: ||R - (A - zI) q||_2."""
        R = _c128(R)
        q = _c128(q)
        return lib().orc_residual_norm(*self._args(), z.real, z.imag, _ptr(R), _ptr(q))

    def gmres(self, z, R, restart=0, rel_tol=1e-12, max_iter=1000):
        """Section 3 GMRES / GMRES(k) from q0 = 0.  Returns (q, info)."""
        R = _c128(R)
        q = np.zeros(self.n, dtype=np.complex128)
        out = np.zeros(3)
        st = lib().orc_gmres(*self._args(), z.real, z.imag, _ptr(R), int(restart),
                             float(rel_tol), int(max_iter), _ptr(q), _ptr(out))
        return q, {"status": st, "iters": int(out[0]), "rel_residual": out[1],
                   "restarts": int(out[2])}

    def qmr(self, z, R, rel_tol=1e-12, max_iter=1000, library=None):
        """Section 3 J-symmetric QMR-from-BCG (J = D), q0 = 0.  Returns (q, info).
        `library` runs another build of the oracle's source (see `load`)."""
        R = _c128(R)
        q = np.zeros(self.n, dtype=np.complex128)
        out = np.zeros(3)
        st = (library or lib()).orc_qmr(self.kind, self.n, _ptr(self.D), _ptr(self.xyz), _ptr(self.eta),
                           _ptr(self.rowptr), _ptr(self.col), _ptr(self.val), z.real, z.imag,
                           _ptr(R), float(rel_tol), int(max_iter), _ptr(q), _ptr(out))
        return q, {"status": st, "iters": int(out[0]), "rel_residual": out[1]}


def lu_solve(A, z, R):
    """Direct solve of (A - zI) q = R by LU with partial pivoting (Section 4's reference)."""
    A = _f64(A)
    R = _c128(R)
    q = np.empty(len(A), dtype=np.complex128)
    st = lib().orc_lu_solve(len(A), _ptr(A), z.real, z.imag, _ptr(R), _ptr(q))
    if st != 0:
        raise ArithmeticError("zero pivot in oracle LU")
    return q


def alpha(xyz, q, E0=1.0):
    """alpha_{k'} = sum_i q_i r_{i,k'} / E0 for k' = x, y, z (from Eq. 28)."""
    xyz = _f64(xyz)
    q = _c128(q)
    out = np.empty(6)
    lib().orc_alpha(len(xyz), _ptr(xyz), _ptr(q), float(E0), _ptr(out))
    return out[0::2] + 1j * out[1::2]


def apply_rows(xyz, p, z, x, rows, eta=None):
    """Selected rows of (A - zI) x with D recomputed from Eq. 3 and each row's neighbours
    found by a brute-force scan (no N x N storage, no CSR), plus the per-row rounding
    scale sum_p Kbar_ip (s_i + s_j) + |z||x_i|, s = |D||x|."""
    xyz = _f64(xyz)
    n = len(xyz)
    eta = _eta_vec(n, p["eta"] if eta is None else eta)
    x = _c128(x)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty(len(rows), dtype=np.complex128)
    bound = np.empty(len(rows))
    lib().orc_apply_rows(n, _ptr(xyz), _ptr(eta), p["r0"], p["d_fermi"], p["s_fermi"], p["area"],
                         p["cutoff_eps"], z.real, z.imag, _ptr(x), len(rows), _ptr(rows), _ptr(y), _ptr(bound))
    return y, bound


def rhs_rows(xyz, p, kdir, rows, E0=1.0):
    """Selected rows of R (Eq. 13, Eq. 2), each row's neighbours by a brute-force scan."""
    xyz = _f64(xyz)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    kd = _f64(np.asarray(kdir, dtype=np.float64))
    out = np.empty(len(rows))
    lib().orc_rhs_rows(len(xyz), _ptr(xyz), p["r0"], p["d_fermi"], p["s_fermi"], p["area"], p["cutoff_eps"],
                       _ptr(kd), float(E0), len(rows), _ptr(rows), _ptr(out))
    return out


def vdot(u, v):
    u = _c128(u)
    v = _c128(v)
    out = np.empty(2)
    lib().orc_vdot(len(u), _ptr(u), _ptr(v), _ptr(out))
    return complex(out[0], out[1])


# ---------------------------------------------------------------- convenience


class System:
    """Everything the oracle assembles for one structure: D, Kbar (dense or CSR),
    and, for small N, A by Eq. 11.  `solve` returns q for (omega, direction)."""

    def __init__(self, xyz, p, eta=None, dense=None, cutoff_eps=None, assemble_a=None):
        self.xyz = _f64(xyz)
        self.p = dict(p)
        self.n = n = len(self.xyz)
        self.eta = _eta_vec(n, p["eta"] if eta is None else eta)
        if dense is None:
            dense = n <= 5000
        self.dense = dense
        if dense:
            self.D = d_matrix(self.xyz, self.eta)
            self.K = kbar_matrix(self.xyz, self.p)
            rowptr = np.arange(0, n * n + 1, n, dtype=np.int64)
            self.csr = (rowptr, np.tile(np.arange(n, dtype=np.int64), n), self.K.ravel())
        else:
            self.D = None
            self.K = None
            self.csr = kbar_csr(self.xyz, self.p, cutoff_eps)
        if assemble_a is None:
            assemble_a = dense and n <= 2000
        self.A = a_matrix(self.D, self.K) if assemble_a else None

    def rhs(self, kdir, E0=1.0):
        if self.K is not None:
            return rhs_dense(self.xyz, self.K, kdir, E0)
        return rhs_csr(self.xyz, self.csr, kdir, E0)

    def z(self, omega):
        return z_of_omega(omega, self.p)

    def operator(self, stored=True):
        if self.D is not None and stored:
            return Operator.stored(self.D, self.csr)
        return Operator.on_the_fly(self.xyz, self.eta, self.csr)

    def solve(self, omega, kdir, E0=1.0, method="lu", rel_tol=1e-12, max_iter=2000, restart=0):
        R = self.rhs(kdir, E0).astype(np.complex128)
        z = self.z(omega)
        if method == "lu":
            if self.A is None:
                raise ValueError("LU needs the assembled A (small N)")
            return lu_solve(self.A, z, R), {"method": "lu"}
        op = self.operator()
        if method == "gmres":
            return op.gmres(z, R, restart=restart, rel_tol=rel_tol, max_iter=max_iter)
        if method == "qmr":
            return op.qmr(z, R, rel_tol=rel_tol, max_iter=max_iter)
        raise ValueError(method)
