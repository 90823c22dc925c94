"""FP64 CPU oracle for the polynomial-filtered interior eigensolver (arXiv 1902.07041).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``. The product library never imports, links or runs it.

The arithmetic lives in ``oracle.c`` (plain C, scalar CSR, column-major multivectors, its own
dense linear algebra and its own Philox4x32-10 generator). This module compiles it with gcc on
first use and wraps it with ctypes; it adds no arithmetic of its own beyond argument marshalling,
except ``exact_interval`` which calls LAPACK (numpy.linalg.eigh) as a library step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

DAMPING = {"none": 0, "jackson": 1, "lanczos": 2}

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double
_U64 = ctypes.c_uint64
_U32 = ctypes.c_uint32


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared object (idempotent unless ``force``)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _sig(lib, name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        _sig(lib, "or_csr_free", None, [_P])
        _sig(lib, "or_csr_n", _I64, [_P])
        _sig(lib, "or_csr_nnz", _I64, [_P])
        _sig(lib, "or_csr_export", None, [_P, _P, _P, _P])
        _sig(lib, "or_csr_from_arrays", _P, [_I64, _P, _P, _P])
        _sig(lib, "or_csr_from_springs", _P, [_I32, _I64, _P, _P, _P, _P, _P])
        _sig(lib, "or_spmm", None, [_P, _I32, _P, _I64, _P, _I64])
        _sig(lib, "or_residuals", None, [_P, _I32, _P, _P, _I64, _P])
        _sig(lib, "or_participation_ratio", None, [_I64, _I32, _P, _I64, _P])
        _sig(lib, "or_dirac_coeffs", None, [_D, _I32, ctypes.c_int, _P])
        _sig(lib, "or_dirac_gamma", _D, [_D, _D, _I32, ctypes.c_int])
        _sig(lib, "or_dirac_degree", _I32, [_D, _D, _D, ctypes.c_int, _I32])
        _sig(lib, "or_plane_wave_content", None, [_I64, _I32, _P, _I64, _P, _I32, _P, _P])
        _sig(lib, "or_pq_coeffs", None, [_D, _D, _D, _I32, _P])
        _sig(lib, "or_chi_coeffs", None, [_D, _D, _I32, _P])
        _sig(lib, "or_damping", None, [ctypes.c_int, _I32, _P])
        _sig(lib, "or_series_value", _D, [_P, _I32, _D])
        _sig(lib, "or_select_degree", _I32, [_D, _D, _D, _D, ctypes.c_int, _I32])
        _sig(lib, "or_cheb_filter", _I64, [_P, _D, _D, _P, _I32, _I32, _P, _I64, _P, _I64])
        _sig(lib, "or_philox4x32_10", None, [_P, _P, _P])
        _sig(lib, "or_normal", _D, [_U64, _U32, _U32, _U32])
        _sig(lib, "or_normal_block", None, [_U64, _U32, _I64, _I32, _I32, _P, _I64])
        _sig(lib, "or_jacobi_eig", None, [_I32, _P, _P, _P])
        _sig(lib, "or_householder_qr", ctypes.c_int, [_I64, _I32, _P, _I64, _P])
        _sig(lib, "or_tridiagonalize", None, [_I32, _P, _P, _P])
        _sig(lib, "or_count_below", _I64, [_I32, _P, _P, _D])
        _sig(lib, "or_lanczos_lmax", ctypes.c_int, [_P, _I32, _U64, _P, _P, _P])
        _sig(lib, "or_count_estimate", _D, [_P, _D, _D, _D, _D, _I32, ctypes.c_int, _I32, _U64])
        _sig(lib, "or_si_solve", ctypes.c_int,
             [_P, _D, _D, _D, _D, _P, _I32, _I32, _P, _D, _I32, _I32, _P, _P, _P, _P, _P, _P])
        _sig(lib, "or_si_alg4_diag", _I32, [_I64, _P, _I32, _I32, _I32, _D, _P, _I32])
        _sig(lib, "or_bks_solve", ctypes.c_int,
             [_P, _D, _D, _D, _D, _P, _I32, _I32, _I32, _I32, _P, _D, _D, _I32, _I32, _P, _P, _P, _P, _P, _P])
        _sig(lib, "or_filter_adjoint", ctypes.c_int,
             [_P, _D, _D, _P, _I32, _I32, _P, _I64, _P, _I64, _P, _I64, _P])
        _sig(lib, "or_chain_springs", None, [_P, _I32, _I64, _P, _P, _P, _P, _P, _P, _P, _P])
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _fortran(a):
    return np.asfortranarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data


class CSR:
    """Scalar CSR matrix owned by the oracle (FP64)."""

    def __init__(self, handle):
        if not handle:
            raise MemoryError("oracle: CSR allocation failed")
        self._h = handle
        self._lib = _load()

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.or_csr_free(h)

    @property
    def handle(self):
        return self._h

    @property
    def n(self) -> int:
        return int(self._lib.or_csr_n(self._h))

    @property
    def nnz(self) -> int:
        return int(self._lib.or_csr_nnz(self._h))

    def arrays(self):
        rp = np.zeros(self.n + 1, np.int64)
        ci = np.zeros(self.nnz, np.int32)
        v = np.zeros(self.nnz, np.float64)
        self._lib.or_csr_export(self._h, _ptr(rp), _ptr(ci), _ptr(v))
        return rp, ci, v

    def dense(self) -> np.ndarray:
        rp, ci, v = self.arrays()
        A = np.zeros((self.n, self.n))
        for i in range(self.n):
            A[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
        return A

    def matmul(self, X: np.ndarray) -> np.ndarray:
        X = _fortran(X.reshape(self.n, -1))
        Y = np.zeros_like(X, order="F")
        self._lib.or_spmm(self._h, X.shape[1], _ptr(X), self.n, _ptr(Y), self.n)
        return Y


def csr_from_springs(glass) -> CSR:
    """Mass-weighted Hessian H_ij = Delta_ij / sqrt(m_i m_j) of a glassgen.Glass (eqs. (1)-(2))."""
    lib = _load()
    bi = np.ascontiguousarray(glass.bi, np.int32)
    bj = np.ascontiguousarray(glass.bj, np.int32)
    k = _f64(glass.k)
    rh = _f64(glass.rhat)
    m = _f64(glass.mass)
    return CSR(lib.or_csr_from_springs(glass.n_atoms, bi.shape[0], _ptr(bi), _ptr(bj), _ptr(k), _ptr(rh), _ptr(m)))


def csr_from_arrays(rp, ci, v) -> CSR:
    rp = np.ascontiguousarray(rp, np.int64)
    ci = np.ascontiguousarray(ci, np.int32)
    v = _f64(v)
    return CSR(_load().or_csr_from_arrays(rp.shape[0] - 1, _ptr(rp), _ptr(ci), _ptr(v)))


def csr_diagonal(d) -> CSR:
    d = _f64(d)
    n = d.shape[0]
    return csr_from_arrays(np.arange(n + 1), np.arange(n), d)


# ---------------------------------------------------------------- coefficients and degree
def pq_coeffs(xi, eta, eps, m) -> np.ndarray:
    g = np.zeros(m + 1)
    _load().or_pq_coeffs(xi, eta, eps, m, _ptr(g))
    return g


def chi_coeffs(xi, eta, m) -> np.ndarray:
    g = np.zeros(m + 1)
    _load().or_chi_coeffs(xi, eta, m, _ptr(g))
    return g


def damping(kind, k) -> np.ndarray:
    g = np.zeros(k + 1)
    _load().or_damping(DAMPING[kind] if isinstance(kind, str) else int(kind), k, _ptr(g))
    return g


def series_value(c, x) -> float:
    c = _f64(c)
    return float(_load().or_series_value(_ptr(c), c.shape[0] - 1, float(x)))


def select_degree(xi, eta, eps, r, kind="jackson", kmax=20000) -> int:
    return int(_load().or_select_degree(xi, eta, eps, r, DAMPING[kind], kmax))


def filter_coeffs(xi, eta, eps, m, kind="jackson") -> np.ndarray:
    """Damped coefficients g_j gamma_j of the piecewise-quadratic filter of degree m."""
    return pq_coeffs(xi, eta, eps, m) * damping(kind, m)


# ---------------------------------------------------------------- filter and friends
def cheb_filter(H: CSR, c, d, coef, X) -> np.ndarray:
    """Alg. 2 on each column of X with Ht = (H - cI)/d."""
    coef = _f64(coef)
    X = _fortran(X.reshape(H.n, -1))
    Y = np.zeros_like(X, order="F")
    _load().or_cheb_filter(H.handle, c, d, _ptr(coef), coef.shape[0] - 1, X.shape[1], _ptr(X), H.n, _ptr(Y), H.n)
    return Y


def philox(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return [int(x) for x in o]


def normal_block(seed, stream, n, k, col0=0) -> np.ndarray:
    X = np.zeros((n, k), order="F")
    _load().or_normal_block(seed, stream, n, k, col0, _ptr(X), n)
    return X


def jacobi_eig(A):
    A = _fortran(A).copy(order="F")
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), order="F")
    _load().or_jacobi_eig(n, _ptr(A), _ptr(w), _ptr(V))
    return w, V


def householder_qr(X):
    X = _fortran(X).copy(order="F")
    n, q = X.shape
    R = np.zeros((q, q), order="F")
    if _load().or_householder_qr(n, q, _ptr(X), n, _ptr(R)) != 0:
        raise ValueError("householder_qr: n < q")
    return X, R


def tridiagonalize(A):
    A = _fortran(A).copy(order="F")
    n = A.shape[0]
    d = np.zeros(n)
    e = np.zeros(max(n - 1, 1))
    _load().or_tridiagonalize(n, _ptr(A), _ptr(d), _ptr(e))
    return d, e[: n - 1]


def count_below(diag, off, sigma) -> int:
    d = _f64(diag)
    e = _f64(off) if len(off) else np.zeros(1)
    return int(_load().or_count_below(d.shape[0], _ptr(d), _ptr(e), float(sigma)))


def inertia_count(A_dense, a, b) -> int:
    """Number of eigenvalues in [a, b): nu(A - bI) - nu(A - aI) from the Sturm pivots."""
    d, e = tridiagonalize(A_dense)
    return count_below(d, e, b) - count_below(d, e, a)


def lanczos_lmax(H: CSR, steps=30, seed=0):
    th, rb, est = _D(), _D(), _D()
    rc = _load().or_lanczos_lmax(H.handle, steps, seed, ctypes.byref(th), ctypes.byref(rb), ctypes.byref(est))
    if rc != 0:
        raise ValueError("lanczos_lmax: bad arguments")
    return th.value, rb.value, est.value


def count_estimate(H: CSR, c, d, xi, eta, degree=100, kind="none", M=30, seed=0) -> float:
    return float(_load().or_count_estimate(H.handle, c, d, xi, eta, degree, DAMPING[kind], M, seed))


def residuals(H: CSR, lam, V) -> np.ndarray:
    lam = _f64(lam)
    V = _fortran(V.reshape(H.n, -1))
    r = np.zeros(V.shape[1])
    _load().or_residuals(H.handle, V.shape[1], _ptr(lam), _ptr(V), H.n, _ptr(r))
    return r


@dataclass
class SIResult:
    status: int
    lam: np.ndarray
    vecs: np.ndarray
    res: np.ndarray
    iters: int
    matvecs: int


def si_solve(H: CSR, a, b, lmin, lmax, coef, q, X0, tol=1e-8, max_iter=100, cap=None) -> SIResult:
    """Filtered subspace iteration with Rayleigh-Ritz on H and locking (see oracle.c)."""
    coef = _f64(coef)
    X0 = _fortran(X0.reshape(H.n, q))
    cap = q if cap is None else cap
    lam = np.zeros(cap)
    vec = np.zeros((H.n, cap), order="F")
    res = np.zeros(cap)
    nf, it, mv = _I32(), _I32(), _I64()
    st = _load().or_si_solve(H.handle, a, b, lmin, lmax, _ptr(coef), coef.shape[0] - 1, q, _ptr(X0), tol,
                             max_iter, cap, ctypes.byref(nf), _ptr(lam), _ptr(vec), _ptr(res), ctypes.byref(it),
                             ctypes.byref(mv))
    if st < 0:
        raise ValueError(f"si_solve: bad arguments ({st})")
    k = min(nf.value, cap)
    return SIResult(st, lam[:k].copy(), vec[:, :k].copy(), res[:k].copy(), it.value, mv.value)


def bks_solve(H: CSR, a, b, lmin, lmax, coef, bs, maxbasis, keep_min, X0, theta_cut, tol=1e-8, max_restarts=50,
              cap=None) -> SIResult:
    """Thick-restart block Lanczos on p(Ht), then Rayleigh-Ritz with H (see oracle.c)."""
    coef = _f64(coef)
    X0 = _fortran(X0.reshape(H.n, bs))
    cap = maxbasis if cap is None else cap
    lam = np.zeros(cap)
    vec = np.zeros((H.n, cap), order="F")
    res = np.zeros(cap)
    nf, it, mv = _I32(), _I32(), _I64()
    st = _load().or_bks_solve(H.handle, a, b, lmin, lmax, _ptr(coef), coef.shape[0] - 1, bs, maxbasis, keep_min,
                              _ptr(X0), theta_cut, tol, max_restarts, cap, ctypes.byref(nf), _ptr(lam), _ptr(vec),
                              _ptr(res), ctypes.byref(it), ctypes.byref(mv))
    if st < 0:
        raise ValueError(f"bks_solve: bad arguments ({st})")
    k = min(nf.value, cap)
    return SIResult(st, lam[:k].copy(), vec[:, :k].copy(), res[:k].copy(), it.value, mv.value)


def si_alg4_diag(pd, q, p, n_rr, tau, X0, max_k=200) -> int:
    pd = _f64(pd)
    X0 = _fortran(X0)
    return int(_load().or_si_alg4_diag(pd.shape[0], _ptr(pd), q, p, n_rr, tau, _ptr(X0), max_k))


def filter_adjoint(H: CSR, c, d, coef, X, Ybar):
    """Reverse sweep of Alg. 2: returns (Xbar, vbar per stored CSR entry)."""
    coef = _f64(coef)
    X = _fortran(X.reshape(H.n, -1))
    Yb = _fortran(Ybar.reshape(H.n, -1))
    Xb = np.zeros_like(X, order="F")
    vb = np.zeros(H.nnz)
    rc = _load().or_filter_adjoint(H.handle, c, d, _ptr(coef), coef.shape[0] - 1, X.shape[1], _ptr(X), H.n,
                                   _ptr(Yb), H.n, _ptr(Xb), H.n, _ptr(vb))
    if rc != 0:
        raise MemoryError("filter_adjoint: out of memory")
    return Xb, vb


def chain_springs(H: CSR, glass, vbar):
    """dL/dk per bond and dL/dm per atom from dL/dH per stored entry."""
    bi = np.ascontiguousarray(glass.bi, np.int32)
    bj = np.ascontiguousarray(glass.bj, np.int32)
    k = _f64(glass.k)
    rh = _f64(glass.rhat)
    m = _f64(glass.mass)
    vb = _f64(vbar)
    kb = np.zeros(bi.shape[0])
    mb = np.zeros(glass.n_atoms)
    _load().or_chain_springs(H.handle, glass.n_atoms, bi.shape[0], _ptr(bi), _ptr(bj), _ptr(k), _ptr(rh), _ptr(m),
                             _ptr(vb), _ptr(kb), _ptr(mb))
    return kb, mb


def exact_interval(H: CSR, a, b):
    """All eigenpairs of the (small) dense H with eigenvalue in [a, b], by LAPACK dsyevd."""
    w, V = np.linalg.eigh(H.dense())
    sel = (w >= a) & (w <= b)
    return w[sel], V[:, sel], w


def participation_ratio(V) -> np.ndarray:
    """Normalised participation ratio of each column (Sec. 4.4, eq. (PR_def) divided by N)."""
    V = _fortran(np.asarray(V, np.float64).reshape(np.shape(V)[0], -1))
    pr = np.zeros(V.shape[1])
    _load().or_participation_ratio(V.shape[0] // 3, V.shape[1], _ptr(V), V.shape[0], _ptr(pr))
    return pr


def plane_wave_content(V, pos, kvecs) -> np.ndarray:
    """(k, nk, 2): longitudinal and transverse plane-wave content of each column (Sec. 4.4)."""
    V = _fortran(np.asarray(V, np.float64).reshape(np.shape(V)[0], -1))
    pos = _f64(np.asarray(pos).reshape(-1))
    kv = _f64(np.asarray(kvecs).reshape(-1, 3))
    out = np.zeros((V.shape[1], kv.shape[0], 2))
    _load().or_plane_wave_content(V.shape[0] // 3, V.shape[1], _ptr(V), V.shape[0], _ptr(pos), kv.shape[0], _ptr(kv),
                                  _ptr(out))
    return out


def dirac_coeffs(gamma, k, kind="jackson") -> np.ndarray:
    """Damped coefficients of the Dirac filter rho_k(x) centred at gamma (eq. (cheby-delta.1))."""
    c = np.zeros(k + 1)
    _load().or_dirac_coeffs(float(gamma), int(k), DAMPING[kind], _ptr(c))
    return c


def dirac_gamma(xi, eta, k, kind="jackson") -> float:
    """Centre gamma in (xi, eta) with rho_k(xi) = rho_k(eta)."""
    return _load().or_dirac_gamma(float(xi), float(eta), int(k), DAMPING[kind])


def dirac_degree(xi, eta, phi, kind="jackson", kmax=20000) -> int:
    """Smallest degree whose balanced Dirac filter has rho(xi) / rho(gamma) <= phi."""
    return _load().or_dirac_degree(float(xi), float(eta), float(phi), DAMPING[kind], int(kmax))
