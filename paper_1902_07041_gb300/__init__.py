"""Python binding of libpfe, the GB300 polynomial-filtered interior eigensolver (arXiv 1902.07041).

Thin ctypes marshalling over the C ABI declared in include/pfe.h: every function here has the
name of the C entry point it calls and does no arithmetic of its own. Device pointers may be given
as integers or as torch CUDA tensors. A failed call raises PfeError with the library's message.

The compiled library (libpfe.so, next to this file) is required: importing works without it, but
the first call raises if it has not been built (python -m paper_1902_07041_gb300.build).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpfe.so")

# status codes (pfe_status)
PFE_OK, PFE_E_ARG, PFE_E_NOMEM, PFE_E_CUDA, PFE_E_NOTSYM, PFE_E_CAPACITY = 0, 1, 2, 3, 4, 5
PFE_E_NOCONV, PFE_E_BREAKDOWN, PFE_E_BOUND, PFE_E_TIMEOUT, PFE_E_STATE = 6, 7, 8, 9, 10
STATUS_NAMES = {0: "PFE_OK", 1: "PFE_E_ARG", 2: "PFE_E_NOMEM", 3: "PFE_E_CUDA", 4: "PFE_E_NOTSYM",
                5: "PFE_E_CAPACITY", 6: "PFE_E_NOCONV", 7: "PFE_E_BREAKDOWN", 8: "PFE_E_BOUND",
                9: "PFE_E_TIMEOUT", 10: "PFE_E_STATE"}
# flags
PFE_DEVICE_PTRS, PFE_SKIP_SYM_CHECK = 0x1, 0x2
# dtypes
PFE_F64, PFE_F32 = 0, 1
# parameter keys
PFE_P_DEGREE, PFE_P_EPS_FRAC, PFE_P_RATE, PFE_P_DAMPING, PFE_P_WIDTH = 1, 2, 3, 4, 5
PFE_P_WIDTH_FACTOR, PFE_P_TOL, PFE_P_PRECISION, PFE_P_MAX_ITERS, PFE_P_SEED = 6, 7, 8, 9, 10
PFE_P_LAMBDA_MAX, PFE_P_LAMBDA_MIN, PFE_P_COUNT_M, PFE_P_COUNT_DEGREE = 11, 12, 13, 14
PFE_P_LANCZOS_STEPS, PFE_P_COUNT_DAMPING, PFE_P_MIN_WIDTH, PFE_P_REFINE_TOL = 15, 16, 17, 18
PFE_P_STEP_SHAPE_F64, PFE_P_STEP_SHAPE_F32 = 19, 20
PFE_P_METHOD, PFE_P_BLOCK, PFE_P_BASIS_FACTOR, PFE_P_BATCH_THREADS, PFE_P_RANK1 = 21, 22, 23, 24, 25
PFE_P_FILTER, PFE_P_PHI, PFE_P_DIRAC_CUT, PFE_P_SLICE_TARGET, PFE_P_OVERLAP = 26, 27, 28, 29, 30
PFE_P_DEGREE_RULE = 31

# every entry point declared in include/pfe.h
EXPORTS = ("pfe_springs_to_bsr", "pfe_create", "pfe_destroy", "pfe_last_error", "pfe_set_param",
           "pfe_get_param", "pfe_set_interval", "pfe_estimate", "pfe_get_filter", "pfe_solve",
           "pfe_get_eigenpairs", "pfe_get_stats", "pfe_filter_apply", "pfe_filter_adjoint",
           "pfe_chain_springs", "pfe_solve_batch", "pfe_filter_apply_noalloc", "pfe_participation_ratio",
           "pfe_plane_wave_content", "pfe_solve_sliced", "pfe_design_filter", "pfe_solve_begin",
           "pfe_solve_iterate", "pfe_solve_end", "pfe_probe_fp64_fma")


class PfeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class PfeStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("width", ctypes.c_int32), ("degree", ctypes.c_int32),
                ("n_found", ctypes.c_int32), ("matvecs", ctypes.c_int64), ("lambda_max", ctypes.c_double),
                ("count_estimate", ctypes.c_double), ("seconds_total", ctypes.c_double),
                ("seconds_filter", ctypes.c_double), ("seconds_orth", ctypes.c_double),
                ("seconds_rr", ctypes.c_double), ("max_residual", ctypes.c_double),
                ("fp64_sweeps", ctypes.c_int32), ("status", ctypes.c_int32), ("window_estimate", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("filter_launches", ctypes.c_int64),
                ("filter_col_steps", ctypes.c_int64), ("filter_col_steps_f32", ctypes.c_int64),
                ("seconds_filter_f32", ctypes.c_double), ("batch_replays", ctypes.c_int64),
                ("restarts", ctypes.c_int32), ("basis", ctypes.c_int32), ("filter_shape_f64", ctypes.c_int32),
                ("filter_shape_f32", ctypes.c_int32), ("slices", ctypes.c_int32), ("active", ctypes.c_int32),
                ("locked", ctypes.c_int32), ("cholqr_shifts", ctypes.c_int32),
                ("filter_col_steps_forced", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_P, _I32, _I64, _D, _U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32


def load(path: str | None = None):
    """Load libpfe.so; raises if it is missing (there is no fallback implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libpfe.so is not built ({path}); run `python -m paper_1902_07041_gb300.build`")
    lib = ctypes.CDLL(path)
    sig = {
        "pfe_springs_to_bsr": (ctypes.c_int, [_I32, _I64, _P, _P, _P, _P, _I64, _P, _P, _P, _P]),
        "pfe_create": (ctypes.c_int, [_P, _I32, _I64, _P, _P, _P, _P, _U32, _P]),
        "pfe_destroy": (None, [_P]),
        "pfe_last_error": (ctypes.c_char_p, [_P]),
        "pfe_set_param": (ctypes.c_int, [_P, ctypes.c_int, _D]),
        "pfe_get_param": (ctypes.c_int, [_P, ctypes.c_int, _P]),
        "pfe_set_interval": (ctypes.c_int, [_P, _D, _D]),
        "pfe_estimate": (ctypes.c_int, [_P, _P, _P]),
        "pfe_get_filter": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P]),
        "pfe_solve": (ctypes.c_int, [_P, _P]),
        "pfe_solve_begin": (ctypes.c_int, [_P]),
        "pfe_solve_iterate": (ctypes.c_int, [_P, _P]),
        "pfe_solve_end": (ctypes.c_int, [_P, _P]),
        "pfe_probe_fp64_fma": (ctypes.c_int, [_I32, _I32, _P, _P, _P]),
        "pfe_get_eigenpairs": (ctypes.c_int, [_P, _I32, _P, _P, _P, _U32]),
        "pfe_get_stats": (ctypes.c_int, [_P, _P]),
        "pfe_filter_apply": (ctypes.c_int, [_P, _I32, _P, _I32, _P, _I64, _P, _I64, ctypes.c_int, _P]),
        "pfe_filter_adjoint": (ctypes.c_int, [_P, _I32, _P, _I32, _P, _I64, _P, _I64, _P, _I64, _P, _P]),
        "pfe_chain_springs": (ctypes.c_int, [_P, _I64, _P, _P, _P, _P, _P, _P, _P]),
        "pfe_solve_batch": (ctypes.c_int, [_P, _I32, _P]),
        "pfe_filter_apply_noalloc": (ctypes.c_int, [_P, _I32, _P, _I32, _P, _I64, _P, _I64, _P]),
        "pfe_participation_ratio": (ctypes.c_int, [_P, _I32, _P]),
        "pfe_plane_wave_content": (ctypes.c_int, [_P, _P, _I32, _P, _I32, _P]),
        "pfe_solve_sliced": (ctypes.c_int, [_P, _I32, _P, _P]),
        "pfe_design_filter": (ctypes.c_int, [ctypes.c_int, _D, _D, _D, _D, _D, ctypes.c_int, _I32, _I32, _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st: int, ctx=None, what: str = ""):
    if st != PFE_OK:
        msg = pfe_last_error(ctx) if ctx else what
        raise PfeError(st, msg or what)


def _dptr(x) -> int:
    """Device address of a torch tensor or an integer pointer."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return int(getattr(s, "cuda_stream", 0))


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------------------------------ ABI
def pfe_springs_to_bsr(n_atoms, bi, bj, k, rhat):
    """Host assembly of Delta from springs; returns (row_ptr, col_idx, vals) as numpy arrays."""
    lib = load()
    bi, bj = _host(bi, np.int32), _host(bj, np.int32)
    k, rhat = _host(k, np.float64), _host(rhat, np.float64)
    nb = ctypes.c_int64(0)
    st = lib.pfe_springs_to_bsr(n_atoms, bi.shape[0], bi.ctypes.data, bj.ctypes.data, k.ctypes.data,
                                rhat.ctypes.data, 0, None, None, None, ctypes.byref(nb))
    if st not in (PFE_OK, PFE_E_CAPACITY):
        _check(st, what="pfe_springs_to_bsr: invalid bonds")
    nnzb = nb.value
    rp = np.zeros(n_atoms + 1, np.int32)
    ci = np.zeros(nnzb, np.int32)
    vals = np.zeros(9 * nnzb, np.float64)
    st = lib.pfe_springs_to_bsr(n_atoms, bi.shape[0], bi.ctypes.data, bj.ctypes.data, k.ctypes.data,
                                rhat.ctypes.data, nnzb, rp.ctypes.data, ci.ctypes.data, vals.ctypes.data,
                                ctypes.byref(nb))
    _check(st, what="pfe_springs_to_bsr failed")
    return rp, ci, vals


def pfe_create(n_atoms, row_ptr, col_idx, vals, masses=None, flags=0, stream=None):
    """Create a context. Host numpy arrays, or device tensors with flags |= PFE_DEVICE_PTRS."""
    lib = load()
    out = ctypes.c_void_p(0)
    if flags & PFE_DEVICE_PTRS:
        nnzb = int(col_idx.numel())
        args = (_dptr(row_ptr), _dptr(col_idx), _dptr(vals), _dptr(masses))
        keep = None
    else:
        row_ptr, col_idx = _host(row_ptr, np.int32), _host(col_idx, np.int32)
        vals = _host(vals, np.float64)
        masses = None if masses is None else _host(masses, np.float64)
        nnzb = int(col_idx.shape[0])
        args = (row_ptr.ctypes.data, col_idx.ctypes.data, vals.ctypes.data,
                None if masses is None else masses.ctypes.data)
        keep = (row_ptr, col_idx, vals, masses)
    st = lib.pfe_create(ctypes.byref(out), int(n_atoms), nnzb, *args, int(flags), _stream(stream))
    del keep
    _check(st, what="pfe_create failed (invalid structure, values or CUDA error)")
    return out.value


def pfe_destroy(ctx):
    if ctx:
        load().pfe_destroy(ctx)


def pfe_last_error(ctx) -> str:
    r = load().pfe_last_error(ctx)
    return r.decode() if r else ""


def pfe_set_param(ctx, key, value):
    _check(load().pfe_set_param(ctx, int(key), float(value)), ctx)


def pfe_get_param(ctx, key) -> float:
    v = ctypes.c_double(0)
    _check(load().pfe_get_param(ctx, int(key), ctypes.byref(v)), ctx, "unknown key")
    return v.value


def pfe_set_interval(ctx, a, b):
    _check(load().pfe_set_interval(ctx, float(a), float(b)), ctx)


def pfe_estimate(ctx):
    """Returns (lambda_max bound, eigenvalue-count estimate or nan)."""
    lm, ce = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().pfe_estimate(ctx, ctypes.byref(lm), ctypes.byref(ce)), ctx)
    return lm.value, ce.value


def pfe_get_filter(ctx):
    """Returns (degree m, damped coefficients[m+1], c, d)."""
    m, c, d = ctypes.c_int32(0), ctypes.c_double(0), ctypes.c_double(0)
    _check(load().pfe_get_filter(ctx, 0, ctypes.byref(m), None, ctypes.byref(c), ctypes.byref(d)), ctx)
    coef = np.zeros(m.value + 1)
    _check(load().pfe_get_filter(ctx, coef.shape[0], ctypes.byref(m), coef.ctypes.data, None, None), ctx)
    return m.value, coef, c.value, d.value


def pfe_solve(ctx, raise_on_error=True):
    """Returns (n_found, status)."""
    nf = ctypes.c_int32(0)
    st = load().pfe_solve(ctx, ctypes.byref(nf))
    if raise_on_error:
        _check(st, ctx)
    return nf.value, st


def pfe_solve_begin(ctx):
    """Set-up of a stepwise subspace-iteration solve."""
    _check(load().pfe_solve_begin(ctx), ctx)


def pfe_solve_iterate(ctx) -> bool:
    """One outer iteration; returns True once the solve has ended."""
    done = ctypes.c_int32(0)
    _check(load().pfe_solve_iterate(ctx, ctypes.byref(done)), ctx)
    return bool(done.value)


def pfe_solve_end(ctx, raise_on_error=True):
    """Results of a stepwise solve. Returns (n_found, status)."""
    nf = ctypes.c_int32(0)
    st = load().pfe_solve_end(ctx, ctypes.byref(nf))
    if raise_on_error:
        _check(st, ctx)
    return nf.value, st


def pfe_get_eigenpairs(ctx, n, cap, vecs_out=None):
    """Host copies (lambda, vecs n x cap column-major as an (n, cap) array, resid); with a torch
    tensor `vecs_out` (column-major n x cap storage, e.g. shape (cap, n)) the vectors go there: to the
    device for a CUDA tensor (or an integer device pointer), to host memory (e.g. pinned) for a CPU one."""
    lam = np.zeros(cap)
    res = np.zeros(cap)
    if vecs_out is None:
        vecs = np.zeros((cap, n))  # row c holds eigenvector c: column-major n x cap
        st = load().pfe_get_eigenpairs(ctx, cap, lam.ctypes.data, vecs.ctypes.data, res.ctypes.data, 0)
        _check(st, ctx)
        return lam, vecs.T, res
    flags = PFE_DEVICE_PTRS if getattr(vecs_out, "is_cuda", True) else 0
    st = load().pfe_get_eigenpairs(ctx, cap, lam.ctypes.data, _dptr(vecs_out), res.ctypes.data, flags)
    _check(st, ctx)
    return lam, vecs_out, res


def pfe_get_stats(ctx) -> dict:
    s = PfeStats()
    _check(load().pfe_get_stats(ctx, ctypes.byref(s)), ctx)
    return s.as_dict()


def pfe_filter_apply(ctx, m, coeffs, k, X, ldx, Y, ldy, dtype=PFE_F64, stream=None):
    """Y = p_m(Ht) X on device buffers (column-major n x k). coeffs None = the solver's filter."""
    if coeffs is not None:
        coeffs = _host(coeffs, np.float64)
        cptr = coeffs.ctypes.data
    else:
        cptr = None
    st = load().pfe_filter_apply(ctx, int(m), cptr, int(k), _dptr(X), int(ldx), _dptr(Y), int(ldy), int(dtype),
                                 _stream(stream))
    _check(st, ctx)


def pfe_filter_adjoint(ctx, m, coeffs, k, X, ldx, Ybar, ldyb, Xbar, ldxb, vals_bar, stream=None):
    if coeffs is not None:
        coeffs = _host(coeffs, np.float64)
        cptr = coeffs.ctypes.data
    else:
        cptr = None
    st = load().pfe_filter_adjoint(ctx, int(m), cptr, int(k), _dptr(X), int(ldx), _dptr(Ybar), int(ldyb),
                                   _dptr(Xbar), int(ldxb), _dptr(vals_bar), _stream(stream))
    _check(st, ctx)


def pfe_chain_springs(ctx, nbonds, bi, bj, rhat, vals_bar, k_bar, m_bar, stream=None):
    st = load().pfe_chain_springs(ctx, int(nbonds), _dptr(bi), _dptr(bj), _dptr(rhat), _dptr(vals_bar),
                                  _dptr(k_bar), _dptr(m_bar), _stream(stream))
    _check(st, ctx)


def pfe_solve_batch(ctxs):
    """Returns (n_found list, first failing status)."""
    arr = (ctypes.c_void_p * len(ctxs))(*ctxs)
    nf = np.zeros(len(ctxs), np.int32)
    st = load().pfe_solve_batch(arr, len(ctxs), nf.ctypes.data)
    return [int(x) for x in nf], st


def pfe_filter_apply_noalloc(ctx, m, coeffs, k, X, ldx, Y, ldy, stream=None):
    """pfe_filter_apply (FP64) with its work buffers in the library's fixed device array: no device
    allocation. Returns the status (raises on any status other than PFE_OK)."""
    coeffs = _host(coeffs, np.float64)
    st = load().pfe_filter_apply_noalloc(ctx, int(m), coeffs.ctypes.data, int(k), _dptr(X), int(ldx), _dptr(Y),
                                         int(ldy), _stream(stream))
    _check(st, ctx)


def pfe_participation_ratio(ctx, cap):
    """Participation ratio (normalised by N) of each found eigenvector, in eigenpair order."""
    pr = np.zeros(max(int(cap), 0))
    _check(load().pfe_participation_ratio(ctx, int(cap), pr.ctypes.data), ctx)
    return pr


def pfe_plane_wave_content(ctx, pos, kvecs, cap):
    """(cap, nk, 2) array: longitudinal and transverse plane-wave content of each found eigenvector."""
    pos = _host(pos, np.float64).reshape(-1)
    kv = _host(kvecs, np.float64).reshape(-1, 3)
    out = np.zeros((max(int(cap), 0), kv.shape[0], 2))
    st = load().pfe_plane_wave_content(ctx, pos.ctypes.data, kv.shape[0], np.ascontiguousarray(kv).ctypes.data,
                                       int(cap), out.ctypes.data)
    _check(st, ctx)
    return out


def pfe_solve_sliced(ctx, edges=None, raise_on_error=True):
    """Spectrum slicing of the context's interval; edges None = automatic (PFE_P_SLICE_TARGET per
    slice), else the interior edges. Returns (n_found, status)."""
    nf = ctypes.c_int32(0)
    if edges is None or len(edges) == 0:
        st = load().pfe_solve_sliced(ctx, 0, None, ctypes.byref(nf))
    else:
        ed = _host(edges, np.float64)
        st = load().pfe_solve_sliced(ctx, int(ed.size), ed.ctypes.data, ctypes.byref(nf))
    if raise_on_error and st != PFE_OK:
        _check(st, ctx)
    return nf.value, st


def pfe_probe_fp64_fma(iters, reps, sink, stream=None) -> float:
    """Measured FP64 FMA throughput (TFLOP/s) of this GPU; sink: a device tensor of >= 1 double."""
    t = ctypes.c_double(0)
    _check(load().pfe_probe_fp64_fma(int(iters), int(reps), _stream(stream), _dptr(sink), ctypes.byref(t)), None,
           "pfe_probe_fp64_fma failed")
    return t.value


DAMPING_KINDS = {"none": 0, "jackson": 1, "lanczos": 2}


def pfe_design_filter(kind, xi, eta, eps=0.0, r=0.0, phi=0.0, damping="none", degree=0):
    """Filter design on the host (no context, no GPU): kind "pq" (eps, r) or "dirac" (phi).
    Returns (degree, damped Chebyshev coefficients)."""
    k = {"pq": 0, "dirac": 1}[kind]
    dmp = DAMPING_KINDS[damping] if isinstance(damping, str) else int(damping)
    m = ctypes.c_int32(0)
    _check(load().pfe_design_filter(k, float(xi), float(eta), float(eps), float(r), float(phi), dmp, int(degree), 0,
                                    ctypes.byref(m), None), None, "pfe_design_filter: invalid arguments")
    c = np.zeros(m.value + 1)
    _check(load().pfe_design_filter(k, float(xi), float(eta), float(eps), float(r), float(phi), dmp, int(degree),
                                    c.size, ctypes.byref(m), c.ctypes.data), None, "pfe_design_filter failed")
    return m.value, c

