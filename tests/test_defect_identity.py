"""The splitting behind the defect-corrected FP32 filter (PRECISION 2), checked on the CPU.

For a block X with Rayleigh quotients theta, Ht = (H - cI)/d, theta_t = (theta - c)/d and the
residual block Rt = (H X - X diag(theta)) / d, the differences D_j = T_j(Ht) X - X diag(T_j(theta_t))
follow D_0 = 0, D_1 = Rt, D_{j+1} = 2 Ht D_j - D_{j-1} + 2 Rt diag(T_j(theta_t)), and
    p(Ht) X = X diag(p(theta_t)) + sum_j g_j D_j
exactly.  The library's kernels run the D recurrence in FP32 and form the first term in FP64.  The
tests check, against the oracle's Alg. 2 (FP64), that the identity holds to rounding in FP64 and
that with the recurrence in FP32 the error follows ||Rt|| instead of staying at the FP32 level of
the plain recurrence.  Everything here is numpy on a 60-atom glass.
"""
import numpy as np
import pytest

import glassgen
import oracle


@pytest.fixture(scope="module")
def setup():
    g = glassgen.generate(60, 11)
    H = oracle.csr_from_springs(g)
    A = H.dense()
    w, V = np.linalg.eigh(A)
    lmax = 1.01 * w[-1]
    c = d = lmax / 2
    a, b = 0.05 * lmax, 0.12 * lmax
    xi, eta = (a - c) / d, (b - c) / d
    coef = oracle.filter_coeffs(xi, eta, 0.25 * (eta - xi), 60, "none")
    inside = np.where((w >= a) & (w <= b))[0]
    return H, A, V, c, d, coef, inside


def _block(A, V, inside, pert, seed):
    """Orthonormal block near six interval eigenvectors, its Rayleigh quotients."""
    rng = np.random.default_rng(seed)
    X, _ = np.linalg.qr(V[:, inside[:6]] + pert * rng.standard_normal((A.shape[0], 6)))
    theta = np.einsum("ij,ij->j", X, A @ X)
    return X, theta


def _defect_filter(A, X, theta, c, d, coef, dt):
    """X p(theta_t) in FP64 plus the D recurrence in precision dt (its sum accumulated in FP64)."""
    n = A.shape[0]
    m = len(coef) - 1
    Ht = ((A - c * np.eye(n)) / d).astype(dt)
    tt = (theta - c) / d
    Rt = ((A @ X - X * theta) / d).astype(dt)
    Dm, D = np.zeros_like(Rt), Rt.copy()
    S = coef[1] * D.astype(np.float64)
    tm, tj = np.ones_like(tt), tt.copy()
    for j in range(1, m):
        Dn = 2 * (Ht @ D) - Dm + (2 * tj).astype(dt) * Rt
        S += coef[j + 1] * Dn.astype(np.float64)
        Dm, D = D, Dn
        tm, tj = tj, 2 * tt * tj - tm
    return X * np.polynomial.chebyshev.chebval(tt, coef) + S


def _plain_filter32(A, X, c, d, coef):
    """Alg. 2 with the recurrence in FP32 (its sum accumulated in FP64)."""
    n = A.shape[0]
    Ht = ((A - c * np.eye(n)) / d).astype(np.float32)
    T0 = X.astype(np.float32)
    T1 = Ht @ T0
    Y = coef[0] * T0.astype(np.float64) + coef[1] * T1.astype(np.float64)
    for j in range(1, len(coef) - 1):
        T2 = 2 * (Ht @ T1) - T0
        Y += coef[j + 1] * T2.astype(np.float64)
        T0, T1 = T1, T2
    return Y


@pytest.mark.parametrize("pert", [1e-2, 1e-4, 1e-6])
def test_defect_splitting_is_alg2_in_fp64(setup, pert):
    H, A, V, c, d, coef, inside = setup
    X, theta = _block(A, V, inside, pert, 3)
    ref = oracle.cheb_filter(H, c, d, coef, X)
    got = _defect_filter(A, X, theta, c, d, coef, np.float64)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_defect_error_follows_the_residual_in_fp32(setup):
    H, A, V, c, d, coef, inside = setup
    errs, rhos = [], []
    for pert in (1e-2, 1e-4, 1e-6):
        X, theta = _block(A, V, inside, pert, 3)
        ref = oracle.cheb_filter(H, c, d, coef, X)
        rho = np.linalg.norm((A @ X - X * theta) / d) / np.linalg.norm(X)
        err = np.linalg.norm(_defect_filter(A, X, theta, c, d, coef, np.float32) - ref) / np.linalg.norm(ref)
        # FP32 unit roundoff 6e-8 times a growth factor of the degree-60 recurrence, times ||Rt|| / ||X||
        assert err <= 1e-5 * rho, (pert, err, rho)
        errs.append(err)
        rhos.append(rho)
    plain = np.linalg.norm(_plain_filter32(A, X, c, d, coef) - ref) / np.linalg.norm(ref)
    assert plain >= 1e-8  # the plain FP32 recurrence stays at the FP32 level
    assert errs[-1] <= 1e-3 * plain  # near convergence the split form is far below it
    assert errs[0] > errs[1] > errs[2]
