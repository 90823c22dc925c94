"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a printed value of the paper
(tests/golden/, each with its citation), a closed form, a special case that reduces to a library
routine (LAPACK through numpy), an invariant, or a finite-difference derivative.
"""
import math

import numpy as np
import pytest

import glassgen
import oracle


# ------------------------------------------------------------------ printed values of the paper
def test_degrees_tables_1_3(golden):
    """All 27 degrees of Tables 1-3: coefficients (App. A), damping (Sec. 2.3), eq. (thresh)."""
    g = golden("degrees_tables_1_3.json")
    rs = [0.1, 0.1 ** 0.5, 0.1 ** 0.25]
    for case in g["cases"]:
        for ri, r in enumerate(rs):
            got = [oracle.select_degree(case["xi"], case["eta"], case["eps"], r, kind, kmax=7000)
                   for kind in g["columns"]]
            assert got == case["degrees"][ri], (case["table"], r, got)


def test_fig3_values(golden):
    f = golden("figures_2_3.json")["fig3"]
    xi, eta, eps, k = f["xi"], f["eta"], f["eps"], f["degree"]
    cj = oracle.filter_coeffs(xi, eta, eps, k, "jackson")
    cl = oracle.filter_coeffs(xi, eta, eps, k, "lanczos")
    half_ulp = 0.5 * 10 ** -f["printed_digits"]
    assert abs(oracle.series_value(cj, xi - eps) - f["jackson_left"]) <= half_ulp
    assert abs(oracle.series_value(cj, eta + eps) - f["jackson_right"]) <= half_ulp
    assert abs(oracle.series_value(cl, xi - eps) - f["lanczos_left"]) <= 0.5e-4
    assert abs(oracle.series_value(cl, eta + eps) - f["lanczos_right"]) <= 0.5e-4


def test_fig2_shape(golden):
    """The undamped series converges to p: p(xi) = p(eta) = 1, p(mid) = 1 + (eta-xi)/(2 eps) = 3,
    p = 0 outside [xi - eps, eta + eps]; q = p' has q(xi) = 2/eps = 80 (by differencing the series)."""
    f = golden("figures_2_3.json")["fig2"]
    xi, eta, eps = f["xi"], f["eta"], f["eps"]
    c = oracle.filter_coeffs(xi, eta, eps, 3000, "none")
    assert abs(oracle.series_value(c, 0.5 * (xi + eta)) - f["p_mid"]) < 1e-3
    assert abs(oracle.series_value(c, xi) - 1.0) < 1e-3
    assert abs(oracle.series_value(c, eta) - 1.0) < 1e-3
    for x in (-0.5, 0.0, xi - 2 * eps, eta + 2 * eps, 0.8):
        assert abs(oracle.series_value(c, x)) < 1e-3
    h = 1e-4
    dq = (oracle.series_value(c, xi + h) - oracle.series_value(c, xi - h)) / (2 * h)
    assert abs(dq - f["q_xi"]) < 1.0  # q has a kink at xi: the differentiated series converges like 1/k
    # coefficients of a C^1 piecewise quadratic decay like j^-3 (Sec. 2.6)
    j = np.arange(50, 3000)
    assert np.max(np.abs(c[50:3000]) * j ** 3) < 10 * np.max(np.abs(c[50:100]) * j[:50] ** 3)


def test_transform_example(golden):
    """Eq. (transf.1) folded into Alg. 2: with coefficients e_1 the filter returns Ht x = (H - c)/d x."""
    g = golden("transform_example.json")
    lmin, lmax = g["lambda_min"], g["lambda_max"]
    c, d = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    lam = np.array([p[0] for p in g["points"]])
    H = oracle.csr_diagonal(lam)
    y = oracle.cheb_filter(H, c, d, [0.0, 1.0], np.ones(3))[:, 0]
    for (l0, num, den), v in zip(g["fractions"], y):
        assert v == pytest.approx(num / den, abs=1e-15)


def test_philox_known_answers(golden):
    for v in golden("philox_kat.json")["vectors"]:
        out = oracle.philox([int(x, 16) for x in v["ctr"]], [int(x, 16) for x in v["key"]])
        assert out == [int(x, 16) for x in v["out"]]


def test_normals_moments():
    z = oracle.normal_block(7, 0, 200000, 1)[:, 0]
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    assert abs(np.mean(z ** 4) - 3.0) < 0.1


# ------------------------------------------------------------------ closed forms
def test_damping_factors():
    for k in (1, 5, 11, 200):
        gj = oracle.damping("jackson", k)
        gl = oracle.damping("lanczos", k)
        assert gj[0] == pytest.approx(1.0, abs=1e-14) and gl[0] == 1.0
        assert np.all(np.diff(gj) <= 1e-14) and np.all(gj >= -1e-14)  # decreasing to ~0
        assert gl[-1] == pytest.approx(math.sin(k * math.pi / (k + 1)) / (k * math.pi / (k + 1)))
    # Jackson damping keeps a nonnegative target nonnegative (monotone approximation, Sec. 2.3)
    xs = np.linspace(-1, 1, 801)
    for k in (11, 60, 150):
        c = oracle.chi_coeffs(-0.2, 0.2, k) * oracle.damping("jackson", k)
        assert min(oracle.series_value(c, x) for x in xs) > -1e-12
        c0 = oracle.chi_coeffs(-0.2, 0.2, k)
        assert min(oracle.series_value(c0, x) for x in xs) < -1e-3  # the undamped series has Gibbs dips


def test_chi_coeffs_closed_form():
    xi, eta = -0.3, 0.4
    c = oracle.chi_coeffs(xi, eta, 4000)
    assert c[0] == pytest.approx((math.acos(xi) - math.acos(eta)) / math.pi, rel=1e-15)
    assert oracle.series_value(c, 0.0) == pytest.approx(1.0, abs=2e-3)
    assert oracle.series_value(c, 0.8) == pytest.approx(0.0, abs=2e-3)
    assert oracle.series_value(c, xi) == pytest.approx(0.5, abs=2e-3)  # average of the jump


def test_series_value_closed_form():
    rng = np.random.default_rng(0)
    c = rng.standard_normal(40)
    for x in (-0.99, -0.3, 0.0, 0.7):
        ref = sum(cj * math.cos(j * math.acos(x)) for j, cj in enumerate(c))
        assert oracle.series_value(c, x) == pytest.approx(ref, abs=1e-12)


def test_cheb_filter_diagonal_closed_form():
    """Alg. 2 on a diagonal H: y_i = sum_j gamma_j cos(j arccos(lt_i)) x_i, lt = (lam - c)/d."""
    rng = np.random.default_rng(1)
    lam = np.sort(rng.uniform(0.0, 2.0, 60))
    c, d = 1.0, 1.0
    coef = oracle.filter_coeffs(-0.5, -0.3, 0.05, 37, "jackson")
    X = rng.standard_normal((60, 3))
    Y = oracle.cheb_filter(oracle.csr_diagonal(lam), c, d, coef, X)
    lt = (lam - c) / d
    pv = np.array([sum(g * math.cos(j * math.acos(t)) for j, g in enumerate(coef)) for t in lt])
    assert np.allclose(Y, pv[:, None] * X, atol=1e-13, rtol=0)


@pytest.fixture(scope="module")
def small_glass():
    g = glassgen.generate(60, 11)
    H = oracle.csr_from_springs(g)
    return g, H, H.dense()


def test_cheb_filter_vs_eigendecomposition(small_glass):
    """p(Ht) X = V p(lt) V^T X with LAPACK's eigendecomposition of a non-diagonal H."""
    g, H, A = small_glass
    w, V = np.linalg.eigh(A)
    lmax = w[-1] * 1.01
    c = d = lmax / 2
    coef = oracle.filter_coeffs(-0.9, -0.7, 0.05, 50, "lanczos")
    X = np.random.default_rng(2).standard_normal((H.n, 4))
    Y = oracle.cheb_filter(H, c, d, coef, X)
    lt = (w - c) / d
    pv = np.array([oracle.series_value(coef, t) for t in lt])
    ref = V @ (pv[:, None] * (V.T @ X))
    assert np.allclose(Y, ref, atol=1e-12 * np.abs(ref).max(), rtol=0)


# ------------------------------------------------------------------ model invariants
def _residuals_ld(H, lam, V, ld):
    """or_residuals called directly with a leading dimension ld >= n (V: ld x k, column-major)."""
    lam = np.ascontiguousarray(lam, np.float64)
    V = np.asfortranarray(V, np.float64)
    r = np.zeros(V.shape[1])
    oracle._load().or_residuals(H.handle, V.shape[1], oracle._ptr(lam), oracle._ptr(V), ld, oracle._ptr(r))
    return r


def test_residuals_diagonal_closed_form():
    """Alg. 3's residual r = ||H v - lambda v|| on a diagonal H, where it has a closed form:
    for v = alpha e_i + beta e_j, H v - mu v = alpha (d_i - mu) e_i + beta (d_j - mu) e_j, so
    r = sqrt(alpha^2 (d_i - mu)^2 + beta^2 (d_j - mu)^2); for a unit vector e_i it is |d_i - mu|.
    The columns sit in a block whose leading dimension exceeds n, with NaN in the padding rows: a
    stride slip reads them; a dropped square root, a wrong sign or a wrong index changes the value."""
    n, ld = 7, 11
    d = np.array([0.5, -1.25, 2.0, 3.75, -0.125, 1.5, 4.0])
    H = oracle.csr_diagonal(d)
    cols = [(2, 1.0, None, 0.0, 0.75), (0, 1.0, None, 0.0, -2.0), (4, 0.6, 6, 0.8, 1.0), (1, 3.0, 5, -4.0, 0.0)]
    V = np.full((ld, len(cols)), np.nan)
    V[:n] = 0.0
    lam, want = [], []
    for c, (i, a, j, b, mu) in enumerate(cols):
        V[i, c] = a
        if j is not None:
            V[j, c] = b
        lam.append(mu)
        want.append(math.hypot(a * (d[i] - mu), 0.0 if j is None else b * (d[j] - mu)))
    r = _residuals_ld(H, lam, V, ld)
    assert np.all(np.isfinite(r))
    assert np.allclose(r, want, rtol=4e-16, atol=0)
    assert r[0] == abs(d[2] - 0.75) and r[1] == abs(d[0] + 2.0)  # unit vectors: exact
    # the Python wrapper (leading dimension n) on the same columns
    assert np.allclose(oracle.residuals(H, lam, V[:n]), want, rtol=4e-16, atol=0)


def test_residuals_of_exact_eigenpairs(small_glass):
    """Exact eigenpairs of the glass Hessian (LAPACK) have residual at rounding level, and a shifted
    eigenvalue lambda + delta gives exactly |delta| (||v|| = 1, H v = lambda v)."""
    _, H, Hd = small_glass
    w, U = np.linalg.eigh(Hd)
    sel = [0, 5, 100, U.shape[1] - 1]
    nrm = np.abs(w).max()
    r = oracle.residuals(H, w[sel], U[:, sel])
    assert np.all(r <= 1e-13 * nrm)
    delta = np.array([1e-3, -2e-2, 0.5, -1.0]) * nrm
    r2 = oracle.residuals(H, w[sel] + delta, U[:, sel])
    assert np.allclose(r2, np.abs(delta), rtol=1e-10, atol=1e-13 * nrm)


def test_hessian_invariants(small_glass):
    g, H, A = small_glass
    assert np.array_equal(A, A.T)  # bitwise symmetric
    nrm = np.linalg.norm(A, 2)
    for ax in range(3):  # three translation modes sqrt(m_i) e_x (eq. (2))
        v = np.zeros((g.n_atoms, 3))
        v[:, ax] = np.sqrt(g.mass)
        v = v.ravel()
        assert np.linalg.norm(A @ v) <= 1e-14 * nrm * np.linalg.norm(v)
    w = np.linalg.eigvalsh(A)
    assert np.trace(A) == pytest.approx(w.sum(), rel=1e-12)
    assert w[0] > -1e-13 * nrm  # positive semidefinite
    # the quadratic form of eq. (1): q^T Delta q = sum_bonds k (r.(q_i - q_j))^2, Delta = M^1/2 H M^1/2
    q = np.random.default_rng(3).standard_normal((g.n_atoms, 3))
    sm = np.repeat(np.sqrt(g.mass), 3)
    quad = (q.ravel() * sm) @ A @ (q.ravel() * sm)
    dq = q[g.bi] - q[g.bj]
    ref = np.sum(g.k * np.einsum("ij,ij->i", g.rhat, dq) ** 2)
    assert quad == pytest.approx(ref, rel=1e-12)


def test_hellmann_feynman(small_glass):
    """d lambda / d k_e = ((v_i.r)/sqrt(m_i) - (v_j.r)/sqrt(m_j))^2 for a simple eigenpair (eq. (2))."""
    g, H, A = small_glass
    w, V = np.linalg.eigh(A)
    idx = int(np.argmin(np.abs(w - 0.3 * w[-1])))
    assert min(w[idx + 1] - w[idx], w[idx] - w[idx - 1]) > 1e-6
    v = V[:, idx].reshape(-1, 3)
    rng = np.random.default_rng(4)
    for e in rng.choice(g.n_bonds, 5, replace=False):
        i, j, r = g.bi[e], g.bj[e], g.rhat[e]
        hf = (v[i] @ r / math.sqrt(g.mass[i]) - v[j] @ r / math.sqrt(g.mass[j])) ** 2
        h = 1e-6 * g.k[e]
        vals = []
        for s in (+1, -1):
            g2 = glassgen.Glass(**{**g.__dict__, "k": g.k.copy()})
            g2.k[e] += s * h
            vals.append(np.linalg.eigvalsh(oracle.csr_from_springs(g2).dense())[idx])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert fd == pytest.approx(hf, rel=1e-5, abs=1e-10)


# ------------------------------------------------------------------ dense building blocks vs LAPACK
def test_jacobi_vs_lapack():
    rng = np.random.default_rng(5)
    B = rng.standard_normal((40, 40))
    A = B + B.T
    w, V = oracle.jacobi_eig(A)
    assert np.allclose(w, np.linalg.eigvalsh(A), atol=1e-12)
    assert np.allclose(A @ V, V * w, atol=1e-11)
    assert np.allclose(V.T @ V, np.eye(40), atol=1e-13)


def test_householder_qr_vs_lapack():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((300, 17))
    Q, R = oracle.householder_qr(X)
    assert np.allclose(Q.T @ Q, np.eye(17), atol=1e-14)
    assert np.allclose(Q @ R, X, atol=1e-13)
    assert np.allclose(np.tril(R, -1), 0.0)
    _, Rl = np.linalg.qr(X)
    assert np.allclose(np.abs(R), np.abs(Rl), atol=1e-12)


def test_sturm_counts_vs_lapack(small_glass):
    g, H, A = small_glass
    w = np.linalg.eigvalsh(A)
    d, e = oracle.tridiagonalize(A)
    assert np.allclose(np.linalg.eigvalsh(np.diag(d) + np.diag(e, 1) + np.diag(e, -1)), w, atol=1e-13)
    for s in np.linspace(-0.01, w[-1] * 1.1, 23):
        if np.min(np.abs(w - s)) < 1e-9:
            continue
        assert oracle.count_below(d, e, s) == int(np.sum(w < s))


def test_lanczos_upper_bound(small_glass):
    g, H, A = small_glass
    lmax = np.linalg.eigvalsh(A)[-1]
    for seed in range(4):
        th, rb, est = oracle.lanczos_lmax(H, 30, seed)
        assert th <= lmax * (1 + 1e-12)
        assert est >= lmax
        # the Ritz pair's residual norm |beta_s s_s| bounds its distance to the spectrum (Krylov-Weinstein)
        assert abs(lmax - th) <= rb + 1e-12 * lmax
        # 30 steps with full reorthogonalisation on n = 180 converge the top Ritz value; the bound is
        # not looser than its 1 % margin plus that residual
        assert th == pytest.approx(lmax, rel=1e-10)
        assert est <= 1.01 * lmax + rb + 1e-12 * lmax


def test_count_estimator_expectation(small_glass):
    """E[v^T psi(Ht) v] = trace(psi(Ht)) / n for normalised Gaussian v (Sec. 2.4)."""
    g, H, A = small_glass
    w = np.linalg.eigvalsh(A)
    lmax = 1.01 * w[-1]
    c = d = lmax / 2
    a, b = 0.2 * lmax, 0.4 * lmax
    xi, eta = (a - c) / d, (b - c) / d
    coef = oracle.chi_coeffs(xi, eta, 100)
    trace = sum(oracle.series_value(coef, (x - c) / d) for x in w)
    ests = [oracle.count_estimate(H, c, d, xi, eta, 100, "none", 30, s) for s in range(20)]
    sd = np.std(ests) / math.sqrt(len(ests))
    assert abs(np.mean(ests) - trace) < 5 * sd + 1e-9
    assert abs(np.mean(ests) - np.sum((w >= a) & (w <= b))) < 0.25 * np.sum((w >= a) & (w <= b)) + 5 * sd


# ------------------------------------------------------------------ the solver
def test_si_solve_matches_lapack():
    """Filtered SI + Rayleigh-Ritz + locking against the exact interval eigenpairs."""
    g = glassgen.generate(150, 2)
    H = oracle.csr_from_springs(g)
    A = H.dense()
    w, V = np.linalg.eigh(A)
    th, rb, lmax = oracle.lanczos_lmax(H, 30, 0)
    a, b = 0.02 * lmax, 0.05 * lmax
    sel = (w >= a) & (w <= b)
    c = d = lmax / 2
    xi, eta = (a - c) / d, (b - c) / d
    eps = 0.25 * (eta - xi)
    m = oracle.select_degree(xi, eta, eps, 0.1 ** 0.5, "jackson")
    coef = oracle.filter_coeffs(xi, eta, eps, m, "jackson")
    nwin = int(np.sum((w >= c + d * (xi - eps)) & (w <= c + d * (eta + eps))))
    q = nwin + 6
    X0 = oracle.normal_block(0, 0, H.n, q)
    r = oracle.si_solve(H, a, b, 0.0, lmax, coef, q, X0, tol=1e-10, max_iter=60)
    assert r.status == 0
    assert r.lam.size == int(sel.sum())
    assert np.allclose(r.lam, w[sel], rtol=1e-10, atol=0)
    assert np.all(oracle.residuals(H, r.lam, r.vecs) / lmax <= 1e-10)
    # principal angles between the computed and exact interval subspaces
    s = np.linalg.svd(V[:, sel].T @ r.vecs, compute_uv=False)
    assert np.min(s) > 1 - 1e-12


def test_alg4_table1_schedule(golden):
    """Alg. 4 as printed converges at step 7 (r = 0.1) and 13 (r = sqrt 0.1) on test case 1."""
    g = golden("si_schedule_table1.json")
    n = g["n"]
    lam = -1 + (2 * np.arange(1, n + 1) - 1) / n
    X0 = oracle.normal_block(0, 3, n, g["q"])
    for case in (g["cases"][0], g["cases"][3]):
        coef = oracle.filter_coeffs(g["xi"], g["eta"], g["eps"], case["degree"], case["damping"])
        pd = np.array([oracle.series_value(coef, x) for x in lam])
        k = oracle.si_alg4_diag(pd, g["q"], g["p"], g["n_rr"], g["tau"], X0, 40)
        assert k == case["steps"]
        assert k * g["q"] * case["degree"] == case["matvecs"]


# ------------------------------------------------------------------ the adjoint
def test_adjoint_symmetry_and_fd(small_glass):
    g, H, A = small_glass
    lmax = 1.01 * np.linalg.eigvalsh(A)[-1]
    c = d = lmax / 2
    coef = oracle.filter_coeffs(-0.9, -0.8, 0.03, 25, "jackson")
    rng = np.random.default_rng(8)
    X = rng.standard_normal((H.n, 2))
    Yb = rng.standard_normal((H.n, 2))
    Xb, vb = oracle.filter_adjoint(H, c, d, coef, X, Yb)
    assert np.allclose(Xb, oracle.cheb_filter(H, c, d, coef, Yb), atol=1e-12 * np.abs(Xb).max())
    rp, ci, v = H.arrays()

    def loss(vals):
        Hp = oracle.csr_from_arrays(rp, ci, vals)
        return float(np.sum(Yb * oracle.cheb_filter(Hp, c, d, coef, X)))

    for p in rng.choice(H.nnz, 12, replace=False):
        h = 1e-6 * max(abs(v[p]), 1e-3)
        vp, vm = v.copy(), v.copy()
        vp[p] += h
        vm[p] -= h
        fd = (loss(vp) - loss(vm)) / (2 * h)
        assert fd == pytest.approx(vb[p], rel=1e-5, abs=1e-7 * np.abs(vb).max())


def test_adjoint_daleckii_krein(small_glass):
    """The reverse sweep against the Daleckii-Krein formula for the derivative of a matrix function:
    with Ht = Q diag(l) Q^T, d p(Ht)[E] = Q (F o (Q^T E Q)) Q^T, F_ij the divided difference of p at
    l_i, l_j (p'(l_i) on coinciding values), so dL/dHt for L = <Ybar, p(Ht) X> is
    Q (F o (Q^T Ybar X^T Q)) Q^T, and dL/dH = that / d.  Every stored entry is compared."""
    g, H, A = small_glass
    lmax = 1.01 * np.linalg.eigvalsh(A)[-1]
    c = d = lmax / 2
    coef = oracle.filter_coeffs(-0.9, -0.8, 0.03, 30, "jackson")
    rng = np.random.default_rng(12)
    X = rng.standard_normal((H.n, 3))
    Yb = rng.standard_normal((H.n, 3))
    _, vb = oracle.filter_adjoint(H, c, d, coef, X, Yb)
    lam, Q = np.linalg.eigh((A - c * np.eye(H.n)) / d)
    p = np.polynomial.chebyshev.chebval(lam, coef)
    dp = np.polynomial.chebyshev.chebval(lam, np.polynomial.chebyshev.chebder(coef))
    gap = lam[:, None] - lam[None, :]
    close = np.abs(gap) < 1e-7
    F = np.where(close, 0.5 * (dp[:, None] + dp[None, :]), (p[:, None] - p[None, :]) / np.where(close, 1.0, gap))
    G = Q @ (F * (Q.T @ Yb @ X.T @ Q)) @ Q.T / d
    rp, ci, _ = H.arrays()
    rows = np.repeat(np.arange(H.n), np.diff(rp))
    want = G[rows, ci]
    assert np.abs(vb - want).max() <= 1e-9 * np.abs(want).max()


def test_chain_springs_fd(small_glass):
    g, H, A = small_glass
    lmax = 1.01 * np.linalg.eigvalsh(A)[-1]
    c = d = lmax / 2
    coef = oracle.filter_coeffs(-0.9, -0.8, 0.03, 20, "jackson")
    rng = np.random.default_rng(9)
    X = rng.standard_normal((H.n, 2))
    Yb = rng.standard_normal((H.n, 2))
    _, vb = oracle.filter_adjoint(H, c, d, coef, X, Yb)
    kb, mb = oracle.chain_springs(H, g, vb)

    def loss(gl):
        return float(np.sum(Yb * oracle.cheb_filter(oracle.csr_from_springs(gl), c, d, coef, X)))

    for e in rng.choice(g.n_bonds, 6, replace=False):
        h = 1e-6 * g.k[e]
        gp = glassgen.Glass(**{**g.__dict__, "k": g.k.copy()})
        gm = glassgen.Glass(**{**g.__dict__, "k": g.k.copy()})
        gp.k[e] += h
        gm.k[e] -= h
        assert (loss(gp) - loss(gm)) / (2 * h) == pytest.approx(kb[e], rel=1e-5, abs=1e-7 * np.abs(kb).max())
    for i in rng.choice(g.n_atoms, 4, replace=False):
        h = 1e-6 * g.mass[i]
        gp = glassgen.Glass(**{**g.__dict__, "mass": g.mass.copy()})
        gm = glassgen.Glass(**{**g.__dict__, "mass": g.mass.copy()})
        gp.mass[i] += h
        gm.mass[i] -= h
        assert (loss(gp) - loss(gm)) / (2 * h) == pytest.approx(mb[i], rel=1e-5, abs=1e-7 * np.abs(mb).max())


def test_block_lanczos_matches_lapack_with_fewer_matvecs():
    """Thick-restart block Lanczos on p(Ht) + Rayleigh-Ritz with H (Sec. 2.5): the exact interval
    eigenpairs, with fewer single-vector products than the subspace iteration on the same filter
    (the relation Tables 1-3 report for block Krylov-Schur against subspace iteration)."""
    g = glassgen.generate(300, 5)
    H = oracle.csr_from_springs(g)
    th, rb, lmax = oracle.lanczos_lmax(H, 30, 0)
    w = np.linalg.eigvalsh(H.dense())
    a, b = 0.05 * lmax, 0.12 * lmax
    c = d = lmax / 2
    xi, eta = (a - c) / d, (b - c) / d
    eps = 0.25 * (eta - xi)
    r = 0.1 ** 0.5
    m = oracle.select_degree(xi, eta, eps, r, "none")
    coef = oracle.filter_coeffs(xi, eta, eps, m, "none")
    tau = min(oracle.series_value(coef, xi), oracle.series_value(coef, eta))
    bks = oracle.bks_solve(H, a, b, 0.0, lmax, coef, 16, 368, 150, oracle.normal_block(0, 0, H.n, 16),
                           math.sqrt(r) * tau, tol=1e-8, max_restarts=30)
    sel = (w >= a) & (w <= b)
    assert bks.status == 0 and bks.lam.size == int(sel.sum())
    assert np.allclose(bks.lam, w[sel], rtol=1e-10, atol=0)
    assert np.all(oracle.residuals(H, bks.lam, bks.vecs) / lmax <= 1e-8)
    si = oracle.si_solve(H, a, b, 0.0, lmax, coef, 203, oracle.normal_block(0, 0, H.n, 203), tol=1e-8, max_iter=60)
    assert si.status == 0 and si.lam.size == bks.lam.size
    assert bks.matvecs < si.matvecs


def _lattice_plane_wave(L, kint, zeta, phase="sin"):
    """Atoms on the integer points of a periodic L^3 cube; q_i = sqrt(2/N) zeta sin(k . r_i) with the
    allowed k = 2 pi kint / L (Sec. 4.4)."""
    g = np.stack(np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij"), -1).reshape(-1, 3).astype(float)
    N = g.shape[0]
    k = 2 * np.pi * np.asarray(kint, float) / L
    f = np.sin(g @ k) if phase == "sin" else np.cos(g @ k)
    q = np.sqrt(2.0 / N) * f[:, None] * np.asarray(zeta, float)[None, :]
    return g, k, q.reshape(-1)


def test_participation_ratio_closed_forms():
    """Sec. 4.4: PR = 1 for |q_i| = 1/sqrt(N), 1/N for a single atom, 2/3 for a plane wave; a
    translation mode sqrt(m_i) e_x of the glass gives (sum m)^2 / (N sum m^2)."""
    N = 125
    uni = np.zeros((3 * N, 2))
    uni[0::3, 0] = 1 / np.sqrt(N)
    uni[:, 1] = np.random.default_rng(0).choice([-1.0, 1.0], 3 * N) / np.sqrt(3 * N)  # |q_i| = 1/sqrt(N) too
    one = np.zeros((3 * N, 1))
    one[3 * 17 + 1, 0] = 1.0
    _, _, pw = _lattice_plane_wave(5, (1, 0, 0), (0, 0, 1))
    pr = oracle.participation_ratio(np.column_stack([uni, one, pw, 3.0 * pw]))
    assert np.allclose(pr, [1.0, 1.0, 1.0 / N, 2.0 / 3.0, 2.0 / 3.0], rtol=1e-14, atol=0)
    g = glassgen.generate(200, 3)
    t = np.zeros(3 * g.n_atoms)
    t[0::3] = np.sqrt(g.mass)
    assert np.isclose(oracle.participation_ratio(t[:, None])[0],
                      g.mass.sum() ** 2 / (g.n_atoms * (g.mass ** 2).sum()), rtol=1e-14)


def test_plane_wave_content_closed_forms():
    """A lattice plane wave of an allowed k is 1 in its own polarisation and wave vector, 0 in the
    other polarisation and in other allowed wave vectors (orthogonality of the lattice sums)."""
    L = 5
    pos, k, qt = _lattice_plane_wave(L, (1, 2, 0), (0, 0, 1))             # transverse (zeta _|_ k)
    _, _, ql = _lattice_plane_wave(L, (1, 2, 0), np.array([1, 2, 0]) / np.sqrt(5), "cos")  # longitudinal
    ks = 2 * np.pi / L * np.array([[1, 2, 0], [-1, -2, 0], [2, 1, 0], [0, 0, 1]], float)
    out = oracle.plane_wave_content(np.column_stack([qt, ql]), pos, ks)
    assert np.allclose(out[0, 0], [0.0, 1.0], atol=1e-13) and np.allclose(out[1, 0], [1.0, 0.0], atol=1e-13)
    assert np.allclose(out[:, 1], out[:, 0], atol=1e-13)  # -k is the same plane wave
    assert np.allclose(out[:, 2:], 0.0, atol=1e-13)
    # content is a sum of squared projections onto orthonormal functions: at most 1 in total
    q = np.random.default_rng(3).standard_normal(3 * L ** 3)
    kall = 2 * np.pi / L * np.array([[a, b, c] for a in range(3) for b in range(-2, 3) for c in range(-2, 3)
                                     if (a, b, c) > (0, 0, 0)], float)
    tot = oracle.plane_wave_content(q[:, None], pos, kall).sum()
    assert tot <= 1.0 + 1e-12


def test_dirac_filter_degrees_tables_1_3(golden):
    """All 18 Dirac-filter degrees printed in Tables 1-3 (phi = 0.8, 0.6; Jackson, Lanczos, none):
    the smallest degree whose filter, centred so that rho(xi) = rho(eta), has rho(xi) / rho(gamma) <= phi."""
    fx = golden("dirac_degrees_tables_1_3.json")
    for case in fx["cases"]:
        for i, phi in enumerate(fx["rows_phi"]):
            for j, kind in enumerate(fx["columns"]):
                assert oracle.dirac_degree(case["xi"], case["eta"], phi, kind) == case["degrees"][i][j], \
                    (case["table"], phi, kind)


def test_dirac_filter_is_the_delta_projection():
    """rho_k = sum_j T_j(gamma) T_j / <T_j, T_j>: undamped, its integral against any polynomial f of
    degree <= k with the Chebyshev weight returns f(gamma) (the defining property of delta); the
    balanced centre gives equal edge values."""
    gm, k = -0.37, 12
    c = oracle.dirac_coeffs(gm, k, "none")
    x, w = np.polynomial.chebyshev.chebgauss(64)  # exact for degree <= 127 with weight 1/sqrt(1-x^2)
    for deg in (0, 3, 7, 12):
        f = np.polynomial.chebyshev.Chebyshev.basis(deg) + 0.5 * np.polynomial.chebyshev.Chebyshev.basis(max(deg - 2, 0))
        integral = np.sum(w * f(x) * np.polynomial.chebyshev.chebval(x, c))
        assert abs(integral - f(gm)) <= 1e-12
    xi, eta = -0.9, -0.885
    g = oracle.dirac_gamma(xi, eta, 128, "jackson")
    c = oracle.dirac_coeffs(g, 128, "jackson")
    assert xi < g < eta
    assert abs(oracle.series_value(c, xi) - oracle.series_value(c, eta)) <= 1e-12 * oracle.series_value(c, g)


def test_block_lanczos_with_the_dirac_filter():
    """The paper's production pairing (Sec. 4.1, Tables 1-3): block Lanczos on the Dirac filter rho (phi = 0.8,
    Jackson), wanted Ritz values >= 0.9 rho(xi), then Rayleigh-Ritz with H: the exact interval eigenpairs."""
    g = glassgen.generate(300, 5)
    H = oracle.csr_from_springs(g)
    th, rb, lmax = oracle.lanczos_lmax(H, 30, 0)
    w = np.linalg.eigvalsh(H.dense())
    a, b = 0.05 * lmax, 0.12 * lmax
    c = d = lmax / 2
    xi, eta = (a - c) / d, (b - c) / d
    m = oracle.dirac_degree(xi, eta, 0.8, "jackson")
    gm = oracle.dirac_gamma(xi, eta, m, "jackson")
    coef = oracle.dirac_coeffs(gm, m, "jackson")
    tau = oracle.series_value(coef, xi)
    bks = oracle.bks_solve(H, a, b, 0.0, lmax, coef, 16, 368, 150, oracle.normal_block(0, 0, H.n, 16), 0.9 * tau,
                           tol=1e-8, max_restarts=30)
    sel = (w >= a) & (w <= b)
    assert bks.status == 0 and bks.lam.size == int(sel.sum())
    assert np.allclose(bks.lam, w[sel], rtol=1e-10, atol=0)
    assert np.all(oracle.residuals(H, bks.lam, bks.vecs) / lmax <= 1e-8)
