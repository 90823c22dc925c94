"""Edge cases of the filtered subspace iteration on the GPU, through the C ABI, against the oracle
and closed forms: an interval without eigenvalues, the zero (translation) modes at lambda = 0, the
top of the spectrum, exactly degenerate eigenvalues, and the synthetic diagonal problem of the
paper's Sec. 4.1 (test case 1, equally distributed eigenvalues) with known eigenpairs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import glassgen  # noqa: E402
import oracle  # noqa: E402
import paper_1902_07041_gb300 as pfe  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    pfe.load()


def _solve(rp, ci, vals, n_atoms, masses, lo, hi, absolute=False, **params):
    ctx = pfe.pfe_create(n_atoms, rp, ci, vals, masses)
    try:
        for k, v in params.items():
            pfe.pfe_set_param(ctx, getattr(pfe, "PFE_P_" + k), v)
        lmax, _ = pfe.pfe_estimate(ctx)
        a, b = (lo, hi) if absolute else (lo * lmax, hi * lmax)
        pfe.pfe_set_interval(ctx, a, b)
        nf, st = pfe.pfe_solve(ctx, raise_on_error=False)
        lam, V, res = pfe.pfe_get_eigenpairs(ctx, 3 * n_atoms, nf) if nf else (np.zeros(0), None, None)
        return st, nf, lam, V, lmax, a, b
    finally:
        pfe.pfe_destroy(ctx)


def _glass(n, seed):
    g = glassgen.generate(n, seed)
    return g, pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)


def test_interval_without_eigenvalues():
    g, (rp, ci, vals) = _glass(200, 31)
    w = np.linalg.eigvalsh(oracle.csr_from_springs(g).dense())
    gaps = np.diff(w)
    i = int(np.argmax(gaps[len(w) // 4: len(w) // 2])) + len(w) // 4  # a wide gap in the lower spectrum
    a, b = w[i] + 0.3 * gaps[i], w[i] + 0.7 * gaps[i]
    st, nf, lam, _, _, _, _ = _solve(rp, ci, vals, g.n_atoms, g.mass, a, b, absolute=True)
    assert st == pfe.PFE_OK and nf == 0


def test_zero_modes_at_the_bottom_of_the_spectrum():
    """[0, b] starts at the three translation modes sqrt(m_i) e_x (lambda = 0).  Computed in FP64 they
    sit within rounding of the edge a = 0 and may fall on either side of it (boundary-ambiguous);
    every other eigenvalue of [0, b] must be found, and whatever is found near 0 must lie in the
    translation space."""
    g, (rp, ci, vals) = _glass(150, 32)
    st, nf, lam, V, lmax, a, b = _solve(rp, ci, vals, g.n_atoms, g.mass, 0.0, 0.04)
    H = oracle.csr_from_springs(g)
    w, _, _ = oracle.exact_interval(H, 1e-9 * lmax, b)
    assert st == pfe.PFE_OK
    nz = lam > 1e-9 * lmax
    assert int(nz.sum()) == w.size and nf - int(nz.sum()) <= 3
    assert np.allclose(lam[nz], w, rtol=1e-10, atol=0)
    T = np.zeros((H.n, 3))
    for ax in range(3):
        T[ax::3, ax] = np.sqrt(g.mass)
    T /= np.linalg.norm(T, axis=0)
    Z = V[:, ~nz]
    if Z.shape[1]:
        assert np.allclose(np.linalg.norm(T.T @ Z, axis=0), 1.0, atol=1e-8)  # inside the translation space


def test_top_of_the_spectrum():
    g, (rp, ci, vals) = _glass(150, 33)
    st, nf, lam, V, lmax, a, b = _solve(rp, ci, vals, g.n_atoms, g.mass, 0.85, 1.0)
    H = oracle.csr_from_springs(g)
    w, _, _ = oracle.exact_interval(H, a, b)
    assert st == pfe.PFE_OK and nf == w.size and nf > 0
    assert np.allclose(lam, w, rtol=1e-10, atol=0)


def _block_diagonal(diag_values):
    """BSR of a block-diagonal matrix with 3x3 diagonal blocks diag(d_3i, d_3i+1, d_3i+2)."""
    n = diag_values.size
    N = n // 3
    rp = np.arange(N + 1, dtype=np.int32)
    ci = np.arange(N, dtype=np.int32)
    vals = np.zeros(9 * N)
    for i in range(N):
        vals[9 * i + 0], vals[9 * i + 4], vals[9 * i + 8] = diag_values[3 * i:3 * i + 3]
    return rp, ci, vals


def test_exactly_degenerate_eigenvalues():
    """Eigenvalues of multiplicity 3 (each diagonal value repeated in a whole block): the count is
    exact and each eigenvalue's computed space is the coordinate space of its value."""
    base = np.repeat(np.linspace(0.0, 1.0, 400), 3)  # each value 3 times, blocks identical multiples
    rp, ci, vals = _block_diagonal(base)
    st, nf, lam, V, lmax, a, b = _solve(rp, ci, vals, 400, None, 0.30, 0.36, absolute=True, LAMBDA_MAX=1.01)
    sel = (base >= a) & (base <= b)
    assert st == pfe.PFE_OK and nf == int(sel.sum())
    assert np.allclose(lam, np.sort(base[sel]), rtol=0, atol=1e-12)
    # the computed subspace equals the span of the selected coordinate vectors
    assert np.allclose(np.linalg.norm(V[sel, :], axis=0), 1.0, atol=1e-10)


def test_paper_diagonal_test_case_1():
    """Sec. 4.1, test case 1: equally distributed eigenvalues lambda_i = -1 + (2i - 1)/n shifted by +1
    into [0, 2] (H must be PSD here); the 50 eigenvalues of (-0.9, -0.898) + 1, eigenvectors e_i."""
    n = 50001  # 16,667 atoms: the paper's n = 50,000 plus one eigenvalue at the top
    lam_all = -1 + (2 * np.arange(1, 50001) - 1) / 50000.0 + 1.0
    lam_all = np.append(lam_all, 2.0)
    rp, ci, vals = _block_diagonal(lam_all)
    st, nf, lam, V, lmax, a, b = _solve(rp, ci, vals, n // 3, None, 0.1, 0.102, absolute=True, LAMBDA_MAX=2.0,
                                        EPS_FRAC=0.25)
    sel = (lam_all >= a) & (lam_all <= b)
    assert int(sel.sum()) == 50
    assert st == pfe.PFE_OK and nf == 50
    assert np.allclose(lam, lam_all[sel], rtol=0, atol=1e-12)
    idx = np.nonzero(sel)[0]
    assert np.allclose(np.abs(V[idx, np.arange(50)]), 1.0, atol=1e-8)


def test_lambda_max_bound_below_the_spectrum():
    """Alg. 3 bounds the spectrum before filtering; a bound set below the true lambda_max (0.9 x the
    exact one) puts eigenvalues outside [-1, 1], where the filter amplifies them, and the solver must
    stop with PFE_E_BOUND when a Ritz value exceeds the bound instead of returning wrong pairs."""
    g, (rp, ci, vals) = _glass(300, 5)
    lmax_true = np.linalg.eigvalsh(oracle.csr_from_springs(g).dense())[-1]
    st, nf, *_ = _solve(rp, ci, vals, g.n_atoms, g.mass, 0.05 * lmax_true, 0.12 * lmax_true, absolute=True,
                        LAMBDA_MAX=0.9 * lmax_true, DEGREE=8, WIDTH=64)
    assert st == pfe.PFE_E_BOUND and nf == 0


def test_rank_deficient_filtered_block_takes_the_shifted_cholqr():
    """A filtered block that is numerically rank deficient: 87 of the 90 eigenvalues of a diagonal H
    sit on the root of the degree-1 filter p(x) = g_0 + g_1 x (the solver's own design, computed here
    by pfe_design_filter), so p(H) X has rank 3 up to rounding.  The Cholesky factor of its Gram
    matrix breaks down; the shifted retry (Fukaya et al.) must run, and the solve must return the 3
    eigenpairs of [a, b] exactly, or PFE_E_BREAKDOWN."""
    lmax, a, b = 1.01, 0.05, 0.06
    c = d = 0.5 * lmax
    xi, eta = (a - c) / d, (b - c) / d
    _, coef = pfe.pfe_design_filter("pq", xi, eta, eps=0.25 * (eta - xi), r=0.1 ** 0.5, degree=1)
    x0 = -coef[0] / coef[1]
    lam0 = c + d * x0
    assert 0.0 < lam0 < lmax and lam0 > b + 0.1  # the root lies in the spectrum, far above [a, b]
    vals_diag = np.full(90, lam0)
    vals_diag[[10, 41, 77]] = [0.052, 0.055, 0.058]
    rp, ci, vals = _block_diagonal(vals_diag)
    ctx = pfe.pfe_create(30, rp, ci, vals, None)
    try:
        for k, v in (("LAMBDA_MAX", lmax), ("DEGREE", 1), ("WIDTH", 90)):
            pfe.pfe_set_param(ctx, getattr(pfe, "PFE_P_" + k), v)
        pfe.pfe_set_interval(ctx, a, b)
        nf, st = pfe.pfe_solve(ctx, raise_on_error=False)
        stats = pfe.pfe_get_stats(ctx)
        lam, V, _ = pfe.pfe_get_eigenpairs(ctx, 90, nf) if st == pfe.PFE_OK else (None, None, None)
    finally:
        pfe.pfe_destroy(ctx)
    assert st in (pfe.PFE_OK, pfe.PFE_E_BREAKDOWN)
    if st == pfe.PFE_OK:
        assert stats["cholqr_shifts"] >= 1
        assert nf == 3 and np.allclose(lam, [0.052, 0.055, 0.058], rtol=0, atol=1e-12)
        assert np.allclose(np.abs(V[[10, 41, 77], np.arange(3)]), 1.0, atol=1e-8)


def test_subspace_narrower_than_the_interval_count():
    """Width 8 against 20 copies of one eigenvalue in [a, b]: the 8 columns converge inside the
    degenerate eigenspace, fill the subspace, and the solver reports PFE_E_CAPACITY (raise the width)
    with the 8 pairs it found."""
    d = np.linspace(0.0, 1.0, 90)
    d[20:40] = 0.5
    d[(d > 0.4) & (d < 0.6) & (d != 0.5)] = 0.3  # nothing else in the margin window
    rp, ci, vals = _block_diagonal(d)
    st, nf, lam, V, *_ = _solve(rp, ci, vals, 30, None, 0.45, 0.55, absolute=True, LAMBDA_MAX=1.01, WIDTH=8)
    assert st == pfe.PFE_E_CAPACITY and nf == 8
    assert np.allclose(lam, 0.5, rtol=0, atol=1e-12)
    assert np.allclose(np.linalg.norm(V[20:40], axis=0), 1.0, atol=1e-8)


def _cross_pairs_within_residual_bound(lam, V, r):
    """For symmetric H, two approximate eigenpairs (l_i, v_i), (l_j, v_j) with residual norms r_i, r_j
    satisfy (l_j - l_i) v_i^T v_j = v_i^T (H v_j - l_j v_j) - (H v_i - l_i v_i)^T v_j, hence
    |v_i^T v_j| <= (r_i + r_j) / |l_i - l_j| (plus rounding of the dot product)."""
    G = np.abs(V.T @ V - np.eye(lam.size))
    gap = np.abs(lam[:, None] - lam[None, :])
    np.fill_diagonal(gap, np.inf)
    bound = (r[:, None] + r[None, :]) / gap + 1e-13
    np.fill_diagonal(bound, 1e-12)
    return bool(np.all(G <= bound))


@pytest.mark.parametrize("table,xi,eta", [(1, -0.9, -0.898), (2, -0.9, -0.896), (3, -0.9, -0.885)])
def test_library_dirac_degrees_match_tables(golden, table, xi, eta):
    """The library's own Dirac-filter degree selection reproduces the degrees printed in Tables 1-3
    (transformed interval [xi, eta] with lambda in [0, 2]: a = 1 + xi, b = 1 + eta)."""
    fx = golden("dirac_degrees_tables_1_3.json")
    case = [c for c in fx["cases"] if c["table"] == table][0]
    rp, ci, vals = _block_diagonal(np.linspace(0.0, 2.0, 300))
    ctx = pfe.pfe_create(100, rp, ci, vals, None)
    try:
        pfe.pfe_set_param(ctx, pfe.PFE_P_LAMBDA_MAX, 2.0)
        pfe.pfe_set_param(ctx, pfe.PFE_P_FILTER, 1)
        for i, phi in enumerate(fx["rows_phi"]):
            for j, kind in enumerate(fx["columns"]):
                pfe.pfe_set_param(ctx, pfe.PFE_P_PHI, phi)
                pfe.pfe_set_param(ctx, pfe.PFE_P_DAMPING, {"none": 0, "jackson": 1, "lanczos": 2}[kind])
                pfe.pfe_set_interval(ctx, 1.0 + xi, 1.0 + eta)
                m, coef, c, d = pfe.pfe_get_filter(ctx)
                assert m == case["degrees"][i][j], (table, phi, kind, m)
                g = oracle.dirac_gamma(xi, eta, m, kind)
                assert np.allclose(coef, oracle.dirac_coeffs(g, m, kind), rtol=1e-9, atol=1e-12 * np.abs(coef).max())
    finally:
        pfe.pfe_destroy(ctx)


def test_block_lanczos_dirac_filter_paper_test_case_1():
    """Sec. 4.1 test case 1 with the paper's production solver: block Lanczos on the Dirac filter
    (phi = 0.8, Jackson smoothing), the 50 eigenvalues of [0.1, 0.102] and their coordinate vectors."""
    lam_all = -1 + (2 * np.arange(1, 50001) - 1) / 50000.0 + 1.0
    lam_all = np.append(lam_all, 2.0)
    rp, ci, vals = _block_diagonal(lam_all)
    st, nf, lam, V, lmax, a, b = _solve(rp, ci, vals, 50001 // 3, None, 0.1, 0.102, absolute=True, LAMBDA_MAX=2.0,
                                        METHOD=1, FILTER=1, DAMPING=1, BLOCK=16)
    sel = (lam_all >= a) & (lam_all <= b)
    assert st == pfe.PFE_OK and nf == 50
    assert np.allclose(lam, lam_all[sel], rtol=0, atol=1e-12)
    idx = np.nonzero(sel)[0]
    assert np.allclose(np.abs(V[idx, np.arange(50)]), 1.0, atol=1e-8)


def test_block_lanczos_dirac_filter_glass():
    g, (rp, ci, vals) = _glass(300, 5)
    st, nf, lam, V, lmax, a, b = _solve(rp, ci, vals, g.n_atoms, g.mass, 0.05, 0.12, METHOD=1, FILTER=1, DAMPING=1,
                                        BLOCK=32)
    H = oracle.csr_from_springs(g)
    w, _, _ = oracle.exact_interval(H, a, b)
    assert st == pfe.PFE_OK and nf == w.size
    assert np.allclose(lam, w, rtol=1e-10, atol=0)
    assert np.all(oracle.residuals(H, lam, V) <= 1e-8 * lmax)


def test_subspace_iteration_refuses_the_dirac_filter():
    g, (rp, ci, vals) = _glass(100, 5)
    st, nf, *_ = _solve(rp, ci, vals, g.n_atoms, g.mass, 0.05, 0.12, FILTER=1)
    assert st == pfe.PFE_E_ARG and nf == 0


@pytest.mark.parametrize("method", [0, 1])
def test_spectrum_slicing_matches_exact(method):
    """pfe_solve_sliced with automatic, count-guided edges (about 40 eigenvalues a slice): the union is
    every eigenpair of [a, b] exactly once."""
    g, (rp, ci, vals) = _glass(1000, 0)
    ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
    try:
        pfe.pfe_set_param(ctx, pfe.PFE_P_METHOD, method)
        pfe.pfe_set_param(ctx, pfe.PFE_P_BLOCK, 16)
        pfe.pfe_set_param(ctx, pfe.PFE_P_SLICE_TARGET, 40)
        lmax, _ = pfe.pfe_estimate(ctx)
        a, b = 0.02 * lmax, 0.05 * lmax
        pfe.pfe_set_interval(ctx, a, b)
        nf, st = pfe.pfe_solve_sliced(ctx)
        stats = pfe.pfe_get_stats(ctx)
        lam, V, res = pfe.pfe_get_eigenpairs(ctx, g.n, nf)
    finally:
        pfe.pfe_destroy(ctx)
    H = oracle.csr_from_springs(g)
    w, _, _ = oracle.exact_interval(H, a, b)
    assert st == pfe.PFE_OK and stats["slices"] >= 3
    assert nf == w.size and np.allclose(lam, w, rtol=1e-10, atol=0)
    r = oracle.residuals(H, lam, V)
    assert np.all(r <= 1e-8 * lmax)
    # vectors of different slices are orthogonal to the accuracy their residuals and gaps allow
    assert _cross_pairs_within_residual_bound(lam, V, r)


def test_spectrum_slicing_edges_on_eigenvalues():
    """Explicit edges placed exactly on a simple and on a double eigenvalue: both neighbouring slices
    find those pairs, and the merge keeps each eigenpair once (the double one as a 2-dimensional
    space)."""
    d = np.linspace(0.01, 1.0, 600)
    d[300] = d[301] = 0.5  # a double eigenvalue
    simple = d[250]
    rp, ci, vals = _block_diagonal(np.concatenate([d, [1.0, 1.0, 1.0]]))
    N = (d.size + 3) // 3
    ctx = pfe.pfe_create(N, rp, ci, vals, None)
    try:
        pfe.pfe_set_param(ctx, pfe.PFE_P_LAMBDA_MAX, 1.01)
        a, b = 0.38, 0.62
        pfe.pfe_set_interval(ctx, a, b)
        nf, st = pfe.pfe_solve_sliced(ctx, [simple, 0.5])
        lam, V, res = pfe.pfe_get_eigenpairs(ctx, 3 * N, nf)
        stats = pfe.pfe_get_stats(ctx)
    finally:
        pfe.pfe_destroy(ctx)
    full = np.concatenate([d, [1.0, 1.0, 1.0]])
    sel = np.sort(full[(full >= a) & (full <= b)])
    assert st == pfe.PFE_OK and stats["slices"] == 3
    assert nf == sel.size and np.allclose(lam, sel, rtol=0, atol=1e-12)
    # vectors from different slices: orthogonal to (r_i + r_j) / gap
    r = np.linalg.norm(full[:, None] * V - V * lam, axis=0)  # H is diagonal: H v = full * v
    assert _cross_pairs_within_residual_bound(lam, V, r)
    # the double eigenvalue's two vectors span the coordinates 300 and 301
    j = np.nonzero(np.abs(lam - 0.5) < 1e-9)[0]
    assert j.size == 2 and np.allclose(np.linalg.norm(V[[300, 301]][:, j], axis=0), 1.0, atol=1e-8)
