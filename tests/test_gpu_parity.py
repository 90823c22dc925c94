"""GPU parity: the CUDA path, called through the C ABI, against the FP64 CPU oracle on the same
seeded inputs.

Tolerances (derived from the arithmetic):
  FP64 filter, degree m: each step adds O(u * nnz_row) relative rounding to bounded Chebyshev
    vectors (|T_j(Ht)| <= 1), so |Y_gpu - Y_oracle| <= 1e-11 * max|X| * sum|g_j| for m <= 100.
  FP32 filter: the same bound with u_32 = 6e-8: 2e-4 * max|X| * sum|g_j|.
  Eigenpairs: eigenvalue relative error <= 1e-10, residual ||Hv - lambda v|| <= 1e-8 lambda_max,
    counts exact (Sturm/LDL^T inertia and LAPACK), and for each cluster of nearly equal eigenvalues
    the largest principal angle within the Davis-Kahan bound ||R||_F / gap.
"""
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


def make_ctx(g, **params):
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
    for k, v in params.items():
        pfe.pfe_set_param(ctx, getattr(pfe, "PFE_P_" + k), v)
    return ctx, (rp, ci, vals)


def dev_colmajor(X, dtype=torch.float64):
    """numpy (n, k) -> device storage of a column-major n x k matrix (ld = n)."""
    return torch.from_numpy(np.ascontiguousarray(X.T)).to(device="cuda", dtype=dtype)


def filter_gpu(ctx, coef, X, dtype=pfe.PFE_F64):
    n, k = X.shape
    tdt = torch.float64 if dtype == pfe.PFE_F64 else torch.float32
    Xd = dev_colmajor(X, tdt)
    Yd = torch.full((k, n), float("nan"), device="cuda", dtype=tdt)
    pfe.pfe_filter_apply(ctx, len(coef) - 1, coef, k, Xd, n, Yd, n, dtype)
    torch.cuda.synchronize()
    return Yd.double().cpu().numpy().T


def cluster_angles_ok(H, lam, V, w_all, U_sel, w_sel, lmax):
    """Davis-Kahan: for each cluster of nearly equal eigenvalues, the sine of the largest principal
    angle between computed and exact eigenvectors is at most ||H V - V Lambda||_F / gap, gap being
    the distance from the cluster to the rest of the spectrum."""
    i = 0
    while i < lam.size:
        j = i + 1
        while j < lam.size and w_sel[j] - w_sel[j - 1] < 1e-6 * lmax:
            j += 1
        others = np.concatenate([w_all[w_all < w_sel[i] - 1e-6 * lmax], w_all[w_all > w_sel[j - 1] + 1e-6 * lmax]])
        gap = np.min(np.minimum(np.abs(others - w_sel[i]), np.abs(others - w_sel[j - 1])))
        R = H.matmul(V[:, i:j]) - V[:, i:j] * lam[i:j]
        # sine of the largest principal angle as ||(I - U U^T) V||_2, accurate to rounding (the
        # form sqrt(1 - cos^2) cannot resolve angles below ~1e-8)
        Uc, Vc = U_sel[:, i:j], V[:, i:j]
        sin_t = np.linalg.norm(Vc - Uc @ (Uc.T @ Vc), 2)
        if sin_t > 2.0 * np.linalg.norm(R) / gap + 1e-12:
            return False
        i = j
    return True


# ------------------------------------------------------------------ a0 + a4: the filter
@pytest.mark.parametrize("N,seed,k,m", [(300, 5, 5, 17), (300, 5, 37, 40), (411, 7, 100, 23), (1000, 0, 48, 40)])
def test_filter_fp64_parity(N, seed, k, m):
    g = glassgen.generate(N, seed)
    ctx, _ = make_ctx(g, LAMBDA_MAX=0.0)
    try:
        lmax, _ = pfe.pfe_estimate(ctx)
        c = d = 0.5 * lmax
        coef = oracle.filter_coeffs(-0.96, -0.9, 0.015, m, "jackson")
        X = np.random.default_rng(seed).standard_normal((g.n, k))
        Y = filter_gpu(ctx, coef, X)
        ref = oracle.cheb_filter(oracle.csr_from_springs(g), c, d, coef, X)
        tol = 1e-11 * np.abs(X).max() * np.abs(coef).sum()
        assert np.max(np.abs(Y - ref)) <= tol
    finally:
        pfe.pfe_destroy(ctx)


@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11])
def test_filter_every_kernel_shape(shape):
    """Each kernel shape of the fused step (forced instead of autotuned), FP64 and FP32, ragged k;
    shapes 7-11 run on the rank-1 form of the spring network's operator, shape 10 (FP32) with each
    tile's neighbour rows staged in shared memory (333 atoms: a ragged last tile of 13), shape 11 at six
    resident CTAs per SM."""
    g = glassgen.generate(333, 13)
    ctx, _ = make_ctx(g, LAMBDA_MAX=0.25)
    try:
        coef = oracle.filter_coeffs(-0.95, -0.9, 0.02, 21, "none")
        ref_c = oracle.csr_from_springs(g)
        for dt, key, tol in ((pfe.PFE_F64, "STEP_SHAPE_F64", 1e-11), (pfe.PFE_F32, "STEP_SHAPE_F32", 2e-4)):
            pfe.pfe_set_param(ctx, getattr(pfe, "PFE_P_" + key), shape)
            for k in (7, 45, 133):
                X = np.random.default_rng(k).standard_normal((g.n, k))
                Y = filter_gpu(ctx, coef, X, dt)
                ref = oracle.cheb_filter(ref_c, 0.125, 0.125, coef, X)
                assert np.max(np.abs(Y - ref)) <= tol * np.abs(X).max() * np.abs(coef).sum(), (dt, k)
            pfe.pfe_set_param(ctx, getattr(pfe, "PFE_P_" + key), -1)
        assert pfe.pfe_get_param(ctx, pfe.PFE_P_RANK1) == 1  # the spring network has the rank-1 form
    finally:
        pfe.pfe_destroy(ctx)


def _bsr_to_oracle_csr(rp, ci, vals):
    """Scalar CSR (oracle) of a BSR matrix with 3x3 row-major blocks."""
    N = rp.size - 1
    rows = [[] for _ in range(3 * N)]
    for i in range(N):
        for p in range(rp[i], rp[i + 1]):
            for r in range(3):
                for c in range(3):
                    rows[3 * i + r].append((3 * ci[p] + c, vals[9 * p + 3 * r + c]))
    rpc = np.zeros(3 * N + 1, np.int32)
    cic, vc = [], []
    for r, row in enumerate(rows):
        row.sort()
        rpc[r + 1] = rpc[r] + len(row)
        cic += [c for c, _ in row]
        vc += [v for _, v in row]
    return oracle.csr_from_arrays(rpc, np.array(cic, np.int32), np.array(vc))


@pytest.mark.parametrize("rank1", [0, 1])
def test_general_blocks_use_the_full_form(rank1):
    """Off-diagonal blocks that are not -k r r^T (a symmetric perturbation of a spring network):
    the rank-1 form is refused and the filter and the solve run on the full 3x3 blocks."""
    g = glassgen.generate(120, 21)
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    rng = np.random.default_rng(5)
    H = vals.copy()
    N = g.n_atoms
    for i in range(N):  # mass weighting here; the context gets H directly (masses None)
        for p in range(rp[i], rp[i + 1]):
            H[9 * p:9 * p + 9] /= np.sqrt(g.mass[i] * g.mass[ci[p]])
    blk = {(i, int(ci[p])): p for i in range(N) for p in range(rp[i], rp[i + 1])}
    for (i, j), p in blk.items():
        if i < j:
            S = rng.standard_normal((3, 3)) * 1e-3
            S = S + S.T
            H[9 * p:9 * p + 9] += S.ravel()
            q = blk[(j, i)]
            H[9 * q:9 * q + 9] += S.T.ravel()
    ctx = pfe.pfe_create(N, rp, ci, H, None)
    try:
        pfe.pfe_set_param(ctx, pfe.PFE_P_RANK1, rank1)
        lmax, _ = pfe.pfe_estimate(ctx)
        coef = oracle.filter_coeffs(-0.95, -0.9, 0.02, 30, "none")
        X = np.random.default_rng(2).standard_normal((g.n, 9))
        Y = filter_gpu(ctx, coef, X)
        assert pfe.pfe_get_param(ctx, pfe.PFE_P_RANK1) == 0
        Hc = _bsr_to_oracle_csr(rp, ci, H)
        ref = oracle.cheb_filter(Hc, 0.5 * lmax, 0.5 * lmax, coef, X)
        assert np.max(np.abs(Y - ref)) <= 1e-11 * np.abs(X).max() * np.abs(coef).sum()
        lo, hi = 0.05 * lmax, 0.12 * lmax
        pfe.pfe_set_interval(ctx, lo, hi)
        nf, _ = pfe.pfe_solve(ctx)
        lam, _, _ = pfe.pfe_get_eigenpairs(ctx, g.n, nf)
        w, _, _ = oracle.exact_interval(Hc, lo, hi)
        assert nf == w.size and np.allclose(lam, w, rtol=1e-10, atol=0)
    finally:
        pfe.pfe_destroy(ctx)


@pytest.mark.parametrize("rank1", [0, 1])
def test_solve_with_and_without_rank1_form(rank1):
    st = _solve_and_check(glassgen.generate(300, 5), 0.05, 0.12, RANK1=rank1)
    assert st["iterations"] >= 2


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_filter_low_degrees(m, dtype):
    """Degrees 1-5: the y accumulation that skips odd steps must still add every term (the last
    step adds its own term when it is odd)."""
    g = glassgen.generate(150, 3)
    ctx, _ = make_ctx(g, LAMBDA_MAX=0.3)
    try:
        coef = np.random.default_rng(m).standard_normal(m + 1)
        X = np.random.default_rng(7).standard_normal((g.n, 9))
        dt = pfe.PFE_F64 if dtype == "f64" else pfe.PFE_F32
        Y = filter_gpu(ctx, coef, X, dt)
        ref = oracle.cheb_filter(oracle.csr_from_springs(g), 0.15, 0.15, coef, X)
        tol = 1e-12 if dtype == "f64" else 1e-5
        assert np.max(np.abs(Y - ref)) <= tol * np.abs(X).max() * np.abs(coef).sum()
    finally:
        pfe.pfe_destroy(ctx)


def test_filter_first_step_is_transformed_hessian():
    """Coefficients e_1 give Ht X = (H - cI)/d X: mass weighting (a0) and the transform."""
    g = glassgen.generate(200, 9)
    ctx, _ = make_ctx(g, LAMBDA_MAX=0.3)
    try:
        X = np.random.default_rng(1).standard_normal((g.n, 7))
        Y = filter_gpu(ctx, np.array([0.0, 1.0]), X)
        H = oracle.csr_from_springs(g)
        ref = (H.matmul(X) - 0.15 * X) / 0.15
        assert np.max(np.abs(Y - ref)) <= 1e-13 * np.abs(ref).max()
    finally:
        pfe.pfe_destroy(ctx)


@pytest.mark.parametrize("k", [3, 64, 130])
def test_filter_fp32_parity(k):
    g = glassgen.generate(500, 12)
    ctx, _ = make_ctx(g)
    try:
        lmax, _ = pfe.pfe_estimate(ctx)
        coef = oracle.filter_coeffs(-0.95, -0.9, 0.02, 60, "lanczos")
        X = np.random.default_rng(k).standard_normal((g.n, k))
        Y = filter_gpu(ctx, coef, X, pfe.PFE_F32)
        ref = oracle.cheb_filter(oracle.csr_from_springs(g), 0.5 * lmax, 0.5 * lmax, coef, X)
        assert np.max(np.abs(Y - ref)) <= 2e-4 * np.abs(X).max() * np.abs(coef).sum()
    finally:
        pfe.pfe_destroy(ctx)


def test_filter_degree_zero_and_empty_block():
    g = glassgen.generate(50, 2)
    ctx, _ = make_ctx(g)
    try:
        X = np.random.default_rng(0).standard_normal((g.n, 4))
        Y = filter_gpu(ctx, np.array([2.5]), X)
        assert np.array_equal(Y, 2.5 * X)
        pfe.pfe_filter_apply(ctx, 3, np.ones(4), 0, 0, g.n, 0, g.n)  # k = 0 is a no-op
    finally:
        pfe.pfe_destroy(ctx)


# ------------------------------------------------------------------ a1, a2, a3
def test_lanczos_bound_and_filter_match_oracle():
    g = glassgen.generate(1000, 0)
    ctx, _ = make_ctx(g)
    try:
        lmax, _ = pfe.pfe_estimate(ctx)
        H = oracle.csr_from_springs(g)
        th, rb, est = oracle.lanczos_lmax(H, 30, 0)
        assert lmax == pytest.approx(est, rel=1e-9)
        assert lmax >= np.linalg.eigvalsh(H.dense())[-1]
        pfe.pfe_set_interval(ctx, 0.02 * lmax, 0.05 * lmax)
        m, coef, c, d = pfe.pfe_get_filter(ctx)
        xi, eta = (0.02 * lmax - c) / d, (0.05 * lmax - c) / d
        eps = 0.25 * (eta - xi)
        assert m == oracle.select_degree(xi, eta, eps, 0.1 ** 0.5, "none")
        assert np.allclose(coef, oracle.filter_coeffs(xi, eta, eps, m, "none"), rtol=0, atol=1e-12)
        for kind, code in (("jackson", 1), ("lanczos", 2)):
            pfe.pfe_set_param(ctx, pfe.PFE_P_DAMPING, code)
            m, coef, _, _ = pfe.pfe_get_filter(ctx)
            assert m == oracle.select_degree(xi, eta, eps, 0.1 ** 0.5, kind)
            assert np.allclose(coef, oracle.filter_coeffs(xi, eta, eps, m, kind), rtol=0, atol=1e-12)
    finally:
        pfe.pfe_destroy(ctx)


def test_count_estimate_matches_oracle():
    g = glassgen.generate(400, 4)
    ctx, _ = make_ctx(g, COUNT_M=12, COUNT_DEGREE=60, SEED=3)
    try:
        lmax, _ = pfe.pfe_estimate(ctx)
        a, b = 0.05 * lmax, 0.15 * lmax
        pfe.pfe_set_interval(ctx, a, b)
        _, est = pfe.pfe_estimate(ctx)
        c = d = 0.5 * lmax
        ref = oracle.count_estimate(oracle.csr_from_springs(g), c, d, (a - c) / d, (b - c) / d, 60, "none", 12, 3)
        assert est == pytest.approx(ref, rel=1e-9, abs=1e-9)
    finally:
        pfe.pfe_destroy(ctx)


# ------------------------------------------------------------------ a5-a7: the solve
def _solve_and_check(g, lo, hi, precision=0, **params):
    ctx, _ = make_ctx(g, PRECISION=precision, **params)
    try:
        lmax, _ = pfe.pfe_estimate(ctx)
        a, b = lo * lmax, hi * lmax
        pfe.pfe_set_interval(ctx, a, b)
        nf, _ = pfe.pfe_solve(ctx)
        lam, V, res = pfe.pfe_get_eigenpairs(ctx, g.n, nf)
        stats = pfe.pfe_get_stats(ctx)
    finally:
        pfe.pfe_destroy(ctx)
    H = oracle.csr_from_springs(g)
    w, U, w_all = oracle.exact_interval(H, a, b)
    d, e = oracle.tridiagonalize(H.dense())
    count = oracle.count_below(d, e, b) - oracle.count_below(d, e, a)
    assert nf == w.size == count, (nf, w.size, count)
    assert np.allclose(lam, w, rtol=1e-10, atol=0)
    r = oracle.residuals(H, lam, V)
    assert np.all(r <= 1e-8 * lmax)
    assert np.allclose(res, r, rtol=1e-3, atol=1e-14 * lmax)
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0, atol=1e-12)
    assert cluster_angles_ok(H, lam, V, w_all, U, w, lmax)
    return stats


def test_solve_small_glass_fp64():
    st = _solve_and_check(glassgen.generate(300, 5), 0.05, 0.12)
    assert st["iterations"] >= 2 and st["width"] >= 177  # 177 eigenvalues lie in the margin window


def test_solve_config_n1000_fp64():
    """N = 1000, seed 0, [0.02, 0.05] lambda_max, automatic degree and width."""
    _solve_and_check(glassgen.generate(1000, 0), 0.02, 0.05)


@pytest.mark.parametrize("rule", [0, 1])
def test_degree_rule(rule):
    """DEGREE_RULE 0 keeps the degree of eq. (thresh) (r = sqrt(0.1)), the library's own host design of
    it; 1 may only raise it (the work model's candidates start there).  Both solve exactly."""
    g = glassgen.generate(1000, 0)
    st = _solve_and_check(g, 0.02, 0.05, DEGREE_RULE=rule)
    lmax = st["lambda_max"]
    xi, eta = (0.02 * lmax - lmax / 2) / (lmax / 2), (0.05 * lmax - lmax / 2) / (lmax / 2)
    m0, _ = pfe.pfe_design_filter("pq", xi, eta, eps=0.25 * (eta - xi), r=0.1 ** 0.5)
    if rule == 0:
        assert st["degree"] == m0
    else:
        assert m0 <= st["degree"] <= 4 * m0


def test_solve_config_n1000_degree40():
    """The same workload with the fixed degree 40 (a weak filter: more iterations)."""
    _solve_and_check(glassgen.generate(1000, 0), 0.02, 0.05, DEGREE=40, WIDTH=256, MAX_ITERS=200)


@pytest.mark.parametrize("overlap", [1, 0])
def test_solve_mixed_precision_matches_fp64_accuracy(overlap):
    """Mixed precision, with the FP32 and FP64 column groups on two streams (1) or on one (0)."""
    st = _solve_and_check(glassgen.generate(300, 5), 0.05, 0.12, precision=1, OVERLAP=overlap)
    assert st["filter_col_steps_f32"] > 0 and st["filter_col_steps"] > 0  # both precisions were used


@pytest.mark.parametrize("N,seed,lo,hi,shape", [(300, 5, 0.05, 0.12, -1), (1000, 0, 0.02, 0.05, -1),
                                                (1000, 0, 0.02, 0.05, 10)])
def test_solve_defect_corrected_fp32_filter_reaches_fp64_accuracy(N, seed, lo, hi, shape):
    """PRECISION 2: every filter application runs in FP32 (below the hand-over residual by defect
    correction: x p(theta) in FP64 plus the recurrence on the residual in FP32).  The plain FP32 filter
    alone stalls near its rounding level (~1e-4 of lambda_max); reaching the 1e-8 residuals, the exact
    count and the 1e-10 eigenvalues with no FP64 filter sweep shows the correction at work."""
    try:  # shape 10: the forced steps too run with the tile's neighbour rows in shared memory
        st = _solve_and_check(glassgen.generate(N, seed), lo, hi, precision=2, STEP_SHAPE_F32=shape)
    finally:
        ctx, _ = make_ctx(glassgen.generate(20, 1), STEP_SHAPE_F32=-1)  # the shape is process-wide
        pfe.pfe_destroy(ctx)
    assert st["filter_col_steps_f32"] > 0 and st["filter_col_steps"] == 0 and st["fp64_sweeps"] == 0
    assert st["filter_col_steps_forced"] > 0


@pytest.mark.parametrize("block", [16, 64])
def test_solve_block_lanczos(block):
    """Thick-restart block Lanczos on p(Ht) + Rayleigh-Ritz with H (PFE_P_METHOD = 1)."""
    st = _solve_and_check(glassgen.generate(300, 5), 0.05, 0.12, METHOD=1, BLOCK=block)
    assert st["basis"] >= 3 * block


def test_solve_block_lanczos_n1000():
    _solve_and_check(glassgen.generate(1000, 0), 0.02, 0.05, METHOD=1, BLOCK=32)


@pytest.mark.parametrize("threads", [0, 1, 3])
def test_solve_batch_equals_solo(threads):
    """Batched lockstep solve (one persistent filter launch per step over all samples, replayed from
    a CUDA graph; the samples' dense steps from `threads` host threads, 0 = automatic): every sample
    matches the exact interval eigenpairs and its own solo solve."""
    sizes = (150, 420, 180, 300, 95)
    gs = [glassgen.generate(n, glassgen.subseed(3, i)) for i, n in enumerate(sizes)]
    ctxs = []
    try:
        for g in gs:
            ctx, _ = make_ctx(g, BATCH_THREADS=threads)
            lmax, _ = pfe.pfe_estimate(ctx)
            pfe.pfe_set_interval(ctx, 0.05 * lmax, 0.15 * lmax)
            ctxs.append(ctx)
        nfs, st = pfe.pfe_solve_batch(ctxs)
        assert st == pfe.PFE_OK, [pfe.pfe_last_error(c) for c in ctxs]
        for g, ctx, nf in zip(gs, ctxs, nfs):
            lam, V, res = pfe.pfe_get_eigenpairs(ctx, g.n, nf)
            stats = pfe.pfe_get_stats(ctx)
            assert stats["batch_replays"] >= 2
            lmax = stats["lambda_max"]
            H = oracle.csr_from_springs(g)
            w, _, _ = oracle.exact_interval(H, 0.05 * lmax, 0.15 * lmax)
            assert nf == w.size
            assert np.allclose(lam, w, rtol=1e-10, atol=0)
            assert np.all(oracle.residuals(H, lam, V) <= 1e-8 * lmax)
            # the same sample solved alone
            solo, _ = make_ctx(g)
            try:
                pfe.pfe_set_param(solo, pfe.PFE_P_LAMBDA_MAX, lmax)
                pfe.pfe_set_interval(solo, 0.05 * lmax, 0.15 * lmax)
                nf1, _ = pfe.pfe_solve(solo)
                lam1, _, _ = pfe.pfe_get_eigenpairs(solo, g.n, nf1)
            finally:
                pfe.pfe_destroy(solo)
            assert nf1 == nf and np.allclose(lam1, lam, rtol=1e-10, atol=0)
    finally:
        for c in ctxs:
            pfe.pfe_destroy(c)


def test_solve_batch_block_lanczos_members():
    """A batch of block Lanczos samples (solved concurrently from host threads): exact eigenpairs."""
    gs = [glassgen.generate(n, glassgen.subseed(5, i)) for i, n in enumerate((220, 300, 160, 260))]
    ctxs = []
    try:
        for g in gs:
            ctx, _ = make_ctx(g, METHOD=1, BLOCK=16)
            lmax, _ = pfe.pfe_estimate(ctx)
            pfe.pfe_set_interval(ctx, 0.05 * lmax, 0.12 * lmax)
            ctxs.append(ctx)
        nfs, st = pfe.pfe_solve_batch(ctxs)
        assert st == pfe.PFE_OK, [pfe.pfe_last_error(c) for c in ctxs]
        for g, ctx, nf in zip(gs, ctxs, nfs):
            lam, V, _ = pfe.pfe_get_eigenpairs(ctx, g.n, nf)
            lmax = pfe.pfe_get_stats(ctx)["lambda_max"]
            H = oracle.csr_from_springs(g)
            w, _, _ = oracle.exact_interval(H, 0.05 * lmax, 0.12 * lmax)
            assert nf == w.size and np.allclose(lam, w, rtol=1e-10, atol=0)
            assert np.all(oracle.residuals(H, lam, V) <= 1e-8 * lmax)
    finally:
        for c in ctxs:
            pfe.pfe_destroy(c)


def test_solve_batch_mixed_precision_members():
    """A batch whose members use different filter precisions (FP64, the FP64 hand-over, the defect-
    corrected FP32 filter) still matches the exact eigenpairs."""
    gs = [glassgen.generate(n, 40 + i) for i, n in enumerate((200, 260, 230))]
    ctxs = []
    try:
        for i, g in enumerate(gs):
            ctx, _ = make_ctx(g, PRECISION=i % 3)
            lmax, _ = pfe.pfe_estimate(ctx)
            pfe.pfe_set_interval(ctx, 0.05 * lmax, 0.12 * lmax)
            ctxs.append(ctx)
        nfs, st = pfe.pfe_solve_batch(ctxs)
        assert st == pfe.PFE_OK, [pfe.pfe_last_error(c) for c in ctxs]
        for g, ctx, nf in zip(gs, ctxs, nfs):
            lam, _, _ = pfe.pfe_get_eigenpairs(ctx, g.n, nf)
            lmax = pfe.pfe_get_stats(ctx)["lambda_max"]
            w, _, _ = oracle.exact_interval(oracle.csr_from_springs(g), 0.05 * lmax, 0.12 * lmax)
            assert nf == w.size and np.allclose(lam, w, rtol=1e-10, atol=0)
    finally:
        for c in ctxs:
            pfe.pfe_destroy(c)


# ------------------------------------------------------------------ a9: the adjoint
def _bsr_to_csr_index(rp_b, ci_b, rp_c):
    """For each BSR entry 9p + 3r + s the index of the oracle's CSR entry (3i+r, 3j+s)."""
    idx = np.zeros(9 * ci_b.size, np.int64)
    for i in range(rp_b.size - 1):
        for p in range(rp_b[i], rp_b[i + 1]):
            for r in range(3):
                base = rp_c[3 * i + r] + 3 * (p - rp_b[i])
                idx[9 * p + 3 * r:9 * p + 3 * r + 3] = base + np.arange(3)
    return idx


@pytest.mark.parametrize("m,k", [(0, 2), (1, 3), (2, 4), (14, 3), (16, 8), (37, 11)])
def test_adjoint_and_chain_parity(m, k):
    """Degrees that give one, several, exactly filled and ragged checkpoint segments (S = ceil(sqrt m));
    odd and even block widths."""
    g = glassgen.generate(90, 6)
    ctx, (rp, ci, vals) = make_ctx(g, LAMBDA_MAX=0.2)
    try:
        c = d = 0.1
        coef = oracle.filter_coeffs(-0.9, -0.8, 0.03, m, "jackson")
        rng = np.random.default_rng(4 + m)
        X = rng.standard_normal((g.n, k))
        Yb = rng.standard_normal((g.n, k))
        Xd, Ybd = dev_colmajor(X), dev_colmajor(Yb)
        Xbd = torch.zeros((k, g.n), device="cuda", dtype=torch.float64)
        vb = torch.zeros(9 * ci.size, device="cuda", dtype=torch.float64)
        pfe.pfe_filter_adjoint(ctx, len(coef) - 1, coef, k, Xd, g.n, Ybd, g.n, Xbd, g.n, vb)
        kb = torch.zeros(g.n_bonds, device="cuda", dtype=torch.float64)
        mb = torch.zeros(g.n_atoms, device="cuda", dtype=torch.float64)
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)  # noqa: E731
        pfe.pfe_chain_springs(ctx, g.n_bonds, t(g.bi, torch.int32), t(g.bj, torch.int32), t(g.rhat, torch.float64),
                              vb, kb, mb)
        torch.cuda.synchronize()
        H = oracle.csr_from_springs(g)
        Xb_ref, vb_ref = oracle.filter_adjoint(H, c, d, coef, X, Yb)
        assert np.max(np.abs(Xbd.cpu().numpy().T - Xb_ref)) <= 1e-11 * np.abs(Xb_ref).max()
        rp_c, _, _ = H.arrays()
        vb_gpu = np.zeros(H.nnz)
        vb_gpu[_bsr_to_csr_index(rp, ci, rp_c)] = vb.cpu().numpy()
        assert np.max(np.abs(vb_gpu - vb_ref)) <= 1e-10 * np.abs(vb_ref).max()
        kb_ref, mb_ref = oracle.chain_springs(H, g, vb_ref)
        assert np.max(np.abs(kb.cpu().numpy() - kb_ref)) <= 1e-10 * np.abs(kb_ref).max()
        assert np.max(np.abs(mb.cpu().numpy() - mb_ref)) <= 1e-10 * np.abs(mb_ref).max()
    finally:
        pfe.pfe_destroy(ctx)


def test_create_from_device_pointers():
    g = glassgen.generate(120, 8)
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)  # noqa: E731
    ctx = pfe.pfe_create(g.n_atoms, t(rp, torch.int32), t(ci, torch.int32), t(vals, torch.float64),
                         t(g.mass, torch.float64), flags=pfe.PFE_DEVICE_PTRS)
    try:
        pfe.pfe_set_param(ctx, pfe.PFE_P_LAMBDA_MAX, 0.4)
        X = np.random.default_rng(0).standard_normal((g.n, 2))
        Y = filter_gpu(ctx, np.array([0.0, 1.0]), X)
        H = oracle.csr_from_springs(g)
        assert np.max(np.abs(Y - (H.matmul(X) - 0.2 * X) / 0.2)) <= 1e-13 * np.abs(Y).max()
    finally:
        pfe.pfe_destroy(ctx)
