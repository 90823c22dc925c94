"""Mode analysis of Sec. 4.4 on the GPU (participation ratio, plane-wave content), through the C ABI,
against the oracle on eigenvectors that the oracle or the construction fixes."""
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


def test_single_atom_modes_of_a_diagonal_matrix():
    """Diagonal H with distinct entries: every eigenvector is a coordinate vector e_{3i+d}, so
    PR = 1/N and the plane-wave content is (2/N) (khat_d^2, 1 - khat_d^2).  Solved by block Lanczos,
    whose residuals sit near rounding: the content is linear in the eigenvector error (the
    participation ratio of a coordinate vector only quadratic)."""
    N = 300
    d = np.linspace(0.01, 1.0, 3 * N)
    rp = np.arange(N + 1, dtype=np.int32)
    ci = np.arange(N, dtype=np.int32)
    vals = np.zeros(9 * N)
    for i in range(N):
        vals[9 * i], vals[9 * i + 4], vals[9 * i + 8] = d[3 * i:3 * i + 3]
    ctx = pfe.pfe_create(N, rp, ci, vals, None)
    try:
        pfe.pfe_set_param(ctx, pfe.PFE_P_LAMBDA_MAX, 1.01)
        pfe.pfe_set_param(ctx, pfe.PFE_P_METHOD, 1)
        pfe.pfe_set_param(ctx, pfe.PFE_P_BLOCK, 16)
        pfe.pfe_set_interval(ctx, 0.30, 0.34)
        nf, _ = pfe.pfe_solve(ctx)
        sel = np.nonzero((d >= 0.30) & (d <= 0.34))[0]
        assert nf == sel.size
        pr = pfe.pfe_participation_ratio(ctx, nf)
        assert np.allclose(pr, 1.0 / N, rtol=1e-12, atol=0)
        pos = np.random.default_rng(1).uniform(0, 10, (N, 3))
        ks = np.array([[0.3, -0.2, 0.5], [1.0, 0.0, 0.0]])
        out = pfe.pfe_plane_wave_content(ctx, pos, ks, nf)
        E = np.zeros((3 * N, nf))
        E[sel, np.arange(nf)] = 1.0
        ref = oracle.plane_wave_content(E, pos, ks)
        assert np.allclose(out, ref, rtol=1e-9, atol=1e-13)
    finally:
        pfe.pfe_destroy(ctx)


def test_glass_modes_match_exact_eigenvectors():
    """Glass N = 400: PR and plane-wave content of the block Lanczos eigenvectors (residuals near
    rounding) against the oracle on the exact eigenvectors, for modes separated from their
    neighbours (the quantities are basis dependent inside a degenerate cluster)."""
    g = glassgen.generate(400, 11)
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
    try:
        pfe.pfe_set_param(ctx, pfe.PFE_P_METHOD, 1)
        pfe.pfe_set_param(ctx, pfe.PFE_P_BLOCK, 16)
        lmax, _ = pfe.pfe_estimate(ctx)
        a, b = 0.02 * lmax, 0.08 * lmax
        pfe.pfe_set_interval(ctx, a, b)
        nf, _ = pfe.pfe_solve(ctx)
        H = oracle.csr_from_springs(g)
        w, U, w_all = oracle.exact_interval(H, a, b)
        assert nf == w.size
        pr = pfe.pfe_participation_ratio(ctx, nf)
        L = g.box
        ks = 2 * np.pi / L * np.array([[1, 0, 0], [0, 1, 1], [1, -1, 2]], float)
        out = pfe.pfe_plane_wave_content(ctx, g.pos, ks, nf)
        pr_ref = oracle.participation_ratio(U)
        out_ref = oracle.plane_wave_content(U, g.pos, ks)
        gaps = np.array([np.min(np.abs(np.delete(w_all, np.argmin(np.abs(w_all - x))) - x)) for x in w])
        iso = gaps > 1e-4 * lmax
        assert iso.sum() >= nf // 2
        assert np.allclose(pr[iso], pr_ref[iso], rtol=1e-8, atol=0)
        assert np.allclose(out[iso], out_ref[iso], rtol=1e-8, atol=1e-12)
        assert np.all((pr > 0) & (pr <= 1.0 + 1e-12))
    finally:
        pfe.pfe_destroy(ctx)


def test_mode_analysis_errors():
    g = glassgen.generate(60, 2)
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
    try:
        with pytest.raises(pfe.PfeError):  # no solve results yet
            pfe.pfe_participation_ratio(ctx, 10)
        lmax, _ = pfe.pfe_estimate(ctx)
        pfe.pfe_set_interval(ctx, 0.05 * lmax, 0.2 * lmax)
        nf, _ = pfe.pfe_solve(ctx)
        assert nf > 1
        with pytest.raises(pfe.PfeError):  # capacity below the eigenpair count
            pfe.pfe_participation_ratio(ctx, nf - 1)
        with pytest.raises(pfe.PfeError):  # zero wave vector
            pfe.pfe_plane_wave_content(ctx, g.pos, np.zeros((1, 3)), nf)
    finally:
        pfe.pfe_destroy(ctx)
