"""GPU parity of the filter adjoint (pfe_filter_adjoint + pfe_chain_springs behind
torch.autograd.Function) against the oracle's reverse sweep, central finite differences at the
N = 50,000 adjoint workload, and Hellmann-Feynman eigenvalue derivatives."""
import math

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


def _net(g):
    from paper_1902_07041_gb300.autograd import SpringNetwork

    return SpringNetwork(g.n_atoms, g.bi, g.bj, g.rhat)


def test_autograd_matches_oracle_adjoint():
    from paper_1902_07041_gb300.autograd import cheb_filter

    g = glassgen.generate(120, 21)
    lmax = 0.2
    coef = oracle.filter_coeffs(-0.9, -0.8, 0.03, 16, "none")
    rng = np.random.default_rng(2)
    X = torch.tensor(rng.standard_normal((g.n, 3)), device="cuda", requires_grad=True)
    kk = torch.tensor(g.k, device="cuda", requires_grad=True)
    mm = torch.tensor(g.mass, device="cuda", requires_grad=True)
    Yb = rng.standard_normal((g.n, 3))
    Y = cheb_filter(X, kk, mm, _net(g), coef, lmax)
    (Y * torch.tensor(Yb, device="cuda")).sum().backward()
    H = oracle.csr_from_springs(g)
    Y_ref = oracle.cheb_filter(H, lmax / 2, lmax / 2, coef, X.detach().cpu().numpy())
    assert np.max(np.abs(Y.detach().cpu().numpy() - Y_ref)) <= 1e-11 * np.abs(Y_ref).max()
    Xb_ref, vb_ref = oracle.filter_adjoint(H, lmax / 2, lmax / 2, coef, X.detach().cpu().numpy(), Yb)
    kb_ref, mb_ref = oracle.chain_springs(H, g, vb_ref)
    assert np.max(np.abs(X.grad.cpu().numpy() - Xb_ref)) <= 1e-11 * np.abs(Xb_ref).max()
    assert np.max(np.abs(kk.grad.cpu().numpy() - kb_ref)) <= 1e-10 * np.abs(kb_ref).max()
    assert np.max(np.abs(mm.grad.cpu().numpy() - mb_ref)) <= 1e-10 * np.abs(mb_ref).max()


def test_adjoint_central_differences_n50k():
    """N = 50,000 (seed 4), degree 60, k = 64 columns, FP64: dL/dk on 32 random springs against
    central differences with a 1e-6 relative step, L = <Ybar, p(Ht) X>."""
    from paper_1902_07041_gb300.autograd import cheb_filter

    g = glassgen.generate(50_000, 4)
    net = _net(g)
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
    lmax, _ = pfe.pfe_estimate(ctx)
    pfe.pfe_destroy(ctx)
    coef = oracle.filter_coeffs(2 * 0.02 / 1.01 - 1, 2 * 0.04 / 1.01 - 1, 0.25 * 0.04 / 1.01, 60, "none")
    gen = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn(g.n, 64, device="cuda", dtype=torch.float64, generator=gen)
    Yb = torch.randn(g.n, 64, device="cuda", dtype=torch.float64, generator=gen)
    kk = torch.tensor(g.k, device="cuda", requires_grad=True)
    mm = torch.tensor(g.mass, device="cuda")
    (cheb_filter(X, kk, mm, net, coef, lmax) * Yb).sum().backward()
    kb = kk.grad.cpu().numpy()
    rng = np.random.default_rng(6)
    for e in rng.choice(g.n_bonds, 32, replace=False):
        h = 1e-6 * g.k[e]
        vals_pm = []
        for sgn in (1, -1):
            k2 = torch.tensor(g.k, device="cuda")
            k2[e] += sgn * h
            with torch.no_grad():
                vals_pm.append(float((cheb_filter(X, k2, mm, net, coef, lmax) * Yb).sum()))
        fd = (vals_pm[0] - vals_pm[1]) / (2 * h)
        assert fd == pytest.approx(kb[e], rel=2e-5, abs=1e-6 * np.abs(kb).max())


def test_adjoint_hellmann_feynman_on_converged_eigenpairs():
    """For a converged simple eigenpair (lambda, v) and L = v^T p(Ht) v with v held fixed,
    dL/dk_e = p'(lt) / d * dlambda/dk_e (the derivative of a matrix function along an eigenvector),
    and Hellmann-Feynman gives dlambda/dk_e = ((v_i.r)/sqrt(m_i) - (v_j.r)/sqrt(m_j))^2."""
    from numpy.polynomial import chebyshev as C

    from paper_1902_07041_gb300.autograd import cheb_filter

    g = glassgen.generate(3000, 4)
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
    try:
        lmax, _ = pfe.pfe_estimate(ctx)
        pfe.pfe_set_param(ctx, pfe.PFE_P_TOL, 1e-10)
        pfe.pfe_set_interval(ctx, 0.02 * lmax, 0.04 * lmax)
        nf, _ = pfe.pfe_solve(ctx)
        lam, V, _ = pfe.pfe_get_eigenpairs(ctx, g.n, nf)
    finally:
        pfe.pfe_destroy(ctx)
    assert nf > 20
    c = d = lmax / 2
    coef = oracle.filter_coeffs(-0.97, -0.9, 0.02, 40, "none")
    dcoef = C.chebder(coef)
    gaps = np.minimum(np.diff(lam, prepend=-np.inf), np.diff(lam, append=np.inf))
    picks = [i for i in np.argsort(-gaps)[:6]]
    net = _net(g)
    mm = torch.tensor(g.mass, device="cuda")
    rng = np.random.default_rng(7)
    bonds = rng.choice(g.n_bonds, 8, replace=False)
    for i in picks:
        v = V[:, i]
        vt = torch.tensor(v[:, None], device="cuda")
        kk = torch.tensor(g.k, device="cuda", requires_grad=True)
        (cheb_filter(vt, kk, mm, net, coef, lmax) * vt).sum().backward()
        lt = (lam[i] - c) / d
        scale = C.chebval(lt, dcoef) / d
        vr = v.reshape(-1, 3)
        for e in bonds:
            a, b, r = g.bi[e], g.bj[e], g.rhat[e]
            hf = (vr[a] @ r / math.sqrt(g.mass[a]) - vr[b] @ r / math.sqrt(g.mass[b])) ** 2
            assert float(kk.grad[e]) == pytest.approx(scale * hf, rel=1e-6, abs=1e-9 * abs(scale) * lmax)
