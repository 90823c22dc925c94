"""The stepwise solve (pfe_solve_begin / pfe_solve_iterate / pfe_solve_end) through the C ABI: it is
pfe_solve one outer iteration at a time (Alg. 4), so it must return the exact interval eigenpairs of
the oracle, report the iteration in progress, end early on request with only converged pairs, and
refuse calls out of order."""
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


@pytest.fixture(scope="module")
def glass():
    g = glassgen.generate(300, 5)
    return g, pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)


def _ctx(glass, lo=0.05, hi=0.12, **params):
    g, (rp, ci, vals) = glass
    ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
    for k, v in params.items():
        pfe.pfe_set_param(ctx, getattr(pfe, "PFE_P_" + k), v)
    lmax, _ = pfe.pfe_estimate(ctx)
    pfe.pfe_set_interval(ctx, lo * lmax, hi * lmax)
    return ctx, lmax


def test_stepwise_solve_matches_pfe_solve_and_exact(glass):
    g, _ = glass
    ctx, lmax = _ctx(glass)
    try:
        pfe.pfe_solve_begin(ctx)
        seen = []
        done = False
        while not done:
            st = pfe.pfe_get_stats(ctx)
            seen.append((st["iterations"], st["active"], st["locked"], st["width"]))
            done = pfe.pfe_solve_iterate(ctx)
        assert pfe.pfe_solve_iterate(ctx) is True  # a finished solve stays finished
        nf, status = pfe.pfe_solve_end(ctx)
        lam, V, res = pfe.pfe_get_eigenpairs(ctx, g.n, nf)
        final = pfe.pfe_get_stats(ctx)
    finally:
        pfe.pfe_destroy(ctx)
    assert status == pfe.PFE_OK
    # progress: one iteration per call, the active block shrinks as pairs lock, width fixed
    assert [s[0] for s in seen] == list(range(len(seen)))
    q = seen[0][3]
    assert seen[0][1:3] == (q, 0) and all(s[3] == q for s in seen)
    assert all(s[1] + s[2] == q for s in seen)
    assert all(b[1] <= a[1] for a, b in zip(seen, seen[1:]))
    assert final["iterations"] == len(seen) and final["active"] == 0 and final["locked"] == 0
    # the same solve in one call
    ctx, _ = _ctx(glass)
    try:
        nf2, _ = pfe.pfe_solve(ctx)
        lam2, _, _ = pfe.pfe_get_eigenpairs(ctx, g.n, nf2)
        st2 = pfe.pfe_get_stats(ctx)
    finally:
        pfe.pfe_destroy(ctx)
    assert nf2 == nf and st2["iterations"] == final["iterations"] and st2["matvecs"] == final["matvecs"]
    assert np.allclose(lam2, lam, rtol=1e-12, atol=0)
    # and the oracle's exact eigenpairs of [a, b]
    H = oracle.csr_from_springs(g)
    w, _, _ = oracle.exact_interval(H, 0.05 * lmax, 0.12 * lmax)
    assert nf == w.size and np.allclose(lam, w, rtol=1e-10, atol=0)
    assert np.all(oracle.residuals(H, lam, V) <= 1e-8 * lmax)


def test_stepwise_solve_ended_early(glass):
    """Ending after two iterations: PFE_E_NOCONV, and the pairs returned are only converged ones."""
    g, _ = glass
    ctx, lmax = _ctx(glass)
    try:
        pfe.pfe_solve_begin(ctx)
        for _ in range(2):
            pfe.pfe_solve_iterate(ctx)
        nf, status = pfe.pfe_solve_end(ctx, raise_on_error=False)
        lam, V, res = pfe.pfe_get_eigenpairs(ctx, g.n, nf) if nf else (np.zeros(0), None, None)
        st = pfe.pfe_get_stats(ctx)
        # nothing is in progress any more
        with pytest.raises(pfe.PfeError) as e:
            pfe.pfe_solve_iterate(ctx)
        assert e.value.status == pfe.PFE_E_STATE
    finally:
        pfe.pfe_destroy(ctx)
    assert status == pfe.PFE_E_NOCONV and st["iterations"] == 2 and st["status"] == pfe.PFE_E_NOCONV
    if nf:
        H = oracle.csr_from_springs(g)
        w_all = np.linalg.eigvalsh(H.dense())
        assert np.all(oracle.residuals(H, lam, V) <= 1e-8 * lmax)
        assert np.all(np.min(np.abs(lam[:, None] - w_all[None, :]), axis=1) <= 1e-8 * lmax)


def test_stepwise_calls_out_of_order(glass):
    g, (rp, ci, vals) = glass
    ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
    try:
        for call in (lambda: pfe.pfe_solve_iterate(ctx), lambda: pfe.pfe_solve_end(ctx)):
            with pytest.raises(pfe.PfeError) as e:
                call()
            assert e.value.status == pfe.PFE_E_STATE
        with pytest.raises(pfe.PfeError) as e:  # no interval yet
            pfe.pfe_solve_begin(ctx)
        assert e.value.status == pfe.PFE_E_STATE
        lmax, _ = pfe.pfe_estimate(ctx)
        pfe.pfe_set_interval(ctx, 0.05 * lmax, 0.12 * lmax)
        pfe.pfe_set_param(ctx, pfe.PFE_P_METHOD, 1)  # block Lanczos has no stepwise form
        with pytest.raises(pfe.PfeError) as e:
            pfe.pfe_solve_begin(ctx)
        assert e.value.status == pfe.PFE_E_ARG
    finally:
        pfe.pfe_destroy(ctx)
