"""The allocation-free filter entry point, for callers that cannot let the library allocate device
memory (their memory is owned by another allocator, or cudaMalloc's implicit synchronisation is
not acceptable).  Called through the C ABI and compared with pfe_filter_apply, the entry point
that allocates its own work buffers, on two calls in a row.

This file is collected last on purpose: the entry point shares one fixed device array across
calls, and the test must pass both alone in a fresh process and after every other test."""
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


def _filter(ctx, coef, X, noalloc):
    n, k = X.shape
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    Yd = torch.full((k, n), float("nan"), device="cuda", dtype=torch.float64)
    if noalloc:
        pfe.pfe_filter_apply_noalloc(ctx, len(coef) - 1, coef, k, Xd, n, Yd, n)
    else:
        pfe.pfe_filter_apply(ctx, len(coef) - 1, coef, k, Xd, n, Yd, n, pfe.PFE_F64)
    torch.cuda.synchronize()
    return Yd.cpu().numpy().T


def test_noalloc_filter_matches_allocating_filter_twice():
    g = glassgen.generate(300, 5)
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
    try:
        pfe.pfe_set_param(ctx, pfe.PFE_P_LAMBDA_MAX, 0.2)
        coef = oracle.filter_coeffs(-0.96, -0.9, 0.015, 33, "none")
        rng = np.random.default_rng(11)
        X1 = rng.standard_normal((g.n, 37))
        X2 = rng.standard_normal((g.n, 5))
        # without the operator built by an allocating call, the entry point refuses to run
        with pytest.raises(pfe.PfeError) as e:
            _filter(ctx, coef, X1, True)
        assert e.value.status == pfe.PFE_E_STATE
        ref1 = _filter(ctx, coef, X1, False)
        ref2 = _filter(ctx, coef, X2, False)
        tol = 1e-11 * np.abs(coef).sum()
        # the allocating filter itself against the oracle's Alg. 2 (c = d = lambda_max / 2)
        H = oracle.csr_from_springs(g)
        assert np.max(np.abs(ref1 - oracle.cheb_filter(H, 0.1, 0.1, coef, X1))) <= tol * np.abs(X1).max()
        for _ in range(2):  # two calls in a row share (and reuse) the fixed array
            y1 = _filter(ctx, coef, X1, True)
            assert np.max(np.abs(y1 - ref1)) <= tol * np.abs(X1).max()
            y2 = _filter(ctx, coef, X2, True)
            assert np.max(np.abs(y2 - ref2)) <= tol * np.abs(X2).max()
            assert np.max(np.abs(y1 - oracle.cheb_filter(H, 0.1, 0.1, coef, X1))) <= tol * np.abs(X1).max()
        # a caller stream other than the context's, right after an allocating call that builds the
        # filter operator on the context's stream (a fresh context: nothing built before)
        ctx3 = pfe.pfe_create(g.n_atoms, *pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat), g.mass)
        try:
            pfe.pfe_set_param(ctx3, pfe.PFE_P_LAMBDA_MAX, 0.2)
            n, k = X1.shape
            Xd = torch.from_numpy(np.ascontiguousarray(X1.T)).cuda()
            Ya = torch.full((k, n), float("nan"), device="cuda", dtype=torch.float64)
            Yb = torch.full((k, n), float("nan"), device="cuda", dtype=torch.float64)
            torch.cuda.synchronize()
            side = torch.cuda.Stream()
            pfe.pfe_filter_apply(ctx3, len(coef) - 1, coef, k, Xd, n, Ya, n, pfe.PFE_F64)  # context stream
            pfe.pfe_filter_apply_noalloc(ctx3, len(coef) - 1, coef, k, Xd, n, Yb, n, stream=side)
            side.synchronize()
            torch.cuda.synchronize()
            assert np.max(np.abs(Yb.cpu().numpy().T - ref1)) <= tol * np.abs(X1).max()
            assert np.max(np.abs(Ya.cpu().numpy().T - ref1)) <= tol * np.abs(X1).max()
        finally:
            pfe.pfe_destroy(ctx3)
        # sizes beyond the fixed array are rejected with a clear error
        big = glassgen.generate(20000, 2)
        rp, ci, vals = pfe.pfe_springs_to_bsr(big.n_atoms, big.bi, big.bj, big.k, big.rhat)
        ctx2 = pfe.pfe_create(big.n_atoms, rp, ci, vals, big.mass)
        try:
            pfe.pfe_set_param(ctx2, pfe.PFE_P_LAMBDA_MAX, 0.3)
            Xb = np.ones((big.n, 20))
            _filter(ctx2, coef, Xb[:, :1], False)
            with pytest.raises(pfe.PfeError) as e:
                _filter(ctx2, coef, Xb, True)
            assert e.value.status == pfe.PFE_E_CAPACITY
        finally:
            pfe.pfe_destroy(ctx2)
    finally:
        pfe.pfe_destroy(ctx)
