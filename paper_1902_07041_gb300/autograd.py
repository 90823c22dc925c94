"""Differentiable Chebyshev filter Y = p_m(Ht(k, m)) X behind torch.autograd.Function.

The forward pass assembles Delta from the spring constants (eq. (1)), forms H = M^-1/2 Delta M^-1/2
(eq. (2)) and applies Alg. 2 through pfe_filter_apply.  The backward pass calls pfe_filter_adjoint
(X_bar = p(Ht) Y_bar, and dL/dH per stored entry from the reverse sweep of the three-term recurrence,
recomputed from about sqrt(m) checkpoints) and pfe_chain_springs (dL/dk per bond, dL/dm per atom).
The spectral transform Ht = (H - cI)/d is held fixed: c and d come from the given lambda bounds,
they are not differentiated.

Tensors: X is (n, k) float64 on the GPU (n = 3N); k_springs (nbonds,) and masses (N,) float64.
"""
from __future__ import annotations

import weakref

import numpy as np
import torch

import paper_1902_07041_gb300 as pfe


class SpringNetwork:
    """Bond structure (which atoms, unit vectors) of a spring network; values are passed per call."""

    def __init__(self, n_atoms, bi, bj, rhat):
        self.n_atoms = int(n_atoms)
        self.bi = np.ascontiguousarray(bi, np.int32)
        self.bj = np.ascontiguousarray(bj, np.int32)
        self.rhat = np.ascontiguousarray(rhat, np.float64)
        self._dev = None

    def device_arrays(self):
        if self._dev is None:
            self._dev = (torch.from_numpy(self.bi).cuda(), torch.from_numpy(self.bj).cuda(),
                         torch.from_numpy(self.rhat).cuda())
        return self._dev


class ChebFilter(torch.autograd.Function):
    @staticmethod
    def forward(fctx, X, k_springs, masses, net, coeffs, lambda_max, lambda_min=0.0):
        rp, ci, vals = pfe.pfe_springs_to_bsr(net.n_atoms, net.bi, net.bj, k_springs.detach().cpu().numpy(), net.rhat)
        handle = pfe.pfe_create(net.n_atoms, rp, ci, vals, masses.detach().cpu().numpy())
        try:
            pfe.pfe_set_param(handle, pfe.PFE_P_LAMBDA_MAX, float(lambda_max))
            pfe.pfe_set_param(handle, pfe.PFE_P_LAMBDA_MIN, float(lambda_min))
            coeffs = np.ascontiguousarray(coeffs, np.float64)
            n, k = X.shape
            Xc = X.detach().t().contiguous()  # column-major n x k storage
            Yc = torch.empty_like(Xc)
            pfe.pfe_filter_apply(handle, coeffs.shape[0] - 1, coeffs, k, Xc, n, Yc, n, pfe.PFE_F64)
        except Exception:
            pfe.pfe_destroy(handle)
            raise
        if not any(fctx.needs_input_grad[:3]):
            pfe.pfe_destroy(handle)
            return Yc.t()
        # the context lives until backward runs, or until the autograd graph is freed
        fctx.release = weakref.finalize(fctx, pfe.pfe_destroy, handle)
        fctx.handle = handle
        fctx.nnzb = int(ci.size)
        fctx.net = net
        fctx.coeffs = coeffs
        fctx.save_for_backward(Xc)
        return Yc.t()

    @staticmethod
    def backward(fctx, Ybar):
        (Xc,) = fctx.saved_tensors
        handle = fctx.handle
        try:
            k, n = Xc.shape
            Ybc = Ybar.detach().to(torch.float64).t().contiguous()
            Xbc = torch.empty_like(Xc)
            vbar = torch.empty(9 * fctx.nnzb, device=Xc.device, dtype=torch.float64)
            pfe.pfe_filter_adjoint(handle, fctx.coeffs.shape[0] - 1, fctx.coeffs, k, Xc, n, Ybc, n, Xbc, n, vbar)
            bi, bj, rhat = fctx.net.device_arrays()
            kbar = torch.empty(bi.shape[0], device=Xc.device, dtype=torch.float64)
            mbar = torch.empty(fctx.net.n_atoms, device=Xc.device, dtype=torch.float64)
            pfe.pfe_chain_springs(handle, bi.shape[0], bi, bj, rhat, vbar, kbar, mbar)
            torch.cuda.synchronize()
        finally:
            fctx.release()
            fctx.handle = None
        return Xbc.t(), kbar, mbar, None, None, None, None


def cheb_filter(X, k_springs, masses, net, coeffs, lambda_max, lambda_min=0.0):
    """Y = p(Ht) X with gradients to X, the spring constants and the masses (one backward per call)."""
    return ChebFilter.apply(X, k_springs, masses, net, coeffs, lambda_max, lambda_min)
