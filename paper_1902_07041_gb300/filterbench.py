"""Time the fused Chebyshev filter (Alg. 2) of libpfe on a synthetic glass.

    python -m paper_1902_07041_gb300.filterbench --n-atoms 100000 --k 128 --dtype f64 --degree 8 --reps 3

Prints one JSON line per repetition: seconds per filter step, algorithmic GB/s and GFLOP/s.
The multivectors are column-major n x k device buffers, as at the C ABI.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    import torch

    import glassgen
    import paper_1902_07041_gb300 as pfe

    ap = argparse.ArgumentParser()
    ap.add_argument("--n-atoms", type=int, default=100_000)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--k", type=int, default=128)
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    ap.add_argument("--degree", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--shape", type=int, default=-1, help="kernel shape 0..9, -1 = autotuned")
    ap.add_argument("--rank1", type=int, default=1, help="1: the rank-1 form of the spring network when it has one")
    ap.add_argument("--adjoint", action="store_true", help="time pfe_filter_adjoint (FP64) at this degree instead")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    g = glassgen.generate(a.n_atoms, a.seed)
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
    try:
        pfe.pfe_set_param(ctx, pfe.PFE_P_STEP_SHAPE_F64 if a.dtype == "f64" else pfe.PFE_P_STEP_SHAPE_F32, a.shape)
        pfe.pfe_set_param(ctx, pfe.PFE_P_RANK1, a.rank1)
        pfe.pfe_estimate(ctx)
        tdt = torch.float64 if a.dtype == "f64" else torch.float32
        dt = pfe.PFE_F64 if a.dtype == "f64" else pfe.PFE_F32
        X = torch.randn(a.k, g.n, device="cuda", dtype=tdt)
        Y = torch.empty_like(X)
        s = 8 if a.dtype == "f64" else 4
        kt = 64 if s == 8 else 128
        nnzb = ci.size
        # vector passes: gather t_j, read t_{j-1}, write t_{j+1}, and y read and written every other step
        step_bytes = -(-a.k // kt) * (nnzb * (9 * s + 4) + 4 * (g.n_atoms + 1)) + 4 * g.n * a.k * s
        step_flops = 18 * nnzb * a.k + 6 * g.n * a.k
        noff = nnzb - g.n_atoms
        # the rank-1 form: 3 values and 6 FMAs per off-diagonal block and column, full diagonal blocks
        r1_bytes = -(-a.k // kt) * (noff * (3 * s + 4) + g.n_atoms * 6 * s + 4 * (g.n_atoms + 1)) + 4 * g.n * a.k * s
        r1_flops = 12 * noff * a.k + 18 * g.n_atoms * a.k + 6 * g.n * a.k
        if a.adjoint:
            coef = np.ones(a.degree + 1) / (a.degree + 1)
            Xb = torch.empty_like(X)
            vb = torch.empty(9 * ci.size, device="cuda", dtype=torch.float64)
            pfe.pfe_filter_adjoint(ctx, a.degree, coef, a.k, X, g.n, Y, g.n, Xb, g.n, vb)
            torch.cuda.synchronize()
            for _ in range(a.reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                pfe.pfe_filter_adjoint(ctx, a.degree, coef, a.k, X, g.n, Y, g.n, Xb, g.n, vb)
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / 1e3
                # forward (m steps), segment recomputation (~m steps), reverse (m steps) and the
                # outer products (9 FMA per block and column per step)
                flops = 3 * a.degree * step_flops + a.degree * 18 * nnzb * a.k
                print(json.dumps({"n_atoms": g.n_atoms, "k": a.k, "degree": a.degree, "adjoint_s": t,
                                  "alg_gflops": flops / t / 1e9}), flush=True)
            return
        times = {}
        for m in (1, a.degree + 1):
            coef = np.ones(m + 1) / (m + 1)
            pfe.pfe_filter_apply(ctx, m, coef, a.k, X, g.n, Y, g.n, dt)
            torch.cuda.synchronize()
            best = []
            for _ in range(a.reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                pfe.pfe_filter_apply(ctx, m, coef, a.k, X, g.n, Y, g.n, dt)
                e1.record()
                torch.cuda.synchronize()
                best.append(e0.elapsed_time(e1) / 1e3)
            times[m] = best
        r1 = pfe.pfe_get_param(ctx, pfe.PFE_P_RANK1) == 1 and (a.shape < 0 or a.shape >= 7)
        byts, flops = (r1_bytes, r1_flops) if r1 else (step_bytes, step_flops)
        for r in range(a.reps):
            per = (times[a.degree + 1][r] - times[1][r]) / a.degree
            print(json.dumps({"n_atoms": g.n_atoms, "k": a.k, "dtype": a.dtype, "shape": a.shape,
                              "form": "rank1" if r1 else "bsr", "s_per_step": per,
                              "alg_gbs": byts / per / 1e9, "alg_gflops": flops / per / 1e9}), flush=True)
    finally:
        pfe.pfe_destroy(ctx)


if __name__ == "__main__":
    main()
