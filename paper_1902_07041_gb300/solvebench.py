"""Time one interval solve of libpfe on a synthetic glass and print its statistics.

    python -m paper_1902_07041_gb300.solvebench --n-atoms 100000 --seed 1 --lo 0.02 --hi 0.0214 --method 0

Prints one JSON line per solve: wall time around pfe_estimate + pfe_solve, the solver's own
statistics (pfe_get_stats) and the status.  --method 1 selects the thick-restart block Lanczos
solver (--block, --basis-factor); --precision 1 the mixed-precision subspace iteration.
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    import torch

    import glassgen
    import paper_1902_07041_gb300 as pfe

    ap = argparse.ArgumentParser()
    ap.add_argument("--n-atoms", type=int, default=100_000)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--lo", type=float, default=0.02)
    ap.add_argument("--hi", type=float, default=0.0214)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--method", type=int, default=0)
    ap.add_argument("--block", type=int, default=64)
    ap.add_argument("--basis-factor", type=float, default=2.0)
    ap.add_argument("--rank1", type=int, default=1)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--filter", type=int, default=0, help="0 piecewise quadratic, 1 Dirac (with --method 1)")
    ap.add_argument("--damping", type=int, default=0, help="0 none, 1 Jackson, 2 Lanczos")
    ap.add_argument("--sliced", type=int, default=0, help="spectrum slicing with this many eigenvalues a slice")
    ap.add_argument("--rate", type=float, default=0.0,
                    help="r of eq. (thresh) (piecewise quadratic filter); 0: the method's default and degree rule")
    ap.add_argument("--phi", type=float, default=0.8, help="phi of the Dirac filter")
    ap.add_argument("--degree", type=int, default=0, help="filter degree (0: chosen by eq. (thresh))")
    ap.add_argument("--width", type=int, default=0, help="subspace width (0: automatic)")
    ap.add_argument("--overlap", type=int, default=1, help="mixed precision: FP32 and FP64 groups on two streams")
    ap.add_argument("--refine-tol", type=float, default=1e-4, help="mixed precision: hand-over residual to FP64")
    ap.add_argument("--degree-rule", type=int, default=1, help="1: cost-model degree (automatic degree only)")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    g = glassgen.generate(a.n_atoms, a.seed)
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    for _ in range(a.repeat):
        ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
        try:
            for key, v in (("PRECISION", a.precision), ("METHOD", a.method), ("BLOCK", a.block),
                           ("BASIS_FACTOR", a.basis_factor), ("RANK1", a.rank1), ("FILTER", a.filter),
                           ("DAMPING", a.damping), ("PHI", a.phi), ("DEGREE", a.degree),
                           ("WIDTH", a.width), ("OVERLAP", a.overlap), ("REFINE_TOL", a.refine_tol),
                           ("DEGREE_RULE", a.degree_rule)):
                pfe.pfe_set_param(ctx, getattr(pfe, "PFE_P_" + key), v)
            if a.rate > 0:
                pfe.pfe_set_param(ctx, pfe.PFE_P_RATE, a.rate)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lmax, _ = pfe.pfe_estimate(ctx)
            pfe.pfe_set_interval(ctx, a.lo * lmax, a.hi * lmax)
            if a.sliced > 0:
                pfe.pfe_set_param(ctx, pfe.PFE_P_SLICE_TARGET, a.sliced)
                nf, st = pfe.pfe_solve_sliced(ctx, raise_on_error=False)
            else:
                nf, st = pfe.pfe_solve(ctx, raise_on_error=False)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            stats = pfe.pfe_get_stats(ctx)
            print(json.dumps({"n_atoms": a.n_atoms, "seed": a.seed, "lo": a.lo, "hi": a.hi, "method": a.method,
                              "precision": a.precision, "block": a.block, "basis_factor": a.basis_factor,
                              "filter": a.filter, "damping": a.damping, "sliced": a.sliced, "rate": a.rate,
                              "phi": a.phi, "degree_set": a.degree, "width_set": a.width, "overlap": a.overlap,
                              "refine_tol": a.refine_tol, "degree_rule": a.degree_rule,
                              "rank1_in_use": pfe.pfe_get_param(ctx, pfe.PFE_P_RANK1), "wall_s": wall,
                              "status": st, **stats}), flush=True)
        finally:
            pfe.pfe_destroy(ctx)


if __name__ == "__main__":
    main()
