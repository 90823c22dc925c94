"""Solve one glass's interval problem in several forms (FP64 subspace iteration, the two mixed-precision
forms, block Lanczos) and compare each form's eigenpairs with the first form's, pair by pair.

    python -m paper_1902_07041_gb300.comparebench --n-atoms 500000 --seed 2 --lo 0.02 --hi 0.02047 \
        --forms p2,p0 [--out per_pair.csv] [--sliced 700]

Forms: p0 = FP64 subspace iteration, p1 = mixed with the FP64 hand-over, p2 = mixed by defect
correction, bks = block Lanczos (FP64).  Prints one JSON line per form (time to all eigenpairs by
CUDA events around pfe_estimate + pfe_solve, the solver's statistics) and one line comparing every
form with the first: largest and median relative eigenvalue difference and the sine of the largest
principal angle between the two computed invariant subspaces.  --out writes the pairs side by side.
"""
from __future__ import annotations

import argparse
import json


def main():
    import numpy as np
    import torch

    import glassgen
    import paper_1902_07041_gb300 as pfe

    ap = argparse.ArgumentParser()
    ap.add_argument("--n-atoms", type=int, default=500_000)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--lo", type=float, default=0.02)
    ap.add_argument("--hi", type=float, default=0.02047)
    ap.add_argument("--forms", default="p2,p0")
    ap.add_argument("--out", default="")
    ap.add_argument("--sliced", type=int, default=0,
                    help="spectrum slicing (pfe_solve_sliced) with about this many eigenvalues a slice")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    g = glassgen.generate(a.n_atoms, a.seed)
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    n = g.n
    ref = None  # the first form: (name, eigenvalues, residuals, eigenvectors, lambda_max)
    rows, hdr = [], []
    for form in a.forms.split(","):
        ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
        try:
            if form == "bks":
                pfe.pfe_set_param(ctx, pfe.PFE_P_METHOD, 1)
            else:
                pfe.pfe_set_param(ctx, pfe.PFE_P_PRECISION, int(form[1:]))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            lmax, _ = pfe.pfe_estimate(ctx)
            pfe.pfe_set_interval(ctx, a.lo * lmax, a.hi * lmax)
            if a.sliced > 0:
                pfe.pfe_set_param(ctx, pfe.PFE_P_SLICE_TARGET, a.sliced)
                nf, st = pfe.pfe_solve_sliced(ctx, raise_on_error=False)
            else:
                nf, st = pfe.pfe_solve(ctx, raise_on_error=False)
            e1.record()
            torch.cuda.synchronize()
            stats = pfe.pfe_get_stats(ctx)
            V = torch.empty((max(nf, 1), n), dtype=torch.float64, device="cuda")
            lam, _, res = pfe.pfe_get_eigenpairs(ctx, n, nf, vecs_out=V) if nf else (np.zeros(0), V, np.zeros(0))
        finally:
            pfe.pfe_destroy(ctx)
        torch.cuda.synchronize()
        V = V[:nf]
        print(json.dumps({"form": form, "n_atoms": a.n_atoms, "seed": a.seed, "lo": a.lo, "hi": a.hi, "sliced": a.sliced,
                          "seconds": e0.elapsed_time(e1) / 1e3, "status": st, "n_found": nf,
                          "max_rel_residual": float(res.max() / lmax) if nf else 0.0, **stats}), flush=True)
        if ref is None:  # every later form is compared with this one as soon as it has finished
            ref = (form, lam, res, V, lmax)
            rows += [lam, res / lmax]
            hdr += ["lambda_" + form, "rel_residual_" + form]
            continue
        name0, lam0, _, V0, _ = ref
        out = {"compare": form, "with": name0, "n_found": [int(lam0.size), int(lam.size)]}
        if lam.size == lam0.size and lam.size > 0:
            rel = np.abs(lam - lam0) / np.abs(lam0)
            # sine of the largest principal angle between the two spaces: ||V - V0 (V0^T V)||_2
            P = V0 @ V.T
            D = V - P.T @ V0
            sin_max = float(torch.linalg.eigvalsh(D @ D.T).max().clamp(min=0).sqrt())
            out.update({"max_eig_rel_diff": float(rel.max()), "median_eig_rel_diff": float(np.median(rel)),
                        "subspace_sin_max": sin_max})
            rows += [lam, res / lmax, rel]
            hdr += ["lambda_" + form, "rel_residual_" + form, "eig_rel_diff_" + form]
            del P, D
        print(json.dumps(out), flush=True)
        del V
        torch.cuda.empty_cache()
    if a.out and rows and all(r.size == rows[0].size for r in rows):
        np.savetxt(a.out, np.column_stack(rows), delimiter=",", header=",".join(hdr), comments="", fmt="%.17g")


if __name__ == "__main__":
    main()
