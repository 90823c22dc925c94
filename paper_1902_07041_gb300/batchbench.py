"""Time the batched solve (pfe_solve_batch) of many independent glass samples against solving
them one after another.

    python -m paper_1902_07041_gb300.batchbench --samples 48 --n-min 5000 --n-max 40000 --seed 3 \
        --lo 0.02 --hi 0.026 [--precision 1] [--solo]

Sample sizes are uniform integers in [n-min, n-max] (seeded); sample i uses glassgen sub-seed
SplitMix64(seed ^ i).  Each sample's interval is [lo, hi] times its own lambda_max bound.
Prints one JSON line with the batched wall time, the filter time and the per-sample counts.
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
    ap.add_argument("--samples", type=int, default=48)
    ap.add_argument("--n-min", type=int, default=5000)
    ap.add_argument("--n-max", type=int, default=40000)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--lo", type=float, default=0.02)
    ap.add_argument("--hi", type=float, default=0.026)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--solo", action="store_true", help="also time the samples solved one by one")
    ap.add_argument("--no-batch", action="store_true", help="with --solo: time only the one-by-one solves")
    ap.add_argument("--threads", type=int, default=0, help="host threads for the per-sample steps (0: automatic)")
    ap.add_argument("--method", type=int, default=0, help="0 subspace iteration (lockstep), 1 block Lanczos")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    sizes = glassgen.batch_sizes(a.samples, a.seed, a.n_min, a.n_max)
    problems = []
    for i, n in enumerate(sizes):
        g = glassgen.generate(n, glassgen.subseed(a.seed, i))
        problems.append((g, pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)))

    def make_all():  # every sample's context, set up (lambda_max bound, interval) outside the timed region
        ctxs = []
        for g, (rp, ci, vals) in problems:
            ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
            pfe.pfe_set_param(ctx, pfe.PFE_P_PRECISION, a.precision)
            pfe.pfe_set_param(ctx, pfe.PFE_P_BATCH_THREADS, a.threads)
            pfe.pfe_set_param(ctx, pfe.PFE_P_METHOD, a.method)
            lmax, _ = pfe.pfe_estimate(ctx)
            pfe.pfe_set_interval(ctx, a.lo * lmax, a.hi * lmax)
            ctxs.append(ctx)
        return ctxs

    out = {"samples": a.samples, "atoms_total": int(sum(sizes)), "precision": a.precision, "method": a.method}
    if not a.no_batch:
        ctxs = make_all()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nfs, st = pfe.pfe_solve_batch(ctxs)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        stats = [pfe.pfe_get_stats(c) for c in ctxs]
        for c in ctxs:
            pfe.pfe_destroy(c)
        out.update({"status": st, "batch_s": t_batch, "batch_filter_s": stats[0]["seconds_filter"],
                    "replays": stats[0]["batch_replays"], "modes_total": int(sum(nfs)),
                    "iterations_max": max(s["iterations"] for s in stats),
                    "matvecs_total": sum(s["matvecs"] for s in stats), "widths": [s["width"] for s in stats],
                    "n_found": nfs})
    if a.solo:
        # one sample at a time: set up like the batch (untimed), solve (timed), release its memory
        solo_s, solo = 0.0, []
        for g, (rp, ci, vals) in problems:
            ctx = pfe.pfe_create(g.n_atoms, rp, ci, vals, g.mass)
            try:
                pfe.pfe_set_param(ctx, pfe.PFE_P_PRECISION, a.precision)
                pfe.pfe_set_param(ctx, pfe.PFE_P_METHOD, a.method)
                lmax, _ = pfe.pfe_estimate(ctx)
                pfe.pfe_set_interval(ctx, a.lo * lmax, a.hi * lmax)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                solo.append(pfe.pfe_solve(ctx, raise_on_error=False))
                torch.cuda.synchronize()
                solo_s += time.perf_counter() - t0
            finally:
                pfe.pfe_destroy(ctx)
        out["solo_s"] = solo_s
        out["solo_status"] = max(s for _, s in solo)
        out["solo_modes_total"] = int(sum(nf for nf, _ in solo))
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
