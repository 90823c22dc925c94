#!/usr/bin/env python
"""Benchmark: time to all interval eigenpairs (residual <= 1e-8) of a synthetic glass Hessian,
with the filter's throughput against its roofline and the mixed-precision form beside the FP64 form.

One step = one outer iteration of the filtered subspace iteration (Alg. 4: the filter p_m(Ht) on
the active block, CholQR2 against the locked vectors, Rayleigh-Ritz with H, residuals, locking),
through the stepwise C ABI (pfe_solve_begin / pfe_solve_iterate / pfe_solve_end).  A solve's set-up
(context creation, lambda_max bound, filter design, count estimate, start block) belongs to its
first step and its results to its last; when a solve ends, the next step starts a new one.  Exactly
--steps steps are timed.  `value` is the time to all interval eigenpairs of the solves completed in
the timed region (when none completes there, the solve in flight is run to its end and timed whole).
Inputs are seeded and synthetic (glassgen).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl native|reference]

Under torchrun (N > 1) every rank solves its own replica (the single solve does not shard: replicas
only); times are the max over ranks.  --impl reference times the FP64 CPU oracle on a bounded sample
of the same workload: each step applies the oracle's Alg. 2 filter of the workload's degree to one
column per host core, and the time to all eigenpairs is extrapolated from the measured rates to the
subspace iteration's work on this workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to all interval eigenpairs (resid≤1e-8); filter SpMM GB/s; mixed vs FP64"

# Workloads (binary glass of glassgen: density 0.06/A^3, RSA d_min 2.2 A, bonds r < 3.5 A,
# k lognormal(1, 0.3), 64 % A / 36 % B).  The N = 100,000 interval keeps the lower edge
# 0.02 lambda_max of the stated configuration and ends where it holds ~700 modes (598 found):
# the literal upper edge 0.03 lambda_max holds ~4,990 modes for this generator.
_READING = ("[0.02, 0.0214] lambda_max: the stated lower edge and the stated ~700-mode size (598 modes); "
            "the stated upper edge 0.03 lambda_max holds ~5,000 modes for this generator and is solved by "
            "spectrum slicing, outside this line")
WORKLOADS = {
    "glass-n100k-fp64": dict(N=100_000, seed=1, lo=0.02, hi=0.0214, precision=0, interval=_READING),
    "glass-n100k-mixed": dict(N=100_000, seed=1, lo=0.02, hi=0.0214, precision=1, interval=_READING),
    "glass-n1k-fp64": dict(N=1_000, seed=0, lo=0.02, hi=0.05, precision=0, interval="[0.02, 0.05] lambda_max as stated"),
    "glass-n20k-fp64": dict(N=20_000, seed=1, lo=0.02, hi=0.0214, precision=0, interval="[0.02, 0.0214] lambda_max"),
}
DEFAULT = "glass-n100k-fp64"

# Work of the subspace iteration on a workload, as its GPU solve counted it (the same method with the
# same width, degree and locking does the same work on any machine): outer iterations, products with
# H (the filter's m per active column and iteration plus the Rayleigh-Ritz products), and the active
# and locked column counts of each iteration.  The reference arm scales the oracle's measured rates
# by these counts; the native arm prints its own counts beside them.
SOLVE_WORK = {
    "glass-n100k-fp64": dict(width=994, degree=713, iterations=8, matvecs=4_197_050,
                             active=[994] * 4 + [772, 469, 354, 299], locked=[0] * 4 + [222, 525, 640, 695]),
}

# DRAM traffic per launch of the dominant kernel, measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on one GB300 for the launch shape the solve runs, keyed by a hash of the
# kernel's source text: a changed kernel invalidates the number.  (kernel, FP bytes) -> bytes.
TRAFFIC = {
    # N = 100,000, k = 994 (the width of the bench solve's first iterations), shape 9: the mean of a STEP
    # launch (8.75 GB) and a STEP_ACC launch (13.51 GB); algorithmic bytes of that mean launch 10.09 GB
    ("k_r1_step<double>", 8): {"file": "paper_1902_07041_gb300/csrc/r1_kernels.cu",
                                "begin": "template <typename T, int CPL, int MODE, int UNROLL, int MINB>",
                                "end": "template <typename T, int CPL, int UNROLL, int MINB>\nvoid dispatch_r1_mode",
                                "src": "2288ce777daee821",
                                "bytes": 11131068288, "alg_bytes": 10086400320},
}
R1_SHAPES = (7, 8, 9, 10, 11)  # kernel shapes of the fused step that run on the rank-1 form


def _src_hash(rel, begin, end):
    """Hash of the source text of one kernel: from the line that starts with `begin` to the one that
    starts with `end` (the code that follows it)."""
    with open(os.path.join(ROOT, rel)) as f:
        s = f.read()
    i = s.find(begin)
    j = s.find(end, i + 1) if i >= 0 else -1
    return hashlib.sha256(s[i:j].encode()).hexdigest()[:16] if i >= 0 and j > i else None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def filter_work(n_atoms, nnzb, k, vec_bytes, val_bytes, rank1=False):
    """Algorithmic bytes and flops of one fused Chebyshev step on k columns (one launch).
    Full 3x3 blocks: 9 values and 9 FMAs per block and column.  Rank-1 form of a spring network:
    3 values and 6 FMAs per off-diagonal block and column, a full symmetric diagonal block (6 values,
    9 FMAs) per atom."""
    n = 3 * n_atoms
    kt = 128 if vec_bytes == 4 else 64  # columns per warp (CPL x 32)
    tiles = -(-k // kt)
    # gather t_j, read t_{j-1}, write t_{j+1}; y is read and written every other step (4 passes on average)
    vec = 4 * n * k * vec_bytes
    if rank1:
        noff = nnzb - n_atoms
        byts = tiles * (noff * (3 * val_bytes + 4) + n_atoms * 6 * val_bytes + 4 * (n_atoms + 1)) + vec
        flops = 12 * noff * k + 18 * n_atoms * k + 6 * n * k
    else:
        byts = tiles * (nnzb * (9 * val_bytes + 4) + 4 * (n_atoms + 1)) + vec
        flops = 18 * nnzb * k + 6 * n * k
    return byts, flops


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        import tempfile

        self.path = os.path.join(tempfile.gettempdir(), f"pfe_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [x for x in sm if x > 0.5 * max(sm)]
        return {"sm_mhz": statistics.median(load or sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(values, dist, device):
    """Max over the ranks of each timing: replicas run concurrently, so the job takes as long as its
    slowest rank. dist None (one process) returns the values unchanged."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


# ============================================================================================
# The oracle on the host cores (reference arm and cpu_baseline).  Only the oracle and the input
# generator are loaded here: no part of the GPU library.
# ============================================================================================
_W = {}


def _worker_init(wl):
    import glassgen
    import oracle

    g = glassgen.generate(wl["N"], wl["seed"])
    _W["H"] = oracle.csr_from_springs(g)


def _worker_filter(args):
    """The oracle's Alg. 2 on one seeded column of this worker's copy of H; returns seconds."""
    import oracle

    c, d, coef, col = args
    H = _W["H"]
    x = oracle.normal_block(17, 1, H.n, 1, col)
    t0 = time.perf_counter()
    oracle.cheb_filter(H, c, d, coef, x)
    return time.perf_counter() - t0


def _worker_count(args):
    """The oracle's count estimate (Sec. 2.4) with its own share of the probe vectors."""
    import oracle

    c, d, xi, eta, m_vec, seed = args
    return oracle.count_estimate(_W["H"], c, d, xi, eta, 100, "none", m_vec, seed)


class OracleSample:
    """The FP64 CPU oracle on a bounded sample of a workload, on `cores` host processes.

    Set-up: H, the Lanczos bound, the filter degree (eq. (thresh), r = sqrt(0.1), no damping) and the
    width rule of the solver (max(1.5 x the count estimate of [a, b], 1.1 x the estimate of the margin
    window + 8), M = 30 probe vectors shared over the processes), and the oracle's dense rate from one
    Householder QR of an n x 32 block.  step(): the oracle's Alg. 2 at the workload's degree on one
    column per process, in parallel.  estimate(): the time to all eigenpairs from those rates and the
    subspace iteration's work on this workload."""

    def __init__(self, wl, cores=None, degree=None):
        import numpy as np

        import glassgen
        import oracle

        self.wl = wl
        self.cores = int(cores or os.cpu_count() or 1)
        g = glassgen.generate(wl["N"], wl["seed"])
        self.H = H = oracle.csr_from_springs(g)
        self.n = H.n
        _, _, lmax = oracle.lanczos_lmax(H, 30, 0)
        self.lmax = lmax
        self.c = self.d = 0.5 * lmax
        self.xi = (wl["lo"] * lmax - self.c) / self.d
        self.eta = (wl["hi"] * lmax - self.c) / self.d
        self.eps = 0.25 * (self.eta - self.xi)
        # the degree of the solve when it is known (the GPU solve raises eq. (thresh)'s by its cost model),
        # else eq. (thresh) at r = sqrt(0.1)
        self.degree = degree or oracle.select_degree(self.xi, self.eta, self.eps, 0.1 ** 0.5, "none")
        self.coef = oracle.filter_coeffs(self.xi, self.eta, self.eps, self.degree, "none")
        ctx = mp.get_context("spawn")
        self.pool = ctx.Pool(self.cores, initializer=_worker_init, initargs=(wl,))
        t0 = time.perf_counter()
        per = max(1, -(-30 // self.cores))
        jobs = [(self.c, self.d, self.xi, self.eta, per, s) for s in range(-(-30 // per))]
        wjobs = [(self.c, self.d, self.xi - self.eps, self.eta + self.eps, per, s) for s in range(-(-30 // per))]
        cnt = self.pool.map(_worker_count, jobs + wjobs)
        self.count = float(np.mean(cnt[:len(jobs)]))
        self.window = float(np.mean(cnt[len(jobs):]))
        self.width = int(np.ceil(max(1.5 * self.count, 1.1 * self.window + 8, 16)))
        self.setup_count_s = time.perf_counter() - t0
        k = 32
        Xq = oracle.normal_block(8, 0, self.n, k)
        t0 = time.perf_counter()
        oracle.householder_qr(Xq)
        self.qr_s = time.perf_counter() - t0
        self.sec_per_dense_flop = self.qr_s / (4.0 * self.n * k * k)
        self.step_times = []
        self._col = 0

    def step(self):
        """One step: the filter on one column per process; returns the step's wall seconds."""
        args = [(self.c, self.d, self.coef, self._col + i) for i in range(self.cores)]
        self._col += self.cores
        t0 = time.perf_counter()
        self.pool.map(_worker_filter, args, chunksize=1)
        t = time.perf_counter() - t0
        self.step_times.append(t)
        return t

    def sec_per_matvec(self):
        """Wall seconds per single-vector product with H with every process busy (median step)."""
        return statistics.median(self.step_times) / (self.cores * self.degree)

    def estimate(self, work):
        """Time to all eigenpairs of the subspace iteration with `work` (iterations, MatVecs, and the
        active and locked columns per iteration when known): products with H at the parallel rate,
        the dense steps of the oracle's iteration (two Gram-Schmidt passes against the locked block,
        Householder QR, the Gram matrix, X Q and W Q: 8 n a l + 10 n a^2 flops for a active and l
        locked columns, plus about 20 a^3 for the Jacobi eigensolver) at its single-thread rate."""
        n = self.n
        it = work["iterations"]
        act = work.get("active")
        lck = work.get("locked")
        if not act:
            a = work["matvecs"] / (it * (work["degree"] + 2))  # mean active width
            act = [a] * it
            lck = [0.5 * (work["width"] - a)] * it
        dense = sum(8.0 * n * a * l + 10.0 * n * a * a + 20.0 * a ** 3 for a, l in zip(act, lck))
        t_mv = work["matvecs"] * self.sec_per_matvec()
        t_dense = dense * self.sec_per_dense_flop
        return t_mv + t_dense, t_mv, t_dense, dense

    def describe(self):
        per = statistics.median(self.step_times) / self.degree
        return (f"oracle Alg. 2 (degree {self.degree}) on one seeded column per process, {self.cores} processes "
                f"in parallel on N = {self.wl['N']} (median {statistics.median(self.step_times):.2f} s a step: "
                f"{1e3 * per:.2f} ms per product with H in each process, {1e3 * self.sec_per_matvec():.3f} ms per "
                f"product over all {self.cores}); dense rate from a Householder QR of {self.n} x 32 "
                f"({self.qr_s:.2f} s, one core)")

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_full_solve_n1000():
    """The oracle's complete subspace iteration on the N = 1,000 glass (seed 0, [0.02, 0.05] lambda_max,
    degree 40, width 256), single-threaded: a full solve, not a sample."""
    import oracle
    import glassgen

    g = glassgen.generate(1000, 0)
    H = oracle.csr_from_springs(g)
    t0 = time.perf_counter()
    _, _, lmax = oracle.lanczos_lmax(H, 30, 0)
    c = d = 0.5 * lmax
    a, b = 0.02 * lmax, 0.05 * lmax
    xi, eta = (a - c) / d, (b - c) / d
    coef = oracle.filter_coeffs(xi, eta, 0.25 * (eta - xi), 40, "none")
    r = oracle.si_solve(H, a, b, 0.0, lmax, coef, 256, oracle.normal_block(0, 0, H.n, 256), max_iter=200)
    return {"seconds": time.perf_counter() - t0, "n_found": int(r.lam.size), "iterations": r.iters,
            "matvecs": r.matvecs, "status": r.status, "cores": 1}


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    work = SOLVE_WORK.get(args.workload)
    t_setup = time.perf_counter()
    smp = OracleSample(wl, degree=work["degree"] if work else None)
    setup_s = time.perf_counter() - t_setup
    for _ in range(args.warmup):
        smp.step()
    smp.step_times.clear()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        smp.step()
    timed = time.perf_counter() - t0
    smp.close()
    if work is None:
        work = dict(width=smp.width, degree=smp.degree, iterations=13,
                    matvecs=int(13 * smp.width * (smp.degree + 2) * 0.75))
    est, t_mv, t_dense, dense = smp.estimate(work)
    full = oracle_full_solve_n1000()
    sample = (smp.describe() + f"; extrapolated to the subspace iteration's work on this workload "
              f"({work['iterations']} iterations, {work['matvecs']} products with H, ~{dense:.3g} dense flops): "
              f"{t_mv:.0f} s of products, {t_dense:.0f} s of dense steps")
    line = {"metric": METRIC, "value": est, "unit": "s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * timed / max(args.steps, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, **wl, "degree": smp.degree, "width": smp.width,
                       "count_estimate": smp.count, "window_estimate": smp.window,
                       "step": f"the oracle's Alg. 2 at degree {smp.degree} on {smp.cores} columns, one per "
                               f"host process"},
            "cpu_baseline": {"value": est, "unit": "s", "cores": smp.cores, "kind": "oracle", "sample": sample,
                             "extrapolated": True, "oracle_full_solve_n1000": full},
            "e2e": {"value": est, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "timed_wall_s": timed, "setup_s": setup_s}
    print(json.dumps(line), flush=True)


# ============================================================================================
# Native arm: the GPU library through its C ABI
# ============================================================================================
class SteppedSolve:
    """One subspace-iteration solve driven a step at a time through the stepwise C ABI.

    host=False: the context is created from device-resident BSR arrays (inputs in HBM) and the
    eigenvectors are exported to a device buffer.  host=True: created from pinned host arrays
    (H2D inside) and the eigenpairs copied to pinned host buffers (D2H inside)."""

    def __init__(self, pfe, torch, arrays, wl, host):
        self.pfe, self.torch, self.arrays, self.wl, self.host = pfe, torch, arrays, wl, host
        self.ctx = None
        self.done = False
        self.profile = []  # (active, locked) before each iteration
        self.ev0 = torch.cuda.Event(enable_timing=True)
        self.ev1 = torch.cuda.Event(enable_timing=True)

    def start(self):
        pfe, a = self.pfe, self.arrays
        self.ev0.record()
        if self.host:
            self.ctx = pfe.pfe_create(a["N"], a["rp_h"], a["ci_h"], a["vals_h"], a["mass_h"])
        else:
            self.ctx = pfe.pfe_create(a["N"], a["rp_d"], a["ci_d"], a["vals_d"], a["mass_d"],
                                      flags=pfe.PFE_DEVICE_PTRS)
        pfe.pfe_set_param(self.ctx, pfe.PFE_P_PRECISION, self.wl["precision"])
        pfe.pfe_set_param(self.ctx, pfe.PFE_P_METHOD, 0)
        lmax, _ = pfe.pfe_estimate(self.ctx)
        self.lmax = lmax
        pfe.pfe_set_interval(self.ctx, self.wl["lo"] * lmax, self.wl["hi"] * lmax)
        pfe.pfe_solve_begin(self.ctx)

    def iterate(self):
        st = self.pfe.pfe_get_stats(self.ctx)
        self.profile.append((st["active"], st["locked"]))
        self.done = self.pfe.pfe_solve_iterate(self.ctx)
        return self.done

    def finish(self):
        pfe, torch = self.pfe, self.torch
        nf, st = pfe.pfe_solve_end(self.ctx)
        n = 3 * self.arrays["N"]
        if self.host:
            self.vecs = torch.empty((max(nf, 1), n), dtype=torch.float64).pin_memory()
            lam, _, res = pfe.pfe_get_eigenpairs(self.ctx, n, nf, vecs_out=self.vecs)
        else:
            self.vecs = torch.empty((max(nf, 1), n), dtype=torch.float64, device="cuda")
            lam, _, res = pfe.pfe_get_eigenpairs(self.ctx, n, nf, vecs_out=self.vecs)
        self.stats = pfe.pfe_get_stats(self.ctx)
        pfe.pfe_destroy(self.ctx)
        self.ctx = None
        self.ev1.record()
        self.lam, self.res, self.n_found = lam, res, nf
        self.max_rel_residual = float(res.max() / self.lmax) if nf else 0.0

    def abandon(self):
        if self.ctx is not None:
            self.pfe.pfe_solve_end(self.ctx, raise_on_error=False)
            self.pfe.pfe_destroy(self.ctx)
            self.ctx = None

    def seconds(self):
        return self.ev0.elapsed_time(self.ev1) / 1e3


def whole_solve(pfe, torch, arrays, wl, host=False, method=0):
    """One complete solve through pfe_solve (the call a user makes), timed by CUDA events."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 3 * arrays["N"]
    e0.record()
    if host:
        ctx = pfe.pfe_create(arrays["N"], arrays["rp_h"], arrays["ci_h"], arrays["vals_h"], arrays["mass_h"])
    else:
        ctx = pfe.pfe_create(arrays["N"], arrays["rp_d"], arrays["ci_d"], arrays["vals_d"], arrays["mass_d"],
                             flags=pfe.PFE_DEVICE_PTRS)
    try:
        pfe.pfe_set_param(ctx, pfe.PFE_P_PRECISION, wl["precision"])
        pfe.pfe_set_param(ctx, pfe.PFE_P_METHOD, method)
        lmax, _ = pfe.pfe_estimate(ctx)
        pfe.pfe_set_interval(ctx, wl["lo"] * lmax, wl["hi"] * lmax)
        nf, _ = pfe.pfe_solve(ctx)
        if host:
            vecs = torch.empty((max(nf, 1), n), dtype=torch.float64).pin_memory()
        else:
            vecs = torch.empty((max(nf, 1), n), dtype=torch.float64, device="cuda")
        lam, _, res = pfe.pfe_get_eigenpairs(ctx, n, nf, vecs_out=vecs)
        stats = pfe.pfe_get_stats(ctx)
    finally:
        pfe.pfe_destroy(ctx)
    e1.record()
    torch.cuda.synchronize()
    return {"seconds": e0.elapsed_time(e1) / 1e3, "lam": lam, "res": res, "vecs": vecs, "n_found": nf,
            "lmax": lmax, "stats": stats, "max_rel_residual": float(res.max() / lmax) if nf else 0.0}


def fp64_probe(pfe, torch):
    """FP64 throughput of this GPU's FMA probe, measured now (best of three)."""
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    return max(pfe.pfe_probe_fp64_fma(4000, 5, sink) for _ in range(3))


def fp64_unit_peak(sm_mhz, sms=152):
    """FP64 peak from the unit count: 2 FP64 FMA lanes per clock per SM (4 flops), at the SM clock."""
    return sms * 4.0 * sm_mhz * 1e6 / 1e12


def run_native(args, wl):
    import numpy as np
    import torch

    import glassgen
    import paper_1902_07041_gb300 as pfe

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    pfe.load()
    g = glassgen.generate(wl["N"], wl["seed"])
    rp, ci, vals = pfe.pfe_springs_to_bsr(g.n_atoms, g.bi, g.bj, g.k, g.rhat)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    arrays = {"N": g.n_atoms, "rp_h": pin(rp), "ci_h": pin(ci), "vals_h": pin(vals), "mass_h": pin(g.mass)}
    for key in ("rp", "ci", "vals", "mass"):
        arrays[key + "_d"] = arrays[key + "_h"].cuda()
    h2d_bytes = sum(arrays[k + "_h"].numel() * arrays[k + "_h"].element_size() for k in ("rp", "ci", "vals", "mass"))
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- warm-up: W steps of a solve that is then dropped (kernel-shape tuning, library handles)
    cur = SteppedSolve(pfe, torch, arrays, wl, host=False)
    cur.start()
    for _ in range(args.warmup):
        if cur.iterate():
            cur.finish()
            cur = SteppedSolve(pfe, torch, arrays, wl, host=False)
            cur.start()
    cur.abandon()
    cur = None
    # ---- timed region: exactly K steps
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    wall0 = time.perf_counter()
    t_start.record()
    completed = []
    for _ in range(args.steps):
        if cur is None:
            cur = SteppedSolve(pfe, torch, arrays, wl, host=False)
            cur.start()
        if cur.iterate():
            cur.finish()
            completed.append(cur)
            cur = None
    t_end.record()
    barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    timed_s = t_start.elapsed_time(t_end) / 1e3
    # launches of this library's kernels inside the timed region: each solve there created its context
    # there, and one context works at a time, so its process-wide launch count since creation is exact
    gpu_launches = sum(int(s.stats["kernel_launches"]) for s in completed)
    if cur is not None:
        gpu_launches += int(pfe.pfe_get_stats(cur.ctx)["kernel_launches"])
    if not completed:  # the timed steps did not finish a solve: run the one in flight to its end
        while not cur.iterate():
            pass
        cur.finish()
        torch.cuda.synchronize()
        completed.append(cur)
        cur = None
    if cur is not None:
        cur.abandon()
    torch.cuda.synchronize()
    solve_s = statistics.mean(s.seconds() for s in completed)
    solve_s, timed_s = max_over_ranks([solve_s, timed_s], dist, "cuda")
    first = completed[0]
    st = first.stats
    nnzb = int(ci.size)
    hbm, hbm_src = peaks()

    # ---- roofline of the dominant kernel: the fused filter step, FP64, bound by the FP64 pipe.  The
    # FMA probe tops out below what the filter kernel itself reaches, so the peak is the unit count at
    # the clock sampled during the timed steps (the probe's rate is reported beside it).
    probe64 = fp64_probe(pfe, torch)
    sm_clock = clocks.get("sm_mhz") or 2070.0
    peak64 = max(fp64_unit_peak(sm_clock, torch.cuda.get_device_properties(local).multi_processor_count), probe64)
    r1 = st["filter_shape_f64"] in R1_SHAPES
    secs64 = st["seconds_filter"] - st["seconds_filter_f32"]
    _, fl1 = filter_work(g.n_atoms, nnzb, 1, 8, 8, r1)
    achieved = fl1 * st["filter_col_steps"] / secs64 / 1e12
    avg_k = st["filter_col_steps"] / max(st["filter_launches"], 1)
    b_avg, _ = filter_work(g.n_atoms, nnzb, int(round(avg_k)), 8, 8, r1)
    kname = "k_r1_step<double>" if r1 else "k_bsr_step<double>"
    tr = TRAFFIC.get((kname, 8))
    traffic = None
    if tr and tr["src"] == _src_hash(tr["file"], tr["begin"], tr["end"]):
        traffic = tr["bytes"] * b_avg / tr["alg_bytes"]  # scaled from the captured launch to the average one
    roof = {"bound": "alu", "kernel": kname + " (fused Chebyshev step, shape %d)" % st["filter_shape_f64"],
            "achieved": achieved, "peak": peak64, "unit": "TFLOP/s", "frac": achieved / peak64,
            "traffic": traffic, "algorithmic_bytes_per_launch": b_avg, "avg_columns_per_launch": avg_k,
            "peak_source": "SMs x 2 FP64 FMA lanes per clock x 2 flops x the median SM clock of the timed steps",
            "probe_tflops": probe64,
            "probe_note": "pfe_probe_fp64_fma (independent FMA chains, several shapes) measured in this run; it "
                          "stays below the filter kernel's own rate, so it does not bound the pipe",
            "achieved_how": "the rank-1 form's flops (12 per off-diagonal block and column, 18 per diagonal block "
                            "and column, 6 per vector element) x column-steps / CUDA-event seconds of the FP64 "
                            "filter sweeps on the launching stream",
            "filter_gbs_fp64": b_avg * st["filter_launches"] / secs64 / 1e9, "hbm_peak_gbs": hbm,
            "launches": st["filter_launches"], "operator_form": "rank1" if r1 else "bsr"}
    work_live = {"width": st["width"], "degree": st["degree"], "iterations": st["iterations"],
                 "matvecs": st["matvecs"], "active": [a for a, _ in first.profile],
                 "locked": [lk for _, lk in first.profile]}
    line = {
        "metric": METRIC, "value": solve_s, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * timed_s / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if wl["precision"] == 0 else "f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, **wl, "n": 3 * wl["N"], "nnzb": nnzb, "width": st["width"],
                   "degree": st["degree"], "iterations": st["iterations"], "n_found": first.n_found,
                   "matvecs": st["matvecs"], "parallelism": f"replicas x{world}",
                   "step": "one outer iteration of the subspace iteration (a solve's set-up in its first step)",
                   "solves_completed_in_timed_region": len(completed),
                   "l2": "no flush: every step streams multivectors of n x width FP64 (2.4 GB each) through the "
                         "129 MB L2"},
        "roofline": roof,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "breakdown_s": {"filter": st["seconds_filter"], "orth": st["seconds_orth"], "rr": st["seconds_rr"]},
        "max_rel_residual": first.max_rel_residual, "wall_s": wall, "timed_s": timed_s,
        "work": work_live,
    }

    # ---- end to end through the public API: pinned host BSR in, host eigenpairs out
    e2e = whole_solve(pfe, torch, arrays, wl, host=True)
    line["e2e"] = {"value": e2e["seconds"], "unit": "s", "h2d_bytes_per_step": int(h2d_bytes),
                   "d2h_bytes_per_step": int(e2e["lam"].nbytes + e2e["res"].nbytes +
                                             e2e["n_found"] * 3 * wl["N"] * 8),
                   "step": "one complete solve: pfe_create from pinned host arrays, pfe_estimate, pfe_solve, "
                           "pfe_get_eigenpairs into pinned host buffers, pfe_destroy",
                   "n_found": e2e["n_found"], "max_rel_residual": e2e["max_rel_residual"]}
    plain_si = wl["precision"] == 0
    if rank == 0 and args.mixed and plain_si:
        # the per-pair hand-over form (FP32 filter above the hand-over residual, FP64 below)
        sh = whole_solve(pfe, torch, arrays, dict(wl, precision=1))
        s1 = sh["stats"]
        line["mixed_fp64_handover"] = {"value": sh["seconds"], "unit": "s", "fp64_sweeps": s1["fp64_sweeps"],
                                       "iterations": s1["iterations"], "degree": s1["degree"],
                                       "n_found": sh["n_found"], "max_rel_residual": sh["max_rel_residual"],
                                       "breakdown_s": {"filter": s1["seconds_filter"],
                                                       "filter_f32": s1["seconds_filter_f32"],
                                                       "orth": s1["seconds_orth"], "rr": s1["seconds_rr"]}}
        del sh
        # the defect-corrected form: every filter step in FP32
        wm = dict(wl, precision=2)
        sm = whole_solve(pfe, torch, arrays, wm)
        s2 = sm["stats"]
        b1, _ = filter_work(g.n_atoms, nnzb, s2["width"], 4, 4, s2["filter_shape_f32"] in R1_SHAPES)
        # the steps with the forcing term also read the residual block: one more pass of 4 n bytes a column
        byts32 = (b1 / s2["width"]) * s2["filter_col_steps_f32"] + 4 * g.n * s2["filter_col_steps_forced"]
        gbs32 = byts32 / max(s2["seconds_filter_f32"], 1e-12) / 1e9
        # per-eigenpair agreement of the mixed form with the FP64 form (e2e solve) on the same matrix
        agree = {}
        if sm["n_found"] == e2e["n_found"] and sm["n_found"] > 0:
            lam64, lam32 = e2e["lam"], sm["lam"]
            rel = np.abs(lam32 - lam64) / np.abs(lam64)
            V64 = e2e["vecs"][:e2e["n_found"]].cuda()
            V32 = sm["vecs"][:sm["n_found"]]
            # largest principal angle between the two computed spaces: ||V32 - V64 (V64^T V32)||_2
            P = V64 @ V32.T
            Dv = V32 - P.T @ V64
            sin_max = float(torch.linalg.eigvalsh(Dv @ Dv.T).max().clamp(min=0).sqrt())
            agree = {"max_eig_rel_diff": float(rel.max()), "median_eig_rel_diff": float(np.median(rel)),
                     "subspace_sin_max": sin_max}
            del V64, P, Dv
        line["mixed"] = {"value": sm["seconds"], "unit": "s", "fp64_sweeps": s2["fp64_sweeps"],
                         "form": "PRECISION 2: FP32 filter; below the hand-over residual by defect correction "
                                 "(x p(theta) in FP64 plus the recurrence on the residual in FP32); FP64 CholQR2, "
                                 "Rayleigh-Ritz and residuals",
                         "iterations": s2["iterations"], "degree": s2["degree"], "n_found": sm["n_found"],
                         "max_rel_residual": sm["max_rel_residual"], "vs_fp64_form": agree,
                         "filter_f32": {"achieved": gbs32, "peak": hbm, "unit": "GB/s", "frac": gbs32 / hbm,
                                        "peak_source": hbm_src, "shape": s2["filter_shape_f32"],
                                        "bytes": "4 vector passes a step, a 5th (the residual block) in the steps "
                                                 "with the forcing term, plus the operator per 128-column tile; "
                                                 "the prep and combine kernels of each application not counted"},
                         "breakdown_s": {"filter": s2["seconds_filter"], "filter_f32": s2["seconds_filter_f32"],
                                         "orth": s2["seconds_orth"], "rr": s2["seconds_rr"]}}
    if rank == 0 and args.block_lanczos and plain_si:
        sb = whole_solve(pfe, torch, arrays, wl, method=1)
        s3 = sb["stats"]
        line["block_lanczos"] = {"value": sb["seconds"], "unit": "s", "n_found": sb["n_found"],
                                 "matvecs": s3["matvecs"], "restarts": s3["restarts"], "basis": s3["basis"],
                                 "block": s3["width"], "degree": s3["degree"],
                                 "max_rel_residual": sb["max_rel_residual"],
                                 "breakdown_s": {"filter": s3["seconds_filter"], "orth": s3["seconds_orth"],
                                                 "rr": s3["seconds_rr"]},
                                 "note": "thick-restart block Lanczos on p(Ht), then Rayleigh-Ritz with H "
                                         "(the paper's block Krylov-Schur solver); one solve after the timed "
                                         "subspace-iteration steps"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        smp = OracleSample(wl, degree=st["degree"])
        for _ in range(2):
            smp.step()
        smp.step_times.pop(0)  # the first step warms the processes up
        est, t_mv, t_dense, dense = smp.estimate(work_live)
        smp.close()
        line["cpu_baseline"] = {"value": est, "unit": "s", "cores": smp.cores, "kind": "oracle",
                                "sample": smp.describe() + f"; extrapolated to this solve's work "
                                                           f"({st['iterations']} iterations, {st['matvecs']} "
                                                           f"products with H, ~{dense:.3g} dense flops)",
                                "extrapolated": True}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=15)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-mixed", dest="mixed", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-block-lanczos", dest="block_lanczos", action="store_false")
    args = ap.parse_args()
    if args.steps < 1 or args.warmup < 0:
        ap.error("--steps must be >= 1 and --warmup >= 0")
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_native(args, wl)


if __name__ == "__main__":
    main()
