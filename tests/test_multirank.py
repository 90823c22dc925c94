"""The multi-process path of bench.py on CPU: two gloo ranks (replicas), the max-over-ranks timing,
and the reference arm's rank handling. No GPU is used."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "measured" (r + 1) s for the solve and 10 r s end to end
        res = bench.max_over_ranks([rank + 1.0, 10.0 * rank], dist, "cpu")
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        assert out[0] == [2.0, 10.0] and out[1] == [2.0, 10.0]


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([3.0, 4.0], None, "cpu") == [3.0, 4.0]


def test_reference_arm_nonzero_rank_does_no_work():
    """Under torchrun only rank 0 runs and prints the oracle's line; the others exit 0 at once."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "glass-n1k-fp64"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_runs_the_oracle_only():
    """The reference arm on a small workload: one JSON line whose per-step time covers the timed
    steps, measured on the host cores with the oracle; the GPU library is never loaded."""
    code = ("import runpy, sys; sys.argv = ['bench.py', '--impl', 'reference', '--steps', '2', '--warmup', '1', "
            "'--workload', 'glass-n1k-fp64']; runpy.run_path('bench.py', run_name='__main__'); "
            "maps = open('/proc/self/maps').read(); print('LIBPFE_LOADED' if 'libpfe' in maps else 'LIBPFE_ABSENT')")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert lines[-1] == "LIBPFE_ABSENT"
    import json

    rec = json.loads(lines[-2])
    assert rec["impl"] == "reference" and rec["steps"] == 2 and rec["warmup"] == 1
    assert rec["unit"] == "s" and rec["higher_is_better"] is False and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1
    assert rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["ms_per_step"] * rec["steps"] <= 1e3 * rec["timed_wall_s"] * 1.001 + 1.0
    full = rec["cpu_baseline"]["oracle_full_solve_n1000"]
    assert full["status"] == 0 and full["n_found"] == 144  # the exact count of [0.02, 0.05] lambda_max


def test_recorded_traffic_matches_the_current_kernel_source():
    """roofline.traffic is only reported while the captured kernel's source text is unchanged: every
    recorded DRAM capture must still hash to the kernel in the tree, and its algorithmic bytes must
    be those of the launch model for the captured shape (N = 100,000, nnzb 1,128,572, k = 994)."""
    sys.path.insert(0, ROOT)
    import bench

    for (kernel, fp_bytes), tr in bench.TRAFFIC.items():
        assert bench._src_hash(tr["file"], tr["begin"], tr["end"]) == tr["src"], kernel
        assert tr["bytes"] >= tr["alg_bytes"] > 0
    tr = bench.TRAFFIC[("k_r1_step<double>", 8)]
    assert bench.filter_work(100_000, 1_128_572, 994, 8, 8, rank1=True)[0] == tr["alg_bytes"]


def test_clock_sampler_reads_median_under_load_and_throttle_reasons(tmp_path):
    """The clocks field of the bench line from nvidia-smi's CSV (no GPU: the sampler's output file is
    written here and its process is a stand-in)."""
    sys.path.insert(0, ROOT)
    import bench

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    rows = ["0, 120, 2070, 90.1, 0x0, Not Active, Not Active, Not Active, Not Active"]  # idle before the load
    rows += ["0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active"] * 5
    rows += ["0, 1980, 2070, 1398.0, 0x4, Not Active, Not Active, Not Active, Active"]
    rows += ["garbage line", "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    with open(cs.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    cs.fh = open(cs.path)
    cs.proc = _Done()
    got = cs.stop()
    assert got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"]
    assert got["samples"] == 7
    off = bench.ClockSampler(0)
    assert off.stop()["reasons"] == ["nvidia-smi unavailable"]
