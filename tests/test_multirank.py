"""The N > 1 path of bench.py on the CPU with the gloo backend (world size 2).

The chains are independent, so several GPUs are replicas only: each rank runs its own
chains and the ranks meet only to turn their timings and unit counts into whole-job
figures (the MAX of the times, the SUM of the units).  These tests cover that host
logic and the reference arm's launch under torchrun, where rank 0 alone runs.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r timed 1.5 + r ms and processed (r + 1, 10 (r + 1), 1) units
        t, units = bench.reduce_over_ranks(1.5 + rank, [rank + 1, 10 * (rank + 1), 1], dist, device="cpu")
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"t": t, "units": list(map(float, units))}, f)
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_takes_max_time_and_sums_units(tmp_path):
    world = 2
    tmp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        d = json.load(open(tmp_path / f"rank{r}.json"))
        assert d["t"] == 2.5
        assert d["units"] == [3.0, 30.0, 2.0]


def test_reduce_over_ranks_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    t, units = bench.reduce_over_ranks(3.25, [1.0, 2.0], None)
    assert t == 3.25 and np.array_equal(units, [1.0, 2.0])


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    """bench.py --impl reference at world size 2: one JSON line (rank 0), the same metric,
    unit and config keys as the GPU arm, exit status 0 on every rank."""
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-cores", "2"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["unit"] == "atom-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["parallelism"] == "replicas x2"
    assert d["config"]["workload"].startswith("LJ electrolyte 4000 ions")
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == 2
