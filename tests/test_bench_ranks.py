"""The multi-rank path of bench.py on the CPU: with N ranks every rank runs an
independent replica ensemble (its own seed, no collective on the data path);
the job's time is the slowest rank's, taken with one max all-reduce, and the
job's throughput counts the site updates of all ranks.  Two gloo ranks on
127.0.0.1 stand in for two GPUs; the reference arm works on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1 + r ms on the device and 10 - r s end to end
        got = bench.max_over_ranks(dist, [1.0 + rank, 10.0 - rank])
        q.put((rank, got, bench.replica_seed(rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank_and_distinct_replicas():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        results = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, got, _ in results:
        assert got == [2.0, 10.0], (rank, got)  # max of (1, 2) and of (10, 9) on every rank
    assert len({seed for _, _, seed in results}) == 2


def test_single_process_and_job_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, [3.0, 4.5]) == [3.0, 4.5]
    # 2 ranks x 1000 sites x 500 steps in 0.25 s
    assert bench.job_glups(1000, 500, 2, 0.25) == pytest.approx(1000 * 500 * 2 / 0.25 / 1e9)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_its_contract_line_on_rank_zero():
    """At N = 1 the reference arm times the oracle on the host cores and prints
    one JSON line with the metric of the GPU arm, its own CPU baseline and an
    end-to-end figure without host-device copies."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GLUPS"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    # the single-threaded rate of one process, at most the aggregate (within timing noise)
    assert 0 < cb["per_core"] <= 1.2 * cb["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("GKTL batched ensemble")
