"""Multi-rank logic of the benchmark on CPU (gloo, world size 2).

The estimator shards by independent pairs: every rank runs its own stream
with no collective on the data path, and the job's time is the slowest
rank's.  These tests run the benchmark's reduction helpers in two gloo
processes, and the reference arm under torchrun with two ranks (rank 0
alone works and prints; rank 1 exits 0 without output).
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local_seconds = [2.0, 3.5][rank]                     # rank 1 is the slow one
    worst = bench.reduce_max(local_seconds, dist, "cpu")
    rate = bench.whole_job_rate(1000, ws, worst)
    dist.barrier()
    q.put((rank, worst, rate))
    dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time_and_units_add_up():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, worst, rate in res:
        assert worst == 3.5
        assert rate == pytest.approx(2 * 1000 / 3.5)


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_max(1.25) == 1.25
    assert bench.whole_job_rate(30, 1, 2.0) == 15.0


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_two_ranks():
    env = dict(os.environ, OMP_NUM_THREADS="4")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == 4  # the threads the oracle ran on (OMP_NUM_THREADS above)
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # the same workload config as the GPU arm's line at this rank count
    import bench
    cfg = dict(d["config"])
    cfg.pop("step")
    assert cfg == bench.workload_config(bench.FRAMES1, 2)
