"""The multi-process (replica) host logic of bench.py on CPU with gloo,
world size 2: every rank gets the slowest rank's time and the whole-job
rate; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t = bench.replica_time(1.0 + rank, ws, "cpu")            # rank 1 is the slow one
        r = bench.replica_rate(4, 1.0 + 0.5 * rank, ws, "cpu")
        ws_env, rank_env, local_env = bench._dist()
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{t} {r} {ws_env} {rank_env}")
    finally:
        dist.destroy_process_group()


def test_replica_time_and_rate_gloo_world_size_2(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        t, r, ws_env, rank_env = open(tmp_path / f"r{rank}.txt").read().split()
        assert float(t) == 2.0                                     # max over ranks, on every rank
        assert abs(float(r) - 2 * 4 / 1.5) < 1e-12                 # units of all ranks / slowest time
        assert int(ws_env) == 2 and int(rank_env) == rank


def test_replica_logic_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_time(3.0, 1, "cpu") == 3.0
    assert bench.replica_rate(5, 2.0, 1, "cpu") == 2.5


def test_reference_arm_runs_on_rank_0_only():
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
