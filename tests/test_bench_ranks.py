"""The multi-rank host logic of bench.py on CPU: world size 2 over gloo.

Every GPU runs an independent replica (images are independent and nothing is
exchanged), so the only cross-rank steps are the barriers around the timed
region, the maximum of the step time over the ranks and the whole-job rate.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench._dist()
        bench._barrier(ws)
        # the slower replica (rank 1) sets the job's time
        t = bench._max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")
        rate = bench._job_rate(ws, 1000.0, t)
        bench._barrier(ws)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{got_ws} {got_rank} {got_local} {t!r} {rate!r}\n")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(ws)]
    for r, row in enumerate(rows):
        assert row[:3] == [str(ws), str(r), str(r)]
        # both ranks see the slowest rank's time and the same whole-job rate:
        # 2 replicas x 1000 units in 15 s
        assert float(row[3]) == 15.0
        assert float(row[4]) == pytest.approx(2 * 1000.0 / 15.0, rel=0, abs=1e-12)


def test_one_rank_needs_no_process_group():
    import bench

    assert bench._max_over_ranks(3.25, 1, "cpu") == 3.25
    assert bench._job_rate(1, 100.0, 4.0) == 25.0
    bench._barrier(1)  # no process group: nothing to wait for


def test_reference_arm_other_ranks_exit_without_work():
    # under torchrun only rank 0 times the oracle; the others leave at once
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
