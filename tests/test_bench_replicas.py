"""The N > 1 path of bench.py on CPU: two gloo ranks (world size 2).

`bench.py --gpus N` runs replicas only: every rank solves its own copy and
the process group is used for the barriers around the timed region and for
the maximum per-solve time over ranks.  The reference arm runs on rank 0
alone; the other ranks exit 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    reps = bench.Replicas("gloo")
    assert (reps.world, reps.rank, reps.local) == (world, rank, rank)
    reps.barrier()
    # per-rank "solve times": rank r reports (10 + r, 5 - r)
    got = reps.max([10.0 + rank, 5.0 - rank], "cpu")
    reps.barrier()
    reps.close()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(got, f)


def test_replicas_max_over_ranks_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        got = json.load(open(tmp_path / f"rank{r}.json"))
        assert got == [10.0 + world - 1, 5.0], got


def test_replicas_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        reps = bench.Replicas("gloo")
        assert reps.world == 1 and reps.max([3.0, 4.0], "cpu") == [3.0, 4.0]
        reps.barrier()
        reps.close()
    finally:
        os.environ.update(env)


def test_reference_arm_nonzero_rank_exits_without_work():
    """Under torchrun the reference arm's rank 1 prints nothing and exits 0
    (it never touches the oracle)."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
