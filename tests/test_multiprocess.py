"""The N > 1 path of bench.py on CPU: two ranks over gloo (the launch the
driver uses, torchrun-style environment variables, rendezvous on 127.0.0.1).
The path is replicas only -- nothing in the method exchanges data -- so what
is tested is the host logic around it: process-group set-up, the barrier, the
max-over-ranks time, the whole-job rate, and that ranks other than 0 of the
reference arm exit without work."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup()
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    slowest = bench.max_over_ranks(1.5 + rank, w)   # rank 1 is the slow one
    rate = bench.whole_job_rate(10, w, slowest)
    bench.barrier(w)
    with open(os.path.join(out_dir, f"{rank}.json"), "w") as f:
        json.dump({"ws": w, "rank": r, "local": local, "slowest": slowest, "rate": rate}, f)
    dist.destroy_process_group()


@pytest.mark.skipif(torch.cuda.is_available(), reason="CPU (gloo) test of the multi-rank host logic")
def test_two_ranks_over_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert (d["ws"], d["rank"], d["local"]) == (2, r, r)
        assert d["slowest"] == 2.5                # the max over ranks
        assert d["rate"] == pytest.approx(10 * 2 / 2.5)  # units of both ranks / slowest time


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0
    assert p.stdout.strip() == ""
