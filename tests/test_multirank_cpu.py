"""The multi-rank path of bench.py on CPU: two gloo ranks, as torchrun would start them.
Every rank runs an independent replica; the helpers must give the slowest rank's time and
the whole-job rate (weak scaling), and the reference arm must print from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks("gloo")
    r.barrier()
    slowest = r.max(10.0 + rank)          # rank r took 10 + r ms
    total = r.sum(1000.0 * (rank + 1))    # rank r processed 1000 (r + 1) units
    rate = bench.whole_job_rate(1000.0 * (rank + 1), 10.0 + rank, r)
    r.close()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "total": total, "rate": rate}, f)


def test_rank_helpers_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    for rank in range(2):
        d = json.loads((tmp_path / f"rank{rank}.json").read_text())
        assert d["slowest"] == 11.0
        assert d["total"] == 3000.0
        assert d["rate"] == pytest.approx(3000.0 / 11e-3)


@pytest.mark.slow
def test_reference_arm_prints_once_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "3",
           "--warmup", "3"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
