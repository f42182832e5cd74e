"""The multi-GPU path of bench.py on the host: replicas only (every rank steps
its own atmosphere; only the timing is combined), so what there is to test
without GPUs is the rank plumbing over gloo with world size 2: the barrier,
the maximum over ranks of the timed region, the whole-job rate, and the
reference arm under torchrun printing one line from rank 0 only."""

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


def _rank_main(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks()
    r.barrier()
    got = r.max(1.5 + rank)                      # rank 1's time is the larger
    r.barrier()
    rate = bench.whole_job_rate(r.world, 1000.0, got)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"world": r.world, "max": got, "rate": rate}, f)
    r.close()


def test_ranks_over_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(i, port, str(tmp_path))) for i in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / f"rank{i}.json")) for i in range(2)]
    for r in res:
        assert r["world"] == 2 and r["max"] == 2.5
        assert r["rate"] == pytest.approx(2 * 1000.0 / 2.5)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    pytest.importorskip("torch")
    port = _free_port()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--gpus", "2", "--impl", "reference",
           "--workload", "hs_g4", "--steps", "1", "--warmup", "3"]
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle"
