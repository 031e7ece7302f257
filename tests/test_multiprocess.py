"""The N > 1 launch path of bench.py on CPU (gloo, world size 2): replicas synchronise only
through the barrier and the max-over-ranks timing reduction; the reference arm runs on rank 0
alone and the other rank exits 0 without work."""
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


def _rank_main(rank, world, port, outdir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    ws, r, local = bench.init_dist("gloo")
    bench.barrier()
    t = bench.max_over_ranks(1.5 + r)
    bench.barrier()
    with open(os.path.join(outdir, "rank%d.json" % r), "w") as f:
        json.dump({"ws": ws, "rank": r, "local": local, "max": t}, f)
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world_size_2(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    assert [x["rank"] for x in res] == [0, 1] and all(x["ws"] == 2 for x in res)
    assert all(x["max"] == 2.5 for x in res)


def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` launched like the GPU arm (torchrun, 2 ranks, 127.0.0.1):
    exactly one JSON line, from rank 0, with the reference keys."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
