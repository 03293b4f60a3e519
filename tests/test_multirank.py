"""The N > 1 path of bench.py on CPU: two gloo ranks (no GPU).  Every rank
fits its own batch (weak scaling); the only cross-rank steps are the barrier
around the timed region and the maximum of the ranks' times; under torchrun
the reference arm runs on rank 0 alone."""
import hashlib
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _digest(sets) -> str:
    h = hashlib.sha256()
    for ts in sets:
        for a in (ts.par0, ts.hpos):
            h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _rank_main(rank, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": "2", "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    bench.set_nevt(1)
    world, r, local = bench.dist_setup(2, backend="gloo")
    bench.barrier(world)
    slowest = bench.max_over_ranks(world, 1.5 + r)
    digest = _digest(bench.workload(r))
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": world, "rank": r, "max": slowest, "digest": digest}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_agree_on_the_slowest(tmp_path):
    mp.start_processes(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert [x["world"] for x in res] == [2, 2]
    assert [x["max"] for x in res] == [2.5, 2.5]  # both ranks report the slowest time
    # each rank draws its own batch, and the same one a lone process draws
    assert res[0]["digest"] != res[1]["digest"]
    sys.path.insert(0, ROOT)
    import bench
    bench.set_nevt(1)
    try:
        assert res[1]["digest"] == _digest(bench.workload(1))
    finally:
        bench.set_nevt(100)


def test_reference_arm_under_torchrun_prints_one_line(tmp_path):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
