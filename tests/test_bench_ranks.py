"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the
max-over-ranks reduction of step times and the reference arm printing from
rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    v = bench.reduce_max(1.5 + rank, world, torch.device("cpu"))
    # the reference arm: rank 0 prints one line, the other ranks nothing
    args = bench.parse_args(["--impl", "reference", "--gpus", str(world), "--steps", "1",
                             "--warmup", "0", "--p", "40", "--n", "60", "--cpu-budget", "0.2"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    dist.destroy_process_group()
    q.put((rank, v, buf.getvalue()))


def test_max_over_ranks_and_rank0_output():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict()
    for _ in range(world):
        rank, v, text = q.get(timeout=300)
        out[rank] = (v, text)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 2.5
    assert out[1][1] == ""
    lines = out[0][1].strip().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == world
    assert rec["value"] > 0 and rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["cpu_baseline"]["cores"] >= 1 and rec["cpu_baseline"]["nproc"] >= 1
    assert rec["e2e"]["h2d_bytes_per_step"] == 0
