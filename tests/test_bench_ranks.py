"""The benchmark's multi-rank logic on CPU (gloo, world size 2): the path
shards by independent problems, so ranks exchange only timings and unit
counts — the max of the per-rank times and the sum of the per-rank units —
and the reference arm runs on rank 0 alone."""

import contextlib
import io
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx = bench.over_ranks(dist, 10.0 + rank, "max", "cpu")
        sm = bench.over_ranks(dist, 100.0 * (rank + 1), "sum", "cpu")
        # the reference arm prints its line on rank 0 only
        a = types.SimpleNamespace(workload="sk100", lr=6.0, mu=0.0, steps=1, warmup=0)
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(a, rank, world)
        dist.barrier()
        out[rank] = (mx, sm, buf.getvalue())
    finally:
        dist.destroy_process_group()


def test_over_ranks_and_reference_on_rank0_only():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import json
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0][:2] == (11.0, 300.0) and res[1][:2] == (11.0, 300.0)
    assert res[1][2] == ""
    line = json.loads(res[0][2].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def test_over_ranks_without_a_process_group():
    import bench
    assert bench.over_ranks(None, 3.5, "max", "cpu") == 3.5
    assert bench.over_ranks(None, 7.0, "sum", "cpu") == 7.0
