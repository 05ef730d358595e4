"""bench.py's multi-rank path on CPU (world size 2, gloo): each rank times its own replica (the path
shards into independent propagations, no data-path collective); the job's time is the slowest
rank's (all-reduce MAX) and its value counts every rank's ADO-RHS evaluations.  The reference arm
under torchrun runs on rank 0 only; the other ranks exit 0 without work."""
import io
import json
import os
import socket
import sys
import types
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, _ = bench._dist()
        bench._barrier(w)
        m = bench._max_over_ranks(10.0 + 5.0 * rank, w)  # rank 1 is the slow one
        out[rank] = (w, r, m, bench._job_value(w, 1000, 3, m))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    ws = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
    for rank in range(ws):
        w, r, m, v = out[rank]
        assert (w, r) == (ws, rank)
        assert m == 15.0                               # the slowest rank's time
        assert v == pytest.approx(2 * 1000 * 4 * 3 / 0.015)  # both replicas' evaluations


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(gpus=2, steps=1, warmup=0)
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.reference_arm(args, 2, 1) == 0
    assert buf.getvalue() == ""
    with redirect_stdout(buf):
        assert bench.reference_arm(args, 2, 0) == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    for k in ("metric", "unit", "steps", "warmup", "ms_per_step", "cpu_baseline", "e2e", "config"):
        assert k in line
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
