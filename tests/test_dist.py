"""The multi-rank host logic of bench.py on CPU: two gloo ranks (spawned
processes) run the barrier and the max-over-ranks reduction, and the
reference arm does its work on rank 0 only (rank 1 exits at once, silently).
Every rank of a GPU run is an independent replica, so nothing else crosses
ranks."""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, port: int, q) -> None:
    os.environ.update(WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import types

    import bench
    d = bench.Dist()
    try:
        d.barrier()
        m = d.max(3.0 * (rank + 1))
        out = io.StringIO()
        if rank == 1:
            args = types.SimpleNamespace(warmup=1, steps=1, gpus=2)
            with redirect_stdout(out):
                bench.run_reference(args, d)
        d.barrier()
        q.put((rank, m, out.getvalue()))
    finally:
        d.close()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, m, out = q.get(timeout=180)
        res[rank] = (m, out)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # max over ranks reaches every rank
    assert res[0][0] == res[1][0] == 6.0
    # the reference arm prints nothing and does no work on rank 1
    assert res[1][1] == ""


def test_reference_arm_json_line():
    """The reference arm on rank 0 (one warm-up and one timed view of the
    1M-Gaussian workload through the FP64 oracle on the host cores) prints
    one JSON line carrying the fields the contract names."""
    import json
    import types

    sys.path.insert(0, ROOT)
    import bench

    class OneRank:
        rank, world = 0, 1

    out = io.StringIO()
    with redirect_stdout(out):
        bench.run_reference(types.SimpleNamespace(warmup=1, steps=1, gpus=1), OneRank())
    lines = [l for l in out.getvalue().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == bench.WORKLOAD
