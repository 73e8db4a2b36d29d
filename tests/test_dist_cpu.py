"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the
max / sum aggregation over ranks, and the reference arm running on rank 0
only."""
import io
import json
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _agg_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, dist = bench._dist()
    q.put((r, w, bench.aggregate(dist, float(rank + 1), "max"),
           bench.aggregate(dist, float(rank + 1), "sum")))
    dist.destroy_process_group()


def _ref_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3",
                         "--ref-angles", "2"])
    q.put((rank, rc, buf.getvalue()))


def _run(target, world=2, timeout=600):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=timeout) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def test_aggregate_over_two_gloo_ranks():
    pytest.importorskip("torch.distributed")
    res = sorted(_run(_agg_worker))
    assert [r[:2] for r in res] == [(0, 2), (1, 2)]
    for _, _, mx, sm in res:
        assert mx == 2.0 and sm == 3.0


def test_reference_arm_prints_on_rank_zero_only():
    pytest.importorskip("torch.distributed")
    res = sorted(_run(_ref_worker))
    (r0, rc0, out0), (r1, rc1, out1) = res
    assert rc0 == 0 and rc1 == 0 and out1.strip() == ""
    line = json.loads(out0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
