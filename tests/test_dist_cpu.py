"""Host logic of the multi-rank benchmark path on CPU ranks (gloo, world size 2): the max-over-ranks
timing reduction, the whole-job rate, per-rank batch seeds, and the reference arm on rank > 0."""
import io
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


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = bench.reduce_max(10.0 + 5.0 * rank, dist, "cpu")   # rank 1 is the slow one
    rate = bench.whole_job_rate(1000, ws, ms)
    seed = bench.batch_seed(rank)
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.run_reference(type("A", (), {"steps": 1, "warmup": 3, "members": 2})()) if rank == 1 else 0
    q.put((rank, ms, rate, seed, rc, buf.getvalue()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, rate0, seed0, _, _), (r1, ms1, rate1, seed1, rc1, printed1) = out
    assert ms0 == ms1 == 15.0                    # both ranks see the slowest rank's time
    assert rate0 == rate1 == 2 * 1000 / 15e-3    # whole-job nonzeros over the max time
    assert seed0 != seed1                        # each rank evaluates its own batch
    assert rc1 == 0 and printed1 == ""           # reference arm: only rank 0 runs and prints
