"""The N > 1 path of bench.py: independent replicas (one density per rank per
step, no data-path collective), timed by the slowest rank.  Two gloo ranks
on the CPU check the per-rank units, the max-over-ranks time, the whole-job
value, and that the reference arm runs and prints on rank 0 only."""

import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    try:
        _work(rank, world, port, q)
    except BaseException as exc:  # report instead of leaving the parent waiting
        q.put((rank, "error", repr(exc)))
        raise


def _work(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    w, r, _ = bench.dist_setup(False)  # gloo
    t = 1.0 + 0.5 * r                  # a slower rank 1
    t_max = bench.max_over_ranks(t, w)
    value = bench.job_value(w, 10, t_max)
    # the reference arm: rank 0 alone runs (a stand-in for the oracle sample)
    # and prints one JSON line; the other ranks return without output
    bench.oracle_sample = lambda rho, node_frac=1.0: (0.5, None, "stand-in sample",
                                                      {"i1": 0.0, "type2": 0.0, "type1": 0.0,
                                                       "node_frac": 1.0})
    args = type("A", (), {"steps": 2, "warmup": 1})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    dist.barrier()
    q.put((r, w, bench.replica_seed(r), t_max, value, buf.getvalue()))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in range(2))
    assert all(r[1] != "error" for r in res), res
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, s0, t0, v0, out0), (r1, w1, s1, t1, v1, out1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert s0 != s1                      # each rank solves its own density
    assert t0 == t1 == 1.5               # the job's time is the slowest rank's
    assert v0 == v1 == 2 * 10 / 1.5      # units of all ranks over that time
    line = json.loads(out0.strip())
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] == 2.0
    assert out1 == ""
