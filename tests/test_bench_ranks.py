"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): rendezvous, barrier, the max-over-ranks
timing reduction, that only rank 0 runs and reports the reference arm, and the row strips of the
row-sharded mode (one image split across ranks)."""
import os
import socket
import sys
import types

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup(world)
    slowest = bench.max_over_ranks(0.5 + rank, w)  # each rank's own step time
    bench.barrier(w)
    ref = bench.run_reference(types.SimpleNamespace(steps=1, warmup=0), w, r) if r != 0 else "rank0-skipped"
    # row-sharded mode: every rank's strip, gathered
    strips = [None] * w
    dist.all_gather_object(strips, bench.rank_rows(w, r))
    out.put((r, w, slowest, ref, strips))
    dist.destroy_process_group()


def bench_H():
    sys.path.insert(0, ROOT)
    import bench
    return bench.H


def test_two_gloo_ranks_reduce_timing_and_only_rank0_reports():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, out)) for k in range(2)]
    for pr in procs:
        pr.start()
    results = sorted(out.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert [r[1] for r in results] == [2, 2]
    assert all(r[2] == 1.5 for r in results)  # max over ranks of 0.5 and 1.5
    assert results[1][3] is None              # rank 1 runs no reference work and prints nothing
    # the two ranks' row strips tile the image's rows without overlap, the same on both ranks
    strips = results[0][4]
    assert strips == results[1][4]
    assert strips[0][0] == 0 and strips[0][1] == strips[1][0] and strips[1][1] == bench_H()
