"""The bench's multi-rank bookkeeping on CPU with gloo (world size 2): rank r
evaluates block r of the job's batch (weak scaling, no data-path
collective), or with --split its part of one batch (strong scaling); the
timed region is closed by a barrier, the time is the maximum over ranks and
the throughput counts the units of all ranks.  Both arms of the bench
describe the same job in the same config object."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w = bench.init_dist("gloo")
    assert (r, w) == (rank, world)
    my_seconds = 1.0 + rank  # rank 1 is the slower one
    bench.barrier()
    slowest = bench.max_over_ranks(my_seconds)
    rate = bench.whole_job_rate(1000.0, w, slowest)
    from paper_2403_04006_gb300 import workloads as W
    blk = W.ragged(count=256, block=rank, sizes_only=True)  # this rank's block
    terms = bench.glynn_terms(blk, range(blk.batch))
    job = bench.sum_over_ranks(terms)
    # --split: one batch, each rank its part of the library's partition
    import numpy as np

    from paper_2403_04006_gb300 import api
    full = W.ragged(count=256, sizes_only=True)
    rank_of, per_rank = api.partition_batch(full, w)
    mine = full.subset(np.nonzero(rank_of == rank)[0])
    split_job = bench.sum_over_ranks(bench.glynn_terms(mine, range(mine.batch)))
    q.put((rank, slowest, rate, terms, job,
           (split_job, int(per_rank.sum()), bench.glynn_terms(full, range(full.batch)))))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    block_terms = [g[3] for g in got]
    assert block_terms[0] != block_terms[1]  # two different blocks
    for rank, slowest, rate, terms, job, (split_job, per_rank, whole) in got:
        assert slowest == 2.0          # max over ranks
        assert rate == 1000.0 * 2 / 2.0  # all ranks' units / slowest time
        assert job == sum(block_terms)   # the job's terms: every rank's block
        assert split_job == per_rank == whole  # a split batch counts its terms once


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
    assert bench.max_over_ranks(3.0) == 3.0  # no process group: identity
    assert bench.sum_over_ranks(3.0) == 3.0


def test_both_arms_describe_the_same_job():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.bench_config(bench.WORKLOAD, 65536, 176370045, 1)
    b = bench.bench_config(bench.WORKLOAD, 65536, 176370045, 1)
    assert a == b and set(a) == {"workload", "permanents", "terms", "parallelism", "l2"}
    weak = bench.bench_config(bench.WORKLOAD, 2 * 65536, 352740090, 2)
    split = bench.bench_config(bench.WORKLOAD, 65536, 176370045, 2, split=True)
    assert "block r" in weak["parallelism"] and "pq_partition_batch" in split["parallelism"]
    assert bench.bench_config(bench.WORKLOAD, 65536, 1, 1, split=True) == \
        bench.bench_config(bench.WORKLOAD, 65536, 1, 1)  # one GPU: the same job
