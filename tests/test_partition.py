"""A batch split over ranks by whole permanents (independent problems: no
exchange step beyond gathering the outputs): the library's balanced
partition (pq_partition_batch, host only) and the gather of the ranks'
outputs across two gloo ranks on CPU, each rank evaluating its items with
the oracle."""
import math
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2403_04006_gb300 import api, pq  # noqa: E402
from paper_2403_04006_gb300 import workloads as W  # noqa: E402


def gray_terms(m) -> int:
    """Terms of the Gray code over one side with multiplicities m: the least
    repeated entry keeps one copy fixed, prod_{i != f} (m_i + 1) * m_f."""
    m = [int(x) for x in m if x > 0]
    if not m:
        return 0
    f = int(np.argmin(m))
    return math.prod(x if i == f else x + 1 for i, x in enumerate(m))


def item_terms(pb) -> np.ndarray:
    out = np.zeros(pb.batch, dtype=np.int64)
    for b in range(pb.batch):
        _, r, c = pb.item(b)
        out[b] = min(gray_terms(r), gray_terms(c))
    return out


@pytest.fixture(scope="module")
def sizes():
    return W.ragged(count=8192, sizes_only=True)


@pytest.mark.parametrize("ranks", [1, 2, 3, 8])
def test_partition_covers_every_item_once_and_balances(sizes, ranks):
    rank_of, terms = api.partition_batch(sizes, ranks)
    assert rank_of.shape == (sizes.batch,) and terms.shape == (ranks,)
    assert rank_of.min() >= 0 and rank_of.max() < ranks
    t = item_terms(sizes)
    for r in range(ranks):  # each rank's reported terms are those of its items
        assert terms[r] == t[rank_of == r].sum()
    assert terms.sum() == t.sum()
    # largest first to the least loaded rank: within one item of the mean
    assert terms.max() <= terms.mean() + t.max()
    assert terms.max() <= 1.01 * terms.mean()
    again, _ = api.partition_batch(sizes, ranks)
    assert np.array_equal(again, rank_of)  # a function of the sizes alone


def test_equal_items_go_round_robin():
    """Equal work everywhere: ties go to the lower rank, so items 0, 1, 2, ...
    land on ranks 0, 1, 2, 0, 1, 2, ..."""
    items = [(np.zeros((3, 3)), [1, 1, 1], [1, 1, 1])] * 7
    rank_of, terms = api.partition_batch(W.pack_batch(items), 3)
    assert rank_of.tolist() == [0, 1, 2, 0, 1, 2, 0]
    assert terms.tolist() == [12, 8, 8]  # 4 Gray-code terms per 3 x 3 permanent


def test_partition_edge_cases():
    empty = W.pack_batch([])
    rank_of, terms = api.partition_batch(empty, 4)
    assert rank_of.size == 0 and terms.tolist() == [0, 0, 0, 0]
    one = W.pack_batch([(np.zeros((0, 0)), [], [])])  # n = 0: no terms, still placed
    rank_of, terms = api.partition_batch(one, 2)
    assert rank_of.tolist() == [0] and terms.tolist() == [0, 0]
    for bad in (0, -1, 65537):
        with pytest.raises(pq.PQError) as e:
            api.partition_batch(one, bad)
        assert e.value.code == pq.PQ_ERR_ARG


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def small_batch():
    rng = np.random.default_rng(71)
    items = []
    for _ in range(40):
        n = int(rng.integers(1, 9))
        r = W._parts(n, rng)
        c = W._parts(n, rng)
        B = rng.standard_normal((len(r), len(c))) + 1j * rng.standard_normal((len(r), len(c)))
        items.append((B / math.sqrt(2 * n), r, c))
    return W.pack_batch(items)


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_2403_04006_gb300 import api as A
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pb = small_batch()
    rank_of, _ = A.partition_batch(pb, world)
    sub = pb.subset(np.nonzero(rank_of == rank)[0])  # this rank's items, in item order
    local = O.perm_batch(sub.mats, sub.mat_off, sub.k, sub.l, sub.row_mult, sub.row_off,
                         sub.col_mult, sub.col_off, gold=True)
    full = A.gather_partitioned(torch.from_numpy(np.asarray(local)), rank_of)
    q.put((rank, np.asarray(full).tolist(), int((rank_of == rank).sum())))
    dist.destroy_process_group()


def test_gather_over_two_gloo_ranks():
    import oracle as O
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
    pb = small_batch()
    want = np.asarray(O.perm_batch(pb.mats, pb.mat_off, pb.k, pb.l, pb.row_mult, pb.row_off,
                                   pb.col_mult, pb.col_off, gold=True))
    assert got[0][2] > 0 and got[1][2] > 0 and got[0][2] + got[1][2] == pb.batch
    for _, full, _ in got:  # every rank holds the whole batch, in item order
        assert np.array_equal(np.array(full), want)


def test_single_process_gather_is_local():
    t = torch.arange(5, dtype=torch.float64).to(torch.complex128)
    assert api.gather_partitioned(t, np.zeros(5, dtype=np.int32)) is t
