"""Host side of a permanent split over ranks (the exchange step of one large
permanent spread across GPUs): the library's double-double combination of
the shards' partial sums (pq_combine_partials_host, the host twin of the
device kernel pq_combine_partials), pinned by exact rational arithmetic, and
the all_gather of the partials across two gloo ranks on CPU."""
import os
import socket
import sys
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2403_04006_gb300 import api  # noqa: E402


def dd_random(rng, size, scale):
    """Pairs (hi, lo) with lo = a fraction of an ulp of hi: exact values with
    about 106 significant bits."""
    hi = rng.standard_normal(size) * scale
    lo = rng.uniform(-0.5, 0.5, size) * np.spacing(hi)
    return hi, lo


def exact(hi, lo):
    return Fraction(float(hi)) + Fraction(float(lo))


def make_parts(rng, nshards, batch):
    parts = []
    for _ in range(nshards):
        p = np.zeros((batch, 4))
        p[:, 0], p[:, 1] = dd_random(rng, batch, 1.0)
        p[:, 2], p[:, 3] = dd_random(rng, batch, 1.0)
        parts.append(p)
    # heavy cancellation in item 0: shard values nearly cancel, the sum is
    # carried by the low parts
    parts[0][0, 0], parts[0][0, 1] = 1.0e6, 3.0e-11
    parts[-1][0, 0], parts[-1][0, 1] = -1.0e6, 4.0e-11
    for p in parts[1:-1]:
        p[0, :2] = 0.0
    if nshards >= 3:
        # item 2 (imaginary part): 1 + 2^-60 - 1, whose value is only the
        # rounding error of the first high-part addition
        for p in parts:
            p[2, 2:] = 0.0
        parts[0][2, 2], parts[1][2, 2], parts[2][2, 2] = 1.0, 2.0 ** -60, -1.0
    return parts


@pytest.mark.parametrize("nshards", [1, 2, 3, 5])
def test_combination_is_the_exact_sum_rounded(nshards):
    rng = np.random.default_rng(90 + nshards)
    batch = 16
    parts = make_parts(rng, nshards, batch)
    n = rng.integers(1, 30, batch)
    n[0] = 1  # the cancelling item, unscaled
    n[1] = 0  # n = 0: no scaling
    got = api.combine_partials(parts, n)
    for b in range(batch):
        re = sum(exact(p[b, 0], p[b, 1]) for p in parts)
        im = sum(exact(p[b, 2], p[b, 3]) for p in parts)
        scale = Fraction(1) if n[b] == 0 else Fraction(1, 2 ** int(n[b] - 1))
        for g, w in ((got[b].real, re * scale), (got[b].imag, im * scale)):
            # one rounding of the exact sum, plus double-double rounding far below it
            assert abs(Fraction(float(g)) - w) <= abs(w) * Fraction(1, 2 ** 52) + Fraction(1, 2 ** 200)
    if nshards > 1:
        # the cancelling item: a plain double sum would lose it entirely
        assert abs(got[0].real - 7.0e-11) <= 1e-24
    if nshards >= 3:
        assert got[2].imag == np.ldexp(2.0 ** -60, 1 - int(n[2]))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    from paper_2403_04006_gb300 import api as A
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = make_parts(np.random.default_rng(7), world, 8)  # same on every rank
    local = torch.from_numpy(parts[rank])                   # this rank's shard
    gathered = A.gather_partials(local)
    n = np.arange(8) + 1
    q.put((rank, [g.tolist() for g in gathered], A.combine_partials(gathered, n).tolist()))
    dist.destroy_process_group()


def test_gather_over_two_gloo_ranks():
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
    parts = make_parts(np.random.default_rng(7), 2, 8)
    want = api.combine_partials(parts, np.arange(8) + 1)
    for rank, gathered, combined in got:
        assert [np.array(g) for g in gathered][0].tolist() == parts[0].tolist()
        assert [np.array(g) for g in gathered][1].tolist() == parts[1].tolist()
        assert np.array_equal(np.array(combined), want)  # identical on every rank


def test_single_process_gather_is_local():
    t = torch.arange(8, dtype=torch.float64).reshape(2, 4)
    g = api.gather_partials(t)
    assert len(g) == 1 and np.array_equal(g[0].numpy(), t.numpy())


def test_combine_argument_errors():
    from paper_2403_04006_gb300 import pq
    parts = np.zeros((2, 3, 4))
    with pytest.raises(pq.PQError) as e:
        pq.pq_combine_partials_host(parts, np.array([1, 2, 49]))  # n above PQ_MAX_N
    assert e.value.code == pq.PQ_ERR_ARG
    with pytest.raises(ValueError):
        pq.pq_combine_partials_host(parts, np.array([1, 2]))
    assert pq.pq_combine_partials_host(np.zeros((1, 0, 4)), np.zeros(0)).shape == (0,)
    one = np.zeros((3, 1, 4))
    one[1, 0, 0] = 1.0  # n = 0: the shard that held the permanent contributes 1
    assert pq.pq_combine_partials_host(one, np.array([0]))[0] == 1.0
