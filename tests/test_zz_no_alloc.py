"""pq_permanent_noalloc: the permanent of one base matrix for callers that
cannot allocate device memory (code inside a framework whose caching
allocator owns the device memory, processes held to a fixed device-memory
budget, latency-critical paths where an allocation may synchronise the
device).  It must give what the regular entry point pq_permanent_batched
gives, call after call, although every call reuses the same static device
workspace, and it must match the oracle within the tolerance of the other
parity tests.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process.
"""
import math
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2403_04006_gb300 import api, pq  # noqa: E402
from paper_2403_04006_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the relative tolerance of the parity tests for n <= 20
TOL30 = 1e-8  # ... and at n = 30
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pq.load_library()
    return torch.device("cuda:0")


def cases():
    rng = np.random.default_rng(909)
    out = []
    n = 18  # collision-free, many warp tasks
    B = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2 * n)
    out.append((B, [1] * n, [1] * n))
    B = (rng.standard_normal((5, 4)) + 1j * rng.standard_normal((5, 4))) / 3
    out.append((B, [2, 1, 3, 1, 2], [3, 2, 2, 2]))  # repeated rows and columns
    out.append((np.array([[0.4 - 0.9j]]), [1], [1]))  # n = 1
    out.append((np.zeros((2, 2), dtype=complex), [0, 0], [0, 0]))  # n = 0
    return out


def regular_entry_point(items, dev):
    pb = W.pack_batch(items)
    return api.permanent_batched(api.DeviceBatch(pb, dev), api.Plan.for_batch(pb)).cpu().numpy()


def noalloc(B, r, c, dev):
    """One pq_permanent_noalloc call through the C ABI; the output buffer starts as NaN."""
    Bd = torch.from_numpy(np.ascontiguousarray(B, dtype=np.complex128)).to(dev)
    out = torch.full((1,), complex(float("nan"), float("nan")), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    pq.pq_permanent_noalloc(Bd.data_ptr() if Bd.numel() else None, B.shape[0], B.shape[1],
                            np.asarray(r), np.asarray(c), out.data_ptr(), stream)
    return out.cpu().numpy()[0]


def test_noalloc_matches_regular_entry_point_twice(dev):
    items = cases()
    ref = regular_entry_point(items, dev)
    gold = [O.perm_ryser(B, r, c, gold=True) for B, r, c in items]
    for _call in range(2):  # the second call reuses the workspace the first left behind
        for (B, r, c), want, w_or in zip(items, ref, gold):
            got = noalloc(B, r, c, dev)
            assert abs(got - want) <= TOL * abs(want), (B.shape, r, c, got, want)
            assert abs(got - w_or) <= TOL * abs(w_or), (B.shape, r, c, got, w_or)


def test_noalloc_large_permanents(dev):
    """n = 30 against the stored gold value (16384 warp tasks), and n = 31, whose
    2^30 terms need longer chunks than the default so that the task list fits
    the static workspace, against the regular entry point; each twice."""
    sys.path.insert(0, os.path.join(HERE, "golden"))
    from make_golden import read_matrix_file
    A, vals = read_matrix_file(os.path.join(HERE, "golden", "single_large_n30.txt"))
    A31 = W.single_large(31)
    want31 = regular_entry_point([(A31, [1] * 31, [1] * 31)], dev)[0]
    for _call in range(2):
        got30 = noalloc(A, [1] * 30, [1] * 30, dev)
        assert abs(got30 - vals["per_gold"]) <= TOL30 * abs(vals["per_gold"]), got30
        got31 = noalloc(A31, [1] * 31, [1] * 31, dev)
        assert abs(got31 - want31) <= TOL * abs(want31), (got31, want31)


def test_noalloc_rejects_bad_and_oversized_input(dev):
    out = torch.empty(1, dtype=torch.complex128, device=dev)
    B = torch.ones((2, 2), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(pq.PQError) as e:  # 3 row copies against 2 column copies
        pq.pq_permanent_noalloc(B.data_ptr(), 2, 2, np.array([1, 2]), np.array([1, 1]),
                                out.data_ptr(), stream)
    assert e.value.code == pq.PQ_ERR_ARG
    n = 40  # 2^39 Gray-code terms: more warp tasks than the static workspace holds
    Bn = torch.ones((n, n), dtype=torch.complex128, device=dev)
    with pytest.raises(pq.PQError) as e:
        pq.pq_permanent_noalloc(Bn.data_ptr(), n, n, np.ones(n), np.ones(n), out.data_ptr(),
                                stream)
    assert e.value.code == pq.PQ_ERR_UNSUPPORTED
