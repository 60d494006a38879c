"""GPU Algorithm A sampler (pq_bs_sample) against the oracle's sampler on the
same random inputs, and its sample frequencies against Eq. (BS_prob).

The selection of each photon's mode is an integer decided by floating point:
both sides sum the weights in mode order in double precision and compare
with u * total, so with the same draws they pick the same modes unless a
uniform falls within rounding distance of a cumulative boundary (which these
seeded draws do not)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
scipy_stats = pytest.importorskip("scipy.stats")

import oracle as O  # noqa: E402
from paper_2403_04006_gb300 import api, pq  # noqa: E402
from paper_2403_04006_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pq.load_library()
    return torch.device("cuda:0")


@pytest.mark.parametrize("case", ["bs_small", "repeated_inputs"])
def test_same_draws_same_samples(dev, case):
    if case == "bs_small":
        U, s, _ = W.bs_small()
        ns, seed = 200, 41
    else:
        U = W.haar_unitary(6, np.random.default_rng(42))
        s = np.array([2, 1, 0, 1, 0, 0], dtype=np.int32)
        ns, seed = 120, 43
    n = int(s.sum())
    order, unif = W.sampler_draws(ns, n, seed)
    got = api.bs_sample(torch.from_numpy(U).to(dev), s, order, unif)
    want = O.algorithm_a(U, s, order, unif)
    assert got.shape == want.shape
    assert (got.sum(axis=1) == n).all()
    assert np.array_equal(got, want)


def all_patterns(n, m):
    if m == 1:
        return [[n]]
    return [[v] + rest for v in range(n + 1) for rest in all_patterns(n - v, m - 1)]


def test_sample_frequencies_follow_bs_prob(dev):
    U = W.haar_unitary(5, np.random.default_rng(44))
    s = np.array([1, 1, 1, 0, 0], dtype=np.int32)
    ns = 20000
    order, unif = W.sampler_draws(ns, 3, 45)
    got = api.bs_sample(torch.from_numpy(U).to(dev), s, order, unif)
    pats = np.array(all_patterns(3, 5))
    p, _ = O.bs_probs(U, s, pats)
    index = {tuple(t): q for q, t in enumerate(pats)}
    counts = np.zeros(len(pats))
    for row in got:
        counts[index[tuple(row)]] += 1
    stat = scipy_stats.power_divergence(counts, ns * p / p.sum(), lambda_="log-likelihood")
    assert stat.pvalue > 1e-4


def test_sampler_argument_errors(dev):
    U = torch.from_numpy(W.haar_unitary(3, np.random.default_rng(46))).to(dev)
    s = np.array([1, 1, 0], dtype=np.int32)
    with pytest.raises(pq.PQError) as e:  # not a permutation
        api.bs_sample(U, s, np.array([[0, 0]], dtype=np.int32), np.array([[0.1, 0.2]]))
    assert e.value.code == pq.PQ_ERR_ARG
    with pytest.raises(pq.PQError) as e:  # uniform outside [0, 1)
        api.bs_sample(U, s, np.array([[0, 1]], dtype=np.int32), np.array([[0.1, 1.0]]))
    assert e.value.code == pq.PQ_ERR_ARG
