"""GPU Algorithm A sampler (pq_bs_sample) against the oracle's sampler on the
same random inputs, and its sample frequencies against Eq. (BS_prob).

The selection of each photon's mode is an integer decided by floating point:
photon k goes to the first mode whose running weight sum (modes in order)
exceeds u_k times the total.  The GPU forms the weights by expanding each
step's permanents along the new photon's row, the oracle by Ryser's formula
in double-double, so their weights differ in the last bits; a pick whose
threshold lies that close to a cumulative boundary may go either way.  The
test therefore enumerates, with the oracle's weights, every outcome whose
picks all lie in their mode's cumulative interval widened by the path's
weight tolerance, and requires each GPU sample to be one of them; where no
boundary lies within that width the outcome is unique and must equal the
oracle sampler's sample exactly."""
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


WEIGHT_TOL = 4e-10  # 2 x the 1e-10 permanent tolerance for |per|^2, for the sums and the total


def valid_outcomes(U, s, order, unif, rel=WEIGHT_TOL):
    """Every output occupation one sample can reach when each photon's pick
    lies in its mode's cumulative-weight interval widened by rel x total
    (oracle weights, gold mode).  Returns (set of outcomes, ambiguous steps)."""
    m = U.shape[0]
    cols = [j for j in range(m) for _ in range(int(s[j]))]
    n = len(cols)
    found, ambiguous = set(), [0]

    def rec(k, occ):
        if k > n:
            found.add(tuple(int(x) for x in occ))
            return
        sk = np.zeros(m, dtype=np.int32)
        for q in range(k):
            sk[cols[int(order[q])]] += 1
        cand = np.repeat(occ[None, :], m, axis=0)
        cand[np.arange(m), np.arange(m)] += 1
        _, amps = O.bs_probs(U, sk, cand, gold=True, nthreads=1)
        w = [float(abs(a) ** 2) for a in amps]
        total = 0.0
        for x in w:
            total += x
        thr, e = float(unif[k - 1]) * total, rel * total
        picks, cum = [], 0.0
        for i, x in enumerate(w):
            lo, cum = cum, cum + x
            if x > 0.0 and lo - e <= thr < cum + e:
                picks.append(i)
        ambiguous[0] += len(picks) > 1
        for i in picks:
            nxt = occ.copy()
            nxt[i] += 1
            rec(k + 1, nxt)

    rec(1, np.zeros(m, dtype=np.int32))
    return found, ambiguous[0]


@pytest.mark.parametrize("case", ["bs_small", "repeated_inputs"])
def test_samples_are_valid_draws_for_their_uniforms(dev, case):
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
    assert got.shape == (ns, U.shape[0])
    assert (got.sum(axis=1) == n).all()
    unique = []
    for b in range(ns):
        outs, _amb = valid_outcomes(U, s, order[b], unif[b])
        assert tuple(int(x) for x in got[b]) in outs, (b, got[b], outs)
        if len(outs) == 1:
            unique.append(b)
    # where the draw is unambiguous, the oracle sampler gives the same sample
    assert len(unique) >= ns - 2
    want = O.algorithm_a(U, s, order[unique], unif[unique])
    assert np.array_equal(got[unique], want)


def test_validity_check_rejects_a_wrong_pick():
    """The enumeration pins the selection rule: a sample with one photon moved
    to another mode is not a valid outcome of its uniforms."""
    U, s, _ = W.bs_small()
    order, unif = W.sampler_draws(5, 4, 41)
    want = O.algorithm_a(U, s, order, unif)
    for b in range(5):
        outs, amb = valid_outcomes(U, s, order[b], unif[b])
        if amb:
            continue
        assert outs == {tuple(int(x) for x in want[b])}
        moved = want[b].copy()
        src = int(np.nonzero(moved)[0][0])
        moved[src] -= 1
        moved[(src + 1) % len(moved)] += 1
        assert tuple(int(x) for x in moved) not in outs


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


def test_sampler_plan_runs_match_the_one_shot_call(dev):
    """A planned sampler run gives, sample for sample, what pq_bs_sample gives
    for the same interferometer, column orders and uniforms: on three runs in
    a row with different interferometers and draws (the workspace is reused),
    and with the step plans made once."""
    s = np.array([1, 0, 1, 1, 0, 1, 0, 0], dtype=np.int32)
    m, ns, n = 8, 300, 4
    plan = api.SamplerPlan(m, s, ns)
    try:
        for run in range(3):
            U = torch.from_numpy(W.haar_unitary(m, np.random.default_rng(50 + run))).to(dev)
            order, unif = W.sampler_draws(ns, n, 60 + run)
            got = plan.run(U, order, unif)
            want = api.bs_sample(U, s, order, unif)
            assert np.array_equal(got, want), run
            assert (got.sum(axis=1) == n).all()
        with pytest.raises(ValueError):
            plan.run(U, order[:10], unif[:10])
        with pytest.raises(pq.PQError) as e:  # not a permutation: checked before any launch
            bad = order.copy()
            bad[3, 1] = bad[3, 0]
            plan.run(U, bad, unif)
        assert e.value.code == pq.PQ_ERR_ARG
        assert np.array_equal(plan.run(U, order, unif), want)  # usable after the error
    finally:
        plan.close()
