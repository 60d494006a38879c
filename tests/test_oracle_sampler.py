"""Pins of the oracle's Algorithm A sampler against what fixes it: outputs of
a permutation interferometer are deterministic, and sample frequencies follow
Eq. (BS_prob) (likelihood-ratio test against the exact distribution)."""
import math

import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")

import oracle as O  # noqa: E402
from paper_2403_04006_gb300 import workloads as W  # noqa: E402


def all_patterns(n, m):
    if m == 1:
        return [[n]]
    return [[v] + rest for v in range(n + 1) for rest in all_patterns(n - v, m - 1)]


def frequency_test(U, s, nsamples, seed):
    n = int(np.sum(s))
    m = U.shape[0]
    order, unif = W.sampler_draws(nsamples, n, seed)
    out = O.algorithm_a(U, s, order, unif)
    pats = np.array(all_patterns(n, m))
    p, _ = O.bs_probs(U, s, pats)
    index = {tuple(t): q for q, t in enumerate(pats)}
    counts = np.zeros(len(pats))
    for row in out:
        counts[index[tuple(row)]] += 1
    keep = p > 0
    assert counts[~keep].sum() == 0  # never an impossible outcome
    stat = scipy_stats.power_divergence(counts[keep], nsamples * p[keep] / p[keep].sum(),
                                        lambda_="log-likelihood")
    return stat.pvalue


def test_permutation_interferometer_is_deterministic():
    m = 4
    perm = [2, 0, 3, 1]  # input mode j -> output mode perm[j]
    U = np.zeros((m, m), dtype=complex)
    for j, o in enumerate(perm):
        U[o, j] = np.exp(0.3j * j)
    s = np.array([1, 2, 0, 1])
    order, unif = W.sampler_draws(50, 4, 7)
    out = O.algorithm_a(U, s, order, unif)
    want = np.zeros(m, dtype=int)
    for j in range(m):
        want[perm[j]] += s[j]
    assert (out == want).all()


def test_single_photon_frequencies():
    U = W.haar_unitary(4, np.random.default_rng(31))
    assert frequency_test(U, np.array([0, 1, 0, 0]), 3000, 11) > 1e-4


def test_two_photons_frequencies():
    U = W.haar_unitary(3, np.random.default_rng(32))
    assert frequency_test(U, np.array([1, 1, 0]), 4000, 12) > 1e-4


def test_repeated_input_mode_frequencies():
    U = W.haar_unitary(3, np.random.default_rng(33))
    assert frequency_test(U, np.array([2, 0, 1]), 3000, 13) > 1e-4


def test_hong_ou_mandel_never_coincident():
    U = O.beamsplitter_block(math.pi / 4, 0.2)
    order, unif = W.sampler_draws(400, 2, 14)
    out = O.algorithm_a(U, [1, 1], order, unif)
    assert not np.any((out[:, 0] == 1) & (out[:, 1] == 1))
    assert 150 < np.sum(out[:, 0] == 2) < 250
