"""Pins of the oracle's lossy boson-sampling probabilities (Sec. 3.2.4): no
loss reduces to Eq. (BS_prob); probabilities over all detection patterns
(every photon count) sum to one; with equal loss on every mode the number of
detected photons is binomial; one photon is seen in mode i with probability
|A_ij|^2 and lost with the rest."""
import math

import numpy as np

import oracle as O
from paper_2403_04006_gb300 import workloads as W


def patterns_upto(n, m):
    def comp(k, mm):
        if mm == 1:
            return [[k]]
        return [[v] + r for v in range(k + 1) for r in comp(k - v, mm - 1)]
    out = []
    for k in range(n + 1):
        out += comp(k, m)
    return np.array(out, dtype=np.int32)


def factors(m, seed):
    rng = np.random.default_rng(seed)
    return W.haar_unitary(m, rng), rng.uniform(0.2, 0.95, m), W.haar_unitary(m, rng)


def test_no_loss_is_lossless_bs():
    V, _, Wm = factors(4, 1)
    s = np.array([1, 0, 1, 1])
    t = patterns_upto(3, 4)
    p = O.lossy_probs(V, np.ones(4), Wm, s, t)
    full = t.sum(axis=1) == 3
    ref, _ = O.bs_probs(V @ Wm, s, t[full])
    assert np.abs(p[full] - ref).max() <= 1e-14
    assert np.abs(p[~full]).max() <= 1e-15


def test_total_probability_is_one():
    V, eta, Wm = factors(4, 2)
    s = np.array([2, 0, 1, 0])
    p = O.lossy_probs(V, eta, Wm, s, patterns_upto(3, 4))
    assert abs(p.sum() - 1.0) <= 1e-13
    assert (p >= 0).all()


def test_equal_loss_gives_binomial_photon_count():
    m, n, eta = 3, 3, 0.63
    V, _, Wm = factors(m, 3)
    s = np.array([1, 1, 1])
    t = patterns_upto(n, m)
    p = O.lossy_probs(V, np.full(m, eta), Wm, s, t)
    for k in range(n + 1):
        want = math.comb(n, k) * eta ** k * (1 - eta) ** (n - k)
        assert abs(p[t.sum(axis=1) == k].sum() - want) <= 1e-13


def test_single_photon():
    V, eta, Wm = factors(5, 4)
    A = V @ np.diag(np.sqrt(eta)) @ Wm
    j = 2
    s = np.zeros(5, dtype=int)
    s[j] = 1
    t = patterns_upto(1, 5)
    p = O.lossy_probs(V, eta, Wm, s, t)
    assert abs(p[0] - (1 - np.sum(np.abs(A[:, j]) ** 2))) <= 1e-14
    for i in range(5):
        row = np.zeros(5, dtype=int)
        row[i] = 1
        q = int(np.nonzero((t == row).all(axis=1))[0][0])
        assert abs(p[q] - abs(A[i, j]) ** 2) <= 1e-14
