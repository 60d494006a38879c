"""Pins of the oracle's hafnian (Eq. (haf_def), Sec. 4.1): hand values, closed
forms, exact arithmetic, and the grouped formula against the definition on
expanded matrices."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from exact import to_gaussian_ints

RNG = np.random.default_rng(4242)


def sym(k, rng=RNG):
    a = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    return (a + a.T) / 2


def expand(B, r):
    return np.repeat(np.repeat(np.asarray(B), r, axis=0), r, axis=1)


def double_factorial(m):
    return math.prod(range(m, 0, -2)) if m > 0 else 1


def exact_haf(a):
    """Exact hafnian by recursion over perfect matchings on Gaussian integers."""
    re, im, E = to_gaussian_ints(a)
    N = re.shape[0]

    def rec(rem):
        if not rem:
            return (1, 0)
        p, rest = rem[0], rem[1:]
        tot = (0, 0)
        for idx, q in enumerate(rest):
            sub = rec(rest[:idx] + rest[idx + 1:])
            x = (re[p, q], im[p, q])
            prod = (x[0] * sub[0] - x[1] * sub[1], x[0] * sub[1] + x[1] * sub[0])
            tot = (tot[0] + prod[0], tot[1] + prod[1])
        return tot

    t = rec(tuple(range(N)))
    scale = 1 << (E * (N // 2))
    return complex(float(Fraction(t[0], scale)), float(Fraction(t[1], scale)))


def test_hand_values():
    a = np.array([[0, 2, 3, 4], [2, 0, 5, 6], [3, 5, 0, 7], [4, 6, 7, 0]], dtype=float)
    # matchings {01,23}, {02,13}, {03,12}: 2*7 + 3*6 + 4*5
    assert O.haf_bruteforce(a) == 52
    assert O.haf_bruteforce([[9.0, 1.5], [1.5, 9.0]]) == 1.5  # diagonal never used
    assert O.haf_bruteforce(np.zeros((0, 0))) == 1
    assert abs(O.haf_grouped(a) - 52) <= 1e-12


@pytest.mark.parametrize("N", [2, 4, 6, 8, 10])
def test_all_ones_counts_perfect_matchings(N):
    want = double_factorial(N - 1)
    assert O.haf_bruteforce(np.ones((N, N))) == want
    assert abs(O.haf_grouped(np.ones((N, N))) - want) <= 1e-12 * want
    # one base index repeated N times expands to the same all-ones matrix
    assert abs(O.haf_grouped([[1.0]], [N]) - want) <= 1e-12 * want


def test_block_diagonal_pairs_and_scaling():
    vals = [0.3 + 1j, -1.2, 0.5 - 0.25j]
    a = np.zeros((6, 6), dtype=complex)
    for q, v in enumerate(vals):
        a[2 * q, 2 * q + 1] = a[2 * q + 1, 2 * q] = v
    assert abs(O.haf_bruteforce(a) - np.prod(vals)) <= 1e-15
    assert abs(O.haf_grouped(a) - np.prod(vals)) <= 1e-14
    b = sym(6)
    d = RNG.standard_normal(6) + 1j * RNG.standard_normal(6)
    h = O.haf_bruteforce(b)
    assert abs(O.haf_bruteforce(np.diag(d) @ b @ np.diag(d)) - np.prod(d) * h) <= 1e-12 * abs(h) * 10


@pytest.mark.parametrize("N", [2, 4, 6, 8])
def test_bruteforce_matches_exact(N):
    a = sym(N)
    assert abs(O.haf_bruteforce(a) - exact_haf(a)) <= 1e-13 * max(1, abs(exact_haf(a)))


@pytest.mark.parametrize("r", [[1, 1, 1, 1], [2, 2], [2, 1, 1], [3, 1], [2, 2, 2], [1, 3, 2, 2],
                               [4], [2, 2, 2, 2]])
def test_grouped_formula_matches_definition_on_expanded_matrix(r):
    B = sym(len(r))
    A = expand(B, r)
    ref = O.haf_bruteforce(A)
    got, scale = O.haf_grouped(B, r, info=True)
    assert abs(got - ref) <= 1e-13 * max(abs(ref), scale)


def test_odd_size_is_zero():
    assert O.haf_grouped(sym(3), [1, 1, 1]) == 0
    with pytest.raises(ValueError):
        O.haf_bruteforce(np.ones((3, 3)))


# ---------------------------------------------------------------- loop hafnian

def telephone(N):
    """Number of involutions of N elements (matchings with loops of K_N)."""
    t = [1, 1]
    for m in range(2, N + 1):
        t.append(t[-1] + (m - 1) * t[-2])
    return t[N]


def filldiag(B, gamma, r):
    A = expand(B, r)
    np.fill_diagonal(A, np.repeat(np.asarray(gamma), r))
    return A


def exact_lhaf(a):
    """Exact loop hafnian on Gaussian integers (loops from the diagonal)."""
    re, im, E = to_gaussian_ints(a)
    N = re.shape[0]

    def mul(x, y):
        return (x[0] * y[0] - x[1] * y[1], x[0] * y[1] + x[1] * y[0])

    def rec(rem):
        # returns (value, number of loops used is folded into the scale below)
        if not rem:
            return {0: (1, 0)}
        p, rest = rem[0], rem[1:]
        out = {}
        for loops, v in rec(rest).items():  # p takes its loop
            w = mul((re[p, p], im[p, p]), v)
            o = out.get(loops + 1, (0, 0))
            out[loops + 1] = (o[0] + w[0], o[1] + w[1])
        for idx, q in enumerate(rest):
            for loops, v in rec(rest[:idx] + rest[idx + 1:]).items():
                w = mul((re[p, q], im[p, q]), v)
                o = out.get(loops, (0, 0))
                out[loops] = (o[0] + w[0], o[1] + w[1])
        return out

    tot_re, tot_im = Fraction(0), Fraction(0)
    for loops, v in rec(tuple(range(N))).items():
        factors = loops + (N - loops) // 2  # entries multiplied in each product
        scale = 1 << (E * factors)
        tot_re += Fraction(v[0], scale)
        tot_im += Fraction(v[1], scale)
    return complex(float(tot_re), float(tot_im))


@pytest.mark.parametrize("N", [0, 1, 2, 3, 4, 5, 6, 7, 8])
def test_lhaf_all_ones_counts_involutions(N):
    want = telephone(N)
    assert O.lhaf_bruteforce(np.ones((N, N))) == want
    if N:
        assert abs(O.lhaf_grouped([[1.0]], [1.0], [N]) - want) <= 1e-12 * want
        assert abs(O.lhaf_grouped(np.ones((N, N)), np.ones(N)) - want) <= 1e-12 * want


def test_lhaf_reduces_to_haf_and_to_diagonal_product():
    B = sym(6)
    np.fill_diagonal(B, 0)
    assert abs(O.lhaf_bruteforce(B) - O.haf_bruteforce(B)) <= 1e-14 * abs(O.haf_bruteforce(B))
    g0 = np.zeros(6)
    assert abs(O.lhaf_grouped(B, g0) - O.haf_bruteforce(B)) <= 1e-12 * abs(O.haf_bruteforce(B))
    d = RNG.standard_normal(5) + 1j * RNG.standard_normal(5)
    D = np.diag(d)
    assert abs(O.lhaf_bruteforce(D) - np.prod(d)) <= 1e-14
    assert abs(O.lhaf_grouped(np.zeros((5, 5)), d) - np.prod(d)) <= 1e-13


def test_lhaf_hand_value_three():
    # 3 x 3: three loops, or one pair and the remaining loop
    a = np.array([[2.0, 3, 5], [3, 7, 11], [5, 11, 13]])
    want = 2 * 7 * 13 + 3 * 13 + 5 * 7 + 11 * 2
    assert O.lhaf_bruteforce(a) == want
    assert abs(O.lhaf_grouped(a, np.diag(a)) - want) <= 1e-12 * want


@pytest.mark.parametrize("N", [1, 2, 5, 8, 11])
def test_lhaf_single_index_closed_form(N):
    # one index repeated N times: sum_j C(N, 2j) (2j-1)!! b^j c^{N-2j}
    b, c = 0.7 - 0.2j, -0.4 + 0.9j
    want = sum(math.comb(N, 2 * j) * double_factorial(2 * j - 1) * b ** j * c ** (N - 2 * j)
               for j in range(N // 2 + 1))
    got = O.lhaf_grouped([[b]], [c], [N])
    assert abs(got - want) <= 1e-13 * max(1.0, abs(want))


@pytest.mark.parametrize("N", [3, 4, 6, 7])
def test_lhaf_bruteforce_matches_exact(N):
    a = sym(N)
    ref = exact_lhaf(a)
    assert abs(O.lhaf_bruteforce(a) - ref) <= 1e-13 * max(1, abs(ref))


@pytest.mark.parametrize("r", [[1, 1, 1], [2, 1], [2, 2], [3, 1, 1], [1, 2, 2, 2], [5],
                               [2, 2, 2, 1], [1, 0, 3]])
def test_lhaf_grouped_matches_definition_on_filled_matrix(r):
    B = sym(len(r))
    gamma = RNG.standard_normal(len(r)) + 1j * RNG.standard_normal(len(r))
    ref = O.lhaf_bruteforce(filldiag(B, gamma, r))
    got, scale = O.lhaf_grouped(B, gamma, r, info=True)
    assert abs(got - ref) <= 1e-13 * max(abs(ref), scale)
