"""Pins of the CPU oracle against what the paper and mathematics fix.

Each check below would fail under a plausible bug in the oracle: a dropped
term, a wrong sign, a wrong binomial weight, a transposed operand or index,
or rounding beyond the stated bound.  None of them compares the oracle with
itself.  Passages: Eq. (per_def) and Eq. (BS_prob) (Appendix A, "Particle
number measurement"); row/column multiplicities (Sec. 4.2, "Boson
Sampling"); beamsplitter block (Appendix A, "Beamsplitter gate").
"""
import math

import numpy as np
import pytest

import oracle as O
from exact import abs_err, exact_perm_definition, exact_perm_grouped, to_complex

RNG = np.random.default_rng(20240306)


def crandn(*shape, rng=RNG):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def expand(B, r, c):
    return np.repeat(np.repeat(np.asarray(B), r, axis=0), c, axis=1)


# ---------------------------------------------------------------- definition
def test_hand_computed_values():
    # 2x2: per [[a,b],[c,d]] = ad + bc
    assert O.perm_bruteforce([[1, 2], [3, 4]]) == 10
    # 3x3 of 1..9: 45 + 48 + 72 + 84 + 96 + 105
    assert O.perm_bruteforce(np.arange(1, 10).reshape(3, 3)) == 450
    assert O.perm_ryser(np.arange(1, 10).reshape(3, 3)) == 450
    # [[i,1],[1,i]]: i*i + 1*1 = 0 (the HOM cancellation in miniature)
    assert O.perm_bruteforce([[1j, 1], [1, 1j]]) == 0
    assert O.perm_ryser(np.array([[1j, 1], [1, 1j]])) == 0
    # column index convention: A[sigma(i), i] with a non-symmetric 3x3
    A = np.array([[1, 2, 0], [0, 1, 5], [3, 0, 1]], dtype=float)
    # permutations with nonzero products: identity (1*1*1) and the 3-cycle 2*5*3
    assert O.perm_bruteforce(A) == 31
    assert O.perm_ryser(A) == 31


def test_exact_helpers_agree_on_definition():
    """The exact grouped sum equals the exact permutation sum (n <= 6)."""
    for n in range(1, 7):
        A = np.round(crandn(n, n) * 8) / 8
        assert exact_perm_definition(A) == exact_perm_grouped(A, [1] * n, [1] * n)
    B = np.round(crandn(3, 2) * 4) / 4
    r, c = [2, 1, 2], [3, 2]
    assert exact_perm_definition(expand(B, r, c)) == exact_perm_grouped(B, r, c)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 8])
def test_bruteforce_matches_exact(n):
    A = crandn(n, n)
    ex = exact_perm_definition(A)
    val = O.perm_bruteforce(A)
    assert abs_err(val, ex) <= 1e-13 * max(1.0, abs(to_complex(ex)))


# ---------------------------------------------------------------- Ryser vs exact
@pytest.mark.parametrize("gold", [False, True])
@pytest.mark.parametrize("n", [1, 2, 4, 7, 10, 13])
def test_ryser_within_bound_of_exact(n, gold):
    A = crandn(n, n) / math.sqrt(2 * n)
    ex = exact_perm_grouped(A, [1] * n, [1] * n)
    per, sumabs, bound = O.perm_ryser(A, gold=gold, info=True)
    err = abs_err(per, ex)
    assert err <= bound, (err, bound)
    assert err <= 1e-11 * sumabs


@pytest.mark.parametrize("gold", [False, True])
def test_ryser_multiplicities_within_bound_of_exact(gold):
    rng = np.random.default_rng(7)
    for trial in range(12):
        k = int(rng.integers(1, 5))
        l = int(rng.integers(1, 5))
        r = rng.integers(1, 4, size=k)
        c = list(rng.integers(1, 4, size=l))
        # adjust the column multiplicities to the same total
        n = int(r.sum())
        while sum(c) < n:
            c[int(rng.integers(0, l))] += 1
        while sum(c) > n:
            j = int(rng.integers(0, l))
            if c[j] > 1:
                c[j] -= 1
            elif all(x == 1 for x in c):
                break
        if sum(c) != n:
            continue
        B = crandn(k, l, rng=rng) / 2
        ex = exact_perm_grouped(B, r, c)
        per, sumabs, bound = O.perm_ryser(B, r, c, gold=gold, info=True)
        assert abs_err(per, ex) <= bound


def test_multiplicities_equal_expanded_matrix():
    """Grouped rows/columns == Ryser on the expanded matrix == brute force."""
    rng = np.random.default_rng(11)
    cases = [([2, 1, 1], [1, 3]), ([3], [1, 1, 1]), ([1, 2, 2], [2, 2, 1]), ([2, 2], [1, 1, 1, 1])]
    for r, c in cases:
        B = crandn(len(r), len(c), rng=rng)
        A = expand(B, r, c)
        g = O.perm_ryser(B, r, c)
        e = O.perm_ryser(A)
        bf = O.perm_bruteforce(A)
        scale = max(1.0, abs(bf))
        assert abs(g - bf) <= 1e-12 * scale
        assert abs(e - bf) <= 1e-12 * scale


def test_zero_multiplicity_rows_and_columns_drop_out():
    B = crandn(3, 3)
    full = O.perm_ryser(B[[0, 2]][:, [1, 2]], [2, 1], [1, 2])
    assert abs(O.perm_ryser(B, [2, 0, 1], [0, 1, 2]) - full) <= 1e-13 * max(1, abs(full))


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [1, 2, 3, 6, 9, 12, 16, 20])
def test_all_ones_is_factorial(n):
    # Ryser's terms reach ~n^n here, so fast mode is only as good as its
    # a-posteriori bound (the precision gap Sec. 4.2 describes); gold is tight.
    per, _, bound = O.perm_ryser(np.ones((n, n)), info=True)
    assert abs(per - math.factorial(n)) <= bound
    g = O.perm_ryser(np.ones((n, n)), gold=True)
    assert abs(g - math.factorial(n)) <= 1e-15 * math.factorial(n)


def derangements(n):
    d = [1, 0]
    for i in range(2, n + 1):
        d.append((i - 1) * (d[i - 1] + d[i - 2]))
    return d[n]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 8, 12, 16, 18])
def test_ones_minus_identity_is_derangements(n):
    A = np.ones((n, n)) - np.eye(n)
    per, _, bound = O.perm_ryser(A, info=True)
    assert abs(per - derangements(n)) <= bound
    g = O.perm_ryser(A, gold=True)
    assert abs(g - derangements(n)) <= 1e-15 * max(1, derangements(n))


def test_diagonal_and_triangular():
    d = crandn(9)
    assert abs(O.perm_ryser(np.diag(d)) - np.prod(d)) <= 1e-13 * abs(np.prod(d))
    T = np.triu(crandn(9, 9))
    want = np.prod(np.diag(T))
    per, _, bound = O.perm_ryser(T, info=True)  # heavy cancellation: judge by the bound
    assert abs(per - want) <= bound
    assert abs(O.perm_ryser(T, gold=True) - want) <= 1e-14 * abs(want)
    assert abs(O.perm_bruteforce(T[:7, :7]) - np.prod(np.diag(T)[:7])) <= 1e-12 * abs(
        np.prod(np.diag(T)[:7]))


def test_scaling_transpose_and_permutations():
    n = 9
    A = crandn(n, n)
    d1, d2 = crandn(n), crandn(n)
    p = O.perm_ryser(A)
    scaled = O.perm_ryser(np.diag(d1) @ A @ np.diag(d2))
    assert abs(scaled - np.prod(d1) * np.prod(d2) * p) <= 1e-11 * abs(scaled)
    assert abs(O.perm_ryser(A.T) - p) <= 1e-12 * abs(p)
    pr, pc = RNG.permutation(n), RNG.permutation(n)
    assert abs(O.perm_ryser(A[pr][:, pc]) - p) <= 1e-12 * abs(p)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_single_entry_repeated(n):
    """1x1 base a with r = c = n: the expanded matrix is a*J_n, per = n! a^n.
    This exercises the binomial weights of one digit with radix n+1."""
    a = 0.7 - 0.4j
    per, _, bound = O.perm_ryser([[a]], [n], [n], info=True)
    want = math.factorial(n) * a ** n
    assert abs(per - want) <= max(bound, 1e-14 * abs(want))


def test_laplace_row_expansion():
    n = 8
    A = crandn(n, n)
    p = O.perm_ryser(A)
    for i in (0, 3, 7):
        acc = 0j
        for j in range(n):
            minor = np.delete(np.delete(A, i, axis=0), j, axis=1)
            acc += A[i, j] * O.perm_ryser(minor)
        assert abs(acc - p) <= 1e-11 * abs(p)


def test_threads_do_not_change_result_beyond_bound():
    A = crandn(16, 16) / 4
    p1, _, b1 = O.perm_ryser(A, nthreads=1, info=True)
    p8, _, b8 = O.perm_ryser(A, nthreads=8, info=True)
    assert abs(p1 - p8) <= b1 + b8


def test_gold_and_fast_agree_n22():
    A = crandn(22, 22) / math.sqrt(44)
    f, _, bf = O.perm_ryser(A, nthreads=8, info=True)
    g, _, bg = O.perm_ryser(A, gold=True, nthreads=8, info=True)
    assert abs(f - g) <= bf + bg
    assert bg < 1e-6 * bf


def test_argument_errors():
    with pytest.raises(ValueError):
        O.perm_ryser(crandn(2, 2), [1, 1], [1, 2])  # sum r != sum c
    with pytest.raises(ValueError):
        O.perm_ryser(crandn(2, 2), [1, -1], [0, 0])
    assert O.perm_ryser(np.zeros((0, 0))) == 1


# ---------------------------------------------------------------- gradients
def test_grad_matches_finite_differences():
    rng = np.random.default_rng(5)
    B = crandn(3, 4, rng=rng)
    r, c = [2, 1, 2], [1, 2, 1, 1]
    G = O.perm_grad(B, r, c)
    h = 1e-6
    for i in range(3):
        for j in range(4):
            E = np.zeros_like(B)
            E[i, j] = h
            d_re = (O.perm_ryser(B + E, r, c) - O.perm_ryser(B - E, r, c)) / (2 * h)
            d_im = (O.perm_ryser(B + 1j * E, r, c) - O.perm_ryser(B - 1j * E, r, c)) / (2 * h)
            # holomorphic: d/dRe = dP/db, d/dIm = i dP/db
            assert abs(d_re - G[i, j]) <= 1e-7 * np.abs(G).max()
            assert abs(d_im - 1j * G[i, j]) <= 1e-7 * np.abs(G).max()


def test_grad_euler_homogeneity():
    """per is homogeneous of degree r_i in base row i and c_j in column j."""
    B = crandn(4, 3)
    r, c = [1, 2, 1, 3], [3, 2, 2]
    p = O.perm_ryser(B, r, c)
    G = O.perm_grad(B, r, c)
    for i in range(4):
        assert abs(np.sum(B[i] * G[i]) - r[i] * p) <= 1e-12 * max(1, abs(p)) * 10
    for j in range(3):
        assert abs(np.sum(B[:, j] * G[:, j]) - c[j] * p) <= 1e-12 * max(1, abs(p)) * 10


def test_grad_of_expanded_matrix_sums_entries():
    """d per / d b_ij of the grouped form = sum of d per(A)/dA over the r_i c_j
    copies, where the expanded gradient is checked entry by entry from minors."""
    B = crandn(2, 2)
    r, c = [2, 1], [1, 2]
    A = expand(B, r, c)
    GA = O.perm_grad(A)
    rowmap = np.repeat(np.arange(2), r)
    colmap = np.repeat(np.arange(2), c)
    G = O.perm_grad(B, r, c)
    for i in range(2):
        for j in range(2):
            want = GA[np.ix_(rowmap == i, colmap == j)].sum()
            assert abs(G[i, j] - want) <= 1e-13 * max(1, abs(want))
    # and the expanded gradient itself is the minor permanent
    for p in range(3):
        for q in range(3):
            minor = np.delete(np.delete(A, p, axis=0), q, axis=1)
            assert abs(GA[p, q] - O.perm_bruteforce(minor)) <= 1e-13 * 10


# ---------------------------------------------------------------- boson sampling
def haar(m, rng):
    z = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / math.sqrt(2)
    q, rr = np.linalg.qr(z)
    d = np.diagonal(rr)
    return q * (d / np.abs(d))[None, :]


def all_patterns(n, m):
    if m == 1:
        return [[n]]
    return [[v] + rest for v in range(n + 1) for rest in all_patterns(n - v, m - 1)]


def test_probabilities_sum_to_one():
    """Unitarity: sum_t p(s, t) = 1 over all C(n+m-1, n) outputs."""
    rng = np.random.default_rng(1001)
    U = haar(8, rng)
    s = [1, 1, 1, 1, 0, 0, 0, 0]
    t = np.array(all_patterns(4, 8))
    assert t.shape[0] == math.comb(11, 4)
    p, _ = O.bs_probs(U, s, t)
    assert abs(p.sum() - 1.0) <= 1e-13
    assert (p >= 0).all()
    # with a repeated input mode as well
    s2 = [2, 0, 1, 0, 1, 0, 0, 0]
    p2, _ = O.bs_probs(U, s2, t)
    assert abs(p2.sum() - 1.0) <= 1e-13


def test_single_photon_probability():
    rng = np.random.default_rng(3)
    U = haar(5, rng)
    for i in range(5):
        for j in range(5):
            s = np.zeros(5, dtype=int)
            s[j] = 1
            t = np.zeros(5, dtype=int)
            t[i] = 1
            p, a = O.bs_probs(U, s, t[None])
            # U[out, in]: output mode i, input mode j
            assert abs(p[0] - abs(U[i, j]) ** 2) <= 1e-15
            assert abs(a[0] - U[i, j]) <= 1e-15


def test_hong_ou_mandel():
    """50:50 beamsplitter (theta = pi/4) on |1,1>: p(1,1) = 0, p(2,0) = p(0,2) = 1/2."""
    U = O.beamsplitter_block(math.pi / 4, 0.3)
    p, _ = O.bs_probs(U, [1, 1], np.array([[1, 1], [2, 0], [0, 2]]))
    assert abs(p[0]) <= 1e-16
    assert abs(p[1] - 0.5) <= 1e-15 and abs(p[2] - 0.5) <= 1e-15


def test_two_photons_same_mode_normalisation():
    """|2,0> through a beamsplitter: p(2,0) = |t|^4, p(1,1) = 2|t|^2|r|^2,
    p(0,2) = |r|^4 (binomial law), which fixes the factorial normalisation."""
    th, ph = 0.37, 1.1
    U = O.beamsplitter_block(th, ph)
    p, _ = O.bs_probs(U, [2, 0], np.array([[2, 0], [1, 1], [0, 2]]))
    c2, s2 = math.cos(th) ** 2, math.sin(th) ** 2
    assert np.allclose(p, [c2 * c2, 2 * c2 * s2, s2 * s2], rtol=0, atol=1e-15)


def test_bs_grad_matches_finite_differences():
    rng = np.random.default_rng(9)
    U = haar(4, rng)
    s = [1, 1, 0, 1]
    t = np.array([[1, 0, 2, 0], [0, 1, 1, 1], [3, 0, 0, 0], [1, 1, 1, 0]])
    g = rng.uniform(0.5, 1.5, size=len(t))
    G = O.bs_grad_U(U, s, t, g)
    h = 1e-6

    def L(V):
        p, _ = O.bs_probs(V, s, t)
        return float(np.dot(g, p))

    for a in range(4):
        for b in range(4):
            E = np.zeros((4, 4), dtype=complex)
            E[a, b] = h
            dre = (L(U + E) - L(U - E)) / (2 * h)
            dim = (L(U + 1j * E) - L(U - 1j * E)) / (2 * h)
            assert abs(dre - G[a, b].real) <= 1e-7 * np.abs(G).max()
            assert abs(dim - G[a, b].imag) <= 1e-7 * np.abs(G).max()


# ---------------------------------------------------------------- Clements mesh
def test_clements_layout_counts():
    js = O.clements_layout(16)
    assert len(js) == 120
    assert js[:8] == [0, 2, 4, 6, 8, 10, 12, 14] and js[8:15] == [1, 3, 5, 7, 9, 11, 13]


def test_beamsplitter_block_matches_paper():
    th, ph = 0.3, 1.2
    Bk = O.beamsplitter_block(th, ph)
    t, r = math.cos(th), np.exp(1j * ph) * math.sin(th)
    assert np.allclose(Bk, [[t, -np.conj(r)], [r, t]], atol=0, rtol=0)
    assert np.allclose(Bk @ Bk.conj().T, np.eye(2), atol=1e-15)


def test_clements_unitary_structure():
    rng = np.random.default_rng(17)
    m = 16
    th = rng.uniform(0, 2 * math.pi, 120)
    ph = rng.uniform(0, 2 * math.pi, 120)
    U = O.clements_unitary(th, ph, m)
    assert np.abs(U @ U.conj().T - np.eye(m)).max() <= 1e-13
    assert np.abs(O.clements_unitary(np.zeros(120), ph, m) - np.eye(m)).max() == 0
    # one active beamsplitter k sits on modes (j, j+1)
    for k in (0, 9, 119):
        th1 = np.zeros(120)
        th1[k] = 0.8
        V = O.clements_unitary(th1, ph, m)
        j = O.clements_layout(m)[k]
        W = np.eye(m, dtype=complex)
        W[j:j + 2, j:j + 2] = O.beamsplitter_block(0.8, ph[k])
        assert np.abs(V - W).max() <= 1e-15
    # order: T_1 T_0 (T_0 acts first) on overlapping pairs (0,1) then (1,2)
    m3 = 3
    js = O.clements_layout(m3)  # [0, 1, 0]
    th3 = np.array([0.4, 0.9, 0.0])
    ph3 = np.array([0.1, 0.7, 0.0])
    T0 = np.eye(3, dtype=complex)
    T0[0:2, 0:2] = O.beamsplitter_block(0.4, 0.1)
    T1 = np.eye(3, dtype=complex)
    T1[1:3, 1:3] = O.beamsplitter_block(0.9, 0.7)
    assert js == [0, 1, 0]
    assert np.abs(O.clements_unitary(th3, ph3, 3) - T1 @ T0).max() <= 1e-15


def test_clements_grad_matches_finite_differences():
    rng = np.random.default_rng(23)
    m = 6
    L = m * (m - 1) // 2
    th = rng.uniform(0, 2 * math.pi, L)
    ph = rng.uniform(0, 2 * math.pi, L)
    C = crandn(m, m, rng=rng)

    def loss(a, b):  # a real function of U: Re sum conj(C) U
        return float(np.real(np.sum(np.conj(C) * O.clements_unitary(a, b, m))))

    gt, gp = O.clements_grad(th, ph, m, C)  # dL/dU = C for this loss
    h = 1e-6
    for k in range(L):
        e = np.zeros(L)
        e[k] = h
        assert abs((loss(th + e, ph) - loss(th - e, ph)) / (2 * h) - gt[k]) <= 1e-8
        assert abs((loss(th, ph + e) - loss(th, ph - e)) / (2 * h) - gp[k]) <= 1e-8
