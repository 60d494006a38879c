"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/pq.h declares, rejects bad arguments on the host, and its
planner and Gray-code walk (the code the kernels run, compiled for the host)
behave as the method requires (Sec. 4.2: mixed-radix Gray code whose digit
for a row runs over 0..multiplicity)."""
import ctypes
import itertools
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

from paper_2403_04006_gb300 import build as B
from paper_2403_04006_gb300 import pq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pq.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return pq.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|const char\*)\s+(pq_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_named_calls():
    names = declared_functions()
    for must in ("pq_permanent_batched", "pq_bs_probs", "pq_permanent_backward",
                 "pq_bs_probs_backward", "pq_clements_forward", "pq_clements_backward",
                 "pq_plan_create", "pq_plan_create_bs", "pq_plan_destroy", "pq_autotune",
                 "pq_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_no_error(lib):
    assert "sm_103a" in pq.pq_version()


def test_host_argument_errors_without_gpu(lib):
    # null arguments are rejected before any CUDA call
    assert lib.pq_plan_create(None, None, None) == pq.PQ_ERR_ARG
    assert lib.pq_permanent_batched(None, None, None, None) == pq.PQ_ERR_ARG
    assert lib.pq_bs_probs(None, 4, None, None, 1, None, None, None, None) == pq.PQ_ERR_ARG
    assert lib.pq_clements_forward(None, None, 4, None, None) == pq.PQ_ERR_ARG
    assert "null" in pq.pq_last_error()


class ItemInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("k", ctypes.c_int32), ("l", ctypes.c_int32),
                ("transposed", ctypes.c_int32), ("ndig", ctypes.c_int32), ("J", ctypes.c_int32),
                ("terms", ctypes.c_int64), ("chunk_len", ctypes.c_int64),
                ("chunks", ctypes.c_int64), ("radix", ctypes.c_int32 * 48),
                ("row_of_digit", ctypes.c_int32 * 48)]


def item_info(lib, r, c, log2=0):
    r = np.ascontiguousarray(r, dtype=np.int32)
    c = np.ascontiguousarray(c, dtype=np.int32)
    info = ItemInfo()
    rc = lib.pq_plan_item_info(len(r), len(c), r.ctypes.data_as(ctypes.c_void_p),
                               c.ctypes.data_as(ctypes.c_void_p), log2, ctypes.byref(info))
    return rc, info


def side_terms(m):
    m = [x for x in m if x > 0]
    f = int(np.argmin(m))
    return int(np.prod([x if i == f else x + 1 for i, x in enumerate(m)]))


@pytest.mark.parametrize("r,c", [([1] * 12, [1] * 12), ([2, 1, 3], [1, 1, 1, 1, 1, 1]),
                                 ([1, 1, 1, 1], [4]), ([2, 2, 2], [3, 3]), ([3], [3]),
                                 ([0, 2, 0, 1], [1, 0, 2]), ([1] * 30, [1] * 30),
                                 ([1], [1]), ([0, 1], [1, 0]), ([2], [1, 1])])
def test_planner_side_choice_and_term_count(lib, r, c):
    rc, info = item_info(lib, r, c)
    assert rc == 0
    n = sum(r)
    assert info.n == n
    Tr, Tc = side_terms(r), side_terms(c)
    assert info.terms == min(Tr, Tc)
    assert info.transposed == (1 if Tc < Tr else 0)
    rad = list(info.radix[:info.ndig])
    # the chunk's (low) digits first, then the others, each in ascending radix
    assert rad[:info.J] == sorted(rad[:info.J]) and rad[info.J:] == sorted(rad[info.J:])
    assert math.prod(rad) == info.terms
    assert info.chunk_len == math.prod(rad[:info.J])
    assert info.chunks * info.chunk_len == info.terms
    # collision-free: Glynn's 2^(n-1) sign vectors
    if all(x == 1 for x in r) and all(x == 1 for x in c):
        assert info.terms == 2 ** (n - 1)


def test_planner_rejects(lib):
    assert item_info(lib, [1, 2], [1, 1])[0] == pq.PQ_ERR_ARG  # 3 != 2
    assert item_info(lib, [-1, 2], [1])[0] == pq.PQ_ERR_ARG
    # one column repeated 41 times is the cheap side to sum, which leaves 41
    # product-side columns: above PQ_MAX_PRODUCT_COLS
    assert item_info(lib, [1] * 41, [41])[0] == pq.PQ_ERR_UNSUPPORTED
    assert item_info(lib, [1] * 49, [1] * 49)[0] == pq.PQ_ERR_UNSUPPORTED  # n > PQ_MAX_N
    rc, info = item_info(lib, [0, 0], [0])
    assert rc == 0 and info.n == 0


@pytest.mark.parametrize("radix", [[2], [3], [2, 2, 2], [2, 3, 4], [3, 2, 4], [2, 2, 3, 3],
                                   [4, 4], [15], [2] * 10, [5, 3, 2]])
def test_gray_walk_visits_every_code_once_with_unit_steps(lib, radix):
    total = math.prod(radix)
    steps = total - 1
    rad = np.asarray(radix, dtype=np.int32)
    dig = np.zeros(max(steps, 1), dtype=np.int32)
    dr = np.zeros(max(steps, 1), dtype=np.int32)
    rc = lib.pq_gray_walk(rad.ctypes.data_as(ctypes.c_void_p), len(radix), steps,
                          dig.ctypes.data_as(ctypes.c_void_p), dr.ctypes.data_as(ctypes.c_void_p))
    assert rc == 0
    g = [0] * len(radix)
    seen = {tuple(g)}
    for s in range(steps):
        d, u = int(dig[s]), int(dr[s])
        assert u in (1, -1)
        g[d] += u
        assert 0 <= g[d] < radix[d]
        seen.add(tuple(g))
    assert len(seen) == total
    assert seen == set(itertools.product(*[range(x) for x in radix]))


def test_gray_walk_rejects_too_many_steps(lib):
    rad = np.asarray([2, 3], dtype=np.int32)
    buf = np.zeros(16, dtype=np.int32)
    assert lib.pq_gray_walk(rad.ctypes.data_as(ctypes.c_void_p), 2, 6,
                            buf.ctypes.data_as(ctypes.c_void_p),
                            buf.ctypes.data_as(ctypes.c_void_p)) == pq.PQ_ERR_ARG


def test_loop_poly_factors_closed_forms(lib):
    # N = 2: He_2 = x^2 - 1, one root z = -1/2;  N = 4: He_4 = x^4 - 6x^2 + 3
    # gives the pair a = 1, b = 1/12 (q^2/2 + q l^2/2 + l^4/24 = (q^2 + q s + s^2/12)/2)
    assert np.allclose(pq.pq_loop_poly_factors(2), [1.0, -0.5], rtol=1e-15, atol=0)
    assert np.allclose(pq.pq_loop_poly_factors(3), [1.0, -1.0 / 6.0], rtol=1e-15, atol=0)
    assert np.allclose(pq.pq_loop_poly_factors(4), [0.5, 1.0, 1.0 / 12.0], rtol=1e-14, atol=0)
    assert np.array_equal(pq.pq_loop_poly_factors(0), [1.0])
    assert np.array_equal(pq.pq_loop_poly_factors(1), [1.0])
    with pytest.raises(pq.PQError):
        pq.pq_loop_poly_factors(49)


@pytest.mark.parametrize("N", list(range(0, 49)))
def test_loop_poly_factors_reproduce_the_polynomial(lib, N):
    """The factored form equals sum_j q^j l^{N-2j} / (j! (N-2j)!) (the degree-N
    part of exp(q + l) used by the loop hafnian) at random points."""
    cf = pq.pq_loop_poly_factors(N)
    J, P = N // 2, N // 4
    rng = np.random.default_rng(N)
    for _ in range(4):
        q, l = complex(*rng.standard_normal(2)), complex(*rng.standard_normal(2))
        s = l * l
        terms = [q ** j * l ** (N - 2 * j) / (math.factorial(j) * math.factorial(N - 2 * j))
                 for j in range(J + 1)]
        direct, scale = sum(terms), sum(abs(t) for t in terms)
        h = cf[0]
        for p in range(P):
            h *= q * q + cf[1 + 2 * p] * q * s + cf[2 + 2 * p] * s * s
        if J % 2:
            h *= q - cf[1 + 2 * P] * s
        if N % 2:
            h *= l
        assert abs(h - direct) <= 1e-13 * scale, (N, h, direct)


def fixsum(lib, hi, lo):
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    out = np.zeros(2)
    rc = lib.pq_fixsum_host(hi.ctypes.data_as(ctypes.c_void_p), lo.ctypes.data_as(ctypes.c_void_p),
                            len(hi), out.ctypes.data_as(ctypes.c_void_p))
    return rc, out


def _trunc53(x):
    """Leading 53 bits of the rational x, truncated towards zero, as a double."""
    if x == 0:
        return 0.0
    s = -1 if x < 0 else 1
    a = abs(x)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    ulp = Fraction(2) ** (e - 52)
    return s * float(math.floor(a / ulp) * ulp)


@pytest.mark.parametrize("case", ["random", "cancel", "spread", "tiny", "signs"])
def test_exact_warp_sum_is_the_truncated_exact_sum(lib, case):
    """The forward kernels' lane reduction adds 32 double-double lane sums in
    128-bit integers: out[0] must be the exact sum's leading 53 bits and
    out[1] the rest's, for inputs whose bits all lie within 2^-64 of the
    largest value's last bit (then nothing is dropped); zeros, cancellation,
    subnormal-free spreads of exponent and mixed signs."""
    rng = np.random.default_rng({"random": 1, "cancel": 2, "spread": 3, "tiny": 4, "signs": 5}[case])
    n = 32
    hi = rng.standard_normal(n) * 2.0 ** rng.integers(-8, 8, n)
    if case == "cancel":
        hi[16:] = -hi[:16] * (1 + 2.0 ** -50)
    if case == "spread":
        hi = hi * 2.0 ** rng.integers(-10, 0, n)
    if case == "tiny":
        hi = hi * 1e-280
    if case == "signs":
        hi[::3] = 0.0
    lo = np.array([h * 2.0 ** -53 * u for h, u in zip(hi, rng.uniform(-1, 1, n))])
    # keep every bit within 2^-64 of the largest value's last significand bit
    unit = 2.0 ** (math.frexp(float(np.abs(hi).max()))[1] - 1 - 52 - 64)
    lo = np.round(lo / unit) * unit
    rc, out = fixsum(lib, hi, lo)
    assert rc == 0
    exact = sum((Fraction(float(h)) + Fraction(float(l)) for h, l in zip(hi, lo)), Fraction(0))
    assert out[0] == _trunc53(exact)
    assert out[1] == _trunc53(exact - Fraction(float(out[0])))


def test_exact_warp_sum_drops_only_bits_far_below_the_largest(lib):
    """A value more than 64 bits below the largest one's last bit is dropped
    (truncated), an error below 2^-116 relative to the largest; lane counts 0
    and 1; bad arguments."""
    hi = np.array([1.0, 2.0 ** -120, -(2.0 ** -125)])
    lo = np.array([2.0 ** -60, 0.0, 0.0])
    rc, out = fixsum(lib, hi, lo)
    assert rc == 0
    exact = Fraction(1) + Fraction(2) ** -60
    assert Fraction(float(out[0])) + Fraction(float(out[1])) == exact
    rc, out = fixsum(lib, [], [])
    assert rc == 0 and out[0] == 0.0 and out[1] == 0.0
    rc, out = fixsum(lib, [-3.5], [2.0 ** -60])
    assert rc == 0 and Fraction(float(out[0])) + Fraction(float(out[1])) == Fraction(-7, 2) + Fraction(2) ** -60
    assert fixsum(lib, [np.inf], [0.0])[0] == pq.PQ_ERR_ARG
    assert fixsum(lib, np.ones(33), np.zeros(33))[0] == pq.PQ_ERR_ARG


def test_chunk_digits_fill_the_warp_tasks(lib):
    """The batched cut may take any radices as a chunk's digits: rows
    (2, 2, 2, 3, 3) against 12 single columns give Gray radices 2, 3, 3, 4, 4
    (T = 288); the prefix cut (2, 3: chunks of 6) leaves 48 chunks, two warp
    tasks with 16 idle lanes, while the chunk digits (3, 3) give 32 chunks of
    9 terms, one full task."""
    rc, info = item_info(lib, [2, 2, 2, 3, 3], [1] * 12)
    assert rc == 0 and info.terms == 288
    rad = list(info.radix[:info.ndig])
    assert sorted(rad) == [2, 3, 3, 4, 4]
    assert rad[:info.J] == [3, 3] and info.chunk_len == 9 and info.chunks == 32
