"""Exact rational arithmetic for pinning the oracle (test helper).

Every IEEE double is a dyadic rational, so a complex128 matrix scaled by a
common power of two is a matrix of Gaussian integers.  Permanents of such
matrices are computed here exactly with Python integers: once from the
definition (Eq. (per_def), sum over permutations) and once by grouped Ryser
enumeration in exact arithmetic.  No floating point is involved until the
final comparison, so these values carry no rounding error at all.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np


def to_gaussian_ints(a):
    """(re, im, E): integer arrays (Python ints, object dtype) with
    a == (re + i im) / 2^E exactly."""
    a = np.asarray(a, dtype=np.complex128)
    parts = [float(x) for x in a.real.ravel()] + [float(x) for x in a.imag.ravel()]
    E = 0
    for x in parts:
        den = x.as_integer_ratio()[1]
        E = max(E, den.bit_length() - 1)

    def conv(x):
        p, q = float(x).as_integer_ratio()
        return p * ((1 << E) // q)

    re = np.array([conv(x) for x in a.real.ravel()], dtype=object).reshape(a.shape)
    im = np.array([conv(x) for x in a.imag.ravel()], dtype=object).reshape(a.shape)
    return re, im, E


def _gmul(x, y):
    return (x[0] * y[0] - x[1] * y[1], x[0] * y[1] + x[1] * y[0])


def exact_perm_definition(a) -> tuple[Fraction, Fraction]:
    """per(a) = sum_sigma prod_i a[sigma(i), i], exactly (n <= 8)."""
    re, im, E = to_gaussian_ints(a)
    n = re.shape[0]
    tot = (0, 0)
    for sigma in itertools.permutations(range(n)):
        t = (1, 0)
        for i in range(n):
            t = _gmul(t, (re[sigma[i], i], im[sigma[i], i]))
        tot = (tot[0] + t[0], tot[1] + t[1])
    scale = 1 << (E * n)
    return Fraction(tot[0], scale), Fraction(tot[1], scale)


def exact_perm_grouped(b, r, c) -> tuple[Fraction, Fraction]:
    """Permanent of the matrix repeating row i r[i] times and column j c[j]
    times, exactly, by the grouped inclusion-exclusion sum
    (-1)^n sum_k (-1)^{sum k} prod C(r_i,k_i) prod_j (sum_i k_i b_ij)^{c_j}."""
    re, im, E = to_gaussian_ints(b)
    k, l = re.shape
    n = int(sum(int(x) for x in r))
    assert n == int(sum(int(x) for x in c))
    tot = (0, 0)
    for ks in itertools.product(*[range(int(ri) + 1) for ri in r]):
        w = 1
        for i in range(k):
            w *= math.comb(int(r[i]), ks[i])
        if sum(ks) % 2:
            w = -w
        p = (w, 0)
        for j in range(l):
            s = (sum(ks[i] * re[i, j] for i in range(k)), sum(ks[i] * im[i, j] for i in range(k)))
            for _ in range(int(c[j])):
                p = _gmul(p, s)
        tot = (tot[0] + p[0], tot[1] + p[1])
    if n % 2:
        tot = (-tot[0], -tot[1])
    scale = 1 << (E * n)
    return Fraction(tot[0], scale), Fraction(tot[1], scale)


def abs_err(value: complex, exact: tuple[Fraction, Fraction]) -> float:
    """|value - exact| evaluated exactly, then rounded."""
    dr = Fraction(value.real) - exact[0]
    di = Fraction(value.imag) - exact[1]
    return math.sqrt(float(dr * dr + di * di))


def to_complex(exact: tuple[Fraction, Fraction]) -> complex:
    return complex(float(exact[0]), float(exact[1]))
