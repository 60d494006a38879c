"""CPU oracle for permanents with repeated rows/columns, boson-sampling
probabilities and their gradients, and for the Clements beamsplitter mesh.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_2403_04006_gb300``):
neither imports the other, and the two meet only through the seeded inputs of
``paper_2403_04006_gb300.workloads``.

The arithmetic lives in ``pq_oracle.c`` (plain C, built with
``-ffp-contract=off``); this module only marshals numpy arrays into it, except
for the Clements mesh (``clements.py``, numpy).  Paper: "Piquasso: A Photonic
Quantum Computer Simulation Software Platform", arXiv 2403.04006.

Functions and the passage each follows:

* ``perm_bruteforce``      -- Eq. (per_def), Appendix A "Particle number measurement".
* ``perm_ryser``           -- Ryser's formula (the variant Sec. 4.2 "Boson Sampling"
                              compares BB/FG against), with the row/column
                              multiplicities of Sec. 4.2 grouped into binomials.
* ``perm_batch``           -- the same, over a ragged batch.
* ``perm_grad``            -- Laplace-minor derivative of Eq. (per_def).
* ``bs_probs``             -- Eq. (BS_prob).
* ``haf_*``                -- Eq. (haf_def), by matchings and by the grouped
                              sign-vector formula for repeated indices (Sec. 4.1).
* ``lhaf_*``               -- Eq. (loop_hafnian) with the filldiag of the
                              displaced detection probability, the same two ways.
* ``bs_grad_U``            -- chain rule through Eq. (BS_prob) and ``perm_grad``.
* ``clements_*``           -- beamsplitter matrix of Appendix A "Beamsplitter gate",
                              arranged as a Clements mesh (layout is a reading, the
                              paper only says the interferometer is decomposed into
                              beamsplitters, Fig. BS_Setup).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .clements import (clements_layout, beamsplitter_block, clements_unitary,  # noqa: F401
                       clements_grad)
from .sampler import algorithm_a  # noqa: F401
from .lossy import lossy_probs  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pq_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0


def build(force: bool = False) -> str:
    """Compile ``pq_oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_int64)
        i64 = ctypes.c_int64
        ci = ctypes.c_int
        lib.oracle_perm_bruteforce.argtypes = [dp, ci, dp]
        lib.oracle_perm_ryser.argtypes = [dp, ci, ci, ip, ip, ci, ci, dp]
        lib.oracle_perm_grad.argtypes = [dp, ci, ci, ip, ip, ci, ci, dp]
        lib.oracle_perm_batch.argtypes = [i64, dp, lp, ip, ip, ip, lp, ip, lp, ci, ci, dp]
        lib.oracle_bs_probs.argtypes = [dp, ci, ip, ip, i64, ci, ci, dp, dp]
        lib.oracle_bs_grad_U.argtypes = [dp, ci, ip, ip, i64, dp, ci, dp]
        lib.oracle_haf_bruteforce.argtypes = [dp, ci, dp]
        lib.oracle_haf_grouped.argtypes = [dp, ci, ip, dp]
        lib.oracle_lhaf_bruteforce.argtypes = [dp, ci, dp]
        lib.oracle_lhaf_grouped.argtypes = [dp, dp, ci, ip, dp]
        for f in ("oracle_perm_bruteforce", "oracle_perm_ryser", "oracle_perm_grad",
                  "oracle_perm_batch", "oracle_bs_probs", "oracle_bs_grad_U",
                  "oracle_haf_bruteforce", "oracle_haf_grouped", "oracle_lhaf_bruteforce",
                  "oracle_lhaf_grouped"):
            getattr(lib, f).restype = ci
        _lib = lib
        return lib


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _lptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _check(rc: int, what: str):
    if rc != ORC_OK:
        raise ValueError(f"{what}: oracle returned {rc}")


def perm_bruteforce(a) -> complex:
    """per(a) as the sum over all n! permutations of prod_i a[sigma(i), i]
    (Eq. (per_def)); n <= 12."""
    a = _c128(a)
    n = a.shape[0]
    assert a.shape == (n, n)
    out = np.zeros(3)
    _check(_load().oracle_perm_bruteforce(_dptr(a), n, _dptr(out)), "perm_bruteforce")
    return complex(out[0], out[1])


def perm_ryser(b, r=None, c=None, gold: bool = False, nthreads: int | None = None,
               info: bool = False):
    """Permanent of the matrix that repeats base row i r[i] times and base
    column j c[j] times (defaults: all ones), by Ryser's formula.

    Returns the complex permanent, or ``(per, sum_abs_terms, bound)`` if
    ``info`` is set, where ``bound`` is the a-posteriori error bound."""
    b = _c128(b)
    if b.ndim != 2:
        raise ValueError("b must be 2-D")
    k, l = b.shape
    r = _i32(np.ones(k) if r is None else r)
    c = _i32(np.ones(l) if c is None else c)
    out = np.zeros(4)
    nt = 1 if nthreads is None else int(nthreads)
    _check(_load().oracle_perm_ryser(_dptr(b), k, l, _iptr(r), _iptr(c), int(gold), nt,
                                     _dptr(out)), "perm_ryser")
    per = complex(out[0], out[1])
    if info:
        return per, float(out[2]), float(out[3])
    return per


def perm_batch(mats, mat_off, k, l, row_mult, row_off, col_mult, col_off,
               gold: bool = False, nthreads: int | None = None, info: bool = False):
    """Ragged batch of ``perm_ryser`` calls in the packed layout (offsets in
    complex elements for ``mats``, in entries for the multiplicities)."""
    mats = _c128(mats)
    mat_off, row_off, col_off = _i64(mat_off), _i64(row_off), _i64(col_off)
    k, l, row_mult, col_mult = _i32(k), _i32(l), _i32(row_mult), _i32(col_mult)
    batch = k.shape[0]
    out = np.zeros((batch, 4))
    nt = default_threads() if nthreads is None else int(nthreads)
    _check(_load().oracle_perm_batch(batch, _dptr(mats), _lptr(mat_off), _iptr(k), _iptr(l),
                                     _iptr(row_mult), _lptr(row_off), _iptr(col_mult),
                                     _lptr(col_off), int(gold), nt, _dptr(out)), "perm_batch")
    per = out[:, 0] + 1j * out[:, 1]
    if info:
        return per, out[:, 2], out[:, 3]
    return per


def perm_grad(b, r=None, c=None, gold: bool = False) -> np.ndarray:
    """d per / d b_ij = r_i c_j per(B; r - e_i, c - e_j), a k x l complex array."""
    b = _c128(b)
    k, l = b.shape
    r = _i32(np.ones(k) if r is None else r)
    c = _i32(np.ones(l) if c is None else c)
    g = np.zeros((k, l), dtype=np.complex128)
    _check(_load().oracle_perm_grad(_dptr(b), k, l, _iptr(r), _iptr(c), int(gold), 1,
                                    _dptr(g)), "perm_grad")
    return g


def bs_probs(U, s, t, gold: bool = False, nthreads: int | None = None):
    """Eq. (BS_prob) for input occupation ``s`` (length m) and each row of
    ``t`` (B x m output occupations); U is indexed U[out, in].
    Returns ``(probs, amps)`` with amps = per(U_{s,t})."""
    U = _c128(U)
    m = U.shape[0]
    s = _i32(s)
    t = _i32(np.atleast_2d(t))
    B = t.shape[0]
    probs = np.zeros(B)
    amps = np.zeros(B, dtype=np.complex128)
    nt = default_threads() if nthreads is None else int(nthreads)
    _check(_load().oracle_bs_probs(_dptr(U), m, _iptr(s), _iptr(t), B, int(gold), nt,
                                   _dptr(probs), _dptr(amps)), "bs_probs")
    return probs, amps


def haf_bruteforce(a) -> complex:
    """haf(a) as the sum over perfect matchings of prod a_ij, Eq. (haf_def);
    a symmetric, even size <= 16."""
    a = _c128(a)
    N = a.shape[0]
    out = np.zeros(3)
    _check(_load().oracle_haf_bruteforce(_dptr(a), N, _dptr(out)), "haf_bruteforce")
    return complex(out[0], out[1])


def haf_grouped(b, r=None, info: bool = False):
    """Hafnian of the matrix repeating base index i r[i] times, by the grouped
    sign-vector formula in double-double (every term from scratch)."""
    b = _c128(b)
    k = b.shape[0]
    r = _i32(np.ones(k) if r is None else r)
    out = np.zeros(3)
    _check(_load().oracle_haf_grouped(_dptr(b), k, _iptr(r), _dptr(out)), "haf_grouped")
    h = complex(out[0], out[1])
    return (h, float(out[2])) if info else h


def lhaf_bruteforce(a) -> complex:
    """lhaf(a) as the sum over matchings with loops (the diagonal entries are
    the loop weights), Eq. (loop_hafnian); a symmetric, size <= 14."""
    a = _c128(a)
    N = a.shape[0]
    out = np.zeros(3)
    _check(_load().oracle_lhaf_bruteforce(_dptr(a), N, _dptr(out)), "lhaf_bruteforce")
    return complex(out[0], out[1])


def lhaf_grouped(b, gamma, r=None, info: bool = False):
    """Loop hafnian of filldiag(b repeated by r, gamma repeated by r) by the
    grouped sign-vector formula in double-double."""
    b = _c128(b)
    k = b.shape[0]
    g = _c128(gamma)
    r = _i32(np.ones(k) if r is None else r)
    out = np.zeros(3)
    _check(_load().oracle_lhaf_grouped(_dptr(b), _dptr(g), k, _iptr(r), _dptr(out)),
           "lhaf_grouped")
    h = complex(out[0], out[1])
    return (h, float(out[2])) if info else h


def bs_grad_U(U, s, t, grad_probs, gold: bool = False) -> np.ndarray:
    """Gradient of sum_b grad_probs[b] * p_b with respect to U, in the
    convention dL/dRe U + i dL/dIm U (the one torch uses for complex tensors)."""
    U = _c128(U)
    m = U.shape[0]
    s = _i32(s)
    t = _i32(np.atleast_2d(t))
    g = np.ascontiguousarray(np.asarray(grad_probs, dtype=np.float64))
    out = np.zeros((m, m), dtype=np.complex128)
    _check(_load().oracle_bs_grad_U(_dptr(U), m, _iptr(s), _iptr(t), t.shape[0], _dptr(g),
                                    int(gold), _dptr(out)), "bs_grad_U")
    return out
