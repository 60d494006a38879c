"""Clifford and Clifford's "Algorithm A" boson sampler, written plainly on top
of the oracle's permanents (TEST INFRASTRUCTURE ONLY; see the package
docstring).  The paper samples boson-sampling outputs with this algorithm
(Sec. 4.2, "Boson Sampling").

For input occupation s (n photons), A holds the columns of U of the occupied
input modes (mode j repeated s_j times) in the order col_order[b] of sample b.
Photon k (k = 1 .. n) is placed in output mode i with probability
proportional to |per(A[{r_1 .. r_{k-1}, i}, 1 .. k])|^2.  The random numbers
are inputs: the column orders and one uniform per photon; a photon goes to
the first mode whose running weight sum (modes in order, plain sequential
double additions) exceeds u * total, or to the last mode with a positive
weight if rounding leaves none.
"""
from __future__ import annotations

import numpy as np


def algorithm_a(U, s, col_order, uniforms, gold: bool = True) -> np.ndarray:
    from . import bs_probs  # the oracle's per(U_{s,t}) via Ryser's formula

    U = np.asarray(U, dtype=np.complex128)
    m = U.shape[0]
    s = np.asarray(s, dtype=np.int64)
    cols = [j for j in range(m) for _ in range(int(s[j]))]
    n = len(cols)
    col_order = np.asarray(col_order)
    uniforms = np.asarray(uniforms, dtype=np.float64)
    nsamples = col_order.shape[0]
    out = np.zeros((nsamples, m), dtype=np.int32)
    for b in range(nsamples):
        occ = np.zeros(m, dtype=np.int32)
        for k in range(1, n + 1):
            sk = np.zeros(m, dtype=np.int32)  # input modes of the first k columns
            for q in range(k):
                sk[cols[int(col_order[b, q])]] += 1
            cand = np.repeat(occ[None, :], m, axis=0)
            cand[np.arange(m), np.arange(m)] += 1  # candidate i adds a photon to mode i
            _, amps = bs_probs(U, sk, cand, gold=gold, nthreads=1)
            w = [float(abs(a) ** 2) for a in amps]
            total = 0.0
            for x in w:
                total += x
            thr = float(uniforms[b, k - 1]) * total
            run, pick, last = 0.0, -1, -1
            for i, x in enumerate(w):
                if x > 0.0:
                    last = i
                run += x
                if pick < 0 and run > thr:
                    pick = i
            if pick < 0:
                pick = last
            occ[pick] += 1
        out[b] = occ
    return out
