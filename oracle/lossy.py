"""Lossy boson sampling, written plainly (TEST INFRASTRUCTURE ONLY; see the
package docstring).

Paper Sec. 3.2.4 (Figs. BS_Setup, BS_LossModel): a lossy interferometer is
A = V diag(sqrt(eta)) W; a photon in mode i survives with probability eta_i,
modelled as a beamsplitter sending it to an inaccessible mode.  The m system
modes plus m loss modes form a unitary whose input-mode columns are
[V diag(sqrt(eta)) W ; diag(sqrt(1 - eta)) W]; the probability of seeing t on
the system modes is Eq. (BS_prob) on that 2m-mode unitary summed over every
occupation u of the loss modes with |u| = n - |t|.
"""
from __future__ import annotations

import numpy as np


def _compositions(k: int, m: int):
    if m == 1:
        yield [k]
        return
    for v in range(k + 1):
        for rest in _compositions(k - v, m - 1):
            yield [v] + rest


def dilation(V, eta, W) -> np.ndarray:
    V = np.asarray(V, dtype=np.complex128)
    W = np.asarray(W, dtype=np.complex128)
    eta = np.asarray(eta, dtype=np.float64)
    m = V.shape[0]
    U = np.zeros((2 * m, 2 * m), dtype=np.complex128)
    U[:m, :m] = V @ np.diag(np.sqrt(eta)) @ W
    U[m:, :m] = np.diag(np.sqrt(1.0 - eta)) @ W
    # columns m..2m-1 (photons entering loss modes) never occur; any
    # completion to a unitary leaves these probabilities unchanged
    return U


def lossy_probs(V, eta, W, s, t, gold: bool = True) -> np.ndarray:
    from . import bs_probs

    U = dilation(V, eta, W)
    m = U.shape[0] // 2
    s = np.asarray(s, dtype=np.int32)
    n = int(s.sum())
    sbig = np.concatenate([s, np.zeros(m, dtype=np.int32)])
    t = np.atleast_2d(np.asarray(t, dtype=np.int32))
    out = np.zeros(t.shape[0])
    for b, tb in enumerate(t):
        pats = np.array([np.concatenate([tb, u]) for u in _compositions(n - int(tb.sum()), m)],
                        dtype=np.int32)
        p, _ = bs_probs(U, sbig, pats, gold=gold, nthreads=1)
        total = 0.0
        for x in p:  # in pattern order
            total += float(x)
        out[b] = total
    return out
