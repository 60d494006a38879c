"""Clements beamsplitter mesh U(theta, phi) and its parameter gradient, written
plainly with full m x m matrix products (numpy ``@`` is the only library step).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Beamsplitter (Appendix A, "Beamsplitter gate"): on the pair of modes (j, j+1)
the ladder operators transform with the 2 x 2 block [[t, -conj(r)], [r, t]],
t = cos(theta), r = exp(i phi) sin(theta).

Mesh layout (a reading: the paper only says the interferometer decomposes
into two-mode beamsplitters, caption of Fig. BS_Setup): m layers; layer q
holds the beamsplitters on pairs (j, j+1) with j = q mod 2, q mod 2 + 2, ...,
j + 1 < m.  Beamsplitters are numbered in that order (layer-major, j
ascending), k = 0 .. L-1 with L = m(m-1)/2, and U = T_{L-1} ... T_1 T_0
(T_0 acts first).  U is indexed U[out, in].
"""
from __future__ import annotations

import numpy as np


def clements_layout(m: int) -> list[int]:
    """Lower mode j of every beamsplitter (j, j+1), in application order."""
    js = []
    for q in range(m):
        j = q % 2
        while j + 1 < m:
            js.append(j)
            j += 2
    return js


def beamsplitter_block(theta: float, phi: float) -> np.ndarray:
    t = np.cos(theta)
    r = np.exp(1j * phi) * np.sin(theta)
    return np.array([[t, -np.conj(r)], [r, t]], dtype=np.complex128)


def _dblock_dtheta(theta: float, phi: float) -> np.ndarray:
    # d/dtheta of [[cos, -e^{-i phi} sin], [e^{i phi} sin, cos]]
    return np.array([[-np.sin(theta), -np.exp(-1j * phi) * np.cos(theta)],
                     [np.exp(1j * phi) * np.cos(theta), -np.sin(theta)]], dtype=np.complex128)


def _dblock_dphi(theta: float, phi: float) -> np.ndarray:
    # d/dphi of the same block
    return np.array([[0.0, 1j * np.exp(-1j * phi) * np.sin(theta)],
                     [1j * np.exp(1j * phi) * np.sin(theta), 0.0]], dtype=np.complex128)


def _embed(block: np.ndarray, j: int, m: int, identity: bool) -> np.ndarray:
    T = np.eye(m, dtype=np.complex128) if identity else np.zeros((m, m), dtype=np.complex128)
    T[j:j + 2, j:j + 2] = block
    return T


def clements_unitary(theta, phi, m: int) -> np.ndarray:
    """U = T_{L-1} ... T_0 with T_k the identity carrying beamsplitter k."""
    js = clements_layout(m)
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    assert theta.shape == (len(js),) and phi.shape == (len(js),)
    U = np.eye(m, dtype=np.complex128)
    for k, j in enumerate(js):
        U = _embed(beamsplitter_block(theta[k], phi[k]), j, m, True) @ U
    return U


def clements_grad(theta, phi, m: int, G) -> tuple[np.ndarray, np.ndarray]:
    """dL/dtheta_k and dL/dphi_k for a real loss L whose gradient with respect
    to U is G = dL/dRe U + i dL/dIm U.  Since dL = Re sum conj(G) dU,
    dL/dtheta_k = Re sum conj(G) * (T_{L-1}..T_{k+1}) dT_k/dtheta (T_{k-1}..T_0),
    evaluated here with explicit prefix and suffix products."""
    js = clements_layout(m)
    L = len(js)
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    G = np.asarray(G, dtype=np.complex128)
    Ts = [_embed(beamsplitter_block(theta[k], phi[k]), j, m, True) for k, j in enumerate(js)]
    before = [np.eye(m, dtype=np.complex128)]  # before[k] = T_{k-1} ... T_0
    for k in range(L):
        before.append(Ts[k] @ before[k])
    after = [np.eye(m, dtype=np.complex128) for _ in range(L + 1)]  # after[k] = T_{L-1}..T_{k+1}
    for k in range(L - 2, -1, -1):
        after[k] = after[k + 1] @ Ts[k + 1]
    gt = np.zeros(L)
    gp = np.zeros(L)
    for k, j in enumerate(js):
        dUt = after[k] @ _embed(_dblock_dtheta(theta[k], phi[k]), j, m, False) @ before[k]
        dUp = after[k] @ _embed(_dblock_dphi(theta[k], phi[k]), j, m, False) @ before[k]
        gt[k] = np.real(np.sum(np.conj(G) * dUt))
        gp[k] = np.real(np.sum(np.conj(G) * dUp))
    return gt, gp
