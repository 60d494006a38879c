"""Seeded synthetic inputs for the permanent path.

This module holds input generation only (random unitaries, occupation
patterns, ragged batches, mesh angles) and none of the permanent, probability
or mesh arithmetic, so that the CUDA path and the CPU oracle can both be fed
from it without sharing any of the method's code.

Workloads (all seeded; config c uses base seed 1000 + c):

1. ``bs_small``       m = 8 Haar unitary, input |1,1,1,1,0,0,0,0>, all C(11,4) = 330
                      output patterns with 4 photons, lexicographic order.
2. ``single_large``   top-left 30 x 30 block of a Haar 60 x 60 unitary, no repetitions.
3. ``bs_batched``     m = 24 Haar, 12 photons in modes 0..11, 4096 output patterns:
                      2048 collision-free, 2048 with occupations up to 3.
4. ``ragged``         65536 permanents, n ~ U{4..20}, row/column multiplicities with
                      parts from {1, 2, 3}, each a submatrix of its own Haar 2n x 2n.
5. ``gradient``       m = 16 Clements mesh angles theta, phi ~ U[0, 2 pi) (120 each),
                      8 photons in modes 0..7, 1024 distinct output patterns.

The Haar measure follows Mezzadri's recipe: QR of a complex Ginibre matrix
with the phases of R's diagonal moved into Q.  The paper measures on no public
dataset; these generators stand in for its "Haar-random interferometer"
workloads (Sec. 4.2 benchmarks use random inputs as well).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 1000


def rng_for(config: int, stream: int = 0) -> np.random.Generator:
    """Generator for sub-stream ``stream`` of workload ``config``."""
    return np.random.Generator(np.random.PCG64((BASE_SEED + config) * (1 << 20) + stream))


def haar_unitary(m: int, rng: np.random.Generator) -> np.ndarray:
    z = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return np.ascontiguousarray(q * (d / np.abs(d))[None, :])


def haar_unitaries(count: int, m: int, rng: np.random.Generator) -> np.ndarray:
    """``count`` independent m x m Haar unitaries (batched QR)."""
    z = (rng.standard_normal((count, m, m)) + 1j * rng.standard_normal((count, m, m))) \
        / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    return np.ascontiguousarray(q * (d / np.abs(d))[:, None, :])


def compositions(n: int, m: int) -> np.ndarray:
    """All occupation patterns t in N^m with sum n, in lexicographic order
    (first mode most significant, ascending)."""
    out = []

    def rec(prefix, left, slots):
        if slots == 1:
            out.append(prefix + [left])
            return
        for v in range(0, left + 1):
            rec(prefix + [v], left - v, slots - 1)

    rec([], n, m)
    return np.asarray(out, dtype=np.int32)


# --------------------------------------------------------------------------
# packed ragged batch of base matrices
# --------------------------------------------------------------------------
@dataclass
class PermBatch:
    """Ragged batch in the packed layout of the C ABI.

    mats      complex128, all base matrices row-major, concatenated
    mat_off   int64[batch], offset of item b in ``mats`` (complex elements)
    k, l      int32[batch], base rows / columns of item b
    row_mult  int32, concatenated row multiplicities; row_off int64[batch]
    col_mult  int32, concatenated column multiplicities; col_off int64[batch]
    """
    mats: np.ndarray
    mat_off: np.ndarray
    k: np.ndarray
    l: np.ndarray
    row_mult: np.ndarray
    row_off: np.ndarray
    col_mult: np.ndarray
    col_off: np.ndarray

    @property
    def batch(self) -> int:
        return int(self.k.shape[0])

    def item(self, b: int):
        """(base matrix, r, c) of item b."""
        k, l = int(self.k[b]), int(self.l[b])
        o = int(self.mat_off[b])
        B = self.mats[o:o + k * l].reshape(k, l)
        r = self.row_mult[int(self.row_off[b]):int(self.row_off[b]) + k]
        c = self.col_mult[int(self.col_off[b]):int(self.col_off[b]) + l]
        return B, r, c

    def subset(self, idx) -> "PermBatch":
        return pack_batch([self.item(int(b)) for b in idx])


def pack_batch(items) -> PermBatch:
    """Pack a list of (B, r, c) into the ragged layout."""
    mats, mo, ks, ls, rm, ro, cm, co = [], [], [], [], [], [], [], []
    off = roff = coff = 0
    for B, r, c in items:
        B = np.asarray(B, dtype=np.complex128)
        k, l = B.shape
        mats.append(B.reshape(-1))
        mo.append(off)
        ks.append(k)
        ls.append(l)
        rm.append(np.asarray(r, dtype=np.int32).reshape(-1))
        ro.append(roff)
        cm.append(np.asarray(c, dtype=np.int32).reshape(-1))
        co.append(coff)
        off += k * l
        roff += k
        coff += l
    cat = (lambda xs, dt: np.ascontiguousarray(np.concatenate(xs)).astype(dt)
           if xs else np.zeros(0, dtype=dt))
    return PermBatch(cat(mats, np.complex128), np.asarray(mo, dtype=np.int64),
                     np.asarray(ks, dtype=np.int32), np.asarray(ls, dtype=np.int32),
                     cat(rm, np.int32), np.asarray(ro, dtype=np.int64),
                     cat(cm, np.int32), np.asarray(co, dtype=np.int64))


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def bs_small():
    """(U 8x8, s, t[330, 8])."""
    U = haar_unitary(8, rng_for(1))
    s = np.array([1, 1, 1, 1, 0, 0, 0, 0], dtype=np.int32)
    t = compositions(4, 8)
    return U, s, t


def single_large(n: int = 30):
    """Top-left n x n block of a Haar 2n x 2n unitary (2n = 60 for n = 30)."""
    U = haar_unitary(2 * n, rng_for(2))
    return np.ascontiguousarray(U[:n, :n])


def _pattern_collision_free(m: int, n: int, rng) -> np.ndarray:
    t = np.zeros(m, dtype=np.int32)
    t[rng.choice(m, size=n, replace=False)] = 1
    return t


def _pattern_with_collisions(m: int, n: int, cap: int, rng) -> np.ndarray:
    while True:
        t = np.zeros(m, dtype=np.int32)
        placed = 0
        while placed < n:
            mode = int(rng.integers(0, m))
            if t[mode] < cap:
                t[mode] += 1
                placed += 1
        if t.max() > 1:
            return t


def bs_batched(m: int = 24, n: int = 12, count: int = 4096, cap: int = 3):
    """(U m x m, s, t[count, m]): first half collision-free, second half with
    photons dropped one by one into modes of capacity ``cap`` (redrawn when the
    result happens to be collision-free)."""
    U = haar_unitary(m, rng_for(3))
    s = np.zeros(m, dtype=np.int32)
    s[:n] = 1
    rng = rng_for(3, 1)
    half = count // 2
    t = np.zeros((count, m), dtype=np.int32)
    for b in range(half):
        t[b] = _pattern_collision_free(m, n, rng)
    for b in range(half, count):
        t[b] = _pattern_with_collisions(m, n, cap, rng)
    return U, s, t


def _parts(n: int, rng) -> list[int]:
    """Multiplicities with parts drawn uniformly from {1,2,3}, the last one
    clipped so that they sum to n."""
    out, left = [], n
    while left > 0:
        p = min(int(rng.integers(1, 4)), left)
        out.append(p)
        left -= p
    return out


def ragged(count: int = 65536, nmin: int = 4, nmax: int = 20, block: int = 0,
           sizes_only: bool = False) -> PermBatch:
    """Ragged batch: n ~ U{nmin..nmax}; row and column multiplicities drawn
    independently as ``_parts``; distinct row modes and distinct column modes
    drawn from 0..2n-1 of the item's own Haar 2n x 2n unitary.

    ``block`` b > 0 draws another batch of the same recipe from seed streams
    of its own (sizes from stream 1000 b, unitaries of size 2n from stream
    1000 b + n): block r is rank r's part of a batch of several blocks split
    over ranks.  Block 0 is the benchmark batch.  ``sizes_only`` skips the
    unitaries (all base matrices zero): the sizes and multiplicities alone."""
    rng = rng_for(4) if block == 0 else rng_for(4, 1000 * block)
    ns = rng.integers(nmin, nmax + 1, size=count)
    rows_l, cols_l, rs, cs = [], [], [], []
    for b in range(count):
        n = int(ns[b])
        r = _parts(n, rng)
        c = _parts(n, rng)
        rows_l.append(rng.choice(2 * n, size=len(r), replace=False))
        cols_l.append(rng.choice(2 * n, size=len(c), replace=False))
        rs.append(r)
        cs.append(c)
    items = [None] * count
    if sizes_only:
        return pack_batch([(np.zeros((len(rs[b]), len(cs[b])), dtype=np.complex128), rs[b], cs[b])
                           for b in range(count)])
    for n in range(nmin, nmax + 1):
        idx = np.nonzero(ns == n)[0]
        if idx.size == 0:
            continue
        Us = haar_unitaries(idx.size, 2 * n, rng_for(4, n if block == 0 else 1000 * block + n))
        for q, b in enumerate(idx):
            B = Us[q][np.ix_(rows_l[b], cols_l[b])]
            items[b] = (B, rs[b], cs[b])
    return pack_batch(items)


def _unrank_combination(rank: int, n: int, k: int) -> list[int]:
    """k-subset of {0..n-1} with the given rank in lexicographic order."""
    out, x = [], 0
    for i in range(k):
        while True:
            cnt = math.comb(n - x - 1, k - i - 1)
            if rank < cnt:
                out.append(x)
                x += 1
                break
            rank -= cnt
            x += 1
    return out


def gradient_workload(m: int = 16, n: int = 8, count: int = 1024):
    """(theta[L], phi[L], s, t[count, m]) with L = m(m-1)/2.  Output patterns
    are drawn without replacement by rank among the C(n+m-1, n) occupation
    patterns (stars and bars: a pattern is an n-subset of n+m-1 slots)."""
    L = m * (m - 1) // 2
    rng = rng_for(5)
    theta = rng.uniform(0.0, 2.0 * math.pi, size=L)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=L)
    s = np.zeros(m, dtype=np.int32)
    s[:n] = 1
    total = math.comb(n + m - 1, n)
    ranks = rng_for(5, 1).choice(total, size=count, replace=False)
    t = np.zeros((count, m), dtype=np.int32)
    for b, rk in enumerate(ranks):
        bars = _unrank_combination(int(rk), n + m - 1, m - 1)  # positions of the m-1 bars
        prev = -1
        for mode, pos in enumerate(bars):
            t[b, mode] = pos - prev - 1
            prev = pos
        t[b, m - 1] = n + m - 1 - prev - 1
    return theta, phi, s, t


def paper_repeated(k: int, seed_stream: int = 0):
    """Workload of the paper's repeated-permanent benchmark (Sec. 4.2, Fig.
    permanent): a k x k block of a Haar 2k x 2k unitary with every row and
    column repeated twice.  Returns (B, r, c)."""
    U = haar_unitary(2 * k, rng_for(6, 100 * k + seed_stream))
    B = np.ascontiguousarray(U[:k, :k])
    return B, np.full(k, 2, dtype=np.int32), np.full(k, 2, dtype=np.int32)


def sampler_draws(nsamples: int, n: int, seed: int):
    """Random inputs of a boson sampler run: for every sample a uniformly
    random order of its n photon columns and one uniform in [0, 1) per photon."""
    rng = np.random.Generator(np.random.PCG64(seed))
    order = np.stack([rng.permutation(n) for _ in range(nsamples)]).astype(np.int32) \
        if nsamples else np.zeros((0, n), dtype=np.int32)
    uniforms = rng.random((nsamples, n))
    return np.ascontiguousarray(order.reshape(nsamples, n)), np.ascontiguousarray(uniforms)


def gbs_matrix(k: int, rng: np.random.Generator, squeezing: float = math.asinh(1.0)):
    """Symmetric k x k matrix U diag(tanh r) U^T of a Haar interferometer U
    after k equal single-mode squeezers (the Gaussian boson-sampling setting
    of Sec. 4.1 / Fig. gaussian_boson_sampling_benchmark, r = arcsinh 1)."""
    U = haar_unitary(k, rng)
    A = (U * math.tanh(squeezing)) @ U.T
    return np.ascontiguousarray((A + A.T) / 2)  # exactly symmetric


def paper_repeated_hafnian(k: int, loop: bool = False, seed_stream: int = 0):
    """Workload of the paper's repeated (loop) hafnian benchmarks (Figs.
    hafnian and loop_hafnian): a k x k symmetric GBS matrix with every index
    repeated twice (N = 2k); for the loop hafnian also loop weights gamma with
    entries ~ CN(0, 1/2).  Returns (B, r, gamma or None)."""
    rng = rng_for(8, 100 * k + seed_stream + (50 if loop else 0))
    B = gbs_matrix(k, rng)
    gamma = None
    if loop:
        gamma = (rng.standard_normal(k) + 1j * rng.standard_normal(k)) * 0.5
    return B, np.full(k, 2, dtype=np.int32), gamma


def hafnian_batch(count: int, kmin: int = 1, kmax: int = 8, rmax: int = 3, seed_stream: int = 0):
    """Ragged batch of repeated-hafnian items: k ~ U{kmin..kmax}, repetitions
    ~ U{0..rmax} per index, GBS base matrices, loop weights ~ CN(0, 1/2).
    Returns packed (mats, mat_off, k, rep, rep_off, gamma)."""
    rng = rng_for(9, seed_stream)
    mats, gam, reps = [], [], []
    ks = rng.integers(kmin, kmax + 1, size=count)
    mat_off = np.zeros(count, dtype=np.int64)
    rep_off = np.zeros(count, dtype=np.int64)
    mo = ro = 0
    for b, k in enumerate(ks):
        k = int(k)
        mats.append(gbs_matrix(k, rng).reshape(-1))
        reps.append(rng.integers(0, rmax + 1, size=k).astype(np.int32))
        gam.append((rng.standard_normal(k) + 1j * rng.standard_normal(k)) * 0.5)
        mat_off[b], rep_off[b] = mo, ro
        mo += k * k
        ro += k
    cat = (lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dtype=dt))
    return (cat(mats, np.complex128), mat_off, ks.astype(np.int32), cat(reps, np.int32), rep_off,
            cat(gam, np.complex128))
