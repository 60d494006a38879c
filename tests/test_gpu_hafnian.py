"""GPU hafnians and loop hafnians with repeated indices (pq_hafnian_repeated,
pq_loop_hafnian_repeated; Sec. 4.1, Eqs. (haf_def), (loop_hafnian)) against the
oracle on the same seeded inputs.

Tolerance: every term of the sign-vector sum is formed in FP64 from q and l,
which the Gray walk updates incrementally over at most 1024 steps per chunk,
and raised to a power <= 24, so a term carries a relative error of a few 1e-13
at most; the sum is double-double.  The GPU error is therefore bounded by a
few 1e-13 times sum |terms| (the oracle's normalised sum of term magnitudes,
the scale of the cancellation).  Wherever that bound is below the tolerance
-- a cancellation ratio sum |terms| / |value| of at most 1e4, which holds for
every item of the ragged batches and the (2, ..., 2) shapes here (the largest
ratio is about 600) -- the check is relative: |gpu - oracle| <= 1e-10 |oracle|.
Exact zeros (odd N) must come out exactly zero.  The block-diagonal N = 32
case, whose full sum the oracle cannot evaluate and whose ratio is about 2e4,
is checked relative to the product of its blocks' hafnians (each block's
ratio is below 1e3, so that product is accurate to about 1e-12); the lanes'
sums are exact integer sums, and the GPU's error there measured 3e-13 to
4e-13 relative.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2403_04006_gb300 import api, pq  # noqa: E402
from paper_2403_04006_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pq.load_library()
    return torch.device("cuda:0")


def run(dev, mats, mat_off, k, rep, rep_off, gamma=None):
    m = torch.from_numpy(np.ascontiguousarray(mats, dtype=np.complex128)).to(dev)
    g = None if gamma is None else torch.from_numpy(
        np.ascontiguousarray(gamma, dtype=np.complex128)).to(dev)
    return api.hafnian_repeated(m, mat_off, k, rep, rep_off, gamma=g).cpu().numpy()


def pack(items):
    """items: list of (B, r[, gamma]) -> packed arrays."""
    mats, reps, gams, mo, ro, ks = [], [], [], [], [], []
    a = b = 0
    for it in items:
        B, r = np.asarray(it[0], dtype=np.complex128), np.asarray(it[1], dtype=np.int32)
        g = it[2] if len(it) > 2 and it[2] is not None else np.zeros(len(r))
        k = B.shape[0]
        mats.append(B.reshape(-1))
        reps.append(r)
        gams.append(np.asarray(g, dtype=np.complex128))
        mo.append(a)
        ro.append(b)
        ks.append(k)
        a += k * k
        b += k
    cat = (lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dtype=dt))
    return (cat(mats, np.complex128), np.array(mo, dtype=np.int64), np.array(ks, dtype=np.int32),
            cat(reps, np.int32), np.array(ro, dtype=np.int64), cat(gams, np.complex128))


KAPPA_MAX = 1e4  # cancellation ratio up to which the relative check applies


def check(got, ref, scale, tol=TOL):
    """Relative check where the cancellation allows it (see the module
    docstring); returns True if it was the relative one."""
    if ref == 0:
        assert got == 0, (got, scale)
        return True
    if scale <= KAPPA_MAX * abs(ref):
        assert abs(got - ref) <= tol * abs(ref), (got, ref, scale)
        return True
    assert abs(got - ref) <= tol * scale, (got, ref, scale)
    return False


@pytest.mark.parametrize("loop", [False, True])
def test_ragged_batch_matches_oracle(dev, loop):
    mats, mo, k, rep, ro, gam = W.hafnian_batch(300, kmin=1, kmax=6, rmax=3,
                                                seed_stream=int(loop))
    got = run(dev, mats, mo, k, rep, ro, gam if loop else None)
    for b in range(len(k)):
        kb = int(k[b])
        B = mats[mo[b]:mo[b] + kb * kb].reshape(kb, kb)
        r = rep[ro[b]:ro[b] + kb]
        if loop:
            ref, scale = O.lhaf_grouped(B, gam[ro[b]:ro[b] + kb], r, info=True)
        else:
            ref, scale = O.haf_grouped(B, r, info=True)
        assert check(got[b], ref, scale)


@pytest.mark.parametrize("loop", [False, True])
def test_paper_repetitions_two(dev, loop):
    """(2, ..., 2) repetitions as in Figs. hafnian / loop_hafnian, k = 1 .. 9."""
    items = [W.paper_repeated_hafnian(k, loop=loop) for k in range(1, 10)]
    got = run(dev, *pack(items)[:5], gamma=pack(items)[5] if loop else None)
    for b, (B, r, g) in enumerate(items):
        ref, scale = (O.lhaf_grouped(B, g, r, info=True) if loop
                      else O.haf_grouped(B, r, info=True))
        assert check(got[b], ref, scale)  # relative 1e-10 for every k


@pytest.mark.parametrize("loop", [False, True])
def test_block_diagonal_factorises_at_large_size(dev, loop):
    """haf / lhaf of a block-diagonal base is the product of the blocks'; at
    k = 16 (N = 32, 2 * 3^15 terms) only the GPU evaluates the whole sum."""
    B1, r1, g1 = W.paper_repeated_hafnian(8, loop=True, seed_stream=1)
    B2, r2, g2 = W.paper_repeated_hafnian(8, loop=True, seed_stream=2)
    B = np.zeros((16, 16), dtype=np.complex128)
    B[:8, :8], B[8:, 8:] = B1, B2
    r = np.concatenate([r1, r2])
    g = np.concatenate([g1, g2])
    got = run(dev, *pack([(B, r, g)])[:5], gamma=g if loop else None)[0]
    if loop:
        (h1, s1), (h2, s2) = O.lhaf_grouped(B1, g1, r1, info=True), O.lhaf_grouped(B2, g2, r2, info=True)
    else:
        (h1, s1), (h2, s2) = O.haf_grouped(B1, r1, info=True), O.haf_grouped(B2, r2, info=True)
    ref = h1 * h2
    # The reference is a product of two k = 8 sums whose own cancellation is
    # mild (term scale over value below 1e3 each), so it holds to about
    # 1e-12 relative; the GPU's whole N = 32 sum cancels far more (term scale
    # about 2e4 |ref|) and is held to the relative tolerance of the other
    # parity tests (measured on a GB300: 3e-13 and 4e-13).
    assert s1 < 1e3 * abs(h1) and s2 < 1e3 * abs(h2), (s1 / abs(h1), s2 / abs(h2))
    assert abs(got - ref) <= TOL * abs(ref), (got, ref, abs(got - ref) / abs(ref))


def test_edge_cases(dev):
    a = 0.3 - 0.8j
    items = [
        (np.array([[a]]), [3]),                # odd N -> 0
        (np.array([[a]]), [0]),                # N = 0 -> 1
        (np.zeros((0, 0)), np.zeros(0)),       # empty base -> 1
        (np.array([[a]]), [6]),                # 5!! a^3
        (np.array([[a]]), [1, ]),              # odd
        (np.ones((6, 6)), np.ones(6)),         # all ones: 5!! matchings
        (np.array([[0, a], [a, 0]]), [1, 1]),  # one pair
        (np.array([[2.0, a], [a, 5.0]]), [0, 2]),  # second index twice: B_11 = 5
    ]
    got = run(dev, *pack(items)[:5])
    want = [0, 1, 1, 15 * a ** 3, 0, 15, a, 5.0]
    for g, w in zip(got, want):
        assert abs(g - w) <= 1e-13 * max(1, abs(w)), (g, w)
    assert got[0] == 0 and got[4] == 0


def test_loop_edge_cases(dev):
    b, c = 0.7 - 0.2j, -0.4 + 0.9j
    items = [(np.array([[b]]), [N], [c]) for N in (0, 1, 2, 5, 9)]
    items.append((np.ones((5, 5)), np.ones(5), np.ones(5)))  # 26 involutions
    got = run(dev, *pack(items)[:5], gamma=pack(items)[5])
    for gv, (_, r, _) in zip(got[:5], items[:5]):
        N = int(r[0])
        want = sum(math.comb(N, 2 * j) * math.prod(range(2 * j - 1, 0, -2)) * b ** j
                   * c ** (N - 2 * j) for j in range(N // 2 + 1))
        assert abs(gv - want) <= 1e-13 * max(1, abs(want)), (N, gv, want)
    assert abs(got[5] - 26) <= 1e-12


def test_loop_with_zero_weights_equals_hafnian(dev):
    mats, mo, k, rep, ro, gam = W.hafnian_batch(64, kmin=2, kmax=6, rmax=2, seed_stream=3)
    h = run(dev, mats, mo, k, rep, ro)
    lh = run(dev, mats, mo, k, rep, ro, np.zeros_like(gam))
    N = np.array([rep[ro[b]:ro[b] + k[b]].sum() for b in range(len(k))])
    assert (lh[N % 2 == 1] == 0).all()
    for b in range(len(k)):
        assert abs(lh[b] - h[b]) <= 1e-12 * max(1, abs(h[b]))


def test_deterministic(dev):
    items = [W.paper_repeated_hafnian(k, loop=True) for k in (9, 11, 12)]
    p = pack(items)
    a1 = run(dev, *p[:5], gamma=p[5])
    a2 = run(dev, *p[:5], gamma=p[5])
    assert (a1 == a2).all()
    h1 = run(dev, *p[:5])
    h2 = run(dev, *p[:5])
    assert (h1 == h2).all()


def test_errors(dev):
    B = torch.eye(2, dtype=torch.complex128, device=dev)
    with pytest.raises(pq.PQError) as e:
        api.hafnian_repeated(B, [0], [2], [1, -1], [0])
    assert e.value.code == pq.PQ_ERR_ARG
    with pytest.raises(pq.PQError) as e:
        api.hafnian_repeated(B, [0], [2], [25, 25], [0])
    assert e.value.code == pq.PQ_ERR_UNSUPPORTED
    out = torch.empty(1, dtype=torch.complex128, device=dev)
    with pytest.raises(pq.PQError) as e:
        pq.pq_hafnian_repeated(B.data_ptr(), [0], [2], [1, 1], [0], out.data_ptr(), None,
                               gamma_ptr=None, loop=True)
    assert e.value.code == pq.PQ_ERR_ARG
    assert api.hafnian_repeated(B, [], [], [], []).numel() == 0


@pytest.mark.parametrize("loop", [False, True])
def test_plan_runs_match_the_one_shot_call(dev, loop):
    """A hafnian plan evaluates the same values as the one-shot call, run
    after run, for new matrix values each time."""
    mats, mo, k, rep, ro, gam = W.hafnian_batch(120, kmin=1, kmax=7, rmax=3, seed_stream=11)
    plan = api.HafnianPlan(mo, k, rep, ro, loop=loop)
    rng = np.random.default_rng(12)
    for _ in range(3):
        m = (rng.standard_normal(mats.shape) + 1j * rng.standard_normal(mats.shape)) * 0.4
        g = (rng.standard_normal(gam.shape) + 1j * rng.standard_normal(gam.shape)) * 0.5
        for b in range(len(k)):  # keep every base symmetric
            kb = int(k[b])
            blk = m[mo[b]:mo[b] + kb * kb].reshape(kb, kb)
            m[mo[b]:mo[b] + kb * kb] = ((blk + blk.T) / 2).reshape(-1)
        md = torch.from_numpy(m).to(dev)
        gd = torch.from_numpy(g).to(dev) if loop else None
        got = plan.run(md, gamma=gd).cpu().numpy()
        want = run(dev, m, mo, k, rep, ro, g if loop else None)
        assert np.array_equal(got, want)  # same schedule, same order of operations
    plan.close()


def test_plan_errors(dev):
    plan = api.HafnianPlan([0], [2], [1, 1], [0], loop=True)
    B = torch.eye(2, dtype=torch.complex128, device=dev)
    with pytest.raises(pq.PQError) as e:
        plan.run(B)  # a loop plan needs loop weights
    assert e.value.code == pq.PQ_ERR_ARG
    with pytest.raises(pq.PQError) as e:
        api.HafnianPlan([0], [2], [1, -1], [0])
    assert e.value.code == pq.PQ_ERR_ARG
    empty = api.HafnianPlan([], [], [], [])
    assert empty.run(B).numel() == 0
