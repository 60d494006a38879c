"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle
on identical seeded inputs.

Tolerances (stated requirement of the path): relative error <= 1e-10 for
n <= 20, <= 1e-8 at n = 30, gradients within 1e-7 (max-norm, relative to the
reference's max-norm).  Expected values come from the oracle's gold mode
(double-double throughout), whose own error bound is checked to be far below
these tolerances; exact zeros (Hong-Ou-Mandel) are compared absolutely.
"""
import ctypes
import math
import os
import sys
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2403_04006_gb300 import api, pq  # noqa: E402
from paper_2403_04006_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
from make_golden import read_matrix_file  # noqa: E402

TOL = 1e-10
TOL30 = 1e-8
TOLG = 1e-7


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pq.load_library()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def ragged_pb():
    """Workload 4 (65536 permanents), generated once for the module."""
    return W.ragged()


def rel_err(x, ref):
    x = np.asarray(x)
    ref = np.asarray(ref)
    return np.abs(x - ref) / np.abs(ref)


def random_parts(n, rng, maxpart=3):
    out, left = [], n
    while left:
        p = min(int(rng.integers(1, maxpart + 1)), left)
        out.append(p)
        left -= p
    return out


def random_items(count, nmin, nmax, rng, maxpart=3):
    items = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        r = random_parts(n, rng, maxpart)
        c = random_parts(n, rng, maxpart)
        B = (rng.standard_normal((len(r), len(c))) + 1j * rng.standard_normal((len(r), len(c))))
        B /= math.sqrt(2 * n)
        items.append((B, r, c))
    return items


def oracle_items(items):
    return np.array([O.perm_ryser(B, r, c, gold=True) for B, r, c in items])


def gpu_perms(pb, dev, method="batched", use_graph=False, chunk_log2=0):
    db = api.DeviceBatch(pb, dev)
    plan = api.Plan.for_batch(pb, method=method, use_graph=use_graph, chunk_log2=chunk_log2)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out = api.permanent_batched(db, plan)
    s.synchronize()
    return out.cpu().numpy(), plan


# ------------------------------------------------------------------ forward
def test_random_batch_with_multiplicities(dev):
    rng = np.random.default_rng(101)
    items = random_items(300, 1, 14, rng)
    pb = W.pack_batch(items)
    ref = oracle_items(items)
    got_b, _ = gpu_perms(pb, dev, "batched")
    got_p, _ = gpu_perms(pb, dev, "plain")
    assert rel_err(got_b, ref).max() <= TOL
    # the plain method cuts every permanent finer (one launch must fill the GPU)
    assert rel_err(got_p, ref).max() <= TOL


@pytest.mark.parametrize("chunk_log2", [1, 3, 6, 12])
def test_chunking_does_not_change_results(dev, chunk_log2):
    rng = np.random.default_rng(202)
    items = random_items(64, 6, 16, rng)
    pb = W.pack_batch(items)
    ref = oracle_items(items)
    got, _ = gpu_perms(pb, dev, chunk_log2=chunk_log2)
    assert rel_err(got, ref).max() <= TOL


def test_edge_cases(dev):
    rng = np.random.default_rng(303)
    items, want = [], []
    # n = 0: empty base and all-zero multiplicities -> per = 1
    items.append((np.zeros((0, 0)), [], []))
    want.append(1.0)
    items.append((rng.standard_normal((2, 3)) + 0j, [0, 0], [0, 0, 0]))
    want.append(1.0)
    # n = 1
    items.append((np.array([[0.3 - 0.7j]]), [1], [1]))
    want.append(0.3 - 0.7j)
    # 1 x 1 base repeated: per = n! a^n
    a = 0.8 + 0.35j
    for n in (2, 3, 5, 9, 12):
        items.append((np.array([[a]]), [n], [n]))
        want.append(math.factorial(n) * a ** n)
    # all ones and ones minus identity (derangements)
    for n in (4, 9, 13):
        items.append((np.ones((n, n)) + 0j, [1] * n, [1] * n))
        want.append(float(math.factorial(n)))
    d = [1, 0]
    for i in range(2, 14):
        d.append((i - 1) * (d[-1] + d[-2]))
    for n in (5, 10, 13):
        items.append((np.ones((n, n)) - np.eye(n) + 0j, [1] * n, [1] * n))
        want.append(float(d[n]))
    # zero-multiplicity rows/columns among live ones
    B = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    items.append((B, [2, 0, 1, 0], [0, 1, 0, 2]))
    want.append(O.perm_ryser(B[[0, 2]][:, [1, 3]], [2, 1], [1, 2], gold=True))
    # widest product side: 2 rows repeated 20 times against 40 single columns
    B = (rng.standard_normal((2, 40)) + 1j * rng.standard_normal((2, 40))) / 4
    items.append((B, [20, 20], [1] * 40))
    want.append(O.perm_ryser(B, [20, 20], [1] * 40, gold=True))
    # one row, one column, tall and wide bases
    B = rng.standard_normal((1, 5)) + 1j * rng.standard_normal((1, 5))
    items.append((B, [5], [1] * 5))
    want.append(O.perm_ryser(B, [5], [1] * 5, gold=True))
    B = rng.standard_normal((6, 1)) + 1j * rng.standard_normal((6, 1))
    items.append((B, [1] * 6, [6]))
    want.append(O.perm_ryser(B, [1] * 6, [6], gold=True))
    pb = W.pack_batch(items)
    got, _ = gpu_perms(pb, dev)
    want = np.array(want, dtype=np.complex128)
    for (B, r, c), g, w in zip(items, got, want):
        # J_n and J - I cancel heavily in any inclusion-exclusion sum: allow
        # the a-priori rounding bound of the Glynn sum as well as TOL
        n = int(sum(r))
        bound = 0.0
        if 0 < n <= 14:
            bound = 8 * n * 2.0 ** -53 * glynn_abs_sum(np.repeat(np.repeat(B, r, 0), c, 1))
        assert abs(g - w) <= max(TOL * abs(w), bound), (n, g, w)


def glynn_abs_sum(A):
    """2^-(n-1) sum over sign vectors (first fixed) of prod_j |sum_i d_i a_ij|."""
    n = A.shape[0]
    if n == 1:
        return abs(A[0, 0])
    signs = np.array(np.meshgrid(*[[1.0, -1.0]] * (n - 1), indexing="ij")).reshape(n - 1, -1).T
    d = np.concatenate([np.ones((signs.shape[0], 1)), signs], axis=1)
    return float(np.prod(np.abs(d @ A), axis=1).sum()) / 2 ** (n - 1)


def test_argument_errors_on_device(dev):
    pb = W.pack_batch([(np.ones((2, 2)) + 0j, [1, 2], [1, 1])])  # 3 != 2
    with pytest.raises(pq.PQError) as e:
        api.Plan.for_batch(pb)
    assert e.value.code == pq.PQ_ERR_ARG


def test_bs_small_probabilities(dev):
    """Workload 1: m = 8, |1,1,1,1,0,0,0,0>, all 330 outputs; sum p = 1."""
    U, s, t = W.bs_small()
    p_ref, a_ref = O.bs_probs(U, s, t, gold=True)
    for method in ("batched", "plain"):
        plan = api.Plan.for_bs(8, s, t, method=method)
        p, a = api.bs_probs(torch.from_numpy(U).to(dev), torch.from_numpy(s).to(dev),
                            torch.from_numpy(t).to(dev), plan)
        torch.cuda.synchronize()
        p, a = p.cpu().numpy(), a.cpu().numpy()
        assert abs(p.sum() - 1.0) <= 1e-13
        assert rel_err(a, a_ref).max() <= TOL
        assert rel_err(p, p_ref).max() <= 2 * TOL
    # the convenience path without a plan
    p2, _ = api.bs_probs(torch.from_numpy(U).to(dev), torch.from_numpy(s).to(dev),
                         torch.from_numpy(t).to(dev), None)
    assert rel_err(p2.cpu().numpy(), p_ref).max() <= 2 * TOL


def test_hong_ou_mandel(dev):
    U = O.beamsplitter_block(math.pi / 4, 0.4)
    s = np.array([1, 1], dtype=np.int32)
    t = np.array([[1, 1], [2, 0], [0, 2]], dtype=np.int32)
    p, _ = api.bs_probs(torch.from_numpy(U).to(dev), torch.from_numpy(s).to(dev),
                        torch.from_numpy(t).to(dev), api.Plan.for_bs(2, s, t))
    p = p.cpu().numpy()
    assert abs(p[0]) <= 1e-16
    assert abs(p[1] - 0.5) <= 1e-15 and abs(p[2] - 0.5) <= 1e-15


def test_bs_batched_workload(dev):
    """Workload 3: m = 24, 12 photons, 4096 patterns (half with collisions)."""
    U, s, t = W.bs_batched()
    p_ref, a_ref = O.bs_probs(U, s, t, gold=True)
    Ud, sd, td = (torch.from_numpy(x).to(dev) for x in (U, s, t))
    for method, graph in (("batched", False), ("batched", True), ("plain", False)):
        plan = api.Plan.for_bs(24, s, t, method=method, use_graph=graph)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            p, a = api.bs_probs(Ud, sd, td, plan)
            if graph:  # replay the captured graph
                p, a = api.bs_probs(Ud, sd, td, plan)
        st.synchronize()
        assert rel_err(a.cpu().numpy(), a_ref).max() <= TOL
        assert rel_err(p.cpu().numpy(), p_ref).max() <= 2 * TOL


def test_ragged_workload_sampled(dev, ragged_pb):
    """Workload 4 at full size in the launch configuration the benchmark
    times (one graph-captured persistent launch, chunks autotuned per size
    class): every 16th item checked against the oracle plus every item of
    n = 20."""
    pb = ragged_pb
    db = api.DeviceBatch(pb, dev)
    plan = api.Plan.for_batch(pb, method="batched", use_graph=True)
    saved = pq.pq_tune_table_get()
    try:
        plan.autotune(db)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            out = api.permanent_batched(db, plan)
            out = api.permanent_batched(db, plan)  # the replay of the captured graph
        s.synchronize()
    finally:
        pq.pq_tune_table_set(saved)
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    ns = np.array([int(pb.row_mult[pb.row_off[b]:pb.row_off[b] + pb.k[b]].sum())
                   for b in range(pb.batch)])
    idx = sorted(set(range(0, pb.batch, 16)) | set(np.nonzero(ns == 20)[0][:256].tolist()))
    sub = pb.subset(idx)
    ref = O.perm_batch(sub.mats, sub.mat_off, sub.k, sub.l, sub.row_mult, sub.row_off,
                       sub.col_mult, sub.col_off, gold=True)
    assert rel_err(got[idx], ref).max() <= TOL
    assert plan.stats()["launches_forward"] == 1


def test_ragged_workload_plain_sampled(dev, ragged_pb):
    """Workload 4 by the plain method: 65536 launches, one per permanent, each
    cut to fill the GPU (the launch set the benchmark times as the plain
    path); every 64th item against the oracle."""
    pb = ragged_pb
    got, plan = gpu_perms(pb, dev, method="plain")
    assert plan.stats()["launches_forward"] == pb.batch
    assert np.isfinite(got).all()
    idx = list(range(0, pb.batch, 64))
    sub = pb.subset(idx)
    ref = O.perm_batch(sub.mats, sub.mat_off, sub.k, sub.l, sub.row_mult, sub.row_off,
                       sub.col_mult, sub.col_off, gold=True)
    assert rel_err(got[idx], ref).max() <= TOL


def product_columns(pb):
    """Columns on the product side of every item, as the planner orients it
    (pq_plan_item_info, host only)."""
    lib = pq.load_library()

    class Info(ctypes.Structure):
        _fields_ = [("n", ctypes.c_int32), ("k", ctypes.c_int32), ("l", ctypes.c_int32),
                    ("transposed", ctypes.c_int32), ("ndig", ctypes.c_int32),
                    ("J", ctypes.c_int32), ("terms", ctypes.c_int64),
                    ("chunk_len", ctypes.c_int64), ("chunks", ctypes.c_int64),
                    ("radix", ctypes.c_int32 * 48), ("row_of_digit", ctypes.c_int32 * 48)]

    out = np.zeros(pb.batch, dtype=np.int64)
    info = Info()
    for b in range(pb.batch):
        _, r, c = pb.item(b)
        r = np.ascontiguousarray(r, dtype=np.int32)
        c = np.ascontiguousarray(c, dtype=np.int32)
        assert lib.pq_plan_item_info(len(r), len(c), r.ctypes.data, c.ctypes.data, 0,
                                     ctypes.byref(info)) == 0
        out[b] = info.l
    return out


def test_ragged_workload_backward_sampled(dev, ragged_pb):
    """Backward of workload 4 at full size: the batched plan's launch per
    product-column class over all 65536 permanents plus the scatter (the
    launch set the benchmark times), against Laplace-minor permanents (gold)
    for every 64th item and every item of the widest class present (product
    columns in (14, 16]; this batch has none wider), at the gradient
    tolerance."""
    pb = ragged_pb
    db = api.DeviceBatch(pb, dev)
    plan = api.Plan.for_batch(pb)
    rng = np.random.default_rng(4004)
    gout = rng.standard_normal(pb.batch) + 1j * rng.standard_normal(pb.batch)
    g = api.permanent_backward(db, torch.from_numpy(gout).to(dev), plan).cpu().numpy()
    assert np.isfinite(g).all()
    lprod = product_columns(pb)
    assert lprod.max() == 16
    assert plan.stats()["launches_backward"] == 8 + 1  # classes l <= 2, 4, ..., 16; scatter
    wide = np.nonzero(lprod > 14)[0].tolist()
    assert len(wide) >= 16
    idx = sorted(set(range(0, pb.batch, 64)) | set(wide))

    def minors(b):
        B, r, c = pb.item(b)
        return O.perm_grad(B, r, c, gold=True)

    with ThreadPoolExecutor(O.default_threads()) as ex:
        refs = list(ex.map(minors, idx))
    for b, G in zip(idx, refs):
        B, r, c = pb.item(b)
        ref = gout[b] * np.conj(G)
        o = int(pb.mat_off[b])
        got = g[o:o + B.size].reshape(B.shape)
        assert np.abs(got - ref).max() <= TOLG * np.abs(ref).max(), b


def test_single_large_n30(dev):
    """Workload 2: n = 30 (2^29 Gray-code terms) against the stored gold value."""
    A, vals = read_matrix_file(os.path.join(HERE, "golden", "single_large_n30.txt"))
    assert vals["bound_gold"] < 1e-12 * abs(vals["per_gold"])
    pb = W.pack_batch([(A, [1] * 30, [1] * 30)])
    got, plan = gpu_perms(pb, dev)
    assert plan.stats()["terms"] == 2 ** 29
    assert rel_err(got[0], vals["per_gold"]) <= TOL30
    # the generator still produces this workload
    assert np.abs(W.single_large(30) - A).max() <= 1e-12


def test_results_are_deterministic(dev):
    U, s, t = W.bs_batched()
    plan = api.Plan.for_bs(24, s, t)
    Ud, sd, td = (torch.from_numpy(x).to(dev) for x in (U, s, t))
    p1, a1 = api.bs_probs(Ud, sd, td, plan)
    p2, a2 = api.bs_probs(Ud, sd, td, plan)
    torch.cuda.synchronize()
    assert torch.equal(a1, a2) and torch.equal(p1, p2)


def test_autotune_then_parity(dev):
    U, s, t = W.bs_batched()
    Ud, sd, td = (torch.from_numpy(x).to(dev) for x in (U, s, t))
    plan = api.Plan.for_bs(24, s, t)
    assert plan.stats()["column_sums"] == "registers"  # one column class
    plan.autotune(U=Ud)
    assert plan.stats()["column_sums"] in ("registers", "shared")  # the faster one
    p, a = api.bs_probs(Ud, sd, td, plan)
    p_ref, a_ref = O.bs_probs(U, s, t, gold=True)
    assert rel_err(a.cpu().numpy(), a_ref).max() <= TOL


def test_autotune_chooses_the_faster_column_sums_and_keeps_parity(dev):
    """A batch of one column class (collision-free n = 12): the autotuner
    times the plan with column sums in registers and in shared memory, keeps
    one, and the result still matches the oracle; forcing either form in
    the options keeps it through tuning."""
    A = W.single_large(30)
    items = [(A[i:i + 12, :12], [1] * 12, [1] * 12) for i in range(0, 18, 2)] * 64
    pb = W.pack_batch(items)
    db = api.DeviceBatch(pb, dev)
    ref = oracle_items(items[:9])
    for cs in ("auto", "shared", "registers"):
        plan = api.Plan.for_batch(pb, column_sums=cs)
        plan.autotune(db)
        form = plan.stats()["column_sums"]
        assert form == ("registers" if cs == "registers" else "shared") or cs == "auto"
        got = api.permanent_batched(db, plan).cpu().numpy()
        assert rel_err(got[:9], ref).max() <= TOL
        assert np.array_equal(got.view(np.float64), np.tile(got[:9], 64).view(np.float64))


# ------------------------------------------------------------------ backward
def test_permanent_backward_vs_minors(dev):
    rng = np.random.default_rng(404)
    items = random_items(60, 1, 10, rng)
    items.append((np.array([[0.5 + 0.1j]]), [1], [1]))
    items.append((np.zeros((0, 0)), [], []))
    pb = W.pack_batch(items)
    db = api.DeviceBatch(pb, dev)
    gout = (rng.standard_normal(pb.batch) + 1j * rng.standard_normal(pb.batch))
    for method in ("batched", "plain"):
        plan = api.Plan.for_batch(pb, method=method)
        g = api.permanent_backward(db, torch.from_numpy(gout).to(dev), plan).cpu().numpy()
        for b, (B, r, c) in enumerate(items):
            if B.size == 0:
                continue
            ref = gout[b] * np.conj(O.perm_grad(B, r, c, gold=True))
            o = int(pb.mat_off[b])
            got = g[o:o + B.size].reshape(B.shape)
            assert np.abs(got - ref).max() <= TOLG * max(np.abs(ref).max(), 1e-300)


def test_permanent_backward_large_product_sides(dev):
    """Backward launch classes for wide product sides (l up to 15) and narrow
    ones in one batch, both methods, against the Laplace minors."""
    rng = np.random.default_rng(406)
    items = random_items(3, 13, 15, rng, maxpart=1)   # every column distinct: l = n
    items += random_items(3, 14, 18, rng, maxpart=2)
    items += random_items(6, 2, 6, rng)
    pb = W.pack_batch(items)
    db = api.DeviceBatch(pb, dev)
    gout = (rng.standard_normal(pb.batch) + 1j * rng.standard_normal(pb.batch))
    refs = [gout[b] * np.conj(O.perm_grad(B, r, c)) for b, (B, r, c) in enumerate(items)]
    for method in ("batched", "plain"):
        plan = api.Plan.for_batch(pb, method=method)
        g = api.permanent_backward(db, torch.from_numpy(gout).to(dev), plan).cpu().numpy()
        assert plan.stats()["fp64_instr_backward"] > 0
        for b, (B, r, c) in enumerate(items):
            o = int(pb.mat_off[b])
            got = g[o:o + B.size].reshape(B.shape)
            assert np.abs(got - refs[b]).max() <= TOLG * np.abs(refs[b]).max()


def width_items(rng):
    """For every product width l = 1 .. 16 one item with distinct product
    columns and one with repeated ones (up to 4 copies for l <= 8, 2 above),
    the summed side repeated more (parts of 2 to 4), so that the planner keeps
    the repeated columns on the product side."""
    items = []
    for l in range(1, 17):
        for cmax in ((1, 4) if l <= 8 else (1, 2)):
            c = sorted((int(x) for x in rng.integers(1, cmax + 1, size=l)), reverse=True)
            if cmax > 1:
                c[0] = cmax
            n = sum(c)
            r, left = [], n
            while left:
                p = min(int(rng.integers(2, 5)), left)
                r.append(p)
                left -= p
            B = (rng.standard_normal((len(r), l)) + 1j * rng.standard_normal((len(r), l)))
            items.append((B / math.sqrt(2 * n), r, c))
    return items


def test_backward_every_product_width(dev):
    """Every backward launch class: product widths 1 .. 14 (the
    register-resident walk, odd and even widths of each class bound) and 15,
    16 (the shared-memory kernel), with and without repeated product columns,
    both methods, against the oracle's Laplace minors."""
    items = width_items(np.random.default_rng(408))
    pb = W.pack_batch(items)
    widths = product_columns(pb)
    assert set(range(1, 17)) <= set(int(w) for w in widths)
    db = api.DeviceBatch(pb, dev)
    rng = np.random.default_rng(409)
    gout = (rng.standard_normal(pb.batch) + 1j * rng.standard_normal(pb.batch))
    refs = [gout[b] * np.conj(O.perm_grad(B, r, c, gold=True)) for b, (B, r, c) in enumerate(items)]
    for method in ("batched", "plain"):
        plan = api.Plan.for_batch(pb, method=method)
        g = api.permanent_backward(db, torch.from_numpy(gout).to(dev), plan).cpu().numpy()
        for b, (B, r, c) in enumerate(items):
            o = int(pb.mat_off[b])
            got = g[o:o + B.size].reshape(B.shape)
            assert np.abs(got - refs[b]).max() <= TOLG * np.abs(refs[b]).max(), (method, b)
        assert pq.pq_plan_device_error(plan.handle) == (0, 0)


def walk_items(rng):
    """Product widths 1 .. 20 in one batch: random ragged items with repeated
    rows and columns (n <= 14), the width items of the backward test and
    all-distinct permanents of widths 17 .. 20."""
    items = random_items(80, 1, 14, rng) + width_items(rng)
    A = W.single_large(30)
    for l in range(17, 21):
        items.append((A[:l, :l], [1] * l, [1] * l))
    return items


@pytest.mark.parametrize("method", ["batched", "plain"])
def test_register_and_shared_walks_agree(dev, method):
    """The forward walk with column sums in registers (one instantiation per
    class of product widths; a batch mixing classes runs them all in one
    launch) and in shared memory: with the same chunks the same bits, and
    the oracle's permanents; a batch of one width class takes registers by
    default, a mixed one shared memory."""
    rng = np.random.default_rng(410)
    items = walk_items(rng)
    pb = W.pack_batch(items)
    db = api.DeviceBatch(pb, dev)
    outs = {}
    for cs in ("shared", "registers"):
        plan = api.Plan.for_batch(pb, method=method, chunk_log2=6, column_sums=cs)
        assert plan.stats()["column_sums"] == cs
        outs[cs] = api.permanent_batched(db, plan).cpu().numpy()
        assert pq.pq_plan_device_error(plan.handle) == (0, 0)
    assert np.array_equal(outs["shared"].view(np.float64), outs["registers"].view(np.float64))
    ref = oracle_items(items)
    assert rel_err(outs["registers"], ref).max() <= TOL
    assert api.Plan.for_batch(pb).stats()["column_sums"] == "shared"
    w = product_columns(pb)
    idx = np.nonzero((w == 11) | (w == 12))[0]
    assert idx.size >= 2
    assert api.Plan.for_batch(pb.subset(idx)).stats()["column_sums"] == "registers"


@pytest.mark.parametrize("method", ["batched", "plain"])
def test_register_walk_of_one_class_narrower_than_its_bound(dev, method):
    """Batches of one column class whose widest permanent is narrower than
    the class's register count (at most 3 product columns: 4 registers; 5: 6;
    11: 12), run by default with the column sums in registers: the oracle's
    and the shared-memory walk's permanents, no device error."""
    rng = np.random.default_rng(411)
    items = walk_items(rng)
    pb = W.pack_batch(items)
    w = product_columns(pb)
    ref_all = oracle_items(items)
    for sel in (w <= 3, w == 5, w == 11):
        idx = np.nonzero(sel)[0]
        assert idx.size >= 1
        sub = pb.subset(idx)
        db = api.DeviceBatch(sub, dev)
        plan = api.Plan.for_batch(sub, method=method)
        assert plan.stats()["column_sums"] == "registers"
        got = api.permanent_batched(db, plan).cpu().numpy()
        assert pq.pq_plan_device_error(plan.handle) == (0, 0)
        assert rel_err(got, ref_all[idx]).max() <= TOL
        shared = api.Plan.for_batch(sub, method=method, column_sums="shared")
        assert rel_err(got, api.permanent_batched(db, shared).cpu().numpy()).max() <= TOL


def test_permanent_gradcheck(dev):
    rng = np.random.default_rng(505)
    items = random_items(4, 2, 5, rng)
    pb = W.pack_batch(items)
    db = api.DeviceBatch(pb, dev)
    plan = api.Plan.for_batch(pb)
    mats = torch.from_numpy(pb.mats).to(dev).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: api.Permanent.apply(x, db, plan), (mats,),
                                    eps=1e-6, atol=1e-8, rtol=1e-6)


def test_clements_forward(dev):
    th, ph, s, t = W.gradient_workload()
    U = api.clements_forward(torch.from_numpy(th).to(dev), torch.from_numpy(ph).to(dev), 16)
    ref = O.clements_unitary(th, ph, 16)
    assert np.abs(U.cpu().numpy() - ref).max() <= 1e-13


def test_gradient_workload(dev):
    """Workload 5: Clements mesh (m = 16, 120 beamsplitters) -> probabilities of
    1024 patterns with 8 photons -> L = sum p; dL/dU against Laplace-minor
    permanents, dL/d(theta, phi) against the oracle's chain rule and against
    central finite differences (h = 1e-6) of the oracle's L."""
    th, ph, s, t = W.gradient_workload()
    thd = torch.from_numpy(th).to(dev).requires_grad_(True)
    phd = torch.from_numpy(ph).to(dev).requires_grad_(True)
    sd, td = torch.from_numpy(s).to(dev), torch.from_numpy(t).to(dev)
    plan = api.Plan.for_bs(16, s, t)
    U = api.ClementsMesh.apply(thd, phd, 16)
    U.retain_grad()
    L = api.BSProbs.apply(U, sd, td, plan).sum()
    L.backward()
    torch.cuda.synchronize()
    Uref = O.clements_unitary(th, ph, 16)
    p_ref, _ = O.bs_probs(Uref, s, t, gold=True)
    assert abs(L.item() - p_ref.sum()) <= TOL * p_ref.sum()
    G_ref = O.bs_grad_U(Uref, s, t, np.ones(len(t)), gold=True)
    G = U.grad.cpu().numpy()
    assert np.abs(G - G_ref).max() <= TOLG * np.abs(G_ref).max()
    gt_ref, gp_ref = O.clements_grad(th, ph, 16, G_ref)
    gt, gp = thd.grad.cpu().numpy(), phd.grad.cpu().numpy()
    scale = max(np.abs(gt_ref).max(), np.abs(gp_ref).max())
    assert np.abs(gt - gt_ref).max() <= TOLG * scale
    assert np.abs(gp - gp_ref).max() <= TOLG * scale

    def L_oracle(a, b):
        return O.bs_probs(O.clements_unitary(a, b, 16), s, t)[0].sum()

    h = 1e-6
    for k in (0, 7, 8, 59, 119):
        e = np.zeros(120)
        e[k] = h
        fd_t = (L_oracle(th + e, ph) - L_oracle(th - e, ph)) / (2 * h)
        fd_p = (L_oracle(th, ph + e) - L_oracle(th, ph - e)) / (2 * h)
        assert abs(gt[k] - fd_t) <= TOLG * scale
        assert abs(gp[k] - fd_p) <= TOLG * scale


def test_bs_backward_plain_matches_batched(dev):
    th, ph, s, t = W.gradient_workload()
    U = torch.from_numpy(O.clements_unitary(th, ph, 16)).to(dev)
    sd, td = torch.from_numpy(s).to(dev), torch.from_numpy(t).to(dev)
    g = torch.linspace(0.5, 1.5, len(t), dtype=torch.float64, device=dev)
    outs = []
    for method in ("batched", "plain"):
        plan = api.Plan.for_bs(16, s, t, method=method)
        p, a = api.bs_probs(U, sd, td, plan)
        outs.append(api.bs_probs_backward(U, sd, td, g, a, plan).cpu().numpy())
    # the two methods chunk the forward differently, so the amplitudes fed to
    # the backward may differ in the last bits
    assert np.abs(outs[0] - outs[1]).max() <= 1e-12 * np.abs(outs[0]).max()


def test_fp64_probe_runs(dev):
    flops, ms = api.probe_fp64_peak(1 << 12)
    assert flops > 1e11 and ms > 0


def test_later_plan_with_smaller_workspace_keeps_earlier_plan_working(dev):
    """A plan made later with less shared memory per block must not lower the
    launch limit an earlier, larger plan relies on."""
    A = W.single_large(26)
    big = W.pack_batch([(A, [1] * 26, [1] * 26)])
    ref = O.perm_ryser(A, gold=True, nthreads=O.default_threads())
    db = api.DeviceBatch(big, dev)
    plan_big = api.Plan.for_batch(big)
    small = W.pack_batch([(np.array([[0.5 + 0.5j]]), [1], [1])])
    plan_small = api.Plan.for_batch(small)
    api.permanent_batched(api.DeviceBatch(small, dev), plan_small)
    got = api.permanent_batched(db, plan_big).cpu().numpy()
    assert rel_err(got[0], ref) <= TOL


@pytest.mark.parametrize("method", ["batched", "plain"])
def test_paper_repeated_permanents(dev, method):
    """The shape of the paper's repeated-permanent benchmark (Sec. 4.2, Fig.
    permanent): a k x k Haar block with every row and column repeated twice,
    k = 4 .. 14 (2 * 3^(k-1) Gray-code terms), one permanent per k."""
    items = [W.paper_repeated(k) for k in range(4, 15)]
    pb = W.pack_batch(items)
    ref = np.array([O.perm_ryser(B, r, c, gold=True, nthreads=O.default_threads())
                    for B, r, c in items])
    got, plan = gpu_perms(pb, dev, method)
    assert plan.stats()["terms"] == sum(2 * 3 ** (k - 1) for k in range(4, 15))
    assert rel_err(got, ref).max() <= TOL


@pytest.mark.parametrize("use_graph", [False, True])
def test_plans_run_inside_a_callers_graph_capture(dev, use_graph):
    """An executed plan allocates nothing, reads no host memory and does not
    synchronise, so a caller can capture it (forward, boson-sampling
    probabilities and, after the first backward call, the backward) into its
    own CUDA graph; replays follow new input values."""
    rng = np.random.default_rng(707)
    items = random_items(40, 2, 9, rng)
    pb = W.pack_batch(items)
    db = api.DeviceBatch(pb, dev)
    plan = api.Plan.for_batch(pb, use_graph=use_graph)
    out = torch.empty(pb.batch, dtype=torch.complex128, device=dev)
    gout = torch.ones(pb.batch, dtype=torch.complex128, device=dev)
    api.permanent_backward(db, gout, plan)  # plans the backward outside the capture
    U, s, t = W.bs_small()
    Ud, sd, td = (torch.from_numpy(x).to(dev) for x in (U, s, t))
    bplan = api.Plan.for_bs(8, s, t, use_graph=use_graph)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        api.permanent_batched(db, plan, out=out)
        grad = api.permanent_backward(db, gout, plan)
        probs, _ = api.bs_probs(Ud, sd, td, bplan)
    for rep in range(2):
        new = (rng.standard_normal(pb.mats.shape) + 1j * rng.standard_normal(pb.mats.shape)) * 0.3
        db.mats.copy_(torch.from_numpy(new))
        Ud.copy_(torch.from_numpy(W.haar_unitary(8, rng)))
        g.replay()
        torch.cuda.synchronize()
        ref_out = api.permanent_batched(db, plan).cpu().numpy()
        ref_grad = api.permanent_backward(db, gout, plan).cpu().numpy()
        ref_p, _ = api.bs_probs(Ud, sd, td, bplan)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref_out)
        assert np.array_equal(grad.cpu().numpy(), ref_grad)
        assert np.array_equal(probs.cpu().numpy(), ref_p.cpu().numpy())
        # and the values are the permanents of the new matrices
        for b in range(0, pb.batch, 7):
            B, r, c = items[b]
            o = int(pb.mat_off[b])
            Bn = new[o:o + B.size].reshape(B.shape)
            ref = O.perm_ryser(Bn, r, c, gold=True)
            assert abs(ref_out[b] - ref) <= TOL * max(abs(ref), 1e-300)


@pytest.mark.parametrize("nshards", [1, 2, 3, 7])
def test_sharded_plans_sum_to_the_permanents(dev, nshards):
    """Every shard's plan covers its range of each permanent's warp tasks; the
    shards' partials, combined in double-double, give the permanents.  The
    shards run one after another on this GPU (no shard waits on another)."""
    rng = np.random.default_rng(808)
    A = W.single_large(30)[:20, :20]
    items = [(A, [1] * 20, [1] * 20)]                 # 2^19 terms: many tasks
    items += random_items(10, 2, 12, rng)             # fewer tasks than shards
    items.append((np.zeros((0, 0)), [], []))          # n = 0
    pb = W.pack_batch(items)
    db = api.DeviceBatch(pb, dev)
    ref = api.permanent_batched(db, api.Plan.for_batch(pb)).cpu().numpy()
    parts = []
    for r in range(nshards):
        plan = api.Plan.for_batch(pb, shard=(r, nshards))
        parts.append(api.permanent_partials(db, plan).cpu().numpy())
    n = np.array([int(np.sum(r)) for _, r, _ in items])
    got = api.combine_partials(parts, n)
    assert got[-1] == 1.0
    for b, (B, r, c) in enumerate(items[:-1]):
        assert abs(got[b] - ref[b]) <= 1e-13 * abs(ref[b])
    w0 = O.perm_ryser(A, gold=True)
    assert abs(got[0] - w0) <= TOL * abs(w0)


def test_sharded_plan_misuse(dev):
    pb = W.pack_batch([(np.eye(3) + 0j, [1, 1, 1], [1, 1, 1])])
    db = api.DeviceBatch(pb, dev)
    sh = api.Plan.for_batch(pb, shard=(0, 2))
    plain = api.Plan.for_batch(pb)
    for call, code in ((lambda: api.permanent_batched(db, sh), pq.PQ_ERR_STATE),
                       (lambda: api.permanent_partials(db, plain), pq.PQ_ERR_STATE),
                       (lambda: sh.autotune(db), pq.PQ_ERR_STATE),
                       (lambda: api.permanent_backward(
                           db, torch.ones(1, dtype=torch.complex128, device=dev), sh),
                        pq.PQ_ERR_STATE),
                       (lambda: api.Plan.for_batch(pb, shard=(2, 2)), pq.PQ_ERR_ARG),
                       (lambda: api.Plan.for_bs(3, [1, 1, 1], [[1, 1, 1]], shard=(0, 2)),
                        pq.PQ_ERR_UNSUPPORTED)):
        with pytest.raises(pq.PQError) as e:
            call()
        assert e.value.code == code


@pytest.mark.parametrize("method", ["batched", "plain"])
def test_overflowing_permanent_is_not_finite(dev, method):
    """A permanent whose terms overflow FP64 (1 x 1 base 1e200 repeated twice:
    per = 2 * 1e400) comes out infinite or NaN, as FP64 arithmetic gives it,
    not as a finite number made up by the integer lane sum; the permanents
    beside it in the batch are unaffected."""
    rng = np.random.default_rng(77)
    items = random_items(6, 2, 8, rng) + [(np.array([[1e200 + 0j]]), [2], [2])]
    pb = W.pack_batch(items)
    got = api.permanent_batched(api.DeviceBatch(pb, dev), api.Plan.for_batch(pb, method=method))
    got = got.cpu().numpy()
    assert not np.isfinite(got[-1])
    ref = oracle_items(items[:-1])
    assert rel_err(got[:-1], ref).max() <= TOL
