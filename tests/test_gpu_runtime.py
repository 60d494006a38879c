"""Runtime services on the GPU: device allocations that fail part-way leave
nothing behind, the kernels' task guards catch a corrupted plan and record
it instead of reading out of bounds, and the device combination of shard
partials equals the host one bit for bit."""
import gc

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2403_04006_gb300 import api, pq  # noqa: E402
from paper_2403_04006_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pq.load_library()
    return torch.device("cuda:0")


def small_items(seed, count=24, nmax=9):
    rng = np.random.default_rng(seed)
    items = []
    for _ in range(count):
        n = int(rng.integers(2, nmax + 1))
        r, c = [], []
        for out in (r, c):
            left = n
            while left:
                p = min(int(rng.integers(1, 3)), left)
                out.append(p)
                left -= p
        B = (rng.standard_normal((len(r), len(c))) + 1j * rng.standard_normal((len(r), len(c))))
        items.append((B / np.sqrt(2 * n), r, c))
    return items


def every_allocating_call(dev, pb, db):
    """Plans and runs each allocating entry point once, closing what it made."""
    plans = []
    try:
        plan = api.Plan.for_batch(pb)
        plans.append(plan)
        api.permanent_batched(db, plan)
        api.permanent_backward(db, torch.ones(pb.batch, dtype=torch.complex128, device=dev), plan)
        U, s, t = W.bs_small()
        Ud, sd, td = (torch.from_numpy(x).to(dev) for x in (U, s, t))
        bplan = api.Plan.for_bs(8, s, t[:40])
        plans.append(bplan)
        p, a = api.bs_probs(Ud, sd, td[:40], bplan)
        api.bs_probs_backward(Ud, sd, td[:40], torch.ones_like(p), a, bplan)
        api.permanent_batched(db, None)  # convenience path: plans and frees inside
        B, r, g = W.paper_repeated_hafnian(4, loop=True)
        Bd = torch.from_numpy(B.reshape(-1)).to(dev)
        api.hafnian_repeated(Bd, [0], [4], r, [0], gamma=torch.from_numpy(g).to(dev))
        hp = api.HafnianPlan([0], [4], r, [0])
        plans.append(hp)
        hp.run(Bd)
        V = torch.from_numpy(W.haar_unitary(3, np.random.default_rng(5))).to(dev)
        api.bs_probs_lossy(V, torch.full((3,), 0.7, dtype=torch.float64, device=dev), V,
                           [1, 1, 0], [[1, 0, 0], [1, 1, 0]])
        order, unif = W.sampler_draws(4, 2, 6)
        api.bs_sample(V, np.array([1, 1, 0], dtype=np.int32), order, unif)
        sp = api.SamplerPlan(3, np.array([1, 1, 0], dtype=np.int32), 4)
        plans.append(sp)
        sp.run(V, order, unif)
        lp = api.LossyPlan(3, [1, 1, 0], [[1, 0, 0], [1, 1, 0]])
        plans.append(lp)
        lp.run(V, torch.full((3,), 0.7, dtype=torch.float64, device=dev), V)
        torch.cuda.synchronize()
    finally:
        for p in plans:
            p.close()


def test_failed_allocations_leave_nothing_behind(dev):
    pb = W.pack_batch(small_items(31))
    db = api.DeviceBatch(pb, dev)
    every_allocating_call(dev, pb, db)  # warm: kernel attributes, lazy module loads
    gc.collect()
    base = pq.pq_debug_live_allocations()
    failures = 0
    after = 0
    while True:
        pq.pq_debug_fail_allocation(after)
        try:
            every_allocating_call(dev, pb, db)
            done = True
        except pq.PQError as e:
            assert e.code == pq.PQ_ERR_NOMEM, (after, str(e))
            failures += 1
            done = False
        finally:
            pq.pq_debug_fail_allocation(-1)
        gc.collect()
        assert pq.pq_debug_live_allocations() == base, after
        if done:
            break
        after += 1
    assert failures >= 20  # every allocation of every call was made to fail once


def corrupted_run(dev, what, method):
    items = small_items(32, count=40, nmax=12)
    pb = W.pack_batch(items)
    db = api.DeviceBatch(pb, dev)
    clean = api.permanent_batched(db, api.Plan.for_batch(pb, method=method)).cpu().numpy()
    plan = api.Plan.for_batch(pb, method=method)
    assert pq.pq_plan_device_error(plan.handle) == (0, 0)
    pq.pq_debug_corrupt_plan(plan.handle, what)
    out = torch.full((pb.batch,), complex(7.0, 7.0), dtype=torch.complex128, device=dev)
    api.permanent_batched(db, plan, out=out)
    got = out.cpu().numpy()
    code, task = pq.pq_plan_device_error(plan.handle, clear=True)
    assert pq.pq_plan_device_error(plan.handle) == (0, 0)  # cleared
    plan.close()
    return clean, got, code, task


@pytest.mark.parametrize("method", ["batched", "plain"])
def test_guard_catches_task_outside_the_batch(dev, method):
    clean, got, code, task = corrupted_run(dev, 1, method)
    assert code == pq.PQ_DEVERR_TASK_PERM and task == 0
    # only the permanent whose task was lost stays unwritten
    bad = np.nonzero(got != clean)[0]
    assert len(bad) <= 1 and (len(bad) == 0 or got[bad[0]] == complex(7.0, 7.0))


def test_guard_catches_descriptor_beyond_the_launch_layout(dev):
    clean, got, code, task = corrupted_run(dev, 2, "batched")
    assert code == pq.PQ_DEVERR_LAYOUT
    assert got[0] == complex(7.0, 7.0)  # permanent 0 skipped
    assert np.array_equal(got[1:], clean[1:])


def test_clean_runs_record_nothing(dev):
    pb = W.pack_batch(small_items(33))
    db = api.DeviceBatch(pb, dev)
    for method in ("batched", "plain"):
        plan = api.Plan.for_batch(pb, method=method)
        api.permanent_batched(db, plan)
        api.permanent_backward(db, torch.ones(pb.batch, dtype=torch.complex128, device=dev), plan)
        assert pq.pq_plan_device_error(plan.handle) == (0, 0)
        plan.close()


def test_device_combine_equals_host_combine(dev):
    """Shards of a batch (run one after another on this GPU) combined by the
    device kernel and by the host twin: the same bits, and the oracle's
    permanents."""
    items = small_items(34, count=30, nmax=14)
    A = W.single_large(30)[:18, :18]
    items.append((A, [1] * 18, [1] * 18))
    items.append((np.zeros((0, 0)), [], []))
    pb = W.pack_batch(items)
    db = api.DeviceBatch(pb, dev)
    for R in (2, 5):
        parts = torch.stack([api.permanent_partials(db, api.Plan.for_batch(pb, shard=(r, R)))
                             for r in range(R)])
        n = api.photon_numbers(pb)
        d = api.combine_partials_device(parts, torch.from_numpy(n).to(dev)).cpu().numpy()
        h = api.combine_partials([p for p in parts.cpu().numpy()], n)
        assert np.array_equal(d.view(np.float64), h.view(np.float64))
        assert d[-1] == 1.0
        for b, (B, r, c) in enumerate(items[:-1]):
            ref = O.perm_ryser(B, r, c, gold=True)
            assert abs(d[b] - ref) <= 1e-10 * abs(ref), (R, b)


def test_shards_balance_small_permanents(dev):
    """A permanent with fewer tasks than shards goes to a shard that depends
    on its index, so single-task permanents spread over all shards."""
    items = small_items(35, count=64, nmax=6)  # one warp task each
    pb = W.pack_batch(items)
    db = api.DeviceBatch(pb, dev)
    R = 4
    held = []
    for r in range(R):
        p = api.permanent_partials(db, api.Plan.for_batch(pb, shard=(r, R))).cpu().numpy()
        held.append(int((np.abs(p).sum(axis=1) > 0).sum()))
    assert sum(held) == pb.batch
    assert min(held) >= pb.batch // R - 1


def test_tune_cache_under_the_current_device_name(dev, tmp_path):
    """Without a key the cache is filed under this GPU's name and SM count;
    a plan made after loading it uses the stored chunk length (2^5 terms for
    n = 16: the warp tasks of a plan asked for 2^5, not those of the default
    plan, which lowers its cap for a batch this small) and still gives the
    oracle's permanent."""
    import json
    A = W.single_large(16)
    pb = W.pack_batch([(A, [1] * 16, [1] * 16)])
    saved = pq.pq_tune_table_get()
    try:
        pq.pq_tune_table_set(np.zeros(pq.PQ_MAX_N + 1, dtype=np.int32))
        default_tasks = api.Plan.for_batch(pb).stats()["tasks"]
        fixed_tasks = api.Plan.for_batch(pb, chunk_log2=5).stats()["tasks"]
        assert fixed_tasks != default_tasks
        t = np.zeros(pq.PQ_MAX_N + 1, dtype=np.int32)
        t[16] = 5
        pq.pq_tune_table_set(t)
        path = str(tmp_path / "tune.json")
        pq.pq_tune_cache_save(path)
        key, = json.load(open(path))["tables"].keys()
        assert torch.cuda.get_device_name(0) in key and "SMs" in key
        pq.pq_tune_table_set(np.zeros_like(t))
        assert pq.pq_tune_cache_load(path)
        assert pq.pq_tune_table_get()[16] == 5
        plan = api.Plan.for_batch(pb)
        assert plan.stats()["tasks"] == fixed_tasks
        got = api.permanent_batched(api.DeviceBatch(pb, dev), plan).cpu().numpy()[0]
        ref = O.perm_ryser(A, gold=True)
        assert abs(got - ref) <= 1e-10 * abs(ref)
    finally:
        pq.pq_tune_table_set(saved)


def test_partitioned_batch_matches_the_whole(dev):
    """The items of each rank of a 3-way partition (pq_partition_batch),
    evaluated one rank after another on this GPU and put back in item order,
    give the whole batch's permanents (a smaller batch may cut its Gray codes
    into other chunks, so to 1e-11 relative) and the oracle's; without a
    process group the partitioned call evaluates the whole batch."""
    items = small_items(36, count=60, nmax=14)
    items.append((np.zeros((0, 0)), [], []))
    pb = W.pack_batch(items)
    whole = api.permanent_batched(api.DeviceBatch(pb, dev), api.Plan.for_batch(pb)).cpu().numpy()
    rank_of, terms = api.partition_batch(pb, 3)
    assert (np.bincount(rank_of, minlength=3) > 0).all()
    got = np.full(pb.batch, complex(7.0, 7.0))
    for r in range(3):
        idx = np.nonzero(rank_of == r)[0]
        sub = pb.subset(idx)
        got[idx] = api.permanent_batched(api.DeviceBatch(sub, dev),
                                         api.Plan.for_batch(sub)).cpu().numpy()
    assert np.all(np.abs(got - whole) <= 1e-11 * np.abs(whole))
    for b, (B, r, c) in enumerate(items):
        ref = O.perm_ryser(B, r, c, gold=True)
        assert abs(got[b] - ref) <= 1e-10 * abs(ref), b
    solo = api.permanent_partitioned(pb, dev).cpu().numpy()
    assert np.all(np.abs(solo - whole) <= 1e-11 * np.abs(whole))
