"""Runtime services of the library that need no GPU: the tuning table and its
JSON cache on disk, and the allocation-failure test hook on the host objects
the library creates."""
import json
import os

import numpy as np
import pytest

from paper_2403_04006_gb300 import build as B
from paper_2403_04006_gb300 import pq


@pytest.fixture(scope="module")
def lib():
    B.build()
    return pq.load_library()


@pytest.fixture
def table_restored(lib):
    saved = pq.pq_tune_table_get()
    yield
    pq.pq_tune_table_set(saved)


def test_tune_table_set_and_get(lib, table_restored):
    t = np.zeros(pq.PQ_MAX_N + 1, dtype=np.int32)
    t[12], t[20] = 6, 8
    pq.pq_tune_table_set(t)
    assert np.array_equal(pq.pq_tune_table_get(), t)
    bad = t.copy()
    bad[3] = 31
    with pytest.raises(pq.PQError) as e:
        pq.pq_tune_table_set(bad)
    assert e.value.code == pq.PQ_ERR_ARG
    assert np.array_equal(pq.pq_tune_table_get(), t)  # a rejected table changes nothing


def test_tune_cache_round_trip_keeps_other_devices(lib, table_restored, tmp_path):
    path = str(tmp_path / "tune.json")
    assert not pq.pq_tune_cache_load(path, "gpu-a")  # no file yet: not found, no error
    a = np.zeros(pq.PQ_MAX_N + 1, dtype=np.int32)
    a[4:21] = np.arange(17) % 5 + 4
    pq.pq_tune_table_set(a)
    pq.pq_tune_cache_save(path, "gpu-a")
    b = np.full(pq.PQ_MAX_N + 1, 10, dtype=np.int32)
    pq.pq_tune_table_set(b)
    pq.pq_tune_cache_save(path, 'gpu "b"')  # a key that needs escaping
    doc = json.load(open(path))
    assert set(doc["tables"]) == {"gpu-a", 'gpu "b"'}
    assert doc["tables"]["gpu-a"] == a.tolist()
    pq.pq_tune_table_set(np.zeros(pq.PQ_MAX_N + 1, dtype=np.int32))
    assert pq.pq_tune_cache_load(path, "gpu-a")
    assert np.array_equal(pq.pq_tune_table_get(), a)
    assert pq.pq_tune_cache_load(path, 'gpu "b"')
    assert np.array_equal(pq.pq_tune_table_get(), b)
    assert not pq.pq_tune_cache_load(path, "gpu-c")
    assert np.array_equal(pq.pq_tune_table_get(), b)  # unknown key: table untouched


def test_tune_cache_reads_foreign_members_and_rejects_garbage(lib, table_restored, tmp_path):
    path = str(tmp_path / "tune.json")
    t = list(range(pq.PQ_MAX_N + 1))
    t = [x % 13 for x in t]
    with open(path, "w") as f:
        json.dump({"comment": ["x", {"y": None}], "tables": {"k": t}, "extra": 1.5e3}, f)
    assert pq.pq_tune_cache_load(path, "k")
    assert pq.pq_tune_table_get().tolist() == t
    pq.pq_tune_cache_save(path, "k2")
    assert set(json.load(open(path))["tables"]) == {"k", "k2"}
    with open(path, "w") as f:
        f.write('{"tables": {"k": [1, 2')
    with pytest.raises(pq.PQError) as e:
        pq.pq_tune_cache_load(path, "k")
    assert e.value.code == pq.PQ_ERR_ARG
    with pytest.raises(pq.PQError):
        pq.pq_tune_cache_save(path, "k")  # does not overwrite a file it cannot read
    with open(path, "w") as f:
        json.dump({"tables": {"short": [1, 2, 3]}}, f)
    with pytest.raises(pq.PQError) as e:
        pq.pq_tune_cache_load(path, "short")
    assert e.value.code == pq.PQ_ERR_ARG


def test_allocation_hook_fails_plan_creation_and_leaks_nothing(lib):
    """The plan object is the first allocation of pq_plan_create, before any
    CUDA call, so the hook's failure is visible without a GPU."""
    import ctypes
    r = np.array([1, 1], dtype=np.int32)
    z = np.array([0], dtype=np.int64)
    k = np.array([2], dtype=np.int32)
    s = pq.pq_batch_sizes()
    s.batch = 1
    s.mat_off, s.k, s.l, s.row_mult, s.row_off, s.col_mult, s.col_off = (
        z.ctypes.data, k.ctypes.data, k.ctypes.data, r.ctypes.data, z.ctypes.data,
        r.ctypes.data, z.ctypes.data)
    before = pq.pq_debug_live_allocations()
    out = ctypes.c_void_p()
    pq.pq_debug_fail_allocation(0)
    try:
        assert lib.pq_plan_create(ctypes.byref(s), None, ctypes.byref(out)) == pq.PQ_ERR_NOMEM
    finally:
        pq.pq_debug_fail_allocation(-1)
    assert out.value is None
    assert pq.pq_debug_live_allocations() == before
    assert "allocation" in pq.pq_last_error()
    # disarmed: the same call gets past the allocation; here it stops at the
    # missing GPU (or succeeds on a GPU host), and still leaks nothing
    rc = lib.pq_plan_create(ctypes.byref(s), None, ctypes.byref(out))
    if rc == pq.PQ_OK:
        pq.pq_plan_destroy(out.value)
    else:
        assert rc == pq.PQ_ERR_CUDA
    assert pq.pq_debug_live_allocations() == before


def test_hook_is_one_shot_and_counts_successful_allocations(lib):
    import ctypes
    r = np.array([1], dtype=np.int32)
    z = np.array([0], dtype=np.int64)
    k = np.array([1], dtype=np.int32)
    s = pq.pq_batch_sizes()
    s.batch = 1
    s.mat_off, s.k, s.l, s.row_mult, s.row_off, s.col_mult, s.col_off = (
        z.ctypes.data, k.ctypes.data, k.ctypes.data, r.ctypes.data, z.ctypes.data,
        r.ctypes.data, z.ctypes.data)
    out = ctypes.c_void_p()
    pq.pq_debug_fail_allocation(0)
    try:
        assert lib.pq_plan_create(ctypes.byref(s), None, ctypes.byref(out)) == pq.PQ_ERR_NOMEM
        rc = lib.pq_plan_create(ctypes.byref(s), None, ctypes.byref(out))  # hook spent
        assert rc in (pq.PQ_OK, pq.PQ_ERR_CUDA)
        if rc == pq.PQ_OK:
            pq.pq_plan_destroy(out.value)
    finally:
        pq.pq_debug_fail_allocation(-1)
