"""Thin Python binding of the C ABI in include/pq.h.

Every ``pq_*`` function here has the name of the C entry point it calls and
only marshals arguments (torch tensors to device pointers, numpy arrays to
host pointers); all arithmetic of the permanent path runs in the CUDA
library.  The library must have been built (``paper_2403_04006_gb300.build``);
if it is missing every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpq_gb300.so")

PQ_OK = 0
PQ_ERR_ARG = -1
PQ_ERR_UNSUPPORTED = -2
PQ_ERR_CUDA = -3
PQ_ERR_TIMEOUT = -4
PQ_ERR_NOMEM = -5
PQ_ERR_STATE = -6
PQ_METHOD_BATCHED = 0
PQ_METHOD_PLAIN = 1
PQ_SUMS_AUTO, PQ_SUMS_SHARED, PQ_SUMS_REGISTERS = 0, 1, 2
PQ_MAX_N = 48
PQ_DEVERR_TASK_PERM = 1
PQ_DEVERR_TASK_PART = 2
PQ_DEVERR_LAYOUT = 3
PQ_DEVERR_DIGITS = 4
PQ_DEVERR_INDEX = 5

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


class pq_batch(ctypes.Structure):
    _fields_ = [("batch", _i64), ("mats", _vp), ("mat_off", _vp), ("k", _vp), ("l", _vp),
                ("row_mult", _vp), ("row_off", _vp), ("col_mult", _vp), ("col_off", _vp)]


class pq_batch_sizes(ctypes.Structure):
    _fields_ = [("batch", _i64), ("mat_off", _vp), ("k", _vp), ("l", _vp), ("row_mult", _vp),
                ("row_off", _vp), ("col_mult", _vp), ("col_off", _vp)]


class pq_plan_options(ctypes.Structure):
    _fields_ = [("method", _i32), ("use_graph", _i32), ("chunk_log2", _i32),
                ("warps_per_block", _i32), ("blocks_per_sm", _i32), ("shard_index", _i32),
                ("shard_count", _i32), ("column_sums", _i32)]


class pq_plan_stats(ctypes.Structure):
    _fields_ = [("permanents", _i64), ("terms", _i64), ("flops_forward", ctypes.c_double),
                ("flops_backward", ctypes.c_double), ("tasks", _i64),
                ("launches_forward", _i64), ("launches_backward", _i64), ("lmax", _i32),
                ("column_sums", _i32), ("fp64_instr_forward", ctypes.c_double),
                ("fp64_instr_backward", ctypes.c_double),
                ("fp64_instr_forward_executed", ctypes.c_double)]


# name -> (restype, argtypes)
_SIGNATURES = {
    "pq_plan_create": (_i32, [ctypes.POINTER(pq_batch_sizes), ctypes.POINTER(pq_plan_options),
                              ctypes.POINTER(_vp)]),
    "pq_plan_create_bs": (_i32, [_i32, _vp, _vp, _i64, ctypes.POINTER(pq_plan_options),
                                 ctypes.POINTER(_vp)]),
    "pq_plan_destroy": (_i32, [_vp]),
    "pq_permanent_batched": (_i32, [ctypes.POINTER(pq_batch), _vp, _vp, _vp]),
    "pq_permanent_partials": (_i32, [ctypes.POINTER(pq_batch), _vp, _vp, _vp]),
    "pq_bs_probs": (_i32, [_vp, _i32, _vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "pq_permanent_backward": (_i32, [ctypes.POINTER(pq_batch), _vp, _vp, _vp, _vp]),
    "pq_bs_probs_backward": (_i32, [_vp, _i32, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    "pq_clements_forward": (_i32, [_vp, _vp, _i32, _vp, _vp]),
    "pq_clements_backward": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "pq_autotune": (_i32, [_vp, ctypes.POINTER(pq_batch), _vp, _vp]),
    "pq_plan_get_stats": (_i32, [_vp, ctypes.POINTER(pq_plan_stats)]),
    "pq_probe_fp64_peak": (_i32, [_i64, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), _vp]),
    "pq_probe_fp64_sweep": (_i32, [_i32, _i32, _i32, _i64, ctypes.POINTER(ctypes.c_double), _vp]),
    "pq_permanent_noalloc": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp, _vp]),
    "pq_bs_sample": (_i32, [_vp, _i32, _vp, _i64, _vp, _vp, _vp, _vp]),
    "pq_bs_probs_lossy": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _i64, _vp, _vp]),
    "pq_lossy_plan_create": (_i32, [_i32, _vp, _vp, _i64, ctypes.POINTER(_vp)]),
    "pq_lossy_plan_run": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "pq_lossy_plan_destroy": (_i32, [_vp]),
    "pq_partition_batch": (_i32, [ctypes.POINTER(pq_batch_sizes), _i32, _vp, _vp]),
    "pq_sampler_plan_create": (_i32, [_i32, _vp, _i64, ctypes.POINTER(_vp)]),
    "pq_sampler_plan_run": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "pq_sampler_plan_destroy": (_i32, [_vp]),
    "pq_hafnian_repeated": (_i32, [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "pq_loop_hafnian_repeated": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "pq_hafnian_plan_create": (_i32, [_vp, _vp, _vp, _vp, _i64, _i32, ctypes.POINTER(_vp)]),
    "pq_hafnian_plan_run": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "pq_hafnian_plan_destroy": (_i32, [_vp]),
    "pq_plan_item_info": (_i32, [_i32, _i32, _vp, _vp, _i32, _vp]),
    "pq_gray_walk": (_i32, [_vp, _i32, _i64, _vp, _vp]),
    "pq_fixsum_host": (_i32, [_vp, _vp, _i32, _vp]),
    "pq_fixsum_device": (_i32, [_vp, _vp, _i32, _vp, _vp]),
    "pq_loop_poly_factors": (_i32, [_i32, _vp]),
    "pq_combine_partials": (_i32, [_vp, _i32, _i64, _vp, _vp, _vp]),
    "pq_combine_partials_host": (_i32, [_vp, _i32, _i64, _vp, _vp]),
    "pq_tune_table_get": (_i32, [_vp]),
    "pq_tune_table_set": (_i32, [_vp]),
    "pq_tune_cache_save": (_i32, [ctypes.c_char_p, ctypes.c_char_p]),
    "pq_tune_cache_load": (_i32, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(_i32)]),
    "pq_plan_device_error": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64), _i32]),
    "pq_debug_fail_allocation": (_i32, [_i64]),
    "pq_debug_live_allocations": (_i32, [ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "pq_debug_corrupt_plan": (_i32, [_vp, _i32]),
    "pq_last_error": (ctypes.c_char_p, []),
    "pq_version": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def load_library(path: str | None = None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing "
                               "(run paper_2403_04006_gb300.build.build())")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class PQError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} returned {code}: {msg}")
        self.code = code


def _check(rc: int, where: str):
    if rc != PQ_OK:
        msg = load_library().pq_last_error().decode(errors="replace")
        raise PQError(rc, where, msg)


# --------------------------------------------------------------------------
# raw entry points (same names as the C ABI)
# --------------------------------------------------------------------------
def pq_plan_create(sizes: pq_batch_sizes, opts: pq_plan_options | None = None) -> int:
    out = _vp()
    _check(load_library().pq_plan_create(ctypes.byref(sizes),
                                         ctypes.byref(opts) if opts else None,
                                         ctypes.byref(out)), "pq_plan_create")
    return out.value


def pq_partition_batch(sizes: pq_batch_sizes, ranks: int) -> tuple[np.ndarray, np.ndarray]:
    """(rank of every item, Gray-code terms per rank) of the balanced split."""
    rank_of = np.zeros(max(int(sizes.batch), 0), dtype=np.int32)
    terms = np.zeros(max(int(ranks), 0), dtype=np.int64)
    _check(load_library().pq_partition_batch(ctypes.byref(sizes), int(ranks),
                                             rank_of.ctypes.data if rank_of.size else None,
                                             terms.ctypes.data if terms.size else None),
           "pq_partition_batch")
    return rank_of, terms


def pq_plan_create_bs(m: int, input_occ: np.ndarray, output_occ: np.ndarray, B: int,
                      opts: pq_plan_options | None = None) -> int:
    out = _vp()
    _check(load_library().pq_plan_create_bs(m, input_occ.ctypes.data, output_occ.ctypes.data, B,
                                            ctypes.byref(opts) if opts else None,
                                            ctypes.byref(out)), "pq_plan_create_bs")
    return out.value


def pq_plan_destroy(plan: int):
    _check(load_library().pq_plan_destroy(plan), "pq_plan_destroy")


def pq_permanent_batched(b: pq_batch, out_ptr: int, plan: int | None, stream: int | None):
    _check(load_library().pq_permanent_batched(ctypes.byref(b), out_ptr, plan, stream),
           "pq_permanent_batched")


def pq_permanent_partials(b: pq_batch, partials_ptr: int, plan: int, stream: int | None):
    _check(load_library().pq_permanent_partials(ctypes.byref(b), partials_ptr, plan, stream),
           "pq_permanent_partials")


def pq_bs_probs(U_ptr, m, in_ptr, out_ptr, B, probs_ptr, amps_ptr, plan, stream):
    _check(load_library().pq_bs_probs(U_ptr, m, in_ptr, out_ptr, B, probs_ptr, amps_ptr, plan,
                                      stream), "pq_bs_probs")


def pq_permanent_backward(b: pq_batch, grad_out_ptr, grad_mats_ptr, plan, stream):
    _check(load_library().pq_permanent_backward(ctypes.byref(b), grad_out_ptr, grad_mats_ptr,
                                                plan, stream), "pq_permanent_backward")


def pq_bs_probs_backward(U_ptr, m, in_ptr, out_ptr, B, grad_probs_ptr, amps_ptr, grad_U_ptr,
                         plan, stream):
    _check(load_library().pq_bs_probs_backward(U_ptr, m, in_ptr, out_ptr, B, grad_probs_ptr,
                                               amps_ptr, grad_U_ptr, plan, stream),
           "pq_bs_probs_backward")


def pq_clements_forward(theta_ptr, phi_ptr, m, U_ptr, stream):
    _check(load_library().pq_clements_forward(theta_ptr, phi_ptr, m, U_ptr, stream),
           "pq_clements_forward")


def pq_clements_backward(theta_ptr, phi_ptr, m, U_ptr, gU_ptr, gtheta_ptr, gphi_ptr, stream):
    _check(load_library().pq_clements_backward(theta_ptr, phi_ptr, m, U_ptr, gU_ptr, gtheta_ptr,
                                               gphi_ptr, stream), "pq_clements_backward")


def pq_autotune(plan: int, b: pq_batch | None, U_ptr, stream):
    _check(load_library().pq_autotune(plan, ctypes.byref(b) if b is not None else None, U_ptr,
                                      stream), "pq_autotune")


def pq_plan_get_stats(plan: int) -> pq_plan_stats:
    s = pq_plan_stats()
    _check(load_library().pq_plan_get_stats(plan, ctypes.byref(s)), "pq_plan_get_stats")
    return s


def pq_probe_fp64_peak(iters: int, stream=None) -> tuple[float, float]:
    f = ctypes.c_double()
    ms = ctypes.c_double()
    _check(load_library().pq_probe_fp64_peak(iters, ctypes.byref(f), ctypes.byref(ms), stream),
           "pq_probe_fp64_peak")
    return f.value, ms.value


def pq_probe_fp64_sweep(op: int, warps_per_sm: int, chains: int, iters: int,
                        stream=None) -> float:
    """Lane operations per second per SM of op (0 DFMA, 1 DADD, 2 DMUL)."""
    r = ctypes.c_double()
    _check(load_library().pq_probe_fp64_sweep(op, warps_per_sm, chains, iters, ctypes.byref(r),
                                              stream), "pq_probe_fp64_sweep")
    return r.value


def pq_permanent_noalloc(B_ptr, k: int, l: int, row_mult: np.ndarray, col_mult: np.ndarray,
                         out_ptr, stream):
    """Permanent of one base matrix with no device allocation (static device
    workspace shared by all calls; serialise calls).  row_mult / col_mult are
    host int32 arrays."""
    r = np.ascontiguousarray(row_mult, dtype=np.int32)
    c = np.ascontiguousarray(col_mult, dtype=np.int32)
    _check(load_library().pq_permanent_noalloc(B_ptr, k, l, r.ctypes.data if r.size else None,
                                               c.ctypes.data if c.size else None, out_ptr,
                                               stream), "pq_permanent_noalloc")


def pq_bs_sample(U_ptr, m: int, input_occ: np.ndarray, col_order: np.ndarray,
                 uniforms: np.ndarray, stream) -> np.ndarray:
    """Algorithm A samples; col_order (nsamples x n int32) and uniforms
    (nsamples x n float64) are host arrays.  Returns nsamples x m occupations."""
    s = np.ascontiguousarray(input_occ, dtype=np.int32)
    co = np.ascontiguousarray(col_order, dtype=np.int32)
    un = np.ascontiguousarray(uniforms, dtype=np.float64)
    ns = co.shape[0]
    out = np.zeros((ns, m), dtype=np.int32)
    _check(load_library().pq_bs_sample(U_ptr, m, s.ctypes.data, ns,
                                       co.ctypes.data if co.size else None,
                                       un.ctypes.data if un.size else None,
                                       out.ctypes.data if out.size else None, stream),
           "pq_bs_sample")
    return out


def pq_hafnian_repeated(mats_ptr, mat_off: np.ndarray, k: np.ndarray, rep: np.ndarray,
                        rep_off: np.ndarray, out_ptr, stream, gamma_ptr=None, loop: bool = False):
    """Hafnians (or, with ``loop``, loop hafnians with loop weights at
    ``gamma_ptr``) of bases repeated by ``rep``; mat_off / k / rep / rep_off
    are host arrays, mats, gamma and out device pointers."""
    mo = np.ascontiguousarray(mat_off, dtype=np.int64)
    kk = np.ascontiguousarray(k, dtype=np.int32)
    r = np.ascontiguousarray(rep, dtype=np.int32)
    ro = np.ascontiguousarray(rep_off, dtype=np.int64)
    nb = kk.shape[0]
    lib = load_library()
    args = (mo.ctypes.data if nb else None, kk.ctypes.data if nb else None,
            r.ctypes.data if r.size else (kk.ctypes.data if nb else None),
            ro.ctypes.data if nb else None, nb, out_ptr, stream)
    if loop:
        _check(lib.pq_loop_hafnian_repeated(mats_ptr, gamma_ptr, *args),
               "pq_loop_hafnian_repeated")
    else:
        _check(lib.pq_hafnian_repeated(mats_ptr, *args), "pq_hafnian_repeated")


def pq_hafnian_plan_create(mat_off, k, rep, rep_off, loop: bool) -> int:
    """Plan a (loop) hafnian batch from host sizes and repetitions; returns the handle."""
    mo = np.ascontiguousarray(mat_off, dtype=np.int64)
    kk = np.ascontiguousarray(k, dtype=np.int32)
    r = np.ascontiguousarray(rep, dtype=np.int32)
    ro = np.ascontiguousarray(rep_off, dtype=np.int64)
    nb = kk.shape[0]
    h = _vp()
    _check(load_library().pq_hafnian_plan_create(
        mo.ctypes.data if nb else None, kk.ctypes.data if nb else None,
        r.ctypes.data if r.size else (kk.ctypes.data if nb else None),
        ro.ctypes.data if nb else None, nb, 1 if loop else 0, ctypes.byref(h)),
        "pq_hafnian_plan_create")
    return h.value


def pq_hafnian_plan_run(plan: int, mats_ptr, gamma_ptr, out_ptr, stream):
    _check(load_library().pq_hafnian_plan_run(plan, mats_ptr, gamma_ptr, out_ptr, stream),
           "pq_hafnian_plan_run")


def pq_hafnian_plan_destroy(plan: int):
    _check(load_library().pq_hafnian_plan_destroy(plan), "pq_hafnian_plan_destroy")


def pq_loop_poly_factors(N: int) -> np.ndarray:
    """Host-only: the factors of the loop-hafnian polynomial of size N."""
    out = np.zeros(N // 2 + 1)
    _check(load_library().pq_loop_poly_factors(N, out.ctypes.data), "pq_loop_poly_factors")
    return out


def pq_bs_probs_lossy(V_ptr, eta_ptr, W_ptr, m: int, input_occ: np.ndarray,
                      output_occ: np.ndarray, probs_ptr, stream):
    s = np.ascontiguousarray(input_occ, dtype=np.int32)
    t = np.ascontiguousarray(output_occ, dtype=np.int32).reshape(-1, m)
    _check(load_library().pq_bs_probs_lossy(V_ptr, eta_ptr, W_ptr, m, s.ctypes.data, t.ctypes.data,
                                            t.shape[0], probs_ptr, stream), "pq_bs_probs_lossy")


def pq_combine_partials(parts_ptr, nshards: int, batch: int, n_ptr, out_ptr, stream):
    """Device pointers: parts (nshards x batch x 4 doubles), n (int32), out (complex)."""
    _check(load_library().pq_combine_partials(parts_ptr, nshards, batch, n_ptr, out_ptr, stream),
           "pq_combine_partials")


def pq_combine_partials_host(parts: np.ndarray, n: np.ndarray) -> np.ndarray:
    """Host arrays: parts (nshards, batch, 4) float64, n (batch,) int; returns
    the complex permanents."""
    p = np.ascontiguousarray(parts, dtype=np.float64)
    if p.ndim != 3 or p.shape[2] != 4:
        raise ValueError("parts must have shape (nshards, batch, 4)")
    nn = np.ascontiguousarray(n, dtype=np.int32)
    batch = p.shape[1]
    if nn.shape != (batch,):
        raise ValueError("n must have one entry per permanent")
    out = np.zeros(batch, dtype=np.complex128)
    _check(load_library().pq_combine_partials_host(p.ctypes.data if p.size else None, p.shape[0],
                                                   batch, nn.ctypes.data if nn.size else None,
                                                   out.ctypes.data if out.size else None),
           "pq_combine_partials_host")
    return out


def pq_tune_table_get() -> np.ndarray:
    t = np.zeros(PQ_MAX_N + 1, dtype=np.int32)
    _check(load_library().pq_tune_table_get(t.ctypes.data), "pq_tune_table_get")
    return t


def pq_tune_table_set(table) -> None:
    t = np.ascontiguousarray(table, dtype=np.int32)
    if t.shape != (PQ_MAX_N + 1,):
        raise ValueError(f"the tuning table has {PQ_MAX_N + 1} entries")
    _check(load_library().pq_tune_table_set(t.ctypes.data), "pq_tune_table_set")


def pq_tune_cache_save(path: str, device_key: str | None = None) -> None:
    _check(load_library().pq_tune_cache_save(os.fsencode(path),
                                             None if device_key is None else device_key.encode()),
           "pq_tune_cache_save")


def pq_tune_cache_load(path: str, device_key: str | None = None) -> bool:
    found = _i32()
    _check(load_library().pq_tune_cache_load(os.fsencode(path),
                                             None if device_key is None else device_key.encode(),
                                             ctypes.byref(found)), "pq_tune_cache_load")
    return bool(found.value)


def pq_plan_device_error(plan: int, clear: bool = False) -> tuple[int, int]:
    code, task = _i32(), _i64()
    _check(load_library().pq_plan_device_error(plan, ctypes.byref(code), ctypes.byref(task),
                                               1 if clear else 0), "pq_plan_device_error")
    return code.value, task.value


def pq_debug_fail_allocation(after: int) -> None:
    _check(load_library().pq_debug_fail_allocation(after), "pq_debug_fail_allocation")


def pq_debug_live_allocations() -> tuple[int, int]:
    d, h = _i64(), _i64()
    _check(load_library().pq_debug_live_allocations(ctypes.byref(d), ctypes.byref(h)),
           "pq_debug_live_allocations")
    return d.value, h.value


def pq_debug_corrupt_plan(plan: int, what: int) -> None:
    _check(load_library().pq_debug_corrupt_plan(plan, what), "pq_debug_corrupt_plan")


def pq_lossy_plan_create(m: int, input_occ, output_occ) -> int:
    """Plan lossy probabilities for host occupations; returns the handle."""
    s = np.ascontiguousarray(input_occ, dtype=np.int32)
    t = np.ascontiguousarray(output_occ, dtype=np.int32).reshape(-1, m)
    h = _vp()
    _check(load_library().pq_lossy_plan_create(m, s.ctypes.data, t.ctypes.data if t.size else None,
                                               t.shape[0], ctypes.byref(h)),
           "pq_lossy_plan_create")
    return h.value


def pq_lossy_plan_run(plan: int, V_ptr, eta_ptr, W_ptr, probs_ptr, stream):
    _check(load_library().pq_lossy_plan_run(plan, V_ptr, eta_ptr, W_ptr, probs_ptr, stream),
           "pq_lossy_plan_run")


def pq_lossy_plan_destroy(plan: int):
    _check(load_library().pq_lossy_plan_destroy(plan), "pq_lossy_plan_destroy")


def pq_sampler_plan_create(m: int, input_occ, nsamples: int) -> int:
    """Plan nsamples Algorithm A draws per run for a host input occupation."""
    s = np.ascontiguousarray(input_occ, dtype=np.int32)
    h = _vp()
    _check(load_library().pq_sampler_plan_create(m, s.ctypes.data, nsamples, ctypes.byref(h)),
           "pq_sampler_plan_create")
    return h.value


def pq_sampler_plan_run(plan: int, U_ptr, m: int, col_order: np.ndarray, uniforms: np.ndarray,
                        stream) -> np.ndarray:
    """One planned run; col_order and uniforms are host arrays (nsamples x n).
    Returns nsamples x m occupations."""
    co = np.ascontiguousarray(col_order, dtype=np.int32)
    un = np.ascontiguousarray(uniforms, dtype=np.float64)
    out = np.zeros((co.shape[0], m), dtype=np.int32)
    _check(load_library().pq_sampler_plan_run(plan, U_ptr, co.ctypes.data if co.size else None,
                                              un.ctypes.data if un.size else None,
                                              out.ctypes.data if out.size else None, stream),
           "pq_sampler_plan_run")
    return out


def pq_sampler_plan_destroy(plan: int):
    _check(load_library().pq_sampler_plan_destroy(plan), "pq_sampler_plan_destroy")


def pq_version() -> str:
    return load_library().pq_version().decode()


def pq_last_error() -> str:
    return load_library().pq_last_error().decode()
