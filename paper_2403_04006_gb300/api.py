"""Torch-facing API over the C ABI: device batches, plans and autograd
Functions.  Tensors only carry device memory and streams; every step of the
permanent path runs in the CUDA library (no CPU fallback)."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import pq as _pq
from .workloads import PermBatch


def _stream_handle(stream: torch.cuda.Stream | None = None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


_SUMS = {"auto": _pq.PQ_SUMS_AUTO, "shared": _pq.PQ_SUMS_SHARED,
         "registers": _pq.PQ_SUMS_REGISTERS}


def _opts(method: str, use_graph: bool, chunk_log2: int, warps_per_block: int = 0,
          blocks_per_sm: int = 0, shard: tuple[int, int] | None = None,
          column_sums: str = "auto") -> _pq.pq_plan_options:
    o = _pq.pq_plan_options()
    o.column_sums = _SUMS[column_sums]
    o.method = {"batched": _pq.PQ_METHOD_BATCHED, "plain": _pq.PQ_METHOD_PLAIN}[method]
    o.use_graph = 1 if use_graph else 0
    o.chunk_log2 = int(chunk_log2)
    o.warps_per_block = int(warps_per_block)
    o.blocks_per_sm = int(blocks_per_sm)
    if shard is not None:
        o.shard_index, o.shard_count = int(shard[0]), int(shard[1])
    return o


class DeviceBatch:
    """A ragged batch of base matrices resident on the GPU, plus the host
    copy of its sizes that planning needs."""

    def __init__(self, pb: PermBatch, device: str | torch.device = "cuda",
                 mats: torch.Tensor | None = None):
        self.host = pb
        dev = torch.device(device)
        self.mats = (mats if mats is not None
                     else torch.from_numpy(pb.mats).to(dev))
        self.mat_off = torch.from_numpy(pb.mat_off).to(dev)
        self.k = torch.from_numpy(pb.k).to(dev)
        self.l = torch.from_numpy(pb.l).to(dev)
        self.row_mult = torch.from_numpy(pb.row_mult).to(dev)
        self.row_off = torch.from_numpy(pb.row_off).to(dev)
        self.col_mult = torch.from_numpy(pb.col_mult).to(dev)
        self.col_off = torch.from_numpy(pb.col_off).to(dev)

    @property
    def batch(self) -> int:
        return self.host.batch

    def c_struct(self, mats: torch.Tensor | None = None) -> _pq.pq_batch:
        m = self.mats if mats is None else mats
        b = _pq.pq_batch()
        b.batch = self.batch
        b.mats = _ptr(m) if m.numel() else None
        for f in ("mat_off", "k", "l", "row_mult", "row_off", "col_mult", "col_off"):
            t = getattr(self, f)
            setattr(b, f, _ptr(t) if t.numel() else None)
        return b

    def sizes_struct(self):
        h = self.host
        keep = [np.ascontiguousarray(x) for x in
                (h.mat_off, h.k, h.l, h.row_mult, h.row_off, h.col_mult, h.col_off)]
        s = _pq.pq_batch_sizes()
        s.batch = h.batch
        s.mat_off, s.k, s.l, s.row_mult, s.row_off, s.col_mult, s.col_off = [
            x.ctypes.data if x.size else None for x in keep]
        return s, keep


class Plan:
    """Owns a pq_plan (host schedule + device workspace)."""

    def __init__(self, handle: int, kind: str):
        self.handle = handle
        self.kind = kind

    @classmethod
    def for_batch(cls, pb: PermBatch | DeviceBatch, method: str = "batched",
                  use_graph: bool = False, chunk_log2: int = 0, warps_per_block: int = 0,
                  blocks_per_sm: int = 0, shard: tuple[int, int] | None = None,
                  column_sums: str = "auto") -> "Plan":
        """Plan a ragged batch; ``shard=(index, count)`` makes a plan for one
        shard of every permanent's warp tasks (see ``permanent_partials``);
        ``column_sums`` is "auto", "shared" or "registers" (PQ_SUMS_*)."""
        db = pb if isinstance(pb, DeviceBatch) else None
        host = db.host if db is not None else pb
        keep = [np.ascontiguousarray(x) for x in
                (host.mat_off, host.k, host.l, host.row_mult, host.row_off, host.col_mult,
                 host.col_off)]
        s = _pq.pq_batch_sizes()
        s.batch = host.batch
        s.mat_off, s.k, s.l, s.row_mult, s.row_off, s.col_mult, s.col_off = [
            x.ctypes.data if x.size else None for x in keep]
        h = _pq.pq_plan_create(s, _opts(method, use_graph, chunk_log2, warps_per_block,
                                        blocks_per_sm, shard, column_sums))
        return cls(h, "batch")

    @classmethod
    def for_bs(cls, m: int, s, t, method: str = "batched", use_graph: bool = False,
               chunk_log2: int = 0, warps_per_block: int = 0, blocks_per_sm: int = 0,
               shard: tuple[int, int] | None = None, column_sums: str = "auto") -> "Plan":
        s = np.ascontiguousarray(np.asarray(s, dtype=np.int32))
        t = np.ascontiguousarray(np.asarray(t, dtype=np.int32).reshape(-1, m))
        h = _pq.pq_plan_create_bs(int(m), s, t, int(t.shape[0]),
                                  _opts(method, use_graph, chunk_log2, warps_per_block,
                                        blocks_per_sm, shard, column_sums))
        return cls(h, "bs")

    def stats(self) -> dict:
        st = _pq.pq_plan_get_stats(self.handle)
        d = {f: getattr(st, f) for f, _ in _pq.pq_plan_stats._fields_}
        d["column_sums"] = {v: k for k, v in _SUMS.items()}[d["column_sums"]]
        return d

    def autotune(self, db: DeviceBatch | None = None, U: torch.Tensor | None = None,
                 stream=None):
        b = db.c_struct() if db is not None else None
        _pq.pq_autotune(self.handle, b, _ptr(U), _stream_handle(stream))

    def close(self):
        if self.handle:
            _pq.pq_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# functional API
# --------------------------------------------------------------------------
def permanent_batched(db: DeviceBatch, plan: Plan | None = None, out: torch.Tensor | None = None,
                      mats: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    dev = db.mats.device
    if out is None:
        out = torch.empty(db.batch, dtype=torch.complex128, device=dev)
    _pq.pq_permanent_batched(db.c_struct(mats), _ptr(out) if db.batch else None,
                             plan.handle if plan else None, _stream_handle(stream))
    return out


def permanent_partials(db: DeviceBatch, plan: Plan, out: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
    """This shard's unscaled double-double sums, a (batch, 4) float64 tensor
    (re hi, re lo, im hi, im lo) on the batch's device; ``plan`` must be made
    with ``shard=(index, count)``."""
    if out is None:
        out = torch.empty((db.batch, 4), dtype=torch.float64, device=db.mats.device)
    _pq.pq_permanent_partials(db.c_struct(), _ptr(out) if db.batch else None, plan.handle,
                              _stream_handle(stream))
    return out


def combine_partials(parts, n) -> np.ndarray:
    """Permanents from the shards' partial sums (host arrays of shape
    (batch, 4), in shard order) and each permanent's photon number ``n``:
    the library adds them in double-double and scales by 2^{-(n-1)}
    (pq_combine_partials_host)."""
    stacked = np.stack([np.asarray(p, dtype=np.float64) for p in parts])
    return _pq.pq_combine_partials_host(stacked, np.asarray(n))


def combine_partials_device(parts: torch.Tensor, n: torch.Tensor, out: torch.Tensor | None = None,
                            stream=None) -> torch.Tensor:
    """The same on the GPU (pq_combine_partials): ``parts`` a (nshards,
    batch, 4) float64 CUDA tensor, ``n`` an int32 CUDA tensor of photon
    numbers; returns the complex128 permanents on the same device."""
    parts = parts.contiguous()
    n32 = n.to(torch.int32).contiguous()
    batch = parts.shape[1]
    if out is None:
        out = torch.empty(batch, dtype=torch.complex128, device=parts.device)
    _pq.pq_combine_partials(_ptr(parts) if batch else None, parts.shape[0], batch,
                            _ptr(n32) if batch else None, _ptr(out) if batch else None,
                            _stream_handle(stream))
    return out


def gather_partials(local: torch.Tensor, group=None) -> list:
    """Every shard's partials, in rank order, on every rank (one all_gather of
    32 bytes per permanent: the exchange step of a split permanent), as a
    list of tensors on the device of ``local`` when the backend is NCCL, on
    the CPU otherwise.  Without an initialised process group, this rank's
    partials alone."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [local]
    world = dist.get_world_size(group)
    t = local if dist.get_backend(group) == "nccl" else local.cpu()
    bufs = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(bufs, t.contiguous(), group=group)
    return bufs


def photon_numbers(pb: PermBatch) -> np.ndarray:
    """n of every permanent of a batch (the sum of its row multiplicities)."""
    return np.array([int(pb.row_mult[pb.row_off[b]:pb.row_off[b] + pb.k[b]].sum())
                     for b in range(pb.batch)], dtype=np.int32)


def permanent_distributed(db: DeviceBatch, plan: Plan, group=None, stream=None) -> torch.Tensor:
    """Permanents of a batch whose Gray codes are split over the ranks of a
    process group: each rank passes the plan of its shard (``shard=(rank,
    world)``, all planned under the same tuning table); every rank gets the
    complex permanents, combined by the library from the all-gathered
    partials (on the GPU with NCCL, on the host otherwise)."""
    part = permanent_partials(db, plan, stream=stream)
    parts = gather_partials(part, group)
    n = photon_numbers(db.host)
    if parts[0].is_cuda:
        return combine_partials_device(torch.stack(parts),
                                       torch.from_numpy(n).to(parts[0].device), stream=stream)
    return torch.from_numpy(combine_partials([p.numpy() for p in parts], n))


def partition_batch(pb: PermBatch, ranks: int) -> tuple[np.ndarray, np.ndarray]:
    """The library's balanced split of a batch over ``ranks`` ranks by whole
    permanents (pq_partition_batch): the rank of every item and the Gray-code
    terms of every rank.  Host only; every rank computes the same split."""
    keep = [np.ascontiguousarray(x) for x in
            (pb.mat_off, pb.k, pb.l, pb.row_mult, pb.row_off, pb.col_mult, pb.col_off)]
    s = _pq.pq_batch_sizes()
    s.batch = pb.batch
    s.mat_off, s.k, s.l, s.row_mult, s.row_off, s.col_mult, s.col_off = [
        x.ctypes.data if x.size else None for x in keep]
    return _pq.pq_partition_batch(s, ranks)


def gather_partitioned(local: torch.Tensor, rank_of: np.ndarray, group=None) -> torch.Tensor:
    """The outputs of a batch split by ``partition_batch``, in item order, on
    every rank: rank r holds the outputs of its items (ascending item index)
    in ``local``; one all_gather of equal-length padded buffers, no
    arithmetic.  The result lives on the device of ``local`` with NCCL, on
    the CPU otherwise.  Without an initialised process group ``local`` is the
    whole batch."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return local
    world = dist.get_world_size(group)
    counts = np.bincount(rank_of, minlength=world)
    t = local if dist.get_backend(group) == "nccl" else local.cpu()
    width = int(counts.max()) if counts.size else 0
    pad = torch.zeros(width, dtype=t.dtype, device=t.device)
    pad[:t.numel()] = t
    bufs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad, group=group)
    out = torch.empty(len(rank_of), dtype=t.dtype, device=t.device)
    for r in range(world):
        idx = torch.from_numpy(np.nonzero(rank_of == r)[0]).to(t.device)
        out[idx] = bufs[r][:int(counts[r])]
    return out


def permanent_partitioned(pb: PermBatch, device, group=None, use_graph: bool = False,
                          stream=None) -> torch.Tensor:
    """Permanents of a batch split over the ranks of a process group by whole
    permanents: this rank plans and evaluates its items of
    ``partition_batch(pb, world)`` and every rank gets all outputs in item
    order (``gather_partitioned``)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        rank, world = dist.get_rank(group), dist.get_world_size(group)
    else:
        rank, world = 0, 1
    rank_of, _ = partition_batch(pb, world)
    sub = pb.subset(np.nonzero(rank_of == rank)[0])
    db = DeviceBatch(sub, device)
    plan = Plan.for_batch(sub, use_graph=use_graph)
    local = permanent_batched(db, plan, stream=stream)
    if stream is not None:
        stream.synchronize()
    plan.close()
    return gather_partitioned(local, rank_of, group)


def permanent_backward(db: DeviceBatch, grad_out: torch.Tensor, plan: Plan | None = None,
                       mats: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    m = db.mats if mats is None else mats
    grad = torch.empty_like(m)
    go = grad_out.contiguous()  # held until the call returns
    _pq.pq_permanent_backward(db.c_struct(mats), _ptr(go), _ptr(grad),
                              plan.handle if plan else None, _stream_handle(stream))
    return grad


def bs_probs(U: torch.Tensor, s: torch.Tensor, t: torch.Tensor, plan: Plan | None = None,
             want_amps: bool = True, stream=None):
    m = U.shape[0]
    B = t.shape[0]
    probs = torch.empty(B, dtype=torch.float64, device=U.device)
    amps = torch.empty(B, dtype=torch.complex128, device=U.device) if want_amps else None
    _pq.pq_bs_probs(_ptr(U), m, _ptr(s), _ptr(t), B, _ptr(probs), _ptr(amps),
                    plan.handle if plan else None, _stream_handle(stream))
    return probs, amps


def bs_probs_backward(U, s, t, grad_probs, amps, plan: Plan | None = None, stream=None):
    m = U.shape[0]
    gU = torch.empty_like(U)
    gp = grad_probs.contiguous()  # held until the call returns
    _pq.pq_bs_probs_backward(_ptr(U), m, _ptr(s), _ptr(t), t.shape[0],
                             _ptr(gp), _ptr(amps), _ptr(gU),
                             plan.handle if plan else None, _stream_handle(stream))
    return gU


def clements_forward(theta: torch.Tensor, phi: torch.Tensor, m: int, stream=None):
    U = torch.empty((m, m), dtype=torch.complex128, device=theta.device)
    _pq.pq_clements_forward(_ptr(theta), _ptr(phi), m, _ptr(U), _stream_handle(stream))
    return U


def clements_backward(theta, phi, m, U, grad_U, stream=None):
    gt = torch.empty_like(theta)
    gp = torch.empty_like(phi)
    gUc = grad_U.contiguous()  # held until the call returns
    _pq.pq_clements_backward(_ptr(theta), _ptr(phi), m, _ptr(U), _ptr(gUc),
                             _ptr(gt), _ptr(gp), _stream_handle(stream))
    return gt, gp


# --------------------------------------------------------------------------
# autograd
# --------------------------------------------------------------------------
class Permanent(torch.autograd.Function):
    """per of every item of a ragged batch; ``mats`` is the packed complex128
    matrix tensor of the batch (differentiable)."""

    @staticmethod
    def forward(ctx, mats, db: DeviceBatch, plan: Plan | None):
        mats = mats.contiguous()
        ctx.db, ctx.plan = db, plan
        ctx.save_for_backward(mats)
        return permanent_batched(db, plan, mats=mats)

    @staticmethod
    def backward(ctx, grad_out):
        (mats,) = ctx.saved_tensors
        g = permanent_backward(ctx.db, grad_out.to(torch.complex128), ctx.plan, mats=mats)
        return g, None, None


class BSProbs(torch.autograd.Function):
    """Boson-sampling probabilities p(s, t_b) of Eq. (BS_prob) as a function of U."""

    @staticmethod
    def forward(ctx, U, s, t, plan: Plan | None):
        U = U.contiguous()
        probs, amps = bs_probs(U, s, t, plan)
        ctx.plan = plan
        ctx.save_for_backward(U, s, t, amps)
        return probs

    @staticmethod
    def backward(ctx, grad_probs):
        U, s, t, amps = ctx.saved_tensors
        gU = bs_probs_backward(U, s, t, grad_probs.to(torch.float64), amps, ctx.plan)
        return gU, None, None, None


class ClementsMesh(torch.autograd.Function):
    """U(theta, phi) of the Clements beamsplitter mesh."""

    @staticmethod
    def forward(ctx, theta, phi, m: int):
        theta = theta.contiguous()
        phi = phi.contiguous()
        U = clements_forward(theta, phi, m)
        ctx.m = m
        ctx.save_for_backward(theta, phi, U)
        return U

    @staticmethod
    def backward(ctx, grad_U):
        theta, phi, U = ctx.saved_tensors
        gt, gp = clements_backward(theta, phi, ctx.m, U, grad_U.to(torch.complex128))
        return gt, gp, None


def probe_fp64_peak(iters: int = 1 << 16, stream=None) -> tuple[float, float]:
    """Measured FP64 rate of this GPU (FLOP/s, FMA = 2) and the probe's ms."""
    return _pq.pq_probe_fp64_peak(iters, _stream_handle(stream))


def bs_probs_lossy(V: torch.Tensor, eta: torch.Tensor, W: torch.Tensor, s, t,
                   stream=None) -> torch.Tensor:
    """Detection probabilities of the lossy interferometer V diag(sqrt(eta)) W
    for input occupation s and output patterns t (host arrays, |t| <= n)."""
    t = np.atleast_2d(np.asarray(t, dtype=np.int32))
    m = V.shape[0]
    probs = torch.empty(t.shape[0], dtype=torch.float64, device=V.device)
    # Contiguous copies are bound to names so that none is freed (and its
    # block reused by the next copy) before the call reads it.
    Vc, etac, Wc = V.contiguous(), eta.contiguous(), W.contiguous()
    _pq.pq_bs_probs_lossy(_ptr(Vc), _ptr(etac), _ptr(Wc), m,
                          np.asarray(s), t, _ptr(probs), _stream_handle(stream))
    return probs


class LossyPlan:
    """Lossy detection probabilities of fixed patterns (pq_lossy_plan_*):
    planned once for input occupation ``s`` and output patterns ``t`` (host
    arrays), ``run`` evaluates them for an interferometer V diag(sqrt(eta)) W
    without host work, allocation or synchronisation."""

    def __init__(self, m: int, s, t):
        t = np.atleast_2d(np.asarray(t, dtype=np.int32))
        self.m, self.count = int(m), int(t.shape[0])
        self.handle = _pq.pq_lossy_plan_create(self.m, np.asarray(s), t)

    def run(self, V: torch.Tensor, eta: torch.Tensor, W: torch.Tensor,
            out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.count, dtype=torch.float64, device=V.device)
        Vc, etac, Wc = V.contiguous(), eta.contiguous(), W.contiguous()
        _pq.pq_lossy_plan_run(self.handle, _ptr(Vc), _ptr(etac), _ptr(Wc),
                              _ptr(out) if self.count else None, _stream_handle(stream))
        return out

    def close(self):
        if self.handle:
            _pq.pq_lossy_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bs_sample(U: torch.Tensor, s, col_order, uniforms, stream=None) -> np.ndarray:
    """Boson-sampling outputs by Algorithm A (pq_bs_sample): U on the GPU,
    input occupation s, and the run's random column orders and uniforms
    (host arrays, nsamples x n).  Returns nsamples x m occupations."""
    Uc = U.contiguous()
    return _pq.pq_bs_sample(_ptr(Uc), U.shape[0], np.asarray(s), col_order,
                            uniforms, _stream_handle(stream))


class SamplerPlan:
    """Algorithm A with the host work done once (pq_sampler_plan_*): planned
    for m modes, input occupation ``s`` and ``nsamples`` draws per run; ``run``
    takes U on the GPU and the run's column orders and uniforms (host arrays,
    nsamples x n) and returns nsamples x m occupations, the samples that
    ``bs_sample`` gives for the same arguments."""

    def __init__(self, m: int, s, nsamples: int):
        self.m, self.nsamples = int(m), int(nsamples)
        self.handle = _pq.pq_sampler_plan_create(self.m, np.asarray(s), self.nsamples)

    def run(self, U: torch.Tensor, col_order, uniforms, stream=None) -> np.ndarray:
        col_order = np.asarray(col_order, dtype=np.int32)
        uniforms = np.asarray(uniforms, dtype=np.float64)
        if col_order.shape[0] != self.nsamples or uniforms.shape != col_order.shape:
            raise ValueError("col_order and uniforms must be nsamples x n")
        Uc = U.contiguous()
        return _pq.pq_sampler_plan_run(self.handle, _ptr(Uc), self.m, col_order, uniforms,
                                       _stream_handle(stream))

    def close(self):
        if self.handle:
            _pq.pq_sampler_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hafnian_repeated(mats: torch.Tensor, mat_off, k, rep, rep_off, gamma: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    """Hafnians of symmetric bases with repeated indices (pq_hafnian_repeated),
    or loop hafnians with loop weights ``gamma`` (pq_loop_hafnian_repeated;
    packed like ``rep``): ``mats`` packed complex128 on the GPU, the offsets,
    sizes and repetitions host arrays.  Returns one complex128 per item."""
    mc = mats.contiguous()
    gc = None if gamma is None else gamma.contiguous()
    nb = len(k)
    out = torch.empty(nb, dtype=torch.complex128, device=mats.device)
    _pq.pq_hafnian_repeated(_ptr(mc), np.asarray(mat_off), np.asarray(k), np.asarray(rep),
                            np.asarray(rep_off), _ptr(out) if nb else None,
                            _stream_handle(stream), gamma_ptr=_ptr(gc), loop=gc is not None)
    return out


class HafnianPlan:
    """A planned batch of hafnians (or loop hafnians with ``loop=True``) of
    fixed sizes and repetitions (pq_hafnian_plan_*): ``run`` evaluates it for
    new matrix values (and loop weights) without planning, allocating in the
    library or synchronising."""

    def __init__(self, mat_off, k, rep, rep_off, loop: bool = False):
        self.batch = len(k)
        self.loop = bool(loop)
        self.handle = _pq.pq_hafnian_plan_create(np.asarray(mat_off), np.asarray(k),
                                                 np.asarray(rep), np.asarray(rep_off), loop)

    def run(self, mats: torch.Tensor, gamma: torch.Tensor | None = None,
            out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.batch, dtype=torch.complex128, device=mats.device)
        mc = mats.contiguous()
        gc = None if gamma is None else gamma.contiguous()
        _pq.pq_hafnian_plan_run(self.handle, _ptr(mc), _ptr(gc), _ptr(out) if self.batch else None,
                                _stream_handle(stream))
        return out

    def close(self):
        if self.handle:
            _pq.pq_hafnian_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
