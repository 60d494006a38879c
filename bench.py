"""Benchmark of the permanent path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one graph-captured persistent forward over the ragged batch of
65536 permanents (n ~ U{4..20}, row/column multiplicities with parts in
{1,2,3}, each a submatrix of its own Haar unitary of size 2n), with the
batch resident in HBM and L2 flushed before every step.  The metric is
Gray-code terms per second (every permanent counts the exact number of terms
of the side its Gray code sums); permanents/s, the plain one-launch-per-
permanent path on the same batch, the single n = 30 permanent, the batched
boson-sampling workload and the Clements-mesh forward+backward workload are
reported in the same JSON line under "extra".

``--impl reference`` times the CPU oracle (Ryser's formula in FP64 with
double-double accumulation, all host cores) on the same batch (by default the
whole of it, a few seconds per step on 16 host cores) and prints the same line
with "impl": "reference".

Under torchrun (N > 1) the job evaluates a batch of N x 65536 permanents
split over the ranks: rank r evaluates block r of it (block 0 is the batch
above, the others the same recipe from their own seed streams), on its own
GPU, with no collective on the data path (weak scaling: 65536 permanents per
GPU).  Rank 0 prints the line with the terms of all blocks over the slowest
rank's time.

Profiling cases (``--workload``; same JSON line, smaller or different work,
never the benchmark figure): ``ragged4096`` and ``single30`` run the same
forward on a 4096-permanent batch of the recipe or the n = 30 permanent;
``ragged-backward`` and ``ragged4096-backward`` time the backward (one launch
per product-column class and the scatter) on the benchmark batch or the
4096-permanent batch; ``hafnian-2x`` and
``loop-hafnian-2x`` time the repeated (loop) hafnian of a k x k GBS matrix
with every index repeated twice (``--k``); ``gradient-m16`` times the
Clements mesh (m = 16) -> 1024 boson-sampling probabilities -> sum ->
backward through both; ``fp64-sweep`` measures the FP64
pipe (DFMA, DADD, DMUL) against resident warps per SM and independent chains
per thread.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gray-code terms/sec & permanents/sec (FP64 roofline %), batched vs plain, 1 GB300"
UNIT = "terms/s"
WORKLOAD = ("ragged batch: 65536 permanents, n ~ U{4..20}, row/col multiplicities with parts "
            "in {1,2,3}, submatrices of per-item Haar 2n x 2n unitaries (seed 1004)")
FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64, NVIDIA's figure
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "glynn_fwd_persistent_ragged65536.md")
KERNEL_SOURCES = ["paper_2403_04006_gb300/csrc/glynn_fwd.cu",
                  "paper_2403_04006_gb300/csrc/pq_fixsum.cuh",
                  "paper_2403_04006_gb300/csrc/pq_device.cuh",
                  "paper_2403_04006_gb300/csrc/pq_internal.h"]


# ---------------------------------------------------------------- distributed helpers
def rank_env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init_dist(backend: str):
    import torch.distributed as dist
    rank, world, _ = rank_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return rank, world


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units all ranks processed (each the same count) divided by the slowest
    rank's time."""
    return units_per_rank * world / seconds_max


def sum_over_ranks(x: float, device=None) -> float:
    """The sum of x over the ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampled every 100 ms while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"pq_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the persistent forward kernel from the
    committed ncu summary, if it was taken on the current kernel source."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    text = open(PROFILE_SUMMARY).read()
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    b = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not m or not b or m.group(1) != kernel_hash():
        return None
    return float(b.group(1))


PROFILE_CASES = ("ragged-backward", "ragged4096-backward", "bs-m24", "hafnian-2x", "loop-hafnian-2x",
                 "gradient-m16", "fp64-sweep")


def load_workload(name: str, block: int = 0):
    """(PermBatch, description).  'ragged' is the benchmark workload (block
    ``block`` of it under torchrun); the others are smaller cases of the same
    kernel for profiling."""
    from paper_2403_04006_gb300 import workloads as W
    if name == "ragged":
        if block == 0:
            return W.ragged(), WORKLOAD
        return W.ragged(block=block), WORKLOAD + f", block {block} (own seed streams)"
    if name == "ragged-backward":
        return W.ragged(), WORKLOAD + ", backward (profiling case)"
    if name in ("ragged4096", "ragged4096-backward"):
        return W.ragged(count=4096), "ragged recipe with 4096 permanents (profiling case)"
    if name == "single30":
        A = W.single_large(30)
        return (W.pack_batch([(A, [1] * 30, [1] * 30)]),
                "single permanent n = 30, top-left block of a Haar 60 x 60 (seed 1002)")
    raise ValueError(f"unknown workload {name}")


def bench_config(desc: str, permanents: int, terms: int, world: int, split: bool = False) -> dict:
    """The workload the line measures; both arms print this same object."""
    if world == 1:
        par = "1 GPU"
    elif split:
        par = (f"{world} ranks, one batch of {permanents} permanents split by whole permanents "
               "with balanced work (pq_partition_batch), outputs all-gathered in every timed step")
    else:
        par = (f"{world} ranks, block r of a batch of {world} x {permanents // world} "
               "permanents on rank r, no collective on the data path")
    return {"workload": desc, "permanents": permanents, "terms": terms,
            "parallelism": par,
            "l2": "GPU arm: flushed (256 MB write) before every timed step; "
                  "CPU arm: inputs in host memory"}


def max_sm_clock_mhz(gpu_index: int) -> float:
    try:
        out = subprocess.run(["nvidia-smi", f"--id={gpu_index}", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=20)
        return float(out.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return 2070.0  # GB300 maximum SM clock


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


ARM_PARTS = {"0xd0c": "Neoverse N1", "0xd40": "Neoverse V1", "0xd49": "Neoverse N2",
             "0xd4f": "Neoverse V2", "0xd8e": "Neoverse N3", "0xd84": "Neoverse V3"}


def cpu_model() -> str:
    """The host CPU's model name, or for Arm cores the name of their part number."""
    part = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":", 1)[0].strip().lower()
            if key == "model name":
                return line.split(":", 1)[1].strip()
            if key == "cpu part" and part is None:
                part = line.split(":", 1)[1].strip().lower()
    except OSError:
        pass
    if part is not None:
        return f"Arm {ARM_PARTS.get(part, 'part ' + part)}"
    return "unknown"


def oracle_sample(pb, target_ryser_terms: float):
    """Items of the batch taken with a fixed stride until the oracle's Ryser
    term count reaches the target: a bounded, representative sample."""
    order = list(range(0, pb.batch, 7)) + [b for b in range(pb.batch) if b % 7]
    picked, tot = [], 0.0
    for b in order:
        r = pb.row_mult[pb.row_off[b]:pb.row_off[b] + pb.k[b]]
        tot += float(np.prod(r.astype(np.float64) + 1.0))
        picked.append(b)
        if tot >= target_ryser_terms:
            break
    return sorted(picked)


def glynn_terms(pb, idx) -> int:
    """Gray-code terms of the cheaper side of each item (the count the GPU sums)."""
    def side(m):
        m = [int(x) for x in m if x > 0]
        if not m:
            return 0
        f = int(np.argmin(m))
        return math.prod(x if i == f else x + 1 for i, x in enumerate(m))
    tot = 0
    for b in idx:
        r = pb.row_mult[pb.row_off[b]:pb.row_off[b] + pb.k[b]]
        c = pb.col_mult[pb.col_off[b]:pb.col_off[b] + pb.l[b]]
        tot += min(side(r), side(c))
    return tot


def run_oracle_sample(pb, idx, threads):
    import oracle as O
    sub = pb.subset(idx)
    t0 = time.perf_counter()
    O.perm_batch(sub.mats, sub.mat_off, sub.k, sub.l, sub.row_mult, sub.row_off, sub.col_mult,
                 sub.col_off, gold=False, nthreads=threads)
    return time.perf_counter() - t0


# ---------------------------------------------------------------- our arm
def bench_ours(args):
    import torch

    from paper_2403_04006_gb300 import api, pq
    from paper_2403_04006_gb300 import workloads as W

    rank, world, local = rank_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    init_dist("nccl")
    pq.load_library()

    if args.workload in PROFILE_CASES:
        return bench_case(args, dev)
    split = args.split and world > 1
    if split:
        # strong scaling: one batch, each rank its share of whole permanents
        full, workload_desc = load_workload(args.workload, block=0)
        rank_of, _ = api.partition_batch(full, world)
        pb = full.subset(np.nonzero(rank_of == rank)[0])
    else:
        pb, workload_desc = load_workload(args.workload, block=rank)
    db = api.DeviceBatch(pb, dev)
    plan = api.Plan.for_batch(pb, method="batched", use_graph=True, chunk_log2=args.chunk_log2)
    if not args.no_autotune and args.chunk_log2 == 0:
        plan.autotune(db)
    st = plan.stats()
    out = torch.empty(pb.batch, dtype=torch.complex128, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    def step():
        api.permanent_batched(db, plan, out=out, stream=stream)
        if split:  # every rank ends the step with the whole batch's outputs
            api.gather_partitioned(out, rank_of)

    # FP64 peak: 2 lane-operations per clock per SM (the pipe the path loads),
    # and the DFMA-chain probe measured in this run beside it
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clock_mhz = max_sm_clock_mhz(local)
    peak_tflops = sms * clock_mhz * 1e6 * 2 * 2 / 1e12
    peak_flops, _ = api.probe_fp64_peak(1 << 16, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            step()
    stream.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(dev)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        t_wall0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed_region")  # lets a profiler select these launches
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.fill_(1.0)  # L2 flush, outside the events
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
        stream.synchronize()
        torch.cuda.nvtx.range_pop()
        t_wall = time.perf_counter() - t_wall0
        barrier(dev)
        torch.cuda.synchronize(dev)
    clk = clocks.summary()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_mean = sum(step_ms) / len(step_ms)
    ms_max = max_over_ranks(ms_mean, dev)
    # every rank holds its own block: the job's units are the sum over ranks
    job_terms = sum_over_ranks(st["terms"], dev)
    job_perms = sum_over_ranks(st["permanents"], dev)
    value = job_terms / (ms_max * 1e-3)
    perms_per_s = job_perms / (ms_max * 1e-3)
    achieved_tflops = st["flops_forward"] / (ms_mean * 1e-3) / 1e12

    # ---- end to end through the C ABI with host buffers
    host = {k: torch.from_numpy(getattr(pb, k)).pin_memory()
            for k in ("mats", "mat_off", "k", "l", "row_mult", "row_off", "col_mult", "col_off")}
    out_host = torch.empty(full.batch if split else pb.batch,
                           dtype=torch.complex128).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = out_host.numel() * out_host.element_size()

    def e2e_step():
        with torch.cuda.stream(stream):
            for k, t in host.items():
                getattr(db, k).copy_(t, non_blocking=True)
            api.permanent_batched(db, plan, out=out, stream=stream)
            res = api.gather_partitioned(out, rank_of) if split else out
            out_host.copy_(res, non_blocking=True)
        stream.synchronize()

    for _ in range(2):
        e2e_step()
    e2e_times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_step()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e_times) / len(e2e_times), dev)
    e2e_value = job_terms / e2e_s

    extra = {}
    if rank == 0 and not args.quick:
        extra = extra_measurements(args, dev, stream, flush, peak_tflops,
                                   2.0 * sms * clock_mhz * 1e6)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = host_cores()
        idx = oracle_sample(pb, args.cpu_sample_terms)
        # repeat the sample until about 10 s of host time have been measured
        runs, secs = 0, 0.0
        while runs < 8 and (runs == 0 or secs < 10.0):
            secs += run_oracle_sample(pb, idx, threads)
            runs += 1
        per = secs / runs
        cpu = {"value": glynn_terms(pb, idx) / per, "unit": UNIT, "cores": threads,
               "kind": "oracle",
               "sample": f"{len(idx)} of {pb.batch} permanents (stride-7 order), {runs} run(s), "
                         f"{per:.2f} s each, Ryser FP64 + double-double accumulation, "
                         f"{cpu_model()}"}

    traffic = profiled_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "strong" if split else "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": bench_config(WORKLOAD if args.workload == "ragged" else workload_desc,
                               int(job_perms), int(job_terms), world, split),
        "method": "batched persistent kernel, CUDA graph, " + (
            f"chunks of about 2^{args.chunk_log2} terms" if args.chunk_log2 else
            "default chunks" if args.no_autotune else "autotuned chunks"),
        "permanents_per_s": perms_per_s,
        "roofline": {"bound": "alu", "achieved": achieved_tflops,
                     "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved_tflops / peak_tflops, "traffic": traffic,
                     "peak_source": f"derived: {sms} SMs x {clock_mhz:.0f} MHz x 2 FP64 lane-ops "
                                    "per clock per SM x 2 flop (FMA)",
                     "peak_probe_measured": peak_flops / 1e12,
                     "frac_of_probe": achieved_tflops / (peak_flops / 1e12),
                     "fp64_pipe_frac": st["fp64_instr_forward"] / (ms_mean * 1e-3)
                                       / (2.0 * sms * clock_mhz * 1e6),
                     "fp64_pipe_frac_executed": st["fp64_instr_forward_executed"]
                                                / (ms_mean * 1e-3) / (2.0 * sms * clock_mhz * 1e6),
                     "flops_per_step": st["flops_forward"],
                     "fp64_instr_per_step": st["fp64_instr_forward"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * int(st["launches_forward"]),
        "clocks": clk,
        "wall_s_timed_region": t_wall,
        "cpu_baseline": cpu,
        "extra": extra,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def extra_measurements(args, dev, stream, flush, peak_tflops, fp64_lane_ops):
    """Secondary numbers of the same path, one JSON object each."""
    import torch

    from paper_2403_04006_gb300 import api
    from paper_2403_04006_gb300 import workloads as W

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        with torch.cuda.stream(stream):
            fn()
            for _ in range(reps):
                flush.fill_(1.0)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    res = {}
    # plain path on the same ragged batch
    pb = W.ragged()
    db = api.DeviceBatch(pb, dev)
    plan_p = api.Plan.for_batch(pb, method="plain")
    out = torch.empty(pb.batch, dtype=torch.complex128, device=dev)
    st = plan_p.stats()
    ms = timed(lambda: api.permanent_batched(db, plan_p, out=out, stream=stream), 3)
    res["ragged_plain"] = {"terms_per_s": st["terms"] / ms * 1e3,
                           "permanents_per_s": st["permanents"] / ms * 1e3, "ms": ms,
                           "launches": st["launches_forward"]}
    plan_b = api.Plan.for_batch(pb, method="batched")
    gout = torch.ones(pb.batch, dtype=torch.complex128, device=dev)

    def bwd_entry(plan, ms):
        # stats after the first backward call, which plans the backward;
        # the algorithmic flop count includes a k x l rank-1 update per term
        # that the kernel's correction scheme avoids, so it can exceed the
        # peak: the FP64-instruction fraction is the roofline figure
        st_ = plan.stats()
        return {"terms_per_s": st_["terms"] / ms * 1e3, "ms": ms,
                "fp64_pipe_frac": st_["fp64_instr_backward"] / (ms * 1e-3) / fp64_lane_ops,
                "fp64_instr": st_["fp64_instr_backward"],
                "tflops_algorithmic": st_["flops_backward"] / ms / 1e9,
                "launches": st_["launches_backward"]}

    ms = timed(lambda: api.permanent_backward(db, gout, plan_b, stream=stream), 3)
    res["ragged_backward_batched"] = bwd_entry(plan_b, ms)
    plan_pb = api.Plan.for_batch(pb, method="plain")
    ms = timed(lambda: api.permanent_backward(db, gout, plan_pb, stream=stream), 1)
    res["ragged_backward_plain"] = bwd_entry(plan_pb, ms)
    del plan_pb
    del db, plan_p, plan_b
    # single n = 30
    A = W.single_large(30)
    pb30 = W.pack_batch([(A, [1] * 30, [1] * 30)])
    db30 = api.DeviceBatch(pb30, dev)
    plan30 = api.Plan.for_batch(pb30)
    out30 = torch.empty(1, dtype=torch.complex128, device=dev)
    st = plan30.stats()
    ms = timed(lambda: api.permanent_batched(db30, plan30, out=out30, stream=stream), 3)
    res["single_n30"] = {"terms_per_s": st["terms"] / ms * 1e3, "ms": ms,
                         "tflops": st["flops_forward"] / ms / 1e9,
                         "frac": st["flops_forward"] / ms / 1e9 / peak_tflops}
    # the paper's repeated-permanent benchmark shape (Sec. 4.2, Fig. permanent):
    # k x k Haar block, every row and column repeated twice, one launch each
    sweep = {}
    for k in range(4, 17):
        B, r, c = W.paper_repeated(k)
        pbk = W.pack_batch([(B, r, c)])
        dbk = api.DeviceBatch(pbk, dev)
        plank = api.Plan.for_batch(pbk, method="plain")
        outk = torch.empty(1, dtype=torch.complex128, device=dev)
        stk = plank.stats()
        ms = timed(lambda: api.permanent_batched(dbk, plank, out=outk, stream=stream), 5)
        sweep[str(k)] = {"ms": ms, "terms": stk["terms"], "terms_per_s": stk["terms"] / ms * 1e3}
    res["paper_repeated_2x"] = sweep
    # the paper's repeated hafnian / loop hafnian benchmark shape (Figs.
    # hafnian, loop_hafnian): k x k GBS matrix, every index repeated twice
    # (N = 2k); one synchronous call each (planning and upload included), and
    # the launch of a plan made once
    for loop in (False, True):
        hs = {}
        for k in range(4, 21, 2):
            B, r, g = W.paper_repeated_hafnian(k, loop=loop)
            Bd = torch.from_numpy(B.reshape(-1)).to(dev)
            gd = torch.from_numpy(g).to(dev) if loop else None
            terms = 2 * 3 ** (k - 1)
            ms = timed(lambda: api.hafnian_repeated(Bd, [0], [k], r, [0], gamma=gd,
                                                    stream=stream), 3)
            # the same through a plan made once: the launch alone
            hplan = api.HafnianPlan([0], [k], r, [0], loop=loop)
            hout = torch.empty(1, dtype=torch.complex128, device=dev)
            ms_p = timed(lambda: hplan.run(Bd, gamma=gd, out=hout, stream=stream), 3)
            hplan.close()
            hs[str(k)] = {"N": 2 * k, "ms": ms, "terms": terms, "terms_per_s": terms / ms * 1e3,
                          "ms_planned": ms_p, "terms_per_s_planned": terms / ms_p * 1e3}
        res["paper_loop_hafnian_2x" if loop else "paper_hafnian_2x"] = hs
    # Algorithm A sampler (one batched launch per photon over all samples),
    # m = 16 Haar interferometer, 8 photons, 2000 samples
    Us = torch.from_numpy(W.haar_unitary(16, W.rng_for(7))).to(dev)
    s8 = np.zeros(16, dtype=np.int32)
    s8[:8] = 1
    order, unif = W.sampler_draws(2000, 8, 1007)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    api.bs_sample(Us, s8, order, unif)
    secs = time.perf_counter() - t0
    # the same draws through a plan made once: each run is the upload, the
    # 8 steps' launches and the read-back
    splan = api.SamplerPlan(16, s8, 2000)
    splan.run(Us, order, unif)
    t0 = time.perf_counter()
    for _ in range(5):
        splan.run(Us, order, unif)
    secs_p = (time.perf_counter() - t0) / 5
    splan.close()
    res["sampler_m16_n8"] = {"samples": 2000, "s": secs, "samples_per_s": 2000 / secs,
                             "s_planned": secs_p, "samples_per_s_planned": 2000 / secs_p}
    # a larger sampler run: m = 40 Haar, 20 photons in modes 0..19, 100 samples
    # (the last steps evaluate 20 minors of size 19, 2^18 terms each, per sample)
    U40 = torch.from_numpy(W.haar_unitary(40, W.rng_for(7, 1))).to(dev)
    s20 = np.zeros(40, dtype=np.int32)
    s20[:20] = 1
    order20, unif20 = W.sampler_draws(100, 20, 1008)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    api.bs_sample(U40, s20, order20, unif20)
    secs = time.perf_counter() - t0
    splan = api.SamplerPlan(40, s20, 100)
    splan.run(U40, order20, unif20)
    t0 = time.perf_counter()
    splan.run(U40, order20, unif20)
    secs_p = time.perf_counter() - t0
    splan.close()
    res["sampler_m40_n20"] = {"samples": 100, "s": secs, "samples_per_s": 100 / secs,
                              "s_planned": secs_p, "samples_per_s_planned": 100 / secs_p}
    # lossy boson sampling (Sec. 3.2.4): m = 10 Haar factors V, W, transmissions
    # eta ~ U[0.5, 0.95], 5 photons in modes 0..4, every output pattern with at
    # most 5 photons (3003 patterns, 42504 permanents of the 20-mode dilation);
    # one synchronous call, planning included
    rl = W.rng_for(10)
    Vl, Wl = W.haar_unitary(10, rl), W.haar_unitary(10, rl)
    etal = rl.uniform(0.5, 0.95, 10)
    sl = np.zeros(10, dtype=np.int32)
    sl[:5] = 1
    tl = np.concatenate([W.compositions(k, 10) for k in range(6)])
    Vd, Wd, etad = (torch.from_numpy(x).to(dev) for x in (Vl, Wl, etal))
    ms = timed(lambda: api.bs_probs_lossy(Vd, etad, Wd, sl, tl, stream=stream), 3)
    lplan = api.LossyPlan(10, sl, tl)  # the same, planned once: each run is three launches
    ms_p = timed(lambda: lplan.run(Vd, etad, Wd, stream=stream), 5)
    lplan.close()
    res["lossy_m10_n5"] = {"patterns": int(tl.shape[0]), "permanents": 42504, "ms": ms,
                           "patterns_per_s": tl.shape[0] / ms * 1e3, "ms_planned": ms_p,
                           "patterns_per_s_planned": tl.shape[0] / ms_p * 1e3}
    # batched boson sampling, m = 24, 4096 patterns
    U, s, t = W.bs_batched()
    Ud, sd, td = (torch.from_numpy(x).to(dev) for x in (U, s, t))
    for method in ("batched", "plain"):
        plan = api.Plan.for_bs(24, s, t, method=method, use_graph=(method == "batched"))
        st = plan.stats()
        ms = timed(lambda: api.bs_probs(Ud, sd, td, plan, stream=stream), 10)
        res[f"bs_m24_{method}"] = {"terms_per_s": st["terms"] / ms * 1e3,
                                   "permanents_per_s": st["permanents"] / ms * 1e3, "ms": ms}
    # Clements mesh -> probabilities -> sum -> backward, m = 16, 1024 patterns
    th, ph, s5, t5 = W.gradient_workload()
    thd = torch.from_numpy(th).to(dev).requires_grad_(True)
    phd = torch.from_numpy(ph).to(dev).requires_grad_(True)
    sd5, td5 = torch.from_numpy(s5).to(dev), torch.from_numpy(t5).to(dev)
    plan5 = api.Plan.for_bs(16, s5, t5)

    def step5():
        U5 = api.ClementsMesh.apply(thd, phd, 16)
        api.BSProbs.apply(U5, sd5, td5, plan5).sum().backward()

    ms = timed(step5, 10)
    res["gradient_m16"] = {"ms_fwd_bwd": ms, "terms": plan5.stats()["terms"]}
    return res


def bench_case(args, dev):
    """One profiling case (PROFILE_CASES): time the operation over --steps
    launches (L2 flushed before each, CUDA events on the launching stream)
    and print a JSON line for it."""
    import torch

    from paper_2403_04006_gb300 import api
    from paper_2403_04006_gb300 import workloads as W

    stream = torch.cuda.Stream(device=dev)
    if args.workload == "fp64-sweep":
        from paper_2403_04006_gb300 import pq
        hz = max_sm_clock_mhz(dev.index) * 1e6
        table = {}
        for op, name in enumerate(("DFMA", "DADD", "DMUL")):
            for w in (1, 2, 4, 8, 16, 32, 64):
                table[f"{name} {w} warps/SM"] = {
                    f"ch{c}": round(pq.pq_probe_fp64_sweep(op, w, c, 1 << 14, stream.cuda_stream)
                                    / hz, 3) for c in (1, 2, 4, 8)}
        print(json.dumps({"profiling_case": "fp64-sweep",
                          "unit": "lane operations per clock per SM at the maximum SM clock",
                          "sm_max_mhz": hz / 1e6, "table": table}), flush=True)
        return
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    extra = {}
    if args.workload in ("ragged-backward", "ragged4096-backward"):
        pb, desc = load_workload(args.workload)
        db = api.DeviceBatch(pb, dev)
        plan = api.Plan.for_batch(pb, method="batched")
        gout = torch.ones(pb.batch, dtype=torch.complex128, device=dev)

        def op():
            api.permanent_backward(db, gout, plan, stream=stream)
        terms_of = lambda: plan.stats()["terms"]  # noqa: E731
        if args.workload == "ragged4096-backward":
            desc = desc.replace("(profiling case)", "backward (profiling case)")
    elif args.workload == "bs-m24":
        U3, s3, t3 = W.bs_batched()
        Ud3, sd3, td3 = (torch.from_numpy(x).to(dev) for x in (U3, s3, t3))
        plan3 = api.Plan.for_bs(24, s3, t3, use_graph=True)

        def op():
            api.bs_probs(Ud3, sd3, td3, plan3, stream=stream)
        terms_of = lambda: plan3.stats()["terms"]  # noqa: E731
        extra = {"column_sums": plan3.stats()["column_sums"]}
        desc = ("boson sampling m = 24, 12 photons in modes 0..11, 4096 output patterns, "
                "batched plan (profiling case)")
    elif args.workload == "gradient-m16":
        th, ph, s5, t5 = W.gradient_workload()
        thd = torch.from_numpy(th).to(dev).requires_grad_(True)
        phd = torch.from_numpy(ph).to(dev).requires_grad_(True)
        sd5, td5 = torch.from_numpy(s5).to(dev), torch.from_numpy(t5).to(dev)
        plan5 = api.Plan.for_bs(16, s5, t5)

        def op():
            U5 = api.ClementsMesh.apply(thd, phd, 16)
            api.BSProbs.apply(U5, sd5, td5, plan5).sum().backward()
        terms_of = lambda: plan5.stats()["terms"]  # noqa: E731
        desc = ("Clements mesh m = 16 (120 beamsplitters) -> probabilities of 1024 patterns with "
                "8 photons -> sum -> backward (profiling case)")
    else:
        loop = args.workload.startswith("loop")
        B, r, g = W.paper_repeated_hafnian(args.k, loop=loop)
        Bd = torch.from_numpy(B.reshape(-1)).to(dev)
        gd = torch.from_numpy(g).to(dev) if loop else None
        hplan = api.HafnianPlan([0], [args.k], r, [0], loop=loop)
        hout = torch.empty(1, dtype=torch.complex128, device=dev)

        def op():
            hplan.run(Bd, gamma=gd, out=hout, stream=stream)
        terms_of = lambda: 2 * 3 ** (args.k - 1)  # noqa: E731
        desc = (f"{'loop ' if loop else ''}hafnian of a {args.k} x {args.k} GBS matrix, every "
                f"index repeated twice (N = {2 * args.k}; profiling case)")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            op()
    stream.synchronize()
    ms = []
    torch.cuda.nvtx.range_push("timed_region")
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            e0.record(stream)
            op()
            e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    torch.cuda.nvtx.range_pop()
    if args.workload in ("ragged-backward", "ragged4096-backward"):
        st = plan.stats()
        extra = {"fp64_instr_backward": st["fp64_instr_backward"],
                 "launches": st["launches_backward"]}
    mean = sum(ms) / len(ms)
    terms = terms_of()
    print(json.dumps({
        "metric": METRIC, "value": terms / (mean * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "profiling_case": args.workload,
        "config": {"workload": desc, "terms": terms,
                   "l2": "flushed (256 MB write) before every timed step"},
        "ms_per_launch_set": ms, "extra": extra}), flush=True)


# ---------------------------------------------------------------- reference arm
def bench_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return  # the CPU oracle runs once, on rank 0
    from paper_2403_04006_gb300 import workloads as W
    import oracle as O
    O.build()
    pb = W.ragged()
    threads = host_cores()
    idx = oracle_sample(pb, args.cpu_sample_terms)
    terms = glynn_terms(pb, idx)
    # the job the GPU arm measures: blocks 0 .. world-1, or with --split block 0
    # alone (the oracle times block 0)
    job_terms = glynn_terms(pb, range(pb.batch))
    for blk in range(1, 1 if args.split else world):
        bs = W.ragged(block=blk, sizes_only=True)
        job_terms += glynn_terms(bs, range(bs.batch))
    for _ in range(args.warmup):
        run_oracle_sample(pb, idx[: max(1, len(idx) // 8)], threads)
    secs = [run_oracle_sample(pb, idx, threads) for _ in range(args.steps)]
    per = sum(secs) / len(secs)
    value = terms / per
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "strong" if args.split and world > 1 else "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": bench_config(WORKLOAD, pb.batch * (1 if args.split else world),
                               int(job_terms), world, args.split),
        "method": "CPU oracle: Ryser FP64 + double-double accumulation, all host cores",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{len(idx)} of {pb.batch} permanents per step "
                                   f"({terms} Gray-code terms), Ryser FP64 + double-double "
                                   f"accumulation, {cpu_model()}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quick", action="store_true", help="skip the extra measurements")
    ap.add_argument("--workload", choices=["ragged", "ragged4096", "single30", *PROFILE_CASES],
                    default="ragged", help="ragged is the benchmark; the others are profiling cases")
    ap.add_argument("--no-autotune", action="store_true",
                    help="plan with the built-in chunk lengths instead of timing candidates first")
    ap.add_argument("--chunk-log2", type=int, default=0,
                    help="plan every permanent with chunks of about 2^K terms (0: per class)")
    ap.add_argument("--k", type=int, default=18,
                    help="hafnian profiling cases: base size k (N = 2k)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--split", action="store_true",
                    help="with N > 1: split one batch over the ranks by whole permanents and "
                         "all-gather the outputs (strong scaling) instead of one block per rank")
    ap.add_argument("--cpu-sample-terms", type=float, default=math.inf,
                    help="Ryser terms of the oracle sample (default: the whole batch, "
                         "about 2-3 s on 16 host cores; repeated to about 10 s)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
