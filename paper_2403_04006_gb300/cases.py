"""Single entry-point runs on the seeded workloads, for timing and profiling.

    python -m paper_2403_04006_gb300.cases hafnian --k 16 [--reps 3] [--loop]
    python -m paper_2403_04006_gb300.cases backward --count 4096 [--reps 3]

Each case uploads its inputs once, runs the call ``--reps`` times on one
stream and prints the per-call times (CUDA events) as one JSON line.  The
runs are small enough to sit under a profiler.
"""
from __future__ import annotations

import argparse
import json


def hafnian_case(k: int, loop: bool, reps: int):
    import torch

    from . import api
    from . import workloads as W

    dev = torch.device("cuda", 0)
    B, r, g = W.paper_repeated_hafnian(k, loop=loop)
    Bd = torch.from_numpy(B.reshape(-1)).to(dev)
    gd = torch.from_numpy(g).to(dev) if loop else None
    stream = torch.cuda.Stream(device=dev)
    ms = []
    val = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        val = api.hafnian_repeated(Bd, [0], [k], r, [0], gamma=gd, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    terms = 2 * 3 ** (k - 1)
    return {"case": "loop_hafnian" if loop else "hafnian", "k": k, "N": 2 * k, "terms": terms,
            "ms": ms, "terms_per_s": terms / min(ms) * 1e3, "value": [val[0].real.item(),
                                                                      val[0].imag.item()]}


def backward_case(count: int, reps: int):
    import torch

    from . import api
    from . import workloads as W

    dev = torch.device("cuda", 0)
    pb = W.ragged(count=count)
    db = api.DeviceBatch(pb, dev)
    plan = api.Plan.for_batch(pb, method="batched")
    gout = torch.ones(pb.batch, dtype=torch.complex128, device=dev)
    stream = torch.cuda.Stream(device=dev)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        api.permanent_backward(db, gout, plan, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    st = plan.stats()
    return {"case": "backward", "permanents": count, "terms": st["terms"], "ms": ms,
            "terms_per_s": st["terms"] / min(ms) * 1e3,
            "fp64_instr_backward": st["fp64_instr_backward"],
            "launches": st["launches_backward"]}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("case", choices=["hafnian", "backward"])
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--loop", action="store_true")
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    if a.case == "hafnian":
        print(json.dumps(hafnian_case(a.k, a.loop, a.reps)), flush=True)
    else:
        print(json.dumps(backward_case(a.count, a.reps)), flush=True)


if __name__ == "__main__":
    main()
