"""Write the stored expected values under tests/golden/ from the CPU oracle.

Only the oracle computes anything here (plus the seeded input generator for
the input matrix itself).  Run from the repository root:

    python tests/golden/make_golden.py [--threads N]

single_large_n30.txt
    Workload "single large permanent": the top-left 30 x 30 block of the seeded
    Haar 60 x 60 unitary, no repetitions.  The input matrix is stored too
    (hex floats), so the value does not depend on the LAPACK build that
    generated it; a test checks that the generator still reproduces it.
    The expected permanent comes from the oracle's gold mode (Ryser's formula,
    Sec. 4.2's comparison variant, with column sums, products and accumulation
    in double-double), whose a-posteriori bound is stored alongside.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2403_04006_gb300 import workloads as W  # noqa: E402


def write_matrix_file(path, A, per, bound, per_fast, bound_fast, note, seconds):
    n = A.shape[0]
    with open(path, "w") as f:
        f.write(f"# {note}\n")
        f.write("# written by tests/golden/make_golden.py (CPU oracle, gold mode)\n")
        f.write(f"# oracle seconds: {seconds:.1f}\n")
        f.write(f"n {n}\n")
        for i in range(n):
            for j in range(n):
                z = A[i, j]
                f.write(f"{float(z.real).hex()} {float(z.imag).hex()}\n")
        f.write(f"per_gold {per.real.hex()} {per.imag.hex()}\n")
        f.write(f"bound_gold {bound.hex()}\n")
        f.write(f"per_fast {per_fast.real.hex()} {per_fast.imag.hex()}\n")
        f.write(f"bound_fast {bound_fast.hex()}\n")


def read_matrix_file(path):
    """(A, {key: value}) from a file written by write_matrix_file."""
    vals = {}
    rows = []
    n = None
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "n":
                n = int(parts[1])
            elif parts[0] in ("per_gold", "per_fast"):
                vals[parts[0]] = complex(float.fromhex(parts[1]), float.fromhex(parts[2]))
            elif parts[0] in ("bound_gold", "bound_fast"):
                vals[parts[0]] = float.fromhex(parts[1])
            else:
                rows.append(complex(float.fromhex(parts[0]), float.fromhex(parts[1])))
    A = np.array(rows, dtype=np.complex128).reshape(n, n)
    return A, vals


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=O.default_threads())
    args = ap.parse_args()
    A = W.single_large(30)
    t0 = time.time()
    per_f, _, bound_f = O.perm_ryser(A, gold=False, nthreads=args.threads, info=True)
    t1 = time.time()
    per_g, _, bound_g = O.perm_ryser(A, gold=True, nthreads=args.threads, info=True)
    t2 = time.time()
    note = ("single large permanent: top-left 30x30 block of the seeded Haar 60x60 unitary "
            "(workloads.single_large), r = c = 1; paper Sec. 4.2 / Eq. (per_def)")
    write_matrix_file(os.path.join(HERE, "single_large_n30.txt"), A, per_g, bound_g, per_f,
                      bound_f, note, t2 - t1)
    print(f"fast {per_f} bound {bound_f:.3e} ({t1 - t0:.1f} s)")
    print(f"gold {per_g} bound {bound_g:.3e} ({t2 - t1:.1f} s)")
    print(f"|fast - gold| / |gold| = {abs(per_f - per_g) / abs(per_g):.3e}")


if __name__ == "__main__":
    main()
