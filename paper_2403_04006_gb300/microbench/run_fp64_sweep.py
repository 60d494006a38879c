"""Build and run the FP64 pipe sweep (``fp64_sweep.cu``) on the current GPU.

    python -m paper_2403_04006_gb300.microbench.run_fp64_sweep
"""
import os
import subprocess
import sys

from ..build import ARCH, nvcc

HERE = os.path.dirname(os.path.abspath(__file__))
EXE = os.path.join(os.path.dirname(HERE), "_build", "fp64_sweep")


def main() -> int:
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    subprocess.run([nvcc(), *ARCH, "-O3", "-o", EXE, os.path.join(HERE, "fp64_sweep.cu")],
                   check=True)
    return subprocess.run([EXE]).returncode


if __name__ == "__main__":
    sys.exit(main())
