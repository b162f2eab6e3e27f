"""Build and run the instruction-rate microbenchmarks.

instruction_rates.cu measures, with register-only loops on every SM, the
throughput of LOP3 and of the legacy warp-level tensor instructions mma.sync
s8, b1 (and.popc) and f16; mma_rates.cu measures the tcgen05.mma issue rate
(FP8 and block-scaled FP4 kinds, M = 128, several N) with operands resident in
shared memory.  These rates decide which instruction each form of the GF(2)
slice GEMM is built on and bound what its kernels can reach.
Usage: python paper_1111_6900_gb300/microbench/run.py
"""
import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    rc = 0
    with tempfile.TemporaryDirectory() as tmp:
        for name in ("instruction_rates", "mma_rates"):
            exe = os.path.join(tmp, name)
            subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                            os.path.join(HERE, name + ".cu"), "-o", exe], check=True)
            rc |= subprocess.run([exe]).returncode
    return rc


if __name__ == "__main__":
    sys.exit(main())
