"""Build and run the instruction-rate microbenchmark (instruction_rates.cu).

Measures, with register-only loops on every SM, the throughput of LOP3 and
of the legacy warp-level tensor instructions mma.sync s8, b1 (and.popc) and
f16 on the current GPU.  These rates decide which instruction each form of
the GF(2) slice GEMM is built on.  Usage: python paper_1111_6900_gb300/microbench/run.py
"""
import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "instruction_rates")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                        os.path.join(HERE, "instruction_rates.cu"), "-o", exe], check=True)
        return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
