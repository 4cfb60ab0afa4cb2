"""Build and run the pipe-throughput diagnostic (csrc/pipe_rates.cu): rates
of the FP64 operations the stage kernels use, and of FP32 FMA, on cuda:0.

  python -m paper_2603_26272_gb300.pipe_rates
"""
import os
import subprocess
import sys

from . import build as wbuild


def main():
    os.makedirs(wbuild.BUILD, exist_ok=True)
    exe = os.path.join(wbuild.BUILD, "pipe_rates")
    src = os.path.join(wbuild.CSRC, "pipe_rates.cu")
    subprocess.run([wbuild.nvcc(), "-O3", wbuild.ARCH, "-o", exe, src], check=True)
    sys.exit(subprocess.run([exe]).returncode)


if __name__ == "__main__":
    main()
