"""Compile and run the host<->device bandwidth probe (csrc/probe/c2c_peak.cu).

Prints copy-engine rates (1, 2 and 4 streams per direction, each direction
alone and both at once) and SM rates (a kernel loading and storing pinned
host memory through its device mapping): the ceilings of a staged copy
pipeline and of a kernel working on host buffers directly.

    python -m paper_1305_4376_gb300.c2c_peak
"""
import os
import subprocess
import sys

from paper_1305_4376_gb300.build import ARCH, BUILD, nvcc

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "c2c_peak")
    src = os.path.join(HERE, "csrc", "probe", "c2c_peak.cu")
    subprocess.run([nvcc()] + ARCH + ["-O3", "-o", exe, src], check=True)
    return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
