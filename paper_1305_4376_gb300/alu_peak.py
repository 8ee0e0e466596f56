"""Compile and run the integer-pipe throughput probe (csrc/probe/alu_peak.cu).

Prints LOP3, IMAD and mixed instruction rates per SM per clock; the LOP3 rate
times the SM count and the maximum SM clock is the ALU roofline peak of the
bitsliced kernel.

    python -m paper_1305_4376_gb300.alu_peak
"""
import os
import subprocess
import sys

from paper_1305_4376_gb300.build import ARCH, BUILD, nvcc

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "alu_peak")
    src = os.path.join(HERE, "csrc", "probe", "alu_peak.cu")
    subprocess.run([nvcc()] + ARCH + ["-O3", "-o", exe, src], check=True)
    return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
