"""Build and run the integer-throughput probe (alu_peak.cu) on the current GPU.

Prints lane-operations per SM per clock for LOP3, IMAD, SHF, POPC, FFMA,
DP4A, SHFL and mixes: the unit counts behind the roofline of the walk kernel
(peak = SMs x lanes/clk x SM clock).
"""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "alu_peak")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                        os.path.join(HERE, "alu_peak.cu")], check=True)
        return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
