"""The unit counts behind the roofline denominators, measured on the GPU:
population counts (the XU pipe) at 16 lanes per clock per SM and LOP3 / IMAD
at 64, as the CUDA throughput table for compute capability 10.x gives them.
bench.py's popcount roofline divides by 152 SMs x 16 x the maximum clock, so a
device whose rates differ fails here rather than reporting a wrong fraction.
Run with -s to see the measured rates."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_integer_unit_rates(tmp_path):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    exe = tmp_path / "unit_rates"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", str(exe),
                    os.path.join(HERE, "unit_rates", "unit_rates.cu")], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True, timeout=300).stdout
    print(out)
    rates = {}
    for line in out.splitlines():
        parts = line.split()
        if len(parts) == 3 and parts[0] != "device":
            rates[parts[0]] = float(parts[1])
    assert rates["POPC"] == pytest.approx(16.0, rel=0.03)
    assert rates["LOP3"] == pytest.approx(64.0, rel=0.03)
    assert rates["IMAD"] == pytest.approx(64.0, rel=0.03)
    # POPC and LOP3 issue to different pipes: together they exceed either alone
    assert rates["POPC+LOP3"] > 1.5 * rates["POPC"]
