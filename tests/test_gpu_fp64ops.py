"""The sweep's refined FP64 reciprocal (three FMAs on the hardware's
approximate reciprocal) and its x / sqrt(x) square root, against the
IEEE-rounded 1/x and sqrt on the GPU: within one and two ulps over normal
arguments of every exponent, and the IEEE division itself outside the
refined range (zero, subnormals, the largest exponents, inf, NaN).  The
integer-pipe FP64 -> FP32 (round to nearest even) and FP32 -> FP64
conversions must equal the hardware's bit for bit."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _build(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "fp64ops_check")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                           os.path.join(HERE, "fp64ops_check.cu"), "-o", exe])
    return exe


def test_fp64ops_check_builds(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_fp64ops_within_ulps(tmp_path):
    exe = _build(tmp_path)
    out = subprocess.run([exe, str(1 << 22)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    f = out.stdout.split()
    assert f[0] == "recip" and f[3] == "sqrt" and f[6] == "d2f" and f[8] == "f2d", out.stdout
    assert int(f[7]) == 0 and int(f[9]) == 0, out.stdout
    r_ulp, r_bad, s_ulp, s_bad = float(f[1]), int(f[2]), float(f[4]), int(f[5])
    assert r_ulp <= 1.0, out.stdout
    assert r_bad == 0, out.stdout
    assert s_ulp <= 2.0, out.stdout
    assert s_bad == 0, out.stdout
