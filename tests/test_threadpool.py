"""The host worker pool shared by the tessellation tiles, the batch's
simulations and the server's lanes (csrc/threadpool.h), checked on the CPU:
concurrent callers with priorities, nested calls and tasks of very
different lengths; every task runs exactly once and every call returns
only after its own tasks are done."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_pool_concurrent_callers(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not found")
    exe = str(tmp_path / "threadpool_check")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-pthread", os.path.join(HERE, "threadpool_check.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
