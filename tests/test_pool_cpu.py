"""The server's pool allocator (first fit with coalescing), compiled for the
host from its header and exercised without a GPU."""
import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2411_03416_b300", "csrc")


def test_pool_allocator():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "pool_check")
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", CSRC, os.path.join(HERE, "pool_check.cpp"),
                               "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
