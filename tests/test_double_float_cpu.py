"""The double-float arithmetic of the recursions (df64: hi + lo of two
floats, from Knuth's two-sum, Dekker's fast two-sum and the FMA two-product),
compiled for the host from the device header and checked against its error
bounds, 2^-48 scale per operation (tests/df_check.cpp).  Contraction is off,
as in the device build's round-to-nearest intrinsics.  No GPU needed."""
import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2411_03416_b300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


def test_double_float_error_bounds():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "df_check")
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-I", CSRC, "-I", CUDA_INC,
                               os.path.join(HERE, "df_check.cpp"), "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
