"""Float-float arithmetic (csrc/df64.cuh) checked on the host: the
error-free transformations are exact, add / multiply / multiply-subtract
and the reciprocal square root stay within a few units of 2^-48, and a
Cholesky factorisation with inverse of Jacobi-scaled damped matrices gives
the single-precision inverse factors of an exact (long double) computation.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2602_08266_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "df64_host_check.cpp")


@pytest.fixture(scope="module")
def results():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "df64_check")
        subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-I", CSRC,
                        "-o", exe, SRC], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}


def test_error_free_transformations_are_exact(results):
    assert results["two_sum_inexact"] == 0
    assert results["fast_two_sum_inexact"] == 0
    assert results["two_prod_inexact"] == 0


def test_operations_near_df64_precision(results):
    assert results["add_rel_err_log2"] < -46
    assert results["mul_rel_err_log2"] < -45
    assert results["fms_rel_err_log2"] < -45
    assert results["rsqrt_rel_err_log2"] < -44


def test_factorisation_matches_exact_after_rounding(results):
    assert results["factor_equal_fraction"] > 0.999
    assert results["factor_worst_rel_row"] < 1e-7
    # the same comparison separates plain single precision clearly
    assert results["float_equal_fraction"] < 0.5
    assert results["float_worst_rel_row"] > 1e-6
