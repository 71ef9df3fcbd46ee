"""The fine search's double-float arithmetic, compiled as host code: the table-and-series
exp(-2 pi i f), the per-point constants against central differences, and the per-sample
sums of F, its gradient and its Hessian (Eqs. OS and Fab and their derivatives) over a
2-day, 2 s series against the same sums in FP64."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_double_float_fine_search_sums_match_fp64(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "refine_check")
    # no contraction on the host: the double-float steps rely on the roundings they write
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-Xcompiler", "-ffp-contract=off",
                        "-x", "cu", os.path.join(HERE, "host", "refine_check.cu"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout
