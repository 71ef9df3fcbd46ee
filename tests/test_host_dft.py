"""The register DFTs of the transform kernels, compiled as host code: the FMA-fused
decimation-in-time butterflies with zero-input and output pruning against a direct
double-precision DFT (Eq. eq:DFT), for every size and pruning the kernels use."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_register_dfts_match_direct_dft(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "dft_check")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-x", "cu",
                        os.path.join(HERE, "host", "dft_check.cu"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout
