"""NVTX ranges over the library's stages: a small search run with a recording NVTX
tool (tests/host/nvtx_recorder.c, loaded by the NVTX calls through
NVTX_INJECTION64_PATH) sees the preparation, search, demodulation and transform
ranges, in that order."""
import os
import shutil
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, %r)
import numpy as np, torch
from paper_1003_0844_gb300 import build, fstat as fs, workloads as W
build.build()
wl = W.WORKLOADS["tiny"]
x = torch.as_tensor(np.random.default_rng(3).standard_normal(wl.n).astype(np.float32), device="cuda")
alpha, delta = (torch.as_tensor(v, device="cuda") for v in W.sky_grid(2))
f1 = torch.as_tensor(W.spin_grid(2, *wl.f1_range), device="cuda")
ctx = fs.Context(W.detector_for(wl))
seg = fs.Segment(ctx, x, wl.dt, wl.nfft, wl.fl, wl.S0)
fs.search(ctx, seg, alpha, delta, f1, wl.F_thr)
torch.cuda.synchronize()
assert ctx.sync_status() == 0
print("done")
"""


def _cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    return inc if os.path.exists(os.path.join(inc, "nvtx3", "nvToolsExt.h")) else None


def test_stages_are_nvtx_ranges(tmp_path):
    gcc, inc = shutil.which("gcc"), _cuda_include()
    if gcc is None or inc is None:
        pytest.skip("gcc or the NVTX headers are missing")
    tool = str(tmp_path / "libnvtxrec.so")
    r = subprocess.run([gcc, "-shared", "-fPIC", "-O2", "-I", inc, os.path.join(ROOT, "tests", "host", "nvtx_recorder.c"),
                        "-o", tool], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    rec = tmp_path / "ranges.txt"
    env = dict(os.environ, NVTX_INJECTION64_PATH=tool, NVTX_RECORD_FILE=str(rec))
    r = subprocess.run([sys.executable, "-c", SCRIPT % ROOT], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0 and "done" in r.stdout, r.stderr[-3000:]
    names = [ln for ln in rec.read_text().splitlines() if ln.startswith("fs.")]
    assert names[:4] == ["fs.prepare", "fs.search", "fs.demodulate", "fs.transform"], names
