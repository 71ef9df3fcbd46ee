"""The debug build (-DFS_DEBUG): device bounds checks on every workspace and
output index of the transform kernels and guard words around the transform ring
and the queue counters.  A small search in the persistent launch (F up to
Nyquist), in the per-batch launches (F on all bins) and through the
allocation-free entry point runs clean with it: no check fires (FS_OK from
fs_sync_status, where a hit would read FS_ERR_CORRUPT), the guard entries the
caller places around its candidate buffer are untouched, and F equals the release
build's F."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import ctypes, json, sys
sys.path.insert(0, %(root)r)
import numpy as np, torch
from paper_1003_0844_gb300 import fstat as fs, workloads as W
fs.load_library(%(lib)r)
wl = W.WORKLOADS["small"]
x = torch.as_tensor(np.random.default_rng(11).standard_normal(wl.n).astype(np.float32), device="cuda")
a, d = (torch.as_tensor(v, device="cuda") for v in W.sky_grid(3))
f1 = torch.as_tensor(W.spin_grid(3, *wl.f1_range), device="cuda")
ctx = fs.Context(W.detector_for(wl))
seg = fs.Segment(ctx, x, wl.dt, wl.nfft, wl.fl, wl.S0)
out, status = {}, []
cap, pad = 1 << 12, 64
GUARD = 0x5A5A5A5A
for nbins in (wl.nfft // 2, wl.nfft):
    full = torch.full((pad + cap + pad, 4), GUARD, dtype=torch.int32, device="cuda")
    res = fs.search(ctx, seg, a, d, f1, 8.0, nbins=nbins, cand=full[pad:pad + cap], cand_cap=cap)
    status.append(ctx.sync_status())
    g = torch.cat([full[:pad], full[pad + cap:]])
    out["guards_%%d" %% nbins] = bool(torch.all(g == GUARD).item())
    np.save(%(prefix)r + "_F%%d.npy" %% nbins, res.F.cpu().numpy())
lib = fs.load_library()
nb = wl.nfft // 2
F = torch.empty((9, nb), dtype=torch.float32, device="cuda")
cand = torch.zeros((cap, 4), dtype=torch.int32, device="cuda")
nc = torch.zeros(1, dtype=torch.int64, device="cuda")
st = lib.fs_search_noalloc(ctx.handle, seg.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(d.data_ptr()), 3,
                           ctypes.c_void_p(f1.data_ptr()), 3, ctypes.c_float(8.0), ctypes.c_void_p(F.data_ptr()),
                           ctypes.c_int64(nb), ctypes.c_void_p(cand.data_ptr()), ctypes.c_int64(cap),
                           ctypes.c_void_p(nc.data_ptr()), None)
status += [st, ctx.sync_status()]
np.save(%(prefix)r + "_Fnoalloc.npy", F.cpu().numpy())
out["status"] = status
print(json.dumps(out))
"""


def _run(lib, prefix):
    r = subprocess.run([sys.executable, "-c", SCRIPT % {"root": ROOT, "lib": lib, "prefix": prefix}],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_runs_clean(tmp_path):
    from paper_1003_0844_gb300 import build
    rel = build.build()
    dbg = build.build_debug()
    d = _run(dbg, str(tmp_path / "dbg"))
    r = _run(rel, str(tmp_path / "rel"))
    assert d["status"] == [0, 0, 0, 0], d
    assert r["status"] == [0, 0, 0, 0], r
    assert all(v for k, v in d.items() if k.startswith("guards_")), d
    for tag in ("_F%d" % (1 << 13), "_F%d" % (1 << 14), "_Fnoalloc"):
        Fd = np.load(str(tmp_path / ("dbg" + tag + ".npy")))
        Fr = np.load(str(tmp_path / ("rel" + tag + ".npy")))
        assert np.all(np.isfinite(Fd))
        assert np.max(np.abs(Fd - Fr) / np.maximum(Fr, 1.0)) < 1e-6, tag
