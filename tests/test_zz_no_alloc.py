"""fs_search_noalloc, the allocation-free search, against fs_search.

Some callers cannot allocate device memory while they search: an application
whose framework already owns the GPU's memory through its own caching pool,
or a latency-sensitive loop that cannot absorb the device-wide synchronisation
of cudaFree.  fs_search_noalloc serves them from one fixed array that the
library holds per device.  This test calls it through the C ABI twice in a row
(the array keeps the previous call's contents, so the second call checks that
everything that must start from zero is cleared) and compares F and the
candidates with fs_search on the same inputs, within the FP32 parity tolerance.
It shows that the calls allocate nothing: on a fresh context that never ran
fs_search, the context's workspaces do not grow and the device's free memory is
the same before and after the calls (after one first call, which may make the
CUDA driver load the library's kernels).  It also checks that a
request larger than the fixed array is refused, and the lattice search's
allocation-free form against fs_search_lattice.
"""
import ctypes

import numpy as np
import pytest
import torch

from tests.helpers import F32_TOL, make_case, max_rel_dF

pytestmark = pytest.mark.gpu

FS_ERR_SCRATCH = 9


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _cand_set(cand, n):
    c = cand[: min(n, cand.shape[0])].cpu().numpy()
    return set(map(tuple, c[:, :3].tolist()))


def _noalloc_call(lib, ctx, seg, a, d, f, nsky, nspin, thr, F, nbins, cand, cap, ncand, stream):
    return lib.fs_search_noalloc(ctx.handle, seg.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                 nsky, ctypes.c_void_p(f.data_ptr()), nspin, ctypes.c_float(thr),
                                 ctypes.c_void_p(F.data_ptr()), ctypes.c_int64(nbins),
                                 ctypes.c_void_p(cand.data_ptr()), ctypes.c_int64(cap),
                                 ctypes.c_void_p(ncand.data_ptr()), stream)


def test_noalloc_search_allocates_nothing_on_a_fresh_context():
    """A context that never ran fs_search: its workspaces do not grow across the
    calls (segment preparation holds the only one), and the device's free memory
    does not move between the second and the fourth call (every output is
    allocated before the first reading)."""
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    from paper_1003_0844_gb300 import build, fstat as fs
    build.build()
    lib = fs.load_library()
    wl, det, x, alpha, delta, _ = make_case("single_fp64", n=30011, nfft=1 << 16, nsky=3, nspin=4)
    f1 = np.linspace(-1e-8, 0.0, 4)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    a, d, f = _dev(alpha), _dev(delta), _dev(f1)
    nbins, cap = wl.nfft // 2, 1 << 12
    outs = [(torch.empty((len(alpha) * len(f1), nbins), dtype=torch.float32, device="cuda"),
             torch.zeros((cap, 4), dtype=torch.int32, device="cuda"),
             torch.zeros((1,), dtype=torch.int64, device="cuda")) for _ in range(4)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ws0 = ctx.stats(reset=False)["workspace_bytes"]
    free = []
    for i, (F, cand, ncand) in enumerate(outs):
        st = _noalloc_call(lib, ctx, seg, a, d, f, len(alpha), len(f1), 15.0, F, nbins, cand, cap, ncand, stream)
        assert st == 0, "call %d returned %d" % (i, st)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    assert ctx.sync_status() == 0
    assert ctx.stats(reset=False)["workspace_bytes"] == ws0
    assert free[1] == free[2] == free[3], free
    for F, cand, ncand in outs[1:]:
        assert torch.equal(F, outs[0][0]) and int(ncand.item()) == int(outs[0][2].item())
    seg.close()
    ctx.close()


def test_noalloc_search_matches_search_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    from paper_1003_0844_gb300 import build, fstat as fs
    build.build()
    lib = fs.load_library()
    wl, det, x, alpha, delta, _ = make_case("single_fp64", n=30011, nfft=1 << 16, nsky=3, nspin=4)
    f1 = np.linspace(-1e-8, 0.0, 4)
    thr = 15.0
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    a, d, f = _dev(alpha), _dev(delta), _dev(f1)
    ref = fs.search(ctx, seg, a, d, f, thr)
    assert ctx.sync_status() == 0
    F_ref = ref.F.double().cpu().numpy()
    n_ref = int(ref.n_cand.item())
    want = _cand_set(ref.cand, n_ref)

    nbins = wl.nfft // 2
    cap = 1 << 12
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        F = torch.full((len(alpha) * len(f1), nbins), float("nan"), dtype=torch.float32, device="cuda")
        cand = torch.zeros((cap, 4), dtype=torch.int32, device="cuda")
        ncand = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        st = lib.fs_search_noalloc(ctx.handle, seg.handle, ctypes.c_void_p(a.data_ptr()),
                                   ctypes.c_void_p(d.data_ptr()), len(alpha), ctypes.c_void_p(f.data_ptr()),
                                   len(f1), ctypes.c_float(thr), ctypes.c_void_p(F.data_ptr()),
                                   ctypes.c_int64(nbins), ctypes.c_void_p(cand.data_ptr()), ctypes.c_int64(cap),
                                   ctypes.c_void_p(ncand.data_ptr()), stream)
        assert st == 0, "call %d returned %d" % (call, st)
        assert ctx.sync_status() == 0
        got = F.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        assert max_rel_dF(got, F_ref) < F32_TOL
        n = int(ncand.item())
        assert n == n_ref
        assert _cand_set(cand, n) == want


def test_noalloc_lattice_search_matches_lattice_search():
    """fs_search_lattice_noalloc (per-template spindowns and bin offsets, one sky row
    per launch) against fs_search_lattice on the same inputs, twice in a row."""
    import math
    from oracle import grid as og
    from paper_1003_0844_gb300 import build, fstat as fs
    build.build()
    lib = fs.load_library()
    wl, det, x, _, _, _ = make_case("small")
    G = og.linear_model_fisher(wl.n, wl.dt, det)
    B, _, _ = og.constrained_lattice(G, 0.75, 2 * math.pi / (wl.nfft * wl.dt))
    al, de, f1, off = fs.lattice_templates(B, det, wl.fl, wl.nfft, wl.dt, (-2e-9, 0.0), (0.30, 0.45, -0.10, 0.05))
    thr = 12.0
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    a, d, f, o = _dev(al), _dev(de), _dev(f1), _dev(off)
    ref = fs.search_lattice(ctx, seg, a, d, f, o, thr)
    assert ctx.sync_status() == 0
    n_ref = int(ref.n_cand.item())
    want = _cand_set(ref.cand, n_ref)
    nsky, nspin = f1.shape
    nbins = wl.nfft // 2
    cap = 1 << 16
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        F = torch.full((nsky * nspin, nbins), float("nan"), dtype=torch.float32, device="cuda")
        cand = torch.zeros((cap, 4), dtype=torch.int32, device="cuda")
        ncand = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        st = lib.fs_search_lattice_noalloc(ctx.handle, seg.handle, ctypes.c_void_p(a.data_ptr()),
                                           ctypes.c_void_p(d.data_ptr()), nsky, ctypes.c_void_p(f.data_ptr()),
                                           ctypes.c_void_p(o.data_ptr()), nspin, ctypes.c_float(thr),
                                           ctypes.c_void_p(F.data_ptr()), ctypes.c_int64(nbins),
                                           ctypes.c_void_p(cand.data_ptr()), ctypes.c_int64(cap),
                                           ctypes.c_void_p(ncand.data_ptr()), stream)
        assert st == 0, "call %d returned %d" % (call, st)
        assert ctx.sync_status() == 0
        got = F.double().cpu().numpy()
        assert max_rel_dF(got, ref.F.double().cpu().numpy()) < F32_TOL
        n = int(ncand.item())
        assert n == n_ref
        assert _cand_set(cand, n) == want
    seg.close()
    ctx.close()


def test_noalloc_search_refuses_requests_larger_than_its_array():
    from paper_1003_0844_gb300 import build, fstat as fs
    build.build()
    lib = fs.load_library()
    wl, det, x, alpha, delta, f1 = make_case("grid_2d", inject=False, nsky=1, nspin=1)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)  # Nfft = 2^18
    F = torch.empty((1, wl.nfft // 2), dtype=torch.float32, device="cuda")
    cand = torch.zeros((16, 4), dtype=torch.int32, device="cuda")
    ncand = torch.zeros(1, dtype=torch.int64, device="cuda")
    a, d, f = _dev(alpha), _dev(delta), _dev(f1)
    st = lib.fs_search_noalloc(ctx.handle, seg.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                               1, ctypes.c_void_p(f.data_ptr()), 1, ctypes.c_float(20.0),
                               ctypes.c_void_p(F.data_ptr()), ctypes.c_int64(wl.nfft // 2),
                               ctypes.c_void_p(cand.data_ptr()), ctypes.c_int64(16),
                               ctypes.c_void_p(ncand.data_ptr()), None)
    assert st == FS_ERR_SCRATCH
    assert ctx.sync_status() == 0
