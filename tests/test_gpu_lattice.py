"""FFT search of the constrained lattice on the GPU (fs_search_lattice): F on every
bin of every template (per-sky spindown rows, bins shifted by the lines' offsets)
against the oracle, the plain product grid reproduced bit for bit with zero offsets,
and an injection inside the searched patch recovered within the lattice's mismatch,
at a node whose exact F confirms the reported frequency; the plain FP64 form of the
lattice search; the same on the 2^21 transform (two 2^20 sub-transforms per
template)."""
import dataclasses
import math

import numpy as np
import pytest
import torch

from oracle import fstat as ofs
from oracle import grid as og
from oracle import resample as ors
from oracle import response as orsp
from paper_1003_0844_gb300 import workloads as W
from tests.helpers import F32_TOL, F64_TOL, check_candidates, max_rel_dF

pytestmark = pytest.mark.gpu

BOX = (0.30, 0.45, -0.10, 0.05)   # ecliptic n_x, n_y of the searched patch (near an ecliptic pole)
F1R = (-2e-9, 0.0)


@pytest.fixture(scope="module")
def fs():
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    from paper_1003_0844_gb300 import build, fstat
    build.build()
    fstat.load_library()
    return fstat


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _templates(fs, wl, det):
    G = og.linear_model_fisher(wl.n, wl.dt, det)
    B, _, _ = og.constrained_lattice(G, 0.75, 2 * math.pi / (wl.nfft * wl.dt))
    return fs.lattice_templates(B, det, wl.fl, wl.nfft, wl.dt, F1R, BOX)


def test_lattice_search_matches_oracle(fs):
    wl = W.WORKLOADS["small"]
    det = W.detector_for(wl)
    a, d, f1, off = _templates(fs, wl, det)
    x = (W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)).astype(np.float32)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    thr = 12.0
    res = fs.search_lattice(ctx, seg, _dev(a), _dev(d), _dev(f1), _dev(off), thr)
    assert ctx.sync_status() == 0
    F = res.F.double().cpu().numpy()
    so = ors.Segment(x.astype(np.float64), wl.dt)
    ns, nm = f1.shape
    ref = np.stack([ofs.fstat(so, a[s], d[s], f1[s, m], wl.fl, det, wl.S0, wl.nfft, bin_offset=off[s, m])
                    for s in range(ns) for m in range(nm)])
    assert max_rel_dF(F, ref) <= F32_TOL
    missing, bad = check_candidates(*res.candidates(), ref, thr, nm)
    assert not missing and not bad
    # zero offsets and one shared spindown row: the plain product grid, bit for bit
    f1s = W.spin_grid(nm, *F1R)
    r0 = fs.search_lattice(ctx, seg, _dev(a), _dev(d), _dev(np.tile(f1s, (ns, 1))), _dev(np.zeros((ns, nm))), thr)
    r1 = fs.search(ctx, seg, _dev(a), _dev(d), _dev(f1s), thr)
    assert torch.equal(r0.F, r1.F)
    # the plain FP64 form of the same lattice search
    seg64 = fs.Segment(ctx, _dev(x.astype(np.float64)), wl.dt, wl.nfft, wl.fl, wl.S0, precision="f64")
    r64 = fs.search_lattice(ctx, seg64, _dev(a), _dev(d), _dev(f1), _dev(off), thr)
    assert ctx.sync_status() == 0
    assert r64.F.dtype == torch.float64
    assert max_rel_dF(r64.F.cpu().numpy(), ref) <= F64_TOL
    missing, bad = check_candidates(*r64.candidates(), ref, thr, nm)
    assert not missing and not bad
    seg64.close()
    # what the lattice search refuses
    with pytest.raises(fs.FstatError) as e:
        seg_ib = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, interbin=True)
        fs.search_lattice(ctx, seg_ib, _dev(a), _dev(d), _dev(f1), _dev(off), thr)
    assert e.value.status == 7
    ctx.close()


def test_lattice_search_finds_an_injection_in_the_patch(fs):
    """A noise-free signal at a random point of the patch: the largest F of the
    lattice search is within the lattice's mismatch of the F at the true point (the
    linear model's minimal match 0.75 near the ecliptic poles) and sits next to the
    injected frequency."""
    wl = W.WORKLOADS["small"]
    det = W.detector_for(wl)
    a, d, f1, off = _templates(fs, wl, det)
    ce, se = math.cos(det.eps), math.sin(det.eps)
    g = np.random.default_rng(11)
    nx, ny = g.uniform(BOX[0] + 0.03, BOX[1] - 0.03), g.uniform(BOX[2] + 0.03, BOX[3] - 0.03)
    nz = math.sqrt(1 - nx * nx - ny * ny)
    ex, ey, ez = nx, ce * ny - se * nz, se * ny + ce * nz
    inj = W.Injection(f0=float(g.uniform(*wl.f0_range)), f1=float(g.uniform(*F1R)),
                      alpha=math.atan2(ey, ex) % (2 * math.pi),
                      delta=math.asin(ez), psi=0.4, cos_iota=0.3, phi0=0.7, snr=30.0)
    x = orsp.inject(wl.n, wl.dt, [inj], wl.fl, det, wl.sigma).astype(np.float32)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    res = fs.search_lattice(ctx, seg, _dev(a), _dev(d), _dev(f1), _dev(off), 1e9)
    F = res.F.double().cpu().numpy()
    t, k = np.unravel_index(np.argmax(F), F.shape)
    s, m = divmod(t, f1.shape[1])
    F_true = float(fs.fstat_points(ctx, seg, _dev(np.array([[inj.f0, inj.f1, inj.alpha, inj.delta]])),
                                   grad=False)[0].cpu()[0])
    assert F.max() >= 0.6 * F_true
    # the best node is reported at f0 = (k + d) / (Nfft dt): the exact F there agrees with
    # the search's (over one day the maximum may sit far along the f0-sky Doppler ridge)
    node = np.array([[(k + off[s, m]) / (wl.nfft * wl.dt), f1[s, m], a[s], d[s]]])
    F_node = float(fs.fstat_points(ctx, seg, _dev(node), grad=False)[0].cpu()[0])
    assert F_node == pytest.approx(F.max(), rel=0.03)
    ctx.close()


@pytest.mark.parametrize("n,dt", [(300000, 2.0), (1033968, 0.5)])
def test_lattice_search_2p21_matches_oracle(fs, n, dt):
    """nfft = 2^21, both data lengths (at most half of a 2^20 sub-transform, and nearly
    all of it): the first nodes of the lattice lines of a small patch against the
    oracle on every bin; zero offsets and a shared spindown row give the plain 2^21
    search bit for bit."""
    nfft = 1 << 21
    wl = dataclasses.replace(W.WORKLOADS["wide_6d"], dt=dt)
    det = W.detector_for(wl)
    G = og.linear_model_fisher(n, dt, det)
    B, _, _ = og.constrained_lattice(G, 0.75, 2 * math.pi / (nfft * dt))
    a, d, f1, off = fs.lattice_templates(B, det, wl.fl, nfft, dt, F1R, (0.30, 0.32, -0.10, -0.08))
    assert a.size >= 1 and f1.shape[1] >= 3
    a, d = a[:2].copy(), d[:2].copy()
    f1, off = f1[:2, :3].copy(), off[:2, :3].copy()
    injs = [W.Injection(f0=0.1 + 0.37 / (n * dt), f1=float(f1[0, 1]), alpha=float(a[0]), delta=float(d[0]),
                        psi=0.4, cos_iota=0.5, phi0=0.2, snr=20.0)]
    x = (np.random.default_rng(5).standard_normal(n) * wl.sigma
         + orsp.inject(n, dt, injs, wl.fl, det, wl.sigma)).astype(np.float32)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), dt, nfft, wl.fl, wl.S0)
    res = fs.search_lattice(ctx, seg, _dev(a), _dev(d), _dev(f1), _dev(off), wl.F_thr)
    assert ctx.sync_status() == 0
    F = res.F.double().cpu().numpy()
    assert F.shape == (f1.size, nfft // 2)
    so = ors.Segment(x.astype(np.float64), dt)
    ns, nm = f1.shape
    ref = np.stack([ofs.fstat(so, a[s], d[s], f1[s, m], wl.fl, det, wl.S0, nfft, bin_offset=off[s, m])
                    for s in range(ns) for m in range(nm)])
    assert max_rel_dF(F, ref) <= F32_TOL
    assert ref.max() > 100
    missing, bad = check_candidates(*res.candidates(), ref, wl.F_thr, nm)
    assert not missing and not bad
    f1s = f1[0]
    r0 = fs.search_lattice(ctx, seg, _dev(a), _dev(d), _dev(np.tile(f1s, (ns, 1))), _dev(np.zeros((ns, nm))),
                           wl.F_thr)
    r1 = fs.search(ctx, seg, _dev(a), _dev(d), _dev(f1s), wl.F_thr)
    assert torch.equal(r0.F, r1.F)
    seg.close()
    ctx.close()


def test_lattice_workload_full_configuration_sampled(fs):
    """The lattice benchmark's launch configuration (every sky row of the patch, every
    spindown node, the library's own lattice, one search call as the benchmark makes
    it): sampled template rows against the oracle and their candidates, and for all
    templates the count of crossings equals the number of F values above threshold."""
    wl = W.WORKLOADS["grid_2d"]
    det = W.detector_for(wl)
    x = (W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)).astype(np.float32)
    G = fs.linear_model_fisher(det, wl.n, wl.dt)
    B, _ = fs.lattice(G, W.LATTICE_MATCH, 2 * math.pi / (wl.nfft * wl.dt))
    a, d, f1, off = fs.lattice_templates(B, det, wl.fl, wl.nfft, wl.dt, wl.f1_range, W.LATTICE_BOX)
    ns, nm = f1.shape
    assert ns * nm > 4096
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    res = fs.search_lattice(ctx, seg, _dev(a), _dev(d), _dev(f1), _dev(off), wl.F_thr, cand_cap=1 << 20)
    assert ctx.sync_status() == 0
    F = res.F
    assert F.shape == (ns * nm, wl.nbins)
    assert bool(torch.isfinite(F).all()) and float(F.min()) >= 0.0
    assert int(res.n_cand.item()) == int((F > wl.F_thr).sum().item())
    sky, spin, bins, Fc = res.candidates()
    g = np.random.default_rng(7)
    picks = sorted({0, ns * nm - 1, *g.integers(0, ns * nm, 4).tolist()})
    so = ors.Segment(x.astype(np.float64), wl.dt)
    for t in picks:
        s, m = divmod(t, nm)
        ref = ofs.fstat(so, a[s], d[s], f1[s, m], wl.fl, det, wl.S0, wl.nfft, bin_offset=off[s, m])
        row = F[t].double().cpu().numpy()
        assert max_rel_dF(row, ref) <= F32_TOL, (t, max_rel_dF(row, ref))
        mine = (sky == s) & (spin == m)
        missing, bad = check_candidates(np.zeros(mine.sum(), dtype=np.int64), np.zeros(mine.sum(), dtype=np.int64),
                                        bins[mine], Fc[mine], ref[None, :], wl.F_thr, 1)
        assert not missing and not bad, (t, missing, bad)
    seg.close()
    ctx.close()
