"""Parity of the batched multi-segment search, the transform splits the tuner
chooses from, the 2^21 transform (two half-bin-shifted 2^20 sub-transforms) and
segment epochs, all through the C ABI against the CPU oracle."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import earth as oe
from oracle import fstat as ofs
from oracle import resample as ors
from oracle import response as orsp
from paper_1003_0844_gb300 import workloads as W
from tests.helpers import F32_TOL, check_candidates, make_case, max_rel_dF, oracle_F

pytestmark = pytest.mark.gpu


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


def _search_F(fs, ctx, seg, alpha, delta, f1, thr, nbins=None):
    res = fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), thr, nbins=nbins)
    assert ctx.sync_status() == 0
    return res.F.double().cpu().numpy(), res.candidates()


# ------------------------------------------------------------------ transform splits

@pytest.mark.parametrize("name,nfft,n1", [("small", 1 << 14, 256), ("small", 1 << 14, 128),
                                          ("small", 1 << 16, 512), ("small", 1 << 16, 128),
                                          ("grid_2d", 1 << 18, 1024), ("grid_2d", 1 << 18, 256)])
def test_split_matches_oracle(fs, name, nfft, n1):
    wl, det, x, alpha, delta, f1 = make_case(name, nfft=nfft, nsky=2, nspin=2)
    if name == "grid_2d":
        alpha, delta, f1 = alpha[:1], delta[:1], f1[:2]
    ref = oracle_F(x, wl, det, alpha, delta, f1)
    ctx = fs.Context(det)
    ctx.set_tuning(nfft, n1=n1, queue_round=3, queue_lag=2)
    assert ctx.get_tuning(nfft)["n1"] == n1
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    F, cand = _search_F(fs, ctx, seg, alpha, delta, f1, wl.F_thr)
    assert max_rel_dF(F, ref) <= F32_TOL
    missing, bad = check_candidates(*cand, ref, wl.F_thr, len(f1))
    assert not missing and not bad


def test_tuning_arguments(fs):
    wl, det, x, *_ = make_case("tiny")
    ctx = fs.Context(det)
    assert ctx.get_tuning(1 << 14) is None
    with pytest.raises(fs.FstatError) as e:
        ctx.set_tuning(1 << 14, n1=32)          # 32 x 512 is not built
    assert e.value.status == 1
    with pytest.raises(fs.FstatError) as e:
        ctx.set_tuning(3000, n1=0)
    assert e.value.status == 2
    ctx.set_tuning(1 << 16, n1=128, queue_round=5)
    t = ctx.get_tuning(1 << 16)
    assert (t["n1"], t["queue_round"], t["queue_lag"]) == (128, 5, 0)
    ctx.clear_tuning(1 << 16)
    assert ctx.get_tuning(1 << 16) is None


# ------------------------------------------------------------------ 2^21 transform

@pytest.mark.parametrize("n,dt", [(300000, 2.0), (1033968, 0.5)])
def test_nfft_2p21_matches_oracle(fs, n, dt):
    """nfft = 2^21: both data lengths (at most half of a 2^20 sub-transform, and
    nearly all of it, the 6-day 0.5 s segment)."""
    wl = dataclasses.replace(W.WORKLOADS["wide_6d"], dt=dt, nsky=1, nspin=1)
    det = W.detector_for(wl)
    x = W.noise(wl)[:n] if n <= wl.n else np.random.default_rng(5).standard_normal(n)
    injs = [W.Injection(f0=0.1 + 0.37 / (n * dt), f1=-2e-9, alpha=1.0, delta=0.3, psi=0.4, cos_iota=0.5,
                        phi0=0.2, snr=20.0)]
    x = x + orsp.inject(n, dt, injs, wl.fl, det, wl.sigma)
    alpha, delta = np.array([injs[0].alpha]), np.array([injs[0].delta])
    f1 = np.array([injs[0].f1])
    ref = oracle_F(x, wl, det, alpha, delta, f1)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), dt, 1 << 21, wl.fl, wl.S0)
    F, cand = _search_F(fs, ctx, seg, alpha, delta, f1, wl.F_thr)
    assert F.shape == (1, 1 << 20)
    assert max_rel_dF(F, ref) <= F32_TOL
    missing, bad = check_candidates(*cand, ref, wl.F_thr, 1)
    assert not missing and not bad
    # the injected source's peak is in the band and found
    assert ref.max() > 100 and int(np.argmax(F)) == int(np.argmax(ref))


def test_nfft_2p21_f64_and_limits(fs):
    wl = dataclasses.replace(W.WORKLOADS["wide_6d"], dt=2.0, nsky=1, nspin=1)
    det = W.detector_for(wl)
    n = 200000
    x = W.noise(wl)[:n]
    alpha, delta = W.sky_grid(1)
    f1 = np.array([-3e-9])
    ref = oracle_F(x, wl, det, alpha, delta, f1)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x), 2.0, 1 << 21, wl.fl, wl.S0, precision="f64")
    F, _ = _search_F(fs, ctx, seg, alpha, delta, f1, 1e9)
    assert max_rel_dF(F, ref) <= 1e-8
    # FP32 2^21 needs the data to fit one 2^20 sub-transform
    xl = torch.zeros((1 << 20) + 2, dtype=torch.float32, device="cuda")
    with pytest.raises(fs.FstatError) as e:
        fs.Segment(ctx, xl, 0.5, 1 << 21, wl.fl, wl.S0)
    assert e.value.status == 2


# ------------------------------------------------------------------ batches and epochs

def _batch_case(name="uneven_small"):
    b = W.BATCHES[name]
    det = W.detector_for(b)
    segs = b.segments()
    t0 = b.epochs()
    xs = []
    for i, wl in enumerate(segs):
        de = oe.detector_at_epoch(det, t0[i])
        x = W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, de, wl.sigma)
        xs.append(x)
    alpha, delta = W.sky_grid(b.nsky)
    f1 = W.spin_grid(b.nspin, *b.f1_range)
    return b, det, segs, t0, xs, alpha, delta, f1


def test_batch_matches_oracle_and_single_searches(fs):
    b, det, segs, t0, xs, alpha, delta, f1 = _batch_case()
    ctx = fs.Context(det)
    handles = [fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, t0=t0[i])
               for i, (wl, x) in enumerate(zip(segs, xs))]
    A, D, F1 = _dev(alpha), _dev(delta), _dev(f1)
    res = fs.search_batch(ctx, handles, A, D, F1, b.F_thr, cand_cap=4096)
    assert ctx.sync_status() == 0
    for i, (wl, x) in enumerate(zip(segs, xs)):
        got = res.candidates(i)
        single = fs.search(ctx, handles[i], A, D, F1, b.F_thr, write_F=True)
        assert ctx.sync_status() == 0
        sc = single.candidates()
        key = lambda c: sorted(zip(c[0].tolist(), c[1].tolist(), c[2].tolist(), c[3].tolist()))
        assert key(got) == key(sc)                      # same kernels, same configuration: bit-exact
        ref = oracle_F(x, wl, oe.detector_at_epoch(det, t0[i]), alpha, delta, f1)
        assert max_rel_dF(single.F.double().cpu().numpy(), ref) <= F32_TOL
        missing, bad = check_candidates(*got, ref, b.F_thr, len(f1))
        assert not missing and not bad
    # the epoch matters: a segment searched as if it started at t = 0 differs
    wl, x = segs[2], xs[2]
    s0 = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, t0=0.0)
    F0, _ = _search_F(fs, ctx, s0, alpha, delta, f1, b.F_thr)
    ref = oracle_F(x, wl, oe.detector_at_epoch(det, t0[2]), alpha, delta, f1)
    assert max_rel_dF(F0, ref) > 10 * F32_TOL


def test_lattice_batch_matches_single_lattice_searches(fs):
    """fs_search_lattice_batch: every segment of the uneven batch with its own lattice
    of the same sky patch (its own Fisher matrix at its epoch, so its own counts of sky
    rows and spindown nodes) reports the same candidates as fs_search_lattice on that
    segment alone (same kernels, same configuration: bit-exact), on the first call and
    on the recorded graph's replay; an interbinning segment is refused."""
    import math
    b, det, segs, t0, xs, _, _, _ = _batch_case()
    ctx = fs.Context(det)
    handles = [fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, t0=t0[i])
               for i, (wl, x) in enumerate(zip(segs, xs))]
    tpl = []
    for i, wl in enumerate(segs):
        G = fs.linear_model_fisher(det, wl.n, wl.dt, float(t0[i]))
        B, _ = fs.lattice(G, 0.75, 2 * math.pi / (wl.nfft * wl.dt))
        a, d, f1, off = fs.lattice_templates(B, det, wl.fl, wl.nfft, wl.dt, (-2e-9, 0.0), (0.30, 0.45, -0.10, 0.05))
        tpl.append(tuple(_dev(v) for v in (a, d, f1, off)))
    assert len({tuple(t[2].shape) for t in tpl}) > 2
    key = lambda c: sorted(zip(c[0].tolist(), c[1].tolist(), c[2].tolist(), c[3].tolist()))
    res = fs.search_lattice_batch(ctx, handles, tpl, b.F_thr, cand_cap=1 << 20)
    assert ctx.sync_status() == 0
    first = [key(res.candidates(i)) for i in range(len(segs))]
    assert sum(len(c) for c in first) > 0
    res.cand.zero_()
    res.n_cand.fill_(-1)
    res2 = fs.search_lattice_batch(ctx, handles, tpl, b.F_thr, cand_cap=1 << 20, cand=res.cand, n_cand=res.n_cand)
    assert ctx.sync_status() == 0
    assert [key(res2.candidates(i)) for i in range(len(segs))] == first
    for i, h in enumerate(handles):
        single = fs.search_lattice(ctx, h, *tpl[i], b.F_thr, write_F=False, cand_cap=1 << 20)
        assert ctx.sync_status() == 0
        assert first[i] == key(single.candidates()), i
    wl = segs[0]
    ib = fs.Segment(ctx, _dev(xs[0], torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, t0=t0[0], interbin=True)
    with pytest.raises(fs.FstatError) as e:
        fs.search_lattice_batch(ctx, [ib] + handles[1:], tpl, b.F_thr)
    assert e.value.status == 7
    ctx.close()


def test_batch_full_configuration_sampled(fs):
    """The benchmark's batch (64 segments of 1/2/3/6 days, 2^16-2^20, 64 skies x 64
    spindowns, one graph): for one template of each segment kind, the crossings the
    batch reports equal the oracle's F above threshold (FFT mode, that template)."""
    b = W.BATCHES["uneven_64"]
    det = W.detector_for(b)
    segs, t0 = b.segments(), b.epochs()
    a_all, d_all = W.sky_grid(b.nsky)
    alpha, delta = a_all[:64], d_all[:64]
    f1 = W.spin_grid(b.nspin, *b.f1_range)
    ctx = fs.Context(det)
    xs, handles = [], []
    for i, wl in enumerate(segs):
        de = oe.detector_at_epoch(det, t0[i])
        x = (W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, de, wl.sigma)).astype(np.float32)
        xs.append(x)
        handles.append(fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, t0=t0[i]))
    res = fs.search_batch(ctx, handles, _dev(alpha), _dev(delta), _dev(f1), b.F_thr, cand_cap=1 << 16)
    assert ctx.sync_status() == 0
    g = np.random.default_rng(3)
    seen = set()
    for i, wl in enumerate(segs):
        if (wl.days, wl.nfft) in seen:
            continue
        seen.add((wl.days, wl.nfft))
        s, m = int(g.integers(0, len(alpha))), int(g.integers(0, len(f1)))
        so = ors.Segment(xs[i].astype(np.float64), wl.dt)
        ref = ofs.fstat(so, alpha[s], delta[s], f1[m], wl.fl, oe.detector_at_epoch(det, t0[i]), wl.S0, wl.nfft)
        sky, spin, bins, Fc = res.candidates(i)
        mine = (sky == s) & (spin == m)
        z = np.zeros(int(mine.sum()), dtype=np.int64)
        missing, bad = check_candidates(z, z, bins[mine], Fc[mine], ref[None, :], b.F_thr, 1)
        assert not missing and not bad, (i, s, m, missing, bad)
    assert len(seen) == 4
    ctx.close()


def test_batch_graph_replay_and_reload(fs):
    b, det, segs, t0, xs, alpha, delta, f1 = _batch_case()
    ctx = fs.Context(det)
    handles = [fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, t0=t0[i])
               for i, (wl, x) in enumerate(zip(segs, xs))]
    A, D, F1 = _dev(alpha), _dev(delta), _dev(f1)
    cand = torch.zeros((len(segs), 4096, 4), dtype=torch.int32, device="cuda")
    ncand = torch.zeros(len(segs), dtype=torch.int64, device="cuda")
    ctx.stats(reset=True)
    r1 = fs.search_batch(ctx, handles, A, D, F1, b.F_thr, cand=cand, n_cand=ncand)
    first = [r1.candidates(i) for i in range(len(segs))]
    l1 = ctx.stats(reset=True)["launches"]
    r2 = fs.search_batch(ctx, handles, A, D, F1, b.F_thr, cand=cand, n_cand=ncand)   # graph replay
    assert ctx.sync_status() == 0
    assert ctx.stats(reset=True)["launches"] == l1 > 0
    key = lambda c: sorted(zip(c[0].tolist(), c[1].tolist(), c[2].tolist(), c[3].tolist()))
    for i in range(len(segs)):
        assert key(r2.candidates(i)) == key(first[i])
    # reload segment 1 with other data: the replayed graph searches the new data
    wl = segs[1]
    xn = W.noise(wl, seed_stream=9) + orsp.inject(wl.n, wl.dt, W.injections(wl, seed_stream=8), wl.fl,
                                                  oe.detector_at_epoch(det, t0[1]), wl.sigma)
    handles[1].load(_dev(xn, torch.float32))
    r3 = fs.search_batch(ctx, handles, A, D, F1, b.F_thr, cand=cand, n_cand=ncand)
    assert ctx.sync_status() == 0
    single = fs.search(ctx, handles[1], A, D, F1, b.F_thr, write_F=False)
    assert key(r3.candidates(1)) == key(single.candidates())
    for i in (0, 2, 3):
        assert key(r3.candidates(i)) == key(first[i])


def test_autotune_picks_a_valid_split(fs):
    wl, det, x, alpha, delta, f1 = make_case("small", nfft=1 << 16, nsky=4, nspin=3)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    t = ctx.autotune(seg, _dev(alpha), _dev(delta), _dev(f1), reps=2)
    assert t["n1"] in (128, 256, 512) and t["queue_round"] >= 1 and t["queue_lag"] in (1, 2)
    assert t["ms_per_template"] > 0
    assert ctx.get_tuning(1 << 16)["n1"] == t["n1"]
    F, cand = _search_F(fs, ctx, seg, alpha, delta, f1, wl.F_thr)
    ref = oracle_F(x, wl, det, alpha, delta, f1)
    assert max_rel_dF(F, ref) <= F32_TOL
    missing, bad = check_candidates(*cand, ref, wl.F_thr, len(f1))
    assert not missing and not bad


def test_autotune_interbinning_segment(fs):
    """The tuner times an interbinning segment on its own half-bin row and keeps a
    split whose search still matches the oracle."""
    from oracle import fstat as ofs_
    wl, det, x, alpha, delta, f1 = make_case("small", nfft=1 << 15, nsky=2, nspin=2)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, interbin=True)
    t = ctx.autotune(seg, _dev(alpha), _dev(delta), _dev(f1), reps=1)
    assert t["n1"] in (64, 128, 256, 512) and t["ms_per_template"] > 0
    res = fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), wl.F_thr)
    assert ctx.sync_status() == 0
    so = ors.Segment(x, wl.dt)
    ref = np.stack([ofs_.fstat_interbinned(so, a, d, s1, wl.fl, det, wl.S0, wl.nfft)
                    for a, d in zip(alpha, delta) for s1 in f1])
    assert max_rel_dF(res.F.double().cpu().numpy(), ref) <= F32_TOL


# ------------------------------------------------------------------ interbinning

@pytest.mark.parametrize("name,n,nfft,precision", [("small", None, 1 << 14, "f32"), ("small", None, 1 << 14, "f64"),
                                                   ("grid_2d", None, 1 << 17, "f32"),
                                                   ("wide_6d", 1033968, 1 << 20, "f32")])
def test_interbinning_matches_oracle(fs, name, n, nfft, precision):
    from oracle import fstat as ofs
    wl, det, x, alpha, delta, f1 = make_case(name, nfft=nfft, nsky=2, nspin=2, n=n)
    if name != "small":
        alpha, delta, f1 = alpha[:1], delta[:1], f1[:1]
    seg_o = ors.Segment(x, wl.dt)
    ref = np.stack([ofs.fstat_interbinned(seg_o, a, d, s1, wl.fl, det, wl.S0, nfft)
                    for a, d in zip(alpha, delta) for s1 in f1])
    ctx = fs.Context(det)
    xd = _dev(x, torch.float32 if precision == "f32" else torch.float64)
    seg = fs.Segment(ctx, xd, wl.dt, nfft, wl.fl, wl.S0, precision=precision, interbin=True)
    res = fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), wl.F_thr)
    assert ctx.sync_status() == 0
    F = res.F.double().cpu().numpy()
    assert F.shape == (len(alpha) * len(f1), nfft)
    assert max_rel_dF(F, ref) <= (F32_TOL if precision == "f32" else 1e-8)
    missing, bad = check_candidates(*res.candidates(), ref, wl.F_thr, len(f1))
    assert not missing and not bad
    # argument rules: the F row is nfft long; the batch and allocation-free paths refuse
    with pytest.raises(fs.FstatError) as e:
        fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), wl.F_thr, nbins=nfft // 2)
    assert e.value.status == 2
    if precision == "f32":
        # the batched search takes interbinning segments: the same crossings, bit for bit
        rb = fs.search_batch(ctx, [seg], _dev(alpha), _dev(delta), _dev(f1), wl.F_thr)
        assert ctx.sync_status() == 0
        key = lambda c: sorted(zip(c[0].tolist(), c[1].tolist(), c[2].tolist(), c[3].tolist()))
        assert key(rb.candidates(0)) == key(res.candidates())


@pytest.mark.parametrize("name,nfft,n1,qround,nsky,nspin", [
    ("tiny", 1 << 12, 0, 0, 3, 2),        # 64 x 64: two rows per warp, 16-row tiles
    ("small", 1 << 15, 0, 1, 2, 3),       # 256 x 128, one template per queue round
    ("small", 1 << 16, 512, 0, 1, 2),     # 512 x 128: no interbinning items, per-batch launches
    ("grid_2d", 1 << 17, 512, 0, 1, 2),   # 512 x 256 (the default 2^17 interbinning split is 256 x 512)
])
def test_interbinning_persistent_splits(fs, name, nfft, n1, qround, nsky, nspin):
    """The interbinning items of the persistent queue (tile-interior odd bins) and the
    edge kernel (odd bins between tiles, the wrap to row 0 and X(Nfft/2)) on every
    bin against the oracle, for splits and queue shapes the default test does not reach."""
    from oracle import fstat as ofs
    wl, det, x, alpha, delta, f1 = make_case(name, nfft=nfft, nsky=nsky, nspin=nspin)
    seg_o = ors.Segment(x, wl.dt)
    ref = np.stack([ofs.fstat_interbinned(seg_o, a, d, s1, wl.fl, det, wl.S0, nfft)
                    for a, d in zip(alpha, delta) for s1 in f1])
    ctx = fs.Context(det)
    if n1 or qround:
        ctx.set_tuning(nfft, n1=n1, queue_round=qround)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, nfft, wl.fl, wl.S0, interbin=True)
    thr = float(np.quantile(ref, 0.999))   # enough crossings to exercise the compaction on both grids
    res = fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), thr)
    assert ctx.sync_status() == 0
    F = res.F.double().cpu().numpy()
    assert max_rel_dF(F, ref) <= F32_TOL
    assert max_rel_dF(F[:, 1::2], ref[:, 1::2]) <= F32_TOL
    missing, bad = check_candidates(*res.candidates(), ref, thr, len(f1))
    assert not missing and not bad
    # candidates only (no F written) give the same crossings
    res2 = fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), thr, write_F=False)
    c1 = sorted(zip(*[a.tolist() for a in res.candidates()[:3]]))
    c2 = sorted(zip(*[a.tolist() for a in res2.candidates()[:3]]))
    assert c1 == c2
