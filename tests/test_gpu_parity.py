"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same
seeded inputs: each stage (upsampling, injection, per-sky demodulation) and
the whole search (F on every bin and the candidate list), for FFT shapes that
span several tiles and a ragged tail, both precisions, and the edge cases."""
import math

import numpy as np
import pytest
import torch

from oracle import fstat as ofs
from oracle import resample as ors
from oracle import response as orsp
from paper_1003_0844_gb300 import workloads as W
from tests.helpers import F32_TOL, F64_TOL, check_candidates, make_case, max_rel_dF, oracle_F

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


def _run(fs, wl, det, x, alpha, delta, f1, precision="f32", interp="spline", nbins=None, thr=None,
         x_dtype=torch.float32, cand_cap=1 << 16):
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, x_dtype), wl.dt, wl.nfft, wl.fl, wl.S0, precision=precision, interp=interp)
    res = fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), wl.F_thr if thr is None else thr,
                    nbins=nbins, cand_cap=cand_cap)
    status = ctx.sync_status()
    F = res.F.double().cpu().numpy()
    cand = res.candidates()
    ncand = int(res.n_cand.item())
    seg.close()
    ctx.close()
    return F, cand, ncand, status


# ------------------------------------------------------------------ stages

@pytest.mark.parametrize("name,xdt", [("tiny", torch.float32), ("small", torch.float64)])
def test_upsample_matches_oracle(fs, name, xdt):
    wl, det, x, *_ = make_case(name)
    x = x.astype(np.float32).astype(np.float64) if xdt == torch.float32 else x
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, xdt), wl.dt, wl.nfft, wl.fl, wl.S0)
    x2 = seg.upsampled().cpu().numpy()
    ref = ors.fourier_upsample2(x)
    assert np.max(np.abs(x2 - ref)) < 1e-11 * np.max(np.abs(x))
    assert np.array_equal(x2[::2], x)


def test_inject_matches_oracle(fs):
    wl = W.WORKLOADS["small"]
    det = W.detector_for(wl)
    injs = W.injections(wl)
    ctx = fs.Context(det)
    xg = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    fs.inject(ctx, xg, wl.dt, wl.fl, wl.sigma, injs)
    ref = orsp.inject(wl.n, wl.dt, injs, wl.fl, det, wl.sigma)
    assert np.max(np.abs(xg.cpu().numpy() - ref)) < 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("interp", ["spline", "nearest"])
def test_demodulate_matches_oracle(fs, precision, interp):
    wl, det, x, alpha, delta, _ = make_case("small")
    x = x.astype(np.float32).astype(np.float64)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, precision=precision, interp=interp)
    oseg = ors.Segment(x, wl.dt)
    for s in range(len(alpha)):
        ya, yb, ts, ab = fs.demodulate(ctx, seg, alpha[s], delta[s])
        ref = ofs.demodulate(oseg, alpha[s], delta[s], 0.0, wl.fl, det, interp=interp)
        ts = ts.cpu().numpy()
        ya = ya.cpu().numpy()
        yb = yb.cpu().numpy()
        a2, b2 = ab.cpu().numpy()
        tol_t = 2e-6 if precision == "f32" else 1e-9
        assert np.max(np.abs(ts - ref.t_src)) < tol_t
        tol = 2e-5 if precision == "f32" else 1e-9
        rms = math.sqrt(np.mean(np.abs(ref.ya) ** 2))
        assert np.max(np.abs(ya - ref.ya)) < tol * rms * 10
        assert np.max(np.abs(yb - ref.yb)) < tol * rms * 10
        tol_m = 1e-6 if precision == "f32" else 1e-12
        assert abs(a2 / ref.a2 - 1) < tol_m and abs(b2 / ref.b2 - 1) < tol_m


# ------------------------------------------------------------------ whole search

SHAPES = [
    # (workload, n, nfft): FFT splits 64x64, 128x64, 128x128, 256x128, 256x256, 512x256
    ("tiny", None, 1 << 12),
    ("tiny", None, 1 << 13),
    ("small", None, 1 << 14),
    ("small", None, 1 << 15),
    ("single_fp64", 30011, 1 << 16),
    ("single_fp64", None, 1 << 17),
    # 1024-point column DFTs: 3 sidereal days (zero upper half pruned), an unpruned
    # 2^19 case, and 6 sidereal days on 1024 x 1024
    ("grid_2d", 129246, 1 << 19),
    ("grid_2d", 300000, 1 << 19),
    ("grid_2d", 258492, 1 << 20),
]


@pytest.mark.parametrize("name,n,nfft", SHAPES)
def test_search_f32_matches_oracle(fs, name, n, nfft):
    nsky, nspin = (3, 2) if nfft <= (1 << 15) else ((2, 2) if nfft <= (1 << 18) else (2, 1))
    wl, det, x, alpha, delta, f1 = make_case(name, n=n, nfft=nfft, nsky=nsky, nspin=nspin)
    if name == "single_fp64":
        f1 = np.array([-1e-9, -7e-9])
    x32 = x.astype(np.float32).astype(np.float64)
    F, (cs, cm, cb, cF), ncand, status = _run(fs, wl, det, x32, alpha, delta, f1, thr=15.0)
    assert status == 0
    Fref = oracle_F(x32, wl, det, alpha, delta, f1)
    assert max_rel_dF(F, Fref) < F32_TOL
    missing, bad = check_candidates(cs, cm, cb, cF, Fref, 15.0, len(f1))
    assert not missing and not bad
    assert ncand == len(cs)
    assert np.all(np.abs(cF - F[cs * len(f1) + cm, cb]) == 0.0)


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_search_f64_matches_oracle(fs, name):
    wl, det, x, alpha, delta, f1 = make_case(name)
    F, (cs, cm, cb, cF), ncand, status = _run(fs, wl, det, x, alpha, delta, f1, precision="f64",
                                              x_dtype=torch.float64)
    assert status == 0
    Fref = oracle_F(x, wl, det, alpha, delta, f1)
    assert max_rel_dF(F, Fref) < F64_TOL
    missing, bad = check_candidates(cs, cm, cb, cF, Fref, wl.F_thr, len(f1), rel=1e-7)
    assert not missing and not bad


def test_search_f64_headline_shape_matches_oracle(fs):
    """The plain FP64 form at the 2-sidereal-day shape of the benchmark (N = 86,164,
    Nfft = 2^18, every bin up to Nyquist): two templates against the oracle."""
    wl, det, x, alpha, delta, f1 = make_case("grid_2d", nsky=2, nspin=1)
    F, (cs, cm, cb, cF), ncand, status = _run(fs, wl, det, x, alpha, delta, f1, precision="f64",
                                              x_dtype=torch.float64)
    assert status == 0
    assert F.shape == (2, wl.nfft // 2)
    Fref = oracle_F(x, wl, det, alpha, delta, f1)
    assert max_rel_dF(F, Fref) < F64_TOL
    missing, bad = check_candidates(cs, cm, cb, cF, Fref, wl.F_thr, len(f1), rel=1e-7)
    assert not missing and not bad


def test_search_all_bins_and_nearest(fs):
    wl, det, x, alpha, delta, f1 = make_case("tiny")
    x32 = x.astype(np.float32).astype(np.float64)
    F, *_ = _run(fs, wl, det, x32, alpha, delta, f1, nbins=wl.nfft)
    Fref = oracle_F(x32, wl, det, alpha, delta, f1, nbins=wl.nfft)
    assert max_rel_dF(F, Fref) < F32_TOL
    Fn, *_ = _run(fs, wl, det, x32, alpha, delta, f1, interp="nearest")
    Fnref = oracle_F(x32, wl, det, alpha, delta, f1, interp="nearest")
    assert max_rel_dF(Fn, Fnref) < F32_TOL


def test_search_full_size_2day_sampled_templates(fs):
    # the 2-sidereal-day shape (N = 86,164, Nfft = 2^18) in the launch
    # configuration of the benchmark; a few templates against the oracle's FFT mode
    wl, det, x, alpha, delta, f1 = make_case("grid_2d", nsky=3, nspin=2)
    x32 = x.astype(np.float32).astype(np.float64)
    F, (cs, cm, cb, cF), ncand, status = _run(fs, wl, det, x32, alpha, delta, f1)
    assert status == 0
    Fref = oracle_F(x32, wl, det, alpha, delta, f1)
    assert max_rel_dF(F, Fref) < F32_TOL
    missing, bad = check_candidates(cs, cm, cb, cF, Fref, wl.F_thr, len(f1))
    assert not missing and not bad


def test_search_is_deterministic(fs):
    wl, det, x, alpha, delta, f1 = make_case("small")
    F1, c1, n1, _ = _run(fs, wl, det, x, alpha, delta, f1)
    F2, c2, n2, _ = _run(fs, wl, det, x, alpha, delta, f1)
    assert np.array_equal(F1, F2)
    assert n1 == n2
    k1 = sorted(zip(c1[0], c1[1], c1[2]))
    k2 = sorted(zip(c2[0], c2[1], c2[2]))
    assert k1 == k2


# ------------------------------------------------------------------ statistics and signal

def _kept_weight(x, wl, det, al, de, f1, interp):
    """E[F] / 2 for white noise under nearest-neighbour resampling: the a^2- (b^2-)
    weighted fraction of output samples whose source time falls inside the data."""
    dm = ofs.demodulate(ors.Segment(x, wl.dt), al, de, f1, wl.fl, det, interp=interp)
    k = np.rint(dm.t_src / wl.dt)
    kept = (k >= 0) & (k < wl.n)
    a, b = orsp.ab(dm.t_src, al, de, det)
    return 0.5 * (np.sum(a[kept] ** 2) / np.sum(a * a) + np.sum(b[kept] ** 2) / np.sum(b * b))


def test_noise_only_F_is_chi2_4dof_on_gpu(fs):
    from scipy.stats import chi2, kstest
    # independent noise realizations (templates sharing one realization are correlated);
    # nearest-neighbour resampling keeps the noise white, so E[F] = 2 x kept weight exactly.
    # The band mean of one realization follows that realization's energy (~3% scatter),
    # so the check uses the empirical spread of the realization means.
    ratios, shapes = [], []
    for r in range(16):
        wl, det, x, alpha, delta, f1 = make_case("small", inject=False, seed_stream=100 + r, nsky=2, nspin=1)
        al, de = alpha[r % 2: r % 2 + 1], delta[r % 2: r % 2 + 1]
        F, *_ = _run(fs, wl, det, x, al, de, f1, thr=1e9, interp="nearest")
        nb = F.shape[1]
        core = F[0, nb // 20: 19 * nb // 20]
        w = _kept_weight(x, wl, det, al[0], de[0], f1[0], "nearest")
        ratios.append(core.mean() / (2.0 * w))
        shapes.append(4.0 * core[::3] / core.mean())  # 2F normalised to mean 4; bins 3 apart
    ratios = np.array(ratios)
    sem = ratios.std(ddof=1) / math.sqrt(len(ratios))
    assert abs(ratios.mean() - 1.0) < max(4 * sem, 0.005) and abs(ratios.mean() - 1.0) < 0.03
    # shape: 2F ~ chi^2 with 4 degrees of freedom
    assert kstest(np.concatenate(shapes), chi2(4).cdf).pvalue > 1e-4


def test_noise_free_injection_peaks_at_injected_bin(fs):
    wl = W.WORKLOADS["small"]
    det = W.detector_for(wl)
    inj = W.injections(wl, on_bin=True)[0]
    x = orsp.inject(wl.n, wl.dt, [inj], wl.fl, det, wl.sigma)
    F, *_ = _run(fs, wl, det, x, np.array([inj.alpha]), np.array([inj.delta]), np.array([inj.f1]), thr=1e9)
    k0 = int(round(inj.f0 * wl.nfft * wl.dt))
    assert abs(int(np.argmax(F[0])) - k0) <= 1
    # F = rho^2/2 up to the resampling approximation and the samples lost at the edges
    assert abs(F[0].max() / (inj.snr ** 2 / 2) - 1.0) < 0.02


# ------------------------------------------------------------------ edge cases and errors

def test_nonfinite_input_is_reported(fs):
    wl, det, x, alpha, delta, f1 = make_case("tiny")
    x = x.copy()
    x[17] = np.nan
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    assert ctx.sync_status() == 4  # FS_ERR_NONFINITE
    assert ctx.sync_status() == 0  # cleared after reading


def test_candidate_overflow_counts_exactly(fs):
    wl, det, x, alpha, delta, f1 = make_case("tiny")
    F, (cs, *_), ncand, status = _run(fs, wl, det, x, alpha, delta, f1, thr=3.0, cand_cap=5)
    assert status == 3  # FS_ERR_CAPACITY
    assert ncand == int(np.sum(F > 3.0)) and ncand > 5
    assert len(cs) == 5


def test_argument_errors(fs):
    wl, det, x, alpha, delta, f1 = make_case("tiny")
    ctx = fs.Context(det)
    xd = _dev(x, torch.float32)
    with pytest.raises(fs.FstatError) as e:
        fs.Segment(ctx, xd, wl.dt, 3000, wl.fl, wl.S0)  # not a power of two
    assert e.value.status == 2
    with pytest.raises(fs.FstatError) as e:
        fs.Segment(ctx, xd, -1.0, wl.nfft, wl.fl, wl.S0)
    assert e.value.status == 1
    with pytest.raises(fs.FstatError) as e:
        fs.Segment(ctx, xd, wl.dt, 1 << 22, wl.fl, wl.S0)  # transforms up to 2^21
    assert e.value.status == 2
    seg = fs.Segment(ctx, xd, wl.dt, wl.nfft, wl.fl, wl.S0)
    with pytest.raises(fs.FstatError) as e:
        fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), 10.0, nbins=wl.nfft // 4)
    assert e.value.status == 2


@pytest.mark.parametrize("name", ["grid_2d", "grid_2d_ib", "wide_6d"])
def test_full_configuration_sampled(fs, name):
    """The benchmark's launch configuration (all 256 skies x 16 spindowns in one sky
    group, the persistent queue sized as the bench sizes it): sampled template rows
    against the oracle (FFT mode) and their candidates; for all templates the count of
    crossings equals the number of F values above threshold, and every template's F
    (the 6-day 2^21 grid: every 32nd sky's) agrees with the plain FP64 form."""
    wl = W.WORKLOADS[name]
    det = W.detector_for(wl)
    x = (W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)).astype(np.float32)
    alpha, delta = W.sky_grid(wl.nsky)
    f1 = W.spin_grid(wl.nspin, *wl.f1_range)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, interbin=wl.interbin)
    res = fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), wl.F_thr, cand_cap=1 << 20)
    assert ctx.sync_status() == 0
    F = res.F
    assert F.shape == (wl.nsky * wl.nspin, wl.nbins)
    assert bool(torch.isfinite(F).all()) and float(F.min()) >= 0.0
    n = int(res.n_cand.item())
    assert n == int((F > wl.F_thr).sum().item())
    sky, spin, bins, Fc = res.candidates()
    g = np.random.default_rng(5)
    picks = sorted({0, wl.nsky * wl.nspin - 1, *g.integers(0, wl.nsky * wl.nspin, 4).tolist()})
    so = ors.Segment(x.astype(np.float64), wl.dt)
    for t in picks:
        s, m = divmod(t, wl.nspin)
        if wl.interbin:
            ref = ofs.fstat_interbinned(so, alpha[s], delta[s], f1[m], wl.fl, det, wl.S0, wl.nfft)
        else:
            ref = ofs.fstat(so, alpha[s], delta[s], f1[m], wl.fl, det, wl.S0, wl.nfft)
        row = F[t].double().cpu().numpy()
        assert max_rel_dF(row, ref) <= F32_TOL, (t, max_rel_dF(row, ref))
        mine = (sky == s) & (spin == m)
        missing, bad = check_candidates(np.zeros(mine.sum(), dtype=np.int64), np.zeros(mine.sum(), dtype=np.int64),
                                        bins[mine], Fc[mine], ref[None, :], wl.F_thr, 1)
        assert not missing and not bad, (t, missing, bad)
    # every template (the 2^21 grid: every 32nd sky) against the plain FP64 form on the
    # same GPU, itself parity-tested against the oracle at 1e-8, by chunks of skies
    seg64 = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, precision="f64",
                       interbin=wl.interbin)
    skies = np.arange(0, wl.nsky, 32 if wl.nfft > (1 << 20) else 1)
    per = max(1, (1 << 28) // (wl.nspin * wl.nbins * 8))
    worst = 0.0
    for c0 in range(0, skies.size, per):
        sk = skies[c0:c0 + per]
        r64 = fs.search(ctx, seg64, _dev(alpha[sk]), _dev(delta[sk]), _dev(f1), 1e30, cand_cap=1)
        rows = torch.as_tensor((sk[:, None] * wl.nspin + np.arange(wl.nspin)[None, :]).ravel(), device="cuda")
        d = ((F[rows].double() - r64.F).abs() / torch.clamp(r64.F, min=1.0)).max().item()
        worst = max(worst, d)
    assert ctx.sync_status() == 0
    assert worst <= F32_TOL, worst
    seg64.close()
    seg.close()
    ctx.close()


def test_bounded_wait_runs_out_and_the_context_recovers(fs):
    """A wait of the persistent queue on a counter that nothing increments runs out
    after its iteration bound, latches FS_ERR_TIMEOUT for the host and returns; the
    same context then searches normally."""
    import time
    wl, det, x, alpha, delta, f1 = make_case("tiny")
    ctx = fs.Context(det)
    t0 = time.perf_counter()
    ctx.selftest_wait()
    assert ctx.sync_status() == 6          # FS_ERR_TIMEOUT
    elapsed = time.perf_counter() - t0
    assert elapsed < 120.0
    print("bounded wait ran out after %.1f s" % elapsed)
    assert ctx.sync_status() == 0          # cleared by the read
    seg = fs.Segment(ctx, _dev(x.astype(np.float32), torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    res = fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), wl.F_thr)
    assert ctx.sync_status() == 0
    ref = oracle_F(x.astype(np.float32).astype(np.float64), wl, det, alpha, delta, f1)
    assert max_rel_dF(res.F.double().cpu().numpy(), ref) < F32_TOL
    seg.close()
    ctx.close()
