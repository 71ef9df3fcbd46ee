"""The coarse search's F at continuous points and its gradient (the adjoint kernel,
through the C ABI) against the oracle's FP64 restatement, against the search's own
F map on the Fourier grid, and through the autograd wrapper."""
import numpy as np
import pytest
import torch

from oracle import adjoint as oad
from oracle import refine as orf
from oracle import resample as ors
from oracle import response as orsp
from paper_1003_0844_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# FP32 arithmetic with double-float phases, as the coarse search: F within 1e-4 of
# max(F, 1) (the coarse path's bound); each gradient component within 1e-4 of the sum
# of the magnitudes of the terms it is made of (its size before they cancel near a
# maximum), i.e. the same relative precision carried through the quotient rule.
F_TOL = 1e-4
G_TOL = 1e-4


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


def _case(name="small", snr=25.0):
    wl = W.WORKLOADS[name]
    det = W.detector_for(wl)
    inj = W.Injection(f0=0.0213 if name == "small" else 0.1234, f1=-4e-9, alpha=2.1, delta=0.45, psi=0.3,
                      cos_iota=0.4, phi0=1.1, snr=snr)
    x = orsp.inject(wl.n, wl.dt, [inj], wl.fl, det, wl.sigma) + W.noise(wl)
    theta = np.array([inj.f0, inj.f1, inj.alpha, inj.delta])
    return wl, det, x.astype(np.float32), theta


def _points(wl, det, x, th):
    _, _, G0 = orf.fstat_point(x.astype(np.float64), wl.dt, th, wl.fl, det, wl.S0, grad=True)
    width = 1.0 / np.sqrt(np.diag(G0))
    offs = np.array([[0, 0, 0, 0], [0.7, -0.4, 0.3, 0.5], [-1.5, 0.8, -0.6, 0.2], [3.0, 2.0, -2.0, -1.0],
                     [0.1, 0.1, 5.0, -4.0]])
    return th + offs * width


@pytest.mark.parametrize("name", ["small", "grid_2d"])
def test_F_and_gradient_match_oracle(fs, name):
    wl, det, x, th = _case(name)
    P = _points(wl, det, x, th)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    F = fs.fstat_resampled(ctx, seg, _dev(P))
    F2, g = fs.fstat_resampled_grad(ctx, seg, _dev(P))
    assert ctx.sync_status() == 0
    assert torch.equal(F, F2)  # the same sums in both calls
    F, g = F.cpu().numpy(), g.cpu().numpy()
    oseg = ors.Segment(x.astype(np.float64), wl.dt)  # the samples the segment holds
    for p in range(len(P)):
        Fr, gr, scale = oad.resampled_fstat_point(oseg, P[p], wl.fl, det, wl.S0, grad=True)
        assert abs(F[p] - Fr) <= F_TOL * max(Fr, 1.0), (p, F[p], Fr)
        assert np.all(np.abs(g[p] - gr) <= G_TOL * scale), (p, g[p], gr, scale)


def test_segment_epoch(fs):
    """A segment starting t0 after the detector's t = 0 (Sec. V: orbital and sidereal
    angles at its first sample): the adjoint against the oracle on the detector at
    that epoch."""
    from oracle import earth as oe
    wl, det, x, th = _case("small")
    t0 = 123456.7
    P = _points(wl, oe.detector_at_epoch(det, t0), x, th)[:3]
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, t0=t0)
    F, g = fs.fstat_resampled_grad(ctx, seg, _dev(P))
    assert ctx.sync_status() == 0
    F, g = F.cpu().numpy(), g.cpu().numpy()
    oseg = ors.Segment(x.astype(np.float64), wl.dt)
    for p in range(len(P)):
        Fr, gr, scale = oad.resampled_fstat_point(oseg, P[p], wl.fl, oe.detector_at_epoch(det, t0), wl.S0, grad=True)
        assert abs(F[p] - Fr) <= F_TOL * max(Fr, 1.0), (p, F[p], Fr)
        assert np.all(np.abs(g[p] - gr) <= G_TOL * scale), (p, g[p], gr, scale)


def test_on_the_fourier_grid_it_is_the_searchs_F(fs):
    """Points at f0 = k / (Nfft dt) with the templates of a search: F equals the
    search's F map at bin k (the transform and the direct sum are two routes to the
    same zero-padded DFT, Eq. eq:DFT)."""
    wl, det, x, th = _case("small")
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    alpha, delta = np.array([th[2], 1.0]), np.array([th[3], -0.3])
    f1 = np.array([th[1], 0.0])
    res = fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), F_thr=1e30, cand_cap=1)
    Fmap = res.F.cpu().numpy()  # [nsky * nspin, nbins]
    k0 = int(round(th[0] * wl.nfft * wl.dt))
    bins = np.array([1, k0 - 3, k0, k0 + 1, wl.nfft // 2 - 2])
    P, ref = [], []
    for s in range(2):
        for m in range(2):
            for k in bins:
                P.append([k / (wl.nfft * wl.dt), f1[m], alpha[s], delta[s]])
                ref.append(Fmap[s * 2 + m, k])
    F = fs.fstat_resampled(ctx, seg, _dev(np.array(P))).cpu().numpy()
    ref = np.array(ref)
    assert np.all(np.abs(F - ref) <= F_TOL * np.maximum(ref, 1.0)), np.max(np.abs(F - ref) / np.maximum(ref, 1.0))
    assert ref.max() > 100.0  # the injected template's bin


def test_autograd_backward_is_the_adjoint_call(fs):
    wl, det, x, th = _case("small")
    P = _dev(_points(wl, det, x, th))
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    pts = P.clone().requires_grad_(True)
    F = fs.fstat_resampled_at(ctx, seg, pts)
    w = torch.linspace(0.5, 2.0, F.numel(), dtype=torch.float64, device="cuda")
    (F * w).sum().backward()
    F1, g1 = fs.fstat_resampled_grad(ctx, seg, P)
    _, gw = fs.fstat_resampled_grad(ctx, seg, P, gF=w)
    assert torch.equal(F.detach(), F1)
    assert torch.equal(pts.grad, gw)
    assert torch.allclose(gw, w[:, None] * g1, rtol=1e-14, atol=0.0)


def test_gradient_against_differences_on_the_gpu(fs):
    """Central differences of the GPU's own F along each coordinate, steps of 0.05 of a
    correlation width: FP32 rounding of F (~1e-5 F) bounds their precision to ~1e-3 F
    per width, enough to catch a wrong term or sign."""
    wl, det, x, th = _case("small")
    _, _, G0 = orf.fstat_point(x.astype(np.float64), wl.dt, th, wl.fl, det, wl.S0, grad=True)
    width = 1.0 / np.sqrt(np.diag(G0))
    p0 = th + np.array([0.4, -0.3, 0.3, -0.2]) * width
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    F0, g = fs.fstat_resampled_grad(ctx, seg, _dev(p0[None, :]))
    F0, g = float(F0[0]), g[0].cpu().numpy()
    P = []
    for i in range(4):
        for s in (1, -1):
            q = p0.copy()
            q[i] += s * 0.05 * width[i]
            P.append(q)
    Fd = fs.fstat_resampled(ctx, seg, _dev(np.array(P))).cpu().numpy()
    for i in range(4):
        fd = (Fd[2 * i] - Fd[2 * i + 1]) / (0.1 * width[i])
        assert abs(fd - g[i]) <= 5e-3 * F0 / width[i] + 1e-2 * abs(g[i]), (i, fd, g[i])


@pytest.mark.parametrize("kind", ["f64", "nearest", "table"])
def test_unsupported_segments_are_refused(fs, kind):
    wl, det, x, th = _case("small")
    ctx = fs.Context(det)
    if kind == "f64":
        seg = fs.Segment(ctx, _dev(x.astype(np.float64)), wl.dt, wl.nfft, wl.fl, wl.S0, precision="f64")
    elif kind == "nearest":
        seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, interp="nearest")
    else:
        from oracle import earth as oe
        tab = oe.tabulate(wl.n, wl.dt, det)
        seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0,
                         eph=(_dev(tab.r), _dev(tab.v)))
    with pytest.raises(fs.FstatError) as e:
        fs.fstat_resampled(ctx, seg, _dev(th[None, :]))
    assert e.value.status == 7
    with pytest.raises(fs.FstatError):
        fs.fstat_resampled_grad(ctx, seg, _dev(th[None, :]))


def test_gradient_ascent_never_lowers_F(fs):
    """fs_refine_resampled on the 1-day case: F never decreases with more steps, the
    returned F is the F at the returned point, and the oracle agrees there."""
    wl, det, x, th = _case("small")
    _, _, G0 = orf.fstat_point(x.astype(np.float64), wl.dt, th, wl.fl, det, wl.S0, grad=True)
    width = 1.0 / np.sqrt(np.diag(G0))
    starts = th + width * np.array([[0.9, -0.8, 0.7, -0.6], [-0.5, 0.6, 0.4, 0.9], [0.3, 0.3, -0.8, -0.2]])
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    prev = fs.fstat_resampled(ctx, seg, _dev(starts)).cpu().numpy()
    for k in (1, 2, 4, 8, 20):
        out, Fk = fs.refine_resampled(ctx, seg, _dev(starts), nsteps=k)
        Fk = Fk.cpu().numpy()
        assert np.all(Fk >= prev)
        prev = Fk
    assert ctx.sync_status() == 0
    assert np.array_equal(prev, fs.fstat_resampled(ctx, seg, out).cpu().numpy())
    oseg = ors.Segment(x.astype(np.float64), wl.dt)
    out = out.cpu().numpy()
    for p in range(len(starts)):
        Fr = oad.resampled_fstat_point(oseg, out[p], wl.fl, det, wl.S0)
        assert abs(prev[p] - Fr) <= F_TOL * Fr, (p, prev[p], Fr)


def test_gradient_ascent_reaches_the_simplex_maximum(fs):
    """The 2-day series of the differentiation workload: from three starts up to a
    correlation width away, 20 quasi-Newton steps reach the oracle's simplex maximum of
    the resampled F to 1e-3 of F, i.e. (F(theta + tau) ~ F (1 - tau^T G tau), Eq.
    TaylorC2) to about 0.03 of a correlation length; near the peak the FP32 rounding of
    F (~1e-5) decides the last accepted steps."""
    wl, det, x, th = _case("grid_2d")
    _, _, G0 = orf.fstat_point(x.astype(np.float64), wl.dt, th, wl.fl, det, wl.S0, grad=True)
    width = 1.0 / np.sqrt(np.diag(G0))
    starts = th + width * np.array([[0.9, -0.8, 0.7, -0.6], [-0.5, 0.6, 0.4, 0.9], [0.3, 0.3, -0.8, -0.2]])
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    F0 = fs.fstat_resampled(ctx, seg, _dev(starts)).cpu().numpy()
    out, F = fs.refine_resampled(ctx, seg, _dev(starts), nsteps=20)
    assert ctx.sync_status() == 0
    out, F = out.cpu().numpy(), F.cpu().numpy()
    oseg = ors.Segment(x.astype(np.float64), wl.dt)
    _, Fb = oad.resampled_fine_search(oseg, starts[1], wl.fl, det, wl.S0, width)
    for p in range(len(starts)):
        assert F[p] > F0[p]
        assert F[p] >= Fb * (1 - 1e-3), (p, F[p], Fb)
        Fr = oad.resampled_fstat_point(oseg, out[p], wl.fl, det, wl.S0)
        assert abs(F[p] - Fr) <= F_TOL * Fr, (p, F[p], Fr)


def test_gradient_ascent_refuses_unsupported_segments(fs):
    wl, det, x, th = _case("small")
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x.astype(np.float64)), wl.dt, wl.nfft, wl.fl, wl.S0, precision="f64")
    with pytest.raises(fs.FstatError) as e:
        fs.refine_resampled(ctx, seg, _dev(th[None, :]), nsteps=2)
    assert e.value.status == 7


def test_six_day_segment(fs):
    """The 6-day, 0.5 s series of the wide-band workload (N = 1,033,968): two points
    against the oracle (phases to ~1e6 cycles in the heterodyne term)."""
    wl, det, x, th = _case("wide_6d")
    P = np.array([th, th + np.array([2e-7, 1e-10, 1e-4, -1e-4])])
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    F, g = fs.fstat_resampled_grad(ctx, seg, _dev(P))
    assert ctx.sync_status() == 0
    F, g = F.cpu().numpy(), g.cpu().numpy()
    oseg = ors.Segment(x.astype(np.float64), wl.dt)
    for p in range(len(P)):
        Fr, gr, scale = oad.resampled_fstat_point(oseg, P[p], wl.fl, det, wl.S0, grad=True)
        assert abs(F[p] - Fr) <= F_TOL * max(Fr, 1.0), (p, F[p], Fr)
        assert np.all(np.abs(g[p] - gr) <= G_TOL * scale), (p, g[p], gr, scale)


def test_interbinning_segment_gives_the_same_sums(fs):
    """The resampled series does not depend on the transform's options: a segment with
    interbinning (Eq. intbin) gives the same F and gradient bit for bit."""
    wl, det, x, th = _case("small")
    P = _dev(_points(wl, det, x, th))
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    seg_ib = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, interbin=True)
    F1, g1 = fs.fstat_resampled_grad(ctx, seg, P)
    F2, g2 = fs.fstat_resampled_grad(ctx, seg_ib, P)
    assert ctx.sync_status() == 0
    assert torch.equal(F1, F2) and torch.equal(g1, g2)
