"""The caller's position table (fs_prepare_segment_eph, the ephemerides of Sec. V)
on the GPU against the oracle's TabulatedDetector: F on every bin of the FP32
and FP64 searches and the candidates, the fine search's exact F, gradient and
Hessian, a table of the analytic Earth against the analytic path, and the
table's validation."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import earth
from oracle import refine as orf
from oracle import resample as ors
from oracle import response as orsp
from paper_1003_0844_gb300 import workloads as W
from tests.helpers import F32_TOL, F64_TOL, check_candidates, max_rel_dF, oracle_F

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


def _perturbed(n, dt, det):
    """Analytic positions in a shifted, drifting frame (not the analytic model)."""
    c0 = np.array([3.0, -2.0, 1.5])[:, None]
    c1 = np.array([2e-6, -1e-6, 5e-7])[:, None]
    return earth.tabulate(n, dt, det, r_fn=lambda t: earth.detector_position_ls(t, det) + c0 + c1 * t,
                          v_fn=lambda t: earth.detector_velocity_ls(t, det) + c1)


def _case(name, nfft=None):
    wl = W.WORKLOADS[name]
    if nfft is not None:
        wl = dataclasses.replace(wl, nfft=nfft)
    det = W.detector_for(wl)
    tab = _perturbed(wl.n, wl.dt, det)
    # signals that follow the table, so the candidates come from the table's delays
    x = W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, tab, wl.sigma)
    alpha, delta = W.sky_grid(wl.nsky)
    f1 = W.spin_grid(wl.nspin, *wl.f1_range)
    return wl, det, tab, x, alpha, delta, f1


def _eph(tab):
    return _dev(tab.r), _dev(tab.v)


@pytest.mark.parametrize("name,nfft,precision", [("tiny", None, "f32"), ("small", None, "f32"),
                                                   ("small", 1 << 15, "f32"), ("tiny", None, "f64")])
def test_search_with_table_matches_oracle(fs, name, nfft, precision):
    wl, det, tab, x, alpha, delta, f1 = _case(name, nfft)
    x32 = x.astype(np.float32)
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x32, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, precision=precision,
                     eph=_eph(tab))
    res = fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), wl.F_thr)
    assert ctx.sync_status() == 0
    F = res.F.double().cpu().numpy()
    ref = oracle_F(x32.astype(np.float64), wl, tab, alpha, delta, f1)
    tol = F32_TOL if precision == "f32" else F64_TOL
    assert max_rel_dF(F, ref) <= tol
    sky, spin, bins, Fc = res.candidates()
    missing, bad = check_candidates(sky, spin, bins, Fc, ref, wl.F_thr, len(f1))
    assert not missing and not bad
    assert ref.max() > wl.F_thr   # the injections are found with the table
    seg.close()
    ctx.close()


def test_table_of_the_analytic_earth_matches_the_analytic_path(fs):
    """dt = 8 s: the table's extrapolation error (< 1e-9 s) is far inside the FP32 tolerance."""
    wl = W.WORKLOADS["small"]
    det = W.detector_for(wl)
    tab = earth.tabulate(wl.n, wl.dt, det)
    x = (W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)).astype(np.float32)
    alpha, delta = W.sky_grid(wl.nsky)
    f1 = W.spin_grid(wl.nspin, *wl.f1_range)
    ctx = fs.Context(det)
    out = []
    for eph in (None, _eph(tab)):
        seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0, eph=eph)
        out.append(fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), wl.F_thr).F.double().cpu().numpy())
        seg.close()
    assert ctx.sync_status() == 0
    assert max_rel_dF(out[1], out[0]) <= 2e-5
    ctx.close()


def test_fine_search_with_table_matches_oracle(fs):
    wl = W.WORKLOADS["small"]
    det = W.detector_for(wl)
    tab = _perturbed(wl.n, wl.dt, det)
    inj = W.Injection(f0=0.0213, f1=-4e-9, alpha=2.1, delta=0.45, psi=0.3, cos_iota=0.4, phi0=1.1, snr=25.0)
    x = W.noise(wl) + orsp.inject(wl.n, wl.dt, [inj], wl.fl, tab, wl.sigma)
    th = np.array([inj.f0, inj.f1, inj.alpha, inj.delta])
    _, _, G0 = orf.fstat_point(x, wl.dt, th, wl.fl, tab, wl.S0, grad=True)
    wd0 = 1.0 / np.sqrt(np.diag(G0))
    P = th + np.array([[0, 0, 0, 0], [0.7, -0.4, 0.3, 0.5], [-1.5, 0.8, -0.6, 0.2]]) * wd0
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x), wl.dt, wl.nfft, wl.fl, wl.S0, precision="f64", eph=_eph(tab))
    F, g, m, h = fs.fstat_points(ctx, seg, _dev(P), grad=True, metric=True, hess=True)
    assert ctx.sync_status() == 0
    F, g, m, h = F.cpu().numpy(), g.cpu().numpy(), m.cpu().numpy(), h.cpu().numpy()
    iu = np.triu_indices(4)
    for p in range(len(P)):
        Fr, gr, Gr, Hr = orf.fstat_point(x, wl.dt, P[p], wl.fl, tab, wl.S0, grad=True, hess=True)
        wd = 1.0 / np.sqrt(np.diag(Gr))
        assert abs(F[p] - Fr) <= 1e-9 * max(Fr, 1.0), (p, F[p], Fr)
        assert np.all(np.abs(g[p] - gr) <= 1e-7 * np.abs(gr) + 1e-8 * max(Fr, 1.0) / wd), (p, g[p], gr)
        scale = np.sqrt(np.outer(np.diag(Gr), np.diag(Gr)))[iu]
        assert np.all(np.abs(m[p] - Gr[iu]) <= 1e-9 * scale), (p, m[p], Gr[iu])
        hs = (max(Fr, 1.0) / np.outer(wd, wd))[iu]
        assert np.all(np.abs(h[p] - Hr[iu]) <= 1e-7 * np.abs(Hr[iu]) + 1e-8 * hs), (p, h[p], Hr[iu])
    # the climb from a displaced point reaches the table's maximum, not the analytic one
    _, Fc = fs.refine(ctx, seg, _dev(P[1:2]), nsteps=20)
    assert float(Fc.cpu()[0]) >= 0.95 * orf.fstat_point(x, wl.dt, th, wl.fl, tab, wl.S0)
    seg.close()
    ctx.close()


@pytest.mark.parametrize("bad", ["nan", "far"])
def test_invalid_table_latches_nonfinite(fs, bad):
    wl = W.WORKLOADS["tiny"]
    det = W.detector_for(wl)
    tab = earth.tabulate(wl.n, wl.dt, det)
    r = tab.r.copy()
    r[1, wl.n // 3] = np.nan if bad == "nan" else 700.0
    ctx = fs.Context(det)
    x = _dev(W.noise(wl), torch.float32)
    seg = fs.Segment(ctx, x, wl.dt, wl.nfft, wl.fl, wl.S0, eph=(_dev(r), _dev(tab.v)))
    assert ctx.sync_status() == 4   # FS_ERR_NONFINITE
    seg.close()
    ctx.close()


def test_table_arguments_are_checked(fs):
    wl = W.WORKLOADS["tiny"]
    det = W.detector_for(wl)
    ctx = fs.Context(det)
    x = _dev(W.noise(wl), torch.float32)
    r = torch.zeros((3, wl.n), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        fs.Segment(ctx, x, wl.dt, wl.nfft, wl.fl, wl.S0, eph=(r[:, :-1].contiguous(), r))
    with pytest.raises(ValueError):
        fs.Segment(ctx, x, wl.dt, wl.nfft, wl.fl, wl.S0, eph=(r.float(), r))
    ctx.close()
