"""Pins of the resampled F at continuous points and of its gradient (the adjoint's
oracle): the coarse search's FFT F on the Fourier grid, the spline's slope against
scipy, the source times' sky derivatives and every sum's derivative against finite
differences, and reduced cases that isolate the small terms."""
import math

import numpy as np
import pytest

from oracle import adjoint as oad
from oracle import earth as oe
from oracle import fstat as ofs
from oracle import refine as orf
from oracle import resample as ors
from oracle import response as orsp
from paper_1003_0844_gb300 import workloads as W


def _case(noise=True, snr=25.0):
    wl = W.WORKLOADS["small"]
    det = W.detector_for(wl)
    inj = W.Injection(f0=0.0213, f1=-4e-9, alpha=2.1, delta=0.45, psi=0.3, cos_iota=0.4, phi0=1.1, snr=snr)
    x = orsp.inject(wl.n, wl.dt, [inj], wl.fl, det, wl.sigma)
    if noise:
        x = x + W.noise(wl)
    theta = np.array([inj.f0, inj.f1, inj.alpha, inj.delta])
    return wl, det, ors.Segment(x, wl.dt), x, theta


def _widths(wl, det, x, theta):
    """Correlation widths of F along each coordinate (1/sqrt(G_ii) of the reduced Fisher
    matrix, Eq. redFm-def): the natural step scale for differences."""
    _, _, G = orf.fstat_point(x, wl.dt, theta, wl.fl, det, wl.S0, grad=True)
    return 1.0 / np.sqrt(np.diag(G))


def test_on_the_fourier_grid_it_is_the_coarse_searchs_F():
    """f0 = k / (Nfft dt): the single-frequency sum is the zero-padded DFT at bin k, here
    against the FFT route of the coarse-search oracle (Eq. eq:DFT)."""
    wl, det, seg, _, th = _case()
    Fmap = ofs.fstat(seg, th[2], th[3], th[1], wl.fl, det, wl.S0, wl.nfft)
    k0 = int(round(th[0] * wl.nfft * wl.dt))
    for k in (3, k0 - 1, k0, k0 + 2, wl.nfft // 2 - 5):
        F = oad.resampled_fstat_point(seg, (k / (wl.nfft * wl.dt), th[1], th[2], th[3]), wl.fl, det, wl.S0)
        assert abs(F - Fmap[k]) <= 1e-9 * Fmap[k] + 1e-12, (k, F, Fmap[k])
    # and the injected signal's F is large there
    assert Fmap[k0] > 100.0


def test_spline_slope_matches_scipy():
    interp = pytest.importorskip("scipy.interpolate")
    g = np.random.default_rng(3)
    x = g.standard_normal(257)
    seg = ors.Segment(x, 2.0)
    cs = interp.CubicSpline(np.arange(seg.x2.size) * 1.0, seg.x2, bc_type="natural")
    t = np.concatenate([g.uniform(0.0, (seg.n - 1) * seg.dt, 500), [0.0, 1.0, (seg.n - 1) * seg.dt]])
    ref = cs(2.0 * t / seg.dt, 1) * (2.0 / seg.dt)
    assert np.max(np.abs(seg.interpolate_derivative(t) - ref)) <= 1e-12 * np.max(np.abs(ref))
    out = np.array([-0.5, (seg.n - 1) * seg.dt + 0.5])
    assert np.all(seg.interpolate_derivative(out) == 0.0)


def test_source_time_sky_derivatives_match_differences():
    wl, det, _, _, th = _case()
    tau = np.arange(0, wl.n, 97, dtype=np.float64) * wl.dt
    a, d = th[2], th[3]
    t = ors.source_times(tau, a, d, det)
    t_a, t_d = oad.source_time_sky_derivatives(t, a, d, det)
    h = 1e-5
    fa = (ors.source_times(tau, a + h, d, det) - ors.source_times(tau, a - h, d, det)) / (2 * h)
    fd = (ors.source_times(tau, a, d + h, det) - ors.source_times(tau, a, d - h, det)) / (2 * h)
    # truncation h^2 t''' / 6 ~ 1e-10 s; rounding ~ 1e-12 s / h ~ 1e-7 s on terms of ~500 s
    tol = 1e-6 * max(np.max(np.abs(t_a)), np.max(np.abs(t_d)))
    assert np.max(np.abs(fa - t_a)) <= tol
    assert np.max(np.abs(fd - t_d)) <= tol
    # the factor 1 / (1 + dphi/dt) (dphi/dt ~ 1e-4) is resolved: without it the check fails
    ca, sa, cd = math.cos(a), math.sin(a), math.cos(d)
    n0_a = oe.ecliptic_rotation(det.eps) @ np.array([-sa * cd, ca * cd, 0.0])
    assert np.max(np.abs(fa + n0_a @ oe.detector_position_ls(t, det))) > 10 * tol


def _fd5(fun, th, i, h):
    """Five-point central difference of fun along coordinate i (truncation h^4)."""
    e = np.zeros(4)
    e[i] = h
    return (-fun(th + 2 * e) + 8 * fun(th + e) - 8 * fun(th - e) + fun(th - 2 * e)) / (12 * h)


@pytest.mark.parametrize("offset", [0.0, 0.4])
def test_gradient_matches_central_differences(offset):
    wl, det, seg, x, th = _case()
    width = _widths(wl, det, x, th)
    th = th + offset * width * np.array([1.0, -0.7, 0.5, 0.8])
    F0, g, scale = oad.resampled_fstat_point(seg, th, wl.fl, det, wl.S0, grad=True)
    fun = lambda p: oad.resampled_fstat_point(seg, p, wl.fl, det, wl.S0)
    for i in range(4):
        fd = _fd5(fun, th, i, 1e-2 * width[i])
        assert abs(fd - g[i]) <= 1e-6 * scale[i], (i, fd, g[i], scale[i])


def test_every_sums_derivative_matches_differences():
    """Sa, Sb, <a^2>, <b^2> one by one, each against its own scale: the terms of da/dsky
    enter dSa at ~1e-6 of the phase terms, and <a^2>'s sky derivative carries the
    Omega_r dt/dsky term of da/dsky at a few per cent of its size."""
    wl, det, seg, x, th = _case()
    width = _widths(wl, det, x, th)
    r = oad.resampled_terms(seg, th, wl.fl, det, grad=True)
    # Sa itself turns with the heterodyne phase fl phi_m, ~2 pi fl |dt/dsky| ~ 1e6 rad per
    # radian of sky, far faster than |Sa|^2 varies: sky steps of 1e-4 widths
    for key, dkey in (("Sa", "dSa"), ("Sb", "dSb")):
        fun = lambda p, key=key: oad.resampled_terms(seg, p, wl.fl, det)[key]
        for i in range(4):
            fd = _fd5(fun, th, i, (1e-2 if i < 2 else 1e-4) * width[i])
            # the da/dsky terms are ~3e-4 |Sa| / width here: 10x above the bound
            assert abs(fd - r[dkey][i]) <= 2e-5 * abs(r[key]) / width[i], (key, i, fd, r[dkey][i])
    for key, dkey in (("A2", "dA2"), ("B2", "dB2")):
        assert r[dkey][0] == 0.0 and r[dkey][1] == 0.0  # no dependence on f0, f1
        fun = lambda p, key=key: oad.resampled_terms(seg, p, wl.fl, det)[key]
        for i in (2, 3):
            fd = _fd5(fun, th, i, 1e-3)
            assert abs(fd - r[dkey][i]) <= 1e-6 * abs(r[dkey][i]), (key, i, fd, r[dkey][i])
    # the Omega_r term is well above that tolerance: |Omega_r dt/dalpha| reaches a few 1e-2
    t = ors.source_times(np.arange(wl.n) * wl.dt, th[2], th[3], det)
    t_a, _ = oad.source_time_sky_derivatives(t, th[2], th[3], det)
    assert np.max(np.abs(oe.OMEGA_R * t_a)) > 0.02


def test_amplitude_terms_alone():
    """fl = 0, f1 = 0 and a constant series: the phase no longer depends on the sky and
    x~' = 0 inside the data, so dSa/dsky is the sum of da/dsky exp(-2 pi i f0 tau) alone;
    against differences of Sa."""
    wl, det, _, _, th = _case(noise=False)
    seg = ors.Segment(np.ones(wl.n), wl.dt)
    th0 = np.array([th[0], 0.0, th[2], th[3]])
    r = oad.resampled_terms(seg, th0, 0.0, det, grad=True)
    # no source time within reach of the data's ends (the series steps from 0 to 1 there)
    t = ors.source_times(np.arange(wl.n) * wl.dt, th[2], th[3], det)
    t_a, t_d = oad.source_time_sky_derivatives(t, th[2], th[3], det)
    h = 1e-5
    edge = np.minimum(np.abs(t), np.abs(t - (wl.n - 1) * wl.dt))
    assert np.all(edge > 3 * h * (np.abs(t_a) + np.abs(t_d)))
    for key, dkey in (("Sa", "dSa"), ("Sb", "dSb")):
        fun = lambda p, key=key: oad.resampled_terms(seg, p, 0.0, det)[key]
        for i in (2, 3):
            fd = _fd5(fun, th0, i, h)
            assert abs(fd - r[dkey][i]) <= 1e-8 * abs(r[dkey]).max() + 1e-9, (key, i, fd, r[dkey][i])
    # the spline of a constant is that constant
    assert np.max(np.abs(seg.interpolate_derivative(t[(t > 0) & (t < (wl.n - 1) * wl.dt)]))) < 1e-9


def test_caller_table_is_refused():
    wl, det, seg, _, th = _case(noise=False)
    tab = oe.tabulate(wl.n, wl.dt, det)
    with pytest.raises(NotImplementedError):
        oad.resampled_fstat_point(seg, th, wl.fl, tab, wl.S0, grad=True)


def test_resampled_F_near_the_injection():
    """Noise-free injection: at the injected parameters the resampled F is the exact F
    less the interpolation loss of Sec. VI.A (here ~2%), its gradient nearly vanishes
    there, and the simplex maximum stays within a per cent of the exact F's peak.
    (Over one day the f0-sky correlation makes a long, flat ridge: the maximum can
    sit many single-axis widths from the injection at nearly the same F.)"""
    wl, det, seg, x, th = _case(noise=False)
    width = _widths(wl, det, x, th)
    F, g, _ = oad.resampled_fstat_point(seg, th, wl.fl, det, wl.S0, grad=True)
    Fex = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0)
    assert 0.95 < F / Fex <= 1.0, (F, Fex)
    assert np.all(np.abs(g) * width < 2e-3 * F), g * width / F
    start = th + width * np.array([0.4, -0.3, 0.3, 0.2])
    best, Fb = oad.resampled_fine_search(seg, start, wl.fl, det, wl.S0, width)
    assert F <= Fb <= 1.01 * Fex, (F, Fb, Fex)
    _, gb, _ = oad.resampled_fstat_point(seg, best, wl.fl, det, wl.S0, grad=True)
    assert np.all(np.abs(gb) * width < 1e-3 * Fb), gb * width / Fb
