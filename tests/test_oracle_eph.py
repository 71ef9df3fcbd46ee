"""Pins of the oracle's tabulated detector position (the ephemeris table that
stands in for the files of Sec. V): the interpolation rule against its error
bound, the analytic velocity against finite differences, and the zero table,
which removes the Doppler and leaves F as the plain zero-padded DFT of
x a exp(-2 pi i f1 t^2/2) (Eqs. OS, Fab with phi_m = 0)."""
import math

import numpy as np
import pytest

from oracle import earth, fstat as ofs, refine as orf, resample as ors, response as orsp
from paper_1003_0844_gb300 import workloads as W


def _perturbed_table(n, dt, det):
    """Analytic positions plus a constant offset and a uniform drift (an SSB
    frame that differs from the analytic one), with the matching velocity."""
    c0 = np.array([3.0, -2.0, 1.5])[:, None]
    c1 = np.array([2e-6, -1e-6, 5e-7])[:, None]
    return earth.tabulate(n, dt, det, r_fn=lambda t: earth.detector_position_ls(t, det) + c0 + c1 * t,
                          v_fn=lambda t: earth.detector_velocity_ls(t, det) + c1)


def test_velocity_is_the_derivative_of_the_position():
    det = W.detector_for(W.WORKLOADS["tiny"])
    t = np.linspace(0.0, 3 * 86400.0, 97)
    h = 5.0    # truncation (third derivative) h^2/6 ~ 3.5e-14, rounding spacing(500)/(2h) ~ 1e-14
    fd = (earth.detector_position_ls(t + h, det) - earth.detector_position_ls(t - h, det)) / (2 * h)
    v = earth.detector_velocity_ls(t, det)
    assert np.abs(fd - v).max() <= 2e-13


@pytest.mark.parametrize("dt", [2.0, 64.0])
def test_table_interpolation_error_bound(dt):
    """Inside the grid the linear extrapolation from the nearest point differs from
    the analytic delay by at most |r''| dt^2 / 8, |r''| <= (AU Omega_o^2 + r_e Omega_r^2)/c."""
    det = W.detector_for(W.WORKLOADS["tiny"])
    n = int(86400 / dt)
    tab = earth.tabulate(n, dt, det)
    r_e, _ = earth.site_equatorial_radius_and_z(det.lat)
    acc = (earth.AU_M * earth.OMEGA_O ** 2 + r_e * earth.OMEGA_R ** 2) / earth.C_LIGHT
    bound = acc * dt * dt / 8.0
    t = np.random.default_rng(5).uniform(0.0, (n - 1) * dt, 20000)
    for a, d in [(0.3, 0.2), (2.5, -1.1), (4.0, 1.4)]:
        err = np.abs(earth.phi_m(t, a, d, tab) - earth.phi_m(t, a, d, det))
        assert err.max() <= bound * 1.001 + 1e-12
        assert err.max() >= 0.05 * bound       # the rule is linear, not exact
    # on the grid points the table is exact
    tg = np.arange(0, n, 7) * dt
    assert np.abs(earth.phi_m(tg, 0.3, 0.2, tab) - earth.phi_m(tg, 0.3, 0.2, det)).max() < 1e-12


def test_table_clamps_to_the_end_points():
    det = W.detector_for(W.WORKLOADS["tiny"])
    tab = _perturbed_table(100, 10.0, det)
    t = np.array([-300.0, -4.9, 990.0 + 250.0])
    p = tab.position(t)
    assert np.allclose(p[:, 0], tab.r[:, 0] - 300.0 * tab.v[:, 0], rtol=0, atol=1e-12)
    assert np.allclose(p[:, 1], tab.r[:, 0] - 4.9 * tab.v[:, 0], rtol=0, atol=1e-12)
    assert np.allclose(p[:, 2], tab.r[:, 99] + 250.0 * tab.v[:, 99], rtol=0, atol=1e-12)


def test_zero_table_is_the_plain_dft():
    """phi_m = 0: source times equal the output times, the spline returns the
    samples, no heterodyne, and F_k is 2/(S0 To) dt^2 (|sum x a c e_k|^2/<a^2> +
    |sum x b c e_k|^2/<b^2>) with c = exp(-2 pi i f1 t^2/2), e_k = exp(-2 pi i jk/Nfft)."""
    wl = W.WORKLOADS["tiny"]
    det = W.detector_for(wl)
    n, dt = wl.n, wl.dt
    tab = earth.TabulatedDetector(det, np.zeros((3, n)), np.zeros((3, n)), dt)
    x = W.noise(wl) + orsp.inject(n, dt, W.injections(wl), wl.fl, det, wl.sigma)
    seg = ors.Segment(x, dt)
    a_, d_, f1 = 1.3, -0.7, -3e-9
    F = ofs.fstat(seg, a_, d_, f1, wl.fl, tab, wl.S0, wl.nfft)
    t = np.arange(n) * dt
    a, b = orsp.ab(t, a_, d_, det)
    c = np.exp(-2j * math.pi * f1 * t * t / 2)
    ks = np.arange(0, wl.nfft // 2, 37)
    E = np.exp(-2j * math.pi * np.outer(ks, np.arange(n)) / wl.nfft)
    Fa, Fb = dt * (E @ (x * a * c)), dt * (E @ (x * b * c))
    ref = 2.0 / (wl.S0 * n * dt) * (np.abs(Fa) ** 2 / np.mean(a * a) + np.abs(Fb) ** 2 / np.mean(b * b))
    assert np.allclose(F[ks], ref, rtol=1e-9, atol=1e-9 * ref.max())
    # the exact F of the fine search at the same points (f0 = k / (Nfft dt)) agrees
    for k in ks[:4]:
        Fp = orf.fstat_point(x, dt, (k / (wl.nfft * dt), f1, a_, d_), wl.fl, tab, wl.S0)
        assert Fp == pytest.approx(F[k], rel=1e-9, abs=1e-9 * ref.max())


def test_table_of_the_analytic_model_gives_the_analytic_F():
    """dt = 8 s: the delay error of the table (< 1e-9 s) moves F by far less
    than the FP32 path's tolerance."""
    wl = W.WORKLOADS["small"]
    det = W.detector_for(wl)
    tab = earth.tabulate(wl.n, wl.dt, det)
    x = W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)
    seg = ors.Segment(x, wl.dt)
    F0 = ofs.fstat(seg, 0.9, 0.4, -2e-9, wl.fl, det, wl.S0, wl.nfft)
    F1 = ofs.fstat(seg, 0.9, 0.4, -2e-9, wl.fl, tab, wl.S0, wl.nfft)
    assert np.max(np.abs(F1 - F0) / np.maximum(F0, 1.0)) < 1e-6


def test_perturbed_table_moves_the_signal():
    """A table in a shifted, drifting frame is not the analytic one: the F of an
    injection made with the table peaks with the table, not with the analytic model."""
    wl = W.WORKLOADS["small"]
    det = W.detector_for(wl)
    tab = _perturbed_table(wl.n, wl.dt, det)
    inj = W.injections(wl, on_bin=True)[0]
    x = orsp.inject(wl.n, wl.dt, [inj], wl.fl, tab, wl.sigma)
    seg = ors.Segment(x, wl.dt)
    k = int(round(inj.f0 * wl.nfft * wl.dt))
    bins = [k]
    Ft = ofs.fstat(seg, inj.alpha, inj.delta, inj.f1, wl.fl, tab, wl.S0, wl.nfft, bins=bins)[0]
    Fa = ofs.fstat(seg, inj.alpha, inj.delta, inj.f1, wl.fl, det, wl.S0, wl.nfft, bins=bins)[0]
    assert Ft > 2.0 * Fa
