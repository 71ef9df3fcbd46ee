"""Pins for the CPU oracle: each test checks the oracle against something other
than itself (a textbook construction, a library routine, brute force, a closed
form or a number printed in the paper), chosen so that a dropped term, a wrong
sign or index or a transposed operand in the oracle fails one of them."""
import math

import numpy as np
import pytest

from oracle import earth, fstat, resample, response
from paper_1003_0844_gb300 import workloads as W
from tests.helpers import golden

DET = W.Detector(lambda_e0=1.234, theta_g0=0.3)


# --------------------------------------------------------------------------- Earth model (Sec. II, V)

def test_site_matches_textbook_geodetic_to_cartesian():
    # prime-vertical radius form: X = N cos(phi), Z = N (1 - e^2) sin(phi), N = a / sqrt(1 - e^2 sin^2 phi)
    for lat_deg in (0.0, 10.0, 43.63, 60.0, -35.0, 89.0):
        lat = math.radians(lat_deg)
        e2 = earth.ELL_FLAT * (2.0 - earth.ELL_FLAT)
        Nv = earth.ELL_A_M / math.sqrt(1.0 - e2 * math.sin(lat) ** 2)
        r_e, z = earth.site_equatorial_radius_and_z(lat)
        assert abs(r_e - Nv * math.cos(lat)) < 1e-6
        assert abs(z - Nv * (1.0 - e2) * math.sin(lat)) < 1e-6


def test_phi_m_scalar_product_equals_matrix_form():
    # the four-term scalar product of Sec. II against n0 (Eq. pha4) . r_d (Eq. pha5) in matrix form
    rng = np.random.default_rng(5)
    t = rng.uniform(-1e5, 6e5, 64)
    for _ in range(20):
        al, de = rng.uniform(0, 2 * math.pi), math.asin(rng.uniform(-1, 1))
        n0 = earth.sky_vector(al, de, DET.eps)
        rd = earth.detector_position_ls(t, DET)
        ref = n0 @ rd
        got = earth.phi_m(t, al, de, DET)
        assert np.max(np.abs(got - ref)) < 1e-12 * 500


def test_orbit_radius_speed_and_diurnal_speed():
    t = np.linspace(0, 86164.0, 7)
    r = earth.earth_orbit_ls(t, DET)
    assert np.allclose(np.linalg.norm(r, axis=0), 149_597_870_700.0 / 299_792_458.0, rtol=1e-14)
    h = 1.0
    v = (earth.earth_orbit_ls(t + h, DET) - earth.earth_orbit_ls(t - h, DET)) / (2 * h)
    # orbital speed / c: 2 pi AU / sidereal year / c ~ 9.93e-5
    assert np.allclose(np.linalg.norm(v, axis=0), 2 * math.pi * 499.00478383615643 / (365.25636 * 86400), rtol=1e-9)
    vs = (earth.site_equatorial_ls(t + h, DET) - earth.site_equatorial_ls(t - h, DET)) / (2 * h)
    r_e, _ = earth.site_equatorial_radius_and_z(DET.lat)
    # diurnal speed v0 = Omega_r r_e, directed East (Sec. V)
    assert np.allclose(np.linalg.norm(vs, axis=0), 7.2921151467e-5 * r_e / 299_792_458.0, rtol=1e-8)
    th = earth.sidereal_angle(t, DET)
    east = np.stack([-np.sin(th), np.cos(th), np.zeros_like(th)])
    assert np.allclose(np.sum(vs * east, axis=0), np.linalg.norm(vs, axis=0), rtol=1e-8)


# --------------------------------------------------------------------------- amplitude modulation (Sec. II)

def _tensor_beam_norm(t, al, de, det):
    """F+^2 + Fx^2 from the detector tensor d = (u u - v v)/2 of an L-shaped
    interferometer whose arms' bisector is at gamma from East; independent of
    the restated a, b formulas and of the polarisation-angle convention."""
    th = float(earth.sidereal_angle(t, det))
    l, g = det.lat, det.gamma
    E = np.array([-math.sin(th), math.cos(th), 0.0])
    N = np.array([-math.sin(l) * math.cos(th), -math.sin(l) * math.sin(th), math.cos(l)])
    u = math.cos(g + math.pi / 4) * E + math.sin(g + math.pi / 4) * N
    v = math.cos(g - math.pi / 4) * E + math.sin(g - math.pi / 4) * N
    d = 0.5 * (np.outer(u, u) - np.outer(v, v))
    n = np.array([math.cos(de) * math.cos(al), math.cos(de) * math.sin(al), math.sin(de)])
    p = np.array([math.sin(al), -math.cos(al), 0.0])
    q = np.cross(n, p)
    Fp = p @ d @ p - q @ d @ q
    Fx = 2.0 * p @ d @ q
    return Fp * Fp + Fx * Fx


def test_ab_norm_matches_detector_tensor():
    rng = np.random.default_rng(7)
    for _ in range(300):
        det = W.Detector(lat=math.asin(rng.uniform(-1, 1)), gamma=rng.uniform(0, math.pi), theta_g0=rng.uniform(0, 6))
        t = rng.uniform(0, 3e5)
        al, de = rng.uniform(0, 2 * math.pi), math.asin(rng.uniform(-1, 1))
        a, b = response.ab(np.array([t]), al, de, det)
        assert abs(a[0] ** 2 + b[0] ** 2 - _tensor_beam_norm(t, al, de, det)) < 1e-13


def test_ab_unit_norm_at_zenith():
    # a source at the detector's zenith sees |F+|^2 + |Fx|^2 = 1 for any arm orientation
    t = np.array([12345.0])
    for g in (0.0, 0.3, math.radians(19.4), 1.2):
        det = W.Detector(gamma=g)
        al = float(earth.sidereal_angle(t, det)[0])
        a, b = response.ab(t, al, det.lat, det)
        assert abs(a[0] ** 2 + b[0] ** 2 - 1.0) < 1e-13


def test_ab_cross_average_vanishes_and_closed_form_means():
    # <ab> = 0 over a whole number of sidereal days (Sec. III.A); closed-form <a^2>, <b^2>
    Tsid = 2 * math.pi / earth.OMEGA_R
    m = 20000
    t = (np.arange(m) + 0.5) * (2 * Tsid / m)  # two sidereal days, midpoint rule (exact for harmonics)
    rng = np.random.default_rng(3)
    for _ in range(10):
        al, de = rng.uniform(0, 2 * math.pi), math.asin(rng.uniform(-1, 1))
        a, b = response.ab(t, al, de, DET)
        assert abs(np.mean(a * b)) < 1e-14
        a2c, b2c = response.ab_mean_squares_closed(de, DET)
        assert abs(np.mean(a * a) - a2c) < 1e-13
        assert abs(np.mean(b * b) - b2c) < 1e-13


def test_four_amplitude_signal_equals_polarisation_form():
    # Eq. sig with A_i of Eq. eq:ampone == Eq. resp with Eqs. patt, hphc
    wl = W.WORKLOADS["tiny"]
    t = np.arange(500) * 173.0
    rng = np.random.default_rng(11)
    for _ in range(10):
        inj = W.Injection(f0=rng.uniform(0.001, 0.006), f1=-rng.uniform(0, 1e-8), alpha=rng.uniform(0, 6.28),
                          delta=math.asin(rng.uniform(-1, 1)), psi=rng.uniform(0, math.pi),
                          cos_iota=rng.uniform(-1, 1), phi0=rng.uniform(0, 6.28), snr=10.0)
        h1 = response.signal_unit(t, inj, wl.fl, DET)
        h2 = response.signal_polarisations(t, inj, wl.fl, DET)
        # the heterodyned phase reaches ~1.4e6 rad, whose FP64 spacing is ~2e-10 rad
        assert np.max(np.abs(h1 - h2)) < 1e-9


# --------------------------------------------------------------------------- resampling (Sec. VI.A)

@pytest.mark.parametrize("n", [16, 17, 40, 41])
def test_upsample_matches_brute_force_trig_interpolant(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    x2 = resample.fourier_upsample2(x)
    # brute force: the real trigonometric interpolant with the Nyquist term split symmetrically
    k = np.arange(n)
    X = np.array([np.sum(x * np.exp(-2j * math.pi * k * kk / n)) for kk in range(n)])
    ts = np.arange(2 * n) / 2.0
    ref = np.zeros(2 * n)
    for kk in range(n):
        if n % 2 == 0 and kk == n // 2:
            ref += (X[kk] * np.cos(math.pi * ts)).real / n  # cos(pi t) carries the Nyquist term
            continue
        f = kk if kk < (n + 1) // 2 else kk - n
        ref += (X[kk] * np.exp(2j * math.pi * f * ts / n)).real / n
    assert np.max(np.abs(x2 - ref)) < 1e-12
    assert np.max(np.abs(x2[::2] - x)) < 1e-12


def test_upsample_reproduces_bandlimited_tone():
    n = 1000
    j = np.arange(n)
    x = np.cos(2 * math.pi * 37 * j / n + 0.4) + 0.5 * np.sin(2 * math.pi * 211 * j / n)
    x2 = resample.fourier_upsample2(x)
    ts = np.arange(2 * n) / 2.0
    ref = np.cos(2 * math.pi * 37 * ts / n + 0.4) + 0.5 * np.sin(2 * math.pi * 211 * ts / n)
    assert np.max(np.abs(x2 - ref)) < 1e-12


def test_natural_spline_matches_scipy_and_reproduces_lines():
    from scipy.interpolate import CubicSpline
    rng = np.random.default_rng(2)
    y = rng.standard_normal(3001)
    M = resample.natural_spline_second_derivatives(y)
    cs = CubicSpline(np.arange(y.size), y, bc_type="natural")
    u = np.concatenate([rng.uniform(0, y.size - 1, 5000), np.arange(y.size, dtype=float)])
    assert np.max(np.abs(resample.spline_eval(y, M, u) - cs(u))) < 1e-12
    assert np.max(np.abs(M - cs(np.arange(y.size), 2))) < 1e-11
    assert M[0] == 0.0 and M[-1] == 0.0
    lin = 0.3 - 1.7 * np.arange(50.0)
    Ml = resample.natural_spline_second_derivatives(lin)
    uu = np.linspace(0, 49, 777)
    assert np.max(np.abs(resample.spline_eval(lin, Ml, uu) - (0.3 - 1.7 * uu))) < 1e-12


def test_source_times_solve_barycentric_equation():
    tb = np.arange(0, 2 * 86164, 1000.0)
    for al, de in ((0.1, 0.2), (3.0, -1.2), (5.5, 1.5)):
        t = resample.source_times(tb, al, de, DET)
        resid = t + earth.phi_m(t, al, de, DET) - tb
        assert np.max(np.abs(resid)) < 1e-9
        assert np.max(np.abs(tb - t)) < 510.0


# --------------------------------------------------------------------------- transforms (Sec. VI.B)

def test_direct_dft_matches_matrix_dft_and_fft():
    rng = np.random.default_rng(4)
    for n, nfft in ((7, 16), (100, 256), (1000, 4096)):
        y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        bins = list(range(0, nfft, max(1, nfft // 37))) + [nfft - 1]
        Xd = fstat.dft_direct(y, nfft, bins)
        yp = np.zeros(nfft, complex)
        yp[:n] = y
        Xm = np.array([np.sum(yp * np.exp(-2j * math.pi * np.arange(nfft) * k / nfft)) for k in bins])
        assert np.max(np.abs(Xd - Xm)) < 1e-9 * math.sqrt(n)
        Xf = fstat.dft_fft(y, nfft, nfft)[bins]
        assert np.max(np.abs(Xd - Xf)) < 1e-9 * math.sqrt(n)


def test_tone_on_bin_has_full_amplitude():
    n = 4096
    j = np.arange(n)
    y = np.exp(2j * math.pi * 300 * j / n)
    X = fstat.dft_direct(y, n, [299, 300, 301])
    assert abs(abs(X[1]) - n) < 1e-8
    assert abs(X[0]) < 1e-8 and abs(X[2]) < 1e-8


def _worst_loss(pad):
    """Largest amplitude loss at the best bin over sub-bin offsets of a tone."""
    n = 2048
    j = np.arange(n)
    worst = 0.0
    for off in np.linspace(0.0, 1.0, 41):
        y = np.exp(2j * math.pi * (500 + off) * j / n)
        nfft = n * pad
        X = fstat.dft_fft(y, nfft, nfft)
        worst = max(worst, 1.0 - np.max(np.abs(X)) / n)
    return worst


def test_zero_padding_losses_printed_in_paper():
    # Sec. VI.B (tests/golden/sec6b_losses.txt): worst loss without padding and with N zeros
    g = golden("sec6b_losses.txt")
    assert abs(_worst_loss(1) - g["loss_no_padding"]) < 1e-3
    assert abs(_worst_loss(2) - g["loss_padding_2"]) < 1e-3


# --------------------------------------------------------------------------- F-statistic (Sec. III)

def test_false_alarm_probability_is_chi2_4dof_survival():
    from scipy.stats import chi2
    F0 = np.linspace(0, 40, 81)
    assert np.allclose(fstat.false_alarm_probability(F0), chi2(4).sf(2 * F0), rtol=1e-10, atol=1e-300)


def test_exact_F_noise_is_chi2_4dof():
    from scipy.stats import kstest, chi2
    wl = W.WORKLOADS["tiny"]
    rng = np.random.default_rng(21)
    vals = []
    for r in range(40):
        x = rng.standard_normal(wl.n)
        df = 1.0 / (wl.n * wl.dt)
        f0s = (np.arange(25) * 2 + 10) * df  # bins two natural bins apart: nearly independent
        vals.append(fstat.fstat_exact(x, wl.dt, 1.1, 0.4, -3e-9, wl.fl, DET, wl.S0, f0s))
    v = np.concatenate(vals)
    assert abs(v.mean() - 2.0) < 4 * math.sqrt(2.0 / v.size) * 1.2
    assert kstest(2 * v, chi2(4).cdf).pvalue > 1e-3


def _noise_free(wl, inj, det):
    x = response.inject(wl.n, wl.dt, [inj], wl.fl, det, wl.sigma)
    return x


def test_exact_F_noise_free_signal_is_rho2_over_2():
    # E[F] = 2 + rho^2/2 with noise; without noise F = rho^2/2 at the true parameters
    wl = W.WORKLOADS["small"]
    rng = np.random.default_rng(8)
    for _ in range(4):
        inj = W.Injection(f0=rng.uniform(0.01, 0.04), f1=-rng.uniform(0, 1e-8), alpha=rng.uniform(0, 6.28),
                          delta=math.asin(rng.uniform(-1, 1)), psi=rng.uniform(0, math.pi),
                          cos_iota=rng.uniform(-1, 1), phi0=rng.uniform(0, 6.28), snr=20.0)
        x = _noise_free(wl, inj, DET)
        F = fstat.fstat_exact(x, wl.dt, inj.alpha, inj.delta, inj.f1, wl.fl, DET, wl.S0, [inj.f0])[0]
        assert abs(F / (inj.snr ** 2 / 2) - 1.0) < 0.01


def test_resampled_F_identity_when_delay_vanishes(monkeypatch):
    # with phi_m = 0 the source times equal the output times, the spline passes
    # through the data, and F is the periodogram of x a exp(-2 pi i f1 t^2/2)
    wl = W.WORKLOADS["tiny"]
    x = W.noise(wl)
    monkeypatch.setattr(earth, "phi_m", lambda t, al, de, det: np.zeros_like(np.asarray(t, dtype=float)))
    seg = resample.Segment(x, wl.dt)
    al, de, f1 = 0.7, -0.2, -5e-9
    F = fstat.fstat(seg, al, de, f1, wl.fl, DET, wl.S0, wl.nfft)
    t = np.arange(wl.n) * wl.dt
    a, b = response.ab(t, al, de, DET)
    rot = np.exp(-2j * math.pi * f1 * t * t / 2)
    Xa = np.fft.fft(x * a * rot, wl.nfft)[: wl.nfft // 2] * wl.dt
    Xb = np.fft.fft(x * b * rot, wl.nfft)[: wl.nfft // 2] * wl.dt
    To = wl.n * wl.dt
    ref = 2 / (wl.S0 * To) * (np.abs(Xa) ** 2 / np.mean(a * a) + np.abs(Xb) ** 2 / np.mean(b * b))
    assert np.max(np.abs(F - ref) / np.maximum(ref, 1.0)) < 1e-10


def test_resampled_F_tracks_exact_F_for_noise_free_signal():
    # Sec. VI.A: two-step resampling reproduces the exact matched filter (rms/max ~ 0.1%)
    # and nearest-neighbour resampling does much worse (~5%)
    wl = W.WORKLOADS["small"]
    rng = np.random.default_rng(12)
    errs, errs_nn = [], []
    for _ in range(3):
        inj = W.Injection(f0=rng.uniform(0.01, 0.04), f1=-rng.uniform(0, 1e-8), alpha=rng.uniform(0, 6.28),
                          delta=math.asin(rng.uniform(-1, 1)), psi=rng.uniform(0, math.pi),
                          cos_iota=rng.uniform(-1, 1), phi0=rng.uniform(0, 6.28), snr=30.0)
        x = _noise_free(wl, inj, DET)
        seg = resample.Segment(x, wl.dt)
        k0 = int(round(inj.f0 * wl.nfft * wl.dt))
        bins = np.arange(k0 - 40, k0 + 41)
        f0s = bins / (wl.nfft * wl.dt)
        Fe = fstat.fstat_exact(x, wl.dt, inj.alpha, inj.delta, inj.f1, wl.fl, DET, wl.S0, f0s)
        Fr = fstat.fstat(seg, inj.alpha, inj.delta, inj.f1, wl.fl, DET, wl.S0, wl.nfft, bins=bins)
        Fn = fstat.fstat(seg, inj.alpha, inj.delta, inj.f1, wl.fl, DET, wl.S0, wl.nfft, bins=bins,
                         interp="nearest")
        errs.append(np.sqrt(np.mean((Fr - Fe) ** 2)) / Fe.max())
        errs_nn.append(np.sqrt(np.mean((Fn - Fe) ** 2)) / Fe.max())
    assert max(errs) < 3e-3
    assert 0.01 < np.mean(errs_nn) < 0.2
    assert np.mean(errs_nn) > 5 * np.mean(errs)


def test_resampled_F_noise_mean_matches_kept_weight():
    # white noise: E|Fa_k|^2 / (sigma^2 N <a^2>) is the a^2-weighted fraction of output
    # samples whose source time stays inside the data (nearest neighbour keeps the noise
    # white, so this is exact); the spline lowers it slightly (up to a few % near the
    # band top).  Independent realizations: templates sharing one realization correlate.
    wl = W.WORKLOADS["small"]
    rng = np.random.default_rng(31)
    r_nn, r_sp = [], []
    for al, de in ((0.3, 0.1), (2.0, -0.9), (4.0, 1.1), (5.2, 0.4), (1.1, -0.3), (3.3, 0.8)):
        seg = resample.Segment(rng.standard_normal(wl.n), wl.dt)
        for interp, out in (("nearest", r_nn), ("spline", r_sp)):
            dm = fstat.demodulate(seg, al, de, -2e-9, wl.fl, DET, interp=interp)
            k = np.rint(dm.t_src / wl.dt)
            kept = (k >= 0) & (k < wl.n)
            a, _ = response.ab(dm.t_src, al, de, DET)
            w = np.sum(a[kept] ** 2) / np.sum(a * a)
            P = np.abs(np.fft.fft(dm.ya, wl.nfft)[: wl.nfft // 2]) ** 2 / (wl.n * dm.a2)
            nb = P.size
            out.append(P[nb // 20: 19 * nb // 20].mean() / w)
    # sigma of each mean over ~6 x 4800 independent bins: ~0.6% (|Fa|^2 part alone)
    assert abs(np.mean(r_nn) - 1.0) < 0.02
    assert 0.95 < np.mean(r_sp) < 1.0 + 0.02


def test_epoch_shift_is_a_time_translation():
    """A segment starting at t0 sees the detector where the unshifted detector is
    at t0 + t: phi_m and the detector position agree at every t."""
    det = W.detector_for(W.WORKLOADS["grid_2d"])
    t0 = 1.7e7 + 123.25
    d2 = earth.detector_at_epoch(det, t0)
    t = np.linspace(0.0, 3 * 86164.0, 257)
    a, dl = 1.1, -0.4
    assert np.max(np.abs(earth.phi_m(t0 + t, a, dl, det) - earth.phi_m(t, a, dl, d2))) < 1e-8
    assert np.max(np.abs(earth.detector_position_ls(t0 + t, det) - earth.detector_position_ls(t, d2))) < 1e-8
    # a whole number of sidereal rotations leaves the site, not the orbit, unchanged
    day = 2 * math.pi / earth.OMEGA_R
    d3 = earth.detector_at_epoch(det, 5 * day)
    assert abs(math.remainder(earth.sidereal_angle(0.0, d3) - earth.sidereal_angle(0.0, det), 2 * math.pi)) < 1e-9
    assert abs(d3.lambda_e0 - det.lambda_e0 - earth.OMEGA_O * 5 * day) < 1e-15


def test_search_false_alarm_and_threshold():
    """Eq. FP against the chi^2_4 survival (Eq. PF), its small-alpha limit, and the
    inversion to a threshold."""
    from scipy.stats import chi2
    for F0 in (0.5, 5.0, 20.0, 35.0):
        a1, nf = fstat.search_false_alarm(F0, 1.0)
        assert abs(a1 - chi2.sf(2 * F0, 4)) <= 1e-12 * max(a1, 1e-300) + 1e-15
        aN, nfN = fstat.search_false_alarm(F0, 1e6)
        assert abs(nfN - 1e6 * a1) <= 1e-9 * nfN
        if nfN < 1e-3:                                 # rare: alpha ~ expected number
            assert abs(aN / nfN - 1.0) < 1e-3
    for alpha, nc in ((0.01, 1e9), (1e-3, 4.3e6), (0.5, 10.0)):
        F0 = fstat.threshold_for_false_alarm(alpha, nc)
        assert abs(fstat.search_false_alarm(F0, nc)[0] - alpha) < 1e-12
    assert fstat.threshold_for_false_alarm(0.999999, 1e6) == 0.0 or \
        fstat.search_false_alarm(fstat.threshold_for_false_alarm(0.999999, 1e6), 1e6)[0] <= 1.0


def test_cell_count_is_the_ellipsoid_volume():
    """V_cell of Eq. vc is the volume of tau^T G tau <= 1: Monte Carlo in 2 and 4 dimensions."""
    rng = np.random.default_rng(7)
    for G in (np.array([[1 / 12, 1 / 12], [1 / 12, 4 / 45]]),
              np.array([[3.0, 0.4, 0.1, 0.0], [0.4, 2.0, 0.2, 0.1], [0.1, 0.2, 1.5, 0.3], [0.0, 0.1, 0.3, 1.0]])):
        M = G.shape[0]
        half = 1.0 / np.sqrt(np.linalg.eigvalsh(G).min())     # box half-width covering the ellipsoid
        u = rng.uniform(-half, half, size=(400000, M))
        frac = np.mean(np.einsum("ij,jk,ik->i", u, G, u) <= 1.0)
        v_mc = frac * (2 * half) ** M
        v_cell = 1.0 / fstat.cell_count(G, 1.0)
        assert abs(v_mc / v_cell - 1.0) < 0.02, (v_mc, v_cell)


def test_interbinning_worst_loss_is_13_percent():
    """Sec. VI.B: interbinning (Eq. intbin) loses at most ~13% of the amplitude of a tone
    between Fourier frequencies (the plain DFT loses 36.3% at half a bin)."""
    N = 4096
    j = np.arange(N)
    worst_ib, worst_plain = 0.0, 0.0
    for frac in np.linspace(0.0, 1.0, 201):
        X = np.fft.fft(np.exp(2j * math.pi * (100 + frac) * j / N))
        H = (X[1:] - X[:-1]) / math.sqrt(2.0)
        best = max(np.max(np.abs(X[95:106])), np.max(np.abs(H[95:106])))
        worst_ib = max(worst_ib, 1.0 - best / N)
        worst_plain = max(worst_plain, 1.0 - np.max(np.abs(X[95:106])) / N)
    g = golden("sec6b_losses.txt")
    assert abs(worst_plain - g["loss_no_padding"]) < 2e-3
    assert abs(worst_ib - g["loss_interbinning"]) < 6e-3, worst_ib


def test_interbinned_F_even_entries_are_the_plain_bins():
    wl = W.WORKLOADS["tiny"]
    det = W.detector_for(wl)
    x = W.noise(wl) + response.inject(wl.n, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)
    seg = resample.Segment(x, wl.dt)
    nfft = 2048                      # >= N = 1346, no doubling
    a, d = W.sky_grid(2)
    Fi = fstat.fstat_interbinned(seg, a[1], d[1], -3e-9, wl.fl, det, wl.S0, nfft)
    Fp = fstat.fstat(seg, a[1], d[1], -3e-9, wl.fl, det, wl.S0, nfft)
    assert Fi.shape == (nfft,)
    assert np.allclose(Fi[0::2], Fp, rtol=1e-13, atol=1e-13)
    # the half bins track the doubly padded transform's odd bins (an approximation)
    F2 = fstat.fstat(seg, a[1], d[1], -3e-9, wl.fl, det, wl.S0, 2 * nfft)
    assert np.allclose(Fi[0::2], F2[0::2], rtol=1e-12, atol=1e-12)
    assert np.corrcoef(Fi[1::2], F2[1::2])[0, 1] > 0.6
