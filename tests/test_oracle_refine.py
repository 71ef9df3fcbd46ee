"""Pins of the fine-search oracle (exact F at continuous points, its gradient, the
reduced Fisher matrix and the Nelder-Mead maximisation) against finite
differences, closed forms and the injected signal."""
import math

import numpy as np
import pytest

from oracle import fstat as ofs
from oracle import refine as orf
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
    return wl, det, x, theta


def test_point_F_is_the_exact_F():
    wl, det, x, th = _case()
    F = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0)
    ref = ofs.fstat_exact(x, wl.dt, th[2], th[3], th[1], wl.fl, det, wl.S0, [th[0]])[0]
    assert abs(F - ref) <= 1e-10 * ref   # phases of ~2e5 cycles: rounding order only


@pytest.mark.parametrize("offset", [0.0, 0.4])
def test_gradient_matches_central_differences(offset):
    wl, det, x, th = _case()
    F0, g, G = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True)
    width = 1.0 / np.sqrt(np.diag(G))
    th = th + offset * width * np.array([1.0, -0.7, 0.5, 0.8])
    F0, g, G = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True)
    width = 1.0 / np.sqrt(np.diag(G))
    for i in range(4):
        h = 1e-3 * width[i]
        e = np.zeros(4)
        e[i] = h
        fd = (orf.fstat_point(x, wl.dt, th + e, wl.fl, det, wl.S0)
              - orf.fstat_point(x, wl.dt, th - e, wl.fl, det, wl.S0)) / (2 * h)
        # truncation ~ h^2 F'''; scale-free bound: 1e-5 of F per width
        assert abs(fd - g[i]) <= 1e-4 * abs(g[i]) + 1e-5 * F0 / width[i], (i, fd, g[i])


@pytest.mark.parametrize("offset", [0.0, 0.6])
def test_hessian_matches_differences_of_the_gradient(offset):
    wl, det, x, th = _case()
    _, _, G = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True)
    width = 1.0 / np.sqrt(np.diag(G))
    th = th + offset * width * np.array([0.5, 1.0, -0.8, 0.4])
    F0, g, G, H = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True, hess=True)
    assert np.allclose(H, H.T)
    for j in range(4):
        h = 1e-3 * width[j]
        e = np.zeros(4)
        e[j] = h
        col = (orf.fstat_point(x, wl.dt, th + e, wl.fl, det, wl.S0, grad=True)[1]
               - orf.fstat_point(x, wl.dt, th - e, wl.fl, det, wl.S0, grad=True)[1]) / (2 * h)
        for i in range(4):
            assert abs(col[i] - H[i, j]) <= 1e-4 * abs(H[i, j]) + 1e-5 * F0 / (width[i] * width[j]), \
                (i, j, col[i], H[i, j])


def test_reduced_fisher_closed_forms():
    """Frequency and spindown rows: m_0 = 2 pi (t + phi), m_1 = 2 pi (t^2/2 + t phi); over
    t uniform in [0, To) with |phi| varying by a few seconds, G_00 -> (2 pi)^2 (N^2 - 1) dt^2 / 12
    and G_11 -> (2 pi)^2 To^4 / 45."""
    wl, det, x, th = _case()
    _, _, G = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True)
    n, dt = wl.n, wl.dt
    To = n * dt
    assert abs(G[0, 0] / ((2 * math.pi) ** 2 * (n * n - 1) * dt * dt / 12.0) - 1.0) < 2e-3
    assert abs(G[1, 1] / ((2 * math.pi) ** 2 * To ** 4 / 45.0) - 1.0) < 2e-2
    assert np.allclose(G, G.T)
    assert np.all(np.linalg.eigvalsh(G) > 0)


@pytest.mark.parametrize("i", [0, 1, 2, 3])
def test_metric_is_the_curvature_of_the_autocovariance(i):
    """G = -(1/2) d^2 C / dtau^2 with C(tau) = |<exp(2 pi i (Phi(theta + tau) - Phi(theta)))>|^2
    (Eqs. auto5, G, redFm-def): C from the phase model of the response module (the
    4-term scalar product of phi_m), G from the refine module (n0 . r_d and its
    derivatives)."""
    wl, det, x, th = _case()
    _, _, G = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True)
    t = np.arange(wl.n) * wl.dt
    tau = math.sqrt(0.002 / G[i, i])             # 1 - C ~ 0.2% (quartic terms ~ 1e-3 of it)
    ph0 = orsp.heterodyned_phase_cycles(t, th[0], th[1], wl.fl, th[2], th[3], det)
    loss = []
    for sgn in (1, -1):
        q = th.copy()
        q[i] += sgn * tau
        d = orsp.heterodyned_phase_cycles(t, q[0], q[1], wl.fl, q[2], q[3], det) - ph0
        loss.append(1.0 - abs(np.mean(np.exp(2j * math.pi * d))) ** 2)
    assert abs(0.5 * (loss[0] + loss[1]) / 0.002 - 1.0) < 2e-3, loss


def test_signal_loss_follows_the_metric_in_order_of_magnitude():
    """Noise-free signal: the F loss is quadratic in the offset and of the size the metric
    gives (within a factor the daily amplitude modulation a^2, b^2 sets on one day)."""
    wl, det, x, th = _case(noise=False)
    F0, _, G = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True)
    for i in range(4):
        e = np.zeros(4)
        e[i] = math.sqrt(0.01 / G[i, i])
        l1 = 1 - 0.5 * sum(orf.fstat_point(x, wl.dt, th + s * e, wl.fl, det, wl.S0) for s in (1, -1)) / F0
        l2 = 1 - 0.5 * sum(orf.fstat_point(x, wl.dt, th + 2 * s * e, wl.fl, det, wl.S0) for s in (1, -1)) / F0
        assert 0.2 < l1 / 0.01 < 1.5
        assert abs(l2 / l1 - 4.0) < 0.2           # quadratic near the maximum


def test_nelder_mead_recovers_the_injection():
    wl, det, x, th = _case(noise=False)
    F0, _, G = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True)
    width = 1.0 / np.sqrt(np.diag(G))
    start = th + width * np.array([0.9, -0.8, 0.7, -0.6])
    assert orf.fstat_point(x, wl.dt, start, wl.fl, det, wl.S0) < 0.9 * F0
    best, Fb = orf.fine_search(x, wl.dt, start, wl.fl, det, wl.S0)
    assert Fb >= F0 * (1 - 1e-4)
    assert np.all(np.abs(best - th) < 0.05 * width), (best - th) / width


def test_amplitude_estimates_recover_the_injected_amplitudes():
    """Noise-free signal over (nearly) one sidereal day at the true template: the
    estimators of Eq. amle0 return the A_i of Eq. eq:ampone up to <ab> != 0 terms."""
    wl, det, x, th = _case(noise=False)
    inj = W.Injection(f0=th[0], f1=th[1], alpha=th[2], delta=th[3], psi=0.3, cos_iota=0.4, phi0=1.1, snr=25.0)
    t = np.arange(wl.n) * wl.dt
    h = orsp.signal_unit(t, inj, wl.fl, det)
    h0 = inj.snr / math.sqrt(2.0 / wl.S0 * wl.dt * float(np.dot(h, h)))     # the amplitude inject() applies
    A = orsp.amplitudes(h0, inj.cos_iota, inj.psi, inj.phi0)
    Ah = orf.amplitude_estimates(x, wl.dt, th, wl.fl, det)
    assert np.max(np.abs(Ah - A)) < 0.02 * np.max(np.abs(A)), (Ah, A)
    # with noise the estimates scatter around the truth by ~ sqrt(2/(<a^2> To/S0)) ...
    wl, det, xn, th = _case(noise=True)
    An = orf.amplitude_estimates(xn, wl.dt, th, wl.fl, det)
    a, b = orsp.ab(t, th[2], th[3], det)
    sig = np.sqrt([2 * wl.S0 / (wl.n * wl.dt * np.mean(v * v)) for v in (a, b, a, b)])
    assert np.all(np.abs(An - A) < 5 * sig), ((An - A) / sig)
