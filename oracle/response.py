"""Detector response and signal model (oracle, FP64).

Test infrastructure only (see the package docstring).

Sec. II defers the explicit amplitude modulation functions of an
interferometer to Eqs. (12)-(13) of the first paper of the series (Jaranowski,
Krolak, Schutz 1998); they are restated here from that published form.  With
x = alpha - theta(t), lambda the site latitude and gamma the orientation of
the arms' bisector (counter-clockwise from local East):

  a = (1/16) sin2g (3 - cos2l)(3 - cos2d) cos2x - (1/4) cos2g sinl (3 - cos2d) sin2x
      + (1/4) sin2g sin2l sin2d cosx - (1/2) cos2g cosl sin2d sinx
      + (3/4) sin2g cos^2 l cos^2 d
  b = cos2g sinl sind cos2x + (1/4) sin2g (3 - cos2l) sind sin2x
      + cos2g cosl cosd cosx + (1/2) sin2g sin2l cosd sinx
"""
from __future__ import annotations

import math

import numpy as np

from . import earth


def ab_coefficients(delta: float, det):
    """Fourier coefficients of a and b in x = alpha - theta.

    Returns (e, f): a = e0 + e1c cos x + e1s sin x + e2c cos 2x + e2s sin 2x and
    b = f1c cos x + f1s sin x + f2c cos 2x + f2s sin 2x, as dicts.
    """
    g, l, d = det.gamma, det.lat, delta
    s2g, c2g = math.sin(2 * g), math.cos(2 * g)
    sl, cl, s2l, c2l = math.sin(l), math.cos(l), math.sin(2 * l), math.cos(2 * l)
    sd, cd, s2d, c2d = math.sin(d), math.cos(d), math.sin(2 * d), math.cos(2 * d)
    e = dict(
        c2=s2g * (3 - c2l) * (3 - c2d) / 16.0,
        s2=-c2g * sl * (3 - c2d) / 4.0,
        c1=s2g * s2l * s2d / 4.0,
        s1=-c2g * cl * s2d / 2.0,
        c0=0.75 * s2g * cl * cl * cd * cd,
    )
    f = dict(
        c2=c2g * sl * sd,
        s2=s2g * (3 - c2l) * sd / 4.0,
        c1=c2g * cl * cd,
        s1=s2g * s2l * cd / 2.0,
    )
    return e, f


def ab(t, alpha: float, delta: float, det):
    """a(t), b(t) at the times t (seconds from the segment start)."""
    x = alpha - earth.sidereal_angle(t, det)
    e, f = ab_coefficients(delta, det)
    c1, s1, c2, s2 = np.cos(x), np.sin(x), np.cos(2 * x), np.sin(2 * x)
    a = e["c2"] * c2 + e["s2"] * s2 + e["c1"] * c1 + e["s1"] * s1 + e["c0"]
    b = f["c2"] * c2 + f["s2"] * s2 + f["c1"] * c1 + f["s1"] * s1
    return a, b


def ab_mean_squares_closed(delta: float, det):
    """<a^2>, <b^2> averaged over a whole number of sidereal days (closed form).

    Over whole days each harmonic of x averages to 1/2 in square and the
    cross products vanish, so <a^2> = e0^2 + (e1c^2 + e1s^2 + e2c^2 + e2s^2)/2
    and <b^2> = (f1c^2 + f1s^2 + f2c^2 + f2s^2)/2.
    """
    e, f = ab_coefficients(delta, det)
    a2 = e["c0"] ** 2 + 0.5 * (e["c1"] ** 2 + e["s1"] ** 2 + e["c2"] ** 2 + e["s2"] ** 2)
    b2 = 0.5 * (f["c1"] ** 2 + f["s1"] ** 2 + f["c2"] ** 2 + f["s2"] ** 2)
    return a2, b2


def amplitudes(h0: float, cos_iota: float, psi: float, phi0: float):
    """A_1..A_4 of Eq. eq:ampone with h0+ and h0x from Eq. h0iota (zeta = 90 deg)."""
    hp = 0.5 * h0 * (1.0 + cos_iota ** 2)
    hc = h0 * cos_iota
    c2p, s2p = math.cos(2 * psi), math.sin(2 * psi)
    cp, sp = math.cos(phi0), math.sin(phi0)
    return np.array([
        hp * c2p * cp - hc * s2p * sp,
        hp * s2p * cp + hc * c2p * sp,
        -hp * c2p * sp - hc * s2p * cp,
        -hp * s2p * sp + hc * c2p * cp,
    ])


def heterodyned_phase_cycles(t, f0: float, f1: float, fl: float, alpha: float, delta: float, det):
    """Phase of the narrow-band series in cycles.

    The full phase of Eq. pha3 with one spindown is w0 (t + phi_m) + phi_s with
    w0 = 2 pi (fl + f0).  The narrow-band series is the band above fl shifted
    down by fl, so its phase is that minus 2 pi fl t:
      f0 (t + phi_m) + fl phi_m + f1 (t^2/2 + t phi_m)       [cycles]
    """
    t = np.asarray(t, dtype=np.float64)
    pm = earth.phi_m(t, alpha, delta, det)
    return f0 * (t + pm) + fl * pm + f1 * (0.5 * t * t + t * pm)


def signal_unit(t, inj, fl: float, det, h0: float = 1.0):
    """h(t) of Eq. sig: sum_i A_i h_i with h_i = a cos(phi), b cos(phi), a sin(phi), b sin(phi)."""
    a, b = ab(t, inj.alpha, inj.delta, det)
    ph = 2.0 * math.pi * heterodyned_phase_cycles(t, inj.f0, inj.f1, fl, inj.alpha, inj.delta, det)
    A = amplitudes(h0, inj.cos_iota, inj.psi, inj.phi0)
    cph, sph = np.cos(ph), np.sin(ph)
    return A[0] * a * cph + A[1] * b * cph + A[2] * a * sph + A[3] * b * sph


def signal_polarisations(t, inj, fl: float, det, h0: float = 1.0):
    """h(t) of Eq. resp with the beam patterns of Eq. patt and polarisations of Eq. hphc."""
    a, b = ab(t, inj.alpha, inj.delta, det)
    ph = 2.0 * math.pi * heterodyned_phase_cycles(t, inj.f0, inj.f1, fl, inj.alpha, inj.delta, det)
    c2p, s2p = math.cos(2 * inj.psi), math.sin(2 * inj.psi)
    Fp = a * c2p + b * s2p
    Fx = b * c2p - a * s2p
    hp = 0.5 * h0 * (1.0 + inj.cos_iota ** 2) * np.cos(ph + inj.phi0)
    hx = h0 * inj.cos_iota * np.sin(ph + inj.phi0)
    return Fp * hp + Fx * hx


def inject(n: int, dt: float, injections, fl: float, det, sigma: float):
    """Sum of injections sampled at t_k = k dt, each scaled to its target SNR.

    The optimal SNR of Eq. snr-def with the scalar product of Eq. approx1 and
    S0 = 2 sigma^2 dt is rho^2 = (2/S0) dt sum_k h_k^2 = sum_k h_k^2 / sigma^2.
    """
    t = np.arange(n, dtype=np.float64) * dt
    S0 = 2.0 * sigma ** 2 * dt
    out = np.zeros(n)
    for inj in injections:
        h = signal_unit(t, inj, fl, det)
        rho_unit = math.sqrt(2.0 / S0 * dt * float(np.dot(h, h)))
        out += h * (inj.snr / rho_unit)
    return out
