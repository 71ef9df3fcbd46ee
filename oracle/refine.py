"""The fine search of Sec. VI.C (oracle, FP64): F at a continuous template point,
its gradient, the reduced Fisher matrix, and the Nelder-Mead maximisation.

Test infrastructure only (see the package docstring).

In the fine search of the Monte Carlo simulations (Sec. VII) the F-statistic is
evaluated exactly, by the direct sums of Eqs. OS and Fab over the original samples
(no resampling).  A template point is
theta = (f0, f1, alpha, delta): f0 the frequency above the band edge fl [Hz]
(the bin frequency k / (Nfft dt) of the coarse search, now continuous), f1 the
spindown [Hz/s], alpha and delta the sky position.  With t_k = k dt,
phi_k = phi_m(t_k) (Eq. pham) and a_k, b_k the amplitude modulation functions:

  Phi_k = f0 (t_k + phi_k) + fl phi_k + f1 (t_k^2/2 + t_k phi_k)      [cycles]
  Sa = sum_k x_k a_k exp(-2 pi i Phi_k),  Sb likewise with b_k
  F = 2 dt / (S0 N) (|Sa|^2 / <a^2> + |Sb|^2 / <b^2>)               (Eqs. OS, Fab)

Derivatives (chain rule written out here; pinned by finite differences):

  dPhi/df0 = t + phi,  dPhi/df1 = t^2/2 + t phi,
  dPhi/dsky = (f0 + fl + f1 t) dphi/dsky,
  dSa/dtheta = sum_k x_k (da_k/dtheta - 2 pi i a_k dPhi_k/dtheta) exp(-2 pi i Phi_k),
  dF = c [2 Re(conj(Sa) dSa) / <a^2> - |Sa|^2 d<a^2> / <a^2>^2 + (same for b)],

where a depends on alpha through x = alpha - theta(t) and on delta through its
coefficients.  Second derivatives follow by differentiating once more:

  d2Sa/dtheta_i dtheta_j = sum_k x_k [a_ij - 2 pi i (a_i dPhi_j + a_j dPhi_i + a dPhi_ij)
                                      - 4 pi^2 a dPhi_i dPhi_j] exp(-2 pi i Phi_k),
  d2(P/A) = P_ij/A - (P_i A_j + P_j A_i)/A^2 - P A_ij/A^2 + 2 P A_i A_j/A^3, P = |Sa|^2.

The reduced Fisher matrix (Eq. redFm-def) takes the phase derivatives
m_i = 2 pi dPhi/dtheta_i:  G_ij = <m_i m_j> - <m_i><m_j>, and
near a maximum F(theta + tau) ~ F(theta) (1 - tau^T G tau) (Eq. TaylorC2).
"""
from __future__ import annotations

import math

import numpy as np

from . import earth, response


def _geometry(n: int, dt: float, alpha: float, delta: float, det, second: bool = False):
    """t_k, phi_k and its alpha/delta derivatives, a_k, b_k and their derivatives
    (with second=True also the second derivatives: phi_aa, phi_ad, phi_dd and the
    same for a and b)."""
    t = np.arange(n, dtype=np.float64) * dt
    rd = earth.detector_position_ls(t, det)                    # (3, n)
    ca, sa, cd, sd = math.cos(alpha), math.sin(alpha), math.cos(delta), math.sin(delta)
    R = earth.ecliptic_rotation(det.eps)
    n0 = R @ np.array([ca * cd, sa * cd, sd])
    n0_a = R @ np.array([-sa * cd, ca * cd, 0.0])
    n0_d = R @ np.array([-ca * sd, -sa * sd, cd])
    phi, phi_a, phi_d = n0 @ rd, n0_a @ rd, n0_d @ rd
    # a, b and derivatives: x = alpha - theta(t); coefficients depend on delta
    x = alpha - earth.sidereal_angle(t, det)
    c1, s1, c2, s2 = np.cos(x), np.sin(x), np.cos(2 * x), np.sin(2 * x)
    e, f = response.ab_coefficients(delta, det)
    ed, fd = _ab_coefficients_ddelta(delta, det)
    a = e["c2"] * c2 + e["s2"] * s2 + e["c1"] * c1 + e["s1"] * s1 + e["c0"]
    b = f["c2"] * c2 + f["s2"] * s2 + f["c1"] * c1 + f["s1"] * s1
    a_a = -2 * e["c2"] * s2 + 2 * e["s2"] * c2 - e["c1"] * s1 + e["s1"] * c1
    b_a = -2 * f["c2"] * s2 + 2 * f["s2"] * c2 - f["c1"] * s1 + f["s1"] * c1
    a_d = ed["c2"] * c2 + ed["s2"] * s2 + ed["c1"] * c1 + ed["s1"] * s1 + ed["c0"]
    b_d = fd["c2"] * c2 + fd["s2"] * s2 + fd["c1"] * c1 + fd["s1"] * s1
    first = (t, phi, phi_a, phi_d, a, b, a_a, b_a, a_d, b_d)
    if not second:
        return first
    n0_aa = R @ np.array([-ca * cd, -sa * cd, 0.0])
    n0_ad = R @ np.array([sa * sd, -ca * sd, 0.0])
    n0_dd = R @ np.array([-ca * cd, -sa * cd, -sd])
    phi2 = (n0_aa @ rd, n0_ad @ rd, n0_dd @ rd)
    edd, fdd = _ab_coefficients_ddelta2(delta, det)
    a_aa = -4 * e["c2"] * c2 - 4 * e["s2"] * s2 - e["c1"] * c1 - e["s1"] * s1
    b_aa = -4 * f["c2"] * c2 - 4 * f["s2"] * s2 - f["c1"] * c1 - f["s1"] * s1
    a_ad = -2 * ed["c2"] * s2 + 2 * ed["s2"] * c2 - ed["c1"] * s1 + ed["s1"] * c1
    b_ad = -2 * fd["c2"] * s2 + 2 * fd["s2"] * c2 - fd["c1"] * s1 + fd["s1"] * c1
    a_dd = edd["c2"] * c2 + edd["s2"] * s2 + edd["c1"] * c1 + edd["s1"] * s1 + edd["c0"]
    b_dd = fdd["c2"] * c2 + fdd["s2"] * s2 + fdd["c1"] * c1 + fdd["s1"] * s1
    return first + (phi2, (a_aa, a_ad, a_dd), (b_aa, b_ad, b_dd))


def _ab_coefficients_ddelta(delta: float, det):
    """d/ddelta of the coefficients of response.ab_coefficients."""
    g, l, d = det.gamma, det.lat, delta
    s2g, c2g = math.sin(2 * g), math.cos(2 * g)
    sl, cl, s2l, c2l = math.sin(l), math.cos(l), math.sin(2 * l), math.cos(2 * l)
    sd, cd, s2d, c2d = math.sin(d), math.cos(d), math.sin(2 * d), math.cos(2 * d)
    e = dict(
        c2=s2g * (3 - c2l) * 2 * s2d / 16.0,
        s2=-c2g * sl * 2 * s2d / 4.0,
        c1=s2g * s2l * 2 * c2d / 4.0,
        s1=-c2g * cl * c2d,
        c0=-0.75 * s2g * cl * cl * s2d,
    )
    f = dict(
        c2=c2g * sl * cd,
        s2=s2g * (3 - c2l) * cd / 4.0,
        c1=-c2g * cl * sd,
        s1=-s2g * s2l * sd / 2.0,
    )
    return e, f


def _ab_coefficients_ddelta2(delta: float, det):
    """d^2/ddelta^2 of the coefficients of response.ab_coefficients."""
    g, l, d = det.gamma, det.lat, delta
    s2g, c2g = math.sin(2 * g), math.cos(2 * g)
    sl, cl, s2l, c2l = math.sin(l), math.cos(l), math.sin(2 * l), math.cos(2 * l)
    sd, cd, s2d, c2d = math.sin(d), math.cos(d), math.sin(2 * d), math.cos(2 * d)
    e = dict(
        c2=s2g * (3 - c2l) * 4 * c2d / 16.0,
        s2=-c2g * sl * c2d,
        c1=-s2g * s2l * s2d,
        s1=2 * c2g * cl * s2d,
        c0=-1.5 * s2g * cl * cl * c2d,
    )
    f = dict(
        c2=-c2g * sl * sd,
        s2=-s2g * (3 - c2l) * sd / 4.0,
        c1=-c2g * cl * cd,
        s1=-s2g * s2l * cd / 2.0,
    )
    return e, f


def fstat_point(x, dt: float, theta, fl: float, det, S0: float, grad: bool = False, hess: bool = False):
    """Exact F at theta = (f0, f1, alpha, delta); with grad=True also dF/dtheta (4,)
    and the reduced Fisher matrix G (4, 4) in rad^2 per unit parameter^2; with
    hess=True as well the Hessian of F (4, 4) as a fourth value."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    f0, f1, alpha, delta = (float(v) for v in theta)
    geo = _geometry(n, dt, alpha, delta, det, second=hess)
    t, phi, phi_a, phi_d, a, b, a_a, b_a, a_d, b_d = geo[:10]
    ph = f0 * (t + phi) + fl * phi + f1 * (0.5 * t * t + t * phi)
    rot = np.exp(-2j * math.pi * (ph - np.floor(ph)))
    Sa, Sb = np.dot(x * a, rot), np.dot(x * b, rot)
    A, B = float(np.mean(a * a)), float(np.mean(b * b))
    c = 2.0 * dt / (S0 * n)
    F = c * (abs(Sa) ** 2 / A + abs(Sb) ** 2 / B)
    if not grad:
        return F
    w = f0 + fl + f1 * t
    dPhi = [t + phi, t * (0.5 * t + phi), w * phi_a, w * phi_d]
    da = [0.0, 0.0, a_a, a_d]
    db = [0.0, 0.0, b_a, b_d]
    g = np.empty(4)
    for i in range(4):
        dSa = np.dot(x * (da[i] - 2j * math.pi * a * dPhi[i]), rot)
        dSb = np.dot(x * (db[i] - 2j * math.pi * b * dPhi[i]), rot)
        dA = 2.0 * float(np.mean(a * da[i])) if i >= 2 else 0.0
        dB = 2.0 * float(np.mean(b * db[i])) if i >= 2 else 0.0
        g[i] = c * (2.0 * (np.conj(Sa) * dSa).real / A - abs(Sa) ** 2 * dA / A ** 2
                    + 2.0 * (np.conj(Sb) * dSb).real / B - abs(Sb) ** 2 * dB / B ** 2)
    m = np.stack([2.0 * math.pi * d for d in dPhi])             # (4, n)
    mm = m.mean(axis=1)
    G = (m @ m.T) / n - np.outer(mm, mm)
    if not hess:
        return F, g, G
    phi2, a2s, b2s = geo[10:]
    zero = np.zeros(n)
    # second derivatives of Phi (cycles) and of a, b, indexed (i, j)
    d2P = {(0, 0): zero, (0, 1): zero, (0, 2): phi_a, (0, 3): phi_d, (1, 1): zero, (1, 2): t * phi_a,
           (1, 3): t * phi_d, (2, 2): w * phi2[0], (2, 3): w * phi2[1], (3, 3): w * phi2[2]}
    d2a = {(2, 2): a2s[0], (2, 3): a2s[1], (3, 3): a2s[2]}
    d2b = {(2, 2): b2s[0], (2, 3): b2s[1], (3, 3): b2s[2]}
    H = np.empty((4, 4))
    for (u, S, amp, damp, d2amp, M) in ((0, Sa, a, da, d2a, A), (1, Sb, b, db, d2b, B)):
        dS = [np.dot(x * (damp[i] - 2j * math.pi * amp * dPhi[i]), rot) for i in range(4)]
        dM = [2.0 * float(np.mean(amp * damp[i])) if i >= 2 else 0.0 for i in range(4)]
        P = abs(S) ** 2
        dP_ = [2.0 * (np.conj(S) * dS[i]).real for i in range(4)]
        for i in range(4):
            for j in range(i, 4):
                aij = d2amp.get((i, j), 0.0)
                ai = damp[i] if i >= 2 else 0.0
                aj = damp[j] if j >= 2 else 0.0
                d2S = np.dot(x * (aij - 2j * math.pi * (ai * dPhi[j] + aj * dPhi[i] + amp * d2P[(i, j)])
                                  - 4.0 * math.pi ** 2 * amp * dPhi[i] * dPhi[j]), rot)
                Mij = 2.0 * float(np.mean(ai * aj + amp * aij)) if (i >= 2 and j >= 2) else 0.0
                Pij = 2.0 * (np.conj(dS[i]) * dS[j] + np.conj(S) * d2S).real
                h = (Pij / M - (dP_[i] * dM[j] + dP_[j] * dM[i]) / M ** 2 - P * Mij / M ** 2
                     + 2.0 * P * dM[i] * dM[j] / M ** 3)
                if u == 0:
                    H[i, j] = h
                else:
                    H[i, j] += h
    H = c * H
    for i in range(4):
        for j in range(i):
            H[i, j] = H[j, i]
    return F, g, G, H


def fine_search(x, dt: float, theta0, fl: float, det, S0: float, scale=None, xatol: float = 1e-4,
                maxiter: int = 2000):
    """Maximise the exact F from theta0 with the Nelder-Mead simplex (Sec. VI.C).

    The simplex works in coordinates u = (theta - theta0) / scale; `scale`
    defaults to the widths G_ii^(-1/2) of the reduced Fisher matrix at theta0,
    so that one unit is about one correlation length in each parameter."""
    from scipy.optimize import minimize
    theta0 = np.asarray(theta0, dtype=np.float64)
    if scale is None:
        _, _, G = fstat_point(x, dt, theta0, fl, det, S0, grad=True)
        scale = 1.0 / np.sqrt(np.diag(G))
    scale = np.asarray(scale, dtype=np.float64)
    res = minimize(lambda u: -fstat_point(x, dt, theta0 + u * scale, fl, det, S0), np.zeros(4),
                   method="Nelder-Mead", options=dict(xatol=xatol, fatol=1e-10, maxiter=maxiter,
                                                      initial_simplex=0.3 * np.vstack([np.zeros(4), np.eye(4)])))
    return theta0 + res.x * scale, -res.fun


def amplitude_estimates(x, dt: float, theta, fl: float, det):
    """ML estimators of the amplitudes (Eq. amle0): A1 = 2 <x h1>/<a^2>,
    A2 = 2 <x h2>/<b^2>, A3 = 2 <x h3>/<a^2>, A4 = 2 <x h4>/<b^2> with
    h1..h4 = a cos(phi), b cos(phi), a sin(phi), b sin(phi) (Eq. sig) at the
    template theta, time averages over the samples."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    t = np.arange(n, dtype=np.float64) * dt
    f0, f1, alpha, delta = (float(v) for v in theta)
    a, b = response.ab(t, alpha, delta, det)
    cyc = response.heterodyned_phase_cycles(t, f0, f1, fl, alpha, delta, det)
    ph = 2.0 * math.pi * (cyc - np.floor(cyc))
    c, s = np.cos(ph), np.sin(ph)
    A, B = np.mean(a * a), np.mean(b * b)
    return np.array([2 * np.mean(x * a * c) / A, 2 * np.mean(x * b * c) / B,
                     2 * np.mean(x * a * s) / A, 2 * np.mean(x * b * s) / B])
