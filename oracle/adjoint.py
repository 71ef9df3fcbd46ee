"""F of the resampled series at a continuous template point, and its gradient
(oracle, FP64): the coarse search's F of Sec. VI (Eqs. eq:Bt, ia, Fab, OS with the
resampling of Sec. VI.A) taken off the Fourier grid, and dF/d(f0, f1, alpha, delta)
by the chain rule through the resampling.

Test infrastructure only (see the package docstring).

For theta = (f0, f1, alpha, delta) and the barycentric output grid tau_j = j dt, j < N:

  t_j solves t_j + phi_m(t_j) = tau_j                                  (Eq. eq:Bt)
  x~_j = x(t_j) by Fourier x2 and the natural cubic spline          (Sec. VI.A)
  Psi_j = fl phi_m(t_j) + f1 (t_j^2/2 + t_j phi_m(t_j)) + f0 tau_j      [cycles]
  Sa = sum_j x~_j a(t_j) exp(-2 pi i Psi_j),   Sb likewise with b
  F = c (|Sa|^2 / <a^2> + |Sb|^2 / <b^2>),  c = 2 dt / (S0 N),  <a^2> the mean of a(t_j)^2.

At f0 = k / (Nfft dt) the last phase term is j k / Nfft and F is the coarse search's
F_k (the zero-padded DFT of Eq. eq:DFT at bin k); between Fourier frequencies it is
the same sum off the grid.

Derivatives.  tau_j is fixed and t_j moves with the sky; differentiating Eq. eq:Bt
(partial derivatives of phi_m taken at t_j):

  dt_j/dsky = -(d phi_m/dsky) / (1 + d phi_m/dt),
  dx~_j/dsky = x~'(t_j) dt_j/dsky                 (the spline's slope),
  da_j/dalpha = a_x (1 - Omega_r dt_j/dalpha),     a_x = da/dx, x = alpha - theta(t),
  da_j/ddelta = a_delta - Omega_r a_x dt_j/ddelta,   a_delta through the coefficients,
  dPsi_j/dsky = dt_j/dsky (f1 phi_m(t_j) - fl)       (since phi_m(t_j) = tau_j - t_j),
  dPsi_j/df0 = tau_j,   dPsi_j/df1 = t_j^2/2 + t_j phi_m(t_j),
  dSa = sum_j [d(x~ a)_j - 2 pi i x~_j a_j dPsi_j] exp(-2 pi i Psi_j),
  d<a^2> = 2 mean(a da),
  dF = c [2 Re(conj(Sa) dSa) / <a^2> - |Sa|^2 d<a^2> / <a^2>^2 + (the same for b)].

Only the analytic Earth of ``earth`` is supported (a caller's position table is not).
"""
from __future__ import annotations

import math

import numpy as np

from . import earth, resample, response
from .refine import _ab_coefficients_ddelta


def _check_detector(det):
    if isinstance(det, earth.TabulatedDetector):
        raise NotImplementedError("the resampled F's gradient takes the analytic Earth only")


def source_time_sky_derivatives(t: np.ndarray, alpha: float, delta: float, det):
    """dt_j/dalpha and dt_j/ddelta at the source times t (Eq. eq:Bt differentiated with
    tau_j fixed): -(d phi_m/dsky) / (1 + d phi_m/dt), phi_m = n0 . r_d / c."""
    _check_detector(det)
    ca, sa, cd, sd = math.cos(alpha), math.sin(alpha), math.cos(delta), math.sin(delta)
    R = earth.ecliptic_rotation(det.eps)
    n0 = R @ np.array([ca * cd, sa * cd, sd])
    n0_a = R @ np.array([-sa * cd, ca * cd, 0.0])
    n0_d = R @ np.array([-ca * sd, -sa * sd, cd])
    rd = earth.detector_position_ls(t, det)
    vd = earth.detector_velocity_ls(t, det)
    den = 1.0 + n0 @ vd
    return -(n0_a @ rd) / den, -(n0_d @ rd) / den


def resampled_terms(seg: resample.Segment, theta, fl: float, det, grad: bool = False):
    """The sums F is made of: Sa, Sb (complex), <a^2>, <b^2>; with grad=True also their
    derivatives along (f0, f1, alpha, delta): dSa, dSb (complex, shape (4,)) and dA2,
    dB2 (shape (4,)).  Returned as a dict."""
    f0, f1, alpha, delta = (float(v) for v in theta)
    n, dt = seg.n, seg.dt
    tau = np.arange(n, dtype=np.float64) * dt
    t = resample.source_times(tau, alpha, delta, det)
    pm = earth.phi_m(t, alpha, delta, det)
    xr = seg.interpolate(t)
    a, b = response.ab(t, alpha, delta, det)
    psi = fl * pm + f1 * (0.5 * t * t + t * pm) + f0 * tau
    e = np.exp(-2j * math.pi * (psi - np.floor(psi)))
    out = dict(Sa=np.dot(xr * a, e), Sb=np.dot(xr * b, e), A2=float(np.mean(a * a)), B2=float(np.mean(b * b)))
    if not grad:
        return out
    t_a, t_d = source_time_sky_derivatives(t, alpha, delta, det)
    xp = seg.interpolate_derivative(t)
    # a, b as functions of x = alpha - theta(t) and of delta through the coefficients
    x = alpha - earth.sidereal_angle(t, det)
    c1, s1, c2, s2 = np.cos(x), np.sin(x), np.cos(2 * x), np.sin(2 * x)
    ce, cf = response.ab_coefficients(delta, det)
    de, dfc = _ab_coefficients_ddelta(delta, det)
    a_x = -2 * ce["c2"] * s2 + 2 * ce["s2"] * c2 - ce["c1"] * s1 + ce["s1"] * c1
    b_x = -2 * cf["c2"] * s2 + 2 * cf["s2"] * c2 - cf["c1"] * s1 + cf["s1"] * c1
    a_dl = de["c2"] * c2 + de["s2"] * s2 + de["c1"] * c1 + de["s1"] * s1 + de["c0"]
    b_dl = dfc["c2"] * c2 + dfc["s2"] * s2 + dfc["c1"] * c1 + dfc["s1"] * s1
    w = earth.OMEGA_R
    zero = np.zeros(n)
    da = (zero, zero, a_x * (1.0 - w * t_a), a_dl - w * a_x * t_d)
    db = (zero, zero, b_x * (1.0 - w * t_a), b_dl - w * b_x * t_d)
    dx = (zero, zero, xp * t_a, xp * t_d)
    dpsi = (tau, 0.5 * t * t + t * pm, t_a * (f1 * pm - fl), t_d * (f1 * pm - fl))
    dSa = np.empty(4, dtype=np.complex128)
    dSb = np.empty(4, dtype=np.complex128)
    dA2 = np.empty(4)
    dB2 = np.empty(4)
    for i in range(4):
        dSa[i] = np.dot(dx[i] * a + xr * da[i] - 2j * math.pi * xr * a * dpsi[i], e)
        dSb[i] = np.dot(dx[i] * b + xr * db[i] - 2j * math.pi * xr * b * dpsi[i], e)
        dA2[i] = 2.0 * float(np.mean(a * da[i]))
        dB2[i] = 2.0 * float(np.mean(b * db[i]))
    out.update(dSa=dSa, dSb=dSb, dA2=dA2, dB2=dB2)
    return out


def resampled_fstat_point(seg: resample.Segment, theta, fl: float, det, S0: float, grad: bool = False):
    """F of the resampled series at theta = (f0, f1, alpha, delta); with grad=True
    (F, dF/dtheta (4,), scale (4,)), scale_i being the sum of the magnitudes of the
    terms that make dF/dtheta_i (the size it has before they cancel near a maximum)."""
    r = resampled_terms(seg, theta, fl, det, grad=grad)
    c = 2.0 * seg.dt / (S0 * seg.n)
    Pa, Pb = abs(r["Sa"]) ** 2, abs(r["Sb"]) ** 2
    F = c * (Pa / r["A2"] + Pb / r["B2"])
    if not grad:
        return F
    dF = np.empty(4)
    scale = np.empty(4)
    for i in range(4):
        ta = 2.0 * (np.conj(r["Sa"]) * r["dSa"][i]).real / r["A2"]
        tb = 2.0 * (np.conj(r["Sb"]) * r["dSb"][i]).real / r["B2"]
        ua = Pa * r["dA2"][i] / r["A2"] ** 2
        ub = Pb * r["dB2"][i] / r["B2"] ** 2
        dF[i] = c * (ta - ua + tb - ub)
        scale[i] = c * (2.0 * abs(r["Sa"]) * abs(r["dSa"][i]) / r["A2"] + abs(ua)
                        + 2.0 * abs(r["Sb"]) * abs(r["dSb"][i]) / r["B2"] + abs(ub))
    return F, dF, scale


def resampled_fine_search(seg: resample.Segment, theta0, fl: float, det, S0: float, scale, xatol: float = 1e-4,
                          maxiter: int = 2000):
    """Maximise the resampled F from theta0 with the Nelder-Mead simplex, in coordinates
    u = (theta - theta0) / scale (scale: about one correlation length per parameter)."""
    from scipy.optimize import minimize
    theta0 = np.asarray(theta0, dtype=np.float64)
    scale = np.asarray(scale, dtype=np.float64)
    res = minimize(lambda u: -resampled_fstat_point(seg, theta0 + u * scale, fl, det, S0), np.zeros(4),
                   method="Nelder-Mead", options=dict(xatol=xatol, fatol=1e-10, maxiter=maxiter,
                                                      initial_simplex=0.3 * np.vstack([np.zeros(4), np.eye(4)])))
    return theta0 + res.x * scale, -res.fun
