"""The F-statistic (oracle, FP64): Eqs. OS, Fab, ia, eq:DFT, PF.

Test infrastructure only (see the package docstring).

For a template (alpha, delta, f1) and a segment x_k = x(k dt), k < N:

 1. barycentric output grid t_b,j = j dt (j < N) and source times t_j with
    t_j + phi_m(t_j) = t_b,j (Eq. eq:Bt);
 2. x~_j = x(t_j) by Fourier x2 + cubic spline (Sec. VI.A), a_j = a(t_j),
    b_j = b(t_j);
 3. the frequency-independent part of the phase of the narrow-band series
    Phi_j = fl phi_m(t_j) + f1 (t_j^2/2 + t_j phi_m(t_j))  [cycles]
    (Eq. phas with one spindown, plus the heterodyne term);
 4. y^a_j = x~_j a_j exp(-2 pi i Phi_j), y^b_j likewise with b_j;
 5. Fa_k = dt sum_j y^a_j exp(-2 pi i j k / Nfft), the zero-padded DFT of
    Eq. eq:DFT evaluated at the Fourier frequencies f0_k = k / (Nfft dt);
 6. F_k = 2 / (S0 To) (|Fa_k|^2 / <a^2> + |Fb_k|^2 / <b^2>) with To = N dt
    and <a^2>, <b^2> the means of a_j^2, b_j^2 over the N output samples.

Step 5 is either a direct sum at each requested bin (twiddles looked up by
the exact integer (j k mod Nfft)) or, for whole spectra, numpy's FFT.
"""
from __future__ import annotations

import math

import numpy as np

from . import earth, resample, response


class Demodulated:
    """Resampled, demodulated series of one template (steps 1-4)."""

    def __init__(self, ya, yb, a2, b2, t_src, phase_cycles):
        self.ya = ya
        self.yb = yb
        self.a2 = a2          # <a^2>
        self.b2 = b2          # <b^2>
        self.t_src = t_src
        self.phase_cycles = phase_cycles


def demodulate(seg: resample.Segment, alpha: float, delta: float, f1: float, fl: float, det,
               interp: str = "spline") -> Demodulated:
    n, dt = seg.n, seg.dt
    tb = np.arange(n, dtype=np.float64) * dt
    t = resample.source_times(tb, alpha, delta, det)
    pm = earth.phi_m(t, alpha, delta, det)
    xr = seg.interpolate(t) if interp == "spline" else seg.nearest(t)
    a, b = response.ab(t, alpha, delta, det)
    phase = fl * pm + f1 * (0.5 * t * t + t * pm)
    # reduce the phase to [0, 1) cycles in FP64 before the complex exponential
    frac = phase - np.floor(phase)
    rot = np.exp(-2j * math.pi * frac)
    return Demodulated(xr * a * rot, xr * b * rot, float(np.mean(a * a)), float(np.mean(b * b)),
                       t, phase)


def dft_direct(y: np.ndarray, nfft: int, bins) -> np.ndarray:
    """X_k = sum_j y_j exp(-2 pi i j k / Nfft) by direct summation (Eq. eq:DFT)."""
    y = np.asarray(y, dtype=np.complex128)
    j = np.arange(y.size, dtype=np.int64)
    tw = np.exp(-2j * math.pi * np.arange(nfft, dtype=np.float64) / nfft)
    out = np.empty(len(bins), dtype=np.complex128)
    for i, k in enumerate(bins):
        out[i] = np.dot(y, tw[(j * int(k)) % nfft])
    return out


def dft_fft(y: np.ndarray, nfft: int, nbins: int) -> np.ndarray:
    """First nbins coefficients of the length-Nfft DFT of y zero-padded (numpy FFT)."""
    return np.fft.fft(np.asarray(y, dtype=np.complex128), n=nfft)[:nbins]


def fstat_from_transforms(Xa, Xb, dm: Demodulated, n: int, dt: float, S0: float) -> np.ndarray:
    To = n * dt
    Fa = dt * Xa
    Fb = dt * Xb
    return 2.0 / (S0 * To) * (np.abs(Fa) ** 2 / dm.a2 + np.abs(Fb) ** 2 / dm.b2)


def fstat(seg: resample.Segment, alpha, delta, f1, fl, det, S0, nfft, bins=None, nbins=None,
          interp="spline", bin_offset=0.0):
    """F on the requested bins (direct sums) or on bins [0, nbins) (FFT).

    bin_offset: F at the frequencies (k + bin_offset) / (Nfft dt) instead of the
    Fourier frequencies: X(k + d) = sum_j y_j exp(-2 pi i j (k + d) / Nfft) is the
    DFT at bin k of y_j exp(-2 pi i d j / Nfft) (Eq. eq:DFT off the Fourier grid;
    used to search lattice nodes that fall between Fourier frequencies, Sec. IV)."""
    dm = demodulate(seg, alpha, delta, f1, fl, det, interp=interp)
    if bin_offset:
        j = np.arange(seg.n, dtype=np.float64)
        c = bin_offset * j / nfft
        rot = np.exp(-2j * math.pi * (c - np.floor(c)))
        dm.ya = dm.ya * rot
        dm.yb = dm.yb * rot
    if bins is not None:
        Xa = dft_direct(dm.ya, nfft, bins)
        Xb = dft_direct(dm.yb, nfft, bins)
    else:
        nb = nfft // 2 if nbins is None else nbins
        Xa = dft_fft(dm.ya, nfft, nb)
        Xb = dft_fft(dm.yb, nfft, nb)
    return fstat_from_transforms(Xa, Xb, dm, seg.n, seg.dt, S0)


def fstat_interbinned(seg: resample.Segment, alpha, delta, f1, fl, det, S0, nfft, interp="spline"):
    """F on the half-bin grid f = j / (2 Nfft dt), j < Nfft, from a length-Nfft DFT and
    interbinning (Eq. intbin, Sec. VI.B): even j = 2k take X(k); odd j = 2k+1 take
    X(k + 1/2) ~ (X(k+1) - X(k)) / sqrt(2), for both Fa and Fb."""
    dm = demodulate(seg, alpha, delta, f1, fl, det, interp=interp)
    nb = nfft // 2
    Xa = np.fft.fft(np.asarray(dm.ya, dtype=np.complex128), n=nfft)[:nb + 1]
    Xb = np.fft.fft(np.asarray(dm.yb, dtype=np.complex128), n=nfft)[:nb + 1]
    Ha = (Xa[1:] - Xa[:-1]) / math.sqrt(2.0)
    Hb = (Xb[1:] - Xb[:-1]) / math.sqrt(2.0)
    out = np.empty(2 * nb)
    out[0::2] = fstat_from_transforms(Xa[:nb], Xb[:nb], dm, seg.n, seg.dt, S0)
    out[1::2] = fstat_from_transforms(Ha, Hb, dm, seg.n, seg.dt, S0)
    return out


def fstat_exact(x: np.ndarray, dt: float, alpha, delta, f1, fl, det, S0, f0s) -> np.ndarray:
    """F of Eqs. OS/Fab by direct summation over the original samples, no resampling.

    Fa(f0) = dt sum_k x_k a(t_k) exp(-2 pi i Phi(t_k; f0)) with the full
    heterodyned phase Phi = f0 (t + phi_m) + fl phi_m + f1 (t^2/2 + t phi_m),
    and <a^2> the mean of a(t_k)^2 over the samples.
    """
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    t = np.arange(n, dtype=np.float64) * dt
    pm = earth.phi_m(t, alpha, delta, det)
    a, b = response.ab(t, alpha, delta, det)
    base = fl * pm + f1 * (0.5 * t * t + t * pm)
    tb = t + pm
    a2, b2 = float(np.mean(a * a)), float(np.mean(b * b))
    To = n * dt
    out = np.empty(len(f0s))
    for i, f0 in enumerate(f0s):
        ph = f0 * tb + base
        ph = ph - np.floor(ph)
        rot = np.exp(-2j * math.pi * ph)
        Fa = dt * np.dot(x * a, rot)
        Fb = dt * np.dot(x * b, rot)
        out[i] = 2.0 / (S0 * To) * (abs(Fa) ** 2 / a2 + abs(Fb) ** 2 / b2)
    return out


def candidates(F: np.ndarray, thr: float):
    """Threshold crossings of an F array of shape (..., nbins): index tuples with F > thr."""
    idx = np.nonzero(F > thr)
    return idx, F[idx]


def false_alarm_probability(F0):
    """P_F(F0) = (1 + F0) exp(-F0): survival of F when 2F ~ chi^2 with 4 dof (Eq. PF)."""
    F0 = np.asarray(F0, dtype=np.float64)
    return (1.0 + F0) * np.exp(-F0)


def search_false_alarm(F0, n_cells):
    """False-alarm probability of a search over n_cells independent cells,
    alpha = 1 - (1 - P_F(F0))^Nc (Eq. FP), and the expected number of false
    alarms Nc P_F(F0) (Eq. NF)."""
    P = float(false_alarm_probability(F0))
    # 1 - (1 - P)^Nc written with log1p/expm1 so that it keeps its digits when P is tiny
    return -math.expm1(n_cells * math.log1p(-P)) if P < 1.0 else 1.0, n_cells * P


def threshold_for_false_alarm(alpha: float, n_cells: float) -> float:
    """The threshold F0 whose search false-alarm probability is alpha (Eq. FP
    inverted), by bracketing and bisection on the definition."""
    from scipy.optimize import brentq
    f = lambda F0: search_false_alarm(F0, n_cells)[0] - alpha
    if f(0.0) <= 0.0:
        return 0.0
    hi = 1.0
    while f(hi) > 0.0:
        hi *= 2.0
    return brentq(f, 0.0, hi, xtol=1e-14, rtol=1e-15)


def cell_count(G, v_total: float) -> float:
    """N_c = V_total / V_cell with V_cell = pi^(M/2) / (Gamma(M/2 + 1) sqrt(det G))
    (Eqs. NT, vc), G the M x M reduced Fisher matrix."""
    G = np.asarray(G, dtype=np.float64)
    M = G.shape[0]
    v_cell = math.pi ** (M / 2) / (math.gamma(M / 2 + 1) * math.sqrt(np.linalg.det(G)))
    return v_total / v_cell
