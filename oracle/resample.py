"""Resampling to barycentric time (oracle, FP64), Sec. VI.A.

Test infrastructure only (see the package docstring).

Readings taken where the paper is silent:
  * the upsampler pads the DFT with N zeros in the middle (between the
    positive and negative frequencies); for even N the Nyquist coefficient is
    split in equal halves between bins N/2 and 3N/2 of the 2N grid, and the
    result is scaled so that the even samples reproduce the input exactly;
  * the spline is the natural cubic spline (zero second derivative at both
    ends) through all 2N upsampled points at unit spacing (dt/2);
  * the interpolated series is zero where the source time falls outside
    [0, (N-1) dt];
  * the source time solves t + phi_m(t) = t_b exactly (fixed-point
    iteration), and the Jacobian dt/dt_b is dropped, as in Eq. ia.
"""
from __future__ import annotations

import numpy as np

from . import earth


def fourier_upsample2(x: np.ndarray) -> np.ndarray:
    """Fourier x2 upsampling: DFT, pad with N zeros, inverse DFT of length 2N."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    X = np.fft.fft(x)
    Y = np.zeros(2 * n, dtype=np.complex128)
    if n % 2 == 0:
        h = n // 2
        Y[:h] = X[:h]
        Y[h] = 0.5 * X[h]
        Y[2 * n - h] = 0.5 * X[h]
        Y[2 * n - h + 1:] = X[h + 1:]
    else:
        h = (n + 1) // 2
        Y[:h] = X[:h]
        Y[2 * n - (n - h):] = X[h:]
    # numpy's inverse carries 1/(2N); the factor 2 restores the amplitude
    return 2.0 * np.fft.ifft(Y).real


def natural_spline_second_derivatives(y: np.ndarray) -> np.ndarray:
    """Second derivatives M of the natural cubic spline through y at unit spacing.

    M_0 = M_{n-1} = 0 and M_{i-1} + 4 M_i + M_{i+1} = 6 (y_{i+1} - 2 y_i + y_{i-1})
    for the interior points, solved by forward elimination and back
    substitution (the Thomas algorithm).
    """
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    M = np.zeros(n)
    m = n - 2
    if m <= 0:
        return M
    rhs = 6.0 * (y[2:] - 2.0 * y[1:-1] + y[:-2])
    cp = np.empty(m)
    dp = np.empty(m)
    cp[0] = 1.0 / 4.0
    dp[0] = rhs[0] / 4.0
    for i in range(1, m):
        den = 4.0 - cp[i - 1]
        cp[i] = 1.0 / den
        dp[i] = (rhs[i] - dp[i - 1]) / den
    sol = np.empty(m)
    sol[-1] = dp[-1]
    for i in range(m - 2, -1, -1):
        sol[i] = dp[i] - cp[i] * sol[i + 1]
    M[1:-1] = sol
    return M


def spline_eval(y: np.ndarray, M: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Evaluate the cubic spline with knot values y and second derivatives M at u.

    Standard form on the interval [i, i+1] with f = u - i:
      S = (1-f) y_i + f y_{i+1} + ((1-f)^3 - (1-f)) M_i / 6 + (f^3 - f) M_{i+1} / 6.
    u must lie in [0, n-1].
    """
    u = np.asarray(u, dtype=np.float64)
    n = y.size
    i = np.minimum(np.floor(u).astype(np.int64), n - 2)
    f = u - i
    g = 1.0 - f
    return g * y[i] + f * y[i + 1] + ((g ** 3 - g) * M[i] + (f ** 3 - f) * M[i + 1]) / 6.0


def spline_eval_derivative(y: np.ndarray, M: np.ndarray, u: np.ndarray) -> np.ndarray:
    """dS/du of the spline of spline_eval: on [i, i+1] with f = u - i, g = 1 - f,
      dS/du = y_{i+1} - y_i + ((1 - 3 g^2) M_i + (3 f^2 - 1) M_{i+1}) / 6."""
    u = np.asarray(u, dtype=np.float64)
    n = y.size
    i = np.minimum(np.floor(u).astype(np.int64), n - 2)
    f = u - i
    g = 1.0 - f
    return y[i + 1] - y[i] + ((1.0 - 3.0 * g * g) * M[i] + (3.0 * f * f - 1.0) * M[i + 1]) / 6.0


def source_times(tb: np.ndarray, alpha: float, delta: float, det, tol: float = 1e-10,
                 max_iter: int = 50) -> np.ndarray:
    """Solve t + phi_m(t) = t_b (Eq. eq:Bt) for the source time t by fixed-point iteration.

    Stops when the largest step is below tol or below 8 FP64 spacings of the
    largest time (the finer of the two that FP64 can resolve)."""
    tb = np.asarray(tb, dtype=np.float64)
    t = tb.copy()
    if tb.size:
        tol = max(tol, 8.0 * np.spacing(np.max(np.abs(tb)) + 600.0))
    for _ in range(max_iter):
        t_new = tb - earth.phi_m(t, alpha, delta, det)
        step = np.max(np.abs(t_new - t)) if t.size else 0.0
        t = t_new
        if step < tol:
            # one more pass to settle the last rounding
            return tb - earth.phi_m(t, alpha, delta, det)
    raise RuntimeError("source-time iteration did not converge")


class Segment:
    """Template-independent part of the resampler for one data segment:
    the x2 upsampled series and its natural-spline second derivatives."""

    def __init__(self, x: np.ndarray, dt: float):
        self.x = np.asarray(x, dtype=np.float64)
        self.n = self.x.size
        self.dt = float(dt)
        self.x2 = fourier_upsample2(self.x)
        self.M = natural_spline_second_derivatives(self.x2)

    def interpolate(self, t: np.ndarray) -> np.ndarray:
        """x at source times t via the spline on the x2 grid; 0 outside [0, (N-1) dt]."""
        t = np.asarray(t, dtype=np.float64)
        inside = (t >= 0.0) & (t <= (self.n - 1) * self.dt)
        out = np.zeros(t.size)
        u = 2.0 * t[inside] / self.dt
        out[inside] = spline_eval(self.x2, self.M, u)
        return out

    def interpolate_derivative(self, t: np.ndarray) -> np.ndarray:
        """d/dt of interpolate: the spline's slope times du/dt = 2/dt; 0 outside [0, (N-1) dt]."""
        t = np.asarray(t, dtype=np.float64)
        inside = (t >= 0.0) & (t <= (self.n - 1) * self.dt)
        out = np.zeros(t.size)
        out[inside] = spline_eval_derivative(self.x2, self.M, 2.0 * t[inside] / self.dt) * (2.0 / self.dt)
        return out

    def nearest(self, t: np.ndarray) -> np.ndarray:
        """Nearest-neighbour ("stroboscopic") resampling of Sec. VI.A; 0 outside the data."""
        t = np.asarray(t, dtype=np.float64)
        k = np.rint(t / self.dt).astype(np.int64)
        inside = (k >= 0) & (k < self.n)
        out = np.zeros(t.size)
        out[inside] = self.x[k[inside]]
        return out
