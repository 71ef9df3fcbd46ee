"""Analytic Earth model for the detector-to-SSB delay (oracle, FP64).

Test infrastructure only (see the package docstring).

The paper obtains the detector position from JPL ephemerides (Sec. V).  Here
the Earth moves on a circular 1 AU orbit in the ecliptic and rotates with the
NOVAS angular velocity; the site sits on the reference ellipsoid at zero
height.  All positions are returned in light-seconds.

A detector may instead carry a caller's table of its SSB position and velocity
on the sample grid (``TabulatedDetector``), standing in for the ephemeris files
of Sec. V: the delay then comes from the table, the sidereal angle (for a, b)
still from the site model.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299_792_458.0             # m/s
AU_M = 149_597_870_700.0            # m
OMEGA_R = 7.2921151467e-5           # rad/s, Earth rotation (Sec. V, NOVAS value)
SIDEREAL_YEAR_S = 365.25636 * 86400.0
OMEGA_O = 2.0 * math.pi / SIDEREAL_YEAR_S   # rad/s, orbital angular velocity
ELL_A_M = 6_378_140.0               # m, semi-major axis of the ellipsoid (Sec. V)
ELL_FLAT = 0.00335281               # flattening, NOVAS value (Sec. V)


def site_equatorial_radius_and_z(lat: float):
    """Site on the ellipsoid at zero height (Sec. V, site coordinates).

    Reduced latitude Psi = arctan(b tan(phi)/a); the equatorial component of
    the radius vector is a cos(Psi) and the polar component b sin(Psi), with
    b = a (1 - flattening).  Returns (r_e, z) in metres.
    """
    b = ELL_A_M * (1.0 - ELL_FLAT)
    psi = math.atan(b * math.tan(lat) / ELL_A_M)
    return ELL_A_M * math.cos(psi), b * math.sin(psi)


@dataclasses.dataclass(frozen=True, eq=False)
class TabulatedDetector:
    """A detector whose position r_d/c comes from a table on the segment's sample
    grid t_m = m dt, m = 0..n-1 (the role of the ephemerides of Sec. V).

    site: the detector (latitude, orientation, obliquity, sidereal angle: every
      attribute other than the position is read from it);
    r, v: arrays (3, n), r_d(t_m)/c in light-seconds and v_d(t_m)/c, components
      in the SSB frame of Eq. pha5 (ecliptic axes).
    Between and beyond the grid points the position is extrapolated linearly
    from the nearest grid point m, clamped to [0, n): r(t) = r_m + (t - t_m) v_m
    (the reading used for a table; inside the grid its error is at most
    |r''| dt^2 / 8 for a trajectory with acceleration r'')."""
    site: object
    r: np.ndarray
    v: np.ndarray
    dt: float

    def __getattr__(self, name):
        if name.startswith("__") or name in ("site", "r", "v", "dt"):
            raise AttributeError(name)
        return getattr(self.site, name)

    def position(self, t):
        t = np.asarray(t, dtype=np.float64)
        n = self.r.shape[1]
        m = np.clip(np.rint(t / self.dt), 0, n - 1).astype(np.int64)
        tau = t - m * self.dt
        return self.r[:, m] + tau * self.v[:, m]


def detector_at_epoch(det, t0: float):
    """The detector seen from a segment that starts t0 seconds after the
    detector's t = 0: the orbital longitude and the sidereal angle at the
    segment's first sample are those at t0 (Sec. V), and the segment keeps
    t = 0 at its first sample.  A table already holds the segment's own
    positions: only its site's sidereal angle moves."""
    if isinstance(det, TabulatedDetector):
        return dataclasses.replace(det, site=detector_at_epoch(det.site, t0))
    return dataclasses.replace(det, lambda_e0=det.lambda_e0 + OMEGA_O * t0, theta_g0=det.theta_g0 + OMEGA_R * t0)


def sidereal_angle(t, det):
    """Local sidereal angle theta(t) = theta_g0 + lon + Omega_r t (Sec. V)."""
    return det.theta_g0 + det.lon + OMEGA_R * np.asarray(t, dtype=np.float64)


def earth_orbit_ls(t, det):
    """SSB -> Earth centre in the SSB ecliptic frame, light-seconds (Eq. pha5, R_ES).

    Circular orbit of radius 1 AU in the ecliptic plane; ecliptic longitude
    lambda_e0 + Omega_o t.  Returns an array of shape (3, len(t)).
    """
    t = np.asarray(t, dtype=np.float64)
    lam = det.lambda_e0 + OMEGA_O * t
    r = AU_M / C_LIGHT
    return np.stack([r * np.cos(lam), r * np.sin(lam), np.zeros_like(t)])


def site_equatorial_ls(t, det):
    """Earth centre -> detector in the celestial (equatorial) frame, light-seconds.

    X = r_e cos(theta), Y = r_e sin(theta), Z = z (Sec. V).
    """
    r_e, z = site_equatorial_radius_and_z(det.lat)
    th = sidereal_angle(t, det)
    return np.stack([r_e * np.cos(th), r_e * np.sin(th), np.full_like(th, z)]) / C_LIGHT


def ecliptic_rotation(eps: float) -> np.ndarray:
    """The matrix of Eqs. pha4/pha5 taking celestial components to SSB-frame components."""
    c, s = math.cos(eps), math.sin(eps)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, s], [0.0, -s, c]])


def sky_vector(alpha: float, delta: float, eps: float) -> np.ndarray:
    """Unit vector n0 towards the source in the SSB frame (Eq. pha4)."""
    v = np.array([math.cos(alpha) * math.cos(delta), math.sin(alpha) * math.cos(delta), math.sin(delta)])
    return ecliptic_rotation(eps) @ v


def detector_position_ls(t, det):
    """r_d(t)/c in the SSB frame (Eq. pha5): R_ES + Rot(eps) R_E, or the table's
    position for a TabulatedDetector.  Shape (3, n)."""
    if isinstance(det, TabulatedDetector):
        return det.position(t)
    return earth_orbit_ls(t, det) + ecliptic_rotation(det.eps) @ site_equatorial_ls(t, det)


def detector_velocity_ls(t, det):
    """v_d(t)/c of the analytic model, the time derivative of detector_position_ls:
    Omega_o AU/c (-sin lambda, cos lambda, 0) + Rot(eps) Omega_r r_e/c (-sin theta, cos theta, 0)."""
    t = np.asarray(t, dtype=np.float64)
    lam = det.lambda_e0 + OMEGA_O * t
    orb = (AU_M / C_LIGHT) * OMEGA_O * np.stack([-np.sin(lam), np.cos(lam), np.zeros_like(t)])
    r_e, _ = site_equatorial_radius_and_z(det.lat)
    th = sidereal_angle(t, det)
    rot = (r_e / C_LIGHT) * OMEGA_R * np.stack([-np.sin(th), np.cos(th), np.zeros_like(th)])
    return orb + ecliptic_rotation(det.eps) @ rot


def tabulate(n: int, dt: float, det, r_fn=None, v_fn=None) -> TabulatedDetector:
    """A table of n grid points t_m = m dt from position and velocity functions
    of t (default: the analytic model of this module)."""
    t = np.arange(n, dtype=np.float64) * dt
    r = (r_fn or (lambda tt: detector_position_ls(tt, det)))(t)
    v = (v_fn or (lambda tt: detector_velocity_ls(tt, det)))(t)
    return TabulatedDetector(det, np.ascontiguousarray(r, dtype=np.float64),
                             np.ascontiguousarray(v, dtype=np.float64), float(dt))


def phi_m(t, alpha: float, delta: float, det):
    """phi_m(t) = n0 . r_d(t) / c in seconds (Eq. pham), by the explicit scalar
    product of Sec. II:

      cos(a)cos(d)(R_ES^x + R_E^x) + (sin(a)cos(d)cos(eps) + sin(d)sin(eps)) R_ES^y
      + sin(a)cos(d) R_E^y + sin(d) R_E^z

    For a TabulatedDetector: n0 . r(t) with n0 of Eq. pha4 and the table's r(t).
    """
    if isinstance(det, TabulatedDetector):
        return sky_vector(alpha, delta, det.eps) @ det.position(t)
    res = earth_orbit_ls(t, det)
    rE = site_equatorial_ls(t, det)
    ca, sa = math.cos(alpha), math.sin(alpha)
    cd, sd = math.cos(delta), math.sin(delta)
    ce, se = math.cos(det.eps), math.sin(det.eps)
    return (ca * cd * (res[0] + rE[0])
            + (sa * cd * ce + sd * se) * res[1]
            + sa * cd * rE[1] + sd * rE[2])
