"""Seeded synthetic inputs for the coherent F-statistic search.

This module holds only input generation: the named workloads (segment length,
sampling, FFT length, template grid sizes), white Gaussian noise, the sky and
spindown grids, and random draws of injection parameters.  It contains none of
the method's arithmetic (no detector response, no phase model, no resampling,
no transform): both the CUDA path and the CPU oracle consume what it returns.

The workloads take the shape of the paper's narrow-band data (Sec. VII): a
real series in a narrow band whose lower edge is 435.1875 Hz, whole sidereal
days of observation, and zero padding to a power of two.  The paper's VSR1
data and JPL/IERS ephemerides are not available, so seeded white noise and an
analytic Earth stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SIDEREAL_DAY_S = 86164.0  # whole-second sidereal day used to size segments
BASE_SEED = 10030844       # seed base; the workload index is added to it


@dataclasses.dataclass(frozen=True)
class Detector:
    """Detector site and analytic-Earth parameters (all angles in radians).

    lat/lon: geodetic latitude and east longitude of the site (Sec. V, site
    coordinates); gamma: orientation of the arms' bisector counter-clockwise
    from local East (the gamma of the amplitude modulation functions);
    eps: obliquity of the ecliptic (Eq. pha4); lambda_e0: ecliptic longitude
    of the Earth seen from the SSB at t = 0; theta_g0: Greenwich sidereal angle
    at t = 0 (the local sidereal angle is theta_g0 + lon + Omega_r t).
    """

    lat: float = math.radians(43.63)
    lon: float = math.radians(10.50)
    gamma: float = math.radians(19.4)
    eps: float = math.radians(23.44)
    lambda_e0: float = 0.0
    theta_g0: float = 0.0


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    days: int           # whole sidereal days
    dt: float           # sampling interval [s]
    nfft: int           # zero-padded FFT length
    nsky: int
    nspin: int
    n_inj: int
    snr: tuple          # (lo, hi) target optimal SNR of each injection
    fl: float = 435.1875  # lower band edge [Hz] (Sec. VII)
    f1_range: tuple = (-1e-8, 0.0)
    f0_range: tuple = (0.05, 0.20)
    F_thr: float = 20.0
    sigma: float = 1.0
    interbin: bool = False  # F on the half-bin grid of an unpadded transform (Sec. VI.B)

    @property
    def n(self) -> int:
        return int(math.floor(self.days * SIDEREAL_DAY_S / self.dt))

    @property
    def nbins(self) -> int:
        return self.nfft if self.interbin else self.nfft // 2

    @property
    def S0(self) -> float:
        # one-sided spectral density of white noise with variance sigma^2
        return 2.0 * self.sigma ** 2 * self.dt


# Named workloads.  "single_fp64" is the 1-day single-template case; "grid_2d"
# is the 2-sidereal-day coarse grid (256 sky x 16 spindowns, 2^18 FFT).
WORKLOADS = {
    "single_fp64": Workload("single_fp64", days=1, dt=2.0, nfft=1 << 16, nsky=1, nspin=1,
                            n_inj=1, snr=(10.0, 10.0)),
    "grid_2d": Workload("grid_2d", days=2, dt=2.0, nfft=1 << 18, nsky=256, nspin=16,
                        n_inj=4, snr=(8.0, 20.0)),
    # the 2-day grid with interbinning in place of padding by two: transform of 2^17
    # points, F on the same 2^17-point half-bin grid as the padded 2^18 transform
    "grid_2d_ib": Workload("grid_2d_ib", days=2, dt=2.0, nfft=1 << 17, nsky=256, nspin=16,
                           n_inj=4, snr=(8.0, 20.0), interbin=True),
    "wide_6d": Workload("wide_6d", days=6, dt=0.5, nfft=1 << 21, nsky=512, nspin=32,
                        n_inj=8, snr=(8.0, 20.0), f0_range=(0.05, 0.95)),
    # small cases for tests: same structure, quick to evaluate on the CPU
    "tiny": Workload("tiny", days=1, dt=64.0, nfft=1 << 12, nsky=3, nspin=2,
                     n_inj=1, snr=(30.0, 30.0), f0_range=(0.001, 0.006), F_thr=15.0),
    "small": Workload("small", days=1, dt=8.0, nfft=1 << 14, nsky=4, nspin=3,
                      n_inj=2, snr=(25.0, 40.0), f0_range=(0.005, 0.05), F_thr=15.0),
}

# The constrained-lattice workload on the 2-day data of "grid_2d": the A4* lattice of
# minimal match LATTICE_MATCH (Sec. IV) over this patch of ecliptic (n_x, n_y) near
# the ecliptic pole, spindowns in the grid's range.
LATTICE_BOX = (0.30, 0.45, -0.10, 0.05)
LATTICE_MATCH = 0.75


@dataclasses.dataclass(frozen=True)
class BatchWorkload:
    """Many segments of uneven length searched with one template grid (the
    coherent first stage of a hierarchical search, Sec. I).  `parts` lists
    (days, nfft, count) per kind of segment; the kinds are interleaved and the
    segments follow each other in time without gaps."""
    name: str
    parts: tuple
    dt: float
    nsky: int
    nspin: int
    n_inj: int          # injections per segment
    snr: tuple
    fl: float = 435.1875
    f1_range: tuple = (-1e-8, 0.0)
    f0_range: tuple = (0.05, 0.20)
    F_thr: float = 20.0
    sigma: float = 1.0

    def segments(self) -> list:
        """One Workload per segment (name "<batch>/<index>") in time order."""
        out = []
        for c in range(max(p[2] for p in self.parts)):
            for days, nfft, count in self.parts:
                if c < count:
                    out.append(Workload("%s/%d" % (self.name, len(out)), days=days, dt=self.dt, nfft=nfft,
                                        nsky=self.nsky, nspin=self.nspin, n_inj=self.n_inj, snr=self.snr,
                                        fl=self.fl, f1_range=self.f1_range, f0_range=self.f0_range,
                                        F_thr=self.F_thr, sigma=self.sigma))
        return out

    def epochs(self) -> np.ndarray:
        """Start time [s] of each segment after the first one's start."""
        segs = self.segments()
        t = np.zeros(len(segs))
        for i in range(1, len(segs)):
            t[i] = t[i - 1] + segs[i - 1].n * segs[i - 1].dt
        return t


# Batches of uneven segments: 16 each of 1, 2, 3 and 6 sidereal days with
# transforms of 2^16, 2^18, 2^18 and 2^20 points, 4096 sky x 64 spindowns, and
# a small one for tests.
BATCHES = {
    "uneven_64": BatchWorkload("uneven_64", parts=((1, 1 << 16, 16), (2, 1 << 18, 16), (3, 1 << 18, 16),
                                                   (6, 1 << 20, 16)),
                               dt=2.0, nsky=4096, nspin=64, n_inj=1, snr=(10.0, 20.0)),
    "uneven_small": BatchWorkload("uneven_small", parts=((1, 1 << 12, 2), (2, 1 << 13, 1), (3, 1 << 14, 1)),
                                  dt=64.0, nsky=3, nspin=2, n_inj=1, snr=(30.0, 30.0), f0_range=(0.001, 0.006),
                                  F_thr=15.0),
}


def rng_for(workload: str, stream: int = 0) -> np.random.Generator:
    """Seeded generator of a named workload, or of segment i of a batch ("<batch>/<i>")."""
    if "/" in workload:
        batch, i = workload.split("/")
        idx = 100 + list(BATCHES).index(batch)
        return np.random.default_rng([BASE_SEED + idx, 1000 + int(i), stream])
    if workload in BATCHES:
        return np.random.default_rng([BASE_SEED + 100 + list(BATCHES).index(workload), stream])
    idx = list(WORKLOADS).index(workload)
    return np.random.default_rng([BASE_SEED + idx, stream])


def noise(wl: Workload, seed_stream: int = 1, rng: np.random.Generator | None = None) -> np.ndarray:
    """White Gaussian noise N(0, sigma^2), float64 array of length wl.n."""
    g = rng if rng is not None else rng_for(wl.name, seed_stream)
    return wl.sigma * g.standard_normal(wl.n)


def detector_for(wl, seed_stream: int = 2) -> Detector:
    """The detector of the paper's simulations; the orbital phase at t = 0 is seeded
    (a batch's segments share the detector of the batch)."""
    g = rng_for(wl.name.split("/")[0], seed_stream)
    return Detector(lambda_e0=float(g.uniform(0.0, 2.0 * math.pi)))


def sky_grid(n: int):
    """Fibonacci lattice on the sphere: n (alpha, delta) pairs, quasi-uniform."""
    i = np.arange(n, dtype=np.float64)
    golden = (1.0 + math.sqrt(5.0)) / 2.0
    alpha = 2.0 * math.pi * np.mod(i * golden, 1.0)
    sin_delta = 1.0 - (2.0 * i + 1.0) / n
    delta = np.arcsin(sin_delta)
    return alpha, delta


def spin_grid(n: int, lo: float, hi: float) -> np.ndarray:
    """n spindowns evenly spaced over [lo, hi], both ends included."""
    if n == 1:
        return np.array([lo], dtype=np.float64)
    return np.linspace(lo, hi, n, dtype=np.float64)


@dataclasses.dataclass(frozen=True)
class Injection:
    f0: float     # frequency offset above the band edge at the SSB, t = 0 [Hz]
    f1: float     # spindown [Hz/s]
    alpha: float
    delta: float
    psi: float
    cos_iota: float
    phi0: float
    snr: float    # target optimal SNR; the amplitude h0 is fixed from it


def injections(wl: Workload, seed_stream: int = 3, on_bin: bool = False) -> list:
    """Random injection parameters: isotropic sky, uniform psi, cos(iota), phi0.

    With on_bin=True the frequency is rounded to the nearest Fourier bin of the
    zero-padded transform (so the peak lands exactly on a bin).
    """
    g = rng_for(wl.name, seed_stream)
    out = []
    for _ in range(wl.n_inj):
        f0 = float(g.uniform(*wl.f0_range))
        if on_bin:
            df = 1.0 / (wl.nfft * wl.dt)
            f0 = round(f0 / df) * df
        f1 = -1e-9 if wl.name == "single_fp64" else float(g.uniform(*wl.f1_range))
        out.append(Injection(
            f0=f0, f1=f1,
            alpha=float(g.uniform(0.0, 2.0 * math.pi)),
            delta=float(math.asin(g.uniform(-1.0, 1.0))),
            psi=float(g.uniform(0.0, math.pi)),
            cos_iota=float(g.uniform(-1.0, 1.0)),
            phi0=float(g.uniform(0.0, 2.0 * math.pi)),
            snr=float(g.uniform(*wl.snr)),
        ))
    return out
