"""Shared test helpers: seeded cases built from the workload generators and
the oracle's injection model, and the F / candidate comparison rules."""
import math
import os

import numpy as np

from oracle import fstat as ofs
from oracle import resample as ors
from oracle import response as orsp
from paper_1003_0844_gb300 import workloads as W

# Parity bar for the FP32 path: max_k |F - F_ref| / max(F_ref, 1) <= 1e-4.
F32_TOL = 1e-4
# FP64 path: both sides in double; differences come from summation order and
# the ~1e6-rad heterodyne phase (spacing ~2e-10 rad).
F64_TOL = 1e-8


def make_case(name, inject=True, seed_stream=1, n=None, nfft=None, nsky=None, nspin=None):
    """(workload, detector, x, alpha, delta, f1) for a named workload, optionally resized."""
    wl = W.WORKLOADS[name]
    if n is not None or nfft is not None or nsky is not None or nspin is not None:
        import dataclasses
        kw = {}
        if nfft is not None:
            kw["nfft"] = nfft
        if nsky is not None:
            kw["nsky"] = nsky
        if nspin is not None:
            kw["nspin"] = nspin
        wl = dataclasses.replace(wl, **kw)
    det = W.detector_for(wl)
    N = wl.n if n is None else n
    x = W.noise(wl, seed_stream)[:N] if N <= wl.n else np.random.default_rng(seed_stream).standard_normal(N)
    if inject:
        x = x + orsp.inject(N, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)
    alpha, delta = W.sky_grid(wl.nsky)
    f1 = W.spin_grid(wl.nspin, *wl.f1_range)
    return wl, det, x, alpha, delta, f1


def oracle_F(x, wl, det, alpha, delta, f1, nbins=None, interp="spline", seg=None):
    """Oracle F for every template (FFT mode), shape (nsky*nspin, nbins)."""
    if seg is None:
        seg = ors.Segment(x, wl.dt)
    nb = wl.nfft // 2 if nbins is None else nbins
    out = np.empty((len(alpha) * len(f1), nb))
    for s in range(len(alpha)):
        for m in range(len(f1)):
            out[s * len(f1) + m] = ofs.fstat(seg, alpha[s], delta[s], f1[m], wl.fl, det, wl.S0, wl.nfft,
                                             nbins=nb, interp=interp)
    return out


def max_rel_dF(F, Fref):
    return float(np.max(np.abs(F - Fref) / np.maximum(Fref, 1.0)))


def check_candidates(sky, spin, bins, Fc, Fref, thr, nspin, rel=1e-4):
    """Candidate rule: every (template, bin) with F_ref > thr (1 + rel) is found,
    and no candidate has F_ref < thr (1 - rel); bins inside the band are free."""
    got = set(zip((sky * nspin + spin).tolist(), bins.tolist()))
    t_idx, b_idx = np.nonzero(Fref > thr * (1 + rel))
    must = set(zip(t_idx.tolist(), b_idx.tolist()))
    missing = must - got
    bad = [(t, b) for (t, b) in got if Fref[t, b] < thr * (1 - rel)]
    return missing, bad


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    """Values of a fixture under tests/golden/ ("key = value  # comment" lines)."""
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (x.strip() for x in line.split("=", 1))
            out[k] = float(v)
    return out
