"""Pins of the oracle's FFT search of the constrained lattice (Sec. IV, Sec. VII):
F off the Fourier grid against the direct sum at the shifted frequency, the offset
of one bin against the next bin, and the templates against the lattice itself
(every template line holds lattice nodes only, and a brute-force sweep of lattice
coefficients finds no node the templates miss)."""
import itertools
import math

import numpy as np
import pytest

from oracle import earth, fstat as ofs, grid as og, resample as ors, response as orsp
from paper_1003_0844_gb300 import workloads as W


def _seg(name="tiny"):
    wl = W.WORKLOADS[name]
    det = W.detector_for(wl)
    x = W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)
    return wl, det, x, ors.Segment(x, wl.dt)


def test_fractional_bin_is_the_direct_sum_at_the_shifted_frequency():
    wl, det, x, seg = _seg()
    a, d, f1, off = 1.1, -0.3, -4e-9, 0.37
    ks = [0, 5, 91, wl.nfft // 2 - 1]
    F = ofs.fstat(seg, a, d, f1, wl.fl, det, wl.S0, wl.nfft, bin_offset=off)
    dm = ofs.demodulate(seg, a, d, f1, wl.fl, det)
    j = np.arange(wl.n, dtype=np.float64)
    for k in ks:
        e = np.exp(-2j * math.pi * j * (k + off) / wl.nfft)
        Fa, Fb = wl.dt * np.dot(dm.ya, e), wl.dt * np.dot(dm.yb, e)
        ref = 2.0 / (wl.S0 * wl.n * wl.dt) * (abs(Fa) ** 2 / dm.a2 + abs(Fb) ** 2 / dm.b2)
        assert F[k] == pytest.approx(ref, rel=1e-10, abs=1e-12)


def test_offset_of_one_bin_is_the_next_bin():
    wl, det, x, seg = _seg()
    F0 = ofs.fstat(seg, 2.0, 0.5, -1e-9, wl.fl, det, wl.S0, wl.nfft)
    F1 = ofs.fstat(seg, 2.0, 0.5, -1e-9, wl.fl, det, wl.S0, wl.nfft, bin_offset=1.0)
    assert np.allclose(F1[:-1], F0[1:], rtol=1e-10, atol=1e-10 * F0.max())


def _lattice(name="small"):
    wl = W.WORKLOADS[name]
    det = W.detector_for(wl)
    G = og.linear_model_fisher(wl.n, wl.dt, det)
    dp0 = 2 * math.pi / (wl.nfft * wl.dt)
    gen, _, _ = og.constrained_lattice(G, 0.75, dp0)
    return wl, det, gen


def test_templates_are_lattice_nodes_and_complete():
    wl, det, B = _lattice()
    box = (0.30, 0.45, -0.10, 0.05)
    f1lo, f1hi = -2e-9, 0.0
    T = og.lattice_templates(B, det, wl.fl, wl.nfft, wl.dt, f1lo, f1hi, box=box)
    assert len(T) > 4
    tp = 2 * math.pi
    w_ref = tp * (wl.fl + 0.5 / wl.dt)
    Binv = np.linalg.inv(B)
    ce, se = math.cos(det.eps), math.sin(det.eps)
    found = set()
    for alpha, delta, rows in T:
        n_eq = np.array([math.cos(alpha) * math.cos(delta), math.sin(alpha) * math.cos(delta), math.sin(delta)])
        ny = ce * n_eq[1] + se * n_eq[2]
        nx = n_eq[0]
        assert box[0] - 1e-12 <= nx <= box[1] + 1e-12 and box[2] - 1e-12 <= ny <= box[3] + 1e-12
        for f1, d, k1 in rows:
            assert 0.0 <= d < 1.0 and f1lo <= f1 <= f1hi
            for k in (0, 17, wl.nfft // 2 - 1):
                node = np.array([tp * (wl.fl + (k + d) / (wl.nfft * wl.dt)), tp * f1, w_ref * ny, w_ref * nx])
                c = node @ Binv
                assert np.allclose(c, np.rint(c), atol=1e-6), c
                assert int(np.rint(c[1])) == k1
            found.add((int(np.rint(c[1])), int(np.rint(c[2])), int(np.rint(c[3]))))
    # brute force over a wider coefficient box: every lattice line with its sky node in the
    # box and its spindown in range is among the templates
    S = B[2:4, 2:4]
    k23 = np.linalg.solve(S.T, np.array([[w_ref * box[2], w_ref * box[0]], [w_ref * box[3], w_ref * box[1]],
                                          [w_ref * box[2], w_ref * box[1]], [w_ref * box[3], w_ref * box[0]]]).T)
    lo, hi = np.floor(k23.min(axis=1)) - 3, np.ceil(k23.max(axis=1)) + 3
    want = set()
    for k2 in range(int(lo[0]), int(hi[0]) + 1):
        for k3 in range(int(lo[1]), int(hi[1]) + 1):
            a1, a2 = k2 * B[2, 2] + k3 * B[3, 2], k2 * B[2, 3] + k3 * B[3, 3]
            ny, nx = a1 / w_ref, a2 / w_ref
            if not (box[0] <= nx <= box[1] and box[2] <= ny <= box[3]) or nx * nx + ny * ny > 1:
                continue
            c1 = k2 * B[2, 1] + k3 * B[3, 1]
            for k1 in range(-400, 401):
                om1 = k1 * B[1, 1] + c1
                if tp * f1lo <= om1 <= tp * f1hi:
                    want.add((k1, k2, k3))
    assert want and want == found
