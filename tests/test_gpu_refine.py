"""Fine search on the GPU (through the C ABI) against the oracle: exact F at
continuous points, its gradient and the reduced Fisher matrix, the autograd
wrapper, and the hill climb against the oracle's Nelder-Mead maximum."""
import math

import numpy as np
import pytest
import torch

from oracle import refine as orf
from oracle import response as orsp
from paper_1003_0844_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    from paper_1003_0844_gb300 import build, fstat
    build.build()
    fstat.load_library()
    return fstat


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _case(name="small", noise=True, snr=25.0):
    wl = W.WORKLOADS[name]
    det = W.detector_for(wl)
    inj = W.Injection(f0=0.0213 if name == "small" else 0.1234, f1=-4e-9, alpha=2.1, delta=0.45, psi=0.3,
                      cos_iota=0.4, phi0=1.1, snr=snr)
    x = orsp.inject(wl.n, wl.dt, [inj], wl.fl, det, wl.sigma)
    if noise:
        x = x + W.noise(wl)
    theta = np.array([inj.f0, inj.f1, inj.alpha, inj.delta])
    return wl, det, x, theta


def _points(th, width):
    offs = np.array([[0, 0, 0, 0], [0.7, -0.4, 0.3, 0.5], [-1.5, 0.8, -0.6, 0.2], [3.0, 2.0, -2.0, -1.0],
                     [0.1, 0.1, 5.0, -4.0]])
    return th + offs * width


@pytest.mark.parametrize("precision,name", [("f32", "small"), ("f64", "small"), ("f32", "grid_2d")])
def test_points_match_oracle(fs, precision, name):
    wl, det, x, th = _case(name)
    _, _, G0 = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True)
    width = 1.0 / np.sqrt(np.diag(G0))
    P = _points(th, width)
    ctx = fs.Context(det)
    xd = _dev(x, torch.float32 if precision == "f32" else torch.float64)
    seg = fs.Segment(ctx, xd, wl.dt, wl.nfft, wl.fl, wl.S0, precision=precision)
    F, g, m, h = fs.fstat_points(ctx, seg, _dev(P), grad=True, metric=True, hess=True)
    F2, g2, _ = fs.fstat_points(ctx, seg, _dev(P), grad=True)       # the variant without Hessian, metric
    assert ctx.sync_status() == 0
    assert torch.equal(F, F2) and torch.equal(g, g2)
    F, g, m, h = F.cpu().numpy(), g.cpu().numpy(), m.cpu().numpy(), h.cpu().numpy()
    xo = xd.double().cpu().numpy()   # the oracle sums the same samples the segment holds
    iu = np.triu_indices(4)
    for p in range(len(P)):
        Fr, gr, Gr, Hr = orf.fstat_point(xo, wl.dt, P[p], wl.fl, det, wl.S0, grad=True, hess=True)
        wd = 1.0 / np.sqrt(np.diag(Gr))
        assert abs(F[p] - Fr) <= 1e-9 * max(Fr, 1.0), (p, F[p], Fr)
        assert np.all(np.abs(g[p] - gr) <= 1e-7 * np.abs(gr) + 1e-8 * max(Fr, 1.0) / wd), (p, g[p], gr)
        scale = np.sqrt(np.outer(np.diag(Gr), np.diag(Gr)))[iu]
        assert np.all(np.abs(m[p] - Gr[iu]) <= 1e-9 * scale), (p, m[p], Gr[iu])
        hs = (max(Fr, 1.0) / np.outer(wd, wd))[iu]
        assert np.all(np.abs(h[p] - Hr[iu]) <= 1e-7 * np.abs(Hr[iu]) + 1e-8 * hs), (p, h[p], Hr[iu])


def test_autograd_and_central_differences(fs):
    wl, det, x, th = _case()
    _, _, G0 = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True)
    width = 1.0 / np.sqrt(np.diag(G0))
    P = _points(th, width)[:3]
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x), wl.dt, wl.nfft, wl.fl, wl.S0, precision="f64")
    pts = _dev(P).requires_grad_(True)
    F = fs.fstat_at(ctx, seg, pts)
    (F * torch.tensor([1.0, 2.0, -0.5], dtype=torch.float64, device="cuda")).sum().backward()
    _, g, _ = fs.fstat_points(ctx, seg, _dev(P))
    w = torch.tensor([1.0, 2.0, -0.5], dtype=torch.float64, device="cuda")[:, None]
    assert torch.allclose(pts.grad, w * g, rtol=0, atol=0)
    for i in range(4):
        h = 1e-3 * width[i]
        e = np.zeros((1, 4))
        e[0, i] = h
        Fp, _, _ = fs.fstat_points(ctx, seg, _dev(P + e), grad=False)
        Fm, _, _ = fs.fstat_points(ctx, seg, _dev(P - e), grad=False)
        fd = ((Fp - Fm) / (2 * h)).cpu().numpy()
        gi = g[:, i].cpu().numpy()
        Fv = F.detach().cpu().numpy()
        assert np.all(np.abs(fd - gi) <= 1e-4 * np.abs(gi) + 1e-5 * Fv / width[i]), (i, fd, gi)


def test_refine_reaches_the_nelder_mead_maximum(fs):
    wl, det, x, th = _case()
    _, _, G0 = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True)
    width = 1.0 / np.sqrt(np.diag(G0))
    starts = th + width * np.array([[0.9, -0.8, 0.7, -0.6], [-0.5, 0.6, 0.4, 0.9], [0.3, 0.3, -0.8, -0.2]])
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    x32 = _dev(x, torch.float32).double().cpu().numpy()
    F0, _, _ = fs.fstat_points(ctx, seg, _dev(starts), grad=False)
    prev = F0.cpu().numpy()
    for k in (1, 2, 4, 8):
        _, Fk = fs.refine(ctx, seg, _dev(starts), nsteps=k)
        Fk = Fk.cpu().numpy()
        assert np.all(Fk >= prev - 1e-12 * prev)        # F never decreases
        prev = Fk
    out, F = fs.refine(ctx, seg, _dev(starts), nsteps=20)
    assert ctx.sync_status() == 0
    out, F = out.cpu().numpy(), F.cpu().numpy()
    for p in range(len(starts)):
        best, Fb = orf.fine_search(x32, wl.dt, starts[p], wl.fl, det, wl.S0)
        assert F[p] >= Fb * (1 - 1e-7), (p, F[p], Fb)
        assert np.all(np.abs(out[p] - best) < 0.05 * width), (p, (out[p] - best) / width)
        # the refined F is the F at the refined point
        Fr = orf.fstat_point(x32, wl.dt, out[p], wl.fl, det, wl.S0)
        assert abs(F[p] - Fr) <= 1e-9 * Fr


def test_points_from_candidates(fs):
    wl, det, x, th = _case()
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x, torch.float32), wl.dt, wl.nfft, wl.fl, wl.S0)
    alpha, delta = W.sky_grid(wl.nsky)
    f1 = W.spin_grid(wl.nspin, *wl.f1_range)
    res = fs.search(ctx, seg, _dev(alpha), _dev(delta), _dev(f1), wl.F_thr, write_F=False)
    n = min(int(res.n_cand.item()), res.cand.shape[0])
    assert n > 0
    pts = fs.points_from_candidates(ctx, seg, res.cand, n, _dev(alpha), _dev(delta), _dev(f1)).cpu().numpy()
    sky, spin, bins, Fc = res.candidates()
    assert np.array_equal(pts[:, 0], bins / (wl.nfft * wl.dt))
    assert np.array_equal(pts[:, 1], f1[spin])
    assert np.array_equal(pts[:, 2], alpha[sky]) and np.array_equal(pts[:, 3], delta[sky])
    # the fine search never lowers F below the exact F at the starting points
    F0, _, _ = fs.fstat_points(ctx, seg, _dev(pts), grad=False)
    _, F = fs.refine(ctx, seg, _dev(pts), nsteps=5)
    assert torch.all(F >= F0)


def test_amplitudes_match_oracle(fs):
    wl, det, x, th = _case()
    _, _, G0 = orf.fstat_point(x, wl.dt, th, wl.fl, det, wl.S0, grad=True)
    P = _points(th, 1.0 / np.sqrt(np.diag(G0)))[:3]
    ctx = fs.Context(det)
    xd = _dev(x, torch.float32)
    seg = fs.Segment(ctx, xd, wl.dt, wl.nfft, wl.fl, wl.S0)
    amp = fs.amplitudes(ctx, seg, _dev(P)).cpu().numpy()
    assert ctx.sync_status() == 0
    xo = xd.double().cpu().numpy()
    for p in range(len(P)):
        ref = orf.amplitude_estimates(xo, wl.dt, P[p], wl.fl, det)
        assert np.max(np.abs(amp[p] - ref)) <= 1e-9 * np.max(np.abs(ref)), (p, amp[p], ref)


def test_constrained_lattice_covers_an_injected_signal(fs):
    """The grid of Sec. IV (fs_lattice, fs_lattice_nodes) around a noise-free signal,
    every node evaluated with the exact F: the best node keeps about C0 of the
    signal's F.  The metric is the linear model's (Eq. philin), which fixes the
    ecliptic components n_x, n_y of the sky direction and drops the part of r_d
    perpendicular to the ecliptic (a diurnal phase omega0 (r_E/c) sin(eps) n_z, about
    23 n_z rad here); between neighbouring nodes n_z changes by
    -(n_x dn_x + n_y dn_y)/n_z, small near the ecliptic poles and large near the
    ecliptic, so the source is placed at ecliptic latitude ~70 degrees."""
    wl = W.WORKLOADS["small"]
    det = W.detector_for(wl)
    ce, se = math.cos(det.eps), math.sin(det.eps)
    n_ecl = np.array([0.2, 0.25, math.sqrt(1 - 0.2 ** 2 - 0.25 ** 2)])
    n_eq = np.array([n_ecl[0], ce * n_ecl[1] - se * n_ecl[2], se * n_ecl[1] + ce * n_ecl[2]])
    alpha = math.atan2(n_eq[1], n_eq[0]) % (2 * math.pi)
    delta = math.asin(n_eq[2])
    inj = W.Injection(f0=0.0213, f1=-4e-9, alpha=alpha, delta=delta, psi=0.3, cos_iota=0.4, phi0=1.1, snr=25.0)
    x = orsp.inject(wl.n, wl.dt, [inj], wl.fl, det, wl.sigma)
    th = np.array([inj.f0, inj.f1, inj.alpha, inj.delta])
    To = wl.n * wl.dt
    C0 = 0.75
    G = fs.linear_model_fisher(det, wl.n, wl.dt)
    B, theta = fs.lattice(G, C0, math.pi / To)
    assert 1.7655 < theta < 3.0
    # the box spans the correlation ellipsoid's projections (one day: a sky offset trades
    # against hundreds of frequency bins), then keeps the nodes within metric distance 1
    half = math.sqrt(1 - C0) * np.sqrt(np.diag(np.linalg.inv(G))) / (2 * math.pi)
    nodes = fs.lattice_nodes(B, det, wl.fl, (th[0] - 1.2 * half[0], th[0] + 1.2 * half[0]),
                             (th[1] - 1.5 * half[1], th[1] + 1.5 * half[1]), cap=1 << 26)
    tp = 2 * math.pi
    ce, se = math.cos(det.eps), math.sin(det.eps)

    def xi(p):
        om0 = tp * (wl.fl + p[:, 0])
        nx = np.cos(p[:, 2]) * np.cos(p[:, 3])
        ny = ce * np.sin(p[:, 2]) * np.cos(p[:, 3]) + se * np.sin(p[:, 3])
        return np.stack([om0, tp * p[:, 1], om0 * ny, om0 * nx], axis=1)

    d = xi(nodes) - xi(th[None, :])
    near = nodes[np.einsum("ij,jk,ik->i", d, G, d) <= 1.0]
    assert 10 < len(near) < 100000
    nodes = near
    ctx = fs.Context(det)
    seg = fs.Segment(ctx, _dev(x), wl.dt, wl.nfft, wl.fl, wl.S0, precision="f64")
    F0, _, _ = fs.fstat_points(ctx, seg, _dev(th[None, :]), grad=False)
    Fn, _, _ = fs.fstat_points(ctx, seg, _dev(nodes), grad=False)
    assert ctx.sync_status() == 0
    ratio = float(Fn.max() / F0[0])
    assert ratio >= C0 - 0.05, ratio
