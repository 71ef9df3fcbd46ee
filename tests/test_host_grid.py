"""Grid construction in the library (host functions, no device work) against the
grid oracle: the linear-model Fisher matrix, the constrained lattice, and the
enumeration of its nodes in a band."""
import math

import numpy as np
import pytest

from oracle import grid as og
from paper_1003_0844_gb300 import workloads as W


@pytest.fixture(scope="module")
def fs():
    from paper_1003_0844_gb300 import build, fstat
    build.build()
    fstat.load_library()
    return fstat


def _case():
    wl = W.WORKLOADS["grid_2d"]
    return wl, W.detector_for(wl)


def test_linear_model_fisher_matches_oracle(fs):
    wl, det = _case()
    for t0 in (0.0, 3.1e6):
        G = fs.linear_model_fisher(det, wl.n, wl.dt, t0)
        from oracle import earth
        Go = og.linear_model_fisher(wl.n, wl.dt, earth.detector_at_epoch(det, t0))
        scale = np.sqrt(np.outer(np.diag(Go), np.diag(Go)))
        assert np.max(np.abs(G - Go) / scale) < 1e-9


def test_two_dimensional_lattice_matches_oracle(fs):
    G = np.array([[1 / 12, 1 / 12], [1 / 12, 4 / 45]])
    B, th = fs.lattice(G, 0.75, math.pi, constraint2=False)
    Bo, tho, _ = og.constrained_lattice(G, 0.75, math.pi)
    assert th == pytest.approx(tho, rel=1e-9)
    assert np.allclose(B[0], [math.pi, 0.0], atol=0)
    U = B @ np.linalg.inv(Bo)                       # same lattice: a unimodular change of basis
    assert np.allclose(U, np.rint(U), atol=1e-8) and abs(abs(np.linalg.det(np.rint(U))) - 1) < 1e-9


def test_four_dimensional_lattice_meets_the_constraints(fs):
    wl, det = _case()
    G = fs.linear_model_fisher(det, wl.n, wl.dt)
    dp0 = math.pi / (wl.n * wl.dt)
    B, th = fs.lattice(G, 0.75, dp0)
    Bo, tho, d = og.constrained_lattice(G, 0.75, dp0)
    assert th == pytest.approx(tho, rel=1e-5)
    assert abs(np.linalg.det(B)) == pytest.approx(abs(np.linalg.det(Bo)), rel=1e-5)
    assert np.array_equal(B[0], [dp0, 0.0, 0.0, 0.0])
    assert B[1, 2] == 0.0 and B[1, 3] == 0.0
    assert np.allclose(d["Mx"].T @ G @ d["Mx"], np.eye(4), atol=1e-8)
    x = B @ np.linalg.inv(d["Mx"].T)
    assert og.covering_radius(x)[0] == pytest.approx(d["R"], rel=1e-6)


def test_nodes_are_the_lattice_points_of_the_band(fs):
    """Every node is a lattice point of the box (integer coordinates), each appears once
    per hemisphere, and random lattice points of the box are all among them."""
    wl, det = _case()
    G = fs.linear_model_fisher(det, wl.n, wl.dt)
    To = wl.n * wl.dt
    B, _ = fs.lattice(G, 0.75, math.pi / To)
    f0r, f1r = (0.1, 0.1 + 2 / To), (-2.0e-9, -1.8e-9)
    pts = fs.lattice_nodes(B, det, wl.fl, f0r, f1r)
    assert len(pts) > 100
    tp = 2 * math.pi
    ce, se = math.cos(det.eps), math.sin(det.eps)
    om0 = tp * (wl.fl + pts[:, 0])
    nx = np.cos(pts[:, 2]) * np.cos(pts[:, 3])                      # ecliptic components of n0
    ny = ce * np.sin(pts[:, 2]) * np.cos(pts[:, 3]) + se * np.sin(pts[:, 3])
    nz = -se * np.sin(pts[:, 2]) * np.cos(pts[:, 3]) + ce * np.sin(pts[:, 3])
    xi = np.stack([om0, tp * pts[:, 1], om0 * ny, om0 * nx], axis=1)
    k = xi @ np.linalg.inv(B)
    assert np.max(np.abs(k - np.rint(k))) < 1e-4
    keys = set(zip(*np.rint(k).astype(np.int64).T, nz > 0))
    assert len(keys) == len(pts)
    # random lattice points near the box: those inside must be present
    rng = np.random.default_rng(11)
    kk = np.rint(k).astype(np.int64)
    found = 0
    for _ in range(20000):
        base = kk[rng.integers(len(kk))]
        cand = base + rng.integers(-2, 3, size=4)
        x = cand @ B
        if not (tp * (wl.fl + f0r[0]) <= x[0] <= tp * (wl.fl + f0r[1]) and tp * f1r[0] <= x[1] <= tp * f1r[1]):
            continue
        if x[2] ** 2 + x[3] ** 2 >= x[0] ** 2:
            continue
        found += 1
        assert (int(cand[0]), int(cand[1]), int(cand[2]), int(cand[3]), True) in keys
        assert (int(cand[0]), int(cand[1]), int(cand[2]), int(cand[3]), False) in keys
    assert found > 100
