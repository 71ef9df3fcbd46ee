"""Pins of the grid oracle (Sec. IV): the printed A2* and A4* generators, covering
radius from the Voronoi cell against brute force, the two-dimensional example,
the linear-model Fisher matrix, and the constrained four-dimensional lattice."""
import math

import numpy as np
import pytest

from oracle import grid as og
from paper_1003_0844_gb300 import workloads as W
from tests.helpers import golden


def _brute_covering_radius(gen, n=60000, seed=3):
    """Largest distance of random points of the fundamental cell to the lattice."""
    dim = gen.shape[0]
    B = og._lll(gen)
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0, 1, size=(n, dim)) @ B
    ks = np.array(np.meshgrid(*[np.arange(-2, 3)] * dim)).reshape(dim, -1).T
    L = ks @ B
    best = np.full(n, np.inf)
    for i in range(0, len(L), 64):
        d = np.linalg.norm(pts[:, None, :] - L[None, i:i + 64, :], axis=2).min(axis=1)
        best = np.minimum(best, d)
    return best.max()


@pytest.mark.parametrize("dim,key", [(2, "theta_A2star"), (4, "theta_A4star")])
def test_printed_a_star_generators(dim, key):
    """Eqs. A2gen and gen: covering radius R and the printed thicknesses
    (tests/golden/sec4_lattice_thickness.txt), hexagonal = 2 pi / (3 sqrt 3)."""
    theta = golden("sec4_lattice_thickness.txt")[key]
    R = 0.5
    M0 = og.a_star_generator(dim, R)
    Rv, holes = og.covering_radius(M0)
    assert abs(Rv - R) < 1e-12
    assert og.thickness(M0, Rv) == pytest.approx(theta, abs=1e-4)
    if dim == 2:
        assert theta == pytest.approx(2 * math.pi / (3 * math.sqrt(3)), abs=1e-4)
    rb = _brute_covering_radius(M0)
    assert 0.97 * R < rb <= R * (1 + 1e-9)


def test_two_dimensional_example():
    """Sec. IV.C: G of Eq. gamma2d, a0 = (pi, 0), C0 = 3/4.  The printed |M^-1 a0|, the
    length of l and mu are reproduced; nu is fixed by the covering radius staying R
    (Eq. condition), which for this l gives the thinnest lattice with a0 as a basis
    vector: the isosceles Delaunay triangle on a0 with circumradius R."""
    g = golden("sec4c_example_2d.txt")
    G = np.array([[g["G_11"], g["G_12"]], [g["G_12"], g["G_22"]]])
    gen, th, d = og.constrained_lattice(G, g["C0"], g["a0_1"])
    R, L = 0.5, g["norm_Minv_a0"]
    assert np.linalg.norm(d["e0"]) == pytest.approx(L, rel=1e-12)
    assert np.linalg.norm(d["l"]) == pytest.approx(math.hypot(g["l_1"], g["l_2"]), rel=1e-12)
    assert d["mu"] == pytest.approx(g["mu"], rel=1e-12)
    assert th == pytest.approx(math.pi * R * R / (L * (R + math.sqrt(R * R - L * L / 4))), rel=1e-9)
    assert np.allclose(gen[0], [math.pi, 0.0], atol=1e-12)
    x = gen @ np.linalg.inv(d["Mx"].T)                  # the lattice in x = M^-1 tau
    assert og.covering_radius(x)[0] == pytest.approx(R, rel=1e-9)
    assert 0.97 * R < _brute_covering_radius(x) <= R * (1 + 1e-9)


def test_printed_nu_of_the_example_is_not_a_tight_covering():
    """The example's printed nu = sqrt(108 - pi^2)/9 (thickness 18/sqrt(108 - pi^2) ~ 1.8171
    assuming radius R) leaves the covering radius at ~0.908 R for the same l and mu,
    so it does not meet Eq. condition: the reading used solves that condition."""
    g = golden("sec4c_example_2d.txt")
    R = 0.5
    M0 = og.a_star_generator(2, R)
    l = np.array([g["l_1"], g["l_2"]])
    O1 = og._frame(l / np.linalg.norm(l))
    mu, nu = g["mu"], g["nu_printed"]
    M = M0 @ O1 @ np.diag([mu, 1.0]) @ O1.T @ O1 @ np.diag([1.0, nu]) @ O1.T
    r = og.covering_radius(M)[0]
    assert r / R == pytest.approx(0.908, abs=1e-3)
    assert og.thickness(M0, R) / (mu * nu) == pytest.approx(g["theta_printed"], abs=1e-4)


def test_linear_model_fisher_closed_forms():
    wl = W.WORKLOADS["grid_2d"]
    G = og.linear_model_fisher(wl.n, wl.dt, W.detector_for(wl))
    n, dt = wl.n, wl.dt
    T = n * dt
    assert G[0, 0] == pytest.approx((n * n - 1) * dt * dt / 12.0, rel=1e-12)
    assert G[0, 1] == pytest.approx(T ** 3 / 24.0, rel=2e-4)
    assert G[1, 1] == pytest.approx(T ** 4 / 45.0, rel=2e-4)
    assert np.allclose(G, G.T) and np.all(np.linalg.eigvalsh(G) > 0)


def test_constrained_four_dimensional_lattice():
    """2-day segment, C0 = 3/4, frequency resolution of a transform padded by two:
    a0 = (dp0, 0, 0, 0) is the first basis vector, the second has no sky components
    (Eq. constraint2), the covering radius is R, and the thickness is a little above
    A4*'s 1.7655 (the paper quotes ~2.1 for its 2-day case)."""
    wl = W.WORKLOADS["grid_2d"]
    G = og.linear_model_fisher(wl.n, wl.dt, W.detector_for(wl))
    To = wl.n * wl.dt
    dp0 = math.pi / To
    gen, th, d = og.constrained_lattice(G, 0.75, dp0)
    assert np.allclose(gen[0], [dp0, 0, 0, 0], rtol=0, atol=1e-12 * np.abs(gen).max())
    sky_scale = np.abs(gen[:, 2:]).max()
    assert np.all(np.abs(gen[1, 2:]) <= 1e-12 * sky_scale)
    assert abs(abs(np.linalg.det(gen)) - abs(np.linalg.det(d["gen_images"]))) <= 1e-9 * abs(np.linalg.det(gen))
    assert np.allclose(d["Mx"].T @ G @ d["Mx"], np.eye(4), atol=1e-8)
    x = gen @ np.linalg.inv(d["Mx"].T)
    assert og.covering_radius(x)[0] == pytest.approx(d["R"], rel=1e-9)
    assert _brute_covering_radius(x, n=20000) <= d["R"] * (1 + 1e-9)
    assert 1.7655 < th < 2.2
