"""Grid in the parameter space (Sec. IV; oracle, FP64): the reduced Fisher matrix of
the linear phase model, the thinnest lattice coverings A2* and A4*, covering
radius and deep holes from the Voronoi cell, and the constrained lattice of
Eqs. opt and opt2.

Test infrastructure only (see the package docstring).

Linear model (Eq. philin, one spindown): xi = (omega0, omega1, alpha1, alpha2),
m(t) = (t, t^2/2, mu1(t), mu2(t)) with mu1 = (R_ES^y + R_E^y cos eps)/c and
mu2 = (R_ES^x + R_E^x)/c (ecliptic SSB frame for R_ES, equatorial for R_E), so
that alpha1 = omega0 n0_y and alpha2 = omega0 n0_x (Eq. albe).  The reduced
Fisher matrix is G_kl = <m_k m_l> - <m_k><m_l> (Eq. redFm-def).

Construction (Sec. IV.B): with G = U0 D0^2 U0^T and M = U0 D0^-1 the correlation
ellipsoid tau^T G tau = 1 - C0 becomes the sphere of radius R = sqrt(1 - C0) in
x = M^-1 tau (any M with M^T G M = I does; it is computed from the unit-diagonal
scaling of G for accuracy).  Start from the generator M0 of A_n* (rows are basis vectors,
covering radius R); pick a lattice vector l with |l| >= |e0|, e0 = M^-1 a0,
a0 = (dp0, 0, ...); shrink along l by mu = |e0|/|l|; expand perpendicular to l
by nu so that the covering radius returns to R (Eq. condition: the minimal match
is exactly C0; solved directly by bisection -- the printed iteration
nu_i = R / (R_i sin phi_i) does not keep that condition); keep
the l with the largest det S = mu nu^(n-1); rotate l onto e0 (O2) and, for the
second constraint, rotate about e0 (O3) so that a second lattice vector f has
no sky components; map back with M^T.  All in row-vector form: a lattice vector
r of A_n* becomes r O1 S O2^T O3^T M^T.

Search of the lattice with the FFT (Sec. IV, Sec. VII): with a0 the Fourier
spacing dp0 = 2 pi / (Nfft dt) and a1 free of sky components, the nodes
k0 a0 + k1 a1 + k2 b2 + k3 b3 group into lines along a0 that one zero-padded
transform evaluates at once: per sky node (k2, k3) and spindown node k1, the line
omega0 = c0 + k0 dp0 with c0 = k1 a1_0 + k2 b2_0 + k3 b3_0 falls on the bins k of
the transform shifted by the fraction d = frac(c0/dp0 - fl Nfft dt) of a bin.  The
sky position of (alpha1, alpha2) = omega0 (n0_y, n0_x) (Eq. albe) is taken at one
reference frequency for the whole line (reading: the band's upper edge,
fl + 1/(2 dt)), both ecliptic hemispheres.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import earth


def linear_model_fisher(n: int, dt: float, det) -> np.ndarray:
    """Reduced Fisher matrix of xi = (omega0, omega1, alpha1, alpha2) over t_k = k dt."""
    t = np.arange(n, dtype=np.float64) * dt
    res = earth.earth_orbit_ls(t, det)                 # R_ES / c, ecliptic frame (3, n)
    rE = earth.site_equatorial_ls(t, det)              # R_E / c, equatorial frame (3, n)
    mu1 = res[1] + rE[1] * math.cos(det.eps)
    mu2 = res[0] + rE[0]
    m = np.stack([t, 0.5 * t * t, mu1, mu2])
    mm = m.mean(axis=1)
    return (m @ m.T) / n - np.outer(mm, mm)


def a_star_generator(dim: int, R: float) -> np.ndarray:
    """Generator matrix (rows = basis vectors) of A2* (Eq. A2gen) or A4* (Eq. gen)
    with covering radius R."""
    if dim == 2:
        return R * math.sqrt(3.0) * np.array([[1.0, 0.0], [0.5, math.sqrt(3.0) / 2.0]])
    if dim == 4:
        s2, s3, s5, s6 = math.sqrt(2.0), math.sqrt(3.0), math.sqrt(5.0), math.sqrt(6.0)
        M = np.array([
            [s2, 0.0, 0.0, 0.0],
            [1 / s2, math.sqrt(2.0 / 3.0) + 1 / s6, 0.0, 0.0],
            [1 / s2, 1 / s6, 1 / (2 * s3) + s3 / 2, 0.0],
            [-1 / (5 * s2) - 2 * s2 / 5, 1 / (5 * s6) - s6 / 5, -1 / (5 * s3) - s3 / 10, -1 / (2 * s5)],
        ])
        return R * math.sqrt(5.0 / 2.0) * M
    raise ValueError("dimension 2 or 4")


def _short_vectors(gen: np.ndarray, kmax: int = 2):
    """Nonzero lattice vectors sum k_i a_i with |k_i| <= kmax (enough after reduction)."""
    dim = gen.shape[0]
    out = []
    for k in itertools.product(range(-kmax, kmax + 1), repeat=dim):
        if any(k):
            out.append(np.asarray(k, dtype=np.float64) @ gen)
    return np.array(out)


def _lll(gen: np.ndarray) -> np.ndarray:
    """LLL-reduced basis of the same lattice (delta = 3/4), rows."""
    B = np.array(gen, dtype=np.float64)
    n = B.shape[0]

    def gs(B):
        Bs = np.zeros_like(B)
        mu = np.zeros((n, n))
        for i in range(n):
            v = B[i].copy()
            for j in range(i):
                mu[i, j] = B[i] @ Bs[j] / (Bs[j] @ Bs[j])
                v -= mu[i, j] * Bs[j]
            Bs[i] = v
        return Bs, mu

    Bs, mu = gs(B)
    k = 1
    while k < n:
        for j in range(k - 1, -1, -1):
            q = round(mu[k, j])
            if q:
                B[k] -= q * B[j]
                Bs, mu = gs(B)
        if Bs[k] @ Bs[k] >= (0.75 - mu[k, k - 1] ** 2) * (Bs[k - 1] @ Bs[k - 1]):
            k += 1
        else:
            B[[k, k - 1]] = B[[k - 1, k]]
            Bs, mu = gs(B)
            k = max(k - 1, 1)
    return B


def voronoi_vertices(gen: np.ndarray):
    """Vertices of the Voronoi cell of the origin: points x with x.v <= |v|^2/2 for
    every lattice vector v, equality for dim of them (brute force over the short
    vectors of an LLL-reduced basis)."""
    B = _lll(gen)
    dim = B.shape[0]
    V = _short_vectors(B, 2)
    h = 0.5 * np.einsum("ij,ij->i", V, V)
    # Voronoi-relevant vectors: the midpoint v/2 lies on the cell boundary
    keep = []
    for i, v in enumerate(V):
        others = np.delete(np.arange(len(V)), i)
        if np.all(V[others] @ (v / 2) <= h[others] + 1e-12 * (v @ v)):
            keep.append(i)
    rel = V[keep]
    idx = np.array(list(itertools.combinations(range(len(rel)), dim)))
    A = rel[idx]                                          # (ncomb, dim, dim)
    d = np.linalg.det(A)
    ok = np.abs(d) > 1e-10 * np.prod(np.linalg.norm(A, axis=2), axis=1)
    A = A[ok]
    rhs = 0.5 * np.einsum("cij,cij->ci", A, A)
    X = np.linalg.solve(A, rhs[..., None])[..., 0]       # (ncomb, dim)
    inside = np.all(X @ V.T <= h[None, :] + 1e-9 * (1.0 + np.einsum("ij,ij->i", X, X))[:, None], axis=1)
    X = X[inside]
    # unique up to rounding
    if len(X) == 0:
        return X
    scale = 1e-9 * (1.0 + np.abs(X).max())
    _, first = np.unique(np.round(X / scale), axis=0, return_index=True)
    return X[np.sort(first)]


def covering_radius(gen: np.ndarray):
    """Covering radius and the deep holes (Voronoi vertices at that distance)."""
    vv = voronoi_vertices(gen)
    r = np.linalg.norm(vv, axis=1)
    R = r.max()
    return R, vv[r >= R * (1 - 1e-9)]


def thickness(gen: np.ndarray, R: float) -> float:
    """Covering thickness: volume of the covering sphere over the fundamental cell."""
    dim = gen.shape[0]
    vsph = math.pi ** (dim / 2) / math.gamma(dim / 2 + 1) * R ** dim
    return vsph / abs(np.linalg.det(gen))


def _int_coeffs(gen: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Integer coordinates of the lattice vector v in the basis gen (rows)."""
    c = np.linalg.solve(gen.T, v)
    k = np.rint(c)
    assert np.allclose(c, k, atol=1e-6), c
    return k.astype(np.int64)


def _unimodular_with_rows(rows) -> np.ndarray:
    """An integer matrix of determinant +-1 whose first rows are the given integer
    vectors (a primitive set), up to adding multiples of earlier rows to later ones:
    column operations (extended Euclid) bring row i to the unit vector e_i, and the
    inverse of the accumulated operations is returned."""
    dim = len(rows[0])
    V = np.eye(dim, dtype=np.int64)
    for i, r in enumerate(rows):
        r = np.asarray(r, dtype=np.int64) @ V
        for j in range(dim - 1, i, -1):          # zero r[j] against r[i] by column Euclid
            while r[j] != 0:
                q = r[i] // r[j]
                V[:, i] -= q * V[:, j]
                r[i] -= q * r[j]
                V[:, [i, j]] = V[:, [j, i]]
                r[[i, j]] = r[[j, i]]
        if abs(r[i]) != 1:
            raise ValueError("rows are not part of a basis")
        if r[i] < 0:
            V[:, i] = -V[:, i]
    U = np.rint(np.linalg.inv(V)).astype(np.int64)
    return U


def _frame(u: np.ndarray) -> np.ndarray:
    """Orthogonal matrix whose first column is the unit vector u."""
    dim = u.size
    A = np.eye(dim)
    A[:, 0] = u
    Q, _ = np.linalg.qr(A)
    if Q[:, 0] @ u < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def expand_to_radius(gen: np.ndarray, l: np.ndarray, R: float, rtol: float = 1e-12):
    """The factor nu >= 1 of the expansion perpendicular to l after which the
    covering radius is R again (the condition that defines nu in Sec. IV.B;
    the covering radius grows continuously with nu: bracketed, then solved by
    regula falsi with the Illinois modification).  Returns the expanded
    generator and nu."""
    O1 = _frame(l / np.linalg.norm(l))
    dim = gen.shape[0]

    def expand(nu):
        return gen @ O1 @ np.diag([1.0] + [nu] * (dim - 1)) @ O1.T

    def g(nu):
        return covering_radius(expand(nu))[0] - R

    lo, hi = 1.0, 2.0
    glo, ghi = g(lo), g(hi)
    while ghi < 0:
        lo, glo = hi, ghi
        hi *= 2.0
        ghi = g(hi)
    side = 0
    for _ in range(200):
        mid = (lo * ghi - hi * glo) / (ghi - glo)
        gm = g(mid)
        if gm > 0:
            hi, ghi = mid, gm
            if side == -1:
                glo *= 0.5
            side = -1
        else:
            lo, glo = mid, gm
            if side == 1:
                ghi *= 0.5
            side = 1
        if hi - lo <= rtol * hi or abs(gm) <= 1e-15 * R:
            break
    nu = mid
    return expand(nu), nu


def constrained_lattice(G: np.ndarray, C0: float, dp0: float, n_candidates: int = 4, second: bool = True):
    """Generator (rows, in parameter units) of the thinnest lattice covering found by
    the construction of Sec. IV.B with a0 = (dp0, 0, ...) a lattice vector and, if
    second (4 dimensions), a second lattice vector with no sky components
    (Eq. constraint2).  Returns (generator, thickness, details)."""
    G = np.asarray(G, dtype=np.float64)
    dim = G.shape[0]
    R = math.sqrt(1.0 - C0)
    # tau = Mx x with Mx^T G Mx = I; G's entries span many decades (s^2 to s^4), so the
    # eigendecomposition is taken of the unit-diagonal matrix D^-1 G D^-1, D = diag(G)^1/2
    dg = np.sqrt(np.diag(G))
    w, U0 = np.linalg.eigh(G / np.outer(dg, dg))
    Mx = np.diag(1.0 / dg) @ U0 @ np.diag(1.0 / np.sqrt(w))
    a0 = np.zeros(dim)
    a0[0] = dp0
    e0 = np.linalg.solve(Mx, a0)
    M0 = a_star_generator(dim, R)
    theta_min = thickness(M0, R)
    # lattice vectors of A* by increasing length, |l| >= |e0|, one of each +-pair
    vecs = _short_vectors(M0, 3)
    vecs = vecs[np.argsort(np.linalg.norm(vecs, axis=1))]
    # one candidate per length shell: A_n* is symmetric enough that vectors of one
    # length give congruent results (the final rotation takes l onto e0 anyway)
    cands = []
    for v in vecs:
        if np.linalg.norm(v) >= np.linalg.norm(e0) * (1 - 1e-12) and \
                not any(abs(np.linalg.norm(v) - np.linalg.norm(c)) <= 1e-9 * np.linalg.norm(v) for c in cands):
            cands.append(v)
        if len(cands) >= n_candidates:
            break
    best = None
    for l in cands:
        mu = np.linalg.norm(e0) / np.linalg.norm(l)
        O1 = _frame(l / np.linalg.norm(l))
        M1 = M0 @ O1 @ np.diag([mu] + [1.0] * (dim - 1)) @ O1.T
        _, nu = expand_to_radius(M1, l, R)
        detS = mu * nu ** (dim - 1)
        if best is None or detS > best[0] * (1 + 1e-12):
            best = (detS, l, mu, nu, O1)
    detS, l, mu, nu, O1 = best
    S = np.diag([mu] + [nu] * (dim - 1))
    O2 = _frame(e0 / np.linalg.norm(e0))
    # row map r -> r O1 S O2^T (then O3^T, then Mx^T)
    X = M0 @ O1 @ S @ O2.T
    O3 = np.eye(dim)
    f = None
    if second and dim == 4:
        # second lattice vector: the shortest one not parallel to l
        for v in vecs:
            if abs(abs(v @ l) - np.linalg.norm(v) * np.linalg.norm(l)) > 1e-9 * (v @ v):
                try:
                    _unimodular_with_rows([_int_coeffs(M0, l), _int_coeffs(M0, v)])
                except ValueError:
                    continue
                f = v
                break
        yf = f @ O1 @ S @ O2.T                        # its image in x (row)
        e0h = e0 / np.linalg.norm(e0)
        # x-space directions with no sky components: kernel of the sky rows of Mx
        K = np.linalg.svd(Mx[2:4, :])[2][2:].T           # 4 x 2 basis of {x: (Mx x)_sky = 0}
        # the unit vector of that kernel orthogonal to e0
        k1 = K[:, 0] - (K[:, 0] @ e0h) * e0h
        if np.linalg.norm(k1) < 1e-8:
            k1 = K[:, 1] - (K[:, 1] @ e0h) * e0h
        wv = k1 / np.linalg.norm(k1)
        yperp = yf - (yf @ e0h) * e0h
        u = yperp / np.linalg.norm(yperp)
        # rotation in the plane (u, wv) taking u to wv (identity on the rest; fixes e0)
        c = float(np.clip(u @ wv, -1.0, 1.0))
        v2 = wv - c * u
        if np.linalg.norm(v2) > 1e-14:
            v2 /= np.linalg.norm(v2)
            s = math.sqrt(max(0.0, 1.0 - c * c))
            P = np.outer(u, u) + np.outer(v2, v2)
            O3 = np.eye(4) - P + c * P + s * (np.outer(v2, u) - np.outer(u, v2))
        X = X @ O3.T
    gen_all = X @ Mx.T                                   # images of the rows of M0
    # a basis of the same lattice whose first vector is the image of l (= a0) and,
    # with the second constraint, whose second is f's image minus a multiple of a0
    rows = [_int_coeffs(M0, l)] + ([_int_coeffs(M0, f)] if f is not None else [])
    U = _unimodular_with_rows(rows)
    gen = U @ gen_all
    details = dict(l=l, mu=mu, nu=nu, e0=e0, Mx=Mx, theta_min=theta_min, f=f, R=R, O1=O1, O2=O2, O3=O3, S=S,
                   U=U, gen_images=gen_all)
    return gen, theta_min / detS, details


def lattice_templates(basis, det, fl: float, nfft: int, dt: float, f1_min: float, f1_max: float,
                      box=(-1.0, 1.0, -1.0, 1.0)):
    """Templates of the FFT search of a 4-dimensional lattice with both constraints
    (basis rows a0 = (dp0, 0, 0, 0), a1 = (a1_0, a1_1, 0, 0), b2, b3 in
    (omega0, omega1, alpha1, alpha2) units, dp0 = 2 pi / (Nfft dt)): a list, one
    entry per sky node and hemisphere, of (alpha, delta, [(f1, d, k1), ...]) with the
    spindown nodes in [f1_min, f1_max] Hz/s (k1 increasing) and the bin offsets d in
    [0, 1).  box = (nx_lo, nx_hi, ny_lo, ny_hi) limits the ecliptic components of the
    sky nodes (the whole sky by default).  Sky nodes run over k2, then k3 (both
    increasing), north before south."""
    B = np.array(basis, dtype=np.float64).reshape(4, 4)
    tp = 2.0 * math.pi
    dp0 = B[0, 0]
    scale = np.abs(B).max(axis=0)
    if abs(dp0 - tp / (nfft * dt)) > 1e-9 * dp0 or np.any(np.abs(B[0, 1:]) > 1e-9 * scale[1:]) or \
            np.any(np.abs(B[1, 2:]) > 1e-9 * scale[2:]):
        raise ValueError("basis is not a constrained lattice on this transform's Fourier spacing")
    B[0, 1:] = 0.0          # exact zeros of the constraints (rounding of the construction)
    B[1, 2:] = 0.0
    w_ref = tp * (fl + 0.5 / dt)
    w1lo, w1hi = tp * f1_min, tp * f1_max
    S = B[2:4, 2:4]
    Sinv = np.linalg.inv(S)
    k2r = int(math.ceil(w_ref * np.linalg.norm(Sinv[:, 0]))) + 1
    k3r = int(math.ceil(w_ref * np.linalg.norm(Sinv[:, 1]))) + 1
    ce, se = math.cos(det.eps), math.sin(det.eps)
    out = []
    for k2 in range(-k2r, k2r + 1):
        for k3 in range(-k3r, k3r + 1):
            a1 = k2 * B[2, 2] + k3 * B[3, 2]
            a2 = k2 * B[2, 3] + k3 * B[3, 3]
            ny, nx = a1 / w_ref, a2 / w_ref        # ecliptic n0_y, n0_x (Eq. albe)
            r2 = nx * nx + ny * ny
            if r2 > 1.0 or not (box[0] <= nx <= box[1] and box[2] <= ny <= box[3]):
                continue
            c1 = k2 * B[2, 1] + k3 * B[3, 1]
            lo, hi = sorted(((w1lo - c1) / B[1, 1], (w1hi - c1) / B[1, 1]))
            rows = []
            for k1 in range(int(math.ceil(lo)), int(math.floor(hi)) + 1):
                om1 = k1 * B[1, 1] + c1
                if om1 < w1lo or om1 > w1hi:
                    continue
                c0 = k1 * B[1, 0] + k2 * B[2, 0] + k3 * B[3, 0]
                x = c0 / dp0 - fl * nfft * dt
                rows.append((om1 / tp, x - math.floor(x), k1))
            if not rows:
                continue
            nz_abs = math.sqrt(max(0.0, 1.0 - r2))
            for nz in ((nz_abs, -nz_abs) if nz_abs > 0.0 else (0.0,)):
                ex, ey, ez = nx, ce * ny - se * nz, se * ny + ce * nz   # n_eq = Rot(eps)^T n0
                alpha = math.atan2(ey, ex) % tp
                delta = math.asin(max(-1.0, min(1.0, ez)))
                out.append((alpha, delta, rows))
    return out
