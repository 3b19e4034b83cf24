"""Pins of the oracle's element quadrature (Sec. 3.4.1, 3.5.2), CPU only.

Facts fixed independently of the oracle's own loops:
  * one flat triangle, target off the triangle: the 4x4 collapsed Gauss rule
    must reproduce the element integral of the linearly interpolated density
    against G^l (single) or T^l n(z) (double), computed here by a converged
    high-order Gauss rule over a Cartesian sweep of the triangle's plane (a
    different parametrisation), to the 4x4 rule's error on a smooth integrand;
  * one flat triangle, target at a vertex: the polar 4x4 rule of the parent
    triangle (and n-tilde in the double layer) against a converged high-order
    rule in physical polar coordinates about the vertex (whose Jacobian rho
    removes the 1/r singularity);
  * a sphere carrying q = n: the flow is exactly zero (an isotropic pressure
    inside), so the single layer vanishes and the adjoint double layer is
    lambda n with lambda = 4 pi (1 - 2 V / V_box): by Gauss's law the interior
    pressure of the single layer is -8 pi mu, the on-surface value is the mean
    of the inside and outside stresses, and the zero-mean pressure gauge of
    the k = 0 mode shifts it by 8 pi mu V / V_box.  Both errors must shrink
    with the mesh, as the discretisation error of linear flat elements does
    (O(N_tri^-1), Sec. 5.2).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W

ALPHA, RCUT = 2.0, 2.0


def _frame(x0, x1, x2):
    """In-plane Cartesian frame: origin x0, u along x1 - x0."""
    e1 = x1 - x0
    L = np.linalg.norm(e1)
    e1 = e1 / L
    nt = np.cross(x1 - x0, x2 - x0)
    nt /= np.linalg.norm(nt)
    e2 = np.cross(nt, e1)
    a, b = (x2 - x0) @ e1, (x2 - x0) @ e2
    return e1, e2, nt, L, a, b


def _bary(u, v, L, a, b):
    """Barycentric coordinates of (u, v) in the triangle (0,0), (L,0), (a,b)."""
    p2 = v / b
    p1 = (u - a * p2) / L
    return 1.0 - p1 - p2, p1, p2


def _integrand(x0, x1, x2, z, qv, layer, nz, tilde, u, v):
    """Density times kernel at in-plane points (u, v), one row per point;
    tilde = index of the target vertex for n-tilde (None: the constant nz)."""
    e1, e2, nt, L, a, b = _frame(x0, x1, x2)
    p0, p1, p2 = _bary(u, v, L, a, b)
    y = x0 + u[:, None] * e1 + v[:, None] * e2
    q = p0[:, None] * qv[0] + p1[:, None] * qv[1] + p2[:, None] * qv[2]
    G, _, T = O.kernels(ALPHA, z - y)
    if layer == 0:
        return np.einsum("nji,ni->nj", G, q)
    if tilde is None:
        n = np.broadcast_to(nz, q.shape)
    else:
        pt = (p0, p1, p2)[tilde]
        n = pt[:, None] * nt + (1.0 - pt)[:, None] * nz
    return np.einsum("njik,ni,nk->nj", T, q, n)


def _gl(n):
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def _sweep(x0, x1, x2, z, qv, layer, nz, n):
    """Cartesian sweep: v in [0, b], u between the edges (0,0)-(a,b) and
    (L,0)-(a,b); n x n Gauss-Legendre (smooth integrand: converges fast)."""
    _, _, _, L, a, b = _frame(x0, x1, x2)
    t, w = _gl(n)
    V = b * t
    lo, hi = a * V / b, L + (a - L) * V / b
    U = lo[:, None] + (hi - lo)[:, None] * t[None]
    W_ = (b * w)[:, None] * (hi - lo)[:, None] * w[None]
    Vv = np.broadcast_to(V[:, None], U.shape)
    f = _integrand(x0, x1, x2, z, qv, layer, nz, None, U.ravel(), Vv.ravel())
    return (f * W_.ravel()[:, None]).sum(0)


def _polar(x0, x1, x2, vertex, qv, layer, nz, n):
    """Physical polar coordinates about the target vertex in the triangle's
    plane: theta over the vertex angle, rho from 0 to the opposite edge; the
    Jacobian rho removes the 1/r singularity, n x n Gauss-Legendre."""
    xs = [x0, x1, x2]
    e1, e2, nt, L, a, b = _frame(x0, x1, x2)
    P = [np.array([0.0, 0.0]), np.array([L, 0.0]), np.array([a, b])]
    c = P[vertex]
    pa, pb = P[(vertex + 1) % 3] - c, P[(vertex + 2) % 3] - c
    th0, th1 = np.arctan2(pa[1], pa[0]), np.arctan2(pb[1], pb[0])
    if th1 < th0:
        th1 += 2.0 * np.pi
    t, w = _gl(n)
    TH = th0 + (th1 - th0) * t
    d = np.stack([np.cos(TH), np.sin(TH)], 1)
    # distance along d to the opposite edge pa + s (pb - pa)
    e = pb - pa
    R = (pa[0] * e[1] - pa[1] * e[0]) / (d[:, 0] * e[1] - d[:, 1] * e[0])
    RHO = R[:, None] * t[None]
    U = c[0] + RHO * d[:, 0:1]
    V = c[1] + RHO * d[:, 1:2]
    W_ = ((th1 - th0) * w)[:, None] * (R[:, None] * w[None]) * RHO
    f = _integrand(x0, x1, x2, xs[vertex], qv, layer, nz, vertex, U.ravel(), V.ravel())
    return (f * W_.ravel()[:, None]).sum(0)


def _triangle():
    rng = np.random.default_rng(11)
    x0 = np.array([4.0, 0.1, 4.0])
    x1 = x0 + np.array([0.19, 0.05, 0.02])
    x2 = x0 + np.array([0.03, 0.16, 0.14])
    q = rng.standard_normal((3, 3))
    return x0, x1, x2, q


@pytest.mark.parametrize("layer", [0, 1])
def test_regular_rule_matches_adaptive_integral(layer):
    x0, x1, x2, q = _triangle()
    z = x0 + np.array([0.33, -0.21, 0.27])
    nz = np.array([0.3, 0.8, -0.2])
    nz /= np.linalg.norm(nz)
    box = W.box_single_sphere()
    xs = np.stack([x0, x1, x2, z])
    qs = np.vstack([q, np.zeros((1, 3))])
    nrm = np.vstack([np.zeros((3, 3)), nz[None]])
    got = O.local_elem(box, ALPHA, RCUT, layer, xs, np.array([[0, 1, 2]]), qs, nrm=nrm,
                       targets=[3])[0]
    ref = _sweep(x0, x1, x2, z, q, layer, nz, 48)
    assert np.abs(ref - _sweep(x0, x1, x2, z, q, layer, nz, 96)).max() < 1e-12
    # the 4x4 rule's own error on this smooth integrand is ~1e-5
    assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("layer", [0, 1])
@pytest.mark.parametrize("vertex", [0, 1, 2])
def test_polar_rule_matches_adaptive_integral(layer, vertex):
    """The target is one vertex of the triangle; the oracle relabels it as
    vertex 1 of the parent triangle and integrates in polar coordinates."""
    x0, x1, x2, q = _triangle()
    xs = np.stack([x0, x1, x2])
    _, _, nt, *_ = _frame(x0, x1, x2)
    nz = nt + np.array([0.08, -0.05, 0.11])    # node normal tilted from the element's
    nz /= np.linalg.norm(nz)
    nrm = np.zeros((3, 3))
    nrm[vertex] = nz
    box = W.box_single_sphere()
    got = O.local_elem(box, ALPHA, RCUT, layer, xs, np.array([[0, 1, 2]]), q, nrm=nrm,
                       targets=[vertex])[0]
    ref = _polar(x0, x1, x2, vertex, q, layer, nz, 48)
    assert np.abs(ref - _polar(x0, x1, x2, vertex, q, layer, nz, 96)).max() < 1e-10
    # the polar 4x4 rule's own error here is up to 1.3e-3 (the same map with
    # 8x8 points is within 6e-8); a dropped Jacobian factor or basis mix-up is O(1)
    assert np.abs(got - ref).max() < 3e-3 * np.abs(ref).max()


def _sphere_case(level):
    V, F = W.icosphere(level)
    box = W.Box(Lx=8.0, Lz=8.0, W=8.0, y0=-4.0, Nx=64, Ny=65, Nz=64)
    c = np.array([4.0, 0.0, 4.0])
    x = V + c
    s = W.Suspension(box=box, x=x, tri=F, particle=np.zeros(len(x), np.int32),
                     centres=c[None], radius=1.0)
    _, _, _, nb = O.geometry(x, F)
    vol = abs(np.einsum("ij,ij->i", x[F[:, 0]] - c,
                        np.cross(x[F[:, 1]] - c, x[F[:, 2]] - c)).sum()) / 6.0
    w = O.single_layer(s, nb, alpha=ALPHA)
    v = O.double_layer(s, nb, alpha=ALPHA)
    lam_exact = 4.0 * math.pi * (1.0 - 2.0 * vol / (8.0 * 8.0 * 8.0))
    return w, v, nb, lam_exact


@pytest.mark.slow
def test_sphere_with_normal_density():
    res = [_sphere_case(level) for level in (2, 3)]
    werr, lerr, perr = [], [], []
    for w, v, nb, lam_exact in res:
        lam = np.einsum("ij,ij->i", v, nb)
        werr.append(np.abs(w).max())
        lerr.append(abs(lam.mean() - lam_exact) / lam_exact)
        perr.append(np.abs(v - lam.mean() * nb).max() / lam_exact)
    # level 3 has 4x the elements of level 2: errors fall by >= 2x (O(h) or better)
    assert werr[1] < 0.5 * werr[0] and werr[1] < 5e-3
    assert lerr[1] < 0.5 * lerr[0] and lerr[1] < 5e-3
    assert perr[1] < 0.5 * perr[0] and perr[1] < 3e-3
