"""Capsule dynamics oracle: membrane traction jump, undisturbed flows, the
right-hand side of the Fredholm equation and the time step, in plain FP64
numpy on top of oracle.oracle.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may import this module.  It shares no code with the
CUDA library.

Paper: Kumar & Graham, arXiv 1109.6587.
  * membrane traction jump (Sec. 4): each flat triangle k stores the elastic
    energy A0_k W(lambda_1, lambda_2) of a neo-Hookean membrane, Eq. (eq_WNH),
    with the principal stretches of the triangle's uniform deformation from
    its reference (undeformed) shape; the force on a vertex follows from the
    principle of virtual work (the gradient of the stored energy), and the
    traction jump at node p is that force over the node's area A_p (a third
    of the areas of its triangles), Eq. (cntr2);
  * undisturbed flows and their stress (App. B): pressure-driven flow and
    simple shear, f_inf = sigma_inf . n, Eq. (straction);
  * right-hand side of Eq. (qa): b = -(Delta f/(lambda + 1) + kappa f_inf)/(4 pi mu);
  * velocity u = u_inf + int q G dS, Eq. (bi_ua), and the midpoint (second
    order Runge-Kutta) step of dx/dt = u, Sec. 5, with the time step rule
    gamma_dot dt = 0.5 Ca h_min / a;
  * volume and the volume correction, overlap correction (Sec. 5, 7.1).

Readings (the paper is silent or leaves the detail to its references):
  * the virtual-work force of Charrier et al. is taken as the exact gradient
    of E = sum_k A0_k W with respect to the vertex positions, and the traction
    jump as +grad E / A_p (so that a uniformly stretched sphere has the
    outward Laplace jump 2T/R: the paper's reaction force F_p is the force the
    membrane exerts on the node, -grad E);
  * A_p uses the current (deformed) triangle areas;
  * simple shear is u = gamma_dot (y - y_mid) e_x about the slit mid-plane;
    the pressure of the pressure-driven flow is -8 mu U0 x / H^2 with x the
    node's own (unwrapped) coordinate, as printed;
  * volume correction: the nodes of a particle whose volume left V0 by more
    than the threshold move along their normals by (V0 - V)/S, S its area,
    repeated until within the threshold (one pass leaves a second-order
    residual on a faceted mesh);
  * overlap correction: the gap of two particles is their smallest node to
    node distance (minimum image); pairs closer than the minimum gap move
    apart rigidly along their line of centres (node centroids) by half the
    deficit each, all pairs of a sweep at once from the positions at its
    start (a particle in several pairs moves by the sum), sweeps repeated
    until no pair violates it.  Node distances see near contacts,
    not deep overlaps (nodes of interpenetrating meshes can stay a node
    spacing apart); the correction exists to keep gaps from closing.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O


# ------------------------------------------------------------ membrane (Sec. 4)

def _tri_vectors(x, tri):
    x = np.asarray(x, dtype=np.float64)
    x1, x2, x3 = x[tri[:, 0]], x[tri[:, 1]], x[tri[:, 2]]
    return x2 - x1, x3 - x1


def _metric(e1, e2):
    g11 = np.einsum("ki,ki->k", e1, e1)
    g12 = np.einsum("ki,ki->k", e1, e2)
    g22 = np.einsum("ki,ki->k", e2, e2)
    return g11, g12, g22


def membrane_energy(x, x_ref, tri, shear_modulus):
    """Stored energy E = sum_k A0_k W_NH of the mesh x relative to x_ref,
    W_NH = (G/2)(lambda_1^2 + lambda_2^2 + 1/(lambda_1 lambda_2)^2 - 3)
    (Eq. (eq_WNH)); lambda_1^2 + lambda_2^2 and lambda_1^2 lambda_2^2 are the
    trace and determinant of the triangle's right Cauchy-Green tensor."""
    E1, E2 = _tri_vectors(x_ref, tri)
    e1, e2 = _tri_vectors(x, tri)
    G11, G12, G22 = _metric(E1, E2)
    g11, g12, g22 = _metric(e1, e2)
    detG = G11 * G22 - G12 * G12
    detg = g11 * g22 - g12 * g12
    trC = (G22 * g11 - 2.0 * G12 * g12 + G11 * g22) / detG
    detC = detg / detG
    A0 = 0.5 * np.sqrt(detG)
    W = 0.5 * shear_modulus * (trC + 1.0 / detC - 3.0)
    return float((A0 * W).sum())


def membrane_forces(x, x_ref, tri, shear_modulus):
    """Gradient of membrane_energy with respect to every node, [N, 3]."""
    E1, E2 = _tri_vectors(x_ref, tri)
    e1, e2 = _tri_vectors(x, tri)
    G11, G12, G22 = _metric(E1, E2)
    g11, g12, g22 = _metric(e1, e2)
    detG = G11 * G22 - G12 * G12
    detg = g11 * g22 - g12 * g12
    A0 = 0.5 * np.sqrt(detG)
    # inverse reference metric
    i11, i12, i22 = G22 / detG, -G12 / detG, G11 / detG
    # d trC / d e1 = 2 (i11 e1 + i12 e2), d trC / d e2 = 2 (i12 e1 + i22 e2)
    dtr1 = 2.0 * (i11[:, None] * e1 + i12[:, None] * e2)
    dtr2 = 2.0 * (i12[:, None] * e1 + i22[:, None] * e2)
    # d detg / d e1 = 2 (g22 e1 - g12 e2), d detg / d e2 = 2 (g11 e2 - g12 e1)
    ddet1 = 2.0 * (g22[:, None] * e1 - g12[:, None] * e2)
    ddet2 = 2.0 * (g11[:, None] * e2 - g12[:, None] * e1)
    # d (1/detC) = -(detG / detg^2) d detg
    c = (detG / (detg * detg))[:, None]
    s = (0.5 * shear_modulus * A0)[:, None]
    f2 = s * (dtr1 - c * ddet1)
    f3 = s * (dtr2 - c * ddet2)
    f1 = -(f2 + f3)
    out = np.zeros((np.asarray(x).shape[0], 3))
    for v, f in ((0, f1), (1, f2), (2, f3)):
        np.add.at(out, tri[:, v], f)
    return out


def traction_jump(x, x_ref, tri, shear_modulus):
    """Delta f at the nodes: the energy gradient over the node's area A_p, a
    third of the current areas of its triangles (Eq. (cntr2))."""
    _, _, Ab, _ = O.geometry(x, tri)
    return membrane_forces(x, x_ref, tri, shear_modulus) / Ab[:, None]


# ------------------------------------------------------ undisturbed flows (App. B)

def undisturbed(box, x, kind, strength, mu=1.0):
    """(u_inf [N, 3], sigma_inf [N, 3, 3]) at the points x.
    kind "shear": u = strength (y - y_mid) e_x, sigma = mu strength e;
    kind "poiseuille": u = 4 U0 s (1 - s) e_x, s = (y - y0)/H, U0 = strength,
    sigma = (8 mu U0 / H^2) x delta + (4 mu U0 / H)(1 - 2 s) e;
    e the symmetric xy unit tensor."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    u = np.zeros((n, 3))
    sig = np.zeros((n, 3, 3))
    if kind == "shear":
        u[:, 0] = strength * (x[:, 1] - (box.y0 + 0.5 * box.W))
        sig[:, 0, 1] = sig[:, 1, 0] = mu * strength
    elif kind == "poiseuille":
        H = box.W
        s = (x[:, 1] - box.y0) / H
        u[:, 0] = 4.0 * strength * s * (1.0 - s)
        p = -8.0 * mu * strength / H ** 2 * x[:, 0]
        for i in range(3):
            sig[:, i, i] = -p
        sig[:, 0, 1] = sig[:, 1, 0] = 4.0 * mu * strength / H * (1.0 - 2.0 * s)
    elif kind != "none":
        raise ValueError(kind)
    return u, sig


def f_inf(box, x, normals, kind, strength, mu=1.0):
    """Undisturbed traction sigma_inf . n (Eq. (straction))."""
    _, sig = undisturbed(box, x, kind, strength, mu)
    return np.einsum("nij,nj->ni", sig, normals)


# ------------------------------------------------- right-hand side and step

def capsule_rhs(susp, x_ref, lam, shear_modulus, kind, strength, mu=1.0):
    """b of Eq. (qa) at the nodes and kappa: b = -(Delta f/(lam + 1) +
    kappa f_inf)/(4 pi mu), kappa = (lam - 1)/(lam + 1); lam [N] per node."""
    lam = np.asarray(lam, dtype=np.float64)
    kappa = (lam - 1.0) / (lam + 1.0)
    df = traction_jump(susp.x, x_ref, susp.tri, shear_modulus)
    _, _, _, nb = O.geometry(susp.x, susp.tri)
    fi = f_inf(susp.box, susp.x, nb, kind, strength, mu)
    b = -(df / (lam + 1.0)[:, None] + kappa[:, None] * fi) / (4.0 * math.pi * mu)
    return kappa, b


def velocity(susp, x_ref, lam, shear_modulus, kind, strength, q0=None, tol=1e-10,
             quadrature="element", mu=1.0):
    """Node velocities u = u_inf + int q G dS (Eq. (bi_ua)) with q from
    Eq. (qa).  Returns (u, q, GMRES iterations)."""
    kappa, b = capsule_rhs(susp, x_ref, lam, shear_modulus, kind, strength, mu)
    q, its, rr, ok = O.bie_solve(susp, kappa, b, q0=b if q0 is None else q0, tol=tol,
                                 quadrature=quadrature, mu=mu)
    ui, _ = undisturbed(susp.box, susp.x, kind, strength, mu)
    return ui + O.single_layer(susp, q, quadrature, mu), q, its


def _moved(susp, x):
    from copy import copy
    s = copy(susp)
    s.x = np.ascontiguousarray(x)
    return s


def midpoint_step(susp, x_ref, lam, shear_modulus, kind, strength, dt, q0=None, tol=1e-10,
                  quadrature="element", mu=1.0):
    """One second-order midpoint (Runge-Kutta) step of dx/dt = u (Sec. 5):
    x_half = x + dt/2 u(x), x_new = x + dt u(x_half); each stage's solve
    starts from the previous stage's density.  Returns (x_new, q of the
    second stage, total GMRES iterations)."""
    u1, q1, i1 = velocity(susp, x_ref, lam, shear_modulus, kind, strength, q0, tol,
                          quadrature, mu)
    half = _moved(susp, susp.x + 0.5 * dt * u1)
    u2, q2, i2 = velocity(half, x_ref, lam, shear_modulus, kind, strength, q1, tol,
                          quadrature, mu)
    return susp.x + dt * u2, q2, i1 + i2


def min_separation(x, box=None):
    """Smallest distance between two distinct nodes (any particles), by brute
    force; with a box, the minimum image in x and z (the periodic system)."""
    x = np.asarray(x, dtype=np.float64)
    best = np.inf
    for i in range(len(x) - 1):
        d = x[i + 1:] - x[i]
        if box is not None:
            d[:, 0] -= box.Lx * np.round(d[:, 0] / box.Lx)
            d[:, 2] -= box.Lz * np.round(d[:, 2] / box.Lz)
        best = min(best, np.linalg.norm(d, axis=1).min())
    return float(best)


def time_step(x, ca, radius, gamma_dot, box=None):
    """dt with gamma_dot dt = 0.5 Ca h_min / a (Sec. 5)."""
    return 0.5 * ca * min_separation(x, box) / (radius * gamma_dot)


# ------------------------------------------------------ volume and overlaps

def volumes(x, tri, particle, n_particles):
    """Enclosed volume of every particle (divergence theorem over its
    outward-oriented triangles: sum x1 . (x2 x x3) / 6)."""
    x = np.asarray(x, dtype=np.float64)
    x1, x2, x3 = x[tri[:, 0]], x[tri[:, 1]], x[tri[:, 2]]
    v = np.einsum("ki,ki->k", x1, np.cross(x2, x3)) / 6.0
    out = np.zeros(n_particles)
    np.add.at(out, np.asarray(particle)[tri[:, 0]], v)
    return out


def volume_correct(x, tri, particle, v0, threshold=1e-4, passes=10):
    """Nodes of every particle whose volume differs from v0 by more than
    threshold * v0 move along their unit normals by (v0 - V)/S, S its area;
    repeated (at most `passes` times) until every particle is within the
    threshold: on a faceted mesh one pass leaves a residual of second order.
    Returns (x, passes made)."""
    x = np.array(x, dtype=np.float64)
    particle = np.asarray(particle)
    n_p = len(v0)
    for k in range(passes):
        v = volumes(x, tri, particle, n_p)
        off = np.abs(v - v0) > threshold * np.abs(v0)
        if not off.any():
            return x, k
        _, _, Ab, nb = O.geometry(x, tri)
        S = np.zeros(n_p)
        np.add.at(S, particle, Ab)
        d = np.where(off, (v0 - v) / S, 0.0)
        x = x + d[particle][:, None] * nb
    return x, passes


def centroids(x, particle, n_particles):
    """Mean node position of every particle (unwrapped meshes)."""
    x = np.asarray(x, dtype=np.float64)
    c = np.zeros((n_particles, 3))
    cnt = np.zeros(n_particles)
    np.add.at(c, np.asarray(particle), x)
    np.add.at(cnt, np.asarray(particle), 1.0)
    return c / cnt[:, None]


def overlap_correct(x, particle, n_particles, box, h_min, max_sweeps=100):
    """Minimum-gap correction (Sec. 7.1).  Each sweep finds every pair of
    particles whose closest nodes (minimum image in x, z) are nearer than
    h_min, from the positions at the start of the sweep, and moves both
    rigidly along their line of centres (node centroids, minimum image) by
    half the deficit each; a particle in several pairs moves by the sum.
    Sweeps repeat until no pair violates the gap (gaps within 1e-9 h_min of
    it count as met: a corrected pair lands on h_min up to rounding).
    Returns (x, pair moves)."""
    x = np.array(x, dtype=np.float64)
    particle = np.asarray(particle)
    moves = 0

    def image(d):
        d = d.copy()
        d[..., 0] -= box.Lx * np.round(d[..., 0] / box.Lx)
        d[..., 2] -= box.Lz * np.round(d[..., 2] / box.Lz)
        return d

    for _ in range(max_sweeps):
        c = centroids(x, particle, n_particles)
        disp = np.zeros((n_particles, 3))
        found = 0
        for p in range(n_particles):
            xp = x[particle == p]
            for q in range(p + 1, n_particles):
                xq = x[particle == q]
                gap = np.linalg.norm(image(xp[:, None, :] - xq[None, :, :]), axis=2).min()
                if gap < h_min * (1.0 - 1e-9):             # corrected gaps land on h_min
                    d = image(c[q] - c[p])
                    e = d / np.linalg.norm(d)
                    s = 0.5 * (h_min - gap)
                    disp[p] -= s * e
                    disp[q] += s * e
                    found += 1
        if not found:
            break
        x += disp[particle]
        moves += found
    return x, moves
