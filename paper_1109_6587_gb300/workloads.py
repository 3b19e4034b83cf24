"""Seeded synthetic inputs: capsule meshes, suspensions and point forces.

This module only builds inputs (geometry and random numbers).  It holds none of
the GGEM arithmetic, so both the CPU oracle and the CUDA path can draw from it.

Meshes follow the paper's surface discretisation (Sec. 3.3): an icosahedron
whose faces are split recursively into four, with every vertex pushed onto the
sphere, giving N_tri = 20*4^k triangles and N_b = N_tri/2 + 2 nodes.  Triangles
are oriented so that (x2-x1) x (x3-x1) points out of the capsule.

Workload recipe (all seeded through numpy's PCG64):
  * capsule centres drawn uniformly in the box, rejected when closer than
    2a(1 + 0.05/2) to an earlier centre (minimum gap 0.05a, Sec. 7.1) or
    when the capsule would come within ``wall_gap`` of a wall;
  * point forces / densities i.i.d. N(0, 1) per component.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def icosphere(level: int):
    """Unit-sphere triangulation by recursive subdivision (Sec. 3.3).

    Returns (vertices [N_b, 3] float64, triangles [N_tri, 3] int32).
    """
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v.append((0.0, a, b))
            v.append((a, b, 0.0))
            v.append((b, 0.0, a))
    verts = np.array(v, dtype=np.float64)
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    # faces: triples of mutually adjacent vertices (edge = shortest distance)
    d = np.linalg.norm(verts[:, None, :] - verts[None, :, :], axis=2)
    edge = np.min(d[d > 1e-9])
    adj = np.abs(d - edge) < 1e-6
    faces = []
    for i in range(12):
        for j in range(i + 1, 12):
            if not adj[i, j]:
                continue
            for k in range(j + 1, 12):
                if adj[i, k] and adj[j, k]:
                    faces.append((i, j, k))
    faces = np.array(faces, dtype=np.int64)
    assert faces.shape == (20, 3)
    verts_l = [tuple(p) for p in verts]
    for _ in range(level):
        cache = {}
        new_faces = []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                p = (np.asarray(verts_l[a]) + np.asarray(verts_l[b])) * 0.5
                p /= np.linalg.norm(p)
                cache[key] = len(verts_l)
                verts_l.append(tuple(p))
            return cache[key]

        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = np.array(new_faces, dtype=np.int64)
    verts = np.array(verts_l, dtype=np.float64)
    # orient outward
    x1, x2, x3 = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    nrm = np.cross(x2 - x1, x3 - x1)
    flip = np.einsum("ij,ij->i", nrm, x1 + x2 + x3) < 0
    faces[flip] = faces[flip][:, [0, 2, 1]]
    assert verts.shape[0] == 20 * 4 ** level // 2 + 2
    return verts, faces.astype(np.int32)


@dataclasses.dataclass
class Box:
    """Periodic slit: x in [0, Lx), z in [0, Lz) periodic; walls at y0 and y0+W."""
    Lx: float
    Lz: float
    W: float
    y0: float
    Nx: int
    Ny: int
    Nz: int


@dataclasses.dataclass
class Suspension:
    box: Box
    x: np.ndarray          # [N, 3] node positions (each capsule unwrapped)
    tri: np.ndarray        # [M, 3] int32 node indices, outward oriented
    particle: np.ndarray   # [N] int32 capsule id of each node
    centres: np.ndarray    # [Np, 3]
    radius: float


def place_centres(n_p, box: Box, radius, rng, min_gap=0.05, wall_gap=0.05,
                  max_tries=2_000_000):
    """Uniform non-overlapping capsule centres (rejection sampling)."""
    dmin = 2.0 * radius + min_gap * radius
    ylo = box.y0 + radius + wall_gap * radius
    yhi = box.y0 + box.W - radius - wall_gap * radius
    if yhi <= ylo:
        raise ValueError("slit too narrow for the capsules")
    # cell grid for O(1) overlap checks
    h = dmin
    ncx, ncz = max(1, int(box.Lx // h)), max(1, int(box.Lz // h))
    ncy = max(1, int((yhi - ylo) // h) + 1)
    cells = {}
    out = []
    tries = 0
    while len(out) < n_p:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"could only place {len(out)} of {n_p} capsules")
        c = np.array([rng.uniform(0, box.Lx), rng.uniform(ylo, yhi),
                      rng.uniform(0, box.Lz)])
        ci = (int(c[0] / box.Lx * ncx) % ncx, min(int((c[1] - ylo) / h), ncy - 1),
              int(c[2] / box.Lz * ncz) % ncz)
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = ((ci[0] + dx) % ncx, ci[1] + dy, (ci[2] + dz) % ncz)
                    for j in cells.get(key, ()):
                        d = c - out[j]
                        d[0] -= box.Lx * round(d[0] / box.Lx)
                        d[2] -= box.Lz * round(d[2] / box.Lz)
                        if d @ d < dmin * dmin:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            cells.setdefault(ci, []).append(len(out))
            out.append(c)
    return np.array(out)


def suspension(n_p, box: Box, level=3, radius=1.0, seed=0, centres=None):
    """n_p spherical capsules of the given icosphere level in the slit."""
    rng = np.random.default_rng(seed)
    if centres is None:
        centres = place_centres(n_p, box, radius, rng)
    v, t = icosphere(level)
    nb = v.shape[0]
    x = (centres[:, None, :] + radius * v[None, :, :]).reshape(-1, 3)
    tri = (t[None, :, :] + nb * np.arange(len(centres))[:, None, None]).reshape(-1, 3)
    part = np.repeat(np.arange(len(centres), dtype=np.int32), nb)
    return Suspension(box, np.ascontiguousarray(x), tri.astype(np.int32), part,
                      centres, radius)


def normal_forces(n, seed=0, comps=3):
    """i.i.d. N(0,1) values, shape [n, comps]."""
    return np.random.default_rng(seed).standard_normal((n, comps))


# ---- the workloads -------------------------------------------------------

def box_single_sphere():
    """One capsule of radius 1 in an 8 x [-2,2] x 8 slit; 32 x 33 x 32 grid."""
    return Box(Lx=8.0, Lz=8.0, W=4.0, y0=-2.0, Nx=32, Ny=33, Nz=32)


def single_sphere(seed=0, radius=1.0):
    """162-node icosphere centred at (4, 0, 4).

    With radius 1 every node has its antipode exactly at r_cut = 2 (alpha = 2
    on the 32 x 33 x 32 grid), so whether those pairs count is decided by
    rounding; a radius a little below 1 removes that tie."""
    return suspension(1, box_single_sphere(), level=2, radius=radius, seed=seed,
                      centres=np.array([[4.0, 0.0, 4.0]]))


def box_100_capsules():
    """40 x [-5,5] x 40 slit, 128 x 65 x 128 grid."""
    return Box(Lx=40.0, Lz=40.0, W=10.0, y0=-5.0, Nx=128, Ny=65, Nz=128)


def capsules_100(seed=0):
    """100 capsules x 642 nodes (64,200 points)."""
    return suspension(100, box_100_capsules(), level=3, radius=1.0, seed=seed)


def box_1000_capsules():
    """80 x [-10,10] x 80 slit, 256 x 97 x 256 grid."""
    return Box(Lx=80.0, Lz=80.0, W=20.0, y0=-10.0, Nx=256, Ny=97, Nz=256)


def capsules_1000(seed=0):
    """1000 capsules x 642 nodes (642,000 points)."""
    return suspension(1000, box_1000_capsules(), level=3, radius=1.0, seed=seed)


def capsules_at_phi(box: Box, phi, seed=0, level=3, radius=1.0):
    """Spherical capsules filling the slit to the volume fraction phi
    (n = round(phi Lx Lz W / (4/3 pi a^3)))."""
    n = int(round(phi * box.Lx * box.Lz * box.W / (4.0 / 3.0 * math.pi * radius ** 3)))
    return suspension(n, box, level=level, radius=radius, seed=seed)


def capsules_100_phi(seed=0):
    """The 100-capsule slit and grid filled to phi = 0.1: 382 capsules x 642
    nodes (245,244 points)."""
    return capsules_at_phi(box_100_capsules(), 0.1, seed=seed)


def capsules_1000_phi(seed=0):
    """The 1000-capsule slit and grid filled to phi = 0.2: 6112 capsules x 642
    nodes (3,923,904 points)."""
    return capsules_at_phi(box_1000_capsules(), 0.2, seed=seed)


# ---- generated suspensions for the learned warm start ---------------------

def box_training(nx=64):
    """Slit of the training suspensions: gap 10a, x-z spacing and Chebyshev
    grid of the 100-capsule workload (alpha = 1.6, r_cut = 2.5), a periodic
    cell of nx x nx intervals (20 x 20 for nx = 64)."""
    return Box(Lx=0.3125 * nx, Lz=0.3125 * nx, W=10.0, y0=-5.0, Nx=nx, Ny=65, Nz=nx)


# (volume fraction, viscosity ratio, cell intervals) of the training suspensions:
# 48 to 382 capsules of 642 nodes, phi from 0.05 to 0.3, lambda in {0.2, 1, 5}
TRAINING_SET = ((0.05, 5.0, 64), (0.1, 0.2, 64), (0.2, 1.0, 64), (0.3, 5.0, 64),
                (0.1, 1.0, 128), (0.2, 5.0, 64))


def training_suspensions(seed=1):
    """Generated suspensions for training the learned warm start: for each
    entry of TRAINING_SET, spherical level-3 capsules filling box_training(nx)
    to that volume fraction (seed, seed + 1, ...), with its viscosity ratio.
    Returns [(suspension, lambda)]."""
    return [(capsules_at_phi(box_training(nx), phi, seed=seed + k), lam)
            for k, (phi, lam, nx) in enumerate(TRAINING_SET)]


# Evans-Fung biconcave profile of a red blood cell in units of its radius R0:
# half-thickness h(rho) = (R0/2) sqrt(1 - rho^2) (C0 + C1 rho^2 + C2 rho^4),
# rho the distance from the axis over R0 (Evans and Fung 1972).
EVANS_FUNG = (0.2072, 2.0026, -1.1228)


def rbc_mesh(level=3, radius=1.0):
    """Biconcave capsule: the icosphere's vertices mapped onto the Evans-Fung
    profile about the y axis (x, z scaled by the radius, y replaced by the
    signed half-thickness at that distance from the axis).  The map keeps the
    triangles' orientation (outward normals)."""
    v, t = icosphere(level)
    rho2 = np.clip(v[:, 0] ** 2 + v[:, 2] ** 2, 0.0, 1.0)
    c0, c1, c2 = EVANS_FUNG
    h = 0.5 * radius * np.sqrt(1.0 - rho2) * (c0 + c1 * rho2 + c2 * rho2 * rho2)
    x = np.stack([radius * v[:, 0], np.sign(v[:, 1]) * h, radius * v[:, 2]], 1)
    return x, t


def random_rotations(n, rng):
    """n uniformly random rotation matrices (QR of Gaussian matrices, sign
    fixed so that the factor is a proper rotation)."""
    out = np.empty((n, 3, 3))
    for k in range(n):
        q, r = np.linalg.qr(rng.standard_normal((3, 3)))
        q = q * np.sign(np.diag(r))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        out[k] = q
    return out


def box_rbc_4000():
    """150 x [-15, 15] x 150 slit, 512 x 129 x 512 grid."""
    return Box(Lx=150.0, Lz=150.0, W=30.0, y0=-15.0, Nx=512, Ny=129, Nz=512)


def rbc_4000(seed=0, level=3, radius=1.0):
    """4000 biconcave capsules x 642 nodes (2,568,000 points), each randomly
    oriented, centres placed as for spheres of the cell's radius (which
    bounds it) with the minimum gap 0.05a."""
    box = box_rbc_4000()
    rng = np.random.default_rng(seed)
    centres = place_centres(4000, box, radius, rng)
    rot = random_rotations(len(centres), rng)
    v, t = rbc_mesh(level, radius)
    nb = v.shape[0]
    x = (centres[:, None, :] + np.einsum("pij,nj->pni", rot, v)).reshape(-1, 3)
    tri = (t[None, :, :] + nb * np.arange(len(centres))[:, None, None]).reshape(-1, 3)
    part = np.repeat(np.arange(len(centres), dtype=np.int32), nb)
    return Suspension(box, np.ascontiguousarray(x), tri.astype(np.int32), part, centres,
                      radius)


# ---- Fredholm-solve inputs and emulated time steps ------------------------

def bie_rhs(susp: Suspension, lam=5.0, gamma=1.0, seed=0, step=0, mu=1.0):
    """Synthetic right-hand side of the Fredholm system, Eq. (qa):
        b = -(dF / (lam + 1) + kappa f_inf) / (4 pi mu),  kappa = (lam-1)/(lam+1),
    with f_inf = mu gamma (r_y, r_x, 0) the traction of the shear flow
    u_inf = (gamma y, 0, 0) on the undeformed spheres (r the unit radial
    vector from each capsule's centre), and dF a smooth random membrane load
    per capsule, dF = a_p + B_p r with a_p ~ N(0, 1/4), B_p ~ N(0, 1) per
    entry; `step` drifts the load by 0.05 * step of a second random field.
    Returns (kappa [N], b [N, 3])."""
    rng = np.random.default_rng(seed)
    n_p = len(susp.centres)
    a0, B0 = 0.5 * rng.standard_normal((n_p, 3)), rng.standard_normal((n_p, 3, 3))
    a1, B1 = 0.5 * rng.standard_normal((n_p, 3)), rng.standard_normal((n_p, 3, 3))
    a = a0 + 0.05 * step * a1
    B = B0 + 0.05 * step * B1
    p = susp.particle
    r = susp.x - susp.centres[p]
    r /= np.linalg.norm(r, axis=1, keepdims=True)
    dF = a[p] + np.einsum("nij,nj->ni", B[p], r)
    f_inf = mu * gamma * np.stack([r[:, 1], r[:, 0], np.zeros(len(r))], 1)
    kappa = (lam - 1.0) / (lam + 1.0)
    b = -(dF / (lam + 1.0) + kappa * f_inf) / (4.0 * math.pi * mu)
    return np.full(len(r), kappa), b


def rigid_step(susp: Suspension, seed=0, step=1, amp=0.01):
    """The suspension after `step` emulated time steps: every capsule moved
    rigidly by the sum of `step` random displacements of size amp * radius
    (standing in for the membrane mechanics and time stepper)."""
    rng = np.random.default_rng(seed)
    n_p = len(susp.centres)
    shift = np.zeros((n_p, 3))
    for _ in range(step):
        d = rng.standard_normal((n_p, 3))
        shift += amp * susp.radius * d / np.linalg.norm(d, axis=1, keepdims=True)
    c = susp.centres + shift
    return Suspension(susp.box, np.ascontiguousarray(susp.x + shift[susp.particle]),
                      susp.tri, susp.particle, c, susp.radius)
