"""Pins of the capsule-dynamics oracle (oracle/capsule.py), CPU only.

Membrane (Sec. 4, Eq. (eq_WNH)):
  * the nodal forces are the gradient of the stored energy: central finite
    differences of the energy on a randomly deformed mesh (1e-6);
  * an undeformed mesh, and any rigid rotation plus translation of it, carry
    no force;
  * isotropic stretch by lambda about the centre: every flat triangle has
    lambda_1 = lambda_2 = lambda exactly, so E = S0 (G/2)(2 lambda^2 +
    lambda^-4 - 3), and Euler's relation sum_b (x_b - c) . F_b = lambda dE/dlambda
    = S0 G (2 lambda^2 - 2 lambda^-4) holds to rounding;
  * Laplace's law: the traction jump of the stretched sphere approaches the
    outward 2 T / R n, T = G (1 - lambda^-6) the isotropic tension of the
    neo-Hookean membrane; the mean error falls about 4x per mesh level.
Undisturbed flows (App. B): the pressure-driven flow and simple shear satisfy
the Stokes equations and their wall conditions, and their printed stress
equals -p I + mu (grad u + grad u^T) (finite differences of u and p).
Velocity of a spherical drop (Eqs. (bi_ua), (qa)): with no interfacial force
(an undeformed membrane) in simple shear, a sphere of any viscosity ratio
turns with half the fluid's vorticity, and its surface moves normally at
5/(2 lambda + 3) times the undisturbed straining rate (the classical result
for a drop in a linear flow; 1 for lambda = 1); 642 nodes, walls 5 radii
away: within 3 % (the error shrinks with the mesh: 3.9 % -> 1.6 % at
lambda = 5 from 162 to 642 nodes).
Time stepping (Sec. 5):
  * the midpoint rule is second order: a relaxing ellipsoidal capsule
    integrated over a fixed time with 2, 4 and 8 steps differs from the
    8-step result by a ratio of 5 (exact second order) -- first order would
    give 3;
  * the relaxing capsule's elastic energy decreases at every step (Stokes
    flow dissipates) and its volume stays within 1e-3.
Volumes, volume correction and overlap correction: the volume of a mesh
equals its convex hull's (scipy); the correction removes the volume error to
second order; two capsules closer than the minimum gap end at least that far
apart, displaced along their line of centres; all violating pairs of a sweep
move at once (a chain of three: the middle one stays).
"""
import math

import numpy as np
import pytest

from oracle import capsule as C
from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W


def _rotation(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_membrane_forces_are_the_energy_gradient():
    V, F = W.icosphere(1)
    rng = np.random.default_rng(1)
    x = V * 1.05 + 0.04 * rng.standard_normal(V.shape)
    g = C.membrane_forces(x, V, F, 0.7)
    h = 1e-6
    for b in rng.choice(len(V), 8, replace=False):
        for i in range(3):
            xp, xm = x.copy(), x.copy()
            xp[b, i] += h
            xm[b, i] -= h
            fd = (C.membrane_energy(xp, V, F, 0.7) - C.membrane_energy(xm, V, F, 0.7)) / (2 * h)
            assert abs(fd - g[b, i]) < 1e-6 * max(1.0, abs(fd)), (b, i, fd, g[b, i])


def test_rigid_motion_carries_no_force():
    V, F = W.icosphere(2)
    assert np.abs(C.membrane_forces(V, V, F, 1.0)).max() < 1e-12
    x = V @ _rotation(3).T + np.array([3.0, -1.0, 2.0])
    assert np.abs(C.membrane_forces(x, V, F, 1.0)).max() < 1e-12
    assert abs(C.membrane_energy(x, V, F, 1.0)) < 1e-12


def test_isotropic_stretch_energy_and_euler_relation():
    V, F = W.icosphere(2)
    Ak, _, _, _ = O.geometry(V, F)
    S0 = Ak.sum()
    G = 1.3
    c = np.array([1.0, 2.0, -0.5])
    for lam in (0.9, 1.1, 1.4):
        x = c + lam * V
        E = C.membrane_energy(x, V + c, F, G)
        assert E == pytest.approx(S0 * 0.5 * G * (2 * lam ** 2 + lam ** -4 - 3), rel=1e-12)
        f = C.membrane_forces(x, V + c, F, G)
        euler = np.einsum("ni,ni->", x - c, f)
        assert euler == pytest.approx(S0 * G * (2 * lam ** 2 - 2 * lam ** -4), rel=1e-12)


def test_laplace_law_on_a_stretched_sphere():
    lam, G = 1.1, 1.0
    T = G * (1.0 - lam ** -6)
    errs = []
    for level in (1, 2, 3):
        V, F = W.icosphere(level)
        x = lam * V
        df = C.traction_jump(x, V, F, G)
        _, _, _, nb = O.geometry(x, F)
        dn = np.einsum("ni,ni->n", df, nb)
        errs.append(np.abs(dn / (2 * T / lam) - 1).mean())
        tang = np.linalg.norm(df - dn[:, None] * nb, axis=1).max()
        assert tang < 0.01 * 2 * T / lam
    assert errs[1] < errs[0] / 2.5 and errs[2] < errs[1] / 2.5
    assert errs[2] < 0.006


@pytest.mark.parametrize("kind", ["shear", "poiseuille"])
def test_undisturbed_flows(kind):
    box = W.Box(Lx=16.0, Lz=16.0, W=6.0, y0=-3.0, Nx=32, Ny=33, Nz=32)
    mu, s = 1.7, 0.8
    rng = np.random.default_rng(4)
    x = np.column_stack([rng.uniform(0, 16, 20), rng.uniform(-2.5, 2.5, 20), rng.uniform(0, 16, 20)])
    h = 1e-4

    def up(pts):
        u, sig = C.undisturbed(box, pts, kind, s, mu)
        p = -np.trace(sig, axis1=1, axis2=2) / 3.0          # sigma = -p I + deviatoric
        return u, p

    grad = np.zeros((20, 3, 3))
    lap = np.zeros((20, 3))
    gp = np.zeros((20, 3))
    u0, p0 = up(x)
    for k in range(3):
        d = np.zeros(3)
        d[k] = h
        (ua, pa), (ub, pb) = up(x + d), up(x - d)
        grad[:, :, k] = (ua - ub) / (2 * h)                 # du_i / dx_k
        lap += (ua - 2 * u0 + ub) / h ** 2
        gp[:, k] = (pa - pb) / (2 * h)
    assert np.abs(mu * lap - gp).max() < 1e-5               # Stokes momentum balance
    assert np.abs(np.trace(grad, axis1=1, axis2=2)).max() < 1e-8
    _, sig = C.undisturbed(box, x, kind, s, mu)
    ref = -p0[:, None, None] * np.eye(3) + mu * (grad + grad.transpose(0, 2, 1))
    assert np.abs(sig - ref).max() < 1e-6
    walls = np.array([[3.0, -3.0, 5.0], [3.0, 3.0, 5.0]])
    uw, _ = C.undisturbed(box, walls, kind, s, mu)
    want = [[-s * 3.0, 0, 0], [s * 3.0, 0, 0]] if kind == "shear" else [[0, 0, 0], [0, 0, 0]]
    assert np.allclose(uw, want, atol=1e-14)


@pytest.mark.parametrize("lam", [0.2, 5.0])
def test_spherical_drop_in_shear(lam):
    box = W.Box(Lx=16.0, Lz=16.0, W=10.0, y0=-5.0, Nx=32, Ny=33, Nz=32)
    s = W.suspension(1, box, level=3, centres=np.array([[8.0, 0.0, 8.0]]))
    r = s.x - s.centres[0]
    _, _, _, nb = O.geometry(s.x, s.tri)
    gd = 1.0
    u, q, its = C.velocity(s, s.x, np.full(len(s.x), lam), 1.0, "shear", gd, tol=1e-8)
    # rigid part U + Omega x r by least squares
    A = np.zeros((3 * len(r), 6))
    for k, (rx, ry, rz) in enumerate(r):
        A[3 * k:3 * k + 3, :3] = np.eye(3)
        A[3 * k:3 * k + 3, 3:] = [[0, rz, -ry], [-rz, 0, rx], [ry, -rx, 0]]
    sol, *_ = np.linalg.lstsq(A, u.ravel(), rcond=None)
    assert np.abs(sol[:3]).max() < 1e-3 * gd
    assert sol[5] == pytest.approx(-0.5 * gd, rel=0.01)
    assert np.abs(sol[3:5]).max() < 1e-3 * gd
    a = np.linalg.norm(r, axis=1)
    nEn = a * gd * nb[:, 0] * nb[:, 1]                      # a n.E.n, E_xy = gd/2
    ratio = (np.einsum("ni,ni->n", u, nb) @ nEn) / (nEn @ nEn)
    assert ratio == pytest.approx(5.0 / (2.0 * lam + 3.0), rel=0.03)


@pytest.fixture(scope="module")
def relaxing():
    box = W.Box(Lx=16.0, Lz=16.0, W=10.0, y0=-5.0, Nx=32, Ny=33, Nz=32)
    s0 = W.suspension(1, box, level=1, centres=np.array([[8.0, 0.0, 8.0]]))
    c = s0.centres[0]
    S = np.diag([1.25, 1.25 ** -0.5, 1.25 ** -0.5])
    return s0, s0.x.copy(), c + (s0.x - c) @ S.T


def _run(s0, x_ref, x0, n, T):
    s = C._moved(s0, x0)
    q = None
    energies, vols = [C.membrane_energy(x0, x_ref, s0.tri, 1.0)], []
    for _ in range(n):
        xn, q, _ = C.midpoint_step(s, x_ref, np.ones(len(x0)), 1.0, "none", 0.0, T / n, q)
        s = C._moved(s0, xn)
        energies.append(C.membrane_energy(xn, x_ref, s0.tri, 1.0))
        vols.append(C.volumes(xn, s0.tri, s0.particle, 1)[0])
    return s.x, energies, vols


def test_midpoint_rule_is_second_order(relaxing):
    s0, x_ref, x0 = relaxing
    T = 0.4
    x2, _, _ = _run(s0, x_ref, x0, 2, T)
    x4, _, _ = _run(s0, x_ref, x0, 4, T)
    x8, e8, v8 = _run(s0, x_ref, x0, 8, T)
    ratio = np.abs(x2 - x8).max() / np.abs(x4 - x8).max()
    assert 4.0 < ratio < 6.5, ratio
    assert np.abs(x8 - x0).max() > 0.02                     # it did relax
    assert all(b < a for a, b in zip(e8, e8[1:]))           # energy decreases every step
    v0 = C.volumes(x0, s0.tri, s0.particle, 1)[0]
    assert np.abs(np.asarray(v8) / v0 - 1).max() < 1e-3


def test_volumes_and_volume_correction():
    spatial = pytest.importorskip("scipy.spatial")
    box = W.Box(Lx=16.0, Lz=16.0, W=10.0, y0=-5.0, Nx=32, Ny=33, Nz=32)
    s = W.suspension(2, box, level=2, centres=np.array([[4.0, 0.0, 4.0], [11.0, 1.0, 9.0]]),
                     radius=1.3)
    v = C.volumes(s.x, s.tri, s.particle, 2)
    for p in range(2):
        assert v[p] == pytest.approx(spatial.ConvexHull(s.x[s.particle == p]).volume, rel=1e-12)
    x = s.x.copy()
    x[s.particle == 1] = s.centres[1] + 1.002 * (x[s.particle == 1] - s.centres[1])
    v1 = C.volumes(x, s.tri, s.particle, 2)
    assert abs(v1[1] / v[1] - 1) > 5e-3
    x1, k1 = C.volume_correct(x, s.tri, s.particle, v, passes=1)
    e1 = abs(C.volumes(x1, s.tri, s.particle, 2)[1] / v[1] - 1)
    assert e1 < abs(v1[1] / v[1] - 1) / 50                   # one pass: second-order residual
    xc, k = C.volume_correct(x, s.tri, s.particle, v)
    v2 = C.volumes(xc, s.tri, s.particle, 2)
    assert abs(v2[1] / v[1] - 1) <= 1e-4 and k <= 3
    assert np.array_equal(xc[s.particle == 0], x[s.particle == 0])   # within threshold


def test_overlap_correction():
    box = W.Box(Lx=16.0, Lz=16.0, W=10.0, y0=-5.0, Nx=32, Ny=33, Nz=32)
    # two spheres whose icosahedron vertices face each other 0.03 apart along
    # the line of centres, across the periodic boundary in x
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([phi, 0.0, 1.0]) / math.hypot(phi, 1.0)
    c0 = np.array([15.5, 0.0, 8.0])
    c1 = c0 + 2.03 * v
    c1[0] -= box.Lx
    s = W.suspension(2, box, level=2, centres=np.array([c0, c1]))
    h = 0.05
    x, moves = C.overlap_correct(s.x, s.particle, 2, box, h)
    assert moves >= 1
    d = s.centres[1] - s.centres[0]
    d[0] -= box.Lx * round(d[0] / box.Lx)
    shift = s.centres[1] - s.centres[0] - d
    xp = x[s.particle == 0]
    xq = x[s.particle == 1] - shift
    gap = np.linalg.norm(xp[:, None] - xq[None], axis=2).min()
    assert gap >= h * (1 - 1e-9)
    # each particle moved rigidly along the line of centres
    for p, sign in ((0, -1.0), (1, 1.0)):
        disp = x[s.particle == p] - s.x[s.particle == p]
        assert np.abs(disp - disp[0]).max() < 1e-12
        e = d / np.linalg.norm(d)
        assert np.linalg.norm(np.cross(disp[0], e)) < 1e-12 and sign * disp[0] @ e > 0


def test_overlap_correction_sweeps_all_pairs_at_once():
    # a chain of three spheres along an icosahedron vertex direction, each
    # facing pair of vertices 0.03 apart: the middle one is pushed equally
    # both ways in every sweep and stays, so each end closes half of its gap's
    # deficit per sweep (0.03 -> 0.04 -> 0.045 ...) and ends 0.02 further out
    box = W.Box(Lx=16.0, Lz=16.0, W=10.0, y0=-5.0, Nx=32, Ny=33, Nz=32)
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([phi, 0.0, 1.0]) / math.hypot(phi, 1.0)
    c = np.array([8.0, 0.0, 8.0])
    s = W.suspension(3, box, level=2, centres=np.array([c - 2.03 * v, c, c + 2.03 * v]))
    x1, m1 = C.overlap_correct(s.x, s.particle, 3, box, 0.05, max_sweeps=1)
    assert m1 == 2
    assert np.allclose(x1[s.particle == 2][0] - s.x[s.particle == 2][0], 0.01 * v, atol=1e-15)
    x, moves = C.overlap_correct(s.x, s.particle, 3, box, 0.05)
    assert moves % 2 == 0 and moves > 4                     # two pairs per sweep
    disp = [x[s.particle == p][0] - s.x[s.particle == p][0] for p in range(3)]
    assert np.abs(disp[1]).max() < 1e-15
    assert np.allclose(disp[0], -0.02 * v, atol=1e-10) and np.allclose(disp[2], 0.02 * v, atol=1e-10)
