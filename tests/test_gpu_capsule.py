"""Capsule dynamics on the GPU against the oracle (oracle/capsule.py).

Workload: two capsules of 162 nodes in a 16 x [-5, 5] x 16 slit (grid
32 x 33 x 32), deformed from their spherical reference by a seeded random
displacement plus a stretch, viscosity ratios 0.2 and 5, element quadrature.

  * traction jump (FP64 on both sides, only the summation order differs):
    1e-12 of its largest entry;
  * undisturbed velocity and traction, shear and pressure-driven: 1e-14;
  * node velocities of Eqs. (bi_ua), (qa): FP64 plan against the oracle, both
    solved to 1e-11, 1e-9; mixed plan (FP64 true residuals, mixed operator
    and single layer) 1e-5;
  * one midpoint step: the new positions within 1e-8 of the displacement the
    step made;
  * smallest node separation (minimum image) equal to brute force to
    rounding; volumes 1e-13; the volume correction lands within its threshold
    and on the oracle's positions (1e-12);
  * overlap correction: a pair across the periodic boundary and a chain of
    three, the same pair moves as the oracle and its positions (1e-12).
"""
import numpy as np
import pytest

from oracle import capsule as C
from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ggem():
    from paper_1109_6587_gb300 import _build
    _build.build()
    from paper_1109_6587_gb300 import ggem as G
    return G


def _box():
    return W.Box(Lx=16.0, Lz=16.0, W=10.0, y0=-5.0, Nx=32, Ny=33, Nz=32)


@pytest.fixture(scope="module")
def capsules():
    box = _box()
    # the second capsule straddles the periodic boundary in x
    s = W.suspension(2, box, level=2, centres=np.array([[6.0, 1.0, 7.0], [15.3, -1.5, 10.0]]))
    x_ref = s.x.copy()
    rng = np.random.default_rng(11)
    S = np.diag([1.12, 0.95, 1.0 / (1.12 * 0.95)])
    x = s.x.copy()
    for p in range(2):
        m = s.particle == p
        x[m] = s.centres[p] + (x[m] - s.centres[p]) @ S.T + 0.01 * rng.standard_normal((m.sum(), 3))
    s.x = np.ascontiguousarray(x)
    lam = np.where(s.particle == 0, 0.2, 5.0).astype(np.float64)
    return s, x_ref, lam


def _plan(ggem, s, prec):
    P = ggem.Plan.for_box(s.box, precision=prec, quadrature="element", max_points=len(s.x),
                          max_tris=len(s.tri))
    P.mesh_set(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.tri, device="cuda"))
    P.mesh_particles(s.particle, len(s.centres))
    return P


def test_traction_and_flows(ggem, capsules):
    s, x_ref, lam = capsules
    P = _plan(ggem, s, "fp64")
    P.membrane_reference(x_ref)
    G = 0.7
    df = P.membrane_traction(G)
    ref = C.traction_jump(s.x, x_ref, s.tri, G)
    assert np.abs(df - ref).max() < 1e-12 * np.abs(ref).max()
    _, _, _, nb = O.geometry(s.x, s.tri)
    for kind in ("shear", "poiseuille"):
        u, f = P.undisturbed(kind, 0.8)
        ur, sr = C.undisturbed(s.box, s.x, kind, 0.8)
        fr = np.einsum("nij,nj->ni", sr, nb)
        assert np.abs(u - ur).max() < 1e-14 * max(1.0, np.abs(ur).max())
        assert np.abs(f - fr).max() < 1e-13 * max(1.0, np.abs(fr).max())


@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-11, 1e-9), ("mixed", 1e-9, 1e-5)])
def test_capsule_velocity(ggem, capsules, prec, tol, bar):
    s, x_ref, lam = capsules
    P = _plan(ggem, s, prec)
    P.membrane_reference(x_ref)
    u, q, its, rr = P.capsule_velocity(lam, "shear", 0.5, shear_modulus=0.7, tol=tol,
                                       restart=40, maxit=400)
    ur, qr, _ = C.velocity(s, x_ref, lam, 0.7, "shear", 0.5, tol=1e-11)
    assert rr <= tol
    assert np.abs(u - ur).max() < bar * np.abs(ur).max()
    P.check()


def test_midpoint_step(ggem, capsules):
    s, x_ref, lam = capsules
    P = _plan(ggem, s, "fp64")
    P.membrane_reference(x_ref)
    dt = 0.05
    x1, q, its, rr = P.capsule_step(lam, dt, "shear", 0.5, shear_modulus=0.7, tol=1e-11,
                                    restart=40, maxit=400)
    xr, qr, _ = C.midpoint_step(s, x_ref, lam, 0.7, "shear", 0.5, dt, tol=1e-11)
    moved = np.abs(xr - s.x).max()
    assert moved > 1e-3
    assert np.abs(x1 - xr).max() < 1e-8 * moved
    assert np.array_equal(P.mesh_positions(), x1)
    P.check()


def test_separation_and_volumes(ggem, capsules):
    s, x_ref, lam = capsules
    P = _plan(ggem, s, "fp64")
    h = P.min_separation()
    assert h == pytest.approx(C.min_separation(s.x, s.box), rel=1e-14)
    v = P.particle_volumes()
    vr = C.volumes(s.x, s.tri, s.particle, 2)
    assert np.abs(v - vr).max() < 1e-13 * vr.max()
    v0 = vr * np.array([1.003, 1.0])                     # particle 0 lost 0.3 % of its volume
    passes = P.volume_correct(v0, 1e-4, 10)
    xc = P.mesh_positions()
    xo, k = C.volume_correct(s.x, s.tri, s.particle, v0)
    assert passes == k and passes >= 1
    assert np.abs(xc - xo).max() < 1e-12
    vc = P.particle_volumes()
    assert np.abs(vc / v0 - 1).max() <= 1e-4


def _facing(box, centres_along, level=2):
    """Spheres placed by centres_along(v), v an icosahedron vertex direction
    (facing vertices of neighbours lie on their line of centres)."""
    import math
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([phi, 0.0, 1.0]) / math.hypot(phi, 1.0)
    centres = np.array(centres_along(v))
    return v, W.suspension(len(centres), box, level=level, centres=centres)


@pytest.mark.parametrize("case", ["pair_across_boundary", "chain_of_three"])
def test_overlap_correction(ggem, case):
    box = _box()
    if case == "pair_across_boundary":
        def along(v):
            c0 = np.array([15.5, 0.0, 8.0])
            c1 = c0 + 2.03 * v
            c1[0] -= box.Lx
            return [c0, c1]
    else:
        def along(v):
            c = np.array([8.0, 0.0, 8.0])
            return [c - 2.03 * v, c, c + 2.03 * v]
    _, s = _facing(box, along)
    n_p = len(s.centres)
    P = _plan(ggem, s, "fp64")
    moves = P.overlap_correct(0.05)
    x = P.mesh_positions()
    xo, mo = C.overlap_correct(s.x, s.particle, n_p, box, 0.05)
    assert moves == mo and moves >= 1
    assert np.abs(x - xo).max() < 1e-12
    assert P.overlap_correct(0.05) == 0                    # nothing left to correct


def test_capsule_argument_errors(ggem, capsules):
    s, x_ref, lam = capsules
    P = ggem.Plan.for_box(s.box, precision="fp64", quadrature="element", max_points=len(s.x),
                          max_tris=len(s.tri))
    P.mesh_set(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.tri, device="cuda"))
    with pytest.raises(ggem.GGEMError):             # no membrane reference yet
        P.membrane_traction(1.0)
    with pytest.raises(ggem.GGEMError):
        P.capsule_velocity(lam, "shear", 1.0)
    with pytest.raises(ggem.GGEMError):             # particle ids not set
        P.particle_volumes()
    with pytest.raises(ggem.GGEMError):
        P.overlap_correct(0.05)
    P.membrane_reference(x_ref)
    P.mesh_particles(s.particle, 2)
    with pytest.raises(ggem.GGEMError):             # dt must be positive
        P.capsule_step(lam, 0.0, "shear", 1.0)
    with pytest.raises(ggem.GGEMError):             # the gap must fit a cell
        P.overlap_correct(100.0)
    with pytest.raises(KeyError):                   # unknown flow name (binding)
        P.undisturbed("couette", 1.0)
    bad = ggem.lib().ggem_undisturbed(P.h, 7, 1.0, None, None)
    assert bad == 1                                 # GGEM_ERR_INVALID_ARG for an unknown flow
    # a new triangle set drops the membrane reference
    P.mesh_set(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.tri.copy(), device="cuda"))
    with pytest.raises(ggem.GGEMError):
        P.membrane_traction(1.0)
    P.check()
