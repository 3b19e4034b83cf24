"""Pins of the oracle's rigid-particle solve (Sec. 6.1, Eq. (sl_r) with force
and torque balance), CPU only.  One sphere of radius a = 1 (162 nodes) at the
mid-plane of a slit of gap W = 10 (lambda = a / (W/2) = 0.2), box 16 x 16.

  * rigid-body modes: in a uniform flow the particle moves with it, in a
    rigid rotation it turns with it, and the tractions vanish (exact
    solutions of the discrete system);
  * torque about the wall normal: Omega = T / (8 pi mu a^3) (Stokes); the
    walls change it only at O(lambda^3) (~0.2 %) and periodic images of a
    torque about the normal decay exponentially in a slit, so 1.5 % covers
    the surface discretisation;
  * sedimentation parallel to the walls: U = F / (6 pi mu a) + u_reg(c), the
    first reflection, u_reg being the regular part of the periodic slit
    Green's function at the centre (the point-force velocity at its own
    position without the free-space self term); the next corrections are
    O(lambda^3) of the wall part (Faxen: 0.418 lambda^3 ~ 0.3 %), 1 % bound.
    u_reg includes the mean flow that a net force drives through a periodic
    slit, which is 18 % of the Stokes velocity here;
  * the returned tractions balance the external load: sum A_b f_b = -F,
    sum A_b (x_b - c) x f_b = -T, and mirror symmetry about the mid-plane
    leaves the other velocity components zero.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W


@pytest.fixture(scope="module")
def sphere():
    box = W.Box(Lx=16.0, Lz=16.0, W=10.0, y0=-5.0, Nx=32, Ny=33, Nz=32)
    return W.suspension(1, box, level=2, centres=np.array([[8.0, 0.0, 8.0]]))


def _balance(s, f):
    _, _, Ab, _ = O.geometry(s.x, s.tri)
    r = s.x - s.centres[0]
    return (Ab[:, None] * f).sum(0), (Ab[:, None] * np.cross(r, f)).sum(0)


def test_uniform_flow_is_followed(sphere):
    s = sphere
    e = np.array([0.3, -0.2, 0.5])
    f, uo, its, rr, ok = O.rigid_solve(s, s.centres, np.tile(e, (len(s.x), 1)), tol=1e-8)
    assert ok and rr <= 1e-8
    assert np.abs(uo[0, :3] - e).max() < 1e-6
    assert np.abs(uo[0, 3:]).max() < 1e-6
    assert np.abs(f).max() < 1e-5


def test_rigid_rotation_is_followed(sphere):
    s = sphere
    om = np.array([0.1, 0.4, -0.3])
    f, uo, its, rr, ok = O.rigid_solve(s, s.centres, np.cross(om, s.x - s.centres[0]),
                                       tol=1e-8)
    assert ok
    assert np.abs(uo[0, 3:] - om).max() < 1e-6
    assert np.abs(uo[0, :3]).max() < 1e-6
    assert np.abs(f).max() < 1e-5


def test_torque_about_wall_normal(sphere):
    s = sphere
    T = 1.0
    ext = np.array([[0.0, 0.0, 0.0, 0.0, T, 0.0]])
    f, uo, its, rr, ok = O.rigid_solve(s, s.centres, np.zeros_like(s.x), ext=ext, tol=1e-8)
    assert ok
    ratio = uo[0, 4] * 8.0 * math.pi / T
    assert abs(ratio - 1.0) < 0.015, ratio
    assert np.abs(uo[0, [0, 1, 2, 3, 5]]).max() < 1e-6 * abs(uo[0, 4])
    F, Tq = _balance(s, f)
    assert np.abs(F).max() < 1e-6 and np.abs(Tq + ext[0, 3:]).max() < 1e-6


def test_sedimentation_parallel_to_walls(sphere):
    s = sphere
    Fx = 1.0
    ext = np.array([[Fx, 0.0, 0.0, 0.0, 0.0, 0.0]])
    f, uo, its, rr, ok = O.rigid_solve(s, s.centres, np.zeros_like(s.x), ext=ext, tol=1e-8)
    assert ok
    ureg, _ = O.point_forces(s.box, s.centres, np.array([[Fx, 0.0, 0.0]]))
    u_pred = Fx / (6.0 * math.pi) + ureg[0, 0]
    assert ureg[0, 0] < -0.1 * Fx / (6.0 * math.pi)     # the slit slows it markedly
    assert abs(uo[0, 0] / u_pred - 1.0) < 0.01, (uo[0, 0], u_pred)
    assert np.abs(uo[0, 1:]).max() < 1e-6 * uo[0, 0]
    F, Tq = _balance(s, f)
    assert np.abs(F + ext[0, :3]).max() < 1e-6 and np.abs(Tq).max() < 1e-6
