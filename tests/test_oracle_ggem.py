"""Pins of the oracle's whole GGEM point-force evaluation (CPU only).

Facts fixed by the physics, independent of the oracle's own formulas:
  * plane average: averaging the slit Green's function over a periodic x-z
    plane gives the exact piecewise-linear profile of a force sheet between
    no-slip walls, mu u'' = -g delta(y - y_s)/(Lx Lz); where the local part
    vanishes (|y - y_s| >= r_cut) the GGEM field must match it to the level of
    the rho_g truncation (7.6e-6, Eq. rho_l_g with r_cut = 4/alpha);
  * no slip at the walls (Sec. 3.2.2) at off-grid wall points, converging as
    the grid is refined;
  * alpha-invariance: the split of Eq. (rho_l_g) must not change the total
    (Eq. tot_l_g); differences shrink with the mesh like the interpolation
    error (Sec. 3.2.3, error ~ (alpha dy_m)^5 off the mesh);
  * reciprocity G_ij(x, y) = G_ji(y, x) (self-adjointness, Sec. 3.1).
"""
import dataclasses

import numpy as np

from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W


def _refined(box, n):
    return dataclasses.replace(box, Nx=n, Nz=n, Ny=n + 1)


def test_plane_average_is_force_sheet_profile():
    box = W.box_single_sphere()
    xs = np.array([[3.1, -0.7, 4.3]])
    g = np.array([[0.8, -0.5, 1.3]])
    for b in (box, _refined(box, 48)):
        rc = O.default_rcut(O.default_alpha(b))
        ug, _, _ = O.global_fields(b, xs, g)
        yj = O.grid_y(b)
        far = np.abs(yj - xs[0, 1]) >= rc
        assert far.sum() >= 5
        ubar = ug.mean(axis=(2, 3))
        ys, yy = xs[0, 1] - b.y0, yj - b.y0
        prof = np.where(yy < ys, yy * (b.W - ys) / b.W, ys * (b.W - yy) / b.W)
        exact = np.stack([g[0, 0] * prof, 0 * prof, g[0, 2] * prof]) / (b.Lx * b.Lz)
        err = np.abs(ubar[:, far] - exact[:, far]).max() / np.abs(exact).max()
        assert err < 2e-5


def test_no_slip_at_off_grid_wall_points_converges():
    box = W.box_single_sphere()
    s = W.suspension(1, box, level=2, centres=np.array([[4.0, -0.5, 4.0]]))
    g = W.normal_forces(s.x.shape[0])
    rng = np.random.default_rng(0)
    px, pz = rng.uniform(0, 8, (2, 40))
    errs = []
    for b in (box, _refined(box, 48)):
        xt = np.concatenate([np.stack([px, np.full(40, b.y0), pz], 1),
                             np.stack([px, np.full(40, b.y0 + b.W), pz], 1)])
        u, _ = O.point_forces(b, s.x, g, xt)
        uref, _ = O.point_forces(b, s.x, g)
        errs.append(np.abs(u).max() / np.abs(uref).max())
    assert errs[0] < 1.5e-3
    assert errs[1] < 3e-4 and errs[1] < errs[0] / 3


def test_alpha_invariance():
    box = W.box_single_sphere()
    s = W.single_sphere()
    g = W.normal_forces(s.x.shape[0])
    fine = _refined(box, 64)
    u15, _ = O.point_forces(fine, s.x, g, alpha=1.5)
    u20, _ = O.point_forces(fine, s.x, g, alpha=2.0)
    ucoarse, _ = O.point_forces(box, s.x, g)          # alpha dy_m = 0.5 (recommended)
    scale = np.abs(u15).max()
    assert np.abs(u15 - u20).max() / scale < 3e-4
    assert np.abs(ucoarse - u15).max() / scale < 1e-2


def test_reciprocity():
    box = W.box_single_sphere()
    xa, xb = np.array([[2.0, 0.3, 5.0]]), np.array([[3.1, -1.2, 4.4]])
    errs = []
    for b in (box, _refined(box, 48)):
        M1, M2 = np.zeros((3, 3)), np.zeros((3, 3))
        for j in range(3):
            e = np.zeros((1, 3)); e[0, j] = 1.0
            M1[:, j] = O.point_forces(b, xb, e, xa)[0][0]
            M2[:, j] = O.point_forces(b, xa, e, xb)[0][0]
        errs.append(np.abs(M1 - M2.T).max() / np.abs(M1).max())
    assert errs[0] < 5e-4 and errs[1] < 5e-5


def test_wide_slit_matches_periodic_oseen_lattice_sum():
    """With the walls far away (H = 20, sources and targets within 2.5 of the
    mid-plane) the slit solution is the free-space x-z periodic one.  For a
    force quadrupole -- g at c +- d e_x, -g at c +- d e_z: zero net force and
    zero first moment, so every image decays like 1/r^3 -- that is the
    absolutely convergent lattice sum of Oseen tensors, summed here directly
    over (2R + 1)^2 images.  The spectral off-grid evaluation reproduces it to
    the walls' and the grid's level (2e-6 measured); 5-point interpolation is
    limited by its own error (2e-3 measured)."""
    box = W.Box(Lx=8.0, Lz=8.0, W=40.0, y0=-20.0, Nx=32, Ny=161, Nz=32)
    c, d = np.array([4.0, 0.0, 4.0]), 0.5
    g0 = np.array([0.3, -0.8, 0.5])
    xs = np.array([c + [d, 0, 0], c - [d, 0, 0], c + [0, 0, d], c - [0, 0, d]])
    g = np.array([g0, g0, -g0, -g0])
    xt = np.array([[4.3, 1.2, 5.1], [2.5, -0.7, 3.0], [6.0, 0.4, 1.5], [4.0, 2.5, 4.0],
                   [0.5, -1.5, 7.5]])
    R = 60
    p = np.arange(-R, R + 1)
    P, Q = [a.ravel() for a in np.meshgrid(p, p, indexing="ij")]
    shifts = np.stack([P * box.Lx, 0.0 * P, Q * box.Lz], 1)
    ref = np.zeros((len(xt), 3))
    for xi, gi in zip(xs, g):
        for k, x in enumerate(xt):
            r = x - xi - shifts
            rn = np.linalg.norm(r, axis=1)
            ref[k] += (gi / rn[:, None] + r * ((r @ gi) / rn ** 3)[:, None]).sum(0)
    ref /= 8.0 * np.pi
    scale = np.abs(ref).max()
    # alpha 1.2 (width 0.8): the Gaussian resolved by the Chebyshev nodes at
    # the mid-plane, where their spacing is pi/2 times the mean
    u, _ = O.point_forces(box, xs, g, xt, alpha=1.2, offgrid="spectral")
    assert np.abs(u - ref).max() / scale < 1e-5
    u, _ = O.point_forces(box, xs, g, xt, alpha=1.2)
    assert np.abs(u - ref).max() / scale < 5e-3
