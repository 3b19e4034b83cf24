"""Pins of the oracle's spectral off-grid evaluation (CPU only).

Sec. 3.2.3: on the mesh the global solution converges exponentially with the
number of modes, off the mesh 5-point Lagrange interpolation limits it to
~h^5; summing the expansion itself (what a non-uniform FFT does to its
tolerance) removes that limit.  Facts that fix the oracle's
``spectral_eval``, independent of its own formulas:
  * a field that is a trigonometric polynomial in x, z (no Nyquist mode) times
    a polynomial of degree <= Ny - 1 in y is reproduced exactly anywhere in
    the slit, including outside the periodic cell and on the walls, whatever
    the signs, phases and the ratio Lx / Lz (a transposed axis, a wrong sign
    of a wavenumber or a wrong y map fails this);
  * on the grid nodes the evaluation returns the grid values of a solved
    field (its Nyquist modes are zero);
  * the total GGEM velocity no longer depends on alpha beyond the truncation
    of rho_g (Eq. (tot_l_g)): with Lagrange interpolation the split shows at
    1e-4, with the spectral evaluation it drops below 1e-6 on the same grid;
  * no slip at off-grid wall points converges faster than h^5.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W


def _refined(box, n):
    return dataclasses.replace(box, Nx=n, Nz=n, Ny=n + 1)


def _analytic_field(box):
    # (l, m, n, phase_x, phase_z, amplitude): l, m below the Nyquist index,
    # n up to the top Chebyshev degree
    terms = [(3, 2, 5, 0.3, 1.1, 0.7), (-7, 4, 11, -1.2, 0.2, -0.4),
             (0, -9, 0, 0.5, 0.9, 1.3), (box.Nx // 2 - 1, box.Nz // 2 - 1, box.Ny - 1,
                                         2.0, 0.1, 0.25)]

    def f(x, y, z):
        yb = np.clip(2.0 * (y - box.y0) / box.W - 1.0, -1.0, 1.0)
        v = 0.2 + 0.0 * x
        for l, m, n, p1, p2, a in terms:
            v = v + (a * np.cos(2 * np.pi * l * x / box.Lx + p1)
                     * np.cos(2 * np.pi * m * z / box.Lz + p2) * np.cos(n * np.arccos(yb)))
        return v
    return f


def test_band_limited_field_is_reproduced_exactly():
    box = dataclasses.replace(W.box_single_sphere(), Lx=8.0, Lz=6.0)
    f = _analytic_field(box)
    Y, Z, X = np.meshgrid(O.grid_y(box), O.grid_z(box), O.grid_x(box), indexing="ij")
    field = np.stack([f(X, Y, Z), -2.0 * f(X, Y, Z)])
    rng = np.random.default_rng(1)
    xt = np.stack([rng.uniform(-3, 11, 50), rng.uniform(box.y0, box.y0 + box.W, 50),
                   rng.uniform(-2, 9, 50)], 1)
    xt[0, 1], xt[1, 1] = box.y0, box.y0 + box.W
    v = O.spectral_eval(box, field, xt)
    exact = f(xt[:, 0], xt[:, 1], xt[:, 2])
    assert np.abs(v[:, 0] - exact).max() < 1e-12
    assert np.abs(v[:, 1] + 2.0 * exact).max() < 1e-12
    # the 5-point interpolant is far off on the same field
    assert np.abs(O.interp(box, field, xt)[:, 0] - exact).max() > 1e-2


def test_grid_nodes_return_grid_values():
    box = W.box_single_sphere()
    s = W.suspension(1, box, level=1, centres=np.array([[4.0, -0.5, 3.0]]))
    g = W.normal_forces(s.x.shape[0])
    ug, _, sg = O.global_fields(box, s.x, g, want_stress=True)
    ix, jy, iz = [3, 17, 30], [0, 7, 32], [5, 0, 31]
    xt = np.stack([O.grid_x(box)[ix], O.grid_y(box)[jy], O.grid_z(box)[iz]], 1)
    want = ug[:, jy, iz, ix].T
    assert np.abs(O.spectral_eval(box, ug, xt) - want).max() < 1e-12 * np.abs(ug).max()
    want = sg[:, jy, iz, ix].T
    assert np.abs(O.spectral_eval(box, sg, xt) - want).max() < 1e-12 * np.abs(sg).max()


def test_alpha_invariance_limited_by_truncation_only():
    box = W.box_single_sphere()
    s = W.single_sphere()
    g = W.normal_forces(s.x.shape[0])
    fine = _refined(box, 64)
    d = {}
    for og in ("lagrange", "spectral"):
        u15, _ = O.point_forces(fine, s.x, g, alpha=1.5, offgrid=og)
        u20, _ = O.point_forces(fine, s.x, g, alpha=2.0, offgrid=og)
        ucoarse, _ = O.point_forces(box, s.x, g, offgrid=og)   # alpha dy_m = 0.5
        scale = np.abs(u15).max()
        d[og] = (np.abs(u15 - u20).max() / scale, np.abs(ucoarse - u15).max() / scale)
    assert d["lagrange"][0] > 3e-5                # the interpolation error shows
    assert d["spectral"][0] < 1e-6
    assert d["spectral"][1] < 3e-5 and d["spectral"][1] < d["lagrange"][1] / 100


def test_no_slip_at_off_grid_wall_points_converges_faster():
    box = W.box_single_sphere()
    s = W.suspension(1, box, level=2, centres=np.array([[4.0, -0.5, 4.0]]))
    g = W.normal_forces(s.x.shape[0])
    rng = np.random.default_rng(0)
    px, pz = rng.uniform(0, 8, (2, 40))
    errs = {"lagrange": [], "spectral": []}
    for b in (_refined(box, 48), _refined(box, 64)):
        xt = np.concatenate([np.stack([px, np.full(40, b.y0), pz], 1),
                             np.stack([px, np.full(40, b.y0 + b.W), pz], 1)])
        uref, _ = O.point_forces(b, s.x, g)
        for og in errs:
            u, _ = O.point_forces(b, s.x, g, xt, offgrid=og)
            errs[og].append(np.abs(u).max() / np.abs(uref).max())
    assert errs["spectral"][1] < 5e-6
    assert errs["spectral"][1] < errs["lagrange"][1] / 3
    assert errs["spectral"][0] / errs["spectral"][1] > 5.0


def test_layers_at_sampled_nodes_match_all_nodes():
    s = W.single_sphere(radius=0.97)
    q = W.normal_forces(s.x.shape[0], seed=3)
    tsel = np.array([0, 5, 77, 161])
    for quad in ("nodal", "element"):
        full = O.single_layer(s, q, quad, offgrid="spectral")
        part = O.single_layer(s, q, quad, targets=tsel, offgrid="spectral")
        assert np.abs(full[tsel] - part).max() < 1e-13 * np.abs(full).max()


@pytest.mark.parametrize("mistake", ["sign_kx", "swap_xz", "y_reversed"])
def test_planted_mistakes_fail_the_pin(monkeypatch, mistake):
    """The band-limited pin catches the plausible slips of a spectral sum: a
    wavenumber of the wrong sign, x and z exchanged, the Chebyshev variable
    running the wrong way."""
    box = dataclasses.replace(W.box_single_sphere(), Lx=8.0, Lz=6.0)
    f = _analytic_field(box)
    Y, Z, X = np.meshgrid(O.grid_y(box), O.grid_z(box), O.grid_x(box), indexing="ij")
    field = f(X, Y, Z)[None]
    rng = np.random.default_rng(1)
    xt = np.stack([rng.uniform(-3, 11, 30), rng.uniform(box.y0, box.y0 + box.W, 30),
                   rng.uniform(-2, 9, 30)], 1)
    exact = f(xt[:, 0], xt[:, 1], xt[:, 2])
    good = O.mode_wavenumbers
    if mistake == "sign_kx":
        monkeypatch.setattr(O, "mode_wavenumbers",
                            lambda b: (lambda KX, KZ, nyq: (-KX, KZ, nyq))(*good(b)))
        v = O.spectral_eval(box, field, xt)[:, 0]
    elif mistake == "swap_xz":
        v = O.spectral_eval(box, field, xt[:, [2, 1, 0]])[:, 0]
    else:
        ymir = 2 * box.y0 + box.W - xt[:, 1]
        v = O.spectral_eval(box, field, np.stack([xt[:, 0], ymir, xt[:, 2]], 1))[:, 0]
    assert np.abs(v - exact).max() > 1e-3


def test_convergence_study_of_section_3_2_3():
    """The point-force test of Sec. 3.2.3 (Fig. ggem_conv): a cube slit of side
    L = 1, force (1, 1, 1) at (0.25, 0.25, 0.25), alpha = 80/3 fixed, targets
    at the box centre (a mesh point) and at (0.4312, 0.3734, 0.5234) (not one),
    errors against a fine solution (r_cut = 13/alpha, grid 128 x 129 x 128).
    As the paper reports: on the mesh point the error falls exponentially with
    1/(alpha dy_m) and, for r_cut = 4/alpha, levels off near 1e-6 while a
    larger r_cut keeps falling; off the mesh the 5-point interpolation error
    dominates at the finer mesh, and the spectral evaluation removes it."""
    alpha = 80.0 / 3.0
    xs, g = np.array([[0.25, 0.25, 0.25]]), np.array([[1.0, 1.0, 1.0]])
    xt = np.array([[0.5, 0.5, 0.5], [0.4312, 0.3734, 0.5234]])

    def ux(n, c, og):
        b = W.Box(Lx=1.0, Lz=1.0, W=1.0, y0=0.0, Nx=n, Ny=n + 1, Nz=n)
        return O.point_forces(b, xs, g, xt, alpha=alpha, rcut=c / alpha, offgrid=og)[0][:, 0]

    ref = ux(128, 13.0, "spectral")

    def err(n, c, og):
        return np.abs(ux(n, c, og) - ref) / np.abs(ref)
    e32, e64_4, e64_6 = err(32, 4.0, "spectral"), err(64, 4.0, "spectral"), err(64, 6.0, "spectral")
    # mesh point: 1/(alpha dy_m) 1.2 -> 2.4 gains > 100x (exponential convergence)
    assert e32[0] > 100 * e64_6[0]
    # r_cut = 4/alpha levels off at O(1e-6) (truncation of the local part)
    assert 1e-7 < e64_4[0] < 3e-5 and e64_4[0] > 100 * e64_6[0]
    # off the mesh: interpolation dominates Lagrange, not the spectral evaluation
    lag = err(64, 6.0, "lagrange")
    assert lag[1] > 1e-6 and lag[1] > 100 * e64_6[1]
