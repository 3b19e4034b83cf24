"""Pins of the oracle's global (Fourier x Chebyshev) Stokes solver (CPU only).

  * Chebyshev transform / derivative against numpy.polynomial.chebyshev;
  * a manufactured divergence-free 3-D solution (sympy) whose y-dependence is
    polynomial of degree <= N: the Chebyshev-tau Kleiser-Schumann solve of
    App. C is then exact, so velocity, pressure and stress must agree to
    round-off -- this fixes signs (the Eq. press_helm garble), the i k_x / i k_z
    convention, the FFT normalisation and the stress assembly;
  * a non-polynomial single-mode solution: error falls spectrally with N_y;
  * App. B: the k = 0 mode reproduces the printed Poiseuille profile;
  * the 5-point Lagrange interpolation is exact for degree-4 polynomials.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1109_6587_gb300.workloads import Box

sp = pytest.importorskip("sympy")


def test_chebyshev_transform_matches_numpy():
    Ny = 17
    rng = np.random.default_rng(0)
    a = rng.normal(size=Ny)
    yb = np.cos(np.pi * np.arange(Ny) / (Ny - 1))
    f = np.polynomial.chebyshev.chebval(yb, a)
    np.testing.assert_allclose(O.cheb_forward(Ny) @ f, a, atol=1e-13)
    np.testing.assert_allclose(O.cheb_inverse(Ny) @ a, f, atol=1e-13)
    d = np.polynomial.chebyshev.chebder(a)
    np.testing.assert_allclose((O.cheb_deriv(Ny) @ a)[:-1], d, atol=1e-11)
    bot, top = O.cheb_at_walls(Ny)
    assert abs(bot @ a - np.polynomial.chebyshev.chebval(-1.0, a)) < 1e-13
    assert abs(top @ a - np.polynomial.chebyshev.chebval(1.0, a)) < 1e-13


def _manufactured(box, mu):
    """Divergence-free u = curl(psi), pressure p, forcing f = -grad p + mu lap u."""
    x, y, z = sp.symbols("x y z", real=True)
    kx = 2 * sp.pi / box.Lx
    kz = 2 * sp.pi * 2 / box.Lz
    A = 0.3 * y ** 3 - 0.2 * y ** 2 + 0.5 * y + 0.1
    B = 0.2 * y ** 4 - 0.1 * y + 0.4
    C = -0.15 * y ** 5 + 0.25 * y ** 2 - 0.3
    psi = [A * sp.sin(kz * z + 0.2), B * sp.cos(kx * x + kz * z), C * sp.cos(kx * x)]
    u = [sp.diff(psi[2], y) - sp.diff(psi[1], z),
         sp.diff(psi[0], z) - sp.diff(psi[2], x),
         sp.diff(psi[1], x) - sp.diff(psi[0], y)]
    u[0] = u[0] + 0.4 * y ** 2 - 0.2 * y + 0.1           # k = 0 parts (v_00 = 0)
    u[2] = u[2] - 0.3 * y ** 3 + 0.2
    yc = box.y0 + box.W / 2
    P0 = 0.7 * ((y - yc) ** 2 - (box.W ** 2) / 12)       # zero mean over the slit
    p = 0.5 * y ** 2 * sp.cos(kx * x) + (0.2 * y - 0.3) * sp.sin(kz * z) + P0
    X = (x, y, z)
    f = [-sp.diff(p, X[i]) + mu * sum(sp.diff(u[i], X[k], 2) for k in range(3))
         for i in range(3)]
    sig = {}
    for c, (i, j) in enumerate(O._SYM6):
        sig[c] = (-p if i == j else 0) + mu * (sp.diff(u[i], X[j]) + sp.diff(u[j], X[i]))
    div = sp.simplify(sum(sp.diff(u[i], X[i]) for i in range(3)))
    assert div == 0
    lam = lambda e: sp.lambdify((x, y, z), e, "numpy")
    return [lam(e) for e in u], lam(p), [lam(e) for e in f], [lam(sig[c]) for c in range(6)]


def _on_grid(fun, box, y=None):
    X, Y, Z = np.meshgrid(O.grid_x(box), O.grid_y(box) if y is None else np.array([y]),
                          O.grid_z(box), indexing="xy")
    # meshgrid(x, y, z, 'xy') -> [Ny, Nx, Nz]; reorder to [Ny, Nz, Nx]
    v = fun(X, Y, Z) * np.ones_like(X)
    return np.transpose(v, (0, 2, 1))


@pytest.mark.parametrize("mu", [1.0, 0.7])
def test_global_solve_exact_for_polynomial_manufactured_solution(mu):
    box = Box(Lx=6.0, Lz=5.0, W=2.0, y0=-1.0, Nx=16, Ny=17, Nz=16)
    u, p, f, sig = _manufactured(box, mu)
    F = np.stack([_on_grid(fi, box) for fi in f])
    gb = np.stack([_on_grid(ui, box, y=box.y0)[0] for ui in u])
    gt = np.stack([_on_grid(ui, box, y=box.y0 + box.W)[0] for ui in u])
    ug, pg, sg = O.global_solve(box, F, gb, gt, mu, want_stress=True)
    U = np.stack([_on_grid(ui, box) for ui in u])
    S = np.stack([_on_grid(si, box) for si in sig])
    P = _on_grid(p, box)
    assert np.abs(ug - U).max() / np.abs(U).max() < 1e-11
    assert np.abs(pg - P).max() / np.abs(P).max() < 1e-11
    assert np.abs(sg - S).max() / np.abs(S).max() < 1e-11


def test_single_mode_spectral_convergence():
    """Smooth non-polynomial mode: error falls spectrally with Ny."""
    Lx, Lz, W, mu = 6.0, 5.0, 2.0, 1.0
    kx, kz = 2 * np.pi / Lx, 2 * np.pi * 3 / Lz
    k2 = kx * kx + kz * kz
    y = sp.symbols("y", real=True)
    V = sp.sin(2 * y + 0.3) * sp.exp(0.2 * y)
    Pp = sp.cos(1.5 * y) + 0.3 * y
    ikx, ikz = sp.I * kx, sp.I * kz
    Uh = ikx / k2 * sp.diff(V, y)
    Wh = ikz / k2 * sp.diff(V, y)
    lapl = lambda e: sp.diff(e, y, 2) - k2 * e
    Fx = -ikx * Pp + mu * lapl(Uh)
    Fy = -sp.diff(Pp, y) + mu * lapl(V)
    Fz = -ikz * Pp + mu * lapl(Wh)
    errs = []
    for Ny in (7, 9, 11, 21):
        box = Box(Lx=Lx, Lz=Lz, W=W, y0=-1.0, Nx=8, Ny=Ny, Nz=8)
        yj = O.grid_y(box)
        ev = lambda e: np.array([complex(e.subs(y, v)) for v in yj])
        Cf = O.cheb_forward(Ny)
        Fh = np.stack([Cf @ ev(Fx), Cf @ ev(Fy), Cf @ ev(Fz)])[None]
        gb = np.array([[complex(e.subs(y, -1.0)) for e in (Uh, V, Wh)]])
        gt = np.array([[complex(e.subs(y, 1.0)) for e in (Uh, V, Wh)]])
        uc, vc, wc, pc = O.ks_solve(box, Fh, gb, gt, mu, np.array([kx]), np.array([kz]))
        Ci = O.cheb_inverse(Ny)
        e = max(np.abs(Ci @ uc[0] - ev(Uh)).max(), np.abs(Ci @ vc[0] - ev(V)).max(),
                np.abs(Ci @ pc[0] - ev(Pp)).max())
        errs.append(e)
    print(errs)
    assert errs[-1] < 1e-10
    assert errs[0] > 10 * errs[1] > 100 * errs[2]   # geometric (spectral) decay


def test_k0_mode_is_poiseuille_of_appendix_b():
    """Body force f_x = -8 mu U0/H^2 gives u = 4 U0 (y/H)(1 - y/H) (App. B)."""
    H, U0, mu = 3.0, 1.7, 0.8
    box = Box(Lx=4.0, Lz=4.0, W=H, y0=0.0, Nx=8, Ny=17, Nz=8)
    F = np.zeros((3, box.Ny, box.Nz, box.Nx))
    F[0] = -8 * mu * U0 / H ** 2
    zero = np.zeros((3, box.Nz, box.Nx))
    ug, pg, _ = O.global_solve(box, F, zero, zero, mu)
    yj = O.grid_y(box)
    expect = 4 * U0 * (yj / H) * (1 - yj / H)
    assert np.abs(ug[0] - expect[:, None, None]).max() < 1e-12
    assert np.abs(ug[1]).max() < 1e-12 and np.abs(ug[2]).max() < 1e-12
    # plane Couette: top wall moving, no forcing -> linear profile
    gt = zero.copy(); gt[0] = U0
    ug, _, _ = O.global_solve(box, 0 * F, zero, gt, mu)
    assert np.abs(ug[0] - (U0 * yj / H)[:, None, None]).max() < 1e-12


def test_interpolation_exact_for_quartics():
    box = Box(Lx=6.0, Lz=5.0, W=2.0, y0=-1.0, Nx=24, Ny=17, Nz=20)
    rng = np.random.default_rng(3)
    cx, cy, cz = rng.normal(size=(3, 5))
    poly = lambda X, Y, Z: (np.polyval(cx, X) * np.polyval(cy, Y) * np.polyval(cz, Z))
    F = _on_grid(poly, box)[None]
    n = 50
    dx, dz = box.Lx / box.Nx, box.Lz / box.Nz
    xt = np.stack([rng.uniform(3 * dx, box.Lx - 4 * dx, n),
                   rng.uniform(box.y0, box.y0 + box.W, n),
                   rng.uniform(3 * dz, box.Lz - 4 * dz, n)], axis=1)
    got = O.interp(box, F, xt)[:, 0]
    ref = poly(xt[:, 0], xt[:, 1], xt[:, 2])
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-11
