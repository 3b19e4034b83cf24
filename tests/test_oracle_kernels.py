"""Pins of the oracle's local kernels and quadrature (CPU only).

Each test checks the oracle against a fact the paper or the mathematics fixes,
not against a retyped formula:
  * T^l is the stress of (G^l, P^l):  T = -P delta + dG + dG^T  (Eq. u_g, with
    mu = 1) -- finite differences;
  * G^l is divergence free and solves the local Stokes problem of Eq.
    (stokes_l): -grad P^l + lap G^l = 8 pi rho_g delta away from the pole;
  * rho_g has unit mass (Eq. rho_l_g: rho_g + rho_l = delta);
  * G^l -> Oseen and T^l -> -6 xxx/r^5 as alpha -> 0 (textbook free-space
    Stokeslet/stresslet), and Oseen - G^l -> (4 alpha/sqrt(pi)) delta as r -> 0;
  * the Gauss-Legendre rule matches numpy's and integrates degree 7 exactly.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W

HERE = os.path.dirname(__file__)


def _pts(n, alpha, seed=1, rmin=0.3, rmax=3.0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 3))
    X *= (rng.uniform(rmin, rmax, size=n) / alpha / np.linalg.norm(X, axis=1))[:, None]
    return X


def _grad(fun, X, h=1e-5):
    """Central-difference gradient of fun(X) -> [n, ...]; result [..., 3]."""
    out = []
    for k in range(3):
        e = np.zeros(3); e[k] = h
        out.append((fun(X + e) - fun(X - e)) / (2 * h))
    return np.stack(out, axis=-1)


@pytest.mark.parametrize("alpha", [0.7, 1.6, 3.0])
def test_stress_kernel_is_stress_of_G_and_P(alpha):
    X = _pts(40, alpha)
    G, P, T = O.kernels(alpha, X)
    dG = _grad(lambda Y: O.kernels(alpha, Y)[0], X, h=1e-5 / alpha)   # [n,i,j,k]
    I = np.eye(3)
    Tfd = (-P[:, None, :, None] * I[None, :, None, :] + dG
           + np.transpose(dG, (0, 3, 2, 1)))
    assert np.abs(Tfd - T).max() / np.abs(T).max() < 1e-7


@pytest.mark.parametrize("alpha", [0.7, 1.6, 3.0])
def test_local_stokeslet_divergence_free(alpha):
    X = _pts(40, alpha, seed=2)
    G, _, _ = O.kernels(alpha, X)
    dG = _grad(lambda Y: O.kernels(alpha, Y)[0], X, h=1e-5 / alpha)
    div = np.einsum("niji->nj", dG)
    assert np.abs(div).max() / np.abs(G).max() < 1e-7


@pytest.mark.parametrize("alpha", [0.9, 2.0])
def test_local_solution_solves_local_stokes_problem(alpha):
    """-dP_j/dx_i + lap G_ij = 8 pi rho_g(r) delta_ij for r > 0."""
    X = _pts(30, alpha, seed=3, rmin=0.4, rmax=2.5)
    h = 2e-4 / alpha
    G0, P0, _ = O.kernels(alpha, X)
    lap = -6.0 * G0
    for k in range(3):
        e = np.zeros(3); e[k] = h
        lap += O.kernels(alpha, X + e)[0] + O.kernels(alpha, X - e)[0]
    lap /= h * h
    dP = _grad(lambda Y: O.kernels(alpha, Y)[1], X, h=1e-5 / alpha)    # [n, j, i]
    lhs = -np.transpose(dP, (0, 2, 1)) + lap
    rho = O.rho_g(alpha, np.linalg.norm(X, axis=1))
    rhs = 8 * math.pi * rho[:, None, None] * np.eye(3)[None]
    scale = np.abs(lap).max()
    assert np.abs(lhs - rhs).max() / scale < 2e-5


@pytest.mark.parametrize("alpha", [0.5, 1.6, 4.0])
def test_rho_g_unit_mass_and_truncation(alpha):
    r = np.linspace(0.0, 12.0 / alpha, 200001)
    f = 4 * math.pi * r * r * O.rho_g(alpha, r)
    mass = np.trapezoid(f, r)
    assert abs(mass - 1.0) < 1e-9
    rc = O.default_rcut(alpha)
    inside = np.trapezoid(np.where(r < rc, f, 0.0), r)
    # mass beyond X = alpha r (integrating Eq. rho_l_g a by parts):
    #   (2/sqrt(pi)) (X - X^3) e^{-X^2} + erfc(X)  = -7.6e-6 at X = 4
    x = 4.0
    tail = 2.0 / math.sqrt(math.pi) * (x - x ** 3) * math.exp(-x * x) + math.erfc(x)
    assert abs(tail + 7.6e-6) < 1e-7
    assert abs((1.0 - inside) - tail) < 1e-9


def test_alpha_to_zero_limits_are_oseen_and_stresslet():
    X = _pts(20, 1.0, seed=4)
    G, _, T = O.kernels(1e-9, X)
    r = np.linalg.norm(X, axis=1)
    oseen = (np.eye(3)[None] / r[:, None, None]
             + X[:, :, None] * X[:, None, :] / r[:, None, None] ** 3)
    stresslet = -6 * np.einsum("ni,nj,nk->nijk", X, X, X) / r[:, None, None, None] ** 5
    assert np.abs(G - oseen).max() / np.abs(oseen).max() < 1e-8
    assert np.abs(T - stresslet).max() / np.abs(stresslet).max() < 1e-8


@pytest.mark.parametrize("alpha", [1.0, 2.5])
def test_self_limit(alpha):
    """Oseen - G^l -> (4 alpha / sqrt(pi)) delta as r -> 0 (regular part)."""
    X = _pts(10, alpha, seed=5, rmin=1e-4, rmax=2e-4)
    G, _, _ = O.kernels(alpha, X)
    r = np.linalg.norm(X, axis=1)
    oseen = (np.eye(3)[None] / r[:, None, None]
             + X[:, :, None] * X[:, None, :] / r[:, None, None] ** 3)
    lim = 4 * alpha / math.sqrt(math.pi) * np.eye(3)
    assert np.abs((oseen - G) - lim).max() / lim.max() < 1e-5


def test_gauss_legendre_rule():
    t, w = O.gauss_legendre01(4)
    x, wn = np.polynomial.legendre.leggauss(4)
    np.testing.assert_allclose(np.sort(t), np.sort((x + 1) / 2), atol=1e-15)
    np.testing.assert_allclose(np.sort(w), np.sort(wn / 2), atol=1e-15)
    for d in range(8):
        assert abs((w * t ** d).sum() - 1.0 / (d + 1)) < 1e-14


def test_icosphere_counts_match_paper():
    with open(os.path.join(HERE, "golden", "paper_constants.json")) as fh:
        pc = json.load(fh)
    v, t = W.icosphere(3)
    assert t.shape[0] == pc["icosphere_1280"]["n_tri"]
    assert v.shape[0] == pc["icosphere_1280"]["n_nodes"]
    deg = np.bincount(t.ravel())
    assert (deg == 5).sum() == 12 and (deg == 6).sum() == v.shape[0] - 12
