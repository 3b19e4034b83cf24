"""Spectral off-grid evaluation on the GPU (ggem_set_offgrid, Sec. 3.2.3)
against the oracle's expansion summed at each point.

The GPU evaluates the expansion by a Gaussian-window non-uniform FFT (2x
oversampling) in x, z and theta = arccos of the normalised y (where the
Chebyshev series is a cosine series), so it differs from the oracle's direct
sum by the window's tolerance (~1e-13 at the FP64 default half-width 12,
~2e-7 at the mixed default 6) on top of the usual parity.  Bars as everywhere: 1e-10 for FP64 and FP64-emulated plans, 1e-5 for
mixed, max |gpu - oracle| / max |oracle|.
"""
import math

import numpy as np
import pytest
from _parity import assert_close

from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp64_emulated": 1e-10, "mixed": 1e-5}


@pytest.fixture(scope="module")
def ggem():
    from paper_1109_6587_gb300 import _build
    _build.build()
    from paper_1109_6587_gb300 import ggem as G
    return G


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
    return np.abs(a - b).max() / np.abs(b).max()


def _sym6(s33):
    return np.stack([s33[:, i, j] for (i, j) in O._SYM6], axis=1)


def _targets(box, nt=97, seed=5):
    rng = np.random.default_rng(seed)
    xt = np.stack([rng.uniform(-3, 11, nt), rng.uniform(box.y0, box.y0 + box.W, nt),
                   rng.uniform(-3, 11, nt)], 1)
    xt[:10, 1] = box.y0                          # on the walls
    xt[10:20, 1] = box.y0 + box.W
    # exactly on grid nodes (x, z on the Fourier nodes, y on a Chebyshev node)
    xt[20:24] = np.stack([O.grid_x(box)[[0, 5, 17, 31]], O.grid_y(box)[[3, 0, 16, 32]],
                          O.grid_z(box)[[9, 31, 0, 2]]], 1)
    return xt


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_point_forces_free_targets(ggem, prec):
    s = W.single_sphere(radius=0.97)
    g = W.normal_forces(s.x.shape[0], seed=2)
    xt = _targets(s.box)
    u_ref, s_ref = O.point_forces(s.box, s.x, g, xt, want_sig=True, offgrid="spectral")
    P = ggem.Plan.for_box(s.box, precision=prec, max_points=1000, offgrid="spectral")
    u, sig = P.point_forces(_dev(s.x), _dev(g), _dev(xt), want_sigma=True)
    torch.cuda.synchronize()
    assert_close(u, u_ref, TOL[prec])
    assert_close(sig, _sym6(s_ref), TOL[prec])
    P.check()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_point_forces_self_targets(ggem, prec):
    s = W.single_sphere(radius=0.97)
    g = W.normal_forces(s.x.shape[0], seed=1)
    u_ref, s_ref = O.point_forces(s.box, s.x, g, want_sig=True, offgrid="spectral")
    P = ggem.Plan.for_box(s.box, precision=prec, max_points=1000, offgrid="spectral")
    u, sig = P.point_forces(_dev(s.x), _dev(g), want_sigma=True)
    torch.cuda.synchronize()
    assert_close(u, u_ref, TOL[prec])
    assert_close(sig, _sym6(s_ref), TOL[prec])


@pytest.mark.parametrize("prec,quad", [("fp64", "nodal"), ("fp64", "element"),
                                       ("fp64_emulated", "element"), ("mixed", "nodal"),
                                       ("mixed", "element")])
def test_layers_single_capsule(ggem, prec, quad):
    s = W.single_sphere(radius=0.97)
    q = W.normal_forces(s.x.shape[0], seed=4)
    w_ref = O.single_layer(s, q, quad, offgrid="spectral")
    v_ref = O.double_layer(s, q, quad, offgrid="spectral")
    P = ggem.Plan.for_box(s.box, precision=prec, quadrature=quad, max_points=s.x.shape[0],
                          max_tris=s.tri.shape[0], offgrid="spectral")
    P.mesh_set(_dev(s.x), torch.as_tensor(s.tri, device="cuda"))
    assert_close(P.single_layer(_dev(q)), w_ref, TOL[prec])
    assert_close(P.double_layer(_dev(q)), v_ref, TOL[prec])
    P.check()


def test_window_width_converges(ggem):
    """The window error falls as the half-width grows (Greengard & Lee)."""
    s = W.single_sphere(radius=0.97)
    g = W.normal_forces(s.x.shape[0], seed=6)
    xt = _targets(s.box, seed=8)
    u_ref, _ = O.point_forces(s.box, s.x, g, xt, offgrid="spectral")
    P = ggem.Plan.for_box(s.box, precision="fp64", max_points=1000)
    errs = []
    for w in (4, 6, 8, 12):
        P.set_offgrid("spectral", w)
        u, _ = P.point_forces(_dev(s.x), _dev(g), _dev(xt))
        errs.append(_rel(u, u_ref))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[0] < 1e-3 and errs[3] < 1e-10


def test_switching_modes(ggem):
    """Lagrange results do not change after a spectral evaluation on the same
    plan (to the rounding of the order in which the spreading's reductions
    land); the two evaluations differ by the interpolation error."""
    s = W.single_sphere(radius=0.97)
    q = W.normal_forces(s.x.shape[0], seed=9)
    P = ggem.Plan.for_box(s.box, precision="fp64", quadrature="element",
                          max_points=s.x.shape[0], max_tris=s.tri.shape[0])
    P.mesh_set(_dev(s.x), torch.as_tensor(s.tri, device="cuda"))
    a = P.double_layer(_dev(q)).cpu().numpy()
    P.set_offgrid("spectral")
    b = P.double_layer(_dev(q)).cpu().numpy()
    P.set_offgrid("lagrange")
    c = P.double_layer(_dev(q)).cpu().numpy()
    assert np.abs(a - c).max() < 1e-13 * np.abs(a).max()
    assert np.abs(a - b).max() > 1e-8 * np.abs(a).max()


def test_argument_errors(ggem):
    s = W.single_sphere()
    P = ggem.Plan.for_box(s.box, precision="mixed", max_points=1000)
    for w in (1, 17, -1):
        with pytest.raises(ggem.GGEMError):
            P.set_offgrid("spectral", w)
    assert ggem.lib().ggem_set_offgrid(P.h, 2, 0) == 1      # unknown mode
    assert ggem.lib().ggem_set_offgrid(None, 1, 0) == 1     # no plan
    with pytest.raises(KeyError):
        P.set_offgrid("cubic")
    P.check()


def test_mixed_solve_with_spectral_offgrid(ggem):
    """The refinement's FP64 twin follows the setting, so the mixed solve
    converges on the spectral operator: the oracle's residual of the GPU
    solution with that operator is within the tolerance."""
    V, F = W.icosphere(2)
    box = W.Box(Lx=8.0, Lz=8.0, W=4.0, y0=-2.0, Nx=32, Ny=33, Nz=32)
    c = np.array([4.0, 0.1, 4.0])
    s = W.Suspension(box=box, x=0.97 * V + c, tri=F, particle=np.zeros(len(V), np.int32),
                     centres=c[None], radius=0.97)
    n = s.x.shape[0]
    rng = np.random.default_rng(21)
    kappa = np.where(rng.random(n) < 0.5, 2.0 / 3.0, -2.0 / 3.0)
    b = rng.standard_normal((n, 3))
    P = ggem.Plan.for_box(box, precision="mixed", quadrature="element", max_points=n,
                          max_tris=F.shape[0], offgrid="spectral")
    P.mesh_set(_dev(s.x), torch.as_tensor(s.tri, device="cuda"))
    q, its, rr, st = P.bie_solve(_dev(kappa), _dev(b), tol=1e-6)
    assert rr <= 1e-6
    q = q.cpu().numpy()
    r = b - (q + kappa[:, None] / (4.0 * math.pi)
             * O.double_layer(s, q, "element", offgrid="spectral"))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-6 + 1e-9


@pytest.fixture(scope="module")
def capsules100():
    s = W.capsules_100()
    q = W.normal_forces(s.x.shape[0], seed=12)
    rng = np.random.default_rng(13)
    idx = np.sort(rng.choice(s.x.shape[0], 200, replace=False))
    w_ref = O.single_layer(s, q, "element", targets=idx, offgrid="spectral")
    v_ref = O.double_layer(s, q, "element", targets=idx, offgrid="spectral")
    return s, q, idx, w_ref, v_ref


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_100_capsules_sampled(ggem, capsules100, prec):
    """The bench's workload (64,200 nodes, 128 x 65 x 128 grid): element-rule
    layers at every node on the GPU, the oracle at 200 sampled nodes."""
    s, q, idx, w_ref, v_ref = capsules100
    P = ggem.Plan.for_box(s.box, precision=prec, quadrature="element",
                          max_points=s.x.shape[0], max_tris=s.tri.shape[0], offgrid="spectral")
    P.mesh_set(_dev(s.x), torch.as_tensor(s.tri, device="cuda"))
    qd = _dev(q)
    assert_close(P.single_layer(qd).cpu().numpy()[idx], w_ref, TOL[prec])
    assert_close(P.double_layer(qd).cpu().numpy()[idx], v_ref, TOL[prec])
    P.check()
