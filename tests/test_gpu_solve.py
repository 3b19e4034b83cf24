"""Parity of the CUDA Fredholm solve (bie_solve, Sec. 5) with the oracle.

The oracle solves the same discrete system (I + kappa/(4 pi) D) q = b with
its own GMRES; both stop on the true FP64 residual.  Checks:
  * FP64 plan, tol 1e-12: the solution within 1e-9 of the oracle's, the same
    iteration count to within one, and the oracle's own residual of the GPU
    solution below 5e-11 (operator parity 1e-10);
  * mixed plan, tol 1e-6: the oracle's residual of the GPU solution <= the
    tolerance (plus the 1e-10 FP64 operator parity), the reported residual
    equal to it, and the refinement visible in the work counts;
  * kappa = 0 (operator I), the iteration limit, host arrays, ||b|| = 0;
  * 100 capsules (64,200 nodes), mixed, tol 1e-6: the residual at sampled
    nodes recomputed by the oracle.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OK, NOT_CONVERGED, BREAKDOWN = 0, 5, 6


@pytest.fixture(scope="module")
def ggem():
    from paper_1109_6587_gb300 import _build
    _build.build()
    from paper_1109_6587_gb300 import ggem as G
    return G


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _sphere(level=2):
    V, F = W.icosphere(level)
    box = W.Box(Lx=8.0, Lz=8.0, W=4.0, y0=-2.0, Nx=32, Ny=33, Nz=32)
    c = np.array([4.0, 0.1, 4.0])
    return W.Suspension(box=box, x=0.97 * V + c, tri=F,
                        particle=np.zeros(len(V), np.int32), centres=c[None], radius=0.97)


def _plan(ggem, s, prec, quad):
    P = ggem.Plan.for_box(s.box, precision=prec, quadrature=quad,
                          max_points=s.x.shape[0], max_tris=s.tri.shape[0])
    P.mesh_set(_dev(s.x), torch.as_tensor(s.tri, device="cuda"))
    return P


def _oracle_relres(s, kappa, q, b, quad):
    r = b - O.bie_operator(s, kappa, q, quad)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def case():
    s = _sphere()
    n = s.x.shape[0]
    rng = np.random.default_rng(21)
    kappa = np.where(rng.random(n) < 0.5, 2.0 / 3.0, -2.0 / 3.0)   # lambda = 5 and 0.2
    b = rng.standard_normal((n, 3))
    return s, kappa, b


@pytest.mark.parametrize("quad", ["nodal", "element"])
def test_fp64_solve_matches_oracle(ggem, case, quad):
    s, kappa, b = case
    q_ref, its_ref, rr_ref, ok = O.bie_solve(s, kappa, b, tol=1e-12, quadrature=quad)
    assert ok
    P = _plan(ggem, s, "fp64", quad)
    q, its, rr, st = P.bie_solve(_dev(kappa), _dev(b), tol=1e-12)
    q = q.cpu().numpy()
    assert st in (OK, BREAKDOWN) and rr <= 1e-12
    assert np.abs(q - q_ref).max() < 1e-9 * np.abs(q_ref).max()
    assert abs(its - its_ref) <= 1
    # the GPU operator matches the oracle's to ~1e-10 relative
    assert _oracle_relres(s, kappa, q, b, quad) < 5e-11


@pytest.mark.parametrize("quad", ["nodal", "element"])
def test_mixed_solve_reaches_true_fp64_residual(ggem, case, quad):
    s, kappa, b = case
    P = _plan(ggem, s, "mixed", quad)
    q, its, rr, st = P.bie_solve(_dev(kappa), _dev(b), tol=1e-6)
    q = q.cpu().numpy()
    assert st == OK and rr <= 1e-6
    rr_oracle = _oracle_relres(s, kappa, q, b, quad)
    assert rr_oracle <= 1e-6 + 1e-9
    assert abs(rr_oracle - rr) < 1e-9
    cycles, mv64, mvmix = P.solve_stats()
    # residual of the guess with the mixed operator, one FP64 residual per cycle
    # (one cycle suffices when the mixed operator is accurate enough)
    assert cycles >= 1 and mv64 == cycles and mvmix == its + 1
    # the refined solution agrees with the FP64 solution to about the tolerance
    q_ref, *_ = O.bie_solve(s, kappa, b, tol=1e-12, quadrature=quad)
    assert np.abs(q - q_ref).max() < 1e-5 * np.abs(q_ref).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_identity_operator_and_zero_rhs(ggem, case, prec):
    s, _, b = case
    n = s.x.shape[0]
    P = _plan(ggem, s, prec, "nodal")
    q, its, rr, st = P.bie_solve(_dev(np.zeros(n)), _dev(b), q=_dev(b), tol=1e-10)
    assert st == OK and its == 0 and rr == 0.0
    q, its, rr, st = P.bie_solve(_dev(np.zeros(n)), _dev(b), q=_dev(np.zeros((n, 3))),
                                 tol=1e-10)
    assert st == BREAKDOWN and its == 1 and rr < 1e-14
    assert np.abs(q.cpu().numpy() - b).max() < 1e-14 * np.abs(b).max()
    q, its, rr, st = P.bie_solve(_dev(np.zeros(n)), _dev(np.zeros((n, 3))),
                                 q=_dev(b), tol=1e-10)
    assert st == OK and its == 0 and not q.abs().max().item()


def test_iteration_limit_and_host_arrays(ggem, case):
    s, kappa, b = case
    P = _plan(ggem, s, "fp64", "nodal")
    q0 = np.zeros_like(b)
    q, its, rr, st = P.bie_solve(kappa, b, q=q0, tol=1e-14, restart=3, maxit=4)
    assert st == NOT_CONVERGED and its == 4 and q is q0
    assert abs(_oracle_relres(s, kappa, q, b, "nodal") - rr) < 1e-10
    qd, its_d, rr_d, _ = P.bie_solve(_dev(kappa), _dev(b), q=_dev(np.zeros_like(b)),
                                     tol=1e-14, restart=3, maxit=4)
    assert its_d == its and abs(rr_d - rr) < 1e-15
    assert np.abs(qd.cpu().numpy() - q).max() < 1e-14 * np.abs(q).max()


def test_argument_errors(ggem, case):
    s, kappa, b = case
    P = _plan(ggem, s, "fp64", "nodal")
    for kw in ({"restart": 0}, {"restart": 65}, {"tol": 0.0}, {"maxit": -1},
               {"use_mlp": True}):
        args = dict(tol=1e-6, restart=30, maxit=10)
        args.update(kw)
        with pytest.raises(ggem.GGEMError) as e:
            P.bie_solve(_dev(kappa), _dev(b), **args)
        assert e.value.status == 1


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_non_finite_inputs(ggem, case, prec):
    """Injected faults on the host: a NaN in the right-hand side ends the solve
    with GGEM_ERR_NUMERICAL (non-finite residual), a NaN node coordinate is
    refused by ggem_mesh_set; the plan stays usable after both."""
    s, kappa, b = case
    P = _plan(ggem, s, prec, "nodal")
    bad = b.copy()
    bad[7, 1] = np.nan
    with pytest.raises(ggem.GGEMError) as e:
        P.bie_solve(_dev(kappa), _dev(bad), tol=1e-6)
    assert e.value.status == 4
    x = s.x.copy()
    x[3, 0] = np.nan
    with pytest.raises(ggem.GGEMError) as e:
        P.mesh_set(_dev(x), torch.as_tensor(s.tri, device="cuda"))
    assert e.value.status == 1
    with pytest.raises(ggem.GGEMError):          # the refused mesh leaves none set
        P.single_layer(_dev(b))
    P.mesh_set(_dev(s.x), torch.as_tensor(s.tri, device="cuda"))
    q, its, rr, st = P.bie_solve(_dev(kappa), _dev(b), tol=1e-6)
    assert st == OK and rr <= 1e-6
    P.check()


def test_mixed_solve_100_capsules_sampled_residual(ggem):
    s = W.capsules_100()
    n = s.x.shape[0]
    rng = np.random.default_rng(31)
    kappa = np.full(n, 2.0 / 3.0)
    b = rng.standard_normal((n, 3))
    P = _plan(ggem, s, "mixed", "element")
    q, its, rr, st = P.bie_solve(_dev(kappa), _dev(b), tol=1e-6)
    assert st == OK and rr <= 1e-6 and its < 30
    q = q.cpu().numpy()
    idx = np.sort(rng.choice(n, 200, replace=False))
    Dq = O.double_layer(s, q, quadrature="element", targets=idx)
    r = b[idx] - (q[idx] + kappa[idx, None] / (4.0 * math.pi) * Dq)
    # relres <= 1e-6 in the 2-norm: entries of size ~1e-6 rms(b), FP64 operator
    # parity adds ~1e-10
    assert np.abs(r).max() < 1e-5 * np.sqrt((b ** 2).mean())
