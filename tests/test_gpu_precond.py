"""Per-particle block preconditioner of the Fredholm solve (ggem_precond_set)
against the oracle (oracle.reference_block_inverse, particle_block_solve).

The paper's solve (Sec. 5) uses no preconditioner; the oracle's reference
applies the inverse block of one isolated reference capsule, turned to each
particle's orientation, to every particle.  Checks:
  * the block the GPU builds (3 n_ref double-layer evaluations on a small
    cell, FP64 Gauss-Jordan) equals the oracle's inverse of the assembled
    operator of the same capsule on the same cell: 1e-9 in an FP64 plan,
    1e-4 in a mixed one (the operator's 1e-5 parity times the block's
    condition);
  * two turned biconcave capsules, FP64 plan, tol 1e-10: the oracle's
    iteration count of the preconditioned solve to within one, the solution
    within 1e-9 of the oracle's plain solve, and fewer iterations than the
    GPU's own unpreconditioned solve;
  * mixed plan, tol 1e-6: the oracle's residual of the GPU solution <= tol;
  * 100 capsules (64,200 nodes), mixed, tol 1e-6: fewer GMRES iterations with
    the block, the same solution to the tolerance;
  * argument errors: enabling without a block, particles whose node count
    differs from the reference.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA = 2.0 / 3.0


@pytest.fixture(scope="module")
def ggem():
    from paper_1109_6587_gb300 import _build
    _build.build()
    from paper_1109_6587_gb300 import ggem as G
    return G


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _ref_capsule():
    V, F = W.rbc_mesh(level=1)
    return V - V.mean(0), F


def _pair():
    """Two randomly turned biconcave capsules in a small slit."""
    V, F = _ref_capsule()
    # alpha = 2 (grid spacing 0.25), r_cut = 2: alpha L = 16 > 8 for the slit
    # and for the reference cell of 32 x 32 intervals
    box = W.Box(Lx=8.0, Lz=8.0, W=4.0, y0=-2.0, Nx=32, Ny=17, Nz=32)
    rot = W.random_rotations(2, np.random.default_rng(8))
    cs = [np.array([2.2, 0.1, 4.0]), np.array([5.5, -0.3, 4.5])]
    x = np.concatenate([V @ rot[p].T + cs[p] for p in range(2)])
    s = W.Suspension(box=box, x=x, tri=np.concatenate([F, F + len(V)]),
                     particle=np.repeat([0, 1], len(V)).astype(np.int32),
                     centres=np.stack(cs), radius=1.0)
    return s, rot


def _plan(ggem, s, prec):
    P = ggem.Plan.for_box(s.box, precision=prec, quadrature="element",
                          max_points=s.x.shape[0], max_tris=s.tri.shape[0])
    P.mesh_set(_dev(s.x), torch.as_tensor(s.tri, device="cuda"))
    P.mesh_particles(s.particle, len(s.centres))
    return P


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_block_matches_oracle(ggem, prec, tol):
    s, _ = _pair()
    V, F = _ref_capsule()
    P = _plan(ggem, s, prec)
    assert P.precond_set(V, F, KAPPA, 32, 32) == (32, 32)
    B = P.precond_block()
    Bref = O.reference_block_inverse(s.box, V, F, KAPPA, 32, 32)
    assert np.abs(B - Bref).max() < tol * np.abs(Bref).max()
    P.check()


def test_preconditioned_fp64_solve_matches_oracle(ggem):
    s, rot = _pair()
    V, F = _ref_capsule()
    n = s.x.shape[0]
    kappa = np.full(n, KAPPA)
    b = np.random.default_rng(9).standard_normal((n, 3))
    q_ref, its_plain_ref, _, ok = O.bie_solve(s, kappa, b, tol=1e-10)
    assert ok
    Minv = O.reference_block_inverse(s.box, V, F, KAPPA, 32, 32)
    _, its_pc_ref, _, ok = O.particle_block_solve(s, kappa, b, Minv, tol=1e-10, rotations=rot)
    assert ok
    P = _plan(ggem, s, "fp64")
    q0 = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    _, its_plain, rr, st = P.bie_solve(_dev(kappa), _dev(b), q=q0.clone(), tol=1e-10)
    P.precond_set(V, F, KAPPA, 32, 32)
    q, its, rr, st = P.bie_solve(_dev(kappa), _dev(b), q=q0.clone(), tol=1e-10)
    assert st in (0, 6) and rr <= 1e-10
    q = q.cpu().numpy()
    assert np.abs(q - q_ref).max() < 1e-9 * np.abs(q_ref).max()
    assert abs(its - its_pc_ref) <= 1, (its, its_pc_ref)
    assert its < its_plain and its <= its_plain // 2 + 2, (its, its_plain)
    # switched off: the plain solve again
    P.precond_enable(False)
    _, its_off, _, _ = P.bie_solve(_dev(kappa), _dev(b), q=q0.clone(), tol=1e-10)
    assert its_off == its_plain
    P.check()


def test_preconditioned_mixed_solve_residual(ggem):
    s, _ = _pair()
    V, F = _ref_capsule()
    n = s.x.shape[0]
    kappa = np.full(n, KAPPA)
    b = np.random.default_rng(10).standard_normal((n, 3))
    P = _plan(ggem, s, "mixed")
    P.precond_set(V, F, KAPPA, 32, 32)
    q, its, rr, st = P.bie_solve(_dev(kappa), _dev(b), tol=1e-6)
    assert st in (0, 6)
    q = q.cpu().numpy()
    r = b - O.bie_operator(s, kappa, q)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-6 + 1e-9
    P.check()


def test_preconditioner_on_100_capsules(ggem):
    s = W.capsules_100()
    n = s.x.shape[0]
    kappa, b = W.bie_rhs(s, seed=3)
    P = _plan(ggem, s, "mixed")
    kd, bd = _dev(kappa), _dev(b)
    q1, its_plain, rr1, st1 = P.bie_solve(kd, bd, tol=1e-6)
    V, F = W.icosphere(3)
    P.precond_set(V, F, KAPPA)
    q2, its_pc, rr2, st2 = P.bie_solve(kd, bd, tol=1e-6)
    assert rr1 <= 1e-6 and rr2 <= 1e-6
    assert its_pc < its_plain, (its_pc, its_plain)
    nb = float(torch.linalg.norm(bd))
    assert float(torch.linalg.norm(q1 - q2)) < 4e-6 * nb
    P.check()


def test_precond_argument_errors(ggem):
    s, _ = _pair()
    P = _plan(ggem, s, "mixed")
    with pytest.raises(ggem.GGEMError):
        P.precond_enable(True)                   # nothing set yet
    V, F = W.rbc_mesh(level=2)                   # 162 nodes: the particles have 42
    P.precond_set(V, F, KAPPA, 32, 32)
    n = s.x.shape[0]
    with pytest.raises(ggem.GGEMError):
        P.bie_solve(_dev(np.full(n, KAPPA)), _dev(np.ones((n, 3))), tol=1e-6)
    with pytest.raises(ggem.GGEMError):
        P.precond_set(V, F, KAPPA, 24, 32)       # not a power of two
