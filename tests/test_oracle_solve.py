"""Pins of the oracle's Fredholm solve (Sec. 5), CPU only.

  * GMRES against numpy's dense LU on random well-conditioned systems, with
    restarts forced (m < n): the solution to 1e-10 and the reported residual
    equal to the recomputed one;
  * the iteration limit reports non-convergence with the true residual;
  * kappa = 0 makes the operator the identity: q = b, one Arnoldi step from
    a zero guess (happy breakdown) and none from the guess b;
  * the discretised operator (I + kappa/(4 pi) D) on a small sphere, assembled
    column by column, solved by LU, against GMRES on the same system;
  * a sphere carrying q = n: by the double-layer identity D n = lambda n the
    solution for b = n is n / (1 + kappa lambda/(4 pi)), lambda measured from
    the operator itself at the same mesh.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W


def _system(n, seed):
    rng = np.random.default_rng(seed)
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / math.sqrt(n)
    b = rng.standard_normal(n)
    return A, b


@pytest.mark.parametrize("restart", [5, 12, 60])
def test_gmres_matches_dense_solve(restart):
    A, b = _system(60, 3)
    x, its, rr, ok = O.gmres(lambda v: A @ v, b, tol=1e-13, restart=restart, maxit=500)
    xd = np.linalg.solve(A, b)
    assert ok
    assert np.abs(x - xd).max() < 1e-10 * np.abs(xd).max()
    assert abs(rr - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) < 1e-15
    assert its <= 60 if restart == 60 else its > 0


def test_gmres_iteration_limit():
    A, b = _system(40, 5)
    x, its, rr, ok = O.gmres(lambda v: A @ v, b, tol=1e-14, restart=4, maxit=6)
    assert not ok and its == 6
    assert rr == pytest.approx(np.linalg.norm(b - A @ x) / np.linalg.norm(b), rel=1e-12)
    assert rr > 1e-14


def test_gmres_identity_and_zero_rhs():
    b = np.random.default_rng(1).standard_normal(30)
    x, its, rr, ok = O.gmres(lambda v: v, b, tol=1e-12)
    assert ok and its == 1 and np.abs(x - b).max() < 1e-15
    x, its, rr, ok = O.gmres(lambda v: v, b, x0=b, tol=1e-12)
    assert ok and its == 0
    x, its, rr, ok = O.gmres(lambda v: 2 * v, np.zeros(30), tol=1e-12)
    assert ok and its == 0 and not x.any()


def _small_sphere(level=1):
    V, F = W.icosphere(level)
    box = W.Box(Lx=8.0, Lz=8.0, W=4.0, y0=-2.0, Nx=24, Ny=25, Nz=24)
    c = np.array([4.0, 0.1, 4.0])
    return W.Suspension(box=box, x=V + c, tri=F, particle=np.zeros(len(V), np.int32),
                        centres=c[None], radius=1.0)


def test_kappa_zero_gives_b():
    s = _small_sphere()
    b = np.random.default_rng(2).standard_normal(s.x.shape)
    q, its, rr, ok = O.bie_solve(s, np.zeros(len(s.x)), b, q0=b)
    assert ok and its == 0 and np.array_equal(q, b)


@pytest.mark.slow
@pytest.mark.parametrize("quadrature", ["nodal", "element"])
def test_bie_solve_matches_dense_lu(quadrature):
    s = _small_sphere()
    n = s.x.shape[0]
    rng = np.random.default_rng(4)
    kappa = np.full(n, 2.0 / 3.0)              # viscosity ratio 5
    b = rng.standard_normal((n, 3))
    A = np.zeros((3 * n, 3 * n))
    for c in range(3 * n):
        e = np.zeros(3 * n)
        e[c] = 1.0
        A[:, c] = O.bie_operator(s, kappa, e.reshape(n, 3), quadrature).ravel()
    qd = np.linalg.solve(A, b.ravel()).reshape(n, 3)
    q, its, rr, ok = O.bie_solve(s, kappa, b, tol=1e-12, quadrature=quadrature)
    assert ok and its < 3 * n
    assert np.abs(q - qd).max() < 1e-9 * np.abs(qd).max()
    # a Fredholm operator of the second kind with |kappa| < 1 is well conditioned
    assert np.linalg.cond(A) < 20


def test_normal_density_solution():
    s = _small_sphere(2)
    n = s.x.shape[0]
    _, _, _, nb = O.geometry(s.x, s.tri)
    kappa = np.full(n, -0.6)
    Dn = O.double_layer(s, nb)
    lam = np.einsum("ij,ij->i", Dn, nb).mean()
    q, its, rr, ok = O.bie_solve(s, kappa, nb, tol=1e-10)
    expect = nb / (1.0 + kappa[0] * lam / (4.0 * math.pi))
    # D n = lam n holds up to the mesh/grid error of the operator (~1e-2 here)
    assert ok and np.abs(q - expect).max() < 0.05 * np.abs(expect).max()


def test_block_diagonal_preconditioner_ceiling():
    """What a learned 3x3 block-diagonal preconditioner could at best gain:
    the exact inverse of every node's 3x3 diagonal block of the discrete
    operator (I + kappa/4pi D) as a right preconditioner saves no GMRES
    iteration on two capsules, while the exact inverse of each particle's
    whole block halves the count, and so does one block shared by both (the
    inverse of an isolated capsule's block at the slit centre): the operator's
    spread comes from coupling across each particle, not from node-local
    coupling."""
    V, F = W.icosphere(1)
    box = W.Box(Lx=8.0, Lz=8.0, W=4.0, y0=-2.0, Nx=16, Ny=17, Nz=16)
    c1, c2 = np.array([2.2, 0.1, 4.0]), np.array([5.0, -0.4, 4.5])
    s = W.Suspension(box=box, x=np.concatenate([0.97 * V + c1, 0.97 * V + c2]),
                     tri=np.concatenate([F, F + len(V)]),
                     particle=np.repeat([0, 1], len(V)).astype(np.int32),
                     centres=np.stack([c1, c2]), radius=0.97)
    n, m = s.x.shape[0], 3 * len(V)
    for kap in (2.0 / 3.0, -2.0 / 3.0):
        kappa = np.full(n, kap)
        A = np.stack([O.bie_operator(s, kappa, e.reshape(n, 3)).ravel()
                      for e in np.eye(3 * n)], 1)
        b = np.random.default_rng(0).standard_normal(3 * n)

        def its(M):
            return O.gmres(lambda y: A @ (M @ y), b, tol=1e-6)[1]
        node = np.zeros_like(A)
        for i in range(n):
            sl = slice(3 * i, 3 * i + 3)
            node[sl, sl] = np.linalg.inv(A[sl, sl])
        part = np.zeros_like(A)
        for p in range(2):
            sl = slice(p * m, (p + 1) * m)
            part[sl, sl] = np.linalg.inv(A[sl, sl])
        plain = its(np.eye(3 * n))
        assert its(node) >= plain - 1
        assert its(part) <= plain // 2 + 1
        # one shared block, from an isolated capsule at the slit centre, for both
        c = np.array([4.0, 0.0, 4.0])
        r = W.Suspension(box=box, x=0.97 * V + c, tri=F, particle=np.zeros(len(V), np.int32),
                         centres=c[None], radius=0.97)
        Ar = np.stack([O.bie_operator(r, np.full(len(V), kap), e.reshape(len(V), 3)).ravel()
                       for e in np.eye(m)], 1)
        shared = np.zeros_like(A)
        for p in range(2):
            sl = slice(p * m, (p + 1) * m)
            shared[sl, sl] = np.linalg.inv(Ar)
        assert its(shared) <= plain // 2 + 1


def test_particle_block_preconditioned_solve():
    """The reference for a per-particle block preconditioner: with the
    identity as the block it is plain GMRES (same iterations, same solution);
    with the inverse of an isolated capsule's block it solves the same system
    to the same tolerance in about half the iterations."""
    V, F = W.icosphere(1)
    box = W.Box(Lx=8.0, Lz=8.0, W=4.0, y0=-2.0, Nx=16, Ny=17, Nz=16)
    c1, c2 = np.array([2.2, 0.1, 4.0]), np.array([5.0, -0.4, 4.5])
    s = W.Suspension(box=box, x=np.concatenate([0.97 * V + c1, 0.97 * V + c2]),
                     tri=np.concatenate([F, F + len(V)]),
                     particle=np.repeat([0, 1], len(V)).astype(np.int32),
                     centres=np.stack([c1, c2]), radius=0.97)
    n = s.x.shape[0]
    kappa = np.full(n, 2.0 / 3.0)
    b = np.random.default_rng(4).standard_normal((n, 3))
    q_ref, its_ref, rr_ref, ok = O.bie_solve(s, kappa, b, tol=1e-10, quadrature="element")
    assert ok
    q, its, rr, ok = O.particle_block_solve(s, kappa, b, np.eye(3 * len(V)), tol=1e-10)
    assert ok and its == its_ref and np.abs(q - q_ref).max() < 1e-12 * np.abs(q_ref).max()
    c = np.array([4.0, 0.0, 4.0])
    r = W.Suspension(box=box, x=0.97 * V + c, tri=F, particle=np.zeros(len(V), np.int32),
                     centres=c[None], radius=0.97)
    Minv = np.linalg.inv(O.assembled_operator(r, np.full(len(V), 2.0 / 3.0)))
    q, its_p, rr, ok = O.particle_block_solve(s, kappa, b, Minv, tol=1e-10)
    assert ok and rr <= 1e-10
    assert np.abs(q - q_ref).max() < 1e-8 * np.abs(q_ref).max()
    assert its_p <= its_ref // 2 + 2


def _rot_y(angle):
    c, s = np.cos(angle), np.sin(angle)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def test_operator_rotation_about_the_wall_normal():
    """Pin of the rotation used by the per-particle block preconditioner: a
    quarter turn about the wall normal maps a square slit's grid (capsule
    centred on a grid node, Nx = Nz, Lx = Lz) onto itself, so the discrete
    operator of the turned capsule is (I x R) A (I x R^T) exactly -- the
    identity that lets one reference block serve particles of any
    orientation; a wrong transpose or index order fails it."""
    V, F = W.rbc_mesh(level=1)
    box = W.Box(Lx=8.0, Lz=8.0, W=4.0, y0=-2.0, Nx=16, Ny=17, Nz=16)
    c = np.array([4.0, 0.0, 4.0])
    R = _rot_y(0.5 * np.pi)
    n = len(V)
    kappa = np.full(n, 2.0 / 3.0)

    def susp(x):
        return W.Suspension(box=box, x=x + c, tri=F, particle=np.zeros(n, np.int32),
                            centres=c[None], radius=1.0)
    A = O.assembled_operator(susp(V), kappa)
    Ar = O.assembled_operator(susp(V @ R.T), kappa)
    K = np.kron(np.eye(n), R)
    assert np.abs(Ar - K @ A @ K.T).max() < 1e-10 * np.abs(A).max()
    # the reference block of the preconditioner is this capsule's inverse
    Minv = O.reference_block_inverse(box, V, F, 2.0 / 3.0, 16, 16)
    assert np.abs(Minv @ A - np.eye(3 * n)).max() < 1e-10
    rb = O.reference_box(box, 8, 8)
    assert (rb.Lx, rb.Lz, rb.Nx, rb.Nz, rb.Ny, rb.W) == (4.0, 4.0, 8, 8, 17, 4.0)
    assert O.default_alpha(rb) == O.default_alpha(box)


def test_rotated_block_preconditioner():
    """Two randomly oriented biconcave capsules: the isolated unrotated
    capsule's inverse block, turned to each particle's orientation, solves
    the system to the plain solve's solution in about half its iterations,
    and in fewer than the same block left unturned."""
    V, F = W.rbc_mesh(level=1)
    box = W.Box(Lx=8.0, Lz=8.0, W=4.0, y0=-2.0, Nx=16, Ny=17, Nz=16)
    rot = W.random_rotations(2, np.random.default_rng(8))
    cs = [np.array([2.2, 0.1, 4.0]), np.array([5.5, -0.3, 4.5])]
    x = np.concatenate([V @ rot[p].T + cs[p] for p in range(2)])
    s = W.Suspension(box=box, x=x, tri=np.concatenate([F, F + len(V)]),
                     particle=np.repeat([0, 1], len(V)).astype(np.int32),
                     centres=np.stack(cs), radius=1.0)
    n = x.shape[0]
    kappa = np.full(n, 2.0 / 3.0)
    b = np.random.default_rng(9).standard_normal((n, 3))
    q_ref, its_ref, _, ok = O.bie_solve(s, kappa, b, tol=1e-10)
    assert ok
    Minv = O.reference_block_inverse(box, V, F, 2.0 / 3.0, 16, 16)
    q, its_rot, rr, ok = O.particle_block_solve(s, kappa, b, Minv, tol=1e-10, rotations=rot)
    assert ok and rr <= 1e-10
    assert np.abs(q - q_ref).max() < 1e-8 * np.abs(q_ref).max()
    _, its_plain_block, _, ok2 = O.particle_block_solve(s, kappa, b, Minv, tol=1e-10)
    print("plain", its_ref, "rotated block", its_rot, "unrotated block", its_plain_block)
    assert its_rot <= its_ref // 2 + 2
    assert its_rot < its_plain_block
