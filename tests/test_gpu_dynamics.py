"""Capsule time stepping on the GPU (paper_1109_6587_gb300/dynamics.py, Sec. 5).

  * two full time steps of a capsule in simple shear (viscosity ratio 1,
    Ca = 0.3, 162 nodes), FP64 plan, against the same steps taken with the
    oracle: dt from the node separation, the midpoint step, the volume and
    the overlap corrections; positions within 1e-8 of the displacement;
  * twelve steps of the same capsule: it deforms (the Taylor parameter grows
    from 0 while the strain is small), every step keeps its volume within
    1e-4 of the initial one after the correction, and every stage's solve
    reaches its tolerance;
  * checkpoint and resume: a run saved after two steps and resumed on a
    fresh plan takes the same third step (positions within 1e-10 of the
    displacement; viscosity ratio 5, so the saved density seeds a real
    GMRES solve), with the same GMRES iteration count.
"""
import numpy as np
import pytest

from oracle import capsule as C
from paper_1109_6587_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ggem():
    from paper_1109_6587_gb300 import _build
    _build.build()
    from paper_1109_6587_gb300 import ggem as G
    return G


def _capsule():
    box = W.Box(Lx=16.0, Lz=16.0, W=10.0, y0=-5.0, Nx=32, Ny=33, Nz=32)
    return W.suspension(1, box, level=2, centres=np.array([[8.0, 0.0, 8.0]]))


def _plan(ggem, s, prec):
    P = ggem.Plan.for_box(s.box, precision=prec, quadrature="element", max_points=len(s.x),
                          max_tris=len(s.tri))
    P.mesh_set(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.tri, device="cuda"))
    return P


def _suspension(ggem, s, prec="fp64", lam=1.0):
    from paper_1109_6587_gb300 import dynamics as D
    P = _plan(ggem, s, prec)
    return P, D.Suspension(P, s.particle, 1, lam=np.array([lam]), ca=0.3, flow="shear",
                           strength=1.0, tri=s.tri)


def test_two_steps_match_the_oracle(ggem):
    s = _capsule()
    P, S = _suspension(ggem, s)
    x_ref = s.x.copy()
    v0 = C.volumes(s.x, s.tri, s.particle, 1)
    G = 1.0 / 0.3
    lam = np.ones(len(s.x))
    x = s.x.copy()
    for _ in range(2):
        rec = S.step(tol=1e-11, restart=40, maxit=400)
        dt = C.time_step(x, 0.3, 1.0, 1.0, s.box)
        assert rec["dt"] == pytest.approx(dt, rel=1e-12)
        sx = C._moved(s, x)
        xn, _, _ = C.midpoint_step(sx, x_ref, lam, G, "shear", 1.0, dt, tol=1e-11)
        xn, _ = C.volume_correct(xn, s.tri, s.particle, v0)
        xn, _ = C.overlap_correct(xn, s.particle, 1, s.box, 0.05)
        moved = np.abs(xn - x).max()
        x = xn
        assert np.abs(P.mesh_positions() - x).max() < 1e-8 * moved


def test_capsule_deforms_in_shear(ggem):
    s = _capsule()
    P, S = _suspension(ggem, s, "mixed")
    D = [S.deformation()[0]]
    for _ in range(12):
        rec = S.step(tol=1e-8)
        assert rec["relres"] <= 1e-8
        v = P.particle_volumes()
        assert abs(v[0] / S.v0[0] - 1) <= 1e-4
        D.append(S.deformation()[0])
    assert all(b > a for a, b in zip(D, D[1:]))             # deformation grows from rest
    assert 0.02 < D[-1] < 0.3
    P.check()


def test_checkpoint_resume(ggem, tmp_path):
    from paper_1109_6587_gb300 import dynamics as D
    s = _capsule()
    P, S = _suspension(ggem, s, "fp64", lam=5.0)
    for _ in range(2):
        S.step(tol=1e-10)
    path = tmp_path / "ckpt.npz"
    S.save(path)
    x2 = P.mesh_positions()
    rec_a = S.step(tol=1e-10)
    x_a = P.mesh_positions()
    P2 = ggem.Plan.for_box(s.box, precision="fp64", quadrature="element",
                           max_points=len(s.x), max_tris=len(s.tri))
    S2 = D.Suspension.resume(P2, path)
    assert S2.steps == 2 and S2.t == pytest.approx(S.t - rec_a["dt"], rel=1e-15)
    rec_b = S2.step(tol=1e-10)
    x_b = P2.mesh_positions()
    moved = np.abs(x_a - x2).max()
    assert moved > 1e-3
    assert np.abs(x_b - x_a).max() < 1e-10 * moved
    assert rec_b["iters"] == rec_a["iters"] and rec_b["dt"] == pytest.approx(rec_a["dt"], rel=1e-14)


def test_checkpoint_keeps_the_learned_model_and_its_adam_state(ggem, tmp_path):
    """A checkpoint of a plan holding a learned model keeps the model, its
    Adam moments and step count: the resumed plan holds the same state, and
    one more training epoch on the same samples moves both plans'
    parameters alike."""
    from paper_1109_6587_gb300 import dynamics as D
    s = _capsule()
    P, S = _suspension(ggem, s, "mixed", lam=5.0)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((600, 12))
    T = 0.3 * rng.standard_normal((600, 3))
    P.mlp_train(X, T, init=True, seed=2, epochs=3, batch=200, lr=1e-3)
    m, v, step = P.mlp_adam_state()
    assert step == 9 and np.abs(m).max() > 0 and v.min() >= 0
    path = tmp_path / "ckpt.npz"
    S.save(path)
    P2 = ggem.Plan.for_box(s.box, precision="mixed", quadrature="element",
                           max_points=len(s.x), max_tris=len(s.tri))
    D.Suspension.resume(P2, path)
    m2, v2, step2 = P2.mlp_adam_state()
    assert step2 == step and np.array_equal(m2, m) and np.array_equal(v2, v)
    assert np.array_equal(P2.mlp_save(), P.mlp_save())
    before = P.mlp_save()[25:]
    P.mlp_train(X, T, init=False, seed=5, epochs=1, batch=600, lr=1e-3)
    P2.mlp_train(X, T, init=False, seed=5, epochs=1, batch=600, lr=1e-3)
    a, b = P.mlp_save()[25:], P2.mlp_save()[25:]
    assert np.abs(a - before).max() > 1e-5
    assert np.abs(a - b).max() <= 1e-6 * (1.0 + np.abs(a).max())
    P.check()
    P2.check()
