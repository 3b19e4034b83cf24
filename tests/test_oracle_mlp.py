"""Pins of the learned warm start's oracle (oracle/mlp.py), CPU only.

  * bfloat16 rounding: ties to even at 1 + 2^-8 and 1 + 3 * 2^-8, and equal to
    torch's float32 -> bfloat16 conversion on random values;
  * backpropagation: gradients of the loss equal central finite differences
    (exact arithmetic, no rounding) for every parameter tensor;
  * Adam: the first step moves each parameter by lr * g / (|g| + eps);
  * features: r and its double layer enter divided by rms(r) (so the
    features of c r equal those of r), n and kappa are copied, the wall
    distance is exact; crowding is 0 for a particle out of reach and
    n_other / n_own when every node of the other particle is within r_cut;
  * training: Adam on a target the network can represent lowers the loss by
    more than 100x.
"""
import math

import numpy as np
import pytest

from oracle import mlp as M
from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W


def test_bf16_rounding():
    one = 1.0
    assert M.bf16(one + 2.0 ** -8) == 1.0                   # tie -> even (1.0)
    assert M.bf16(one + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6    # tie -> even (mantissa 2)
    assert M.bf16(one + 2.0 ** -7) == 1.0 + 2.0 ** -7        # representable
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).integers(-5, 5, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), ref)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    params = M.init_params(5)
    params = [p + 0.05 * rng.standard_normal(p.shape) for p in params]   # non-zero biases
    X = rng.standard_normal((7, M.NF))
    Y = rng.standard_normal((7, 3))
    loss, grads = M.loss_and_grads(params, X, Y)
    h = 1e-6
    for k, p in enumerate(params):
        flat = p.reshape(-1)
        idx = rng.choice(flat.size, min(flat.size, 12), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp, _ = M.loss_and_grads(params, X, Y)
            flat[i] = old - h
            lm, _ = M.loss_and_grads(params, X, Y)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[k].reshape(-1)[i]) < 1e-6 * max(1.0, abs(fd)), (k, i)


def test_adam_first_step():
    p = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -4.0, 1e-9])]
    state = []
    M.adam_step(p, g, state, lr=0.01, step=1)
    expect = np.array([1.0, -2.0, 0.5]) - 0.01 * g[0] / (np.abs(g[0]) + 1e-8)
    assert np.allclose(p[0], expect, rtol=0, atol=1e-15)


def _sphere(centre, radius, level=2):
    V, F = W.icosphere(level)
    return radius * V + centre, F


def test_features_on_spheres():
    box = W.Box(Lx=16.0, Lz=16.0, W=6.0, y0=-3.0, Nx=32, Ny=33, Nz=32)
    x1, F1 = _sphere(np.array([4.0, 0.2, 4.0]), 1.3)
    n1 = len(x1)
    rcut = 2.0
    # second particle: far away (no node within r_cut)
    x2, F2 = _sphere(np.array([12.0, 0.0, 12.0]), 0.5)
    x = np.vstack([x1, x2])
    tri = np.vstack([F1, F2 + n1])
    part = np.r_[np.zeros(n1, int), np.ones(len(x2), int)]
    kappa = np.r_[np.full(n1, 0.6), np.full(len(x2), -0.2)]
    rng = np.random.default_rng(2)
    r = rng.standard_normal(x.shape)
    Dr = rng.standard_normal(x.shape)
    _, _, _, nrm = O.geometry(x, tri)
    f, s = M.features(box, kappa, r, Dr, rcut, x, part, nrm)
    assert s == pytest.approx(np.sqrt((r * r).mean()), rel=1e-15)
    assert np.allclose(f[:, 0:3] * s, r, rtol=1e-15, atol=0)
    assert np.allclose(f[:, 3:6] * s, kappa[:, None] / (4 * math.pi) * Dr, rtol=1e-15, atol=0)
    f2, s2 = M.features(box, kappa, 7.0 * r, 7.0 * Dr, rcut, x, part, nrm)
    assert s2 == pytest.approx(7.0 * s) and np.allclose(f2, f, rtol=1e-14, atol=1e-14)
    assert np.array_equal(f[:, 6:9], nrm) and np.array_equal(f[:, 9], kappa)
    assert np.allclose(f[:, 10], np.minimum(x[:, 1] + 3.0, 3.0 - x[:, 1]), rtol=0, atol=1e-14)
    assert not f[:, 11].any()
    # a small particle next to the first: all its nodes within r_cut of the
    # nearest node of the first one
    x3, F3 = _sphere(x1[0] + 0.8 * (x1[0] - np.array([4.0, 0.2, 4.0])) / 1.3, 0.2, level=1)
    x = np.vstack([x1, x3])
    tri = np.vstack([F1, F3 + n1])
    part = np.r_[np.zeros(n1, int), np.ones(len(x3), int)]
    _, _, _, nrm = O.geometry(x, tri)
    f, _ = M.features(box, np.zeros(len(x)), np.ones(x.shape), np.zeros(x.shape), rcut, x,
                      part, nrm)
    assert f[0, 11] == len(x3) / n1


def test_training_reduces_loss():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((512, M.NF))
    A = rng.standard_normal((M.NF, 3)) / math.sqrt(M.NF)
    Y = np.maximum(X @ A, 0.0) - 0.3 * (X @ A)
    params = M.init_params(1)
    state = []
    l0, _ = M.loss_and_grads(params, X, Y)
    for step in range(1, 401):
        idx = rng.choice(len(X), 64, replace=False)
        _, g = M.loss_and_grads(params, X[idx], Y[idx])
        M.adam_step(params, g, state, lr=2e-3, step=step)
    l1, _ = M.loss_and_grads(params, X, Y)
    assert l1 < l0 / 100
