"""Learned warm start on the GPU against its oracle (oracle/mlp.py), and what
it gains in the Fredholm solve.

  * features: FP32 copies of the oracle's FP64 values (1e-6 relative), the
    double-layer columns at the mixed parity (1e-5); the crowding count, an
    integer decided in FP64 on both sides, exactly;
  * forward: the bfloat16 network (tensor-core kernel) against the oracle
    with the same rounding points (FP32 vs FP64 accumulation can move a
    hidden activation by one bfloat16 step: 1e-2 of the output scale), most
    rows, those with no such step, within 1e-5; the learned guess equals
    r + s s_y times the forward output of its own features;
  * gradient of one full-batch pass against the oracle's backpropagation
    (2e-2 relative per parameter tensor), and the loss (1e-3);
  * one Adam step moves the parameters in the oracle's direction, and its
    values equal the oracle's Adam applied to the kernel's own gradient;
  * FP32 mode (no bfloat16 rounding point): forward output and every
    gradient entry against the oracle's FP64 network entry by entry, each
    within 2e-5 of the sum of the magnitudes of its terms (the FP32 error
    bound of a sum), and one Adam step entry by entry;
  * the Fredholm operator (I + kappa/4 pi D) against the oracle's;
  * warm start: trained on emulated time-step series of suspensions, on a
    held-out series the learned guess has a lower residual than the caller's
    guess (b at the first step, the previous density after it) by 2x or more,
    and the solves take fewer GMRES iterations over the series.  (The system
    is of the second kind: GMRES itself reduces the residual about 3x per
    iteration, so a guess 3x better saves about one iteration.)
"""
import numpy as np
import pytest

from oracle import mlp as M
from oracle import oracle as O
from paper_1109_6587_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ggem():
    from paper_1109_6587_gb300 import _build
    _build.build()
    from paper_1109_6587_gb300 import ggem as G
    return G


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _box():
    return W.Box(Lx=16.0, Lz=16.0, W=6.0, y0=-3.0, Nx=32, Ny=33, Nz=32)


def _plan(ggem, s, prec="mixed", quad="nodal"):
    P = ggem.Plan.for_box(s.box, precision=prec, quadrature=quad, max_points=s.x.shape[0],
                          max_tris=s.tri.shape[0])
    P.mesh_set(_dev(s.x), torch.as_tensor(s.tri, device="cuda"))
    P.mesh_particles(s.particle, len(s.centres))
    return P


@pytest.fixture(scope="module")
def susp():
    return W.suspension(8, _box(), level=2, seed=3)


def test_features_match_oracle(ggem, susp):
    s = susp
    P = _plan(ggem, s)
    kappa, b = W.bie_rhs(s, seed=4)
    r = np.random.default_rng(5).standard_normal(s.x.shape)
    f, sc = P.mlp_features(_dev(kappa), _dev(r))
    a, rc = P.info()
    _, _, _, nrm = O.geometry(s.x, s.tri)
    Dr = O.double_layer(s, r, quadrature="nodal")
    ref, sref = M.features(s.box, kappa, r, Dr, rc, s.x, s.particle, nrm)
    assert abs(sc - sref) < 1e-14 * sref
    cols = [c for c in range(12) if c not in (3, 4, 5, 11)]
    scale = np.abs(ref[:, cols]).max(0)
    assert (np.abs(f[:, cols] - ref[:, cols]) / scale).max() < 1e-6
    # (kappa/4 pi) D r / s: the mixed double layer (1e-5 parity)
    assert np.abs(f[:, 3:6] - ref[:, 3:6]).max() < 1e-5 * np.abs(ref[:, 3:6]).max()
    assert np.array_equal(f[:, 11], ref[:, 11].astype(np.float32).astype(np.float64))
    assert ref[:, 11].max() > 0          # the case has crowded nodes


def test_bie_operator_matches_oracle(ggem, susp):
    s = susp
    P = _plan(ggem, s, prec="fp64")
    kappa, _ = W.bie_rhs(s, seed=4)
    q = np.random.default_rng(6).standard_normal(s.x.shape)
    out = P.bie_operator(_dev(kappa), _dev(q)).cpu().numpy()
    ref = O.bie_operator(s, kappa, q, quadrature="nodal")
    assert np.abs(out - ref).max() < 1e-10 * np.abs(ref).max()


def _model(seed):
    rng = np.random.default_rng(seed)
    params = M.init_params(seed)
    params = [p + 0.05 * rng.standard_normal(p.shape) if p.ndim == 1 else p for p in params]
    mu = rng.standard_normal(12) * 0.1
    sigma = 0.5 + rng.random(12)
    s_y = 0.7
    blob = np.concatenate([mu, sigma, [s_y]] + [p.ravel() for p in params])
    return params, mu, sigma, s_y, blob


def test_forward_matches_oracle(ggem, susp):
    P = _plan(ggem, susp)
    params, mu, sigma, s_y, blob = _model(11)
    P.mlp_load(blob)
    assert np.array_equal(P.mlp_save(), blob.astype(np.float32).astype(np.float64))
    X = np.random.default_rng(12).standard_normal((1000, 12))
    out = P.mlp_forward(X)
    _, ref = M.forward(params, (X - mu) / sigma, bf16_round=True)
    assert np.abs(out - ref).max() < 1e-2 * np.abs(ref).max()


def test_tensor_core_forward_rows_and_guess(ggem, susp):
    P = _plan(ggem, susp)
    params, mu, sigma, s_y, blob = _model(13)
    P.mlp_load(blob)
    X = np.random.default_rng(14).standard_normal((3000, 12))
    out = P.mlp_forward(X)
    pf = [_f32(p) for p in params]
    _, ref = M.forward(pf, (_f32(X) - _f32(mu)) / _f32(sigma), bf16_round=True)
    scale = np.abs(ref).max()
    row_err = np.abs(out - ref).max(1) / scale
    assert row_err.max() < 1e-2
    assert (row_err < 1e-5).mean() > 0.8, float((row_err < 1e-5).mean())
    # the learned guess of the solve: r + s s_y y(features of r), same kernel
    kappa, b = W.bie_rhs(susp, seed=15)
    r = np.random.default_rng(16).standard_normal(susp.x.shape)
    f, sc = P.mlp_features(_dev(kappa), _dev(r))
    y = P.mlp_forward(f)
    g = P.mlp_guess(_dev(kappa), _dev(r)).cpu().numpy()
    # mlp_guess evaluates the features again: the double layer's spreading adds
    # in L2 reductions of arbitrary order, so its features differ from f by FP32
    # rounding, which now and then moves a BF16 rounding of the network's input;
    # compare the correction row by row as the forward check above does
    corr = sc * s_y * y
    cerr = np.abs((g - r) - corr).max(1) / np.abs(corr).max()
    assert cerr.max() < 1e-2
    assert (cerr < 1e-5).mean() > 0.95, float((cerr < 1e-5).mean())
    P.check()


def test_gradient_and_adam_match_oracle(ggem, susp):
    P = _plan(ggem, susp)
    params, mu, sigma, s_y, blob = _model(21)
    P.mlp_load(blob)
    rng = np.random.default_rng(22)
    X = rng.standard_normal((700, 12))
    T = rng.standard_normal((700, 3)) * 0.3
    loss, g = P.mlp_train(X, T, init=False, epochs=0, want_grad=True)
    pf = [p.astype(np.float32).astype(np.float64) for p in params]
    ref_loss, ref_g = M.loss_and_grads(pf, (X - mu) / sigma, T / s_y, bf16_round=True)
    assert abs(loss - ref_loss) < 1e-3 * ref_loss
    off = 0
    for rg in ref_g:
        gg = g[off:off + rg.size].reshape(rg.shape)
        off += rg.size
        assert np.linalg.norm(gg - rg) < 2e-2 * np.linalg.norm(rg)
    # one Adam step on the same full batch
    P.mlp_load(blob)
    P.mlp_train(X, T, init=False, epochs=1, batch=700, lr=1e-3)
    new = P.mlp_save()[25:]
    state = []
    M.adam_step(pf, ref_g, state, lr=1e-3, step=1)
    moved_gpu = new - blob[25:].astype(np.float32).astype(np.float64)
    moved_ref = np.concatenate([p.ravel() for p in pf]) - blob[25:].astype(np.float32)
    big = np.abs(np.concatenate([x.ravel() for x in ref_g])) > 1e-6
    assert (np.sign(moved_gpu[big]) == np.sign(moved_ref[big])).mean() > 0.99


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _abs_forward(params, X):
    """Per-entry magnitude scales of the forward pass: |X| through |W| and
    |b| (the sums of the magnitudes of the terms of every activation)."""
    h = np.abs(X)
    for layer in range(4):
        h = h @ np.abs(params[2 * layer]) + np.abs(params[2 * layer + 1])
    return h


def test_fp32_mode_forward_entrywise(ggem, susp):
    P = _plan(ggem, susp)
    P.mlp_precision("fp32")
    params, mu, sigma, s_y, blob = _model(31)
    P.mlp_load(blob)
    X = np.random.default_rng(32).standard_normal((1000, 12))
    out = P.mlp_forward(X)
    pf = [_f32(p) for p in params]
    Z = (_f32(X) - _f32(mu)) / _f32(sigma)
    _, ref = M.forward(pf, Z, bf16_round=False)
    scale = _abs_forward(pf, Z)
    err = np.abs(out - ref)
    assert (err <= 2e-5 * scale + 1e-12).all(), float((err / scale).max())
    # the rounding points matter: the BF16 network differs by far more
    P.mlp_precision("bf16")
    out_bf = P.mlp_forward(X)
    assert np.abs(out_bf - ref).max() > 1e2 * err.max()


def test_fp32_mode_gradient_and_adam_entrywise(ggem, susp):
    P = _plan(ggem, susp)
    P.mlp_precision("fp32")
    params, mu, sigma, s_y, blob = _model(41)
    P.mlp_load(blob)
    rng = np.random.default_rng(42)
    X = rng.standard_normal((700, 12))
    T = rng.standard_normal((700, 3)) * 0.3
    loss, g = P.mlp_train(X, T, init=False, epochs=0, want_grad=True)
    pf = [_f32(p) for p in params]
    Z = (_f32(X) - _f32(mu)) / _f32(sigma)
    Y = _f32(T) / _f32(s_y)
    ref_loss, ref_g = M.loss_and_grads(pf, Z, Y, bf16_round=False)
    assert abs(loss - ref_loss) < 1e-5 * ref_loss
    # magnitude scale of every gradient entry: the same backpropagation with
    # magnitudes (|activations|, |deltas|, |weights|)
    acts, out = M.forward(pf, Z)
    delta = np.abs(2.0 * (out - Y) / out.size)
    scales = [None] * 8
    for layer in range(3, -1, -1):
        h = np.abs(acts[layer])
        scales[2 * layer] = h.T @ delta
        scales[2 * layer + 1] = delta.sum(0)
        if layer > 0:
            delta = (delta @ np.abs(pf[2 * layer]).T) * (acts[layer] > 0)
    off = 0
    tols = []
    for k, rg in enumerate(ref_g):
        gg = g[off:off + rg.size].reshape(rg.shape)
        off += rg.size
        tol = 2e-5 * scales[k] + 1e-12
        bad = np.abs(gg - rg) > tol
        assert not bad.any(), (k, int(bad.sum()), float((np.abs(gg - rg) / tol).max()))
        tols.append(tol.ravel())
    tol = np.concatenate(tols)
    # one Adam step on the same full batch: entries whose gradient sign is
    # decided (|g| far above its error bound) move by the oracle's value
    P.mlp_load(blob)
    P.mlp_train(X, T, init=False, epochs=1, batch=700, lr=1e-3)
    new = P.mlp_save()[25:]
    p0 = np.concatenate([p.ravel() for p in pf])
    state = []
    pr = [p.copy() for p in pf]
    M.adam_step(pr, ref_g, state, lr=1e-3, step=1)
    pr = np.concatenate([p.ravel() for p in pr])
    gr = np.concatenate([x.ravel() for x in ref_g])
    sure = np.abs(gr) > 100 * tol
    assert sure.mean() > 0.9
    assert (np.abs(new[sure] - pr[sure]) <= 2.5e-7 * np.abs(pr[sure]) + 2e-8).all()
    assert (np.abs(new - p0) <= 1e-3 * (1 + 1e-6) + 2.5e-7 * np.abs(p0)).all()


def test_bf16_adam_values_match_oracle_on_the_kernel_gradient(ggem, susp):
    """The Adam kernel entry by entry: the oracle's Adam step applied to the
    gradient the kernels computed gives the parameters the GPU step wrote
    (entries whose gradient is not tiny: the step's own pass accumulates its
    atomics in another order, which can flip the sign of a near-zero one)."""
    P = _plan(ggem, susp)
    params, mu, sigma, s_y, blob = _model(51)
    P.mlp_load(blob)
    rng = np.random.default_rng(52)
    X = rng.standard_normal((500, 12))
    T = rng.standard_normal((500, 3)) * 0.3
    _, g = P.mlp_train(X, T, init=False, epochs=0, want_grad=True)
    P.mlp_load(blob)
    P.mlp_train(X, T, init=False, epochs=1, batch=500, lr=1e-3)
    new = P.mlp_save()[25:]
    pf = [_f32(p) for p in params]
    shapes = [p.shape for p in pf]
    gl, off = [], 0
    for sh in shapes:
        k = int(np.prod(sh))
        gl.append(g[off:off + k].reshape(sh))
        off += k
    state = []
    M.adam_step(pf, gl, state, lr=1e-3, step=1)
    pr = np.concatenate([p.ravel() for p in pf])
    p0 = np.concatenate([_f32(p).ravel() for p in params])
    sure = np.abs(g) > 1e-4 * np.abs(g).max()
    assert sure.mean() > 0.9
    assert (np.abs(new[sure] - pr[sure]) <= 2.5e-7 * np.abs(pr[sure]) + 2e-8).all()
    assert (np.abs(new - p0) <= 1e-3 * (1 + 1e-6) + 2.5e-7 * np.abs(p0)).all()


def test_tensor_core_training_gradient(ggem, susp):
    """BF16 mode trains with tensor-core GEMMs (deltas split into two
    bfloat16 terms): its full-batch gradient against the oracle's with the
    same rounding points, per tensor within 5e-3 in norm, and 99 % of the
    entries within 1e-3 of the sum of their terms' magnitudes (the rest can
    see a hidden activation one bfloat16 step away)."""
    P = _plan(ggem, susp)
    params, mu, sigma, s_y, blob = _model(61)
    P.mlp_load(blob)
    rng = np.random.default_rng(62)
    X = rng.standard_normal((700, 12))
    T = rng.standard_normal((700, 3)) * 0.3
    loss, g = P.mlp_train(X, T, init=False, epochs=0, want_grad=True)
    pf = [_f32(p) for p in params]
    Z = (_f32(X) - _f32(mu)) / _f32(sigma)
    Y = _f32(T) / _f32(s_y)
    ref_loss, ref_g = M.loss_and_grads(pf, Z, Y, bf16_round=True)
    assert abs(loss - ref_loss) < 1e-3 * ref_loss
    acts, out = M.forward(pf, Z, bf16_round=True)
    delta = np.abs(2.0 * (out - Y) / out.size)
    off, near, total = 0, 0, 0
    for layer in range(3, -1, -1):
        h = np.abs(acts[layer])
        sW, sb = h.T @ delta, delta.sum(0)
        for k, sc in ((2 * layer, sW), (2 * layer + 1, sb)):
            rg = ref_g[k]
            o = sum(x.size for x in ref_g[:k])
            gg = g[o:o + rg.size].reshape(rg.shape)
            assert np.linalg.norm(gg - rg) < 5e-3 * np.linalg.norm(rg), k
            near += int((np.abs(gg - rg) <= 1e-3 * sc + 1e-9).sum())
            total += rg.size
        if layer > 0:
            delta = (delta @ np.abs(M.bf16(pf[2 * layer])).T) * (acts[layer] > 0)
    assert near >= 0.99 * total, near / total
    P.check()


def test_learned_warm_start_reduces_iterations(ggem):
    from paper_1109_6587_gb300 import warmstart as WS
    box = _box()
    train_s = [W.suspension(8, box, level=2, seed=100 + i) for i in range(3)]
    P = _plan(ggem, train_s[0])
    F, T = WS.training_set(P, train_s, n_steps=5, seed=200)
    loss = WS.train(P, F, T, seed=1, epochs=150, batch=512, lr=1e-3)
    assert loss < 0.5                     # in units of rms(target)^2
    test_s = W.suspension(8, box, level=2, seed=999)
    plain = WS.solve_series(P, test_s, 4, seed=300, use_mlp=0)
    learned = WS.solve_series(P, test_s, 4, seed=300, use_mlp=1)
    # every step: the learned guess has at most half the residual of the
    # caller's guess (b at step 0, the previous density after it), the solve
    # never takes more GMRES iterations, and over the series it takes fewer
    for p, l in zip(plain, learned):
        assert l["used_mlp"] and l["relres_mlp"] < 0.5 * l["relres_guess"]
        assert l["iters"] <= p["iters"]
        assert l["relres"] <= 1e-6
    assert sum(l["iters"] for l in learned) < sum(p["iters"] for p in plain)
