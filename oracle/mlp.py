"""Oracle of the learned warm start: per-node features, the MLP's forward and
backward passes, the training loss and Adam, in FP64 numpy.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may import this module.  It shares no code with the
CUDA library.

The paper solves the Fredholm system of Sec. 5, A q = b with
A = I + (kappa/4 pi) D, by GMRES from the previous time step's density and
uses no preconditioner.  The learned part approximates A^-1 r - r node by node
for a right-hand side r (b itself, or the residual b - A q_prev of a guess),
to serve as a GMRES initial guess q_prev + A^-1 r.  Its definitions (readings;
the paper has no counterpart):

  scale s = rms(r) over all nodes and components; the network sees r / s and
  predicts (A^-1 r - r) / (s s_y), so it applies to right-hand sides of any
  size (A^-1 is linear).
  features, 12 per node (caller order):
    0-2  r / s
    3-5  (kappa / 4 pi) (D r) / s           one application of the double layer
    6-8  n                                  area-averaged unit node normal
    9    kappa                              (lambda - 1)/(lambda + 1) of the node
    10   min(y - y0, y0 + W - y)            distance to the nearer wall
    11   crowding: nodes of OTHER particles within r_cut (minimum image in
         x, z), divided by the node count of the node's own particle
  network: 12 -> 128 -> 128 -> 128 -> 3, ReLU on the hidden layers; inputs
    standardised by (f - mu)/sigma, outputs scaled by s_y:
      A^-1 r - r ~ s * s_y * MLP((f - mu)/sigma)
  loss: mean over nodes and components of (output - target / s_y)^2, target
    (A^-1 r - r) / s.
  BF16 rounding points (when bf16=True): the standardised input, every weight
    matrix and every hidden activation are rounded to bfloat16 (round to
    nearest even); products accumulate without rounding.
"""
import math

import numpy as np

H = 128
NF = 12
SIZES = [(NF, H), (H, H), (H, H), (H, 3)]     # (fan_in, fan_out) per layer


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def features(box, kappa, r, Dr, rcut, x, particle, normals):
    """The 12 features per node (module docstring) for the right-hand side r
    [n, 3] with its double layer Dr [n, 3]; returns (F [n, 12] FP64, s)."""
    x = np.asarray(x, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    n = x.shape[0]
    s = math.sqrt((r * r).mean())
    F = np.zeros((n, NF))
    F[:, 0:3] = r / s
    F[:, 3:6] = (np.asarray(kappa)[:, None] / (4.0 * math.pi)) * np.asarray(Dr) / s
    F[:, 6:9] = normals
    F[:, 9] = kappa
    F[:, 10] = np.minimum(x[:, 1] - box.y0, box.y0 + box.W - x[:, 1])
    particle = np.asarray(particle)
    counts = np.bincount(particle)
    for i in range(n):
        d = x - x[i]
        d[:, 0] -= box.Lx * np.round(d[:, 0] / box.Lx)
        d[:, 2] -= box.Lz * np.round(d[:, 2] / box.Lz)
        r2 = (d * d).sum(1)
        F[i, 11] = np.count_nonzero((r2 < rcut * rcut) & (particle != particle[i]))
        F[i, 11] /= counts[particle[i]]
    return F, s


def init_params(seed):
    """He-uniform weights W [fan_in, fan_out] and zero biases, FP64."""
    rng = np.random.default_rng(seed)
    ps = []
    for fi, fo in SIZES:
        lim = math.sqrt(6.0 / fi)
        ps.append(rng.uniform(-lim, lim, (fi, fo)))
        ps.append(np.zeros(fo))
    return ps


def forward(params, X, bf16_round=False):
    """Activations [z0 (input), h1, h2, h3] and the output y = h3 W4 + b4."""
    rnd = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    h = rnd(X)
    acts = [h]
    for layer in range(4):
        W, bias = params[2 * layer], params[2 * layer + 1]
        z = h @ rnd(W) + bias
        if layer < 3:
            h = rnd(np.maximum(z, 0.0))
            acts.append(h)
        else:
            return acts, z


def loss_and_grads(params, X, Y, bf16_round=False):
    """Mean squared error over all entries and its gradient with respect to
    every parameter (backpropagation through the ReLU layers; the weights
    used in the backward pass are the same rounded ones as in the forward)."""
    rnd = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    acts, out = forward(params, X, bf16_round)
    m = out.size
    diff = out - Y
    loss = (diff * diff).sum() / m
    delta = 2.0 * diff / m
    grads = [None] * 8
    for layer in range(3, -1, -1):
        W = rnd(params[2 * layer])
        h = acts[layer]
        grads[2 * layer] = h.T @ delta
        grads[2 * layer + 1] = delta.sum(0)
        if layer > 0:
            delta = (delta @ W.T) * (h > 0.0)
    return loss, grads


def adam_step(params, grads, state, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of every parameter, in place; step >= 1."""
    if not state:
        state.extend([np.zeros_like(p) for p in params] + [np.zeros_like(p) for p in params])
    k = len(params)
    for i, (p, g) in enumerate(zip(params, grads)):
        m, v = state[i], state[k + i]
        m *= b1
        m += (1.0 - b1) * g
        v *= b2
        v += (1.0 - b2) * g * g
        mh = m / (1.0 - b1 ** step)
        vh = v / (1.0 - b2 ** step)
        p -= lr * mh / (np.sqrt(vh) + eps)
