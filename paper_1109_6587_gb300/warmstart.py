"""Learned warm start for the Fredholm solve: samples from the solver, training,
and solves that use it.  Host orchestration only -- every computation runs in
libggem's kernels through the C ABI (features, network, training, solve).

A series is a sequence of emulated time steps (workloads.rigid_step moves the
capsules, workloads.bie_rhs drifts the membrane load); step t is solved
starting from the density of step t-1 (from b at t = 0), as the paper's time
stepping does (Sec. 5).  The network estimates A^-1 r for the residual
r = b - A x0 of a guess x0, so the training samples of a step are the
features of r (ggem_mlp_features) and the target (q - x0 - r)/s, s = rms(r),
for the guesses the solver meets: x0 = b and x0 = the previous density.
"""
from __future__ import annotations

import numpy as np

from . import ggem
from . import workloads as W


def _dev(a, device):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)


def solve_series(plan, susp0, n_steps, seed, lam=5.0, tol=1e-6, use_mlp=0, device="cuda",
                 collect=False, restart=30, maxit=300):
    """Run n_steps emulated steps on `plan` (a plan for susp0's box with room
    for its mesh).  Returns a list of per-step dicts: iters, true relative
    residual, GMRES cycles, whether the learned guess was taken and the two
    guesses' residuals; with collect, also 'samples': [(feat [N, 12],
    target [N, 3])] for x0 = b and, from step 1, x0 = the previous density."""
    out = []
    q_prev = None
    import torch
    tri = torch.as_tensor(susp0.tri, device=device)
    for t in range(n_steps):
        s = W.rigid_step(susp0, seed=seed, step=t) if t else susp0
        kappa, b = W.bie_rhs(s, lam=lam, seed=seed, step=t)
        plan.mesh_set(_dev(s.x, device), tri)
        plan.mesh_particles(s.particle, len(s.centres))
        kd, bd = _dev(kappa, device), _dev(b, device)
        q0 = bd.clone() if q_prev is None else q_prev.clone()
        q, its, rr, st = plan.bie_solve(kd, bd, q=q0.clone(), tol=tol, restart=restart,
                                        maxit=maxit, use_mlp=use_mlp)
        used, r_plain, r_mlp = plan.solve_guess()
        rec = {"step": t, "iters": its, "relres": rr, "status": st,
               "cycles": plan.solve_stats()[0], "used_mlp": used,
               "relres_guess": r_plain, "relres_mlp": r_mlp}
        if collect:
            rec["samples"] = []
            for x0 in ([bd] if q_prev is None else [bd, q_prev]):
                r = bd - plan.bie_operator(kd, x0)
                feat, sc = plan.mlp_features(kd, r)
                if not sc > 0.0:
                    # the guess solves the system exactly (e.g. kappa = 0, where
                    # A = I and b is the solution): no residual to learn from
                    continue
                target = ((q - x0 - r) / sc).cpu().numpy()
                rec["samples"].append((feat, target))
        out.append(rec)
        q_prev = q
    return out


def training_set(plan, suspensions, n_steps, seed, lam=5.0, tol=1e-6, device="cuda"):
    """Features and targets of every sample of one series per suspension
    (series seeds seed, seed + 1, ...)."""
    F, T = [], []
    for i, s in enumerate(suspensions):
        for rec in solve_series(plan, s, n_steps, seed + i, lam=lam, tol=tol, device=device,
                                collect=True):
            for f, t in rec["samples"]:
                F.append(f)
                T.append(t)
    return np.concatenate(F), np.concatenate(T)


def generated_training_set(make_plan, pairs, n_steps, seed, tol=1e-6, device="cuda"):
    """Samples from series of generated suspensions of different sizes,
    volume fractions and viscosity ratios (pairs [(suspension, lambda)],
    e.g. workloads.training_suspensions()): each suspension is solved on a
    plan of its own slit, make_plan(suspension), closed afterwards.  The
    features do not depend on the plan, so the samples train any plan's
    model.  Returns (features [n, 12], targets [n, 3])."""
    F, T = [], []
    for i, (s, lam) in enumerate(pairs):
        P = make_plan(s)
        try:
            for rec in solve_series(P, s, n_steps, seed + i, lam=lam, tol=tol, device=device,
                                    collect=True):
                for f, t in rec["samples"]:
                    F.append(f)
                    T.append(t)
        finally:
            P.close()
    F, T = np.concatenate(F), np.concatenate(T)
    ok = np.isfinite(F).all(1) & np.isfinite(T).all(1)
    return F[ok], T[ok]


def train(plan, feat, target, seed=0, epochs=100, batch=512, lr=1e-3):
    """Fresh model on the samples; returns the last epoch's mean loss."""
    return plan.mlp_train(feat, target, init=True, seed=seed, epochs=epochs, batch=batch, lr=lr)
