"""Time stepping of a capsule suspension (Sec. 5, 7.1): host orchestration of
the library's capsule entry points; every computation runs in libggem's
kernels through the C ABI.

One step, as the paper takes it:
  1. dt from gamma_dot dt = 0.5 Ca h_min / a, h_min the smallest node
     separation in the system (ggem_min_separation);
  2. the midpoint step of dx/dt = u (ggem_capsule_step), the Fredholm solve of
     each stage starting from the previous stage's density;
  3. the volume correction of particles that drifted more than 1e-4 of their
     initial volume (ggem_volume_correct);
  4. the minimum-gap correction, h_gap = 0.05 a (ggem_overlap_correct).
"""
from __future__ import annotations

import time

import numpy as np

from .ggem import GGEMError


class Suspension:
    """Capsules on a plan: the plan holds the mesh (moved by every step), the
    membrane reference is the mesh given at construction, lambda per particle."""

    def __init__(self, plan, particle, n_particles, lam, ca=0.3, radius=1.0, flow="shear",
                 strength=1.0, mu=1.0, h_gap=0.05, vol_threshold=1e-4, tri=None, x_ref=None,
                 v0=None):
        """tri (optional): the mesh's triangles, kept for checkpoints; x_ref and
        v0 (optional): membrane reference and initial volumes when resuming
        (default: the plan's current mesh and its volumes)."""
        self.P = plan
        self.particle = np.asarray(particle)
        self.n_particles = int(n_particles)
        self.lam = np.asarray(lam, dtype=np.float64)
        self.lam_nodes = np.ascontiguousarray(self.lam[self.particle])
        self.tri = None if tri is None else np.asarray(tri, dtype=np.int32)
        self.mu = mu
        self.h_gap_factor = h_gap
        self.ca, self.radius, self.flow, self.strength = ca, radius, flow, strength
        # Ca = mu gamma_dot a / G with gamma_dot the shear rate (shear flow) or
        # the wall shear rate 4 U0 / H (pressure-driven flow)
        self.gamma = strength if flow == "shear" else 4.0 * strength / plan.params.W
        self.shear_modulus = mu * self.gamma * radius / ca
        self.h_gap = h_gap * radius
        self.vol_threshold = vol_threshold
        plan.mesh_particles(self.particle, self.n_particles)
        self.x_ref = plan.mesh_positions() if x_ref is None else np.asarray(x_ref, np.float64)
        plan.membrane_reference(np.ascontiguousarray(self.x_ref))
        self.v0 = plan.particle_volumes() if v0 is None else np.asarray(v0, np.float64)
        self.q = np.zeros((plan.n_nodes, 3))
        self.t = 0.0
        self.steps = 0

    # ------------------------------------------------------------ checkpoints
    def save(self, path):
        """Checkpoint (numpy .npz): node positions, triangles, membrane
        reference, the density that seeds the next solve, initial volumes,
        time, step count, viscosity ratios, particle ids and the run's
        parameters; plus, when the plan holds a learned model, the model and
        its Adam moments and step count (a resumed run continues training
        where the saved one stopped)."""
        if self.tri is None:
            raise ValueError("checkpoints need the triangles (pass tri= at construction)")
        extra = {}
        try:
            extra["mlp"] = self.P.mlp_save()
            m, v, st = self.P.mlp_adam_state()
            extra["mlp_m"], extra["mlp_v"], extra["mlp_step"] = m, v, np.array(st)
        except GGEMError:                 # the plan holds no model
            pass
        np.savez(path, x=self.P.mesh_positions(), tri=self.tri, x_ref=self.x_ref,
                 q=np.asarray(self.q.cpu() if hasattr(self.q, "cpu") else self.q),
                 v0=self.v0, t=self.t, steps=self.steps, lam=self.lam, particle=self.particle,
                 params=np.array([self.ca, self.radius, self.strength, self.mu,
                                  self.h_gap_factor, self.vol_threshold]),
                 flow=np.array(self.flow), **extra)

    @classmethod
    def resume(cls, plan, path):
        """A suspension continuing a checkpoint on `plan` (a plan for the same
        box with room for the mesh): the next step reproduces the one the
        saved run would have taken."""
        z = np.load(path)
        ca, radius, strength, mu, h_gap, vol_threshold = (float(v) for v in z["params"])
        plan.mesh_set(np.ascontiguousarray(z["x"]), np.ascontiguousarray(z["tri"]))
        if "mlp" in z:
            plan.mlp_load(z["mlp"])
            if "mlp_m" in z:
                plan.mlp_adam_state((z["mlp_m"], z["mlp_v"], int(z["mlp_step"])))
        S = cls(plan, z["particle"], len(z["lam"]), z["lam"], ca=ca, radius=radius,
                flow=str(z["flow"]), strength=strength, mu=mu, h_gap=h_gap,
                vol_threshold=vol_threshold, tri=z["tri"], x_ref=z["x_ref"], v0=z["v0"])
        S.q = np.array(z["q"])
        S.t = float(z["t"])
        S.steps = int(z["steps"])
        return S

    def dt(self):
        return 0.5 * self.ca * self.P.min_separation() / (self.radius * self.gamma)

    def step(self, tol=1e-6, restart=30, maxit=300, use_mlp=0):
        """One time step; returns its record (dt, GMRES iterations, residual,
        correction passes and pair moves, wall time)."""
        t0 = time.perf_counter()
        dt = self.dt()
        _, self.q, its, rr = self.P.capsule_step(self.lam_nodes, dt, self.flow, self.strength,
                                                 self.shear_modulus, q=self.q, tol=tol,
                                                 restart=restart, maxit=maxit, use_mlp=use_mlp)
        passes = self.P.volume_correct(self.v0, self.vol_threshold, 10)
        moves = self.P.overlap_correct(self.h_gap)
        self.t += dt
        self.steps += 1
        return {"dt": dt, "iters": its, "relres": rr, "volume_passes": passes,
                "overlap_moves": moves, "seconds": time.perf_counter() - t0}

    def deformation(self):
        """Taylor parameter D = (L - B)/(L + B) of every particle in the shear
        plane (x, y): L and B the largest and smallest distance of a node from
        the particle's centroid, taken over nodes near that plane (Sec. 6.3)."""
        x = self.P.mesh_positions()
        out = np.zeros(self.n_particles)
        for p in range(self.n_particles):
            xp = x[self.particle == p]
            r = xp - xp.mean(0)
            d = np.linalg.norm(r, axis=1)
            band = np.abs(r[:, 2]) < 0.25 * d.max()
            L, B = d[band].max(), d[band].min()
            out[p] = (L - B) / (L + B)
        return out
