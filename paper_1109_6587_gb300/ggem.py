"""Thin Python binding of libggem (include/ggem.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
library.  Arrays may be torch CUDA tensors (passed as device pointers, the call
runs on the plan's stream) or numpy arrays (host pointers; the library stages
them and returns when the host output is written).  The library must be built
(``__graft_entry__.build()`` or ``python -m paper_1109_6587_gb300._build``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import pathlib

import numpy as np

_LIB_PATH = pathlib.Path(__file__).resolve().parent / "libggem.so"
_lib = None

GGEM_OK = 0
STATUS = {0: "GGEM_OK", 1: "GGEM_ERR_INVALID_ARG", 2: "GGEM_ERR_CAPACITY",
          3: "GGEM_ERR_CUDA", 4: "GGEM_ERR_NUMERICAL", 5: "GGEM_ERR_NOT_CONVERGED",
          6: "GGEM_OK_BREAKDOWN"}
GGEM_FP64, GGEM_MIXED, GGEM_FP64_EMULATED = 0, 1, 2
GGEM_NODAL, GGEM_ELEMENT = 0, 1


class GGEMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ggem_params(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_double), ("Lz", ctypes.c_double), ("W", ctypes.c_double),
                ("y0", ctypes.c_double), ("Nx", ctypes.c_int), ("Ny", ctypes.c_int),
                ("Nz", ctypes.c_int), ("alpha", ctypes.c_double),
                ("rcut_factor", ctypes.c_double), ("mu", ctypes.c_double),
                ("precision", ctypes.c_int), ("quadrature", ctypes.c_int),
                ("max_points", ctypes.c_int), ("max_tris", ctypes.c_int)]


EXPORTS = ["ggem_plan", "ggem_plan_destroy", "ggem_last_error", "ggem_plan_info",
           "ggem_mesh_set", "ggem_mesh_geometry", "ggem_point_forces", "ggem_local_sum",
           "ggem_single_layer",
           "ggem_double_layer", "ggem_trace_enable", "ggem_trace_stage_count",
           "ggem_trace_stage_name", "ggem_trace_read", "ggem_launch_count",
           "ggem_local_velocity_noalloc", "bie_solve", "ggem_solve_stats", "ggem_solve_guess",
           "ggem_mesh_particles", "ggem_mlp_features", "ggem_mlp_load", "ggem_mlp_save",
           "ggem_mlp_forward", "ggem_mlp_train", "ggem_mlp_guess", "ggem_bie_operator",
           "ggem_check", "ggem_rigid_solve", "ggem_membrane_reference",
           "ggem_membrane_traction", "ggem_undisturbed", "ggem_capsule_velocity",
           "ggem_capsule_step", "ggem_mesh_positions", "ggem_min_separation",
           "ggem_particle_volumes", "ggem_volume_correct", "ggem_overlap_correct",
           "ggem_set_offgrid", "ggem_mlp_precision", "ggem_precond_set",
           "ggem_precond_enable", "ggem_precond_block", "ggem_inject_tc_wait_expiry",
           "ggem_mlp_adam_state", "ggem_probe_l2_reduction",
           "ggem_probe_smem_reduction"]

GGEM_OFFGRID = {"lagrange": 0, "spectral": 1}

GGEM_FLOW = {"none": 0, "shear": 1, "poiseuille": 2}


class ggem_step_params(ctypes.Structure):
    _fields_ = [("flow", ctypes.c_int), ("strength", ctypes.c_double),
                ("shear_modulus", ctypes.c_double), ("dt", ctypes.c_double),
                ("tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("use_mlp", ctypes.c_int)]

MLP_MODEL_SIZE = 25 + 35075


def lib():
    """Load libggem.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise ImportError(f"{_LIB_PATH} is missing: build the CUDA library first "
                              "(python -m paper_1109_6587_gb300._build)")
        L = ctypes.CDLL(str(_LIB_PATH))
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.ggem_plan.argtypes = [ctypes.POINTER(ggem_params), P, ctypes.POINTER(P)]
        L.ggem_plan_destroy.argtypes = [P]
        L.ggem_last_error.argtypes = [P]
        L.ggem_last_error.restype = ctypes.c_char_p
        L.ggem_plan_info.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(D)]
        L.ggem_mesh_set.argtypes = [P, I, P, I, P]
        L.ggem_mesh_geometry.argtypes = [P, P, P]
        L.ggem_point_forces.argtypes = [P, I, P, P, I, P, I, P, P]
        L.ggem_local_sum.argtypes = [P, I, P, P, I, P, I, P, P]
        L.ggem_single_layer.argtypes = [P, P, P]
        L.ggem_double_layer.argtypes = [P, P, P]
        L.bie_solve.argtypes = [P, P, P, P, D, I, I, I, ctypes.POINTER(I), ctypes.POINTER(D)]
        L.ggem_solve_stats.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I),
                                       ctypes.POINTER(I)]
        L.ggem_solve_guess.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(D),
                                       ctypes.POINTER(D)]
        L.ggem_mesh_particles.argtypes = [P, I, P]
        L.ggem_mlp_features.argtypes = [P, P, P, P, ctypes.POINTER(D)]
        L.ggem_mlp_guess.argtypes = [P, P, P, P]
        L.ggem_bie_operator.argtypes = [P, P, P, P]
        L.ggem_check.argtypes = [P]
        L.ggem_rigid_solve.argtypes = [P, I, P, P, P, P, P, D, I, I, ctypes.POINTER(I),
                                       ctypes.POINTER(D)]
        SP = ctypes.POINTER(ggem_step_params)
        L.ggem_membrane_reference.argtypes = [P, P]
        L.ggem_membrane_traction.argtypes = [P, D, P]
        L.ggem_undisturbed.argtypes = [P, I, D, P, P]
        L.ggem_capsule_velocity.argtypes = [P, SP, P, P, P, ctypes.POINTER(I), ctypes.POINTER(D)]
        L.ggem_capsule_step.argtypes = [P, SP, P, P, P, ctypes.POINTER(I), ctypes.POINTER(D)]
        L.ggem_mesh_positions.argtypes = [P, P]
        L.ggem_min_separation.argtypes = [P, ctypes.POINTER(D)]
        L.ggem_particle_volumes.argtypes = [P, P]
        L.ggem_volume_correct.argtypes = [P, P, D, I, ctypes.POINTER(I)]
        L.ggem_overlap_correct.argtypes = [P, D, I, ctypes.POINTER(I)]
        L.ggem_set_offgrid.argtypes = [P, I, I]
        L.ggem_mlp_load.argtypes = [P, P, ctypes.c_size_t]
        L.ggem_mlp_precision.argtypes = [P, I]
        L.ggem_precond_set.argtypes = [P, I, P, I, P, D, I, I]
        L.ggem_precond_enable.argtypes = [P, I]
        L.ggem_precond_block.argtypes = [P, P]
        L.ggem_inject_tc_wait_expiry.argtypes = [ctypes.c_long]
        L.ggem_probe_l2_reduction.argtypes = [ctypes.c_long, I, P, ctypes.POINTER(D),
                                              ctypes.POINTER(D)]
        L.ggem_probe_smem_reduction.argtypes = [I, P, ctypes.POINTER(D), ctypes.POINTER(D)]
        L.ggem_mlp_adam_state.argtypes = [P, I, P, P, ctypes.POINTER(ctypes.c_longlong)]
        L.ggem_mlp_save.argtypes = [P, P, ctypes.c_size_t]
        L.ggem_mlp_forward.argtypes = [P, I, P, P]
        L.ggem_mlp_train.argtypes = [P, I, P, P, I, ctypes.c_ulonglong, I, I, D,
                                     ctypes.POINTER(D), P]
        L.ggem_trace_enable.argtypes = [P, I]
        L.ggem_trace_stage_count.argtypes = []
        L.ggem_trace_stage_name.argtypes = [I]
        L.ggem_trace_read.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_long)]
        L.ggem_launch_count.argtypes = [P, ctypes.POINTER(ctypes.c_long)]
        L.ggem_local_velocity_noalloc.argtypes = [ctypes.POINTER(ggem_params), P, I, P, P, I,
                                                  P, I, P]
        for name in EXPORTS:
            getattr(L, name).restype = (ctypes.c_char_p if name in ("ggem_last_error",
                                                                    "ggem_trace_stage_name")
                                         else ctypes.c_int)
        _lib = L
    return _lib


def _ptr(a, dtype):
    """(pointer, keep-alive) for a torch tensor or numpy array of the given dtype."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):                     # torch tensor
        import torch
        want = torch.float64 if dtype == np.float64 else torch.int32
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return ctypes.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), arr


def _check(status, plan):
    if status not in (0, 6):
        msg = lib().ggem_last_error(plan)
        raise GGEMError(status, msg.decode() if msg else "")
    return status


def _zeros_like_target(ref, shape):
    if hasattr(ref, "data_ptr"):
        import torch
        return torch.zeros(shape, dtype=torch.float64, device=ref.device)
    return np.zeros(shape)


class Plan:
    """A ggem plan (grid, tables, workspaces) bound to one CUDA stream.

    Lx, Lz, W, y0, Nx, Ny, Nz: periodic box, slit and grid (Nx, Nz powers of
    two, Ny Chebyshev-Lobatto nodes); alpha, rcut_factor: the GGEM split (0
    selects alpha = 1/(2h), r_cut = 4/alpha); mu: viscosity; precision: "fp64", "mixed" or
    "fp64_emulated"; quadrature: "nodal" or "element"; max_points, max_tris:
    capacities; stream: a CUDA stream handle (default torch's current one);
    offgrid: "lagrange" (5-point interpolation) or "spectral" (the expansion
    evaluated by a non-uniform FFT, half-width offgrid_width, 0 = default)."""

    def __init__(self, Lx, Lz, W, y0, Nx, Ny, Nz, alpha=0.0, rcut_factor=0.0, mu=1.0,
                 precision="fp64", quadrature="nodal", max_points=1 << 16, max_tris=0,
                 stream=None, offgrid="lagrange", offgrid_width=0):
        prec = {"fp64": GGEM_FP64, "mixed": GGEM_MIXED,
                "fp64_emulated": GGEM_FP64_EMULATED}[precision]
        quad = {"nodal": GGEM_NODAL, "element": GGEM_ELEMENT}[quadrature]
        self.params = ggem_params(Lx, Lz, W, y0, Nx, Ny, Nz, alpha, rcut_factor, mu, prec,
                                  quad, max_points, max_tris)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except Exception:
                stream = 0
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib().ggem_plan(ctypes.byref(self.params), ctypes.c_void_p(stream),
                               ctypes.byref(h)), None)
        self.h = h
        self.n_nodes = 0
        self.n_particles = 0
        if offgrid != "lagrange" or offgrid_width:
            self.set_offgrid(offgrid, offgrid_width)

    def set_offgrid(self, mode, half_width=0):
        """Off-grid evaluation of the global part: 'lagrange' (5-point, Sec.
        3.2.2) or 'spectral' (the expansion itself by a Gaussian-window
        non-uniform FFT, Sec. 3.2.3); half_width 0 = 12 (FP64) / 6 (mixed)."""
        _check(lib().ggem_set_offgrid(self.h, GGEM_OFFGRID[mode], int(half_width)), self.h)

    @classmethod
    def for_box(cls, box, **kw):
        return cls(box.Lx, box.Lz, box.W, box.y0, box.Nx, box.Ny, box.Nz, **kw)

    def close(self):
        if getattr(self, "h", None):
            lib().ggem_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        a, r = ctypes.c_double(), ctypes.c_double()
        _check(lib().ggem_plan_info(self.h, ctypes.byref(a), ctypes.byref(r)), self.h)
        return a.value, r.value

    def mesh_set(self, x, tri=None):
        n = int(x.shape[0])
        px, kx = _ptr(x, np.float64)
        pt, kt = _ptr(tri, np.int32)
        m = 0 if tri is None else int(tri.shape[0])
        _check(lib().ggem_mesh_set(self.h, n, px, m, pt), self.h)
        self.n_nodes = n
        self._mesh_ref = x

    def mesh_geometry(self):
        area = np.zeros(self.n_nodes)
        nrm = np.zeros((self.n_nodes, 3))
        _check(lib().ggem_mesh_geometry(self.h, ctypes.c_void_p(area.ctypes.data),
                                        ctypes.c_void_p(nrm.ctypes.data)), self.h)
        return area, nrm

    def point_forces(self, xs, g, xt=None, want_u=True, want_sigma=False, u=None, sigma=None):
        return self._pf(lib().ggem_point_forces, xs, g, xt, want_u, want_sigma, u, sigma)

    def local_sum(self, xs, g, xt=None, want_u=True, want_sigma=False, u=None, sigma=None):
        """Local part u^l, sigma^l alone (Eq. u_loc)."""
        return self._pf(lib().ggem_local_sum, xs, g, xt, want_u, want_sigma, u, sigma)

    def _pf(self, fn, xs, g, xt, want_u, want_sigma, u, sigma):
        ns = int(xs.shape[0])
        self_t = xt is None
        nt = ns if self_t else int(xt.shape[0])
        pxs, k1 = _ptr(xs, np.float64)
        pg, k2 = _ptr(g, np.float64)
        pxt, k3 = _ptr(xt, np.float64)
        if want_u and u is None:
            u = _zeros_like_target(xs, (nt, 3))
        if want_sigma and sigma is None:
            sigma = _zeros_like_target(xs, (nt, 6))
        pu, k4 = _ptr(u if want_u else None, np.float64)
        psg, k5 = _ptr(sigma if want_sigma else None, np.float64)
        _check(fn(self.h, ns, pxs, pg, nt, pxt, 1 if self_t else 0, pu, psg), self.h)
        return (u if want_u else None), (sigma if want_sigma else None)

    def _layer(self, fn, q, out):
        if out is None:
            out = _zeros_like_target(q, (self.n_nodes, 3))
        pq, k1 = _ptr(q, np.float64)
        po, k2 = _ptr(out, np.float64)
        _check(fn(self.h, pq, po), self.h)
        return out

    def trace(self, on=True):
        _check(lib().ggem_trace_enable(self.h, 1 if on else 0), self.h)

    def trace_read(self):
        """{stage: (total_ms, calls)} for stages that ran."""
        L = lib()
        out = {}
        for i in range(L.ggem_trace_stage_count()):
            ms, calls = ctypes.c_double(), ctypes.c_long()
            _check(L.ggem_trace_read(self.h, i, ctypes.byref(ms), ctypes.byref(calls)), self.h)
            if calls.value:
                out[L.ggem_trace_stage_name(i).decode()] = (ms.value, calls.value)
        return out

    def launch_count(self):
        n = ctypes.c_long()
        _check(lib().ggem_launch_count(self.h, ctypes.byref(n)), self.h)
        return n.value

    def single_layer(self, q, out=None):
        return self._layer(lib().ggem_single_layer, q, out)

    def double_layer(self, q, out=None):
        return self._layer(lib().ggem_double_layer, q, out)

    def bie_solve(self, kappa, b, q=None, tol=1e-6, restart=30, maxit=300, use_mlp=0,
                  check=True):
        """Solve (I + kappa/(4 pi) D) q = b (Sec. 5).  q (in: initial guess, b when
        None; out: the solution) is updated in place when given.  Returns
        (q, iterations, true relative residual, status); with check, an error
        status other than GGEM_ERR_NOT_CONVERGED raises."""
        if q is None:
            q = b.clone() if hasattr(b, "clone") else np.array(b, dtype=np.float64, copy=True)
        pk, kk = _ptr(kappa, np.float64)
        pb, kb = _ptr(b, np.float64)
        pq, kq = _ptr(q, np.float64)
        its = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = lib().bie_solve(self.h, pk, pb, pq, tol, restart, maxit, int(use_mlp),
                             ctypes.byref(its), ctypes.byref(rr))
        if check and st not in (0, 5, 6):
            _check(st, self.h)
        if kq is not q and not hasattr(q, "data_ptr"):
            q[...] = kq
        return q, its.value, rr.value, st

    def rigid_solve(self, centres, u_inf=None, ext=None, f=None, uo=None, tol=1e-6,
                    restart=30, maxit=300, check=True):
        """Tractions and rigid-body velocities of the particles set by
        mesh_particles (Sec. 6.1): centres [P, 3] reference points, u_inf
        [N, 3] undisturbed velocity at the nodes (None: 0), ext [P, 6] external
        force and torque (None: force- and torque-free).  f [N, 3] and uo
        [P, 6] (U, Omega) are the initial guess (zero when None) and are
        updated in place when given.  Returns (f, uo, iterations, true relative
        residual, status); with check, an error status other than
        GGEM_ERR_NOT_CONVERGED raises."""
        n_p = int(np.asarray(centres.cpu() if hasattr(centres, "cpu") else centres).reshape(-1, 3).shape[0])
        ref = u_inf if u_inf is not None else centres
        if f is None:
            f = _zeros_like_target(ref, (self.n_nodes, 3))
        if uo is None:
            uo = _zeros_like_target(ref, (n_p, 6))
        pc, kc = _ptr(centres, np.float64)
        pu, ku = _ptr(u_inf, np.float64)
        pe, ke = _ptr(ext, np.float64)
        pf, kf = _ptr(f, np.float64)
        po, ko = _ptr(uo, np.float64)
        its = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = lib().ggem_rigid_solve(self.h, n_p, pc, pu, pe, pf, po, tol, restart, maxit,
                                    ctypes.byref(its), ctypes.byref(rr))
        if check and st not in (0, 5, 6):
            _check(st, self.h)
        for out, keep in ((f, kf), (uo, ko)):
            if keep is not out and not hasattr(out, "data_ptr"):
                out[...] = keep
        return f, uo, its.value, rr.value, st

    # ------------------------------------------------------- capsule dynamics
    def membrane_reference(self, x_ref):
        """Stress-free shape of the membranes (same triangles as the mesh)."""
        px, kx = _ptr(x_ref, np.float64)
        _check(lib().ggem_membrane_reference(self.h, px), self.h)

    def membrane_traction(self, shear_modulus, out=None):
        """Traction jump Delta f [n, 3] of the neo-Hookean membranes (Sec. 4)."""
        if out is None:
            out = np.zeros((self.n_nodes, 3))
        po, ko = _ptr(out, np.float64)
        _check(lib().ggem_membrane_traction(self.h, float(shear_modulus), po), self.h)
        if ko is not out and not hasattr(out, "data_ptr"):
            out[...] = ko
        return out

    def undisturbed(self, flow, strength):
        """(u_inf, f_inf) [n, 3] at the nodes for flow 'none', 'shear' or
        'poiseuille' (App. B)."""
        u = np.zeros((self.n_nodes, 3))
        f = np.zeros((self.n_nodes, 3))
        _check(lib().ggem_undisturbed(self.h, GGEM_FLOW[flow], float(strength),
                                      u.ctypes.data_as(ctypes.c_void_p),
                                      f.ctypes.data_as(ctypes.c_void_p)), self.h)
        return u, f

    @staticmethod
    def _step_params(flow, strength, shear_modulus, dt, tol, restart, maxit, use_mlp):
        return ggem_step_params(GGEM_FLOW[flow], float(strength), float(shear_modulus),
                                float(dt), float(tol), int(restart), int(maxit), int(use_mlp))

    def capsule_velocity(self, lam, flow="none", strength=0.0, shear_modulus=1.0, q=None,
                         tol=1e-6, restart=30, maxit=300, use_mlp=0):
        """Node velocities of Eqs. (bi_ua), (qa) at the current mesh.  q (guess,
        zero when None) is updated in place when given.  Returns (u, q,
        iterations, true relative residual)."""
        n = self.n_nodes
        if q is None:
            q = np.zeros((n, 3))
        sp = self._step_params(flow, strength, shear_modulus, 0.0, tol, restart, maxit, use_mlp)
        pl, kl = _ptr(lam, np.float64)
        pq, kq = _ptr(q, np.float64)
        u = _zeros_like_target(q, (n, 3))
        pu, ku = _ptr(u, np.float64)
        its, rr = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(lib().ggem_capsule_velocity(self.h, ctypes.byref(sp), pl, pq, pu,
                                           ctypes.byref(its), ctypes.byref(rr)), self.h)
        for out, keep in ((q, kq), (u, ku)):
            if keep is not out and not hasattr(out, "data_ptr"):
                out[...] = keep
        return u, q, its.value, rr.value

    def capsule_step(self, lam, dt, flow="none", strength=0.0, shear_modulus=1.0, q=None,
                     tol=1e-6, restart=30, maxit=300, use_mlp=0):
        """One midpoint step (Sec. 5); the plan's mesh moves.  Returns (x_new
        [n, 3] numpy, q, iterations, larger true relative residual)."""
        n = self.n_nodes
        if q is None:
            q = np.zeros((n, 3))
        sp = self._step_params(flow, strength, shear_modulus, dt, tol, restart, maxit, use_mlp)
        pl, kl = _ptr(lam, np.float64)
        pq, kq = _ptr(q, np.float64)
        x = np.zeros((n, 3))
        its, rr = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(lib().ggem_capsule_step(self.h, ctypes.byref(sp), pl, pq,
                                       x.ctypes.data_as(ctypes.c_void_p), ctypes.byref(its),
                                       ctypes.byref(rr)), self.h)
        if kq is not q and not hasattr(q, "data_ptr"):
            q[...] = kq
        return x, q, its.value, rr.value

    def mesh_positions(self):
        x = np.zeros((self.n_nodes, 3))
        _check(lib().ggem_mesh_positions(self.h, x.ctypes.data_as(ctypes.c_void_p)), self.h)
        return x

    def min_separation(self):
        h = ctypes.c_double(0.0)
        _check(lib().ggem_min_separation(self.h, ctypes.byref(h)), self.h)
        return h.value

    def particle_volumes(self):
        v = np.zeros(self.n_particles)
        _check(lib().ggem_particle_volumes(self.h, v.ctypes.data_as(ctypes.c_void_p)), self.h)
        return v

    def volume_correct(self, v0, threshold=1e-4, max_passes=10):
        """Volume correction (Sec. 5); the plan's mesh moves.  Returns the
        passes made."""
        v = np.ascontiguousarray(v0, dtype=np.float64)
        k = ctypes.c_int(0)
        _check(lib().ggem_volume_correct(self.h, v.ctypes.data_as(ctypes.c_void_p),
                                         float(threshold), int(max_passes), ctypes.byref(k)),
               self.h)
        return k.value

    def overlap_correct(self, h_min, max_sweeps=100):
        """Minimum-gap correction (Sec. 7.1); the plan's mesh moves.  Returns
        the pair moves made."""
        k = ctypes.c_int(0)
        _check(lib().ggem_overlap_correct(self.h, float(h_min), int(max_sweeps),
                                          ctypes.byref(k)), self.h)
        return k.value

    def check(self):
        """Raise if a device-side wait of the plan's kernels expired."""
        _check(lib().ggem_check(self.h), self.h)

    def solve_guess(self):
        """(started from the learned guess, relative residual of the caller's
        guess, relative residual of the learned guess) of the last bie_solve."""
        u, a, b = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        _check(lib().ggem_solve_guess(self.h, ctypes.byref(u), ctypes.byref(a),
                                      ctypes.byref(b)), self.h)
        return bool(u.value), a.value, b.value

    # ---------------------------------------------------- learned warm start
    def mesh_particles(self, particle, n_particles=None):
        part = np.ascontiguousarray(np.asarray(particle.cpu() if hasattr(particle, "cpu")
                                               else particle), dtype=np.int32)
        n_p = int(part.max()) + 1 if n_particles is None else int(n_particles)
        _check(lib().ggem_mesh_particles(self.h, n_p, part.ctypes.data_as(ctypes.c_void_p)),
               self.h)
        self.n_particles = n_p

    def mlp_features(self, kappa, r):
        """(features [n, 12] numpy, s = rms(r)) of the right-hand side r."""
        n = self.n_nodes
        out = np.zeros((n, 12))
        pk, kk = _ptr(kappa, np.float64)
        pr, kr = _ptr(r, np.float64)
        sc = ctypes.c_double(0.0)
        _check(lib().ggem_mlp_features(self.h, pk, pr, out.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.byref(sc)), self.h)
        return out, sc.value

    def mlp_guess(self, kappa, r, out=None):
        """The learned estimate of A^-1 r."""
        return self._apply3(lib().ggem_mlp_guess, kappa, r, out)

    def bie_operator(self, kappa, q, out=None):
        """(I + kappa/(4 pi) D) q."""
        return self._apply3(lib().ggem_bie_operator, kappa, q, out)

    def _apply3(self, fn, kappa, v, out):
        if out is None:
            out = _zeros_like_target(v, (self.n_nodes, 3))
        pk, kk = _ptr(kappa, np.float64)
        pv, kv = _ptr(v, np.float64)
        po, ko = _ptr(out, np.float64)
        _check(fn(self.h, pk, pv, po), self.h)
        if ko is not out and not hasattr(out, "data_ptr"):
            out[...] = ko
        return out

    def precond_set(self, x_ref, tri_ref, kappa, ref_nx=0, ref_nz=0):
        """Build and enable the per-particle block preconditioner of the
        Fredholm solve from one reference capsule (nodes x_ref [n, 3], any
        origin; triangles tri_ref [m, 3]).  ref_nx / ref_nz = 0 pick the
        smallest power of two >= 16 whose cell spans the capsule plus 2 r_cut
        in that direction."""
        x = np.ascontiguousarray(np.asarray(x_ref, dtype=np.float64))
        t = np.ascontiguousarray(np.asarray(tri_ref, dtype=np.int32))
        prm = self.params
        _, rc = self.info()

        def pick(extent, dx):
            nx = 16
            while nx * dx < extent + 2.0 * rc:
                nx *= 2
            return nx
        ext = x.max(0) - x.min(0)
        nx = ref_nx or pick(ext[0], prm.Lx / prm.Nx)
        nz = ref_nz or pick(ext[2], prm.Lz / prm.Nz)
        _check(lib().ggem_precond_set(self.h, x.shape[0], x.ctypes.data_as(ctypes.c_void_p),
                                      t.shape[0], t.ctypes.data_as(ctypes.c_void_p),
                                      float(kappa), int(nx), int(nz)), self.h)
        self._pc_n = x.shape[0]
        return nx, nz

    def precond_enable(self, on=True):
        _check(lib().ggem_precond_enable(self.h, int(bool(on))), self.h)

    def precond_block(self):
        """The block B = (I + kappa/4 pi D_ref)^-1 [3 n_ref, 3 n_ref] (FP64)."""
        n3 = 3 * getattr(self, "_pc_n", 0)
        out = np.zeros((n3, n3))
        _check(lib().ggem_precond_block(self.h, out.ctypes.data_as(ctypes.c_void_p)), self.h)
        return out

    def mlp_precision(self, mode):
        """Network arithmetic: "bf16" (the bfloat16 rounding points, default) or
        "fp32" (none)."""
        _check(lib().ggem_mlp_precision(self.h, {"bf16": 0, "fp32": 1}[mode]), self.h)

    def mlp_load(self, model):
        m = np.ascontiguousarray(np.asarray(model), dtype=np.float64)
        _check(lib().ggem_mlp_load(self.h, m.ctypes.data_as(ctypes.c_void_p), m.size), self.h)

    def mlp_save(self):
        m = np.zeros(MLP_MODEL_SIZE)
        _check(lib().ggem_mlp_save(self.h, m.ctypes.data_as(ctypes.c_void_p), m.size), self.h)
        return m

    def mlp_adam_state(self, state=None):
        """The model's Adam moments and step count (m, v, step); with state =
        (m, v, step), replace them instead."""
        st = ctypes.c_longlong(0)
        if state is None:
            m, v = np.zeros(35075), np.zeros(35075)
            _check(lib().ggem_mlp_adam_state(self.h, 0, m.ctypes.data_as(ctypes.c_void_p),
                                             v.ctypes.data_as(ctypes.c_void_p),
                                             ctypes.byref(st)), self.h)
            return m, v, int(st.value)
        m = np.ascontiguousarray(state[0], dtype=np.float64)
        v = np.ascontiguousarray(state[1], dtype=np.float64)
        st.value = int(state[2])
        _check(lib().ggem_mlp_adam_state(self.h, 1, m.ctypes.data_as(ctypes.c_void_p),
                                         v.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st)),
               self.h)

    def mlp_forward(self, feat):
        f = np.ascontiguousarray(np.asarray(feat.cpu() if hasattr(feat, "cpu") else feat),
                                 dtype=np.float64)
        out = np.zeros((f.shape[0], 3))
        _check(lib().ggem_mlp_forward(self.h, f.shape[0], f.ctypes.data_as(ctypes.c_void_p),
                                      out.ctypes.data_as(ctypes.c_void_p)), self.h)
        return out

    def mlp_train(self, feat, target, init=True, seed=0, epochs=10, batch=2048, lr=1e-3,
                  want_grad=False):
        """Train (or, with epochs=0, evaluate the full-batch loss and gradient).
        Returns loss, or (loss, gradient) with want_grad."""
        pf, kf = _ptr(feat, np.float64)
        pt, kt = _ptr(target, np.float64)
        n = int(feat.shape[0])
        loss = ctypes.c_double(0.0)
        grad = np.zeros(35075) if want_grad else None
        pg = grad.ctypes.data_as(ctypes.c_void_p) if want_grad else None
        _check(lib().ggem_mlp_train(self.h, n, pf, pt, int(bool(init)), int(seed), int(epochs),
                                    int(batch), float(lr), ctypes.byref(loss), pg), self.h)
        return (loss.value, grad) if want_grad else loss.value

    def solve_stats(self):
        """(GMRES cycles, FP64 operator applications, mixed operator applications)
        of the last bie_solve or rigid_solve."""
        c, a, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().ggem_solve_stats(self.h, ctypes.byref(c), ctypes.byref(a),
                                      ctypes.byref(b)), self.h)
        return c.value, a.value, b.value


# The C names, for callers that prefer them.
def ggem_plan(box_or_params, **kw):
    return Plan.for_box(box_or_params, **kw)


def ggem_single_layer(plan, q, out=None):
    return plan.single_layer(q, out)


def ggem_double_layer(plan, q, out=None):
    return plan.double_layer(q, out)


def bie_solve(plan, kappa, b, q=None, tol=1e-6, restart=30, maxit=300, use_mlp=False):
    return plan.bie_solve(kappa, b, q, tol, restart, maxit, use_mlp)


def ggem_rigid_solve(plan, centres, u_inf=None, ext=None, f=None, uo=None, tol=1e-6,
                     restart=30, maxit=300):
    return plan.rigid_solve(centres, u_inf, ext, f, uo, tol, restart, maxit)


def ggem_point_forces(plan, xs, g, xt=None, want_u=True, want_sigma=False):
    return plan.point_forces(xs, g, xt, want_u, want_sigma)


def ggem_mesh_set(plan, x, tri=None):
    return plan.mesh_set(x, tri)


def probe_l2_reduction(nvec=1 << 21, iters=256, stream=None):
    """Throughput of float4 vector reductions into an L2-resident buffer
    (ggem_probe_l2_reduction): (milliseconds, vector reductions per second)."""
    ms, rate = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = lib().ggem_probe_l2_reduction(int(nvec), int(iters), ctypes.c_void_p(stream or 0),
                                       ctypes.byref(ms), ctypes.byref(rate))
    if st != 0:
        raise GGEMError(st, "L2 reduction probe failed")
    return ms.value, rate.value


def probe_smem_reduction(iters=4096, stream=None):
    """Throughput of FP32 atomic adds into shared memory
    (ggem_probe_smem_reduction): (milliseconds, scalar adds per second)."""
    ms, rate = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = lib().ggem_probe_smem_reduction(int(iters), ctypes.c_void_p(stream or 0),
                                         ctypes.byref(ms), ctypes.byref(rate))
    if st != 0:
        raise GGEMError(st, "shared-memory reduction probe failed")
    return ms.value, rate.value
