"""Benchmark of the GGEM slit operators and Fredholm solve on GB300.

Step: one pass of the matvec hot path over the workload -- the single-layer
and the double-layer operators evaluated at every node (Sec. 3.4, 3.5 of
Kumar & Graham, arXiv 1109.6587) for fresh N(0,1) densities.

Workload (default): 100 spherical capsules x 642 nodes = 64,200 points in a
40 x [-5,5] x 40 slit, grid 128 x 65 x 128, mixed precision, element
quadrature (the paper's layer rule; --quadrature nodal for point forces).
Metric: Mpts/s = nodes / (time of one single + one double layer evaluation).
The second half of the metric -- GMRES iterations and seconds per Fredholm
solve at true relative residual 1e-6, per emulated time step, for the plain
FP64 solve, the mixed solve and the mixed solve with the learned warm start
-- is measured on the same workload and reported under "solve".

Other workloads (--workload capsules1000 or rbc4000: 642,000 and 2,568,000
points; capsules100_phi and capsules1000_phi: the 100- and 1000-capsule slits
filled to volume fractions 0.1 and 0.2, 245,244 and 3,923,904 points) measure
the same step at the larger configurations; the pair counts of their roofline
are taken on a sample of 20,000 targets.

The off-grid evaluation of the global part is the paper's 5-point Lagrange
interpolation by default; --offgrid spectral times the spectrally accurate
evaluation instead, and the default run reports the other mode's step under
"offgrid_other".

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
For N > 1 under torchrun each rank runs an independent replica on its own
GPU (the evaluation is one problem per GPU; no collective), value = sum of
the ranks' points / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GGEM slit matvec Mpts/s; GMRES iters & s/solve, learned vs plain at 1e-6"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp64_emulated"])
    ap.add_argument("--quadrature", default="element", choices=["nodal", "element"])
    ap.add_argument("--workload", default="capsules100",
                    choices=["capsules100", "capsules1000", "rbc4000", "capsules100_phi",
                             "capsules1000_phi"],
                    help="capsules100 (default, the benchmark configuration), capsules1000 "
                         "(642,000 points), rbc4000 (2,568,000 points), capsules100_phi / "
                         "capsules1000_phi (the same slits at volume fractions 0.1 / 0.2); "
                         "the CPU baseline runs on the default only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--offgrid", default="lagrange", choices=["lagrange", "spectral"],
                    help="off-grid evaluation of the global part (5-point Lagrange or the "
                         "spectral non-uniform FFT evaluation)")
    return ap.parse_args()


WORKLOADS = {
    "capsules100": ("capsules_100",
                    "100 spherical capsules x 642 nodes (64,200 points), slit 40 x [-5,5] x 40"),
    "capsules1000": ("capsules_1000",
                     "1000 spherical capsules x 642 nodes (642,000 points), slit 80 x [-10,10] x 80"),
    "rbc4000": ("rbc_4000",
                "4000 biconcave capsules x 642 nodes (2,568,000 points), slit 150 x [-15,15] x 150"),
    "capsules100_phi": ("capsules_100_phi",
                        "382 spherical capsules x 642 nodes (245,244 points) at volume "
                        "fraction 0.1, slit 40 x [-5,5] x 40"),
    "capsules1000_phi": ("capsules_1000_phi",
                         "6112 spherical capsules x 642 nodes (3,923,904 points) at volume "
                         "fraction 0.2, slit 80 x [-10,10] x 80"),
}


def _workload(args=None):
    from paper_1109_6587_gb300 import workloads as W
    name = "capsules100" if args is None else args.workload
    return getattr(W, WORKLOADS[name][0])(seed=0)


def _config(susp, args):
    b = susp.box
    return {"workload": WORKLOADS[args.workload][1],
            "n_points": int(susp.x.shape[0]), "grid": [b.Nx, b.Ny, b.Nz],
            "precision": args.precision, "quadrature": args.quadrature,
            "offgrid": args.offgrid,
            "step": "single-layer + double-layer matvec",
            "l2": "flushed (256 MiB write) before every timed step",
            "parallelism": f"replicas x{args.gpus}"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) > 8:
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


SAMPLE_ABOVE = 100_000      # larger workloads count pairs on a sample of targets
SAMPLE_TARGETS = 20_000


def _target_sample(n):
    """All targets, or a seeded sample of SAMPLE_TARGETS of them for large
    workloads; returns (indices, scale to all targets)."""
    if n <= SAMPLE_ABOVE:
        return np.arange(n), 1.0
    idx = np.sort(np.random.default_rng(7).choice(n, SAMPLE_TARGETS, replace=False))
    return idx, n / SAMPLE_TARGETS


def _pair_count(susp, rcut):
    """Number of (target, source) pairs with 0 < r < r_cut (minimum image in x,
    z); counted on a sample of targets for large workloads."""
    from scipy.spatial import cKDTree
    b = susp.box
    x = susp.x.copy()
    x[:, 0] %= b.Lx
    x[:, 2] %= b.Lz
    x[:, 1] -= b.y0
    box = [b.Lx, 4 * b.W + 4 * rcut, b.Lz]
    idx, scale = _target_sample(len(x))
    tree = cKDTree(x, boxsize=box)
    # every sampled target counts itself once at r = 0
    return int(scale * (cKDTree(x[idx], boxsize=box).count_neighbors(tree, rcut) - len(idx)))


def _quad_points(susp):
    """The 16 collapsed-Gauss points of every triangle (Sec. 3.4.1) and the
    triangle each belongs to."""
    t, w = np.polynomial.legendre.leggauss(4)
    t = 0.5 * (t + 1.0)
    eta = np.repeat(t, 4)
    xi = (1.0 - eta) * np.tile(t, 4)
    p = np.stack([1.0 - xi - eta, xi, eta], 1)                    # [16, 3]
    X = susp.x[susp.tri]                                           # [m, 3, 3]
    return np.einsum("qv,mvc->mqc", p, X).reshape(-1, 3), np.repeat(np.arange(len(susp.tri)), 16)


def _elem_pair_count(susp, rcut):
    """(node, quadrature point) pairs with 0 < r < r_cut, minimum image in x, z,
    less the points of triangles that contain the node (polar rule instead)."""
    from scipy.spatial import cKDTree
    b = susp.box
    qx, qt = _quad_points(susp)

    def wrap(a):
        a = a.copy()
        a[:, 0] %= b.Lx
        a[:, 2] %= b.Lz
        a[:, 1] -= b.y0
        return a
    box = [b.Lx, 4 * b.W + 4 * rcut, b.Lz]
    idx, scale = _target_sample(len(susp.x))
    tq = cKDTree(wrap(qx), boxsize=box)
    tn = cKDTree(wrap(susp.x[idx]), boxsize=box)
    total = int(tn.count_neighbors(tq, rcut))
    # the 16 points of each triangle containing a (sampled) node are the polar rule's
    own = np.bincount(susp.tri.ravel(), minlength=len(susp.x))[idx].sum()
    return int(scale * (total - 16 * own))


def aggregate(t_ms, steps, n_points, world, device):
    """Whole-job throughput of independent replicas: the slowest rank's time
    (max over ranks) and the points of all ranks.  Returns (ms per step,
    Mpts/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
        dist.barrier()
    ms_step = t_ms / steps
    return ms_step, world * n_points / (ms_step * 1e-3) / 1e6


def run_mine(args, rank, world):
    import torch
    from paper_1109_6587_gb300 import ggem

    torch.cuda.set_device(rank % max(1, torch.cuda.device_count()))
    dev = torch.device("cuda")
    susp = _workload(args)
    n = susp.x.shape[0]
    P = ggem.Plan.for_box(susp.box, precision=args.precision, quadrature=args.quadrature,
                          max_points=n, max_tris=susp.tri.shape[0], offgrid=args.offgrid)
    P.mesh_set(torch.as_tensor(susp.x, device=dev), torch.as_tensor(susp.tri, device=dev))
    rng = np.random.default_rng(1234 + rank)
    qs = [torch.as_tensor(rng.standard_normal((n, 3)), device=dev) for _ in range(4)]
    w = torch.empty((n, 3), dtype=torch.float64, device=dev)
    v = torch.empty_like(w)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(i):
        P.single_layer(qs[i % 4], w)
        P.double_layer(qs[i % 4], v)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    l0 = P.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step(i)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    launches = P.launch_count() - l0
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_step, value = aggregate(t_ms, args.steps, n, world, dev)

    # per-stage device times (traced pass, same stream)
    P.trace(True)
    for i in range(args.steps):
        flush.zero_()
        step(i)
    torch.cuda.synchronize()
    stages = P.trace_read()
    P.trace(False)

    # end to end through the C ABI with host buffers (copies inside the timer)
    qh = [np.ascontiguousarray(q.cpu().numpy()) for q in qs]
    wh = np.empty((n, 3))
    vh = np.empty((n, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        P.single_layer(qh[i % 4], wh)
        P.double_layer(qh[i % 4], vh)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    return dict(n=n, value=value, ms_step=ms_step, launches=launches, clocks=clk.summary(),
                stages=stages, e2e_s=e2e_s, susp=susp, P=P)


def roofline(res, args):
    """The stage with the most device time against the bound of its kernel:
    the local sum against the FP32 issue rate (algorithmic flops per pair x
    the pairs within r_cut), the other stages against HBM bandwidth
    (algorithmic bytes of one launch)."""
    peaks, kind = _peaks()
    stages = res["stages"]
    name, (tot, calls) = max(stages.items(), key=lambda kv: kv[1][0])
    avg_s = tot / calls * 1e-3
    susp = res["susp"]
    a, rc = res["P"].info()
    n = res["n"]
    b = susp.box
    esz = 4 if args.precision == "mixed" else 8
    plane = b.Nz * b.Nx
    if name == "local_sum":
        pairs = _elem_pair_count(susp, rc) if args.quadrature == "element" else _pair_count(susp, rc)
        # FP32 operations per pair of the kernel's formula (distance, rsqrt and
        # exp2 as one each, the 17-FMA erfcx polynomial, the G^l or n.T^l
        # contraction): single layer 74, double layer 99; the stage averages
        # one launch of each
        flops = pairs * (74.0 + 99.0) / 2.0
        sm_mhz = res["clocks"]["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ach = flops / avg_s / 1e12
        if args.precision != "mixed":
            peak = 1.25           # FP64-accurate work against the nominal FP64 rate
        # dram read + write bytes of one double-layer launch of the mixed
        # element-rule kernel on this workload, from one ncu capture of that
        # launch (its ncu summary is kept with the profiles); other
        # configurations have no capture
        traffic = (94.9e6 + 4.2e6) if (args.precision == "mixed"
                                       and args.quadrature == "element"
                                       and args.workload == "capsules100") else None
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"
                if args.precision == "mixed" else
                "nominal FP64 (the emulated kernel issues FP32 pair arithmetic)"
                if args.precision == "fp64_emulated" else "nominal FP64"}
    # memory-bound stages: algorithmic bytes per launch
    ncomp_out = 4.5  # average of single (3) and double (6) outputs
    bytes_per = {
        "fft_forward": 2 * 2 * (3 * b.Ny + 6) * plane * esz,
        "fft_inverse": 2 * 2 * ncomp_out * b.Ny * plane * esz,
        "cheb_forward": 2 * 3 * b.Ny * plane * esz,
        "cheb_inverse": 2 * ncomp_out * b.Ny * plane * esz,
        "tau_solve": (3 + ncomp_out) * b.Ny * plane * esz + 3 * b.Ny * (plane // 2) * 8,
        "spread": 3 * b.Ny * plane * esz + n * 32,
        "interpolate": ncomp_out * b.Ny * plane * esz + n * 48,
        "wall_local_sum": 6 * plane * esz + n * 32,
    }.get(name, 0)
    ach = bytes_per / avg_s / 1e9
    peak = peaks["hbm_gbs"]
    return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "traffic": None, "peak_source": kind}


def cpu_baseline(susp, args, stride=64):
    """The FP64 oracle as it stands on the host cores, on a bounded sample:
    the single and double layer with their full global parts, the local part
    at every stride-th node, scaled to all nodes."""
    from oracle import oracle as O
    q = np.random.default_rng(99).standard_normal((susp.x.shape[0], 3))
    n = susp.x.shape[0]
    idx = np.arange(0, n, stride)
    a = O.default_alpha(susp.box)
    rc = O.default_rcut(a)
    _, _, _, nb = O.geometry(susp.x, susp.tri)
    t0 = time.perf_counter()
    O.single_layer(susp, q, quadrature=args.quadrature, targets=idx, offgrid=args.offgrid)
    O.double_layer(susp, q, quadrature=args.quadrature, targets=idx, offgrid=args.offgrid)
    t_sample = time.perf_counter() - t0
    t0 = time.perf_counter()
    if args.quadrature == "element":
        O.local_elem(susp.box, a, rc, 0, susp.x, susp.tri, q, targets=idx)
        O.local_elem(susp.box, a, rc, 1, susp.x, susp.tri, q, nrm=nb, targets=idx)
    else:
        g = 8.0 * math.pi * np.asarray(O.geometry(susp.x, susp.tri)[2])[:, None] * q
        O.local_point(susp.box, a, rc, 1.0, susp.x, g, susp.x[idx], want_u=True,
                      want_sig=True)
    t_local = time.perf_counter() - t0
    dt = t_sample + t_local * (n / len(idx) - 1.0)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": n / dt / 1e6, "unit": "Mpts/s", "cores": cores,
            "kind": "oracle", "seconds": dt, "measured_seconds": t_sample + t_local,
            "sample": f"FP64 single + double layer ({args.quadrature} quadrature, "
                      f"{args.offgrid} off-grid evaluation): both global parts in full, the "
                      f"local part at every {stride}th node ({len(idx)} of {n}) scaled to "
                      f"all nodes; OpenMP over targets"}


def solve_metrics(args, susp, dev, train_steps=3, timed_steps=2):
    """GMRES iterations and seconds per Fredholm solve (Sec. 5) at true relative
    residual 1e-6, per emulated time step of the workload (capsules moved
    rigidly by 0.01 radius per step, membrane load drifting; kappa = 2/3,
    viscosity ratio 5; b from Eq. (qa)), each step solved from the previous
    step's density:
      fp64   plain GMRES with the FP64 operator;
      fp64_emulated  plain GMRES with the FP64-accurate operator whose
             element-rule local sum runs in double-float arithmetic;
      mixed  mixed operator with FP64 refinement;
      mixed_learned  mixed, starting from the learned guess when its residual
             is lower (the network trained on steps 0..train_steps-1 of the
             same run, as a running simulation would).
    Steps train_steps .. train_steps + timed_steps - 1 are timed."""
    import torch
    from paper_1109_6587_gb300 import ggem
    from paper_1109_6587_gb300 import warmstart as WS

    n = susp.x.shape[0]
    mk = lambda prec: ggem.Plan.for_box(susp.box, precision=prec, quadrature=args.quadrature,
                                        max_points=n, max_tris=susp.tri.shape[0])
    Pm = mk("mixed")
    t0 = time.perf_counter()
    recs = WS.solve_series(Pm, susp, train_steps, seed=500, collect=True)
    F = np.concatenate([f for r in recs for f, _ in r["samples"]])
    T = np.concatenate([t for r in recs for _, t in r["samples"]])
    t1 = time.perf_counter()
    loss = WS.train(Pm, F, T, seed=1, epochs=20, batch=2048, lr=1e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    out = {"tol": 1e-6, "kappa": 2.0 / 3.0, "rhs": "Eq. (qa), synthetic membrane load + shear",
           "guess": "previous step's density", "restart": 30, "quadrature": args.quadrature,
           "steps_timed": timed_steps,
           "training": {"samples": int(F.shape[0]), "data_s": t1 - t0, "train_s": t2 - t1,
                        "loss": loss, "epochs": 20}}
    P64 = mk("fp64")
    Pem = mk("fp64_emulated")
    variants = (("fp64", P64, 0), ("fp64_emulated", Pem, 0), ("mixed", Pm, 0),
                ("mixed_learned", Pm, 1))
    for name, P, use in variants:
        total = train_steps + timed_steps
        # the series up to the last training step, untimed (warm state), then timed steps
        q_prev = None
        tri = torch.as_tensor(susp.tri, device=dev)
        times, its, rrs, used = [], [], [], []
        for t in range(total):
            s = W_rigid(susp, t)
            kappa, b = W_rhs(s, t)
            P.mesh_set(torch.as_tensor(s.x, device=dev), tri)
            P.mesh_particles(s.particle, len(s.centres))
            kd = torch.as_tensor(kappa, device=dev)
            bd = torch.as_tensor(b, device=dev)
            q0 = bd.clone() if q_prev is None else q_prev.clone()
            timed = t >= train_steps
            if name.startswith("fp64") and not timed and t < train_steps - 1:
                q_prev = None          # FP64 plain: only the last untimed step is needed
                continue
            torch.cuda.synchronize()
            a = time.perf_counter()
            q, it, rr, st = P.bie_solve(kd, bd, q=q0, tol=1e-6, use_mlp=use if timed else 0)
            torch.cuda.synchronize()
            if timed:
                times.append(time.perf_counter() - a)
                its.append(it)
                rrs.append(rr)
                used.append(P.solve_guess()[0])
            q_prev = q
        cyc, m64, mmix = P.solve_stats()
        out[name] = {"iters": float(np.mean(its)), "s_per_solve": float(np.mean(times)),
                     "true_relres_max": float(np.max(rrs)), "learned_guess_used": used,
                     "last_solve_matvec_fp64": m64, "last_solve_matvec_mixed": mmix}
        P.check()
    Pm.close()
    P64.close()
    Pem.close()
    out["speedup_mixed_vs_fp64"] = out["fp64"]["s_per_solve"] / out["mixed"]["s_per_solve"]
    out["speedup_learned_vs_fp64"] = (out["fp64"]["s_per_solve"] /
                                      out["mixed_learned"]["s_per_solve"])
    return out


def dynamics_metrics(args, susp, dev, warm=1, timed=3):
    """Capsule time steps of the workload (Sec. 5, 7.1): simple shear of rate
    1, viscosity ratio 5, Ca = 0.3, membranes stress-free in the initial
    spherical shape.  One step: the dt rule from the smallest node
    separation, the midpoint step (per stage: traction jump, right side of
    Eq. (qa), Fredholm solve to 1e-6 from the previous density, single
    layer), the volume correction and the minimum-gap correction.  `warm`
    untimed steps, then `timed` timed ones; mixed precision."""
    import torch
    from paper_1109_6587_gb300 import dynamics as D
    from paper_1109_6587_gb300 import ggem

    n = susp.x.shape[0]
    P = ggem.Plan.for_box(susp.box, precision="mixed", quadrature=args.quadrature,
                          max_points=n, max_tris=susp.tri.shape[0])
    P.mesh_set(torch.as_tensor(susp.x, device=dev), torch.as_tensor(susp.tri, device=dev))
    S = D.Suspension(P, susp.particle, len(susp.centres), lam=np.full(len(susp.centres), 5.0),
                     ca=0.3, flow="shear", strength=1.0)
    for _ in range(warm):
        S.step()
    recs = [S.step() for _ in range(timed)]
    P.check()
    out = {"flow": "simple shear, rate 1", "lambda": 5.0, "Ca": 0.3, "tol": 1e-6,
           "steps_timed": timed, "s_per_step": float(np.mean([r["seconds"] for r in recs])),
           "gmres_iters_per_step": float(np.mean([r["iters"] for r in recs])),
           "dt": float(np.mean([r["dt"] for r in recs])),
           "volume_passes": int(sum(r["volume_passes"] for r in recs)),
           "overlap_moves": int(sum(r["overlap_moves"] for r in recs)),
           "taylor_D_mean": float(S.deformation().mean()), "strain": S.t}
    P.close()
    return out


def offgrid_metrics(args, susp, dev, warm=3, timed=10):
    """The same step with the other off-grid evaluation (spectral when the
    main line uses Lagrange interpolation, and vice versa): step time and the
    stage times it changes."""
    import torch
    from paper_1109_6587_gb300 import ggem
    other = "spectral" if args.offgrid == "lagrange" else "lagrange"
    n = susp.x.shape[0]
    P = ggem.Plan.for_box(susp.box, precision=args.precision, quadrature=args.quadrature,
                          max_points=n, max_tris=susp.tri.shape[0], offgrid=other)
    P.mesh_set(torch.as_tensor(susp.x, device=dev), torch.as_tensor(susp.tri, device=dev))
    rng = np.random.default_rng(77)
    q = torch.as_tensor(rng.standard_normal((n, 3)), device=dev)
    w = torch.empty((n, 3), dtype=torch.float64, device=dev)
    v = torch.empty_like(w)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        P.single_layer(q, w)
        P.double_layer(q, v)
    torch.cuda.synchronize()
    t_ms = 0.0
    for _ in range(timed):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        P.single_layer(q, w)
        P.double_layer(q, v)
        b.record(stream)
        torch.cuda.synchronize()
        t_ms += a.elapsed_time(b)
    P.trace(True)
    for _ in range(timed):
        flush.zero_()
        P.single_layer(q, w)
        P.double_layer(q, v)
    torch.cuda.synchronize()
    st = P.trace_read()
    P.trace(False)
    ms = t_ms / timed
    out = {"offgrid": other, "ms_per_step": ms, "value": n / (ms * 1e-3) / 1e6,
           "unit": "Mpts/s"}
    for k in ("fft_inverse", "interpolate"):
        if k in st:
            out[k + "_ms"] = st[k][0] / st[k][1]
    P.close()
    return out


def W_rigid(susp, t):
    from paper_1109_6587_gb300 import workloads as W
    return W.rigid_step(susp, seed=500, step=t) if t else susp


def W_rhs(s, t):
    from paper_1109_6587_gb300 import workloads as W
    return W.bie_rhs(s, seed=500, step=t)


def main():
    args = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return
        susp = _workload(args)
        times = []
        for _ in range(args.warmup):
            pass       # the oracle has no warm-up state
        cb = None
        for _ in range(max(1, min(args.steps, 3))):
            cb = cpu_baseline(susp, args)
            times.append(cb["seconds"])
        ms = float(np.median(times)) * 1e3
        val = susp.x.shape[0] / (ms * 1e-3) / 1e6
        cb["value"] = val
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpts/s",
                "n_gpus": args.gpus, "steps": len(times), "warmup": 0, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": _config(susp, args),
                "cpu_baseline": cb,
                "e2e": {"value": val, "unit": "Mpts/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res = run_mine(args, rank, world)
    n = res["n"]
    line = {"metric": METRIC, "value": res["value"], "unit": "Mpts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "f32+f64", "fp64": "f64",
                      "fp64_emulated": "f32-pair+f64"}[args.precision],
            "data": "synthetic", "config": _config(res["susp"], args),
            "e2e": {"value": world * n / res["e2e_s"] / 1e6, "unit": "Mpts/s",
                    "h2d_bytes_per_step": 2 * n * 3 * 8, "d2h_bytes_per_step": 2 * n * 3 * 8},
            "gpu_launches": res["launches"], "clocks": res["clocks"],
            "stages_ms": {k: v[0] / v[1] for k, v in res["stages"].items()}}
    line["roofline"] = roofline(res, args)
    if not args.no_solve:
        import torch
        line["solve"] = solve_metrics(args, res["susp"], torch.device("cuda"))
        line["dynamics"] = dynamics_metrics(args, res["susp"], torch.device("cuda"))
        line["offgrid_other"] = offgrid_metrics(args, res["susp"], torch.device("cuda"))
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "capsules100":
        line["cpu_baseline"] = cpu_baseline(res["susp"], args)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
