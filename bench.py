"""Benchmark of the GGEM slit operators and Fredholm solve on GB300.

Step: one pass of the matvec hot path over the workload -- the single-layer
and the double-layer operators evaluated at every node (Sec. 3.4, 3.5 of
Kumar & Graham, arXiv 1109.6587) for fresh N(0,1) densities.

Workload (default): 4000 biconcave capsules x 642 nodes = 2,568,000 points in
a 150 x [-15,15] x 150 slit, grid 512 x 129 x 512, mixed precision, element
quadrature (the paper's layer rule; --quadrature nodal for point forces).
Metric: Mpts/s = nodes / (time of one single + one double layer evaluation).
The second half of the metric -- GMRES iterations and seconds per Fredholm
solve at true relative residual 1e-6 -- is reported under "solve" on the
1000-capsule workload (642,000 points, viscosity ratio 5) per emulated time
step for the plain FP64 solve, the FP64-accurate emulated one and the mixed
solve with and without the per-particle block preconditioner and the
learned warm start (trained on generated suspensions), and under "dynamics"
as seconds per capsule time step of the default workload in shear.

Other workloads (--workload capsules100 or capsules1000: 64,200 and 642,000
points; capsules100_phi and capsules1000_phi: the 100- and 1000-capsule slits
filled to volume fractions 0.1 and 0.2, 245,244 and 3,923,904 points) measure
the same step; the pair counts of the roofline are taken on a sample of
20,000 targets for workloads above 100,000 points.

The off-grid evaluation of the global part is the paper's 5-point Lagrange
interpolation by default; --offgrid spectral times the spectrally accurate
evaluation instead, and the default run reports the other mode's step under
"offgrid_other".

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
For N > 1 under torchrun each rank runs an independent replica on its own
GPU (the evaluation is one problem per GPU; no collective), value = sum of
the ranks' points / the slowest rank's time.  --impl reference times the FP64
oracle on the host cores, each step a proportional sample of every stage.
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
    ap.add_argument("--workload", default="rbc4000",
                    choices=["capsules100", "capsules1000", "rbc4000", "capsules100_phi",
                             "capsules1000_phi"],
                    help="rbc4000 (default: 4000 biconcave capsules, 2,568,000 points, the "
                         "largest configuration), capsules100 (64,200 points), capsules1000 "
                         "(642,000 points), capsules100_phi / capsules1000_phi (the same "
                         "slits at volume fractions 0.1 / 0.2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--fp64-step", action="store_true",
                    help="also time one capsule time step with the plain native-FP64 solver "
                         "(minutes on the largest workload)")
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


# Algorithmic flops of one (target, source) pair of the local sum (see roofline)
FLOPS_PAIR_SINGLE = 52
FLOPS_PAIR_DOUBLE = 72
# DRAM bytes (read + write) of one local-sum launch, the single- and the
# double-layer launch averaged as the stage is, from ncu captures of the
# kernels as they stand (dram__bytes_read.sum + dram__bytes_write.sum; the
# summaries are kept with the profiles), per (workload, precision, quadrature);
# none for other configurations
LOCAL_TRAFFIC = {
    ("rbc4000", "mixed", "element"): (4687680000 + 41640448 + 5192181248 + 67060480) / 2,
}

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
        # algorithmic flops per (target, source) pair within r_cut, counting
        # add, sub, mul and rsqrt / exp2 as 1 and a fused multiply-add as 2
        # (the peak below counts an FMA as 2): displacement, r^2, 1/r, r,
        # exp(-alpha^2 r^2) as one exp2 of the scaled r^2, erfc(alpha r) =
        # exp(-alpha^2 r^2) erfcx(alpha r) with erfcx = t Q(t),
        # t = 1/(1 + P alpha r), Q of degree 6 (17), x.g -- 33 -- then the
        # single layer's A = erfc/r - c1 e, B = (erfc/r^3 + c1 e/r^2) x.g and
        # u += A g + B x (19: 52 in all) or the double layer's D, E, x.n, g.n
        # and v += x (D x.g x.n + E g.n) + g E x.n + n E x.g with the last
        # term summed as a scalar (39: 72 in all); the stage averages one
        # launch of each
        flops = pairs * (FLOPS_PAIR_SINGLE + FLOPS_PAIR_DOUBLE) / 2.0
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ach = flops / avg_s / 1e12
        if args.precision != "mixed":
            peak = 1.25           # FP64-accurate work against the nominal FP64 rate
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": LOCAL_TRAFFIC.get(
                    (args.workload, args.precision, args.quadrature)),
                "pairs_per_launch": pairs, "pairs_per_s": pairs / avg_s,
                "flops_per_pair": [FLOPS_PAIR_SINGLE, FLOPS_PAIR_DOUBLE],
                "launch_ms": avg_s * 1e3,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x max SM "
                               "clock" if args.precision == "mixed" else
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


# Sample sizes of one oracle step (see oracle_sample_step)
ORACLE_SAMPLE = {"targets": 48, "wall_nodes": 64, "sources": 2048, "triangles": 65536,
                 "planes": 2, "columns": 4096, "modes": 256, "interp_targets": 4096}


def oracle_sample_step(susp, args, seed, aux):
    """One step of the FP64 oracle on a bounded, proportional sample of the
    workload: every stage of the single- and the double-layer evaluation
    (Sec. 3.2-3.5, element quadrature) runs through the oracle's own functions
    on a seeded sample of its independent units -- triangles (geometry),
    target nodes (element-rule local sums), wall grid nodes (wall data),
    sources (spreading), y-planes (x-z FFTs), (x, z) columns (Chebyshev
    transforms), Fourier modes (tau solves, spectral stress) and targets
    (interpolation) -- each stage's time scaled by its units / sampled units.
    Returns (measured seconds, extrapolated seconds of the full step, per-stage
    {name: [sample seconds, scale]})."""
    from oracle import oracle as O
    S = ORACLE_SAMPLE
    box = susp.box
    n, m = susp.x.shape[0], susp.tri.shape[0]
    Ny, Nz, Nx = box.Ny, box.Nz, box.Nx
    rng = np.random.default_rng(seed)
    a, rc, nb, g = aux["alpha"], aux["rcut"], aux["nb"], aux["g"]
    q = aux["q"]
    stages = {}

    def run(name, scale, fn, reps=1):
        t0 = time.perf_counter()
        out = fn()
        stages[name] = [time.perf_counter() - t0, float(scale) * reps]
        return out

    pick = lambda total, k: np.sort(rng.choice(total, min(k, total), replace=False))
    tri_s = pick(m, S["triangles"])
    # geometry: once per layer evaluation (the nodes no sampled triangle touches
    # get 0/0 normals in the sample, which are not used)
    def geometry_sample():
        with np.errstate(invalid="ignore"):
            return O.geometry(susp.x, susp.tri[tri_s])
    run("geometry", m / len(tri_s), geometry_sample, reps=2)
    tg = pick(n, S["targets"]).astype(np.int32)
    run("local_single", n / len(tg),
        lambda: O.local_elem(box, a, rc, 0, susp.x, susp.tri, q, targets=tg))
    run("local_double", n / len(tg),
        lambda: O.local_elem(box, a, rc, 1, susp.x, susp.tri, q, nrm=nb, targets=tg))
    bot, top = O.wall_nodes(box)
    wn = pick(2 * Nx * Nz, S["wall_nodes"])
    walls = np.concatenate([bot, top])[wn]
    run("wall_data", 2 * Nx * Nz / len(wn),
        lambda: O.local_point(box, a, rc, 1.0, susp.x, g, walls), reps=2)
    src = pick(n, S["sources"])
    f = run("spread", n / len(src), lambda: O.spread(box, a, rc, susp.x[src], g[src]), reps=2)
    planes = pick(Ny, S["planes"])
    scale = 1.0 / (Nx * Nz)
    # forward x-z transforms of the 3 forcing planes and the 2 x 3 wall planes
    run("fft_forward", Ny / len(planes),
        lambda: np.fft.fft2(f[:, planes], axes=(2, 3)) * scale, reps=2)
    run("fft_walls", 1.0, lambda: np.fft.fft2(np.zeros((6, Nz, Nx)), axes=(1, 2)) * scale,
        reps=2)
    cols = pick(Nz * Nx, S["columns"])
    Fcol = rng.standard_normal((3, Ny, len(cols))) + 1j * rng.standard_normal((3, Ny, len(cols)))
    Cf = O.cheb_forward(Ny)
    run("cheb_forward", Nz * Nx / len(cols), lambda: np.einsum("nj,cjk->kcn", Cf, Fcol), reps=2)
    KX, KZ, nyq = O.mode_wavenumbers(box)
    sel = np.argwhere((~nyq) & (KX ** 2 + KZ ** 2 > 0))
    md = sel[pick(len(sel), S["modes"])]
    zz, xx = md[:, 0], md[:, 1]
    M = len(md)
    Fh = rng.standard_normal((M, 3, Ny)) + 1j * rng.standard_normal((M, 3, Ny))
    gw = rng.standard_normal((M, 3)) + 0j
    uvwp = run("tau_solve", len(sel) / M,
               lambda: O.ks_solve(box, Fh, gw, gw, 1.0, KX[zz, xx], KZ[zz, xx]), reps=2)
    Ci = O.cheb_inverse(Ny)
    Ccol = rng.standard_normal((len(cols), Ny)) + 1j * rng.standard_normal((len(cols), Ny))
    spec = rng.standard_normal((len(planes), Nz, Nx)) + 1j * rng.standard_normal(
        (len(planes), Nz, Nx))
    # inverse transforms of 14 fields: u, v, w, p for each layer and the 6
    # stress fields of the double layer
    run("cheb_inverse", Nz * Nx / len(cols), lambda: np.einsum("jn,kn->jk", Ci, Ccol), reps=14)
    run("fft_inverse", Ny / len(planes),
        lambda: np.real(np.fft.ifft2(spec, axes=(1, 2)) * (Nx * Nz)), reps=14)
    Dy = (2.0 / box.W) * O.cheb_deriv(Ny)
    U, V, Wc, Pc = uvwp
    ikx, ikz = 1j * KX[zz, xx][:, None], 1j * KZ[zz, xx][:, None]

    def stress():
        dU, dV, dW = U @ Dy.T, V @ Dy.T, Wc @ Dy.T
        return [-Pc + 2 * ikx * U, ikx * V + dU, ikz * U + ikx * Wc, -Pc + 2 * dV,
                ikz * V + dW, -Pc + 2 * ikz * Wc]
    run("spectral_stress", len(sel) / M, stress)
    it = pick(n, S["interp_targets"])
    # 3 velocity components (single layer) + 6 stress components (double layer)
    run("interp", n / len(it), lambda: O.interp(box, aux["F3"], susp.x[it]), reps=3)
    measured = sum(v[0] for v in stages.values())
    extrapolated = sum(v[0] * v[1] for v in stages.values())
    return measured, extrapolated, stages


def oracle_aux(susp):
    """Inputs of the sampled oracle step that are not part of its timing:
    alpha, r_cut, node normals and strengths (computed once)."""
    from oracle import oracle as O
    a = O.default_alpha(susp.box)
    q = np.random.default_rng(99).standard_normal((susp.x.shape[0], 3))
    _, _, Ab, nb = O.geometry(susp.x, susp.tri)
    b = susp.box
    return {"alpha": a, "rcut": O.default_rcut(a), "nb": nb, "q": q,
            "g": 8.0 * math.pi * Ab[:, None] * q, "F3": np.zeros((3, b.Ny, b.Nz, b.Nx))}


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def _sample_note(susp):
    S = ORACLE_SAMPLE
    return (f"FP64 oracle, single + double layer (element quadrature, Lagrange off-grid "
            f"evaluation) on a seeded proportional sample of each stage's independent units: "
            f"{S['targets']} target nodes (element-rule local sums), {S['wall_nodes']} wall "
            f"nodes, {S['sources']} sources (spreading), {S['triangles']} triangles "
            f"(geometry), {S['planes']} y-planes (x-z FFTs), {S['columns']} columns "
            f"(Chebyshev transforms), {S['modes']} Fourier modes (tau solves, spectral "
            f"stress), {S['interp_targets']} targets (interpolation); each stage's time x "
            f"(its units / sampled units); OpenMP in the C parts")


def _spread_updates(susp, rc, sample=2000):
    """Grid-node updates of one spreading call (Eq. (rhog_sum)): the number of
    (source, grid node) pairs with |node - x*| < r_cut, minimum image in x and
    z, Chebyshev nodes in y; counted on a seeded sample of sources and scaled."""
    from oracle import oracle as O
    b = susp.box
    yg = O.grid_y(b)
    n = susp.x.shape[0]
    idx = np.random.default_rng(5).choice(n, min(sample, n), replace=False)
    dx, dz = b.Lx / b.Nx, b.Lz / b.Nz
    total = 0
    for x, y, z in susp.x[idx]:
        ix = np.arange(int(np.floor((x - rc) / dx)), int(np.ceil((x + rc) / dx)) + 1)
        iz = np.arange(int(np.floor((z - rc) / dz)), int(np.ceil((z + rc) / dz)) + 1)
        ex = (ix * dx - x) ** 2
        ez = (iz * dz - z) ** 2
        ey = (yg - y) ** 2
        d2 = ex[:, None, None] + ez[None, :, None] + ey[None, None, :]
        total += int((d2 < rc * rc).sum())
    return total * n / len(idx)


def _stencil(b, yg, rc, x, y, z):
    """Flat indices (j, k, i) of the grid nodes within r_cut of (x, y, z)."""
    dx, dz = b.Lx / b.Nx, b.Lz / b.Nz
    ix = np.arange(int(np.floor((x - rc) / dx)), int(np.ceil((x + rc) / dx)) + 1)
    iz = np.arange(int(np.floor((z - rc) / dz)), int(np.ceil((z + rc) / dz)) + 1)
    d2 = ((ix * dx - x) ** 2)[None, None, :] + ((iz * dz - z) ** 2)[None, :, None] + \
        ((yg - y) ** 2)[:, None, None]
    j, k, i = np.nonzero(d2 < rc * rc)
    return (j * b.Nz + (iz[k] % b.Nz)) * b.Nx + (ix[i] % b.Nx)


def _spread_pair_reductions(susp, rc, sample=1000):
    """Vector reductions the paired spreading issues per call: sources in
    cell order (cells of r_cut/3, as the mesh nodes are sorted), taken two
    at a time, one reduction per node of the union of the two stencils;
    counted on a seeded sample of pairs and scaled."""
    from oracle import oracle as O
    b = susp.box
    yg = O.grid_y(b)
    x = susp.x.copy()
    x[:, 0] %= b.Lx
    x[:, 2] %= b.Lz
    h = rc / 3.0
    ncx, ncy, ncz = int(b.Lx // h), max(1, int(b.W // h)), int(b.Lz // h)
    cx = np.minimum((x[:, 0] / (b.Lx / ncx)).astype(int), ncx - 1)
    cy = np.clip(((x[:, 1] - b.y0) / (b.W / ncy)).astype(int), 0, ncy - 1)
    cz = np.minimum((x[:, 2] / (b.Lz / ncz)).astype(int), ncz - 1)
    order = np.lexsort((np.arange(len(x)), cx, cy, cz))
    npairs = len(x) // 2
    pick = np.random.default_rng(6).choice(npairs, min(sample, npairs), replace=False)
    tot = 0
    for p in pick:
        a, c = order[2 * p], order[2 * p + 1]
        tot += len(np.union1d(_stencil(b, yg, rc, *x[a]), _stencil(b, yg, rc, *x[c])))
    return tot * npairs / len(pick)


def spread_roofline(res, args):
    """The spreading stage against the measured throughput of float4 vector
    reductions into L2 (ggem_probe_l2_reduction): algorithmic node updates per
    call (one vector reduction each) / the stage's time per call."""
    from paper_1109_6587_gb300 import ggem
    stages = res["stages"]
    if "spread" not in stages:
        return None
    tot, calls = stages["spread"]
    avg_s = tot / calls * 1e-3
    _, rc = res["P"].info()
    upd = _spread_updates(res["susp"], rc)
    red = _spread_pair_reductions(res["susp"], rc) if args.precision == "mixed" else upd
    _, peak = ggem.probe_l2_reduction()
    ach = red / avg_s
    return {"kernel": "spread", "bound": "l2_reduction", "achieved": ach, "peak": peak,
            "unit": "vector reductions/s", "frac": ach / peak,
            "reductions_per_call": red, "node_updates_per_call": upd,
            "node_updates_per_s": upd / avg_s, "call_ms": avg_s * 1e3,
            "peak_source": "measured: ggem_probe_l2_reduction (float4 atomic adds, 32 MB "
                           "L2-resident buffer, warps on 32 consecutive vectors)"}


def cpu_baseline(susp, args):
    """The FP64 oracle as it stands on the host cores: one sampled step
    (oracle_sample_step); value = points / extrapolated full-step time."""
    aux = oracle_aux(susp)
    measured, full, stages = oracle_sample_step(susp, args, 1, aux)
    n = susp.x.shape[0]
    return {"value": n / full / 1e6, "unit": "Mpts/s", "cores": _cores(), "kind": "oracle",
            "sample": _sample_note(susp), "measured_seconds": measured,
            "extrapolated_seconds": full, "extrapolation_factor": full / measured,
            "stages": {k: {"sample_s": v[0], "scale": v[1]} for k, v in stages.items()}}


def _mk_plan(susp, prec, quadrature):
    from paper_1109_6587_gb300 import ggem
    return ggem.Plan.for_box(susp.box, precision=prec, quadrature=quadrature,
                             max_points=susp.x.shape[0], max_tris=susp.tri.shape[0])


def train_warm_start(args, model_plan, epochs=20):
    """The learned warm start trained on generated suspensions (none of them
    a timed workload): workloads.training_suspensions -- 48 to 382
    capsules, volume fractions 0.05 to 0.3, viscosity ratios 0.2, 1, 5 --
    each a series of 3 emulated steps solved to 1e-6 (the mixed solver),
    samples from every guess the solver meets; the model lives on
    model_plan."""
    import torch
    from paper_1109_6587_gb300 import warmstart as WS
    from paper_1109_6587_gb300 import workloads as W
    t0 = time.perf_counter()
    pairs = W.training_suspensions(seed=1)
    t1 = time.perf_counter()
    F, T = WS.generated_training_set(lambda s: _mk_plan(s, "mixed", args.quadrature), pairs,
                                     n_steps=3, seed=1000)
    t2 = time.perf_counter()
    loss = WS.train(model_plan, F, T, seed=1, epochs=epochs, batch=2048, lr=1e-3)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    return {"suspensions": [{"capsules": int(len(s.centres)), "lambda": lam,
                             "box": [s.box.Lx, s.box.W, s.box.Lz]} for s, lam in pairs],
            "samples": int(F.shape[0]), "epochs": epochs, "loss": loss,
            "generate_s": t1 - t0, "data_s": t2 - t1, "train_s": t3 - t2}


def solve_metrics(args, dev, model_plan_box=None, warm_steps=2, timed_steps=2):
    """GMRES iterations and seconds per Fredholm solve (Sec. 5) at true
    relative residual 1e-6 on the 1000-capsule workload (642,000 nodes,
    80 x [-10,10] x 80, grid 256 x 97 x 256, viscosity ratio 5: kappa = 2/3,
    b from Eq. (qa)), per emulated time step (capsules moved rigidly by 0.01
    radius, membrane load drifting), each solve from the previous step's
    density.  Steps 0..warm_steps-1 run once with the mixed solver (untimed,
    the warm state every variant starts from); then per variant:
      fp64            plain GMRES, FP64 operator (1 timed step);
      fp64_emulated   plain GMRES, FP64-accurate operator whose element-rule
                      local sum runs in double-float arithmetic (1 step);
      mixed           mixed operator, FP64 refinement (timed_steps steps);
      mixed_precond   the same with the per-particle block preconditioner;
      mixed_learned   mixed, starting from the learned guess when its
                      residual is lower (model trained on generated
                      suspensions, train_warm_start);
      mixed_learned_precond  both."""
    import torch
    from paper_1109_6587_gb300 import workloads as W
    susp = W.capsules_1000(seed=0)
    n = susp.x.shape[0]
    tri = torch.as_tensor(susp.tri, device=dev)
    Pm = _mk_plan(susp, "mixed", args.quadrature)
    training = train_warm_start(args, Pm)
    V, F = W.icosphere(3)

    def prepare(P, t):
        s = W_rigid(susp, t)
        kappa, b = W_rhs(s, t)
        P.mesh_set(torch.as_tensor(s.x, device=dev), tri)
        P.mesh_particles(s.particle, len(s.centres))
        return torch.as_tensor(kappa, device=dev), torch.as_tensor(b, device=dev)

    q = None
    for t in range(warm_steps):
        kd, bd = prepare(Pm, t)
        q, _, _, _ = Pm.bie_solve(kd, bd, q=bd.clone() if q is None else q.clone(), tol=1e-6)
    q_warm = q.clone()
    out = {"workload": "1000 spherical capsules x 642 nodes (642,000 points), slit 80 x "
                       "[-10,10] x 80, grid 256 x 97 x 256", "tol": 1e-6, "kappa": 2.0 / 3.0,
           "rhs": "Eq. (qa), synthetic membrane load + shear", "guess": "previous step's density",
           "restart": 30, "quadrature": args.quadrature, "warm_steps": warm_steps,
           "training": training}
    P64 = _mk_plan(susp, "fp64", args.quadrature)
    Pem = _mk_plan(susp, "fp64_emulated", args.quadrature)
    t0 = time.perf_counter()
    Pm.mesh_set(torch.as_tensor(susp.x, device=dev), tri)
    Pm.mesh_particles(susp.particle, len(susp.centres))
    Pm.precond_set(V, F, 2.0 / 3.0)
    out["precond_setup_s"] = time.perf_counter() - t0
    variants = (("fp64", P64, 0, False, 1), ("fp64_emulated", Pem, 0, False, 1),
                ("mixed", Pm, 0, False, timed_steps), ("mixed_precond", Pm, 0, True, timed_steps),
                ("mixed_learned", Pm, 1, False, timed_steps),
                ("mixed_learned_precond", Pm, 1, True, timed_steps))
    for name, P, use, pc, steps in variants:
        if P is Pm:
            P.precond_enable(pc)
        q = q_warm.clone()
        times, its, rrs, used = [], [], [], []
        for t in range(warm_steps, warm_steps + steps):
            kd, bd = prepare(P, t)
            torch.cuda.synchronize()
            a = time.perf_counter()
            q, it, rr, st = P.bie_solve(kd, bd, q=q, tol=1e-6, use_mlp=use)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - a)
            its.append(it)
            rrs.append(rr)
            used.append(P.solve_guess()[0])
        cyc, m64, mmix = P.solve_stats()
        out[name] = {"steps_timed": steps, "iters": float(np.mean(its)),
                     "s_per_solve": float(np.mean(times)),
                     "true_relres_max": float(np.max(rrs)), "learned_guess_used": used,
                     "last_solve_matvec_fp64": m64, "last_solve_matvec_mixed": mmix}
        P.check()
    out["_model"] = Pm.mlp_save()
    for P in (Pm, P64, Pem):
        P.close()
    for k in ("mixed", "mixed_precond", "mixed_learned", "mixed_learned_precond"):
        out[f"speedup_{k}_vs_fp64"] = out["fp64"]["s_per_solve"] / out[k]["s_per_solve"]
        out[f"speedup_{k}_vs_fp64_emulated"] = (out["fp64_emulated"]["s_per_solve"] /
                                               out[k]["s_per_solve"])
    return out


def dynamics_metrics(args, susp, dev, timed=2, model=None):
    """Capsule time steps of the workload (Sec. 5, 7.1): simple shear of rate
    1, viscosity ratio 5, Ca = 0.3, membranes stress-free in their initial
    shape.  One step: the dt rule from the smallest node separation, the
    midpoint step (per stage: traction jump, right side of Eq. (qa), Fredholm
    solve to 1e-6 from the previous density, single layer), the volume
    correction and the minimum-gap correction.  One untimed mixed step from
    the initial state, checkpointed; every variant resumes that checkpoint on
    a plan of its own and times its steps from the same state:
      mixed (timed steps), mixed_precond (the per-particle block
      preconditioner of the workload's own capsule shape), mixed_learned_precond
      (plus the learned warm start, `model`), fp64_emulated (1 step: plain
      GMRES with the FP64-accurate operator)."""
    import tempfile

    import torch
    from paper_1109_6587_gb300 import dynamics as D
    from paper_1109_6587_gb300 import workloads as W

    n = susp.x.shape[0]
    P = _mk_plan(susp, "mixed", args.quadrature)
    P.mesh_set(torch.as_tensor(susp.x, device=dev), torch.as_tensor(susp.tri, device=dev))
    np_ = len(susp.centres)
    S = D.Suspension(P, susp.particle, np_, lam=np.full(np_, 5.0), ca=0.3, flow="shear",
                     strength=1.0, tri=susp.tri)
    warm = S.step()
    ckpt = os.path.join(tempfile.mkdtemp(), "dyn.npz")
    S.save(ckpt)
    P.close()
    rbc = susp.box.Lx == 150.0
    V, F = W.rbc_mesh(3) if rbc else W.icosphere(3)
    out = {"flow": "simple shear, rate 1", "lambda": 5.0, "Ca": 0.3, "tol": 1e-6,
           "warm_step": {"iters": warm["iters"], "seconds": warm["seconds"]},
           "reference_capsule": "biconcave (Evans-Fung), 642 nodes" if rbc else
           "sphere, 642 nodes"}
    variants = (("mixed", "mixed", False, 0, timed), ("mixed_precond", "mixed", True, 0, timed),
                ("mixed_learned_precond", "mixed", True, 1, timed),
                ("fp64_emulated", "fp64_emulated", False, 0, 1))
    if args.fp64_step:
        variants += (("fp64", "fp64", False, 0, 1),)
    for name, prec, pc, use, steps in variants:
        if use and model is None:
            continue
        P = _mk_plan(susp, prec, args.quadrature)
        S = D.Suspension.resume(P, ckpt)
        if use:
            P.mlp_load(model)
        rec = {}
        if pc:
            t0 = time.perf_counter()
            P.precond_set(V, F, 2.0 / 3.0)
            rec["precond_setup_s"] = time.perf_counter() - t0
        recs = [S.step(use_mlp=use) for _ in range(steps)]
        P.check()
        rec.update({"steps_timed": steps,
                    "s_per_step": float(np.mean([r["seconds"] for r in recs])),
                    "gmres_iters_per_step": float(np.mean([r["iters"] for r in recs])),
                    "dt": float(np.mean([r["dt"] for r in recs])),
                    "volume_passes": int(sum(r["volume_passes"] for r in recs)),
                    "overlap_moves": int(sum(r["overlap_moves"] for r in recs))})
        out[name] = rec
        P.close()
    for k in ("mixed", "mixed_precond", "mixed_learned_precond"):
        for base in ("fp64_emulated", "fp64"):
            if k in out and base in out:
                out[f"speedup_{k}_vs_{base}"] = out[base]["s_per_step"] / out[k]["s_per_step"]
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
        aux = oracle_aux(susp)
        for i in range(args.warmup):
            oracle_sample_step(susp, args, 1000 + i, aux)
        meas, full, last = [], [], None
        for i in range(args.steps):
            m_s, f_s, last = oracle_sample_step(susp, args, i, aux)
            meas.append(m_s)
            full.append(f_s)
        n = susp.x.shape[0]
        t_full = float(np.mean(full))
        val = n / t_full / 1e6
        ms = float(np.mean(meas)) * 1e3
        cfg = _config(susp, args)
        cfg["precision"] = "fp64"
        cb = {"value": val, "unit": "Mpts/s", "cores": _cores(), "kind": "oracle",
              "sample": _sample_note(susp), "measured_seconds_per_step": ms * 1e-3,
              "extrapolated_seconds_per_step": t_full,
              "extrapolation_factor": t_full / (ms * 1e-3),
              "stages_last_step": {k: {"sample_s": v[0], "scale": v[1]} for k, v in last.items()}}
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpts/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms,
                "ms_per_step_note": "measured wall time of one sampled oracle step; value = "
                                    "points / (the step's stage times x their scale "
                                    "factors), i.e. extrapolated to the full workload",
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": cfg, "cpu_baseline": cb,
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
    line["roofline_spread"] = spread_roofline(res, args)
    if not args.no_solve:
        import torch
        dev = torch.device("cuda")
        res["P"].close()
        line["offgrid_other"] = offgrid_metrics(args, res["susp"], dev)
        line["solve"] = solve_metrics(args, dev)
        model = line["solve"].pop("_model", None)
        line["dynamics"] = dynamics_metrics(args, res["susp"], dev, model=model)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(res["susp"], args)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
