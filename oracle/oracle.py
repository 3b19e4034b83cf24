"""GGEM oracle: a plain FP64 CPU implementation of the slit evaluation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may import this module.  It shares no code with the
CUDA library: the pair sums live in ``ggem_oracle.c`` (plain loops), the global
spectral solve is written here with dense matrices and numpy's FFT.

Paper: Kumar & Graham, arXiv 1109.6587.  Steps, in the paper's order:
  1. local sums u^l, sigma^l ........................ Eq. (u_loc), Sec. 3.2.1
  2. wall data for the global problem u^g = -u^l ..... Sec. 3.2.2
  3. global forcing f = -sum g rho_g on the grid ..... Eq. (stokes_gg)
  4. Fourier (x,z) x Chebyshev (y) expansion ......... Eq. (u_expn), App. C
  5. per-mode Kleiser-Schumann influence-matrix solve  App. C, Eqs. (stokes_t_all),
     Chebyshev tau (two top rows = wall conditions)    (bc_vel), (inf_mat), (cheb_sol)
  6. stress sigma^g = -p + mu (grad u + grad u^T) ..... Sec. 3.5.1
  7. 4th-order (5-point) Lagrange interpolation ....... Sec. 3.2.2
     or the expansion summed at each point ............. Sec. 3.2.3, Eq. (u_expn)
  8. u = u^l + u^g ..................................... Eq. (tot_l_g)
Boundary integral operators (Sec. 3.4, 3.5), the Fredholm solve (Sec. 5,
restarted GMRES with modified Gram-Schmidt; a per-particle block-preconditioned
variant, which the paper does not use, as a reference) and the rigid-particle
solve (Sec. 6.1, Eq. (sl_r) with force and torque balance) are built on top.

Readings (the paper is silent, ambiguous or garbled here):
  * alpha = 1/(2 h), h = max(Lx/Nx, W/(Ny-1), Lz/Nz); r_cut = 4/alpha.
  * App. C writes "il, im, k^2": l, m stand for k_x = 2 pi l/Lx, k_z = 2 pi m/Lz.
  * Eq. (press_helm) has the wrong sign on its right side; taking the
    divergence of Eq. (stokes_a) gives (D^2 - k^2) p = -(i kx fx + D fy + i kz fz).
  * The Nyquist modes l = -Nx/2 and m = -Nz/2 of every transformed field are
    set to zero.
  * Mode k = 0: u, w from mu D^2 u = f with the wall values; v is the linear
    interpolant of its two wall values; p from D p = -f_y with zero mean over y.
  * No tau-correction step is applied (the paper mentions none).
  * Interpolation stencils: x, z use nodes i0-2..i0+2, i0 the nearest node
    (ties to even), periodic; y uses the 5 consecutive Chebyshev nodes
    centred on the nearest node, clamped to [0, Ny-5].
  * Point-force targets that coincide with a source: the self pair is left
    out of the local sum (r > 0) and the free-space global self velocity
    (4 alpha / sqrt(pi)) g / (8 pi mu) is subtracted, so the result does not
    depend on alpha.  The global self stress is zero by symmetry.
  * Stress kernel: T = -P delta + dG + dG^T (Eq. (local c) is mu-free);
    physical stress sigma = (1/8 pi) sum T g.  The double layer uses
    sigma/mu (Eq. (st_dbl)).
  * Element form: the global part and the wall data use the trapezoidal nodal
    strengths A_b q_b (Eq. (rhog_sum)); the local part uses the element rule.
  * Spectral off-grid evaluation (Sec. 3.2.3 names the non-uniform FFT as the
    way to exponential accuracy off the mesh without writing it out): the
    value at a point is the trigonometric (x, z; Nyquist modes zero) times
    Chebyshev (y, degree Ny - 1) expansion of the grid field summed there --
    the quantity a non-uniform FFT approximates to its tolerance.
"""
from __future__ import annotations

import ctypes
import math
import os
import pathlib
import subprocess

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_SO = _HERE / "libggem_oracle.so"
_lib = None


def build(force=False):
    """Compile the C half of the oracle (gcc, OpenMP)."""
    src = _HERE / "ggem_oracle.c"
    if force or not _SO.exists() or _SO.stat().st_mtime < src.stat().st_mtime:
        tmp = _SO.with_suffix(f".so.{os.getpid()}")
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC",
                               "-o", str(tmp), str(src), "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Box(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_double), ("Lz", ctypes.c_double),
                ("W", ctypes.c_double), ("y0", ctypes.c_double),
                ("Nx", ctypes.c_int), ("Ny", ctypes.c_int), ("Nz", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(str(_SO))
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        _lib.orc_kernels_batch.argtypes = [d, i, p, p, p, p]
        _lib.orc_local_point.argtypes = [p, d, d, d, i, p, p, i, p, p, p]
        _lib.orc_spread.argtypes = [p, d, d, i, p, p, p]
        _lib.orc_local_elem.argtypes = [p, d, d, i, i, p, i, p, p, p, i, p, p]
        _lib.orc_rhog.argtypes = [d, d]
        _lib.orc_rhog.restype = d
        _lib.orc_gauss_legendre01.argtypes = [i, p, p]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _cbox(box):
    return _Box(box.Lx, box.Lz, box.W, box.y0, box.Nx, box.Ny, box.Nz)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- parameters

def default_alpha(box):
    """alpha = 1/(2h), h the largest mean mesh spacing (alpha*dy_m <= 0.5, Sec. 5)."""
    h = max(box.Lx / box.Nx, box.W / (box.Ny - 1), box.Lz / box.Nz)
    return 1.0 / (2.0 * h)


def default_rcut(alpha):
    """r_cut = 4/alpha (Sec. 3.2.1)."""
    return 4.0 / alpha


# ------------------------------------------------------------ local kernels

def kernels(alpha, x):
    """G^l [n,3,3], P^l [n,3], T^l [n,3,3,3] at displacements x [n,3] (Eq. local)."""
    x = _f64(x).reshape(-1, 3)
    n = x.shape[0]
    G = np.zeros((n, 3, 3)); P = np.zeros((n, 3)); T = np.zeros((n, 3, 3, 3))
    lib().orc_kernels_batch(alpha, n, _ptr(x), _ptr(G), _ptr(P), _ptr(T))
    return G, P, T


def rho_g(alpha, r):
    """Quasi-Gaussian global density of Eq. (rho_l_g a)."""
    r = np.asarray(r, dtype=np.float64)
    a2r2 = alpha * alpha * r * r
    return alpha ** 3 / math.pi ** 1.5 * np.exp(-a2r2) * (2.5 - a2r2)


def local_point(box, alpha, rcut, mu, xs, g, xt, want_u=True, want_sig=False):
    """Local sums of Eq. (u_loc) over pairs with 0 < r < rcut (minimum image)."""
    xs, g, xt = _f64(xs), _f64(g), _f64(xt)
    nt = xt.shape[0]
    u = np.zeros((nt, 3)) if want_u else None
    s = np.zeros((nt, 3, 3)) if want_sig else None
    cb = _cbox(box)
    lib().orc_local_point(ctypes.byref(cb), alpha, rcut, mu, xs.shape[0], _ptr(xs),
                          _ptr(g), nt, _ptr(xt), _ptr(u), _ptr(s))
    return u, s


def spread(box, alpha, rcut, xs, g):
    """Global forcing f = -sum g rho_g on the grid, [3, Ny, Nz, Nx]."""
    xs, g = _f64(xs), _f64(g)
    f = np.zeros((3, box.Ny, box.Nz, box.Nx))
    cb = _cbox(box)
    lib().orc_spread(ctypes.byref(cb), alpha, rcut, xs.shape[0], _ptr(xs), _ptr(g),
                     _ptr(f))
    return f


def gauss_legendre01(n):
    t = np.zeros(n); w = np.zeros(n)
    lib().orc_gauss_legendre01(n, _ptr(t), _ptr(w))
    return t, w


def local_elem(box, alpha, rcut, layer, x, tri, q, nrm=None, targets=None):
    """Local part of the single (layer=0) or double (layer=1) layer by the
    element rule of Sec. 3.4.1 / 3.5.2 at the listed target nodes."""
    x, q = _f64(x), _f64(q)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    if targets is None:
        targets = np.arange(x.shape[0], dtype=np.int32)
    targets = np.ascontiguousarray(targets, dtype=np.int32)
    nrm = _f64(nrm) if nrm is not None else None
    out = np.zeros((targets.shape[0], 3))
    cb = _cbox(box)
    lib().orc_local_elem(ctypes.byref(cb), alpha, rcut, layer, x.shape[0], _ptr(x),
                         tri.shape[0], _ptr(tri), _ptr(q), _ptr(nrm),
                         targets.shape[0], _ptr(targets), _ptr(out))
    return out


# --------------------------------------------------------------------- grid

def grid_x(box):
    return np.arange(box.Nx) * (box.Lx / box.Nx)


def grid_z(box):
    return np.arange(box.Nz) * (box.Lz / box.Nz)


def grid_y(box):
    """Gauss-Lobatto nodes y_j = y0 + W/2 (1 + cos(pi j/(Ny-1))), j = 0..Ny-1 (Sec. 3.2.2)."""
    j = np.arange(box.Ny)
    return box.y0 + 0.5 * box.W * (1.0 + np.cos(np.pi * j / (box.Ny - 1)))


def wall_nodes(box):
    """Grid nodes on the bottom (y0) and top (y0+W) walls, each [Nz*Nx, 3] (z-major)."""
    X, Z = np.meshgrid(grid_x(box), grid_z(box), indexing="xy")
    bot = np.stack([X.ravel(), np.full(X.size, box.y0), Z.ravel()], axis=1)
    top = np.stack([X.ravel(), np.full(X.size, box.y0 + box.W), Z.ravel()], axis=1)
    return bot, top


# ---------------------------------------------------------- Chebyshev (y)

def _cbar(N):
    c = np.ones(N + 1); c[0] = 2.0; c[N] = 2.0
    return c


def cheb_forward(Ny):
    """Matrix of the discrete Chebyshev transform on the Gauss-Lobatto nodes:
    a_n = 2/(N cbar_n) sum_j f_j T_n(ybar_j)/cbar_j, ybar_j = cos(pi j/N)."""
    N = Ny - 1
    n = np.arange(Ny)[:, None]; j = np.arange(Ny)[None, :]
    cb = _cbar(N)
    return 2.0 / (N * cb[:, None] * cb[None, :]) * np.cos(np.pi * n * j / N)


def cheb_inverse(Ny):
    """f_j = sum_n a_n T_n(ybar_j)."""
    N = Ny - 1
    j = np.arange(Ny)[:, None]; n = np.arange(Ny)[None, :]
    return np.cos(np.pi * n * j / N)


def cheb_deriv(Ny):
    """d/dybar in coefficient space: (d/dybar) T_m = sum_{n<m, n+m odd} 2m/c_n T_n."""
    D = np.zeros((Ny, Ny))
    for n in range(Ny):
        cn = 2.0 if n == 0 else 1.0
        for m in range(n + 1, Ny):
            if (n + m) % 2 == 1:
                D[n, m] = 2.0 * m / cn
    return D


def cheb_at_walls(Ny):
    """Rows evaluating a Chebyshev series at ybar = -1 (bottom) and +1 (top)."""
    n = np.arange(Ny)
    return (-1.0) ** n, np.ones(Ny)


def cheb_integrate_zero_mean(G):
    """Coefficients of p with dp/dybar = G and int_{-1}^{1} p dybar = 0, from
    c_{n-1} G_{n-1} - G_{n+1} = 2 n p_n (n >= 1), the series cut at degree N
    (G_{N+1} = 0).  G: [..., Ny]."""
    Ny = G.shape[-1]
    p = np.zeros_like(G)
    for n in range(1, Ny):
        c = 2.0 if n == 1 else 1.0
        gp = G[..., n + 1] if n + 1 < Ny else 0.0
        p[..., n] = (c * G[..., n - 1] - gp) / (2.0 * n)
    for n in range(2, Ny, 2):
        p[..., 0] -= p[..., n] / (1.0 - n * n)
    return p


# --------------------------------------------------------- global problem

def _tau_matrices(Ny, W, k2):
    """Chebyshev-tau operator of (D_y^2 - k^2) for each k2: rows 0..N-2 hold the
    equation in coefficient space, row N-1 the value at the bottom wall and row
    N the value at the top wall (App. C)."""
    Dy = (2.0 / W) * cheb_deriv(Ny)
    D2 = Dy @ Dy
    bot, top = cheb_at_walls(Ny)
    H = np.broadcast_to(D2, (len(k2), Ny, Ny)).copy()
    H -= k2[:, None, None] * np.eye(Ny)[None]
    H[:, Ny - 2, :] = bot
    H[:, Ny - 1, :] = top
    return H


def _with_bc(rhs, bot, top):
    """Replace the two highest equations by the wall values."""
    r = rhs.copy()
    r[..., -2] = bot
    r[..., -1] = top
    return r


def ks_solve(box, Fh, gb, gt, mu, kx, kz):
    """Kleiser-Schumann influence-matrix solve for modes with k^2 > 0 (App. C).

    Fh: [M, 3, Ny] Chebyshev coefficients of (f_x, f_y, f_z) per mode;
    gb, gt: [M, 3] velocity at the bottom / top wall; kx, kz: [M].
    Returns (u, v, w, p) coefficients, each [M, Ny] complex.
    """
    Ny = box.Ny
    M = Fh.shape[0]
    Dy = (2.0 / box.W) * cheb_deriv(Ny)
    bot, top = cheb_at_walls(Ny)
    k2 = kx * kx + kz * kz
    H = _tau_matrices(Ny, box.W, k2).astype(np.complex128)
    ikx, ikz = (1j * kx)[:, None], (1j * kz)[:, None]
    fx, fy, fz = Fh[:, 0], Fh[:, 1], Fh[:, 2]
    # pressure problems: a (forced, p = 0 at walls), b (p = 1 at bottom), c (p = 1 at top)
    rp = -(ikx * fx + fy @ Dy.T + ikz * fz)
    z = np.zeros((M, Ny), complex)
    P = np.stack([_with_bc(rp, 0.0, 0.0), _with_bc(z, 1.0, 0.0), _with_bc(z, 0.0, 1.0)],
                 axis=2)
    pa, pb, pc = np.moveaxis(np.linalg.solve(H, P), 2, 0)

    # velocity problems for a, b, c
    def vel_rhs(f3, p, gbot, gtop):
        ru = _with_bc((f3[0] + ikx * p) / mu, gbot[0], gtop[0])
        rv = _with_bc((f3[1] + p @ Dy.T) / mu, gbot[1], gtop[1])
        rw = _with_bc((f3[2] + ikz * p) / mu, gbot[2], gtop[2])
        return [ru, rv, rw]

    zero3 = [z, z, z]
    zb = np.zeros((3, M), complex)
    cols = (vel_rhs([fx, fy, fz], pa, gb.T, gt.T) + vel_rhs(zero3, pb, zb, zb)
            + vel_rhs(zero3, pc, zb, zb))
    V = np.linalg.solve(H, np.stack(cols, axis=2))
    ua, va, wa, ub, vb, wb, uc, vc, wc = np.moveaxis(V, 2, 0)

    def C(u, v, w, row):
        return (ikx[:, 0] * (u @ row) + (v @ Dy.T) @ row + ikz[:, 0] * (w @ row))

    # influence matrix (Eq. inf_mat): continuity at both walls
    A = np.empty((M, 2, 2), complex)
    A[:, 0, 0] = C(ub, vb, wb, bot); A[:, 0, 1] = C(uc, vc, wc, bot)
    A[:, 1, 0] = C(ub, vb, wb, top); A[:, 1, 1] = C(uc, vc, wc, top)
    rhs = -np.stack([C(ua, va, wa, bot), C(ua, va, wa, top)], axis=1)
    p12 = np.linalg.solve(A, rhs[:, :, None])[:, :, 0]
    p1, p2 = p12[:, 0:1], p12[:, 1:2]
    # Eq. (cheb_sol)
    u = ua + p1 * ub + p2 * uc
    v = va + p1 * vb + p2 * vc
    w = wa + p1 * wb + p2 * wc
    p = pa + p1 * pb + p2 * pc
    return u, v, w, p


def k0_solve(box, Fh, gb, gt, mu):
    """The k = 0 mode (reading): mu D^2 u = f_x, mu D^2 w = f_z with the wall
    values; v linear between its wall values; D p = -f_y, zero mean."""
    Ny = box.Ny
    H = _tau_matrices(Ny, box.W, np.zeros(1))[0].astype(np.complex128)
    u = np.linalg.solve(H, _with_bc(Fh[0] / mu, gb[0], gt[0]))
    w = np.linalg.solve(H, _with_bc(Fh[2] / mu, gb[2], gt[2]))
    v = np.zeros(Ny, complex)
    v[0] = 0.5 * (gb[1] + gt[1])
    v[1] = 0.5 * (gt[1] - gb[1])
    p = cheb_integrate_zero_mean(-(0.5 * box.W) * Fh[1])
    return u, v, w, p


def mode_wavenumbers(box):
    """k_x, k_z for numpy's fft2 layout over axes (z, x); Nyquist flagged."""
    lx = np.fft.fftfreq(box.Nx, 1.0 / box.Nx)   # 0..Nx/2-1, -Nx/2..-1
    mz = np.fft.fftfreq(box.Nz, 1.0 / box.Nz)
    kx = 2.0 * np.pi * lx / box.Lx
    kz = 2.0 * np.pi * mz / box.Lz
    KZ, KX = np.meshgrid(kz, kx, indexing="ij")
    nyq = (np.abs(np.meshgrid(mz, lx, indexing="ij")[0]) == box.Nz // 2) | \
          (np.abs(np.meshgrid(mz, lx, indexing="ij")[1]) == box.Nx // 2)
    return KX, KZ, nyq


def global_solve(box, f, gwall_bot, gwall_top, mu=1.0, want_stress=False, chunk=1024):
    """Solve -grad p + mu lap u = f, div u = 0 in the periodic slit with
    u = gwall_* on the walls (App. C).  f: [3, Ny, Nz, Nx]; gwall_*: [3, Nz, Nx].
    Returns physical-space u [3, Ny, Nz, Nx], p [Ny, Nz, Nx] and, if asked,
    stress [6, Ny, Nz, Nx] ordered xx, xy, xz, yy, yz, zz."""
    Ny, Nz, Nx = box.Ny, box.Nz, box.Nx
    scale = 1.0 / (Nx * Nz)
    Fhat = np.fft.fft2(f, axes=(2, 3)) * scale            # [3, Ny, Nz, Nx]
    Gb = np.fft.fft2(gwall_bot, axes=(1, 2)) * scale       # [3, Nz, Nx]
    Gt = np.fft.fft2(gwall_top, axes=(1, 2)) * scale
    Cf = cheb_forward(Ny)
    Fc = np.einsum("nj,cjzx->zxcn", Cf, Fhat)              # [Nz, Nx, 3, Ny]
    KX, KZ, nyq = mode_wavenumbers(box)
    Uc = np.zeros((Nz, Nx, 4, Ny), complex)                # u, v, w, p coefficients
    k2 = KX ** 2 + KZ ** 2
    sel = (~nyq) & (k2 > 0)
    idx = np.argwhere(sel)
    for s in range(0, len(idx), chunk):
        ii = idx[s:s + chunk]
        zz, xx = ii[:, 0], ii[:, 1]
        u, v, w, p = ks_solve(box, Fc[zz, xx], Gb[:, zz, xx].T, Gt[:, zz, xx].T, mu,
                              KX[zz, xx], KZ[zz, xx])
        Uc[zz, xx, 0], Uc[zz, xx, 1], Uc[zz, xx, 2], Uc[zz, xx, 3] = u, v, w, p
    Uc[0, 0] = np.stack(k0_solve(box, Fc[0, 0], Gb[:, 0, 0], Gt[:, 0, 0], mu))
    Ci = cheb_inverse(Ny)

    def to_phys(coef):                                       # coef [Nz, Nx, Ny]
        spec = np.einsum("jn,zxn->jzx", Ci, coef)
        return np.real(np.fft.ifft2(spec, axes=(1, 2)) * (Nx * Nz))

    u = np.stack([to_phys(Uc[:, :, c]) for c in range(3)])
    p = to_phys(Uc[:, :, 3])
    if not want_stress:
        return u, p, None
    Dy = (2.0 / box.W) * cheb_deriv(Ny)
    ikx, ikz = 1j * KX[:, :, None], 1j * KZ[:, :, None]
    U, V, Wc, Pc = Uc[:, :, 0], Uc[:, :, 1], Uc[:, :, 2], Uc[:, :, 3]
    dU, dV, dW = U @ Dy.T, V @ Dy.T, Wc @ Dy.T
    sig = [
        -Pc + 2 * mu * ikx * U,            # xx
        mu * (ikx * V + dU),               # xy
        mu * (ikz * U + ikx * Wc),         # xz
        -Pc + 2 * mu * dV,                 # yy
        mu * (ikz * V + dW),               # yz
        -Pc + 2 * mu * ikz * Wc,           # zz
    ]
    return u, p, np.stack([to_phys(s_) for s_ in sig])


# ------------------------------------------------------------ interpolation

def _lagrange(t_nodes, t):
    """Lagrange basis values at t [n] for the 5 nodes t_nodes [n, 5]: [n, 5]."""
    L = np.ones(t_nodes.shape)
    for p in range(5):
        for q in range(5):
            if q != p:
                L[..., p] *= (t - t_nodes[..., q]) / (t_nodes[..., p] - t_nodes[..., q])
    return L


def interp_weights(box, xt):
    """Stencil indices and weights of the 5x5x5 Lagrange interpolation."""
    xt = _f64(xt)
    dx, dz = box.Lx / box.Nx, box.Lz / box.Nz
    off = np.arange(-2, 3)
    ix0 = np.rint(xt[:, 0] / dx)                       # ties to even
    iz0 = np.rint(xt[:, 2] / dz)
    tx = xt[:, 0] / dx - ix0
    tz = xt[:, 2] / dz - iz0
    wx = _lagrange(np.broadcast_to(off, (len(xt), 5)).astype(float), tx)
    wz = _lagrange(np.broadcast_to(off, (len(xt), 5)).astype(float), tz)
    ix = (ix0[:, None].astype(np.int64) + off) % box.Nx
    iz = (iz0[:, None].astype(np.int64) + off) % box.Nz
    yg = grid_y(box)
    jn = np.argmin(np.abs(xt[:, 1:2] - yg[None, :]), axis=1)   # nearest node
    j0 = np.clip(jn - 2, 0, box.Ny - 5)
    jy = j0[:, None] + np.arange(5)
    wy = _lagrange(yg[jy], xt[:, 1])
    return (ix, jy, iz), (wx, wy, wz)


def interp(box, field, xt):
    """Evaluate grid fields [C, Ny, Nz, Nx] at points xt [n, 3] -> [n, C]."""
    (ix, jy, iz), (wx, wy, wz) = interp_weights(box, xt)
    vals = field[:, jy[:, :, None, None], iz[:, None, :, None], ix[:, None, None, :]]
    w = wy[:, :, None, None] * wz[:, None, :, None] * wx[:, None, None, :]
    return np.einsum("cnabd,nabd->nc", vals, w)


def spectral_coefficients(box, field):
    """Fourier (x, z) x Chebyshev (y) coefficients of grid fields [C, Ny, Nz, Nx]:
    a[c, n, m, l] with field = sum a T_n(ybar) exp(i (k_l x + k_m z)) at the
    grid nodes (Eq. (u_expn)); the Nyquist modes are zero, as in the solve."""
    coef = np.fft.fft2(field, axes=(2, 3)) / (box.Nx * box.Nz)
    _, _, nyq = mode_wavenumbers(box)
    coef[:, :, nyq] = 0.0
    return np.einsum("nj,cjzx->cnzx", cheb_forward(box.Ny), coef)


def spectral_eval(box, field, xt):
    """Evaluate grid fields [C, Ny, Nz, Nx] at points xt [n, 3] by summing their
    expansion (Eq. (u_expn)) at each point: the exactly convergent off-mesh
    evaluation of Sec. 3.2.3 (what a non-uniform FFT computes to its
    tolerance).  T_n(ybar) = cos(n arccos ybar).  -> [n, C]."""
    xt = _f64(xt)
    a = spectral_coefficients(box, field)
    KX, KZ, _ = mode_wavenumbers(box)
    kx, kz = KX[0], KZ[:, 0]
    n = np.arange(box.Ny)
    out = np.empty((xt.shape[0], field.shape[0]))
    for t, (x, y, z) in enumerate(xt):
        yb = np.clip(2.0 * (y - box.y0) / box.W - 1.0, -1.0, 1.0)
        Tn = np.cos(n * np.arccos(yb))
        ex, ez = np.exp(1j * kx * x), np.exp(1j * kz * z)
        out[t] = np.real(np.einsum("cnml,n,m,l->c", a, Tn, ez, ex, optimize=True))
    return out


# ------------------------------------------------------------- point forces

_SYM6 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def sym6_to_full(s6):
    """[n, 6] (xx, xy, xz, yy, yz, zz) -> [n, 3, 3]."""
    out = np.empty((s6.shape[0], 3, 3))
    for c, (i, j) in enumerate(_SYM6):
        out[:, i, j] = s6[:, c]
        out[:, j, i] = s6[:, c]
    return out


def wall_data(box, alpha, rcut, mu, xs, g):
    """Global wall values u^g = -u^l at the wall grid nodes, each [3, Nz, Nx]."""
    bot, top = wall_nodes(box)
    ub, _ = local_point(box, alpha, rcut, mu, xs, g, bot)
    ut, _ = local_point(box, alpha, rcut, mu, xs, g, top)
    shape = (box.Nz, box.Nx, 3)
    return -np.moveaxis(ub.reshape(shape), 2, 0), -np.moveaxis(ut.reshape(shape), 2, 0)


def global_fields(box, xs, g, mu=1.0, alpha=None, rcut=None, want_stress=False):
    """Global velocity, pressure (and stress) on the grid for point forces g at xs."""
    alpha = default_alpha(box) if alpha is None else alpha
    rcut = default_rcut(alpha) if rcut is None else rcut
    gb, gt = wall_data(box, alpha, rcut, mu, xs, g)
    f = spread(box, alpha, rcut, xs, g)
    return global_solve(box, f, gb, gt, mu, want_stress)


def evaluate(box, field, xt, offgrid="lagrange"):
    """Grid fields at off-grid points: 5-point Lagrange interpolation (Sec. 3.2.2)
    or, with offgrid="spectral", the expansion summed at each point (Sec. 3.2.3)."""
    if offgrid == "spectral":
        return spectral_eval(box, field, xt)
    if offgrid != "lagrange":
        raise ValueError("offgrid must be 'lagrange' or 'spectral'")
    return interp(box, field, xt)


def point_forces(box, xs, g, xt=None, mu=1.0, alpha=None, rcut=None,
                 want_u=True, want_sig=False, offgrid="lagrange"):
    """GGEM velocity [n,3] and stress [n,3,3] at targets due to point forces.

    xt=None means the targets are the sources themselves (self pair left out,
    global self velocity subtracted, see the readings above)."""
    alpha = default_alpha(box) if alpha is None else alpha
    rcut = default_rcut(alpha) if rcut is None else rcut
    self_t = xt is None
    xt = xs if self_t else xt
    ul, sl = local_point(box, alpha, rcut, mu, xs, g, xt, want_u, want_sig)
    ug, pg, sg = global_fields(box, xs, g, mu, alpha, rcut, want_sig)
    u = s = None
    if want_u:
        u = ul + evaluate(box, ug, xt, offgrid)
        if self_t:
            u -= (4.0 * alpha / math.sqrt(math.pi)) * _f64(g) / (8.0 * math.pi * mu)
    if want_sig:
        s = sl + sym6_to_full(evaluate(box, sg, xt, offgrid))
    return u, s


# ------------------------------------------------ boundary integral operators

def geometry(x, tri):
    """Element areas A_k, element unit normals, nodal areas A_b = sum A_k/3 and
    area-averaged unit node normals (Sec. 3.4.2, 3.5.2)."""
    x = _f64(x)
    x1, x2, x3 = x[tri[:, 0]], x[tri[:, 1]], x[tri[:, 2]]
    c = np.cross(x2 - x1, x3 - x1)
    a2 = np.linalg.norm(c, axis=1)
    Ak = 0.5 * a2
    nk = c / a2[:, None]
    Ab = np.zeros(x.shape[0])
    nb = np.zeros_like(x)
    for v in range(3):
        np.add.at(Ab, tri[:, v], Ak / 3.0)
        np.add.at(nb, tri[:, v], Ak[:, None] * nk)
    nb /= np.linalg.norm(nb, axis=1, keepdims=True)
    return Ak, nk, Ab, nb


def single_layer(susp, q, quadrature="element", mu=1.0, alpha=None, rcut=None,
                 targets=None, offgrid="lagrange"):
    """w_j(z) = int q_i G_ji dS at the nodes (Sec. 3.4).  [N, 3] (or targets)."""
    box = susp.box
    alpha = default_alpha(box) if alpha is None else alpha
    rcut = default_rcut(alpha) if rcut is None else rcut
    _, _, Ab, _ = geometry(susp.x, susp.tri)
    g = 8.0 * math.pi * mu * Ab[:, None] * _f64(q)
    tsel = np.arange(susp.x.shape[0]) if targets is None else np.asarray(targets)
    if quadrature == "nodal":
        if targets is None or offgrid == "lagrange":
            u, _ = point_forces(box, susp.x, g, None, mu, alpha, rcut, offgrid=offgrid)
            return u[tsel]
        xt = susp.x[tsel]
        ul, _ = local_point(box, alpha, rcut, mu, susp.x, g, xt)   # r = 0 pairs excluded
        ug, _, _ = global_fields(box, susp.x, g, mu, alpha, rcut)
        return (ul + evaluate(box, ug, xt, offgrid)
                - (4.0 * alpha / math.sqrt(math.pi)) * g[tsel] / (8.0 * math.pi * mu))
    wl = local_elem(box, alpha, rcut, 0, susp.x, susp.tri, q, targets=tsel)
    ug, _, _ = global_fields(box, susp.x, g, mu, alpha, rcut)
    return wl + evaluate(box, ug, susp.x[tsel], offgrid)


def double_layer(susp, q, quadrature="element", mu=1.0, alpha=None, rcut=None,
                 targets=None, offgrid="lagrange"):
    """v_j(z) = n_k(z) int q_i T_jik dS at the nodes (Sec. 3.5).  [N, 3]."""
    box = susp.box
    alpha = default_alpha(box) if alpha is None else alpha
    rcut = default_rcut(alpha) if rcut is None else rcut
    _, _, Ab, nb = geometry(susp.x, susp.tri)
    g = 8.0 * math.pi * mu * Ab[:, None] * _f64(q)
    tsel = np.arange(susp.x.shape[0]) if targets is None else np.asarray(targets)
    xt = susp.x[tsel]
    _, _, sg = global_fields(box, susp.x, g, mu, alpha, rcut, want_stress=True)
    vg = np.einsum("nk,njk->nj", nb[tsel], sym6_to_full(evaluate(box, sg, xt, offgrid))) / mu
    if quadrature == "nodal":
        _, sl = local_point(box, alpha, rcut, mu, susp.x, g, xt, want_u=False,
                            want_sig=True)
        return vg + np.einsum("nk,njk->nj", nb[tsel], sl) / mu
    vl = local_elem(box, alpha, rcut, 1, susp.x, susp.tri, q, nrm=nb, targets=tsel)
    return vg + vl


# ------------------------------------------------------------- Fredholm solve

def bie_operator(susp, kappa, q, quadrature="element", mu=1.0, alpha=None, rcut=None):
    """(I + kappa/(4 pi) D) q at the nodes (Sec. 5): q [N, 3], kappa [N] (the
    kappa_m = (lambda_m - 1)/(lambda_m + 1) of each node's particle, Eq. (qa)),
    D the discretised double layer of Sec. 3.5."""
    q = _f64(q)
    v = double_layer(susp, q, quadrature, mu, alpha, rcut)
    return q + (np.asarray(kappa, dtype=np.float64)[:, None] / (4.0 * math.pi)) * v


def gmres(apply, b, x0=None, tol=1e-6, restart=30, maxit=300):
    """Restarted GMRES(m) (Saad) for A x = b on flat FP64 vectors, with modified
    Gram-Schmidt Arnoldi, Givens rotations and the least-squares update at the
    end of each cycle.  Each cycle starts from the true residual b - A x.
    Stops when ||b - A x|| / ||b|| <= tol (true residual at the end of a cycle,
    the Arnoldi estimate inside one).  Returns (x, iterations, true relative
    residual, converged)."""
    b = np.asarray(b, dtype=np.float64).ravel()
    n = b.size
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros(n), 0, 0.0, True
    its = 0
    while True:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta / nb <= tol:
            return x, its, beta / nb, True
        if its >= maxit:
            return x, its, beta / nb, False
        m = min(restart, maxit - its)
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = apply(V[j])
            its += 1
            for i in range(j + 1):              # modified Gram-Schmidt
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                  # earlier rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            if abs(g[j + 1]) / nb <= tol or H[j, j] == 0.0:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + V[:k].T @ y


def bie_solve(susp, kappa, b, q0=None, tol=1e-6, restart=30, maxit=300,
              quadrature="element", mu=1.0, alpha=None, rcut=None):
    """q with (I + kappa/(4 pi) D) q = b by GMRES (Sec. 5).  b [N, 3] ->
    (q [N, 3], iterations, true relative residual, converged)."""
    n = susp.x.shape[0]

    def apply(v):
        return bie_operator(susp, kappa, v.reshape(n, 3), quadrature, mu, alpha, rcut).ravel()

    x, its, rr, ok = gmres(apply, np.asarray(b).ravel(), None if q0 is None else np.asarray(q0).ravel(),
                           tol, restart, maxit)
    return x.reshape(n, 3), its, rr, ok


def assembled_operator(susp, kappa, quadrature="element", mu=1.0, alpha=None, rcut=None):
    """The matrix of (I + kappa/(4 pi) D) on the flattened [N*3] densities,
    column by column from unit densities (small meshes only)."""
    n = susp.x.shape[0]
    return np.stack([bie_operator(susp, kappa, e.reshape(n, 3), quadrature, mu, alpha,
                                  rcut).ravel() for e in np.eye(3 * n)], 1)


def reference_box(box, ref_nx, ref_nz):
    """Slit of the isolated reference capsule of the per-particle block
    preconditioner: the wall gap, y0, Chebyshev grid and x-z grid spacing of
    `box` on a periodic cell of ref_nx x ref_nz grid intervals."""
    return type(box)(Lx=ref_nx * box.Lx / box.Nx, Lz=ref_nz * box.Lz / box.Nz, W=box.W,
                     y0=box.y0, Nx=ref_nx, Ny=box.Ny, Nz=ref_nz)


def reference_block_inverse(box, x_ref, tri_ref, kappa, ref_nx, ref_nz, quadrature="element",
                            mu=1.0, alpha=None, rcut=None):
    """Inverse of the [3 n, 3 n] matrix of (I + kappa/(4 pi) D) for one capsule
    alone (nodes x_ref [n, 3] relative to its centre, triangles tri_ref) placed
    at the centre of reference_box(box, ref_nx, ref_nz), with the splitting
    parameter and cutoff of `box` (alpha defaults to that of `box`, not of the
    smaller cell)."""
    import types
    rb = reference_box(box, ref_nx, ref_nz)
    alpha = default_alpha(box) if alpha is None else alpha
    c = np.array([0.5 * rb.Lx, rb.y0 + 0.5 * rb.W, 0.5 * rb.Lz])
    x = np.asarray(x_ref, dtype=np.float64) + c
    s = types.SimpleNamespace(box=rb, x=x, tri=np.asarray(tri_ref, dtype=np.int32),
                              particle=np.zeros(len(x), np.int32))
    A = assembled_operator(s, np.full(len(x), float(kappa)), quadrature, mu, alpha, rcut)
    return np.linalg.inv(A)


def particle_block_solve(susp, kappa, b, block_inverse, q0=None, tol=1e-6, restart=30,
                         maxit=300, quadrature="element", mu=1.0, alpha=None, rcut=None,
                         rotations=None):
    """The Fredholm solve of Sec. 5 with a right preconditioner M that applies
    the same dense [3 n_p, 3 n_p] matrix block_inverse to every particle's
    densities (nodes of a particle in increasing index order, n_p nodes each):
    GMRES on A M y = b - A q0, q = q0 + M y.  With rotations ([Np, 3, 3],
    particle p's orientation relative to the block's capsule), particle p's
    block is (I x R_p) block_inverse (I x R_p^T): its densities are turned
    into the reference orientation node by node, multiplied, and turned back.
    The paper uses no preconditioner; this is the reference for a
    per-particle block one.  Returns (q [N, 3], iterations, true relative
    residual of q, converged)."""
    n = susp.x.shape[0]
    parts = [np.flatnonzero(susp.particle == p) for p in range(int(susp.particle.max()) + 1)]
    cols = [np.stack([3 * idx, 3 * idx + 1, 3 * idx + 2], 1).ravel() for idx in parts]

    def A(v):
        return bie_operator(susp, kappa, v.reshape(n, 3), quadrature, mu, alpha, rcut).ravel()

    def M(v):
        out = np.empty_like(v)
        for p, c in enumerate(cols):
            if rotations is None:
                out[c] = block_inverse @ v[c]
            else:
                R = rotations[p]
                u = (v[c].reshape(-1, 3) @ R).ravel()            # R^T v_i at every node
                out[c] = ((block_inverse @ u).reshape(-1, 3) @ R.T).ravel()
        return out

    b = np.asarray(b, dtype=np.float64).ravel()
    q0 = np.zeros_like(b) if q0 is None else np.asarray(q0, dtype=np.float64).ravel()
    r0 = b - A(q0)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros((n, 3)), 0, 0.0, True
    # the inner tolerance is relative to ||r0||; the residual of q is that of y
    y, its, rr, ok = gmres(lambda v: A(M(v)), r0, None, tol * nb / max(np.linalg.norm(r0),
                                                                      1e-300), restart, maxit)
    q = q0 + M(y)
    rel = np.linalg.norm(b - A(q)) / nb
    return q.reshape(n, 3), its, rel, rel <= tol


# ------------------------------------------- rigid particles (Sec. 6.1)

def rigid_scales(susp, mu=1.0):
    """Per particle: surface area S_p = sum of its nodal areas and the radius
    R_p = sqrt(S_p / 4 pi) of the sphere with that area."""
    _, _, Ab, _ = geometry(susp.x, susp.tri)
    n_p = int(susp.particle.max()) + 1
    S = np.zeros(n_p)
    np.add.at(S, susp.particle, Ab)
    return S, np.sqrt(S / (4.0 * math.pi))


def rigid_operator(susp, centres, f, UO, quadrature="element", mu=1.0, alpha=None, rcut=None):
    """The rigid-particle system of Sec. 6.1 applied to (f, U, Omega).

    Velocity rows, one per node b of particle p (Eq. (sl_r) with the surface
    velocity U_p + Omega_p x (x_b - c_p) of a rigid body moved to the left):
        U_p + Omega_p x (x_b - c_p) + 1/(8 pi mu) int f_i G_ji dS
    Balance rows, per particle, in velocity units (reading: the paper states
    the force- and torque-free conditions but no discrete form or scaling):
        -(1/(6 pi mu R_p))   sum_b A_b f_b
        -(1/(8 pi mu R_p^2)) sum_b A_b (x_b - c_p) x f_b
    with the trapezoidal nodal areas A_b.  f [N, 3], UO [P, 6] (U, Omega).
    Returns (rows [N, 3], balance [P, 6])."""
    f = _f64(f)
    UO = _f64(UO).reshape(-1, 6)
    c = _f64(centres).reshape(-1, 3)
    p = susp.particle
    r = susp.x - c[p]
    w = single_layer(susp, f, quadrature, mu, alpha, rcut)
    rows = UO[p, :3] + np.cross(UO[p, 3:], r) + w / (8.0 * math.pi * mu)
    _, _, Ab, _ = geometry(susp.x, susp.tri)
    _, R = rigid_scales(susp, mu)
    n_p = UO.shape[0]
    F = np.zeros((n_p, 3))
    T = np.zeros((n_p, 3))
    np.add.at(F, p, Ab[:, None] * f)
    np.add.at(T, p, Ab[:, None] * np.cross(r, f))
    bal = np.hstack([-F / (6.0 * math.pi * mu * R[:, None]),
                     -T / (8.0 * math.pi * mu * R[:, None] ** 2)])
    return rows, bal


def rigid_rhs(susp, u_inf, ext=None, mu=1.0):
    """Right side of the rigid-particle system: u_inf at the nodes, and the
    external force and torque ext [P, 6] (None: force- and torque-free) in
    the balance rows' units, so that the solution has
    sum_b A_b f_b = -F_ext and sum_b A_b (x_b - c) x f_b = -T_ext."""
    n_p = int(susp.particle.max()) + 1
    _, R = rigid_scales(susp, mu)
    bal = np.zeros((n_p, 6))
    if ext is not None:
        e = _f64(ext).reshape(n_p, 6)
        bal[:, :3] = e[:, :3] / (6.0 * math.pi * mu * R[:, None])
        bal[:, 3:] = e[:, 3:] / (8.0 * math.pi * mu * R[:, None] ** 2)
    return _f64(u_inf).reshape(-1, 3), bal


def rigid_solve(susp, centres, u_inf, ext=None, tol=1e-6, restart=30, maxit=300,
                quadrature="element", mu=1.0, alpha=None, rcut=None, x0=None):
    """Tractions and rigid-body velocities of force- and torque-free (or
    externally loaded) rigid particles in the undisturbed flow u_inf
    (Sec. 6.1), by restarted GMRES on the unknowns (f [N, 3], U, Omega [P, 6]).
    Returns (f, UO, iterations, true relative residual, converged)."""
    n = susp.x.shape[0]
    n_p = int(susp.particle.max()) + 1
    rows_b, bal_b = rigid_rhs(susp, u_inf, ext, mu)
    b = np.concatenate([rows_b.ravel(), bal_b.ravel()])

    def apply(z):
        rows, bal = rigid_operator(susp, centres, z[:3 * n].reshape(n, 3),
                                   z[3 * n:].reshape(n_p, 6), quadrature, mu, alpha, rcut)
        return np.concatenate([rows.ravel(), bal.ravel()])

    z, its, rr, ok = gmres(apply, b, x0, tol, restart, maxit)
    return z[:3 * n].reshape(n, 3), z[3 * n:].reshape(n_p, 6), its, rr, ok
