// Cell list and GGEM local sums (paper Sec. 3.2.1, Eqs. (local), (u_loc)).
//
// Sources are binned into cells no smaller than r_cut/R (R = 2 or 3, the
// grid's search reach) and stored as offsets
// from their cell's corner, so every displacement is formed from small
// numbers (integer cell shift + offset difference) and stays accurate in FP32
// whatever the box size.  x and z are periodic: the neighbour shift of up to
// +-R cells carries the image; as r_cut < L/2 (Sec. 3.2.2, alpha L > 8), at
// most one image of a source lies within r_cut even where a small grid
// visits a cell twice.
#include <type_traits>

#include "ggem_internal.cuh"
#include "ggem_erfcx.cuh"
#include "ggem_ff.cuh"

namespace ggem {

template <typename T> __device__ __forceinline__ T d_rsqrt(T x);
// FP32: the hardware approximations (about 2 ulp); r^2 lies in (0, r_cut^2) and
// the exponent in (-23, 0], far from denormal inputs and results
template <> __device__ __forceinline__ float d_rsqrt<float>(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <> __device__ __forceinline__ double d_rsqrt<double>(double x) { return rsqrt(x); }

// locate a point: cell coordinates and offsets from the cell corner
__device__ __forceinline__ void locate(const GridGeom& geo, const CellGrid& cg, double x,
                                       double y, double z, int& cx, int& cy, int& cz,
                                       double& ox, double& oy, double& oz) {
    double xw = x - geo.Lx * floor(x / geo.Lx);
    double zw = z - geo.Lz * floor(z / geo.Lz);
    double yr = y - cg.y0;
    cx = min(max((int)(xw / cg.hx), 0), cg.ncx - 1);
    cz = min(max((int)(zw / cg.hz), 0), cg.ncz - 1);
    cy = min(max((int)floor(yr / cg.hy), 0), cg.ncy - 1);
    ox = xw - cx * cg.hx;
    oy = yr - cy * cg.hy;
    oz = zw - cz * cg.hz;
}

__global__ void k_cell_count(GridGeom geo, CellGrid cg, int n, const double* __restrict__ x,
                             int* __restrict__ count, int* __restrict__ cell_of) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx, cy, cz;
    double ox, oy, oz;
    locate(geo, cg, x[3 * i], x[3 * i + 1], x[3 * i + 2], cx, cy, cz, ox, oy, oz);
    int c = (cz * cg.ncy + cy) * cg.ncx + cx;
    cell_of[i] = c;
    atomicAdd(&count[c], 1);
}

// exclusive scan of count[0..n) into start[0..n], one block
__global__ void k_scan(int n, const int* __restrict__ count, int* __restrict__ start) {
    __shared__ int part[1024];
    int tid = threadIdx.x, nt = blockDim.x;
    int chunk = (n + nt - 1) / nt;
    int b = tid * chunk, e = min(n, b + chunk);
    int s = 0;
    for (int i = b; i < e; ++i) s += count[i];
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        int v = (tid >= off) ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int run = (tid == 0) ? 0 : part[tid - 1];
    for (int i = b; i < e; ++i) {
        start[i] = run;
        run += count[i];
    }
    if (tid == nt - 1) start[n] = part[nt - 1];
}

template <typename T>
__global__ void k_cell_scatter(GridGeom geo, CellGrid cg, int n, const double* __restrict__ x,
                               const int* __restrict__ cell_of, const int* __restrict__ start,
                               int* __restrict__ cursor, int* __restrict__ src_cell,
                               int* __restrict__ perm, v4_t<T>* __restrict__ pos) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx, cy, cz;
    double ox, oy, oz;
    locate(geo, cg, x[3 * i], x[3 * i + 1], x[3 * i + 2], cx, cy, cz, ox, oy, oz);
    int c = cell_of[i];
    int slot = start[c] + atomicAdd(&cursor[c], 1);
    perm[slot] = i;
    src_cell[slot] = c;
    v4_t<T> p;
    p.x = (T)ox; p.y = (T)oy; p.z = (T)oz; p.w = (T)0;
    pos[slot] = p;
}

__global__ void k_gather_int4(int n, const int* __restrict__ perm, const int4* __restrict__ in,
                              int4* __restrict__ out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) out[s] = in[perm[s]];
}

cudaError_t gather_int4(int n, const int* perm, const int4* in, int4* out, cudaStream_t st) {
    if (n > 0) k_gather_int4<<<(n + 255) / 256, 256, 0, st>>>(n, perm, in, out);
    return cudaGetLastError();
}

cudaError_t scan_counts(int n, const int* count, int* start, cudaStream_t st) {
    if (n > 0) k_scan<<<1, 1024, 0, st>>>(n, count, start);
    return cudaGetLastError();
}

template <typename T>
cudaError_t build_cells(const GridGeom& geo, const CellGrid& cg, int n, const double* x,
                        int* cell_count, int* cell_start, int* cursor, int* src_cell,
                        int* perm, v4_t<T>* pos, cudaStream_t st) {
    int ncell = cg.ncx * cg.ncy * cg.ncz;
    cudaMemsetAsync(cell_count, 0, ncell * sizeof(int), st);
    cudaMemsetAsync(cursor, 0, ncell * sizeof(int), st);
    if (n > 0) {
        // src_cell doubles as the per-source cell scratch before the scatter
        int* cell_of = cursor + ncell;   // caller provides cursor[ncell + n]
        k_cell_count<<<(n + 255) / 256, 256, 0, st>>>(geo, cg, n, x, cell_count, cell_of);
        k_scan<<<1, 1024, 0, st>>>(ncell, cell_count, cell_start);
        k_cell_scatter<T><<<(n + 255) / 256, 256, 0, st>>>(geo, cg, n, x, cell_of, cell_start,
                                                           cursor, src_cell, perm, pos);
    } else {
        cudaMemsetAsync(cell_start, 0, (ncell + 1) * sizeof(int), st);
    }
    return cudaGetLastError();
}

template <typename T>
__global__ void k_gather(int n, const int* __restrict__ perm, const double* __restrict__ q,
                         const double* __restrict__ w, double scale, v4_t<T>* __restrict__ g) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = perm[s];
    double f = scale * (w ? w[i] : 1.0);
    v4_t<T> v;
    v.x = (T)(f * q[3 * i]); v.y = (T)(f * q[3 * i + 1]); v.z = (T)(f * q[3 * i + 2]);
    v.w = (T)0;
    g[s] = v;
}

template <typename T>
cudaError_t gather_strengths(int n, const int* perm, const double* q, const double* w,
                             double scale, v4_t<T>* g, cudaStream_t st) {
    if (n > 0) k_gather<T><<<(n + 255) / 256, 256, 0, st>>>(n, perm, q, w, scale, g);
    return cudaGetLastError();
}

// ------------------------------------------------------------- local sum
// Kernel constants in T, computed on the host so that the kernels execute no
// FP64 instruction (GB300 issues FP64 at a small fraction of the FP32 rate).
template <typename T> struct LocalConst {
    T al, al2, rc2, c1, c2, c3, c4, fU, fS, hx, hy, hz;
    T ke;   // -alpha^2 log2(e): exp(-alpha^2 r^2) = 2^(ke r^2)
    // FP32 element rule (scaled coordinates, set by local_sum_elem): the
    // coordinate scale s, the reciprocal's slope P alpha / s, and -6 s^3
    T sc = (T)1, pt = (T)0, c6 = (T)-6;
};

template <typename T> LocalConst<T> local_const(const GridGeom& geo, const CellGrid& cg) {
    const double sp = 1.7724538509055160273, pi = 3.14159265358979323846;
    double a = geo.alpha;
    LocalConst<T> k;
    k.al = (T)a; k.al2 = (T)(a * a); k.rc2 = (T)(geo.rcut * geo.rcut);
    k.c1 = (T)(2.0 * a / sp); k.c2 = (T)(12.0 * a / sp);
    k.c3 = (T)(8.0 * a * a * a / sp); k.c4 = (T)(4.0 * a * a * a / sp);
    k.fU = (T)(1.0 / (8.0 * pi * geo.mu)); k.fS = (T)(1.0 / (8.0 * pi));
    k.hx = (T)cg.hx; k.hy = (T)cg.hy; k.hz = (T)cg.hz;
    k.ke = (T)(-a * a * 1.4426950408889634074);
    return k;
}

template <typename T> struct LocalArgs {
    GridGeom geo;
    CellGrid cg;
    LocalConst<T> k;
    SortedSources<T> src;
    const int4* qvs;         // element rule: vertices of each sorted point's triangle
    T near2;                 // element rule: points closer than this may share a triangle
    int n_tgt;
    const int* tcell;        // TK_POINTS / TK_WALL: located targets (cell, offsets)
    const v4_t<T>* tpos;
    const int* tperm;        // TK_POINTS: caller index of target t (nullptr: t itself)
    const double* nrm;       // OUT_DBL: [n][3] target normals (caller order)
    T* out;
    int out_stride;
    const int* qinv = nullptr;   // FP32 element rule: padded slot -> sorted point (-1: dummy)
};

// Locate targets once (one thread each, FP64): cell index and offsets from
// the cell corner in T.  kind TK_POINTS reads x[n][3]; TK_WALL generates the
// wall grid nodes (x_i, y0 or y0+W, z_k), index = (wall * Nz + k) * Nx + i.
template <typename T>
__global__ void k_locate(GridGeom geo, CellGrid cg, int n, int kind, const double* __restrict__ x,
                         int* __restrict__ cell, v4_t<T>* __restrict__ pos) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double xx, yy, zz;
    if (kind == TK_POINTS) {
        xx = x[3 * t]; yy = x[3 * t + 1]; zz = x[3 * t + 2];
    } else {
        int nxz = geo.Nz * geo.Nx;
        int w = t / nxz, rem = t - w * nxz;
        int k = rem / geo.Nx, i = rem - k * geo.Nx;
        xx = i * geo.dx; zz = k * geo.dz; yy = geo.y0 + w * geo.W;
    }
    int cx, cy, cz;
    double ox, oy, oz;
    locate(geo, cg, xx, yy, zz, cx, cy, cz, ox, oy, oz);
    cell[t] = (cz * cg.ncy + cy) * cg.ncx + cx;
    v4_t<T> p;
    p.x = (T)ox; p.y = (T)oy; p.z = (T)oz; p.w = (T)0;
    pos[t] = p;
}

template <typename T>
cudaError_t locate_targets(const GridGeom& geo, const CellGrid& cg, int n, int kind,
                           const double* x, int* cell, v4_t<T>* pos, cudaStream_t st) {
    if (n > 0) k_locate<T><<<(n + 255) / 256, 256, 0, st>>>(geo, cg, n, kind, x, cell, pos);
    return cudaGetLastError();
}

// Pair arithmetic of Eq. (local), shared by the local-sum kernels.
// exp(-alpha^2 r^2) and erfc(alpha r) = exp(-x^2) erfcx(x) with the
// approximations of ggem_erfcx.cuh (FP32: t Q(t), t = 1/(1 + P x), Q of degree
// 7; FP64: 8 polynomial pieces of degree 12, coefficients in shared memory),
// so the pair needs one exponential and no erfc call; the FP32 exponential is
// 2^(ke r^2), the FP32 reciprocal the hardware's.
template <typename T> struct PairAcc {
    T ux = 0, uy = 0, uz = 0;
    T sxx = 0, sxy = 0, sxz = 0, syy = 0, syz = 0, szz = 0;
};

__device__ __forceinline__ float rcp_ftz(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void exp_erfc(const LocalConst<float>& k, float r2, float x, float& ex,
                                         float& ec, const double*) {
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ex) : "f"(k.ke * r2));
    ec = ex * erfcx_t(rcp_ftz(fmaf(x, GGEM_ERFCX_P, 1.0f)));
}
__device__ __forceinline__ void exp_erfc(const LocalConst<double>& k, double r2, double x,
                                         double& ex, double& ec, const double* tab) {
    ex = exp(-k.al2 * r2);
    ec = ex * erfcx_poly(x, tab);
}

// adds G^l g (OUT_U), T^l g (OUT_S) or n . T^l g (OUT_DBL) for displacement
// (dx, dy, dz) = target - source, 0 < r2 < rc2
template <typename T, int MODE>
__device__ __forceinline__ void pair_terms(const LocalConst<T>& k, T dx, T dy, T dz, T r2,
                                           const v4_t<T>& g, T nx, T ny, T nz, PairAcc<T>& a,
                                           const double* tab) {
    const T ir = d_rsqrt<T>(r2);
    const T r = r2 * ir;
    T ex, ec;
    exp_erfc(k, r2, k.al * r, ex, ec, tab);
    const T xg = dx * g.x + dy * g.y + dz * g.z;
    if (MODE & OUT_U) {
        const T A = ec * ir - k.c1 * ex;
        const T B = (ec * ir * ir * ir + k.c1 * ex * ir * ir) * xg;
        a.ux += A * g.x + B * dx;
        a.uy += A * g.y + B * dy;
        a.uz += A * g.z + B * dz;
    }
    if (MODE & (OUT_S | OUT_DBL)) {
        const T ir2 = ir * ir;
        const T D = -(T)6 * ec * ir2 * ir2 * ir - k.c2 * ex * ir2 * ir2 - k.c3 * ex * ir2;
        const T E = k.c4 * ex;
        if (MODE & OUT_S) {
            const T Dx = D * xg;
            a.sxx += Dx * dx * dx + E * ((T)2 * g.x * dx + xg);
            a.syy += Dx * dy * dy + E * ((T)2 * g.y * dy + xg);
            a.szz += Dx * dz * dz + E * ((T)2 * g.z * dz + xg);
            a.sxy += Dx * dx * dy + E * (g.y * dx + g.x * dy);
            a.sxz += Dx * dx * dz + E * (g.z * dx + g.x * dz);
            a.syz += Dx * dy * dz + E * (g.z * dy + g.y * dz);
        } else {
            const T xn = dx * nx + dy * ny + dz * nz;
            const T gn = g.x * nx + g.y * ny + g.z * nz;
            const T Dxn = D * xg * xn;
            a.ux += Dxn * dx + E * (dx * gn + g.x * xn + nx * xg);
            a.uy += Dxn * dy + E * (dy * gn + g.y * xn + ny * xg);
            a.uz += Dxn * dz + E * (dz * gn + g.z * xn + nz * xg);
        }
    }
}

// Two candidate pairs at once, FP32 (element rule): the arithmetic of
// pair_terms on paired lanes (add/mul/fma .f32x2), so one issued instruction
// serves two pairs; rsqrt and exp2 stay scalar.  Every multiply-add is an
// explicit FMA.
struct PairAcc2 {
    f2 ux = {0ull}, uy = {0ull}, uz = {0ull};
    f2 sn = {0ull};     // double layer: sum of E x.g (times the target normal at the end)
};

__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_ftz(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// In the FP32 element rule the coordinates are scaled by s = alpha sqrt(log2 e)
// (local_sum_elem), so exp(-alpha^2 r^2) = 2^(-r_s^2) takes no multiply; the
// displacements, r and 1/r below are in scaled units, and the constants
// (c1 / s, c2 s^2, -6 s^3, the output factor s or 1 / s) make every term the
// unscaled one.
template <int MODE>
__device__ __forceinline__ void pair_terms2(const LocalConst<float>& k, f2 dx, f2 dy, f2 dz,
                                            f2 r2, f2 gx, f2 gy, f2 gz, f2 nx, f2 ny, f2 nz,
                                            PairAcc2& a) {
    float lo, hi;
    f2_split(r2, lo, hi);
    const f2 ir = f2_make(rsqrt_ftz(lo), rsqrt_ftz(hi));
    const f2 ex = f2_make(ex2_ftz(-lo), ex2_ftz(-hi));               // exp(-alpha^2 r^2)
    const f2 r = r2 * ir;
    f2_split(fma2(r, f2_splat(k.pt), f2_splat(1.0f)), lo, hi);
    const f2 t = f2_make(rcp_ftz(lo), rcp_ftz(hi));                 // 1/(1 + P alpha r)
    const f2 ec = ex * erfcx_t2(t);                                  // erfc(alpha r)
    const f2 xg = fma2(dz, gz, fma2(dy, gy, dx * gx));
    if (MODE & OUT_U) {
        // A = ec/r - c1 ex,  B = (ec/r^3 + c1 ex/r^2) xg
        const f2 eir = ec * ir;
        const f2 A = fma2(f2_splat(-k.c1), ex, eir);
        const f2 B = (ir * ir) * fma2(f2_splat(k.c1), ex, eir) * xg;
        a.ux = fma2(B, dx, fma2(A, gx, a.ux));
        a.uy = fma2(B, dy, fma2(A, gy, a.uy));
        a.uz = fma2(B, dz, fma2(A, gz, a.uz));
    }
    if (MODE & OUT_DBL) {
        // D = -6 ec/r^5 - c2 ex/r^4 - c3 ex/r^2 = ir2 (ir2 (-6 ec ir - c2 ex) - c3 ex),
        // E = c4 ex; the update D xg xn d + E (d gn + g xn + n xg) regrouped as
        // d (D xg xn + E gn) + g (E xn) + n (E xg), the last term's scalar E xg
        // summed over the pairs and multiplied by the (fixed) target normal once
        const f2 ir2 = ir * ir;
        const f2 t = fma2(f2_splat(k.c6), ec * ir, f2_splat(-k.c2) * ex);
        const f2 D = ir2 * fma2(ir2, t, f2_splat(-k.c3) * ex);
        const f2 E = f2_splat(k.c4) * ex;
        const f2 xn = fma2(dz, nz, fma2(dy, ny, dx * nx));
        const f2 gn = fma2(gz, nz, fma2(gy, ny, gx * nx));
        const f2 cd = fma2(D * xg, xn, E * gn), cg = E * xn;
        a.sn = fma2(E, xg, a.sn);
        a.ux = fma2(dx, cd, fma2(gx, cg, a.ux));
        a.uy = fma2(dy, cd, fma2(gy, cg, a.uy));
        a.uz = fma2(dz, cd, fma2(gz, cg, a.uz));
    }
}

// scaled output of one target in caller order
template <typename T, int MODE>
__device__ __forceinline__ void store_target(const LocalConst<T>& k, const PairAcc<T>& a, T* o) {
    int c = 0;
    if (MODE & (OUT_U | OUT_DBL)) {
        o[0] = k.fU * a.ux; o[1] = k.fU * a.uy; o[2] = k.fU * a.uz;
        c = 3;
    }
    if (MODE & OUT_S) {
        o[c] = k.fS * a.sxx; o[c + 1] = k.fS * a.sxy; o[c + 2] = k.fS * a.sxz;
        o[c + 3] = k.fS * a.syy; o[c + 4] = k.fS * a.syz; o[c + 5] = k.fS * a.szz;
    }
}

// Target t: position in its cell's frame, cell coordinates and caller index.
template <typename T, int KIND>
__device__ __forceinline__ void load_target(const LocalArgs<T>& a, int t, T& ox, T& oy, T& oz,
                                            int& cx, int& cy, int& cz, int& oidx) {
    const CellGrid& cg = a.cg;
    v4_t<T> p;
    int c;
    oidx = t;
    if (KIND == TK_SORTED) {
        p = a.src.pos[t];
        c = a.src.cell[t];
        oidx = a.src.perm[t];
    } else {
        p = a.tpos[t];
        c = a.tcell[t];
        if (a.tperm) oidx = a.tperm[t];
    }
    ox = p.x; oy = p.y; oz = p.z;
    cx = c % cg.ncx;
    cy = (c / cg.ncx) % cg.ncy;
    cz = c / (cg.ncx * cg.ncy);
}

// The warp's list of neighbour cells at offsets -R..R (cells are at least
// r_cut/R wide): the non-empty ones whose nearest point lies within r_cut of
// the target (a slightly widened r_cut, so rounding can only keep more).
// Writes first source, count and offset index of each into the warp's
// shared-memory lists; returns their number (warp-uniform).
template <typename T, int R>
__device__ __forceinline__ int cull_cells(const LocalArgs<T>& a, int lane, T ox, T oy, T oz,
                                          int cx, int cy, int cz, int* s_cst, int* s_cnt,
                                          unsigned short* s_off) {
    const CellGrid& cg = a.cg;
    const unsigned lt = (1u << lane) - 1u;
    const T reach2 = a.k.rc2 * (T)1.0001;
    constexpr int side = 2 * R + 1, nb = side * side * side;
    int nc = 0;
    for (int r = 0; r < (nb + 31) / 32; ++r) {
        const int oi = r * 32 + lane;
        bool keep = false;
        int st = 0, cnt = 0;
        if (oi < nb) {
            const int ix = oi % side - R, iy = (oi / side) % side - R, iz = oi / (side * side) - R;
            const int cyy = cy + iy;
            if (cyy >= 0 && cyy < cg.ncy) {
                const T gx = ix > 0 ? (T)ix * a.k.hx - ox : (ix < 0 ? ox - (T)(ix + 1) * a.k.hx : (T)0);
                const T gy = iy > 0 ? (T)iy * a.k.hy - oy : (iy < 0 ? oy - (T)(iy + 1) * a.k.hy : (T)0);
                const T gz = iz > 0 ? (T)iz * a.k.hz - oz : (iz < 0 ? oz - (T)(iz + 1) * a.k.hz : (T)0);
                if (gx * gx + gy * gy + gz * gz <= reach2) {
                    // ncx, ncz >= 2 R (L > 2 r_cut): one wrap suffices for |i| <= R
                    int cxx = cx + ix, czz = cz + iz;
                    cxx += (cxx < 0) ? cg.ncx : 0;
                    cxx -= (cxx >= cg.ncx) ? cg.ncx : 0;
                    czz += (czz < 0) ? cg.ncz : 0;
                    czz -= (czz >= cg.ncz) ? cg.ncz : 0;
                    const int c = (czz * cg.ncy + cyy) * cg.ncx + cxx;
                    st = a.src.cell_start[c];
                    cnt = a.src.cell_start[c + 1] - st;
                    keep = cnt > 0;
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int slot = nc + __popc(m & lt);
            s_cst[slot] = st;
            s_cnt[slot] = cnt;
            s_off[slot] = (unsigned short)oi;
        }
        nc += __popc(m);
    }
    __syncwarp();
    return nc;
}

// The same culling in batches: rounds of 32 neighbour offsets from *round
// on, stopping before a round could overflow `cap` entries; *round is left at
// the first round not culled (nb rounds = done).  Bit 15 of s_off marks the
// cells within near2 of the target (the only ones that can hold points of
// the triangles around it).
template <typename T, int R>
__device__ __forceinline__ int cull_cells_batch(const LocalArgs<T>& a, int lane, T ox, T oy,
                                                T oz, int cx, int cy, int cz, int* s_cst,
                                                int* s_cnt, unsigned short* s_off, int& round,
                                                int cap) {
    const CellGrid& cg = a.cg;
    const unsigned lt = (1u << lane) - 1u;
    const T reach2 = a.k.rc2 * (T)1.0001;
    constexpr int side = 2 * R + 1, nb = side * side * side, nr = (nb + 31) / 32;
    int nc = 0;
    for (; round < nr && nc + 32 <= cap; ++round) {
        const int oi = round * 32 + lane;
        bool keep = false, nearc = false;
        int st = 0, cnt = 0;
        if (oi < nb) {
            const int ix = oi % side - R, iy = (oi / side) % side - R, iz = oi / (side * side) - R;
            const int cyy = cy + iy;
            if (cyy >= 0 && cyy < cg.ncy) {
                const T gx = ix > 0 ? (T)ix * a.k.hx - ox : (ix < 0 ? ox - (T)(ix + 1) * a.k.hx : (T)0);
                const T gy = iy > 0 ? (T)iy * a.k.hy - oy : (iy < 0 ? oy - (T)(iy + 1) * a.k.hy : (T)0);
                const T gz = iz > 0 ? (T)iz * a.k.hz - oz : (iz < 0 ? oz - (T)(iz + 1) * a.k.hz : (T)0);
                const T d2 = gx * gx + gy * gy + gz * gz;
                nearc = d2 <= a.near2 * (T)1.0001;
                if (d2 <= reach2) {
                    int cxx = cx + ix, czz = cz + iz;
                    cxx += (cxx < 0) ? cg.ncx : 0;
                    cxx -= (cxx >= cg.ncx) ? cg.ncx : 0;
                    czz += (czz < 0) ? cg.ncz : 0;
                    czz -= (czz >= cg.ncz) ? cg.ncz : 0;
                    const int c = (czz * cg.ncy + cyy) * cg.ncx + cxx;
                    st = a.src.cell_start[c];
                    cnt = a.src.cell_start[c + 1] - st;
                    keep = cnt > 0;
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int slot = nc + __popc(m & lt);
            s_cst[slot] = st;
            s_cnt[slot] = cnt;
            s_off[slot] = (unsigned short)(oi | (nearc ? 0x8000 : 0));
        }
        nc += __popc(m);
    }
    __syncwarp();
    return nc;
}

// u_i = sum G^l_ij g_j ; sigma_ik = sum T^l_ijk g_j ; v_i = n_k sigma_ik
// (unscaled in the loop; the caller-facing factors are applied at the end).
//
// One warp per target.  The warp lists the neighbour cells (offsets -R..R)
// that come within r_cut of the target, then walks them one at a time with
// consecutive lanes on consecutive sorted sources (coalesced float4 loads).
// The hits are compacted into a per-warp queue and evaluated 32 at a time.
// Partial sums are reduced with warp shuffles.
constexpr int LW = 8;       // warps (targets) per block
constexpr int kQueue = 64;  // hit queue per warp: < 32 left + <= 32 new always fit
constexpr int kNb = 7 * 7 * 7;   // neighbour cell offsets for the largest reach (3)

// ELEM: sources are element quadrature points and targets are mesh nodes
// (caller index t); points of triangles having the target as a vertex are
// skipped (their integral is done by the polar rule, Sec. 3.4.1).  Used in
// FP64; the FP32 element rule runs in k_local_elem32 below.
template <typename T, int KIND, int MODE, bool ELEM, int REACH>
__global__ void __launch_bounds__(LW * 32) k_local(LocalArgs<T> a) {
    __shared__ int s_cst[LW][kNb];            // this target's cells: first source,
    __shared__ int s_cnt[LW][kNb];            //   source count,
    __shared__ unsigned short s_off[LW][kNb]; //   neighbour offset index
    __shared__ v4_t<T> s_qd[LW][kQueue];     // queued hits: displacement, r^2
    __shared__ int s_qs[LW][kQueue];         // queued hits: sorted source index
    __shared__ double s_tab[sizeof(T) == 8 ? (GGEM_ERFCX64_DEG + 1) * GGEM_ERFCX64_NINT : 1];
    if (sizeof(T) == 8) {
        for (int e = threadIdx.x; e < (GGEM_ERFCX64_DEG + 1) * GGEM_ERFCX64_NINT; e += blockDim.x)
            s_tab[e] = kErfcxTab64[e];
        __syncthreads();
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * LW + wid;
    if (t >= a.n_tgt) return;                     // warp-uniform
    int cx, cy, cz, oidx;
    T ox, oy, oz;
    load_target<T, KIND>(a, t, ox, oy, oz, cx, cy, cz, oidx);
    constexpr int R = REACH, side = 2 * R + 1;
    const unsigned lt = (1u << lane) - 1u;
    const int nc = cull_cells<T, R>(a, lane, ox, oy, oz, cx, cy, cz, s_cst[wid], s_cnt[wid],
                                    s_off[wid]);
    T nx = 0, ny = 0, nz = 0;
    if (MODE & OUT_DBL) {
        nx = (T)a.nrm[3 * oidx]; ny = (T)a.nrm[3 * oidx + 1]; nz = (T)a.nrm[3 * oidx + 2];
    }
    const T rc2 = a.k.rc2;
    PairAcc<T> acc;
    // Lanes test consecutive sources of one cell at a time; hits go to a
    // per-warp ring queue (ballot + popc ranks) and the pair arithmetic runs on
    // 32 queued hits at a time, so no lane idles through it on a miss.
    int head = 0, qn = 0;                         // warp-uniform
    for (int ci = 0; ci < nc; ++ci) {
        const int st = s_cst[wid][ci], cnt = s_cnt[wid][ci], oi = s_off[wid][ci];
        // target position in the frame of this source cell's corner
        const T tx = ox - (T)(oi % side - R) * a.k.hx;
        const T ty = oy - (T)((oi / side) % side - R) * a.k.hy;
        const T tz = oz - (T)(oi / (side * side) - R) * a.k.hz;
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            bool hit = false;
            T dx = 0, dy = 0, dz = 0, r2 = 0;
            int s = 0;
            if (i < cnt) {
                s = st + i;
                const v4_t<T> p = a.src.pos[s];
                dx = tx - p.x;
                dy = ty - p.y;
                dz = tz - p.z;
                r2 = dx * dx + dy * dy + dz * dz;
                hit = r2 < rc2 && r2 > (T)0;
                if (ELEM && hit && r2 < a.near2) {
                    const int4 v = a.qvs[s];
                    hit = !(v.x == oidx || v.y == oidx || v.z == oidx);
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int slot = (head + qn + __popc(m & lt)) & (kQueue - 1);
                v4_t<T> d;
                d.x = dx; d.y = dy; d.z = dz; d.w = r2;
                s_qd[wid][slot] = d;
                s_qs[wid][slot] = s;
            }
            qn += __popc(m);
            if (qn >= 32) {
                __syncwarp();
                const int slot = (head + lane) & (kQueue - 1);
                const v4_t<T> d = s_qd[wid][slot];
                pair_terms<T, MODE>(a.k, d.x, d.y, d.z, d.w, a.src.g[s_qs[wid][slot]], nx, ny,
                                    nz, acc, s_tab);
                head = (head + 32) & (kQueue - 1);
                qn -= 32;
                __syncwarp();
            }
        }
    }
    __syncwarp();
    if (lane < qn) {
        const int slot = (head + lane) & (kQueue - 1);
        const v4_t<T> d = s_qd[wid][slot];
        pair_terms<T, MODE>(a.k, d.x, d.y, d.z, d.w, a.src.g[s_qs[wid][slot]], nx, ny, nz, acc,
                            s_tab);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (MODE & (OUT_U | OUT_DBL)) {
            acc.ux += __shfl_xor_sync(0xffffffffu, acc.ux, o);
            acc.uy += __shfl_xor_sync(0xffffffffu, acc.uy, o);
            acc.uz += __shfl_xor_sync(0xffffffffu, acc.uz, o);
        }
        if (MODE & OUT_S) {
            acc.sxx += __shfl_xor_sync(0xffffffffu, acc.sxx, o);
            acc.sxy += __shfl_xor_sync(0xffffffffu, acc.sxy, o);
            acc.sxz += __shfl_xor_sync(0xffffffffu, acc.sxz, o);
            acc.syy += __shfl_xor_sync(0xffffffffu, acc.syy, o);
            acc.syz += __shfl_xor_sync(0xffffffffu, acc.syz, o);
            acc.szz += __shfl_xor_sync(0xffffffffu, acc.szz, o);
        }
    }
    if (lane != 0) return;
    if (KIND == TK_WALL) {
        // global wall data u^g = -u^l (Sec. 3.2.2), layout [wall][c][Nz][Nx]
        const T f = -a.k.fU;
        const int nxz = a.geo.Nz * a.geo.Nx;
        const int wall = t / nxz, rem = t - wall * nxz;
        T* o = a.out + (size_t)wall * 3 * nxz + rem;
        o[0] = f * acc.ux;
        o[nxz] = f * acc.uy;
        o[2 * nxz] = f * acc.uz;
        return;
    }
    store_target<T, MODE>(a.k, acc, a.out + (size_t)oidx * a.out_stride);
}

// ------------------------------------------------- FP32 element rule
// The element-rule local sum in FP32 reads ~700 quadrature points per cell
// and finds about 80 % of them within r_cut, so no hit queue: every lane
// takes two adjacent candidates of each 64-point step through a cell and
// evaluates both with paired FP32 arithmetic.  The points are read from a
// packed copy, 48 bytes per pair of adjacent points (x0 x1 y0 y1 | z0 z1 gx0
// gx1 | gy0 gy1 gz0 gz1), so a lane's two candidates arrive with three 16-byte
// loads, every coordinate already paired; the layout is padded: each cell
// starts on a multiple of 64 points and fills whole steps with dummies of zero
// strength far away, so a step needs no bounds test.
// Candidates beyond r_cut are evaluated unmasked: their terms carry
// exp(-alpha^2 r^2) <= e^-16 (and erfc(alpha r) <= 1.6e-8), below the FP32
// rounding of the sum, and a step with no candidate within r_cut is skipped.
// Points of the triangles around the target (left to the singular
// correction) can only lie in the cells the culling marks near; only there
// is each candidate within near2 checked and, if excluded, given zero strength.
constexpr int LWE = 4;        // warps (targets) per block; 10 blocks per SM (48 registers)
constexpr int kCap = 128;     // culled cells per batch (a target may need several batches)
constexpr int kChunk = 64;    // candidates per warp step

template <int MODE, int REACH>
__global__ void __launch_bounds__(LWE * 32, 10) k_local_elem32(LocalArgs<float> a,
                                                          const float4* __restrict__ pk) {
    __shared__ int s_cst[LWE][kCap];
    __shared__ int s_cnt[LWE][kCap];
    __shared__ unsigned short s_off[LWE][kCap];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * LWE + wid;
    if (t >= a.n_tgt) return;                     // warp-uniform
    int cx, cy, cz, oidx;
    float ox, oy, oz;
    load_target<float, TK_POINTS>(a, t, ox, oy, oz, cx, cy, cz, oidx);
    ox *= a.k.sc;                                 // scaled coordinates (set by local_sum_elem)
    oy *= a.k.sc;
    oz *= a.k.sc;
    constexpr int R = REACH, side = 2 * R + 1;
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (MODE & OUT_DBL) {
        nx = (float)a.nrm[3 * oidx]; ny = (float)a.nrm[3 * oidx + 1]; nz = (float)a.nrm[3 * oidx + 2];
    }
    const f2 nx2 = f2_splat(nx), ny2 = f2_splat(ny), nz2 = f2_splat(nz);
    const float rc2 = a.k.rc2;
    PairAcc2 acc;
    for (int round = 0; round < (side * side * side + 31) / 32;) {
    const int nc = cull_cells_batch<float, R>(a, lane, ox, oy, oz, cx, cy, cz, s_cst[wid],
                                              s_cnt[wid], s_off[wid], round, kCap);
    for (int ci = 0; ci < nc; ++ci) {
        const int st = s_cst[wid][ci], end = st + s_cnt[wid][ci];
        const int oi = s_off[wid][ci] & 0x7fff;
        const bool nearc = s_off[wid][ci] >> 15;
        // target position in the frame of this source cell's corner
        const f2 tx = f2_splat(ox - (float)(oi % side - R) * a.k.hx);
        const f2 ty = f2_splat(oy - (float)((oi / side) % side - R) * a.k.hy);
        const f2 tz = f2_splat(oz - (float)(oi / (side * side) - R) * a.k.hz);
        // one 64-point step; NEAR: check for points of the target's own triangles
        auto step = [&](int i0, auto near_tag) {
            constexpr bool NEAR = decltype(near_tag)::value;
            const int i = i0 + 2 * lane;          // even: candidates i and i + 1
            const int h = i >> 1;
            // positions and strengths in one go (the strengths before the test,
            // so their latency overlaps the distance arithmetic)
            const float4 pa = pk[3 * h], pb = pk[3 * h + 1], pc = pk[3 * h + 2];
            const f2 dx = tx - f2_make(pa.x, pa.y), dy = ty - f2_make(pa.z, pa.w),
                     dz = tz - f2_make(pb.x, pb.y);
            const f2 r2 = fma2(dz, dz, fma2(dy, dy, dx * dx));
            float r0, r1;
            float2 wx = make_float2(pb.z, pb.w), wy = make_float2(pc.x, pc.y),
                   wz = make_float2(pc.z, pc.w);
            f2_split(r2, r0, r1);
            if (!__any_sync(0xffffffffu, r0 < rc2 || r1 < rc2)) return;
            if (NEAR) {
                if (r0 < a.near2) {
                    const int s = a.qinv[i];
                    if (s >= 0) {
                        const int4 v = a.qvs[s];
                        if (v.x == oidx || v.y == oidx || v.z == oidx) wx.x = wy.x = wz.x = 0.f;
                    }
                }
                if (r1 < a.near2) {
                    const int s = a.qinv[i + 1];
                    if (s >= 0) {
                        const int4 v = a.qvs[s];
                        if (v.x == oidx || v.y == oidx || v.z == oidx) wx.y = wy.y = wz.y = 0.f;
                    }
                }
            }
            pair_terms2<MODE>(a.k, dx, dy, dz, r2, f2_make(wx.x, wx.y), f2_make(wy.x, wy.y),
                              f2_make(wz.x, wz.y), nx2, ny2, nz2, acc);
        };
        if (nearc) {
            for (int i0 = st; i0 < end; i0 += kChunk) step(i0, std::true_type{});
        } else {
            for (int i0 = st; i0 < end; i0 += kChunk) step(i0, std::false_type{});
        }
    }
    __syncwarp();
    }
    float ux = f2_sum(acc.ux), uy = f2_sum(acc.uy), uz = f2_sum(acc.uz);
    if (MODE & OUT_DBL) {
        const float sn = f2_sum(acc.sn);
        ux = fmaf(nx, sn, ux);
        uy = fmaf(ny, sn, uy);
        uz = fmaf(nz, sn, uz);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ux += __shfl_xor_sync(0xffffffffu, ux, o);
        uy += __shfl_xor_sync(0xffffffffu, uy, o);
        uz += __shfl_xor_sync(0xffffffffu, uz, o);
    }
    if (lane == 0) {
        float* o = a.out + (size_t)oidx * a.out_stride;
        o[0] = a.k.fU * ux;
        o[1] = a.k.fU * uy;
        o[2] = a.k.fU * uz;
    }
}

// Order of the sorted points within each cell: 4 x 4 x 4 sub-cells in Morton
// order, so that consecutive points (the 64-point steps of the FP32 element
// rule) lie close together.  One block per cell; a counting sort by the 6-bit
// key into pos_out / perm_out.
__device__ __forceinline__ int subcell_key(float4 p, float ihx, float ihy, float ihz) {
    const int ix = min(3, max(0, (int)(p.x * ihx))), iy = min(3, max(0, (int)(p.y * ihy))),
              iz = min(3, max(0, (int)(p.z * ihz)));
    return (ix & 1) | ((iy & 1) << 1) | ((iz & 1) << 2) | ((ix & 2) << 2) | ((iy & 2) << 3) |
           ((iz & 2) << 4);
}

__global__ void k_cell_subsort(const int* __restrict__ start, const float4* __restrict__ pos,
                               const int* __restrict__ perm, float ihx, float ihy, float ihz,
                               float4* __restrict__ pos_out, int* __restrict__ perm_out) {
    __shared__ int cnt[64];
    const int c = blockIdx.x;
    const int st = start[c], n = start[c + 1] - st;
    if (n == 0) return;                          // block-uniform
    if (threadIdx.x < 64) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        atomicAdd(&cnt[subcell_key(pos[st + i], ihx, ihy, ihz)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < 64; ++k) {
            const int v = cnt[k];
            cnt[k] = run;
            run += v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 p = pos[st + i];
        const int slot = st + atomicAdd(&cnt[subcell_key(p, ihx, ihy, ihz)], 1);
        pos_out[slot] = p;
        perm_out[slot] = perm[st + i];
    }
}

// ----------------------------------- element rule, FP64-accurate in float pairs
// The FP64 element-rule local sum in double-float arithmetic (ggem_ff.cuh):
// same cells, culling and hit queue as k_local<double, ..., ELEM>, with the
// sources read from float-pair copies of the sorted offsets and strengths.
// exp from a 2^(j/16) reduction, erfcx from the FP64 piecewise polynomials
// (degrees 0..9 in pairs, 10..12 in float), 1/r by one Newton step.
constexpr int kFFHead = 9;

struct FFConst {
    ff al, al2, rc2, near2, c1, c2, c3, c4, ln2_16, sixth;
};

struct FFAcc {
    ff ux = {0.f, 0.f}, uy = {0.f, 0.f}, uz = {0.f, 0.f};
};

__device__ __forceinline__ ff ff_dot(ff ax, ff ay, ff az, ff bx, ff by, ff bz) {
    return ff_add(ff_add(ff_mul(ax, bx), ff_mul(ay, by)), ff_mul(az, bz));
}

// erfcx(x), 0 <= x < 4, from the FP64 table in pairs (tab[j * 8 + i])
__device__ __forceinline__ ff ff_erfcx(ff x, const ff* tab) {
    const int i = min((int)(x.hi * 2.0f), GGEM_ERFCX64_NINT - 1);
    const ff u = ff_add_f(ff_mul_f(x, 4.0f), -(float)(2 * i + 1));
    const float uh = u.hi;
    float t = tab[GGEM_ERFCX64_DEG * 8 + i].hi;
    for (int j = GGEM_ERFCX64_DEG - 1; j > kFFHead; --j) t = fmaf(t, uh, tab[j * 8 + i].hi);
    ff p = ff_of(t);
    for (int j = kFFHead; j >= 0; --j) p = ff_add(ff_mul(p, u), tab[j * 8 + i]);
    return p;
}

template <int MODE>
__device__ __forceinline__ void pair_terms_ff(const FFConst& k, ff dx, ff dy, ff dz, ff r2, ff gx,
                                              ff gy, ff gz, ff nx, ff ny, ff nz, const ff* tab,
                                              const ff* t2, FFAcc& a) {
    const ff ir = ff_rsqrt(r2);
    const ff r = ff_mul(r2, ir);
    const ff ex = ff_exp(ff_neg(ff_mul(k.al2, r2)), t2, k.ln2_16, k.sixth);
    const ff ec = ff_mul(ex, ff_erfcx(ff_mul(k.al, r), tab));
    const ff xg = ff_dot(dx, dy, dz, gx, gy, gz);
    const ff ir2 = ff_mul(ir, ir);
    if (MODE & OUT_U) {
        // A = ec/r - c1 ex,  B = (ec/r^3 + c1 ex/r^2) xg
        const ff eir = ff_mul(ec, ir);
        const ff c1ex = ff_mul(k.c1, ex);
        const ff A = ff_sub(eir, c1ex);
        const ff B = ff_mul(ff_mul(ir2, ff_add(eir, c1ex)), xg);
        a.ux = ff_add(a.ux, ff_add(ff_mul(A, gx), ff_mul(B, dx)));
        a.uy = ff_add(a.uy, ff_add(ff_mul(A, gy), ff_mul(B, dy)));
        a.uz = ff_add(a.uz, ff_add(ff_mul(A, gz), ff_mul(B, dz)));
    }
    if (MODE & OUT_DBL) {
        // D = -6 ec/r^5 - c2 ex/r^4 - c3 ex/r^2,  E = c4 ex
        const ff t = ff_sub(ff_mul_f(ff_mul(ec, ir), -6.0f), ff_mul(k.c2, ex));
        const ff D = ff_sub(ff_mul(ff_mul(ir2, ir2), t), ff_mul(ff_mul(k.c3, ex), ir2));
        const ff E = ff_mul(k.c4, ex);
        const ff xn = ff_dot(dx, dy, dz, nx, ny, nz);
        const ff gn = ff_dot(gx, gy, gz, nx, ny, nz);
        const ff Dxn = ff_mul(ff_mul(D, xg), xn);
        const ff nxg[3] = {ff_mul(nx, xg), ff_mul(ny, xg), ff_mul(nz, xg)};
        const ff d[3] = {dx, dy, dz}, g[3] = {gx, gy, gz};
        ff* acc[3] = {&a.ux, &a.uy, &a.uz};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const ff in = ff_add(ff_add(ff_mul(d[c], gn), ff_mul(g[c], xn)), nxg[c]);
            *acc[c] = ff_add(*acc[c], ff_add(ff_mul(Dxn, d[c]), ff_mul(E, in)));
        }
    }
}

template <int MODE, int REACH>
__global__ void __launch_bounds__(LW * 32) k_local_elem_ff(LocalArgs<double> a,
                                                         const float4* __restrict__ qpos,
                                                         const float4* __restrict__ qg) {
    __shared__ int s_cst[LW][kNb];
    __shared__ int s_cnt[LW][kNb];
    __shared__ unsigned short s_off[LW][kNb];
    __shared__ int2 s_q[LW][kQueue];              // queued hits: sorted point, cell slot
    __shared__ ff s_tab[(GGEM_ERFCX64_DEG + 1) * GGEM_ERFCX64_NINT];
    __shared__ ff s_t2[16];
    for (int e = threadIdx.x; e < (GGEM_ERFCX64_DEG + 1) * GGEM_ERFCX64_NINT; e += blockDim.x)
        s_tab[e] = ff_from_double(kErfcxTab64[e]);
    if (threadIdx.x < 16) s_t2[threadIdx.x] = ff_from_double(exp2((double)threadIdx.x / 16.0));
    __syncthreads();
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * LW + wid;
    if (t >= a.n_tgt) return;                     // warp-uniform
    int cx, cy, cz, oidx;
    double ox, oy, oz;
    load_target<double, TK_POINTS>(a, t, ox, oy, oz, cx, cy, cz, oidx);
    constexpr int R = REACH, side = 2 * R + 1;
    const unsigned lt = (1u << lane) - 1u;
    const int nc = cull_cells<double, R>(a, lane, ox, oy, oz, cx, cy, cz, s_cst[wid], s_cnt[wid],
                                         s_off[wid]);
    FFConst k;
    k.al = ff_from_double(a.k.al);
    k.al2 = ff_from_double(a.k.al2);
    k.rc2 = ff_from_double(a.k.rc2);
    k.near2 = ff_from_double(a.near2);
    k.c1 = ff_from_double(a.k.c1);
    k.c2 = ff_from_double(a.k.c2);
    k.c3 = ff_from_double(a.k.c3);
    k.c4 = ff_from_double(a.k.c4);
    k.ln2_16 = ff_from_double(0.043321698784996581);   // ln 2 / 16
    k.sixth = ff_from_double(1.0 / 6.0);
    const ff o[3] = {ff_from_double(ox), ff_from_double(oy), ff_from_double(oz)};
    const ff hc[3] = {ff_from_double(a.k.hx), ff_from_double(a.k.hy), ff_from_double(a.k.hz)};
    ff nx = ff_of(0.f), ny = ff_of(0.f), nz = ff_of(0.f);
    if (MODE & OUT_DBL) {
        nx = ff_from_double(a.nrm[3 * oidx]);
        ny = ff_from_double(a.nrm[3 * oidx + 1]);
        nz = ff_from_double(a.nrm[3 * oidx + 2]);
    }
    // target in the frame of the corner of cell slot ci
    auto target = [&](int ci, ff& tx, ff& ty, ff& tz) {
        const int oi = s_off[wid][ci];
        tx = ff_sub(o[0], ff_mul_f(hc[0], (float)(oi % side - R)));
        ty = ff_sub(o[1], ff_mul_f(hc[1], (float)((oi / side) % side - R)));
        tz = ff_sub(o[2], ff_mul_f(hc[2], (float)(oi / (side * side) - R)));
    };
    auto eval = [&](int s, int ci, FFAcc& acc) {
        ff tx, ty, tz;
        target(ci, tx, ty, tz);
        const float4 ph = qpos[2 * (size_t)s], pl = qpos[2 * (size_t)s + 1];
        const ff dx = ff_sub(tx, {ph.x, pl.x}), dy = ff_sub(ty, {ph.y, pl.y}),
                 dz = ff_sub(tz, {ph.z, pl.z});
        const ff r2 = ff_dot(dx, dy, dz, dx, dy, dz);
        const float4 gh = qg[2 * (size_t)s], gl = qg[2 * (size_t)s + 1];
        pair_terms_ff<MODE>(k, dx, dy, dz, r2, {gh.x, gl.x}, {gh.y, gl.y}, {gh.z, gl.z}, nx, ny,
                            nz, s_tab, s_t2, acc);
    };
    FFAcc acc;
    int head = 0, qn = 0;                         // warp-uniform
    for (int ci = 0; ci < nc; ++ci) {
        const int st = s_cst[wid][ci], cnt = s_cnt[wid][ci];
        ff tx, ty, tz;
        target(ci, tx, ty, tz);
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            bool hit = false;
            int s = 0;
            if (i < cnt) {
                s = st + i;
                const float4 ph = qpos[2 * (size_t)s], pl = qpos[2 * (size_t)s + 1];
                const ff dx = ff_sub(tx, {ph.x, pl.x}), dy = ff_sub(ty, {ph.y, pl.y}),
                         dz = ff_sub(tz, {ph.z, pl.z});
                const ff r2 = ff_dot(dx, dy, dz, dx, dy, dz);
                hit = ff_lt(r2, k.rc2) && r2.hi > 0.f;
                if (hit && ff_lt(r2, k.near2)) {
                    const int4 v = a.qvs[s];
                    hit = !(v.x == oidx || v.y == oidx || v.z == oidx);
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) s_q[wid][(head + qn + __popc(m & lt)) & (kQueue - 1)] = make_int2(s, ci);
            qn += __popc(m);
            if (qn >= 32) {
                __syncwarp();
                const int2 e = s_q[wid][(head + lane) & (kQueue - 1)];
                eval(e.x, e.y, acc);
                head = (head + 32) & (kQueue - 1);
                qn -= 32;
                __syncwarp();
            }
        }
    }
    __syncwarp();
    if (lane < qn) {
        const int2 e = s_q[wid][(head + lane) & (kQueue - 1)];
        eval(e.x, e.y, acc);
    }
    double ux = ff_to_double(acc.ux), uy = ff_to_double(acc.uy), uz = ff_to_double(acc.uz);
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        ux += __shfl_xor_sync(0xffffffffu, ux, o2);
        uy += __shfl_xor_sync(0xffffffffu, uy, o2);
        uz += __shfl_xor_sync(0xffffffffu, uz, o2);
    }
    if (lane == 0) {
        double* out = a.out + (size_t)oidx * a.out_stride;
        out[0] = a.k.fU * ux;
        out[1] = a.k.fU * uy;
        out[2] = a.k.fU * uz;
    }
}

__global__ void k_to_float_pairs(int n, const double* __restrict__ in, float4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* v = in + 4 * (size_t)i;
    const ff x = ff_from_double(v[0]), y = ff_from_double(v[1]), z = ff_from_double(v[2]),
             w = ff_from_double(v[3]);
    out[2 * (size_t)i] = make_float4(x.hi, y.hi, z.hi, w.hi);
    out[2 * (size_t)i + 1] = make_float4(x.lo, y.lo, z.lo, w.lo);
}

template <typename T, int KIND, int REACH>
static void launch_kind(const LocalArgs<T>& a, int mode, cudaStream_t st) {
    dim3 b(LW * 32), g((a.n_tgt + LW - 1) / LW);
    switch (mode) {
        case OUT_U: k_local<T, KIND, OUT_U, false, REACH><<<g, b, 0, st>>>(a); break;
        case OUT_S: k_local<T, KIND, OUT_S, false, REACH><<<g, b, 0, st>>>(a); break;
        case OUT_U | OUT_S:
            k_local<T, KIND, OUT_U | OUT_S, false, REACH><<<g, b, 0, st>>>(a);
            break;
        case OUT_DBL: k_local<T, KIND, OUT_DBL, false, REACH><<<g, b, 0, st>>>(a); break;
        default: break;
    }
}

// the grid's search reach as a compile-time constant (cells >= r_cut/2 or
// r_cut/3; grids of larger cells use reach 2)
template <typename T, int KIND>
static void launch_kind(const LocalArgs<T>& a, int mode, cudaStream_t st) {
    if (a.cg.reach == 3) launch_kind<T, KIND, 3>(a, mode, st);
    else launch_kind<T, KIND, 2>(a, mode, st);
}

// Within-cell sub-sort of sorted points (pos, perm); tmp_* of n entries as scratch.
cudaError_t cell_subsort(const CellGrid& cg, int n, int ncell, const int* start, float4* pos,
                         int* perm, float4* tmp_pos, int* tmp_perm, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_cell_subsort<<<ncell, 256, 0, st>>>(start, pos, perm, (float)(4.0 / cg.hx),
                                          (float)(4.0 / cg.hy), (float)(4.0 / cg.hz), tmp_pos,
                                          tmp_perm);
    cudaMemcpyAsync(pos, tmp_pos, (size_t)n * sizeof(float4), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(perm, tmp_perm, (size_t)n * sizeof(int), cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError();
}

// Padded, packed layout of the sorted points for the FP32 element rule: each
// cell's points start on a multiple of 64 and fill whole 64-point steps; slot
// pair h holds 12 floats x0 x1 y0 y1 z0 z1 gx0 gx1 gy0 gy1 gz0 gz1 (slots 2h,
// 2h + 1); the slots after a cell's last point hold dummies (offset 1e4 from
// the cell corner, strength zero), whose terms are exactly zero.
__global__ void k_pad_counts(int ncell, const int* __restrict__ start, int* __restrict__ pcnt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) pcnt[c] = (start[c + 1] - start[c] + 63) & ~63;
}

__global__ void k_pad_fill(size_t npairs, float4* __restrict__ pack) {
    const size_t h = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= npairs) return;
    pack[3 * h] = make_float4(1e4f, 1e4f, 1e4f, 1e4f);
    pack[3 * h + 1] = make_float4(1e4f, 1e4f, 0.f, 0.f);
    pack[3 * h + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_pad_scatter(int n, const int* __restrict__ cell, const int* __restrict__ start,
                              const int* __restrict__ pstart, const float4* __restrict__ pos,
                              float sc, float* __restrict__ pack, int* __restrict__ inv) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int c = cell[s];
    const int p = pstart[c] + (s - start[c]);
    const float4 v = pos[s];
    float* o = pack + 12 * (size_t)(p >> 1) + (p & 1);
    o[0] = v.x * sc;
    o[2] = v.y * sc;
    o[4] = v.z * sc;
    inv[p] = s;
}

cudaError_t pad_layout_counts(int ncell, const int* start, int* pcnt, int* pstart,
                              cudaStream_t st) {
    if (ncell <= 0) return cudaSuccess;
    k_pad_counts<<<(ncell + 255) / 256, 256, 0, st>>>(ncell, start, pcnt);
    return scan_counts(ncell, pcnt, pstart, st);
}

float elem32_scale(double alpha) { return (float)(alpha * 1.2011224087864498); }

cudaError_t pad_layout_fill(int n, size_t np, const int* cell, const int* start,
                            const int* pstart, const float4* pos, double alpha, float* pack,
                            int* inv, cudaStream_t st) {
    if (np > 0) {
        const size_t npairs = np / 2;
        k_pad_fill<<<(unsigned)((npairs + 255) / 256), 256, 0, st>>>(npairs, (float4*)pack);
        cudaMemsetAsync(inv, 0xff, np * sizeof(int), st);
    }
    if (n > 0)
        k_pad_scatter<<<(n + 255) / 256, 256, 0, st>>>(n, cell, start, pstart, pos,
                                                      elem32_scale(alpha), pack, inv);
    return cudaGetLastError();
}

cudaError_t to_float_pairs(int n, const void* in, void* out, cudaStream_t st) {
    if (n > 0)
        k_to_float_pairs<<<(n + 255) / 256, 256, 0, st>>>(n, (const double*)in, (float4*)out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t local_sum_elem(const GridGeom& geo, const CellGrid& cg, const SortedSources<T>& src,
                           const int4* qvs, double near, const SortedSources<T>& tgt,
                           const double* nrm_tgt, int layer, T* out, int out_stride,
                           cudaStream_t st, const void* aux_pos, const void* aux_g,
                           size_t aux_ld, const int* aux_inv) {
    if (tgt.n <= 0) return cudaSuccess;
    // targets: the mesh nodes in cell order, so the warps of a block mostly
    // scan the same candidate cells (L1 reuse); output in caller order
    LocalArgs<T> a{geo, cg, local_const<T>(geo, cg), src, qvs, (T)(near * near), tgt.n,
                   tgt.cell, tgt.pos, tgt.perm, nrm_tgt, out, out_stride};
    if constexpr (sizeof(T) == 4) {
        (void)aux_g;
        (void)aux_ld;
        if (!aux_pos || !aux_inv) return cudaErrorInvalidValue;
        a.qinv = aux_inv;
        // scaled coordinates: lengths times s = alpha sqrt(log2 e), the
        // packed points scaled likewise at mesh_set (pad_layout_fill)
        {
            const double sc = (double)elem32_scale(geo.alpha);
            LocalConst<float>& k = a.k;
            k.sc = (float)sc;
            k.hx = (float)(cg.hx * sc);
            k.hy = (float)(cg.hy * sc);
            k.hz = (float)(cg.hz * sc);
            k.rc2 = (float)(geo.rcut * geo.rcut * sc * sc);
            a.near2 = (float)(near * near * sc * sc);
            k.pt = (float)(GGEM_ERFCX_P * geo.alpha / sc);
            k.c1 = (float)(2.0 * geo.alpha / 1.7724538509055160273 / sc);
            k.c2 = (float)(12.0 * geo.alpha / 1.7724538509055160273 * sc * sc);
            k.c6 = (float)(-6.0 * sc * sc * sc);
            k.fU = (float)(layer == 0 ? sc : 1.0 / sc) * k.fU;
        }
        const float4* pk = (const float4*)aux_pos;
        dim3 b(LWE * 32), g((tgt.n + LWE - 1) / LWE);
        // ~6 KB of shared memory per block, 10 blocks per SM: ask for a small
        // shared-memory carveout (25 %: the 64 KB configuration) so that the
        // rest of the SM's 256 KB serves as L1
        // for the candidates the warps of a block re-read (a preference; cheap
        // per launch)
        const void* kf = layer == 0 ? (cg.reach == 3 ? (const void*)k_local_elem32<OUT_U, 3>
                                                     : (const void*)k_local_elem32<OUT_U, 2>)
                                    : (cg.reach == 3 ? (const void*)k_local_elem32<OUT_DBL, 3>
                                                     : (const void*)k_local_elem32<OUT_DBL, 2>);
        cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout, 25);
        if (cg.reach == 3) {
            if (layer == 0) k_local_elem32<OUT_U, 3><<<g, b, 0, st>>>(a, pk);
            else k_local_elem32<OUT_DBL, 3><<<g, b, 0, st>>>(a, pk);
        } else {
            if (layer == 0) k_local_elem32<OUT_U, 2><<<g, b, 0, st>>>(a, pk);
            else k_local_elem32<OUT_DBL, 2><<<g, b, 0, st>>>(a, pk);
        }
        return cudaGetLastError();
    }
    dim3 b(LW * 32), g((tgt.n + LW - 1) / LW);
    if constexpr (sizeof(T) == 8) {
        if (aux_pos && aux_g) {
            const float4* fp = (const float4*)aux_pos;
            const float4* fg = (const float4*)aux_g;
            if (cg.reach == 3) {
                if (layer == 0) k_local_elem_ff<OUT_U, 3><<<g, b, 0, st>>>(a, fp, fg);
                else k_local_elem_ff<OUT_DBL, 3><<<g, b, 0, st>>>(a, fp, fg);
            } else {
                if (layer == 0) k_local_elem_ff<OUT_U, 2><<<g, b, 0, st>>>(a, fp, fg);
                else k_local_elem_ff<OUT_DBL, 2><<<g, b, 0, st>>>(a, fp, fg);
            }
            return cudaGetLastError();
        }
    }
    if (cg.reach == 3) {
        if (layer == 0) k_local<T, TK_POINTS, OUT_U, true, 3><<<g, b, 0, st>>>(a);
        else k_local<T, TK_POINTS, OUT_DBL, true, 3><<<g, b, 0, st>>>(a);
    } else {
        if (layer == 0) k_local<T, TK_POINTS, OUT_U, true, 2><<<g, b, 0, st>>>(a);
        else k_local<T, TK_POINTS, OUT_DBL, true, 2><<<g, b, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t local_sum(const GridGeom& geo, const CellGrid& cg, const SortedSources<T>& src,
                      int kind, int n_tgt, const int* tcell, const v4_t<T>* tpos,
                      const double* nrm_tgt, int out_mode, T* out, int out_stride,
                      cudaStream_t st) {
    if (n_tgt <= 0) return cudaSuccess;
    LocalArgs<T> a{geo, cg, local_const<T>(geo, cg), src, nullptr, (T)0, n_tgt, tcell, tpos,
                   nullptr, nrm_tgt, out, out_stride};
    if (kind == TK_SORTED) launch_kind<T, TK_SORTED>(a, out_mode, st);
    else if (kind == TK_POINTS) launch_kind<T, TK_POINTS>(a, out_mode, st);
    else launch_kind<T, TK_WALL>(a, OUT_U, st);
    return cudaGetLastError();
}

#define GGEM_INST_LOCAL(T)                                                                   \
    template cudaError_t build_cells<T>(const GridGeom&, const CellGrid&, int, const double*, \
                                        int*, int*, int*, int*, int*, v4_t<T>*, cudaStream_t); \
    template cudaError_t gather_strengths<T>(int, const int*, const double*, const double*,   \
                                             double, v4_t<T>*, cudaStream_t);                  \
    template cudaError_t local_sum<T>(const GridGeom&, const CellGrid&,                       \
                                      const SortedSources<T>&, int, int, const int*,          \
                                      const v4_t<T>*, const double*, int, T*, int,             \
                                      cudaStream_t);                                           \
    template cudaError_t locate_targets<T>(const GridGeom&, const CellGrid&, int, int,        \
                                           const double*, int*, v4_t<T>*, cudaStream_t);       \
    template cudaError_t local_sum_elem<T>(const GridGeom&, const CellGrid&,                  \
                                           const SortedSources<T>&, const int4*, double,        \
                                           const SortedSources<T>&, const double*, int, T*, int, \
                                           cudaStream_t, const void*, const void*, size_t, \
                                           const int*);
GGEM_INST_LOCAL(float)
GGEM_INST_LOCAL(double)

}  // namespace ggem
