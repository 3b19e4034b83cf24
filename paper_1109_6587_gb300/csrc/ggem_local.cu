// Cell list and GGEM local sums (paper Sec. 3.2.1, Eqs. (local), (u_loc)).
//
// Sources are binned into cells no smaller than r_cut and stored as offsets
// from their cell's corner, so every displacement is formed from small
// numbers (integer cell shift + offset difference) and stays accurate in FP32
// whatever the box size.  x and z are periodic: the neighbour shift of +-1
// cell carries the minimum image (Sec. 3.2.2, alpha L > 8 makes r_cut < L/2).
#include "ggem_internal.cuh"

namespace ggem {

template <typename T> __device__ __forceinline__ T d_erfc(T x);
template <> __device__ __forceinline__ float d_erfc<float>(float x) { return erfcf(x); }
template <> __device__ __forceinline__ double d_erfc<double>(double x) { return erfc(x); }
template <typename T> __device__ __forceinline__ T d_exp(T x);
template <> __device__ __forceinline__ float d_exp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double d_exp<double>(double x) { return exp(x); }
template <typename T> __device__ __forceinline__ T d_rsqrt(T x);
template <> __device__ __forceinline__ float d_rsqrt<float>(float x) { return rsqrtf(x); }
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
template <typename T> struct LocalArgs {
    GridGeom geo;
    CellGrid cg;
    SortedSources<T> src;
    int n_tgt;
    const double* x_tgt;     // TK_POINTS: [n][3] caller order
    const double* nrm;       // OUT_DBL: [n][3] target normals (caller order)
    T* out;
    int out_stride;
};

// u_i = sum G^l_ij g_j ; sigma_ik = sum T^l_ijk g_j ; v_i = n_k sigma_ik
// (unscaled here; the caller-facing factors are applied at the end).
template <typename T, int KIND, int MODE>
__global__ void __launch_bounds__(128) k_local(LocalArgs<T> a) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tgt) return;
    const CellGrid& cg = a.cg;
    int cx, cy, cz, oidx = t;
    T ox, oy, oz;
    double wx = 0, wz = 0;
    int wall = 0;
    if (KIND == TK_SORTED) {
        v4_t<T> p = a.src.pos[t];
        ox = p.x; oy = p.y; oz = p.z;
        int c = a.src.cell[t];
        cx = c % cg.ncx;
        cy = (c / cg.ncx) % cg.ncy;
        cz = c / (cg.ncx * cg.ncy);
        oidx = a.src.perm[t];
    } else {
        double xx, yy, zz;
        if (KIND == TK_POINTS) {
            xx = a.x_tgt[3 * t]; yy = a.x_tgt[3 * t + 1]; zz = a.x_tgt[3 * t + 2];
        } else {
            int nxz = a.geo.Nz * a.geo.Nx;
            wall = t / nxz;
            int rem = t - wall * nxz;
            int k = rem / a.geo.Nx, i = rem - k * a.geo.Nx;
            xx = i * a.geo.dx; zz = k * a.geo.dz;
            yy = a.geo.y0 + wall * a.geo.W;
            wx = i; wz = k;
        }
        double dox, doy, doz;
        locate(a.geo, cg, xx, yy, zz, cx, cy, cz, dox, doy, doz);
        ox = (T)dox; oy = (T)doy; oz = (T)doz;
    }
    T nx = 0, ny = 0, nz = 0;
    if (MODE & OUT_DBL) {
        nx = (T)a.nrm[3 * oidx]; ny = (T)a.nrm[3 * oidx + 1]; nz = (T)a.nrm[3 * oidx + 2];
    }
    const T al = (T)a.geo.alpha, al2 = al * al;
    const T rc2 = (T)(a.geo.rcut * a.geo.rcut);
    const double sp = 1.7724538509055160273;
    const T c1 = (T)(2.0 * a.geo.alpha / sp);
    const T c2 = (T)(12.0 * a.geo.alpha / sp);
    const T c3 = (T)(8.0 * a.geo.alpha * a.geo.alpha * a.geo.alpha / sp);
    const T c4 = (T)(4.0 * a.geo.alpha * a.geo.alpha * a.geo.alpha / sp);
    T ux = 0, uy = 0, uz = 0;
    T sxx = 0, sxy = 0, sxz = 0, syy = 0, syz = 0, szz = 0;
    const T hx = (T)cg.hx, hy = (T)cg.hy, hz = (T)cg.hz;
    for (int dzc = -1; dzc <= 1; ++dzc) {
        int czz = cz + dzc;
        czz += (czz < 0) ? cg.ncz : 0;
        czz -= (czz >= cg.ncz) ? cg.ncz : 0;
        const T shz = -(T)dzc * hz + oz;
        for (int dyc = -1; dyc <= 1; ++dyc) {
            int cyy = cy + dyc;
            if (cyy < 0 || cyy >= cg.ncy) continue;
            const T shy = -(T)dyc * hy + oy;
            for (int dxc = -1; dxc <= 1; ++dxc) {
                int cxx = cx + dxc;
                cxx += (cxx < 0) ? cg.ncx : 0;
                cxx -= (cxx >= cg.ncx) ? cg.ncx : 0;
                const T shx = -(T)dxc * hx + ox;
                int c = (czz * cg.ncy + cyy) * cg.ncx + cxx;
                int s0 = a.src.cell_start[c], s1 = a.src.cell_start[c + 1];
                for (int s = s0; s < s1; ++s) {
                    v4_t<T> p = a.src.pos[s];
                    T dx = shx - p.x, dy = shy - p.y, dz = shz - p.z;
                    T r2 = dx * dx + dy * dy + dz * dz;
                    if (!(r2 < rc2 && r2 > (T)0)) continue;
                    v4_t<T> g = a.src.g[s];
                    T ir = d_rsqrt<T>(r2);
                    T r = r2 * ir;
                    T ec = d_erfc<T>(al * r);
                    T ex = d_exp<T>(-al2 * r2);
                    T xg = dx * g.x + dy * g.y + dz * g.z;
                    if (MODE & OUT_U) {
                        T A = ec * ir - c1 * ex;
                        T B = (ec * ir * ir * ir + c1 * ex * ir * ir) * xg;
                        ux += A * g.x + B * dx;
                        uy += A * g.y + B * dy;
                        uz += A * g.z + B * dz;
                    }
                    if (MODE & (OUT_S | OUT_DBL)) {
                        T ir2 = ir * ir;
                        T D = -(T)6 * ec * ir2 * ir2 * ir - c2 * ex * ir2 * ir2 - c3 * ex * ir2;
                        T E = c4 * ex;
                        if (MODE & OUT_S) {
                            T Dx = D * xg;
                            sxx += Dx * dx * dx + E * ((T)2 * g.x * dx + xg);
                            syy += Dx * dy * dy + E * ((T)2 * g.y * dy + xg);
                            szz += Dx * dz * dz + E * ((T)2 * g.z * dz + xg);
                            sxy += Dx * dx * dy + E * (g.y * dx + g.x * dy);
                            sxz += Dx * dx * dz + E * (g.z * dx + g.x * dz);
                            syz += Dx * dy * dz + E * (g.z * dy + g.y * dz);
                        } else {
                            T xn = dx * nx + dy * ny + dz * nz;
                            T gn = g.x * nx + g.y * ny + g.z * nz;
                            T Dxn = D * xg * xn;
                            ux += Dxn * dx + E * (dx * gn + g.x * xn + nx * xg);
                            uy += Dxn * dy + E * (dy * gn + g.y * xn + ny * xg);
                            uz += Dxn * dz + E * (dz * gn + g.z * xn + nz * xg);
                        }
                    }
                }
            }
        }
    }
    const double pi = 3.14159265358979323846;
    if (KIND == TK_WALL) {
        // global wall data u^g = -u^l (Sec. 3.2.2), layout [wall][c][Nz][Nx]
        T f = (T)(-1.0 / (8.0 * pi * a.geo.mu));
        size_t plane = (size_t)a.geo.Nz * a.geo.Nx;
        size_t o = (size_t)(wall * 3) * plane + (size_t)wz * a.geo.Nx + (size_t)wx;
        a.out[o] = f * ux;
        a.out[o + plane] = f * uy;
        a.out[o + 2 * plane] = f * uz;
        return;
    }
    T* o = a.out + (size_t)oidx * a.out_stride;
    int k = 0;
    if (MODE & (OUT_U | OUT_DBL)) {
        T f = (T)(1.0 / (8.0 * pi * a.geo.mu));
        o[0] = f * ux; o[1] = f * uy; o[2] = f * uz;
        k = 3;
    }
    if (MODE & OUT_S) {
        T f = (T)(1.0 / (8.0 * pi));
        o[k] = f * sxx; o[k + 1] = f * sxy; o[k + 2] = f * sxz;
        o[k + 3] = f * syy; o[k + 4] = f * syz; o[k + 5] = f * szz;
    }
}

template <typename T, int KIND>
static void launch_kind(const LocalArgs<T>& a, int mode, cudaStream_t st) {
    dim3 b(128), g((a.n_tgt + 127) / 128);
    switch (mode) {
        case OUT_U: k_local<T, KIND, OUT_U><<<g, b, 0, st>>>(a); break;
        case OUT_S: k_local<T, KIND, OUT_S><<<g, b, 0, st>>>(a); break;
        case OUT_U | OUT_S: k_local<T, KIND, OUT_U | OUT_S><<<g, b, 0, st>>>(a); break;
        case OUT_DBL: k_local<T, KIND, OUT_DBL><<<g, b, 0, st>>>(a); break;
        default: break;
    }
}

template <typename T>
cudaError_t local_sum(const GridGeom& geo, const CellGrid& cg, const SortedSources<T>& src,
                      int kind, int n_tgt, const double* x_tgt, const double* nrm_tgt,
                      int out_mode, T* out, int out_stride, cudaStream_t st) {
    if (n_tgt <= 0) return cudaSuccess;
    LocalArgs<T> a{geo, cg, src, n_tgt, x_tgt, nrm_tgt, out, out_stride};
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
                                      const SortedSources<T>&, int, int, const double*,       \
                                      const double*, int, T*, int, cudaStream_t);
GGEM_INST_LOCAL(float)
GGEM_INST_LOCAL(double)

}  // namespace ggem
