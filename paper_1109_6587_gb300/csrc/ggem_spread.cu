// Spreading of the global density onto the grid (paper Eqs. (stokes_gg),
// (rho_int), (rhog_sum)):
//   f(node) = - sum_s g_s rho_g(node - x_s*),   |node - x_s*| < r_cut,
//   rho_g(r) = alpha^3 pi^{-3/2} exp(-alpha^2 r^2) (5/2 - alpha^2 r^2).
//
// Source-parallel: a warp takes one sorted source (FP64, k_spread_scatter) or
// two neighbouring ones (FP32, k_spread_pair: the union of their stencils,
// both weights per node, one reduction with their sum), lists the columns,
// rows and planes of its stencil, and adds the weights into an interleaved
// [Ny][Nz][Nx][4] accumulation grid with float4 / double vector reductions in
// L2; k_deinterleave then writes the planar [Ny][3][Nz][Nx] forcing.  The
// Gaussian factor is separable, exp(-a^2 r^2) = exp(-a^2 dx^2)
// exp(-a^2 dy^2) exp(-a^2 dz^2), so each source costs one exponential per
// column, row and plane (the fast Gaussian gridding idea), the remaining
// work per node being a few multiplies.  Displacements come from per-source
// descriptors (integer grid offsets plus small remainders, built once per
// source set), so the kernel runs in T only: no FP64 instruction, accurate in
// large boxes.
#include "ggem_internal.cuh"

namespace ggem {

namespace {

// Per-source descriptor for spreading, computed once per source set (one
// thread per sorted source, FP64): ixb = floor(x/dx) of the wrapped x,
// rx = x - ixb dx; the same for z; jn = nearest Chebyshev node, ry = y - y_jn;
// [jlo, jhi] = a superset of the nodes with |y_j - y| < r_cut.
template <typename T>
__global__ void k_src_desc(GridGeom geo, const double* __restrict__ yj, int n,
                           const int* __restrict__ perm, const double* __restrict__ x,
                           int4* __restrict__ di, v4_t<T>* __restrict__ df) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int src = perm[s];
    double xs = x[3 * src], ys = x[3 * src + 1], zs = x[3 * src + 2];
    xs -= geo.Lx * floor(xs / geo.Lx);
    zs -= geo.Lz * floor(zs / geo.Lz);
    int ixb = min((int)floor(xs / geo.dx), geo.Nx - 1);
    int izb = min((int)floor(zs / geo.dz), geo.Nz - 1);
    const int N = geo.Ny - 1;
    const double pi = 3.14159265358979323846, rc = geo.rcut;
    double yb = fmin(1.0, fmax(-1.0, 2.0 * (ys - geo.y0) / geo.W - 1.0));
    int jn = min(max((int)rint(acos(yb) * N / pi), 0), N);
    double yh = fmin(1.0, yb + 2.0 * rc / geo.W), yl = fmax(-1.0, yb - 2.0 * rc / geo.W);
    int jlo = max(0, (int)floor(acos(yh) * N / pi) - 1);
    int jhi = min(N, (int)ceil(acos(yl) * N / pi) + 1);
    di[s] = make_int4(ixb, izb, jn, jlo | (jhi << 16));
    v4_t<T> f;
    f.x = (T)(xs - ixb * geo.dx);
    f.y = (T)(zs - izb * geo.dz);
    f.z = (T)(ys - yj[jn]);
    f.w = (T)0;
    df[s] = f;
}

template <typename T> __device__ __forceinline__ T sexp(T x);
template <> __device__ __forceinline__ float sexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double sexp<double>(double x) { return exp(x); }

// per-kernel constants in T (computed on the host)
template <typename T> struct SpreadConst {
    T dx, dz, rc2, al2, cn;
};

constexpr int SW = 8;         // warps (sources) per block
constexpr int MAXJ = 272;     // max y nodes of one source stencil (checked on the host)
constexpr int MAXR = 32;      // max columns / rows of one source's stencil

// vector reduction into an interleaved (x, y, z, pad) node
__device__ __forceinline__ void red4(float* p, float a, float b, float c) {
    atomicAdd(reinterpret_cast<float4*>(p), make_float4(a, b, c, 0.f));
}
__device__ __forceinline__ void red4(double* p, double a, double b, double c) {
    atomicAdd(p, a);
    atomicAdd(p + 1, b);
    atomicAdd(p + 2, c);
}

// One warp per source.  The source's stencil is the set of nodes within r_cut:
// columns i with dx^2 < rc^2, rows k with dz^2 < rc^2, planes j in its y-range.
// Lanes build the separable factors e_x, e_z, e_y in shared memory, then walk
// the (column, row) pairs of the disc; each lane runs the planes of its pair
// with dy^2 < rc^2 - dx^2 - dz^2 and adds into the interleaved buffer with one
// vector reduction per node.
// With `list`, warp i handles source list[i] for i < *nlist (the sources the
// paired kernel handed back); otherwise source i for i < n.
template <typename T>
__global__ void __launch_bounds__(SW * 32) k_spread_scatter(
    GridGeom geo, SpreadConst<T> kc, const T* __restrict__ ydiff, int n, int R,
    const int4* __restrict__ sdi, const v4_t<T>* __restrict__ sdf,
    const v4_t<T>* __restrict__ gsrc, T* __restrict__ f4, const int* __restrict__ list,
    const int* __restrict__ nlist) {
    __shared__ T s_xd2[SW][MAXR], s_xe[SW][MAXR], s_zd2[SW][MAXR], s_ze[SW][MAXR];
    __shared__ int s_xi[SW][MAXR], s_zi[SW][MAXR];
    __shared__ T s_yd2[SW][MAXJ], s_ye[SW][MAXJ];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int s = blockIdx.x * SW + wid;
    if (list) {
        if (s >= *nlist) return;                   // warp-uniform
        s = list[s];
    } else if (s >= n) {
        return;                                    // warp-uniform
    }
    const T rc2 = kc.rc2, al2 = kc.al2;
    const int4 di = sdi[s];
    const v4_t<T> df = sdf[s];
    const v4_t<T> g = gsrc[s];
    const int mNx = geo.Nx - 1, mNz = geo.Nz - 1;
    const int nr = 2 * R + 2;                      // candidate offsets -R .. R+1
    // columns and rows within r_cut (lane = offset index)
    T dx2 = (T)1e30, dz2 = (T)1e30;
    if (lane < nr) {
        T vx = fma((T)(lane - R), kc.dx, -df.x);
        T vz = fma((T)(lane - R), kc.dz, -df.y);
        dx2 = vx * vx;
        dz2 = vz * vz;
    }
    const unsigned mx = __ballot_sync(0xffffffffu, dx2 < rc2);
    const unsigned mz = __ballot_sync(0xffffffffu, dz2 < rc2);
    const unsigned lt = (1u << lane) - 1u;
    if (dx2 < rc2) {
        int rk = __popc(mx & lt);
        s_xd2[wid][rk] = dx2;
        s_xe[wid][rk] = sexp<T>(-al2 * dx2);
        s_xi[wid][rk] = (di.x + lane - R) & mNx;
    }
    if (dz2 < rc2) {
        int rk = __popc(mz & lt);
        s_zd2[wid][rk] = dz2;
        s_ze[wid][rk] = sexp<T>(-al2 * dz2);
        s_zi[wid][rk] = (di.y + lane - R) & mNz;
    }
    // planes of the y-range
    const int jlo = di.w & 0xffff, jhi = di.w >> 16, ny = jhi - jlo + 1;
    const T* yrow = ydiff + di.z;
    for (int q = lane; q < ny; q += 32) {
        T d = yrow[(size_t)(jlo + q) * geo.Ny] - df.z;
        T d2 = d * d;
        s_yd2[wid][q] = d2;
        s_ye[wid][q] = sexp<T>(-al2 * d2);
    }
    __syncwarp();
    const T gx = -kc.cn * g.x, gy = -kc.cn * g.y, gz = -kc.cn * g.z;
    const int nxs = __popc(mx), nzs = __popc(mz), npair = nxs * nzs;
    const float inx = 1.0f / (float)nxs;
    const size_t rowst = (size_t)geo.Nx * 4, planest = (size_t)geo.Nz * geo.Nx * 4;
    for (int pi = lane; pi < npair; pi += 32) {
        int b = (int)(((float)pi + 0.5f) * inx);
        int a = pi - b * nxs;
        T dxz = s_xd2[wid][a] + s_zd2[wid][b];
        if (!(dxz < rc2)) continue;
        T exz = s_xe[wid][a] * s_ze[wid][b];
        T* col = f4 + (size_t)s_zi[wid][b] * rowst + (size_t)s_xi[wid][a] * 4;
        for (int q = 0; q < ny; ++q) {
            T r2 = dxz + s_yd2[wid][q];
            if (!(r2 < rc2)) continue;
            T w = exz * s_ye[wid][q] * ((T)2.5 - al2 * r2);
            red4(col + (size_t)(jlo + q) * planest, gx * w, gy * w, gz * w);
        }
    }
}

// Two consecutive sorted sources per warp (FP32).  Neighbouring sources share
// most of their stencils, so the warp walks the union of the two stencils,
// evaluates both weights at every node and issues one vector reduction with
// their sum: fewer reductions, which bound this kernel.  A pair whose union
// does not fit 32 columns or 32 rows (sources far apart in the sorted order)
// is handed to the single-source path.
constexpr int PMAXJ = 272;
__global__ void __launch_bounds__(SW * 32) k_spread_pair(
    GridGeom geo, SpreadConst<float> kc, const float* __restrict__ ydiff, int n, int R,
    const int4* __restrict__ sdi, const float4* __restrict__ sdf,
    const float4* __restrict__ gsrc, float* __restrict__ f4, int* __restrict__ leftover,
    int* __restrict__ nleft) {
    __shared__ float s_xd2[SW][2][32], s_xe[SW][2][32], s_zd2[SW][2][32], s_ze[SW][2][32];
    __shared__ int s_xi[SW][32], s_zi[SW][32];
    __shared__ float s_yd2[SW][2][PMAXJ], s_ye[SW][2][PMAXJ];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s0 = 2 * (blockIdx.x * SW + wid);
    if (s0 >= n) return;                                    // warp-uniform
    const bool two = s0 + 1 < n;
    const int4 d0 = sdi[s0];
    const int4 d1 = two ? sdi[s0 + 1] : d0;
    const int Nx = geo.Nx, Nz = geo.Nz;
    // signed periodic offsets of source 1's base column/row from source 0's
    int ox = d1.x - d0.x, oz = d1.y - d0.y;
    ox -= (ox > Nx / 2) ? Nx : 0;
    ox += (ox < -Nx / 2) ? Nx : 0;
    oz -= (oz > Nz / 2) ? Nz : 0;
    oz += (oz < -Nz / 2) ? Nz : 0;
    const int nr = 2 * R + 2;
    // the union of offsets [-R, R+1] (source 0) and [o - R, o + R + 1] (source 1),
    // relative to source 0's base column / row
    const int bx = min(0, ox) - R, bz = min(0, oz) - R;
    const int spx = max(0, ox) - min(0, ox) + nr, spz = max(0, oz) - min(0, oz) + nr;
    if (!two || spx > 32 || spz > 32) {
        if (lane == 0) {
            leftover[atomicAdd(nleft, 1)] = s0;
            if (two) leftover[atomicAdd(nleft, 1)] = s0 + 1;
        }
        return;
    }
    const float rc2 = kc.rc2, al2 = kc.al2;
    const float4 f0 = sdf[s0], f1 = sdf[s0 + 1];
    // columns and rows of the union: lane = union offset
    {
        const int c = bx + lane;                              // column offset from s0's base
        float v0x = 1e30f, v1x = 1e30f;
        if (lane < spx) {
            const int o0 = c + R, o1 = c - ox + R;            // offsets into each stencil
            if (o0 >= 0 && o0 < nr) { float v = fmaf((float)(o0 - R), kc.dx, -f0.x); v0x = v * v; }
            if (o1 >= 0 && o1 < nr) { float v = fmaf((float)(o1 - R), kc.dx, -f1.x); v1x = v * v; }
        }
        s_xd2[wid][0][lane] = v0x;
        s_xd2[wid][1][lane] = v1x;
        s_xe[wid][0][lane] = v0x < rc2 ? expf(-al2 * v0x) : 0.f;
        s_xe[wid][1][lane] = v1x < rc2 ? expf(-al2 * v1x) : 0.f;
        s_xi[wid][lane] = (d0.x + c) & (Nx - 1);
        const int r = bz + lane;
        float v0z = 1e30f, v1z = 1e30f;
        if (lane < spz) {
            const int o0 = r + R, o1 = r - oz + R;
            if (o0 >= 0 && o0 < nr) { float v = fmaf((float)(o0 - R), kc.dz, -f0.y); v0z = v * v; }
            if (o1 >= 0 && o1 < nr) { float v = fmaf((float)(o1 - R), kc.dz, -f1.y); v1z = v * v; }
        }
        s_zd2[wid][0][lane] = v0z;
        s_zd2[wid][1][lane] = v1z;
        s_ze[wid][0][lane] = v0z < rc2 ? expf(-al2 * v0z) : 0.f;
        s_ze[wid][1][lane] = v1z < rc2 ? expf(-al2 * v1z) : 0.f;
        s_zi[wid][lane] = (d0.y + r) & (Nz - 1);
    }
    // planes: union of the two y-ranges
    const int jlo = min(d0.w & 0xffff, d1.w & 0xffff), jhi = max(d0.w >> 16, d1.w >> 16);
    const int ny = jhi - jlo + 1;
    for (int q = lane; q < ny; q += 32) {
        const float a0 = ydiff[(size_t)(jlo + q) * geo.Ny + d0.z] - f0.z;
        const float a1 = ydiff[(size_t)(jlo + q) * geo.Ny + d1.z] - f1.z;
        s_yd2[wid][0][q] = a0 * a0;
        s_yd2[wid][1][q] = a1 * a1;
        s_ye[wid][0][q] = expf(-al2 * a0 * a0);
        s_ye[wid][1][q] = expf(-al2 * a1 * a1);
    }
    __syncwarp();
    const float4 g0 = gsrc[s0], g1 = gsrc[s0 + 1];
    const float ax = -kc.cn * g0.x, ay = -kc.cn * g0.y, az = -kc.cn * g0.z;
    const float bxg = -kc.cn * g1.x, byg = -kc.cn * g1.y, bzg = -kc.cn * g1.z;
    const int npair = spx * spz;
    const float inx = 1.0f / (float)spx;
    const size_t rowst = (size_t)Nx * 4, planest = (size_t)Nz * Nx * 4;
    for (int pi = lane; pi < npair; pi += 32) {
        const int b = (int)(((float)pi + 0.5f) * inx);
        const int a = pi - b * spx;
        const float e0 = s_xd2[wid][0][a] + s_zd2[wid][0][b];
        const float e1 = s_xd2[wid][1][a] + s_zd2[wid][1][b];
        if (!(e0 < rc2) && !(e1 < rc2)) continue;
        const float x0 = s_xe[wid][0][a] * s_ze[wid][0][b];
        const float x1 = s_xe[wid][1][a] * s_ze[wid][1][b];
        float* col = f4 + (size_t)s_zi[wid][b] * rowst + (size_t)s_xi[wid][a] * 4;
        for (int q = 0; q < ny; ++q) {
            const float r0 = e0 + s_yd2[wid][0][q], r1 = e1 + s_yd2[wid][1][q];
            const float w0 = r0 < rc2 ? x0 * s_ye[wid][0][q] * (2.5f - al2 * r0) : 0.f;
            const float w1 = r1 < rc2 ? x1 * s_ye[wid][1][q] * (2.5f - al2 * r1) : 0.f;
            if (w0 == 0.f && w1 == 0.f) continue;
            red4(col + (size_t)(jlo + q) * planest, fmaf(ax, w0, bxg * w1),
                 fmaf(ay, w0, byg * w1), fmaf(az, w0, bzg * w1));
        }
    }
}

// interleaved [Ny][Nz][Nx][4] -> planar [Ny][3][Nz][Nx]
template <typename T>
__global__ void k_deinterleave(int Ny, int Nz, int Nx, const T* __restrict__ f4,
                               T* __restrict__ grid) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t plane = (size_t)Nz * Nx;
    if (e >= (size_t)Ny * plane) return;
    size_t j = e / plane, r = e - j * plane;
    const T* p = f4 + e * 4;
    T* o = grid + j * 3 * plane + r;
    o[0] = p[0];
    o[plane] = p[1];
    o[2 * plane] = p[2];
}
}  // namespace

template <typename T>
cudaError_t spread_prepare(const GridGeom& geo, const double* yj, int n, const int* perm,
                           const double* x, int4* di, v4_t<T>* df, cudaStream_t st) {
    if (n > 0) k_src_desc<T><<<(n + 255) / 256, 256, 0, st>>>(geo, yj, n, perm, x, di, df);
    return cudaGetLastError();
}

template <typename T>
cudaError_t spread(const GridGeom& geo, const CellGrid& cg, const double* yj, const T* ydiff,
                   const SortedSources<T>& src, const int4* di, const v4_t<T>* df, T* grid,
                   T* work, int* list, cudaStream_t st) {
    (void)cg; (void)yj;
    int R = (int)std::ceil(std::max(geo.rcut / geo.dx, geo.rcut / geo.dz)) + 1;
    if (2 * R + 2 > MAXR || geo.Ny > MAXJ) return cudaErrorInvalidConfiguration;
    const double pi = 3.14159265358979323846;
    SpreadConst<T> kc;
    kc.dx = (T)geo.dx; kc.dz = (T)geo.dz;
    kc.rc2 = (T)(geo.rcut * geo.rcut);
    kc.al2 = (T)(geo.alpha * geo.alpha);
    kc.cn = (T)(geo.alpha * geo.alpha * geo.alpha / (pi * std::sqrt(pi)));
    size_t nodes = (size_t)geo.Ny * geo.Nz * geo.Nx;
    cudaMemsetAsync(work, 0, nodes * 4 * sizeof(T), st);
    if (src.n > 0) {
        bool paired = false;
        if constexpr (sizeof(T) == 4) {
            if (list && geo.Ny <= PMAXJ) {
                // pairs of sources; the pairs that do not fit go back to the single path
                int* nleft = list + src.n;
                cudaMemsetAsync(nleft, 0, sizeof(int), st);
                const int npairs = (src.n + 1) / 2;
                k_spread_pair<<<(npairs + SW - 1) / SW, SW * 32, 0, st>>>(
                    geo, kc, ydiff, src.n, R, di, df, src.g, work, list, nleft);
                k_spread_scatter<T><<<(src.n + SW - 1) / SW, SW * 32, 0, st>>>(
                    geo, kc, ydiff, src.n, R, di, df, src.g, work, list, nleft);
                paired = true;
            }
        }
        if (!paired)
            k_spread_scatter<T><<<(src.n + SW - 1) / SW, SW * 32, 0, st>>>(
                geo, kc, ydiff, src.n, R, di, df, src.g, work, nullptr, nullptr);
    }
    k_deinterleave<T><<<(unsigned)((nodes + 255) / 256), 256, 0, st>>>(geo.Ny, geo.Nz, geo.Nx,
                                                                       work, grid);
    return cudaGetLastError();
}

#define GGEM_INST_SPREAD(T)                                                                  \
    template cudaError_t spread_prepare<T>(const GridGeom&, const double*, int, const int*,    \
                                           const double*, int4*, v4_t<T>*, cudaStream_t);       \
    template cudaError_t spread<T>(const GridGeom&, const CellGrid&, const double*, const T*,   \
                                   const SortedSources<T>&, const int4*, const v4_t<T>*, T*,    \
                                   T*, int*, cudaStream_t);
GGEM_INST_SPREAD(float)
GGEM_INST_SPREAD(double)

// ------------------------------------------------------------------ probe
// Throughput of float4 vector reductions into an L2-resident buffer, the
// operation the spreading is bound by: every warp adds into 32 consecutive
// 16-byte vectors (one per lane, as lanes on consecutive grid columns do) at a
// pseudo-random position of the buffer, `iters` times.  The roof the
// spreading's reduction rate is measured against.
namespace {
__global__ void k_red_probe(float4* __restrict__ buf, unsigned nvec, int iters, unsigned seed) {
    const unsigned w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    unsigned h = (w + 1u) * 2654435761u ^ seed;
    for (int it = 0; it < iters; ++it) {
        h = h * 1664525u + 1013904223u;
        const unsigned base = (h % (nvec >> 5)) << 5;
        atomicAdd(buf + base + lane, make_float4(1.f, 1.f, 1.f, 0.f));
    }
}

// Throughput of FP32 atomic adds into shared memory, the operation a spreading
// staged in shared memory would be bound by: a block holds a tile of 4096
// nodes x 3 components (48 KB, as a 16 x 16 x 16 tile of the grid), and every
// warp adds into 32 consecutive nodes (one per lane: no bank conflict within
// the warp) of each component at a pseudo-random place of the tile, `iters`
// times; the warps of a block collide as the sources of a tile would.  The
// tile is added into `out` at the end so that the adds are kept.
constexpr int kProbeNodes = 4096;
__global__ void k_smem_probe(float* __restrict__ out, int iters, unsigned seed) {
    __shared__ float acc[3 * kProbeNodes];
    for (int e = threadIdx.x; e < 3 * kProbeNodes; e += blockDim.x) acc[e] = 0.f;
    __syncthreads();
    const unsigned w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    unsigned h = (w + 1u) * 2654435761u ^ seed;
    for (int it = 0; it < iters; ++it) {
        h = h * 1664525u + 1013904223u;
        const unsigned base = ((h >> 8) % (kProbeNodes >> 5)) << 5;
        atomicAdd(&acc[base + lane], 1.f);
        atomicAdd(&acc[kProbeNodes + base + lane], 1.f);
        atomicAdd(&acc[2 * kProbeNodes + base + lane], 1.f);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * kProbeNodes; e += blockDim.x) atomicAdd(out + e, acc[e]);
}
}  // namespace

}  // namespace ggem

extern "C" ggem_status ggem_probe_smem_reduction(int iters, void* stream, double* ms,
                                                 double* adds_per_s) {
    if (iters < 1 || iters > (1 << 20) || !ms || !adds_per_s) return GGEM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GGEM_ERR_CUDA;
    const size_t nout = (size_t)3 * ggem::kProbeNodes;
    float* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    ggem_status s = GGEM_OK;
    if (cudaMalloc((void**)&out, nout * sizeof(float)) != cudaSuccess) return GGEM_ERR_CUDA;
    const int blocks = 4 * nsm, threads = 256;     // 48 KB per block: 4 blocks per SM
    if (cudaMemsetAsync(out, 0, nout * sizeof(float), st) != cudaSuccess ||
        cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        s = GGEM_ERR_CUDA;
    } else {
        ggem::k_smem_probe<<<blocks, threads, 0, st>>>(out, iters, 7u);  // warm
        cudaEventRecord(a, st);
        ggem::k_smem_probe<<<blocks, threads, 0, st>>>(out, iters, 11u);
        cudaEventRecord(b, st);
        float t = 0.f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess) {
            s = GGEM_ERR_CUDA;
        } else {
            *ms = t;
            *adds_per_s = 3.0 * blocks * threads * iters / (t * 1e-3);
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(out);
    return s;
}

extern "C" ggem_status ggem_probe_l2_reduction(long nvec, int iters, void* stream, double* ms,
                                               double* vec_per_s) {
    if (nvec < 32 || (nvec & 31) || nvec > (1L << 28) || iters < 1 || !ms || !vec_per_s)
        return GGEM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GGEM_ERR_CUDA;
    float4* buf = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    ggem_status s = GGEM_OK;
    if (cudaMalloc((void**)&buf, (size_t)nvec * sizeof(float4)) != cudaSuccess)
        return GGEM_ERR_CUDA;
    const int blocks = 8 * nsm, threads = 256;
    if (cudaMemsetAsync(buf, 0, (size_t)nvec * sizeof(float4), st) != cudaSuccess ||
        cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        s = GGEM_ERR_CUDA;
    } else {
        ggem::k_red_probe<<<blocks, threads, 0, st>>>(buf, (unsigned)nvec, iters, 7u);  // warm
        cudaEventRecord(a, st);
        ggem::k_red_probe<<<blocks, threads, 0, st>>>(buf, (unsigned)nvec, iters, 11u);
        cudaEventRecord(b, st);
        float t = 0.f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess) {
            s = GGEM_ERR_CUDA;
        } else {
            *ms = t;
            *vec_per_s = (double)blocks * threads * iters / (t * 1e-3);
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(buf);
    return s;
}
