// Per-particle block preconditioner of the Fredholm solve (I + kappa/4 pi D) q = b
// of Sec. 5.  The paper solves it by GMRES without a preconditioner; here the
// solve can be right-preconditioned by M = blockdiag(M_p), one block per
// particle,
//     M_p = (I x R_p) B (I x R_p^T),   B = (I + kappa/4 pi D_ref)^-1,
// D_ref the discrete double layer of one capsule alone at the centre of a small
// periodic cell of the same slit (same wall gap, Chebyshev grid, x-z spacing,
// splitting parameter and cutoff), R_p the rotation that carries that
// reference capsule's node positions onto particle p's (polar factor of their
// cross-covariance).  All particles share the reference mesh: node l of a
// particle (its nodes in increasing index order) corresponds to node l of the
// reference.  The coupling that spreads the operator's spectrum lies across
// each particle, not between a node's own components, so B (dense, 3 n_ref
// square) is the part worth inverting.
//
// Setup: D_ref column by column (3 n_ref double-layer evaluations of unit
// densities on a plan of the small cell), then Gauss-Jordan with partial
// pivoting in FP64 on the device.  Application per GMRES step: densities
// turned into each particle's reference frame and gathered as the rows of a
// [particles][3 n_ref] matrix U, Z = U B^T by a tiled GEMM (FP32 in mixed plans,
// FP64 otherwise), turned back and scattered.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ggem.h"
#include "ggem_host.cuh"

using namespace ggem;

namespace {

// ---------------------------------------------------------------- GEMM
// C[m][n] = sum_k A[m][k] B[n][k]; A rows of stride lda, B rows of stride ldb.
// 64 x 64 tiles of C per block of 16 x 16 threads (4 x 4 each), k in steps of 16.
constexpr int GT = 64, GK = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_nt(int m, int n, int k, const T* __restrict__ A,
                                                 int lda, const T* __restrict__ B, int ldb,
                                                 T* __restrict__ C, int ldc) {
    __shared__ T As[GK][GT + 1];
    __shared__ T Bs[GK][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
    for (int k0 = 0; k0 < k; k0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int r = e / GK, kk = e - r * GK;
            const int ka = k0 + kk;
            As[kk][r] = (m0 + r < m && ka < k) ? A[(size_t)(m0 + r) * lda + ka] : (T)0;
            Bs[kk][r] = (n0 + r < n && ka < k) ? B[(size_t)(n0 + r) * ldb + ka] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = m0 + ty * 4 + i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = n0 + tx * 4 + j;
            if (c < n) C[(size_t)r * ldc + c] = acc[i][j];
        }
    }
}

// --------------------------------------------------------- Gauss-Jordan
// aug [n][2n] = [A | I]; step k: partial pivot in column k, swap, scale the
// pivot row; col[i] = aug[i][k] (the elimination factors, col[k] = 0).
constexpr int GJT = 1024;

__global__ void __launch_bounds__(GJT) k_gj_pivot(int n, int k, double* __restrict__ aug,
                                                  double* __restrict__ col,
                                                  int* __restrict__ singular) {
    __shared__ double sv[GJT / 32];
    __shared__ int si[GJT / 32];
    __shared__ int s_p;
    const size_t ld = 2 * (size_t)n;
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += GJT) {
        const double v = fabs(aug[(size_t)i * ld + k]);
        if (v > best) {
            best = v;
            bi = i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
        }
    }
    if ((threadIdx.x & 31) == 0) {
        sv[threadIdx.x >> 5] = best;
        si[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = -1.0;
        int p = k;
        for (int w = 0; w < GJT / 32; ++w)
            if (sv[w] > b || (sv[w] == b && si[w] < p)) {
                b = sv[w];
                p = si[w];
            }
        if (!(b > 0.0)) atomicOr(singular, 1);
        s_p = p;
    }
    __syncthreads();
    const int p = s_p;
    if (p != k)
        for (size_t j = k + threadIdx.x; j < ld; j += GJT) {
            const double t = aug[(size_t)k * ld + j];
            aug[(size_t)k * ld + j] = aug[(size_t)p * ld + j];
            aug[(size_t)p * ld + j] = t;
        }
    __syncthreads();
    const double piv = aug[(size_t)k * ld + k];
    const double inv = piv != 0.0 ? 1.0 / piv : 0.0;
    __syncthreads();
    for (size_t j = k + threadIdx.x; j < ld; j += GJT) aug[(size_t)k * ld + j] *= inv;
    for (int i = threadIdx.x; i < n; i += GJT) col[i] = i == k ? 0.0 : aug[(size_t)i * ld + k];
}

// aug[i][j] -= col[i] aug[k][j] for every row i != k, columns j >= k
__global__ void k_gj_elim(int n, int k, double* __restrict__ aug,
                          const double* __restrict__ col) {
    const size_t ld = 2 * (size_t)n;
    const size_t j = (size_t)k + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= ld || i == k) return;
    const double f = col[i];
    if (f != 0.0) aug[(size_t)i * ld + j] -= f * aug[(size_t)k * ld + j];
}

// column j of [I + s D | I] from col = D e_j (s = kappa / 4 pi)
__global__ void k_put_column(int n, int j, double s, const double* __restrict__ Dcol,
                             double* __restrict__ aug) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t ld = 2 * (size_t)n;
    aug[(size_t)i * ld + j] = (i == j ? 1.0 : 0.0) + s * Dcol[i];
    aug[(size_t)i * ld + n + j] = i == j ? 1.0 : 0.0;
}

// right half of aug (the inverse) into B64 and B32
__global__ void k_take_inverse(int n, const double* __restrict__ aug, double* __restrict__ B64,
                               float* __restrict__ B32) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * n) return;
    const size_t i = e / n, j = e - i * n;
    const double v = aug[i * 2 * (size_t)n + n + j];
    B64[e] = v;
    B32[e] = (float)v;
}

__global__ void k_set_entry(double* __restrict__ a, int j, double v) { a[j] = v; }

// ------------------------------------------------------------- rotations
constexpr int RT = 128;

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < RT / 32; ++w) t += red[w];
    return t;
}

__device__ void inv3(const double* a, double* o, double* det) {
    o[0] = a[4] * a[8] - a[5] * a[7];
    o[1] = a[2] * a[7] - a[1] * a[8];
    o[2] = a[1] * a[5] - a[2] * a[4];
    o[3] = a[5] * a[6] - a[3] * a[8];
    o[4] = a[0] * a[8] - a[2] * a[6];
    o[5] = a[2] * a[3] - a[0] * a[5];
    o[6] = a[3] * a[7] - a[4] * a[6];
    o[7] = a[1] * a[6] - a[0] * a[7];
    o[8] = a[0] * a[4] - a[1] * a[3];
    const double d = a[0] * o[0] + a[1] * o[3] + a[2] * o[6];
    *det = d;
    const double id = d != 0.0 ? 1.0 / d : 0.0;
    for (int e = 0; e < 9; ++e) o[e] *= id;
}

// R_p (row-major 3 x 3): polar factor of C = sum_l (x_l - c)(xref_l)^T, x_l
// particle p's nodes unwrapped about its first node (minimum image in x, z),
// c their centroid, xref the reference nodes about their centroid; scaled
// Newton iteration X <- (g X + (g X)^-T) / 2, g = |det X|^(-1/3).  Identity
// when C is singular or not orientation-preserving.
__global__ void __launch_bounds__(RT) k_pc_rotations(int nref, const int* __restrict__ pstart,
                                                     const int* __restrict__ pnodes,
                                                     const double* __restrict__ x,
                                                     const double* __restrict__ xref, double Lx,
                                                     double Lz, double* __restrict__ R) {
    __shared__ double red[RT / 32];
    const int p = blockIdx.x;
    const int* nodes = pnodes + pstart[p];
    const int i0 = nodes[0];
    const double x0 = x[3 * i0], y0 = x[3 * i0 + 1], z0 = x[3 * i0 + 2];
    double s[12] = {0};
    for (int l = threadIdx.x; l < nref; l += RT) {
        const int i = nodes[l];
        double d0 = x[3 * i] - x0, d1 = x[3 * i + 1] - y0, d2 = x[3 * i + 2] - z0;
        d0 -= Lx * rint(d0 / Lx);
        d2 -= Lz * rint(d2 / Lz);
        const double r0 = xref[3 * l], r1 = xref[3 * l + 1], r2 = xref[3 * l + 2];
        s[0] += d0 * r0; s[1] += d0 * r1; s[2] += d0 * r2;
        s[3] += d1 * r0; s[4] += d1 * r1; s[5] += d1 * r2;
        s[6] += d2 * r0; s[7] += d2 * r1; s[8] += d2 * r2;
        s[9] += d0; s[10] += d1; s[11] += d2;
    }
    double t[12];
    for (int e = 0; e < 12; ++e) t[e] = block_sum(s[e], red);
    if (threadIdx.x != 0) return;
    // xref is centred, so sum_l (d_l - c) xref_l^T = sum_l d_l xref_l^T: the
    // centroid sums (t[9..11]) drop out and are not needed
    double X[9], Xi[9], det;
    for (int e = 0; e < 9; ++e) X[e] = t[e];
    inv3(X, Xi, &det);
    bool ok = det > 0.0 && isfinite(det);
    for (int it = 0; it < 40 && ok; ++it) {
        const double g = pow(fabs(det), -1.0 / 3.0);
        double d = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                const double v = 0.5 * (g * X[3 * r + c] + Xi[3 * c + r] / g);
                d = fmax(d, fabs(v - X[3 * r + c]));
                X[3 * r + c] = v;
            }
        inv3(X, Xi, &det);
        ok = det > 0.0 && isfinite(det);
        if (d < 1e-15) break;
    }
    for (int e = 0; e < 9; ++e) R[9 * p + e] = ok ? X[e] : (e % 4 == 0 ? 1.0 : 0.0);
}

// U[p][3l + c] = (R_p^T v_i)_c, i the l-th node of particle p
template <typename T>
__global__ void k_pc_gather(int np, int nref, const int* __restrict__ pstart,
                            const int* __restrict__ pnodes, const double* __restrict__ R,
                            const double* __restrict__ v, T* __restrict__ U) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)np * nref) return;
    const int p = (int)(e / nref), l = (int)(e - (size_t)p * nref);
    const int i = pnodes[pstart[p] + l];
    const double* r = R + 9 * (size_t)p;
    const double a = v[3 * i], b = v[3 * i + 1], c = v[3 * i + 2];
    T* u = U + (size_t)p * 3 * nref + 3 * l;
    u[0] = (T)(r[0] * a + r[3] * b + r[6] * c);
    u[1] = (T)(r[1] * a + r[4] * b + r[7] * c);
    u[2] = (T)(r[2] * a + r[5] * b + r[8] * c);
}

// out_i = R_p Z[p][3l .. 3l + 2]
template <typename T>
__global__ void k_pc_scatter(int np, int nref, const int* __restrict__ pstart,
                             const int* __restrict__ pnodes, const double* __restrict__ R,
                             const T* __restrict__ Z, double* __restrict__ out) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)np * nref) return;
    const int p = (int)(e / nref), l = (int)(e - (size_t)p * nref);
    const int i = pnodes[pstart[p] + l];
    const double* r = R + 9 * (size_t)p;
    const T* z = Z + (size_t)p * 3 * nref + 3 * l;
    const double a = z[0], b = z[1], c = z[2];
    out[3 * i] = r[0] * a + r[1] * b + r[2] * c;
    out[3 * i + 1] = r[3] * a + r[4] * b + r[5] * c;
    out[3 * i + 2] = r[6] * a + r[7] * b + r[8] * c;
}

unsigned nb(size_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

template <typename T>
void gemm_nt(int m, int n, int k, const T* A, const T* B, T* C, cudaStream_t st) {
    dim3 g((n + GT - 1) / GT, (m + GT - 1) / GT);
    k_gemm_nt<T><<<g, 256, 0, st>>>(m, n, k, A, k, B, k, C, n);
}

void free_pc(ggem_plan_t* P) {
    for (void* p : {(void*)P->d_pc_B64, (void*)P->d_pc_B32, (void*)P->d_pc_xref,
                    (void*)P->d_pc_R, (void*)P->d_pc_U, (void*)P->d_pc_Z})
        dfree(p);
    P->d_pc_B64 = nullptr;
    P->d_pc_B32 = nullptr;
    P->d_pc_xref = nullptr;
    P->d_pc_R = nullptr;
    P->d_pc_U = nullptr;
    P->d_pc_Z = nullptr;
    P->pc_n = 0;
    P->pc_np = 0;
    P->pc_on = false;
}

}  // namespace

namespace ggem {

// Ready the preconditioner for a solve on the current mesh: particle node
// lists, every particle with the reference's node count, rotations.
void precond_prepare(ggem_plan_t* P) {
    GG_CHECK(P->d_particle && P->n_particles > 0, GGEM_ERR_INVALID_ARG,
             "the block preconditioner needs particle ids (ggem_mesh_particles)");
    particle_node_lists(P);
    const int np = P->n_particles;
    GG_CHECK((long)np * P->pc_n == P->n_nodes, GGEM_ERR_INVALID_ARG,
             "the block preconditioner needs every particle to have the reference's nodes");
    std::vector<int> start(np + 1);
    GG_CUDA(cudaMemcpyAsync(start.data(), P->d_pstart, (size_t)(np + 1) * sizeof(int),
                            cudaMemcpyDeviceToHost, P->st));
    GG_CUDA(cudaStreamSynchronize(P->st));
    for (int p = 0; p < np; ++p)
        GG_CHECK(start[p + 1] - start[p] == P->pc_n, GGEM_ERR_INVALID_ARG,
                 "the block preconditioner needs every particle to have the reference's nodes");
    if (P->pc_np < np) {
        for (void* q : {(void*)P->d_pc_R, (void*)P->d_pc_U, (void*)P->d_pc_Z}) dfree(q);
        P->d_pc_R = nullptr;
        P->d_pc_U = nullptr;
        P->d_pc_Z = nullptr;
        const size_t el = (size_t)np * 3 * P->pc_n;
        dalloc(P, &P->d_pc_R, (size_t)9 * np);
        dalloc(P, &P->d_pc_U, el);              // doubles: room for either precision
        dalloc(P, &P->d_pc_Z, el);
        P->pc_np = np;
    }
    k_pc_rotations<<<np, RT, 0, P->st>>>(P->pc_n, P->d_pstart, P->d_pnodes, P->d_x,
                                         P->d_pc_xref, P->geo.Lx, P->geo.Lz, P->d_pc_R);
    GG_CUDA(cudaGetLastError());
    P->launches += 1;
}

// out = M in (device arrays [n_nodes][3])
void precond_apply(ggem_plan_t* P, const double* in, double* out) {
    const int np = P->n_particles, nref = P->pc_n, n3 = 3 * nref;
    const size_t work = (size_t)np * nref;
    if (P->fp64) {
        double* U = P->d_pc_U;
        double* Z = P->d_pc_Z;
        k_pc_gather<double><<<nb(work), 256, 0, P->st>>>(np, nref, P->d_pstart, P->d_pnodes,
                                                         P->d_pc_R, in, U);
        gemm_nt<double>(np, n3, n3, U, P->d_pc_B64, Z, P->st);
        k_pc_scatter<double><<<nb(work), 256, 0, P->st>>>(np, nref, P->d_pstart, P->d_pnodes,
                                                          P->d_pc_R, Z, out);
    } else {
        float* U = reinterpret_cast<float*>(P->d_pc_U);
        float* Z = reinterpret_cast<float*>(P->d_pc_Z);
        k_pc_gather<float><<<nb(work), 256, 0, P->st>>>(np, nref, P->d_pstart, P->d_pnodes,
                                                        P->d_pc_R, in, U);
        gemm_nt<float>(np, n3, n3, U, P->d_pc_B32, Z, P->st);
        k_pc_scatter<float><<<nb(work), 256, 0, P->st>>>(np, nref, P->d_pstart, P->d_pnodes,
                                                         P->d_pc_R, Z, out);
    }
    GG_CUDA(cudaGetLastError());
    P->launches += 3;
}

void precond_free(ggem_plan_t* P) { free_pc(P); }

}  // namespace ggem

extern "C" {

ggem_status ggem_precond_set(ggem_plan_t* P, int n_ref, const double* x_ref, int n_tri_ref,
                             const int* tri_ref, double kappa, int ref_nx, int ref_nz) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    ggem_plan_t* R = nullptr;
    double *aug = nullptr, *col = nullptr, *e = nullptr, *dcol = nullptr;
    int* sing = nullptr;
    ggem_status s = guarded(P, [&] {
        GG_CHECK(n_ref > 0 && x_ref && n_tri_ref > 0 && tri_ref, GGEM_ERR_INVALID_ARG,
                 "the reference capsule needs nodes and triangles");
        GG_CHECK(std::isfinite(kappa), GGEM_ERR_INVALID_ARG, "kappa must be finite");
        GG_CHECK(ref_nx >= 4 && ref_nz >= 4 && (ref_nx & (ref_nx - 1)) == 0 &&
                     (ref_nz & (ref_nz - 1)) == 0,
                 GGEM_ERR_INVALID_ARG, "ref_nx and ref_nz must be powers of two >= 4");
        GG_CHECK((long)3 * n_ref <= 16384, GGEM_ERR_CAPACITY,
                 "the reference capsule may have at most 5461 nodes");
        free_pc(P);
        // host copies of the reference capsule, centred on its node centroid
        std::vector<double> xr((size_t)3 * n_ref);
        GG_CUDA(cudaMemcpy(xr.data(), x_ref, xr.size() * sizeof(double), cudaMemcpyDefault));
        std::vector<int> tr((size_t)3 * n_tri_ref);
        GG_CUDA(cudaMemcpy(tr.data(), tri_ref, tr.size() * sizeof(int), cudaMemcpyDefault));
        for (int t : tr) GG_CHECK(t >= 0 && t < n_ref, GGEM_ERR_INVALID_ARG,
                                  "reference triangle index out of range");
        double c[3] = {0, 0, 0};
        for (int l = 0; l < n_ref; ++l)
            for (int k = 0; k < 3; ++k) c[k] += xr[3 * l + k] / n_ref;
        for (int l = 0; l < n_ref; ++l)
            for (int k = 0; k < 3; ++k) xr[3 * l + k] -= c[k];
        // the small cell: same wall gap, Chebyshev grid, spacing, alpha, r_cut
        ggem_params rp = P->prm;
        rp.Lx = ref_nx * (P->prm.Lx / P->prm.Nx);
        rp.Lz = ref_nz * (P->prm.Lz / P->prm.Nz);
        rp.Nx = ref_nx;
        rp.Nz = ref_nz;
        rp.alpha = P->geo.alpha;
        rp.rcut_factor = P->geo.rcut * P->geo.alpha;
        rp.max_points = n_ref;
        rp.max_tris = n_tri_ref;
        s = ggem_plan(&rp, P->st, &R);
        GG_CHECK(s == GGEM_OK, s, std::string("reference cell: ") + ggem_last_error(nullptr));
        if (P->offgrid != GGEM_OFFGRID_LAGRANGE) {
            s = ggem_set_offgrid(R, P->offgrid, 0);
            GG_CHECK(s == GGEM_OK, s, std::string("reference cell: ") + ggem_last_error(R));
        }
        std::vector<double> xc(xr);
        const double ctr[3] = {0.5 * rp.Lx, rp.y0 + 0.5 * rp.W, 0.5 * rp.Lz};
        for (int l = 0; l < n_ref; ++l)
            for (int k = 0; k < 3; ++k) xc[3 * l + k] += ctr[k];
        s = ggem_mesh_set(R, n_ref, xc.data(), n_tri_ref, tr.data());
        GG_CHECK(s == GGEM_OK, s, std::string("reference capsule: ") + ggem_last_error(R));
        const int n = 3 * n_ref;
        dalloc(P, &aug, (size_t)n * 2 * n);
        dalloc(P, &col, (size_t)n);
        dalloc(P, &e, (size_t)n);
        dalloc(P, &dcol, (size_t)n);
        dalloc(P, &sing, 1);
        GG_CUDA(cudaMemsetAsync(e, 0, (size_t)n * sizeof(double), P->st));
        GG_CUDA(cudaMemsetAsync(sing, 0, sizeof(int), P->st));
        const double sk = kappa * 0.25 / kPi;
        for (int j = 0; j < n; ++j) {
            k_set_entry<<<1, 1, 0, P->st>>>(e, j, 1.0);
            double_layer_dev(R, e, dcol);
            k_put_column<<<nb(n), 256, 0, P->st>>>(n, j, sk, dcol, aug);
            k_set_entry<<<1, 1, 0, P->st>>>(e, j, 0.0);
        }
        GG_CUDA(cudaGetLastError());
        P->launches += R->launches + 3L * n;
        for (int k = 0; k < n; ++k) {
            k_gj_pivot<<<1, GJT, 0, P->st>>>(n, k, aug, col, sing);
            dim3 g(nb((size_t)2 * n - k), n);
            k_gj_elim<<<g, 256, 0, P->st>>>(n, k, aug, col);
        }
        GG_CUDA(cudaGetLastError());
        P->launches += 2L * n;
        int hs = 0;
        GG_CUDA(cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));
        GG_CHECK(hs == 0, GGEM_ERR_NUMERICAL, "the reference block is singular");
        dalloc(P, &P->d_pc_B64, (size_t)n * n);
        dalloc(P, &P->d_pc_B32, (size_t)n * n);
        dalloc(P, &P->d_pc_xref, (size_t)n);
        k_take_inverse<<<nb((size_t)n * n), 256, 0, P->st>>>(n, aug, P->d_pc_B64, P->d_pc_B32);
        GG_CUDA(cudaMemcpyAsync(P->d_pc_xref, xr.data(), (size_t)n * sizeof(double),
                                cudaMemcpyHostToDevice, P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));       // xr is freed on return
        P->launches += 1;
        P->pc_n = n_ref;
        P->pc_kappa = kappa;
        P->pc_on = true;
    });
    cudaStreamSynchronize(P->st);
    for (void* q : {(void*)aug, (void*)col, (void*)e, (void*)dcol, (void*)sing}) dfree(q);
    if (R) ggem_plan_destroy(R);
    if (s != GGEM_OK) free_pc(P);
    return s;
}

ggem_status ggem_precond_enable(ggem_plan_t* P, int on) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(on == 0 || P->pc_n > 0, GGEM_ERR_INVALID_ARG,
                 "no block preconditioner has been set (ggem_precond_set)");
        P->pc_on = on != 0;
    });
}

ggem_status ggem_precond_block(ggem_plan_t* P, double* out) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->pc_n > 0, GGEM_ERR_INVALID_ARG, "no block preconditioner has been set");
        GG_CHECK(out, GGEM_ERR_INVALID_ARG, "NULL output");
        const size_t n = (size_t)3 * P->pc_n;
        GG_CUDA(cudaMemcpyAsync(out, P->d_pc_B64, n * n * sizeof(double), cudaMemcpyDefault,
                                P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));
    });
}

}  // extern "C"
