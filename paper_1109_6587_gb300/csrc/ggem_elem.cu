// Element quadrature of the local single- and double-layer integrals
// (paper Sec. 3.4.1, Eq. (int_l); Sec. 3.5.2, Eqs. (int_dbl_l), (dbl_l1), (ntilde)).
//
// Every triangle carries the 16 points of the 4x4 Gauss-Legendre product rule
// on the collapsed parent triangle (xi = (1 - eta) s, Jacobian (1 - eta) 2A_k);
// they are point sources of strength 8 pi mu w q(xi, eta) summed by the
// ordinary local-sum kernel.  For a target node z, the triangles having z as a
// vertex need the polar rule instead (Sec. 3.4.1): the local-sum kernel skips
// their regular points, and the correction kernel adds the same 4x4 rule in
// polar coordinates (rho, theta) about z, with n-tilde = n_tri phi1 +
// n(z)(phi2 + phi3) in the double layer.  Displacements in the correction are formed from
// the triangle's edge vectors relative to z, so they are small numbers and
// exact enough in FP32.
#include "ggem_internal.cuh"

namespace ggem {

namespace {

template <typename T> __device__ __forceinline__ T e_erfc(T x);
template <> __device__ __forceinline__ float e_erfc<float>(float x) { return erfcf(x); }
template <> __device__ __forceinline__ double e_erfc<double>(double x) { return erfc(x); }
template <typename T> __device__ __forceinline__ T e_exp(T x);
template <> __device__ __forceinline__ float e_exp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double e_exp<double>(double x) { return exp(x); }
template <typename T> __device__ __forceinline__ T e_rsqrt(T x);
template <> __device__ __forceinline__ float e_rsqrt<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double e_rsqrt<double>(double x) { return rsqrt(x); }

// quadrature-point generation: one thread per (triangle, point)
template <typename T>
__global__ void k_qp_gen(int m, const double* __restrict__ x, const int* __restrict__ tri,
                         const double* __restrict__ tri_area, QuadRule rule,
                         double* __restrict__ xq, int4* __restrict__ qv,
                         v4_t<T>* __restrict__ qw) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * 16) return;
    int k = e >> 4, a = e & 3, c = (e >> 2) & 3;
    int i1 = tri[3 * k], i2 = tri[3 * k + 1], i3 = tri[3 * k + 2];
    double eta = rule.t[c], xi = (1.0 - eta) * rule.t[a];
    double wt = rule.w[a] * rule.w[c] * (1.0 - eta) * 2.0 * tri_area[k];
    double p1 = 1.0 - xi - eta, p2 = xi, p3 = eta;
    for (int d = 0; d < 3; ++d)
        xq[3 * e + d] = p1 * x[3 * i1 + d] + p2 * x[3 * i2 + d] + p3 * x[3 * i3 + d];
    qv[e] = make_int4(i1, i2, i3, 0);
    v4_t<T> w;
    w.x = (T)(p1 * wt); w.y = (T)(p2 * wt); w.z = (T)(p3 * wt); w.w = (T)0;
    qw[e] = w;
}

// strengths of the sorted quadrature points: g = scale * sum_v (phi_v w) q_v,
// from the vertex indices and weights already in point order (qv, qw), into
// interleaved v4 (g); in T throughout (q is the nodal density in T, so FP32
// plans spend no FP64 instruction here -- GB300 runs FP64 at 1/64 of the FP32
// rate)
template <typename T>
__device__ __forceinline__ void qp_strength_of(int s, const int4* __restrict__ qv,
                                               const v4_t<T>* __restrict__ qw,
                                               const T* __restrict__ q, T scale, T& rx, T& ry,
                                               T& rz) {
    const int4 v = qv[s];
    const v4_t<T> w = qw[s];
    const T a = scale * w.x, b = scale * w.y, c = scale * w.z;
    rx = a * q[3 * v.x] + b * q[3 * v.y] + c * q[3 * v.z];
    ry = a * q[3 * v.x + 1] + b * q[3 * v.y + 1] + c * q[3 * v.z + 1];
    rz = a * q[3 * v.x + 2] + b * q[3 * v.y + 2] + c * q[3 * v.z + 2];
}

template <typename T>
__global__ void k_qp_strength(int n, const int4* __restrict__ qv, const v4_t<T>* __restrict__ qw,
                              const T* __restrict__ q, T scale, v4_t<T>* __restrict__ g) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    v4_t<T> r;
    qp_strength_of<T>(s, qv, qw, q, scale, r.x, r.y, r.z);
    r.w = (T)0;
    g[s] = r;
}

// The same for the FP32 element rule, straight into the packed point layout:
// one thread per pair of slots h (slots 2h, 2h + 1; inv maps a slot to its
// sorted point, -1 for a dummy, whose strength stays zero), writing gx, gy, gz
// of both as three 8-byte pairs at floats 6, 8, 10 of the pair's 12
__global__ void k_qp_strength_pack(long npairs, const int* __restrict__ inv,
                                   const int4* __restrict__ qv, const float4* __restrict__ qw,
                                   const float* __restrict__ q, float scale,
                                   float* __restrict__ pack) {
    const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= npairs) return;
    const int s0 = inv[2 * h], s1 = inv[2 * h + 1];
    float x0 = 0.f, y0 = 0.f, z0 = 0.f, x1 = 0.f, y1 = 0.f, z1 = 0.f;
    if (s0 >= 0) qp_strength_of<float>(s0, qv, qw, q, scale, x0, y0, z0);
    if (s1 >= 0) qp_strength_of<float>(s1, qv, qw, q, scale, x1, y1, z1);
    float2* o = reinterpret_cast<float2*>(pack + 12 * h + 6);
    o[0] = make_float2(x0, x1);
    o[1] = make_float2(y0, y1);
    o[2] = make_float2(z0, z1);
}

// out[s] = in[perm[s]] (the quadrature weights into point order)
template <typename T>
__global__ void k_gather_v4(int n, const int* __restrict__ perm, const v4_t<T>* __restrict__ in,
                            v4_t<T>* __restrict__ out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) out[s] = in[perm[s]];
}

// node -> triangle adjacency (CSR)
__global__ void k_adj_count(int m, const int* __restrict__ tri, int* __restrict__ cnt) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    for (int v = 0; v < 3; ++v) atomicAdd(&cnt[tri[3 * k + v]], 1);
}

__global__ void k_adj_fill(int m, const int* __restrict__ tri, const int* __restrict__ start,
                           int* __restrict__ cur, int* __restrict__ list) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    for (int v = 0; v < 3; ++v) {
        int b = tri[3 * k + v];
        list[start[b] + atomicAdd(&cur[b], 1)] = k;
    }
}

// Per target node: for each triangle having it as a vertex, add the 4x4 rule
// in polar coordinates about the node (the local-sum kernel skipped those
// triangles' regular points).  layer 0: out += G^l terms (single);
// layer 1: out += T^l terms with n-tilde (double).  out is the local-sum
// output [n][3] in caller order, already scaled like it (1/(8 pi mu) G g = G w q).
template <typename T>
__global__ void __launch_bounds__(128) k_elem_correct(
    int n, int layer, T alpha, T rc2, const double* __restrict__ x, const int* __restrict__ tri,
    const double* __restrict__ tri_nrm, const double* __restrict__ nrm,
    const int* __restrict__ adj_start, const int* __restrict__ adj,
    const T* __restrict__ q, QuadRule rule, T* __restrict__ out, int out_stride) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const T al = alpha, al2 = alpha * alpha;
    const T sp = (T)1.7724538509055160273;
    const T c1 = (T)2 * al / sp, c2 = (T)12 * al / sp, c3 = (T)8 * al * al2 / sp,
            c4 = (T)4 * al * al2 / sp;
    T nz0 = 0, nz1 = 0, nz2 = 0;
    if (layer == 1) { nz0 = (T)nrm[3 * b]; nz1 = (T)nrm[3 * b + 1]; nz2 = (T)nrm[3 * b + 2]; }
    T rt[4], rw[4], rc_[4], rs_[4], rm[4], rwt[4];
    for (int i = 0; i < 4; ++i) {
        rt[i] = (T)rule.t[i]; rw[i] = (T)rule.w[i]; rc_[i] = (T)rule.cth[i];
        rs_[i] = (T)rule.sth[i]; rm[i] = (T)rule.rmax[i]; rwt[i] = (T)rule.wth[i];
    }
    T acc0 = 0, acc1 = 0, acc2 = 0;
    for (int e = adj_start[b]; e < adj_start[b + 1]; ++e) {
        int k = adj[e];
        int v0 = tri[3 * k], v1 = tri[3 * k + 1], v2 = tri[3 * k + 2];
        // vertex 1 = b (cyclic rotation keeps the orientation)
        int i2 = v1, i3 = v2;
        if (v1 == b) { i2 = v2; i3 = v0; }
        else if (v2 == b) { i2 = v0; i3 = v1; }
        T e2[3], e3[3], q1[3], q2[3], q3[3], nt[3];
        for (int d = 0; d < 3; ++d) {
            e2[d] = (T)(x[3 * i2 + d] - x[3 * b + d]);
            e3[d] = (T)(x[3 * i3 + d] - x[3 * b + d]);
            q1[d] = q[3 * b + d];
            q2[d] = q[3 * i2 + d];
            q3[d] = q[3 * i3 + d];
            nt[d] = (T)tri_nrm[3 * k + d];
        }
        T cx = e2[1] * e3[2] - e2[2] * e3[1], cy = e2[2] * e3[0] - e2[0] * e3[2],
          cz = e2[0] * e3[1] - e2[1] * e3[0];
        T omega = sqrt(cx * cx + cy * cy + cz * cz);     // |x_xi x x_eta| = 2 A_k
        for (int qa = 0; qa < 4; ++qa)
            for (int qc = 0; qc < 4; ++qc) {
                T rmax = rm[qa];
                T rho = rmax * rt[qc];
                T xi = rho * rc_[qa];
                T eta = rho * rs_[qa];
                T wgt = rwt[qa] * rmax * rw[qc] * rho * omega;
                T p1 = (T)1 - xi - eta;
                // displacement target - point = -(xi e2 + eta e3)
                T dx = -(xi * e2[0] + eta * e3[0]);
                T dy = -(xi * e2[1] + eta * e3[1]);
                T dz = -(xi * e2[2] + eta * e3[2]);
                T g0 = (p1 * q1[0] + xi * q2[0] + eta * q3[0]) * wgt;
                T g1 = (p1 * q1[1] + xi * q2[1] + eta * q3[1]) * wgt;
                T g2 = (p1 * q1[2] + xi * q2[2] + eta * q3[2]) * wgt;
                T r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 > (T)0 && r2 < rc2)) continue;
                T ir = e_rsqrt<T>(r2), r = r2 * ir;
                T ec = e_erfc<T>(al * r), ex = e_exp<T>(-al2 * r2);
                T xg = dx * g0 + dy * g1 + dz * g2;
                if (layer == 0) {
                    T A = ec * ir - c1 * ex;
                    T B = (ec * ir * ir * ir + c1 * ex * ir * ir) * xg;
                    acc0 += A * g0 + B * dx;
                    acc1 += A * g1 + B * dy;
                    acc2 += A * g2 + B * dz;
                } else {
                    // n-tilde = n_tri phi1 + n(z)(phi2 + phi3)
                    T s23 = xi + eta;
                    T n0 = nt[0] * p1 + nz0 * s23;
                    T n1 = nt[1] * p1 + nz1 * s23;
                    T n2 = nt[2] * p1 + nz2 * s23;
                    T ir2 = ir * ir;
                    T D = -(T)6 * ec * ir2 * ir2 * ir - c2 * ex * ir2 * ir2 - c3 * ex * ir2;
                    T E = c4 * ex;
                    T xn = dx * n0 + dy * n1 + dz * n2;
                    T gn = g0 * n0 + g1 * n1 + g2 * n2;
                    T Dxn = D * xg * xn;
                    acc0 += Dxn * dx + E * (dx * gn + g0 * xn + n0 * xg);
                    acc1 += Dxn * dy + E * (dy * gn + g1 * xn + n1 * xg);
                    acc2 += Dxn * dz + E * (dz * gn + g2 * xn + n2 * xg);
                }
            }
    }
    T* o = out + (size_t)b * out_stride;
    o[0] += acc0;
    o[1] += acc1;
    o[2] += acc2;
}

}  // namespace

// 4-point Gauss-Legendre rule on [0,1] by Newton iteration on P_4, and the
// polar-rule angles theta_a = (pi/2) t_a with rho_max = 1/(cos + sin).
QuadRule make_quad_rule() {
    QuadRule r;
    const int n = 4;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        r.t[i] = 0.5 * (1.0 - z);
        r.w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    for (int a = 0; a < n; ++a) {
        double th = 0.5 * pi * r.t[a];
        r.th[a] = th;
        r.cth[a] = std::cos(th);
        r.sth[a] = std::sin(th);
        r.rmax[a] = 1.0 / (std::cos(th) + std::sin(th));
        r.wth[a] = 0.5 * pi * r.w[a];
    }
    return r;
}

template <typename T>
cudaError_t elem_setup(int m, const double* x, const int* tri, const double* tri_area,
                       const QuadRule& rule, double* xq, int4* qv, v4_t<T>* qw, int nnodes,
                       int* adj_cnt, int* adj_start, int* adj_cur, int* adj,
                       cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    if (xq)      // quadrature points (element rule only); the adjacency always
        k_qp_gen<T><<<(m * 16 + 255) / 256, 256, 0, st>>>(m, x, tri, tri_area, rule, xq, qv, qw);
    cudaMemsetAsync(adj_cnt, 0, nnodes * sizeof(int), st);
    cudaMemsetAsync(adj_cur, 0, nnodes * sizeof(int), st);
    k_adj_count<<<(m + 255) / 256, 256, 0, st>>>(m, tri, adj_cnt);
    scan_counts(nnodes, adj_cnt, adj_start, st);
    k_adj_fill<<<(m + 255) / 256, 256, 0, st>>>(m, tri, adj_start, adj_cur, adj);
    return cudaGetLastError();
}

template <typename T>
cudaError_t qp_sort_weights(int nq, const int* perm, v4_t<T>* qw, v4_t<T>* tmp, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    k_gather_v4<T><<<(nq + 255) / 256, 256, 0, st>>>(nq, perm, qw, tmp);
    return cudaMemcpyAsync(qw, tmp, (size_t)nq * sizeof(v4_t<T>), cudaMemcpyDeviceToDevice, st);
}

__global__ void k_density_f32(long n, const double* __restrict__ q, float* __restrict__ out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = (float)q[e];
}

template <typename T>
cudaError_t qp_strengths(int nq, const int4* qv, const v4_t<T>* qw, int nnodes, const double* q,
                         T* qT, double scale, v4_t<T>* g, T* pack, const int* inv, long nslots,
                         cudaStream_t st) {
    if constexpr (sizeof(T) == 8) {
        (void)qT;
        (void)pack;
        (void)inv;
        (void)nslots;
        if (nq > 0) k_qp_strength<T><<<(nq + 255) / 256, 256, 0, st>>>(nq, qv, qw, q, scale, g);
    } else {
        if (!qT || !pack || !inv) return cudaErrorInvalidValue;
        const long ne = 3L * nnodes;
        if (ne > 0) k_density_f32<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(ne, q, qT);
        const long npairs = nslots / 2;
        if (npairs > 0)
            k_qp_strength_pack<<<(unsigned)((npairs + 255) / 256), 256, 0, st>>>(
                npairs, inv, qv, qw, qT, (float)scale, pack);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t elem_correct(int n, int layer, const GridGeom& geo, const double* x, const int* tri,
                         const double* tri_nrm, const double* nrm, const int* adj_start,
                         const int* adj, const T* q, const QuadRule& rule, T* out,
                         int out_stride, cudaStream_t st) {
    if (n > 0)
        k_elem_correct<T><<<(n + 127) / 128, 128, 0, st>>>(
            n, layer, (T)geo.alpha, (T)(geo.rcut * geo.rcut), x, tri, tri_nrm, nrm, adj_start,
            adj, q, rule, out, out_stride);
    return cudaGetLastError();
}

#define GGEM_INST_ELEM(T)                                                                     \
    template cudaError_t elem_setup<T>(int, const double*, const int*, const double*,          \
                                       const QuadRule&, double*, int4*, v4_t<T>*, int, int*,    \
                                       int*, int*, int*, cudaStream_t);                         \
    template cudaError_t qp_sort_weights<T>(int, const int*, v4_t<T>*, v4_t<T>*, cudaStream_t); \
    template cudaError_t qp_strengths<T>(int, const int4*, const v4_t<T>*, int, const double*, \
                                         T*, double, v4_t<T>*, T*, const int*, long,           \
                                         cudaStream_t);                                        \
    template cudaError_t elem_correct<T>(int, int, const GridGeom&, const double*, const int*, \
                                         const double*, const double*, const int*, const int*,  \
                                         const T*, const QuadRule&, T*, int, cudaStream_t);
GGEM_INST_ELEM(float)
GGEM_INST_ELEM(double)

}  // namespace ggem
