// Learned warm start for the Fredholm solve A q = b, A = I + (kappa/4 pi) D
// (the paper has no counterpart: it starts GMRES from the previous time step,
// Sec. 5).  A 12-128-128-128-3 ReLU network approximates A^-1 r - r node by
// node for a right-hand side r (the residual of a guess); the solver starts
// from whichever of the guess and the guess + A^-1 r estimate has the lower
// residual.
//
// Features (per node, caller order), FP32, with s = rms(r) (FP64):
//   0-2 r/s, 3-5 (kappa/4 pi)(D r)/s (one double-layer evaluation), 6-8 the
//   area-averaged unit normal, 9 kappa, 10 distance to the nearer wall,
//   11 nodes of other particles within r_cut / nodes of the own particle.
// Network: inputs standardised (f - mu)/sigma; weight matrices and hidden
// activations rounded to bfloat16, products accumulated in FP32; output in
// units of s s_y.  Training: mean squared error, backpropagation in FP32 with
// the same bfloat16 weights, gradients accumulated with atomics, Adam on FP32
// master weights.  FP32 mode (ggem_mlp_precision): the same kernels with no
// bfloat16 rounding point -- FP32 master weights, FP32 inputs and activations.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "ggem.h"
#include "ggem_host.cuh"

using namespace ggem;

namespace {

constexpr int H = 128;        // hidden width
constexpr int NF = 12;        // features
constexpr int TN = 16;        // nodes per block of the network kernels
constexpr int OW1 = 0, OB1 = OW1 + NF * H, OW2 = OB1 + H, OB2 = OW2 + H * H;
constexpr int OW3 = OB2 + H, OB3 = OW3 + H * H, OW4 = OB3 + H, OB4 = OW4 + H * 3;
constexpr int NP = OB4 + 3;   // parameters (35,075)
constexpr int NSTAT = 2 * NF + 1;            // mu[12], sigma[12], s_y

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
// a rounding point of the network: bfloat16 in BF16 mode, none in FP32 mode
template <bool BF> __device__ __forceinline__ float rp(float x) { return BF ? bfr(x) : x; }

// ------------------------------------------------------------- features
// sum of squares of n doubles into *acc (FP64 atomics of block sums)
__global__ void k_sumsq(size_t n, const double* __restrict__ a, double* __restrict__ acc) {
    __shared__ double red[8];
    double t = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        t += a[i] * a[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(acc, s);
    }
}

// Features 0-10 from r, D r and the geometry; ssq = sum of r^2 over 3n entries
__global__ void k_feat_local(int n, const double* __restrict__ x, const double* __restrict__ nrm,
                             const double* __restrict__ kappa, const double* __restrict__ r,
                             const double* __restrict__ Dr, const double* __restrict__ ssq,
                             double y0, double W, float* __restrict__ f) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = sqrt(*ssq / (3.0 * n));
    const double is = s > 0.0 ? 1.0 / s : 0.0;
    const double kc = kappa[i] * (0.25 / 3.14159265358979323846);
    const double y = x[3 * i + 1];
    float* o = f + (size_t)i * NF;
    for (int c = 0; c < 3; ++c) {
        o[c] = (float)(r[3 * i + c] * is);
        o[3 + c] = (float)(kc * Dr[3 * i + c] * is);
        o[6 + c] = (float)nrm[3 * i + c];
    }
    o[9] = (float)kappa[i];
    o[10] = (float)fmin(y - y0, y0 + W - y);
}

// Crowding: nodes of other particles within r_cut (minimum image), one warp
// per node over the mesh cell list (cells at least r_cut/R wide, R = reach).  The
// distance is formed in FP64 with every product and sum rounded separately,
// the same operations in the same order as the oracle, so the integer count
// does not depend on contraction into FMAs.
__global__ void k_feat_crowd(int n, GridGeom geo, CellGrid cg, const double* __restrict__ x,
                             const int* __restrict__ mesh_cell_of, const int* __restrict__ perm,
                             const int* __restrict__ cell_start,
                             const int* __restrict__ particle, const int* __restrict__ pcount,
                             double rc2, float* __restrict__ f) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wid >= n) return;
    const int i = perm[wid];                   // sorted node -> caller index
    const int c = mesh_cell_of[wid];
    const int cx = c % cg.ncx, cy = (c / cg.ncx) % cg.ncy, cz = c / (cg.ncx * cg.ncy);
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    const int pi = particle[i];
    // distinct cells within +-R in x and z (all of them on a grid narrower
    // than 2R + 1 cells), +-R in y; each node is met once
    const int R = cg.reach, side = 2 * R + 1;
    const int nxo = min(side, cg.ncx), nzo = min(side, cg.ncz);
    const int x0 = cg.ncx >= side ? cx - R : 0, z0 = cg.ncz >= side ? cz - R : 0;
    int count = 0;
    for (int a = 0; a < nzo; ++a)
        for (int dy = -R; dy <= R; ++dy) {
            const int cyy = cy + dy;
            if (cyy < 0 || cyy >= cg.ncy) continue;
            const int czz = ((z0 + a) % cg.ncz + cg.ncz) % cg.ncz;
            for (int e = 0; e < nxo; ++e) {
                const int cxx = ((x0 + e) % cg.ncx + cg.ncx) % cg.ncx;
                const int cc = (czz * cg.ncy + cyy) * cg.ncx + cxx;
                for (int s = cell_start[cc] + lane; s < cell_start[cc + 1]; s += 32) {
                    const int j = perm[s];
                    if (particle[j] == pi) continue;
                    double d0 = __dsub_rn(x[3 * j], xi);
                    double d1 = __dsub_rn(x[3 * j + 1], yi);
                    double d2 = __dsub_rn(x[3 * j + 2], zi);
                    d0 = __dsub_rn(d0, __dmul_rn(geo.Lx, rint(__ddiv_rn(d0, geo.Lx))));
                    d2 = __dsub_rn(d2, __dmul_rn(geo.Lz, rint(__ddiv_rn(d2, geo.Lz))));
                    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)),
                                                __dmul_rn(d2, d2));
                    count += r2 < rc2;
                }
            }
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) count += __shfl_xor_sync(0xffffffffu, count, o);
    if (lane == 0) f[(size_t)i * NF + 11] = (float)((double)count / pcount[pi]);
}

// ------------------------------------------------------------- network
struct Net {
    const float* p;               // FP32 master parameters (biases; weights in FP32 mode)
    const __nv_bfloat16* wf;      // bfloat16 weights, [fan_in][fan_out]
    const __nv_bfloat16* wt;      // bfloat16 weights, [fan_out][fan_in] (layers 2-4)
    const float* stats;           // mu[12], sigma[12], s_y
};

// weight W[k][j] of the layer at offset ow with fan_out fo, as the mode uses it
template <bool BF>
__device__ __forceinline__ float wgt(const Net& net, int ow, int fo, int k, int j) {
    return BF ? ld(net.wf + ow + k * fo + j) : net.p[ow + k * fo + j];
}

// out[n][j] = relu(bias[j] + sum_k in[n][k] W[k][j]) (rounded to bfloat16 in
// BF16 mode); thread j of the block, TN nodes
template <int K, bool BF>
__device__ __forceinline__ void hidden_layer(const Net& net, int ow, int ob, const float* in,
                                             float* out) {
    const int j = threadIdx.x;
    float acc[TN];
    const float bj = net.p[ob + j];
#pragma unroll
    for (int m = 0; m < TN; ++m) acc[m] = bj;
    for (int k = 0; k < K; k += 4) {
        const float w0 = wgt<BF>(net, ow, H, k + 0, j), w1 = wgt<BF>(net, ow, H, k + 1, j);
        const float w2 = wgt<BF>(net, ow, H, k + 2, j), w3 = wgt<BF>(net, ow, H, k + 3, j);
#pragma unroll
        for (int m = 0; m < TN; ++m) {
            const float4 h = *reinterpret_cast<const float4*>(in + m * K + k);
            acc[m] = fmaf(h.x, w0, acc[m]);
            acc[m] = fmaf(h.y, w1, acc[m]);
            acc[m] = fmaf(h.z, w2, acc[m]);
            acc[m] = fmaf(h.w, w3, acc[m]);
        }
    }
#pragma unroll
    for (int m = 0; m < TN; ++m) out[m * H + j] = rp<BF>(fmaxf(acc[m], 0.f));
}

struct Acts {
    float a0[TN][NF];
    float a1[TN][H];
    float a2[TN][H];
    float a3[TN][H];
    float out[TN][3];
};

// forward pass of TN nodes (rows >= nv are zero inputs)
template <bool BF>
__device__ void forward_tile(const Net& net, const float* __restrict__ feat, int row0, int nv,
                             Acts& A) {
    for (int t = threadIdx.x; t < TN * NF; t += blockDim.x) {
        const int m = t / NF, k = t - m * NF;
        float v = 0.f;
        if (m < nv) v = (feat[(size_t)(row0 + m) * NF + k] - net.stats[k]) / net.stats[NF + k];
        A.a0[m][k] = rp<BF>(v);
    }
    __syncthreads();
    hidden_layer<NF, BF>(net, OW1, OB1, &A.a0[0][0], &A.a1[0][0]);
    __syncthreads();
    hidden_layer<H, BF>(net, OW2, OB2, &A.a1[0][0], &A.a2[0][0]);
    __syncthreads();
    hidden_layer<H, BF>(net, OW3, OB3, &A.a2[0][0], &A.a3[0][0]);
    __syncthreads();
    if (threadIdx.x < 3 * TN) {
        const int m = threadIdx.x / 3, j = threadIdx.x - 3 * m;
        float acc = net.p[OB4 + j];
        for (int k = 0; k < H; ++k) acc = fmaf(A.a3[m][k], wgt<BF>(net, OW4, 3, k, j), acc);
        A.out[m][j] = acc;
    }
    __syncthreads();
}

// raw network output (units of s_y) of n feature rows
template <bool BF>
__global__ void __launch_bounds__(H) k_mlp_forward(int n, Net net, const float* __restrict__ feat,
                                                   float* __restrict__ out) {
    __shared__ Acts A;
    const int row0 = blockIdx.x * TN, nv = min(TN, n - row0);
    forward_tile<BF>(net, feat, row0, nv, A);
    if (threadIdx.x < 3 * nv) out[(size_t)row0 * 3 + threadIdx.x] = (&A.out[0][0])[threadIdx.x];
}

// out = base + r + s s_y MLP (the A^-1 r estimate added to base), caller order
template <bool BF>
__global__ void __launch_bounds__(H) k_mlp_guess(int n, Net net, const float* __restrict__ feat,
                                                 const double* __restrict__ r,
                                                 const double* __restrict__ ssq,
                                                 const double* __restrict__ base,
                                                 double* __restrict__ out) {
    __shared__ Acts A;
    const int row0 = blockIdx.x * TN, nv = min(TN, n - row0);
    forward_tile<BF>(net, feat, row0, nv, A);
    if (threadIdx.x < 3 * nv) {
        const double s = sqrt(*ssq / (3.0 * n));
        const size_t e = (size_t)row0 * 3 + threadIdx.x;
        out[e] = (base ? base[e] : 0.0) + r[e] +
                 s * (double)net.stats[2 * NF] * (double)(&A.out[0][0])[threadIdx.x];
    }
}

// One minibatch (rows idx[0..nb) of feat/target, target in raw units): forward,
// loss sum((out - target/s_y)^2) / (3 nb) into *loss, gradients added to grad.
template <bool BF>
__global__ void __launch_bounds__(H) k_mlp_train(int nb, const int* __restrict__ idx, Net net,
                                                 const float* __restrict__ feat,
                                                 const float* __restrict__ target,
                                                 float* __restrict__ grad, float* __restrict__ loss) {
    __shared__ Acts A;
    __shared__ float fbuf[TN][NF];
    __shared__ float d3[TN][H];        // delta of the current layer
    __shared__ float d2[TN][H];
    __shared__ float d4[TN][3];
    __shared__ float red[H / 32];
    const int row0 = blockIdx.x * TN, nv = min(TN, nb - row0);
    // gather the minibatch rows into a contiguous tile
    for (int t = threadIdx.x; t < TN * NF; t += blockDim.x) {
        const int m = t / NF, k = t - m * NF;
        fbuf[m][k] = m < nv ? feat[(size_t)idx[row0 + m] * NF + k] : 0.f;
    }
    __syncthreads();
    forward_tile<BF>(net, &fbuf[0][0], 0, nv, A);
    const float scale = 2.f / (3.f * (float)nb), isy = 1.f / net.stats[2 * NF];
    float lsum = 0.f;
    if (threadIdx.x < 3 * TN) {
        const int m = threadIdx.x / 3, j = threadIdx.x - 3 * m;
        float dlt = 0.f;
        if (m < nv) {
            const float e = A.out[m][j] - target[(size_t)idx[row0 + m] * 3 + j] * isy;
            lsum = e * e;
            dlt = scale * e;
        }
        d4[m][j] = dlt;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int q = 0; q < H / 32; ++q) s += red[q];
        atomicAdd(loss, s / (3.f * (float)nb));
    }
    const int t = threadIdx.x;                 // 0..127
    // layer 4: dW4[k][j] = sum_m a3[m][k] d4[m][j]; d3 = (W4 d4) * (a3 > 0)
    {
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        const float w0 = wgt<BF>(net, OW4, 3, t, 0), w1 = wgt<BF>(net, OW4, 3, t, 1),
                    w2 = wgt<BF>(net, OW4, 3, t, 2);
#pragma unroll
        for (int m = 0; m < TN; ++m) {
            const float a = A.a3[m][t];
            g0 = fmaf(a, d4[m][0], g0);
            g1 = fmaf(a, d4[m][1], g1);
            g2 = fmaf(a, d4[m][2], g2);
            const float back = d4[m][0] * w0 + d4[m][1] * w1 + d4[m][2] * w2;
            d3[m][t] = a > 0.f ? back : 0.f;
        }
        atomicAdd(grad + OW4 + t * 3, g0);
        atomicAdd(grad + OW4 + t * 3 + 1, g1);
        atomicAdd(grad + OW4 + t * 3 + 2, g2);
        if (t < 3) {
            float s = 0.f;
            for (int m = 0; m < TN; ++m) s += d4[m][t];
            atomicAdd(grad + OB4 + t, s);
        }
    }
    __syncthreads();
    // hidden layers l = 3, 2, 1: dW_l[k][j] = sum_m in[m][k] d[m][j] (thread j),
    // db_l[j] = sum_m d[m][j]; d_prev[m][k] = (sum_j W_l[k][j] d[m][j]) * (in > 0)
    float (*dcur)[H] = d3;
    float (*dnext)[H] = d2;
    for (int l = 3; l >= 1; --l) {
        const int ow = l == 3 ? OW3 : (l == 2 ? OW2 : OW1);
        const int ob = l == 3 ? OB3 : (l == 2 ? OB2 : OB1);
        const float* in = l == 3 ? &A.a2[0][0] : (l == 2 ? &A.a1[0][0] : &A.a0[0][0]);
        const int K = l == 1 ? NF : H;
        {
            float dj[TN];
            float sb = 0.f;
#pragma unroll
            for (int m = 0; m < TN; ++m) {
                dj[m] = dcur[m][t];
                sb += dj[m];
            }
            atomicAdd(grad + ob + t, sb);
            for (int k = 0; k < K; ++k) {
                float g = 0.f;
#pragma unroll
                for (int m = 0; m < TN; ++m) g = fmaf(in[m * K + k], dj[m], g);
                atomicAdd(grad + ow + k * H + t, g);
            }
        }
        if (l > 1) {
            // thread t = input index k of layer l
            float acc[TN];
#pragma unroll
            for (int m = 0; m < TN; ++m) acc[m] = 0.f;
            for (int j = 0; j < H; j += 4) {
                // W_l[t][j .. j + 3]: the transposed bfloat16 copy (coalesced) or
                // the FP32 masters
                const float w0 = BF ? ld(net.wt + ow + (j + 0) * H + t) : net.p[ow + t * H + j],
                            w1 = BF ? ld(net.wt + ow + (j + 1) * H + t) : net.p[ow + t * H + j + 1],
                            w2 = BF ? ld(net.wt + ow + (j + 2) * H + t) : net.p[ow + t * H + j + 2],
                            w3 = BF ? ld(net.wt + ow + (j + 3) * H + t) : net.p[ow + t * H + j + 3];
#pragma unroll
                for (int m = 0; m < TN; ++m) {
                    const float4 dv = *reinterpret_cast<const float4*>(&dcur[m][j]);
                    acc[m] = fmaf(dv.x, w0, acc[m]);
                    acc[m] = fmaf(dv.y, w1, acc[m]);
                    acc[m] = fmaf(dv.z, w2, acc[m]);
                    acc[m] = fmaf(dv.w, w3, acc[m]);
                }
            }
            __syncthreads();                     // dnext may alias a buffer still read
#pragma unroll
            for (int m = 0; m < TN; ++m) dnext[m][t] = in[m * K + t] > 0.f ? acc[m] : 0.f;
            __syncthreads();
            float (*tmp)[H] = dcur;
            dcur = dnext;
            dnext = tmp;
        }
    }
}

// Adam on the FP32 masters; gradients cleared; bfloat16 copies refreshed
__global__ void k_mlp_adam(float* __restrict__ p, float* __restrict__ grad, float* __restrict__ m1,
                           float* __restrict__ m2, __nv_bfloat16* __restrict__ wf,
                           __nv_bfloat16* __restrict__ wt, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float g = grad[i];
    grad[i] = 0.f;
    const float a = 0.9f * m1[i] + 0.1f * g;
    const float v = 0.999f * m2[i] + 0.001f * g * g;
    m1[i] = a;
    m2[i] = v;
    const float w = p[i] - lr * (a / c1) / (sqrtf(v / c2) + 1e-8f);
    p[i] = w;
    const __nv_bfloat16 wb = __float2bfloat16_rn(w);
    if (i < OB1) {
        wf[i] = wb;
    } else if (i >= OW2 && i < OB2) {
        const int k = (i - OW2) / H, j = (i - OW2) % H;
        wf[i] = wb;
        wt[OW2 + j * H + k] = wb;
    } else if (i >= OW3 && i < OB3) {
        const int k = (i - OW3) / H, j = (i - OW3) % H;
        wf[i] = wb;
        wt[OW3 + j * H + k] = wb;
    } else if (i >= OW4 && i < OB4) {
        const int k = (i - OW4) / 3, j = (i - OW4) % 3;
        wf[i] = wb;
        wt[OW4 + j * H + k] = wb;
    }
}

// refresh both bfloat16 copies from the masters (after a load or init)
__global__ void k_mlp_round(const float* __restrict__ p, __nv_bfloat16* __restrict__ wf,
                            __nv_bfloat16* __restrict__ wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const __nv_bfloat16 wb = __float2bfloat16_rn(p[i]);
    wf[i] = wb;
    if (i >= OW2 && i < OB2) wt[OW2 + ((i - OW2) % H) * H + (i - OW2) / H] = wb;
    else if (i >= OW3 && i < OB3) wt[OW3 + ((i - OW3) % H) * H + (i - OW3) / H] = wb;
    else if (i >= OW4 && i < OB4) wt[OW4 + ((i - OW4) % 3) * H + (i - OW4) / 3] = wb;
}

// per-feature sums of x and x^2 and the sum of squared targets (FP64)
__global__ void k_mlp_moments(int n, const float* __restrict__ feat,
                              const float* __restrict__ target, double* __restrict__ acc) {
    __shared__ double s[2 * NF + 1];
    for (int t = threadIdx.x; t < 2 * NF + 1; t += blockDim.x) s[t] = 0.0;
    __syncthreads();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        for (int k = 0; k < NF; ++k) {
            const double v = feat[(size_t)r * NF + k];
            atomicAdd(&s[k], v);
            atomicAdd(&s[NF + k], v * v);
        }
        const double t0 = target[3 * (size_t)r], t1 = target[3 * (size_t)r + 1],
                     t2 = target[3 * (size_t)r + 2];
        atomicAdd(&s[2 * NF], t0 * t0 + t1 * t1 + t2 * t2);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * NF + 1; t += blockDim.x) atomicAdd(&acc[t], s[t]);
}

__global__ void k_to_float(size_t n, const double* __restrict__ a, float* __restrict__ b) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

__global__ void k_to_double(size_t n, const float* __restrict__ a, double* __restrict__ b) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

unsigned nblk(size_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

void ensure_mlp(ggem_plan_t* P) {
    if (P->d_mlp) return;
    dalloc(P, &P->d_mlp, NP);
    dalloc(P, &P->d_mlp_grad, NP);
    dalloc(P, &P->d_mlp_m, NP);
    dalloc(P, &P->d_mlp_v, NP);
    dalloc(P, &P->d_mlp_wf, NP);
    dalloc(P, &P->d_mlp_wt, NP);
    dalloc(P, &P->d_mlp_stats, NSTAT);
    dalloc(P, &P->d_feat, (size_t)P->cap * NF);
    dalloc(P, &P->d_mlp_out, (size_t)P->cap * 3);
    dalloc(P, &P->d_mlp_dr, (size_t)P->cap * 3);
    dalloc(P, &P->d_mlp_ssq, 1);
    dalloc(P, &P->d_mlp_tc, mlp_tc_image_elems());
    GG_CUDA(cudaMemsetAsync(P->d_mlp_grad, 0, NP * sizeof(float), P->st));
}

Net net_of(ggem_plan_t* P) {
    return Net{P->d_mlp, (const __nv_bfloat16*)P->d_mlp_wf, (const __nv_bfloat16*)P->d_mlp_wt,
               P->d_mlp_stats};
}

// one minibatch's forward, loss and gradient (added to P->d_mlp_grad): FP32
// mode on the SIMT kernel, BF16 mode as tensor-core GEMMs (ggem_mlp_tc.cu)
void train_batch(ggem_plan_t* P, int nb, const int* idx, const float* f, const float* t,
                 float* dloss) {
    if (P->mlp_fp32) {
        k_mlp_train<false><<<nblk(nb, TN), H, 0, P->st>>>(nb, idx, net_of(P), f, t,
                                                          P->d_mlp_grad, dloss);
        P->launches += 1;
    } else {
        GG_CHECK(nb <= P->mlp_tcs_rows, GGEM_ERR_INVALID_ARG, "training scratch too small");
        GG_CUDA(mlp_tc_train_batch(nb, idx, f, t, P->d_mlp, P->d_mlp_stats, P->d_mlp_grad, dloss,
                                   P->d_mlp_tcs, P->d_tc_err, P->st));
        P->launches += 15;
    }
}

// tensor-core training scratch for minibatches of up to rows rows
void ensure_train_scratch(ggem_plan_t* P, int rows) {
    if (P->mlp_fp32 || P->mlp_tcs_rows >= rows) return;
    dfree(P->d_mlp_tcs);
    P->d_mlp_tcs = nullptr;
    P->mlp_tcs_rows = 0;
    dalloc(P, reinterpret_cast<unsigned char**>(&P->d_mlp_tcs), mlp_tc_train_scratch(rows));
    P->mlp_tcs_rows = rows;
}

// features of the right-hand side r (device [n][3]) on the current mesh into
// P->d_feat; P->d_mlp_ssq gets sum(r^2)
void features_impl(ggem_plan_t* P, const double* kappa, const double* r) {
    const int n = P->n_nodes;
    cudaStream_t st = P->st;
    double_layer_dev(P, r, P->d_mlp_dr);
    GG_CUDA(cudaMemsetAsync(P->d_mlp_ssq, 0, sizeof(double), st));
    k_sumsq<<<152, 256, 0, st>>>((size_t)n * 3, r, P->d_mlp_ssq);
    k_feat_local<<<nblk(n), 256, 0, st>>>(n, P->d_x, P->d_nrm, kappa, r, P->d_mlp_dr,
                                          P->d_mlp_ssq, P->geo.y0, P->geo.W, P->d_feat);
    k_feat_crowd<<<nblk((size_t)n * 32), 256, 0, st>>>(
        n, P->geo, P->cg, P->d_x, P->d_mesh_cell, P->d_mesh_perm, P->d_mesh_start, P->d_particle,
        P->d_pcount, P->geo.rcut * P->geo.rcut, P->d_feat);
    GG_CUDA(cudaGetLastError());
    P->launches += 3;
}

__global__ void k_count_particles(int n, const int* __restrict__ part, int np,
                                  int* __restrict__ cnt, int* __restrict__ bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = part[i];
    if (p < 0 || p >= np) atomicAdd(bad, 1);
    else atomicAdd(&cnt[p], 1);
}

}  // namespace

namespace ggem {
void mlp_guess_dev(ggem_plan_t* P, const double* kappa, const double* r, const double* base,
                   double* out) {
    GG_CHECK(P->mlp_ready, GGEM_ERR_INVALID_ARG, "no learned warm start is loaded");
    GG_CHECK(P->d_particle, GGEM_ERR_INVALID_ARG, "particle ids not set (ggem_mesh_particles)");
    features_impl(P, kappa, r);
    if (P->mlp_fp32) {
        k_mlp_guess<false><<<nblk(P->n_nodes, TN), H, 0, P->st>>>(P->n_nodes, net_of(P),
                                                                  P->d_feat, r, P->d_mlp_ssq,
                                                                  base, out);
        P->launches += 1;
    } else {
        // BF16 network on the tensor cores (ggem_mlp_tc.cu)
        GG_CUDA(mlp_tc_prepare(P->d_mlp, P->d_mlp_tc, P->st));
        GG_CUDA(mlp_tc_forward(P->n_nodes, 1, P->d_mlp_tc, P->d_mlp, P->d_mlp_stats, P->d_feat,
                               nullptr, r, P->d_mlp_ssq, base, out, P->d_tc_err, P->nsm,
                               P->st));
        P->launches += 2;
    }
    GG_CUDA(cudaGetLastError());
}
}  // namespace ggem

extern "C" {

ggem_status ggem_mesh_particles(ggem_plan_t* P, int n_particles, const int* particle) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready, GGEM_ERR_INVALID_ARG, "no mesh set");
        GG_CHECK(particle && n_particles > 0 && n_particles <= P->n_nodes, GGEM_ERR_INVALID_ARG,
                 "particle ids need 1 <= n_particles <= n_nodes");
        if (!P->d_particle) dalloc(P, &P->d_particle, (size_t)P->cap);
        if (P->pcount_cap < n_particles) {
            dfree(P->d_pcount);
            P->d_pcount = nullptr;
            dalloc(P, &P->d_pcount, (size_t)n_particles + 1);
            P->pcount_cap = n_particles;
        }
        const int n = P->n_nodes;
        GG_CUDA(cudaMemcpyAsync(P->d_particle, particle, (size_t)n * sizeof(int),
                                is_device_ptr(particle) ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyHostToDevice, P->st));
        GG_CUDA(cudaMemsetAsync(P->d_pcount, 0, ((size_t)n_particles + 1) * sizeof(int), P->st));
        int* bad = P->d_pcount + n_particles;
        k_count_particles<<<nblk(n), 256, 0, P->st>>>(n, P->d_particle, n_particles, P->d_pcount,
                                                      bad);
        int hbad = 0;
        GG_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));
        GG_CHECK(hbad == 0, GGEM_ERR_INVALID_ARG, "particle ids must lie in [0, n_particles)");
        P->n_particles = n_particles;
        P->particles_n = n;
        P->pcsr_ready = false;
        P->tcsr_ready = false;
    });
}

ggem_status ggem_mlp_features(ggem_plan_t* P, const double* kappa, const double* r,
                              double* feat, double* scale) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready && P->n_tris > 0, GGEM_ERR_INVALID_ARG, "needs a triangle mesh");
        GG_CHECK(P->d_particle, GGEM_ERR_INVALID_ARG, "particle ids not set");
        GG_CHECK(kappa && r && feat, GGEM_ERR_INVALID_ARG, "NULL argument");
        ensure_mlp(P);
        const size_t n3 = (size_t)P->n_nodes * 3;
        const double* kd = stage_in(P, kappa, P->d_in1, P->n_nodes);
        const double* rd = stage_in(P, r, P->d_in2, n3);
        features_impl(P, kd, rd);
        const size_t nf = (size_t)P->n_nodes * NF;
        double* tmp = nullptr;
        dalloc(P, &tmp, nf);
        k_to_double<<<nblk(nf), 256, 0, P->st>>>(nf, P->d_feat, tmp);
        GG_CUDA(cudaMemcpyAsync(feat, tmp, nf * sizeof(double), cudaMemcpyDefault, P->st));
        double ssq = 0.0;
        GG_CUDA(cudaMemcpyAsync(&ssq, P->d_mlp_ssq, sizeof(double), cudaMemcpyDeviceToHost,
                                P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));
        dfree(tmp);
        if (scale) *scale = std::sqrt(ssq / (double)n3);
    });
}

ggem_status ggem_mlp_guess(ggem_plan_t* P, const double* kappa, const double* r, double* delta) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready && P->n_tris > 0, GGEM_ERR_INVALID_ARG, "needs a triangle mesh");
        GG_CHECK(kappa && r && delta, GGEM_ERR_INVALID_ARG, "NULL argument");
        ensure_mlp(P);
        const size_t n3 = (size_t)P->n_nodes * 3;
        const double* kd = stage_in(P, kappa, P->d_in1, P->n_nodes);
        const double* rd = stage_in(P, r, P->d_in2, n3);
        OutMap mo = stage_out(delta, P->d_out0, n3);
        mlp_guess_dev(P, kd, rd, nullptr, mo.dev);
        finish_out(P, mo);
        GG_CUDA(cudaStreamSynchronize(P->st));
    });
}

ggem_status ggem_mlp_precision(ggem_plan_t* P, int mode) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(mode == GGEM_MLP_BF16 || mode == GGEM_MLP_FP32, GGEM_ERR_INVALID_ARG,
                 "mode must be GGEM_MLP_BF16 or GGEM_MLP_FP32");
        P->mlp_fp32 = mode == GGEM_MLP_FP32;
    });
}

ggem_status ggem_mlp_load(ggem_plan_t* P, const double* blob, size_t count) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(blob && count == (size_t)(NSTAT + NP), GGEM_ERR_INVALID_ARG,
                 "a model is 25 + 35075 doubles (mu, sigma, s_y, parameters)");
        ensure_mlp(P);
        std::vector<double> h(count);
        GG_CUDA(cudaMemcpy(h.data(), blob, count * sizeof(double), cudaMemcpyDefault));
        for (int k = 0; k < NF; ++k)
            GG_CHECK(h[NF + k] > 0.0, GGEM_ERR_INVALID_ARG, "sigma must be positive");
        GG_CHECK(h[2 * NF] > 0.0, GGEM_ERR_INVALID_ARG, "s_y must be positive");
        std::vector<float> s(h.begin(), h.begin() + NSTAT), p(h.begin() + NSTAT, h.end());
        GG_CUDA(cudaMemcpy(P->d_mlp_stats, s.data(), NSTAT * sizeof(float),
                           cudaMemcpyHostToDevice));
        GG_CUDA(cudaMemcpy(P->d_mlp, p.data(), NP * sizeof(float), cudaMemcpyHostToDevice));
        GG_CUDA(cudaMemset(P->d_mlp_m, 0, NP * sizeof(float)));
        GG_CUDA(cudaMemset(P->d_mlp_v, 0, NP * sizeof(float)));
        k_mlp_round<<<nblk(NP), 256, 0, P->st>>>(P->d_mlp, (__nv_bfloat16*)P->d_mlp_wf,
                                                 (__nv_bfloat16*)P->d_mlp_wt);
        GG_CUDA(cudaStreamSynchronize(P->st));
        P->mlp_step = 0;
        P->mlp_ready = true;
    });
}

ggem_status ggem_mlp_save(ggem_plan_t* P, double* blob, size_t count) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mlp_ready, GGEM_ERR_INVALID_ARG, "no model");
        GG_CHECK(blob && count == (size_t)(NSTAT + NP), GGEM_ERR_INVALID_ARG,
                 "a model is 25 + 35075 doubles");
        std::vector<float> s(NSTAT), p(NP);
        GG_CUDA(cudaMemcpyAsync(s.data(), P->d_mlp_stats, NSTAT * sizeof(float),
                                cudaMemcpyDeviceToHost, P->st));
        GG_CUDA(cudaMemcpyAsync(p.data(), P->d_mlp, NP * sizeof(float), cudaMemcpyDeviceToHost,
                                P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));
        std::vector<double> h(count);
        for (int i = 0; i < NSTAT; ++i) h[i] = s[i];
        for (int i = 0; i < NP; ++i) h[NSTAT + i] = p[i];
        GG_CUDA(cudaMemcpy(blob, h.data(), count * sizeof(double), cudaMemcpyDefault));
    });
}

ggem_status ggem_mlp_adam_state(ggem_plan_t* P, int set, double* m, double* v,
                                long long* step) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mlp_ready, GGEM_ERR_INVALID_ARG, "no model");
        GG_CHECK(m && v && step, GGEM_ERR_INVALID_ARG, "NULL argument");
        std::vector<float> hm(NP), hv(NP);
        if (set) {
            GG_CHECK(*step >= 0, GGEM_ERR_INVALID_ARG, "step must be >= 0");
            std::vector<double> dm(NP), dv(NP);
            GG_CUDA(cudaMemcpy(dm.data(), m, NP * sizeof(double), cudaMemcpyDefault));
            GG_CUDA(cudaMemcpy(dv.data(), v, NP * sizeof(double), cudaMemcpyDefault));
            for (int i = 0; i < NP; ++i) {
                GG_CHECK(std::isfinite(dm[i]) && std::isfinite(dv[i]) && dv[i] >= 0.0,
                         GGEM_ERR_INVALID_ARG, "moments must be finite, second moments >= 0");
                hm[i] = (float)dm[i];
                hv[i] = (float)dv[i];
            }
            GG_CUDA(cudaMemcpy(P->d_mlp_m, hm.data(), NP * sizeof(float), cudaMemcpyHostToDevice));
            GG_CUDA(cudaMemcpy(P->d_mlp_v, hv.data(), NP * sizeof(float), cudaMemcpyHostToDevice));
            P->mlp_step = (long)*step;
        } else {
            GG_CUDA(cudaMemcpyAsync(hm.data(), P->d_mlp_m, NP * sizeof(float),
                                    cudaMemcpyDeviceToHost, P->st));
            GG_CUDA(cudaMemcpyAsync(hv.data(), P->d_mlp_v, NP * sizeof(float),
                                    cudaMemcpyDeviceToHost, P->st));
            GG_CUDA(cudaStreamSynchronize(P->st));
            std::vector<double> dm(hm.begin(), hm.end()), dv(hv.begin(), hv.end());
            GG_CUDA(cudaMemcpy(m, dm.data(), NP * sizeof(double), cudaMemcpyDefault));
            GG_CUDA(cudaMemcpy(v, dv.data(), NP * sizeof(double), cudaMemcpyDefault));
            *step = P->mlp_step;
        }
    });
}

ggem_status ggem_mlp_forward(ggem_plan_t* P, int n, const double* feat, double* out) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mlp_ready, GGEM_ERR_INVALID_ARG, "no model");
        GG_CHECK(n >= 0 && feat && out, GGEM_ERR_INVALID_ARG, "bad arguments");
        if (n == 0) return;
        float *f = nullptr, *o = nullptr;
        double *fd = nullptr, *od = nullptr;
        dalloc(P, &f, (size_t)n * NF);
        dalloc(P, &o, (size_t)n * 3);
        dalloc(P, &fd, (size_t)n * NF);
        dalloc(P, &od, (size_t)n * 3);
        GG_CUDA(cudaMemcpyAsync(fd, feat, (size_t)n * NF * sizeof(double), cudaMemcpyDefault,
                                P->st));
        k_to_float<<<nblk((size_t)n * NF), 256, 0, P->st>>>((size_t)n * NF, fd, f);
        if (P->mlp_fp32) {
            k_mlp_forward<false><<<nblk(n, TN), H, 0, P->st>>>(n, net_of(P), f, o);
        } else {
            GG_CUDA(mlp_tc_prepare(P->d_mlp, P->d_mlp_tc, P->st));
            GG_CUDA(mlp_tc_forward(n, 0, P->d_mlp_tc, P->d_mlp, P->d_mlp_stats, f, o, nullptr,
                                   nullptr, nullptr, nullptr, P->d_tc_err, P->nsm, P->st));
        }
        k_to_double<<<nblk((size_t)n * 3), 256, 0, P->st>>>((size_t)n * 3, o, od);
        GG_CUDA(cudaMemcpyAsync(out, od, (size_t)n * 3 * sizeof(double), cudaMemcpyDefault,
                                P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));
        dfree(f); dfree(o); dfree(fd); dfree(od);
    });
}

// Train on n samples (features [n][12], targets q - b [n][3], host or device):
// a fresh model (seeded He-uniform weights, statistics of these samples) when
// init != 0, else continue; epochs over shuffled minibatches of `batch` rows.
// *loss gets the mean minibatch loss of the last epoch; when grad_out is
// given and epochs == 0, it receives the gradient of one full-batch pass
// (rows in order) instead of training.
ggem_status ggem_mlp_train(ggem_plan_t* P, int n, const double* feat, const double* target,
                           int init, unsigned long long seed, int epochs, int batch, double lr,
                           double* loss, double* grad_out) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(n > 0 && feat && target, GGEM_ERR_INVALID_ARG, "need samples");
        GG_CHECK(epochs >= 0 && batch >= 1 && lr > 0.0, GGEM_ERR_INVALID_ARG, "bad schedule");
        GG_CHECK(init || P->mlp_ready, GGEM_ERR_INVALID_ARG, "no model to continue");
        ensure_mlp(P);
        cudaStream_t st = P->st;
        float *f = nullptr, *t = nullptr, *dloss = nullptr;
        double *fd = nullptr, *td = nullptr, *mom = nullptr;
        int* idx = nullptr;
        dalloc(P, &f, (size_t)n * NF);
        dalloc(P, &t, (size_t)n * 3);
        dalloc(P, &fd, (size_t)n * NF);
        dalloc(P, &td, (size_t)n * 3);
        dalloc(P, &idx, (size_t)n);
        dalloc(P, &dloss, 1);
        dalloc(P, &mom, NSTAT);
        auto release = [&] {
            dfree(f); dfree(t); dfree(fd); dfree(td); dfree(idx); dfree(dloss); dfree(mom);
        };
        try {
            GG_CUDA(cudaMemcpyAsync(fd, feat, (size_t)n * NF * sizeof(double), cudaMemcpyDefault,
                                    st));
            GG_CUDA(cudaMemcpyAsync(td, target, (size_t)n * 3 * sizeof(double),
                                    cudaMemcpyDefault, st));
            k_to_float<<<nblk((size_t)n * NF), 256, 0, st>>>((size_t)n * NF, fd, f);
            k_to_float<<<nblk((size_t)n * 3), 256, 0, st>>>((size_t)n * 3, td, t);
            std::mt19937_64 rng(seed);
            if (init) {
                GG_CUDA(cudaMemsetAsync(mom, 0, NSTAT * sizeof(double), st));
                k_mlp_moments<<<152, 256, 0, st>>>(n, f, t, mom);
                std::vector<double> hm(NSTAT);
                GG_CUDA(cudaMemcpyAsync(hm.data(), mom, NSTAT * sizeof(double),
                                        cudaMemcpyDeviceToHost, st));
                GG_CUDA(cudaStreamSynchronize(st));
                for (int k = 0; k < NSTAT; ++k)
                    GG_CHECK(std::isfinite(hm[k]), GGEM_ERR_NUMERICAL,
                             "non-finite training features or targets");
                std::vector<float> sv(NSTAT);
                for (int k = 0; k < NF; ++k) {
                    const double mu = hm[k] / n, var = hm[NF + k] / n - mu * mu;
                    const double sd = var > 0.0 ? std::sqrt(var) : 0.0;
                    sv[k] = (float)mu;
                    // a constant feature keeps sigma = 1
                    sv[NF + k] = sd > 1e-6 * (std::fabs(mu) + 1e-6) ? (float)sd : 1.f;
                }
                const double ys = std::sqrt(hm[2 * NF] / (3.0 * n));
                sv[2 * NF] = ys > 0.0 ? (float)ys : 1.f;
                std::vector<float> p(NP, 0.f);
                const int fan[4][2] = {{NF, H}, {H, H}, {H, H}, {H, 3}};
                const int ow[4] = {OW1, OW2, OW3, OW4};
                std::uniform_real_distribution<double> U(-1.0, 1.0);
                for (int l = 0; l < 4; ++l) {
                    const double lim = std::sqrt(6.0 / fan[l][0]);
                    for (int e = 0; e < fan[l][0] * fan[l][1]; ++e) p[ow[l] + e] = (float)(lim * U(rng));
                }
                GG_CUDA(cudaMemcpyAsync(P->d_mlp_stats, sv.data(), NSTAT * sizeof(float),
                                        cudaMemcpyHostToDevice, st));
                GG_CUDA(cudaMemcpyAsync(P->d_mlp, p.data(), NP * sizeof(float),
                                        cudaMemcpyHostToDevice, st));
                GG_CUDA(cudaMemsetAsync(P->d_mlp_m, 0, NP * sizeof(float), st));
                GG_CUDA(cudaMemsetAsync(P->d_mlp_v, 0, NP * sizeof(float), st));
                GG_CUDA(cudaMemsetAsync(P->d_mlp_grad, 0, NP * sizeof(float), st));
                k_mlp_round<<<nblk(NP), 256, 0, st>>>(P->d_mlp, (__nv_bfloat16*)P->d_mlp_wf,
                                                      (__nv_bfloat16*)P->d_mlp_wt);
                GG_CUDA(cudaStreamSynchronize(st));
                P->mlp_step = 0;
                P->mlp_ready = true;
            }
            std::vector<int> order(n);
            for (int i = 0; i < n; ++i) order[i] = i;
            ensure_train_scratch(P, epochs == 0 ? n : std::min(batch, n));
            if (epochs == 0) {
                // one full-batch gradient, rows in order
                GG_CUDA(cudaMemcpyAsync(idx, order.data(), (size_t)n * sizeof(int),
                                        cudaMemcpyHostToDevice, st));
                GG_CUDA(cudaMemsetAsync(dloss, 0, sizeof(float), st));
                GG_CUDA(cudaMemsetAsync(P->d_mlp_grad, 0, NP * sizeof(float), st));
                train_batch(P, n, idx, f, t, dloss);
                float hl = 0.f;
                GG_CUDA(cudaMemcpyAsync(&hl, dloss, sizeof(float), cudaMemcpyDeviceToHost, st));
                if (grad_out) {
                    double* gd = nullptr;
                    dalloc(P, &gd, NP);
                    k_to_double<<<nblk(NP), 256, 0, st>>>(NP, P->d_mlp_grad, gd);
                    GG_CUDA(cudaMemcpyAsync(grad_out, gd, NP * sizeof(double), cudaMemcpyDefault,
                                            st));
                    GG_CUDA(cudaStreamSynchronize(st));
                    dfree(gd);
                }
                GG_CUDA(cudaMemsetAsync(P->d_mlp_grad, 0, NP * sizeof(float), st));
                GG_CUDA(cudaStreamSynchronize(st));
                if (loss) *loss = hl;
                release();
                return;
            }
            double last = 0.0;
            for (int ep = 0; ep < epochs; ++ep) {
                std::shuffle(order.begin(), order.end(), rng);
                GG_CUDA(cudaMemcpyAsync(idx, order.data(), (size_t)n * sizeof(int),
                                        cudaMemcpyHostToDevice, st));
                GG_CUDA(cudaMemsetAsync(dloss, 0, sizeof(float), st));
                int nbatches = 0;
                for (int r0 = 0; r0 < n; r0 += batch) {
                    const int nb = std::min(batch, n - r0);
                    train_batch(P, nb, idx + r0, f, t, dloss);
                    P->mlp_step++;
                    const float c1 = 1.f - std::pow(0.9f, (float)P->mlp_step);
                    const float c2 = 1.f - std::pow(0.999f, (float)P->mlp_step);
                    k_mlp_adam<<<nblk(NP), 256, 0, st>>>(
                        P->d_mlp, P->d_mlp_grad, P->d_mlp_m, P->d_mlp_v,
                        (__nv_bfloat16*)P->d_mlp_wf, (__nv_bfloat16*)P->d_mlp_wt, (float)lr, c1,
                        c2);
                    ++nbatches;
                }
                GG_CUDA(cudaGetLastError());
                float hl = 0.f;
                GG_CUDA(cudaMemcpyAsync(&hl, dloss, sizeof(float), cudaMemcpyDeviceToHost, st));
                GG_CUDA(cudaStreamSynchronize(st));
                last = hl / nbatches;
            }
            if (loss) *loss = last;
        } catch (...) {
            release();
            throw;
        }
        release();
    });
}

}  // extern "C"
