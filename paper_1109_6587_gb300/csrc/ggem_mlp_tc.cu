// Forward pass of the learned warm start's network on the 5th-generation tensor
// cores (tcgen05), BF16 mode: the same network as the SIMT kernels of
// ggem_mlp.cu -- inputs standardised and rounded to bfloat16, bfloat16
// weights, FP32 accumulation, hidden activations relu'd and rounded to
// bfloat16 -- with every layer a 128-row tile GEMM:
//     layer 1: [128 x 16] (12 features, zero padded)  x W1 [16 x 128]
//     layers 2, 3: [128 x 128] x W [128 x 128]
//     layer 4: [128 x 128] x W4 [128 x 16] (3 outputs, zero padded)
// One CTA of 4 warps (128 threads = 128 TMEM lanes = the tile's rows) per
// tile, persistent over tiles, two CTAs per SM.  The four weight matrices are
// staged once per CTA from a prepared image (k_mlp_tc_prep, the canonical
// layout below); each layer's activations are written by the epilogue of the
// previous one straight into the A operand of the next.  One thread issues the
// MMAs (M = 128, K = 16 per instruction) and commits them to an mbarrier;
// every wait is bounded: on expiry the kernel records the failure in *err,
// stops, waits (bounded) for MMAs in flight, frees its tensor memory and
// returns.
//
// Operand layout: K-major, no swizzle, canonical core matrices of 8 rows x 16
// bytes (8 bfloat16 along K); the next core matrix along K lies 128 bytes
// away, the next 8-row group (Kp / 8) * 128 bytes away.  B operands hold W^T
// ([N][K]).
#include <cuda_bf16.h>

#include <cstdint>

#include "ggem.h"
#include "ggem_host.cuh"

namespace {

constexpr int H = 128, NF = 12, K1 = 16, N4 = 16;
constexpr int OW1 = 0, OB1 = OW1 + NF * H, OW2 = OB1 + H, OB2 = OW2 + H * H;
constexpr int OW3 = OB2 + H, OB3 = OW3 + H * H, OW4 = OB3 + H, OB4 = OW4 + H * 3;
// prepared image (bfloat16 elements): B1 [128][16], B2, B3 [128][128], B4 [16][128]
constexpr int IB1 = 0, IB2 = IB1 + H * K1, IB3 = IB2 + H * H, IB4 = IB3 + H * H;
constexpr int IMG = IB4 + N4 * H;                 // 36,864 bfloat16 = 73,728 bytes
constexpr int TPB = 128;
constexpr long kWaitLimit = 1L << 24;

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ int canon(int r, int k, int Kp) {
    return ((r >> 3) * (Kp >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint64_t mdesc(uint32_t a, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    for (long it = 0; it < kWaitLimit && !done; ++it)
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity));
    return done != 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

// Writes one row's 128 relu'd, bfloat16-rounded activations (acc + bias) into
// the next layer's A operand (canonical, Kp = 128), 32 columns at a time.
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem_row, const float* bias,
                                                __nv_bfloat16* A, int row) {
#pragma unroll 1
    for (int c0 = 0; c0 < H; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem_row + (uint32_t)c0, r);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = c0 + 8 * g + 2 * q;
                const float a = fmaxf(__uint_as_float(r[8 * g + 2 * q]) + bias[j], 0.f);
                const float b = fmaxf(__uint_as_float(r[8 * g + 2 * q + 1]) + bias[j + 1], 0.f);
                w[q] = pack_bf16(a, b);
            }
            *reinterpret_cast<uint4*>(A + canon(row, c0 + 8 * g, H)) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// mode 0: out32[n][3] = raw network output (units of s_y)
// mode 1: out64[e] = (base ? base[e] : 0) + r[e] + s s_y y[e], s = sqrt(ssq / 3n)
__global__ void __launch_bounds__(TPB)
    k_mlp_fwd_tc(int n, int mode, const uint4* __restrict__ img, const float* __restrict__ p,
                 const float* __restrict__ stats, const float* __restrict__ feat,
                 float* __restrict__ out32, const double* __restrict__ r,
                 const double* __restrict__ ssq, const double* __restrict__ base,
                 double* __restrict__ out64, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __nv_bfloat16* W = reinterpret_cast<__nv_bfloat16*>(sm);          // weight image
    __nv_bfloat16* A = W + IMG;                                        // [128][128] activations
    __nv_bfloat16* A1 = A + H * H;                                     // [128][16] inputs
    float* bias = reinterpret_cast<float*>(A1 + H * K1);               // b1 b2 b3 [128], b4 [16]
    float* st = bias + 3 * H + N4;                                     // mu, sigma, s_y
    uint64_t* mbar = reinterpret_cast<uint64_t*>(st + 32);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5;

    for (int e = tid; e < IMG / 8; e += TPB) reinterpret_cast<uint4*>(W)[e] = img[e];
    for (int j = tid; j < H; j += TPB) {
        bias[j] = p[OB1 + j];
        bias[H + j] = p[OB2 + j];
        bias[2 * H + j] = p[OB3 + j];
    }
    if (tid < N4) bias[3 * H + tid] = tid < 3 ? p[OB4 + tid] : 0.f;
    if (tid < 2 * NF + 1) st[tid] = stats[tid];
    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tslot)),
                     "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);      // this warp's 32 lanes
    // D f32, A and B bf16 (both K-major), M = 128, N = 128 or 16
    const uint32_t id128 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    const uint32_t id16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N4 >> 3) << 17) |
                          ((uint32_t)(128 >> 4) << 24);
    const double s = mode == 1 ? sqrt(*ssq / (3.0 * n)) : 0.0;
    const long ntiles = (n + 127) / 128;
    uint32_t parity = 0;
    bool fail = false;

    // issue one layer's MMAs (K = kp) from thread 0 and wait for them
    auto layer = [&](uint32_t a_addr, int kp, uint32_t b_addr, uint32_t idesc) -> bool {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t sbo = (uint32_t)(kp / 8) * 128;
            for (int ks = 0; ks < kp / 16; ++ks) {
                const uint32_t o = (uint32_t)ks * 256;
                mma_bf16(tmem, mdesc(a_addr + o, 128, sbo), mdesc(b_addr + o, 128, sbo), idesc,
                         ks > 0);
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    saddr(mbar)));
        }
        const bool ok = wait_phase(saddr(mbar), parity);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                s_fail = 1;
                atomicOr(err, 1);
            }
            return false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return true;
    };

    for (long tile = blockIdx.x; tile < ntiles && !fail; tile += gridDim.x) {
        const long row0 = tile * 128;
        const long g = row0 + tid;
        // inputs: standardised, rounded to bfloat16, padded to 16 with zeros
        {
            float v[K1];
#pragma unroll
            for (int k = 0; k < K1; ++k) v[k] = 0.f;
            if (g < n) {
                const float4* f = reinterpret_cast<const float4*>(feat + g * NF);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float4 x = f[q];
                    v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
                }
#pragma unroll
                for (int k = 0; k < NF; ++k) v[k] = (v[k] - st[k]) / st[NF + k];
            }
#pragma unroll
            for (int h8 = 0; h8 < 2; ++h8)
                *reinterpret_cast<uint4*>(A1 + canon(tid, 8 * h8, K1)) =
                    make_uint4(pack_bf16(v[8 * h8], v[8 * h8 + 1]),
                               pack_bf16(v[8 * h8 + 2], v[8 * h8 + 3]),
                               pack_bf16(v[8 * h8 + 4], v[8 * h8 + 5]),
                               pack_bf16(v[8 * h8 + 6], v[8 * h8 + 7]));
        }
        if (!layer(saddr(A1), K1, saddr(W + IB1), id128)) { fail = true; break; }
        hidden_epilogue(trow, bias, A, tid);
        if (!layer(saddr(A), H, saddr(W + IB2), id128)) { fail = true; break; }
        hidden_epilogue(trow, bias + H, A, tid);
        if (!layer(saddr(A), H, saddr(W + IB3), id128)) { fail = true; break; }
        hidden_epilogue(trow, bias + 2 * H, A, tid);
        if (!layer(saddr(A), H, saddr(W + IB4), id16)) { fail = true; break; }
        {
            uint32_t o[16];
            tmem_ld16(trow, o);
            if (g < n) {
                const float y0 = __uint_as_float(o[0]) + bias[3 * H];
                const float y1 = __uint_as_float(o[1]) + bias[3 * H + 1];
                const float y2 = __uint_as_float(o[2]) + bias[3 * H + 2];
                if (mode == 0) {
                    out32[3 * g] = y0;
                    out32[3 * g + 1] = y1;
                    out32[3 * g + 2] = y2;
                } else {
                    const double f = s * (double)st[2 * NF];
                    const double y[3] = {y0, y1, y2};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const long e = 3 * g + c;
                        out64[e] = (base ? base[e] : 0.0) + r[e] + f * y[c];
                    }
                }
            }
        }
        // the next tile's first MMA overwrites the accumulator the loads above read
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (s_fail && tid == 0) wait_phase(saddr(mbar), parity ^ 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(128));
}

// The weight image of the tensor-core forward from the FP32 masters:
// B1 = W1^T [128][16], B2 = W2^T, B3 = W3^T [128][128], B4 = W4^T [16][128],
// bfloat16 (round to nearest even), zero padded, canonical K-major layout.
__global__ void k_mlp_tc_prep(const float* __restrict__ p, __nv_bfloat16* __restrict__ img) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= IMG) return;
    float v = 0.f;
    int o;
    if (e < IB2) {                                // B1: n = hidden unit j, k = feature
        const int j = e / K1, k = e - j * K1;
        if (k < NF) v = p[OW1 + k * H + j];
        o = IB1 + canon(j, k, K1);
    } else if (e < IB4) {                         // B2, B3: n = unit j, k = input unit
        const int l = e < IB3 ? 0 : 1, q = e - (l ? IB3 : IB2);
        const int j = q / H, k = q - j * H;
        v = p[(l ? OW3 : OW2) + k * H + j];
        o = (l ? IB3 : IB2) + canon(j, k, H);
    } else {                                      // B4: n = output c, k = hidden unit
        const int q = e - IB4, c = q / H, k = q - c * H;
        if (c < 3) v = p[OW4 + k * 3 + c];
        o = IB4 + canon(c, k, H);
    }
    img[o] = __float2bfloat16_rn(v);
}

constexpr size_t kSmem = (size_t)IMG * 2 + (size_t)H * H * 2 + (size_t)H * K1 * 2 +
                         (3 * H + N4 + 32) * 4 + 16;

}  // namespace

namespace ggem {

size_t mlp_tc_image_elems() { return IMG; }

cudaError_t mlp_tc_prepare(const float* p, void* img, cudaStream_t st) {
    k_mlp_tc_prep<<<(IMG + 255) / 256, 256, 0, st>>>(p, static_cast<__nv_bfloat16*>(img));
    return cudaGetLastError();
}

// BF16 forward on the tensor cores (see the top of this file); feat [n][12]
// must be 16-byte aligned, img 16-byte aligned.
cudaError_t mlp_tc_forward(int n, int mode, const void* img, const float* p, const float* stats,
                           const float* feat, float* out32, const double* r, const double* ssq,
                           const double* base, double* out64, int* err, int nsm,
                           cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = grant_max_smem((const void*)k_mlp_fwd_tc);
    if (e != cudaSuccess) return e;
    const long ntiles = (n + 127) / 128;
    const long grid = ntiles < 2L * nsm ? ntiles : 2L * nsm;
    k_mlp_fwd_tc<<<(unsigned)grid, TPB, kSmem, st>>>(n, mode, static_cast<const uint4*>(img), p,
                                                      stats, feat, out32, r, ssq, base, out64,
                                                      err);
    return cudaGetLastError();
}

}  // namespace ggem

// ===================================================================== training
// BF16 training on the tensor cores: every product of the forward and backward
// passes of one minibatch is a tile GEMM
//     C[m][n] = sum_k A[m][k] B[n][k]        (A [M][K], B [N][K], bfloat16, row-major)
// with FP32 accumulation in tensor memory and an epilogue per role:
//   ACT    hidden layer: relu(C + bias), rounded to bfloat16, stored row-major
//          and transposed (the transposed copy is the A operand of the layer's
//          weight gradient);
//   OUT    output layer: C + bias (first nreal columns), FP32;
//   DELTA  backpropagated delta: C where the layer's activation is positive,
//          split into bfloat16 hi + lo (so the products keep ~16 more bits),
//          stored row-major and transposed, and its column sums (bias
//          gradient) added to the gradient;
//   GRAD   weight gradient: C added to the gradient (atomics, split over K).
// Deltas enter the products as hi + lo (two MMAs per step); activations and
// weights are bfloat16 by the network's definition, so the gradients match
// backpropagation with unrounded deltas to about 2^-16 of each term.
// A CTA (4 warps, 128 threads = 128 TMEM lanes) computes one 128-row tile of C
// over a range of K, staging K in chunks of 64 (canonical K-major layout, as
// above) and waiting on each chunk's MMAs (bounded wait).
namespace {

enum { EP_ACT = 0, EP_OUT = 1, EP_DELTA = 2, EP_GRAD = 3 };
constexpr int KC = 64;                      // K per staged chunk

struct TcGemm {
    int M, N, K;                            // N a multiple of 16 (<= 128), K of 16
    const __nv_bfloat16 *A, *Alo;           // A [M][lda] (Alo may be null)
    int lda;
    const __nv_bfloat16 *B, *Blo;           // B [N][ldb]
    int ldb;
    int kspan;                              // K per CTA (grid.y splits K)
    int mode, nreal;                        // epilogue; columns that exist
    const float* bias;                      // ACT, OUT: [N]
    const __nv_bfloat16* mask;              // DELTA: activation [M][ldmask]
    int ldmask;
    __nv_bfloat16 *out, *out_lo;            // ACT, DELTA: row-major [M][ldo]
    int ldo;
    __nv_bfloat16 *outT, *outT_lo;          // ACT, DELTA: transposed [N][ldt]
    int ldt;
    float* out32;                           // OUT: [M][ld32]; GRAD: gradient base
    int ld32;
    int gtrans;                             // GRAD: element (m, n) at n * ld32 + m
    float* bgrad;                           // DELTA: bias gradient [N] (atomics)
    int* err;
};

__device__ __forceinline__ void stage_rows(const __nv_bfloat16* src, int ld, int rows, int nrow,
                                           int k0, int kend, __nv_bfloat16* dst, int tid) {
    // rows x KC chunk of a row-major operand into the canonical layout (Kp = KC),
    // zero outside [0, nrow) x [k0, kend); 16-byte pieces, consecutive threads
    // on consecutive pieces of one row
    for (int e = tid; e < rows * (KC / 8); e += TPB) {
        const int r = e / (KC / 8), kg = e - r * (KC / 8);
        const int k = k0 + 8 * kg;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (r < nrow && k < kend) v = *reinterpret_cast<const uint4*>(src + (size_t)r * ld + k);
        *reinterpret_cast<uint4*>(dst + canon(r, 8 * kg, KC)) = v;
    }
}

__global__ void __launch_bounds__(TPB) k_gemm_tc(TcGemm g) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(sm);     // [128][KC]
    __nv_bfloat16* sAl = sA + 128 * KC;
    __nv_bfloat16* sB = sAl + 128 * KC;                           // [128][KC]
    __nv_bfloat16* sBl = sB + 128 * KC;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sBl + 128 * KC);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128;
    const int k_beg = blockIdx.y * g.kspan, k_end = min(g.K, k_beg + g.kspan);
    const uint32_t tcols = g.N <= 32 ? 32 : (g.N <= 64 ? 64 : 128);
    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tslot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(g.N >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    const uint32_t sbo = (uint32_t)(KC / 8) * 128;
    const int mrows = min(128, g.M - m0);
    uint32_t parity = 0;
    bool first = true, fail = false;
    for (int k0 = k_beg; k0 < k_end; k0 += KC) {
        stage_rows(g.A + (size_t)m0 * g.lda, g.lda, 128, mrows, k0, k_end, sA, tid);
        if (g.Alo) stage_rows(g.Alo + (size_t)m0 * g.lda, g.lda, 128, mrows, k0, k_end, sAl, tid);
        stage_rows(g.B, g.ldb, g.N, g.N, k0, k_end, sB, tid);
        if (g.Blo) stage_rows(g.Blo, g.ldb, g.N, g.N, k0, k_end, sBl, tid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const int nks = (min(KC, k_end - k0) + 15) / 16;
            for (int ks = 0; ks < nks; ++ks) {
                const uint32_t o = (uint32_t)ks * 256;
                const uint64_t da = mdesc(saddr(sA) + o, 128, sbo), db = mdesc(saddr(sB) + o, 128, sbo);
                mma_bf16(tmem, da, db, idesc, first ? 0u : 1u);
                first = false;
                if (g.Blo) mma_bf16(tmem, da, mdesc(saddr(sBl) + o, 128, sbo), idesc, 1u);
                if (g.Alo) mma_bf16(tmem, mdesc(saddr(sAl) + o, 128, sbo), db, idesc, 1u);
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    saddr(mbar)));
        }
        first = false;
        const bool ok = wait_phase(saddr(mbar), parity);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                s_fail = 1;
                atomicOr(g.err, 1);
            }
            fail = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!fail && k_beg < k_end) {
        const int m = m0 + tid;                            // this thread's row
        const bool live = tid < mrows;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < g.N; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(trow + (uint32_t)c0, r);
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
            if (g.mode == EP_ACT) {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + g.bias[c0 + j], 0.f);
                if (live) {
                    uint32_t w[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) w[q] = pack_bf16(v[2 * q], v[2 * q + 1]);
                    uint4* o = reinterpret_cast<uint4*>(g.out + (size_t)m * g.ldo + c0);
                    o[0] = make_uint4(w[0], w[1], w[2], w[3]);
                    o[1] = make_uint4(w[4], w[5], w[6], w[7]);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        g.outT[(size_t)(c0 + j) * g.ldt + m] = __float2bfloat16_rn(v[j]);
                }
            } else if (g.mode == EP_OUT) {
                if (live)
                    for (int j = 0; j < 16; ++j)
                        if (c0 + j < g.nreal) g.out32[(size_t)m * g.ld32 + c0 + j] = v[j] + g.bias[c0 + j];
            } else if (g.mode == EP_DELTA) {
                float col[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const bool on = live && __bfloat162float(g.mask[(size_t)m * g.ldmask + c0 + j]) > 0.f;
                    v[j] = on ? v[j] : 0.f;
                    col[j] = v[j];
                }
                if (live) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const __nv_bfloat16 h = __float2bfloat16_rn(v[j]);
                        const __nv_bfloat16 l = __float2bfloat16_rn(v[j] - __bfloat162float(h));
                        if (g.out) {
                            g.out[(size_t)m * g.ldo + c0 + j] = h;
                            g.out_lo[(size_t)m * g.ldo + c0 + j] = l;
                        }
                        g.outT[(size_t)(c0 + j) * g.ldt + m] = h;
                        g.outT_lo[(size_t)(c0 + j) * g.ldt + m] = l;
                    }
                }
                // bias gradient: column sums over the tile's rows
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float t = col[j];
                    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                    if (lane == 0 && c0 + j < g.nreal) atomicAdd(g.bgrad + c0 + j, t);
                }
            } else {                                       // EP_GRAD
                if (live)
                    for (int j = 0; j < 16; ++j)
                        if (c0 + j < g.nreal) {
                            const size_t e = g.gtrans ? (size_t)(c0 + j) * g.ld32 + m
                                                      : (size_t)m * g.ld32 + c0 + j;
                            atomicAdd(g.out32 + e, v[j]);
                        }
            }
        }
    }
    if (s_fail && tid == 0) wait_phase(saddr(mbar), parity ^ 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(tcols));
}

constexpr size_t kGemmSmem = (size_t)4 * 128 * KC * 2 + 16;

// inputs of one minibatch: X0 [nbp][16] = standardised features (bfloat16,
// zero past 12 and past nb), its transpose X0T [16][nbp]; targets / s_y into
// T [nbp][3] (zero past nb)
__global__ void k_train_inputs(int nb, int nbp, const int* __restrict__ idx,
                               const float* __restrict__ feat, const float* __restrict__ target,
                               const float* __restrict__ stats, __nv_bfloat16* __restrict__ X0,
                               __nv_bfloat16* __restrict__ X0T, float* __restrict__ T) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nbp) return;
    const bool live = r < nb;
    const int row = live ? idx[r] : 0;
    for (int k = 0; k < K1; ++k) {
        float v = 0.f;
        if (live && k < NF) v = (feat[(size_t)row * NF + k] - stats[k]) / stats[NF + k];
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        X0[(size_t)r * K1 + k] = b;
        X0T[(size_t)k * nbp + r] = b;
    }
    const float isy = 1.f / stats[2 * NF];
    for (int c = 0; c < 3; ++c) T[(size_t)r * 3 + c] = live ? target[(size_t)row * 3 + c] * isy : 0.f;
}

// output delta d4 = 2 (y - t) / (3 nb) (rows < nb), split hi + lo, row-major
// [nbp][16] and transposed [16][nbp]; loss and the output bias gradient
__global__ void k_train_out_delta(int nb, int nbp, const float* __restrict__ Y,
                                  const float* __restrict__ T, __nv_bfloat16* __restrict__ D,
                                  __nv_bfloat16* __restrict__ Dl, __nv_bfloat16* __restrict__ DT,
                                  __nv_bfloat16* __restrict__ DTl, float* __restrict__ grad_b4,
                                  float* __restrict__ loss) {
    __shared__ float red[4][TPB / 32];
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float sq = 0.f, db[3] = {0.f, 0.f, 0.f};
    if (r < nbp) {
        const float scale = 2.f / (3.f * (float)nb);
        for (int c = 0; c < N4; ++c) {
            float d = 0.f;
            if (c < 3 && r < nb) {
                const float e = Y[(size_t)r * 3 + c] - T[(size_t)r * 3 + c];
                sq += e * e;
                d = scale * e;
                db[c] = d;
            }
            const __nv_bfloat16 h = __float2bfloat16_rn(d);
            const __nv_bfloat16 l = __float2bfloat16_rn(d - __bfloat162float(h));
            D[(size_t)r * N4 + c] = h;
            Dl[(size_t)r * N4 + c] = l;
            DT[(size_t)c * nbp + r] = h;
            DTl[(size_t)c * nbp + r] = l;
        }
    }
    float v[4] = {sq, db[0], db[1], db[2]};
    for (int q = 0; q < 4; ++q) {
        float t = v[q];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[q][w] = t;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        float t = 0.f;
        for (int q = 0; q < TPB / 32; ++q) t += red[threadIdx.x][q];
        if (threadIdx.x == 0) atomicAdd(loss, t / (3.f * (float)nb));
        else atomicAdd(grad_b4 + threadIdx.x - 1, t);
    }
}

// operand images of the training GEMMs from the FP32 masters (bfloat16, row-major):
// forward B operands W^T: W1T [128][16], W2T, W3T [128][128], W4T [16][128];
// backward B operands W as [fan_in][fan_out]: W4n [128][16], W3n, W2n [128][128]
constexpr int TW1T = 0, TW2T = TW1T + H * K1, TW3T = TW2T + H * H, TW4T = TW3T + H * H;
constexpr int TW4N = TW4T + N4 * H, TW3N = TW4N + H * N4, TW2N = TW3N + H * H;
constexpr int TIMG = TW2N + H * H;

__global__ void k_train_weights(const float* __restrict__ p, __nv_bfloat16* __restrict__ w) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= TIMG) return;
    float v = 0.f;
    if (e < TW2T) {                                   // W1T[j][k] = W1[k][j]
        const int j = e / K1, k = e % K1;
        if (k < NF) v = p[OW1 + k * H + j];
    } else if (e < TW4T) {                            // W2T, W3T [j][k] = W[k][j]
        const int l = e < TW3T ? 0 : 1, q = e - (l ? TW3T : TW2T), j = q / H, k = q % H;
        v = p[(l ? OW3 : OW2) + k * H + j];
    } else if (e < TW4N) {                            // W4T[c][k] = W4[k][c]
        const int q = e - TW4T, c = q / H, k = q % H;
        if (c < 3) v = p[OW4 + k * 3 + c];
    } else if (e < TW3N) {                            // W4n[k][c] = W4[k][c]
        const int q = e - TW4N, k = q / N4, c = q % N4;
        if (c < 3) v = p[OW4 + k * 3 + c];
    } else {                                          // W3n, W2n [k][j] = W[k][j]
        const int l = e < TW2N ? 0 : 1, q = e - (l ? TW2N : TW3N);
        v = p[(l ? OW2 : OW3) + q];
    }
    w[e] = __float2bfloat16_rn(v);
}

}  // namespace

namespace ggem {

// scratch of one minibatch of up to nb rows (bfloat16 elements and floats)
size_t mlp_tc_train_scratch(int nb) {
    const size_t nbp = (size_t)(nb + 127) / 128 * 128;
    const size_t bf = TIMG + 2 * nbp * K1 + 6 * nbp * H + 4 * nbp * N4 + 12 * nbp * H;
    return bf * 2 + nbp * 6 * 4 + 256;
}

// One minibatch (rows idx[0..nb)): loss added to *loss, gradients added to grad.
cudaError_t mlp_tc_train_batch(int nb, const int* idx, const float* feat, const float* target,
                               const float* p, const float* stats, float* grad, float* loss,
                               void* scratch, int* err, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    cudaError_t e = grant_max_smem((const void*)k_gemm_tc);
    if (e != cudaSuccess) return e;
    const int nbp = (nb + 127) / 128 * 128;
    __nv_bfloat16* w = static_cast<__nv_bfloat16*>(scratch);
    __nv_bfloat16* X0 = w + TIMG;
    __nv_bfloat16* X0T = X0 + (size_t)nbp * K1;
    __nv_bfloat16* Aact[3];
    __nv_bfloat16* AT[3];
    __nv_bfloat16* cur = X0T + (size_t)nbp * K1;
    for (int l = 0; l < 3; ++l) {
        Aact[l] = cur;
        AT[l] = cur + (size_t)nbp * H;
        cur += 2 * (size_t)nbp * H;
    }
    __nv_bfloat16 *D4 = cur, *D4l = D4 + (size_t)nbp * N4, *D4T = D4l + (size_t)nbp * N4,
                  *D4Tl = D4T + (size_t)nbp * N4;
    cur = D4Tl + (size_t)nbp * N4;
    __nv_bfloat16 *Dh[3], *Dl[3], *DTh[3], *DTl[3];      // deltas of hidden layers 3, 2, 1
    for (int l = 0; l < 3; ++l) {
        Dh[l] = cur;
        Dl[l] = cur + (size_t)nbp * H;
        DTh[l] = cur + 2 * (size_t)nbp * H;
        DTl[l] = cur + 3 * (size_t)nbp * H;
        cur += 4 * (size_t)nbp * H;
    }
    float* Y = reinterpret_cast<float*>(cur);
    float* T = Y + (size_t)nbp * 3;
    k_train_weights<<<(TIMG + 255) / 256, 256, 0, st>>>(p, w);
    k_train_inputs<<<nbp / TPB, TPB, 0, st>>>(nb, nbp, idx, feat, target, stats, X0, X0T, T);
    auto gemm = [&](TcGemm g, int ksplit) {
        g.err = err;
        dim3 grid((g.M + 127) / 128, ksplit);
        k_gemm_tc<<<grid, TPB, kGemmSmem, st>>>(g);
    };
    const int nt = nbp / 128;
    // forward
    const __nv_bfloat16* fin[4] = {X0, Aact[0], Aact[1], Aact[2]};
    const int fk[4] = {K1, H, H, H};
    const __nv_bfloat16* fw[4] = {w + TW1T, w + TW2T, w + TW3T, w + TW4T};
    const int fb[4] = {OB1, OB2, OB3, OB4};
    for (int l = 0; l < 4; ++l) {
        TcGemm g{};
        g.M = nbp; g.N = l < 3 ? H : N4; g.K = fk[l];
        g.A = fin[l]; g.lda = fk[l]; g.B = fw[l]; g.ldb = fk[l]; g.kspan = fk[l];
        g.bias = p + fb[l];
        if (l < 3) {
            g.mode = EP_ACT; g.nreal = H;
            g.out = Aact[l]; g.ldo = H; g.outT = AT[l]; g.ldt = nbp;
        } else {
            g.mode = EP_OUT; g.nreal = 3; g.out32 = Y; g.ld32 = 3;
        }
        gemm(g, 1);
    }
    k_train_out_delta<<<nbp / TPB, TPB, 0, st>>>(nb, nbp, Y, T, D4, D4l, D4T, D4Tl, grad + OB4,
                                                 loss);
    // layer 4: dW4 = A3^T d4 (split over the batch), delta3 = (d4 W4^T) * (a3 > 0)
    {
        TcGemm g{};
        g.M = H; g.N = N4; g.K = nbp; g.A = AT[2]; g.lda = nbp; g.B = D4T; g.Blo = D4Tl;
        g.ldb = nbp; g.kspan = 128; g.mode = EP_GRAD; g.nreal = 3; g.out32 = grad + OW4;
        g.ld32 = 3;
        gemm(g, nt);
        TcGemm d{};
        d.M = nbp; d.N = H; d.K = N4; d.A = D4; d.Alo = D4l; d.lda = N4; d.B = w + TW4N;
        d.ldb = N4; d.kspan = N4; d.mode = EP_DELTA; d.nreal = H; d.mask = Aact[2]; d.ldmask = H;
        d.out = Dh[0]; d.out_lo = Dl[0]; d.ldo = H; d.outT = DTh[0]; d.outT_lo = DTl[0];
        d.ldt = nbp; d.bgrad = grad + OB3;
        gemm(d, 1);
    }
    // layers 3, 2: dW = A_prev^T delta; delta_prev = (delta W^T) * (a_prev > 0)
    const int owl[2] = {OW3, OW2}, obp[2] = {OB2, OB1}, wn[2] = {TW3N, TW2N};
    for (int q = 0; q < 2; ++q) {
        TcGemm g{};
        g.M = H; g.N = H; g.K = nbp; g.A = AT[1 - q]; g.lda = nbp; g.B = DTh[q]; g.Blo = DTl[q];
        g.ldb = nbp; g.kspan = 128; g.mode = EP_GRAD; g.nreal = H; g.out32 = grad + owl[q];
        g.ld32 = H;
        gemm(g, nt);
        TcGemm d{};
        d.M = nbp; d.N = H; d.K = H; d.A = Dh[q]; d.Alo = Dl[q]; d.lda = H; d.B = w + wn[q];
        d.ldb = H; d.kspan = H; d.mode = EP_DELTA; d.nreal = H; d.mask = Aact[1 - q];
        d.ldmask = H; d.out = q == 0 ? Dh[1] : nullptr; d.out_lo = q == 0 ? Dl[1] : nullptr;
        d.ldo = H; d.outT = DTh[q + 1]; d.outT_lo = DTl[q + 1]; d.ldt = nbp;
        d.bgrad = grad + obp[q];
        gemm(d, 1);
    }
    // layer 1: dW1^T = delta1^T X0 (element (j, k) of dW1^T is W1's (k, j))
    {
        TcGemm g{};
        g.M = H; g.N = K1; g.K = nbp; g.A = DTh[2]; g.Alo = DTl[2]; g.lda = nbp; g.B = X0T;
        g.ldb = nbp; g.kspan = 128; g.mode = EP_GRAD; g.nreal = NF; g.out32 = grad + OW1;
        g.ld32 = H; g.gtrans = 1;
        gemm(g, nt);
    }
    return cudaGetLastError();
}

}  // namespace ggem
