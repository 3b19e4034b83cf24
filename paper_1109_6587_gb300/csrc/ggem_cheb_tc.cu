// Chebyshev transforms in y on the 5th-generation tensor cores (tcgen05), for
// the mixed-precision path.  Every transform of Sec. 3.2.2 / App. C is the
// dense contraction
//     out[n][c] = sum_j M[n][j] in[j][c],   M: Ny x Ny, c = 0 .. cols-1,
// (forward DCT-I coefficients or their evaluation at the Gauss-Lobatto nodes)
// over all Fourier modes and field components at once.
//
// Split BF16x3 ("3 products of 2-term splits"): every FP32 operand x is split
// as x = hi + lo with hi = bf16(x), lo = bf16(x - hi), and
//     M in ~ M_hi in_hi + M_hi in_lo + M_lo in_hi
// accumulated in FP32 in tensor memory (the dropped M_lo in_lo and the split
// remainders are ~2^-16 of each product).
//
// Persistent CTAs over 128-column tiles, two per SM when their shared memory
// fits.  M's split is prepared once per plan (k_cheb_tc_prep) and copied into
// shared memory with 16-byte loads; each tile of `in` is split while it is
// staged, one 16-byte core-matrix row per thread and item.  Both
// operands use the K-major no-swizzle canonical layout: core matrices of 8
// rows x 16 bytes (8 bf16 along K), the next core matrix along K 128 bytes
// away, the next 8-row group along M/N (Kp/8) * 128 bytes away.  One thread
// issues the MMAs (M = 128 per row block, N = tile width, K = 16 per
// instruction) and commits them to an mbarrier; the four warps then read the
// accumulator rows (TMEM lanes) with tcgen05.ld and store them.  Every
// mbarrier wait is bounded: on expiry the kernel records the failure in *err,
// stops, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>

#include "ggem_internal.cuh"

namespace ggem {

namespace {

constexpr int TCT = 128;                 // threads per CTA (4 warps = 128 TMEM lanes)
constexpr long kWaitLimit = 1L << 24;    // mbarrier polls before giving up

// Failure injection for tests (ggem_inject_tc_wait_expiry): when > 0, the next
// launch skips issuing and committing the MMAs of every CTA's first tile and
// polls at most this many times, so that its wait expires with nothing in flight.
std::atomic<long> g_inject_polls{0};

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// element (r, k) of an R x Kp K-major operand in the canonical layout
__device__ __forceinline__ int canon(int r, int k, int Kp) {
    return ((r >> 3) * (Kp >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// shared-memory matrix descriptor: no swizzle, version 1
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

__device__ __forceinline__ void split(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(v);
    l = __float2bfloat16_rn(v - __bfloat162float(h));
}

__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity, long limit) {
    uint32_t done = 0;
    for (long it = 0; it < limit && !done; ++it)
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

__global__ void __launch_bounds__(TCT)
    k_cheb_tc(int Ny, int Kp, int MB, int NT, uint32_t tcols, const uint4* __restrict__ Mprep,
              const float* __restrict__ in, float* __restrict__ out, long cols, long ntiles,
              int* __restrict__ err, long wait_limit, int skip_first) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __nv_bfloat16* Ah = reinterpret_cast<__nv_bfloat16*>(sm);
    __nv_bfloat16* Al = Ah + (size_t)MB * 128 * Kp;
    __nv_bfloat16* Bh = Al + (size_t)MB * 128 * Kp;
    __nv_bfloat16* Bl = Bh + (size_t)NT * Kp;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(Bl + (size_t)NT * Kp);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // M split (hi then lo, canonical layout), prepared once per plan
    {
        uint4* dst = reinterpret_cast<uint4*>(Ah);
        const int n16 = 2 * MB * 128 * Kp / 8;
        for (int e = tid; e < n16; e += TCT) dst[e] = Mprep[e];
    }
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
    // D f32, A and B bf16, both K-major, N = NT, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    const uint32_t kstep = 2 * 128;                    // 16 bf16 along K = 2 core matrices
    const uint32_t sbo = (uint32_t)(Kp / 8) * 128;
    uint32_t parity = 0;
    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long c0 = tile * NT;
        // one core-matrix row per item: column n, rows 8 kg .. 8 kg + 7 (zero past Ny),
        // consecutive threads on consecutive columns (coalesced loads), one
        // 16-byte store each for hi and lo
        for (int e = tid; e < NT * (Kp / 8); e += TCT) {
            const int kg = e / NT, n = e - kg * NT;
            const long c = c0 + n;
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                const int k = kg * 8 + j;
                const float v0 = (k < Ny && c < cols) ? in[(long)k * cols + c] : 0.f;
                const float v1 = (k + 1 < Ny && c < cols) ? in[(long)(k + 1) * cols + c] : 0.f;
                __nv_bfloat16 h0, l0, h1, l1;
                split(v0, h0, l0);
                split(v1, h1, l1);
                hw[j / 2] = (uint32_t)__bfloat16_as_ushort(h0) |
                            ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                lw[j / 2] = (uint32_t)__bfloat16_as_ushort(l0) |
                            ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
            const int o = canon(n, kg * 8, Kp);
            *reinterpret_cast<uint4*>(Bh + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(Bl + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0 && !(skip_first && tile == blockIdx.x)) {
            const uint32_t bh = saddr(Bh), bl = saddr(Bl);
            for (int mb = 0; mb < MB; ++mb) {
                const uint32_t ah = saddr(Ah + (size_t)mb * 128 * Kp),
                               al = saddr(Al + (size_t)mb * 128 * Kp);
                const uint32_t d = tmem + (uint32_t)(mb * NT);
                for (int ks = 0; ks < Kp / 16; ++ks) {
                    const uint32_t o = ks * kstep;
                    mma_bf16(d, mdesc(ah + o, 128, sbo), mdesc(bh + o, 128, sbo), idesc,
                             ks > 0);
                    mma_bf16(d, mdesc(ah + o, 128, sbo), mdesc(bl + o, 128, sbo), idesc, 1);
                    mma_bf16(d, mdesc(al + o, 128, sbo), mdesc(bh + o, 128, sbo), idesc, 1);
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    saddr(mbar)));
        }
        const bool ok = wait_phase(saddr(mbar), parity, wait_limit);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                s_fail = 1;
                atomicOr(err, 1);
            }
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int mb = 0; mb < MB; ++mb) {
            const int row = mb * 128 + warp * 32 + lane;
            for (int cc = 0; cc < NT; cc += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mb * NT + cc), r);
                if (row < Ny) {
                    float* o = out + (long)row * cols + c0 + cc;
                    if (c0 + cc + 32 <= cols) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *reinterpret_cast<float4*>(o + j) =
                                make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                            __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                    } else {
                        for (int j = 0; j < 32; ++j)
                            if (c0 + cc + j < cols) o[j] = __uint_as_float(r[j]);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    // on a failed wait the MMAs may still be running: give them one more
    // bounded wait before the tensor memory is released
    if (s_fail && tid == 0) wait_phase(saddr(mbar), parity ^ 1u, wait_limit);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(tcols));
}

// M split into hi and lo, zero padded to MB*128 rows and Kp columns, in the
// canonical layout (hi block then lo block)
__global__ void k_cheb_tc_prep(int Ny, int Kp, int MB, const float* __restrict__ Mx,
                               __nv_bfloat16* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= MB * 128 * Kp) return;
    const int r = e / Kp, k = e - r * Kp;
    const float v = (r < Ny && k < Ny) ? Mx[r * Ny + k] : 0.f;
    __nv_bfloat16 h, l;
    split(v, h, l);
    const int o = (r >> 7) * 128 * Kp + canon(r & 127, k, Kp);
    out[o] = h;
    out[(size_t)MB * 128 * Kp + o] = l;
}

}  // namespace

size_t cheb_tc_prep_bytes(int Ny) {
    const int Kp = (Ny + 15) / 16 * 16, MB = (Ny + 127) / 128;
    return (size_t)2 * MB * 128 * Kp * 2;
}

cudaError_t cheb_tc_prepare(int Ny, const float* M, void* prep, cudaStream_t st) {
    const int Kp = (Ny + 15) / 16 * 16, MB = (Ny + 127) / 128;
    const int n = MB * 128 * Kp;
    k_cheb_tc_prep<<<(n + 255) / 256, 256, 0, st>>>(Ny, Kp, MB, M,
                                                    static_cast<__nv_bfloat16*>(prep));
    return cudaGetLastError();
}

// Shared memory of the tensor-core transform for Ny rows and tile width NT.
static size_t cheb_tc_smem(int Ny, int NT) {
    const int Kp = (Ny + 15) / 16 * 16, MB = (Ny + 127) / 128;
    return (size_t)2 * MB * 128 * Kp * 2 + (size_t)2 * NT * Kp * 2 + 16;
}

// out = M in on the tensor cores when the operands fit in shared memory;
// returns cudaErrorNotSupported otherwise (the caller uses the FP32 kernel).
// Requires cols % 4 == 0 and 16-byte aligned rows for the vector stores.
cudaError_t cheb_apply_tc(int Ny, const void* prep, const float* in, float* out, long cols,
                          int* err, int nsm, cudaStream_t st) {
    if (Ny < 1 || cols <= 0) return cudaSuccess;
    if (!prep || cols % 4 != 0 || ((uintptr_t)out & 15) != 0 || ((uintptr_t)prep & 15) != 0)
        return cudaErrorNotSupported;
    const int Kp = (Ny + 15) / 16 * 16, MB = (Ny + 127) / 128;
    int NT = 128;
    size_t smem = cheb_tc_smem(Ny, NT);
    if (smem > 227 * 1024) {
        NT = 64;
        smem = cheb_tc_smem(Ny, NT);
    }
    if (smem > 227 * 1024 || MB > 2) return cudaErrorNotSupported;
    uint32_t tcols = 32;
    while (tcols < (uint32_t)(MB * NT)) tcols <<= 1;
    cudaError_t e = grant_max_smem((const void*)k_cheb_tc);
    if (e != cudaSuccess) return e;
    const long ntiles = (cols + NT - 1) / NT;
    // two CTAs per SM when their shared memory fits (one stages while the other
    // computes); each holds at most 256 of the SM's 512 tensor-memory columns
    const long per_sm = (2 * smem <= 227 * 1024) ? 2 : 1;
    const long grid = ntiles < per_sm * nsm ? ntiles : per_sm * nsm;
    const long inject = g_inject_polls.exchange(0);
    k_cheb_tc<<<(unsigned)grid, TCT, smem, st>>>(Ny, Kp, MB, NT, tcols,
                                                 static_cast<const uint4*>(prep), in, out, cols,
                                                 ntiles, err, inject > 0 ? inject : kWaitLimit,
                                                 inject > 0 ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace ggem

extern "C" ggem_status ggem_inject_tc_wait_expiry(long polls) {
    if (polls < 1 || polls > (1L << 24)) return GGEM_ERR_INVALID_ARG;
    ggem::g_inject_polls.store(polls);
    return GGEM_OK;
}
