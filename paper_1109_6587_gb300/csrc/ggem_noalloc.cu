// Allocation-free local velocity sum.
//
// Some callers cannot call cudaMalloc: code that records its work into a CUDA
// graph while stream capture is active (allocation calls are not allowed in
// a capture), applications whose device memory is owned entirely by another
// allocator or a fixed budget, and loops that must not pay the device-wide
// synchronisation cudaFree implies.  They also cannot create a ggem plan,
// which allocates its workspaces.  ggem_local_velocity_noalloc serves them: it
// runs the same cell-list and local-sum kernels as ggem_local_sum, but the
// cell list lives in the fixed array below, which is part of the library's
// device image (every GPU that loads the library holds it until the process
// exits).
//
// The array's name in host code is only a host-side stand-in for the device
// symbol; its device address is obtained with cudaGetSymbolAddress once per
// device and CUDA context: the first call on a device does this, and so does
// the first call after that device's context was destroyed and created anew
// (cudaDeviceReset), whose module image may sit at another address.  Make
// that first call before any stream capture.  All calls share the array, so
// calls that overlap on the GPU race with one another.
#include <cuda.h>

#include <mutex>

#include "ggem_internal.cuh"

namespace {

constexpr int kMaxPoints = GGEM_NOALLOC_MAX_POINTS;
constexpr int kMaxCells = GGEM_NOALLOC_MAX_CELLS;

constexpr size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kOffCount = 0;
constexpr size_t kOffStart = al256(kOffCount + sizeof(int) * kMaxCells);
constexpr size_t kOffCursor = al256(kOffStart + sizeof(int) * (kMaxCells + 1));
constexpr size_t kOffCell = al256(kOffCursor + sizeof(int) * (kMaxCells + kMaxPoints));
constexpr size_t kOffPerm = al256(kOffCell + sizeof(int) * kMaxPoints);
constexpr size_t kOffPos = al256(kOffPerm + sizeof(int) * kMaxPoints);
constexpr size_t kOffG = al256(kOffPos + sizeof(double4_32a) * kMaxPoints);
constexpr size_t kOffTCell = al256(kOffG + sizeof(double4_32a) * kMaxPoints);
constexpr size_t kOffTPos = al256(kOffTCell + sizeof(int) * kMaxPoints);
constexpr size_t kBytes = al256(kOffTPos + sizeof(double4_32a) * kMaxPoints);

}  // namespace

// The scratch array (about 7.8 MB with the limits in ggem.h).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kBytes];

namespace {

std::mutex g_mu;
void* g_addr[128] = {nullptr};
unsigned long long g_ctx[128] = {0};   // context id the cached address belongs to

using CtxGetCurrent = CUresult (*)(CUcontext*);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// Process-unique id of the current CUDA context (0 when it cannot be read:
// then the address is looked up afresh on every call).
unsigned long long current_context_id() {
    static CtxGetCurrent get_current = nullptr;
    static CtxGetId get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetId)f;
        cudaGetLastError();
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array on the current device, looked up once
// per device and context.
cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
        g_ctx[dev] = ctx;
    }
    *out = (unsigned char*)g_addr[dev];
    return cudaSuccess;
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" ggem_status ggem_local_velocity_noalloc(const ggem_params* prm, void* stream,
                                                   int n_src, const double* x_src,
                                                   const double* g, int n_tgt,
                                                   const double* x_tgt, int tgt_is_src,
                                                   double* u) {
    using namespace ggem;
    if (!prm || !u) return GGEM_ERR_INVALID_ARG;
    if (!(prm->Lx > 0 && prm->Lz > 0 && prm->W > 0 && prm->mu > 0)) return GGEM_ERR_INVALID_ARG;
    if (prm->Nx <= 0 || prm->Nz <= 0 || prm->Ny < 2) return GGEM_ERR_INVALID_ARG;
    if (n_src < 0 || n_tgt < 0) return GGEM_ERR_INVALID_ARG;
    if (n_src > kMaxPoints) return GGEM_ERR_CAPACITY;
    if (tgt_is_src) n_tgt = n_src;
    if (n_src > 0 && !(x_src && g)) return GGEM_ERR_INVALID_ARG;
    if (!tgt_is_src && n_tgt > 0 && !x_tgt) return GGEM_ERR_INVALID_ARG;
    if (n_tgt == 0) return GGEM_OK;
    if (!on_device(u) || (n_src > 0 && (!on_device(x_src) || !on_device(g))) ||
        (!tgt_is_src && !on_device(x_tgt)))
        return GGEM_ERR_INVALID_ARG;

    GridGeom geo;
    geo.Lx = prm->Lx; geo.Lz = prm->Lz; geo.W = prm->W; geo.y0 = prm->y0;
    geo.Nx = prm->Nx; geo.Ny = prm->Ny; geo.Nz = prm->Nz; geo.nkx = prm->Nx / 2;
    geo.dx = prm->Lx / prm->Nx; geo.dz = prm->Lz / prm->Nz;
    geo.mu = prm->mu;
    double h = fmax(fmax(geo.dx, prm->W / (prm->Ny - 1)), geo.dz);
    geo.alpha = prm->alpha > 0 ? prm->alpha : 1.0 / (2.0 * h);
    double rf = prm->rcut_factor > 0 ? prm->rcut_factor : 4.0;
    geo.rcut = rf / geo.alpha;
    if (!(geo.alpha * prm->Lx > 2 * rf && geo.alpha * prm->Lz > 2 * rf))
        return GGEM_ERR_INVALID_ARG;
    CellGrid cg;
    cg.ncx = (int)fmax(1.0, floor(prm->Lx / geo.rcut));
    cg.ncz = (int)fmax(1.0, floor(prm->Lz / geo.rcut));
    cg.ncy = (int)fmax(1.0, floor(prm->W / geo.rcut));
    cg.hx = prm->Lx / cg.ncx; cg.hz = prm->Lz / cg.ncz; cg.hy = prm->W / cg.ncy;
    cg.reach = 2;                                   // cells at least r_cut wide (>= r_cut/2)
    cg.y0 = prm->y0;
    if ((long)cg.ncx * cg.ncy * cg.ncz > kMaxCells) return GGEM_ERR_CAPACITY;

    unsigned char* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return GGEM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int* count = (int*)(base + kOffCount);
    int* start = (int*)(base + kOffStart);
    int* cursor = (int*)(base + kOffCursor);
    int* cell = (int*)(base + kOffCell);
    int* perm = (int*)(base + kOffPerm);
    double4_32a* pos = (double4_32a*)(base + kOffPos);
    double4_32a* gs = (double4_32a*)(base + kOffG);
    int* tcell = (int*)(base + kOffTCell);
    double4_32a* tpos = (double4_32a*)(base + kOffTPos);

    // build_cells clears the counters it accumulates into (cell counts and
    // cursors) before use, so stale contents from an earlier call do not leak.
    if (build_cells<double>(geo, cg, n_src, x_src, count, start, cursor, cell, perm, pos, st) !=
        cudaSuccess)
        return GGEM_ERR_CUDA;
    if (gather_strengths<double>(n_src, perm, g, nullptr, 1.0, gs, st) != cudaSuccess)
        return GGEM_ERR_CUDA;
    SortedSources<double> src{pos, gs, cell, perm, start, n_src};
    if (tgt_is_src) {
        if (local_sum<double>(geo, cg, src, TK_SORTED, n_tgt, nullptr, nullptr, nullptr, OUT_U,
                              u, 3, st) != cudaSuccess)
            return GGEM_ERR_CUDA;
        return GGEM_OK;
    }
    // free targets, located in chunks that fit the scratch array
    for (int t0 = 0; t0 < n_tgt; t0 += kMaxPoints) {
        int nt = n_tgt - t0 < kMaxPoints ? n_tgt - t0 : kMaxPoints;
        if (locate_targets<double>(geo, cg, nt, TK_POINTS, x_tgt + 3 * (size_t)t0, tcell, tpos,
                                   st) != cudaSuccess)
            return GGEM_ERR_CUDA;
        if (local_sum<double>(geo, cg, src, TK_POINTS, nt, tcell, tpos, nullptr, OUT_U,
                              u + 3 * (size_t)t0, 3, st) != cudaSuccess)
            return GGEM_ERR_CUDA;
    }
    return GGEM_OK;
}
