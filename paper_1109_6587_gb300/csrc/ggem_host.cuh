// Host-side helpers shared by the plan and solver translation units: error
// propagation (a failed check throws Fail, converted to a ggem_status at the
// C-ABI boundary by guarded()), device allocation, host/device staging of
// user arrays, and per-stage tracing with CUDA events.
#pragma once

#include <new>
#include <string>

#include "ggem_internal.cuh"

namespace ggem {

constexpr double kPi = 3.14159265358979323846;

struct Fail {
    ggem_status s;
};

#define GG_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            P->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            throw Fail{GGEM_ERR_CUDA};                                                    \
        }                                                                                 \
    } while (0)

#define GG_CHECK(cond, code, msg)                                                         \
    do {                                                                                  \
        if (!(cond)) {                                                                    \
            P->err = (msg);                                                               \
            throw Fail{code};                                                             \
        }                                                                                 \
    } while (0)

template <typename F>
inline ggem_status guarded(ggem_plan_t* P, F&& f) {
    try {
        f();
        return GGEM_OK;
    } catch (const Fail& e) {
        return e.s;
    } catch (const std::bad_alloc&) {
        if (P) P->err = "host allocation failed";
        return GGEM_ERR_CAPACITY;
    } catch (...) {
        if (P) P->err = "unexpected host exception";
        return GGEM_ERR_CUDA;
    }
}

inline bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename X>
void dalloc(ggem_plan_t* P, X** p, size_t n) {
    GG_CUDA(cudaMalloc((void**)p, n * sizeof(X) + 16));
}

inline void dfree(void* p) {
    if (p) cudaFree(p);
}

// Input staging: device pointers pass through; host pointers are copied into
// the plan buffer `stage` (n doubles).
inline const double* stage_in(ggem_plan_t* P, const double* p, double* stage, size_t n) {
    if (!p) return nullptr;
    if (is_device_ptr(p)) return p;
    GG_CUDA(cudaMemcpyAsync(stage, p, n * sizeof(double), cudaMemcpyHostToDevice, P->st));
    return stage;
}

struct OutMap {
    double* user = nullptr;
    double* dev = nullptr;
    size_t n = 0;
    bool host = false;
};

inline OutMap stage_out(double* user, double* stage, size_t n) {
    OutMap m;
    m.user = user;
    m.n = n;
    if (!user) return m;
    m.host = !is_device_ptr(user);
    m.dev = m.host ? stage : user;
    return m;
}

inline void finish_out(ggem_plan_t* P, const OutMap& m) {
    if (m.user && m.host)
        GG_CUDA(cudaMemcpyAsync(m.user, m.dev, m.n * sizeof(double), cudaMemcpyDeviceToHost,
                                P->st));
}

// ------------------------------------------------------------- tracing
enum Stage {
    ST_CELLS, ST_GATHER, ST_LOCAL, ST_WALL, ST_SPREAD, ST_FFT_FWD, ST_CHEB_FWD, ST_KS,
    ST_CHEB_INV, ST_FFT_INV, ST_INTERP, ST_ELEM, ST_KRYLOV, ST_PRECOND, ST_COUNT
};
inline const char* const kStageNames[ST_COUNT] = {
    "cell_list",   "gather",      "local_sum",    "wall_local_sum", "spread",
    "fft_forward", "cheb_forward", "tau_solve",   "cheb_inverse",   "fft_inverse",
    "interpolate", "element_correction", "krylov_vectors", "block_preconditioner"};

// Run one stage (nk kernel launches); with tracing on, time it with events.
template <typename F>
void stage(ggem_plan_t* P, int id, int nk, F&& f) {
    if (P->prof) GG_CUDA(cudaEventRecord(P->ev0, P->st));
    f();
    P->launches += nk;
    if (P->prof) {
        GG_CUDA(cudaEventRecord(P->ev1, P->st));
        GG_CUDA(cudaEventSynchronize(P->ev1));
        float ms = 0.f;
        GG_CUDA(cudaEventElapsedTime(&ms, P->ev0, P->ev1));
        P->prof_ms[id] += ms;
        P->prof_calls[id] += 1;
    }
}

// w = S q (single layer) and v = D q (double layer) at the mesh nodes with the
// plan's precision and quadrature (device arrays [n_nodes][3]); defined with
// the layer pipeline
void single_layer_dev(ggem_plan_t* P, const double* q, double* w);
void double_layer_dev(ggem_plan_t* P, const double* q, double* v);

// node lists of the particles of ggem_mesh_particles (d_pstart / d_pnodes,
// CSR, nodes ascending), built on first use after the ids change; also sizes
// the per-particle arrays d_rc / d_rscale
void particle_node_lists(ggem_plan_t* P);

// per-particle block preconditioner (ggem_precond.cu): rotations and node
// lists for the current mesh; out = M in; release of its arrays
void precond_prepare(ggem_plan_t* P);
void precond_apply(ggem_plan_t* P, const double* in, double* out);
void precond_free(ggem_plan_t* P);

// tensor-core forward of the learned warm start's network (ggem_mlp_tc.cu):
// weight image size (bfloat16 elements), its preparation from the FP32
// masters, and the forward (mode 0: raw outputs into out32 [n][3]; mode 1:
// out64 = base + r + s s_y y)
size_t mlp_tc_image_elems();
cudaError_t mlp_tc_prepare(const float* p, void* img, cudaStream_t st);
cudaError_t mlp_tc_forward(int n, int mode, const void* img, const float* p, const float* stats,
                           const float* feat, float* out32, const double* r, const double* ssq,
                           const double* base, double* out64, int* err, int nsm,
                           cudaStream_t st);
// tensor-core training of one minibatch (ggem_mlp_tc.cu): scratch bytes for
// minibatches of up to nb rows, and the minibatch (loss added to *loss,
// gradient added to grad)
size_t mlp_tc_train_scratch(int nb);
cudaError_t mlp_tc_train_batch(int nb, const int* idx, const float* feat, const float* target,
                               const float* p, const float* stats, float* grad, float* loss,
                               void* scratch, int* err, cudaStream_t st);

// out = base + A^-1 r estimated by the learned warm start (device arrays;
// base may be NULL); defined with the network kernels
void mlp_guess_dev(ggem_plan_t* P, const double* kappa, const double* r, const double* base,
                   double* out);

}  // namespace ggem
