// Linear systems on the mesh, solved by restarted GMRES (Saad) whose Arnoldi
// vectors live in FP64 in HBM: classical Gram-Schmidt applied twice per step
// (two multi-dot passes, each reading the basis once), deterministic two-stage
// reductions, and the small Hessenberg least-squares problem (Givens rotations)
// on the host.
//   * Fredholm solve of Sec. 5: (I + kappa/(4 pi) D) q = b at the mesh nodes,
//     D the discretised double layer (Sec. 3.5), kappa_m = (lambda_m - 1)/
//     (lambda_m + 1) per node (Eq. qa).
//   * Rigid particles of Sec. 6.1: tractions f and rigid-body velocities from
//     Eq. (sl_r) with the force and torque balance of each particle.
//
// FP64 plan: plain restarted GMRES with the FP64 operator.  Each cycle starts
// from the true residual b - A x.
// Mixed plan: iterative refinement.  The outer residual b - A64 x is formed
// with an FP64 twin plan on the same mesh (the first one of a solve with the
// mixed operator, as the first correction needs only ~1e-4); each correction
// is one GMRES cycle with the mixed operator, asked only for the accuracy that
// operator carries.
#include <algorithm>
#include <cmath>
#include <functional>
#include <vector>

#include "ggem.h"
#include "ggem_host.cuh"

using namespace ggem;

namespace {

constexpr int KB = 256;          // threads per block of the vector kernels
constexpr int KNB = 2 * 152;     // blocks of one reduction pass (2 per SM)
constexpr int KG = 8;            // basis vectors per sweep of the multi-dot
constexpr int KMAXM = 64;        // longest restart cycle
constexpr int KH = KMAXM + 2;    // stride of one coefficient array in d_sh

// out = x + s kappa v (b == nullptr), or out = b - (x + s kappa v); s = 1/(4 pi)
__global__ void k_bie_apply(int n, double s, const double* __restrict__ x,
                            const double* __restrict__ v, const double* __restrict__ kappa,
                            const double* __restrict__ b, double* __restrict__ out) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * n) return;
    double a = fma(s * kappa[e / 3], v[e], x[e]);
    out[e] = b ? b[e] - a : a;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// part[i][blk] = the block's grid-stride share of <V_i, w>, i < k
__global__ void __launch_bounds__(KB) k_mdot(size_t n, int k, const double* __restrict__ V,
                                             size_t ldv, const double* __restrict__ w,
                                             double* __restrict__ part) {
    __shared__ double red[KG][KB / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i0 = 0; i0 < k; i0 += KG) {
        const int kk = min(KG, k - i0);
        double acc[KG];
#pragma unroll
        for (int g = 0; g < KG; ++g) acc[g] = 0.0;
        for (size_t e = (size_t)blockIdx.x * KB + threadIdx.x; e < n;
             e += (size_t)gridDim.x * KB) {
            const double we = w[e];
#pragma unroll
            for (int g = 0; g < KG; ++g)
                if (g < kk) acc[g] = fma(V[(size_t)(i0 + g) * ldv + e], we, acc[g]);
        }
#pragma unroll
        for (int g = 0; g < KG; ++g) {
            double t = warp_sum(acc[g]);
            if (lane == 0) red[g][wid] = t;
        }
        __syncthreads();
        if (threadIdx.x < kk) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < KB / 32; ++q) t += red[threadIdx.x][q];
            part[(size_t)(i0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

// h[i] = sum over blocks of part[i][.], one block per i, fixed summation order
__global__ void __launch_bounds__(KB) k_mdot_final(int nb, const double* __restrict__ part,
                                                   double* __restrict__ h) {
    __shared__ double red[KB / 32];
    const int i = blockIdx.x;
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += KB) t += part[(size_t)i * nb + b];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < KB / 32; ++q) s += red[q];
        h[i] = s;
    }
}

// w += sgn * sum_{i<k} h[i] V_i
__global__ void __launch_bounds__(KB) k_mupdate(size_t n, int k, const double* __restrict__ V,
                                                size_t ldv, const double* __restrict__ h,
                                                double sgn, double* __restrict__ w) {
    __shared__ double sh[KMAXM + 2];
    for (int i = threadIdx.x; i < k; i += KB) sh[i] = sgn * h[i];
    __syncthreads();
    for (size_t e = (size_t)blockIdx.x * KB + threadIdx.x; e < n;
         e += (size_t)gridDim.x * KB) {
        double a = w[e];
        for (int i = 0; i < k; ++i) a = fma(sh[i], V[(size_t)i * ldv + e], a);
        w[e] = a;
    }
}

// w /= sqrt(*nrm2) when *nrm2 > 0
__global__ void k_scale(size_t n, const double* __restrict__ nrm2, double* __restrict__ w) {
    const double s2 = *nrm2;
    if (!(s2 > 0.0)) return;
    const double s = 1.0 / sqrt(s2);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        w[e] *= s;
}

int grid_for(size_t n) {
    return (int)std::min<size_t>(KNB, (n + KB - 1) / KB);
}

struct Solver {
    ggem_plan_t* P;      // the plan the caller owns (error messages, stream)
    ggem_plan_t* P64;    // plan whose operator gives true residuals (P or its twin)
    size_t n3, ld;       // length of the unknown vector, stride of the basis
    const double* b;
    double* x;
    double* hs;          // pinned host copy of d_sh
    bool pc = false;     // right preconditioner M (per-particle blocks): A M y = r,
    double* Zb = nullptr;  //   Zb[j] = M V_j kept for the update x += Z y (flexible form)
    // out = A in (b == nullptr) or b - A in, A applied with plan Q's layers
    std::function<void(ggem_plan_t* Q, const double* in, double* out, const double* b)> op;

    void launched(int k) { P->launches += k; }

    // h_out[0..k) = V_i . w
    void mdot(int k, const double* V, const double* w, double* h_out) {
        int g = grid_for(n3);
        k_mdot<<<g, KB, 0, P->st>>>(n3, k, V, ld, w, P->d_spart);
        k_mdot_final<<<k, KB, 0, P->st>>>(g, P->d_spart, h_out);
        GG_CUDA(cudaGetLastError());
        launched(2);
    }
    void mupdate(int k, const double* h, double sgn, double* w, const double* basis = nullptr) {
        k_mupdate<<<grid_for(n3), KB, 0, P->st>>>(n3, k, basis ? basis : P->d_V, ld, h, sgn, w);
        GG_CUDA(cudaGetLastError());
        launched(1);
    }
    // squared norm of w into *slot (device), then w /= norm
    void normalize(double* w, double* slot) {
        mdot(1, w, w, slot);
        k_scale<<<grid_for(n3), KB, 0, P->st>>>(n3, slot, w);
        GG_CUDA(cudaGetLastError());
        launched(1);
    }
    // out = A in, or b - A in when with_b
    void apply(ggem_plan_t* Q, const double* in, double* out, bool with_b) {
        op(Q, in, out, with_b ? b : nullptr);
        if (Q->fp64) P->sol_mv64++;
        else P->sol_mvmix++;
    }
    void to_host(int count) {
        GG_CUDA(cudaMemcpyAsync(hs, P->d_sh, count * sizeof(double), cudaMemcpyDeviceToHost,
                                P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));
    }

    // ||b||
    double norm_b() {
        mdot(1, b, b, P->d_sh);
        to_host(1);
        return std::sqrt(hs[0]);
    }

    // Residual r = b - A x into V_0 (A = Q's operator), its norm returned,
    // V_0 normalised.
    double residual_into_v0(ggem_plan_t* Q) {
        double* v0 = P->d_V;
        apply(Q, x, v0, true);
        normalize(v0, P->d_sh);
        to_host(1);
        return std::sqrt(hs[0]);
    }

    // One GMRES cycle on A_inner d = r, r = beta V_0 already in place, d = 0;
    // x += d at the end.  Stops when |g_{j+1}| <= stop_abs or after m steps.
    // Returns the operator applications made; *breakdown set when the Krylov
    // space became invariant (the cycle's update is then exact).
    int cycle(ggem_plan_t* Ainner, int m, double beta, double stop_abs, bool* breakdown) {
        std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
        auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
        g[0] = beta;
        double* hA = P->d_sh;
        double* hB = P->d_sh + KH;
        double* hN = P->d_sh + 2 * KH;
        int k = 0, steps = 0;
        *breakdown = false;
        for (int j = 0; j < m; ++j) {
            double* vj = P->d_V + (size_t)j * ld;
            double* w = P->d_V + (size_t)(j + 1) * ld;
            if (pc) {
                double* zj = Zb + (size_t)j * ld;
                stage(P, ST_PRECOND, 0, [&] { precond_apply(P, vj, zj); });
                apply(Ainner, zj, w, false);
            } else {
                apply(Ainner, vj, w, false);
            }
            stage(P, ST_KRYLOV, 0, [&] {
                mdot(j + 1, P->d_V, w, hA);          // classical Gram-Schmidt ...
                mupdate(j + 1, hA, -1.0, w);
                mdot(j + 1, P->d_V, w, hB);          // ... applied twice
                mupdate(j + 1, hB, -1.0, w);
                normalize(w, hN);
                to_host(3 * KH);
            });
            double an = hs[2 * KH];                      // ||A v_j||^2
            for (int i = 0; i <= j; ++i) {
                Hij(i, j) = hs[i] + hs[KH + i];
                an += Hij(i, j) * Hij(i, j);
            }
            double hn = std::sqrt(hs[2 * KH]);
            Hij(j + 1, j) = hn;
            for (int i = 0; i < j; ++i) {                // earlier rotations
                double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
                Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
                Hij(i, j) = t;
            }
            double d = std::hypot(Hij(j, j), Hij(j + 1, j));
            steps = j + 1;
            if (d == 0.0) {                              // singular on the Krylov space
                k = j;
                break;
            }
            k = j + 1;
            cs[j] = Hij(j, j) / d;
            sn[j] = Hij(j + 1, j) / d;
            Hij(j, j) = d;
            Hij(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (hn <= 1e-14 * std::sqrt(an)) {           // happy breakdown: exact in the space
                *breakdown = true;
                break;
            }
            if (std::fabs(g[j + 1]) <= stop_abs) break;
        }
        if (k == 0) return steps;
        std::vector<double> y(k);
        for (int i = k - 1; i >= 0; --i) {               // back substitution
            double t = g[i];
            for (int c = i + 1; c < k; ++c) t -= Hij(i, c) * y[c];
            y[i] = t / Hij(i, i);
        }
        GG_CUDA(cudaMemcpyAsync(P->d_sh, y.data(), k * sizeof(double), cudaMemcpyHostToDevice,
                                P->st));
        stage(P, ST_KRYLOV, 0, [&] { mupdate(k, P->d_sh, 1.0, x, pc ? Zb : nullptr); });
        GG_CUDA(cudaStreamSynchronize(P->st));           // y lives on this stack frame
        return steps;
    }
};

// Solver workspace for unknown vectors of up to `len` entries (at least
// 3 cap) and cycles of up to m steps; grows only.
void ensure_solver_ws(ggem_plan_t* P, int m, size_t len) {
    size_t ld = (std::max(len, (size_t)3 * P->cap) + 31) / 32 * 32;
    if (ld > P->sol_ld) {
        for (double** p : {&P->d_sv, &P->d_sb, &P->d_sx, &P->d_V}) {
            dfree(*p);
            *p = nullptr;
        }
        dalloc(P, &P->d_sv, ld);
        dalloc(P, &P->d_sb, ld);
        dalloc(P, &P->d_sx, ld);
        P->sol_ld = ld;
        P->sol_m = 0;
    }
    if (!P->d_sk) {
        dalloc(P, &P->d_sk, (size_t)P->cap);
        dalloc(P, &P->d_spart, (size_t)KH * KNB);
        dalloc(P, &P->d_sh, (size_t)3 * KH);
        GG_CUDA(cudaMallocHost((void**)&P->h_sh, (size_t)3 * KH * sizeof(double)));
    }
    if (P->sol_m < m) {
        dfree(P->d_V);
        P->d_V = nullptr;
        dalloc(P, &P->d_V, (size_t)(m + 1) * P->sol_ld);
        P->sol_m = m;
    }
}

void ensure_twin(ggem_plan_t* P) {
    if (P->fp64 || P->twin) return;
    ggem_params tp = P->prm;
    tp.precision = GGEM_FP64_EMULATED;    // FP64 accuracy, float-pair local sum
    ggem_plan_t* T = nullptr;
    ggem_status s = ggem_plan(&tp, P->st, &T);
    GG_CHECK(s == GGEM_OK, s, std::string("FP64 twin plan: ") + ggem_last_error(nullptr));
    P->twin = T;
    s = ggem_mesh_set(T, P->n_nodes, P->d_x, P->n_tris, P->d_tri);
    GG_CHECK(s == GGEM_OK, s, std::string("FP64 twin mesh: ") + ggem_last_error(T));
    if (P->offgrid != GGEM_OFFGRID_LAGRANGE) {    // the twin evaluates the same operator
        s = ggem_set_offgrid(T, P->offgrid, 0);
        GG_CHECK(s == GGEM_OK, s, std::string("FP64 twin off-grid: ") + ggem_last_error(T));
    }
}

// Solver on plan P for unknown vectors of length n3 (workspace ready).
Solver make_solver(ggem_plan_t* P, size_t n3) {
    Solver S;
    S.P = P;
    S.P64 = P->fp64 ? P : P->twin;
    S.n3 = n3;
    S.ld = P->sol_ld;
    S.hs = P->h_sh;
    return S;
}

// Restarted GMRES (FP64 plan) or iterative refinement (mixed plan) from the
// iterate S.x to the true relative residual tol; nb = ||b|| > 0.  beta0 > 0:
// V_0 already holds the normalised residual of S.x under P's operator, of
// norm beta0.  Returns the status; *its and *rel get the Arnoldi steps and
// the last true relative residual.
ggem_status refine(Solver& S, double nb, double tol, int restart, int maxit, double beta0,
                   int* its_out, double* rel_out) {
    ggem_plan_t* P = S.P;
    ggem_status result = GGEM_OK;
    int its = 0;
    double rel = 0.0;
    bool last_breakdown = false;
    bool have_v0 = beta0 > 0.0;
    // Mixed plan: the first correction needs only ~1e-4, so its residual
    // comes from the mixed operator unless that already looks converged.
    bool first_mixed = !P->fp64;
    for (;;) {
        double beta = have_v0 ? beta0 : S.residual_into_v0(first_mixed ? P : S.P64);
        have_v0 = false;
        rel = beta / nb;
        GG_CHECK(std::isfinite(rel), GGEM_ERR_NUMERICAL, "non-finite residual");
        if (first_mixed) {
            first_mixed = false;
            if (rel <= 10.0 * tol || its >= maxit) continue;   // decide in FP64
        } else if (rel <= tol) {
            result = last_breakdown ? GGEM_OK_BREAKDOWN : GGEM_OK;
            break;
        }
        if (its >= maxit) {
            result = GGEM_ERR_NOT_CONVERGED;
            P->err = "iteration limit reached";
            break;
        }
        int m = std::min(restart, maxit - its);
        // FP64: aim at the final tolerance.  Mixed: after a correction solved
        // to eta relative to r, the true residual is about (eta + eps) ||r||,
        // eps ~ 1e-5 the mixed operator's relative accuracy; asking eta down to
        // eps lets one correction from a warm start (||r|| ~ 1e-2 ||b||) reach
        // 1e-6, so the solve needs a single FP64 residual after it.
        double eta = P->fp64 ? tol * nb / beta : std::max(0.5 * tol * nb / beta, 1e-5);
        bool bd = false;
        int steps = S.cycle(P, m, beta, eta * beta, &bd);
        its += steps;
        P->sol_cycles++;
        last_breakdown = bd;
    }
    *its_out = its;
    *rel_out = rel;
    return result;
}

}  // namespace

ggem_status bie_solve(ggem_plan_t* P, const double* kappa, const double* b, double* q,
                      double tol, int restart, int maxit, int use_mlp, int* iters,
                      double* true_relres) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    ggem_status result = GGEM_OK;
    ggem_status s = guarded(P, [&] {
        GG_CHECK(P->mesh_ready && P->n_tris > 0, GGEM_ERR_INVALID_ARG,
                 "the solve needs a mesh with triangles");
        GG_CHECK(kappa && b && q, GGEM_ERR_INVALID_ARG, "NULL kappa, b or q");
        GG_CHECK(tol > 0.0 && std::isfinite(tol), GGEM_ERR_INVALID_ARG, "tol must be > 0");
        GG_CHECK(restart >= 1 && restart <= KMAXM, GGEM_ERR_INVALID_ARG,
                 "restart must be in 1..64");
        GG_CHECK(maxit >= 0, GGEM_ERR_INVALID_ARG, "maxit must be >= 0");
        GG_CHECK(use_mlp == 0 || use_mlp == 1, GGEM_ERR_INVALID_ARG, "use_mlp must be 0 or 1");
        GG_CHECK(!use_mlp || (P->mlp_ready && P->d_particle), GGEM_ERR_INVALID_ARG,
                 "the learned warm start needs a model and particle ids");
        const int n = P->n_nodes;
        const size_t n3 = (size_t)n * 3;
        ensure_solver_ws(P, restart, n3);
        ensure_twin(P);
        P->sol_cycles = P->sol_mv64 = P->sol_mvmix = 0;
        Solver S = make_solver(P, n3);
        if (P->pc_on) {
            precond_prepare(P);
            if (P->pc_m < restart || !P->d_pc_Zb) {
                dfree(P->d_pc_Zb);
                P->d_pc_Zb = nullptr;
                dalloc(P, &P->d_pc_Zb, (size_t)restart * P->sol_ld);
                P->pc_m = restart;
            }
            S.pc = true;
            S.Zb = P->d_pc_Zb;
        }
        const double* kd = stage_in(P, kappa, P->d_sk, (size_t)n);
        // (I + kappa/(4 pi) D) in, or b - that
        S.op = [P, n, kd](ggem_plan_t* Q, const double* in, double* out, const double* bb) {
            double_layer_dev(Q, in, P->d_sv);
            int nblk = (int)(((size_t)3 * n + KB - 1) / KB);
            k_bie_apply<<<nblk, KB, 0, P->st>>>(n, 0.25 / kPi, in, P->d_sv, kd, bb, out);
            GG_CUDA(cudaGetLastError());
            P->launches += 1;
        };
        S.b = stage_in(P, b, P->d_sb, n3);
        const bool q_host = !is_device_ptr(q);
        S.x = q_host ? P->d_sx : q;
        if (q_host)
            GG_CUDA(cudaMemcpyAsync(S.x, q, n3 * sizeof(double), cudaMemcpyHostToDevice, P->st));
        int its = 0;
        double rel = 0.0;
        const double nb = S.norm_b();
        double beta0 = 0.0;                              // V_0 already formed when > 0
        P->sol_guess_mlp = 0;
        P->sol_rel_plain = P->sol_rel_mlp = 0.0;
        if (use_mlp && nb > 0.0) {
            // r0 = b - A q; learned guess q + A^-1 r0; keep whichever of q and
            // the learned guess has the lower residual under the plan's operator
            if (!P->d_smlp) dalloc(P, &P->d_smlp, S.ld);
            if (!P->d_sres) dalloc(P, &P->d_sres, S.ld);
            S.apply(P, S.x, P->d_sres, true);
            S.mdot(1, P->d_sres, P->d_sres, P->d_sh);
            S.to_host(1);
            const double r_plain = std::sqrt(S.hs[0]) / nb;
            mlp_guess_dev(P, kd, P->d_sres, S.x, P->d_smlp);
            double* xs = S.x;
            S.x = P->d_smlp;
            const double r_mlp = S.residual_into_v0(P) / nb;
            S.x = xs;
            P->sol_rel_plain = r_plain;
            P->sol_rel_mlp = r_mlp;
            // the chosen guess's residual starts GMRES (V_0 = r / beta)
            if (r_mlp < r_plain) {
                GG_CUDA(cudaMemcpyAsync(S.x, P->d_smlp, n3 * sizeof(double),
                                        cudaMemcpyDeviceToDevice, P->st));
                P->sol_guess_mlp = 1;
                beta0 = r_mlp * nb;                      // V_0 holds it already
            } else {
                beta0 = r_plain * nb;
                GG_CUDA(cudaMemcpyAsync(P->d_V, P->d_sres, n3 * sizeof(double),
                                        cudaMemcpyDeviceToDevice, P->st));
                S.normalize(P->d_V, P->d_sh);
            }
        }
        if (nb == 0.0) GG_CUDA(cudaMemsetAsync(S.x, 0, n3 * sizeof(double), P->st));
        else result = refine(S, nb, tol, restart, maxit, beta0, &its, &rel);
        if (q_host)
            GG_CUDA(cudaMemcpyAsync(q, S.x, n3 * sizeof(double), cudaMemcpyDeviceToHost, P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));
        P->sol_iters = its;
        P->sol_relres = rel;
        if (iters) *iters = its;
        if (true_relres) *true_relres = rel;
    });
    return s != GGEM_OK ? s : result;
}

ggem_status ggem_bie_operator(ggem_plan_t* P, const double* kappa, const double* q,
                              double* out) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready && P->n_tris > 0, GGEM_ERR_INVALID_ARG,
                 "the operator needs a mesh with triangles");
        GG_CHECK(kappa && q && out, GGEM_ERR_INVALID_ARG, "NULL argument");
        const size_t n3 = (size_t)P->n_nodes * 3;
        const double* kd = stage_in(P, kappa, P->d_in1, (size_t)P->n_nodes);
        const double* qd = stage_in(P, q, P->d_in2, n3);
        OutMap mo = stage_out(out, P->d_out0, n3);
        double* v = P->d_out1;                       // [6 cap] staging: room for D q
        double_layer_dev(P, qd, v);
        k_bie_apply<<<(unsigned)((n3 + KB - 1) / KB), KB, 0, P->st>>>(
            P->n_nodes, 0.25 / kPi, qd, v, kd, nullptr, mo.dev);
        GG_CUDA(cudaGetLastError());
        P->launches += 1;
        finish_out(P, mo);
        GG_CUDA(cudaStreamSynchronize(P->st));
    });
}

ggem_status ggem_solve_guess(const ggem_plan_t* P, int* used_mlp, double* relres_plain,
                             double* relres_mlp) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    if (used_mlp) *used_mlp = P->sol_guess_mlp;
    if (relres_plain) *relres_plain = P->sol_rel_plain;
    if (relres_mlp) *relres_mlp = P->sol_rel_mlp;
    return GGEM_OK;
}

ggem_status ggem_solve_stats(const ggem_plan_t* P, int* cycles, int* matvec_fp64,
                             int* matvec_mixed) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    if (cycles) *cycles = P->sol_cycles;
    if (matvec_fp64) *matvec_fp64 = P->sol_mv64;
    if (matvec_mixed) *matvec_mixed = P->sol_mvmix;
    return GGEM_OK;
}

// ======================================================= rigid particles
// Sec. 6.1, Eq. (sl_r): on the surface of a rigid particle p the fluid
// velocity is U_p + Omega_p x (x - c_p), so at every node b of p
//     U_p + Omega_p x (x_b - c_p) + 1/(8 pi mu) int f_i G_ji dS = u_inf(x_b),
// closed by the balance of force and torque on each particle,
//     sum_b A_b f_b = -F_p,   sum_b A_b (x_b - c_p) x f_b = -T_p
// (F_p = T_p = 0: force- and torque-free).  The unknown vector is
// [f (3 N) | U_0, Omega_0, U_1, ... (6 P)]; the balance rows are scaled to
// velocity units by the Stokes mobilities of the sphere with the particle's
// surface area, 1/(6 pi mu R_p) and 1/(8 pi mu R_p^2).

namespace {

constexpr int RB = 128;          // threads of the per-particle kernels

// velocity rows: out_b = s w_b + U_p + Omega_p x (x_b - c_p), or b_b - that
__global__ void k_rigid_rows(int n, double s, const double* __restrict__ x,
                             const int* __restrict__ part, const double* __restrict__ c,
                             const double* __restrict__ w, const double* __restrict__ uo,
                             const double* __restrict__ b, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = part[i];
    const double rx = x[3 * i] - c[3 * p], ry = x[3 * i + 1] - c[3 * p + 1],
                 rz = x[3 * i + 2] - c[3 * p + 2];
    const double* U = uo + 6 * (size_t)p;
    const double ox = U[3], oy = U[4], oz = U[5];
    double v0 = fma(s, w[3 * i], U[0] + (oy * rz - oz * ry));
    double v1 = fma(s, w[3 * i + 1], U[1] + (oz * rx - ox * rz));
    double v2 = fma(s, w[3 * i + 2], U[2] + (ox * ry - oy * rx));
    if (b) {
        v0 = b[3 * i] - v0;
        v1 = b[3 * i + 1] - v1;
        v2 = b[3 * i + 2] - v2;
    }
    out[3 * i] = v0;
    out[3 * i + 1] = v1;
    out[3 * i + 2] = v2;
}

// Sum of 7 per-thread values over the block in a fixed order; valid in thread 0.
__device__ void block_sum7(double (&a)[7]) {
    __shared__ double red[7][RB / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        double t = warp_sum(a[k]);
        if (lane == 0) red[k][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            double t = 0.0;
            for (int q = 0; q < RB / 32; ++q) t += red[k][q];
            a[k] = t;
        }
    }
}

// balance rows of particle blockIdx.x: out = -scale (sum A f, sum A r x f),
// or b - that
__global__ void __launch_bounds__(RB) k_rigid_balance(
    const int* __restrict__ pstart, const int* __restrict__ pnodes, const double* __restrict__ x,
    const double* __restrict__ area, const double* __restrict__ c,
    const double* __restrict__ rscale, const double* __restrict__ f,
    const double* __restrict__ b, double* __restrict__ out) {
    const int p = blockIdx.x;
    const double cx = c[3 * p], cy = c[3 * p + 1], cz = c[3 * p + 2];
    double a[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int k = pstart[p] + threadIdx.x; k < pstart[p + 1]; k += RB) {
        const int i = pnodes[k];
        const double A = area[i];
        const double fx = A * f[3 * i], fy = A * f[3 * i + 1], fz = A * f[3 * i + 2];
        const double rx = x[3 * i] - cx, ry = x[3 * i + 1] - cy, rz = x[3 * i + 2] - cz;
        a[0] += fx;
        a[1] += fy;
        a[2] += fz;
        a[3] += ry * fz - rz * fy;
        a[4] += rz * fx - rx * fz;
        a[5] += rx * fy - ry * fx;
    }
    block_sum7(a);
    if (threadIdx.x == 0) {
        const double sf = rscale[2 * p], st = rscale[2 * p + 1];
        for (int k = 0; k < 6; ++k) {
            double v = -(k < 3 ? sf : st) * a[k];
            out[6 * p + k] = b ? b[6 * p + k] - v : v;
        }
    }
}

// per particle: S_p = sum of its nodal areas, R_p = sqrt(S_p / 4 pi), the two
// row scales, and the balance part of the right side (ext [P][6] scaled in
// place; nullptr: zero)
__global__ void __launch_bounds__(RB) k_rigid_setup(const int* __restrict__ pstart,
                                                    const int* __restrict__ pnodes,
                                                    const double* __restrict__ area, double mu,
                                                    double* __restrict__ rscale,
                                                    double* __restrict__ bbal, int has_ext) {
    const int p = blockIdx.x;
    double a[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int k = pstart[p] + threadIdx.x; k < pstart[p + 1]; k += RB) a[6] += area[pnodes[k]];
    block_sum7(a);
    if (threadIdx.x == 0) {
        const double R2 = a[6] / (4.0 * kPi);
        const double sf = 1.0 / (6.0 * kPi * mu * sqrt(R2)), st = 1.0 / (8.0 * kPi * mu * R2);
        rscale[2 * p] = sf;
        rscale[2 * p + 1] = st;
        for (int k = 0; k < 6; ++k)
            bbal[6 * p + k] = has_ext ? (k < 3 ? sf : st) * bbal[6 * p + k] : 0.0;
    }
}

}  // namespace

// node lists of the particles (CSR, nodes ascending within a particle), from
// the plan's particle ids; sizes the per-particle arrays
void ggem::particle_node_lists(ggem_plan_t* P) {
    const int np = P->n_particles, n = P->n_nodes;
    if (P->rig_cap < np) {
        for (void* q : {(void*)P->d_pstart, (void*)P->d_rc, (void*)P->d_rscale}) dfree(q);
        P->d_pstart = nullptr;
        P->d_rc = P->d_rscale = nullptr;
        dalloc(P, &P->d_pstart, (size_t)np + 1);
        dalloc(P, &P->d_rc, (size_t)3 * np);
        dalloc(P, &P->d_rscale, (size_t)2 * np);
        P->rig_cap = np;
    }
    if (!P->d_pnodes) dalloc(P, &P->d_pnodes, (size_t)P->cap);
    if (P->pcsr_ready) return;
    std::vector<int> part(n), start(np + 1, 0), nodes(n);
    GG_CUDA(cudaMemcpyAsync(part.data(), P->d_particle, (size_t)n * sizeof(int),
                            cudaMemcpyDeviceToHost, P->st));
    GG_CUDA(cudaStreamSynchronize(P->st));
    for (int i = 0; i < n; ++i) start[part[i] + 1]++;
    for (int p = 0; p < np; ++p) start[p + 1] += start[p];
    std::vector<int> cur(start.begin(), start.end() - 1);
    for (int i = 0; i < n; ++i) nodes[cur[part[i]]++] = i;      // stable: ascending nodes
    GG_CUDA(cudaMemcpyAsync(P->d_pstart, start.data(), (size_t)(np + 1) * sizeof(int),
                            cudaMemcpyHostToDevice, P->st));
    GG_CUDA(cudaMemcpyAsync(P->d_pnodes, nodes.data(), (size_t)n * sizeof(int),
                            cudaMemcpyHostToDevice, P->st));
    GG_CUDA(cudaStreamSynchronize(P->st));                       // host vectors go out of scope
    P->pcsr_ready = true;
}

namespace {

// copy n doubles from a host or device array into device memory
void copy_in(ggem_plan_t* P, double* dst, const double* src, size_t n) {
    GG_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double),
                            is_device_ptr(src) ? cudaMemcpyDeviceToDevice
                                               : cudaMemcpyHostToDevice, P->st));
}

void copy_out(ggem_plan_t* P, double* dst, const double* src, size_t n) {
    GG_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double),
                            is_device_ptr(dst) ? cudaMemcpyDeviceToDevice
                                               : cudaMemcpyDeviceToHost, P->st));
}

}  // namespace

ggem_status ggem_rigid_solve(ggem_plan_t* P, int n_particles, const double* centres,
                             const double* u_inf, const double* ext, double* f, double* uo,
                             double tol, int restart, int maxit, int* iters,
                             double* true_relres) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    ggem_status result = GGEM_OK;
    ggem_status s = guarded(P, [&] {
        GG_CHECK(P->mesh_ready && P->n_tris > 0, GGEM_ERR_INVALID_ARG,
                 "the solve needs a mesh with triangles");
        GG_CHECK(P->d_particle && P->particles_n == P->n_nodes, GGEM_ERR_INVALID_ARG,
                 "particle ids not set for this mesh (ggem_mesh_particles)");
        GG_CHECK(n_particles == P->n_particles, GGEM_ERR_INVALID_ARG,
                 "n_particles differs from the count given to ggem_mesh_particles");
        GG_CHECK(centres && f && uo, GGEM_ERR_INVALID_ARG, "NULL centres, f or uo");
        GG_CHECK(tol > 0.0 && std::isfinite(tol), GGEM_ERR_INVALID_ARG, "tol must be > 0");
        GG_CHECK(restart >= 1 && restart <= KMAXM, GGEM_ERR_INVALID_ARG,
                 "restart must be in 1..64");
        GG_CHECK(maxit >= 0, GGEM_ERR_INVALID_ARG, "maxit must be >= 0");
        const int n = P->n_nodes, np = n_particles;
        const size_t nf = (size_t)3 * n, nz = nf + (size_t)6 * np;
        ensure_solver_ws(P, restart, nz);
        ensure_twin(P);
        particle_node_lists(P);
        P->sol_cycles = P->sol_mv64 = P->sol_mvmix = 0;
        P->sol_guess_mlp = 0;
        P->sol_rel_plain = P->sol_rel_mlp = 0.0;
        Solver S = make_solver(P, nz);
        copy_in(P, P->d_rc, centres, (size_t)3 * np);
        // right side [u_inf | scaled F, T]
        double* bv = P->d_sb;
        if (u_inf) copy_in(P, bv, u_inf, nf);
        else GG_CUDA(cudaMemsetAsync(bv, 0, nf * sizeof(double), P->st));
        if (ext) copy_in(P, bv + nf, ext, (size_t)6 * np);
        k_rigid_setup<<<np, RB, 0, P->st>>>(P->d_pstart, P->d_pnodes, P->d_area, P->prm.mu,
                                            P->d_rscale, bv + nf, ext ? 1 : 0);
        GG_CUDA(cudaGetLastError());
        P->launches += 1;
        S.b = bv;
        // iterate [f | U, Omega] from the caller's guess
        S.x = P->d_sx;
        copy_in(P, S.x, f, nf);
        copy_in(P, S.x + nf, uo, (size_t)6 * np);
        const double s8 = 1.0 / (8.0 * kPi * P->prm.mu);
        S.op = [P, n, np, nf, s8](ggem_plan_t* Q, const double* in, double* out,
                                  const double* bb) {
            single_layer_dev(Q, in, P->d_sv);
            k_rigid_rows<<<(n + KB - 1) / KB, KB, 0, P->st>>>(n, s8, P->d_x, P->d_particle,
                                                             P->d_rc, P->d_sv, in + nf, bb,
                                                             out);
            k_rigid_balance<<<np, RB, 0, P->st>>>(P->d_pstart, P->d_pnodes, P->d_x, P->d_area,
                                                  P->d_rc, P->d_rscale, in,
                                                  bb ? bb + nf : nullptr, out + nf);
            GG_CUDA(cudaGetLastError());
            P->launches += 2;
        };
        int its = 0;
        double rel = 0.0;
        const double nb = S.norm_b();
        if (nb == 0.0) GG_CUDA(cudaMemsetAsync(S.x, 0, nz * sizeof(double), P->st));
        else result = refine(S, nb, tol, restart, maxit, 0.0, &its, &rel);
        copy_out(P, f, S.x, nf);
        copy_out(P, uo, S.x + nf, (size_t)6 * np);
        GG_CUDA(cudaStreamSynchronize(P->st));
        P->sol_iters = its;
        P->sol_relres = rel;
        if (iters) *iters = its;
        if (true_relres) *true_relres = rel;
    });
    return s != GGEM_OK ? s : result;
}
