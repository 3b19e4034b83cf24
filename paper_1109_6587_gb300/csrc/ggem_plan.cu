// libggem plan, mesh and C-ABI entry points (include/ggem.h).
// Paper: Kumar & Graham, arXiv 1109.6587.  The data flow of one evaluation
// follows Sec. 3.2 / 3.4 / 3.5:
//   local sum (cell list) -> wall data u^g = -u^l -> spread rho_g -> FFT x,z
//   -> Chebyshev transform -> per-mode Kleiser-Schumann tau solve (FP64)
//   -> inverse transforms -> 5-point Lagrange interpolation + local part.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "ggem_internal.cuh"
#include "ggem_host.cuh"

using namespace ggem;

namespace ggem {
void ks_precompute_mode(int Ny, double W, double mu, double k2, double* pb, double* phib,
                        double* vb, double* minv);
void ks_coef_table(int Ny, double* tab);
void ks_thomas_mode(int Ny, double lam, double* tab, double* isq);
void ks_chunk_mode(int Ny, const double* tab, double* out);
}

namespace {

// message of the last failed ggem_plan call on this thread
thread_local std::string g_create_error = "no plan";

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// FFT tables of an Nx x Nz grid (complex, interleaved): twx = the Nx/4
// twiddles of the length-Nx/2 complex FFT, then the Nx/2 post-twiddles
// exp(-2 pi i k/Nx) of the real transform; twz = the Nz/2 twiddles in z.
void fft_tables(int Nx, int Nz, std::vector<double>& twx, std::vector<double>& twz) {
    const int M = Nx / 2;
    twx.assign(2 * (M / 2 + M), 0.0);
    twz.assign(2 * (Nz / 2), 0.0);
    for (int k = 0; k < M / 2; ++k) {
        twx[2 * k] = std::cos(2 * kPi * k / M);
        twx[2 * k + 1] = -std::sin(2 * kPi * k / M);
    }
    for (int k = 0; k < M; ++k) {
        twx[2 * (M / 2 + k)] = std::cos(2 * kPi * k / Nx);
        twx[2 * (M / 2 + k) + 1] = -std::sin(2 * kPi * k / Nx);
    }
    for (int k = 0; k < Nz / 2; ++k) {
        twz[2 * k] = std::cos(2 * kPi * k / Nz);
        twz[2 * k + 1] = -std::sin(2 * kPi * k / Nz);
    }
}

// Window of the spectral off-grid evaluation with oversampling 2 and w
// points per side (Greengard & Lee): variance tau = pi w / (N^2 R (R - 1/2))
// in units where the period is 2 pi, so exp(-(s - s_p)^2 / 4 tau) =
// exp(-c t^2) with t in fine spacings and c = pi (R - 1/2) / (R w).
constexpr double kSpecR = 2.0;
double spec_c(int w) { return kPi * (kSpecR - 0.5) / (kSpecR * w); }

SpecGrid spec_grid(const ggem_plan_t* P) {
    SpecGrid g;
    g.fine = P->d_spec;
    g.Mx = 2 * P->prm.Nx;
    g.Mz = 2 * P->prm.Nz;
    g.w = P->spec_w;
    g.c = spec_c(P->spec_w);
    g.Mt = 4 * (P->prm.Ny - 1);
    g.sx = g.Mx / P->prm.Lx;
    g.sz = g.Mz / P->prm.Lz;
    g.st = g.Mt / (2.0 * kPi);
    g.sy = 2.0 / P->prm.W;
    g.order = nullptr;
    return g;
}

// ------------------------------------------------------------- geometry
__global__ void k_tri_geom(int m, const double* __restrict__ x, const int* __restrict__ tri,
                           double* __restrict__ ta, double* __restrict__ tn,
                           double* __restrict__ area, double* __restrict__ nsum) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    int i1 = tri[3 * k], i2 = tri[3 * k + 1], i3 = tri[3 * k + 2];
    double e2[3], e3[3], c[3];
    for (int d = 0; d < 3; ++d) {
        e2[d] = x[3 * i2 + d] - x[3 * i1 + d];
        e3[d] = x[3 * i3 + d] - x[3 * i1 + d];
    }
    c[0] = e2[1] * e3[2] - e2[2] * e3[1];
    c[1] = e2[2] * e3[0] - e2[0] * e3[2];
    c[2] = e2[0] * e3[1] - e2[1] * e3[0];
    double a2 = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    double A = 0.5 * a2;
    ta[k] = A;
    for (int d = 0; d < 3; ++d) tn[3 * k + d] = c[d] / a2;
    int v[3] = {i1, i2, i3};
    for (int p = 0; p < 3; ++p) {
        atomicAdd(&area[v[p]], A / 3.0);
        for (int d = 0; d < 3; ++d) atomicAdd(&nsum[3 * v[p] + d], 0.5 * c[d]);
    }
}

__global__ void k_normalize(int n, double* __restrict__ nrm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a = nrm[3 * i], b = nrm[3 * i + 1], c = nrm[3 * i + 2];
    double s = 1.0 / sqrt(a * a + b * b + c * c);
    nrm[3 * i] = a * s; nrm[3 * i + 1] = b * s; nrm[3 * i + 2] = c * s;
}

// longest triangle edge (non-negative doubles compare as unsigned 64-bit integers)
__global__ void k_max_edge(int m, const double* __restrict__ x, const int* __restrict__ tri,
                           double* __restrict__ out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    double l = 0.0;
    for (int e = 0; e < 3; ++e) {
        int a = tri[3 * k + e], b = tri[3 * k + (e + 1) % 3];
        double d0 = x[3 * a] - x[3 * b], d1 = x[3 * a + 1] - x[3 * b + 1],
               d2 = x[3 * a + 2] - x[3 * b + 2];
        l = fmax(l, sqrt(d0 * d0 + d1 * d1 + d2 * d2));
    }
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(l));
}

__global__ void k_check_inside(int n, const double* __restrict__ x, double y0, double W,
                               int* __restrict__ bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double y = x[3 * i + 1];
    bool ok = (y > y0) && (y < y0 + W) && isfinite(x[3 * i]) && isfinite(x[3 * i + 2]);
    if (!ok) atomicAdd(bad, 1);
}

// ------------------------------------------------------------ pipeline
template <typename T>
SortedSources<T> sources_of(ggem_plan_t* P, bool mesh) {
    SortedSources<T> s;
    s.pos = (v4_t<T>*)(mesh ? P->d_mesh_pos : P->d_spos);
    s.g = (v4_t<T>*)P->d_sg;
    s.cell = mesh ? P->d_mesh_cell : P->d_src_cell;
    s.perm = mesh ? P->d_mesh_perm : P->d_perm;
    s.cell_start = mesh ? P->d_mesh_start : P->d_cell_start;
    s.n = 0;
    return s;
}

int nout_of(int sel) { return ((sel & 1) ? 3 : 0) + ((sel & 2) ? 6 : 0); }

// Global part: wall data, spread, transforms, tau solves, inverse transforms.
// The physical result is left in gridB as [Ny][nout][Nz][Nx].
template <typename T>
void run_global(ggem_plan_t* P, const SortedSources<T>& src, bool mesh, int out_sel,
                cudaStream_t st) {
    const GridGeom& geo = P->geo;
    T* A = (T*)P->d_gridA;
    T* B = (T*)P->d_gridB;
    T* Wl = (T*)P->d_wall;
    stage(P, ST_WALL, 1, [&] {
        GG_CUDA(local_sum<T>(geo, P->cg, src, TK_WALL, 2 * geo.Nz * geo.Nx, P->d_wall_cell,
                             (const v4_t<T>*)P->d_wall_pos, nullptr, OUT_U, Wl, 0, st));
    });
    stage(P, ST_SPREAD, sizeof(T) == 4 ? 3 : 2, [&] {
        GG_CUDA(spread<T>(geo, P->cg, P->d_yj, (const T*)P->d_ydiff, src,
                          mesh ? P->d_mesh_sdi : P->d_sdi,
                          (const v4_t<T>*)(mesh ? P->d_mesh_sdf : P->d_sdf), A, B,
                          P->d_spread_list, st));
    });
    stage(P, ST_FFT_FWD, 4, [&] {
        GG_CUDA(fft_forward<T>(geo, A, geo.Ny * 3, P->d_tw_x, P->d_tw_z, st));
        GG_CUDA(fft_forward<T>(geo, Wl, 6, P->d_tw_x, P->d_tw_z, st));
    });
    stage(P, ST_CHEB_FWD, 1, [&] {
        GG_CUDA(cheb_apply<T>(geo.Ny, (const T*)P->d_cheb_fwd, A, B, (long)3 * P->nmodes * 2,
                              st, P->d_tc_err, P->nsm, P->d_tc_fwd));
    });
    stage(P, ST_KS, 1, [&] {
        GG_CUDA(ks_modes<T>(geo, B, Wl, (const T*)P->d_ksb, P->d_minv, P->d_kscoef, P->d_thom,
                            P->d_kschunk, P->d_isq, out_sel, A, st));
    });
    int nout = nout_of(out_sel);
    if (P->offgrid == GGEM_OFFGRID_SPECTRAL) {
        // Chebyshev coefficients -> deconvolved theta-node values, then
        // deconvolve in x, z onto the oversampled grid and transform there
        const int nth = 2 * geo.Ny - 1;
        T* mid = (T*)P->d_spec_mid;
        stage(P, ST_CHEB_INV, 1, [&] {
            GG_CUDA(cheb_rect<T>(nth, geo.Ny, (const T*)P->d_spec_ct, A, mid,
                                 (long)nout * P->nmodes * 2, st));
        });
        stage(P, ST_FFT_INV, 3, [&] {
            GridGeom fg = geo;
            fg.Nx = 2 * geo.Nx;
            fg.Nz = 2 * geo.Nz;
            fg.nkx = geo.Nx;
            GG_CUDA(spectral_pad<T>(geo, mid, nth * nout, fg.Nx, fg.Nz, (const T*)P->d_spec_dx,
                                    (const T*)P->d_spec_dz, (T*)P->d_spec, st));
            // (only the coarse grid's Nx/2 columns in x are nonzero for the z pass)
            GG_CUDA(fft_inverse<T>(fg, (T*)P->d_spec, nth * nout, P->d_spec_twx,
                                   P->d_spec_twz, st, geo.Nx / 2));
        });
        return;
    }
    stage(P, ST_CHEB_INV, 1, [&] {
        GG_CUDA(cheb_apply<T>(geo.Ny, (const T*)P->d_cheb_inv, A, B,
                              (long)nout * P->nmodes * 2, st, P->d_tc_err, P->nsm, P->d_tc_inv));
    });
    stage(P, ST_FFT_INV, 2, [&] {
        GG_CUDA(fft_inverse<T>(geo, B, geo.Ny * nout, P->d_tw_x, P->d_tw_z, st));
    });
}

template <typename T>
void point_forces_impl(ggem_plan_t* P, int n_src, const double* xs, const double* g, int n_tgt,
                       const double* xt, int tgt_is_src, double* u, double* s) {
    const GridGeom& geo = P->geo;
    cudaStream_t st = P->st;
    stage(P, ST_CELLS, 4, [&] {
        GG_CUDA(build_cells<T>(geo, P->cg, n_src, xs, P->d_cell_count, P->d_cell_start,
                               P->d_cursor, P->d_src_cell, P->d_perm, (v4_t<T>*)P->d_spos, st));
        GG_CUDA(spread_prepare<T>(geo, P->d_yj, n_src, P->d_perm, xs, P->d_sdi,
                                  (v4_t<T>*)P->d_sdf, st));
    });
    stage(P, ST_GATHER, 1, [&] {
        GG_CUDA(gather_strengths<T>(n_src, P->d_perm, g, nullptr, 1.0, (v4_t<T>*)P->d_sg, st));
    });
    SortedSources<T> src = sources_of<T>(P, false);
    src.n = n_src;
    int mode = (u ? OUT_U : 0) | (s ? OUT_S : 0);
    int stride = (u ? 3 : 0) + (s ? 6 : 0);
    T* loc = (T*)P->d_local;
    stage(P, ST_LOCAL, tgt_is_src ? 1 : 2, [&] {
        if (!tgt_is_src)
            GG_CUDA(locate_targets<T>(geo, P->cg, n_tgt, TK_POINTS, xt, P->d_tgt_cell,
                                      (v4_t<T>*)P->d_tgt_pos, st));
        GG_CUDA(local_sum<T>(geo, P->cg, src, tgt_is_src ? TK_SORTED : TK_POINTS,
                             tgt_is_src ? n_src : n_tgt, P->d_tgt_cell,
                             (const v4_t<T>*)P->d_tgt_pos, nullptr, mode, loc, stride, st));
    });
    int sel = (u ? 1 : 0) | (s ? 2 : 0);
    run_global<T>(P, src, false, sel, P->st);
    const double* xtt = tgt_is_src ? xs : xt;
    int nt = tgt_is_src ? n_src : n_tgt;
    int nout = nout_of(sel);
    SpecGrid sg = spec_grid(P);
    sg.order = tgt_is_src ? P->d_perm : nullptr;    // sources in cell order
    const SpecGrid* spec = P->offgrid == GGEM_OFFGRID_SPECTRAL ? &sg : nullptr;
    stage(P, ST_INTERP, (u ? 1 : 0) + (s ? 1 : 0), [&] {
        if (u) {
            double sc = 4.0 * geo.alpha / std::sqrt(kPi) / (8.0 * kPi * geo.mu);
            GG_CUDA(interp_combine<T>(geo, P->d_yj, (const T*)P->d_gridB, nout, 0, nt, xtt, loc,
                                      stride, nullptr, tgt_is_src ? g : nullptr, nullptr, sc, 0,
                                      u, 3, st, spec));
        }
        if (s)
            GG_CUDA(interp_combine<T>(geo, P->d_yj, (const T*)P->d_gridB, nout, u ? 3 : 0, nt,
                                      xtt, loc + (u ? 3 : 0), stride, nullptr, nullptr, nullptr,
                                      0.0, 1, s, 6, st, spec));
    });
}

template <typename T>
__global__ void k_split_local(int n, const T* __restrict__ loc, int stride, double* __restrict__ u,
                              double* __restrict__ s) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const T* o = loc + (size_t)t * stride;
    int k = 0;
    if (u) {
        for (int c = 0; c < 3; ++c) u[3 * t + c] = (double)o[c];
        k = 3;
    }
    if (s)
        for (int c = 0; c < 6; ++c) s[6 * t + c] = (double)o[k + c];
}

// Local part alone (Eq. u_loc): cell list of the sources, then the pair sum.
template <typename T>
void local_only_impl(ggem_plan_t* P, int n_src, const double* xs, const double* g, int n_tgt,
                     const double* xt, int tgt_is_src, double* u, double* s) {
    const GridGeom& geo = P->geo;
    cudaStream_t st = P->st;
    stage(P, ST_CELLS, 4, [&] {
        GG_CUDA(build_cells<T>(geo, P->cg, n_src, xs, P->d_cell_count, P->d_cell_start,
                               P->d_cursor, P->d_src_cell, P->d_perm, (v4_t<T>*)P->d_spos, st));
        GG_CUDA(spread_prepare<T>(geo, P->d_yj, n_src, P->d_perm, xs, P->d_sdi,
                                  (v4_t<T>*)P->d_sdf, st));
    });
    stage(P, ST_GATHER, 1, [&] {
        GG_CUDA(gather_strengths<T>(n_src, P->d_perm, g, nullptr, 1.0, (v4_t<T>*)P->d_sg, st));
    });
    SortedSources<T> src = sources_of<T>(P, false);
    src.n = n_src;
    int mode = (u ? OUT_U : 0) | (s ? OUT_S : 0);
    int stride = (u ? 3 : 0) + (s ? 6 : 0);
    int nt = tgt_is_src ? n_src : n_tgt;
    T* loc = (T*)P->d_local;
    stage(P, ST_LOCAL, tgt_is_src ? 2 : 3, [&] {
        if (!tgt_is_src)
            GG_CUDA(locate_targets<T>(geo, P->cg, nt, TK_POINTS, xt, P->d_tgt_cell,
                                      (v4_t<T>*)P->d_tgt_pos, st));
        GG_CUDA(local_sum<T>(geo, P->cg, src, tgt_is_src ? TK_SORTED : TK_POINTS, nt,
                             P->d_tgt_cell, (const v4_t<T>*)P->d_tgt_pos, nullptr, mode, loc,
                             stride, st));
        if (nt > 0) k_split_local<T><<<(nt + 255) / 256, 256, 0, st>>>(nt, loc, stride, u, s);
        GG_CUDA(cudaGetLastError());
    });
}

template <typename T>
void layer_impl(ggem_plan_t* P, int layer, const double* q, double* out) {
    const GridGeom& geo = P->geo;
    cudaStream_t st = P->st;
    int n = P->n_nodes;
    const bool elem = P->prm.quadrature == GGEM_ELEMENT;
    stage(P, ST_GATHER, elem ? 2 : 1, [&] {
        GG_CUDA(gather_strengths<T>(n, P->d_mesh_perm, q, P->d_area, 8.0 * kPi * geo.mu,
                                    (v4_t<T>*)P->d_sg, st));
        if (elem)
            GG_CUDA(qp_strengths<T>(P->n_qp, P->d_qv_sorted, (const v4_t<T>*)P->d_qw, n, q,
                                    (T*)P->d_q32, 8.0 * kPi * geo.mu, (v4_t<T>*)P->d_qg,
                                    (T*)P->d_qp_pack, P->d_qp_inv, P->qp_np, st));
        if (elem && P->ff) GG_CUDA(to_float_pairs(P->n_qp, P->d_qg, P->d_qg_ff, st));
    });
    SortedSources<T> src = sources_of<T>(P, true);
    src.n = n;
    T* loc = (T*)P->d_local;
    // The local part and the global part are independent until the combine.
    // The longer of the two -- the local sum under the element rule (~5x the
    // global part), the global part's chain of short kernels with nodal
    // sources -- runs on the plan's second stream, created with the device's
    // greatest priority, so its blocks are scheduled first and the other part
    // fills the SMs it leaves; forked after the strengths are gathered,
    // joined before the interpolation (both on one stream when tracing, so
    // that stage times stay separable).
    const bool overlap = !P->prof && P->st2;
    cudaStream_t ls = overlap && elem ? P->st2 : st;
    cudaStream_t gs = overlap && !elem ? P->st2 : st;
    cudaStream_t side = overlap ? P->st2 : st;
    if (overlap) {
        GG_CUDA(cudaEventRecord(P->ev_fork, st));
        GG_CUDA(cudaStreamWaitEvent(side, P->ev_fork, 0));
    }
    if (!elem) {
        stage(P, ST_LOCAL, 1, [&] {
            GG_CUDA(local_sum<T>(geo, P->cg, src, TK_SORTED, n, nullptr, nullptr, P->d_nrm,
                                 layer == 0 ? OUT_U : OUT_DBL, loc, 3, ls));
        });
    } else if (P->n_qp == 0) {
        // no triangles: every element integral is empty
        GG_CUDA(cudaMemsetAsync(loc, 0, (size_t)n * 3 * sizeof(T), ls));
    } else {
        // local part by the element rule: all quadrature points, then the polar
        // rule on the triangles that touch each node (Sec. 3.4.1, 3.5.2)
        SortedSources<T> qs;
        qs.pos = (v4_t<T>*)P->d_qp_pos;
        qs.g = (v4_t<T>*)P->d_qg;
        qs.cell = P->d_qp_cell;
        qs.perm = P->d_qp_perm;
        qs.cell_start = P->fp64 ? P->d_qp_start : P->d_qp_pstart;   // FP32: padded layout
        qs.n = P->n_qp;
        stage(P, ST_LOCAL, 1, [&] {
            GG_CUDA(local_sum_elem<T>(geo, P->cg, qs, P->d_qv_sorted, 1.01 * P->near_edge, src,
                                      P->d_nrm, layer, loc, 3, ls,
                                      P->fp64 ? P->d_qp_ff : (void*)P->d_qp_pack,
                                      P->fp64 ? P->d_qg_ff : nullptr, P->soa_ld, P->d_qp_inv));
        });
        stage(P, ST_ELEM, 1, [&] {
            GG_CUDA(elem_correct<T>(n, layer, geo, P->d_x, P->d_tri, P->d_tri_nrm, P->d_nrm,
                                    P->d_adj_start, P->d_adj,
                                    P->fp64 ? (const T*)q : (const T*)P->d_q32, P->rule, loc, 3,
                                    ls));
        });
    }
    run_global<T>(P, src, true, layer == 0 ? 1 : 2, gs);
    if (overlap) {
        GG_CUDA(cudaEventRecord(P->ev_join, side));
        GG_CUDA(cudaStreamWaitEvent(st, P->ev_join, 0));
    }
    SpecGrid sg = spec_grid(P);
    sg.order = P->d_mesh_perm;                      // mesh nodes in cell order
    const SpecGrid* spec = P->offgrid == GGEM_OFFGRID_SPECTRAL ? &sg : nullptr;
    stage(P, ST_INTERP, 1, [&] {
        if (layer == 0) {
            // nodal form: remove the free-space global self term (4 alpha/sqrt(pi)) A_b q_b;
            // the element rule integrates the near field itself
            double sc = elem ? 0.0 : 4.0 * geo.alpha / std::sqrt(kPi);
            GG_CUDA(interp_combine<T>(geo, P->d_yj, (const T*)P->d_gridB, 3, 0, n, P->d_x, loc,
                                      3, nullptr, elem ? nullptr : q, P->d_area, sc, 0, out, 3,
                                      st, spec));
        } else {
            GG_CUDA(interp_combine<T>(geo, P->d_yj, (const T*)P->d_gridB, 6, 0, n, P->d_x, loc,
                                      3, P->d_nrm, nullptr, nullptr, 0.0, 2, out, 3, st, spec));
        }
    });
}

}  // namespace

void ggem::single_layer_dev(ggem_plan_t* P, const double* q, double* w) {
    if (P->fp64) layer_impl<double>(P, 0, q, w);
    else layer_impl<float>(P, 0, q, w);
}

void ggem::double_layer_dev(ggem_plan_t* P, const double* q, double* v) {
    if (P->fp64) layer_impl<double>(P, 1, q, v);
    else layer_impl<float>(P, 1, q, v);
}

namespace {

template <typename T>
void upload_tables(ggem_plan_t* P, const std::vector<double>& cf, const std::vector<double>& ci,
                   const std::vector<double>& twx, const std::vector<double>& twz) {
    std::vector<T> a(cf.begin(), cf.end()), b(ci.begin(), ci.end());
    std::vector<T> c(twx.begin(), twx.end()), d(twz.begin(), twz.end());
    dalloc(P, (T**)&P->d_cheb_fwd, a.size());
    dalloc(P, (T**)&P->d_cheb_inv, b.size());
    dalloc(P, (T**)&P->d_tw_x, c.size());
    dalloc(P, (T**)&P->d_tw_z, d.size());
    GG_CUDA(cudaMemcpy(P->d_cheb_fwd, a.data(), a.size() * sizeof(T), cudaMemcpyHostToDevice));
    GG_CUDA(cudaMemcpy(P->d_cheb_inv, b.data(), b.size() * sizeof(T), cudaMemcpyHostToDevice));
    if (sizeof(T) == 4) {
        // split-bf16 copies for the tensor-core transforms
        const int Ny = P->prm.Ny;
        const size_t nb = cheb_tc_prep_bytes(Ny);
        GG_CUDA(cudaMalloc(&P->d_tc_fwd, nb));
        GG_CUDA(cudaMalloc(&P->d_tc_inv, nb));
        GG_CUDA(cheb_tc_prepare(Ny, (const float*)P->d_cheb_fwd, P->d_tc_fwd, 0));
        GG_CUDA(cheb_tc_prepare(Ny, (const float*)P->d_cheb_inv, P->d_tc_inv, 0));
        GG_CUDA(cudaDeviceSynchronize());
    }
    GG_CUDA(cudaMemcpy(P->d_tw_x, c.data(), c.size() * sizeof(T), cudaMemcpyHostToDevice));
    GG_CUDA(cudaMemcpy(P->d_tw_z, d.data(), d.size() * sizeof(T), cudaMemcpyHostToDevice));
}

// Oversampled grid, its FFT tables and the deconvolution factors of the
// spectral off-grid evaluation with window half-width w.  In x (and z) the
// factor of mode l is 1 / (M ghat(l)), ghat(l) = sqrt(tau/pi) exp(-l^2 tau)
// the Fourier coefficient of the periodised window and 1/M the trapezoidal
// weight of the gather on M fine nodes; Nyquist modes get 0.  In theta the
// Chebyshev series sum a_n cos(n theta) has frequencies |n| <= N = Ny - 1, so
// 2N modes oversampled 2x give Mt = 4N nodes over [0, 2 pi), of which the
// 2N + 1 in [0, pi] are stored (the series is even); the deconvolution of
// degree n is folded into the matrix taking the coefficients to those nodes.
template <typename T>
void spec_setup(ggem_plan_t* P, int w) {
    const int Nx = P->prm.Nx, Nz = P->prm.Nz, Ny = P->prm.Ny;
    const int Mx = 2 * Nx, Mz = 2 * Nz, N = Ny - 1, Mt = 4 * N, nth = 2 * N + 1;
    if (!P->d_spec) {
        // up to 9 components: velocity and stress of ggem_point_forces
        dalloc(P, (T**)&P->d_spec, (size_t)nth * 9 * Mz * Mx);
        dalloc(P, (T**)&P->d_spec_mid, (size_t)nth * 9 * Nz * Nx);
        std::vector<double> twx, twz;
        fft_tables(Mx, Mz, twx, twz);
        std::vector<T> a(twx.begin(), twx.end()), b(twz.begin(), twz.end());
        dalloc(P, (T**)&P->d_spec_twx, a.size());
        dalloc(P, (T**)&P->d_spec_twz, b.size());
        GG_CUDA(cudaMemcpy(P->d_spec_twx, a.data(), a.size() * sizeof(T),
                           cudaMemcpyHostToDevice));
        GG_CUDA(cudaMemcpy(P->d_spec_twz, b.data(), b.size() * sizeof(T),
                           cudaMemcpyHostToDevice));
        dalloc(P, (T**)&P->d_spec_dx, (size_t)Nx / 2);
        dalloc(P, (T**)&P->d_spec_dz, (size_t)Nz);
        dalloc(P, (T**)&P->d_spec_ct, (size_t)nth * Ny);
    }
    if (w == P->spec_w) return;
    const double den = kSpecR * (kSpecR - 0.5);
    const double taux = kPi * w / ((double)Nx * Nx * den);
    const double tauz = kPi * w / ((double)Nz * Nz * den);
    const double taut = kPi * w / (4.0 * N * N * den);
    std::vector<T> dx(Nx / 2), dz(Nz), ct((size_t)nth * Ny);
    for (int l = 0; l < Nx / 2; ++l)
        dx[l] = (T)(std::sqrt(kPi / taux) * std::exp((double)l * l * taux) / Mx);
    for (int k = 0; k < Nz; ++k) {
        const int m = k < Nz / 2 ? k : k - Nz;
        dz[k] = k == Nz / 2 ? (T)0
                            : (T)(std::sqrt(kPi / tauz) * std::exp((double)m * m * tauz) / Mz);
    }
    for (int p = 0; p < nth; ++p)
        for (int n = 0; n < Ny; ++n) {
            const double d = std::sqrt(kPi / taut) * std::exp((double)n * n * taut) / Mt;
            const double th = 2.0 * kPi * (double)((long)n * p % Mt) / Mt;
            ct[(size_t)p * Ny + n] = (T)(d * std::cos(th));
        }
    GG_CUDA(cudaStreamSynchronize(P->st));     // no launch may still read the old factors
    GG_CUDA(cudaMemcpy(P->d_spec_dx, dx.data(), dx.size() * sizeof(T), cudaMemcpyHostToDevice));
    GG_CUDA(cudaMemcpy(P->d_spec_dz, dz.data(), dz.size() * sizeof(T), cudaMemcpyHostToDevice));
    GG_CUDA(cudaMemcpy(P->d_spec_ct, ct.data(), ct.size() * sizeof(T), cudaMemcpyHostToDevice));
    P->spec_w = w;
}

void plan_build(ggem_plan_t* P, const ggem_params& prm) {
    P->prm = prm;
    GG_CHECK(is_pow2(prm.Nx) && is_pow2(prm.Nz) && prm.Nx >= 16 && prm.Nz >= 16 &&
                 prm.Nx <= 1024 && prm.Nz <= 1024,
             GGEM_ERR_INVALID_ARG, "Nx and Nz must be powers of two in [16, 1024]");
    GG_CHECK(prm.Ny >= 9 && prm.Ny <= 257, GGEM_ERR_INVALID_ARG, "Ny must lie in [9, 257]");
    GG_CHECK(prm.Lx > 0 && prm.Lz > 0 && prm.W > 0 && prm.mu > 0, GGEM_ERR_INVALID_ARG,
             "Lx, Lz, W and mu must be positive");
    GG_CHECK(prm.precision == GGEM_FP64 || prm.precision == GGEM_MIXED ||
                 prm.precision == GGEM_FP64_EMULATED,
             GGEM_ERR_INVALID_ARG, "precision must be GGEM_FP64, GGEM_MIXED or GGEM_FP64_EMULATED");
    GG_CHECK(prm.quadrature == GGEM_NODAL || prm.quadrature == GGEM_ELEMENT,
             GGEM_ERR_INVALID_ARG, "quadrature must be GGEM_NODAL or GGEM_ELEMENT");
    GG_CHECK(prm.max_points > 0 && prm.max_tris >= 0, GGEM_ERR_INVALID_ARG,
             "max_points must be positive");
    GridGeom& g = P->geo;
    g.Lx = prm.Lx; g.Lz = prm.Lz; g.W = prm.W; g.y0 = prm.y0;
    g.Nx = prm.Nx; g.Ny = prm.Ny; g.Nz = prm.Nz; g.nkx = prm.Nx / 2;
    g.dx = prm.Lx / prm.Nx; g.dz = prm.Lz / prm.Nz;
    g.mu = prm.mu;
    double h = std::fmax(std::fmax(g.dx, prm.W / (prm.Ny - 1)), g.dz);
    g.alpha = prm.alpha > 0 ? prm.alpha : 1.0 / (2.0 * h);
    double rf = prm.rcut_factor > 0 ? prm.rcut_factor : 4.0;
    g.rcut = rf / g.alpha;
    GG_CHECK(g.alpha * prm.Lx > 2 * rf && g.alpha * prm.Lz > 2 * rf, GGEM_ERR_INVALID_ARG,
             "alpha*L must exceed 2*rcut_factor (r_cut below half the period)");
    P->fp64 = prm.precision != GGEM_MIXED;
    P->ff = prm.precision == GGEM_FP64_EMULATED && prm.quadrature == GGEM_ELEMENT;
    P->nmodes = prm.Nz * g.nkx;
    CellGrid& cg = P->cg;
    // cells at least r_cut/R wide; the local sums search +-R cells and keep
    // those within r_cut of each target.  R = 3 for the element rule (dense
    // quadrature points: smaller cells cut the candidates), 2 for nodal sources
    cg.reach = prm.quadrature == GGEM_ELEMENT ? 3 : 2;
    cg.ncx = std::max(1, (int)std::floor(prm.Lx / (g.rcut / cg.reach)));
    cg.ncz = std::max(1, (int)std::floor(prm.Lz / (g.rcut / cg.reach)));
    cg.ncy = std::max(1, (int)std::floor(prm.W / (g.rcut / cg.reach)));
    cg.hx = prm.Lx / cg.ncx; cg.hz = prm.Lz / cg.ncz; cg.hy = prm.W / cg.ncy;
    cg.y0 = prm.y0;
    P->ncell = cg.ncx * cg.ncy * cg.ncz;

    const int Ny = prm.Ny, N = Ny - 1;
    std::vector<double> yj(Ny), cf((size_t)Ny * Ny), ci((size_t)Ny * Ny);
    for (int j = 0; j < Ny; ++j) yj[j] = prm.y0 + 0.5 * prm.W * (1.0 + std::cos(kPi * j / N));
    double inxz = 1.0 / ((double)prm.Nx * prm.Nz);
    for (int n = 0; n < Ny; ++n)
        for (int j = 0; j < Ny; ++j) {
            double cn = (n == 0 || n == N) ? 2.0 : 1.0, cj = (j == 0 || j == N) ? 2.0 : 1.0;
            double c = std::cos(kPi * ((long)n * j % (2 * N)) / N);
            cf[(size_t)n * Ny + j] = 2.0 / (N * cn * cj) * c * inxz;
            ci[(size_t)j * Ny + n] = c;
        }
    std::vector<double> twx, twz;
    fft_tables(prm.Nx, prm.Nz, twx, twz);
    dalloc(P, &P->d_yj, Ny);
    GG_CUDA(cudaMemcpy(P->d_yj, yj.data(), Ny * sizeof(double), cudaMemcpyHostToDevice));
    {
        std::vector<double> yd((size_t)Ny * Ny);
        for (int j = 0; j < Ny; ++j)
            for (int k = 0; k < Ny; ++k) yd[(size_t)j * Ny + k] = yj[j] - yj[k];
        if (P->fp64) {
            dalloc(P, (double**)&P->d_ydiff, yd.size());
            GG_CUDA(cudaMemcpy(P->d_ydiff, yd.data(), yd.size() * sizeof(double),
                               cudaMemcpyHostToDevice));
        } else {
            std::vector<float> yf(yd.begin(), yd.end());
            dalloc(P, (float**)&P->d_ydiff, yf.size());
            GG_CUDA(cudaMemcpy(P->d_ydiff, yf.data(), yf.size() * sizeof(float),
                               cudaMemcpyHostToDevice));
        }
    }
    if (P->fp64) upload_tables<double>(P, cf, ci, twx, twz);
    else upload_tables<float>(P, cf, ci, twx, twz);

    // per-mode homogeneous solutions and inverse influence matrices (App. C)
    const int nm = P->nmodes;
    std::vector<double> ksb((size_t)3 * Ny * nm, 0.0), minv((size_t)4 * nm, 0.0);
    std::vector<double> thom((size_t)4 * Ny * nm, 0.0), isq((size_t)2 * nm, 0.0);
    std::vector<double> kschunk((size_t)48 * nm, 0.0);
#pragma omp parallel
    {
        std::vector<double> pb(Ny), ph(Ny), vb(Ny), th(4 * Ny);
        double mi[4], iq[2];
#pragma omp for schedule(dynamic, 64)
        for (int m = 0; m < nm; ++m) {
            int kzi = m / g.nkx, kxi = m % g.nkx;
            if (kzi == prm.Nz / 2) continue;
            int mz = kzi < prm.Nz / 2 ? kzi : kzi - prm.Nz;
            double kx = 2 * kPi * kxi / prm.Lx, kz = 2 * kPi * mz / prm.Lz;
            double k2 = kx * kx + kz * kz;
            ks_thomas_mode(Ny, k2 * 0.25 * prm.W * prm.W, th.data(), iq);
            for (int c = 0; c < 4; ++c)
                for (int n = 0; n < Ny; ++n) thom[((size_t)c * Ny + n) * nm + m] = th[c * Ny + n];
            ks_chunk_mode(Ny, th.data(), kschunk.data() + (size_t)48 * m);
            isq[m] = iq[0];
            isq[nm + m] = iq[1];
            if (m == 0) continue;
            ks_precompute_mode(Ny, prm.W, prm.mu, k2, pb.data(), ph.data(), vb.data(), mi);
            for (int n = 0; n < Ny; ++n) {
                ksb[((size_t)0 * Ny + n) * nm + m] = pb[n];
                ksb[((size_t)1 * Ny + n) * nm + m] = ph[n];
                ksb[((size_t)2 * Ny + n) * nm + m] = vb[n];
            }
            for (int c = 0; c < 4; ++c) minv[(size_t)c * nm + m] = mi[c];
        }
    }
    dalloc(P, &P->d_thom, thom.size());
    dalloc(P, &P->d_isq, isq.size());
    GG_CUDA(cudaMemcpy(P->d_thom, thom.data(), thom.size() * sizeof(double),
                       cudaMemcpyHostToDevice));
    GG_CUDA(cudaMemcpy(P->d_isq, isq.data(), isq.size() * sizeof(double),
                       cudaMemcpyHostToDevice));
    dalloc(P, &P->d_kschunk, kschunk.size());
    GG_CUDA(cudaMemcpy(P->d_kschunk, kschunk.data(), kschunk.size() * sizeof(double),
                       cudaMemcpyHostToDevice));
    // the homogeneous solutions in the plan's precision: the tau kernel adds
    // them in T
    if (P->fp64) {
        dalloc(P, (double**)&P->d_ksb, ksb.size());
        GG_CUDA(cudaMemcpy(P->d_ksb, ksb.data(), ksb.size() * sizeof(double),
                           cudaMemcpyHostToDevice));
    } else {
        std::vector<float> kf(ksb.begin(), ksb.end());
        dalloc(P, (float**)&P->d_ksb, kf.size());
        GG_CUDA(cudaMemcpy(P->d_ksb, kf.data(), kf.size() * sizeof(float),
                           cudaMemcpyHostToDevice));
    }
    dalloc(P, &P->d_minv, minv.size());
    GG_CUDA(cudaMemcpy(P->d_minv, minv.data(), minv.size() * sizeof(double),
                       cudaMemcpyHostToDevice));

    // workspaces
    size_t esz = P->fp64 ? sizeof(double) : sizeof(float);
    P->grid_elems = (size_t)9 * Ny * prm.Nz * prm.Nx;
    GG_CUDA(cudaMalloc(&P->d_gridA, P->grid_elems * esz));
    GG_CUDA(cudaMalloc(&P->d_gridB, P->grid_elems * esz));
    GG_CUDA(cudaMalloc(&P->d_wall, (size_t)6 * prm.Nz * prm.Nx * esz));
    {
        std::vector<double> tab(3 * Ny);
        ks_coef_table(Ny, tab.data());
        dalloc(P, &P->d_kscoef, tab.size());
        GG_CUDA(cudaMemcpy(P->d_kscoef, tab.data(), tab.size() * sizeof(double),
                           cudaMemcpyHostToDevice));
    }
    int cap = prm.max_points;
    P->cap = cap;
    dalloc(P, &P->d_cell_count, P->ncell);
    dalloc(P, &P->d_cell_start, P->ncell + 1);
    dalloc(P, &P->d_tc_err, 1);
    dalloc(P, &P->d_spread_list, (size_t)cap + 1);
    GG_CUDA(cudaMemset(P->d_tc_err, 0, sizeof(int)));
    {
        int dev = 0;
        GG_CUDA(cudaGetDevice(&dev));
        GG_CUDA(cudaDeviceGetAttribute(&P->nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    dalloc(P, &P->d_cursor, (size_t)P->ncell + std::max<size_t>(cap, (size_t)16 * prm.max_tris));
    dalloc(P, &P->d_src_cell, cap);
    dalloc(P, &P->d_perm, cap);
    size_t v4 = P->fp64 ? sizeof(double4_32a) : sizeof(float4);
    GG_CUDA(cudaMalloc(&P->d_spos, cap * v4 + 32));
    GG_CUDA(cudaMalloc(&P->d_sg, cap * v4 + 32));
    GG_CUDA(cudaMalloc(&P->d_local, (size_t)cap * 9 * esz + 32));
    dalloc(P, &P->d_in0, (size_t)cap * 3);
    dalloc(P, &P->d_in1, (size_t)cap * 3);
    dalloc(P, &P->d_in2, (size_t)cap * 3);
    dalloc(P, &P->d_out0, (size_t)cap * 3);
    dalloc(P, &P->d_out1, (size_t)cap * 6);
    dalloc(P, &P->d_tgt_cell, cap);
    dalloc(P, &P->d_sdi, cap);
    dalloc(P, &P->d_mesh_sdi, cap);
    GG_CUDA(cudaMalloc(&P->d_sdf, cap * v4 + 32));
    GG_CUDA(cudaMalloc(&P->d_mesh_sdf, cap * v4 + 32));
    GG_CUDA(cudaMalloc(&P->d_tgt_pos, cap * v4 + 32));
    {
        int nw = 2 * prm.Nz * prm.Nx;
        dalloc(P, &P->d_wall_cell, nw);
        GG_CUDA(cudaMalloc(&P->d_wall_pos, nw * v4 + 32));
        if (P->fp64)
            GG_CUDA(locate_targets<double>(g, cg, nw, TK_WALL, nullptr, P->d_wall_cell,
                                           (double4_32a*)P->d_wall_pos, nullptr));
        else
            GG_CUDA(locate_targets<float>(g, cg, nw, TK_WALL, nullptr, P->d_wall_cell,
                                          (float4*)P->d_wall_pos, nullptr));
    }
    // mesh tables
    P->cap_tris = prm.max_tris;
    dalloc(P, &P->d_x, (size_t)cap * 3);
    dalloc(P, &P->d_area, cap);
    dalloc(P, &P->d_nrm, (size_t)cap * 3);
    dalloc(P, &P->d_mesh_cell, cap);
    dalloc(P, &P->d_mesh_perm, cap);
    dalloc(P, &P->d_mesh_start, P->ncell + 1);
    GG_CUDA(cudaMalloc(&P->d_mesh_pos, cap * v4 + 32));
    if (prm.max_tris > 0) {
        dalloc(P, &P->d_tri, (size_t)prm.max_tris * 3);
        dalloc(P, &P->d_tri_area, prm.max_tris);
        dalloc(P, &P->d_tri_nrm, (size_t)prm.max_tris * 3);
        dalloc(P, &P->d_adj_cnt, cap);
        dalloc(P, &P->d_adj_start, (size_t)cap + 1);
        dalloc(P, &P->d_adj_cur, cap);
        dalloc(P, &P->d_adj, (size_t)prm.max_tris * 3);
    }
    P->rule = make_quad_rule();
    if (prm.quadrature == GGEM_ELEMENT && prm.max_tris > 0) {
        size_t cq = (size_t)16 * prm.max_tris;
        GG_CHECK(cq < (size_t)1 << 31, GGEM_ERR_CAPACITY, "too many quadrature points");
        P->cap_qp = (int)cq;
        dalloc(P, &P->d_qx, cq * 3);
        dalloc(P, &P->d_qv, cq);
        dalloc(P, &P->d_qv_sorted, cq);
        GG_CUDA(cudaMalloc(&P->d_qw, cq * v4 + 32));
        dalloc(P, &P->d_qp_cell, cq);
        dalloc(P, &P->d_qp_perm, cq);
        dalloc(P, &P->d_qp_start, (size_t)P->ncell + 1);
        GG_CUDA(cudaMalloc(&P->d_qp_pos, cq * v4 + 32));
        GG_CUDA(cudaMalloc(&P->d_qg, cq * v4 + 32));
        if (P->ff) {                       // float-pair copies: [point][hi, lo] float4
            GG_CUDA(cudaMalloc(&P->d_qp_ff, cq * 2 * sizeof(float4) + 32));
            GG_CUDA(cudaMalloc(&P->d_qg_ff, cq * 2 * sizeof(float4) + 32));
        }
        if (!P->fp64) {                    // padded planes; grown at mesh_set if needed
            P->soa_ld = (cq + cq / 8 + 64 + 63) / 64 * 64;
            dalloc(P, &P->d_qp_pack, 6 * P->soa_ld);
            dalloc(P, &P->d_qp_inv, P->soa_ld);
            dalloc(P, &P->d_qp_pstart, (size_t)P->ncell + 1);
            dalloc(P, &P->d_q32, (size_t)3 * cap);
        }
    }
    GG_CUDA(cudaEventCreate(&P->ev0));
    GG_CUDA(cudaEventCreate(&P->ev1));
    {
        int least = 0, greatest = 0;
        GG_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        GG_CUDA(cudaStreamCreateWithPriority(&P->st2, cudaStreamNonBlocking, greatest));
    }
    GG_CUDA(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
    GG_CUDA(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
    GG_CUDA(cudaDeviceSynchronize());
}

void plan_free(ggem_plan_t* P) {
    if (P->ev0) cudaEventDestroy(P->ev0);
    if (P->ev1) cudaEventDestroy(P->ev1);
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->ev_join) cudaEventDestroy(P->ev_join);
    if (P->st2) {
        cudaStreamSynchronize(P->st2);
        cudaStreamDestroy(P->st2);
    }
    void* ptrs[] = {P->d_yj, P->d_cheb_fwd, P->d_cheb_inv, P->d_tw_x, P->d_tw_z, P->d_ksb,
                    P->d_minv, P->d_ydiff, P->d_sdi, P->d_sdf, P->d_mesh_sdi, P->d_mesh_sdf,
                    P->d_kscoef, P->d_thom, P->d_kschunk, P->d_isq, P->d_gridA, P->d_gridB, P->d_wall,
                    P->d_cell_count, P->d_cell_start, P->d_cursor, P->d_src_cell,
                    P->d_perm, P->d_spos, P->d_sg, P->d_src_x, P->d_local, P->d_in0, P->d_in1,
                    P->d_in2, P->d_out0, P->d_out1, P->d_tgt_cell, P->d_tgt_pos,
                    P->d_wall_cell, P->d_wall_pos, P->d_x, P->d_tri, P->d_area, P->d_nrm,
                    P->d_tri_area, P->d_tri_nrm, P->d_mesh_cell, P->d_mesh_perm,
                    P->d_mesh_start, P->d_mesh_pos, P->d_qx, P->d_qv, P->d_qw, P->d_qp_cell,
                    P->d_qp_perm, P->d_qp_start, P->d_qp_pos, P->d_qg, P->d_adj_cnt,
                    P->d_adj_start, P->d_adj_cur, P->d_adj,
                    P->d_qv_sorted, P->d_V, P->d_sv, P->d_sb, P->d_sk, P->d_sx,
                    P->d_spart, P->d_sh, P->d_particle, P->d_pcount, P->d_feat,
                    P->d_mlp, P->d_mlp_grad, P->d_mlp_m, P->d_mlp_v, P->d_mlp_wf,
                    P->d_mlp_wt, P->d_mlp_stats, P->d_mlp_out, P->d_smlp,
                    P->d_sres, P->d_mlp_dr, P->d_mlp_ssq, P->d_tc_err,
                    P->d_tc_fwd, P->d_tc_inv, P->d_spread_list, P->d_pstart,
                    P->d_pnodes, P->d_rc, P->d_rscale, P->d_mref, P->d_cx0, P->d_cdf,
                    P->d_cuinf, P->d_cfinf, P->d_cb, P->d_ckap, P->d_clam, P->d_cw, P->d_cq,
                    P->d_cmin, P->d_tstart, P->d_tlist, P->d_cvol, P->d_orec, P->d_orecd,
                    P->d_ocount, P->d_odisp, P->d_qp_ff, P->d_qg_ff, P->d_qp_pack,
                    P->d_spec, P->d_spec_twx, P->d_spec_twz, P->d_spec_dx,
                    P->d_spec_dz, P->d_spec_mid, P->d_spec_ct, P->d_mlp_tc,
                    P->d_mlp_tcs, P->d_qp_pstart, P->d_qp_inv, P->d_q32};
    for (void* p : ptrs) dfree(p);
    precond_free(P);
    dfree(P->d_pc_Zb);
    if (P->h_sh) cudaFreeHost(P->h_sh);
    if (P->twin) ggem_plan_destroy(P->twin);
}

}  // namespace

// =================================================================== ABI
extern "C" {

ggem_status ggem_plan(const ggem_params* params, void* stream, ggem_plan_t** out) {
    if (!out) return GGEM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params) return GGEM_ERR_INVALID_ARG;
    ggem_plan_t* P = new (std::nothrow) ggem_plan_t();
    if (!P) return GGEM_ERR_CAPACITY;
    P->st = (cudaStream_t)stream;
    ggem_status s = guarded(P, [&] { plan_build(P, *params); });
    if (s != GGEM_OK) {
        g_create_error = P->err;
        plan_free(P);
        delete P;
        return s;
    }
    *out = P;
    return GGEM_OK;
}

ggem_status ggem_plan_destroy(ggem_plan_t* P) {
    if (!P) return GGEM_OK;
    cudaStreamSynchronize(P->st);
    plan_free(P);
    delete P;
    return GGEM_OK;
}

const char* ggem_last_error(const ggem_plan_t* P) {
    if (!P) return g_create_error.c_str();
    return P->err.c_str();
}

ggem_status ggem_set_offgrid(ggem_plan_t* P, int mode, int half_width) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(mode == GGEM_OFFGRID_LAGRANGE || mode == GGEM_OFFGRID_SPECTRAL,
                 GGEM_ERR_INVALID_ARG, "mode must be GGEM_OFFGRID_LAGRANGE or _SPECTRAL");
        GG_CHECK(half_width == 0 || (half_width >= 2 && half_width <= 16), GGEM_ERR_INVALID_ARG,
                 "half_width must be 0 (default) or in [2, 16]");
        if (mode == GGEM_OFFGRID_SPECTRAL) {
            const int w = half_width ? half_width : (P->fp64 ? 12 : 6);
            if (P->fp64) spec_setup<double>(P, w);
            else spec_setup<float>(P, w);
        }
        P->offgrid = mode;
        if (P->twin) {
            ggem_status ts = ggem_set_offgrid(P->twin, mode, 0);
            GG_CHECK(ts == GGEM_OK, ts, std::string("FP64 twin: ") + ggem_last_error(P->twin));
        }
    });
}

ggem_status ggem_plan_info(const ggem_plan_t* P, double* alpha, double* rcut) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    if (alpha) *alpha = P->geo.alpha;
    if (rcut) *rcut = P->geo.rcut;
    return GGEM_OK;
}

ggem_status ggem_mesh_set(ggem_plan_t* P, int n_nodes, const double* x, int n_tris,
                          const int* tri) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(n_nodes > 0 && x, GGEM_ERR_INVALID_ARG, "mesh needs nodes");
        GG_CHECK(n_nodes <= P->cap, GGEM_ERR_CAPACITY, "more nodes than max_points");
        GG_CHECK(n_tris >= 0 && n_tris <= P->cap_tris, GGEM_ERR_CAPACITY,
                 "more triangles than max_tris");
        GG_CHECK(n_tris == 0 || tri, GGEM_ERR_INVALID_ARG, "triangles pointer is NULL");
        P->mesh_ready = false;         // until the new mesh has passed every check
        cudaStream_t st = P->st;
        auto kind = [](const void* p) {
            return is_device_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        };
        // (the plan's own arrays may be passed back: nothing to copy then)
        if (x != P->d_x)
            GG_CUDA(cudaMemcpyAsync(P->d_x, x, (size_t)n_nodes * 3 * sizeof(double), kind(x),
                                    st));
        if (n_tris > 0 && tri != P->d_tri) {
            GG_CUDA(cudaMemcpyAsync(P->d_tri, tri, (size_t)n_tris * 3 * sizeof(int), kind(tri),
                                    st));
            P->mref_ready = false;     // new connectivity: the membrane reference and the
            P->tcsr_ready = false;     // per-particle triangle lists no longer apply
        }
        int* bad = P->d_cell_count;   // scratch int
        GG_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
        k_check_inside<<<(n_nodes + 255) / 256, 256, 0, st>>>(n_nodes, P->d_x, P->geo.y0,
                                                             P->geo.W, bad);
        int hbad = 0;
        GG_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        GG_CUDA(cudaStreamSynchronize(st));
        GG_CHECK(hbad == 0, GGEM_ERR_INVALID_ARG,
                 "mesh nodes must be finite and lie strictly inside the slit");
        GG_CUDA(cudaMemsetAsync(P->d_area, 0, (size_t)n_nodes * sizeof(double), st));
        GG_CUDA(cudaMemsetAsync(P->d_nrm, 0, (size_t)n_nodes * 3 * sizeof(double), st));
        if (n_tris > 0) {
            k_tri_geom<<<(n_tris + 255) / 256, 256, 0, st>>>(n_tris, P->d_x, P->d_tri,
                                                             P->d_tri_area, P->d_tri_nrm,
                                                             P->d_area, P->d_nrm);
            k_normalize<<<(n_nodes + 255) / 256, 256, 0, st>>>(n_nodes, P->d_nrm);
        }
        GG_CUDA(cudaGetLastError());
        if (P->fp64) {
            GG_CUDA(build_cells<double>(P->geo, P->cg, n_nodes, P->d_x, P->d_cell_count,
                                        P->d_mesh_start, P->d_cursor, P->d_mesh_cell,
                                        P->d_mesh_perm, (double4_32a*)P->d_mesh_pos, st));
            GG_CUDA(spread_prepare<double>(P->geo, P->d_yj, n_nodes, P->d_mesh_perm, P->d_x,
                                           P->d_mesh_sdi, (double4_32a*)P->d_mesh_sdf, st));
        } else {
            GG_CUDA(build_cells<float>(P->geo, P->cg, n_nodes, P->d_x, P->d_cell_count,
                                       P->d_mesh_start, P->d_cursor, P->d_mesh_cell,
                                       P->d_mesh_perm, (float4*)P->d_mesh_pos, st));
            GG_CUDA(spread_prepare<float>(P->geo, P->d_yj, n_nodes, P->d_mesh_perm, P->d_x,
                                          P->d_mesh_sdi, (float4*)P->d_mesh_sdf, st));
        }
        const bool elem = P->prm.quadrature == GGEM_ELEMENT && n_tris > 0;
        if (n_tris > 0) {
            // node -> triangle adjacency (element correction, ring features) and,
            // in element-rule plans, the quadrature points
            if (elem)
                GG_CHECK(P->d_qx && P->d_qv && P->d_qw, GGEM_ERR_INVALID_ARG,
                         "element buffers missing");
            if (P->fp64)
                GG_CUDA(elem_setup<double>(n_tris, P->d_x, P->d_tri, P->d_tri_area, P->rule,
                                           elem ? P->d_qx : nullptr, P->d_qv,
                                           (double4_32a*)P->d_qw, n_nodes, P->d_adj_cnt,
                                           P->d_adj_start, P->d_adj_cur, P->d_adj, st));
            else
                GG_CUDA(elem_setup<float>(n_tris, P->d_x, P->d_tri, P->d_tri_area, P->rule,
                                          elem ? P->d_qx : nullptr, P->d_qv, (float4*)P->d_qw,
                                          n_nodes, P->d_adj_cnt, P->d_adj_start, P->d_adj_cur,
                                          P->d_adj, st));
        }
        P->n_qp = 0;
        if (elem) {
            double* dmax = P->d_out0;   // scratch
            GG_CUDA(cudaMemsetAsync(dmax, 0, sizeof(double), st));
            k_max_edge<<<(n_tris + 255) / 256, 256, 0, st>>>(n_tris, P->d_x, P->d_tri, dmax);
            GG_CUDA(cudaMemcpyAsync(&P->near_edge, dmax, sizeof(double), cudaMemcpyDeviceToHost,
                                    st));
            GG_CUDA(cudaStreamSynchronize(st));
            int nq = 16 * n_tris;
            if (P->fp64) {
                GG_CUDA(build_cells<double>(P->geo, P->cg, nq, P->d_qx, P->d_cell_count,
                                            P->d_qp_start, P->d_cursor, P->d_qp_cell,
                                            P->d_qp_perm, (double4_32a*)P->d_qp_pos, st));
                if (P->ff) GG_CUDA(to_float_pairs(nq, P->d_qp_pos, P->d_qp_ff, st));
            } else {
                GG_CUDA(build_cells<float>(P->geo, P->cg, nq, P->d_qx, P->d_cell_count,
                                           P->d_qp_start, P->d_cursor, P->d_qp_cell,
                                           P->d_qp_perm, (float4*)P->d_qp_pos, st));
                // within-cell order (scratch: the strength buffer and the cursors,
                // both free until the first evaluation)
                GG_CUDA(cell_subsort(P->cg, nq, P->ncell, P->d_qp_start, (float4*)P->d_qp_pos,
                                     P->d_qp_perm, (float4*)P->d_qg, P->d_cursor, st));
                // padded layout: whole 64-point steps per cell (the cursors as
                // scratch for the padded counts); the planes grow if it needs more
                GG_CUDA(pad_layout_counts(P->ncell, P->d_qp_start, P->d_cursor, P->d_qp_pstart,
                                          st));
                int np = 0;
                GG_CUDA(cudaMemcpyAsync(&np, P->d_qp_pstart + P->ncell, sizeof(int),
                                        cudaMemcpyDeviceToHost, st));
                GG_CUDA(cudaStreamSynchronize(st));
                if ((size_t)np + 64 > P->soa_ld) {
                    dfree(P->d_qp_pack);
                    dfree(P->d_qp_inv);
                    P->d_qp_pack = nullptr;
                    P->d_qp_inv = nullptr;
                    P->soa_ld = ((size_t)np + (size_t)np / 8 + 64 + 63) / 64 * 64;
                    dalloc(P, &P->d_qp_pack, 6 * P->soa_ld);
                    dalloc(P, &P->d_qp_inv, P->soa_ld);
                }
                GG_CUDA(pad_layout_fill(nq, P->soa_ld, P->d_qp_cell, P->d_qp_start,
                                        P->d_qp_pstart, (const float4*)P->d_qp_pos,
                                        P->geo.alpha, P->d_qp_pack, P->d_qp_inv, st));
                P->qp_np = np;
            }
            GG_CUDA(gather_int4(nq, P->d_qp_perm, P->d_qv, P->d_qv_sorted, st));
            // weights into point order too (scratch: the strength buffer)
            if (P->fp64)
                GG_CUDA(qp_sort_weights<double>(nq, P->d_qp_perm, (double4_32a*)P->d_qw,
                                                (double4_32a*)P->d_qg, st));
            else
                GG_CUDA(qp_sort_weights<float>(nq, P->d_qp_perm, (float4*)P->d_qw,
                                               (float4*)P->d_qg, st));
            P->n_qp = nq;
        }
        P->n_nodes = n_nodes;
        P->n_tris = n_tris;
        P->mesh_ready = true;
        GG_CUDA(cudaStreamSynchronize(st));
        if (P->twin) {                 // the FP64 twin of a mixed plan follows the mesh
            ggem_status ts = ggem_mesh_set(P->twin, n_nodes, P->d_x, n_tris, P->d_tri);
            GG_CHECK(ts == GGEM_OK, ts, std::string("FP64 twin: ") + ggem_last_error(P->twin));
        }
    });
}

ggem_status ggem_mesh_geometry(ggem_plan_t* P, double* area, double* normal) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready, GGEM_ERR_INVALID_ARG, "no mesh set");
        int n = P->n_nodes;
        if (area)
            GG_CUDA(cudaMemcpyAsync(area, P->d_area, n * sizeof(double), cudaMemcpyDefault,
                                    P->st));
        if (normal)
            GG_CUDA(cudaMemcpyAsync(normal, P->d_nrm, (size_t)n * 3 * sizeof(double),
                                    cudaMemcpyDefault, P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));
    });
}

ggem_status ggem_point_forces(ggem_plan_t* P, int n_src, const double* x_src, const double* g,
                              int n_tgt, const double* x_tgt, int tgt_is_src, double* u,
                              double* sigma) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(n_src >= 0 && n_src <= P->cap, GGEM_ERR_CAPACITY, "n_src exceeds max_points");
        GG_CHECK(n_src == 0 || (x_src && g), GGEM_ERR_INVALID_ARG, "NULL source arrays");
        if (tgt_is_src) n_tgt = n_src;
        GG_CHECK(n_tgt >= 0 && n_tgt <= P->cap, GGEM_ERR_CAPACITY, "n_tgt exceeds max_points");
        GG_CHECK(tgt_is_src || n_tgt == 0 || x_tgt, GGEM_ERR_INVALID_ARG, "NULL target array");
        if (!u && !sigma) return;
        const double* xs = stage_in(P, x_src, P->d_in0, (size_t)n_src * 3);
        const double* gd = stage_in(P, g, P->d_in1, (size_t)n_src * 3);
        const double* xt = tgt_is_src ? xs : stage_in(P, x_tgt, P->d_in2, (size_t)n_tgt * 3);
        OutMap mu_ = stage_out(u, P->d_out0, (size_t)n_tgt * 3);
        OutMap ms_ = stage_out(sigma, P->d_out1, (size_t)n_tgt * 6);
        if (P->fp64)
            point_forces_impl<double>(P, n_src, xs, gd, n_tgt, xt, tgt_is_src, mu_.dev, ms_.dev);
        else
            point_forces_impl<float>(P, n_src, xs, gd, n_tgt, xt, tgt_is_src, mu_.dev, ms_.dev);
        finish_out(P, mu_);
        finish_out(P, ms_);
        if (mu_.host || ms_.host) GG_CUDA(cudaStreamSynchronize(P->st));
    });
}

ggem_status ggem_local_sum(ggem_plan_t* P, int n_src, const double* x_src, const double* g,
                           int n_tgt, const double* x_tgt, int tgt_is_src, double* u,
                           double* sigma) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(n_src >= 0 && n_src <= P->cap, GGEM_ERR_CAPACITY, "n_src exceeds max_points");
        GG_CHECK(n_src == 0 || (x_src && g), GGEM_ERR_INVALID_ARG, "NULL source arrays");
        if (tgt_is_src) n_tgt = n_src;
        GG_CHECK(n_tgt >= 0 && n_tgt <= P->cap, GGEM_ERR_CAPACITY, "n_tgt exceeds max_points");
        GG_CHECK(tgt_is_src || n_tgt == 0 || x_tgt, GGEM_ERR_INVALID_ARG, "NULL target array");
        if (!u && !sigma) return;
        const double* xs = stage_in(P, x_src, P->d_in0, (size_t)n_src * 3);
        const double* gd = stage_in(P, g, P->d_in1, (size_t)n_src * 3);
        const double* xt = tgt_is_src ? xs : stage_in(P, x_tgt, P->d_in2, (size_t)n_tgt * 3);
        OutMap mu_ = stage_out(u, P->d_out0, (size_t)n_tgt * 3);
        OutMap ms_ = stage_out(sigma, P->d_out1, (size_t)n_tgt * 6);
        if (P->fp64)
            local_only_impl<double>(P, n_src, xs, gd, n_tgt, xt, tgt_is_src, mu_.dev, ms_.dev);
        else
            local_only_impl<float>(P, n_src, xs, gd, n_tgt, xt, tgt_is_src, mu_.dev, ms_.dev);
        finish_out(P, mu_);
        finish_out(P, ms_);
        if (mu_.host || ms_.host) GG_CUDA(cudaStreamSynchronize(P->st));
    });
}

static ggem_status layer_entry(ggem_plan_t* P, int layer, const double* q, double* out) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready, GGEM_ERR_INVALID_ARG, "no mesh set");
        GG_CHECK(q && out, GGEM_ERR_INVALID_ARG, "NULL density or output");
        GG_CHECK(P->prm.quadrature == GGEM_NODAL || P->n_tris > 0, GGEM_ERR_INVALID_ARG,
                 "element quadrature needs triangles");

        GG_CHECK(layer == 0 || P->n_tris > 0, GGEM_ERR_INVALID_ARG,
                 "the double layer needs triangles (node normals)");
        size_t n3 = (size_t)P->n_nodes * 3;
        const double* qd = stage_in(P, q, P->d_in0, n3);
        OutMap mo = stage_out(out, P->d_out0, n3);
        if (P->fp64) layer_impl<double>(P, layer, qd, mo.dev);
        else layer_impl<float>(P, layer, qd, mo.dev);
        finish_out(P, mo);
        if (mo.host) GG_CUDA(cudaStreamSynchronize(P->st));
    });
}

ggem_status ggem_single_layer(ggem_plan_t* P, const double* q, double* w) {
    return layer_entry(P, 0, q, w);
}

ggem_status ggem_double_layer(ggem_plan_t* P, const double* q, double* v) {
    return layer_entry(P, 1, q, v);
}

ggem_status ggem_check(ggem_plan_t* P) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        int h = 0;
        GG_CUDA(cudaMemcpyAsync(&h, P->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));
        GG_CHECK(h == 0, GGEM_ERR_CUDA,
                 "a tensor-core kernel gave up waiting for its MMAs (results invalid)");
    });
}

ggem_status ggem_trace_enable(ggem_plan_t* P, int on) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    P->prof = on != 0;
    for (int i = 0; i < 16; ++i) {
        P->prof_ms[i] = 0.0;
        P->prof_calls[i] = 0;
    }
    P->launches = 0;
    if (P->twin) ggem_trace_enable(P->twin, on);
    return GGEM_OK;
}

int ggem_trace_stage_count(void) { return ST_COUNT; }

const char* ggem_trace_stage_name(int stage) {
    return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : "";
}

ggem_status ggem_trace_read(const ggem_plan_t* P, int stage, double* total_ms, long* calls) {
    if (!P || stage < 0 || stage >= ST_COUNT) return GGEM_ERR_INVALID_ARG;
    // a mixed plan's FP64 twin (true residuals of the solve) is counted with it
    if (total_ms) *total_ms = P->prof_ms[stage] + (P->twin ? P->twin->prof_ms[stage] : 0.0);
    if (calls) *calls = P->prof_calls[stage] + (P->twin ? P->twin->prof_calls[stage] : 0);
    return GGEM_OK;
}

ggem_status ggem_launch_count(const ggem_plan_t* P, long* launches) {
    if (!P || !launches) return GGEM_ERR_INVALID_ARG;
    *launches = P->launches + (P->twin ? P->twin->launches : 0);
    return GGEM_OK;
}

}  // extern "C"
