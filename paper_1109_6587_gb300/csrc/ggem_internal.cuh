// Internal declarations of libggem: plan layout, kernel launchers.
// Paper: Kumar & Graham, arXiv 1109.6587 (GGEM in a planar slit).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include <mutex>
#include <unordered_map>

#include "ggem.h"

namespace ggem {

// Lets `kernel` use as much dynamic shared memory as the device allows a block
// (the opt-in limit less the kernel's static shared memory).  Set once per
// kernel under a lock, so launches from several host threads (plans of
// different sizes) never lower each other's limit; occupancy still follows
// each launch's own dynamic size.  Returns the status of that one call.
inline cudaError_t grant_max_smem(const void* kernel) {
    static std::mutex mu;
    static std::unordered_map<const void*, cudaError_t> done;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find(kernel);
    if (it != done.end()) return it->second;
    int dev = 0, v = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 v - (int)fa.sharedSizeBytes);
    done[kernel] = e;
    return e;
}

// ------------------------------------------------------------ small types
template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4_32a; };
template <typename T> using v4_t = typename V4<T>::type;

template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };
template <typename T> using c2_t = typename C2<T>::type;

// Cell list over [0,Lx) x [y0,y0+W] x [0,Lz): cells no smaller than r_cut.
struct CellGrid {
    int ncx, ncy, ncz;
    double hx, hy, hz;
    double y0;
    int reach = 3;   // cells are at least r_cut / reach wide; searches span +-reach cells (2 or 3)
};

// Geometry and GGEM constants handed to kernels by value.
struct GridGeom {
    double Lx, Lz, W, y0;
    int Nx, Ny, Nz, nkx;       // nkx = Nx/2 kept Fourier modes in x
    double dx, dz;
    double alpha, rcut, mu;
};

// Point sources sorted by cell: offsets from the cell corner (T precision),
// strengths, permutation sorted -> caller index.
template <typename T> struct SortedSources {
    v4_t<T>* pos;    // (ox, oy, oz, 0)
    v4_t<T>* g;      // (gx, gy, gz, 0)
    int* cell;       // cell index of each sorted source
    int* perm;       // caller index of each sorted source
    int* cell_start; // [ncell + 1]
    int n;
};

// 4x4 Gauss-Legendre product rule on [0,1]^2 and the polar-rule angles
struct QuadRule {
    double t[4], w[4];                // nodes and weights on [0,1]
    double th[4], cth[4], sth[4];     // theta_a = (pi/2) t_a, cos, sin
    double rmax[4], wth[4];           // 1/(cos + sin), (pi/2) w_a
};

}  // namespace ggem

// ----------------------------------------------------------------- the plan
struct ggem_plan {
    ggem_params prm;
    cudaStream_t st = nullptr;
    ggem::GridGeom geo;
    ggem::CellGrid cg;
    int ncell = 0;
    int nmodes = 0;           // Nz * nkx
    bool fp64 = true;
    std::string err;

    // tables
    double* d_yj = nullptr;            // [Ny] Chebyshev nodes (physical y)
    void* d_cheb_fwd = nullptr;        // [Ny][Ny] T, scaled by 1/(Nx Nz)
    void* d_cheb_inv = nullptr;        // [Ny][Ny] T
    void* d_tw_x = nullptr;            // complex T: [Nx/4] FFT-length-Nx/2 twiddles + [Nx/2] post twiddles
    void* d_tw_z = nullptr;            // complex T: [Nz/2]
    void* d_ksb = nullptr;             // [3][Ny][nmodes] T: p_b, phi_b, v_b coefficients
    double* d_minv = nullptr;          // [4][nmodes] inverse influence matrix
    double* d_kscoef = nullptr;        // [3][Ny] recurrence coefficients
    void* d_ydiff = nullptr;           // [Ny][Ny] T, y_j - y_k

    // workspaces
    void* d_gridA = nullptr;           // max(9,3)*Ny*Nz*Nx T
    void* d_gridB = nullptr;
    void* d_wall = nullptr;            // [2][3][Nz][Nx] T
    double* d_thom = nullptr;          // [4][Ny][nmodes] Thomas factors
    double* d_kschunk = nullptr;       // [nmodes][3][2][8] chunk products of the factors
    double* d_isq = nullptr;           // [2][nmodes]
    size_t grid_elems = 0;

    // point sources (sorted)
    int cap = 0;
    int* d_cell_count = nullptr;       // [ncell]
    int* d_cell_start = nullptr;       // [ncell+1]
    int* d_cursor = nullptr;           // [ncell]
    int* d_src_cell = nullptr;         // [cap]
    int* d_perm = nullptr;             // [cap]
    void* d_spos = nullptr;            // [cap] v4 T
    void* d_sg = nullptr;              // [cap] v4 T
    double* d_src_x = nullptr;         // [cap][3] caller-order positions (double)
    void* d_local = nullptr;           // [cap][9] T local-sum output

    // staging for host pointers
    double* d_in0 = nullptr;           // [cap][3]
    double* d_in1 = nullptr;           // [cap][3]
    double* d_in2 = nullptr;           // [cap][3]
    double* d_out0 = nullptr;          // [cap][3]
    double* d_out1 = nullptr;          // [cap][6]
    int* d_tgt_cell = nullptr;         // [cap] located point targets
    void* d_tgt_pos = nullptr;         // [cap] v4 T
    int* d_wall_cell = nullptr;        // [2 Nz Nx] located wall nodes (plan lifetime)
    void* d_wall_pos = nullptr;

    // mesh
    int n_nodes = 0, n_tris = 0, cap_tris = 0;
    bool mesh_ready = false;
    double* d_x = nullptr;             // [cap][3]
    int* d_tri = nullptr;              // [cap_tris][3]
    double* d_area = nullptr;          // [cap] nodal areas
    double* d_nrm = nullptr;           // [cap][3] node normals
    double* d_tri_area = nullptr;      // [cap_tris]
    double* d_tri_nrm = nullptr;       // [cap_tris][3]
    int* d_mesh_cell = nullptr;        // mesh nodes sorted: cell / perm / offsets
    int* d_mesh_perm = nullptr;
    int* d_mesh_start = nullptr;
    void* d_mesh_pos = nullptr;
    int4* d_mesh_sdi = nullptr;        // spreading descriptors of the mesh nodes
    void* d_mesh_sdf = nullptr;
    int4* d_sdi = nullptr;             // spreading descriptors of free sources
    void* d_sdf = nullptr;

    // element quadrature (16 points per triangle)
    ggem::QuadRule rule;
    int cap_qp = 0, n_qp = 0;
    double* d_qx = nullptr;            // [cap_qp][3] point positions
    int4* d_qv = nullptr;              // [cap_qp] triangle vertices
    int4* d_qv_sorted = nullptr;       // [cap_qp] the same, in sorted point order
    double near_edge = 0.0;            // longest triangle edge of the mesh
    void* d_qw = nullptr;              // [cap_qp] v4 T: phi_v * weight (point order once sorted)
    int* d_qp_cell = nullptr;          // sorted points: cell / perm / offsets / start
    int* d_qp_perm = nullptr;
    int* d_qp_start = nullptr;
    void* d_qp_pos = nullptr;
    void* d_qg = nullptr;              // [cap_qp] v4 T sorted strengths
    int* d_adj_cnt = nullptr;          // node -> triangle adjacency (CSR)
    int* d_adj_start = nullptr;
    int* d_adj_cur = nullptr;
    int* d_adj = nullptr;

    // tracing: per-stage device time (CUDA events on the plan's stream)
    bool prof = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // Fredholm solve workspace (allocated by the first solve)
    int sol_m = 0;                     // restart length d_V holds
    size_t sol_ld = 0;                 // stride of the solver vectors (>= 3 cap)
    double* d_V = nullptr;             // [sol_m + 1][sol_ld] Krylov basis
    double* d_sv = nullptr;            // [ld] double-layer output
    double* d_sb = nullptr;            // [ld] staged right-hand side
    double* d_sk = nullptr;            // [cap] staged kappa
    double* d_sx = nullptr;            // [ld] iterate when q is a host array
    double* d_spart = nullptr;         // reduction partials
    double* d_sh = nullptr;            // Arnoldi coefficients / correction weights
    double* h_sh = nullptr;            // pinned host copy of d_sh
    ggem_plan* twin = nullptr;         // FP64 plan on the same mesh (mixed plans)
    // spectral off-grid evaluation (ggem_set_offgrid)
    int offgrid = 0;                   // GGEM_OFFGRID_*
    int spec_w = 0;                    // Gaussian window half-width (fine points per side)
    void* d_spec = nullptr;            // [2Ny-1][9][2Nz][2Nx] T oversampled grid
    void* d_spec_mid = nullptr;        // [2Ny-1][9][Nz][Nx] T theta planes, x-z spectral
    void* d_spec_ct = nullptr;         // [2Ny-1][Ny] T Chebyshev -> theta-node matrix
    void* d_spec_twx = nullptr;        // FFT twiddles of lengths 2Nx and 2Nz, laid out as
    void* d_spec_twz = nullptr;        //   d_tw_x / d_tw_z
    void* d_spec_dx = nullptr;         // [Nx/2] T deconvolution factors, k_x >= 0
    void* d_spec_dz = nullptr;         // [Nz] T deconvolution factors, FFT order in z
    int sol_iters = 0, sol_cycles = 0, sol_mv64 = 0, sol_mvmix = 0;
    double sol_relres = 0.0;
    // learned warm start (allocated by its first use)
    int* d_particle = nullptr;         // [cap] particle id of each node (caller order)
    int* d_pcount = nullptr;           // [pcount_cap + 1] nodes per particle, error flag
    int pcount_cap = 0, n_particles = 0;
    // rigid-particle solve (allocated by its first use)
    bool pcsr_ready = false;           // d_pstart / d_pnodes match d_particle
    int particles_n = 0;               // n_nodes when the particle ids were set
    int* d_pstart = nullptr;           // [pcount_cap + 1] CSR of the nodes of each particle
    int* d_pnodes = nullptr;           // [cap] node indices grouped by particle, ascending
    double* d_rc = nullptr;            // [pcount_cap][3] reference points c_p
    double* d_rscale = nullptr;        // [pcount_cap][2] 1/(6 pi mu R_p), 1/(8 pi mu R_p^2)
    int rig_cap = 0;                   // particles d_pstart / d_rc / d_rscale hold
    // capsule dynamics (allocated by their first use)
    double* d_mref = nullptr;          // [cap_tris][4] reference metric G11, G12, G22, area
    bool mref_ready = false;
    double* d_cx0 = nullptr;           // [3 cap] positions at the start of a step
    double* d_cdf = nullptr;           // [3 cap] traction jump
    double* d_cuinf = nullptr;         // [3 cap] undisturbed velocity
    double* d_cfinf = nullptr;         // [3 cap] undisturbed traction
    double* d_cb = nullptr;            // [3 cap] right side of the Fredholm equation
    double* d_ckap = nullptr;          // [cap] kappa per node
    double* d_clam = nullptr;          // [cap] staged viscosity ratios
    double* d_cw = nullptr;            // [3 cap] single layer of q / stage velocity
    double* d_cq = nullptr;            // [3 cap] density when the caller's q is a host array
    unsigned long long* d_cmin = nullptr;  // reduction word (bits of a positive double)
    int* d_tstart = nullptr;           // [pcount_cap + 1] CSR of the triangles of each particle
    int* d_tlist = nullptr;            // [cap_tris] triangle indices grouped by particle
    double* d_cvol = nullptr;          // [pcount_cap] particle volumes / areas scratch
    bool tcsr_ready = false;
    bool ff = false;                   // element-rule local sum in double-float arithmetic
    void* d_qp_ff = nullptr;           // [cap_qp][2] float4: sorted point offsets, hi / lo
    void* d_qg_ff = nullptr;           // [cap_qp][2] float4: sorted point strengths, hi / lo
    float* d_qp_pack = nullptr;        // [6 soa_ld] FP32 plans: packed point offsets and strengths
    size_t soa_ld = 0;                 // slots of the packed layout: padded size + 64, a multiple of 64
    long qp_np = 0;                    // slots in use (the padded size, even)
    int* d_qp_pstart = nullptr;        // [ncell + 1] FP32 plans: padded cell starts
    int* d_qp_inv = nullptr;           // [soa_ld] padded slot -> sorted point, -1 for dummies
    float* d_q32 = nullptr;            // [cap][3] FP32 plans: the density in FP32
    int* d_orec = nullptr;             // [4 cap][2] overlap records: particle pair
    double* d_orecd = nullptr;         // [4 cap] overlap records: node gap
    int* d_ocount = nullptr;           // record count
    double* d_odisp = nullptr;         // [pcount_cap][3] rigid displacements / centroids
    float* d_feat = nullptr;           // [cap][12] features
    float* d_mlp = nullptr;            // [35075] FP32 master parameters
    float* d_mlp_grad = nullptr;       // gradient accumulator
    float* d_mlp_m = nullptr;          // Adam first moments
    float* d_mlp_v = nullptr;          // Adam second moments
    unsigned short* d_mlp_wf = nullptr;  // bfloat16 weights [fan_in][fan_out]
    unsigned short* d_mlp_wt = nullptr;  // bfloat16 weights [fan_out][fan_in]
    float* d_mlp_stats = nullptr;      // mu[12], sigma[12], s_y
    float* d_mlp_out = nullptr;        // [cap][3] network output
    double* d_smlp = nullptr;          // [3 cap] learned guess of the solve
    double* d_sres = nullptr;          // [3 cap] residual of the caller's guess
    double* d_mlp_dr = nullptr;        // [3 cap] D r of the features
    double* d_mlp_ssq = nullptr;       // sum of r^2 of the features
    bool mlp_ready = false;
    bool mlp_fp32 = false;             // FP32 mode: no bfloat16 rounding points
    unsigned short* d_mlp_tc = nullptr;  // bfloat16 weight image of the tensor-core forward
    void* d_mlp_tcs = nullptr;         // tensor-core training scratch (one minibatch)
    int mlp_tcs_rows = 0;              // rows it holds
    long mlp_step = 0;
    int sol_guess_mlp = 0;             // last solve: 1 if it started from the learned guess
    double sol_rel_plain = 0.0, sol_rel_mlp = 0.0;
    // per-particle block preconditioner of the Fredholm solve (ggem_precond_set)
    int pc_n = 0;                      // nodes of the reference capsule (0: none set)
    bool pc_on = false;                // solves use it
    double pc_kappa = 0.0;             // kappa the block was built for
    double* d_pc_B64 = nullptr;        // [3 pc_n][3 pc_n] block inverse, FP64
    float* d_pc_B32 = nullptr;         //   and FP32
    double* d_pc_xref = nullptr;       // [pc_n][3] reference nodes about their centroid
    int pc_np = 0;                     // particles the arrays below hold
    double* d_pc_R = nullptr;          // [pc_np][9] rotations, reference -> particle
    double* d_pc_U = nullptr;          // [pc_np][3 pc_n] turned densities (FP64 or FP32)
    double* d_pc_Z = nullptr;          // [pc_np][3 pc_n] block products (FP64 or FP32)
    double* d_pc_Zb = nullptr;         // [pc_m][sol_ld] preconditioned Krylov vectors
    int pc_m = 0;
    int* d_tc_err = nullptr;           // tensor-core kernels: expired waits
    int* d_spread_list = nullptr;      // [cap + 1] sources the paired spread hands back
    void* d_tc_fwd = nullptr;          // split-bf16 Chebyshev matrices (mixed plans)
    void* d_tc_inv = nullptr;
    int nsm = 0;                       // multiprocessors of the plan's device
    cudaStream_t st2 = nullptr;        // second stream (greatest priority): the longer of local / global part
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double prof_ms[16] = {0};
    long prof_calls[16] = {0};
    long launches = 0;                 // kernels launched by this plan
};

namespace ggem {

// ------------------------------------------------------------ launchers
// cell list: sort n sources (caller-order double positions x[n][3]) into cells
template <typename T>
cudaError_t build_cells(const GridGeom& geo, const CellGrid& cg, int n, const double* x,
                        int* cell_count, int* cell_start, int* cursor, int* src_cell,
                        int* perm, v4_t<T>* pos, cudaStream_t st);

// gather caller-order strengths (scale * w[i] * q[i], w may be NULL) into sorted order
template <typename T>
cudaError_t gather_strengths(int n, const int* perm, const double* q, const double* w,
                             double scale, v4_t<T>* g, cudaStream_t st);

// local sum targets
enum TargetKind { TK_SORTED = 0, TK_POINTS = 1, TK_WALL = 2 };
// out modes
enum { OUT_U = 1, OUT_S = 2, OUT_DBL = 4 };

// targets: TK_SORTED = the sorted sources themselves (output via perm);
// TK_POINTS / TK_WALL = targets located by locate_targets (cell, offsets)
template <typename T>
cudaError_t local_sum(const GridGeom& geo, const CellGrid& cg, const SortedSources<T>& src,
                      int kind, int n_tgt, const int* tcell, const v4_t<T>* tpos,
                      const double* nrm_tgt, int out_mode, T* out, int out_stride,
                      cudaStream_t st);

// element rule: local sum over sorted quadrature points at the sorted mesh
// nodes tgt (output in caller order), skipping points of triangles that
// contain the target (only tested when closer than `near`); layer 0
// velocity, 1 double layer
// aux_pos / aux_g: FP32, the structure-of-arrays planes of the sorted points
// (x, y, z, stride aux_ld; required); FP64, float-pair copies selecting the
// double-float kernel (nullptr: native FP64)
template <typename T>
cudaError_t local_sum_elem(const GridGeom& geo, const CellGrid& cg, const SortedSources<T>& src,
                           const int4* qvs, double near, const SortedSources<T>& tgt,
                           const double* nrm_tgt, int layer, T* out, int out_stride,
                           cudaStream_t st, const void* aux_pos = nullptr,
                           const void* aux_g = nullptr, size_t aux_ld = 0,
                           const int* aux_inv = nullptr);
// FP32 element rule, padded and packed layout of the sorted points (each cell
// from a multiple of 64, whole 64-point steps, dummies of zero strength far
// away; 12 floats per slot pair: x0 x1 y0 y1 z0 z1 gx0 gx1 gy0 gy1 gz0 gz1):
// padded counts and starts (pcnt: ncell scratch, pstart: ncell + 1), then the
// np slots of pack (np even; dummies at 1e4, strengths zero), the positions
// (scaled by alpha sqrt(log2 e), the local-sum kernel's units), and the map
// slot -> sorted point (inv, -1 for dummies)
cudaError_t pad_layout_counts(int ncell, const int* start, int* pcnt, int* pstart,
                              cudaStream_t st);
cudaError_t pad_layout_fill(int n, size_t np, const int* cell, const int* start,
                            const int* pstart, const float4* pos, double alpha, float* pack,
                            int* inv, cudaStream_t st);
// FP32 element rule: sub-sort the sorted points within each cell (4 x 4 x 4
// sub-cells in Morton order; tmp_* of n entries as scratch)
cudaError_t cell_subsort(const CellGrid& cg, int n, int ncell, const int* start, float4* pos,
                         int* perm, float4* tmp_pos, int* tmp_perm, cudaStream_t st);
// float-pair copy of n double4 (x, y, z, w) values: out[2 i] = hi, out[2 i + 1] = lo
cudaError_t to_float_pairs(int n, const void* in, void* out, cudaStream_t st);
cudaError_t gather_int4(int n, const int* perm, const int4* in, int4* out, cudaStream_t st);

// exclusive scan of count[0..n) into start[0..n] (start[n] = total)
cudaError_t scan_counts(int n, const int* count, int* start, cudaStream_t st);

QuadRule make_quad_rule();
// quadrature points of m triangles and the node -> triangle adjacency
template <typename T>
cudaError_t elem_setup(int m, const double* x, const int* tri, const double* tri_area,
                       const QuadRule& rule, double* xq, int4* qv, v4_t<T>* qw, int nnodes,
                       int* adj_cnt, int* adj_start, int* adj_cur, int* adj, cudaStream_t st);
// quadrature weights qw into point order, qw[s] <- qw[perm[s]] (tmp: nq v4 T)
template <typename T>
cudaError_t qp_sort_weights(int nq, const int* perm, v4_t<T>* qw, v4_t<T>* tmp, cudaStream_t st);
// sorted point strengths g = scale sum_v (phi_v w) q_v from the sorted vertex
// indices and weights, in T: FP64 plans into g (v4); FP32 plans copy the
// nnodes x 3 density q into qT, then fill the strengths of the nslots slots of
// the packed layout (pad_layout_fill; inv: slot -> sorted point)
template <typename T>
cudaError_t qp_strengths(int nq, const int4* qv, const v4_t<T>* qw, int nnodes, const double* q,
                         T* qT, double scale, v4_t<T>* g, T* pack, const int* inv, long nslots,
                         cudaStream_t st);
// polar-rule correction of the local part at the mesh nodes (layer 0 single, 1 double);
// q: the nodal density in T
template <typename T>
cudaError_t elem_correct(int n, int layer, const GridGeom& geo, const double* x, const int* tri,
                         const double* tri_nrm, const double* nrm, const int* adj_start,
                         const int* adj, const T* q, const QuadRule& rule, T* out,
                         int out_stride, cudaStream_t st);

// locate targets: kind TK_POINTS (x[n][3]) or TK_WALL (the 2 Nz Nx wall nodes)
template <typename T>
cudaError_t locate_targets(const GridGeom& geo, const CellGrid& cg, int n, int kind,
                           const double* x, int* cell, v4_t<T>* pos, cudaStream_t st);

// per-source spreading descriptors (once per source set), then
// f = -sum g rho_g on the grid [Ny][3][Nz][Nx]; ydiff[j][k] = y_j - y_k
template <typename T>
cudaError_t spread_prepare(const GridGeom& geo, const double* yj, int n, const int* perm,
                           const double* x, int4* di, v4_t<T>* df, cudaStream_t st);
// work: scratch of 4 Ny Nz Nx T (interleaved accumulation buffer)
template <typename T>
cudaError_t spread(const GridGeom& geo, const CellGrid& cg, const double* yj, const T* ydiff,
                   const SortedSources<T>& src, const int4* di, const v4_t<T>* df, T* grid,
                   T* work, int* list, cudaStream_t st);

template <typename T>
cudaError_t fft_forward(const GridGeom& geo, T* data, int nplanes, const void* tw_x,
                        const void* tw_z, cudaStream_t st);
template <typename T>
cudaError_t fft_inverse(const GridGeom& geo, T* data, int nplanes, const void* tw_x,
                        const void* tw_z, cudaStream_t st, int active_kx = 0);

template <typename T>
cudaError_t cheb_apply(int Ny, const T* M, const T* in, T* out, long cols, cudaStream_t st,
                       int* tc_err = nullptr, int nsm = 0, const void* tc_prep = nullptr);
// split-bf16 copy of an Ny x Ny FP32 matrix for the tensor-core transform
size_t cheb_tc_prep_bytes(int Ny);
cudaError_t cheb_tc_prepare(int Ny, const float* M, void* prep, cudaStream_t st);

// per-mode tau solves; coef = mode-independent recurrence table [3][Ny];
// thom = per-mode Thomas factors [4][Ny][nmodes], isq = [2][nmodes];
// scratch = [5][2][Ny][nmodes] T, then (256-byte aligned) [3][2][Ny][nmodes] double
template <typename T>
cudaError_t ks_modes(const GridGeom& geo, const T* fcoef, const T* wall, const T* ksb,
                     const double* minv, const double* coef, const double* thom,
                     const double* chunk, const double* isq, int out_sel, T* ocoef,
                     cudaStream_t st);

// mode 0: velocity, out = local + interp - self_coef * wself * qself
// mode 1: stress (6), out = local + interp
// mode 2: double layer, out_j = local_j + n_k sigma_jk / mu
// Oversampled grid of the spectral off-grid evaluation: physical values
// [Mt/2 + 1][ncomp_total][Mz][Mx] of the field deconvolved by the Gaussian
// window exp(-c t^2) (t in fine spacings) at theta = 2 pi p / Mt (theta =
// arccos of the normalised y), gathered over w points per side.
struct SpecGrid {
    const void* fine;
    int Mx, Mz, Mt, w;
    double c;
    double sx, sz, st;  // Mx / Lx, Mz / Lz, Mt / (2 pi): fine spacings per unit
    double sy;          // 2 / W: normalised y = (y - y0) sy - 1
    const int* order;   // target processing order (nullptr: 0..n-1)
};

// Combine of local and global parts at the targets: the global grid field
// evaluated by 5-point Lagrange interpolation, or (spec != nullptr) from the
// oversampled grid by the Gaussian window in x, z and the barycentric
// Chebyshev formula in y.
template <typename T>
cudaError_t interp_combine(const GridGeom& geo, const double* yj, const T* grid, int ncomp_total,
                           int comp0, int n_tgt, const double* x_tgt, const T* local,
                           int local_stride, const double* nrm, const double* qself,
                           const double* wself, double self_coef, int mode, double* out,
                           int out_stride, cudaStream_t st, const SpecGrid* spec = nullptr);

// Spectral planes [nplanes][Nz][Nx/2] (complex T, after the Chebyshev
// inverse) -> deconvolved, zero-padded planes [nplanes][Mz][Mx/2] of the
// oversampled grid (complex T), ready for fft_inverse on the Mx x Mz grid.
template <typename T>
cudaError_t spectral_pad(const GridGeom& geo, const T* spec, int nplanes, int Mx, int Mz,
                         const T* dx, const T* dz, T* fine, cudaStream_t st);

// out[p][col] = sum_n M[p][n] in[n][col], M: R x C (row-major), in: [C][cols].
template <typename T>
cudaError_t cheb_rect(int R, int C, const T* M, const T* in, T* out, long cols,
                      cudaStream_t st);

}  // namespace ggem
