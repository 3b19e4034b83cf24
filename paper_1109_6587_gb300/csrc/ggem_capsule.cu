// Capsule dynamics: the membrane traction jump (Sec. 4), the undisturbed flows
// and their traction (App. B), the right side of Eq. (qa), the velocity of
// Eq. (bi_ua) and the midpoint (second-order Runge-Kutta) step of dx/dt = u
// (Sec. 5), the node separation that sets the time step, particle volumes and
// the volume correction (Sec. 5).  All FP64: the work is O(N) and small beside
// the single- and double-layer evaluations the step makes.
//
// Membrane: every flat triangle k stores the neo-Hookean energy
// A0_k W = A0_k (G/2)(tr C + 1/det C - 3) (Eq. (eq_WNH)) of its uniform
// deformation, C the right Cauchy-Green tensor, written with the reference
// metric G_ij = E_i . E_j and the current one g_ij = e_i . e_j of the edge
// vectors e_1 = x_2 - x_1, e_2 = x_3 - x_1: tr C = G^ij g_ij, det C =
// det g / det G.  The force on a vertex is the energy's gradient (the
// principle of virtual work); the traction jump at node p is the summed force
// over its area A_p (a third of its triangles' current areas), Eq. (cntr2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ggem.h"
#include "ggem_host.cuh"

using namespace ggem;

namespace {

constexpr int CB = 256;

__device__ __forceinline__ void load3(const double* x, int i, double& a, double& b, double& c) {
    a = x[3 * i];
    b = x[3 * i + 1];
    c = x[3 * i + 2];
}

// reference metric and area of every triangle: [G11, G12, G22, A0]
__global__ void k_membrane_ref(int m, const double* __restrict__ xr, const int* __restrict__ tri,
                               double* __restrict__ ref) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    double ax, ay, az, bx, by, bz, cx, cy, cz;
    load3(xr, tri[3 * k], ax, ay, az);
    load3(xr, tri[3 * k + 1], bx, by, bz);
    load3(xr, tri[3 * k + 2], cx, cy, cz);
    const double e1x = bx - ax, e1y = by - ay, e1z = bz - az;
    const double e2x = cx - ax, e2y = cy - ay, e2z = cz - az;
    const double G11 = e1x * e1x + e1y * e1y + e1z * e1z;
    const double G12 = e1x * e2x + e1y * e2y + e1z * e2z;
    const double G22 = e2x * e2x + e2y * e2y + e2z * e2z;
    ref[4 * k] = G11;
    ref[4 * k + 1] = G12;
    ref[4 * k + 2] = G22;
    ref[4 * k + 3] = 0.5 * sqrt(G11 * G22 - G12 * G12);
}

// Delta f at node b: the energy gradient of its triangles at b over A_b
__global__ void k_traction(int n, const double* __restrict__ x, const int* __restrict__ tri,
                           const double* __restrict__ ref, const int* __restrict__ adj_start,
                           const int* __restrict__ adj, const double* __restrict__ area,
                           double shear_modulus, double* __restrict__ df) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int a = adj_start[b]; a < adj_start[b + 1]; ++a) {
        const int k = adj[a];
        const int t0 = tri[3 * k], t1 = tri[3 * k + 1], t2 = tri[3 * k + 2];
        double ax, ay, az, bx, by, bz, cx, cy, cz;
        load3(x, t0, ax, ay, az);
        load3(x, t1, bx, by, bz);
        load3(x, t2, cx, cy, cz);
        const double e1x = bx - ax, e1y = by - ay, e1z = bz - az;
        const double e2x = cx - ax, e2y = cy - ay, e2z = cz - az;
        const double g11 = e1x * e1x + e1y * e1y + e1z * e1z;
        const double g12 = e1x * e2x + e1y * e2y + e1z * e2z;
        const double g22 = e2x * e2x + e2y * e2y + e2z * e2z;
        const double G11 = ref[4 * k], G12 = ref[4 * k + 1], G22 = ref[4 * k + 2];
        const double A0 = ref[4 * k + 3];
        const double detG = G11 * G22 - G12 * G12, detg = g11 * g22 - g12 * g12;
        const double i11 = G22 / detG, i12 = -G12 / detG, i22 = G11 / detG;
        const double c = detG / (detg * detg), s = 0.5 * shear_modulus * A0;
        // dE/de1 = s (2 G^1j e_j - c d(det g)/de1), dE/de2 likewise
        const double p1 = 2.0 * i11, q1 = 2.0 * i12, r1 = -2.0 * c * g22, w1 = 2.0 * c * g12;
        const double p2 = 2.0 * i12, q2 = 2.0 * i22, r2 = -2.0 * c * g11, w2 = 2.0 * c * g12;
        // f2 = s ((p1 + r1) e1 + (q1 + w1) e2),  f3 = s ((p2 + w2) e1 + (q2 + r2) e2)
        const double a1 = s * (p1 + r1), b1 = s * (q1 + w1);
        const double a2 = s * (p2 + w2), b2 = s * (q2 + r2);
        double ca, cb;
        if (b == t1) {
            ca = a1;
            cb = b1;
        } else if (b == t2) {
            ca = a2;
            cb = b2;
        } else {
            ca = -(a1 + a2);
            cb = -(b1 + b2);
        }
        fx += ca * e1x + cb * e2x;
        fy += ca * e1y + cb * e2y;
        fz += ca * e1z + cb * e2z;
    }
    const double ia = 1.0 / area[b];
    df[3 * b] = fx * ia;
    df[3 * b + 1] = fy * ia;
    df[3 * b + 2] = fz * ia;
}

// undisturbed velocity and traction sigma . n at the nodes (App. B):
// flow 1 simple shear u = s (y - y_mid) e_x, sigma = mu s e;
// flow 2 pressure-driven u = 4 s eta (1 - eta) e_x, eta = (y - y0)/W,
//        sigma = (8 mu s / W^2) x I + (4 mu s / W)(1 - 2 eta) e
__global__ void k_undisturbed(int n, const double* __restrict__ x, const double* __restrict__ nrm,
                              int flow, double s, double mu, double y0, double W,
                              double* __restrict__ u, double* __restrict__ f) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const double px = x[3 * b], py = x[3 * b + 1];
    double ux = 0.0, iso = 0.0, sxy = 0.0;
    if (flow == GGEM_FLOW_SHEAR) {
        ux = s * (py - (y0 + 0.5 * W));
        sxy = mu * s;
    } else if (flow == GGEM_FLOW_POISEUILLE) {
        const double eta = (py - y0) / W;
        ux = 4.0 * s * eta * (1.0 - eta);
        iso = 8.0 * mu * s / (W * W) * px;
        sxy = 4.0 * mu * s / W * (1.0 - 2.0 * eta);
    }
    if (u) {
        u[3 * b] = ux;
        u[3 * b + 1] = 0.0;
        u[3 * b + 2] = 0.0;
    }
    if (f) {
        const double nx = nrm[3 * b], ny = nrm[3 * b + 1], nz = nrm[3 * b + 2];
        f[3 * b] = iso * nx + sxy * ny;
        f[3 * b + 1] = sxy * nx + iso * ny;
        f[3 * b + 2] = iso * nz;
    }
}

// kappa = (lam - 1)/(lam + 1), b = -(Delta f/(lam + 1) + kappa f_inf)/(4 pi mu)
__global__ void k_capsule_rhs(int n, const double* __restrict__ lam, const double* __restrict__ df,
                              const double* __restrict__ finf, double mu,
                              double* __restrict__ kap, double* __restrict__ rhs) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const double l = lam[b], il = 1.0 / (l + 1.0), k = (l - 1.0) * il;
    const double s = -1.0 / (4.0 * kPi * mu);
    kap[b] = k;
    for (int c = 0; c < 3; ++c) rhs[3 * b + c] = s * (df[3 * b + c] * il + k * finf[3 * b + c]);
}

// out = base + h (u_inf + w)   (base == nullptr: 0)
__global__ void k_advance(int n3, const double* __restrict__ base, const double* __restrict__ uinf,
                          const double* __restrict__ w, double h, double* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n3) return;
    const double v = uinf[e] + w[e];
    out[e] = base ? fma(h, v, base[e]) : h * v;
}

// smallest distance from every node to another node in its own or a
// neighbouring cell (minimum image in x, z), reduced into *out as the bits of
// a positive double
__global__ void k_min_sep(int n, GridGeom geo, CellGrid cg, const int* __restrict__ cell,
                          const int* __restrict__ start, const int* __restrict__ perm,
                          const double* __restrict__ x, unsigned long long* __restrict__ out) {
    __shared__ double red[CB / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double best = INFINITY;
    if (i < n) {
        const int c = cell[i];
        const int cx = c % cg.ncx, cy = (c / cg.ncx) % cg.ncy, cz = c / (cg.ncx * cg.ncy);
        const int me = perm[i];
        const double px = x[3 * me], py = x[3 * me + 1], pz = x[3 * me + 2];
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int yy = cy + dy;
                    if (yy < 0 || yy >= cg.ncy) continue;
                    const int xx = (cx + dx + cg.ncx) % cg.ncx, zz = (cz + dz + cg.ncz) % cg.ncz;
                    const int cc = (zz * cg.ncy + yy) * cg.ncx + xx;
                    for (int j = start[cc]; j < start[cc + 1]; ++j) {
                        if (j == i) continue;
                        const int o = perm[j];
                        double ex = x[3 * o] - px, ey = x[3 * o + 1] - py, ez = x[3 * o + 2] - pz;
                        ex -= geo.Lx * rint(ex / geo.Lx);
                        ez -= geo.Lz * rint(ez / geo.Lz);
                        best = fmin(best, sqrt(ex * ex + ey * ey + ez * ez));
                    }
                }
    }
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = red[0];
        for (int w = 1; w < CB / 32; ++w) m = fmin(m, red[w]);
        if (m < INFINITY) atomicMin(out, (unsigned long long)__double_as_longlong(m));
    }
}

// volume (divergence theorem) and area of particle blockIdx.x from its triangles
__global__ void __launch_bounds__(CB) k_volumes(const int* __restrict__ tstart,
                                                const int* __restrict__ tlist,
                                                const double* __restrict__ x,
                                                const int* __restrict__ tri,
                                                const double* __restrict__ tri_area,
                                                double* __restrict__ vol,
                                                double* __restrict__ surf) {
    __shared__ double rv[CB / 32], rs[CB / 32];
    const int p = blockIdx.x;
    double v = 0.0, s = 0.0;
    for (int a = tstart[p] + threadIdx.x; a < tstart[p + 1]; a += CB) {
        const int k = tlist[a];
        double ax, ay, az, bx, by, bz, cx, cy, cz;
        load3(x, tri[3 * k], ax, ay, az);
        load3(x, tri[3 * k + 1], bx, by, bz);
        load3(x, tri[3 * k + 2], cx, cy, cz);
        v += (ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx)) /
             6.0;
        s += tri_area[k];
    }
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_down_sync(0xffffffffu, v, o);
        s += __shfl_down_sync(0xffffffffu, s, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rv[threadIdx.x >> 5] = v;
        rs[threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tv = 0.0, ts = 0.0;
        for (int w = 0; w < CB / 32; ++w) {
            tv += rv[w];
            ts += rs[w];
        }
        vol[p] = tv;
        if (surf) surf[p] = ts;
    }
}

// x_b += d[particle_b] n_b
__global__ void k_normal_shift(int n, const int* __restrict__ part, const double* __restrict__ d,
                               const double* __restrict__ nrm, double* __restrict__ x) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const double s = d[part[b]];
    for (int c = 0; c < 3; ++c) x[3 * b + c] += s * nrm[3 * b + c];
}

// mean node position of particle blockIdx.x (node lists of the particles)
__global__ void __launch_bounds__(CB) k_centroids(const int* __restrict__ pstart,
                                                  const int* __restrict__ pnodes,
                                                  const double* __restrict__ x,
                                                  double* __restrict__ c) {
    __shared__ double red[3][CB / 32];
    const int p = blockIdx.x;
    double a[3] = {0.0, 0.0, 0.0};
    for (int k = pstart[p] + threadIdx.x; k < pstart[p + 1]; k += CB) {
        const int i = pnodes[k];
        for (int d = 0; d < 3; ++d) a[d] += x[3 * i + d];
    }
    for (int d = 0; d < 3; ++d) {
        double t = a[d];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) red[d][threadIdx.x >> 5] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double inv = 1.0 / (double)(pstart[p + 1] - pstart[p]);
        for (int d = 0; d < 3; ++d) {
            double t = 0.0;
            for (int w = 0; w < CB / 32; ++w) t += red[d][w];
            c[3 * p + d] = t * inv;
        }
    }
}

constexpr int kGapSlots = 4;   // other particles recorded per node

// every node: the closest node of each (of up to kGapSlots) other particles
// nearer than hthr in its own or a neighbouring cell; records (p, q, gap) for
// q > p, p the node's own particle.  count[0]: records; count[1] set when a
// node meets more than kGapSlots other particles (a record would be lost).
__global__ void k_gap_pairs(int n, GridGeom geo, CellGrid cg, const int* __restrict__ cell,
                            const int* __restrict__ start, const int* __restrict__ perm,
                            const int* __restrict__ part, const double* __restrict__ x,
                            double hthr, int cap, int* __restrict__ rec,
                            double* __restrict__ recd, int* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell[i];
    const int cx = c % cg.ncx, cy = (c / cg.ncx) % cg.ncy, cz = c / (cg.ncx * cg.ncy);
    const int me = perm[i], p = part[me];
    const double px = x[3 * me], py = x[3 * me + 1], pz = x[3 * me + 2];
    int sq[kGapSlots];
    double sd[kGapSlots];
    int ns = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int yy = cy + dy;
                if (yy < 0 || yy >= cg.ncy) continue;
                const int xx = (cx + dx + cg.ncx) % cg.ncx, zz = (cz + dz + cg.ncz) % cg.ncz;
                const int cc = (zz * cg.ncy + yy) * cg.ncx + xx;
                for (int j = start[cc]; j < start[cc + 1]; ++j) {
                    const int o = perm[j], q = part[o];
                    if (q <= p) continue;
                    double ex = x[3 * o] - px, ey = x[3 * o + 1] - py, ez = x[3 * o + 2] - pz;
                    ex -= geo.Lx * rint(ex / geo.Lx);
                    ez -= geo.Lz * rint(ez / geo.Lz);
                    const double d = sqrt(ex * ex + ey * ey + ez * ez);
                    if (!(d < hthr)) continue;
                    int k = 0;
                    while (k < ns && sq[k] != q) ++k;
                    if (k < ns) {
                        sd[k] = fmin(sd[k], d);
                    } else if (ns < kGapSlots) {
                        sq[ns] = q;
                        sd[ns] = d;
                        ++ns;
                    } else {
                        atomicOr(count + 1, 1);
                    }
                }
            }
    for (int k = 0; k < ns; ++k) {
        const int r = atomicAdd(count, 1);
        if (r < cap) {
            rec[2 * r] = p;
            rec[2 * r + 1] = sq[k];
            recd[r] = sd[k];
        }
    }
}

// x_b += disp[particle_b]
__global__ void k_translate(int n, const int* __restrict__ part, const double* __restrict__ disp,
                            double* __restrict__ x) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const int p = part[b];
    for (int d = 0; d < 3; ++d) x[3 * b + d] += disp[3 * p + d];
}

unsigned nblk(size_t n) { return (unsigned)((n + CB - 1) / CB); }

void ensure_capsule_ws(ggem_plan_t* P) {
    if (P->d_cx0) return;
    const size_t n3 = (size_t)3 * P->cap;
    for (double** p : {&P->d_cx0, &P->d_cdf, &P->d_cuinf, &P->d_cfinf, &P->d_cb, &P->d_cw,
                       &P->d_cq})
        dalloc(P, p, n3);
    dalloc(P, &P->d_ckap, (size_t)P->cap);
    dalloc(P, &P->d_clam, (size_t)P->cap);
    dalloc(P, &P->d_cmin, 1);
}

void check_flow(ggem_plan_t* P, int flow) {
    GG_CHECK(flow == GGEM_FLOW_NONE || flow == GGEM_FLOW_SHEAR || flow == GGEM_FLOW_POISEUILLE,
             GGEM_ERR_INVALID_ARG, "flow must be GGEM_FLOW_NONE, _SHEAR or _POISEUILLE");
}

void traction_dev(ggem_plan_t* P, double shear_modulus, double* df) {
    const int n = P->n_nodes;
    k_traction<<<nblk(n), CB, 0, P->st>>>(n, P->d_x, P->d_tri, P->d_mref, P->d_adj_start,
                                          P->d_adj, P->d_area, shear_modulus, df);
    GG_CUDA(cudaGetLastError());
    P->launches += 1;
}

void undisturbed_dev(ggem_plan_t* P, int flow, double s, double* u, double* f) {
    const int n = P->n_nodes;
    k_undisturbed<<<nblk(n), CB, 0, P->st>>>(n, P->d_x, P->d_nrm, flow, s, P->prm.mu,
                                             P->prm.y0, P->prm.W, u, f);
    GG_CUDA(cudaGetLastError());
    P->launches += 1;
}

// One stage at the plan's current mesh: velocity u_inf + S q into d_cw (u_inf
// in d_cuinf, S q in d_cw); q (device) is the solve's guess and its result.
void stage_velocity(ggem_plan_t* P, const ggem_step_params& sp, const double* lam, double* q,
                    int* its, double* rr) {
    const int n = P->n_nodes;
    traction_dev(P, sp.shear_modulus, P->d_cdf);
    undisturbed_dev(P, sp.flow, sp.strength, P->d_cuinf, P->d_cfinf);
    k_capsule_rhs<<<nblk(n), CB, 0, P->st>>>(n, lam, P->d_cdf, P->d_cfinf, P->prm.mu,
                                             P->d_ckap, P->d_cb);
    GG_CUDA(cudaGetLastError());
    P->launches += 1;
    const ggem_status s = bie_solve(P, P->d_ckap, P->d_cb, q, sp.tol, sp.restart, sp.maxit,
                                    sp.use_mlp, its, rr);
    GG_CHECK(s == GGEM_OK || s == GGEM_OK_BREAKDOWN, s,
             std::string("Fredholm solve of a stage: ") + ggem_last_error(P));
    single_layer_dev(P, q, P->d_cw);
}

void check_step(ggem_plan_t* P, const ggem_step_params* sp, const double* lambda) {
    GG_CHECK(P->mesh_ready && P->n_tris > 0, GGEM_ERR_INVALID_ARG, "needs a triangle mesh");
    GG_CHECK(P->mref_ready, GGEM_ERR_INVALID_ARG,
             "no membrane reference for this mesh (ggem_membrane_reference)");
    GG_CHECK(sp && lambda, GGEM_ERR_INVALID_ARG, "NULL parameters or lambda");
    check_flow(P, sp->flow);
    GG_CHECK(std::isfinite(sp->strength) && std::isfinite(sp->shear_modulus) &&
                 sp->shear_modulus >= 0.0,
             GGEM_ERR_INVALID_ARG, "strength and shear modulus must be finite, G >= 0");
}

// the per-particle triangle lists (CSR, ascending), from the particle ids
void tri_lists(ggem_plan_t* P) {
    if (P->tcsr_ready) return;
    const int np = P->n_particles, n = P->n_nodes, m = P->n_tris;
    std::vector<int> part(n), tri((size_t)3 * m), start(np + 1, 0), list(m);
    GG_CUDA(cudaMemcpyAsync(part.data(), P->d_particle, (size_t)n * sizeof(int),
                            cudaMemcpyDeviceToHost, P->st));
    GG_CUDA(cudaMemcpyAsync(tri.data(), P->d_tri, (size_t)3 * m * sizeof(int),
                            cudaMemcpyDeviceToHost, P->st));
    GG_CUDA(cudaStreamSynchronize(P->st));
    for (int k = 0; k < m; ++k) start[part[tri[3 * (size_t)k]] + 1]++;
    for (int p = 0; p < np; ++p) start[p + 1] += start[p];
    std::vector<int> cur(start.begin(), start.end() - 1);
    for (int k = 0; k < m; ++k) list[cur[part[tri[3 * (size_t)k]]]++] = k;
    dfree(P->d_tstart);
    dfree(P->d_tlist);
    dfree(P->d_cvol);
    P->d_tstart = P->d_tlist = nullptr;
    P->d_cvol = nullptr;
    dalloc(P, &P->d_tstart, (size_t)np + 1);
    dalloc(P, &P->d_tlist, (size_t)std::max(m, 1));
    dalloc(P, &P->d_cvol, (size_t)2 * np + 1);
    GG_CUDA(cudaMemcpyAsync(P->d_tstart, start.data(), (size_t)(np + 1) * sizeof(int),
                            cudaMemcpyHostToDevice, P->st));
    GG_CUDA(cudaMemcpyAsync(P->d_tlist, list.data(), (size_t)m * sizeof(int),
                            cudaMemcpyHostToDevice, P->st));
    GG_CUDA(cudaStreamSynchronize(P->st));
    P->tcsr_ready = true;
}

void volumes_dev(ggem_plan_t* P, double* vol, double* surf) {
    k_volumes<<<P->n_particles, CB, 0, P->st>>>(P->d_tstart, P->d_tlist, P->d_x, P->d_tri,
                                                P->d_tri_area, vol, surf);
    GG_CUDA(cudaGetLastError());
    P->launches += 1;
}

void copy_host_or_device(ggem_plan_t* P, double* dst, const double* src, size_t n, bool to_dev) {
    cudaMemcpyKind k;
    if (to_dev) k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    else k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    GG_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), k, P->st));
}

}  // namespace

extern "C" {

ggem_status ggem_membrane_reference(ggem_plan_t* P, const double* x_ref) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready && P->n_tris > 0, GGEM_ERR_INVALID_ARG, "needs a triangle mesh");
        GG_CHECK(x_ref, GGEM_ERR_INVALID_ARG, "NULL reference positions");
        ensure_capsule_ws(P);
        if (!P->d_mref) dalloc(P, &P->d_mref, (size_t)4 * P->cap_tris);
        const double* xr = stage_in(P, x_ref, P->d_cw, (size_t)3 * P->n_nodes);
        k_membrane_ref<<<nblk(P->n_tris), CB, 0, P->st>>>(P->n_tris, xr, P->d_tri, P->d_mref);
        GG_CUDA(cudaGetLastError());
        P->launches += 1;
        GG_CUDA(cudaStreamSynchronize(P->st));
        P->mref_ready = true;
    });
}

ggem_status ggem_membrane_traction(ggem_plan_t* P, double shear_modulus, double* df) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready && P->n_tris > 0 && P->mref_ready, GGEM_ERR_INVALID_ARG,
                 "needs a triangle mesh and its membrane reference");
        GG_CHECK(df, GGEM_ERR_INVALID_ARG, "NULL output");
        const size_t n3 = (size_t)3 * P->n_nodes;
        OutMap mo = stage_out(df, P->d_out0, n3);
        traction_dev(P, shear_modulus, mo.dev);
        finish_out(P, mo);
        GG_CUDA(cudaStreamSynchronize(P->st));
    });
}

ggem_status ggem_undisturbed(ggem_plan_t* P, int flow, double strength, double* u_inf,
                             double* f_inf) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready, GGEM_ERR_INVALID_ARG, "no mesh set");
        GG_CHECK(!f_inf || P->n_tris > 0, GGEM_ERR_INVALID_ARG,
                 "the traction needs node normals (triangles)");
        check_flow(P, flow);
        const size_t n3 = (size_t)3 * P->n_nodes;
        OutMap mu = stage_out(u_inf, P->d_out0, n3);
        OutMap mf = stage_out(f_inf, P->d_out1, n3);
        undisturbed_dev(P, flow, strength, u_inf ? mu.dev : nullptr, f_inf ? mf.dev : nullptr);
        if (u_inf) finish_out(P, mu);
        if (f_inf) finish_out(P, mf);
        GG_CUDA(cudaStreamSynchronize(P->st));
    });
}

ggem_status ggem_capsule_velocity(ggem_plan_t* P, const ggem_step_params* sp,
                                  const double* lambda, double* q, double* u, int* iters,
                                  double* true_relres) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        check_step(P, sp, lambda);
        GG_CHECK(q && u, GGEM_ERR_INVALID_ARG, "NULL q or u");
        ensure_capsule_ws(P);
        const int n = P->n_nodes;
        const size_t n3 = (size_t)3 * n;
        const double* lam = stage_in(P, lambda, P->d_clam, (size_t)n);
        const bool qh = !is_device_ptr(q);
        double* qd = qh ? P->d_cq : q;
        if (qh) copy_host_or_device(P, qd, q, n3, true);
        int its = 0;
        double rr = 0.0;
        stage_velocity(P, *sp, lam, qd, &its, &rr);
        OutMap mo = stage_out(u, P->d_out0, n3);
        k_advance<<<nblk(n3), CB, 0, P->st>>>((int)n3, nullptr, P->d_cuinf, P->d_cw, 1.0,
                                              mo.dev);
        GG_CUDA(cudaGetLastError());
        P->launches += 1;
        finish_out(P, mo);
        if (qh) copy_host_or_device(P, q, qd, n3, false);
        GG_CUDA(cudaStreamSynchronize(P->st));
        if (iters) *iters = its;
        if (true_relres) *true_relres = rr;
    });
}

ggem_status ggem_capsule_step(ggem_plan_t* P, const ggem_step_params* sp, const double* lambda,
                              double* q, double* x_out, int* iters, double* true_relres) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        check_step(P, sp, lambda);
        GG_CHECK(q, GGEM_ERR_INVALID_ARG, "NULL q");
        GG_CHECK(std::isfinite(sp->dt) && sp->dt > 0.0, GGEM_ERR_INVALID_ARG, "dt must be > 0");
        ensure_capsule_ws(P);
        const int n = P->n_nodes;
        const size_t n3 = (size_t)3 * n;
        const double* lam = stage_in(P, lambda, P->d_clam, (size_t)n);
        const bool qh = !is_device_ptr(q);
        double* qd = qh ? P->d_cq : q;
        if (qh) copy_host_or_device(P, qd, q, n3, true);
        GG_CUDA(cudaMemcpyAsync(P->d_cx0, P->d_x, n3 * sizeof(double), cudaMemcpyDeviceToDevice,
                                P->st));
        int i1 = 0, i2 = 0;
        double r1 = 0.0, r2 = 0.0;
        // stage 1 at x: x_half = x + dt/2 u(x)
        stage_velocity(P, *sp, lam, qd, &i1, &r1);
        k_advance<<<nblk(n3), CB, 0, P->st>>>((int)n3, P->d_cx0, P->d_cuinf, P->d_cw,
                                              0.5 * sp->dt, P->d_x);
        GG_CUDA(cudaGetLastError());
        P->launches += 1;
        ggem_status s = ggem_mesh_set(P, n, P->d_x, P->n_tris, P->d_tri);
        GG_CHECK(s == GGEM_OK, s, std::string("midpoint mesh: ") + ggem_last_error(P));
        // stage 2 at x_half (guess: stage 1's density): x_new = x + dt u(x_half)
        stage_velocity(P, *sp, lam, qd, &i2, &r2);
        k_advance<<<nblk(n3), CB, 0, P->st>>>((int)n3, P->d_cx0, P->d_cuinf, P->d_cw, sp->dt,
                                              P->d_x);
        GG_CUDA(cudaGetLastError());
        P->launches += 1;
        s = ggem_mesh_set(P, n, P->d_x, P->n_tris, P->d_tri);
        GG_CHECK(s == GGEM_OK, s, std::string("new mesh: ") + ggem_last_error(P));
        if (x_out) copy_host_or_device(P, x_out, P->d_x, n3, false);
        if (qh) copy_host_or_device(P, q, qd, n3, false);
        GG_CUDA(cudaStreamSynchronize(P->st));
        if (iters) *iters = i1 + i2;
        if (true_relres) *true_relres = std::max(r1, r2);
    });
}

ggem_status ggem_mesh_positions(const ggem_plan_t* plan, double* x) {
    if (!plan) return GGEM_ERR_INVALID_ARG;
    ggem_plan_t* P = const_cast<ggem_plan_t*>(plan);   // error message only
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready && x, GGEM_ERR_INVALID_ARG, "no mesh set or NULL output");
        copy_host_or_device(P, x, P->d_x, (size_t)3 * P->n_nodes, false);
        GG_CUDA(cudaStreamSynchronize(P->st));
    });
}

ggem_status ggem_min_separation(ggem_plan_t* P, double* h_min) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready && h_min, GGEM_ERR_INVALID_ARG, "no mesh set or NULL output");
        ensure_capsule_ws(P);
        const unsigned long long inf = (unsigned long long)0x7ff0000000000000ull;
        GG_CUDA(cudaMemcpyAsync(P->d_cmin, &inf, sizeof(inf), cudaMemcpyHostToDevice, P->st));
        const int n = P->n_nodes;
        k_min_sep<<<nblk(n), CB, 0, P->st>>>(n, P->geo, P->cg, P->d_mesh_cell, P->d_mesh_start,
                                             P->d_mesh_perm, P->d_x, P->d_cmin);
        GG_CUDA(cudaGetLastError());
        P->launches += 1;
        unsigned long long bits = 0;
        GG_CUDA(cudaMemcpyAsync(&bits, P->d_cmin, sizeof(bits), cudaMemcpyDeviceToHost, P->st));
        GG_CUDA(cudaStreamSynchronize(P->st));
        double h;
        std::memcpy(&h, &bits, sizeof(h));
        // no pair within neighbouring cells: the separation is at least a cell
        *h_min = std::min(h, std::min(P->cg.hx, std::min(P->cg.hy, P->cg.hz)));
    });
}

ggem_status ggem_particle_volumes(ggem_plan_t* P, double* volumes) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready && P->n_tris > 0, GGEM_ERR_INVALID_ARG, "needs a triangle mesh");
        GG_CHECK(P->d_particle && P->particles_n == P->n_nodes, GGEM_ERR_INVALID_ARG,
                 "particle ids not set for this mesh (ggem_mesh_particles)");
        GG_CHECK(volumes, GGEM_ERR_INVALID_ARG, "NULL output");
        tri_lists(P);
        volumes_dev(P, P->d_cvol, nullptr);
        copy_host_or_device(P, volumes, P->d_cvol, (size_t)P->n_particles, false);
        GG_CUDA(cudaStreamSynchronize(P->st));
    });
}

ggem_status ggem_volume_correct(ggem_plan_t* P, const double* v0, double threshold,
                                int max_passes, int* passes) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready && P->n_tris > 0, GGEM_ERR_INVALID_ARG, "needs a triangle mesh");
        GG_CHECK(P->d_particle && P->particles_n == P->n_nodes, GGEM_ERR_INVALID_ARG,
                 "particle ids not set for this mesh (ggem_mesh_particles)");
        GG_CHECK(v0 && threshold >= 0.0 && max_passes >= 0, GGEM_ERR_INVALID_ARG,
                 "needs v0, threshold >= 0 and max_passes >= 0");
        ensure_capsule_ws(P);
        tri_lists(P);
        const int np = P->n_particles, n = P->n_nodes;
        std::vector<double> ref(np), vs(2 * (size_t)np), d(np);
        if (is_device_ptr(v0)) {
            GG_CUDA(cudaMemcpyAsync(ref.data(), v0, np * sizeof(double), cudaMemcpyDeviceToHost,
                                    P->st));
            GG_CUDA(cudaStreamSynchronize(P->st));
        } else {
            std::copy(v0, v0 + np, ref.begin());
        }
        int k = 0;
        for (; k < max_passes; ++k) {
            volumes_dev(P, P->d_cvol, P->d_cvol + np);
            GG_CUDA(cudaMemcpyAsync(vs.data(), P->d_cvol, 2 * (size_t)np * sizeof(double),
                                    cudaMemcpyDeviceToHost, P->st));
            GG_CUDA(cudaStreamSynchronize(P->st));
            bool any = false;
            for (int p = 0; p < np; ++p) {
                const bool off = std::fabs(vs[p] - ref[p]) > threshold * std::fabs(ref[p]);
                d[p] = off ? (ref[p] - vs[p]) / vs[np + p] : 0.0;
                any = any || off;
            }
            if (!any) break;
            // shifts go through the traction buffer (3 cap >= n_particles)
            GG_CUDA(cudaMemcpyAsync(P->d_cdf, d.data(), np * sizeof(double),
                                    cudaMemcpyHostToDevice, P->st));
            k_normal_shift<<<nblk(n), CB, 0, P->st>>>(n, P->d_particle, P->d_cdf, P->d_nrm,
                                                      P->d_x);
            GG_CUDA(cudaGetLastError());
            P->launches += 1;
            const ggem_status s = ggem_mesh_set(P, n, P->d_x, P->n_tris, P->d_tri);
            GG_CHECK(s == GGEM_OK, s, std::string("corrected mesh: ") + ggem_last_error(P));
        }
        if (passes) *passes = k;
    });
}

ggem_status ggem_overlap_correct(ggem_plan_t* P, double h_min, int max_sweeps, int* moves) {
    if (!P) return GGEM_ERR_INVALID_ARG;
    return guarded(P, [&] {
        GG_CHECK(P->mesh_ready, GGEM_ERR_INVALID_ARG, "no mesh set");
        GG_CHECK(P->d_particle && P->particles_n == P->n_nodes, GGEM_ERR_INVALID_ARG,
                 "particle ids not set for this mesh (ggem_mesh_particles)");
        GG_CHECK(h_min > 0.0 && h_min <= std::min(P->cg.hx, std::min(P->cg.hy, P->cg.hz)),
                 GGEM_ERR_INVALID_ARG, "h_min must be positive and at most a cell width");
        GG_CHECK(max_sweeps >= 0, GGEM_ERR_INVALID_ARG, "max_sweeps must be >= 0");
        particle_node_lists(P);
        const int n = P->n_nodes, np = P->n_particles;
        const int cap = kGapSlots * P->cap;
        if (!P->d_orec) {
            dalloc(P, &P->d_orec, (size_t)2 * cap);
            dalloc(P, &P->d_orecd, (size_t)cap);
            dalloc(P, &P->d_ocount, 2);
        }
        dfree(P->d_odisp);
        P->d_odisp = nullptr;
        dalloc(P, &P->d_odisp, (size_t)3 * np);
        std::vector<double> c(3 * (size_t)np), disp(3 * (size_t)np);
        std::vector<int> rec;
        std::vector<double> recd;
        const double hthr = h_min * (1.0 - 1e-9);   // corrected gaps land on h_min
        int total = 0;
        for (int sweep = 0; sweep < max_sweeps; ++sweep) {
            GG_CUDA(cudaMemsetAsync(P->d_ocount, 0, 2 * sizeof(int), P->st));
            k_gap_pairs<<<nblk(n), CB, 0, P->st>>>(n, P->geo, P->cg, P->d_mesh_cell,
                                                   P->d_mesh_start, P->d_mesh_perm,
                                                   P->d_particle, P->d_x, hthr, cap, P->d_orec,
                                                   P->d_orecd, P->d_ocount);
            k_centroids<<<np, CB, 0, P->st>>>(P->d_pstart, P->d_pnodes, P->d_x, P->d_odisp);
            GG_CUDA(cudaGetLastError());
            P->launches += 2;
            int cnt2[2] = {0, 0};
            GG_CUDA(cudaMemcpyAsync(cnt2, P->d_ocount, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                    P->st));
            GG_CUDA(cudaMemcpyAsync(c.data(), P->d_odisp, c.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost, P->st));
            GG_CUDA(cudaStreamSynchronize(P->st));
            const int cnt = cnt2[0];
            GG_CHECK(cnt <= cap, GGEM_ERR_CAPACITY, "overlap records overflowed");
            GG_CHECK(cnt2[1] == 0, GGEM_ERR_CAPACITY,
                     "a node is within h_min of more than 4 other particles");
            if (cnt == 0) break;
            rec.resize(2 * (size_t)cnt);
            recd.resize(cnt);
            GG_CUDA(cudaMemcpyAsync(rec.data(), P->d_orec, rec.size() * sizeof(int),
                                    cudaMemcpyDeviceToHost, P->st));
            GG_CUDA(cudaMemcpyAsync(recd.data(), P->d_orecd, recd.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost, P->st));
            GG_CUDA(cudaStreamSynchronize(P->st));
            // smallest gap of every violating pair, in pair order
            std::vector<std::pair<std::pair<int, int>, double>> pairs(cnt);
            for (int r = 0; r < cnt; ++r) pairs[r] = {{rec[2 * r], rec[2 * r + 1]}, recd[r]};
            std::sort(pairs.begin(), pairs.end());
            std::fill(disp.begin(), disp.end(), 0.0);
            int found = 0;
            for (size_t r = 0; r < pairs.size(); ++r) {
                if (r > 0 && pairs[r].first == pairs[r - 1].first) continue;   // sorted: first is min
                const int p = pairs[r].first.first, q = pairs[r].first.second;
                const double gap = pairs[r].second;
                double d[3];
                for (int k = 0; k < 3; ++k) d[k] = c[3 * q + k] - c[3 * p + k];
                d[0] -= P->geo.Lx * std::nearbyint(d[0] / P->geo.Lx);
                d[2] -= P->geo.Lz * std::nearbyint(d[2] / P->geo.Lz);
                const double len = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                const double sh = 0.5 * (h_min - gap) / len;
                for (int k = 0; k < 3; ++k) {
                    disp[3 * p + k] -= sh * d[k];
                    disp[3 * q + k] += sh * d[k];
                }
                ++found;
            }
            GG_CUDA(cudaMemcpyAsync(P->d_odisp, disp.data(), disp.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, P->st));
            k_translate<<<nblk(n), CB, 0, P->st>>>(n, P->d_particle, P->d_odisp, P->d_x);
            GG_CUDA(cudaGetLastError());
            P->launches += 1;
            const ggem_status s = ggem_mesh_set(P, n, P->d_x, P->n_tris, P->d_tri);
            GG_CHECK(s == GGEM_OK, s, std::string("corrected mesh: ") + ggem_last_error(P));
            total += found;
        }
        if (moves) *moves = total;
    });
}

}  // extern "C"
