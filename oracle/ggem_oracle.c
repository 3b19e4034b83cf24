/*
 * GGEM oracle, part 1: the pair sums, written plainly in FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct CPU
 * reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the bench's CPU-baseline leg may load it; the library
 * path never does.  It shares no code with the CUDA sources.
 *
 * Paper: Kumar & Graham, "Accelerated boundary integral method for
 * multiphase flow in non-periodic geometries" (arXiv 1109.6587).
 *   - local kernels G^l, P^l, T^l ............ Eq. (local), Sec. 3.2.1
 *   - local sums u^l, sigma^l ................ Eq. (u_loc), Sec. 3.2.1
 *   - cutoff r_cut = 4/alpha, minimum image .. Sec. 3.2.1, Sec. 3.2.2
 *   - global density rho_g ................... Eq. (rho_l_g)
 *   - spreading onto the grid ................ Eqs. (rho_int), (rhog_sum)
 *   - element quadrature, polar map .......... Eq. (int_l), Sec. 3.4.1
 *   - double layer with n-tilde .............. Eqs. (dbl_l1), (ntilde)
 *
 * Readings fixed here (the paper is silent or loose):
 *   - a pair (target z, source x) contributes iff 0 < |z - x*| < r_cut,
 *     where x* is the minimum image of x in the periodic x and z directions;
 *   - grid nodes receive rho_g iff |node - x*| < r_cut;
 *   - in the element rule every quadrature point is a point source and the
 *     cutoff test is applied to it (regular and polar points alike);
 *   - the collapsed-triangle map of Eq. (int_l) is xi = (1-eta) s, with
 *     Jacobian (1-eta) * |x_xi x x_eta|.
 * All units: mu = viscosity; velocities from forces g are (1/8 pi mu) G g.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double Lx, Lz, W, y0;
    int Nx, Ny, Nz;
} orc_box;

static const double PI = 3.14159265358979323846;

/* minimum image in the periodic x and z directions (Sec. 3.2.2) */
static void min_image(const orc_box *b, double d[3]) {
    d[0] -= b->Lx * nearbyint(d[0] / b->Lx);
    d[2] -= b->Lz * nearbyint(d[2] / b->Lz);
}

/* G^l_ij of Eq. (local a); G[3*i+j] */
void orc_Gl(double a, const double *x, double *G) {
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double r = sqrt(r2);
    double ec = erfc(a * r), ex = exp(-a * a * r2);
    double c = 2.0 * a / sqrt(PI);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double d = (i == j) ? 1.0 : 0.0;
            G[3 * i + j] = (d / r + x[i] * x[j] / (r2 * r)) * ec
                           - c * (d - x[i] * x[j] / r2) * ex;
        }
}

/* P^l_j of Eq. (local b) */
void orc_Pl(double a, const double *x, double *P) {
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double r = sqrt(r2);
    double ec = erfc(a * r), ex = exp(-a * a * r2);
    for (int j = 0; j < 3; j++)
        P[j] = 2.0 * x[j] / (r2 * r) * ec
               + 4.0 * a * x[j] / sqrt(PI) * (1.0 / r2 - a * a) * ex;
}

/* T^l_ijk of Eq. (local c); T[9*i+3*j+k] */
void orc_Tl(double a, const double *x, double *T) {
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double r = sqrt(r2);
    double ec = erfc(a * r), ex = exp(-a * a * r2);
    double sp = sqrt(PI);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) {
                double xxx = x[i] * x[j] * x[k];
                double djk = (j == k), dik = (i == k), dij = (i == j);
                T[9 * i + 3 * j + k] =
                    -6.0 * xxx / (r2 * r2 * r) * ec
                    - 12.0 * a / sp * xxx / (r2 * r2) * ex
                    + 4.0 * a * a * a / sp
                          * (djk * x[i] + dik * x[j] + dij * x[k] - 2.0 * xxx / r2) * ex;
            }
}

/* rho_g of Eq. (rho_l_g a), as a function of r^2 */
double orc_rhog(double a, double r2) {
    return a * a * a / pow(PI, 1.5) * exp(-a * a * r2) * (2.5 - a * a * r2);
}

/* batched pointwise kernels, for the identity tests */
void orc_kernels_batch(double a, int n, const double *x, double *G, double *P,
                       double *T) {
    for (int p = 0; p < n; p++) {
        if (G) orc_Gl(a, x + 3 * p, G + 9 * p);
        if (P) orc_Pl(a, x + 3 * p, P + 3 * p);
        if (T) orc_Tl(a, x + 3 * p, T + 27 * p);
    }
}

/*
 * Local point-force sums, Eq. (u_loc):
 *   u_i(z)      = 1/(8 pi mu) sum_nu G^l_ij(z - x_nu*) g_nu_j
 *   sigma_ik(z) = 1/(8 pi)    sum_nu T^l_ijk(z - x_nu*) g_nu_j
 * over pairs with 0 < r < rcut.  u: [nt][3], sig: [nt][3][3] (either NULL).
 */
void orc_local_point(const orc_box *b, double a, double rcut, double mu, int ns,
                     const double *xs, const double *g, int nt, const double *xt,
                     double *u, double *sig) {
    double rc2 = rcut * rcut;
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < nt; t++) {
        double ut[3] = {0, 0, 0}, st[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        double G[9], T[27];
        for (int s = 0; s < ns; s++) {
            double d[3] = {xt[3 * t] - xs[3 * s], xt[3 * t + 1] - xs[3 * s + 1],
                           xt[3 * t + 2] - xs[3 * s + 2]};
            min_image(b, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 > 0.0 && r2 < rc2)) continue;
            const double *gs = g + 3 * s;
            if (u) {
                orc_Gl(a, d, G);
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) ut[i] += G[3 * i + j] * gs[j];
            }
            if (sig) {
                orc_Tl(a, d, T);
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++)
                        for (int k = 0; k < 3; k++)
                            st[3 * i + k] += T[9 * i + 3 * j + k] * gs[j];
            }
        }
        if (u)
            for (int i = 0; i < 3; i++) u[3 * t + i] = ut[i] / (8.0 * PI * mu);
        if (sig)
            for (int i = 0; i < 9; i++) sig[9 * t + i] = st[i] / (8.0 * PI);
    }
}

/*
 * Spreading of the global density onto the grid, Eq. (stokes_gg):
 * the global problem is  -grad p + mu lap u = f  with
 *   f(node) = - sum_nu g_nu rho_g(node - x_nu*),   |node - x_nu*| < rcut.
 * Nodes: x_i = i Lx/Nx, z_k = k Lz/Nz, y_j = y0 + W/2 (1 + cos(pi j/(Ny-1))).
 * f layout: [3][Ny][Nz][Nx].
 */
void orc_spread(const orc_box *b, double a, double rcut, int ns, const double *xs,
                const double *g, double *f) {
    int Nx = b->Nx, Ny = b->Ny, Nz = b->Nz;
    size_t plane = (size_t)Nz * Nx, comp = (size_t)Ny * plane;
    memset(f, 0, 3 * comp * sizeof(double));
    double rc2 = rcut * rcut;
    /* each y-plane is filled by one thread, so no two threads touch a node */
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < Ny; j++) {
        double yj = b->y0 + 0.5 * b->W * (1.0 + cos(PI * j / (Ny - 1)));
        int *ix = malloc(Nx * sizeof(int)), *iz = malloc(Nz * sizeof(int));
        double *dxs = malloc(Nx * sizeof(double)), *dzs = malloc(Nz * sizeof(double));
        for (int s = 0; s < ns; s++) {
            double dy = yj - xs[3 * s + 1];
            if (!(dy * dy < rc2)) continue;
            /* candidate columns: nodes whose minimum-image offset is below rcut */
            int nxc = 0, nzc = 0;
            for (int i = 0; i < Nx; i++) {
                double d[3] = {i * b->Lx / Nx - xs[3 * s], 0.0, 0.0};
                min_image(b, d);
                if (fabs(d[0]) < rcut) { ix[nxc] = i; dxs[nxc++] = d[0]; }
            }
            for (int k = 0; k < Nz; k++) {
                double d[3] = {0.0, 0.0, k * b->Lz / Nz - xs[3 * s + 2]};
                min_image(b, d);
                if (fabs(d[2]) < rcut) { iz[nzc] = k; dzs[nzc++] = d[2]; }
            }
            for (int kk = 0; kk < nzc; kk++)
                for (int ii = 0; ii < nxc; ii++) {
                    double r2 = dxs[ii] * dxs[ii] + dy * dy + dzs[kk] * dzs[kk];
                    if (!(r2 < rc2)) continue;
                    double rho = orc_rhog(a, r2);
                    size_t o = (size_t)j * plane + (size_t)iz[kk] * Nx + ix[ii];
                    for (int c = 0; c < 3; c++) f[c * comp + o] -= g[3 * s + c] * rho;
                }
        }
        free(ix); free(iz); free(dxs); free(dzs);
    }
}

/* n-point Gauss-Legendre rule on [0,1] by Newton iteration on P_n */
void orc_gauss_legendre01(int n, double *t, double *w) {
    for (int i = 0; i < n; i++) {
        double x = cos(PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            /* p1 = P_n(x), p0 = P_{n-1}(x) */
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        t[i] = 0.5 * (1.0 - x);
        w[i] = 1.0 / ((1.0 - x * x) * dp * dp);   /* = 2/((1-x^2)P'^2) / 2 */
    }
}

static void cross(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/*
 * Local part of the single layer (layer=0), Eq. (int_l):
 *   w_j(z) = sum_k int_{S_k} q_i G^l_ji(z, x) dS
 * or of the double layer (layer=1), Eqs. (int_dbl_l), (dbl_l1), (ntilde):
 *   v_j(z) = n_k(z) sum_k int_{S_k} q_i T^l_jik(z, x) dS   (regular elements)
 *            sum_k int_{S_k} q_i T^l_jik(z, x) ntilde_k dS   (elements with z
 *            as a vertex, ntilde = n_tri phi1 + n(z)(phi2 + phi3)).
 * Regular elements: 4x4 Gauss-Legendre product rule on the collapsed triangle.
 * Elements with the target as a vertex: the same rule in polar coordinates
 * (rho, theta) about that vertex (Sec. 3.4.1).  Targets are the nodes listed in
 * tgt (nt of them); out: [nt][3].  nrm: [nn][3] node normals (double only).
 */
void orc_local_elem(const orc_box *b, double a, double rcut, int layer, int nn,
                    const double *x, int ne, const int *tri, const double *q,
                    const double *nrm, int nt, const int *tgt, double *out) {
    (void)nn;
    const int NQ = 4;
    double tg[4], wg[4];
    orc_gauss_legendre01(NQ, tg, wg);
    double rc2 = rcut * rcut;
#pragma omp parallel for schedule(dynamic, 4)
    for (int it = 0; it < nt; it++) {
        int bt = tgt[it];
        const double *z = x + 3 * bt;
        double acc[3] = {0, 0, 0};
        double G[9], T[27];
        for (int k = 0; k < ne; k++) {
            int v0 = tri[3 * k], v1 = tri[3 * k + 1], v2 = tri[3 * k + 2];
            /* conservative skip: no point of the element can be within rcut */
            double cen[3], rad = 0.0;
            for (int c = 0; c < 3; c++)
                cen[c] = (x[3 * v0 + c] + x[3 * v1 + c] + x[3 * v2 + c]) / 3.0;
            int vs[3] = {v0, v1, v2};
            for (int p = 0; p < 3; p++) {
                double e[3] = {x[3 * vs[p]] - cen[0], x[3 * vs[p] + 1] - cen[1],
                               x[3 * vs[p] + 2] - cen[2]};
                double l = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
                if (l > rad) rad = l;
            }
            double dc[3] = {z[0] - cen[0], z[1] - cen[1], z[2] - cen[2]};
            min_image(b, dc);
            if (sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]) > rcut + rad + 1e-12)
                continue;
            int adjacent = (v0 == bt || v1 == bt || v2 == bt);
            /* label the target as vertex 1 (cyclic rotation keeps orientation) */
            int i1 = v0, i2 = v1, i3 = v2;
            if (v1 == bt) { i1 = v1; i2 = v2; i3 = v0; }
            else if (v2 == bt) { i1 = v2; i2 = v0; i3 = v1; }
            const double *x1 = x + 3 * i1, *x2 = x + 3 * i2, *x3 = x + 3 * i3;
            double e2[3] = {x2[0] - x1[0], x2[1] - x1[1], x2[2] - x1[2]};
            double e3[3] = {x3[0] - x1[0], x3[1] - x1[1], x3[2] - x1[2]};
            double nt_[3];
            cross(e2, e3, nt_);
            double omega = sqrt(nt_[0] * nt_[0] + nt_[1] * nt_[1] + nt_[2] * nt_[2]);
            double ntri[3] = {nt_[0] / omega, nt_[1] / omega, nt_[2] / omega};
            for (int qa = 0; qa < NQ; qa++)
                for (int qc = 0; qc < NQ; qc++) {
                    double xi, eta, wgt;
                    if (adjacent) {
                        double th = 0.5 * PI * tg[qa];
                        double rmax = 1.0 / (cos(th) + sin(th));
                        double rho = rmax * tg[qc];
                        xi = rho * cos(th);
                        eta = rho * sin(th);
                        wgt = 0.5 * PI * wg[qa] * rmax * wg[qc] * rho * omega;
                    } else {
                        eta = tg[qc];
                        xi = (1.0 - eta) * tg[qa];
                        wgt = wg[qa] * wg[qc] * (1.0 - eta) * omega;
                    }
                    double p1 = 1.0 - xi - eta, p2 = xi, p3 = eta;
                    double xq[3], qq[3];
                    for (int c = 0; c < 3; c++) {
                        xq[c] = p1 * x1[c] + p2 * x2[c] + p3 * x3[c];
                        qq[c] = p1 * q[3 * i1 + c] + p2 * q[3 * i2 + c] + p3 * q[3 * i3 + c];
                    }
                    double d[3] = {z[0] - xq[0], z[1] - xq[1], z[2] - xq[2]};
                    min_image(b, d);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (!(r2 > 0.0 && r2 < rc2)) continue;
                    if (layer == 0) {
                        orc_Gl(a, d, G);
                        for (int j = 0; j < 3; j++)
                            for (int i = 0; i < 3; i++) acc[j] += G[3 * j + i] * qq[i] * wgt;
                    } else {
                        double nv[3];
                        const double *nz = nrm + 3 * bt;
                        for (int c = 0; c < 3; c++)
                            nv[c] = adjacent ? (ntri[c] * p1 + nz[c] * (p2 + p3)) : nz[c];
                        orc_Tl(a, d, T);
                        for (int j = 0; j < 3; j++)
                            for (int i = 0; i < 3; i++)
                                for (int kk = 0; kk < 3; kk++)
                                    acc[j] += T[9 * j + 3 * i + kk] * qq[i] * nv[kk] * wgt;
                    }
                }
        }
        for (int c = 0; c < 3; c++) out[3 * it + c] = acc[c];
    }
}
