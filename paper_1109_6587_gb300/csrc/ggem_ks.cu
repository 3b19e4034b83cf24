// Per-Fourier-mode Chebyshev-tau Kleiser-Schumann Stokes solve (paper App. C)
// and spectral stress assembly (Sec. 3.5.1), in FP64.
//
// For each mode (k_x, k_z) the tau system of (D_y^2 - k^2) a = r with the two
// highest equations replaced by the wall values is solved in O(N) by the
// even/odd quasi-tridiagonal form: the identity
//   a_n = c_{n-2} d_{n-2} / (4n(n-1)) - e_{n+2} d_n / (2(n^2-1))
//         + e_{n+4} d_{n+2} / (4n(n+1)),        n >= 2,
// between the coefficients a of a degree-N series and d of its second
// derivative (e_m = 1 for m <= N, else 0) turns rows 0..N-2 of the tau system
// into a tridiagonal recurrence within each parity; the two wall rows become
// one full row per parity (sum of the even / odd coefficients).  This is the
// same discrete system as the dense tau matrix, rearranged.
//
// Steps per mode (App. C, Eqs. (stokes_t_all), (bc_vel), (inf_mat), (cheb_sol)):
//   p_a: (D^2 - k^2) p = -(i kx fx + D fy + i kz fz), p = 0 at the walls
//   u_a, v_a, w_a: mu (D^2 - k^2) u = f + grad p_a, u = wall data
//   p_1, p_2 from the precomputed inverse influence matrix and the
//   divergence of the a-solution at both walls; combine with the stored
//   homogeneous b-solution and its mirror image (the c-solution).
// Mode k = 0: mu D^2 u = f_x, mu D^2 w = f_z with wall values, v linear
// between its wall values, D p = -f_y with zero mean over y.
// The Nyquist mode in z is zero.
#include "ggem_internal.cuh"

namespace ggem {

struct dc {
    double x, y;
};
__host__ __device__ __forceinline__ dc mkc(double a, double b) { dc r; r.x = a; r.y = b; return r; }
__host__ __device__ __forceinline__ dc operator+(dc a, dc b) { return mkc(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ dc operator-(dc a, dc b) { return mkc(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ dc operator*(double s, dc a) { return mkc(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ dc times_i(double k, dc a) { return mkc(-k * a.y, k * a.x); }

// Strided views: element n of a coefficient column lives at p[n * sm].
// Solve the tau system of (D^2 - lam) a = rs * r in ybar units with a(-1) = bot,
// a(+1) = top.  X (complex) and YQ (real pairs) are scratch; out may alias r.
__host__ __device__ void helm_solve(double lam, double rs, const dc* r, dc bot, dc top, dc* X,
                                    dc* YQ, dc* out, int N, size_t sm) {
    for (int p = 0; p < 2; ++p) {
        int ntop = N - ((N - p) & 1);
        dc Xn1 = mkc(0, 0);
        double Yn1 = 0.0;
        for (int n = ntop; n >= p + 2; n -= 2) {
            double c2 = (n - 2 == 0) ? 2.0 : 1.0;
            double e2 = (n + 2 <= N) ? 1.0 : 0.0;
            double e4 = (n + 4 <= N) ? 1.0 : 0.0;
            double f1 = c2 / (4.0 * n * (n - 1.0));
            double f2 = e2 / (2.0 * ((double)n * n - 1.0));
            double f3 = e4 / (4.0 * n * (n + 1.0));
            double al = -lam * f1, be = 1.0 + lam * f2, ga = -lam * f3;
            dc rho = f1 * r[(size_t)(n - 2) * sm] - f2 * r[(size_t)n * sm];
            if (n + 2 <= N) rho = rho + f3 * r[(size_t)(n + 2) * sm];
            rho = rs * rho;
            double d = be + ga * Yn1;
            double id = 1.0 / d;
            dc Xn = id * (rho - ga * Xn1);
            double Yn = -al * id;
            X[(size_t)n * sm] = Xn;
            YQ[(size_t)n * sm].x = Yn;
            Xn1 = Xn;
            Yn1 = Yn;
        }
        dc s = (p == 0) ? 0.5 * (top + bot) : 0.5 * (top - bot);
        dc Pp = mkc(0, 0), sP = mkc(0, 0);
        double Qp = 1.0, sQ = 1.0;
        for (int n = p + 2; n <= ntop; n += 2) {
            double Yn = YQ[(size_t)n * sm].x;
            dc Pn = X[(size_t)n * sm] + Yn * Pp;
            double Qn = Yn * Qp;
            X[(size_t)n * sm] = Pn;
            YQ[(size_t)n * sm].y = Qn;
            sP = sP + Pn;
            sQ += Qn;
            Pp = Pn;
            Qp = Qn;
        }
        dc t = (1.0 / sQ) * (s - sP);
        out[(size_t)p * sm] = t;
        for (int n = p + 2; n <= ntop; n += 2)
            out[(size_t)n * sm] = X[(size_t)n * sm] + YQ[(size_t)n * sm].y * t;
    }
}

// b = d/dy a = (2/W) d/dybar a in coefficient space (backward recurrence
// c_n b_n = b_{n+2} + 2 (n+1) a_{n+1}); b must not alias a.
__host__ __device__ void cheb_deriv(const dc* a, dc* b, int N, size_t sm, double scale) {
    dc b1 = mkc(0, 0), b2 = mkc(0, 0);   // b_{n+1}, b_{n+2} (unscaled)
    b[(size_t)N * sm] = mkc(0, 0);
    for (int n = N - 1; n >= 0; --n) {
        dc bn = b2 + (2.0 * (n + 1)) * a[(size_t)(n + 1) * sm];
        if (n == 0) bn = 0.5 * bn;
        b[(size_t)n * sm] = scale * bn;
        b2 = b1;
        b1 = bn;
    }
}

// Host precompute of the homogeneous b-solution of one mode: p_b with p = 1
// at the bottom wall and 0 at the top; phi_b with mu (D^2-k^2) phi = p_b
// (u_b = i kx phi_b, w_b = i kz phi_b); v_b with mu (D^2-k^2) v = D p_b; all
// with zero velocity at the walls.  Returns the inverse 2x2 influence matrix
// (the c-solution is the mirror image of b, so the matrix is [[a, b],[b, a]]).
void ks_precompute_mode(int Ny, double W, double mu, double k2, double* pb, double* phib,
                        double* vb, double* minv) {
    int N = Ny - 1;
    std::vector<dc> r(Ny), X(Ny), YQ(Ny), P(Ny), F(Ny), V(Ny), D(Ny);
    double s2 = 0.25 * W * W, lam = k2 * s2;
    for (int n = 0; n < Ny; ++n) r[n] = mkc(0, 0);
    helm_solve(lam, s2, r.data(), mkc(1, 0), mkc(0, 0), X.data(), YQ.data(), P.data(), N, 1);
    helm_solve(lam, s2 / mu, P.data(), mkc(0, 0), mkc(0, 0), X.data(), YQ.data(), F.data(), N, 1);
    cheb_deriv(P.data(), D.data(), N, 1, 2.0 / W);
    helm_solve(lam, s2 / mu, D.data(), mkc(0, 0), mkc(0, 0), X.data(), YQ.data(), V.data(), N, 1);
    double cb = 0, ct = 0;   // d v_b/dy at the bottom / top wall (phi_b is zero there)
    for (int n = 0; n < Ny; ++n) {
        double n2 = (double)n * n;
        ct += n2 * V[n].x;
        cb += ((n & 1) ? 1.0 : -1.0) * n2 * V[n].x;
        pb[n] = P[n].x;
        phib[n] = F[n].x;
        vb[n] = V[n].x;
    }
    cb *= 2.0 / W;
    ct *= 2.0 / W;
    double det = cb * cb - ct * ct;
    minv[0] = cb / det; minv[1] = -ct / det;
    minv[2] = -ct / det; minv[3] = cb / det;
}

template <typename T> struct KSArgs {
    GridGeom geo;
    const c2_t<T>* f;      // [Ny][3][nmodes]
    const c2_t<T>* wall;   // [2][3][nmodes]
    const double* ksb;     // [3][Ny][nmodes]
    const double* minv;    // [4][nmodes]
    dc* S;                 // [7][Ny][nmodes]
    int out_sel;           // bit0: u, v, w; bit1: stress
    c2_t<T>* o;            // [Ny][nout][nmodes]
};

template <typename T>
__global__ void __launch_bounds__(64) k_ks(KSArgs<T> a) {
    const GridGeom& geo = a.geo;
    const int nkx = geo.nkx;
    const int nm = geo.Nz * nkx;
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nm) return;
    const int Ny = geo.Ny, N = Ny - 1;
    const size_t sm = nm;
    const int nout = ((a.out_sel & 1) ? 3 : 0) + ((a.out_sel & 2) ? 6 : 0);
    int kzi = m / nkx, kxi = m - kzi * nkx;
    if (kzi == geo.Nz / 2) {
        for (int n = 0; n < Ny; ++n)
            for (int c = 0; c < nout; ++c) {
                c2_t<T> z; z.x = 0; z.y = 0;
                a.o[((size_t)n * nout + c) * sm + m] = z;
            }
        return;
    }
    const double pi = 3.14159265358979323846;
    const double kx = 2.0 * pi * kxi / geo.Lx;
    const int mz = (kzi < geo.Nz / 2) ? kzi : kzi - geo.Nz;
    const double kz = 2.0 * pi * mz / geo.Lz;
    const double W = geo.W, mu = geo.mu, s2 = 0.25 * W * W, dsc = 2.0 / W;
    const double lam = (kx * kx + kz * kz) * s2;
    const double inxz = 1.0 / ((double)geo.Nx * geo.Nz);
    dc* S0 = a.S + 0 * Ny * sm + m;
    dc* S1 = a.S + 1 * Ny * sm + m;
    dc* SP = a.S + 2 * Ny * sm + m;
    dc* SU = a.S + 3 * Ny * sm + m;
    dc* SV = a.S + 4 * Ny * sm + m;
    dc* SW = a.S + 5 * Ny * sm + m;
    dc* SY = a.S + 6 * Ny * sm + m;
    for (int n = 0; n < Ny; ++n) {
        const c2_t<T>* fp = a.f + (size_t)n * 3 * sm + m;
        c2_t<T> fx = fp[0], fy = fp[sm], fz = fp[2 * sm];
        SU[n * sm] = mkc(fx.x, fx.y);
        SV[n * sm] = mkc(fy.x, fy.y);
        SW[n * sm] = mkc(fz.x, fz.y);
    }
    dc gb[3], gt[3];
    for (int c = 0; c < 3; ++c) {
        c2_t<T> b = a.wall[(size_t)c * sm + m], t = a.wall[(size_t)(3 + c) * sm + m];
        gb[c] = mkc(b.x * inxz, b.y * inxz);
        gt[c] = mkc(t.x * inxz, t.y * inxz);
    }
    if (m == 0) {
        // k = 0 mode
        helm_solve(0.0, s2 / mu, SU, gb[0], gt[0], S1, SY, SU, N, sm);
        helm_solve(0.0, s2 / mu, SW, gb[2], gt[2], S1, SY, SW, N, sm);
        // pressure: dp/dybar = G = -(W/2) f_y, zero mean
        dc psum = mkc(0, 0);
        for (int n = 1; n < Ny; ++n) {
            double c = (n == 1) ? 2.0 : 1.0;
            dc gm = -0.5 * W * SV[(size_t)(n - 1) * sm];
            dc gp = (n + 1 < Ny) ? -0.5 * W * SV[(size_t)(n + 1) * sm] : mkc(0, 0);
            dc pn = (1.0 / (2.0 * n)) * (c * gm - gp);
            SP[(size_t)n * sm] = pn;
            if ((n & 1) == 0) psum = psum + (1.0 / (1.0 - (double)n * n)) * pn;
        }
        SP[0] = -1.0 * psum;
        for (int n = 0; n < Ny; ++n) SV[(size_t)n * sm] = mkc(0, 0);
        SV[0] = 0.5 * (gb[1] + gt[1]);
        SV[sm] = 0.5 * (gt[1] - gb[1]);
    } else {
        // p_a
        cheb_deriv(SV, S0, N, sm, dsc);
        for (int n = 0; n < Ny; ++n) {
            size_t o = (size_t)n * sm;
            dc v = times_i(kx, SU[o]) + S0[o] + times_i(kz, SW[o]);
            S0[o] = -1.0 * v;
        }
        helm_solve(lam, s2, S0, mkc(0, 0), mkc(0, 0), S1, SY, SP, N, sm);
        // u_a, v_a, w_a
        cheb_deriv(SP, S0, N, sm, dsc);
        for (int n = 0; n < Ny; ++n) {
            size_t o = (size_t)n * sm;
            SU[o] = SU[o] + times_i(kx, SP[o]);
            SV[o] = SV[o] + S0[o];
            SW[o] = SW[o] + times_i(kz, SP[o]);
        }
        helm_solve(lam, s2 / mu, SU, gb[0], gt[0], S1, SY, SU, N, sm);
        helm_solve(lam, s2 / mu, SV, gb[1], gt[1], S1, SY, SV, N, sm);
        helm_solve(lam, s2 / mu, SW, gb[2], gt[2], S1, SY, SW, N, sm);
        // divergence of the a-solution at the walls
        dc ub = mkc(0, 0), ut = mkc(0, 0), wb = mkc(0, 0), wt = mkc(0, 0);
        dc dvb = mkc(0, 0), dvt = mkc(0, 0);
        for (int n = 0; n < Ny; ++n) {
            size_t o = (size_t)n * sm;
            double sg = (n & 1) ? -1.0 : 1.0, n2 = (double)n * n;
            ub = ub + sg * SU[o]; ut = ut + SU[o];
            wb = wb + sg * SW[o]; wt = wt + SW[o];
            dvb = dvb + (-sg * n2) * SV[o]; dvt = dvt + n2 * SV[o];
        }
        dc Cb = times_i(kx, ub) + dsc * dvb + times_i(kz, wb);
        dc Ct = times_i(kx, ut) + dsc * dvt + times_i(kz, wt);
        const double* mi = a.minv + m;
        dc p1 = -1.0 * (mi[0] * Cb + mi[sm] * Ct);
        dc p2 = -1.0 * (mi[2 * sm] * Cb + mi[3 * sm] * Ct);
        const double* pb = a.ksb + m;
        const double* phib = a.ksb + (size_t)Ny * sm + m;
        const double* vb = a.ksb + (size_t)2 * Ny * sm + m;
        for (int n = 0; n < Ny; ++n) {
            size_t o = (size_t)n * sm;
            double sg = (n & 1) ? -1.0 : 1.0;
            dc pp = p1 + sg * p2, pm = p1 - sg * p2;
            dc phi = phib[o] * pp;
            SU[o] = SU[o] + times_i(kx, phi);
            SW[o] = SW[o] + times_i(kz, phi);
            SV[o] = SV[o] + vb[o] * pm;
            SP[o] = SP[o] + pb[o] * pp;
        }
    }
    int c0 = 0;
    if (a.out_sel & 1) {
        for (int n = 0; n < Ny; ++n) {
            size_t o = (size_t)n * sm;
            c2_t<T>* op = a.o + (size_t)n * nout * sm + m;
            c2_t<T> v;
            v.x = (T)SU[o].x; v.y = (T)SU[o].y; op[0] = v;
            v.x = (T)SV[o].x; v.y = (T)SV[o].y; op[sm] = v;
            v.x = (T)SW[o].x; v.y = (T)SW[o].y; op[2 * sm] = v;
        }
        c0 = 3;
    }
    if (a.out_sel & 2) {
        // sigma = -p I + mu (grad u + grad u^T); d/dy by recurrence
        cheb_deriv(SU, S0, N, sm, dsc);
        cheb_deriv(SV, S1, N, sm, dsc);
        cheb_deriv(SW, SY, N, sm, dsc);
        for (int n = 0; n < Ny; ++n) {
            size_t o = (size_t)n * sm;
            dc U = SU[o], V = SV[o], Wc = SW[o], P = SP[o];
            dc s6[6];
            s6[0] = (-1.0 * P) + (2.0 * mu) * times_i(kx, U);
            s6[1] = mu * (times_i(kx, V) + S0[o]);
            s6[2] = mu * (times_i(kz, U) + times_i(kx, Wc));
            s6[3] = (-1.0 * P) + (2.0 * mu) * S1[o];
            s6[4] = mu * (times_i(kz, V) + SY[o]);
            s6[5] = (-1.0 * P) + (2.0 * mu) * times_i(kz, Wc);
            c2_t<T>* op = a.o + ((size_t)n * nout + c0) * sm + m;
            for (int c = 0; c < 6; ++c) {
                c2_t<T> v;
                v.x = (T)s6[c].x; v.y = (T)s6[c].y;
                op[(size_t)c * sm] = v;
            }
        }
    }
}

template <typename T>
cudaError_t ks_modes(const GridGeom& geo, const T* fcoef, const T* wall, const double* ksb,
                     const double* minv, double* scratch, int out_sel, T* ocoef,
                     cudaStream_t st) {
    int nm = geo.Nz * geo.nkx;
    KSArgs<T> a{geo, (const c2_t<T>*)fcoef, (const c2_t<T>*)wall, ksb, minv, (dc*)scratch,
                out_sel, (c2_t<T>*)ocoef};
    k_ks<T><<<(nm + 63) / 64, 64, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t ks_modes<float>(const GridGeom&, const float*, const float*, const double*,
                                     const double*, double*, int, float*, cudaStream_t);
template cudaError_t ks_modes<double>(const GridGeom&, const double*, const double*,
                                      const double*, const double*, double*, int, double*,
                                      cudaStream_t);

}  // namespace ggem
