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
// same discrete system as the dense tau matrix, rearranged.  Elimination from
// the top gives a_n = X_n + Y_n a_{n-2}, then a_n = P_n + Q_n a_p from the
// bottom, and the wall row fixes a_p.
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
//
// GPU mapping: four threads per mode -- real / imaginary part x even / odd
// coefficient index.  The operator is real, so real and imaginary parts only
// meet through the i k_x, i k_z factors, and the two parities only through D;
// both exchanges go through the mode's scratch columns after __syncwarp.  A
// warp holds 8 consecutive modes, so every scratch access is a coalesced run
// of 8 doubles.  The Thomas factors (Y_n, 1/d_n, Q_n) depend on k^2 only; they
// are computed once per mode and shared by the pressure and velocity solves,
// and the mode-independent recurrence coefficients come from a table.
#include "ggem_internal.cuh"

namespace ggem {

struct dc {
    double x, y;
};
__host__ __device__ __forceinline__ dc mkc(double a, double b) { dc r; r.x = a; r.y = b; return r; }
__host__ __device__ __forceinline__ dc operator+(dc a, dc b) { return mkc(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ dc operator-(dc a, dc b) { return mkc(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ dc operator*(double s, dc a) { return mkc(s * a.x, s * a.y); }

// ---------------------------------------------------------------- host side
// Reference form of the recurrence solve, used at plan time for the
// homogeneous b-solution.  Solves the tau system of (D^2 - lam) a = rs * r in
// ybar units with a(-1) = bot, a(+1) = top.
static void helm_solve_host(double lam, double rs, const std::vector<double>& r, double bot,
                            double top, std::vector<double>& out, int N) {
    std::vector<double> X(N + 1), Y(N + 1);
    for (int p = 0; p < 2; ++p) {
        int ntop = N - ((N - p) & 1);
        double Xn1 = 0.0, Yn1 = 0.0;
        for (int n = ntop; n >= p + 2; n -= 2) {
            double c2 = (n - 2 == 0) ? 2.0 : 1.0;
            double e2 = (n + 2 <= N) ? 1.0 : 0.0;
            double e4 = (n + 4 <= N) ? 1.0 : 0.0;
            double f1 = c2 / (4.0 * n * (n - 1.0));
            double f2 = e2 / (2.0 * ((double)n * n - 1.0));
            double f3 = e4 / (4.0 * n * (n + 1.0));
            double al = -lam * f1, be = 1.0 + lam * f2, ga = -lam * f3;
            double rho = f1 * r[n - 2] - f2 * r[n];
            if (n + 2 <= N) rho += f3 * r[n + 2];
            rho *= rs;
            double d = be + ga * Yn1;
            X[n] = (rho - ga * Xn1) / d;
            Y[n] = -al / d;
            Xn1 = X[n];
            Yn1 = Y[n];
        }
        double s = (p == 0) ? 0.5 * (top + bot) : 0.5 * (top - bot);
        double Pp = 0.0, Qp = 1.0, sP = 0.0, sQ = 1.0;
        std::vector<double> P(N + 1, 0.0), Q(N + 1, 0.0);
        for (int n = p + 2; n <= ntop; n += 2) {
            P[n] = X[n] + Y[n] * Pp;
            Q[n] = Y[n] * Qp;
            sP += P[n];
            sQ += Q[n];
            Pp = P[n];
            Qp = Q[n];
        }
        double t = (s - sP) / sQ;
        out[p] = t;
        for (int n = p + 2; n <= ntop; n += 2) out[n] = P[n] + Q[n] * t;
    }
}

static void cheb_deriv_host(const std::vector<double>& a, std::vector<double>& b, int N,
                            double scale) {
    double b1 = 0.0, b2 = 0.0;
    b[N] = 0.0;
    for (int n = N - 1; n >= 0; --n) {
        double bn = b2 + 2.0 * (n + 1) * a[n + 1];
        if (n == 0) bn *= 0.5;
        b[n] = scale * bn;
        b2 = b1;
        b1 = bn;
    }
}

// Homogeneous b-solution of one mode: p_b with p = 1 at the bottom wall and 0
// at the top; phi_b with mu (D^2-k^2) phi = p_b (u_b = i kx phi_b,
// w_b = i kz phi_b); v_b with mu (D^2-k^2) v = D p_b; zero velocity at the
// walls.  Returns the inverse 2x2 influence matrix; the c-solution is the
// mirror image of b, so the influence matrix is [[a, b],[b, a]].
void ks_precompute_mode(int Ny, double W, double mu, double k2, double* pb, double* phib,
                        double* vb, double* minv) {
    int N = Ny - 1;
    std::vector<double> z(Ny, 0.0), P(Ny), F(Ny), V(Ny), D(Ny);
    double s2 = 0.25 * W * W, lam = k2 * s2;
    helm_solve_host(lam, s2, z, 1.0, 0.0, P, N);
    helm_solve_host(lam, s2 / mu, P, 0.0, 0.0, F, N);
    cheb_deriv_host(P, D, N, 2.0 / W);
    helm_solve_host(lam, s2 / mu, D, 0.0, 0.0, V, N);
    double cb = 0, ct = 0;   // d v_b/dy at the bottom / top wall (phi_b vanishes there)
    for (int n = 0; n < Ny; ++n) {
        double n2 = (double)n * n;
        ct += n2 * V[n];
        cb += ((n & 1) ? 1.0 : -1.0) * n2 * V[n];
        pb[n] = P[n];
        phib[n] = F[n];
        vb[n] = V[n];
    }
    cb *= 2.0 / W;
    ct *= 2.0 / W;
    double det = cb * cb - ct * ct;
    minv[0] = cb / det; minv[1] = -ct / det;
    minv[2] = -ct / det; minv[3] = cb / det;
}

// Mode-independent coefficients of the recurrence, [3][Ny]:
//   f1 = c_{n-2}/(4n(n-1)), f2 = e_{n+2}/(2(n^2-1)), f3 = e_{n+4}/(4n(n+1)).
void ks_coef_table(int Ny, double* tab) {
    int N = Ny - 1;
    for (int n = 0; n < Ny; ++n) {
        double f1 = 0, f2 = 0, f3 = 0;
        if (n >= 2) {
            f1 = ((n - 2 == 0) ? 2.0 : 1.0) / (4.0 * n * (n - 1.0));
            f2 = (n + 2 <= N) ? 1.0 / (2.0 * ((double)n * n - 1.0)) : 0.0;
            f3 = (n + 4 <= N) ? 1.0 / (4.0 * n * (n + 1.0)) : 0.0;
        }
        tab[n] = f1;
        tab[Ny + n] = f2;
        tab[2 * Ny + n] = f3;
    }
}

// Per-mode Thomas factors of (D^2 - lam), computed once at plan time:
// for n of parity p, a_n = X_n + Y_n a_{n-2} with
//   X_n = id_n rs rho_n + B_n X_{n+2},   id_n = 1/d_n,  B_n = lam f3_n id_n,
//   d_n = 1 + lam f2_n - lam f3_n Y_{n+2},  Y_n = lam f1_n id_n,
// then a_n = P_n + Q_n a_p (P_n = X_n + Y_n P_{n-2}, Q_n = Y_n Q_{n-2}) and
// the wall row fixes a_p = (s - sum P)/sum Q.  tab: [4][Ny] (Y, id, B, Q),
// isq[2] = 1/sum Q per parity.
void ks_thomas_mode(int Ny, double lam, double* tab, double* isq) {
    int N = Ny - 1;
    std::vector<double> f(3 * Ny);
    ks_coef_table(Ny, f.data());
    const double* f1 = f.data();
    const double* f2 = f1 + Ny;
    const double* f3 = f2 + Ny;
    double* Y = tab;
    double* ID = tab + Ny;
    double* B = tab + 2 * Ny;
    double* Q = tab + 3 * Ny;
    for (int n = 0; n < Ny; ++n) Y[n] = ID[n] = B[n] = Q[n] = 0.0;
    for (int p = 0; p < 2; ++p) {
        int ntop = N - ((N - p) & 1);
        double Yn1 = 0.0;
        for (int n = ntop; n >= p + 2; n -= 2) {
            double d = 1.0 + lam * f2[n] - lam * f3[n] * Yn1;
            ID[n] = 1.0 / d;
            Y[n] = lam * f1[n] * ID[n];
            B[n] = lam * f3[n] * ID[n];
            Yn1 = Y[n];
        }
        double Qp = 1.0, sQ = 1.0;
        for (int n = p + 2; n <= ntop; n += 2) {
            Qp *= Y[n];
            Q[n] = Qp;
            sQ += Qp;
        }
        isq[p] = 1.0 / sQ;
    }
}

// -------------------------------------------------------------- device side
template <typename T> struct KSArgs {
    GridGeom geo;
    const T* f;            // [Ny][3][nmodes] complex T (re, im interleaved)
    const T* wall;         // [2][3][nmodes] complex T
    const double* ksb;     // [3][Ny][nmodes]
    const double* minv;    // [4][nmodes]
    const double* coef;    // [3][Ny]
    const double* thom;    // [4][Ny][nmodes] Y, id, B, Q
    const double* isq;     // [2][nmodes]
    T* SA;                 // aux scratch [5][2][Ny][nmodes] (T)
    double* SX;            // recurrence scratch [3][2][Ny][nmodes] (FP64)
    int out_sel;           // bit0: u, v, w; bit1: stress
    T* o;                  // [Ny][nout][nmodes] complex T
};

enum { AU = 0, AV = 1, AW = 2, AP = 3, AT = 4 };

// Thread (mode, part r, parity p).  FP64 is used where App. C's boundary-value
// solve needs it -- the tau recurrences and the influence matrix; right-hand
// sides, derivatives and combinations run in T.
// SMEM: the mode scratch (SA, SX) lives in the block's shared memory, one warp
// per block and its 8 modes fastest ([row][8]), so the sequential recurrences
// wait on shared-memory latency instead of L2; otherwise it is the global
// scratch ([row][nmodes]).
template <typename T>
__host__ __device__ constexpr size_t ks_coef_doubles(int Ny) {
    return ((size_t)3 * Ny * sizeof(T) + 7) / 8;
}
template <typename T>
__host__ __device__ constexpr size_t ks_smem_bytes(int Ny) {
    return (ks_coef_doubles<T>(Ny) + (((size_t)5 * 2 * Ny * 8 * sizeof(T) + 7) / 8) +
            (size_t)3 * 2 * Ny * 8) * sizeof(double);
}

template <typename T, bool SMEM>
__global__ void __launch_bounds__(SMEM ? 32 : 128) k_ks(KSArgs<T> a) {
    const GridGeom& geo = a.geo;
    const int nkx = geo.nkx, nm = geo.Nz * nkx;
    const int Ny = geo.Ny, N = Ny - 1;
    extern __shared__ double smc[];            // coef table [3][Ny] as T (+ mode scratch)
    T* ct = reinterpret_cast<T*>(smc);
    for (int e = threadIdx.x; e < 3 * Ny; e += blockDim.x) ct[e] = (T)a.coef[e];
    __syncthreads();
    const T* f1 = ct;
    const T* f2 = ct + Ny;
    const T* f3 = ct + 2 * Ny;

    const int lane = threadIdx.x & 31;
    const int mm = lane & 7, p = (lane >> 3) & 1, r = lane >> 4;
    const int m = (blockIdx.x * blockDim.x + threadIdx.x) / 32 * 8 + mm;
    if (m >= nm) return;                        // warp-uniform (nm is a multiple of 8)
    const size_t sm = nm;
    T* saBase;
    double* sxBase;
    size_t sst;                                 // stride between scratch rows
    if (SMEM) {
        T* sa = reinterpret_cast<T*>(smc + ks_coef_doubles<T>(Ny));
        double* sx = smc + ks_coef_doubles<T>(Ny) + ((size_t)5 * 2 * Ny * 8 * sizeof(T) + 7) / 8;
        saBase = sa + mm;
        sxBase = sx + mm;
        sst = 8;
    } else {
        saBase = a.SA + m;
        sxBase = a.SX + m;
        sst = sm;
    }
    auto SA = [&](int A, int R, int n) -> T& {
        return saBase[((size_t)(A * 2 + R) * Ny + n) * sst];
    };
    auto SX = [&](int A, int R, int n) -> double& {
        return sxBase[((size_t)(A * 2 + R) * Ny + n) * sst];
    };
    auto TH = [&](int A, int n) -> double { return a.thom[((size_t)A * Ny + n) * sm + m]; };
    const int nout = ((a.out_sel & 1) ? 3 : 0) + ((a.out_sel & 2) ? 6 : 0);
    const int kzi = m / nkx, kxi = m - kzi * nkx;
    const int ntop = N - ((N - p) & 1);
    if (kzi == geo.Nz / 2) {                    // Nyquist mode in z (warp-uniform)
        for (int n = p; n <= ntop; n += 2)
            for (int c = 0; c < nout; ++c) a.o[2 * (((size_t)n * nout + c) * sm + m) + r] = (T)0;
        return;
    }
    const bool k0 = (m == 0);
    const T kx = (T)(6.283185307179586477 / geo.Lx) * (T)kxi;
    const int mz = (kzi < geo.Nz / 2) ? kzi : kzi - geo.Nz;
    const T kz = (T)(6.283185307179586477 / geo.Lz) * (T)mz;
    const T W = (T)geo.W, mu = (T)geo.mu, s2 = (T)(0.25 * geo.W * geo.W), dsc = (T)(2.0 / geo.W);
    const T inxz = (T)(1.0 / ((double)geo.Nx * geo.Nz));
    const T sgn = (p & 1) ? (T)-1 : (T)1;
    const double isq = a.isq[(size_t)p * sm + m];
    auto F = [&](int c, int R, int n) -> T { return a.f[2 * (((size_t)n * 3 + c) * sm + m) + R]; };
    auto Wl = [&](int w, int c, int R) -> T {
        return a.wall[2 * ((size_t)(w * 3 + c) * sm + m) + R] * inxz;
    };
    auto wallrow = [&](T bot, T top) -> T {
        return (p == 0) ? (T)0.5 * (top + bot) : (T)0.5 * (top - bot);
    };
    // rho_n of the tau recurrence for the series in A (own part), times rs
    auto rho = [&](int A, int n, T rs) -> T {
        T v = f1[n] * SA(A, r, n - 2) - f2[n] * SA(A, r, n);
        if (n + 2 <= N) v += f3[n] * SA(A, r, n + 2);
        return rs * v;
    };
    // one real tau solve of the series in A in place (FP64 recurrence)
    auto solve1 = [&](int A, int X, T rs, T sp) {
        double Xn1 = 0.0;
        for (int n = ntop; n >= p + 2; n -= 2) {
            double xn = fma(TH(2, n), Xn1, (double)rho(A, n, rs) * TH(1, n));
            SX(X, r, n) = xn;
            Xn1 = xn;
        }
        double Pp = 0.0, sP = 0.0;
        for (int n = p + 2; n <= ntop; n += 2) {
            Pp = fma(TH(0, n), Pp, SX(X, r, n));
            SX(X, r, n) = Pp;
            sP += Pp;
        }
        double t = ((double)sp - sP) * isq;
        SA(A, r, p) = (T)t;
        for (int n = p + 2; n <= ntop; n += 2) SA(A, r, n) = (T)fma(TH(3, n), t, SX(X, r, n));
    };
    auto solve3 = [&](T rs, T sp0, T sp1, T sp2) {
        double X0 = 0, X1 = 0, X2 = 0;
        for (int n = ntop; n >= p + 2; n -= 2) {
            double b = TH(2, n), id = TH(1, n);
            X0 = fma(b, X0, (double)rho(AU, n, rs) * id);
            X1 = fma(b, X1, (double)rho(AV, n, rs) * id);
            X2 = fma(b, X2, (double)rho(AW, n, rs) * id);
            SX(0, r, n) = X0;
            SX(1, r, n) = X1;
            SX(2, r, n) = X2;
        }
        double P0 = 0, P1 = 0, P2 = 0, q0 = 0, q1 = 0, q2 = 0;
        for (int n = p + 2; n <= ntop; n += 2) {
            double y = TH(0, n);
            P0 = fma(y, P0, SX(0, r, n));
            P1 = fma(y, P1, SX(1, r, n));
            P2 = fma(y, P2, SX(2, r, n));
            SX(0, r, n) = P0;
            SX(1, r, n) = P1;
            SX(2, r, n) = P2;
            q0 += P0; q1 += P1; q2 += P2;
        }
        double t0 = ((double)sp0 - q0) * isq, t1 = ((double)sp1 - q1) * isq;
        double t2 = ((double)sp2 - q2) * isq;
        SA(AU, r, p) = (T)t0;
        SA(AV, r, p) = (T)t1;
        SA(AW, r, p) = (T)t2;
        for (int n = p + 2; n <= ntop; n += 2) {
            double q = TH(3, n);
            SA(AU, r, n) = (T)fma(q, t0, SX(0, r, n));
            SA(AV, r, n) = (T)fma(q, t1, SX(1, r, n));
            SA(AW, r, n) = (T)fma(q, t2, SX(2, r, n));
        }
    };
    // derivative (own part, own parity) of a series: b_n = b_{n+2} + 2(n+1) a_{n+1}
    auto deriv = [&](auto get, int AD) {
        T b2 = 0;
        int nstart = ntop;
        if (nstart == N) {
            SA(AD, r, N) = 0;
            nstart -= 2;
        }
        for (int n = nstart; n >= p; n -= 2) {
            T bn = b2 + (T)(2 * (n + 1)) * get(n + 1);
            b2 = bn;
            SA(AD, r, n) = dsc * ((n == 0) ? (T)0.5 * bn : bn);
        }
    };

    // Every __syncwarp and shuffle below is reached by all 32 lanes; the
    // k = 0 mode (lanes of warp 0 with mm = 0) only changes per-lane work.
    // ---- stage 1: pressure (k != 0) or the whole k = 0 solve
    if (!k0) {
        deriv([&](int n) { return F(1, r, n); }, AT);
        for (int n = p; n <= ntop; n += 2) {
            T v = (r == 0) ? (kx * F(0, 1, n) - SA(AT, 0, n) + kz * F(2, 1, n))
                           : -(kx * F(0, 0, n) + SA(AT, 1, n) + kz * F(2, 0, n));
            SA(AP, r, n) = v;
        }
        solve1(AP, 0, s2, (T)0);
    } else {
        for (int n = p; n <= ntop; n += 2) {
            SA(AU, r, n) = F(0, r, n);
            SA(AW, r, n) = F(2, r, n);
        }
        solve1(AU, 0, s2 / mu, wallrow(Wl(0, 0, r), Wl(1, 0, r)));
        solve1(AW, 1, s2 / mu, wallrow(Wl(0, 2, r), Wl(1, 2, r)));
        // v linear between its wall values
        T vbw = Wl(0, 1, r), vtw = Wl(1, 1, r);
        for (int n = p; n <= ntop; n += 2)
            SA(AV, r, n) = (n == 0) ? (T)0.5 * (vbw + vtw) : (n == 1) ? (T)0.5 * (vtw - vbw) : (T)0;
        // pressure: dp/dybar = G = -(W/2) f_y, zero mean over y
        T psum = 0;
        for (int n = (p == 0 ? 2 : 1); n <= ntop; n += 2) {
            T c = (n == 1) ? (T)2 : (T)1;
            T gm = -(T)0.5 * W * F(1, r, n - 1);
            T gp = (n + 1 <= N) ? -(T)0.5 * W * F(1, r, n + 1) : (T)0;
            T pn = (c * gm - gp) / (T)(2 * n);
            SA(AP, r, n) = pn;
            if (p == 0) psum += pn / (T)(1 - n * n);
        }
        if (p == 0) SA(AP, r, 0) = -psum;
    }
    __syncwarp();
    // ---- stage 2: velocity of the a-problem, f + grad p_a (k != 0)
    if (!k0) {
        deriv([&](int n) { return SA(AP, r, n); }, AT);
        for (int n = p; n <= ntop; n += 2) {
            T pr = SA(AP, 1 - r, n);
            T ikp_x = (r == 0) ? -kx * pr : kx * pr;
            T ikp_z = (r == 0) ? -kz * pr : kz * pr;
            SA(AU, r, n) = F(0, r, n) + ikp_x;
            SA(AV, r, n) = F(1, r, n) + SA(AT, r, n);
            SA(AW, r, n) = F(2, r, n) + ikp_z;
        }
        solve3(s2 / mu, wallrow(Wl(0, 0, r), Wl(1, 0, r)), wallrow(Wl(0, 1, r), Wl(1, 1, r)),
               wallrow(Wl(0, 2, r), Wl(1, 2, r)));
    }
    __syncwarp();
    // ---- stage 3: influence matrix from the divergence at both walls (FP64)
    double ub = 0, ut = 0, wb = 0, wt = 0, vb = 0, vt = 0;
    if (!k0) {
        for (int n = p; n <= ntop; n += 2) {
            double n2 = (double)(n * n);
            double u = (double)SA(AU, r, n), w = (double)SA(AW, r, n), v = (double)SA(AV, r, n);
            ub += u; ut += u;
            wb += w; wt += w;
            vb += n2 * v; vt += n2 * v;
        }
        // parity sign (-1)^n is constant per thread: apply once
        double sg = (double)sgn;
        ub *= sg; wb *= sg; vb *= -sg;
    }
    ub += __shfl_xor_sync(0xffffffffu, ub, 8);
    ut += __shfl_xor_sync(0xffffffffu, ut, 8);
    wb += __shfl_xor_sync(0xffffffffu, wb, 8);
    wt += __shfl_xor_sync(0xffffffffu, wt, 8);
    vb += __shfl_xor_sync(0xffffffffu, vb, 8);
    vt += __shfl_xor_sync(0xffffffffu, vt, 8);
    double ubo = __shfl_xor_sync(0xffffffffu, ub, 16);
    double uto = __shfl_xor_sync(0xffffffffu, ut, 16);
    double wbo = __shfl_xor_sync(0xffffffffu, wb, 16);
    double wto = __shfl_xor_sync(0xffffffffu, wt, 16);
    double vbo = __shfl_xor_sync(0xffffffffu, vb, 16);
    double vto = __shfl_xor_sync(0xffffffffu, vt, 16);
    if (!k0) {
        dc Ub = r == 0 ? mkc(ub, ubo) : mkc(ubo, ub);
        dc Ut = r == 0 ? mkc(ut, uto) : mkc(uto, ut);
        dc Wb = r == 0 ? mkc(wb, wbo) : mkc(wbo, wb);
        dc Wt = r == 0 ? mkc(wt, wto) : mkc(wto, wt);
        dc Vb = r == 0 ? mkc(vb, vbo) : mkc(vbo, vb);
        dc Vt = r == 0 ? mkc(vt, vto) : mkc(vto, vt);
        double kxd = (double)kx, kzd = (double)kz, dscd = 2.0 / geo.W;
        // C = i kx u + dsc dv + i kz w
        dc Cb = mkc(-kxd * Ub.y + dscd * Vb.x - kzd * Wb.y, kxd * Ub.x + dscd * Vb.y + kzd * Wb.x);
        dc Ct = mkc(-kxd * Ut.y + dscd * Vt.x - kzd * Wt.y, kxd * Ut.x + dscd * Vt.y + kzd * Wt.x);
        const double* mi = a.minv + m;
        dc p1 = -1.0 * (mi[0] * Cb + mi[sm] * Ct);
        dc p2 = -1.0 * (mi[2 * sm] * Cb + mi[3 * sm] * Ct);
        double sg = (double)sgn;
        dc pp = p1 + sg * p2, pm = p1 - sg * p2;
        const double* pbv = a.ksb + m;
        const double* phv = a.ksb + (size_t)Ny * sm + m;
        const double* vbv = a.ksb + (size_t)2 * Ny * sm + m;
        T ppr = (T)(r == 0 ? pp.x : pp.y), pmr = (T)(r == 0 ? pm.x : pm.y);
        T ppo = (T)(r == 0 ? pp.y : pp.x);       // other part of pp
        T ikf = r == 0 ? (T)-1 : (T)1;           // (i z)_r = ikf * z_other
        for (int n = p; n <= ntop; n += 2) {
            size_t o = (size_t)n * sm;
            T ph = (T)phv[o];
            SA(AU, r, n) += ikf * kx * ph * ppo;
            SA(AW, r, n) += ikf * kz * ph * ppo;
            SA(AV, r, n) += (T)vbv[o] * pmr;
            SA(AP, r, n) += (T)pbv[o] * ppr;
        }
    }
    __syncwarp();
    // ---- outputs
    T* op = a.o;
    int c0 = 0;
    if (a.out_sel & 1) {
        for (int n = p; n <= ntop; n += 2) {
            size_t b = ((size_t)n * nout) * sm + m;
            op[2 * b + r] = SA(AU, r, n);
            op[2 * (b + sm) + r] = SA(AV, r, n);
            op[2 * (b + 2 * sm) + r] = SA(AW, r, n);
        }
        c0 = 3;
    }
    if (a.out_sel & 2) {
        // d/dy of u, v, w, one at a time, into the aux row AT
        deriv([&](int n) { return SA(AU, r, n); }, AT);
        __syncwarp();
        T ikf = r == 0 ? (T)-1 : (T)1;
        // first pass: components that use du/dy
        for (int n = p; n <= ntop; n += 2) {
            T P = SA(AP, r, n);
            T Uo = SA(AU, 1 - r, n), Vo = SA(AV, 1 - r, n), Wo = SA(AW, 1 - r, n);
            size_t b = ((size_t)n * nout + c0) * sm + m;
            op[2 * b + r] = -P + (T)2 * mu * ikf * kx * Uo;                       // xx
            op[2 * (b + sm) + r] = mu * (ikf * kx * Vo + SA(AT, r, n));             // xy
            op[2 * (b + 2 * sm) + r] = mu * (ikf * kz * Uo + ikf * kx * Wo);        // xz
            op[2 * (b + 5 * sm) + r] = -P + (T)2 * mu * ikf * kz * Wo;              // zz
        }
        __syncwarp();
        deriv([&](int n) { return SA(AV, r, n); }, AT);
        for (int n = p; n <= ntop; n += 2) {
            size_t b = ((size_t)n * nout + c0) * sm + m;
            op[2 * (b + 3 * sm) + r] = -SA(AP, r, n) + (T)2 * mu * SA(AT, r, n);   // yy
        }
        __syncwarp();
        deriv([&](int n) { return SA(AW, r, n); }, AT);
        for (int n = p; n <= ntop; n += 2) {
            T Vo = SA(AV, 1 - r, n);
            size_t b = ((size_t)n * nout + c0) * sm + m;
            op[2 * (b + 4 * sm) + r] = mu * (ikf * kz * Vo + SA(AT, r, n));         // yz
        }
    }
}

template <typename T>
cudaError_t ks_modes(const GridGeom& geo, const T* fcoef, const T* wall, const double* ksb,
                     const double* minv, const double* coef, const double* thom,
                     const double* isq, void* scratch, int out_sel, T* ocoef, cudaStream_t st) {
    int nm = geo.Nz * geo.nkx;
    size_t naux = (size_t)5 * 2 * geo.Ny * nm;
    T* SA = (T*)scratch;
    double* SX = (double*)((char*)scratch + ((naux * sizeof(T) + 255) & ~(size_t)255));
    KSArgs<T> a{geo, fcoef, wall, ksb, minv, coef, thom, isq, SA, SX, out_sel, ocoef};
    long warps = (long)(nm + 7) / 8;
    // mode scratch in shared memory when a warp's share fits the opt-in limit
    // (the kernel has no static shared memory)
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        grant_max_smem((const void*)k_ks<T, true>) != cudaSuccess)
        optin = 0;
    const size_t bytes = ks_smem_bytes<T>(geo.Ny);
    if (bytes <= (size_t)optin) {
        k_ks<T, true><<<(unsigned)warps, 32, bytes, st>>>(a);
        return cudaGetLastError();
    }
    size_t smem = (size_t)3 * geo.Ny * sizeof(double);
    k_ks<T, false><<<(unsigned)((warps * 32 + 127) / 128), 128, smem, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t ks_modes<float>(const GridGeom&, const float*, const float*, const double*,
                                     const double*, const double*, const double*,
                                     const double*, void*, int, float*, cudaStream_t);
template cudaError_t ks_modes<double>(const GridGeom&, const double*, const double*,
                                      const double*, const double*, const double*,
                                      const double*, const double*, void*, int, double*,
                                      cudaStream_t);

}  // namespace ggem
