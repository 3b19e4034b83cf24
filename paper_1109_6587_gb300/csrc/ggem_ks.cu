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
// GPU mapping: one warp per mode, lane = (real / imaginary part r, parity p,
// chunk j).  The operator is real, so the parts only meet through the i k_x,
// i k_z factors, and the parities only through D; the Ny/2 coefficients of one
// parity are split into 8 contiguous chunks.  Each sequential recurrence of
// the solve (the downward and upward Thomas sweeps, the derivative's suffix
// sum) is a chunk-local sweep, a three-step shuffle scan of the chunks'
// affine maps over the 8 lanes of the (part, parity), and a second local
// sweep from the exact chunk input.  The rows of one mode live in the warp's
// shared memory (11 KB for Ny = 129 in FP32), so a block of 4 modes needs no
// global scratch and several blocks share an SM.  The Thomas factors
// (Y_n, 1/d_n, B_n, Q_n) depend on k^2 only; they come from a plan-time
// table, and so do the products of each chunk's factors that the scans use
// (ks_chunk_mode).
#include <type_traits>

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

// The recurrence indices of chunk j of parity p: coefficients n = p + 2 i,
// ilo <= i < hi; the Ny/2 coefficients of a parity are split into 8 chunks of
// equal length (parity 0, the longer, sets it) and i = 0 (the wall row's
// coefficient a_p) takes no part in the sweeps.
__host__ __device__ inline void ks_chunk_range(int N, int p, int j, int& lo, int& ilo, int& hi) {
    const int ntop = N - ((N - p) & 1);
    const int ch = (N / 2 + 1 + 7) >> 3;
    lo = j * ch;
    hi = (lo + ch < (ntop - p) / 2 + 1) ? lo + ch : (ntop - p) / 2 + 1;
    ilo = lo > 1 ? lo : 1;
}

// Right-hand-side-independent parts of the chunks' affine maps, per parity p
// and chunk j, from the Thomas factors tab [4][Ny] (Y, id, B, Q): the downward
// sweep X_n = B_n X_{n+2} + c_n maps the chunk's input X (just above it) to
// its lowest X by prod B; the upward sweep P_n = Y_n P_{n-2} + X_n maps the
// input P (just below) to its highest P by prod Y and adds
// sum_n prod_{k <= n} Y_k times the input to the chunk's sum of P.
// out[k * 16 + p * 8 + j], k = 0: prod B, 1: prod Y, 2: the sum.
void ks_chunk_mode(int Ny, const double* tab, double* out) {
    const int N = Ny - 1;
    const double* Y = tab;
    const double* B = tab + 2 * Ny;
    for (int p = 0; p < 2; ++p)
        for (int j = 0; j < 8; ++j) {
            int lo, ilo, hi;
            ks_chunk_range(N, p, j, lo, ilo, hi);
            double ab = 1.0, hc = 1.0, sh = 0.0;
            for (int i = ilo; i < hi; ++i) {
                const int n = p + 2 * i;
                ab *= B[n];
                hc *= Y[n];
                sh += hc;
            }
            out[0 * 16 + p * 8 + j] = ab;
            out[1 * 16 + p * 8 + j] = hc;
            out[2 * 16 + p * 8 + j] = sh;
        }
}

// -------------------------------------------------------------- device side
template <typename T> struct KSArgs {
    GridGeom geo;
    const T* f;            // [Ny][3][nmodes] complex T (re, im interleaved)
    const T* wall;         // [2][3][nmodes] complex T
    const T* ksb;          // [3][Ny][nmodes]
    const double* minv;    // [4][nmodes]
    const double* coef;    // [3][Ny]
    const double* thom;    // [4][Ny][nmodes] Y, id, B, Q
    const double* chunk;   // [nmodes][3][2][8] (ks_chunk_mode)
    const double* isq;     // [2][nmodes]
    int out_sel;           // bit0: u, v, w; bit1: stress
    T* o;                  // [Ny][nout][nmodes] complex T
};

enum { AU = 0, AV = 1, AW = 2, AP = 3, AT = 4 };
constexpr int KS_WARPS = 4;     // modes (warps) per block

// Shared memory: the coefficient table [3][Ny] (as T) per block, then per
// warp the series rows SA [5 series][2 parts][ks_row(Ny)] (T) and the
// recurrence rows SX [3 series][2 parts][Ny] (FP64).  The SA row length is
// padded to 16 mod 32 elements so that the two parts fall in different banks.
__host__ __device__ constexpr int ks_row(int Ny) { return Ny + ((16 - Ny % 32) + 32) % 32; }
template <typename T>
__host__ __device__ constexpr size_t ks_coef_bytes(int Ny) {
    return ((size_t)3 * Ny * sizeof(T) + 15) & ~(size_t)15;
}
template <typename T>
__host__ __device__ constexpr size_t ks_warp_bytes(int Ny) {
    return ((((size_t)10 * ks_row(Ny) * sizeof(T)) + 15) & ~(size_t)15) + (size_t)6 * Ny * 8;
}
template <typename T>
__host__ __device__ constexpr size_t ks_smem_bytes(int Ny) {
    return ks_coef_bytes<T>(Ny) + KS_WARPS * ks_warp_bytes<T>(Ny);
}

// Warp (mode m); lane (part r, parity p, chunk j).  FP64 is used where
// App. C's boundary-value solve needs it -- the tau recurrences and the
// influence matrix; right-hand sides, derivatives and combinations run in T.
// Every __syncwarp and shuffle is reached by all 32 lanes: the branches on
// the mode (Nyquist, k = 0) are warp-uniform.
template <typename T>
__global__ void __launch_bounds__(KS_WARPS * 32) k_ks(KSArgs<T> a) {
    const GridGeom& geo = a.geo;
    const int nkx = geo.nkx, nm = geo.Nz * nkx;
    const int Ny = geo.Ny, N = Ny - 1, RS = ks_row(Ny);
    extern __shared__ __align__(16) unsigned char smraw[];
    T* ct = reinterpret_cast<T*>(smraw);
    for (int e = threadIdx.x; e < 3 * Ny; e += blockDim.x) ct[e] = (T)a.coef[e];
    __syncthreads();
    const T* f1 = ct;
    const T* f2 = ct + Ny;
    const T* f3 = ct + 2 * Ny;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = lane & 7, p = (lane >> 3) & 1, r = lane >> 4;
    const int m = blockIdx.x * KS_WARPS + warp;
    if (m >= nm) return;                        // warp-uniform
    const size_t sm = nm;
    unsigned char* wb = smraw + ks_coef_bytes<T>(Ny) + (size_t)warp * ks_warp_bytes<T>(Ny);
    T* sa = reinterpret_cast<T*>(wb);
    double* sx = reinterpret_cast<double*>(wb + ((((size_t)10 * RS * sizeof(T)) + 15) &
                                                 ~(size_t)15));
    auto SA = [&](int A, int R, int n) -> T& { return sa[(A * 2 + R) * RS + n]; };
    auto SX = [&](int S, int R, int n) -> double& { return sx[(S * 2 + R) * Ny + n]; };
    auto TH = [&](int A, int n) -> double { return a.thom[((size_t)A * Ny + n) * sm + m]; };

    // this lane's chunk of the parity-p coefficients: n = p + 2 i, lo <= i < hi
    int lo, ilo, hi;
    ks_chunk_range(N, p, j, lo, ilo, hi);

    const int nout = ((a.out_sel & 1) ? 3 : 0) + ((a.out_sel & 2) ? 6 : 0);
    const int kzi = m / nkx, kxi = m - kzi * nkx;
    if (kzi == geo.Nz / 2) {                    // Nyquist mode in z
        for (int i = lo; i < hi; ++i)
            for (int c = 0; c < nout; ++c)
                a.o[2 * (((size_t)(p + 2 * i) * nout + c) * sm + m) + r] = (T)0;
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
    auto red8 = [](double v) {
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        return v;
    };

    // this chunk's right-hand-side-independent map parts (ks_chunk_mode)
    const double* chk = a.chunk + (size_t)48 * m + p * 8 + j;
    const double Ab = chk[0], Hc = chk[16], SH = chk[32];

    // rho_n of the tau recurrence for the series in A (own part), times rs
    auto rho = [&](int A, int n, T rs) -> T {
        T v = f1[n] * SA(A, r, n - 2) - f2[n] * SA(A, r, n);
        if (n + 2 <= N) v += f3[n] * SA(A, r, n + 2);
        return rs * v;
    };
    // NS real tau solves (series As[s], wall rows sp[s]) in place, FP64
    // recurrences.  Each sweep is a chunk-local pass, a three-step
    // Kogge-Stone scan of the chunks' affine maps over the 8 lanes of the
    // (part, parity), and a second chunk-local pass from the exact input.
    // Entry: SA(As) complete for all lanes (after a __syncwarp).
    auto solve = [&](auto ns_tag, const int* As, T rs, const T* sp) {
        constexpr int NS = decltype(ns_tag)::value;
        double xl[NS], xin[NS], bv[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) xl[s] = 0.0;
        for (int i = hi - 1; i >= ilo; --i) {          // downward, local
            const int n = p + 2 * i;
            const double b = TH(2, n), id = TH(1, n);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const double c = (double)rho(As[s], n, rs) * id;
                xl[s] = fma(b, xl[s], c);
                SX(s, r, n) = c;
            }
        }
        double A = Ab;                                 // suffix scan over chunks
#pragma unroll
        for (int s = 0; s < NS; ++s) bv[s] = xl[s];
#pragma unroll
        for (int d = 1; d < 8; d <<= 1) {
            const double Ao = __shfl_down_sync(0xffffffffu, A, d, 8);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const double bo = __shfl_down_sync(0xffffffffu, bv[s], d, 8);
                if (j + d < 8) bv[s] = fma(A, bo, bv[s]);
            }
            if (j + d < 8) A *= Ao;
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            xin[s] = __shfl_down_sync(0xffffffffu, bv[s], 1, 8);
            if (j == 7) xin[s] = 0.0;
        }
        for (int i = hi - 1; i >= ilo; --i) {          // downward, exact
            const int n = p + 2 * i;
            const double b = TH(2, n);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                xin[s] = fma(b, xin[s], SX(s, r, n));
                SX(s, r, n) = xin[s];
            }
        }
        double pl[NS], spl[NS], pin[NS], t[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) pl[s] = spl[s] = 0.0;
        for (int i = ilo; i < hi; ++i) {               // upward, local
            const int n = p + 2 * i;
            const double y = TH(0, n);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                pl[s] = fma(y, pl[s], SX(s, r, n));
                spl[s] += pl[s];
            }
        }
        A = Hc;                                        // prefix scan over chunks
#pragma unroll
        for (int s = 0; s < NS; ++s) bv[s] = pl[s];
#pragma unroll
        for (int d = 1; d < 8; d <<= 1) {
            const double Ao = __shfl_up_sync(0xffffffffu, A, d, 8);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const double bo = __shfl_up_sync(0xffffffffu, bv[s], d, 8);
                if (j >= d) bv[s] = fma(A, bo, bv[s]);
            }
            if (j >= d) A *= Ao;
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            pin[s] = __shfl_up_sync(0xffffffffu, bv[s], 1, 8);
            if (j == 0) pin[s] = 0.0;
            const double sP = red8(fma(SH, pin[s], spl[s]));
            t[s] = ((double)sp[s] - sP) * isq;
        }
        __syncwarp();                                  // every rho read of SA(As) is done
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if (j == 0) SA(As[s], r, p) = (T)t[s];
        for (int i = ilo; i < hi; ++i) {               // upward, exact; a_n = P_n + Q_n a_p
            const int n = p + 2 * i;
            const double y = TH(0, n), q = TH(3, n);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                pin[s] = fma(y, pin[s], SX(s, r, n));
                SA(As[s], r, n) = (T)fma(q, t[s], pin[s]);
            }
        }
    };
    using one = std::integral_constant<int, 1>;
    using two = std::integral_constant<int, 2>;
    using three = std::integral_constant<int, 3>;
    // derivative (own part, own parity) of a series:
    // b_n = b_{n+2} + 2(n+1) a_{n+1}, b_N = 0; stored as dsc (n == 0 ? b/2 : b)
    auto deriv = [&](auto get, int AD) {
        T s = 0;
        for (int i = lo; i < hi; ++i) {
            const int n = p + 2 * i;
            if (n < N) s += (T)(2 * (n + 1)) * get(n + 1);
        }
        T inc = s;                                     // suffix sum over chunks
#pragma unroll
        for (int d = 1; d < 8; d <<= 1) {
            const T o = __shfl_down_sync(0xffffffffu, inc, d, 8);
            if (j + d < 8) inc += o;
        }
        T b = __shfl_down_sync(0xffffffffu, inc, 1, 8);
        if (j == 7) b = 0;
        for (int i = hi - 1; i >= lo; --i) {
            const int n = p + 2 * i;
            if (n < N) b += (T)(2 * (n + 1)) * get(n + 1);
            SA(AD, r, n) = dsc * ((n == 0) ? (T)0.5 * b : b);
        }
    };

    // ---- stage 1: pressure (k != 0) or the whole k = 0 solve
    if (!k0) {
        deriv([&](int n) { return F(1, r, n); }, AT);
        for (int i = lo; i < hi; ++i) {
            const int n = p + 2 * i;
            T v = (r == 0) ? (kx * F(0, 1, n) - SA(AT, 0, n) + kz * F(2, 1, n))
                           : -(kx * F(0, 0, n) + SA(AT, 1, n) + kz * F(2, 0, n));
            SA(AP, r, n) = v;
        }
        __syncwarp();
        const int As[1] = {AP};
        const T sp[1] = {(T)0};
        solve(one{}, As, s2, sp);
    } else {
        for (int i = lo; i < hi; ++i) {
            const int n = p + 2 * i;
            SA(AU, r, n) = F(0, r, n);
            SA(AW, r, n) = F(2, r, n);
        }
        __syncwarp();
        const int As[2] = {AU, AW};
        const T sp[2] = {wallrow(Wl(0, 0, r), Wl(1, 0, r)), wallrow(Wl(0, 2, r), Wl(1, 2, r))};
        solve(two{}, As, s2 / mu, sp);
        // v linear between its wall values
        T vbw = Wl(0, 1, r), vtw = Wl(1, 1, r);
        for (int i = lo; i < hi; ++i) {
            const int n = p + 2 * i;
            SA(AV, r, n) = (n == 0) ? (T)0.5 * (vbw + vtw) : (n == 1) ? (T)0.5 * (vtw - vbw) : (T)0;
        }
        // pressure: dp/dybar = G = -(W/2) f_y, zero mean over y
        double psum = 0;
        for (int i = lo; i < hi; ++i) {
            const int n = p + 2 * i;
            if (n == 0) continue;
            T c = (n == 1) ? (T)2 : (T)1;
            T gm = -(T)0.5 * W * F(1, r, n - 1);
            T gp = (n + 1 <= N) ? -(T)0.5 * W * F(1, r, n + 1) : (T)0;
            T pn = (c * gm - gp) / (T)(2 * n);
            SA(AP, r, n) = pn;
            if (p == 0) psum += (double)(pn / (T)(1 - n * n));
        }
        psum = red8(psum);
        if (p == 0 && j == 0) SA(AP, r, 0) = (T)(-psum);
    }
    __syncwarp();
    // ---- stage 2: velocity of the a-problem, f + grad p_a (k != 0)
    if (!k0) {
        deriv([&](int n) { return SA(AP, r, n); }, AT);
        for (int i = lo; i < hi; ++i) {
            const int n = p + 2 * i;
            T pr = SA(AP, 1 - r, n);
            T ikp_x = (r == 0) ? -kx * pr : kx * pr;
            T ikp_z = (r == 0) ? -kz * pr : kz * pr;
            SA(AU, r, n) = F(0, r, n) + ikp_x;
            SA(AV, r, n) = F(1, r, n) + SA(AT, r, n);
            SA(AW, r, n) = F(2, r, n) + ikp_z;
        }
        __syncwarp();
        const int As[3] = {AU, AV, AW};
        const T sp[3] = {wallrow(Wl(0, 0, r), Wl(1, 0, r)), wallrow(Wl(0, 1, r), Wl(1, 1, r)),
                         wallrow(Wl(0, 2, r), Wl(1, 2, r))};
        solve(three{}, As, s2 / mu, sp);
    }
    __syncwarp();
    // ---- stage 3: influence matrix from the divergence at both walls (FP64)
    if (!k0) {
        // sums over the chunk: in FP64 plans in FP64; in FP32 plans the terms
        // are FP32 values, summed with compensation (Kahan) in FP32, as
        // accurate as an FP64 sum of the same terms and off the FP64 pipe
        double su, sw, sv;
        if constexpr (sizeof(T) == 8) {
            su = sw = sv = 0;
            for (int i = lo; i < hi; ++i) {
                const int n = p + 2 * i;
                su += SA(AU, r, n);
                sw += SA(AW, r, n);
                sv += (double)(n * n) * SA(AV, r, n);
            }
        } else {
            float s3[3] = {0.f, 0.f, 0.f}, e3[3] = {0.f, 0.f, 0.f};
            auto kadd = [&](int q, float v) {
                const float y = v - e3[q];
                const float t = s3[q] + y;
                e3[q] = (t - s3[q]) - y;
                s3[q] = t;
            };
            for (int i = lo; i < hi; ++i) {
                const int n = p + 2 * i;
                kadd(0, SA(AU, r, n));
                kadd(1, SA(AW, r, n));
                kadd(2, (float)(n * n) * SA(AV, r, n));
            }
            su = (double)s3[0] - (double)e3[0];
            sw = (double)s3[1] - (double)e3[1];
            sv = (double)s3[2] - (double)e3[2];
        }
        su = red8(su);
        sw = red8(sw);
        sv = red8(sv);
        // parity sign (-1)^n is constant per lane: apply once
        const double sg = (double)sgn;
        double ub = sg * su, ut = su, wb = sg * sw, wt = sw, vb = -sg * sv, vt = sv;
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
        dc pp = p1 + sg * p2, pm = p1 - sg * p2;
        const T* pbv = a.ksb + m;
        const T* phv = a.ksb + (size_t)Ny * sm + m;
        const T* vbv = a.ksb + (size_t)2 * Ny * sm + m;
        T ppr = (T)(r == 0 ? pp.x : pp.y), pmr = (T)(r == 0 ? pm.x : pm.y);
        T ppo = (T)(r == 0 ? pp.y : pp.x);       // other part of pp
        T ikf = r == 0 ? (T)-1 : (T)1;           // (i z)_r = ikf * z_other
        for (int i = lo; i < hi; ++i) {
            const int n = p + 2 * i;
            size_t o = (size_t)n * sm;
            const T ph = phv[o];
            SA(AU, r, n) += ikf * kx * ph * ppo;
            SA(AW, r, n) += ikf * kz * ph * ppo;
            SA(AV, r, n) += vbv[o] * pmr;
            SA(AP, r, n) += pbv[o] * ppr;
        }
    }
    __syncwarp();
    // ---- outputs
    T* op = a.o;
    int c0 = 0;
    if (a.out_sel & 1) {
        for (int i = lo; i < hi; ++i) {
            const int n = p + 2 * i;
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
        T ikf = r == 0 ? (T)-1 : (T)1;
        // first pass: components that use du/dy
        for (int i = lo; i < hi; ++i) {
            const int n = p + 2 * i;
            T P = SA(AP, r, n);
            T Uo = SA(AU, 1 - r, n), Vo = SA(AV, 1 - r, n), Wo = SA(AW, 1 - r, n);
            size_t b = ((size_t)n * nout + c0) * sm + m;
            op[2 * b + r] = -P + (T)2 * mu * ikf * kx * Uo;                       // xx
            op[2 * (b + sm) + r] = mu * (ikf * kx * Vo + SA(AT, r, n));             // xy
            op[2 * (b + 2 * sm) + r] = mu * (ikf * kz * Uo + ikf * kx * Wo);        // xz
            op[2 * (b + 5 * sm) + r] = -P + (T)2 * mu * ikf * kz * Wo;              // zz
        }
        deriv([&](int n) { return SA(AV, r, n); }, AT);
        for (int i = lo; i < hi; ++i) {
            const int n = p + 2 * i;
            size_t b = ((size_t)n * nout + c0) * sm + m;
            op[2 * (b + 3 * sm) + r] = -SA(AP, r, n) + (T)2 * mu * SA(AT, r, n);   // yy
        }
        deriv([&](int n) { return SA(AW, r, n); }, AT);
        for (int i = lo; i < hi; ++i) {
            const int n = p + 2 * i;
            T Vo = SA(AV, 1 - r, n);
            size_t b = ((size_t)n * nout + c0) * sm + m;
            op[2 * (b + 4 * sm) + r] = mu * (ikf * kz * Vo + SA(AT, r, n));         // yz
        }
    }
}

template <typename T>
cudaError_t ks_modes(const GridGeom& geo, const T* fcoef, const T* wall, const T* ksb,
                     const double* minv, const double* coef, const double* thom,
                     const double* chunk, const double* isq, int out_sel, T* ocoef,
                     cudaStream_t st) {
    const int nm = geo.Nz * geo.nkx;
    KSArgs<T> a{geo, fcoef, wall, ksb, minv, coef, thom, chunk, isq, out_sel, ocoef};
    // at most 3 x 257 T + 4 x (10 x 272 T + 6 x 257 FP64) = 137 KB (FP64, Ny = 257)
    cudaError_t e = grant_max_smem((const void*)k_ks<T>);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((nm + KS_WARPS - 1) / KS_WARPS);
    k_ks<T><<<blocks, KS_WARPS * 32, ks_smem_bytes<T>(geo.Ny), st>>>(a);
    return cudaGetLastError();
}

template cudaError_t ks_modes<float>(const GridGeom&, const float*, const float*, const float*,
                                     const double*, const double*, const double*,
                                     const double*, const double*, int, float*, cudaStream_t);
template cudaError_t ks_modes<double>(const GridGeom&, const double*, const double*,
                                      const double*, const double*, const double*,
                                      const double*, const double*, const double*, int,
                                      double*, cudaStream_t);

}  // namespace ggem
