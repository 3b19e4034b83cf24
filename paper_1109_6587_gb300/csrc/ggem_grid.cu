// Grid-side kernels of the GGEM global problem (paper Sec. 3.2.2, 3.2.3, 3.4.2,
// App. C): FFTs in x (real) and z (complex), the Chebyshev transforms in y as a
// dense contraction, 5x5x5 Lagrange interpolation back to the targets, and the
// spectral off-grid evaluation (deconvolution onto an oversampled grid and a
// Gaussian-window gather: a type-2 non-uniform FFT).
//
// Grid layout: physical [Ny][comp][Nz][Nx] (real T); after the x transform
// each row of Nx reals holds Nx/2 complex modes k_x = 0..Nx/2-1 in place (the
// Nyquist mode is dropped, i.e. set to zero); spectral [Ny][comp][Nz][Nx/2].
#include <algorithm>

#include "ggem_internal.cuh"

namespace ggem {

// ------------------------------------------------------------------ FFT
template <typename T> struct Cx {
    using C = c2_t<T>;
    static __device__ __forceinline__ C mk(T a, T b) { C c; c.x = a; c.y = b; return c; }
    static __device__ __forceinline__ C add(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ C sub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
    static __device__ __forceinline__ C mul(C a, C b) {
        return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
    }
    static __device__ __forceinline__ C conj(C a) { return mk(a.x, -a.y); }
};

// In-place DIT butterflies on R transforms of length M stored contiguously
// in shared memory, input already in bit-reversed order.
// tw[k] = exp(-2 pi i k / M), k < M/2; inv selects the conjugate twiddles.
// Two radix-2 stages (spans h and 2h) are fused into one radix-4 pass over
// the quadruples i0, i0 + h, i0 + 2h, i0 + 3h: the first stage pairs them with
// the twiddle W_2h^pos, the second with W_4h^pos and W_4h^(pos+h) =
// W_4h^pos * (-i) (+i inverse); an odd number of stages starts with one
// radix-2 pass.  Half the passes over shared memory and half the barriers of
// the radix-2 form, same operations per element.
template <typename T>
__device__ void smem_fft(c2_t<T>* s, int R, int M, int logM, const c2_t<T>* __restrict__ tw,
                         bool inv) {
    using X = Cx<T>;
    int lh = 0;
    if (logM & 1) {                         // one radix-2 pass (h = 1, twiddle 1)
        __syncthreads();
        for (int b = threadIdx.x; b < R * (M >> 1); b += blockDim.x) {
            const int i0 = 2 * b;
            const c2_t<T> a = s[i0], bb = s[i0 + 1];
            s[i0] = X::add(a, bb);
            s[i0 + 1] = X::sub(a, bb);
        }
        lh = 1;
    }
    for (; lh < logM; lh += 2) {
        const int h = 1 << lh;
        const int q = M >> 2;               // quadruples per transform
        __syncthreads();
        for (int b = threadIdx.x; b < R * q; b += blockDim.x) {
            const int r = b / q, jj = b - r * q;
            const int pos = jj & (h - 1), grp = jj >> lh;
            const int i0 = r * M + (grp << (lh + 2)) + pos;
            c2_t<T> w1 = tw[pos << (logM - 1 - lh)];      // W_2h^pos
            c2_t<T> w2 = tw[pos << (logM - 2 - lh)];      // W_4h^pos
            if (inv) { w1.y = -w1.y; w2.y = -w2.y; }
            // W_4h^(pos+h) = W_4h^pos * (-i) forward, * (+i) inverse
            const c2_t<T> w3 = inv ? X::mk(-w2.y, w2.x) : X::mk(w2.y, -w2.x);
            const c2_t<T> a = s[i0], bb = X::mul(s[i0 + h], w1);
            const c2_t<T> c = s[i0 + 2 * h], d = X::mul(s[i0 + 3 * h], w1);
            const c2_t<T> t0 = X::add(a, bb), t1 = X::sub(a, bb);
            const c2_t<T> t2 = X::add(c, d), t3 = X::sub(c, d);
            const c2_t<T> u2 = X::mul(t2, w2), u3 = X::mul(t3, w3);
            s[i0] = X::add(t0, u2);
            s[i0 + 2 * h] = X::sub(t0, u2);
            s[i0 + h] = X::add(t1, u3);
            s[i0 + 3 * h] = X::sub(t1, u3);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int bitrev(int v, int logM) {
    return (int)(__brev((unsigned)v) >> (32 - logM));
}

// Real-to-complex along x for R rows per block: the row of Nx reals is read as
// M = Nx/2 complex values z_n = x_2n + i x_2n+1, transformed with length M, then
// X_k = E_k + exp(-2 pi i k/Nx) O_k with E, O the even/odd-sample spectra.
// Output X_k, k = 0..M-1, in place.
template <typename T>
__global__ void k_fft_x_r2c(c2_t<T>* data, long nrows, int M, int logM,
                            const c2_t<T>* __restrict__ tw, const c2_t<T>* __restrict__ tpost,
                            int R) {
    using X = Cx<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    c2_t<T>* s = reinterpret_cast<c2_t<T>*>(smraw);
    long row0 = (long)blockIdx.x * R;
    int rr = (int)min((long)R, nrows - row0);
    for (int e = threadIdx.x; e < rr * M; e += blockDim.x) {
        int r = e / M, n = e - r * M;
        s[r * M + bitrev(n, logM)] = data[(row0 + r) * M + n];
    }
    for (int e = threadIdx.x; e < (R - rr) * M; e += blockDim.x) s[rr * M + e] = X::mk(0, 0);
    smem_fft<T>(s, R, M, logM, tw, false);
    for (int e = threadIdx.x; e < rr * M; e += blockDim.x) {
        int r = e / M, k = e - r * M;
        c2_t<T> Zk = s[r * M + k];
        c2_t<T> Zc = X::conj(s[r * M + ((M - k) & (M - 1))]);
        c2_t<T> E = X::mk((T)0.5 * (Zk.x + Zc.x), (T)0.5 * (Zk.y + Zc.y));
        // O = (Zk - Zc) / (2i)
        c2_t<T> O = X::mk((T)0.5 * (Zk.y - Zc.y), -(T)0.5 * (Zk.x - Zc.x));
        data[(row0 + r) * M + k] = X::add(E, X::mul(tpost[k], O));
    }
}

// Complex-to-real along x, the inverse of the above with the Hermitian
// extension X_{Nx-k} = conj(X_k), the Nyquist mode zero and Im X_0 ignored:
// x_n = Re X_0 + 2 sum_{k=1}^{Nx/2-1} Re(X_k exp(2 pi i k n/Nx)).
template <typename T>
__global__ void k_fft_x_c2r(c2_t<T>* data, long nrows, int M, int logM,
                            const c2_t<T>* __restrict__ tw, const c2_t<T>* __restrict__ tpost,
                            int R) {
    using X = Cx<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    c2_t<T>* s = reinterpret_cast<c2_t<T>*>(smraw);
    long row0 = (long)blockIdx.x * R;
    int rr = (int)min((long)R, nrows - row0);
    for (int e = threadIdx.x; e < rr * M; e += blockDim.x) {
        int r = e / M, k = e - r * M;
        const c2_t<T>* row = data + (row0 + r) * M;
        c2_t<T> Z;
        if (k == 0) {
            T x0 = row[0].x;
            Z = X::mk(x0, x0);            // E' = O' = Re X_0 (Nyquist is zero)
        } else {
            c2_t<T> Xk = row[k];
            c2_t<T> Xc = X::conj(row[M - k]);
            c2_t<T> Ep = X::add(Xk, Xc);
            c2_t<T> Op = X::mul(X::sub(Xk, Xc), X::conj(tpost[k]));
            Z = X::mk(Ep.x - Op.y, Ep.y + Op.x);   // E' + i O'
        }
        s[r * M + bitrev(k, logM)] = Z;
    }
    for (int e = threadIdx.x; e < (R - rr) * M; e += blockDim.x) s[rr * M + e] = X::mk(0, 0);
    smem_fft<T>(s, R, M, logM, tw, true);
    for (int e = threadIdx.x; e < rr * M; e += blockDim.x) {
        int r = e / M, n = e - r * M;
        data[(row0 + r) * M + n] = s[r * M + n];
    }
}

// Complex transform along z: planes of [Nz][nkx] complex, TB columns per block;
// only the first ncols columns of each plane (the others hold zeros and stay
// zero).
template <typename T>
__global__ void k_fft_z(c2_t<T>* data, int nkx, int ncols, int Nz, int logNz,
                        const c2_t<T>* __restrict__ tw, int TB, bool inv) {
    extern __shared__ __align__(16) unsigned char smraw[];
    c2_t<T>* s = reinterpret_cast<c2_t<T>*>(smraw);
    int ncb = (ncols + TB - 1) / TB;
    long plane = blockIdx.x / ncb;
    int col0 = (blockIdx.x - plane * ncb) * TB;
    int tb = min(TB, ncols - col0);
    c2_t<T>* base = data + plane * (long)Nz * nkx + col0;
    for (int e = threadIdx.x; e < Nz * TB; e += blockDim.x) {
        int z = e / TB, c = e - z * TB;
        c2_t<T> v = Cx<T>::mk(0, 0);
        if (c < tb) v = base[(long)z * nkx + c];
        s[c * Nz + bitrev(z, logNz)] = v;
    }
    smem_fft<T>(s, TB, Nz, logNz, tw, inv);
    for (int e = threadIdx.x; e < Nz * TB; e += blockDim.x) {
        int z = e / TB, c = e - z * TB;
        if (c < tb) base[(long)z * nkx + c] = s[c * Nz + z];
    }
}

static int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

template <typename T>
static cudaError_t fft_x(const GridGeom& geo, T* data, int nplanes, const void* tw_x, bool inv,
                         cudaStream_t st) {
    int M = geo.Nx / 2, logM = ilog2(M);
    long nrows = (long)nplanes * geo.Nz;
    int R = max(1, 2048 / M);
    size_t smem = (size_t)R * M * sizeof(c2_t<T>);
    const c2_t<T>* tw = (const c2_t<T>*)tw_x;
    const c2_t<T>* tpost = tw + M / 2;
    unsigned nb = (unsigned)((nrows + R - 1) / R);
    if (inv) {
        grant_max_smem((const void*)k_fft_x_c2r<T>);
        k_fft_x_c2r<T><<<nb, 256, smem, st>>>((c2_t<T>*)data, nrows, M, logM, tw, tpost, R);
    } else {
        grant_max_smem((const void*)k_fft_x_r2c<T>);
        k_fft_x_r2c<T><<<nb, 256, smem, st>>>((c2_t<T>*)data, nrows, M, logM, tw, tpost, R);
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t fft_z(const GridGeom& geo, T* data, int nplanes, const void* tw_z, bool inv,
                         cudaStream_t st, int ncols = 0) {
    int Nz = geo.Nz, logNz = ilog2(Nz), nkx = geo.Nx / 2;
    if (ncols <= 0 || ncols > nkx) ncols = nkx;
    int TB = min(ncols, 8);
    // (the oversampled grids of the spectral evaluation reach Nz = 2048)
    while (TB > 1 && (size_t)TB * Nz * sizeof(c2_t<T>) > (size_t)160 * 1024) TB >>= 1;
    size_t smem = (size_t)TB * Nz * sizeof(c2_t<T>);
    unsigned nb = (unsigned)((long)nplanes * ((ncols + TB - 1) / TB));
    grant_max_smem((const void*)k_fft_z<T>);
    k_fft_z<T><<<nb, 256, smem, st>>>((c2_t<T>*)data, nkx, ncols, Nz, logNz,
                                      (const c2_t<T>*)tw_z, TB, inv);
    return cudaGetLastError();
}

template <typename T>
cudaError_t fft_forward(const GridGeom& geo, T* data, int nplanes, const void* tw_x,
                        const void* tw_z, cudaStream_t st) {
    cudaError_t e = fft_x<T>(geo, data, nplanes, tw_x, false, st);
    if (e != cudaSuccess) return e;
    return fft_z<T>(geo, data, nplanes, tw_z, false, st);
}

template <typename T>
cudaError_t fft_inverse(const GridGeom& geo, T* data, int nplanes, const void* tw_x,
                        const void* tw_z, cudaStream_t st, int active_kx) {
    cudaError_t e = fft_z<T>(geo, data, nplanes, tw_z, true, st, active_kx);
    if (e != cudaSuccess) return e;
    return fft_x<T>(geo, data, nplanes, tw_x, true, st);
}

// -------------------------------------------------- Chebyshev contraction
// out[n][col] = sum_j M[n][j] in[j][col]  (M: Ny x Ny in shared memory)
template <typename T, int NB>
__global__ void __launch_bounds__(256) k_cheb(int Ny, const T* __restrict__ M,
                                               const T* __restrict__ in, T* __restrict__ out,
                                               long cols) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Ms = reinterpret_cast<T*>(smraw);
    for (int e = threadIdx.x; e < Ny * Ny; e += blockDim.x) Ms[e] = M[e];
    __syncthreads();
    long col = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= cols) return;
    for (int n0 = 0; n0 < Ny; n0 += NB) {
        T acc[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[b] = 0;
        for (int j = 0; j < Ny; ++j) {
            T v = in[(long)j * cols + col];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                int n = n0 + b;
                if (n < Ny) acc[b] += Ms[n * Ny + j] * v;
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (n0 + b < Ny) out[(long)(n0 + b) * cols + col] = acc[b];
    }
}

cudaError_t cheb_apply_tc(int Ny, const void* prep, const float* in, float* out, long cols,
                          int* err, int nsm, cudaStream_t st);

template <typename T>
cudaError_t cheb_apply(int Ny, const T* M, const T* in, T* out, long cols, cudaStream_t st,
                       int* tc_err, int nsm, const void* tc_prep) {
    if (sizeof(T) == 4 && tc_err && tc_prep) {
        // FP32 data: split-BF16 contraction on the tensor cores when it fits
        cudaError_t e = cheb_apply_tc(Ny, tc_prep, (const float*)in, (float*)out, cols, tc_err,
                                      nsm, st);
        if (e != cudaErrorNotSupported) return e;
    }
    size_t smem = (size_t)Ny * Ny * sizeof(T);
    grant_max_smem((const void*)k_cheb<T, 24>);
    k_cheb<T, 24><<<(unsigned)((cols + 255) / 256), 256, smem, st>>>(Ny, M, in, out, cols);
    return cudaGetLastError();
}

// ------------------------------------------------------- interpolation
// Degree-4 Lagrange weights at offset t for nodes -2..2.
template <typename T> __device__ __forceinline__ void lag5_uniform(T t, T w[5]) {
#pragma unroll
    for (int p = 0; p < 5; ++p) {
        T v = 1;
#pragma unroll
        for (int q = 0; q < 5; ++q)
            if (q != p) v *= (t - (T)(q - 2)) / (T)(p - q);
        w[p] = v;
    }
}

template <typename T> struct InterpArgs {
    GridGeom geo;
    const double* yj;
    const T* grid;
    int ncomp_total, comp0, mode;
    int n;
    const double* x;
    const T* local;
    int local_stride;
    const double* nrm;
    const double* qself;
    const double* wself;
    double self_coef;
    double* out;
    int out_stride;
};

template <typename T>
__device__ __forceinline__ void interp_store(const InterpArgs<T>& a, int t, const T* acc);

template <typename T> __device__ __forceinline__ T wexp(T x);
template <> __device__ __forceinline__ float wexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double wexp<double>(double x) { return exp(x); }

// mode 0: velocity (3 comps): out = local + interp - self
// mode 1: stress (6 comps):   out = local + interp
// mode 2: double layer:       out_j = local_j + n_k sigma_jk / mu
template <typename T>
__global__ void __launch_bounds__(128) k_interp(InterpArgs<T> a) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    const GridGeom& geo = a.geo;
    double xt = a.x[3 * t], yt = a.x[3 * t + 1], zt = a.x[3 * t + 2];
    // grid coordinates in FP64 (positions up to the box size), by multiplies:
    // GB300 runs FP64 at 1/64 of FP32 and an FP64 divide is a long sequence
    double ux = xt * (1.0 / geo.dx), uz = zt * (1.0 / geo.dz);
    double i0 = rint(ux), k0 = rint(uz);
    T wx[5], wz[5], wy[5];
    lag5_uniform<T>((T)(ux - i0), wx);
    lag5_uniform<T>((T)(uz - k0), wz);
    int N = geo.Ny - 1;
    double yb = fmin(1.0, fmax(-1.0, (yt - geo.y0) * (2.0 / geo.W) - 1.0));
    // first guess of the nearest Chebyshev node from theta = acos(yb) in FP32
    // (the search below compares the FP64 distances to its neighbours)
    int jc = (int)rintf(acosf((float)yb) * ((float)N * 0.318309886f));
    jc = min(max(jc, 0), N);
    int jbest = jc;
    double dbest = fabs(yt - a.yj[jc]);
    if (jc > 0) {
        double d = fabs(yt - a.yj[jc - 1]);
        if (d <= dbest) { dbest = d; jbest = jc - 1; }
    }
    if (jc < N) {
        double d = fabs(yt - a.yj[jc + 1]);
        if (d < dbest) { dbest = d; jbest = jc + 1; }
    }
    int js = min(max(jbest - 2, 0), geo.Ny - 5);
    double yn[5];
#pragma unroll
    for (int p = 0; p < 5; ++p) yn[p] = a.yj[js + p];
    // Lagrange weights in y: the five FP64 differences to the target and the
    // ten between the nodes, each rounded once to T
    T dt[5], dn[5][5];
#pragma unroll
    for (int q = 0; q < 5; ++q) dt[q] = (T)(yt - yn[q]);
#pragma unroll
    for (int p = 0; p < 5; ++p)
#pragma unroll
        for (int q = p + 1; q < 5; ++q) {
            dn[p][q] = (T)(yn[p] - yn[q]);
            dn[q][p] = -dn[p][q];
        }
#pragma unroll
    for (int p = 0; p < 5; ++p) {
        T v = 1;
#pragma unroll
        for (int q = 0; q < 5; ++q)
            if (q != p) v *= dt[q] / dn[p][q];
        wy[p] = v;
    }
    int ib = (int)(((long)i0 - 2) % geo.Nx); ib += (ib < 0) ? geo.Nx : 0;
    int kb = (int)(((long)k0 - 2) % geo.Nz); kb += (kb < 0) ? geo.Nz : 0;
    const int nc = (a.mode == 0) ? 3 : 6;
    T acc[6] = {0, 0, 0, 0, 0, 0};
    const size_t plane = (size_t)geo.Nz * geo.Nx;
    for (int p = 0; p < 5; ++p) {
        const T* gy = a.grid + ((size_t)(js + p) * a.ncomp_total + a.comp0) * plane;
        for (int q = 0; q < 5; ++q) {
            int kk = kb + q; kk -= (kk >= geo.Nz) ? geo.Nz : 0;
            T wyz = wy[p] * wz[q];
            const T* gz = gy + (size_t)kk * geo.Nx;
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                int ii = ib + r; ii -= (ii >= geo.Nx) ? geo.Nx : 0;
                T w = wyz * wx[r];
                for (int c = 0; c < nc; ++c) acc[c] += w * gz[c * plane + ii];
            }
        }
    }
    interp_store<T>(a, t, acc);
}

// Spectral evaluation of the global field at the targets (GGEM_OFFGRID_SPECTRAL),
// a warp per target: the type-2 non-uniform FFT of Greengard & Lee in all
// three directions.  In theta = arccos(ybar) the Chebyshev series is a cosine
// series, even and 2 pi-periodic, so y is treated like x and z: the
// oversampled grid holds the field deconvolved by the Gaussian window
// g(t) = exp(-c t^2) (t in fine spacings) on Mx x Mz x the Mt/2 + 1 theta
// nodes of [0, pi], and the window gathered over the 2w nearest fine nodes in
// each direction gives the expansion at the target to the window's tolerance
// (theta nodes beyond 0 or pi are their mirror images).  Lanes split into G
// groups of 32/G: a lane owns one x offset, a group every G-th z row of each
// theta plane, so a row's 2w values are one contiguous load per group.  The
// plane and row offsets and the theta and z weights sit in the warp's shared
// memory.  Warps take the targets in sg.order (cell order for mesh nodes) so
// that the stencils of a block overlap in L1.
template <typename T> __device__ __forceinline__ T wacos(T x);
template <> __device__ __forceinline__ float wacos<float>(float x) { return acosf(x); }
template <> __device__ __forceinline__ double wacos<double>(double x) { return acos(x); }

template <typename T>
__global__ void __launch_bounds__(128, 8) k_interp_spectral(InterpArgs<T> a, SpecGrid sg) {
    __shared__ long offs[4][64];                // per warp: 2w theta planes, 2w z rows
    __shared__ T wts[4][64];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int k = blockIdx.x * (blockDim.x >> 5) + wib;
    if (k >= a.n) return;                       // warp-uniform
    const int t = sg.order ? sg.order[k] : k;
    const GridGeom& geo = a.geo;
    const int w = sg.w, w2 = 2 * sg.w, half = sg.Mt / 2;
    const double xt = a.x[3 * (size_t)t], yt = a.x[3 * (size_t)t + 1],
                 zt = a.x[3 * (size_t)t + 2];
    const size_t plane = (size_t)sg.Mz * sg.Mx;
    const size_t pstride = (size_t)a.ncomp_total * plane;
    // fine-grid coordinates: integer part wrapped into the period (FP64), the
    // fraction and the window arithmetic in the plan's precision T
    const double ux = xt * sg.sx, uz = zt * sg.sz;
    const double flx = floor(ux), flz = floor(uz);
    const T fx = (T)(ux - flx), fz = (T)(uz - flz);
    const int px0 = (int)((long long)flx % sg.Mx), pz0 = (int)((long long)flz % sg.Mz);
    const T yb = (T)fmin(1.0, fmax(-1.0, (yt - geo.y0) * sg.sy - 1.0));
    const T ut = wacos<T>(yb) * (T)sg.st;        // theta in fine spacings, [0, Mt/2]
    const int pt0 = min((int)floor(ut), half);
    const T ft = ut - (T)pt0;
    const T cw = (T)sg.c;
    if (lane < w2) {
        const int o = lane - w + 1;
        const T tt = ft - (T)o, tz = fz - (T)o;
        int pt = pt0 + o;                       // mirror about 0 and pi
        pt = pt < 0 ? -pt : pt;
        pt = pt > half ? sg.Mt - pt : pt;
        int pz = (pz0 + o) % sg.Mz;
        pz += pz < 0 ? sg.Mz : 0;
        offs[wib][lane] = (long)pt * (long)pstride;
        offs[wib][32 + lane] = (long)pz * sg.Mx;
        wts[wib][lane] = wexp<T>(-cw * tt * tt);
        wts[wib][32 + lane] = wexp<T>(-cw * tz * tz);
    }
    const int lpg = w2 <= 8 ? 8 : (w2 <= 16 ? 16 : 32);
    const int G = 32 / lpg, g = lane / lpg, xl = lane - g * lpg;
    const bool xv = xl < w2;
    const T tx = fx - (T)(xl - w + 1);
    const T wx = xv ? wexp<T>(-cw * tx * tx) : (T)0;
    int px = (px0 + xl - w + 1) % sg.Mx;
    px += px < 0 ? sg.Mx : 0;
    __syncwarp();
    const int nc = (a.mode == 0) ? 3 : 6;
    const T* F = (const T*)sg.fine + (size_t)a.comp0 * plane + px;
    T acc[6] = {0, 0, 0, 0, 0, 0};
    if (xv) {
        for (int it = 0; it < w2; ++it) {
            const T* Ft = F + offs[wib][it];
            const T wt = wts[wib][it];
            T sum[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 4
            for (int iz = g; iz < w2; iz += G) {
                const T b = wts[wib][32 + iz];
                const T* Fr = Ft + offs[wib][32 + iz];
#pragma unroll
                for (int c = 0; c < 6; ++c)
                    if (c < nc) sum[c] += b * Fr[c * plane];
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[c] += wt * sum[c];
        }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        T v = acc[c] * wx;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[c] = v;
    }
    if (lane == 0) interp_store<T>(a, t, acc);
}

// Rectangular contraction out[p][col] = sum_n M[p][n] in[n][col] (M: R x C),
// for the Chebyshev coefficients -> deconvolved theta-node values of the
// spectral evaluation; a block takes RT rows of M into shared memory.
template <typename T, int NB>
__global__ void __launch_bounds__(256) k_cheb_rect(int R, int C, int RT, const T* __restrict__ M,
                                                    const T* __restrict__ in,
                                                    T* __restrict__ out, long cols) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Ms = reinterpret_cast<T*>(smraw);
    const int r0 = blockIdx.y * RT, rt = min(RT, R - r0);
    for (int e = threadIdx.x; e < rt * C; e += blockDim.x) Ms[e] = M[(size_t)r0 * C + e];
    __syncthreads();
    const long col = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= cols) return;
    for (int q0 = 0; q0 < rt; q0 += NB) {
        T acc[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[b] = 0;
        for (int n = 0; n < C; ++n) {
            const T v = in[(long)n * cols + col];
#pragma unroll
            for (int b = 0; b < NB; ++b)
                if (q0 + b < rt) acc[b] += Ms[(q0 + b) * C + n] * v;
        }
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (q0 + b < rt) out[(long)(r0 + q0 + b) * cols + col] = acc[b];
    }
}

// Deconvolve and zero-pad the spectral planes onto the oversampled grid: fine
// mode (kz', kx') takes the coarse mode with the same signed wavenumbers times
// dx[kx] dz[kz]; modes the coarse grid lacks (and its Nyquist modes) are zero.
template <typename T>
__global__ void k_spec_pad(const c2_t<T>* __restrict__ spec, long nplanes, int Nx, int Nz,
                           int Mx, int Mz, const T* __restrict__ dx, const T* __restrict__ dz,
                           c2_t<T>* __restrict__ fine) {
    const long total = nplanes * (long)Mz * (Mx / 2);
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
         e += (long)gridDim.x * blockDim.x) {
        const int mkx = Mx / 2, nkx = Nx / 2;
        const long pl = e / ((long)Mz * mkx);
        const int r = (int)(e - pl * Mz * (long)mkx);
        const int kzf = r / mkx, kxf = r - kzf * mkx;
        c2_t<T> v;
        v.x = (T)0;
        v.y = (T)0;
        if (kxf < nkx) {
            int kz = -1;
            if (kzf < Nz / 2) kz = kzf;
            else if (kzf > Mz - Nz / 2) kz = kzf - (Mz - Nz);
            if (kz >= 0) {
                const c2_t<T> c = spec[(pl * Nz + kz) * nkx + kxf];
                const T f = dx[kxf] * dz[kz];
                v.x = c.x * f;
                v.y = c.y * f;
            }
        }
        fine[e] = v;
    }
}

template <typename T>
__device__ __forceinline__ void interp_store(const InterpArgs<T>& a, int t, const T* acc) {
    double* o = a.out + (size_t)t * a.out_stride;
    const T* lo = a.local ? a.local + (size_t)t * a.local_stride : nullptr;
    if (a.mode == 0) {
        for (int c = 0; c < 3; ++c) {
            double v = (double)acc[c] + (lo ? (double)lo[c] : 0.0);
            if (a.qself) v -= a.self_coef * (a.wself ? a.wself[t] : 1.0) * a.qself[3 * t + c];
            o[c] = v;
        }
    } else if (a.mode == 1) {
        for (int c = 0; c < 6; ++c) o[c] = (double)acc[c] + (lo ? (double)lo[c] : 0.0);
    } else {
        double n0 = a.nrm[3 * t], n1 = a.nrm[3 * t + 1], n2 = a.nrm[3 * t + 2];
        double s[6];
        for (int c = 0; c < 6; ++c) s[c] = (double)acc[c];
        double v0 = n0 * s[0] + n1 * s[1] + n2 * s[2];
        double v1 = n0 * s[1] + n1 * s[3] + n2 * s[4];
        double v2 = n0 * s[2] + n1 * s[4] + n2 * s[5];
        double im = 1.0 / a.geo.mu;
        o[0] = v0 * im + (lo ? (double)lo[0] : 0.0);
        o[1] = v1 * im + (lo ? (double)lo[1] : 0.0);
        o[2] = v2 * im + (lo ? (double)lo[2] : 0.0);
    }
}

template <typename T>
cudaError_t interp_combine(const GridGeom& geo, const double* yj, const T* grid, int ncomp_total,
                           int comp0, int n_tgt, const double* x_tgt, const T* local,
                           int local_stride, const double* nrm, const double* qself,
                           const double* wself, double self_coef, int mode, double* out,
                           int out_stride, cudaStream_t st, const SpecGrid* spec) {
    if (n_tgt <= 0) return cudaSuccess;
    InterpArgs<T> a{geo, yj, grid, ncomp_total, comp0, mode, n_tgt, x_tgt, local,
                    local_stride, nrm, qself, wself, self_coef, out, out_stride};
    if (spec) {
        // a warp per target, 4 per block
        k_interp_spectral<T><<<(n_tgt + 3) / 4, 128, 0, st>>>(a, *spec);
    } else {
        k_interp<T><<<(n_tgt + 127) / 128, 128, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t cheb_rect(int R, int C, const T* M, const T* in, T* out, long cols,
                      cudaStream_t st) {
    const int RT = 32;
    const dim3 grid((unsigned)((cols + 255) / 256), (unsigned)((R + RT - 1) / RT));
    const size_t smem = (size_t)RT * C * sizeof(T);
    grant_max_smem((const void*)k_cheb_rect<T, 8>);
    k_cheb_rect<T, 8><<<grid, 256, smem, st>>>(R, C, RT, M, in, out, cols);
    return cudaGetLastError();
}

template <typename T>
cudaError_t spectral_pad(const GridGeom& geo, const T* spec, int nplanes, int Mx, int Mz,
                         const T* dx, const T* dz, T* fine, cudaStream_t st) {
    const long total = (long)nplanes * Mz * (Mx / 2);
    const unsigned nb = (unsigned)std::min<long>((total + 255) / 256, 152L * 16);
    k_spec_pad<T><<<nb, 256, 0, st>>>((const c2_t<T>*)spec, nplanes, geo.Nx, geo.Nz, Mx, Mz,
                                      dx, dz, (c2_t<T>*)fine);
    return cudaGetLastError();
}

#define GGEM_INST_GRID(T)                                                                     \
    template cudaError_t fft_forward<T>(const GridGeom&, T*, int, const void*, const void*,    \
                                        cudaStream_t);                                         \
    template cudaError_t fft_inverse<T>(const GridGeom&, T*, int, const void*, const void*,    \
                                        cudaStream_t, int);                                    \
    template cudaError_t cheb_apply<T>(int, const T*, const T*, T*, long, cudaStream_t, int*,  \
                                       int, const void*);                                      \
    template cudaError_t interp_combine<T>(const GridGeom&, const double*, const T*, int, int, \
                                           int, const double*, const T*, int, const double*,   \
                                           const double*, const double*, double, int, double*, \
                                           int, cudaStream_t, const SpecGrid*);                   \
    template cudaError_t spectral_pad<T>(const GridGeom&, const T*, int, int, int, const T*,   \
                                         const T*, T*, cudaStream_t);                          \
    template cudaError_t cheb_rect<T>(int, int, const T*, const T*, T*, long, cudaStream_t);
GGEM_INST_GRID(float)
GGEM_INST_GRID(double)

}  // namespace ggem
