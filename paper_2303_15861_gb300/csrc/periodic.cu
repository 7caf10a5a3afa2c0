// Periodic Fourier pseudospectral contexts: the discretisation of the paper's two-dimensional
// experiment (Section 5.1, Eq. (ad2d)), where A of Eq. (linop) is diagonal in Fourier space and
// its matrix functions are multipliers on the Fourier coefficients (Section 5.1).
//
// FFT: a batched complex radix-2 FFT along one axis at a time, in the Stockham autosort
// formulation (each stage reads one buffer and writes the other in natural order, so no bit
// reversal is needed). A block takes one line of n points (n a power of two <= 1024) into
// shared memory, runs the log2(n) stages there and writes it back; the twiddles
// e^{-2 pi i j / n}, j < n/2, come from a table computed on the host in FP64.
//
// Right-hand side: F(u) = sum_mu D_mu (a_mumu D_mu u + b_mu u) + r(u) with D_mu the spectral
// first derivative (i k_mu; the Nyquist wavenumber is 0), g(u) = F(u) - A u with A u the
// inverse transform of symbol * u^. A stage output cu u + sum cx X + cg g + cF F is one inverse
// transform of (cg + cF) S - cg symbol u^, S = sum_mu i k_mu (flux_mu)^, plus pointwise terms.
#include <cuda_runtime.h>

#include <algorithm>

#include "adr_internal.h"

namespace adr {
namespace {

template <typename T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// Every line along one axis: element j of line (p, q) sits at p n Q + j Q + q.
template <typename T>
__global__ void __launch_bounds__(256) fft_axis_kernel(Cplx<T>* data, int n, int logn, long long Q, long long lines,
                                                       const Cplx<T>* __restrict__ tw, int inverse) {
    extern __shared__ __align__(16) unsigned char fft_smem[];
    Cplx<T>* b0 = reinterpret_cast<Cplx<T>*>(fft_smem);
    Cplx<T>* b1 = b0 + n;
    const int half = n >> 1;
    const T scale = inverse ? T(1) / T(n) : T(1);
    for (long long line = blockIdx.x; line < lines; line += gridDim.x) {
        const long long p = line / Q, q = line % Q;
        Cplx<T>* base = data + p * n * Q + q;
        for (int j = threadIdx.x; j < n; j += blockDim.x) b0[j] = base[(long long)j * Q];
        __syncthreads();
        Cplx<T>* src = b0;
        Cplx<T>* dst = b1;
        for (int s = 0, Ns = 1; s < logn; ++s, Ns <<= 1) {
            for (int j = threadIdx.x; j < half; j += blockDim.x) {
                const int r = j & (Ns - 1);                   // position inside the current sub-transforms
                Cplx<T> w = tw[r * (half / Ns)];              // e^{-2 pi i r / (2 Ns)}
                if (inverse) w.y = -w.y;
                const Cplx<T> v0 = src[j];
                const Cplx<T> v1 = cmul(src[j + half], w);
                const int o = ((j - r) << 1) + r;             // (j / Ns) 2 Ns + r
                dst[o] = {v0.x + v1.x, v0.y + v1.y};
                dst[o + Ns] = {v0.x - v1.x, v0.y - v1.y};
            }
            __syncthreads();
            Cplx<T>* t = src;
            src = dst;
            dst = t;
        }
        for (int j = threadIdx.x; j < n; j += blockDim.x) base[(long long)j * Q] = {src[j].x * scale, src[j].y * scale};
        __syncthreads();
    }
}

// --------------------------------------------------------------------- pointwise kernels
template <typename T>
__global__ void to_cplx_kernel(const T* __restrict__ x, Cplx<T>* c, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        c[i] = {x[i], T(0)};
}

// out = i k_mu in (the spectral derivative along mu); Q, n of that axis
template <typename T>
__global__ void deriv_kernel(const Cplx<T>* __restrict__ in, Cplx<T>* out, const T* __restrict__ k, int n,
                             long long Q, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const T km = k[(i / Q) % n];
        const Cplx<T> v = in[i];
        out[i] = {-km * v.y, km * v.x};
    }
}

// c = a Re(c) + b u (the flux of direction mu, real)
template <typename T>
__global__ void flux_kernel(Cplx<T>* c, const T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ u,
                            long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        c[i] = {a[i] * c[i].x + b[i] * u[i], T(0)};
}

// S (=|+=) i k_mu c
template <typename T>
__global__ void divacc_kernel(const Cplx<T>* __restrict__ c, Cplx<T>* S, const T* __restrict__ k, int n, long long Q,
                              long long N, int first) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const T km = k[(i / Q) % n];
        const Cplx<T> v = c[i];
        const Cplx<T> d = {-km * v.y, km * v.x};
        S[i] = first ? d : Cplx<T>{S[i].x + d.x, S[i].y + d.y};
    }
}

// out = cgF S - cg sym u^
template <typename T>
__global__ void spec_out_kernel(const Cplx<T>* __restrict__ S, const Cplx<T>* __restrict__ U, const Cplx<T>* __restrict__ sym,
                                Cplx<T>* out, T cgF, T cg, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const Cplx<T> au = cmul(sym[i], U[i]);
        out[i] = {cgF * S[i].x - cg * au.x, cgF * S[i].y - cg * au.y};
    }
}

template <typename T>
struct RealOut {
    const T* u;
    const T* X[kMaxExtra];
    int nx;
    T cu, cx[kMaxExtra], cgF, r[4];
};

// out = cu u + sum cx X + Re(c) + cgF r(u)
template <typename T>
__global__ void real_out_kernel(RealOut<T> a, const Cplx<T>* __restrict__ c, T* out, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const T u = a.u[i];
        T v = a.cu * u + c[i].x + a.cgF * (a.r[0] + u * (a.r[1] + u * (a.r[2] + u * a.r[3])));
        for (int e = 0; e < a.nx; ++e) v += a.cx[e] * a.X[e][i];
        out[i] = v;
    }
}

template <typename T>
__global__ void mul_kernel(Cplx<T>* c, const Cplx<T>* __restrict__ M, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        c[i] = cmul(c[i], M[i]);
}

// y = base + alpha Re(c)  (y = Re(c) without base)
template <typename T>
__global__ void axpy_out_kernel(const Cplx<T>* __restrict__ c, const T* base, T* y, T alpha, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        y[i] = base ? base[i] + alpha * c[i].x : c[i].x;
}

int g_sms = 0;
int sms() {
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

unsigned pw_grid(long long N) { return unsigned(std::min<long long>((N + 255) / 256, 8LL * sms())); }

// forward (inverse = 0) or inverse (1, scaled by 1/N) transform over every axis, in place
template <typename T>
cudaError_t fft_all(const PeriodicArgs<T>& P, Cplx<T>* c, int inverse, cudaStream_t st) {
    long long Q = 1;
    for (int mu = 0; mu < P.dim; ++mu) {
        const int n = P.n[mu];
        int logn = 0;
        while ((1 << logn) < n) ++logn;
        const long long lines = P.N / n;
        const unsigned grid = unsigned(std::min<long long>(lines, 4LL * sms()));
        const int threads = std::min(256, std::max(32, n / 2));
        fft_axis_kernel<T><<<grid, threads, 2 * n * sizeof(Cplx<T>), st>>>(c, n, logn, Q, lines, P.tw[mu], inverse);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        Q *= n;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t rhs_impl(const PeriodicArgs<T>& P, const StencilArgs<T>& s, cudaStream_t st) {
    if (s.nout < 1 || s.nout > kMaxOut || s.nx < 0 || s.nx > kMaxExtra || !s.u) return cudaErrorInvalidValue;
    const long long N = P.N;
    const unsigned g = pw_grid(N);
    cudaError_t e;
    to_cplx_kernel<T><<<g, 256, 0, st>>>(s.u, P.Cu, N);
    if ((e = fft_all(P, P.Cu, 0, st)) != cudaSuccess) return e;
    long long Q = 1;
    for (int mu = 0; mu < P.dim; ++mu) {
        deriv_kernel<T><<<g, 256, 0, st>>>(P.Cu, P.Ct, P.k[mu], P.n[mu], Q, N);
        if ((e = fft_all(P, P.Ct, 1, st)) != cudaSuccess) return e;
        flux_kernel<T><<<g, 256, 0, st>>>(P.Ct, P.a[mu], P.b[mu], s.u, N);
        if ((e = fft_all(P, P.Ct, 0, st)) != cudaSuccess) return e;
        divacc_kernel<T><<<g, 256, 0, st>>>(P.Ct, P.Cs, P.k[mu], P.n[mu], Q, N, mu == 0 ? 1 : 0);
        Q *= P.n[mu];
    }
    for (int j = 0; j < s.nout; ++j) {
        const T cgF = T(s.cg[j] + s.cF[j]);
        spec_out_kernel<T><<<g, 256, 0, st>>>(P.Cs, P.Cu, P.sym, P.Ct, cgF, T(s.cg[j]), N);
        if ((e = fft_all(P, P.Ct, 1, st)) != cudaSuccess) return e;
        RealOut<T> ro;
        ro.u = s.u;
        ro.nx = s.nx;
        ro.cu = T(s.cu[j]);
        ro.cgF = cgF;
        for (int q = 0; q < 4; ++q) ro.r[q] = T(P.r[q]);
        for (int x = 0; x < kMaxExtra; ++x) {
            ro.X[x] = s.X[x];
            ro.cx[x] = T(s.cx[j][x]);
        }
        real_out_kernel<T><<<g, 256, 0, st>>>(ro, P.Ct, s.out[j], N);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t multiplier_impl(const PeriodicArgs<T>& P, const Cplx<T>* M, const T* x, T* y, const T* base, double alpha,
                            cudaStream_t st) {
    if (!M || !x || !y) return cudaErrorInvalidValue;
    const long long N = P.N;
    const unsigned g = pw_grid(N);
    cudaError_t e;
    to_cplx_kernel<T><<<g, 256, 0, st>>>(x, P.Ct, N);
    if ((e = fft_all(P, P.Ct, 0, st)) != cudaSuccess) return e;
    mul_kernel<T><<<g, 256, 0, st>>>(P.Ct, M, N);
    if ((e = fft_all(P, P.Ct, 1, st)) != cudaSuccess) return e;
    axpy_out_kernel<T><<<g, 256, 0, st>>>(P.Ct, base, y, T(alpha), N);
    return cudaGetLastError();
}

}  // namespace

int periodic_rhs_launches(int dim, int nout) { return 1 + dim + dim * (2 * dim + 3) + nout * (dim + 2); }
int periodic_multiplier_launches(int dim) { return 2 * dim + 3; }

cudaError_t launch_periodic_rhs(const PeriodicArgs<double>& P, const StencilArgs<double>& s, cudaStream_t st) {
    return rhs_impl(P, s, st);
}
cudaError_t launch_periodic_rhs(const PeriodicArgs<float>& P, const StencilArgs<float>& s, cudaStream_t st) {
    return rhs_impl(P, s, st);
}
cudaError_t launch_periodic_multiplier(const PeriodicArgs<double>& P, const Cplx<double>* M, const double* x, double* y,
                                       const double* base, double alpha, cudaStream_t st) {
    return multiplier_impl(P, M, x, y, base, alpha, st);
}
cudaError_t launch_periodic_multiplier(const PeriodicArgs<float>& P, const Cplx<float>* M, const float* x, float* y,
                                       const float* base, double alpha, cudaStream_t st) {
    return multiplier_impl(P, M, x, y, base, alpha, st);
}

}  // namespace adr
