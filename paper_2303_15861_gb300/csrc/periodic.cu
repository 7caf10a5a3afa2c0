// Periodic Fourier pseudospectral contexts: the discretisation of the paper's two-dimensional
// experiment (Section 5.1, Eq. (ad2d)), where A of Eq. (linop) is diagonal in Fourier space and
// its matrix functions are multipliers on the Fourier coefficients (Section 5.1).
//
// FFT: complex radix-4 transforms (one radix-2 stage first when log2 n is odd) along one axis at
// a time in the Stockham autosort form (each stage reads one shared-memory buffer and writes the
// other in natural order, so no bit reversal is needed), twiddles e^{-2 pi i j / n}, j < n/2,
// from a host FP64 table. A block
// takes G lines of one axis into shared memory: along x1 the lines are contiguous; along the
// other axes it takes G neighbouring lines, so that every global access moves G consecutive
// elements. The inverse transform is unscaled inside the stages; its 1/n is applied once per
// axis where the result is consumed.
//
// Fusion. A d-dimensional transform is d passes. The last axis d is the pivot: there all other
// axes are already transformed, so the pivot pass does the forward transform, the pointwise
// work in Fourier space and the inverse transform in one kernel. The passes along x1 take the
// real-space prologue (a real input) or epilogue (the stage combination).
//   Multiplier y = base + alpha Re F^-1(M F x):   x1 fwd | (x2 fwd) | pivot: F, M, F^-1 |
//                                                (x2 inv) | x1 inv + axpy.          2-D: 3 kernels
//   Right-hand side, F(u) = sum_mu D_mu (a_mumu D_mu u + b_mu u) + r(u), g = F - A u, with the
//   spectral first derivative D_mu = F^-1 i k_mu F (Nyquist wavenumber 0):
//     x1 fwd u | (x2 fwd) | pivot: u^, i k_mu u^ -> d arrays | (x2 inv) |
//     x1: D_mu u -> flux f_mu = a_mumu D_mu u + b_mu u -> forward | (x2 fwd) |
//     pivot: S = sum_mu i k_mu f_mu^, O_j = (cg_j + cF_j) S - cg_j s u^ | (x2 inv) |
//     x1 inv + out_j = cu_j u + sum_e cx_je X_e + Re O_j + (cg_j + cF_j) r(u).      2-D: 5 kernels
//   Stage kept in Fourier space (2-D periodic Lawson-Euler, ETD2RK, exponential Euler, erk2p1,
//   stabilized Lawson-Euler, Lawson2a/2b): the same first three passes, the x1 flux pass also
//   transforming the pointwise part r(u) into CN; the pivot then forms F^ = S + F_d CN,
//   H = cgF F^ - cg s u^ and the whole stage Mu (cu u^) + Mg (H + cgz Z) + cz Z, saves
//   Ms (zu u^ + zF F^ - zg s u^) for a later stage, and transforms back; the last x1 pass
//   writes y.                                                                           2-D: 5 kernels
//   When the next stage's input is this y, the last x1 pass also transforms y forward along x1
//   into Cu, and the next stage starts at its pivot pass.                       2-D: 4 kernels more
#include <cuda_runtime.h>

#include <algorithm>

#include "adr_internal.h"

namespace adr {
namespace {

template <typename T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

enum PassMode {
    PM_FWD_REAL = 0,     // x1: C[0] = F_1 x (x real)
    PM_PLAIN = 1,        // C[a] = F_mu C[a] or F_mu^-1 C[a], a < na
    PM_PIVOT_MULT = 2,   // C[0] = F_d^-1 (M F_d C[0])
    PM_FINAL_AXPY = 3,   // x1: y = base + alpha Re F_1^-1 C[0]  (y = Re ... without base)
    PM_PIVOT_DERIV = 4,  // Cu = F_d Cu (= u^); C[mu] = F_d^-1 (i k_mu u^)
    PM_FLUX = 5,         // x1: C[mu] = F_1 (a_mu Re F_1^-1 C[mu] + b_mu u)
    PM_PIVOT_DIV = 6,    // S = sum_mu i k_mu F_d C[mu]; C[j] = F_d^-1 (cgF_j S - cg_j M Cu)
    PM_FINAL_OUT = 7,    // x1: out_j = cu_j u + sum cx_je X_e + Re F_1^-1 C[j] + cgF_j r(u)
    PM_PIVOT_STAGE = 8,  // F^ = sum_mu i k_mu F_d C[mu] + F_d CN, H = cgF F^ - cg s u^;
                         // C[0] = F_d^-1 (Mu (cu u^) + Mg (H + cgz Z) + cz Z);
                         // Zs = Ms (zu u^ + zF F^ - zg s u^)
    PM_FINAL_FWD = 9,    // x1: y = Re F_1^-1 C[0]; Cu = F_1 y (the next stage's first pass)
};

constexpr int kPassThreads = 256;
constexpr size_t kPassSmemMax = 200 * 1024;

template <typename T>
struct Pass {
    // the pass: axis, its length n = 2^logn, G = 2^logG lines per block, shared-memory row pitch
    int axis, n, logn, G, logG, pitch;
    int logQ;                 // stride of the axis, Q = 2^logQ
    int log_gpp;              // line groups per outer index p (Q > 1): Q / G = 2^log_gpp
    long long groups;         // line groups in the grid
    // all axes (wavenumber lookup)
    int dim, nn[3], logQs[3];
    const Cplx<T>* tw;
    const T* k[3];
    // arrays
    Cplx<T>* Cu;
    Cplx<T>* C[3];
    int na, inverse;
    const Cplx<T>* M;         // multiplier (PM_PIVOT_MULT) or symbol of A (PM_PIVOT_DIV)
    const T* x;               // real input: x (PM_FWD_REAL) or the stage input u
    T* y;
    const T* base;
    T alpha;
    const T* a[3];
    const T* b[3];
    int nout, nx;
    const T* X[kMaxExtra];
    T* out[kMaxOut];
    T cu[kMaxOut], cx[kMaxOut][kMaxExtra], cgF[kMaxOut], cg[kMaxOut], r[4];
    int adelta;               // a Lap u form (see PeriodicArgs)
    T* dif;                   // adelta: sum_mu a_mumu D_mu D_mu u
    // fused stages (PM_FLUX with nonflux, PM_PIVOT_STAGE): the pointwise part of F (r(u), and the
    // a Lap u product) transformed along x1 into CN; the stage's multipliers and saved array
    int nonflux;
    Cplx<T>* CN;
    const Cplx<T>* Mu;
    const Cplx<T>* Mg;
    const Cplx<T>* Ms;
    const Cplx<T>* Z;
    Cplx<T>* Zs;
    T scu, scgF, scg, scgz, scz;
    T szu, szF, szg;
};

// Global index of element j of line g of line group grp.
template <typename T>
__device__ __forceinline__ long long elem_index(const Pass<T>& P, long long grp, int g, int j) {
    if (P.logQ == 0) return (((grp << P.logG) + g) << P.logn) + j;
    const long long p = grp >> P.log_gpp;
    const long long q0 = (grp & ((1LL << P.log_gpp) - 1)) << P.logG;
    return (p << (P.logn + P.logQ)) + ((long long)j << P.logQ) + q0 + g;
}

// Call f(smem offset, global index) for every element of the block's G lines, in the order that
// makes consecutive threads touch consecutive global elements.
template <typename T, typename F>
__device__ __forceinline__ void for_elems(const Pass<T>& P, long long grp, F f) {
    const int total = P.G << P.logn;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int g, j;
        if (P.logQ == 0) { g = idx >> P.logn; j = idx & (P.n - 1); }
        else             { g = idx & (P.G - 1); j = idx >> P.logG; }
        f(g * P.pitch + j, elem_index(P, grp, g, j), j);
    }
}

// Wavenumber of axis mu at global index i (j: position along the pass axis).
template <typename T>
__device__ __forceinline__ T wavenumber(const Pass<T>& P, int mu, long long i, int j) {
    if (mu == P.axis) return P.k[mu][j];
    return P.k[mu][(i >> P.logQs[mu]) & (P.nn[mu] - 1)];
}

// Stockham transform of the G lines in src (destroys src and dst); returns the buffer that holds
// the result (unscaled). Radix-4 stages, after one radix-2 stage when log2 n is odd: a stage over
// sub-transforms of length Ns takes the four points j + q n/4 (q = 0..3) of butterfly j,
// r = j mod Ns, scales point q by e^{-2 pi i q r / (4 Ns)} (conjugated for the inverse), forms
// their 4-point DFT V_k and writes V_k to 4 (j - r) + r + k Ns.
template <typename T>
__device__ Cplx<T>* fft_lines(const Pass<T>& P, const Cplx<T>* tws, Cplx<T>* src, Cplx<T>* dst, bool inverse) {
    const int half = P.n >> 1, quarter = P.n >> 2;
    int s = 0, Ns = 1;
    if (P.logn & 1) {                                     // radix 2 with Ns = 1: all twiddles are 1
        for (int bf = threadIdx.x; bf < P.G * half; bf += blockDim.x) {
            const int g = bf >> (P.logn - 1), jj = bf & (half - 1);
            const Cplx<T>* sl = src + g * P.pitch;
            Cplx<T>* dl = dst + g * P.pitch;
            const Cplx<T> v0 = sl[jj], v1 = sl[jj + half];
            dl[2 * jj] = {v0.x + v1.x, v0.y + v1.y};
            dl[2 * jj + 1] = {v0.x - v1.x, v0.y - v1.y};
        }
        __syncthreads();
        Cplx<T>* t = src;
        src = dst;
        dst = t;
        s = 1;
        Ns = 2;
    }
    for (; s < P.logn; s += 2, Ns <<= 2) {
        const int lstep = P.logn - 2 - s;                 // n / (4 Ns) = 2^lstep
        for (int bf = threadIdx.x; bf < P.G * quarter; bf += blockDim.x) {
            const int g = bf >> (P.logn - 2), jj = bf & (quarter - 1);
            const int r = jj & (Ns - 1);
            const Cplx<T>* sl = src + g * P.pitch;
            Cplx<T>* dl = dst + g * P.pitch;
            Cplx<T> v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = sl[jj + q * quarter];
#pragma unroll
            for (int q = 1; q < 4; ++q) {                 // e^{-2 pi i m / n}, m = q r n / (4 Ns) < 3n/4
                const int m = (q * r) << lstep;
                Cplx<T> w = m < half ? tws[m] : Cplx<T>{-tws[m - half].x, -tws[m - half].y};
                if (inverse) w.y = -w.y;
                v[q] = cmul(v[q], w);
            }
            const Cplx<T> a0 = {v[0].x + v[2].x, v[0].y + v[2].y}, a1 = {v[0].x - v[2].x, v[0].y - v[2].y};
            const Cplx<T> a2 = {v[1].x + v[3].x, v[1].y + v[3].y}, a3 = {v[1].x - v[3].x, v[1].y - v[3].y};
            // -i a3 = (a3.y, -a3.x) for the forward transform, +i a3 for the inverse
            const Cplx<T> ia3 = inverse ? Cplx<T>{-a3.y, a3.x} : Cplx<T>{a3.y, -a3.x};
            const int o = ((jj - r) << 2) + r;
            dl[o] = {a0.x + a2.x, a0.y + a2.y};
            dl[o + Ns] = {a1.x + ia3.x, a1.y + ia3.y};
            dl[o + 2 * Ns] = {a0.x - a2.x, a0.y - a2.y};
            dl[o + 3 * Ns] = {a1.x - ia3.x, a1.y - ia3.y};
        }
        __syncthreads();
        Cplx<T>* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kPassThreads) fourier_pass_kernel(const __grid_constant__ Pass<T> P) {
    extern __shared__ __align__(16) unsigned char fourier_smem[];
    Cplx<T>* tws = reinterpret_cast<Cplx<T>*>(fourier_smem);
    Cplx<T>* B0 = tws + (P.n >> 1);
    const int bsize = P.G * P.pitch;
    Cplx<T>* B1 = B0 + bsize;
    Cplx<T>* B2 = B1 + bsize;
    for (int j = threadIdx.x; j < (P.n >> 1); j += blockDim.x) tws[j] = P.tw[j];
    const T inv_n = T(1) / T(P.n);
    __syncthreads();

    for (long long grp = blockIdx.x; grp < P.groups; grp += gridDim.x) {
        if (MODE == PM_FWD_REAL) {
            for_elems(P, grp, [&](int o, long long i, int) { B0[o] = {P.x[i], T(0)}; });
            __syncthreads();
            Cplx<T>* R = fft_lines(P, tws, B0, B1, false);
            for_elems(P, grp, [&](int o, long long i, int) { P.C[0][i] = R[o]; });
        } else if (MODE == PM_PLAIN) {
            const T sc = P.inverse ? inv_n : T(1);
            for (int a = 0; a < P.na; ++a) {
                Cplx<T>* A = P.C[a];
                for_elems(P, grp, [&](int o, long long i, int) { B0[o] = A[i]; });
                __syncthreads();
                Cplx<T>* R = fft_lines(P, tws, B0, B1, P.inverse != 0);
                for_elems(P, grp, [&](int o, long long i, int) { A[i] = {R[o].x * sc, R[o].y * sc}; });
                __syncthreads();
            }
        } else if (MODE == PM_PIVOT_MULT) {
            for_elems(P, grp, [&](int o, long long i, int) { B0[o] = P.C[0][i]; });
            __syncthreads();
            Cplx<T>* R = fft_lines(P, tws, B0, B1, false);
            for_elems(P, grp, [&](int o, long long i, int) { R[o] = cmul(R[o], P.M[i]); });
            __syncthreads();
            Cplx<T>* R2 = fft_lines(P, tws, R, R == B0 ? B1 : B0, true);
            for_elems(P, grp, [&](int o, long long i, int) { P.C[0][i] = {R2[o].x * inv_n, R2[o].y * inv_n}; });
        } else if (MODE == PM_FINAL_AXPY) {
            for_elems(P, grp, [&](int o, long long i, int) { B0[o] = P.C[0][i]; });
            __syncthreads();
            Cplx<T>* R = fft_lines(P, tws, B0, B1, true);
            for_elems(P, grp, [&](int o, long long i, int) {
                const T v = R[o].x * inv_n;
                P.y[i] = P.base ? P.base[i] + P.alpha * v : v;
            });
        } else if (MODE == PM_FINAL_FWD) {
            for_elems(P, grp, [&](int o, long long i, int) { B0[o] = P.C[0][i]; });
            __syncthreads();
            Cplx<T>* R = fft_lines(P, tws, B0, B1, true);
            for_elems(P, grp, [&](int o, long long i, int) {     // the same values FWD_REAL would read
                const T v = R[o].x * inv_n;
                P.y[i] = v;
                R[o] = {v, T(0)};
            });
            __syncthreads();
            Cplx<T>* R2 = fft_lines(P, tws, R, R == B0 ? B1 : B0, false);
            for_elems(P, grp, [&](int o, long long i, int) { P.Cu[i] = R2[o]; });
        } else if (MODE == PM_PIVOT_DERIV) {
            for_elems(P, grp, [&](int o, long long i, int) { B0[o] = P.Cu[i]; });
            __syncthreads();
            Cplx<T>* U = fft_lines(P, tws, B0, B1, false);   // u^ (kept for every mu)
            Cplx<T>* Fr = (U == B0) ? B1 : B0;
            for_elems(P, grp, [&](int o, long long i, int) { P.Cu[i] = U[o]; });
            for (int mu = 0; mu < P.dim; ++mu) {
                for_elems(P, grp, [&](int o, long long i, int j) {
                    const T km = wavenumber(P, mu, i, j);
                    if (P.adelta) B2[o] = {-km * km * U[o].x, -km * km * U[o].y};   // (i k)^2 u^
                    else          B2[o] = {-km * U[o].y, km * U[o].x};              // i k u^
                });
                __syncthreads();
                Cplx<T>* R = fft_lines(P, tws, B2, Fr, true);
                Cplx<T>* D = P.C[mu];
                for_elems(P, grp, [&](int o, long long i, int) { D[i] = {R[o].x * inv_n, R[o].y * inv_n}; });
                __syncthreads();
            }
        } else if (MODE == PM_FLUX) {
            for (int mu = 0; mu < P.dim; ++mu) {
                Cplx<T>* D = P.C[mu];
                const T* am = P.a[mu];
                const T* bm = P.b[mu];
                for_elems(P, grp, [&](int o, long long i, int) { B0[o] = D[i]; });
                __syncthreads();
                Cplx<T>* R = fft_lines(P, tws, B0, B1, true);
                if (P.adelta) {      // D_mu D_mu u is complete here: a_mumu times it goes to dif; the flux is b_mu u
                    for_elems(P, grp, [&](int o, long long i, int) {
                        const T d2 = am[i] * (R[o].x * inv_n);
                        P.dif[i] = mu == 0 ? d2 : P.dif[i] + d2;
                        R[o] = {bm[i] * P.x[i], T(0)};
                    });
                } else {
                    for_elems(P, grp, [&](int o, long long i, int) {
                        R[o] = {am[i] * (R[o].x * inv_n) + bm[i] * P.x[i], T(0)};
                    });
                }
                __syncthreads();
                Cplx<T>* R2 = fft_lines(P, tws, R, R == B0 ? B1 : B0, false);
                for_elems(P, grp, [&](int o, long long i, int) { D[i] = R2[o]; });
                __syncthreads();
            }
            if (P.nonflux) {   // r(u) (+ the a Lap u product), forward along x1, into CN
                for_elems(P, grp, [&](int o, long long i, int) {
                    const T u = P.x[i];
                    T v = P.r[0] + u * (P.r[1] + u * (P.r[2] + u * P.r[3]));
                    if (P.adelta) v += P.dif[i];
                    B0[o] = {v, T(0)};
                });
                __syncthreads();
                Cplx<T>* R = fft_lines(P, tws, B0, B1, false);
                for_elems(P, grp, [&](int o, long long i, int) { P.CN[i] = R[o]; });
                __syncthreads();
            }
        } else if (MODE == PM_PIVOT_STAGE) {
            for (int mu = 0; mu <= P.dim; ++mu) {      // B2 = sum_mu i k_mu f_mu^ + (pointwise part)^
                const Cplx<T>* src = mu < P.dim ? P.C[mu] : P.CN;
                for_elems(P, grp, [&](int o, long long i, int) { B0[o] = src[i]; });
                __syncthreads();
                Cplx<T>* R = fft_lines(P, tws, B0, B1, false);
                for_elems(P, grp, [&](int o, long long i, int j) {
                    Cplx<T> d = R[o];
                    if (mu < P.dim) {
                        const T km = wavenumber(P, mu, i, j);
                        d = {-km * R[o].y, km * R[o].x};
                    }
                    B2[o] = mu == 0 ? d : Cplx<T>{B2[o].x + d.x, B2[o].y + d.y};
                });
                __syncthreads();
            }
            for_elems(P, grp, [&](int o, long long i, int) {
                const Cplx<T> uh = P.Cu[i];
                const Cplx<T> fh = B2[o];
                const Cplx<T> au = cmul(P.M[i], uh);
                const Cplx<T> z = P.Z ? P.Z[i] : Cplx<T>{T(0), T(0)};
                if (P.Zs) {
                    const Cplx<T> w = {P.szu * uh.x + P.szF * fh.x - P.szg * au.x,
                                       P.szu * uh.y + P.szF * fh.y - P.szg * au.y};
                    P.Zs[i] = P.Ms ? cmul(P.Ms[i], w) : w;
                }
                Cplx<T> h = {P.scgF * fh.x - P.scg * au.x + P.scgz * z.x,
                             P.scgF * fh.y - P.scg * au.y + P.scgz * z.y};
                if (P.Mg) h = cmul(P.Mg[i], h);
                Cplx<T> v = {P.scu * uh.x, P.scu * uh.y};
                if (P.Mu) v = cmul(P.Mu[i], v);
                B0[o] = {v.x + h.x + P.scz * z.x, v.y + h.y + P.scz * z.y};
            });
            __syncthreads();
            Cplx<T>* R = fft_lines(P, tws, B0, B1, true);
            for_elems(P, grp, [&](int o, long long i, int) { P.C[0][i] = {R[o].x * inv_n, R[o].y * inv_n}; });
        } else if (MODE == PM_PIVOT_DIV) {
            for (int mu = 0; mu < P.dim; ++mu) {       // S (in B2) = sum_mu i k_mu f_mu^
                for_elems(P, grp, [&](int o, long long i, int) { B0[o] = P.C[mu][i]; });
                __syncthreads();
                Cplx<T>* R = fft_lines(P, tws, B0, B1, false);
                for_elems(P, grp, [&](int o, long long i, int j) {
                    const T km = wavenumber(P, mu, i, j);
                    const Cplx<T> d = {-km * R[o].y, km * R[o].x};
                    B2[o] = mu == 0 ? d : Cplx<T>{B2[o].x + d.x, B2[o].y + d.y};
                });
                __syncthreads();
            }
            for (int jo = 0; jo < P.nout; ++jo) {
                const T cgF = P.cgF[jo], cg = P.cg[jo];
                for_elems(P, grp, [&](int o, long long i, int) {
                    const Cplx<T> au = cmul(P.M[i], P.Cu[i]);
                    B0[o] = {cgF * B2[o].x - cg * au.x, cgF * B2[o].y - cg * au.y};
                });
                __syncthreads();
                Cplx<T>* R = fft_lines(P, tws, B0, B1, true);
                Cplx<T>* D = P.C[jo];
                for_elems(P, grp, [&](int o, long long i, int) { D[i] = {R[o].x * inv_n, R[o].y * inv_n}; });
                __syncthreads();
            }
        } else if (MODE == PM_FINAL_OUT) {
            for (int jo = 0; jo < P.nout; ++jo) {
                for_elems(P, grp, [&](int o, long long i, int) { B0[o] = P.C[jo][i]; });
                __syncthreads();
                Cplx<T>* R = fft_lines(P, tws, B0, B1, true);
                T* out = P.out[jo];
                for_elems(P, grp, [&](int o, long long i, int) {
                    const T u = P.x[i];
                    T v = P.cu[jo] * u + R[o].x * inv_n +
                          P.cgF[jo] * (P.r[0] + u * (P.r[1] + u * (P.r[2] + u * P.r[3])));
                    if (P.adelta) v += P.cgF[jo] * P.dif[i];
                    for (int e = 0; e < P.nx; ++e) v += P.cx[jo][e] * P.X[e][i];
                    out[i] = v;
                });
                __syncthreads();
            }
        }
        __syncthreads();
    }
}

int ilog2(long long v) {
    int l = 0;
    while ((1LL << l) < v) ++l;
    return l;
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

// Buffers of shared memory a mode needs besides the twiddles.
int mode_buffers(int mode) { return (mode == PM_PIVOT_DERIV || mode == PM_PIVOT_DIV || mode == PM_PIVOT_STAGE) ? 3 : 2; }

size_t pass_smem(int n, int G, int pitch, int nb, size_t cs) { return (size_t(n / 2) + size_t(nb) * G * pitch) * cs; }

// Geometry of a pass along `axis`: G lines per block, as many as keep at least two blocks per
// SM busy and fit the shared memory, and along strided axes at least one full 32-byte sector.
template <typename T>
Pass<T> make_pass(const PeriodicArgs<T>& A, int axis, int mode) {
    Pass<T> P{};
    P.axis = axis;
    P.dim = A.dim;
    long long Q = 1;
    for (int m = 0; m < A.dim; ++m) {
        P.nn[m] = A.n[m];
        P.logQs[m] = ilog2(Q);
        P.k[m] = A.k[m];
        P.a[m] = A.a[m];
        P.b[m] = A.b[m];
        P.C[m] = A.C[m];
        Q *= A.n[m];
    }
    P.n = A.n[axis];
    P.logn = ilog2(P.n);
    P.logQ = P.logQs[axis];
    const long long Qa = 1LL << P.logQ;
    const long long lines = A.N / P.n;
    const long long limit = P.logQ == 0 ? lines : Qa;     // a group stays inside one outer index
    const size_t cs = sizeof(Cplx<T>);
    const int nb = mode_buffers(mode);
    auto pitch_of = [&](int) { return P.logQ == 0 ? P.n : P.n + 1; };
    int G = 1;
    auto fits = [&](int g2) { return g2 <= limit && pass_smem(P.n, g2, pitch_of(g2), nb, cs) <= kPassSmemMax; };
    while (fits(2 * G) && lines / (2 * G) >= 2LL * sms()) G *= 2;
    while (P.logQ > 0 && size_t(G) * cs < 32 && fits(2 * G)) G *= 2;
    P.G = G;
    P.logG = ilog2(G);
    P.pitch = pitch_of(G);
    P.log_gpp = P.logQ > P.logG ? P.logQ - P.logG : 0;
    P.groups = lines / G;
    P.tw = A.tw[axis];
    P.Cu = A.Cu;
    for (int i = 0; i < 4; ++i) P.r[i] = T(A.r[i]);
    P.adelta = A.adelta ? 1 : 0;
    P.dif = A.dif;
    return P;
}

template <typename T, int MODE>
cudaError_t launch_pass_on(const Pass<T>& P, cudaStream_t st) {
    const size_t smem = pass_smem(P.n, P.G, P.pitch, mode_buffers(MODE), sizeof(Cplx<T>));
    const int work = std::max(P.G * (P.n >> 1), 1);
    const int threads = std::min(kPassThreads, (work + 31) / 32 * 32);
    const long long grid = std::min<long long>(P.groups, 64LL * sms());
    fourier_pass_kernel<T, MODE><<<unsigned(grid), threads, smem, st>>>(P);
    return cudaGetLastError();
}

template <typename T>
cudaError_t prepare_impl() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kPassSmemMax));
    };
    set(reinterpret_cast<const void*>(fourier_pass_kernel<T, PM_FWD_REAL>));
    set(reinterpret_cast<const void*>(fourier_pass_kernel<T, PM_PLAIN>));
    set(reinterpret_cast<const void*>(fourier_pass_kernel<T, PM_PIVOT_MULT>));
    set(reinterpret_cast<const void*>(fourier_pass_kernel<T, PM_FINAL_AXPY>));
    set(reinterpret_cast<const void*>(fourier_pass_kernel<T, PM_PIVOT_DERIV>));
    set(reinterpret_cast<const void*>(fourier_pass_kernel<T, PM_FLUX>));
    set(reinterpret_cast<const void*>(fourier_pass_kernel<T, PM_PIVOT_DIV>));
    set(reinterpret_cast<const void*>(fourier_pass_kernel<T, PM_FINAL_OUT>));
    set(reinterpret_cast<const void*>(fourier_pass_kernel<T, PM_PIVOT_STAGE>));
    set(reinterpret_cast<const void*>(fourier_pass_kernel<T, PM_FINAL_FWD>));
    sms();
    return e;
}

// The passes along the middle axes (x2 of a 3-D grid), forward or inverse, on na arrays.
template <typename T>
cudaError_t middle_passes(const PeriodicArgs<T>& A, Cplx<T>* const* arrays, int na, int inverse, cudaStream_t st) {
    for (int ax = 1; ax + 1 < A.dim; ++ax) {
        const int axis = inverse ? A.dim - 1 - ax : ax;
        Pass<T> P = make_pass(A, axis, PM_PLAIN);
        for (int a = 0; a < na; ++a) P.C[a] = arrays[a];
        P.na = na;
        P.inverse = inverse;
        const cudaError_t e = launch_pass_on<T, PM_PLAIN>(P, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t rhs_impl(const PeriodicArgs<T>& A, const StencilArgs<T>& s, cudaStream_t st) {
    if (s.nout < 1 || s.nout > kMaxOut || s.nout > A.dim || s.nx < 0 || s.nx > kMaxExtra || !s.u)
        return cudaErrorInvalidValue;
    const int d = A.dim, last = d - 1;
    cudaError_t e;
    {   // Cu = F_1 u
        Pass<T> P = make_pass(A, 0, PM_FWD_REAL);
        P.x = s.u;
        P.C[0] = A.Cu;
        if ((e = launch_pass_on<T, PM_FWD_REAL>(P, st)) != cudaSuccess) return e;
    }
    Cplx<T>* cu_only[1] = {A.Cu};
    if ((e = middle_passes(A, cu_only, 1, 0, st)) != cudaSuccess) return e;
    {   // u^ and i k_mu u^, back along the pivot axis
        Pass<T> P = make_pass(A, last, PM_PIVOT_DERIV);
        if ((e = launch_pass_on<T, PM_PIVOT_DERIV>(P, st)) != cudaSuccess) return e;
    }
    Cplx<T>* const* Cs = A.C;
    if ((e = middle_passes(A, Cs, d, 1, st)) != cudaSuccess) return e;
    {   // fluxes, forward along x1
        Pass<T> P = make_pass(A, 0, PM_FLUX);
        P.x = s.u;
        if ((e = launch_pass_on<T, PM_FLUX>(P, st)) != cudaSuccess) return e;
    }
    if ((e = middle_passes(A, Cs, d, 0, st)) != cudaSuccess) return e;
    {   // divergence and the stage outputs in Fourier space, back along the pivot axis
        Pass<T> P = make_pass(A, last, PM_PIVOT_DIV);
        P.M = A.sym;
        P.nout = s.nout;
        for (int j = 0; j < s.nout; ++j) {
            P.cgF[j] = T(s.cg[j] + s.cF[j]);
            P.cg[j] = T(s.cg[j]);
        }
        if ((e = launch_pass_on<T, PM_PIVOT_DIV>(P, st)) != cudaSuccess) return e;
    }
    if ((e = middle_passes(A, Cs, s.nout, 1, st)) != cudaSuccess) return e;
    {   // stage outputs in real space
        Pass<T> P = make_pass(A, 0, PM_FINAL_OUT);
        P.x = s.u;
        P.nout = s.nout;
        P.nx = s.nx;
        for (int x = 0; x < kMaxExtra; ++x) P.X[x] = s.X[x];
        for (int j = 0; j < s.nout; ++j) {
            P.out[j] = s.out[j];
            P.cgF[j] = T(s.cg[j] + s.cF[j]);
            state_coefs<T>(s.cu[j], s.cx[j], P.cu[j], P.cx[j]);
        }
        if ((e = launch_pass_on<T, PM_FINAL_OUT>(P, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t multiplier_impl(const PeriodicArgs<T>& A, const Cplx<T>* M, const T* x, T* y, const T* base, double alpha,
                            cudaStream_t st) {
    if (!M || !x || !y) return cudaErrorInvalidValue;
    const int last = A.dim - 1;
    cudaError_t e;
    {
        Pass<T> P = make_pass(A, 0, PM_FWD_REAL);
        P.x = x;
        if ((e = launch_pass_on<T, PM_FWD_REAL>(P, st)) != cudaSuccess) return e;
    }
    Cplx<T>* c0[1] = {A.C[0]};
    if ((e = middle_passes(A, c0, 1, 0, st)) != cudaSuccess) return e;
    {
        Pass<T> P = make_pass(A, last, PM_PIVOT_MULT);
        P.M = M;
        if ((e = launch_pass_on<T, PM_PIVOT_MULT>(P, st)) != cudaSuccess) return e;
    }
    if ((e = middle_passes(A, c0, 1, 1, st)) != cudaSuccess) return e;
    {
        Pass<T> P = make_pass(A, 0, PM_FINAL_AXPY);
        P.y = y;
        P.base = base;
        P.alpha = T(alpha);
        if ((e = launch_pass_on<T, PM_FINAL_AXPY>(P, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One fused stage of a 2-D periodic context, kept in Fourier space from the state's transform to
// the stage's result: y = Re F^-1 (Mu (cu u^) + Mg (cgF (F(u) - pointwise)^ ... ) + cz Z), see
// PeriodicStage. Five launches: x1 forward of u | pivot: u^ and i k_mu u^ back | x1: fluxes and
// the pointwise part forward | pivot: the combination and its multipliers, back | x1 inverse.
template <typename T>
cudaError_t stage_impl(const PeriodicArgs<T>& A, const PeriodicStage<T>& s, cudaStream_t st) {
    if (A.dim != 2 || !s.x || !s.y || !A.CN || (s.Zs && !A.Cu)) return cudaErrorInvalidValue;
    cudaError_t e;
    if (!s.take_over) {      // otherwise the previous stage's last pass left F_1 x in Cu
        Pass<T> P = make_pass(A, 0, PM_FWD_REAL);
        P.x = s.x;
        P.C[0] = A.Cu;
        if ((e = launch_pass_on<T, PM_FWD_REAL>(P, st)) != cudaSuccess) return e;
    }
    {
        Pass<T> P = make_pass(A, 1, PM_PIVOT_DERIV);
        if ((e = launch_pass_on<T, PM_PIVOT_DERIV>(P, st)) != cudaSuccess) return e;
    }
    {
        Pass<T> P = make_pass(A, 0, PM_FLUX);
        P.x = s.x;
        P.nonflux = 1;
        P.CN = A.CN;
        if ((e = launch_pass_on<T, PM_FLUX>(P, st)) != cudaSuccess) return e;
    }
    {
        Pass<T> P = make_pass(A, 1, PM_PIVOT_STAGE);
        P.M = A.sym;
        P.CN = A.CN;
        P.Mu = s.Mu;
        P.Mg = s.Mg;
        P.Ms = s.Ms;
        P.Z = s.Z;
        P.Zs = s.Zs;
        P.scu = T(s.cu);
        P.scgF = T(s.cgF);
        P.scg = T(s.cg);
        P.scgz = T(s.cgz);
        P.scz = T(s.cz);
        P.szu = T(s.zu);
        P.szF = T(s.zF);
        P.szg = T(s.zg);
        if ((e = launch_pass_on<T, PM_PIVOT_STAGE>(P, st)) != cudaSuccess) return e;
    }
    if (s.hand_on) {
        Pass<T> P = make_pass(A, 0, PM_FINAL_FWD);
        P.y = s.y;
        if ((e = launch_pass_on<T, PM_FINAL_FWD>(P, st)) != cudaSuccess) return e;
    } else {
        Pass<T> P = make_pass(A, 0, PM_FINAL_AXPY);
        P.y = s.y;
        P.base = nullptr;
        if ((e = launch_pass_on<T, PM_FINAL_AXPY>(P, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

int periodic_stage_launches(int dim, bool take_over) { return dim == 2 ? (take_over ? 4 : 5) : 0; }
cudaError_t launch_periodic_stage(const PeriodicArgs<double>& P, const PeriodicStage<double>& s, cudaStream_t st) {
    return stage_impl(P, s, st);
}
cudaError_t launch_periodic_stage(const PeriodicArgs<float>& P, const PeriodicStage<float>& s, cudaStream_t st) {
    return stage_impl(P, s, st);
}

cudaError_t periodic_prepare(bool fp64) { return fp64 ? prepare_impl<double>() : prepare_impl<float>(); }

bool periodic_line_fits(int n, int axis, int dim, bool fp64) {
    const int mode = axis == dim - 1 ? PM_PIVOT_DIV : PM_PLAIN;   // the most buffers a pass on that axis uses
    const int pitch = axis == 0 ? n : n + 1;
    return pass_smem(n, 1, pitch, mode_buffers(mode), fp64 ? sizeof(Cplx<double>) : sizeof(Cplx<float>)) <=
           kPassSmemMax;
}

int periodic_rhs_launches(int dim, int nout) { (void)nout; return 5 + 4 * (dim - 2); }
int periodic_multiplier_launches(int dim) { return 3 + 2 * (dim - 2); }

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
