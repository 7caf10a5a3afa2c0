// Batched 2-D instances: one persistent launch per stage over every instance of a batch.
//
// K1 (batch_stencil_kernel): the stencil of stencil.cu (Eq. (adr), Eq. (nonlin), Section 3;
// centred differences, Section 5.2) with per-instance grid sizes and coefficients. A warp
// takes one row (i2) of one instance at a time, lanes along x1 (coalesced); the instance of
// a row comes from a binary search in the row prefix of the batch.
//
// K2 (batch_contract_kernel): the mu-mode products of Section 1 / Section 5.2 for every
// instance, as one list of output tiles. A work item names (instance, tile row, tile
// column, tile shape); the shapes 32x32, 64x64 and 128x128 share one 256-thread block and
// one shared-memory buffer, so items of different instances and shapes mix in one launch.
// Every output accumulates its K products in the same order whatever the tile shape, so the
// result does not depend on the shapes chosen. Epilogues as contract_simt.cu: store, the
// pointwise phi_k(tau (lambda_1 + lambda_2)) scaling (K3) or the stage axpy (K4).
#include <cuda_runtime.h>

#include <cstdint>

#include "adr_internal.h"
#include "phi_device.cuh"
#include "stencil_core.cuh"

namespace adr {
namespace {

// ------------------------------------------------------------------------------- stencil
template <typename T>
struct Combo {
    T cu[kMaxOut], cx[kMaxOut][kMaxExtra], cg[kMaxOut], cF[kMaxOut];
};

__device__ __forceinline__ int find_instance(const long long* row_start, int ninst, long long r) {
    int lo = 0, hi = ninst - 1;      // largest i with row_start[i] <= r
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(row_start + mid) <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(256) batch_stencil_kernel(BatchStencilArgs<T> p, Combo<T> cb, bool needF) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < p.rows; r += warps) {
        const int ii = find_instance(p.row_start, p.ninst, r);
        const BatchInst<T>& in = p.inst[ii];
        const int n1 = in.n1, n2 = in.n2;
        const int i2 = int(r - in.row0);
        Coefs<T> c;
        c.ih2[0] = in.ih2[0]; c.ih2[1] = in.ih2[1]; c.ih2[2] = T(0);
        c.i2h[0] = in.i2h[0]; c.i2h[1] = in.i2h[1]; c.i2h[2] = T(0);
        c.bmb[0] = in.bmb[0]; c.bmb[1] = in.bmb[1]; c.bmb[2] = T(0);
        c.beta[0] = in.beta[0]; c.beta[1] = in.beta[1]; c.beta[2] = T(0);
        c.abar = in.abar;
        c.r0 = in.r[0]; c.r1 = in.r[1]; c.r2 = in.r[2]; c.r3 = in.r[3];
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j) {
            c.cu[j] = cb.cu[j]; c.cg[j] = cb.cg[j]; c.cF[j] = cb.cF[j];
#pragma unroll
            for (int e = 0; e < kMaxExtra; ++e) c.cx[j][e] = cb.cx[j][e];
        }
        const T* u = p.u + in.off + (long long)i2 * n1;
        const T* a = p.a + in.a_off + (long long)(i2 + 1) * in.apitch + 4;   // interior i1 = 0
        const long long row = in.off + (long long)i2 * n1;
        for (int i1 = lane; i1 < n1; i1 += 32) {
            const T u0 = __ldg(u + i1);
            const T uw = i1 > 0 ? __ldg(u + i1 - 1) : T(0);
            const T ue = i1 + 1 < n1 ? __ldg(u + i1 + 1) : T(0);
            const T us = i2 > 0 ? __ldg(u + i1 - n1) : T(0);
            const T un = i2 + 1 < n2 ? __ldg(u + i1 + n1) : T(0);
            const T a0 = __ldg(a + i1);            // the boundary ring makes the four neighbours valid
            const T aw = __ldg(a + i1 - 1), ae = __ldg(a + i1 + 1);
            const T as = __ldg(a + i1 - in.apitch), an = __ldg(a + i1 + in.apitch);
            T F = T(0);
            const T g = stencil_core<T, 2>(c, u0, ue - u0, u0 - uw, un - u0, u0 - us, T(0), T(0), a0 + ae, a0 + aw,
                                           a0 + an, a0 + as, T(0), T(0), needF, F);
#pragma unroll
            for (int j = 0; j < kMaxOut; ++j) {
                if (j < p.nout) {
                    T v = c.cu[j] * u0 + c.cg[j] * g + c.cF[j] * F;
#pragma unroll
                    for (int e = 0; e < kMaxExtra; ++e)
                        if (e < p.nx) v += c.cx[j][e] * __ldg(p.X[e] + row + i1);
                    p.out[j][row + i1] = v;
                }
            }
        }
    }
}

// --------------------------------------------------------------------------- contraction
constexpr int kThreads = 256;
constexpr int kBK = 16;
constexpr int kMaxEdge = 128;

template <typename T>
struct TileSmem {
    T A[kBK][kMaxEdge + 1];
    T B[kBK][kMaxEdge + 1];
};

// The phi factor of one output, kept out of line: the series branch would otherwise take
// registers from the accumulator tile of every shape.
template <typename T>
__device__ __noinline__ T phi_factor(int k, double z) { return phi_eval(k, T(z)); }

// One BM x BN output tile of C = A B (K = the contracted extent) with the fused epilogue.
// A(m, k) = A[m * sam + k] (k contiguous in both modes); B(k, n) = B[k * sbk + n * sbn].
template <typename T, int BM, int BN>
__device__ __forceinline__ void tile_gemm(TileSmem<T>& sm, const T* __restrict__ A, long long sam, const T* __restrict__ B,
                                          long long sbk, long long sbn, int M, int N, int K, int m0, int n0,
                                          const BatchContractArgs<T>& p, const BatchInst<T>& in) {
    constexpr int TM = BM / 16, TN = BN / 16;    // 16 x 16 threads
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const bool b_kfast = (sbk == 1);
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < K; k0 += kBK) {
        for (int e = tid; e < BM * kBK; e += kThreads) {
            const int kk = e % kBK, mm = e / kBK;
            const int gm = m0 + mm, gk = k0 + kk;
            sm.A[kk][mm] = (gm < M && gk < K) ? __ldg(A + (long long)gm * sam + gk) : T(0);
        }
        for (int e = tid; e < BN * kBK; e += kThreads) {
            int nn, kk;
            if (b_kfast) { kk = e % kBK; nn = e / kBK; } else { nn = e % BN; kk = e / BN; }
            const int gn = n0 + nn, gk = k0 + kk;
            sm.B[kk][nn] = (gn < N && gk < K) ? __ldg(B + (long long)gk * sbk + (long long)gn * sbn) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            T ra[TM], rb[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) ra[i] = sm.A[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) rb[j] = sm.B[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(ra[i], rb[j], acc[i][j]);
        }
        __syncthreads();
    }

    // C(m, n) is node (i1 = n, i2 = m) of the instance in both modes
    const double* l1 = (p.epi == EPI_PHI) ? p.lam + in.lam_off[0] : nullptr;
    const double* l2 = (p.epi == EPI_PHI) ? p.lam + in.lam_off[1] : nullptr;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            const long long off = in.off + (long long)gm * in.n1 + gn;
            T v = acc[i][j];
            if (p.epi == EPI_PHI) {
                v *= phi_factor<T>(p.phik, p.tau * (__ldg(l1 + gn) + __ldg(l2 + gm)));
            } else if (p.epi == EPI_AXPY) {
                v = __ldg(p.base + off) + T(p.alpha) * v;
            }
            p.Y[off] = v;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 2 : 1) batch_contract_kernel(BatchContractArgs<T> p) {
    __shared__ TileSmem<T> sm;
    for (int it = blockIdx.x; it < p.nitems; it += gridDim.x) {
        const int4 item = __ldg(p.items + it);
        const BatchInst<T>& in = p.inst[item.x];
        const int n1 = in.n1, n2 = in.n2;
        const T* F = p.factors + in.f_off[p.role][p.mode - 1];
        const T* X = p.X + in.off;
        const int edge = item.w == BT_32 ? 32 : item.w == BT_64 ? 64 : 128;
        const int m0 = item.y * edge, n0 = item.z * edge;
        // mode 1: C (n2 x n1) = X (n2 x n1) * M1^T, K = n1; mode 2: C = M2 (n2 x n2) * X, K = n2
        const T* A = p.mode == 1 ? X : F;
        const long long sam = p.mode == 1 ? n1 : n2;
        const T* B = p.mode == 1 ? F : X;
        const long long sbk = p.mode == 1 ? 1 : n1;
        const long long sbn = p.mode == 1 ? n1 : 1;
        const int K = p.mode == 1 ? n1 : n2;
        if (item.w == BT_32)      tile_gemm<T, 32, 32>(sm, A, sam, B, sbk, sbn, n2, n1, K, m0, n0, p, in);
        else if (item.w == BT_64) tile_gemm<T, 64, 64>(sm, A, sam, B, sbk, sbn, n2, n1, K, m0, n0, p, in);
        else                      tile_gemm<T, 128, 128>(sm, A, sam, B, sbk, sbn, n2, n1, K, m0, n0, p, in);
    }
}

int g_sms = 0;

int sm_count() {
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

template <typename T>
cudaError_t stencil_launch(const BatchStencilArgs<T>& p, cudaStream_t s) {
    if (p.rows <= 0) return cudaSuccess;
    if (!p.inst || !p.row_start || !p.a || !p.u || p.nout < 1 || p.nout > kMaxOut || p.nx < 0 || p.nx > kMaxExtra)
        return cudaErrorInvalidValue;
    Combo<T> cb;
    bool needF = false;
    for (int j = 0; j < kMaxOut; ++j) {
        cb.cu[j] = T(p.cu[j]); cb.cg[j] = T(p.cg[j]); cb.cF[j] = T(p.cF[j]);
        for (int e = 0; e < kMaxExtra; ++e) cb.cx[j][e] = T(p.cx[j][e]);
        if (j < p.nout && p.cF[j] != 0.0) needF = true;
    }
    const long long want = (p.rows + 7) / 8;                 // 8 warps (rows) per block
    long long grid = p.grid > 0 ? p.grid : 8LL * sm_count();
    if (grid > want) grid = want;
    batch_stencil_kernel<T><<<unsigned(grid), 256, 0, s>>>(p, cb, needF);
    return cudaGetLastError();
}

template <typename T>
cudaError_t contract_launch(const BatchContractArgs<T>& p, cudaStream_t s) {
    if (p.nitems <= 0) return cudaSuccess;
    if (!p.inst || !p.items || !p.factors || !p.X || !p.Y || (p.mode != 1 && p.mode != 2)) return cudaErrorInvalidValue;
    if (p.role < 0 || p.role > BR_VINV) return cudaErrorInvalidValue;
    if (p.epi == EPI_PHI && !p.lam) return cudaErrorInvalidValue;
    if (p.epi == EPI_AXPY && !p.base) return cudaErrorInvalidValue;
    long long grid = p.grid > 0 ? p.grid : 2LL * sm_count();
    if (grid > p.nitems) grid = p.nitems;
    batch_contract_kernel<T><<<unsigned(grid), kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_stencil(const BatchStencilArgs<double>& a, cudaStream_t s) { return stencil_launch(a, s); }
cudaError_t launch_batch_stencil(const BatchStencilArgs<float>& a, cudaStream_t s) { return stencil_launch(a, s); }
cudaError_t launch_batch_contract(const BatchContractArgs<double>& a, cudaStream_t s) { return contract_launch(a, s); }
cudaError_t launch_batch_contract(const BatchContractArgs<float>& a, cudaStream_t s) { return contract_launch(a, s); }

}  // namespace adr
