// K2 (SIMT): mu-mode contraction Y = X x_mu M on the FP64 / FP32 FMA pipes, with the
// pointwise phi_k scaling (K3) and the stage axpy (K4) fused into the epilogue.
//
// The mu-mode product of Section 1 (e^{A_d (+) ... (+) A_1} v = vec(V x_1 e^{A_1} ...
// x_d e^{A_d})) is a strided batched GEMM. Viewing the state as [P][n_mu][Q] (P the
// directions slower than mu, Q the faster ones):
//   mode 1 (Q = 1):  Y (P x n) = X (P x n) * M^T
//   mode mu > 1:     Y_p (n x Q) = M (n x n) * X_p (n x Q)   for each p
// The host passes element strides for A, B, C so one kernel serves every mode.
#include <cuda_runtime.h>

#include "adr_internal.h"
#include "phi_device.cuh"

namespace adr {
namespace {

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
contract_kernel(ContractArgs<T> p) {
    constexpr int NT = (BM / TM) * (BN / TN);
    constexpr int NX = BN / TN;   // threads along n
    constexpr int NY = BM / TM;   // threads along m
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];

    const int tid = threadIdx.x;
    const int tx = tid % NX, ty = tid / NX;
    const int b = blockIdx.z;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const T* A = p.A + (long long)b * p.sab;
    const T* B = p.B + (long long)b * p.sbb;
    const bool a_kfast = (p.sak == 1);
    const bool b_kfast = (p.sbk == 1);

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < p.K; k0 += BK) {
        // global -> shared, consecutive threads along the contiguous global index
        for (int e = tid; e < BM * BK; e += NT) {
            int mm, kk;
            if (a_kfast) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < p.M && gk < p.K) ? A[(long long)gm * p.sam + (long long)gk * p.sak] : T(0);
        }
        for (int e = tid; e < BN * BK; e += NT) {
            int nn, kk;
            if (b_kfast) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
            const int gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < p.N && gk < p.K) ? B[(long long)gk * p.sbk + (long long)gn * p.sbn] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T ra[TM], rb[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) ra[i] = As[kk][ty + i * NY];
#pragma unroll
            for (int j = 0; j < TN; ++j) rb[j] = Bs[kk][tx + j * NX];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(ra[i], rb[j], acc[i][j]);
        }
        __syncthreads();
    }

    // epilogue: the C offset is the element's linear index in the state array
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int gm = m0 + ty + i * NY;
        if (gm >= p.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int gn = n0 + tx + j * NX;
            if (gn >= p.N) continue;
            const long long off = (long long)b * p.scb + (long long)gm * p.scm + (long long)gn * p.scn;
            T v = acc[i][j];
            if (p.epi == EPI_PHI) {
                const int i1 = int(off % p.n1);
                const long long t = off / p.n1;
                const int i2 = int(t % p.n2);
                const int i3 = int(t / p.n2);
                double ls = p.lam[0][i1] + p.lam[1][i2];
                if (p.lam[2]) ls += p.lam[2][i3];
                v *= phi_eval(p.phik, T(p.ctau * ls));
            } else if (p.epi == EPI_AXPY) {
                v = p.base[off] + T(p.alpha) * v;
            }
            p.C[off] = v;
        }
    }
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
cudaError_t launch_tiled(const ContractArgs<T>& p, cudaStream_t s) {
    dim3 grid((p.N + BN - 1) / BN, (p.M + BM - 1) / BM, p.batch);
    if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
    contract_kernel<T, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(p);
    return cudaGetLastError();
}

int g_sms = 0;

// Output tiles of a bm x bn tiling of the pass.
template <typename T>
long long ctas(const ContractArgs<T>& p, int bm, int bn) {
    return (long long)((p.N + bn - 1) / bn) * ((p.M + bm - 1) / bm) * p.batch;
}

int sm_count() {
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

}  // namespace

// The largest tile that still gives every SM work: a small grid in one big tile would run on
// one SM (and mostly on padding), which the FP64 pipes of this GPU make very slow. Every
// output accumulates its K products in the same order for every tile shape.
cudaError_t launch_contract(const ContractArgs<double>& p, cudaStream_t s) {
    const long long want = 2LL * sm_count();
    if (ctas(p, 64, 64) >= want) return launch_tiled<double, 64, 64, 16, 4, 4>(p, s);
    if (ctas(p, 32, 32) >= want) return launch_tiled<double, 32, 32, 16, 2, 2>(p, s);
    if (ctas(p, 16, 16) >= want / 2) return launch_tiled<double, 16, 16, 16, 1, 1>(p, s);
    return launch_tiled<double, 8, 8, 16, 1, 1>(p, s);
}

cudaError_t launch_contract(const ContractArgs<float>& p, cudaStream_t s) {
    const long long want = 2LL * sm_count();
    if (ctas(p, 128, 128) >= want) return launch_tiled<float, 128, 128, 8, 8, 8>(p, s);
    if (ctas(p, 64, 64) >= want) return launch_tiled<float, 64, 64, 16, 4, 4>(p, s);
    if (ctas(p, 32, 32) >= want) return launch_tiled<float, 32, 32, 16, 2, 2>(p, s);
    return launch_tiled<float, 16, 16, 16, 1, 1>(p, s);
}

}  // namespace adr
