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

// ------------------------------------------------------------- compensated stencil (mixed)
// Coefficients of the stage combination as double-float pairs (hi, lo) of the host's doubles.
struct Combo2 {
    float cu[kMaxOut][2], cx[kMaxOut][kMaxExtra][2], cg[kMaxOut][2], cF[kMaxOut][2];
};

__device__ __forceinline__ void two_sum2(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// acc (hi, lo) += (ch + cl) (xh + xl), in double-float arithmetic
__device__ __forceinline__ void df_fma(float ch, float cl, float xh, float xl, float& hi, float& lo) {
    const float p = ch * xh;
    float e = fmaf(ch, xh, -p);
    e = fmaf(ch, xl, fmaf(cl, xh, e));
    float s, t;
    two_sum2(hi, p, s, t);
    t += lo + e;
    hi = s + t;
    lo = t - (hi - s);
}

// The stencil of batch_stencil_kernel on a compensated state u + u_lo: each one-sided
// difference is formed from both parts, (u_E - u_C) + (lo_E - lo_C), so that FP32 rounding of
// the state does not enter through the 1/h^2 of the stencil; the differences, coefficients and
// reaction are then FP32 as in the plain kernel. The stage combination is formed in
// double-float arithmetic (inputs with their low parts); an output with a low-part array gets
// both parts, one without gets their FP32 sum. Per output the maximum |out| of each instance is
// recorded (one atomic per row).
__global__ void __launch_bounds__(256) batch_stencil2_kernel(BatchStencil2Args P, Combo<float> cb, Combo2 c2, bool needF) {
    const BatchStencilArgs<float>& p = P.s;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < p.rows; r += warps) {
        const int ii = find_instance(p.row_start, p.ninst, r);
        const BatchInst<float>& in = p.inst[ii];
        const int n1 = in.n1, n2 = in.n2;
        const int i2 = int(r - in.row0);
        Coefs<float> c;
        c.ih2[0] = in.ih2[0]; c.ih2[1] = in.ih2[1]; c.ih2[2] = 0.f;
        c.i2h[0] = in.i2h[0]; c.i2h[1] = in.i2h[1]; c.i2h[2] = 0.f;
        c.bmb[0] = in.bmb[0]; c.bmb[1] = in.bmb[1]; c.bmb[2] = 0.f;
        c.beta[0] = in.beta[0]; c.beta[1] = in.beta[1]; c.beta[2] = 0.f;
        c.abar = in.abar;
        c.r0 = in.r[0]; c.r1 = in.r[1]; c.r2 = in.r[2]; c.r3 = in.r[3];
        const long long row = in.off + (long long)i2 * n1;
        const float* u = p.u + row;
        const float* ul = P.u_lo ? P.u_lo + row : nullptr;
        const float* a = p.a + in.a_off + (long long)(i2 + 1) * in.apitch + 4;   // interior i1 = 0
        float vmax[kMaxOut] = {0.f, 0.f};
        for (int i1 = lane; i1 < n1; i1 += 32) {
            auto ld = [&](const float* base, int di1, int di2, bool inside) -> float {
                return inside ? __ldg(base + di1 + (long long)di2 * n1) : 0.f;
            };
            const bool hw = i1 > 0, he = i1 + 1 < n1, hs = i2 > 0, hn = i2 + 1 < n2;
            const float u0 = __ldg(u + i1);
            const float uw = ld(u + i1, -1, 0, hw), ue = ld(u + i1, 1, 0, he);
            const float us = ld(u + i1, 0, -1, hs), un = ld(u + i1, 0, 1, hn);
            float l0 = 0.f, lw = 0.f, le = 0.f, ls = 0.f, ln = 0.f;
            if (ul) {
                l0 = __ldg(ul + i1);
                lw = ld(ul + i1, -1, 0, hw); le = ld(ul + i1, 1, 0, he);
                ls = ld(ul + i1, 0, -1, hs); ln = ld(ul + i1, 0, 1, hn);
            }
            const float dE = (ue - u0) + (le - l0), dW = (u0 - uw) + (l0 - lw);
            const float dN = (un - u0) + (ln - l0), dS = (u0 - us) + (l0 - ls);
            const float a0 = __ldg(a + i1);
            const float aw = __ldg(a + i1 - 1), ae = __ldg(a + i1 + 1);
            const float as = __ldg(a + i1 - in.apitch), an = __ldg(a + i1 + in.apitch);
            float F = 0.f;
            const float g = stencil_core<float, 2>(c, u0 + l0, dE, dW, dN, dS, 0.f, 0.f, a0 + ae, a0 + aw, a0 + an, a0 + as,
                                                   0.f, 0.f, needF, F);
#pragma unroll
            for (int j = 0; j < kMaxOut; ++j) {
                if (j >= p.nout) continue;
                float hi = 0.f, lo = 0.f;
                if (cb.cu[j] != 0.f) df_fma(c2.cu[j][0], c2.cu[j][1], u0, l0, hi, lo);
#pragma unroll
                for (int e = 0; e < kMaxExtra; ++e)
                    if (e < p.nx && cb.cx[j][e] != 0.f) {
                        const float xh = __ldg(p.X[e] + row + i1);
                        const float xl = P.X_lo[e] ? __ldg(P.X_lo[e] + row + i1) : 0.f;
                        df_fma(c2.cx[j][e][0], c2.cx[j][e][1], xh, xl, hi, lo);
                    }
                if (cb.cg[j] != 0.f) df_fma(c2.cg[j][0], c2.cg[j][1], g, 0.f, hi, lo);
                if (cb.cF[j] != 0.f) df_fma(c2.cF[j][0], c2.cF[j][1], F, 0.f, hi, lo);
                if (P.out_lo[j]) {
                    p.out[j][row + i1] = hi;
                    P.out_lo[j][row + i1] = lo;
                } else {
                    hi = hi + lo;
                    p.out[j][row + i1] = hi;
                }
                if (P.out_hs[j]) P.out_hs[j][row + i1] = hi;
                vmax[j] = fmaxf(vmax[j], fabsf(hi));
            }
        }
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j) {
            if (j >= p.nout || !P.amax[j]) continue;
            float m = vmax[j];
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0 && m > 0.f) atomicMax(P.amax[j] + ii, __float_as_uint(m));
        }
    }
}

// The same node arithmetic as batch_stencil2_kernel, marching: a warp takes 32 consecutive x1
// nodes of one instance (a unit {instance, x1 start, first row, rows}) and walks down its rows,
// keeping the rows above, at and below the current one of u, its low part and (a - abar) in
// registers; the x1 neighbours come from the adjacent lanes, the two at the ends of the strip
// from memory. Each input element is read once per strip instead of five times.
__global__ void __launch_bounds__(256) batch_stencil2_march_kernel(BatchStencil2Args P, const int4* __restrict__ units,
                                                                   int nunits, Combo<float> cb, Combo2 c2, bool needF) {
    const BatchStencilArgs<float>& p = P.s;
    const int lane = threadIdx.x & 31;
    const int warps = int(gridDim.x) * int(blockDim.x >> 5);
    for (int w = int(blockIdx.x) * int(blockDim.x >> 5) + int(threadIdx.x >> 5); w < nunits; w += warps) {
        const int4 un = __ldg(units + w);
        const BatchInst<float>& in = p.inst[un.x];
        const int n1 = in.n1, n2 = in.n2, ap = in.apitch;
        const int i1 = un.y + lane;
        const bool valid = i1 < n1;
        Coefs<float> c;
        c.ih2[0] = in.ih2[0]; c.ih2[1] = in.ih2[1]; c.ih2[2] = 0.f;
        c.i2h[0] = in.i2h[0]; c.i2h[1] = in.i2h[1]; c.i2h[2] = 0.f;
        c.bmb[0] = in.bmb[0]; c.bmb[1] = in.bmb[1]; c.bmb[2] = 0.f;
        c.beta[0] = in.beta[0]; c.beta[1] = in.beta[1]; c.beta[2] = 0.f;
        c.abar = in.abar;
        c.r0 = in.r[0]; c.r1 = in.r[1]; c.r2 = in.r[2]; c.r3 = in.r[3];
        const float* ub = p.u + in.off;
        const float* lb = P.u_lo ? P.u_lo + in.off : nullptr;
        const float* ab = p.a + in.a_off + 4;          // (a - abar) at interior i1 = 0 of ring row 0
        // value of row r (-1..n2) at this lane's node: zero outside the grid (Dirichlet ghosts)
        auto ldu = [&](const float* base, int r) -> float {
            return (base && valid && r >= 0 && r < n2) ? __ldg(base + (long long)r * n1 + i1) : 0.f;
        };
        auto lda = [&](int r) -> float {            // ring rows -1..n2 exist for every node i1 in 0..n1-1
            return valid ? __ldg(ab + (long long)(r + 1) * ap + i1) : 0.f;
        };
        const int r0 = un.z, r1 = un.z + un.w;
        float um = ldu(ub, r0 - 1), uc = ldu(ub, r0);
        float lm = ldu(lb, r0 - 1), lc = ldu(lb, r0);
        float am = lda(r0 - 1), ac = lda(r0);
        float vmax[kMaxOut] = {0.f, 0.f};
        for (int r = r0; r < r1; ++r) {
            const float up = ldu(ub, r + 1), lp = ldu(lb, r + 1), apl = lda(r + 1);
            // x1 neighbours: adjacent lanes, and memory at the two ends of the strip
            float uw = __shfl_up_sync(0xffffffffu, uc, 1), ue = __shfl_down_sync(0xffffffffu, uc, 1);
            float lw = __shfl_up_sync(0xffffffffu, lc, 1), le = __shfl_down_sync(0xffffffffu, lc, 1);
            float aw = __shfl_up_sync(0xffffffffu, ac, 1), ae = __shfl_down_sync(0xffffffffu, ac, 1);
            const long long rowoff = (long long)r * n1;
            const float* arow = ab + (long long)(r + 1) * ap;
            if (lane == 0 && valid) {
                uw = i1 > 0 ? __ldg(ub + rowoff + i1 - 1) : 0.f;
                lw = (lb && i1 > 0) ? __ldg(lb + rowoff + i1 - 1) : 0.f;
                aw = __ldg(arow + i1 - 1);           // the ring column at i1 = -1 exists
            }
            if (valid && (lane == 31 || i1 + 1 >= n1)) {
                ue = i1 + 1 < n1 ? __ldg(ub + rowoff + i1 + 1) : 0.f;
                le = (lb && i1 + 1 < n1) ? __ldg(lb + rowoff + i1 + 1) : 0.f;
                ae = __ldg(arow + i1 + 1);           // the ring column at i1 = n1 exists
            }
            if (valid) {
                const float dE = (ue - uc) + (le - lc), dW = (uc - uw) + (lc - lw);
                const float dN = (up - uc) + (lp - lc), dS = (uc - um) + (lc - lm);
                float F = 0.f;
                const float g = stencil_core<float, 2>(c, uc + lc, dE, dW, dN, dS, 0.f, 0.f, ac + ae, ac + aw, ac + apl,
                                                       ac + am, 0.f, 0.f, needF, F);
                const long long o = in.off + rowoff + i1;
#pragma unroll
                for (int j = 0; j < kMaxOut; ++j) {
                    if (j >= p.nout) continue;
                    float hi = 0.f, lo = 0.f;
                    if (cb.cu[j] != 0.f) df_fma(c2.cu[j][0], c2.cu[j][1], uc, lc, hi, lo);
#pragma unroll
                    for (int e = 0; e < kMaxExtra; ++e)
                        if (e < p.nx && cb.cx[j][e] != 0.f) {
                            const float xh = __ldg(p.X[e] + o);
                            const float xl = P.X_lo[e] ? __ldg(P.X_lo[e] + o) : 0.f;
                            df_fma(c2.cx[j][e][0], c2.cx[j][e][1], xh, xl, hi, lo);
                        }
                    if (cb.cg[j] != 0.f) df_fma(c2.cg[j][0], c2.cg[j][1], g, 0.f, hi, lo);
                    if (cb.cF[j] != 0.f) df_fma(c2.cF[j][0], c2.cF[j][1], F, 0.f, hi, lo);
                    if (P.out_lo[j]) {
                        p.out[j][o] = hi;
                        P.out_lo[j][o] = lo;
                    } else {
                        hi = hi + lo;
                        p.out[j][o] = hi;
                    }
                    if (P.out_hs[j]) P.out_hs[j][o] = hi;
                    vmax[j] = fmaxf(vmax[j], fabsf(hi));
                }
            }
            um = uc; uc = up;
            lm = lc; lc = lp;
            am = ac; ac = apl;
        }
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j) {
            if (j >= p.nout || !P.amax[j]) continue;
            float m = vmax[j];
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0 && m > 0.f) atomicMax(P.amax[j] + un.x, __float_as_uint(m));
        }
    }
}

// --------------------------------------------------------------------------- contraction
constexpr int kThreads = 256;      // 16 x 16 threads per tile of every shape
constexpr int kBK = 16;            // K per shared-memory stage
constexpr int kPad = 4;            // row padding: keeps 16-byte alignment of 4-wide groups
constexpr int kMaxEdge = 128;

template <typename T>
struct TileSmem {
    alignas(16) T A[kBK][kMaxEdge + kPad];   // A^T slice: [k][m]
    alignas(16) T B[kBK][kMaxEdge + kPad];   // B slice:   [k][n]
};

// G consecutive values from shared or global memory (16-byte aligned when G * sizeof(T) >= 16).
template <int G>
__device__ __forceinline__ void ld_group(const float* p, float (&r)[G]) {
    if constexpr (G == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    } else if constexpr (G == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        r[0] = v.x; r[1] = v.y;
    } else {
        r[0] = p[0];
    }
}
template <int G>
__device__ __forceinline__ void ld_group(const double* p, double (&r)[G]) {
    if constexpr (G >= 2) {
#pragma unroll
        for (int h = 0; h < G / 2; ++h) {
            const double2 v = reinterpret_cast<const double2*>(p)[h];
            r[2 * h] = v.x; r[2 * h + 1] = v.y;
        }
    } else {
        r[0] = p[0];
    }
}
__device__ __forceinline__ void st4(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double* v) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void ldg4(const float* p, float* v) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void ldg4(const double* p, double* v) {
    const double2 x = __ldg(reinterpret_cast<const double2*>(p)), y = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

// One kBK-deep slice of an operand tile of edge E, staged through E/16 registers per
// thread. Element (e, k) of the operand (e the row of A or the column of B) sits at
// P[e * s + k] when KFAST (k contiguous), else at P[k * s + e]. VEC: 16-byte loads of 4
// elements along the contiguous index (every row start and extent a multiple of 4).
template <typename T, int E, bool KFAST, bool VEC>
struct Slice {
    static constexpr int R = E / 16;
    T v[R];

    __device__ __forceinline__ void load(const T* __restrict__ P, long long s, int e0, int k0, int Ne, int K) {
        const int tid = threadIdx.x;
        if constexpr (VEC) {
#pragma unroll
            for (int q = 0; q < R / 4; ++q) {
                const int c = tid + kThreads * q;
                const int e = KFAST ? c / (kBK / 4) : (c % (E / 4)) * 4;
                const int k = KFAST ? (c % (kBK / 4)) * 4 : c / (E / 4);
                const int ge = e0 + e, gk = k0 + k;
                if (ge < Ne && gk < K) ldg4(KFAST ? P + (long long)ge * s + gk : P + (long long)gk * s + ge, v + 4 * q);
                else v[4 * q] = v[4 * q + 1] = v[4 * q + 2] = v[4 * q + 3] = T(0);
            }
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int c = tid + kThreads * q;
                const int e = KFAST ? c / kBK : c % E;
                const int k = KFAST ? c % kBK : c / E;
                const int ge = e0 + e, gk = k0 + k;
                v[q] = (ge < Ne && gk < K) ? __ldg(KFAST ? P + (long long)ge * s + gk : P + (long long)gk * s + ge) : T(0);
            }
        }
    }

    __device__ __forceinline__ void store(T (*S)[kMaxEdge + kPad]) const {
        const int tid = threadIdx.x;
        if constexpr (VEC) {
#pragma unroll
            for (int q = 0; q < R / 4; ++q) {
                const int c = tid + kThreads * q;
                if constexpr (KFAST) {
                    const int e = c / (kBK / 4), k = (c % (kBK / 4)) * 4;
#pragma unroll
                    for (int j = 0; j < 4; ++j) S[k + j][e] = v[4 * q + j];
                } else {
                    const int e = (c % (E / 4)) * 4, k = c / (E / 4);
                    st4(&S[k][e], v + 4 * q);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int c = tid + kThreads * q;
                const int e = KFAST ? c / kBK : c % E;
                const int k = KFAST ? c % kBK : c / E;
                S[k][e] = v[q];
            }
        }
    }
};

// The phi factor of one output, kept out of line: the series branch would otherwise take
// registers from the accumulator tile of every shape.
template <typename T>
__device__ __noinline__ T phi_factor(int k, T z) { return phi_eval(k, z); }

// One E x E output tile of C = A B (K = the contracted extent) with the fused epilogue.
// A(m, k) = A[m * sam + k]; B(k, n) = B[n * sb + k] in mode 1 (the factor, k contiguous)
// and B[k * sb + n] in mode 2 (the state, n contiguous). A thread owns TM x TM outputs in
// groups of G consecutive rows and columns: row (i / G) * 16G + ty G + i % G.
template <typename T, int E, int MODE, bool VEC>
__device__ __forceinline__ void tile_gemm(TileSmem<T>& sm, const T* __restrict__ A, long long sam,
                                          const T* __restrict__ B, long long sb, int M, int N, int K, int m0, int n0,
                                          const BatchContractArgs<T>& p, const BatchInst<T>& in) {
    constexpr int TM = E / 16;
    constexpr int G = TM < 4 ? TM : 4;
    constexpr int H = TM / G;
    constexpr bool VA = VEC && E >= 64;          // vector staging needs E/16 >= 4 registers
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = T(0);

    Slice<T, E, true, VA> sa;
    Slice<T, E, MODE == 1, VA> sbl;
    sa.load(A, sam, m0, 0, M, K);
    sbl.load(B, sb, n0, 0, N, K);
    for (int k0 = 0; k0 < K; k0 += kBK) {
        sa.store(sm.A);
        sbl.store(sm.B);
        __syncthreads();
        if (k0 + kBK < K) {                      // the next slice is in flight during the FMAs
            sa.load(A, sam, m0, k0 + kBK, M, K);
            sbl.load(B, sb, n0, k0 + kBK, N, K);
        }
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            T ra[TM], rb[TM];
#pragma unroll
            for (int h = 0; h < H; ++h) {
                T ga[G], gb[G];
                ld_group<G>(&sm.A[kk][h * 16 * G + ty * G], ga);
                ld_group<G>(&sm.B[kk][h * 16 * G + tx * G], gb);
#pragma unroll
                for (int g = 0; g < G; ++g) { ra[h * G + g] = ga[g]; rb[h * G + g] = gb[g]; }
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TM; ++j) acc[i][j] = fma(ra[i], rb[j], acc[i][j]);
        }
        __syncthreads();
    }

    // C(m, n) is node (i1 = n, i2 = m) of the instance in both modes
    const T* z1 = (MODE == 2 && p.epi == EPI_PHI) ? p.zt + in.zt_off[0] : nullptr;
    const T* z2 = (MODE == 2 && p.epi == EPI_PHI) ? p.zt + in.zt_off[1] : nullptr;
    constexpr bool VOUT = (G == 4);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int gm = m0 + (i / G) * 16 * G + ty * G + (i % G);
        if (gm >= M) continue;
        const long long row = in.off + (long long)gm * in.n1;
        const T zr = (MODE == 2 && p.epi == EPI_PHI) ? __ldg(z2 + gm) : T(0);
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int gn0 = n0 + h * 16 * G + tx * G;
            if (gn0 >= N) continue;
            T v[G];
#pragma unroll
            for (int g = 0; g < G; ++g) v[g] = acc[i][h * G + g];
            const bool full = VOUT && VEC && p.aligned && (gn0 + G <= N);
            if (MODE == 2 && p.epi == EPI_PHI) {      // the last forward pass of a 2-D phi action
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (gn0 + g < N) v[g] *= phi_factor<T>(p.phik, zr + __ldg(z1 + gn0 + g));
            } else if (p.epi == EPI_AXPY) {
                T bv[G];
                if constexpr (VOUT) {
                    if (full) ldg4(p.base + row + gn0, bv);
                    else
#pragma unroll
                        for (int g = 0; g < G; ++g) bv[g] = gn0 + g < N ? __ldg(p.base + row + gn0 + g) : T(0);
                } else {
#pragma unroll
                    for (int g = 0; g < G; ++g) bv[g] = gn0 + g < N ? __ldg(p.base + row + gn0 + g) : T(0);
                }
#pragma unroll
                for (int g = 0; g < G; ++g) v[g] = bv[g] + T(p.alpha) * v[g];
            }
            if constexpr (VOUT) {
                if (full) { st4(p.Y + row + gn0, v); continue; }
            }
#pragma unroll
            for (int g = 0; g < G; ++g)
                if (gn0 + g < N) p.Y[row + gn0 + g] = v[g];
        }
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 2 : 1) batch_contract_kernel(BatchContractArgs<T> p) {
    __shared__ TileSmem<T> sm;
    for (int it = blockIdx.x; it < p.nitems; it += gridDim.x) {
        const int4 item = __ldg(p.items + it);
        const BatchInst<T>& in = p.inst[item.x];
        const int n1 = in.n1, n2 = in.n2;
        const T* F = p.factors + in.f_off[p.role][MODE - 1];
        const T* X = p.X + in.off;
        const int edge = item.w == BT_32 ? 32 : item.w == BT_64 ? 64 : 128;
        const int m0 = item.y * edge, n0 = item.z * edge;
        // mode 1: C (n2 x n1) = X (n2 x n1) * M1^T, K = n1; mode 2: C = M2 (n2 x n2) * X, K = n2
        const T* A = MODE == 1 ? X : F;
        const long long sam = MODE == 1 ? n1 : n2;
        const T* B = MODE == 1 ? F : X;
        const long long sb = n1;
        const int K = MODE == 1 ? n1 : n2;
        const bool vec = in.vec && p.aligned;
        if (item.w == BT_32) {
            tile_gemm<T, 32, MODE, false>(sm, A, sam, B, sb, n2, n1, K, m0, n0, p, in);
        } else if (item.w == BT_64) {
            if (vec) tile_gemm<T, 64, MODE, true>(sm, A, sam, B, sb, n2, n1, K, m0, n0, p, in);
            else     tile_gemm<T, 64, MODE, false>(sm, A, sam, B, sb, n2, n1, K, m0, n0, p, in);
        } else {
            if (vec) tile_gemm<T, 128, MODE, true>(sm, A, sam, B, sb, n2, n1, K, m0, n0, p, in);
            else     tile_gemm<T, 128, MODE, false>(sm, A, sam, B, sb, n2, n1, K, m0, n0, p, in);
        }
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
        cb.cg[j] = T(p.cg[j]); cb.cF[j] = T(p.cF[j]);
        state_coefs<T>(p.cu[j], p.cx[j], cb.cu[j], cb.cx[j]);
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
    if (p.role < 0 || p.role >= kBatchRoles) return cudaErrorInvalidValue;
    if (p.epi == EPI_PHI && (!p.zt || p.mode != 2)) return cudaErrorInvalidValue;
    if (p.epi == EPI_AXPY && !p.base) return cudaErrorInvalidValue;
    long long grid = p.grid > 0 ? p.grid : 2LL * sm_count();
    if (grid > p.nitems) grid = p.nitems;
    if (p.mode == 1) batch_contract_kernel<T, 1><<<unsigned(grid), kThreads, 0, s>>>(p);
    else             batch_contract_kernel<T, 2><<<unsigned(grid), kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t stencil2_launch(const BatchStencil2Args& P, cudaStream_t s) {
    const BatchStencilArgs<float>& p = P.s;
    if (p.rows <= 0) return cudaSuccess;
    if (!p.inst || !p.row_start || !p.a || !p.u || p.nout < 1 || p.nout > kMaxOut || p.nx < 0 || p.nx > kMaxExtra)
        return cudaErrorInvalidValue;
    Combo<float> cb;
    Combo2 c2;
    bool needF = false;
    auto split = [](double v, float (&o)[2]) {
        o[0] = float(v);
        o[1] = float(v - double(o[0]));
    };
    for (int j = 0; j < kMaxOut; ++j) {
        cb.cu[j] = float(p.cu[j]); cb.cg[j] = float(p.cg[j]); cb.cF[j] = float(p.cF[j]);
        split(p.cu[j], c2.cu[j]); split(p.cg[j], c2.cg[j]); split(p.cF[j], c2.cF[j]);
        for (int e = 0; e < kMaxExtra; ++e) {
            cb.cx[j][e] = float(p.cx[j][e]);
            split(p.cx[j][e], c2.cx[j][e]);
        }
        if (j < p.nout && p.cF[j] != 0.0) needF = true;
    }
    if (P.units && P.nunits > 0) {   // the marching form over {instance, x1 start, first row, rows} units
        long long grid = (P.nunits + 7) / 8;
        const long long cap = 16LL * sm_count();
        if (grid > cap) grid = cap;
        batch_stencil2_march_kernel<<<unsigned(grid), 256, 0, s>>>(P, P.units, P.nunits, cb, c2, needF);
        return cudaGetLastError();
    }
    const long long want = (p.rows + 7) / 8;
    long long grid = p.grid > 0 ? p.grid : 8LL * sm_count();
    if (grid > want) grid = want;
    batch_stencil2_kernel<<<unsigned(grid), 256, 0, s>>>(P, cb, c2, needF);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_stencil(const BatchStencilArgs<double>& a, cudaStream_t s) { return stencil_launch(a, s); }
cudaError_t launch_batch_stencil(const BatchStencilArgs<float>& a, cudaStream_t s) { return stencil_launch(a, s); }
cudaError_t launch_batch_contract(const BatchContractArgs<double>& a, cudaStream_t s) { return contract_launch(a, s); }
cudaError_t launch_batch_contract(const BatchContractArgs<float>& a, cudaStream_t s) { return contract_launch(a, s); }
cudaError_t launch_batch_stencil2(const BatchStencil2Args& a, cudaStream_t s) { return stencil2_launch(a, s); }

}  // namespace adr
