// K1: variable-coefficient 5/7-point stencil for F(u) and g(u) = F(u) - A u with a fused
// stage-combination epilogue.
//
// Discretisation (Eq. (adr) and Eq. (nonlin), Section 3; centred differences, Section 5.2):
//   g_i = sum_mu [ (a-abar)_{i+1/2} (u_{i+e} - u_i) - (a-abar)_{i-1/2} (u_i - u_{i-e}) ] / h_mu^2
//       + sum_mu (b_mu - beta_mu) (u_{i+e} - u_{i-e}) / (2 h_mu) + r(u_i),
//   (A u)_i = sum_mu abar (u_{i+e} - 2 u_i + u_{i-e}) / h_mu^2 + beta_mu (u_{i+e} - u_{i-e}) / (2 h_mu),
// face coefficient (a-abar)_{i+1/2} = ((a-abar)_i + (a-abar)_{i+e}) / 2 of the nodal field,
// Dirichlet ghosts u = 0. F = g + A u.
//
// Layout: u is n3*n2*n1 (x1 fastest), the nodal (a - abar) is (n3+2)(n2+2)(n1+2).
// A CTA covers 32 x 8 nodes of (x1, x2) and ZCHUNK planes of x3.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "adr_internal.h"
#include "stencil_core.cuh"

namespace adr {
namespace {

constexpr int TX = 32;   // x1 extent of a CTA tile (one warp wide: coalesced rows)
constexpr int TY = 8;    // x2 extent
constexpr int ZCHUNK = 4;   // x3 planes per thread

// One pass over the grid. Each thread owns the nodes (i1, i2, z0 .. z0+ZC-1): it issues
// every load of its column up front (centre column with its x3 halo, the four x1/x2
// neighbours per plane, the extra stage inputs), all independent and warp-coalesced along
// x1, so no barrier is needed and many requests are in flight; x1/x2 neighbours are served
// by L1, x3 neighbours by registers. DIM = 2 has one plane and no x3 terms.
template <typename T, int DIM, int ZC, bool HASLO>
__global__ void __launch_bounds__(TX * TY) stencil_kernel(StencilArgs<T> p, Coefs<T> c, bool needF) {
    const int n1 = p.n1, n2 = p.n2, n3 = p.n3;
    const int A1 = p.apitch, A2 = n2 + 2;
    const long long plane_u = (long long)n1 * n2;
    const long long plane_a = (long long)A1 * A2;
    const int i1 = blockIdx.x * TX + int(threadIdx.x % TX);
    const int i2 = blockIdx.y * TY + int(threadIdx.x / TX);
    const int z0 = (DIM == 3) ? int(blockIdx.z) * ZC : 0;
    const bool inside = (i1 < n1) && (i2 < n2);
    const long long row_u = (long long)i2 * n1 + i1;
    const long long row_a = (long long)(i2 + 1) * A1 + (i1 + 4);   // interior i1 at offset 4

    // loads: u (and its low part) at the node and its 6 neighbours, a at the node and its 6
    T uc[ZC + 2], lc[ZC + 2], ac[ZC + 2];
    T uw[ZC], ue[ZC], us[ZC], un[ZC], lw[ZC], le[ZC], ls[ZC], ln[ZC], aw[ZC], ae[ZC], as_[ZC], an[ZC];
    T xv[ZC][kMaxExtra];
#pragma unroll
    for (int q = 0; q < ZC + 2; ++q) {
        uc[q] = T(0); lc[q] = T(0); ac[q] = T(0);
        const int z = z0 - 1 + q;                  // interior plane index, -1 and n3 are boundary
        if (!inside || (DIM == 2 && q != 1) || (DIM == 3 && z > n3)) continue;
        const long long za = (DIM == 3) ? (long long)(z + 1) * plane_a : 0;
        ac[q] = __ldg(p.a + za + row_a);
        const int zs = (DIM == 3 && p.neumann && z == n3) ? n3 - 2 : z;   // Neumann: mirror ghost plane
        if (DIM == 2 || (zs >= 0 && zs < n3)) {
            const long long zu = (DIM == 3 ? (long long)zs * plane_u : 0) + row_u;
            uc[q] = __ldg(p.u + zu);
            if (HASLO) lc[q] = __ldg(p.u_lo + zu);
        }
    }
#pragma unroll
    for (int q = 0; q < ZC; ++q) {
        const int z = z0 + q;
        uw[q] = ue[q] = us[q] = un[q] = T(0);
        lw[q] = le[q] = ls[q] = ln[q] = T(0);
        aw[q] = ae[q] = as_[q] = an[q] = T(0);
#pragma unroll
        for (int e = 0; e < kMaxExtra; ++e) xv[q][e] = T(0);
        if (!inside || (DIM == 3 && z >= n3)) continue;
        const long long zu = (DIM == 3) ? (long long)z * plane_u : 0;
        const long long za = (DIM == 3) ? (long long)(z + 1) * plane_a : 0;
        const T* uz = p.u + zu + row_u;
        const T* az = p.a + za + row_a;
        // Dirichlet ghosts are zero; a Neumann face at x_mu = 1 mirrors u_{n-1} (p.neumann)
        if (i1 > 0) uw[q] = __ldg(uz - 1);
        if (i1 + 1 < n1) ue[q] = __ldg(uz + 1);
        else if (p.neumann && i1 > 0) ue[q] = uw[q];
        if (i2 > 0) us[q] = __ldg(uz - n1);
        if (i2 + 1 < n2) un[q] = __ldg(uz + n1);
        else if (p.neumann && i2 > 0) un[q] = us[q];
        if (HASLO) {
            const T* lz = p.u_lo + zu + row_u;
            if (i1 > 0) lw[q] = __ldg(lz - 1);
            if (i1 + 1 < n1) le[q] = __ldg(lz + 1);
            else if (p.neumann && i1 > 0) le[q] = lw[q];
            if (i2 > 0) ls[q] = __ldg(lz - n1);
            if (i2 + 1 < n2) ln[q] = __ldg(lz + n1);
            else if (p.neumann && i2 > 0) ln[q] = ls[q];
        }
        aw[q] = __ldg(az - 1);                      // the boundary ring makes these valid
        ae[q] = __ldg(az + 1);
        as_[q] = __ldg(az - A1);
        an[q] = __ldg(az + A1);
#pragma unroll
        for (int e = 0; e < kMaxExtra; ++e)
            if (e < p.nx) xv[q][e] = __ldg(p.X[e] + zu + row_u);
    }
    float outabs[kMaxOut] = {0.f, 0.f};
    float uabs = 0.f;
#pragma unroll
    for (int q = 0; q < ZC; ++q) {
        const int z = z0 + q;
        if (!inside || (DIM == 3 && z >= n3)) continue;
        const T u0 = uc[q + 1], l0 = lc[q + 1], a0 = ac[q + 1];
        // one-sided differences; with a low part, (hi difference) + (lo difference)
        const T dE = (ue[q] - u0) + (le[q] - l0), dW = (u0 - uw[q]) + (l0 - lw[q]);
        const T dN = (un[q] - u0) + (ln[q] - l0), dS = (u0 - us[q]) + (l0 - ls[q]);
        const T dP = DIM == 3 ? (uc[q + 2] - u0) + (lc[q + 2] - l0) : T(0);
        const T dM = DIM == 3 ? (u0 - uc[q]) + (l0 - lc[q]) : T(0);
        const T uC = u0 + l0;
        T F = T(0);
        // face sums (a - abar)_C + (a - abar)_nb; the a Lap u form uses 2 (a - abar)_C on every face
        const T g = p.adelta
            ? stencil_core<T, DIM>(c, uC, dE, dW, dN, dS, dP, dM, a0 + a0, a0 + a0, a0 + a0, a0 + a0, a0 + a0, a0 + a0,
                                   needF, F)
            : stencil_core<T, DIM>(c, uC, dE, dW, dN, dS, dP, dM, a0 + ae[q], a0 + aw[q], a0 + an[q], a0 + as_[q],
                                   a0 + ac[q + 2], a0 + ac[q], needF, F);
        const long long idx = (DIM == 3 ? (long long)z * plane_u : 0) + row_u;
        uabs = fmaxf(uabs, (float)absval(uC));
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j) {
            if (j < p.nout) {
                T v = c.cu[j] * uC + c.cg[j] * g + c.cF[j] * F;
#pragma unroll
                for (int e = 0; e < kMaxExtra; ++e) v += c.cx[j][e] * xv[q][e];
                p.out[j][idx] = v;
                outabs[j] = fmaxf(outabs[j], (float)absval(v));
            }
        }
    }
    // converged warp reductions (amax slots are uniform across the grid)
    if (p.amax_u) block_amax(uabs, p.amax_u);
#pragma unroll
    for (int j = 0; j < kMaxOut; ++j)
        if (j < p.nout && p.amax[j]) block_amax(outabs[j], p.amax[j]);
}

// FP32, n1 % 4 == 0: each thread computes 4 consecutive x1 nodes of ZV planes with 16-byte
// loads; the x1 neighbours of the 4-node group come from the adjacent lanes (shuffles), the
// warp edges load them. A warp covers 128 consecutive x1 nodes of one (x2, x3) row.
constexpr int ZV = 2;
constexpr int kMarchPlanes = 12;   // x3 planes walked by one CTA of the z-marching kernel

__device__ __forceinline__ void f4arr(const float4& v, float (&a)[4]) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; }
__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

template <int DIM, bool HASLO>
__global__ void __launch_bounds__(256) stencil_vec4_kernel(StencilArgs<float> p, Coefs<float> c, bool needF) {
    const int n1 = p.n1, n2 = p.n2, n3 = p.n3;
    const int A1 = p.apitch, A2 = n2 + 2;
    const long long plane_u = (long long)n1 * n2;
    const long long plane_a = (long long)A1 * A2;
    const int lane = threadIdx.x & 31;
    const int i1 = (blockIdx.x * 32 + lane) * 4;
    const int i2 = blockIdx.y * 8 + int(threadIdx.x >> 5);
    const int z0 = (DIM == 3) ? int(blockIdx.z) * ZV : 0;
    const bool inside = (i1 < n1) && (i2 < n2);      // n1 % 4 == 0: all 4 nodes or none
    const long long row_u = (long long)i2 * n1 + i1;
    const long long row_a = (long long)(i2 + 1) * A1 + (i1 + 4);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    float4 uc[ZV + 2], lc[ZV + 2], ac[ZV + 2];
#pragma unroll
    for (int q = 0; q < ZV + 2; ++q) {
        uc[q] = lc[q] = ac[q] = zero4;
        const int z = z0 - 1 + q;
        if (!inside || (DIM == 2 && q != 1) || (DIM == 3 && z > n3)) continue;
        const long long za = (DIM == 3) ? (long long)(z + 1) * plane_a : 0;
        ac[q] = ld4(p.a + za + row_a);
        if (DIM == 2 || (z >= 0 && z < n3)) {
            const long long zu = (DIM == 3 ? (long long)z * plane_u : 0) + row_u;
            uc[q] = ld4(p.u + zu);
            if (HASLO) lc[q] = ld4(p.u_lo + zu);
        }
    }
    float outabs[kMaxOut] = {0.f, 0.f};
    float uabs = 0.f;
#pragma unroll
    for (int q = 0; q < ZV; ++q) {
        const int z = z0 + q;
        const bool plane_ok = (DIM == 2) ? (q == 0) : (z < n3);   // 2-D: a single plane
        const long long zu = (DIM == 3) ? (long long)z * plane_u : 0;
        const long long za = (DIM == 3) ? (long long)(z + 1) * plane_a : 0;
        float4 us = zero4, un = zero4, ls4 = zero4, ln4 = zero4, as4 = zero4, an4 = zero4;
        float xw = 0.f, xe = 0.f, yw = 0.f, ye = 0.f, aw = 0.f, ae = 0.f;
        float4 xv[kMaxExtra];
#pragma unroll
        for (int e = 0; e < kMaxExtra; ++e) xv[e] = zero4;
        // warp edges, and a group whose right neighbour is the boundary, load their halo
        const bool load_e = (lane == 31) || (i1 + 4 >= n1);
        if (inside && plane_ok) {
            const float* uz = p.u + zu + row_u;
            const float* az = p.a + za + row_a;
            if (i2 > 0) us = ld4(uz - n1);
            if (i2 + 1 < n2) un = ld4(uz + n1);
            as4 = ld4(az - A1);
            an4 = ld4(az + A1);
            if (lane == 0 && i1 > 0) xw = __ldg(uz - 1);
            if (load_e && i1 + 4 < n1) xe = __ldg(uz + 4);
            if (lane == 0) aw = __ldg(az - 1);
            if (load_e) ae = __ldg(az + 4);
            if (HASLO) {
                const float* lz = p.u_lo + zu + row_u;
                if (i2 > 0) ls4 = ld4(lz - n1);
                if (i2 + 1 < n2) ln4 = ld4(lz + n1);
                if (lane == 0 && i1 > 0) yw = __ldg(lz - 1);
                if (load_e && i1 + 4 < n1) ye = __ldg(lz + 4);
            }
#pragma unroll
            for (int e = 0; e < kMaxExtra; ++e)
                if (e < p.nx) xv[e] = ld4(p.X[e] + zu + row_u);
        }
        const float4 u0 = uc[q + 1], l0 = lc[q + 1], a0 = ac[q + 1];
        // x1 halo of the group from the neighbouring lanes (all lanes take part)
        const float sw_u = __shfl_up_sync(0xffffffffu, u0.w, 1), se_u = __shfl_down_sync(0xffffffffu, u0.x, 1);
        const float sw_a = __shfl_up_sync(0xffffffffu, a0.w, 1), se_a = __shfl_down_sync(0xffffffffu, a0.x, 1);
        float sw_l = 0.f, se_l = 0.f;
        if (HASLO) {
            sw_l = __shfl_up_sync(0xffffffffu, l0.w, 1);
            se_l = __shfl_down_sync(0xffffffffu, l0.x, 1);
        }
        if (!inside || !plane_ok) continue;
        if (lane != 0) { xw = sw_u; aw = sw_a; yw = sw_l; }
        if (lane != 31 && i1 + 4 < n1) { xe = se_u; ae = se_a; ye = se_l; }
        float U[4], L[4], Aa[4], US[4], UN[4], LS[4], LN[4], AS[4], AN[4], UM[4], UP[4], LM[4], LP[4], AM[4], AP[4];
        f4arr(u0, U); f4arr(l0, L); f4arr(a0, Aa);
        f4arr(us, US); f4arr(un, UN); f4arr(ls4, LS); f4arr(ln4, LN); f4arr(as4, AS); f4arr(an4, AN);
        f4arr(uc[q], UM); f4arr(uc[q + 2], UP); f4arr(lc[q], LM); f4arr(lc[q + 2], LP); f4arr(ac[q], AM); f4arr(ac[q + 2], AP);
        const float UX[6] = {xw, U[0], U[1], U[2], U[3], xe}, LX[6] = {yw, L[0], L[1], L[2], L[3], ye};
        const float AX[6] = {aw, Aa[0], Aa[1], Aa[2], Aa[3], ae};
        float res[kMaxOut][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float uC = U[k], lC = L[k], aC = Aa[k];
            const float dE = (UX[k + 2] - uC) + (LX[k + 2] - lC), dW = (uC - UX[k]) + (lC - LX[k]);
            const float dN = (UN[k] - uC) + (LN[k] - lC), dS = (uC - US[k]) + (lC - LS[k]);
            const float dP = (UP[k] - uC) + (LP[k] - lC), dM = (uC - UM[k]) + (lC - LM[k]);
            const float uF = uC + lC;
            float F = 0.f;
            const float g = stencil_core<float, DIM>(c, uF, dE, dW, dN, dS, dP, dM, aC + AX[k + 2], aC + AX[k],
                                                     aC + AN[k], aC + AS[k], aC + AP[k], aC + AM[k], needF, F);
            uabs = fmaxf(uabs, fabsf(uF));
#pragma unroll
            for (int j = 0; j < kMaxOut; ++j) {
                float v = c.cu[j] * uF + c.cg[j] * g + c.cF[j] * F;
#pragma unroll
                for (int e = 0; e < kMaxExtra; ++e) {
                    float xe4[4];
                    f4arr(xv[e], xe4);
                    v += c.cx[j][e] * xe4[k];
                }
                res[j][k] = v;
            }
        }
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j) {
            if (j < p.nout) {
                *reinterpret_cast<float4*>(p.out[j] + zu + row_u) = make_float4(res[j][0], res[j][1], res[j][2], res[j][3]);
                outabs[j] = fmaxf(outabs[j], fmaxf(fmaxf(fabsf(res[j][0]), fabsf(res[j][1])), fmaxf(fabsf(res[j][2]), fabsf(res[j][3]))));
            }
        }
    }
    if (p.amax_u) block_amax(uabs, p.amax_u);
#pragma unroll
    for (int j = 0; j < kMaxOut; ++j)
        if (j < p.nout && p.amax[j]) block_amax(outabs[j], p.amax[j]);
}

// FP32, 3-D, n1 % 4 == 0: z-marching form. A thread owns 4 consecutive x1 nodes of one
// (x2) row and walks ZB planes of x3: the planes below, at and above the current one stay
// in registers and rotate, and the next plane's centre values (u, its low part, a, the extra
// stage inputs) are loaded one iteration ahead, so each value is read from memory about once
// and the loads of plane z+1 are in flight while plane z is computed. The x1 neighbours come
// from the adjacent lanes (shuffles), the x2 neighbours from the rows of the adjacent warps
// (L1/L2 hits).
template <bool HASLO, int NX, int NOUT>
__global__ void __launch_bounds__(256, HASLO ? 2 : 3) stencil_march_kernel(StencilArgs<float> p, Coefs<float> c, bool needF, int zb) {
    const int n1 = p.n1, n2 = p.n2, n3 = p.n3;
    const int A1 = p.apitch, A2 = n2 + 2;
    const long long plane_u = (long long)n1 * n2;
    const long long plane_a = (long long)A1 * A2;
    const int lane = threadIdx.x & 31;
    const int i1 = (blockIdx.x * 32 + lane) * 4;
    const int i2 = blockIdx.y * 8 + int(threadIdx.x >> 5);
    const int z0 = int(blockIdx.z) * zb;
    const int z1 = min(z0 + zb, n3);
    const bool inside = (i1 < n1) && (i2 < n2);      // n1 % 4 == 0: all 4 nodes or none
    const long long row_u = (long long)i2 * n1 + i1;
    const long long row_a = (long long)(i2 + 1) * A1 + (i1 + 4);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool load_e = (lane == 31) || (i1 + 4 >= n1);

    // planes z-1 (M), z (C), z+1 (P) of u (+ low part) and of a; x1 ghosts of u are 0
    float4 uM = zero4, uC = zero4, uP = zero4, lM = zero4, lC = zero4, lP = zero4;
    float4 aM = zero4, aC = zero4, aP = zero4;
    float4 xC[NX > 0 ? NX : 1], xP[NX > 0 ? NX : 1];
#pragma unroll
    for (int e = 0; e < (NX > 0 ? NX : 1); ++e) xC[e] = xP[e] = zero4;
    if (inside) {
        aM = ld4(p.a + (long long)z0 * plane_a + row_a);              // a plane index z + 1
        aC = ld4(p.a + (long long)(z0 + 1) * plane_a + row_a);
        if (z0 > 0) {
            uM = ld4(p.u + (long long)(z0 - 1) * plane_u + row_u);
            if (HASLO) lM = ld4(p.u_lo + (long long)(z0 - 1) * plane_u + row_u);
        }
        uC = ld4(p.u + (long long)z0 * plane_u + row_u);
        if (HASLO) lC = ld4(p.u_lo + (long long)z0 * plane_u + row_u);
#pragma unroll
        for (int e = 0; e < NX; ++e) xC[e] = ld4(p.X[e] + (long long)z0 * plane_u + row_u);
    }
    float outabs[NOUT];
#pragma unroll
    for (int j = 0; j < NOUT; ++j) outabs[j] = 0.f;
    float uabs = 0.f;
    for (int z = z0; z < z1; ++z) {
        const long long zu = (long long)z * plane_u;
        const long long za = (long long)(z + 1) * plane_a;
        // next plane (in flight during this one)
        if (inside) {
            aP = ld4(p.a + za + plane_a + row_a);                     // a at z + 1 (ring: z + 2 <= n3 + 1)
            if (z + 1 < n3) {
                uP = ld4(p.u + zu + plane_u + row_u);
                if (HASLO) lP = ld4(p.u_lo + zu + plane_u + row_u);
                if (z + 1 < z1) {
#pragma unroll
                    for (int e = 0; e < NX; ++e) xP[e] = ld4(p.X[e] + zu + plane_u + row_u);
                }
            } else if (p.neumann) {          // Neumann face at x3 = 1: mirror ghost plane
                uP = uM;
                lP = lM;
            } else {
                uP = zero4;
                lP = zero4;
            }
        }
        float4 us = zero4, un = zero4, ls4 = zero4, ln4 = zero4, as4 = zero4, an4 = zero4;
        float xw = 0.f, xe = 0.f, yw = 0.f, ye = 0.f, aw = 0.f, ae = 0.f;
        if (inside) {
            const float* uz = p.u + zu + row_u;
            const float* az = p.a + za + row_a;
            if (i2 > 0) us = ld4(uz - n1);
            if (i2 + 1 < n2) un = ld4(uz + n1);
            else if (p.neumann && i2 > 0) un = us;          // Neumann face at x2 = 1
            as4 = ld4(az - A1);
            an4 = ld4(az + A1);
            if (lane == 0 && i1 > 0) xw = __ldg(uz - 1);
            if (load_e && i1 + 4 < n1) xe = __ldg(uz + 4);
            if (lane == 0) aw = __ldg(az - 1);
            if (load_e) ae = __ldg(az + 4);
            if (HASLO) {
                const float* lz = p.u_lo + zu + row_u;
                if (i2 > 0) ls4 = ld4(lz - n1);
                if (i2 + 1 < n2) ln4 = ld4(lz + n1);
                else if (p.neumann && i2 > 0) ln4 = ls4;
                if (lane == 0 && i1 > 0) yw = __ldg(lz - 1);
                if (load_e && i1 + 4 < n1) ye = __ldg(lz + 4);
            }
        }
        // x1 halo of the group from the neighbouring lanes (all lanes take part)
        const float sw_u = __shfl_up_sync(0xffffffffu, uC.w, 1), se_u = __shfl_down_sync(0xffffffffu, uC.x, 1);
        const float sw_a = __shfl_up_sync(0xffffffffu, aC.w, 1), se_a = __shfl_down_sync(0xffffffffu, aC.x, 1);
        float sw_l = 0.f, se_l = 0.f;
        if (HASLO) {
            sw_l = __shfl_up_sync(0xffffffffu, lC.w, 1);
            se_l = __shfl_down_sync(0xffffffffu, lC.x, 1);
        }
        if (inside) {
            if (lane != 0) { xw = sw_u; aw = sw_a; yw = sw_l; }
            if (lane != 31 && i1 + 4 < n1) { xe = se_u; ae = se_a; ye = se_l; }
            if (p.neumann && i1 + 4 >= n1) { xe = uC.z; ye = lC.z; }   // Neumann face at x1 = 1: mirror
            float U[4], L[4], Aa[4], US[4], UN[4], LS[4], LN[4], AS[4], AN[4], UM[4], UP[4], LM[4], LP[4], AM[4], AP[4];
            f4arr(uC, U); f4arr(lC, L); f4arr(aC, Aa);
            f4arr(us, US); f4arr(un, UN); f4arr(ls4, LS); f4arr(ln4, LN); f4arr(as4, AS); f4arr(an4, AN);
            f4arr(uM, UM); f4arr(uP, UP); f4arr(lM, LM); f4arr(lP, LP); f4arr(aM, AM); f4arr(aP, AP);
            const float UX[6] = {xw, U[0], U[1], U[2], U[3], xe}, LX[6] = {yw, L[0], L[1], L[2], L[3], ye};
            const float AX[6] = {aw, Aa[0], Aa[1], Aa[2], Aa[3], ae};
            float res[NOUT][4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float uk = U[k], lk = L[k], ak = Aa[k];
                const float dE = (UX[k + 2] - uk) + (LX[k + 2] - lk), dW = (uk - UX[k]) + (lk - LX[k]);
                const float dN = (UN[k] - uk) + (LN[k] - lk), dS = (uk - US[k]) + (lk - LS[k]);
                const float dP = (UP[k] - uk) + (LP[k] - lk), dM = (uk - UM[k]) + (lk - LM[k]);
                const float uF = uk + lk;
                float F = 0.f;
                const float g = p.adelta
                    ? stencil_core<float, 3>(c, uF, dE, dW, dN, dS, dP, dM, ak + ak, ak + ak, ak + ak, ak + ak, ak + ak,
                                             ak + ak, needF, F)
                    : stencil_core<float, 3>(c, uF, dE, dW, dN, dS, dP, dM, ak + AX[k + 2], ak + AX[k], ak + AN[k],
                                             ak + AS[k], ak + AP[k], ak + AM[k], needF, F);
                uabs = fmaxf(uabs, fabsf(uF));
#pragma unroll
                for (int j = 0; j < NOUT; ++j) {
                    float v = c.cu[j] * uF + c.cg[j] * g + c.cF[j] * F;
#pragma unroll
                    for (int e = 0; e < NX; ++e) {
                        float xe4[4];
                        f4arr(xC[e], xe4);
                        v += c.cx[j][e] * xe4[k];
                    }
                    res[j][k] = v;
                }
            }
#pragma unroll
            for (int j = 0; j < NOUT; ++j) {
                *reinterpret_cast<float4*>(p.out[j] + zu + row_u) = make_float4(res[j][0], res[j][1], res[j][2], res[j][3]);
                outabs[j] = fmaxf(outabs[j], fmaxf(fmaxf(fabsf(res[j][0]), fabsf(res[j][1])), fmaxf(fabsf(res[j][2]), fabsf(res[j][3]))));
            }
        }
        uM = uC; uC = uP; lM = lC; lC = lP; aM = aC; aC = aP;
#pragma unroll
        for (int e = 0; e < NX; ++e) xC[e] = xP[e];
    }
    if (p.amax_u) block_amax(uabs, p.amax_u);
#pragma unroll
    for (int j = 0; j < NOUT; ++j)
        if (p.amax[j]) block_amax(outabs[j], p.amax[j]);
}

template <bool HASLO, int NX>
void launch_march_nout(const StencilArgs<float>& p, const Coefs<float>& c, bool needF, int zb, dim3 g, cudaStream_t s) {
    if (p.nout == 1) stencil_march_kernel<HASLO, NX, 1><<<g, 256, 0, s>>>(p, c, needF, zb);
    else             stencil_march_kernel<HASLO, NX, 2><<<g, 256, 0, s>>>(p, c, needF, zb);
}

template <bool HASLO>
void launch_march_nx(const StencilArgs<float>& p, const Coefs<float>& c, bool needF, int zb, dim3 g, cudaStream_t s) {
    switch (p.nx) {
    case 0: launch_march_nout<HASLO, 0>(p, c, needF, zb, g, s); break;
    case 1: launch_march_nout<HASLO, 1>(p, c, needF, zb, g, s); break;
    case 2: launch_march_nout<HASLO, 2>(p, c, needF, zb, g, s); break;
    default: launch_march_nout<HASLO, 3>(p, c, needF, zb, g, s); break;
    }
}

cudaError_t launch_march(const StencilArgs<float>& p, const Coefs<float>& c, bool needF, int zb, dim3 g, cudaStream_t s) {
    if (p.nout < 1 || p.nout > kMaxOut || p.nx < 0 || p.nx > kMaxExtra) return cudaErrorInvalidValue;
    if (p.u_lo) launch_march_nx<true>(p, c, needF, zb, g, s);
    else        launch_march_nx<false>(p, c, needF, zb, g, s);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_impl(const StencilArgs<T>& p, cudaStream_t s) {
    Coefs<T> c;
    for (int m = 0; m < 3; ++m) {
        c.ih2[m] = T(p.inv_h2[m]);
        c.i2h[m] = T(p.inv_2h[m]);
        c.bmb[m] = T(p.bmb[m]);
        c.beta[m] = T(p.beta[m]);
    }
    c.abar = T(p.abar);
    c.r0 = T(p.r[0]); c.r1 = T(p.r[1]); c.r2 = T(p.r[2]); c.r3 = T(p.r[3]);
    bool needF = false;
    for (int j = 0; j < kMaxOut; ++j) {
        c.cg[j] = T(p.cg[j]); c.cF[j] = T(p.cF[j]);
        state_coefs<T>(p.cu[j], p.cx[j], c.cu[j], c.cx[j]);
        if (j < p.nout && p.cF[j] != 0.0) needF = true;
    }
    dim3 block(TX * TY);
    if constexpr (std::is_same<T, float>::value) {
        bool aligned = (p.n1 % 4 == 0) && (p.apitch % 4 == 0) && (reinterpret_cast<uintptr_t>(p.u) % 16 == 0) &&
                       (reinterpret_cast<uintptr_t>(p.a) % 16 == 0);
        for (int j = 0; j < p.nout; ++j) aligned = aligned && (reinterpret_cast<uintptr_t>(p.out[j]) % 16 == 0);
        for (int e = 0; e < p.nx; ++e) aligned = aligned && (reinterpret_cast<uintptr_t>(p.X[e]) % 16 == 0);
        // the vectorised 2-D kernel has Dirichlet ghosts and the flux form only
        if (p.dim == 2 && (p.neumann || p.adelta)) aligned = false;
        if (p.u_lo) aligned = aligned && (reinterpret_cast<uintptr_t>(p.u_lo) % 16 == 0);
        if (aligned) {
            dim3 g4((p.n1 / 4 + 31) / 32, (p.n2 + 7) / 8, p.dim == 3 ? (p.n3 + ZV - 1) / ZV : 1);
            if (p.dim == 3) {
                if (stencil_tma_usable(p)) return launch_stencil_tma(p, c, needF, s);
                const int zb = kMarchPlanes;
                dim3 gm((p.n1 / 4 + 31) / 32, (p.n2 + 7) / 8, (p.n3 + zb - 1) / zb);
                return launch_march(p, c, needF, zb, gm, s);
            } else {
                if (p.u_lo) stencil_vec4_kernel<2, true><<<g4, 256, 0, s>>>(p, c, needF);
                else        stencil_vec4_kernel<2, false><<<g4, 256, 0, s>>>(p, c, needF);
            }
            return cudaGetLastError();
        }
    }
    dim3 grid((p.n1 + TX - 1) / TX, (p.n2 + TY - 1) / TY, p.dim == 3 ? (p.n3 + ZCHUNK - 1) / ZCHUNK : 1);
    const bool lo = std::is_same<T, float>::value && p.u_lo != nullptr;
    if (p.dim == 3) {
        if (lo) stencil_kernel<T, 3, ZCHUNK, true><<<grid, block, 0, s>>>(p, c, needF);
        else    stencil_kernel<T, 3, ZCHUNK, false><<<grid, block, 0, s>>>(p, c, needF);
    } else {
        if (lo) stencil_kernel<T, 2, 1, true><<<grid, block, 0, s>>>(p, c, needF);
        else    stencil_kernel<T, 2, 1, false><<<grid, block, 0, s>>>(p, c, needF);
    }
    return cudaGetLastError();
}

__global__ void amax_kernel(const float* x, size_t n, unsigned* slot) {
    float m = 0.f;
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    block_amax(m, slot);
}

__global__ void convert_kernel(const double* in, float* out, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        out[i] = float(in[i]);
}

}  // namespace

cudaError_t launch_stencil(const StencilArgs<double>& a, cudaStream_t s) { return launch_impl(a, s); }
cudaError_t launch_stencil(const StencilArgs<float>& a, cudaStream_t s) { return launch_impl(a, s); }

cudaError_t launch_amax(const float* x, size_t n, unsigned* slot, cudaStream_t s) {
    const int blocks = int(std::min<size_t>((n + 255) / 256, 152 * 8));
    amax_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(x, n, slot);
    return cudaGetLastError();
}

cudaError_t launch_convert_f64_to_f32(const double* in, float* out, size_t n, cudaStream_t s) {
    const int blocks = int(std::min<size_t>((n + 255) / 256, 152 * 16));
    convert_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

}  // namespace adr
