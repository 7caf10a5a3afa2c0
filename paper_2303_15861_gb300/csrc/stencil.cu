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

namespace adr {
namespace {

constexpr int TX = 32;   // x1 extent of a CTA tile (one warp wide: coalesced rows)
constexpr int TY = 8;    // x2 extent
constexpr int ZCHUNK = 4;   // x3 planes per thread

template <typename T>
struct Coefs {
    T ih2[3], i2h[3], bmb[3], beta[3], abar, r0, r1, r2, r3;
    T cu[kMaxOut], cx[kMaxOut][kMaxExtra], cg[kMaxOut], cF[kMaxOut];
};

template <typename T>
__device__ __forceinline__ T absval(T v) { return v < T(0) ? -v : v; }

__device__ __forceinline__ void block_amax(float v, unsigned* slot) {
    // Warp max then one atomic per warp; |out| as float bits (monotone for v >= 0).
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(slot, __float_as_uint(v));
}

// One pass over the grid. Each thread owns the nodes (i1, i2, z0 .. z0+ZC-1): it issues
// every load of its column up front (centre column with its x3 halo, the four x1/x2
// neighbours per plane, the extra stage inputs), all independent and warp-coalesced along
// x1, so no barrier is needed and many requests are in flight; x1/x2 neighbours are served
// by L1, x3 neighbours by registers. DIM = 2 has one plane and no x3 terms.
template <typename T, int DIM, int ZC>
__global__ void __launch_bounds__(TX * TY) stencil_kernel(StencilArgs<T> p, Coefs<T> c, bool needF) {
    const int n1 = p.n1, n2 = p.n2, n3 = p.n3;
    const int A1 = p.apitch, A2 = n2 + 2;
    const long long plane_u = (long long)n1 * n2;
    const long long plane_a = (long long)A1 * A2;
    const int i1 = blockIdx.x * TX + int(threadIdx.x % TX);
    const int i2 = blockIdx.y * TY + int(threadIdx.x / TX);
    const int z0 = (DIM == 3) ? int(blockIdx.z) * ZC : 0;
    const bool inside = (i1 < n1) && (i2 < n2);

    T uc[ZC + 2], ac[ZC + 2];
    T uw[ZC], ue[ZC], us[ZC], un[ZC], aw[ZC], ae[ZC], as_[ZC], an[ZC];
    T xv[ZC][kMaxExtra];
    const long long row_u = (long long)i2 * n1 + i1;
    const long long row_a = (long long)(i2 + 1) * A1 + (i1 + 4);   // interior i1 at offset 4
#pragma unroll
    for (int q = 0; q < ZC + 2; ++q) { uc[q] = T(0); ac[q] = T(0); }
    if (inside) {
#pragma unroll
        for (int q = 0; q < ZC + 2; ++q) {
            const int z = z0 - 1 + q;                  // interior plane index, -1 and n3 are boundary
            if (DIM == 2 && q != 1) continue;
            if (DIM == 3 && z > n3) continue;
            const long long za = (DIM == 3) ? (long long)(z + 1) * plane_a : 0;
            ac[q] = __ldg(p.a + za + row_a);
            if (DIM == 2 || (z >= 0 && z < n3)) uc[q] = __ldg(p.u + (DIM == 3 ? (long long)z * plane_u : 0) + row_u);
        }
#pragma unroll
        for (int q = 0; q < ZC; ++q) {
            const int z = z0 + q;
            uw[q] = ue[q] = us[q] = un[q] = T(0);
            aw[q] = ae[q] = as_[q] = an[q] = T(0);
            if (DIM == 3 && z >= n3) continue;
            const long long zu = (DIM == 3) ? (long long)z * plane_u : 0;
            const long long za = (DIM == 3) ? (long long)(z + 1) * plane_a : 0;
            const T* uz = p.u + zu + row_u;
            const T* az = p.a + za + row_a;
            if (i1 > 0) uw[q] = __ldg(uz - 1);
            if (i1 + 1 < n1) ue[q] = __ldg(uz + 1);
            if (i2 > 0) us[q] = __ldg(uz - n1);
            if (i2 + 1 < n2) un[q] = __ldg(uz + n1);
            aw[q] = __ldg(az - 1);                      // the boundary ring makes these valid
            ae[q] = __ldg(az + 1);
            as_[q] = __ldg(az - A1);
            an[q] = __ldg(az + A1);
#pragma unroll
            for (int e = 0; e < kMaxExtra; ++e) xv[q][e] = (e < p.nx) ? __ldg(p.X[e] + zu + row_u) : T(0);
        }
    }
    float outabs[kMaxOut] = {0.f, 0.f};
    float uabs = 0.f;
    const T half = T(0.5), two = T(2);
#pragma unroll
    for (int q = 0; q < ZC; ++q) {
        const int z = z0 + q;
        if (!inside || (DIM == 3 && z >= n3)) continue;
        const T u0 = uc[q + 1], a0 = ac[q + 1];
        // diffusion remainder (a - abar) in flux form and advection remainder
        T g = (half * (a0 + ae[q]) * (ue[q] - u0) - half * (a0 + aw[q]) * (u0 - uw[q])) * c.ih2[0]
            + (half * (a0 + an[q]) * (un[q] - u0) - half * (a0 + as_[q]) * (u0 - us[q])) * c.ih2[1]
            + c.bmb[0] * (ue[q] - uw[q]) * c.i2h[0] + c.bmb[1] * (un[q] - us[q]) * c.i2h[1];
        if (DIM == 3) {
            const T up = uc[q + 2], um = uc[q], ap = ac[q + 2], am = ac[q];
            g += (half * (a0 + ap) * (up - u0) - half * (a0 + am) * (u0 - um)) * c.ih2[2]
               + c.bmb[2] * (up - um) * c.i2h[2];
        }
        g += c.r0 + u0 * (c.r1 + u0 * (c.r2 + u0 * c.r3));
        T F = T(0);
        if (needF) {
            F = g + c.abar * ((ue[q] - two * u0 + uw[q]) * c.ih2[0] + (un[q] - two * u0 + us[q]) * c.ih2[1])
                  + c.beta[0] * (ue[q] - uw[q]) * c.i2h[0] + c.beta[1] * (un[q] - us[q]) * c.i2h[1];
            if (DIM == 3)
                F += c.abar * (uc[q + 2] - two * u0 + uc[q]) * c.ih2[2] + c.beta[2] * (uc[q + 2] - uc[q]) * c.i2h[2];
        }
        const long long idx = (DIM == 3 ? (long long)z * plane_u : 0) + row_u;
        uabs = fmaxf(uabs, (float)absval(u0));
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j) {
            if (j < p.nout) {
                T v = c.cu[j] * u0 + c.cg[j] * g + c.cF[j] * F;
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
template <int DIM>
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
    const bool row_ok = i2 < n2;
    const long long row_u = (long long)i2 * n1 + i1;
    const long long row_a = (long long)(i2 + 1) * A1 + (i1 + 4);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    float4 uc[ZV + 2], ac[ZV + 2];
#pragma unroll
    for (int q = 0; q < ZV + 2; ++q) {
        uc[q] = zero4;
        ac[q] = zero4;
        const int z = z0 - 1 + q;
        if (!inside || (DIM == 2 && q != 1) || (DIM == 3 && z > n3)) continue;
        const long long za = (DIM == 3) ? (long long)(z + 1) * plane_a : 0;
        ac[q] = __ldg(reinterpret_cast<const float4*>(p.a + za + row_a));
        if (DIM == 2 || (z >= 0 && z < n3))
            uc[q] = __ldg(reinterpret_cast<const float4*>(p.u + (DIM == 3 ? (long long)z * plane_u : 0) + row_u));
    }
    float outabs[kMaxOut] = {0.f, 0.f};
    float uabs = 0.f;
#pragma unroll
    for (int q = 0; q < ZV; ++q) {
        const int z = z0 + q;
        const bool plane_ok = (DIM == 2) ? (q == 0) : (z < n3);   // 2-D: a single plane
        const long long zu = (DIM == 3) ? (long long)z * plane_u : 0;
        const long long za = (DIM == 3) ? (long long)(z + 1) * plane_a : 0;
        float4 us = zero4, un = zero4, as4 = zero4, an4 = zero4;
        float xw = 0.f, xe = 0.f, aw = 0.f, ae = 0.f;
        float4 xv[kMaxExtra];
        if (inside && plane_ok) {
            const float* uz = p.u + zu + row_u;
            const float* az = p.a + za + row_a;
            if (i2 > 0) us = __ldg(reinterpret_cast<const float4*>(uz - n1));
            if (i2 + 1 < n2) un = __ldg(reinterpret_cast<const float4*>(uz + n1));
            as4 = __ldg(reinterpret_cast<const float4*>(az - A1));
            an4 = __ldg(reinterpret_cast<const float4*>(az + A1));
            // warp edges, and a group whose right neighbour is the boundary, load their halo
            const bool load_e = (lane == 31) || (i1 + 4 >= n1);
            if (lane == 0 && i1 > 0) xw = __ldg(uz - 1);
            if (load_e && i1 + 4 < n1) xe = __ldg(uz + 4);
            if (lane == 0) aw = __ldg(az - 1);
            if (load_e) ae = __ldg(az + 4);
#pragma unroll
            for (int e = 0; e < kMaxExtra; ++e)
                xv[e] = (e < p.nx) ? __ldg(reinterpret_cast<const float4*>(p.X[e] + zu + row_u)) : zero4;
        }
        const float4 u0 = uc[q + 1], a0 = ac[q + 1];
        // x1 halo of the group from the neighbouring lanes (all lanes take part)
        const float sw_u = __shfl_up_sync(0xffffffffu, u0.w, 1), se_u = __shfl_down_sync(0xffffffffu, u0.x, 1);
        const float sw_a = __shfl_up_sync(0xffffffffu, a0.w, 1), se_a = __shfl_down_sync(0xffffffffu, a0.x, 1);
        if (!inside || !plane_ok) continue;
        if (lane != 0) { xw = sw_u; aw = sw_a; }
        if (lane != 31 && i1 + 4 < n1) { xe = se_u; ae = se_a; }
        const float uu[6] = {xw, u0.x, u0.y, u0.z, u0.w, xe};
        const float aa[6] = {aw, a0.x, a0.y, a0.z, a0.w, ae};
        const float uS[4] = {us.x, us.y, us.z, us.w}, uN[4] = {un.x, un.y, un.z, un.w};
        const float aS[4] = {as4.x, as4.y, as4.z, as4.w}, aN[4] = {an4.x, an4.y, an4.z, an4.w};
        const float uM[4] = {uc[q].x, uc[q].y, uc[q].z, uc[q].w}, uP[4] = {uc[q + 2].x, uc[q + 2].y, uc[q + 2].z, uc[q + 2].w};
        const float aM[4] = {ac[q].x, ac[q].y, ac[q].z, ac[q].w}, aP[4] = {ac[q + 2].x, ac[q + 2].y, ac[q + 2].z, ac[q + 2].w};
        float res[kMaxOut][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float uC = uu[k + 1], aC = aa[k + 1];
            const float uW = uu[k], uE = uu[k + 2], aW = aa[k], aE = aa[k + 2];
            float g = (0.5f * (aC + aE) * (uE - uC) - 0.5f * (aC + aW) * (uC - uW)) * c.ih2[0]
                    + (0.5f * (aC + aN[k]) * (uN[k] - uC) - 0.5f * (aC + aS[k]) * (uC - uS[k])) * c.ih2[1]
                    + c.bmb[0] * (uE - uW) * c.i2h[0] + c.bmb[1] * (uN[k] - uS[k]) * c.i2h[1];
            if (DIM == 3)
                g += (0.5f * (aC + aP[k]) * (uP[k] - uC) - 0.5f * (aC + aM[k]) * (uC - uM[k])) * c.ih2[2]
                   + c.bmb[2] * (uP[k] - uM[k]) * c.i2h[2];
            g += c.r0 + uC * (c.r1 + uC * (c.r2 + uC * c.r3));
            float F = 0.f;
            if (needF) {
                F = g + c.abar * ((uE - 2.f * uC + uW) * c.ih2[0] + (uN[k] - 2.f * uC + uS[k]) * c.ih2[1])
                      + c.beta[0] * (uE - uW) * c.i2h[0] + c.beta[1] * (uN[k] - uS[k]) * c.i2h[1];
                if (DIM == 3) F += c.abar * (uP[k] - 2.f * uC + uM[k]) * c.ih2[2] + c.beta[2] * (uP[k] - uM[k]) * c.i2h[2];
            }
            uabs = fmaxf(uabs, fabsf(uC));
#pragma unroll
            for (int j = 0; j < kMaxOut; ++j) {
                float v = c.cu[j] * uC + c.cg[j] * g + c.cF[j] * F;
#pragma unroll
                for (int e = 0; e < kMaxExtra; ++e) {
                    const float xe4[4] = {xv[e].x, xv[e].y, xv[e].z, xv[e].w};
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
    (void)row_ok;
    if (p.amax_u) block_amax(uabs, p.amax_u);
#pragma unroll
    for (int j = 0; j < kMaxOut; ++j)
        if (j < p.nout && p.amax[j]) block_amax(outabs[j], p.amax[j]);
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
        c.cu[j] = T(p.cu[j]); c.cg[j] = T(p.cg[j]); c.cF[j] = T(p.cF[j]);
        for (int e = 0; e < kMaxExtra; ++e) c.cx[j][e] = T(p.cx[j][e]);
        if (j < p.nout && p.cF[j] != 0.0) needF = true;
    }
    dim3 block(TX * TY);
    if constexpr (std::is_same<T, float>::value) {
        bool aligned = (p.n1 % 4 == 0) && (p.apitch % 4 == 0) && (reinterpret_cast<uintptr_t>(p.u) % 16 == 0) &&
                       (reinterpret_cast<uintptr_t>(p.a) % 16 == 0);
        for (int j = 0; j < p.nout; ++j) aligned = aligned && (reinterpret_cast<uintptr_t>(p.out[j]) % 16 == 0);
        for (int e = 0; e < p.nx; ++e) aligned = aligned && (reinterpret_cast<uintptr_t>(p.X[e]) % 16 == 0);
        if (aligned) {
            dim3 g4((p.n1 / 4 + 31) / 32, (p.n2 + 7) / 8, p.dim == 3 ? (p.n3 + ZV - 1) / ZV : 1);
            if (p.dim == 3) stencil_vec4_kernel<3><<<g4, 256, 0, s>>>(p, c, needF);
            else            stencil_vec4_kernel<2><<<g4, 256, 0, s>>>(p, c, needF);
            return cudaGetLastError();
        }
    }
    dim3 grid((p.n1 + TX - 1) / TX, (p.n2 + TY - 1) / TY, p.dim == 3 ? (p.n3 + ZCHUNK - 1) / ZCHUNK : 1);
    if (p.dim == 3) stencil_kernel<T, 3, ZCHUNK><<<grid, block, 0, s>>>(p, c, needF);
    else            stencil_kernel<T, 2, 1><<<grid, block, 0, s>>>(p, c, needF);
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
