// Node arithmetic of the K1 stencil, shared by the single-grid kernels (stencil.cu) and the
// batched 2-D kernel (batch2d.cu). See stencil.cu for the discretisation (Eq. (adr) and
// Eq. (nonlin), Section 3; centred differences, Section 5.2).
#pragma once

#include <cuda_runtime.h>

#include "adr_internal.h"

namespace adr {

template <typename T>
struct Coefs {
    T ih2[3], i2h[3], bmb[3], beta[3], abar, r0, r1, r2, r3;
    T cu[kMaxOut], cx[kMaxOut][kMaxExtra], cg[kMaxOut], cF[kMaxOut];
};

// The TMA-staged 3-D FP32 stencil (stencil_tma.cu): whether it takes these arguments (Dirichlet
// faces, n1 a multiple of 4 and at least 64, n2 at least 16, 16-byte aligned arrays), and its
// launch.
bool stencil_tma_usable(const StencilArgs<float>& p);
cudaError_t launch_stencil_tma(const StencilArgs<float>& p, const Coefs<float>& c, bool needF, cudaStream_t s);

template <typename T>
__device__ __forceinline__ T absval(T v) { return v < T(0) ? -v : v; }

__device__ __forceinline__ void block_amax(float v, unsigned* slot) {
    // Warp max then one atomic per warp; |out| as float bits (monotone for v >= 0).
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(slot, __float_as_uint(v));
}


// The stencil at one node from its one-sided differences dE = u_E - u_C, dW = u_C - u_W
// (and N/S, P/M for x2, x3), the centre value and the face-coefficient sums
// sE = (a - abar)_C + (a - abar)_E etc. Returns g; F = g + A u when needF.
template <typename T, int DIM>
__device__ __forceinline__ T stencil_core(const Coefs<T>& c, T uC, T dE, T dW, T dN, T dS, T dP, T dM, T sE, T sW,
                                          T sN, T sS, T sP, T sM, bool needF, T& F) {
    const T h = T(0.5);
    T g = (h * sE * dE - h * sW * dW) * c.ih2[0] + (h * sN * dN - h * sS * dS) * c.ih2[1]
        + c.bmb[0] * (dE + dW) * c.i2h[0] + c.bmb[1] * (dN + dS) * c.i2h[1];
    if (DIM == 3) g += (h * sP * dP - h * sM * dM) * c.ih2[2] + c.bmb[2] * (dP + dM) * c.i2h[2];
    g += c.r0 + uC * (c.r1 + uC * (c.r2 + uC * c.r3));
    if (needF) {
        F = g + c.abar * ((dE - dW) * c.ih2[0] + (dN - dS) * c.ih2[1]) + c.beta[0] * (dE + dW) * c.i2h[0]
              + c.beta[1] * (dN + dS) * c.i2h[1];
        if (DIM == 3) F += c.abar * (dP - dM) * c.ih2[2] + c.beta[2] * (dP + dM) * c.i2h[2];
    }
    return g;
}


}  // namespace adr
