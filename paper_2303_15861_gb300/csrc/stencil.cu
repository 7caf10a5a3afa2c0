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
// Each CTA owns a 32 x 8 column of (x1, x2) and marches along x3, keeping the three
// u planes it needs in registers / shared memory so that u and a are read from HBM
// once (plus a one-node halo).
#include <cuda_runtime.h>

#include "adr_internal.h"

namespace adr {
namespace {

constexpr int TX = 32;   // x1 extent of a CTA tile (one warp wide: coalesced rows)
constexpr int TY = 8;    // x2 extent
constexpr int ZCHUNK = 16;  // x3 planes per CTA

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

// One pass over the grid. DIM = 2 uses n3 = 1 and no x3 terms.
template <typename T, int DIM>
__global__ void __launch_bounds__(TX * TY) stencil_kernel(StencilArgs<T> p, Coefs<T> c, bool needF) {
    __shared__ T su[TY + 2][TX + 2];   // u plane with x1/x2 halo
    __shared__ T sa[TY + 2][TX + 2];   // (a - abar) plane with halo

    const int n1 = p.n1, n2 = p.n2, n3 = p.n3;
    const int A1 = n1 + 2, A2 = n2 + 2;
    const long long plane_u = (long long)n1 * n2;
    const long long plane_a = (long long)A1 * A2;

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int i1 = blockIdx.x * TX + tx;
    const int i2 = blockIdx.y * TY + ty;
    const int z0 = (DIM == 3) ? blockIdx.z * ZCHUNK : 0;
    const int z1 = (DIM == 3) ? min(z0 + ZCHUNK, n3) : 1;
    const bool inside = (i1 < n1) && (i2 < n2);
    // a is needed one node past the interior (boundary ring) for the last face
    const bool inside_a = (i1 <= n1) && (i2 <= n2);

    // Register window along x3 (DIM == 3): u and a at z-1, z, z+1 for this thread's column.
    T u_m = T(0), u_c = T(0), u_p = T(0), a_m = T(0), a_c = T(0), a_p = T(0);
    auto load_u = [&](int z) -> T {
        return (inside && z >= 0 && z < n3) ? p.u[(long long)z * plane_u + (long long)i2 * n1 + i1] : T(0);
    };
    auto load_a = [&](int z) -> T {  // z in interior numbering, z = -1 and n3 are boundary nodes
        if (!inside_a) return T(0);
        const long long za = (DIM == 3) ? (long long)(z + 1) : 0;
        return p.a[za * plane_a + (long long)(i2 + 1) * A1 + (i1 + 1)];
    };
    if (DIM == 3) {
        u_m = load_u(z0 - 1); u_c = load_u(z0);
        a_m = load_a(z0 - 1); a_c = load_a(z0);
    } else {
        u_c = load_u(0); a_c = load_a(0);
    }

    for (int z = z0; z < z1; ++z) {
        if (DIM == 3) { u_p = load_u(z + 1); a_p = load_a(z + 1); }
        // stage the current plane with its x1/x2 halo in shared memory
        __syncthreads();
        su[ty + 1][tx + 1] = u_c;
        sa[ty + 1][tx + 1] = a_c;
        const long long zu = (long long)z * plane_u;
        const long long za = (DIM == 3) ? (long long)(z + 1) * plane_a : 0;
        // halo: x1 edges (2 columns of TY) and x2 edges (2 rows of TX)
        if (threadIdx.x < 2 * TY) {
            const int side = threadIdx.x / TY, r = threadIdx.x % TY;
            const int hx = side ? blockIdx.x * TX + TX : blockIdx.x * TX - 1;
            const int hy = blockIdx.y * TY + r;
            T uv = T(0), av = T(0);
            if (hy < n2 && hx >= -1 && hx <= n1) {
                if (hx >= 0 && hx < n1) uv = p.u[zu + (long long)hy * n1 + hx];
                av = p.a[za + (long long)(hy + 1) * A1 + (hx + 1)];
            }
            su[r + 1][side ? TX + 1 : 0] = uv;
            sa[r + 1][side ? TX + 1 : 0] = av;
        } else if (threadIdx.x < 2 * TY + 2 * TX) {
            const int t = threadIdx.x - 2 * TY;
            const int side = t / TX, col = t % TX;
            const int hx = blockIdx.x * TX + col;
            const int hy = side ? blockIdx.y * TY + TY : blockIdx.y * TY - 1;
            T uv = T(0), av = T(0);
            if (hx < n1 && hy >= -1 && hy <= n2) {
                if (hy >= 0 && hy < n2) uv = p.u[zu + (long long)hy * n1 + hx];
                av = p.a[za + (long long)(hy + 1) * A1 + (hx + 1)];
            }
            su[side ? TY + 1 : 0][col + 1] = uv;
            sa[side ? TY + 1 : 0][col + 1] = av;
        }
        __syncthreads();

        float outabs[kMaxOut] = {0.f, 0.f};
        if (inside) {
            const T uw = su[ty + 1][tx], ue = su[ty + 1][tx + 2];
            const T us = su[ty][tx + 1], un = su[ty + 2][tx + 1];
            const T aw = sa[ty + 1][tx], ae = sa[ty + 1][tx + 2];
            const T as_ = sa[ty][tx + 1], an = sa[ty + 2][tx + 1];
            const T half = T(0.5);
            // diffusion remainder (a - abar) in flux form and advection remainder
            T g = (half * (a_c + ae) * (ue - u_c) - half * (a_c + aw) * (u_c - uw)) * c.ih2[0]
                + (half * (a_c + an) * (un - u_c) - half * (a_c + as_) * (u_c - us)) * c.ih2[1]
                + c.bmb[0] * (ue - uw) * c.i2h[0] + c.bmb[1] * (un - us) * c.i2h[1];
            if (DIM == 3) {
                g += (half * (a_c + a_p) * (u_p - u_c) - half * (a_c + a_m) * (u_c - u_m)) * c.ih2[2]
                   + c.bmb[2] * (u_p - u_m) * c.i2h[2];
            }
            g += c.r0 + u_c * (c.r1 + u_c * (c.r2 + u_c * c.r3));
            T F = T(0);
            if (needF) {
                const T two = T(2);
                F = g + c.abar * ((ue - two * u_c + uw) * c.ih2[0] + (un - two * u_c + us) * c.ih2[1])
                      + c.beta[0] * (ue - uw) * c.i2h[0] + c.beta[1] * (un - us) * c.i2h[1];
                if (DIM == 3)
                    F += c.abar * (u_p - two * u_c + u_m) * c.ih2[2] + c.beta[2] * (u_p - u_m) * c.i2h[2];
            }
            const long long idx = zu + (long long)i2 * n1 + i1;
            T xv[kMaxExtra];
#pragma unroll
            for (int e = 0; e < kMaxExtra; ++e) xv[e] = (e < p.nx) ? p.X[e][idx] : T(0);
#pragma unroll
            for (int j = 0; j < kMaxOut; ++j) {
                if (j < p.nout) {
                    T v = c.cu[j] * u_c + c.cg[j] * g + c.cF[j] * F;
#pragma unroll
                    for (int e = 0; e < kMaxExtra; ++e) v += c.cx[j][e] * xv[e];
                    p.out[j][idx] = v;
                    outabs[j] = (float)absval(v);
                }
            }
        }
        // converged warp reduction (amax slots are uniform across the grid)
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j)
            if (j < p.nout && p.amax[j]) block_amax(outabs[j], p.amax[j]);
        if (DIM == 3) { u_m = u_c; u_c = u_p; a_m = a_c; a_c = a_p; }
    }
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
    dim3 grid((p.n1 + TX - 1) / TX, (p.n2 + TY - 1) / TY, p.dim == 3 ? (p.n3 + ZCHUNK - 1) / ZCHUNK : 1);
    if (p.dim == 3) stencil_kernel<T, 3><<<grid, block, 0, s>>>(p, c, needF);
    else            stencil_kernel<T, 2><<<grid, block, 0, s>>>(p, c, needF);
    return cudaGetLastError();
}

__global__ void convert_kernel(const double* in, float* out, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        out[i] = float(in[i]);
}

}  // namespace

cudaError_t launch_stencil(const StencilArgs<double>& a, cudaStream_t s) { return launch_impl(a, s); }
cudaError_t launch_stencil(const StencilArgs<float>& a, cudaStream_t s) { return launch_impl(a, s); }

cudaError_t launch_convert_f64_to_f32(const double* in, float* out, size_t n, cudaStream_t s) {
    const int blocks = int(std::min<size_t>((n + 255) / 256, 152 * 16));
    convert_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

}  // namespace adr
