// K1 on 3-D FP32 grids with Dirichlet faces: the z-marching stencil of stencil.cu with its planes
// staged in shared memory by TMA (cp.async.bulk.tensor) instead of loaded into registers.
//
// A CTA owns a tile of 64 x1 nodes x 16 x2 rows and walks zb planes of x3. One thread stages each
// plane of u (with its low part), of a and of the extra stage inputs into a ring of 4 to 6 slots,
// 2 to 4 planes beyond the one the current step needs, so the loads of several planes are in
// flight while a plane is computed: memory latency is covered by the ring, not by registers or
// warps. The staged planes of u and a carry a halo of one x2 row on each side and four x1 nodes
// (TMA copies start at x1 offsets that are multiples of 16 bytes); copies that reach past the grid
// read zeros, which are the Dirichlet ghosts of u, while a carries its own boundary ring. Every
// thread computes 4 consecutive x1 nodes of one row: the centre values of planes z - 1, z, z + 1
// rotate in registers (each plane's centre is read from shared memory once), the in-plane
// neighbours and the extra inputs come from the staged plane z (where slots with all three extra
// inputs and the low part would not fit, the extra inputs are read from global memory one plane
// ahead instead). The node
// arithmetic is that of stencil_core.cuh with the per-direction weights folded, and the results
// are stored with 16-byte stores.
//
// Bounded waits: a plane that does not arrive within the wait limit records an error code in the
// context's error word and ends the CTA (after waiting, again bounded, for its copies in flight).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "adr_internal.h"
#include "stencil_core.cuh"
#include "tc_common.cuh"

namespace adr {
namespace {
using namespace tc;

constexpr int kTX = 64;                                  // x1 nodes of a tile (16 threads x 4)
constexpr int kTY = 16;                                  // x2 rows of a tile
constexpr int kThreads = 256;
constexpr int kHX = kTX + 8;                             // staged row: 4 halo nodes on each side
constexpr int kHY = kTY + 2;                             // staged rows: 1 halo row on each side
constexpr uint32_t kPlaneBytes = kHX * kHY * 4;          // one staged plane of u, its low part or a
constexpr uint32_t kPlaneSlot = (kPlaneBytes + 127u) / 128u * 128u;
constexpr uint32_t kXBytes = kTX * kTY * 4;              // one staged plane of an extra input
constexpr uint32_t kCtaSmem = 75u * 1024u;               // shared memory of one of three CTAs per SM
constexpr int kMaxRing = 6;
constexpr int kErrStencilWait = 0x40;

struct StencilMaps {
    CUtensorMap u, lo, a, x[kMaxExtra];
};

// Slot layout and ring depth per variant: the extra stage inputs are staged with the plane (XS)
// wherever a ring of at least 3 slots of that size fits the shared memory of three CTAs per SM
// (otherwise they are read from global memory one plane ahead); the ring is as deep as that
// shared memory allows (each step keeps planes z and z + 1). With the low part the register cap
// of three CTAs spills a few values, which is still faster than two CTAs with a deeper ring.
template <bool HASLO, int NX>
struct SCfg {
    static constexpr bool XS = NX > 0 && (kCtaSmem - 256u) / ((HASLO ? 3 : 2) * kPlaneSlot + NX * kXBytes) >= 3;
    static constexpr uint32_t LO = 2 * kPlaneSlot;                       // offset of the low part
    static constexpr uint32_t XO = (HASLO ? 3 : 2) * kPlaneSlot;         // offset of the extra inputs
    static constexpr uint32_t SLOT = XO + (XS ? NX * kXBytes : 0u);
    static constexpr int FIT = int((kCtaSmem - 256u) / SLOT);
    static constexpr int RING = FIT < kMaxRing ? FIT : kMaxRing;
    static constexpr int AHEAD = RING - 2;                               // planes in flight beyond z + 1
    static_assert(RING >= 3, "ring");
    static constexpr uint32_t SMEM = RING * SLOT + 128;
    static_assert(RING <= kMaxRing, "barrier array");
};

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ float4 lds4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds1(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void f4a(float4 v, float (&o)[4]) {
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}

template <bool HASLO, bool NEEDF, bool ADELTA, int NX, int NOUT>
__global__ void __launch_bounds__(kThreads, 3) stencil_tma_kernel(const __grid_constant__ StencilMaps m, StencilArgs<float> p,
                                                               Coefs<float> c, int zb) {
    using C = SCfg<HASLO, NX>;
    constexpr int kRing = C::RING, kAhead = C::AHEAD;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kMaxRing];
    __shared__ volatile int abort_s;

    const uint32_t base = (static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw)) + 127u) & ~127u;
    const uint32_t bar0 = static_cast<uint32_t>(__cvta_generic_to_shared(&full[0]));
    const int n1 = p.n1, n2 = p.n2, n3 = p.n3;
    const int i1_0 = int(blockIdx.x) * kTX, i2_0 = int(blockIdx.y) * kTY;
    const int z0 = int(blockIdx.z) * zb, z1 = min(z0 + zb, n3);
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int i1 = i1_0 + 4 * tx, i2 = i2_0 + ty;
    const bool inside = (i1 < n1) && (i2 < n2);        // n1 % 4 == 0: all 4 nodes or none
    const int nplanes = z1 - z0 + 2;                    // staged planes z0 - 1 .. z1, index q = z - z0 + 1
    const long long plane_u = (long long)n1 * n2;
    const long long row_u = (long long)i2 * n1 + i1;

    if (t == 0) {
        for (int s = 0; s < kRing; ++s) mbar_init(bar0 + 8u * s, 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // thread 0: stage plane index q (plane z0 - 1 + q) into slot q mod kRing
    auto issue = [&](int q) {
        const int pz = z0 - 1 + q;
        const uint32_t slot = base + uint32_t(q % kRing) * C::SLOT;
        const uint32_t bar = bar0 + 8u * uint32_t(q % kRing);
        const bool withx = C::XS && pz >= z0 && pz < z1;
        mbar_arrive_expect_tx(bar, (HASLO ? 3u : 2u) * kPlaneBytes + (withx ? uint32_t(NX) * kXBytes : 0u));
        tma_load_3d(slot, &m.u, i1_0 - 4, i2_0 - 1, pz, bar);
        tma_load_3d(slot + kPlaneSlot, &m.a, i1_0, i2_0, pz + 1, bar);     // a: interior x1 at +4, x2 at +1
        if (HASLO) tma_load_3d(slot + C::LO, &m.lo, i1_0 - 4, i2_0 - 1, pz, bar);
        if (withx) {
#pragma unroll
            for (int e = 0; e < NX; ++e) tma_load_3d(slot + C::XO + e * kXBytes, &m.x[e], i1_0, i2_0, pz, bar);
        }
    };
    auto wait_plane = [&](int q) {
        return mbar_wait(bar0 + 8u * uint32_t(q % kRing), uint32_t(q / kRing) & 1u, p.err, kErrStencilWait, &abort_s);
    };

    int issued = 0;                                    // thread 0's count of staged planes
    if (t == 0) {
        for (; issued < nplanes && issued < kRing; ++issued) issue(issued);
    }
    // offset of the thread's 4 nodes in a staged plane (row ty + 1, column 4 + 4 tx)
    const uint32_t o = uint32_t(((ty + 1) * kHX + 4 + 4 * tx) * 4);
    const uint32_t ox = uint32_t((ty * kTX + 4 * tx) * 4);        // the same nodes in a staged extra input
    constexpr uint32_t kRow = kHX * 4;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    // planes z0 - 1 and z0 (index 0, 1): their centres go to registers
    bool ok = wait_plane(0);
    ok = wait_plane(1) && ok;
    float4 uM = zero4, uC = zero4, lM = zero4, lC = zero4, aM = zero4, aC = zero4;
    float4 xC[NX > 0 ? NX : 1], xP[NX > 0 ? NX : 1];
#pragma unroll
    for (int e = 0; e < (NX > 0 ? NX : 1); ++e) xC[e] = xP[e] = zero4;
    if (ok && inside) {
        const uint32_t s0 = base, s1 = base + C::SLOT;
        uM = lds4(s0 + o); aM = lds4(s0 + kPlaneSlot + o);
        uC = lds4(s1 + o); aC = lds4(s1 + kPlaneSlot + o);
        if (HASLO) { lM = lds4(s0 + C::LO + o); lC = lds4(s1 + C::LO + o); }
        if (!C::XS) {
#pragma unroll
            for (int e = 0; e < NX; ++e) xC[e] = *reinterpret_cast<const float4*>(p.X[e] + z0 * plane_u + row_u);
        }
    }
    // plane 0's slot is refilled in the first step: everyone has read it
    ok = !__syncthreads_or(!ok);
    int waited = ok ? 2 : 0;                           // planes every thread has waited for

    float outabs[NOUT];
#pragma unroll
    for (int j = 0; j < NOUT; ++j) outabs[j] = 0.f;
    float uabs = 0.f;

    // per-direction weights of the node arithmetic: w1 = (1/2)/h^2 on the face-sum form of the
    // diffusion, w2 = (b - beta)/(2h) on the centred advection, and for F the constant part
    // wa = abar/h^2, wb = beta/(2h)
    float w1[3], w2[3], wa[3], wb[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        w1[d] = 0.5f * c.ih2[d];
        w2[d] = c.bmb[d] * c.i2h[d];
        wa[d] = c.abar * c.ih2[d];
        wb[d] = c.beta[d] * c.i2h[d];
    }
    // slots of planes q and q + 1, and the barrier phase of plane q + 1, advanced step by step
    int slot_q = 1 % kRing, slot_n = 2 % kRing;
    uint32_t phase_n = uint32_t(2 / kRing) & 1u;

    for (int z = z0; ok && z < z1; ++z) {
        const int q = z - z0 + 1;
        // the slot of plane q + 1 + kAhead held plane q - 1, released by the barrier that ended
        // the previous step
        if (t == 0 && issued < nplanes && issued == q + 1 + kAhead) issue(issued++);
        const bool w = mbar_wait(bar0 + 8u * uint32_t(slot_n), phase_n, p.err, kErrStencilWait, &abort_s);
        ++waited;
        if (inside && w) {
            const uint32_t sC = base + uint32_t(slot_q) * C::SLOT;
            const uint32_t sP = base + uint32_t(slot_n) * C::SLOT;
            // next plane: centre values (staged); the extra inputs of this plane (staged), or of the
            // next one from global memory (used next step)
            const float4 uP = lds4(sP + o), aP = lds4(sP + kPlaneSlot + o);
            const float4 lP = HASLO ? lds4(sP + C::LO + o) : zero4;
            if (C::XS) {
#pragma unroll
                for (int e = 0; e < NX; ++e) xC[e] = lds4(sC + C::XO + e * kXBytes + ox);
            } else if (z + 1 < z1) {
#pragma unroll
                for (int e = 0; e < NX; ++e) xP[e] = *reinterpret_cast<const float4*>(p.X[e] + (z + 1) * plane_u + row_u);
            }
            // in-plane neighbours of plane z
            const float4 us = lds4(sC + o - kRow), un = lds4(sC + o + kRow);
            const float xw = lds1(sC + o - 4), xe = lds1(sC + o + 16);
            const float4 as4 = lds4(sC + kPlaneSlot + o - kRow), an4 = lds4(sC + kPlaneSlot + o + kRow);
            const float aw = lds1(sC + kPlaneSlot + o - 4), ae = lds1(sC + kPlaneSlot + o + 16);
            float4 ls4 = zero4, ln4 = zero4;
            float yw = 0.f, ye = 0.f;
            if (HASLO) {
                ls4 = lds4(sC + C::LO + o - kRow); ln4 = lds4(sC + C::LO + o + kRow);
                yw = lds1(sC + C::LO + o - 4); ye = lds1(sC + C::LO + o + 16);
            }
            float U[4], L[4], Aa[4], US[4], UN[4], LS[4], LN[4], AS[4], AN[4], UM[4], UP[4], LM[4], LP[4], AM[4], AP[4];
            f4a(uC, U); f4a(lC, L); f4a(aC, Aa);
            f4a(us, US); f4a(un, UN); f4a(ls4, LS); f4a(ln4, LN); f4a(as4, AS); f4a(an4, AN);
            f4a(uM, UM); f4a(uP, UP); f4a(lM, LM); f4a(lP, LP); f4a(aM, AM); f4a(aP, AP);
            const float UX[6] = {xw, U[0], U[1], U[2], U[3], xe}, LX[6] = {yw, L[0], L[1], L[2], L[3], ye};
            const float AX[6] = {aw, Aa[0], Aa[1], Aa[2], Aa[3], ae};
            float res[NOUT][4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float uk = U[k], ak = Aa[k];
                // one-sided differences (with the low part, the differences of the pairs)
                float dE = UX[k + 2] - uk, dW = uk - UX[k], dN = UN[k] - uk, dS = uk - US[k], dP = UP[k] - uk,
                      dM = uk - UM[k], uF = uk;
                if (HASLO) {
                    const float lk = L[k];
                    dE += LX[k + 2] - lk; dW += lk - LX[k]; dN += LN[k] - lk; dS += lk - LS[k];
                    dP += LP[k] - lk; dM += lk - LM[k]; uF += lk;
                }
                // face sums of (a - abar): 2 (a - abar)_C on every face in the a Lap u form
                const float sE = ADELTA ? ak + ak : ak + AX[k + 2], sW = ADELTA ? ak + ak : ak + AX[k];
                const float sN = ADELTA ? ak + ak : ak + AN[k], sS = ADELTA ? ak + ak : ak + AS[k];
                const float sP = ADELTA ? ak + ak : ak + AP[k], sM = ADELTA ? ak + ak : ak + AM[k];
                // g = sum_mu [w1 (s+ d+ - s- d-) + w2 (d+ + d-)] + r(u)
                float g = fmaf(uF, fmaf(uF, fmaf(uF, c.r3, c.r2), c.r1), c.r0);
                g = fmaf(w1[0], fmaf(-sW, dW, sE * dE), g);
                g = fmaf(w2[0], dE + dW, g);
                g = fmaf(w1[1], fmaf(-sS, dS, sN * dN), g);
                g = fmaf(w2[1], dN + dS, g);
                g = fmaf(w1[2], fmaf(-sM, dM, sP * dP), g);
                g = fmaf(w2[2], dP + dM, g);
                float F = 0.f;
                if (NEEDF) {          // F = g + A u: abar times the second differences, beta the first
                    F = fmaf(wa[0], dE - dW, g);
                    F = fmaf(wb[0], dE + dW, F);
                    F = fmaf(wa[1], dN - dS, F);
                    F = fmaf(wb[1], dN + dS, F);
                    F = fmaf(wa[2], dP - dM, F);
                    F = fmaf(wb[2], dP + dM, F);
                }
                uabs = fmaxf(uabs, fabsf(uF));
#pragma unroll
                for (int j = 0; j < NOUT; ++j) {
                    float v = fmaf(c.cg[j], g, c.cu[j] * uF);
                    if (NEEDF) v = fmaf(c.cF[j], F, v);
#pragma unroll
                    for (int e = 0; e < NX; ++e) {
                        float xe4[4];
                        f4a(xC[e], xe4);
                        v = fmaf(c.cx[j][e], xe4[k], v);
                    }
                    res[j][k] = v;
                }
            }
#pragma unroll
            for (int j = 0; j < NOUT; ++j) {
                *reinterpret_cast<float4*>(p.out[j] + z * plane_u + row_u) = make_float4(res[j][0], res[j][1], res[j][2], res[j][3]);
                outabs[j] = fmaxf(outabs[j], fmaxf(fmaxf(fabsf(res[j][0]), fabsf(res[j][1])), fmaxf(fabsf(res[j][2]), fabsf(res[j][3]))));
            }
            uM = uC; uC = uP; lM = lC; lC = lP; aM = aC; aC = aP;
            if (!C::XS) {
#pragma unroll
                for (int e = 0; e < NX; ++e) xC[e] = xP[e];
            }
        }
        slot_q = slot_n;
        if (++slot_n == kRing) {
            slot_n = 0;
            phase_n ^= 1u;
        }
        // every thread is done with plane q: its slot may be refilled (and a timed-out wait ends
        // the walk for the whole CTA)
        if (__syncthreads_or(!w)) break;
    }
    if (t == 0) {               // after an abort: wait (bounded) for the copies still in flight
        for (int q = waited; q < issued; ++q) {
            const long long t0 = clock64();
            while (!mbar_try_wait(bar0 + 8u * uint32_t(q % kRing), uint32_t(q / kRing) & 1u) &&
                   clock64() - t0 < kWaitCycles) {
            }
        }
    }
    if (p.amax_u) block_amax(uabs, p.amax_u);
#pragma unroll
    for (int j = 0; j < NOUT; ++j)
        if (p.amax[j]) block_amax(outabs[j], p.amax[j]);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return EncodeTiledFn(nullptr);
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// 3-D FP32 map over x[d2][d1][d0] (d0 contiguous, row pitch p0 elements) with a box of
// b0 x b1 x 1; reads outside the array return zeros.
bool encode3(CUtensorMap* m, const float* x, long long d0, long long p0, long long d1, long long d2, int b0, int b1) {
    const EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {cuuint64_t(d0), cuuint64_t(d1), cuuint64_t(d2)};
    cuuint64_t strides[2] = {cuuint64_t(p0 * 4), cuuint64_t(p0 * d1 * 4)};
    cuuint32_t box[3] = {cuuint32_t(b0), cuuint32_t(b1), 1u};
    cuuint32_t es[3] = {1u, 1u, 1u};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(x), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int g_sm_count = 0;

template <bool HASLO, bool NEEDF, bool ADELTA, int NX, int NOUT>
cudaError_t launch_variant(const StencilMaps& maps, const StencilArgs<float>& p, const Coefs<float>& c,
                           cudaStream_t s) {
    using C = SCfg<HASLO, NX>;
    static int occ = -1;                       // resident CTAs per SM of this variant
    if (occ < 0) {
        cudaError_t e = cudaFuncSetAttribute(stencil_tma_kernel<HASLO, NEEDF, ADELTA, NX, NOUT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM));
        if (e != cudaSuccess) return e;
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, stencil_tma_kernel<HASLO, NEEDF, ADELTA, NX, NOUT>, kThreads, C::SMEM);
        if (e != cudaSuccess) return e;
        occ = b > 0 ? b : 1;
    }
    const int gx = (p.n1 + kTX - 1) / kTX, gy = (p.n2 + kTY - 1) / kTY;
    // one wave: the x3 extent split so that every resident CTA slot holds one CTA
    int nz = (occ * g_sm_count) / (gx * gy);
    if (nz < 1) nz = 1;
    if (nz > p.n3) nz = p.n3;
    const int zb = (p.n3 + nz - 1) / nz;
    dim3 grid(unsigned(gx), unsigned(gy), unsigned((p.n3 + zb - 1) / zb));
    stencil_tma_kernel<HASLO, NEEDF, ADELTA, NX, NOUT><<<grid, kThreads, C::SMEM, s>>>(maps, p, c, zb);
    return cudaGetLastError();
}

template <bool HASLO, int NX>
cudaError_t launch_nout(const StencilMaps& maps, const StencilArgs<float>& p, const Coefs<float>& c, bool needF,
                        cudaStream_t s) {
    // the a Lap u form and F as compile-time choices: no per-node selects
    if (p.adelta) {
        if (needF) return p.nout == 1 ? launch_variant<HASLO, true, true, NX, 1>(maps, p, c, s)
                                      : launch_variant<HASLO, true, true, NX, 2>(maps, p, c, s);
        return p.nout == 1 ? launch_variant<HASLO, false, true, NX, 1>(maps, p, c, s)
                           : launch_variant<HASLO, false, true, NX, 2>(maps, p, c, s);
    }
    if (needF) return p.nout == 1 ? launch_variant<HASLO, true, false, NX, 1>(maps, p, c, s)
                                  : launch_variant<HASLO, true, false, NX, 2>(maps, p, c, s);
    return p.nout == 1 ? launch_variant<HASLO, false, false, NX, 1>(maps, p, c, s)
                       : launch_variant<HASLO, false, false, NX, 2>(maps, p, c, s);
}

template <bool HASLO>
cudaError_t launch_nx(const StencilMaps& maps, const StencilArgs<float>& p, const Coefs<float>& c, bool needF,
                      cudaStream_t s) {
    switch (p.nx) {
    case 0: return launch_nout<HASLO, 0>(maps, p, c, needF, s);
    case 1: return launch_nout<HASLO, 1>(maps, p, c, needF, s);
    case 2: return launch_nout<HASLO, 2>(maps, p, c, needF, s);
    default: return launch_nout<HASLO, 3>(maps, p, c, needF, s);
    }
}

bool aligned16(const void* x) { return reinterpret_cast<uintptr_t>(x) % 16 == 0; }

}  // namespace

bool stencil_tma_usable(const StencilArgs<float>& p) {
    if (p.dim != 3 || p.neumann || p.n1 % 4 != 0 || p.apitch % 4 != 0) return false;
    if (p.n1 < kTX || p.n2 < kTY || p.n3 < 2) return false;        // boxes no larger than the grid
    if (p.nout < 1 || p.nout > kMaxOut || p.nx < 0 || p.nx > kMaxExtra) return false;
    if (!aligned16(p.u) || !aligned16(p.a) || (p.u_lo && !aligned16(p.u_lo))) return false;
    for (int e = 0; e < p.nx; ++e)
        if (!aligned16(p.X[e])) return false;
    for (int j = 0; j < p.nout; ++j)
        if (!aligned16(p.out[j])) return false;
    return encode_fn() != nullptr;
}

cudaError_t launch_stencil_tma(const StencilArgs<float>& p, const Coefs<float>& c, bool needF, cudaStream_t s) {
    if (!stencil_tma_usable(p)) return cudaErrorInvalidValue;
    if (g_sm_count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    }
    StencilMaps maps;
    const long long n1 = p.n1, n2 = p.n2, n3 = p.n3;
    bool ok = encode3(&maps.u, p.u, n1, n1, n2, n3, kHX, kHY) &&
              encode3(&maps.a, p.a, p.apitch, p.apitch, n2 + 2, n3 + 2, kHX, kHY);
    maps.lo = maps.u;
    if (ok && p.u_lo) ok = encode3(&maps.lo, p.u_lo, n1, n1, n2, n3, kHX, kHY);
    for (int e = 0; e < kMaxExtra; ++e) maps.x[e] = maps.u;
    for (int e = 0; ok && e < p.nx; ++e) ok = encode3(&maps.x[e], p.X[e], n1, n1, n2, n3, kTX, kTY);
    if (!ok) return cudaErrorInvalidValue;
    return p.u_lo ? launch_nx<true>(maps, p, c, needF, s) : launch_nx<false>(maps, p, c, needF, s);
}

}  // namespace adr
