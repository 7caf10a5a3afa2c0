// K2 (tensor cores), TMA-fed form of the mixed-precision mu-mode contraction. Same
// exact-slice arithmetic as contract_tc.cu (see there); what changes is how the FP32 state
// reaches the slicers and how shared memory is spent:
//   * a loader thread brings FP32 state tiles with cp.async.bulk.tensor (TMA) into a
//     staging ring several chunks ahead, so the producer warps only slice shared -> shared;
//   * K chunks of 32 with the 64-byte swizzle halve every slice tile, which leaves room for
//     N = 128 output columns in the precise configuration too (no re-slicing of a state
//     tile per 64 outputs; the precise form keeps one TMEM accumulator set of 4 x 128).
// Used when the x1 extent is a multiple of 4 and the arrays are 16-byte aligned (TMA
// stride and address rules); other shapes use contract_tc.cu.
//
// Tiles. Modes >= 2 (state is A): a position tile is 128 consecutive q of one p (the state
// seen as [P][n][Q]); mode 1 (state is B): 128 consecutive fibres. Output tiles are 128 rows
// of the factor. Warps: 0-7 producers, then 8 (16 with the low part) epilogue warps, the MMA
// issuer and the TMA and factor loader.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "adr_internal.h"
#include "phi_device.cuh"
#include "tc_common.cuh"

namespace adr {
namespace {
using namespace tc;

constexpr int kM = 128;          // UMMA M, TMEM lanes
constexpr int kN = 128;          // UMMA N
constexpr int kKc = 32;          // K per stage: one 64-byte bf16 row (64-byte swizzle)
constexpr int kProducerWarps = 8;
constexpr int kEpiWarp0 = 8;      // epilogue warps from 8: their TMEM lane quarter is warp % 4
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kN >> 3) << 17) | (uint32_t(kM >> 4) << 24);
constexpr uint32_t kIdesc2 = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t((2 * kN) >> 3) << 17) |
                           (uint32_t(kM >> 4) << 24);   // N = 256

// Every pass: four slices of the state and of the factor, ten products into four accumulators,
//     D0 = S0.F0,  D1 = S0.F1 + S1.F0,  D2 = S0.F2 + S1.F1 + S2.F0,
//     D3 = S0.F3 + S1.F2 + S2.F1 + S3.F0,
// integer terms of magnitude at most 2^14. For K <= 256 all four stay within 2^24 even in the
// worst case (D0 and D1 for K <= 512), so they are exact whatever rounding the tensor cores
// apply; beyond that D2 and D3 could pass 2^24 only if hundreds of residual-slice products
// shared the largest magnitude and one sign, and their rounding would weigh 2^-16 and 2^-24 of
// a unit of D0. x.f = D0 + 2^-8 D1 + 2^-16 D2 + 2^-24 D3 up to the products below 2^-32,
// combined once in the epilogue. A time integration applies the same factor to a
// slowly varying state in every step, so any bias of a pass adds up. Measured on the 40-step
// 256^3 Lawson4 run (relative error and mean drift against the FP64 path): six products into
// two accumulators 1.5e-6 / -1.0e-6; seven into three exact accumulators with a 32-bit factor
// but without the 2^-24 cross products S1.F2, S2.F1, S3.F0 2.8e-6 / -1.7e-6; all ten 2.6e-7 /
// +1e-9. PR: the input and the output carry a low part (double-float), for the one exponential
// whose result feeds the stencil that no later exponential smooths.
template <bool PR>
struct Cfg {
    static constexpr int SS = 4;                       // state slices
    static constexpr int FS = 4;                       // factor slices
    static constexpr int NACC = 4;                     // accumulators (128 columns each)
    static constexpr int NSETS = 1;                    // TMEM accumulator sets
    static constexpr int TILE = kM * kKc * 2;          // one bf16 slice tile: 8 KB
    static constexpr int SBYTES = SS * TILE;           // one state-slice stage (32 KB)
    static constexpr int FBYTES = FS * TILE;           // one factor stage (32 KB)
    static constexpr int NSLICE = PR ? 2 : 3;          // state-slice ring
    static constexpr int NF = 3;                       // factor ring (the loader runs it ahead)
    static constexpr int XTILE = kM * kKc * 4;         // one FP32 staging tile: 16 KB
    static constexpr int XSTAGE = PR ? 2 * XTILE : XTILE;   // hi (+ lo)
    static constexpr int NX = 2;
    static constexpr int SMEM = NSLICE * SBYTES + NF * FBYTES + NX * XSTAGE + 1024;
    // warps: producers 0-7, then the epilogue (two per TMEM lane quarter, each half the columns;
    // four per quarter in the double-float configuration, whose epilogue is the longer), the MMA
    // issuer and the loader
    static constexpr int EPIW = PR ? 16 : 8;
    static constexpr int MMAW = kEpiWarp0 + EPIW;
    static constexpr int LOADW = MMAW + 1;
    static constexpr int THREADS = (LOADW + 1) * 32;
    static constexpr int COLS = kN / (EPIW / 4);           // columns per epilogue warp
    static_assert(NACC * kN * NSETS <= 512, "TMEM");
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld8x4(uint32_t t0, uint32_t stride, float (&d)[4][8]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%33];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%34];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%35];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(t0), "r"(t0 + stride), "r"(t0 + 2 * stride), "r"(t0 + 3 * stride)
        : "memory");
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 8; ++j) d[k][j] = __uint_as_float(r[8 * k + j]);
}

// Integer slices of y (+ ylo); see split<> in contract_tc.cu.
template <bool PR>
__device__ __forceinline__ void split(float y, float ylo, uint32_t (&b)[4]) {
    const float s0 = rintf(y);
    const float r0 = PR ? (y - s0) + ylo : (y - s0);
    const float y1 = r0 * 256.f;
    const float s1 = rintf(y1);
    const float y2 = (y1 - s1) * 256.f;
    const float s2 = rintf(y2);
    b[0] = __float_as_uint(s0);
    b[1] = __float_as_uint(s1);
    b[2] = __float_as_uint(s2);
    b[3] = __float_as_uint(rintf((y2 - s2) * 256.f));
}

// Slice 8 values (+ low parts) and store them as 16-byte chunk j of row r of the SS tiles.
template <bool PR>
__device__ __forceinline__ void slice_store8(const float (&v)[8], const float (&vl)[8], float sc, uint32_t tile0, int r,
                                             int j) {
    constexpr int SS = 4;
    uint32_t w[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        uint32_t a[4], c[4];
        split<PR>(v[2 * e] * sc, vl[2 * e] * sc, a);
        split<PR>(v[2 * e + 1] * sc, vl[2 * e + 1] * sc, c);
#pragma unroll
        for (int q = 0; q < SS; ++q) w[q][e] = __byte_perm(a[q], c[q], 0x7632);
    }
    const uint32_t off = swz64(r, j);
#pragma unroll
    for (int q = 0; q < SS; ++q)
        st_shared_v4(tile0 + q * (kM * kKc * 2) + off, make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]));
}

__device__ __forceinline__ float lds(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float4 lds4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// One K step of 16 of the ten products. With X the slices of the A operand and Y those of the
// B operand (X = S, Y = F for modes >= 2; the other way for mode 1), X_i.Y_j goes to D_(i+j).
// The accumulators D0..D3 sit in consecutive 128-column blocks of TMEM and the Y slices in
// consecutive shared-memory tiles, so X_i.[Y_j ; Y_(j+1)] as one N = 256 product adds
// X_i.Y_j to D_(i+j) and X_i.Y_(j+1) to D_(i+j+1): six MMAs (four of N = 256, two of N = 128)
// instead of ten of N = 128, the same tensor work with a fifth less operand traffic from
// shared memory (12 KB per 128 columns x 256 rows instead of 16 KB).
template <bool SA>
__device__ __forceinline__ void mma_kstep(uint32_t d, const uint64_t (&S)[4], const uint64_t (&F)[4], uint64_t adv,
                                          uint32_t first) {
    const uint64_t(&X)[4] = SA ? S : F;
    const uint64_t(&Y)[4] = SA ? F : S;
    auto mma = [&](uint32_t col, int xi, int yj, uint32_t idesc, uint32_t accumulate) {
        tc_mma(d + col, X[xi] + adv, Y[yj] + adv, idesc, accumulate);
    };
    const uint32_t acc = first ? 0u : 1u;
    mma(0 * kN, 0, 0, kIdesc2, acc);     // D0 += X0.Y0, D1 += X0.Y1
    mma(2 * kN, 0, 2, kIdesc2, acc);     // D2 += X0.Y2, D3 += X0.Y3
    mma(1 * kN, 1, 0, kIdesc2, 1u);      // D1 += X1.Y0, D2 += X1.Y1
    mma(3 * kN, 1, 2, kIdesc, 1u);       // D3 += X1.Y2
    mma(2 * kN, 2, 0, kIdesc2, 1u);      // D2 += X2.Y0, D3 += X2.Y1
    mma(3 * kN, 3, 0, kIdesc, 1u);       // D3 += X3.Y0
}

template <bool SA, bool PR, int EPI>
__global__ void __launch_bounds__(Cfg<PR>::THREADS, 1) tma_contract_kernel(const __grid_constant__ TmaArgs p) {
    using C = Cfg<PR>;
    extern __shared__ uint8_t smem_raw[];
    // barriers: xfull[NX] xempty[NX] sfull[NSLICE] sempty[NSLICE] ffull[NF] fempty[NF] accf[2] acce[2] drain
    constexpr uint32_t kXF = 0, kXE = kXF + 8 * C::NX, kSF = kXE + 8 * C::NX, kSE = kSF + 8 * C::NSLICE;
    constexpr uint32_t kFF = kSE + 8 * C::NSLICE, kFE = kFF + 8 * C::NF, kAF = kFE + 8 * C::NF, kAE = kAF + 16;
    constexpr uint32_t kDR = kAE + 16;
    __shared__ __align__(8) uint64_t bars[kDR / 8 + 1];
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;   // state-slice ring
    const uint32_t fbase = sbase + C::NSLICE * C::SBYTES;             // factor ring
    const uint32_t xbase = fbase + C::NF * C::FBYTES;                 // FP32 staging ring
    const uint32_t bar0 = smem_u32(&bars[0]);
    auto xfull = [&](int s) { return bar0 + kXF + 8u * s; };
    auto xempty = [&](int s) { return bar0 + kXE + 8u * s; };
    auto sfull = [&](int s) { return bar0 + kSF + 8u * s; };
    auto sempty = [&](int s) { return bar0 + kSE + 8u * s; };
    auto ffull = [&](int s) { return bar0 + kFF + 8u * s; };
    auto fempty = [&](int s) { return bar0 + kFE + 8u * s; };
    auto accf = [&](int a) { return bar0 + kAF + 8u * a; };
    auto acce = [&](int a) { return bar0 + kAE + 8u * a; };
    const uint32_t drain_bar = bar0 + kDR;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::NX; ++s) {
            mbar_init(xfull(s), 1);                         // loader's expect_tx arrival
            mbar_init(xempty(s), kProducerWarps);           // one arrival per producer warp
        }
        for (int s = 0; s < C::NSLICE; ++s) {
            mbar_init(sfull(s), kProducerWarps);            // one arrival per producer warp
            mbar_init(sempty(s), 1);                        // tcgen05.commit
        }
        for (int s = 0; s < C::NF; ++s) {
            mbar_init(ffull(s), 1);                         // loader's expect_tx arrival
            mbar_init(fempty(s), 1);                        // tcgen05.commit
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf(a), 1);
            mbar_init(acce(a), C::EPIW);                    // one arrival per epilogue warp
        }
        mbar_init(drain_bar, 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == C::MMAW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    const float amax = __uint_as_float(*p.amax_in);
    int es = 0;
    if (amax > 0.f) frexpf(amax, &es);
    const float sc = ldexpf(1.f, 7 - es);
    const float sback = ldexpf(1.f, es - 7);
    const int n = p.n;
    const long long Q = p.Q;
    const long long my_tiles = (p.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const long long items = my_tiles * p.nK;

    // tile -> (position tile, output tile); position tile -> (p, q0) or fibre f0
    auto tile_of = [&](long long it) { return blockIdx.x + (it / p.nK) * gridDim.x; };

    if (warp == C::LOADW) {
        // ------------------------------------------------------------ TMA loader
        // Lane 0 fills the factor ring (pre-sliced factor tiles, consumed directly by the MMA;
        // the slot of item i frees when the MMA of item i - NF retires, so each copy has NF - 1
        // chunks of lead time), lane 1 the FP32 staging ring (state tiles for the producers),
        // each at its own pace: a wait on one ring does not hold back the other.
        if (lane < 2) {
            for (long long it = 0; it < items && !abort_s; ++it) {
                const long long tile = tile_of(it);
                if (lane == 0) {
                    const int s = int(it % C::NF);
                    const uint32_t ph = uint32_t(it / C::NF) & 1u;
                    if (!mbar_wait(fempty(s), ph ^ 1u, p.err, 64, &abort_s, 32)) break;
                    mbar_arrive_expect_tx(ffull(s), C::FBYTES);
                    const uint8_t* src = p.fimg + (size_t(tile % p.nOut) * p.nK + it % p.nK) * C::FBYTES;
                    const uint32_t dst = fbase + s * C::FBYTES;
#pragma unroll
                    bulk_g2s(dst, src, C::FBYTES, ffull(s));
                }
                if (lane == 1) {
                    const int s = int(it % C::NX);
                    const uint32_t ph = uint32_t(it / C::NX) & 1u;
                    if (!mbar_wait(xempty(s), ph ^ 1u, p.err, 16, &abort_s, 32)) break;
                    const long long pt = tile / p.nOut;
                    const int k0 = int(it % p.nK) * kKc;
                    const uint32_t dst = xbase + s * C::XSTAGE;
                    const bool lo = PR && p.has_lo;
                    mbar_arrive_expect_tx(xfull(s), lo ? 2 * C::XTILE : C::XTILE);
                    if (SA) {
                        const int pidx = int(pt / p.nqt), q0 = int(pt % p.nqt) * kM;
                        tma_load_3d(dst, &p.map_x, q0, k0, pidx, xfull(s));
                        if (lo) tma_load_3d(dst + C::XTILE, &p.map_xlo, q0, k0, pidx, xfull(s));
                    } else {
                        const int f0 = int(pt * kN);
                        tma_load_2d(dst, &p.map_x, k0, f0, xfull(s));
                        if (lo) tma_load_2d(dst + C::XTILE, &p.map_xlo, k0, f0, xfull(s));
                    }
                }
            }
        }
    } else if (warp < kProducerWarps) {
        // ------------------------------------------------------------ producers (shared -> shared)
        const int t = threadIdx.x;
        for (long long it = 0; it < items; ++it) {
            const int ss = int(it % C::NSLICE);
            const uint32_t sph = uint32_t(it / C::NSLICE) & 1u;
            // waits decide warp-uniformly: the per-warp arrivals below need every lane
            if (!__all_sync(0xffffffffu, mbar_wait(sempty(ss), sph ^ 1u, p.err, 1, &abort_s, 32))) break;
            const uint32_t sA = sbase + ss * C::SBYTES;
            const int xs = int(it % C::NX);
            const uint32_t xph = uint32_t(it / C::NX) & 1u;
            if (!__all_sync(0xffffffffu, mbar_wait(xfull(xs), xph, p.err, 32, &abort_s))) break;
            const uint32_t xt = xbase + xs * C::XSTAGE;
            float v[2][8], vl[2][8];
            if (SA) {
                // staging tile [k][q] (32 rows of 128 floats); thread: position row, 16 K values
                const int row = t & (kM - 1), half = t >> 7;
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const uint32_t a = xt + uint32_t(((16 * half + 8 * h + e) * kM + row) * 4);
                        v[h][e] = lds(a);
                        vl[h][e] = (PR && p.has_lo) ? lds(a + C::XTILE) : 0.f;
                    }
            } else {
                // staging tile [f][k] (128 rows of 32 floats); thread: chunk j of rows r0, r0 + 64
                const int j = t & 3, r0 = t >> 2;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t a = xt + uint32_t(((r0 + 64 * h) * kKc + 8 * j) * 4);
                    const float4 x0 = lds4(a), x1 = lds4(a + 16);
                    v[h][0] = x0.x; v[h][1] = x0.y; v[h][2] = x0.z; v[h][3] = x0.w;
                    v[h][4] = x1.x; v[h][5] = x1.y; v[h][6] = x1.z; v[h][7] = x1.w;
                    if (PR && p.has_lo) {
                        const float4 y0 = lds4(a + C::XTILE), y1 = lds4(a + C::XTILE + 16);
                        vl[h][0] = y0.x; vl[h][1] = y0.y; vl[h][2] = y0.z; vl[h][3] = y0.w;
                        vl[h][4] = y1.x; vl[h][5] = y1.y; vl[h][6] = y1.z; vl[h][7] = y1.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) vl[h][e] = 0.f;
                    }
                }
            }
            // the staging tile may be refilled: one arrival per warp once every lane has read
            // (256 single-thread arrivals on one barrier word serialise for ~1000 cycles)
            __syncwarp();
            if (lane == 0) mbar_arrive(xempty(xs));
            if (SA) {
                const int row = t & (kM - 1), half = t >> 7;
                slice_store8<PR>(v[0], vl[0], sc, sA, row, 2 * half);
                slice_store8<PR>(v[1], vl[1], sc, sA, row, 2 * half + 1);
            } else {
                const int j = t & 3, r0 = t >> 2;
                slice_store8<PR>(v[0], vl[0], sc, sA, r0, j);
                slice_store8<PR>(v[1], vl[1], sc, sA, r0 + 64, j);
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(sfull(ss));
        }
    } else if (warp < kEpiWarp0 + C::EPIW) {
        // ------------------------------------------------------------ epilogue
        const int ew = (warp - kEpiWarp0) & 3;          // TMEM lane quarter (warp % 4)
        const int part = (warp - kEpiWarp0) >> 2;       // column part
        const int row = ew * 32 + lane;
        long long tl = 0;
        for (long long tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x, ++tl) {
            const int a = int(tl % C::NSETS);
            const uint32_t ph = uint32_t(tl / C::NSETS) & 1u;
            const bool waited = mbar_wait(accf(a), ph, p.err, 2, &abort_s, 64);
            if (!__all_sync(0xffffffffu, waited)) break;
            tc_fence_after();
            const long long pt = tile / p.nOut;
            const int ot = int(tile % p.nOut);
            float vmax = 0.f;
            bool rvalid;
            long long off0, cstep;
            float zrow = 0.f, rscale = 0.f;
            int ncol;
            if (SA) {
                const long long pp = pt / p.nqt, qq = (pt % p.nqt) * kM + row;
                rvalid = qq < Q;
                off0 = (pp * n + ot * kN) * Q + qq;
                cstep = Q;
                ncol = min(kN, n - ot * kN);
                if (EPI == EPI_PHI && rvalid) {
                    zrow = __ldg(p.zq_a + qq % p.na);
                    if (p.zq_b) zrow += __ldg(p.zq_b + qq / p.na);
                    if (p.zp) zrow += __ldg(p.zp + pp);
                }
            } else {
                const int irow = ot * kM + row;
                rvalid = irow < n;
                if (rvalid) rscale = sback * __ldg(p.fscale + irow);
                off0 = pt * kN * (long long)n + irow;
                cstep = n;
                ncol = int(min((long long)kN, p.npos - pt * kN));
            }
            const float* fsc = p.fscale + ot * kN;
            const float* zc = p.zmu + ot * kN;
            float* yrow = p.Y + off0;
            float* ylo = (EPI == EPI_STORE2) ? p.Ylo + off0 : nullptr;
            const float* brow = (EPI == EPI_AXPY) ? p.base + off0 : nullptr;
            const uint32_t tbase = tmem + (uint32_t(ew * 32) << 16) + uint32_t(a) * 256u;
            auto emit = [&](int col, float hi, float lo, float bval, float scale) {
                const long long o = (long long)col * cstep;
                if (EPI == EPI_STORE2) {
                    yrow[o] = hi * scale;
                    ylo[o] = lo * scale;
                    vmax = fmaxf(vmax, fabsf(hi * scale));
                    return;
                }
                float v = (hi + lo) * scale;
                if (EPI == EPI_PHI) v *= phi_eval(p.phik, zrow + __ldg(zc + col));
                if (EPI == EPI_AXPY) v = fmaf(p.alpha, v, bval);
                yrow[o] = v;
                vmax = fmaxf(vmax, fabsf(v));
            };
            // the axpy's base values of the next 8 columns are loaded while the current ones are
            // combined, so their latency does not add to every group
            auto load_base = [&](int j0, float (&b)[8]) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    b[j] = (EPI == EPI_AXPY && rvalid && j0 + j < ncol) ? __ldg(brow + (long long)(j0 + j) * cstep) : 0.f;
            };
            const int jlo = part * C::COLS, jhi = jlo + C::COLS;
            float bcur[8], bnxt[8];
            load_base(jlo, bcur);
#pragma unroll 1
            for (int j0 = jlo; j0 < jhi; j0 += 8) {
                float d[4][8];
                if (j0 + 8 < jhi) load_base(j0 + 8, bnxt);
                __syncwarp();
                tmem_ld8x4(tbase + j0, uint32_t(kN), d);
                if (j0 + 8 >= jhi) {       // the last columns are in registers: TMEM is free
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(acce(a));
                }
                // the column scales of the group (the factor's row scales, padded to whole tiles)
                float scl8[8];
                if (SA) {
                    const float4 s0 = __ldg(reinterpret_cast<const float4*>(fsc + j0));
                    const float4 s1 = __ldg(reinterpret_cast<const float4*>(fsc + j0 + 4));
                    scl8[0] = sback * s0.x; scl8[1] = sback * s0.y; scl8[2] = sback * s0.z; scl8[3] = sback * s0.w;
                    scl8[4] = sback * s1.x; scl8[5] = sback * s1.y; scl8[6] = sback * s1.z; scl8[7] = sback * s1.w;
                }
                auto combine = [&](int j) {
                    const float tail = fmaf(d[3][j], 5.9604644775390625e-08f, d[2][j] * 1.52587890625e-05f);
                    if (EPI == EPI_STORE2) {     // double-float result: D0 + 2^-8 D1 exactly, then the tail
                        float hi, lo;
                        two_sum(d[0][j], d[1][j] * 0.00390625f, hi, lo);
                        lo += tail;
                        const float s = hi + lo;
                        emit(j0 + j, s, lo - (s - hi), bcur[j], SA ? scl8[j] : rscale);
                    } else {                     // one FP32 result: the smaller terms first, D0 last
                        emit(j0 + j, d[0][j] + fmaf(d[1][j], 0.00390625f, tail), 0.f, bcur[j], SA ? scl8[j] : rscale);
                    }
                };
                if (rvalid && j0 + 8 <= ncol) {    // a whole group: no per-column branches
#pragma unroll
                    for (int j = 0; j < 8; ++j) combine(j);
                } else if (rvalid) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j0 + j < ncol) combine(j);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) bcur[j] = bnxt[j];
            }
            for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
            if (lane == 0 && p.amax_out && vmax > 0.f) atomicMax(p.amax_out, __float_as_uint(vmax));
        }
    } else if (warp == C::MMAW && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        long long g = 0, tl = 0;
        for (long long tile = blockIdx.x; tile < p.ntiles && !abort_s; tile += gridDim.x, ++tl) {
            const int a = int(tl % C::NSETS);
            const uint32_t aph = uint32_t(tl / C::NSETS) & 1u;
            if (!mbar_wait(acce(a), aph ^ 1u, p.err, 4, &abort_s)) break;
            tc_fence_after();
            const uint32_t d = tmem + uint32_t(a) * 256u;
            bool ok = true;
            for (int c = 0; c < p.nK; ++c, ++g) {
                const int s = int(g % C::NSLICE);
                const uint32_t ph = uint32_t(g / C::NSLICE) & 1u;
                const int fs = int(g % C::NF);
                const uint32_t fph = uint32_t(g / C::NF) & 1u;
                if (!mbar_wait(ffull(fs), fph, p.err, 128, &abort_s)) { ok = false; break; }
                if (!mbar_wait(sfull(s), ph, p.err, 8, &abort_s)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sS = sbase + s * C::SBYTES;
                const uint32_t sF = fbase + fs * C::FBYTES;
                uint64_t S[4], F[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    S[q] = sdesc64(sS + (q < C::SS ? q : 0) * C::TILE);
                    F[q] = sdesc64(sF + (q < C::FS ? q : 0) * C::TILE);
                }
#pragma unroll
                for (int kk = 0; kk < kKc / 16; ++kk)
                    mma_kstep<SA>(d, S, F, uint64_t(kk * 32) >> 4, (c == 0 && kk == 0) ? 1u : 0u);
                tc_commit(sempty(s));
                tc_commit(fempty(fs));
            }
            if (!ok) break;
            tc_commit(accf(a));
        }
        tc_commit(drain_bar);
        const long long t0 = clock64();
        while (!mbar_try_wait(drain_bar, 0) && clock64() - t0 < kWaitCycles) {}
    }

    tc_fence_before();
    __syncthreads();
    if (warp == C::MMAW) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

int g_sms = 0;

template <bool SA, bool PR, int EPI>
cudaError_t launch_variant(const TmaArgs& a, unsigned grid, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tma_contract_kernel<SA, PR, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Cfg<PR>::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    tma_contract_kernel<SA, PR, EPI><<<grid, Cfg<PR>::THREADS, Cfg<PR>::SMEM, s>>>(a);
    return cudaGetLastError();
}

// FP32 tensor map over the state seen as [P][n][Q] (modes >= 2; box 128 q x 32 k x 1 p) or
// as [P][n] rows of n (mode 1; box 32 k x 128 fibres).
// cuTensorMapEncodeTiled is a driver-API call; the library takes it through the runtime's
// driver entry-point query so that it does not link libcuda itself and still loads (for
// symbol checks) on a machine without a GPU driver.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn() {
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

bool encode_map(CUtensorMap* m, const float* x, bool state_is_a, long long n, long long Q, long long P) {
    if (!x) return true;
    const EncodeTiledFn cuTensorMapEncodeTiled = encode_tiled_fn();
    if (!cuTensorMapEncodeTiled) return false;
    CUresult r;
    if (state_is_a) {
        cuuint64_t dims[3] = {cuuint64_t(Q), cuuint64_t(n), cuuint64_t(P)};
        cuuint64_t strides[2] = {cuuint64_t(Q * 4), cuuint64_t(n * Q * 4)};
        cuuint32_t box[3] = {cuuint32_t(kM), cuuint32_t(kKc), 1u};
        cuuint32_t es[3] = {1u, 1u, 1u};
        r = cuTensorMapEncodeTiled(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(x), dims, strides, box, es,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        cuuint64_t dims[2] = {cuuint64_t(n), cuuint64_t(P)};
        cuuint64_t strides[1] = {cuuint64_t(n * 4)};
        cuuint32_t box[2] = {cuuint32_t(kKc), cuuint32_t(kN)};
        cuuint32_t es[2] = {1u, 1u};
        r = cuTensorMapEncodeTiled(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(x), dims, strides, box, es,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS;
}

}  // namespace

bool tma_supported(int n, long long Q, const void* x, const void* xlo) {
    // TMA: 16-byte aligned base addresses and row strides (Q * 4 or n * 4 bytes)
    if (reinterpret_cast<uintptr_t>(x) % 16 != 0) return false;
    if (xlo && reinterpret_cast<uintptr_t>(xlo) % 16 != 0) return false;
    if (Q == 1) return n % 4 == 0;
    return Q % 4 == 0;
}

cudaError_t launch_contract_tma(TmaArgs a, long long P, cudaStream_t s) {
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (a.n > 512 || a.n < 1) return cudaErrorInvalidValue;
    if (!encode_map(&a.map_x, a.X, a.state_is_a, a.n, a.Q, P)) return cudaErrorInvalidValue;
    a.has_lo = a.precise && a.Xlo != nullptr;
    if (a.has_lo && !encode_map(&a.map_xlo, a.Xlo, a.state_is_a, a.n, a.Q, P)) return cudaErrorInvalidValue;
    const long long grid = a.ntiles < g_sms ? a.ntiles : g_sms;
    if (grid <= 0) return cudaSuccess;
    const unsigned g = unsigned(grid);
    if (a.precise) {
        if (a.epi != EPI_STORE2 && a.epi != EPI_STORE) return cudaErrorInvalidValue;
        if (a.state_is_a) return a.epi == EPI_STORE2 ? launch_variant<true, true, EPI_STORE2>(a, g, s)
                                                     : launch_variant<true, true, EPI_STORE>(a, g, s);
        return a.epi == EPI_STORE2 ? launch_variant<false, true, EPI_STORE2>(a, g, s)
                                   : launch_variant<false, true, EPI_STORE>(a, g, s);
    }
    if (a.state_is_a) {
        if (a.epi == EPI_PHI) return launch_variant<true, false, EPI_PHI>(a, g, s);
        if (a.epi == EPI_AXPY) return launch_variant<true, false, EPI_AXPY>(a, g, s);
        if (a.epi == EPI_STORE2) return launch_variant<true, false, EPI_STORE2>(a, g, s);
        return launch_variant<true, false, EPI_STORE>(a, g, s);
    }
    if (a.epi == EPI_PHI || a.epi == EPI_STORE2) return cudaErrorInvalidValue;
    if (a.epi == EPI_AXPY) return launch_variant<false, false, EPI_AXPY>(a, g, s);
    return launch_variant<false, false, EPI_STORE>(a, g, s);
}

}  // namespace adr
