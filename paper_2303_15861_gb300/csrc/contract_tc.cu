// K2 (tensor cores): mu-mode contraction Y = X x_mu M of the mixed-precision path on the
// 5th-generation tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32 accumulators
// in TMEM), with the pointwise phi_k scaling (K3) and the stage axpy (K4) fused into the
// epilogue. The mu-mode product is the one of Section 1 / Section 5.2:
// e^{A_d (+) ... (+) A_1} v = vec(V x_1 e^{A_1} x_2 ... x_d e^{A_d}).
//
// Exact-slice split. The FP32 state x gets one power-of-two scale 2^es from the max-abs
// that its producing kernel recorded; each row i of the FP64 factor (output index) gets
// its own scale 2^e_i. With integer slices |s_j|, |f_j| <= 128 (exact in BF16):
//     x = 2^(es-7) (s0 + 2^-8 s1 + 2^-16 s2),   f = 2^(e_i-7) (f0 + 2^-8 f1 + 2^-16 f2),
//     sum_k x f = 2^(es+e_i-14) (D0 + 2^-8 D1),
//     D0 = S0.F0,  D1 = S0.F1 + S1.F0 + S0.F2' + S2'.F0 + S1.F1'    (six MMAs per K step;
//     the library runs the precise configuration below instead)
// with F1' = 2^-8 F1, F2' = 2^-8 F2, S2' = 2^-8 S2 (exact scalings). Every term of D0 is
// an integer of magnitude < 2^14 and |D0| < 2^24 for K <= 512, so D0 is exact in the FP32
// accumulator whatever rounding the tensor core applies: the dominant, same-signed part
// of a heat-kernel product carries no accumulation bias. D1 is weighted 2^-8 and its
// terms have random signs. Representation errors are 2^-24 of the scales (as FP32).
//
// Precise configuration, which the library uses for every pass of this kernel (the
// two-accumulator standard configuration above rounds D1, and that biased every pass of a time
// integration): four slices per operand, x = 2^(es-7) sum_j 2^(-8j) s_j (j < 4), the input
// optionally a double-float pair hi + lo, and ten MMAs per K step
//     D0 = S0.F0, D1 = S0.F1 + S1.F0, D2 = S0.F2 + S1.F1 + S2.F0 (all three exact),
//     D3 = S0.F3 + S1.F2 + S2.F1 + S3.F0,
// combined in double-float arithmetic into a hi + lo result (about 2^-31 of the scales).
//
// CTA organisation (persistent, one CTA per SM, 416 threads):
//   warps 0-7  producers: load the FP32 state chunk (coalesced; the next chunk's loads are
//              in flight while the current one is sliced), slice it into S0, S1, S2' and
//              store the 128B-swizzled K-major tiles; thread 0 also bulk-copies the
//              pre-sliced, pre-swizzled factor tiles (F0, F1, F1', F2') of the chunk.
//   warps 8-11 epilogue: tcgen05.ld the two accumulators, combine, fused op, store,
//              record max|y| for the next pass.
//   warp 12    one thread issues the tcgen05.mma chain and commits to mbarriers.
// Two pipeline stages (K chunk of 64; 112 KB standard, 96 KB precise) and two TMEM
// accumulator sets of 256 columns (2 x 128 standard, 4 x 64 precise) let loads, MMAs and
// the epilogue of consecutive tiles overlap.
//
// Operand roles. Modes mu >= 2 (positions contiguous in memory): A = state (128
// positions), B = factor (128 outputs), D[pos][i]; the epilogue store is coalesced along
// positions. Mode 1 (fibres contiguous along K): A = factor (128 outputs), B = state
// (128 fibres), D[i][fibre]; the store is coalesced along outputs.
//
// Every mbarrier wait is bounded (about 2 s of clock64 cycles); on timeout the kernel
// records an error code, stops its roles, drains its MMAs and frees TMEM.
#include <cuda_runtime.h>

#include <cstdint>

#include "adr_internal.h"
#include "phi_device.cuh"
#include "tc_common.cuh"

namespace adr {
namespace {

constexpr int kM = 128;                          // UMMA M, TMEM lanes, rows of the A tile
constexpr int kChunk = 64;                       // K per stage: one 128-byte bf16 row
constexpr int kProducerWarps = 8;
constexpr int kMmaWarp = kProducerWarps + 4;
constexpr int kThreads = (kMmaWarp + 1) * 32;   // 416
constexpr uint32_t kTmemCols = 512;
using namespace tc;

// Compile-time shape of one kernel variant. SA: the state is the A operand (modes >= 2);
// PR: precise configuration.
template <bool SA, bool PR>
struct Cfg {
    static constexpr int N = PR ? 64 : 128;            // UMMA N: columns of each accumulator
    static constexpr int SS = PR ? 4 : 3;              // state slices
    static constexpr int FS = 4;                       // factor slices
    static constexpr int NACC = PR ? 4 : 2;            // accumulators per TMEM set (NACC * N = 256)
    static constexpr int SROWS = SA ? kM : N;          // rows of a state tile (positions or fibres)
    static constexpr int FROWS = SA ? N : kM;          // rows of a factor tile (outputs)
    static constexpr int STILE = SROWS * kChunk * 2;   // bytes of one state slice tile
    static constexpr int FTILE = FROWS * kChunk * 2;   // bytes of one factor slice tile
    static constexpr int SBYTES = SS * STILE;
    static constexpr int FBYTES = FS * FTILE;          // one factor block (output tile, K chunk)
    static constexpr int STAGE = SBYTES + FBYTES;
    static constexpr int SMEM = 2 * STAGE + 1024;      // two stages + alignment slack
    static constexpr int NV = SROWS * kChunk / (kProducerWarps * 32);   // state values per thread
    // instruction descriptor: kind::f16, D = F32, A = B = BF16, K-major, N >> 3, M >> 4
    static constexpr uint32_t IDESC =
        (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(kM >> 4) << 24);
    static_assert(NACC * N == 256, "one accumulator set is 256 TMEM columns");
    static_assert(2 * STAGE + 1024 <= 227 * 1024, "shared memory budget");
};

// Load 16 columns of two accumulators for this warp's 32 lanes, then wait.
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float (&a)[16], float (&b)[16]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta), "r"(tb)
        : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        a[j] = __uint_as_float(r[j]);
        b[j] = __uint_as_float(r[16 + j]);
    }
}

// Load 8 columns of four accumulators (columns 64 apart) for this warp's 32 lanes, then wait.
__device__ __forceinline__ void tmem_ld8x4(uint32_t t0, float (&d)[4][8]) {
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
        : "r"(t0), "r"(t0 + 64u), "r"(t0 + 128u), "r"(t0 + 192u)
        : "memory");
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 8; ++j) d[k][j] = __uint_as_float(r[8 * k + j]);
}

// Integer slices of y (|y| < 128; exact FP32 steps; at most 8 significant bits each, so the
// upper half of each FP32 pattern is its exact BF16 pattern).
//   standard: s0, s1, 2^-8 s2;  precise: s0, s1, s2, s3 of y + ylo (double-float input).
template <bool PR>
__device__ __forceinline__ void split(float y, float ylo, uint32_t (&b)[4]) {
    const float s0 = rintf(y);
    const float r0 = PR ? (y - s0) + ylo : (y - s0);   // the sum with ylo rounds below 2^-32
    const float y1 = r0 * 256.f;
    const float s1 = rintf(y1);
    const float y2 = (y1 - s1) * 256.f;
    const float s2 = rintf(y2);
    b[0] = __float_as_uint(s0);
    b[1] = __float_as_uint(s1);
    if (PR) {
        b[2] = __float_as_uint(s2);
        b[3] = __float_as_uint(rintf((y2 - s2) * 256.f));
    } else {
        b[2] = __float_as_uint(s2 * 0.00390625f);
        b[3] = 0u;
    }
}

// Slice 8 consecutive K values v[o..o+7] (+ low parts) into chunk j of row r of each of the
// SS state tiles (tile stride `stile` bytes).
template <bool PR, int NV>
__device__ __forceinline__ void slice_store8(const float (&v)[NV], const float (&vl)[NV], int o, float sc,
                                             uint32_t tile0, uint32_t stile, int r, int j) {
    constexpr int SS = PR ? 4 : 3;
    uint32_t w[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        uint32_t a[4], c[4];
        split<PR>(v[o + 2 * e] * sc, vl[o + 2 * e] * sc, a);
        split<PR>(v[o + 2 * e + 1] * sc, vl[o + 2 * e + 1] * sc, c);
#pragma unroll
        for (int q = 0; q < SS; ++q) w[q][e] = __byte_perm(a[q], c[q], 0x7632);
    }
    const uint32_t off = swz(r, j);
#pragma unroll
    for (int q = 0; q < SS; ++q) st_shared_v4(tile0 + q * stile + off, make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]));
}

// Producer item `it` of a CTA: K chunk (it % nK) of its (it / nK)-th tile. Loads the NV state
// values (and low parts) of thread t.
template <bool SA, bool PR>
__device__ __forceinline__ void produce_load(const TcArgs& p, long long it, long long items, int t,
                                             float (&v)[Cfg<SA, PR>::NV], float (&vl)[Cfg<SA, PR>::NV]) {
    using C = Cfg<SA, PR>;
    constexpr int NV = C::NV;
    if (it >= items) return;
    const long long tile = blockIdx.x + (it / p.nK) * gridDim.x;
    const long long pt = tile / p.nOut;
    const int k0 = int(it % p.nK) * kChunk;
    const int n = p.n;
    const bool lo = PR && p.Xlo != nullptr;
    if (SA) {
        // thread t: position row t % 128, K part t / 128 (NV = 32 values); warp-coalesced
        const int row = t & (kM - 1), part = t >> 7;
        const long long pos = pt * kM + row;
        const bool valid = pos < p.npos;
        const long long Q = p.Q;
        const long long pp = valid ? pos / Q : 0, qq = valid ? pos % Q : 0;
        const int kb = k0 + NV * part;
        const long long base = (pp * n + kb) * Q + qq;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const bool ok = valid && kb + i < n;
            v[i] = ok ? __ldg(p.X + base + (long long)i * Q) : 0.f;
            vl[i] = (lo && ok) ? __ldg(p.Xlo + base + (long long)i * Q) : 0.f;
        }
    } else {
        // thread t: 16-byte chunk j = t % 8 of fibre rows t / 8 + 32 rr (NV / 8 rows)
        const int j = t & 7, r0 = t >> 3;
        const int kb = k0 + 8 * j;
#pragma unroll
        for (int rr = 0; rr < NV / 8; ++rr) {
            const long long f = pt * C::SROWS + r0 + 32 * rr;
            const bool valid = f < p.npos;
            const long long base = (valid ? f : 0) * n + kb;
            if (valid && p.vec4 && kb + 8 <= n) {
                const float4 a = __ldg(reinterpret_cast<const float4*>(p.X + base));
                const float4 b = __ldg(reinterpret_cast<const float4*>(p.X + base) + 1);
                v[8 * rr + 0] = a.x; v[8 * rr + 1] = a.y; v[8 * rr + 2] = a.z; v[8 * rr + 3] = a.w;
                v[8 * rr + 4] = b.x; v[8 * rr + 5] = b.y; v[8 * rr + 6] = b.z; v[8 * rr + 7] = b.w;
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[8 * rr + e] = (valid && kb + e < n) ? __ldg(p.X + base + e) : 0.f;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) vl[8 * rr + e] = (lo && valid && kb + e < n) ? __ldg(p.Xlo + base + e) : 0.f;
        }
    }
}

template <bool SA, bool PR>
__device__ __forceinline__ void produce_store(const float (&v)[Cfg<SA, PR>::NV], const float (&vl)[Cfg<SA, PR>::NV],
                                              int t, float sc, uint32_t sA) {
    using C = Cfg<SA, PR>;
    if (SA) {
        const int row = t & (kM - 1), part = t >> 7;
#pragma unroll
        for (int j4 = 0; j4 < C::NV / 8; ++j4)
            slice_store8<PR, C::NV>(v, vl, 8 * j4, sc, sA, C::STILE, row, (C::NV / 8) * part + j4);
    } else {
        const int j = t & 7, r0 = t >> 3;
#pragma unroll
        for (int rr = 0; rr < C::NV / 8; ++rr) slice_store8<PR, C::NV>(v, vl, 8 * rr, sc, sA, C::STILE, r0 + 32 * rr, j);
    }
}

// One pipeline item: wait for the stage, start the factor copy, prefetch the next item,
// slice the current one, publish.
template <bool SA, bool PR>
__device__ __forceinline__ bool produce_step(const TcArgs& p, long long it, long long items, int t, float sc,
                                             uint32_t sbase, uint32_t bar0, volatile int* abort_flag,
                                             const float (&cur)[Cfg<SA, PR>::NV], const float (&curl)[Cfg<SA, PR>::NV],
                                             float (&nxt)[Cfg<SA, PR>::NV], float (&nxtl)[Cfg<SA, PR>::NV]) {
    using C = Cfg<SA, PR>;
    const int s = int(it & 1);
    const uint32_t ph = uint32_t(it >> 1) & 1u;
    const uint32_t full = bar0 + 8u * s, empty = bar0 + 16u + 8u * s;
    if (!mbar_wait(empty, ph ^ 1u, p.err, 1, abort_flag, 64)) return false;
    const uint32_t sA = sbase + s * C::STAGE;
    const uint32_t sF = sA + C::SBYTES;
    if (t == 0) {
        const long long tile = blockIdx.x + (it / p.nK) * gridDim.x;
        const int ot = int(tile % p.nOut);
        const int c = int(it % p.nK);
        mbar_arrive_expect_tx(full, C::FBYTES);
        const uint8_t* src = p.fimg + (size_t(ot) * p.nK + c) * C::FBYTES;
#pragma unroll
        for (int q = 0; q < C::FS; ++q) bulk_g2s(sF + q * C::FTILE, src + q * C::FTILE, C::FTILE, full);
    }
    produce_load<SA, PR>(p, it + 1, items, t, nxt, nxtl);
    produce_store<SA, PR>(cur, curl, t, sc, sA);
    fence_proxy_async();
    mbar_arrive(full);
    return true;
}

// Issue the MMAs of one 16-wide K step. Standard: D0 += S0.F0; D1 += S0.F1 + S1.F0 +
// S0.(2^-8 F2) + (2^-8 S2).F0 + S1.(2^-8 F1) (factor tiles F0, F1, 2^-8 F1, 2^-8 F2; state
// tiles S0, S1, 2^-8 S2). Precise: D0..D3 as in the file header (tiles F0..F3, S0..S3).
template <bool SA, bool PR>
__device__ __forceinline__ void mma_kstep(uint32_t d, const uint64_t (&S)[4], const uint64_t (&F)[4], uint64_t adv,
                                          uint32_t first) {
    using C = Cfg<SA, PR>;
    auto mma = [&](int acc, int si, int fi, uint32_t accumulate) {
        const uint32_t dd = d + uint32_t(acc * C::N);
        if (SA) tc_mma(dd, S[si] + adv, F[fi] + adv, C::IDESC, accumulate);
        else    tc_mma(dd, F[fi] + adv, S[si] + adv, C::IDESC, accumulate);
    };
    const uint32_t acc = first ? 0u : 1u;
    if (!PR) {
        mma(0, 0, 0, acc);
        mma(1, 0, 1, acc);
        mma(1, 1, 0, 1u);
        mma(1, 0, 3, 1u);
        mma(1, 2, 0, 1u);
        mma(1, 1, 2, 1u);
    } else {
        mma(0, 0, 0, acc);
        mma(1, 0, 1, acc);
        mma(1, 1, 0, 1u);
        mma(2, 0, 2, acc);
        mma(2, 1, 1, 1u);
        mma(2, 2, 0, 1u);
        mma(3, 0, 3, acc);
        mma(3, 1, 2, 1u);
        mma(3, 2, 1, 1u);
        mma(3, 3, 0, 1u);
    }
}

// TwoSum: s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <bool SA, bool PR, int EPI>
__global__ void __launch_bounds__(kThreads, 1) tc_contract_kernel(TcArgs p) {
    using C = Cfg<SA, PR>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[9];
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t bar0 = smem_u32(&bars[0]);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 16u + 8u * s; };
    auto accf_bar = [&](int a) { return bar0 + 32u + 8u * a; };
    auto acce_bar = [&](int a) { return bar0 + 48u + 8u * a; };
    const uint32_t drain_bar = bar0 + 64u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(full_bar(s), kProducerWarps * 32 + 1);   // producers + 1 expect_tx arrival
            mbar_init(empty_bar(s), 1);                         // tcgen05.commit
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf_bar(a), 1);     // tcgen05.commit
            mbar_init(acce_bar(a), 128);   // epilogue threads
        }
        mbar_init(drain_bar, 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    // scale of the state from the max-abs recorded by its producer (amax < 2^es)
    const float amax = __uint_as_float(*p.amax_in);
    int es = 0;
    if (amax > 0.f) frexpf(amax, &es);
    const float sc = ldexpf(1.f, 7 - es);
    const float sback = ldexpf(1.f, es - 7);

    const int n = p.n;
    const long long Q = p.Q;

    if (warp < kProducerWarps) {
        // ------------------------------------------------------------ producers
        // The loads of the next chunk are issued before the current one is sliced, so
        // global latency overlaps the ALU work.
        const int t = threadIdx.x;
        const long long my_tiles = (p.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
        const long long items = my_tiles * p.nK;
        if (!PR) {
            float va[C::NV], vb[C::NV], la[C::NV], lb[C::NV];   // la, lb stay zero (no low parts)
            produce_load<SA, PR>(p, 0, items, t, va, la);
            for (long long it = 0; it < items; it += 2) {
                if (!produce_step<SA, PR>(p, it, items, t, sc, sbase, bar0, &abort_s, va, la, vb, lb)) break;
                if (it + 1 >= items) break;
                if (!produce_step<SA, PR>(p, it + 1, items, t, sc, sbase, bar0, &abort_s, vb, lb, va, la)) break;
            }
        } else {
            // precise: hi and lo values of one item at a time (registers do not allow a prefetch)
            float v[C::NV], vl[C::NV];
            for (long long it = 0; it < items; ++it) {
                const int s = int(it & 1);
                const uint32_t ph = uint32_t(it >> 1) & 1u;
                if (!mbar_wait(empty_bar(s), ph ^ 1u, p.err, 1, &abort_s, 64)) break;
                const uint32_t sA = sbase + s * C::STAGE;
                const uint32_t sF = sA + C::SBYTES;
                if (t == 0) {
                    const long long tile = blockIdx.x + (it / p.nK) * gridDim.x;
                    mbar_arrive_expect_tx(full_bar(s), C::FBYTES);
                    const uint8_t* src = p.fimg + (size_t(tile % p.nOut) * p.nK + it % p.nK) * C::FBYTES;
#pragma unroll
                    for (int q = 0; q < C::FS; ++q) bulk_g2s(sF + q * C::FTILE, src + q * C::FTILE, C::FTILE, full_bar(s));
                }
                produce_load<SA, PR>(p, it, items, t, v, vl);
                produce_store<SA, PR>(v, vl, t, sc, sA);
                fence_proxy_async();
                mbar_arrive(full_bar(s));
            }
        }
    } else if (warp < kProducerWarps + 4) {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - kProducerWarps;   // TMEM lane quarter of this warp
        const int row = ew * 32 + lane;
        long long tl = 0;
        for (long long tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x, ++tl) {
            const int a = int(tl & 1);
            const uint32_t ph = uint32_t(tl >> 1) & 1u;
            const bool waited = mbar_wait(accf_bar(a), ph, p.err, 2, &abort_s, 64);
            if (!__all_sync(0xffffffffu, waited)) break;   // warp-uniform: TMEM loads are .sync.aligned
            tc_fence_after();
            const long long pt = tile / p.nOut;
            const int ot = int(tile % p.nOut);
            float vmax = 0.f;
            // per-row setup: rows are positions (SA) or outputs; columns the other
            bool rvalid;
            long long off0, cstep;      // offset of (row, column 0) and per-column stride
            float zrow = 0.f, rscale = 0.f;
            int ncol;                    // valid columns of this tile
            if (SA) {
                const long long pos = pt * kM + row;
                rvalid = pos < p.npos;
                const long long pp = rvalid ? pos / Q : 0, qq = rvalid ? pos % Q : 0;
                off0 = (pp * n + ot * C::N) * Q + qq;
                cstep = Q;
                ncol = min(C::N, n - ot * C::N);
                if (EPI == EPI_PHI && rvalid) {
                    // position part of z = tau (l1 + l2 + l3): the directions other than mu
                    zrow = __ldg(p.zq_a + qq % p.na);
                    if (p.zq_b) zrow += __ldg(p.zq_b + qq / p.na);
                    if (p.zp) zrow += __ldg(p.zp + pp);
                }
            } else {
                const int irow = ot * kM + row;
                rvalid = irow < n;
                if (rvalid) rscale = sback * __ldg(p.fscale + irow);
                off0 = pt * C::N * (long long)n + irow;
                cstep = n;
                ncol = int(min((long long)C::N, p.npos - pt * C::N));
            }
            const float* fsc = p.fscale + ot * C::N;      // column scales (SA)
            const float* zc = p.zmu + ot * C::N;          // column part of z (EPI_PHI)
            float* yrow = p.Y + off0;
            float* ylo = (EPI == EPI_STORE2) ? p.Ylo + off0 : nullptr;
            const float* brow = (EPI == EPI_AXPY) ? p.base + off0 : nullptr;
            const uint32_t tbase = tmem + (uint32_t(ew * 32) << 16) + uint32_t(a) * 256u;
            auto emit = [&](int col, float hi, float lo) {
                // hi + lo: the combined accumulators of (row, col) before scaling
                const float scale = SA ? sback * __ldg(fsc + col) : rscale;
                const long long o = (long long)col * cstep;
                if (EPI == EPI_STORE2) {
                    yrow[o] = hi * scale;
                    ylo[o] = lo * scale;
                    vmax = fmaxf(vmax, fabsf(hi * scale));
                    return;
                }
                float v = (hi + lo) * scale;
                if (EPI == EPI_PHI) v *= phi_eval(p.phik, zrow + __ldg(zc + col));
                if (EPI == EPI_AXPY) v = fmaf(p.alpha, v, __ldg(brow + o));
                yrow[o] = v;
                vmax = fmaxf(vmax, fabsf(v));
            };
            if (!PR) {
#pragma unroll 1
                for (int j0 = 0; j0 < C::N; j0 += 16) {
                    float d0[16], d1[16];
                    __syncwarp();
                    tmem_ld16x2(tbase + j0, tbase + uint32_t(C::N) + j0, d0, d1);
                    if (!rvalid || j0 >= ncol) continue;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (j0 + j >= ncol) break;
                        // D0 is an exact integer, 2^-8 D1 an exact scaling
                        const float t1 = d1[j] * 0.00390625f;
                        if (EPI == EPI_STORE2) {
                            float hi, lo;
                            two_sum(d0[j], t1, hi, lo);
                            emit(j0 + j, hi, lo);
                        } else {
                            emit(j0 + j, d0[j] + t1, 0.f);
                        }
                    }
                }
            } else {
#pragma unroll 1
                for (int j0 = 0; j0 < C::N; j0 += 8) {
                    float d[4][8];
                    __syncwarp();
                    tmem_ld8x4(tbase + j0, d);
                    if (!rvalid || j0 >= ncol) continue;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (j0 + j >= ncol) break;
                        // D0 + 2^-8 D1 + 2^-16 D2 + 2^-24 D3 in double-float arithmetic
                        float hi, lo;
                        two_sum(d[0][j], d[1][j] * 0.00390625f, hi, lo);
                        lo += fmaf(d[3][j], 5.9604644775390625e-08f, d[2][j] * 1.52587890625e-05f);
                        const float s = hi + lo;
                        lo = lo - (s - hi);
                        emit(j0 + j, s, lo);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acce_bar(a));
            for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
            if (lane == 0 && p.amax_out && vmax > 0.f) atomicMax(p.amax_out, __float_as_uint(vmax));
        }
    } else if (lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        long long g = 0, tl = 0;
        for (long long tile = blockIdx.x; tile < p.ntiles && !abort_s; tile += gridDim.x, ++tl) {
            const int a = int(tl & 1);
            const uint32_t aph = uint32_t(tl >> 1) & 1u;
            if (!mbar_wait(acce_bar(a), aph ^ 1u, p.err, 4, &abort_s)) break;
            tc_fence_after();
            const uint32_t d = tmem + uint32_t(a) * 256u;
            bool ok = true;
            for (int c = 0; c < p.nK; ++c, ++g) {
                const int s = int(g & 1);
                const uint32_t ph = uint32_t(g >> 1) & 1u;
                if (!mbar_wait(full_bar(s), ph, p.err, 8, &abort_s)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sS = sbase + s * C::STAGE;
                const uint32_t sF = sS + C::SBYTES;
                uint64_t S[4], F[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    S[q] = sdesc(sS + (q < C::SS ? q : 0) * C::STILE);
                    F[q] = sdesc(sF + q * C::FTILE);
                }
#pragma unroll
                for (int kk = 0; kk < kChunk / 16; ++kk)
                    mma_kstep<SA, PR>(d, S, F, uint64_t(kk * 32) >> 4, (c == 0 && kk == 0) ? 1u : 0u);
                tc_commit(empty_bar(s));
            }
            if (!ok) break;
            tc_commit(accf_bar(a));
        }
        // wait for every MMA this thread issued before TMEM is released
        tc_commit(drain_bar);
        {
            const long long t0 = clock64();
            while (!mbar_try_wait(drain_bar, 0) && clock64() - t0 < kWaitCycles) {}
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

int g_num_sms = 0;

template <bool SA, bool PR, int EPI>
cudaError_t launch_variant(const TcArgs& a, unsigned grid, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tc_contract_kernel<SA, PR, EPI>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<SA, PR>::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    tc_contract_kernel<SA, PR, EPI><<<grid, kThreads, Cfg<SA, PR>::SMEM, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Rows of an output tile and of a position tile for a variant (the host tiles with these).
int tc_out_rows(bool state_is_a, bool precise) { return state_is_a ? (precise ? 64 : 128) : 128; }
int tc_pos_rows(bool state_is_a, bool precise) { return state_is_a ? 128 : (precise ? 64 : 128); }

cudaError_t launch_contract_tc(const TcArgs& a, cudaStream_t s) {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (a.n > 512 || a.n < 1) return cudaErrorInvalidValue;
    const long long grid = a.ntiles < g_num_sms ? a.ntiles : g_num_sms;
    if (grid <= 0) return cudaSuccess;
    const unsigned g = unsigned(grid);
    // The library runs every pass in the precise configuration (ten products into exact
    // accumulators); the standard configuration's two accumulators round, and that rounding
    // biased every pass.
    if (!a.precise) return cudaErrorInvalidValue;
    if (a.state_is_a) {
        if (a.epi == EPI_PHI) return launch_variant<true, true, EPI_PHI>(a, g, s);
        if (a.epi == EPI_AXPY) return launch_variant<true, true, EPI_AXPY>(a, g, s);
        if (a.epi == EPI_STORE2) return launch_variant<true, true, EPI_STORE2>(a, g, s);
        return launch_variant<true, true, EPI_STORE>(a, g, s);
    }
    if (a.epi == EPI_PHI) return cudaErrorInvalidValue;   // fused into modes >= 2 only
    if (a.epi == EPI_AXPY) return launch_variant<false, true, EPI_AXPY>(a, g, s);
    if (a.epi == EPI_STORE2) return launch_variant<false, true, EPI_STORE2>(a, g, s);
    return launch_variant<false, true, EPI_STORE>(a, g, s);
}

}  // namespace adr
