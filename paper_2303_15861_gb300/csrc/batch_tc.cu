// K2 on the tensor cores for batched 2-D contexts in mixed precision: the mu-mode products
// of Section 1 / Section 5.2 for every instance of a batch in one persistent launch, with
// compensated (hi + lo) FP32 inputs and outputs, the pointwise phi_k scaling (K3) and the
// stage axpy (K4) fused into the epilogue.
//
// Exact-slice split with five state slices. The input x = hi + lo of instance i gets the
// scale 2^(es_i - 7) from max|x| over that instance (recorded by the kernel that produced
// it); each factor row r its own 2^(e_r - 7):
//     x = 2^(es-7) (S0 + 2^-8 S1 + 2^-16 S2 + 2^-24 S3 + 2^-32 S4)   up to 2^-40 of max|x|,
//     f = 2^(e-7)  (F0 + 2^-8 F1 + 2^-16 F2 + 2^-24 F3)              up to 2^-32 of the row max,
// integer slices |S_j|, |F_j| <= 128, exact in BF16. The fourteen products with i + j <= 4
// go into four TMEM accumulators per output:
//     D0 = S0 F0,   D1 = S0 F1 + S1 F0,   D2 = S0 F2 + S1 F1 + S2 F0,
//     D3 = S0 F3 + S1 F2 + S2 F1 + S3 F0 + 2^-8 (S1 F3 + S2 F2 + S3 F1 + S4 F0),
// the 2^-8 terms through pre-scaled tiles (2^-8 F1, F2, F3 sliced on the host, 2^-8 S4 by the
// producers; exact scalings). For K <= 256 D0, D1 and D2 are sums of integers below 2^24 and
// exact whatever rounding the tensor cores apply; D3 rounds at 2^-24 of itself, some 2^-48 of
// the result. The epilogue forms D0 + 2^-8 D1 + 2^-16 D2 + 2^-24 D3 in double-float
// arithmetic. With four slices of the state (ten products), or without the cross products
// at 2^-32, an FP64 emulation of the batched ETD2RK workload ends at 1.5e-4 on its worst
// instance; with these fourteen at 1.0e-6.
//
// CTA (persistent, one per SM, 416 threads): warps 0-7 load the FP32 pairs of a K chunk of
// 32 (coalesced), slice them and store 64-byte-swizzled K-major BF16 tiles, and thread 0
// bulk-copies the seven pre-sliced factor tiles of the chunk; warps 8-11 are the epilogue
// (one TMEM lane quarter each); warp 12 issues the MMAs. Two pipeline stages and two TMEM
// accumulator sets (2 x 4 x 64 columns) let slicing, MMAs and the epilogue of consecutive
// tiles overlap. Operand roles: mode 2 (K = x2): A = state (128 positions along x1),
// B = factor (64 outputs); mode 1 (K = x1): A = factor (128 outputs), B = state (64 rows).
// In both the epilogue stores are coalesced along x1. Every mbarrier wait is bounded; on a
// timeout the CTA records an error code, drains its MMAs and frees TMEM.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "adr_internal.h"
#include "tc_common.cuh"

namespace adr {
namespace {
using namespace tc;

constexpr int kM = 128;                 // UMMA M, TMEM lanes
constexpr int kN = 64;                  // UMMA N: columns of each accumulator
constexpr int kKc = 32;                 // K per stage: one 64-byte BF16 row
constexpr int kSS = 5;                  // state slice tiles: S0..S3, 2^-8 S4
constexpr int kFS = 7;                  // factor slice tiles: F0..F3, 2^-8 F1..F3
static_assert(kM == kBatchTcRows1 && kN == kBatchTcRows2 && kKc == kBatchTcChunk && kFS == kBatchTcFactorTiles,
              "the host slicing (host_setup.cpp) writes the tiles this kernel reads");
constexpr int kNacc = 4;
constexpr int kProducerWarps = 8;
constexpr int kEpiWarp0 = 8;
constexpr int kMmaWarp = 12;
constexpr int kLoadWarp = 13;           // factor tiles: bulk copies, its own ring, running ahead
constexpr int kThreads = (kLoadWarp + 1) * 32;
constexpr uint32_t kTmemCols = 512;     // two sets of kNacc x kN columns
static_assert(2 * kNacc * kN <= int(kTmemCols), "TMEM");

template <bool SA>
struct BCfg {
    static constexpr int SROWS = SA ? kM : kN;     // rows of a state tile (positions or x2 rows)
    static constexpr int FROWS = SA ? kN : kM;     // rows of a factor tile (outputs)
    static constexpr int STILE = SROWS * kKc * 2;
    static constexpr int FTILE = FROWS * kKc * 2;
    static constexpr int SBYTES = kSS * STILE;
    static constexpr int FBYTES = kFS * FTILE;
    static constexpr int SST = SA ? 3 : 2;         // state-slice ring stages
    static constexpr int FST = 3;                  // factor ring stages
    static constexpr int SMEM = SST * SBYTES + FST * FBYTES + 1024;
    static constexpr int NV = SROWS * kKc / (kProducerWarps * 32);   // values per producer thread
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b|
    s = a + b;
    e = b - (s - a);
}
// (ah + al) (bh + bl) in double-float arithmetic
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& h, float& l) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, fmaf(al, bh, e));
    quick_two_sum(p, e, h, l);
}
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& h, float& l) {
    float s, e;
    two_sum(ah, bh, s, e);
    e += al + bl;
    quick_two_sum(s, e, h, l);
}

// Five integer slices of y + ylo (|y + ylo| <= 128 + a rounding), as FP32 patterns whose upper
// halves are the exact BF16 values: S0..S3 and 2^-8 S4. The steps y - rint(y) and the scalings
// by 256 are exact; the low part enters once through an exact TwoSum, its rounding error at
// the last slice, where only products below 2^-40 of the scale are left out.
__device__ __forceinline__ void split5(float y, float ylo, uint32_t (&b)[kSS]) {
    const float s0 = rintf(y);
    float a = (y - s0) * 256.f;
    const float s1 = rintf(a);
    a = (a - s1) * 256.f;
    float t, e;
    two_sum(a, ylo * 65536.f, t, e);
    const float s2 = rintf(t);
    a = (t - s2) * 256.f;
    const float s3 = rintf(a);
    a = fmaf(e, 65536.f, (a - s3) * 256.f);
    const float s4 = rintf(a);
    b[0] = __float_as_uint(s0);
    b[1] = __float_as_uint(s1);
    b[2] = __float_as_uint(s2);
    b[3] = __float_as_uint(s3);
    b[4] = __float_as_uint(s4 * 0.00390625f);
}

// Slice 8 consecutive K values (+ low parts) into 16-byte chunk j of row r of the five state
// tiles (tile stride stile bytes).
__device__ __forceinline__ void slice_store8(const float* v, const float* vl, float sc, uint32_t tile0, uint32_t stile,
                                             int r, int j) {
    uint32_t w[kSS][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        uint32_t a[kSS], c[kSS];
        split5(v[2 * e] * sc, vl[2 * e] * sc, a);
        split5(v[2 * e + 1] * sc, vl[2 * e + 1] * sc, c);
#pragma unroll
        for (int q = 0; q < kSS; ++q) w[q][e] = __byte_perm(a[q], c[q], 0x7632);
    }
    const uint32_t off = swz64(r, j);
#pragma unroll
    for (int q = 0; q < kSS; ++q) st_shared_v4(tile0 + q * stile + off, make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]));
}

__device__ __forceinline__ void ld8(const float* p, float* v) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Scale of an instance's input from its recorded max|x| (< 2^es): x * 2^(7 - es) in [-128, 128].
__device__ __forceinline__ int input_exponent(const unsigned* amax, int inst) {
    const float m = __uint_as_float(__ldg(amax + inst));
    int es = 0;
    if (m > 0.f) frexpf(m, &es);
    return es;
}

// Prefetch into L2 the lines that K chunk c of a tile will load: one 128-byte line per producer
// thread (mode 2: 32 rows x 4 lines of hi and of lo; mode 1: 64 rows x 1 line of hi and of lo).
template <bool SA>
__device__ __forceinline__ void prefetch_chunk(const BatchTcArgs& p, const BatchTcInst& in, int pt, int c, int t) {
    const int n1 = in.n1, n2 = in.n2;
    const float* base = nullptr;
    long long e = 0;
    if (SA) {
        const int k = c * kKc + ((t >> 2) & 31), q = pt * kM + 32 * (t & 3);
        if (k < n2 && q < n1) { base = (t >> 7) ? p.Xlo : p.X; e = in.off + (long long)k * n1 + q; }
    } else if (t < 128) {
        const int f = pt * kN + (t & 63), k = c * kKc;
        if (f < n2 && k < n1) { base = (t >> 6) ? p.Xlo : p.X; e = in.off + (long long)f * n1 + k; }
    }
    if (base) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + e));
}

// Load the NV state values (and low parts) of producer thread t for K chunk c of a tile.
template <bool SA>
__device__ __forceinline__ void load_chunk(const BatchTcArgs& p, const BatchTcInst& in, int pt, int c, int t,
                                           float (&v)[BCfg<SA>::NV], float (&vl)[BCfg<SA>::NV]) {
    constexpr int NV = BCfg<SA>::NV;
    const int n1 = in.n1, n2 = in.n2;
    if (SA) {
        // mode 2: thread t holds position row t % 128, K values 16 (t / 128) .. + 15 (x2 rows)
        const int row = t & (kM - 1), part = t >> 7;
        const int q = pt * kM + row;
        const bool valid = q < n1;
        const int kb = c * kKc + NV * part;
        const long long base = in.off + (long long)kb * n1 + q;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const bool ok = valid && kb + i < n2;
            v[i] = ok ? __ldg(p.X + base + (long long)i * n1) : 0.f;
            vl[i] = (ok && p.Xlo) ? __ldg(p.Xlo + base + (long long)i * n1) : 0.f;
        }
    } else {
        // mode 1: thread t holds 16-byte chunk t % 4 (8 K values along x1) of row t / 4
        const int j = t & 3, r = t >> 2;
        const int f = pt * kN + r;
        const bool valid = f < n2;
        const int kb = c * kKc + 8 * j;
        const long long base = in.off + (long long)(valid ? f : 0) * n1 + kb;
        if (valid && in.vec && kb + 8 <= n1) {
            ld8(p.X + base, v);
            if (p.Xlo) ld8(p.Xlo + base, vl);
            else
#pragma unroll
                for (int e = 0; e < 8; ++e) vl[e] = 0.f;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const bool ok = valid && kb + e < n1;
                v[e] = ok ? __ldg(p.X + base + e) : 0.f;
                vl[e] = (ok && p.Xlo) ? __ldg(p.Xlo + base + e) : 0.f;
            }
        }
    }
}

// Instruction descriptor of an M = 128 product of N columns (BF16 inputs, FP32 accumulate).
constexpr uint32_t idesc_n(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(kM >> 4) << 24);
}

// One K step of 16 of the fourteen products. The accumulators D0..D3 sit in consecutive kN-column
// blocks of TMEM and the slice tiles of each operand in consecutive shared-memory tiles, so one
// A slice against r consecutive B slices is one product of r kN columns that adds each pair to
// its own accumulator: eight MMAs (N = 256, 192, 128 and five of 64) instead of fourteen of
// N = 64, the same tensor work with less operand traffic from shared memory.
//   SA (A = state): S0.[F0..F3] -> D0..D3, S1.[F0..F2] -> D1..D3, S2.[F0 F1] -> D2 D3, and into
//       D3: S1 (2^-8 F3), S2 (2^-8 F2), S3 F0, S3 (2^-8 F1), (2^-8 S4) F0.
//   mode 1 (A = factor): F0.[S0..S3] -> D0..D3, F1.[S0..S2] -> D1..D3, F2.[S0 S1] -> D2 D3, and
//       into D3: F0 (2^-8 S4), F3 S0, (2^-8 F1) S3, (2^-8 F2) S2, (2^-8 F3) S1.
template <bool SA>
__device__ __forceinline__ void mma_kstep(uint32_t d, const uint64_t (&S)[kSS], const uint64_t (&F)[kFS], uint64_t adv,
                                          uint32_t first) {
    auto mma = [&](int acc, uint64_t a, uint64_t b, int nacc, uint32_t accumulate) {
        tc_mma(d + uint32_t(acc * kN), a + adv, b + adv, idesc_n(nacc * kN), accumulate);
    };
    const uint32_t acc = first ? 0u : 1u;
    if (SA) {
        mma(0, S[0], F[0], 4, acc);
        mma(1, S[1], F[0], 3, 1u);
        mma(2, S[2], F[0], 2, 1u);
        mma(3, S[1], F[6], 1, 1u);
        mma(3, S[2], F[5], 1, 1u);
        mma(3, S[3], F[0], 1, 1u);
        mma(3, S[3], F[4], 1, 1u);
        mma(3, S[4], F[0], 1, 1u);
    } else {
        mma(0, F[0], S[0], 4, acc);
        mma(1, F[1], S[0], 3, 1u);
        mma(2, F[2], S[0], 2, 1u);
        mma(3, F[0], S[4], 1, 1u);
        mma(3, F[3], S[0], 1, 1u);
        mma(3, F[4], S[3], 1, 1u);
        mma(3, F[5], S[2], 1, 1u);
        mma(3, F[6], S[1], 1, 1u);
    }
}

// Load 8 columns of the four accumulators (kN columns apart) for this warp's 32 lanes.
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
        : "r"(t0), "r"(t0 + uint32_t(kN)), "r"(t0 + uint32_t(2 * kN)), "r"(t0 + uint32_t(3 * kN))
        : "memory");
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 8; ++j) d[k][j] = __uint_as_float(r[8 * k + j]);
}

template <bool SA, int EPI>
__global__ void __launch_bounds__(kThreads, 1) batch_tc_kernel(const __grid_constant__ BatchTcArgs p) {
    using C = BCfg<SA>;
    extern __shared__ uint8_t smem_raw[];
    constexpr int kStages = C::SST, kFStages = C::FST;
    // barriers: sfull[SST] sempty[SST] ffull[FST] fempty[FST] accf[2] acce[2] drain
    __shared__ __align__(8) uint64_t bars[2 * kStages + 2 * kFStages + 4 + 1];
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;   // state-slice ring
    const uint32_t fbase = sbase + kStages * C::SBYTES;               // factor ring
    const uint32_t bar0 = smem_u32(&bars[0]);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
    auto ffull_bar = [&](int s) { return bar0 + 8u * (2 * kStages + s); };
    auto fempty_bar = [&](int s) { return bar0 + 8u * (2 * kStages + kFStages + s); };
    const uint32_t acc0 = bar0 + 8u * (2 * kStages + 2 * kFStages);
    auto accf_bar = [&](int a) { return acc0 + 8u * a; };
    auto acce_bar = [&](int a) { return acc0 + 8u * (2 + a); };
    const uint32_t drain_bar = acc0 + 8u * 4;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full_bar(s), kProducerWarps);             // one arrival per producer warp
            mbar_init(empty_bar(s), 1);                         // tcgen05.commit
        }
        for (int s = 0; s < kFStages; ++s) {
            mbar_init(ffull_bar(s), 1);                         // the loader's expect_tx arrival
            mbar_init(fempty_bar(s), 1);                        // tcgen05.commit
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf_bar(a), 1);                          // tcgen05.commit
            mbar_init(acce_bar(a), 4);                          // one arrival per epilogue warp
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
    const int dir = SA ? 1 : 0;                      // direction of the factor (mode - 1)

    if (warp < kProducerWarps) {
        // ------------------------------------------------------------ producers
        // The chunks of this CTA's tiles in order; the global loads of the next chunk are issued
        // before the current one is sliced, so their latency overlaps the slicing.
        const int t = threadIdx.x;
        struct Job {
            int tile = 0, c = 0, nK = 0;
            int4 item;
            const BatchTcInst* in = nullptr;
            float sc = 0.f;
            const uint8_t* img = nullptr;
        };
        auto start = [&](int tile, Job& j) {
            j.tile = tile;
            j.c = 0;
            if (tile >= p.nitems) return;
            j.item = __ldg(p.items + tile);
            j.in = p.inst + j.item.x;
            j.nK = ((SA ? j.in->n2 : j.in->n1) + kKc - 1) / kKc;
            j.sc = ldexpf(1.f, 7 - input_exponent(p.amax_in, j.item.x));
            j.img = p.fimg + j.in->img_off[p.role][dir] + size_t(j.item.z) * j.nK * C::FBYTES;
        };
        auto next = [&](const Job& j, Job& n) {
            if (j.c + 1 < j.nK) { n = j; n.c = j.c + 1; }
            else start(j.tile + int(gridDim.x), n);
        };
        // one chunk: wait for its stage, prefetch the next chunk, slice
        auto step = [&](const Job& j, long long g, const float (&v)[C::NV], const float (&vl)[C::NV], const Job& nj,
                        float (&nv)[C::NV], float (&nvl)[C::NV]) -> bool {
            const int s = int(g % kStages);
            const uint32_t ph = uint32_t(g / kStages) & 1u;
            // warp-uniform decision: the per-warp arrival below needs every lane
            if (!__all_sync(0xffffffffu, mbar_wait(empty_bar(s), ph ^ 1u, p.err, 1, &abort_s, 64))) return false;
            const uint32_t sA = sbase + s * C::SBYTES;
            if (nj.tile < p.nitems) load_chunk<SA>(p, *nj.in, nj.item.y, nj.c, t, nv, nvl);
            if (SA) {
                const int row = t & (kM - 1), part = t >> 7;
                slice_store8(v, vl, j.sc, sA, C::STILE, row, 2 * part);
                slice_store8(v + 8, vl + 8, j.sc, sA, C::STILE, row, 2 * part + 1);
            } else {
                slice_store8(v, vl, j.sc, sA, C::STILE, t >> 2, t & 3);
            }
            // one arrival per warp once every lane's slices are visible to the tensor cores
            // (256 single-thread arrivals on one barrier word serialise)
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(full_bar(s));
            return true;
        };
        Job a, b, pf;
        start(blockIdx.x, a);
        float va[C::NV], vla[C::NV], vb[C::NV], vlb[C::NV];
        if (a.tile < p.nitems) load_chunk<SA>(p, *a.in, a.item.y, a.c, t, va, vla);
        // an L2 prefetch cursor kPrefetch chunks ahead of the chunk being sliced
        constexpr int kPrefetch = 3;
        pf = a;
        for (int i = 0; i < kPrefetch && pf.tile < p.nitems; ++i) {
            prefetch_chunk<SA>(p, *pf.in, pf.item.y, pf.c, t);
            Job nx;
            next(pf, nx);
            pf = nx;
        }
        auto advance_prefetch = [&]() {
            if (pf.tile >= p.nitems) return;
            prefetch_chunk<SA>(p, *pf.in, pf.item.y, pf.c, t);
            Job nx;
            next(pf, nx);
            pf = nx;
        };
        for (long long g = 0; a.tile < p.nitems; g += 2) {
            next(a, b);
            advance_prefetch();
            if (!step(a, g, va, vla, b, vb, vlb)) break;
            if (b.tile >= p.nitems) break;
            next(b, a);
            advance_prefetch();
            if (!step(b, g + 1, vb, vlb, a, va, vla)) break;
        }
    } else if (warp < kEpiWarp0 + 4) {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - kEpiWarp0;        // TMEM lane quarter of this warp
        const int row = ew * 32 + lane;
        const float ah = float(p.alpha);
        const float al = float(p.alpha - double(ah));
        long long tl = 0;
        for (int tile = blockIdx.x; tile < p.nitems; tile += gridDim.x, ++tl) {
            const int a = int(tl & 1);
            const uint32_t ph = uint32_t(tl >> 1) & 1u;
            const bool waited = mbar_wait(accf_bar(a), ph, p.err, 2, &abort_s, 64);
            if (!__all_sync(0xffffffffu, waited)) break;   // warp-uniform: TMEM loads are .sync.aligned
            tc_fence_after();
            const int4 item = __ldg(p.items + tile);
            const BatchTcInst& in = p.inst[item.x];
            const int n1 = in.n1, n2 = in.n2;
            const float sback = ldexpf(1.f, input_exponent(p.amax_in, item.x) - 7);
            const float* fsc = p.fscale + in.fsc_off[p.role][dir];
            bool rvalid;
            long long off0, cstep;
            int col0, ncol;
            float rscale = 0.f;
            if (SA) {       // rows: positions q along x1; columns: outputs along x2
                const int q = item.y * kM + row;
                rvalid = q < n1;
                col0 = item.z * kN;
                off0 = in.off + (long long)col0 * n1 + q;
                cstep = n1;
                ncol = min(kN, n2 - col0);
            } else {        // rows: outputs along x1; columns: x2 rows
                const int o = item.z * kM + row;
                rvalid = o < n1;
                col0 = item.y * kN;
                if (rvalid) rscale = sback * __ldg(fsc + o);
                off0 = in.off + (long long)col0 * n1 + o;
                cstep = n1;
                ncol = min(kN, n2 - col0);
            }
            float vmax = 0.f;
            const uint32_t tbase = tmem + (uint32_t(ew * 32) << 16) + uint32_t(a) * uint32_t(kNacc * kN);
            // the global operands of the next 8 columns (column scales, the phi table or the axpy
            // base) are loaded while the current ones are combined
            auto load_ops = [&](int j0, float (&sc)[8], float2 (&op)[8]) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const bool ok = rvalid && j0 + j < ncol;
                    const long long o = off0 + (long long)(j0 + j) * cstep;
                    sc[j] = SA ? (ok ? sback * __ldg(fsc + col0 + j0 + j) : 0.f) : rscale;
                    if (EPI == EPI_PHI) op[j] = ok ? __ldg(p.phi + o) : make_float2(0.f, 0.f);
                    else if (EPI == EPI_AXPY)
                        op[j] = make_float2(ok ? __ldg(p.base + o) : 0.f, (ok && p.base_lo) ? __ldg(p.base_lo + o) : 0.f);
                    else op[j] = make_float2(0.f, 0.f);
                }
            };
            float sc_c[8], sc_n[8];
            float2 op_c[8], op_n[8];
            load_ops(0, sc_c, op_c);
#pragma unroll 1
            for (int j0 = 0; j0 < kN; j0 += 8) {
                float d[4][8];
                if (j0 + 8 < kN) load_ops(j0 + 8, sc_n, op_n);
                __syncwarp();
                tmem_ld8x4(tbase + j0, d);
                auto combine = [&](int j) {
                    // D0 + 2^-8 D1 + 2^-16 D2 + 2^-24 D3 in double-float arithmetic
                    float hi, lo;
                    two_sum(d[0][j], d[1][j] * 0.00390625f, hi, lo);
                    lo += fmaf(d[3][j], 5.9604644775390625e-08f, d[2][j] * 1.52587890625e-05f);
                    quick_two_sum(hi, lo, hi, lo);
                    hi *= sc_c[j];                 // a power of two: exact
                    lo *= sc_c[j];
                    const long long o = off0 + (long long)(j0 + j) * cstep;
                    if (EPI == EPI_PHI) {
                        df_mul(hi, lo, op_c[j].x, op_c[j].y, hi, lo);
                    } else if (EPI == EPI_AXPY) {
                        float th, tl2;
                        df_mul(ah, al, hi, lo, th, tl2);
                        df_add(op_c[j].x, op_c[j].y, th, tl2, hi, lo);
                    }
                    if (p.Ylo) {
                        p.Y[o] = hi;
                        p.Ylo[o] = lo;
                    } else {
                        hi = hi + lo;
                        p.Y[o] = hi;
                    }
                    if (p.Yhs) p.Yhs[o] = hi;
                    vmax = fmaxf(vmax, fabsf(hi));
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
                for (int j = 0; j < 8; ++j) {
                    sc_c[j] = sc_n[j];
                    op_c[j] = op_n[j];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce_bar(a));
            for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
            if (lane == 0 && p.amax_out && vmax > 0.f) atomicMax(p.amax_out + item.x, __float_as_uint(vmax));
        }
    } else if (warp == kLoadWarp) {
        // ------------------------------------------------------------ factor loader
        // The CTA's chunks in the same order as the MMA issuer; a ring slot frees when the MMAs
        // of the chunk kFStages earlier retire, so each copy has kFStages - 1 chunks of lead.
        if (lane == 0) {
            long long g = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < p.nitems && ok && !abort_s; tile += gridDim.x) {
                const int4 item = __ldg(p.items + tile);
                const BatchTcInst& in = p.inst[item.x];
                const int nK = ((SA ? in.n2 : in.n1) + kKc - 1) / kKc;
                const uint8_t* img = p.fimg + in.img_off[p.role][dir] + size_t(item.z) * nK * C::FBYTES;
                for (int c = 0; c < nK; ++c, ++g) {
                    const int fs = int(g % kFStages);
                    const uint32_t fph = uint32_t(g / kFStages) & 1u;
                    if (!mbar_wait(fempty_bar(fs), fph ^ 1u, p.err, 32, &abort_s, 32)) { ok = false; break; }
                    mbar_arrive_expect_tx(ffull_bar(fs), C::FBYTES);
                    const uint8_t* src = img + size_t(c) * C::FBYTES;
                    bulk_g2s(fbase + fs * C::FBYTES, src, C::FBYTES, ffull_bar(fs));   // the seven tiles are contiguous
                }
            }
        }
    } else if (lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        long long g = 0, tl = 0;
        for (int tile = blockIdx.x; tile < p.nitems && !abort_s; tile += gridDim.x, ++tl) {
            const int4 item = __ldg(p.items + tile);
            const BatchTcInst& in = p.inst[item.x];
            const int nK = ((SA ? in.n2 : in.n1) + kKc - 1) / kKc;
            const int a = int(tl & 1);
            const uint32_t aph = uint32_t(tl >> 1) & 1u;
            if (!mbar_wait(acce_bar(a), aph ^ 1u, p.err, 4, &abort_s)) break;
            tc_fence_after();
            const uint32_t d = tmem + uint32_t(a) * uint32_t(kNacc * kN);
            bool ok = true;
            for (int c = 0; c < nK; ++c, ++g) {
                const int s = int(g % kStages);
                const uint32_t ph = uint32_t(g / kStages) & 1u;
                const int fs = int(g % kFStages);
                const uint32_t fph = uint32_t(g / kFStages) & 1u;
                if (!mbar_wait(ffull_bar(fs), fph, p.err, 16, &abort_s)) { ok = false; break; }
                if (!mbar_wait(full_bar(s), ph, p.err, 8, &abort_s)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sS = sbase + s * C::SBYTES;
                const uint32_t sF = fbase + fs * C::FBYTES;
                uint64_t S[kSS], F[kFS];
#pragma unroll
                for (int q = 0; q < kSS; ++q) S[q] = sdesc64(sS + q * C::STILE);
#pragma unroll
                for (int q = 0; q < kFS; ++q) F[q] = sdesc64(sF + q * C::FTILE);
#pragma unroll
                for (int kk = 0; kk < kKc / 16; ++kk)
                    mma_kstep<SA>(d, S, F, uint64_t(kk * 32) >> 4, (c == 0 && kk == 0) ? 1u : 0u);
                tc_commit(empty_bar(s));
                tc_commit(fempty_bar(fs));
            }
            if (!ok) break;
            tc_commit(accf_bar(a));
        }
        // wait for every MMA this thread issued before TMEM is released
        tc_commit(drain_bar);
        const long long t0 = clock64();
        while (!mbar_try_wait(drain_bar, 0) && clock64() - t0 < kWaitCycles) {}
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

int g_sms = 0;

template <bool SA, int EPI>
cudaError_t launch_variant(const BatchTcArgs& a, unsigned grid, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(batch_tc_kernel<SA, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             BCfg<SA>::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    batch_tc_kernel<SA, EPI><<<grid, kThreads, BCfg<SA>::SMEM, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ small kernels
__global__ void keep_lo_kernel(const float* __restrict__ u, const float* __restrict__ hs, float* __restrict__ lo,
                               long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (u[i] != hs[i]) lo[i] = 0.f;
}

// One warp per row of one instance (rows located through the row prefix), lanes along x1.
__global__ void __launch_bounds__(256) batch_amax_kernel(BatchStencilArgs<float> g, const float* __restrict__ x,
                                                         unsigned* amax) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < g.rows; r += warps) {
        int lo = 0, hi = g.ninst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(g.row_start + mid) <= r) lo = mid; else hi = mid - 1;
        }
        const BatchInst<float>& in = g.inst[lo];
        const float* row = x + in.off + (r - in.row0) * in.n1;
        float m = 0.f;
        for (int i1 = lane; i1 < in.n1; i1 += 32) m = fmaxf(m, fabsf(__ldg(row + i1)));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && m > 0.f) atomicMax(amax + lo, __float_as_uint(m));
    }
}

}  // namespace

cudaError_t launch_batch_tc(const BatchTcArgs& a, cudaStream_t s) {
    if (a.nitems <= 0) return cudaSuccess;
    if (!a.inst || !a.items || !a.fimg || !a.fscale || !a.X || !a.Y || !a.amax_in || (a.mode != 1 && a.mode != 2))
        return cudaErrorInvalidValue;
    if (a.role < 0 || a.role >= kBatchRoles) return cudaErrorInvalidValue;
    if (a.epi == EPI_PHI && (!a.phi || a.mode != 2)) return cudaErrorInvalidValue;
    if (a.epi == EPI_AXPY && !a.base) return cudaErrorInvalidValue;
    if (a.epi != EPI_STORE && a.epi != EPI_PHI && a.epi != EPI_AXPY) return cudaErrorInvalidValue;
    // the mode-1 producers read 16-byte vectors where an instance's rows allow it
    if (reinterpret_cast<uintptr_t>(a.X) % 16 != 0 || (a.Xlo && reinterpret_cast<uintptr_t>(a.Xlo) % 16 != 0))
        return cudaErrorMisalignedAddress;
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    long long grid = a.grid > 0 ? a.grid : g_sms;
    if (grid > a.nitems) grid = a.nitems;
    const unsigned g = unsigned(grid);
    if (a.mode == 2) {
        if (a.epi == EPI_PHI) return launch_variant<true, EPI_PHI>(a, g, s);
        if (a.epi == EPI_AXPY) return launch_variant<true, EPI_AXPY>(a, g, s);
        return launch_variant<true, EPI_STORE>(a, g, s);
    }
    if (a.epi == EPI_AXPY) return launch_variant<false, EPI_AXPY>(a, g, s);
    if (a.epi == EPI_PHI) return cudaErrorInvalidValue;
    return launch_variant<false, EPI_STORE>(a, g, s);
}

cudaError_t launch_batch_keep_lo(const float* u, const float* hs, float* lo, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (!u || !hs || !lo) return cudaErrorInvalidValue;
    long long blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    keep_lo_kernel<<<unsigned(blocks), 256, 0, s>>>(u, hs, lo, n);
    return cudaGetLastError();
}

cudaError_t launch_batch_amax(const BatchStencilArgs<float>& geom, const float* x, unsigned* amax, cudaStream_t s) {
    if (geom.rows <= 0) return cudaSuccess;
    if (!geom.inst || !geom.row_start || !x || !amax) return cudaErrorInvalidValue;
    long long blocks = (geom.rows + 7) / 8;
    if (blocks > 8192) blocks = 8192;
    batch_amax_kernel<<<unsigned(blocks), 256, 0, s>>>(geom, x, amax);
    return cudaGetLastError();
}

}  // namespace adr
