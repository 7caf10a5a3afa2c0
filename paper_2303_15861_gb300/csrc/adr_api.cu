// C ABI of libadr (declared in include/adr.h): context, host setup, step schedules of
// the integrators and CUDA-graph replay.
//
// Schedules (per time step; B*, T* are library workspace arrays of N elements):
//   Lawson--Euler (Appendix):   W = u + tau g(u)                          [K1]
//                               u = e^{tau A} W                          [K2 x d]
//   ETD2RK = exponential RK2 with phi_2, c2 = 1 (Appendix), written with U:
//                               F = F(u), G0 = g(u)                       [K1]
//                               U = u + tau phi_1(tau A) F                [K2 x 2d, K3, K4]
//                               D = g(U) - G0                             [K1]
//                               u = U + tau phi_2(tau A) D                [K2 x 2d, K3, K4]
//   Lawson4 (Lawson's construction on classical RK4, E = e^{tau A / 2}):
//                               W = u + tau/2 g(u)                        [K1]
//                               X = E W (= U2),  Eu = E u                 [K2 x 2d]
//                               W = Eu + tau/2 g(X)        (= U3)
//                               ACC = 2/3 Eu + 1/3 X + tau/3 g(X)         [K1]
//                               X = Eu + tau g(W),  ACC += tau/3 g(W)     [K1]
//                               W = E X (= U4),  X = E ACC                [K2 x 2d]
//                               u = X + tau/6 g(W)                        [K1]
//     using E(u + tau/6 k1) = 2/3 Eu + 1/3 U2, so a step costs four E actions.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/adr.h"
#include "adr_internal.h"

using adr::ContractArgs;
using adr::StencilArgs;

namespace {

// One enqueued operation of a schedule and the kind of kernel it launches.
enum OpKind { OP_MEMSET = 0, OP_AMAX = 1, OP_STENCIL = 2, OP_CONTRACT_SIMT = 3, OP_CONTRACT_TC = 4,
              OP_CONTRACT_TC_PRECISE = 5, OP_PERIODIC_RHS = 6, OP_FOURIER_MULT = 7,
              OP_PERIODIC_STAGE = 8 };
struct Op {
    std::function<cudaError_t(cudaStream_t)> fn;
    int kind;
    int launches = 1;                      // kernels the op launches (0 for a memset)
    cudaError_t operator()(cudaStream_t s) const { return fn(s); }
};

thread_local std::string g_create_error;

// Factor kinds: 0 E(0.5), 1 E(1), 2 V, 3 V^-1, 4 E(0.5) precise, 5 E(alpha); from kLevel0 the
// factors e^{2^i tau A_mu / 2^s} of the phi doubling route, level i = kind - kLevel0.
constexpr int kLevel0 = 8;
constexpr int kMaxLevels = 40;
constexpr int kFactorKinds = kLevel0 + kMaxLevels;

}  // namespace

// Host side of a batched context: the packing of the instances (fixed at adr_create),
// FP64 staging of their coefficients, factors and eigenvalues (filled by adr_set_coeffs),
// the device copies, and the contraction schedule chosen by the autotuner.
struct adr_batch_state {
    int B = 0;
    int tile_force = -1;                   // BatchTile forced by batch_tile, -1: autotune
    std::vector<int> n1, n2, apitch;
    std::vector<long long> off, row0, a_off;
    std::vector<long long> f_off;          // [i][role][dir] -> 2 * kBatchRoles per instance, -1 if absent
    std::vector<long long> zt_off;         // [i][dir] -> 2 per instance, -1 if absent
    long long rows = 0, a_len = 0, f_len = 0, zt_len = 0;
    bool roles[adr::kBatchRoles] = {false, false, false, false, false};
    std::vector<char> set;
    int nset = 0;
    std::vector<double> hA, hF, hZt;       // FP64 staging, packed like the device copies
    std::vector<double> coef;              // [i] -> ih2[2] i2h[2] bmb[2] beta[2] abar r[4]
    std::vector<double> kappa;             // [i][dir]
    // device
    void* d_inst = nullptr;                // BatchInst<T>[B]
    long long* d_row_start = nullptr;      // B + 1
    void* d_a = nullptr;
    void* d_f = nullptr;
    void* d_zt = nullptr;                  // tau * eigenvalues, working precision
    int4* d_items[2] = {nullptr, nullptr};
    int nitems[2] = {0, 0};
    int grid[2] = {0, 0};                  // persistent CTAs of the contraction, per mode
    int sgrid = 0;                         // persistent CTAs of the stencil
    std::vector<int> tile[2];              // BatchTile per instance, per mode
    bool uploaded = false, tuned = false;
    // mixed precision (compensated FP32 pairs, tensor-core contractions; batch_tc.cu)
    bool mixed = false;
    std::vector<adr::BatchTcInst> tci;     // per instance: sizes, image and scale offsets
    void* d_tci = nullptr;
    uint8_t* d_img = nullptr;              // sliced factor images of every instance, role, direction
    float* d_fsc = nullptr;                // their row scales
    float2* d_phi[3] = {nullptr, nullptr, nullptr};   // double-float phi_0, phi_1, phi_2 per node
    int4* d_titems[2] = {nullptr, nullptr};           // tensor-core work items per mode
    int ntitems[2] = {0, 0};
    int4* d_sunits = nullptr;              // marching stencil units {instance, x1 start, first row, rows}
    int nsunits = 0;
    float* d_lo[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};   // low parts of ws[0..5]
    float* d_ulo = nullptr;                // low part of the caller's state
    float* d_uhs = nullptr;                // the high part the library last wrote to the caller's state
    unsigned* d_bslots = nullptr;          // max|x| per (produced array, instance)
};

struct adr_ctx {
    adr_params p{};
    cudaStream_t stream = nullptr;
    int dim = 0;
    int n[3] = {1, 1, 1};
    size_t N = 0;
    size_t nodes = 0;
    int apitch = 0;                        // padded row pitch of the device copy of a
    bool fp64 = true;
    size_t esize = 8;

    bool coeffs_set = false;
    double b[3] = {0, 0, 0}, r[4] = {0, 0, 0, 0};
    double abar = 0, beta[3] = {0, 0, 0};
    double kappa[3] = {0, 0, 0};
    bool eig_real = false;
    adr::Factor1D f[3];

    // device memory (library-owned)
    void* d_a = nullptr;                   // nodal (a - abar)
    void* d_E[3][3] = {{nullptr}};         // e^{c tau A_mu}, c = 0.5 (0), 1 (1), alpha (2)
    void* d_V[3] = {nullptr};
    void* d_Vi[3] = {nullptr};
    double* d_lam[3] = {nullptr};
    void* ws[9] = {nullptr};               // state-sized workspace; ws[6..8]: low parts (mixed)
    void* d_host_state = nullptr;

    // mixed precision (tensor cores): sliced factor images, per-row scales, c tau lambda
    bool tc = false;
    uint8_t* d_img[kFactorKinds][3] = {{nullptr}};    // sliced image per factor kind and direction
    float* d_fsc[kFactorKinds][3] = {{nullptr}};
    uint8_t* d_img2[kFactorKinds][3] = {{nullptr}};   // the same for the TMA-fed kernel (K chunks of 32)
    float* d_fsc2[kFactorKinds][3] = {{nullptr}};
    float* d_zt[3] = {nullptr};            // tau * lambda_mu[j] (FP32)
    unsigned* d_slots = nullptr;           // max-abs slots of the arrays a step produces
    int* d_err = nullptr;                  // device error word (bounded waits)

    // batched 2-D instances (p.batch > 0)
    std::unique_ptr<adr_batch_state> bs;

    // periodic Fourier pseudospectral contexts (p.periodic)
    bool periodic = false;
    void* d_pc[4] = {nullptr, nullptr, nullptr, nullptr};   // complex work: Cu, C[0..dim-1]
    void* d_ptw[3] = {nullptr, nullptr, nullptr};  // twiddles per direction
    void* d_pk[3] = {nullptr, nullptr, nullptr};   // wavenumbers per direction
    void* d_pa[3] = {nullptr, nullptr, nullptr};   // a_mumu at the nodes
    void* d_pb[3] = {nullptr, nullptr, nullptr};   // b_mu at the nodes
    void* d_psym = nullptr;                        // symbol of A
    void* d_pm[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // E(1/2), E(1), E(alpha), phi_1, phi_2
    void* d_pdif = nullptr;                        // a Lap u form: sum_mu a_mumu D_mu D_mu u
    void* d_pcn = nullptr;                         // fused 2-D stages: the pointwise part of F, transformed
    void* d_pz = nullptr;                          // fused 2-D stages: a Fourier-space array kept between stages

    // phi_k route; for the doubling route: X = tau A / 2^s, Taylor terms, level factors
    int phi_route = 0;                     // adr_phi_route in use (0: no phi_k needed)
    int dbl_s = 0, dbl_p = 0;
    void* d_El[kMaxLevels][3] = {{nullptr}};   // e^{2^i tau A_mu / 2^s}, i = 0..s-1
    void* d_a0 = nullptr;                  // zero (a - abar): the stencil then yields A u
    void* wsd[3] = {nullptr, nullptr, nullptr};   // doubling-route workspace

    // graph cache for adr_integrate
    cudaGraph_t graph = nullptr;           // one step
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph_k = nullptr;         // kGraphSteps steps in one graph (fewer replays)
    cudaGraphExec_t gexec_k = nullptr;
    void* graph_u = nullptr;

    std::string err;
};

namespace {

adr_status fail(adr_ctx* c, adr_status s, const std::string& msg) {
    if (c) c->err = msg; else g_create_error = msg;
    return s;
}

adr_status cuda_fail(adr_ctx* c, cudaError_t e, const char* where) {
    return fail(c, ADR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void free_dev(void*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void drop_graph(adr_ctx* c) {
    if (c->gexec_k) cudaGraphExecDestroy(c->gexec_k);
    if (c->graph_k) cudaGraphDestroy(c->graph_k);
    c->gexec_k = nullptr;
    c->graph_k = nullptr;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->graph_u = nullptr;
}

// Upload an FP64 host array in the working precision.
cudaError_t upload(adr_ctx* c, void** dst, const std::vector<double>& src) {
    const size_t bytes = src.size() * c->esize;
    cudaError_t e = cudaSuccess;
    if (!*dst) e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return e;
    if (c->fp64) return cudaMemcpy(*dst, src.data(), bytes, cudaMemcpyHostToDevice);
    std::vector<float> tmp(src.begin(), src.end());
    return cudaMemcpy(*dst, tmp.data(), bytes, cudaMemcpyHostToDevice);
}

// Slice an FP64 factor for the tensor-core kernel and upload image + row scales. Mode 1
// uses the factor as the A operand (128-row tiles), modes >= 2 as the B operand.
cudaError_t upload_tc(adr_ctx* c, int kind, int m, const std::vector<double>& M) {
    const bool precise = (kind == 4);   // FK_EXP_HALF_PRECISE
    // register-fed kernel: every image in the four-slice layout of its precise variant
    const adr::TcFactor f = adr::make_tc_factor(M, c->n[m], adr::tc_out_rows(m >= 1, true), true);
    cudaError_t e = cudaSuccess;
    if (!c->d_img[kind][m]) e = cudaMalloc(reinterpret_cast<void**>(&c->d_img[kind][m]), f.img.size());
    if (e == cudaSuccess && !c->d_fsc[kind][m])
        e = cudaMalloc(reinterpret_cast<void**>(&c->d_fsc[kind][m]), f.fscale.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_img[kind][m], f.img.data(), f.img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_fsc[kind][m], f.fscale.data(), f.fscale.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    // TMA-fed kernel: 128-row output tiles, K chunks of 32
    const adr::TcFactor f2 = adr::make_tc_factor(M, c->n[m], 128, precise, 32);
    if (!c->d_img2[kind][m]) e = cudaMalloc(reinterpret_cast<void**>(&c->d_img2[kind][m]), f2.img.size());
    if (e == cudaSuccess && !c->d_fsc2[kind][m])
        e = cudaMalloc(reinterpret_cast<void**>(&c->d_fsc2[kind][m]), f2.fscale.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_img2[kind][m], f2.img.data(), f2.img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_fsc2[kind][m], f2.fscale.data(), f2.fscale.size() * sizeof(float), cudaMemcpyHostToDevice);
    return e;
}

// ------------------------------------------------------------------ schedule builders
constexpr int kSlots = 4096;
constexpr int kBatchSlots = 64;         // per-instance max-abs slots of a mixed batched step
constexpr int kGraphSteps = 8;             // steps per replay of the multi-step graph

// The ops of one call, plus the max-abs bookkeeping of the mixed path: every array a
// step produces gets a fresh slot (zeroed at the start of the step) that its producer
// fills and its tensor-core consumer reads to choose the slicing scale.
struct Sched {
    const adr_ctx* c;
    std::vector<Op> ops;
    int next = 0;
    std::vector<std::pair<const void*, int>> slot_of;
    // mixed batched contexts: the low part (and the copy of the high part) kept beside an array
    struct Companion {
        const void* hi;
        float* lo;
        float* hs;
    };
    std::vector<Companion> comp;

    bool batch_mixed() const { return c->bs && c->bs->mixed; }
    bool slots_on() const { return c->tc || batch_mixed(); }
    int max_slots() const { return batch_mixed() ? kBatchSlots : kSlots; }
    // a slot is one word, or one word per instance in a batched context
    unsigned* slot(int id) const { return batch_mixed() ? c->bs->d_bslots + size_t(id) * c->bs->B : c->d_slots + id; }

    explicit Sched(const adr_ctx* ctx) : c(ctx) {
        if (c->tc) {
            unsigned* sl = c->d_slots;
            ops.push_back({[sl](cudaStream_t s) { return cudaMemsetAsync(sl, 0, kSlots * sizeof(unsigned), s); }, OP_MEMSET});
        }
        if (batch_mixed()) {
            unsigned* sl = c->bs->d_bslots;
            const size_t bytes = size_t(kBatchSlots) * c->bs->B * sizeof(unsigned);
            ops.push_back({[sl, bytes](cudaStream_t s) { return cudaMemsetAsync(sl, 0, bytes, s); }, OP_MEMSET});
            for (int i = 0; i < 6; ++i) comp.push_back({c->ws[i], c->bs->d_lo[i], nullptr});
        }
    }
    bool overflow = false;
    unsigned* produce(const void* buf) {
        if (!slots_on()) return nullptr;
        if (next >= max_slots()) { overflow = true; return slot(max_slots() - 1); }
        const int id = next++;
        for (auto& e : slot_of)
            if (e.first == buf) { e.second = id; return slot(id); }
        slot_of.push_back({buf, id});
        return slot(id);
    }
    const unsigned* consume(const void* buf);
    float* lo_of(const void* p) const {
        for (const auto& e : comp)
            if (p && e.hi == p) return e.lo;
        return nullptr;
    }
    float* hs_of(const void* p) const {
        for (const auto& e : comp)
            if (p && e.hi == p) return e.hs;
        return nullptr;
    }
    // The caller's state u of a step of a mixed batched context: its low part lives in the
    // library and is kept only where u still holds the high part the library wrote last.
    void bind_state(const void* u) {
        if (!batch_mixed()) return;
        const adr_batch_state& b = *c->bs;
        comp.push_back({u, b.d_ulo, b.d_uhs});
        const float* uu = static_cast<const float*>(u);
        float* hs = b.d_uhs;
        float* lo = b.d_ulo;
        const long long n = static_cast<long long>(c->N);
        ops.push_back({[uu, hs, lo, n](cudaStream_t s) { return adr::launch_batch_keep_lo(uu, hs, lo, n, s); }, OP_AMAX});
    }
};

template <typename T>
ContractArgs<T> mode_args(const adr_ctx* c, int mu, const T* M, const T* X, T* Y) {
    // state viewed as [P][n][Q]; see contract_simt.cu
    const int n = c->n[mu - 1];
    long long Q = 1, P = 1;
    for (int nu = 1; nu < mu; ++nu) Q *= c->n[nu - 1];
    for (int nu = mu + 1; nu <= c->dim; ++nu) P *= c->n[nu - 1];
    ContractArgs<T> a;
    if (mu == 1) {
        a.A = X; a.sam = n; a.sak = 1; a.sab = 0;
        a.B = M; a.sbk = 1; a.sbn = n; a.sbb = 0;    // B[k][j] = M[j][k]
        a.C = Y; a.scm = n; a.scn = 1; a.scb = 0;
        a.M = int(P); a.N = n; a.K = n; a.batch = 1;
    } else {
        a.A = M; a.sam = n; a.sak = 1; a.sab = 0;
        a.B = X; a.sbk = Q; a.sbn = 1; a.sbb = (long long)n * Q;
        a.C = Y; a.scm = Q; a.scn = 1; a.scb = (long long)n * Q;
        a.M = n; a.N = int(Q); a.K = n; a.batch = int(P);
    }
    a.n1 = c->n[0];
    a.n2 = c->n[1];
    return a;
}

enum FactorKind { FK_EXP_HALF = 0, FK_EXP_ONE = 1, FK_V = 2, FK_VINV = 3, FK_EXP_HALF_PRECISE = 4, FK_EXP_ALPHA = 5 };
static_assert(int(FK_EXP_HALF) == adr::BR_EXP_HALF && int(FK_EXP_ONE) == adr::BR_EXP_ONE && int(FK_V) == adr::BR_V &&
                  int(FK_VINV) == adr::BR_VINV,
              "factor kinds and batch roles share their numbering");

bool aligned16(const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

// Mixed batched context: one tensor-core pass over every instance (batch_tc.cu); inputs,
// outputs and the axpy base carry their low parts where the schedule keeps them.
void push_mode_batch_tc(Sched& S, int mu, int kind, const float* x, float* y, int epi, const float* base, double alpha,
                        int phik) {
    const adr_ctx* c = S.c;
    const adr_batch_state& b = *c->bs;
    adr::BatchTcArgs a;
    a.inst = static_cast<const adr::BatchTcInst*>(b.d_tci);
    a.items = b.d_titems[mu - 1];
    a.nitems = b.ntitems[mu - 1];
    a.mode = mu;
    a.role = kind == FK_EXP_ALPHA ? adr::BR_EXP_ALPHA : kind;
    a.fimg = b.d_img;
    a.fscale = b.d_fsc;
    a.X = x;
    a.Xlo = S.lo_of(x);
    a.Y = y;
    a.Ylo = S.lo_of(y);
    a.Yhs = S.hs_of(y);
    a.epi = epi;
    a.base = base;
    a.base_lo = S.lo_of(base);
    a.alpha = alpha;
    a.phi = epi == adr::EPI_PHI ? b.d_phi[phik] : nullptr;
    a.amax_in = S.consume(x);
    a.amax_out = S.produce(y);
    a.err = c->d_err;
    S.ops.push_back({[a](cudaStream_t s) { return adr::launch_batch_tc(a, s); }, OP_CONTRACT_TC});
}

// Batched context: one pass over every instance (one persistent launch).
template <typename T>
void push_mode_batch(Sched& S, int mu, int kind, const T* x, T* y, int epi, const T* base, double alpha, int phik) {
    const adr_ctx* c = S.c;
    const adr_batch_state& b = *c->bs;
    if (b.mixed) {
        if constexpr (sizeof(T) == 4) push_mode_batch_tc(S, mu, kind, x, y, epi, base, alpha, phik);
        return;
    }
    adr::BatchContractArgs<T> a;
    a.inst = static_cast<const adr::BatchInst<T>*>(b.d_inst);
    a.items = b.d_items[mu - 1];
    a.nitems = b.nitems[mu - 1];
    a.mode = mu;
    a.role = kind == FK_EXP_ALPHA ? adr::BR_EXP_ALPHA : kind;
    a.factors = static_cast<const T*>(b.d_f);
    a.zt = static_cast<const T*>(b.d_zt);
    a.X = x;
    a.Y = y;
    a.epi = epi;
    a.base = base;
    a.alpha = alpha;
    a.phik = phik;
    a.aligned = aligned16(x) && aligned16(y) && aligned16(base);
    a.grid = b.grid[mu - 1];
    S.ops.push_back({[a](cudaStream_t s) { return adr::launch_batch_contract(a, s); }, OP_CONTRACT_SIMT});
}

// Batched context: the stage combination of s over every instance, with each instance's
// own coefficients (the grid and coefficient fields of s are not used).
template <typename T>
adr::BatchStencilArgs<T> batch_stencil_args(const adr_ctx* c, const StencilArgs<T>& s) {
    const adr_batch_state& b = *c->bs;
    adr::BatchStencilArgs<T> a;
    a.inst = static_cast<const adr::BatchInst<T>*>(b.d_inst);
    a.row_start = b.d_row_start;
    a.ninst = b.B;
    a.rows = b.rows;
    a.a = static_cast<const T*>(b.d_a);
    a.u = s.u;
    a.nx = s.nx;
    a.nout = s.nout;
    for (int e = 0; e < adr::kMaxExtra; ++e) a.X[e] = s.X[e];
    for (int j = 0; j < adr::kMaxOut; ++j) {
        a.out[j] = s.out[j];
        a.cu[j] = s.cu[j];
        a.cg[j] = s.cg[j];
        a.cF[j] = s.cF[j];
        for (int e = 0; e < adr::kMaxExtra; ++e) a.cx[j][e] = s.cx[j][e];
    }
    a.grid = b.sgrid;
    return a;
}

const unsigned* Sched::consume(const void* buf) {
    for (auto& e : slot_of)
        if (e.first == buf) return slot(e.second);
    // not produced in this schedule (a caller's array): measure it first
    unsigned* sl = produce(buf);
    const float* x = static_cast<const float*>(buf);
    if (batch_mixed()) {
        const adr_batch_state& b = *c->bs;
        adr::BatchStencilArgs<float> g;
        g.inst = static_cast<const adr::BatchInst<float>*>(b.d_inst);
        g.row_start = b.d_row_start;
        g.ninst = b.B;
        g.rows = b.rows;
        ops.push_back({[g, x, sl](cudaStream_t s) { return adr::launch_batch_amax(g, x, sl, s); }, OP_AMAX});
        return sl;
    }
    const size_t N = c->N;
    ops.push_back({[x, N, sl](cudaStream_t s) { return adr::launch_amax(x, N, sl, s); }, OP_AMAX});
    return sl;
}

// One mu-mode pass y = x x_mu M_kind with epilogue (epi, base, alpha, phik).
template <typename T>
void push_mode(Sched& S, int mu, int kind, const T* x, T* y, int epi = adr::EPI_STORE,
               const T* base = nullptr, double alpha = 0.0, int phik = 0, T* ylo = nullptr,
               const T* xlo = nullptr) {
    const adr_ctx* c = S.c;
    if (c->bs) {
        push_mode_batch<T>(S, mu, kind, x, y, epi, base, alpha, phik);
        return;
    }
    if (!c->tc) {
        const void* M = kind >= kLevel0 ? c->d_El[kind - kLevel0][mu - 1]
                      : kind == FK_EXP_HALF ? c->d_E[0][mu - 1] : kind == FK_EXP_ONE ? c->d_E[1][mu - 1]
                      : kind == FK_EXP_ALPHA ? c->d_E[2][mu - 1]
                      : kind == FK_V ? c->d_V[mu - 1] : c->d_Vi[mu - 1];
        auto a = mode_args<T>(c, mu, static_cast<const T*>(M), x, y);
        a.epi = epi; a.base = base; a.alpha = alpha; a.phik = phik; a.ctau = c->p.tau;
        for (int m = 0; m < 3; ++m) a.lam[m] = (m < c->dim) ? c->d_lam[m] : nullptr;
        S.ops.push_back({[a](cudaStream_t s) { return adr::launch_contract(a, s); }, OP_CONTRACT_SIMT});
        return;
    }
    adr::TcArgs a;
    const int n = c->n[mu - 1];
    long long Q = 1, P = 1;
    for (int nu = 1; nu < mu; ++nu) Q *= c->n[nu - 1];
    for (int nu = mu + 1; nu <= c->dim; ++nu) P *= c->n[nu - 1];
    a.X = reinterpret_cast<const float*>(x);
    a.Xlo = reinterpret_cast<const float*>(xlo);
    a.Y = reinterpret_cast<float*>(y);
    a.precise = (kind == FK_EXP_HALF_PRECISE);
    a.fimg = c->d_img[kind][mu - 1];
    a.fscale = c->d_fsc[kind][mu - 1];
    a.n = n;
    a.Q = Q;
    a.state_is_a = (mu >= 2);
    a.vec4 = (mu == 1) && (n % 4 == 0) && (reinterpret_cast<uintptr_t>(x) % 16 == 0);
    a.npos = (mu >= 2) ? P * Q : P;
    a.nK = (n + 63) / 64;
    if (epi == adr::EPI_PHI) {
        // the phi scaling is fused into a mode >= 2 pass: decode (q, p) into the other directions
        a.zmu = c->d_zt[mu - 1];
        a.zq_a = c->d_zt[0];
        a.na = c->n[0];
        a.zq_b = (mu == 3) ? c->d_zt[1] : nullptr;
        a.zp = (mu == 2 && c->dim == 3) ? c->d_zt[2] : nullptr;
    }
    a.epi = epi;
    a.Ylo = reinterpret_cast<float*>(ylo);
    a.base = reinterpret_cast<const float*>(base);
    a.alpha = float(alpha);
    a.phik = phik;
    a.amax_in = S.consume(x);
    a.amax_out = S.produce(y);
    a.err = c->d_err;
    const int tc_kind = a.precise ? OP_CONTRACT_TC_PRECISE : OP_CONTRACT_TC;
    if (adr::tma_supported(n, Q, x, xlo)) {
        // TMA-fed kernel: position tiles of 128 consecutive q of one p, 128-row output tiles
        adr::TmaArgs t;
        static_cast<adr::TcArgs&>(t) = a;
        t.fimg = c->d_img2[kind][mu - 1];
        t.fscale = c->d_fsc2[kind][mu - 1];
        t.nK = (n + 31) / 32;
        t.nOut = (n + 127) / 128;
        t.nqt = (mu >= 2) ? (Q + 127) / 128 : 1;
        t.ntiles = ((mu >= 2) ? P * t.nqt : (P + 127) / 128) * t.nOut;
        const long long PP = P;
        S.ops.push_back({[t, PP](cudaStream_t s) { return adr::launch_contract_tma(t, PP, s); }, tc_kind});
        return;
    }
    // Register-fed kernel (shapes the TMA rules exclude): every pass in its precise variant, the
    // ten-product split into exact accumulators (its images are built in that layout); the low
    // part stays optional.
    adr::TcArgs r = a;
    r.precise = true;
    const int orows = adr::tc_out_rows(r.state_is_a, true), prows = adr::tc_pos_rows(r.state_is_a, true);
    r.nOut = (n + orows - 1) / orows;
    r.ntiles = ((r.npos + prows - 1) / prows) * r.nOut;
    S.ops.push_back({[r](cudaStream_t s) { return adr::launch_contract_tc(r, s); }, tc_kind});
}

// The device arrays of a periodic context as the Fourier kernels take them.
template <typename T>
adr::PeriodicArgs<T> periodic_args(const adr_ctx* c) {
    adr::PeriodicArgs<T> P;
    P.dim = c->dim;
    for (int m = 0; m < 3; ++m) P.n[m] = c->n[m];
    P.N = static_cast<long long>(c->N);
    P.Cu = static_cast<adr::Cplx<T>*>(c->d_pc[0]);
    for (int m = 0; m < c->dim; ++m) P.C[m] = static_cast<adr::Cplx<T>*>(c->d_pc[m + 1]);
    for (int m = 0; m < c->dim; ++m) {
        P.tw[m] = static_cast<const adr::Cplx<T>*>(c->d_ptw[m]);
        P.k[m] = static_cast<const T*>(c->d_pk[m]);
        P.a[m] = static_cast<const T*>(c->d_pa[m]);
        P.b[m] = static_cast<const T*>(c->d_pb[m]);
    }
    P.sym = static_cast<const adr::Cplx<T>*>(c->d_psym);
    for (int i = 0; i < 4; ++i) P.r[i] = c->r[i];
    P.adelta = c->p.form == ADR_FORM_ADELTA;
    P.dif = static_cast<T*>(c->d_pdif);
    P.CN = static_cast<adr::Cplx<T>*>(c->d_pcn);
    return P;
}

// Periodic contexts: y = base + alpha Re(F^-1 (M F x)) for the Fourier multiplier M
// (y = Re(F^-1 (M F x)) without base); mi indexes d_pm.
template <typename T>
void push_fourier(Sched& S, int mi, const T* x, T* y, const T* base, double alpha) {
    const adr_ctx* c = S.c;
    const auto P = periodic_args<T>(c);
    const auto* M = static_cast<const adr::Cplx<T>*>(c->d_pm[mi]);
    Op op{[P, M, x, y, base, alpha](cudaStream_t st) { return adr::launch_periodic_multiplier(P, M, x, y, base, alpha, st); },
          OP_FOURIER_MULT};
    op.launches = adr::periodic_multiplier_launches(c->dim);
    S.ops.push_back(op);
}

// A fused stage of a 2-D periodic context (see PeriodicStage). Multipliers by index into d_pm
// (-1: the identity); the Fourier-space array d_pz is read (cgz or cz nonzero) or written (save).
struct StageSpec {
    int mu = -1;                     // Mu
    double cu = 0;
    int mg = -1;                     // Mg
    double cgF = 0, cg = 0, cgz = 0, cz = 0;
    bool save = false;
    int ms = -1;                     // Ms
    double zu = 1, zF = 0, zg = 0;
    bool hand_on = false, take_over = false;   // chained stages (see PeriodicStage)
};

template <typename T>
void push_periodic_stage(Sched& S, const T* x, T* y, const StageSpec& q) {
    const adr_ctx* c = S.c;
    const auto P = periodic_args<T>(c);
    auto pm = [&](int i) { return i < 0 ? nullptr : static_cast<const adr::Cplx<T>*>(c->d_pm[i]); };
    adr::PeriodicStage<T> st;
    st.x = x;
    st.y = y;
    st.Mu = pm(q.mu);
    st.Mg = pm(q.mg);
    st.cu = q.cu;
    st.cgF = q.cgF;
    st.cg = q.cg;
    st.cgz = q.cgz;
    st.cz = q.cz;
    if (q.cgz != 0.0 || q.cz != 0.0) st.Z = static_cast<const adr::Cplx<T>*>(c->d_pz);
    if (q.save) {
        st.Zs = static_cast<adr::Cplx<T>*>(c->d_pz);
        st.Ms = pm(q.ms);
        st.zu = q.zu;
        st.zF = q.zF;
        st.zg = q.zg;
    }
    st.hand_on = q.hand_on;
    st.take_over = q.take_over;
    Op op{[P, st](cudaStream_t s) { return adr::launch_periodic_stage(P, st, s); }, OP_PERIODIC_STAGE};
    op.launches = adr::periodic_stage_launches(c->dim, q.take_over);
    S.ops.push_back(op);
}

// y = e^{c tau A} x, optionally finished by y = base + alpha * (e^{c tau A} x).
template <typename T>
void push_exp(Sched& S, int ci, const T* x, T* y, const T* base = nullptr, double alpha = 0.0) {
    const adr_ctx* c = S.c;
    if (c->periodic) {   // multipliers d_pm[0..2]: e^{tau s / 2}, e^{tau s}, e^{alpha tau s}
        push_fourier<T>(S, ci == FK_EXP_HALF ? 0 : ci == FK_EXP_ONE ? 1 : 2, x, y, base, alpha);
        return;
    }
    T* t0 = static_cast<T*>(c->ws[4]);
    T* t1 = static_cast<T*>(c->ws[5]);
    const T* in = x;
    for (int mu = 1; mu <= c->dim; ++mu) {
        T* out = (mu == c->dim) ? y : ((mu % 2) ? t0 : t1);
        const bool last = (mu == c->dim) && base;
        push_mode<T>(S, mu, ci, in, out, last ? adr::EPI_AXPY : adr::EPI_STORE, last ? base : nullptr, alpha);
        in = out;
    }
}

// Mixed path: y + ylo = e^{tau A / 2} x with every pass in the precise configuration and
// double-float intermediates (low parts in ws[6], ws[7]).
template <typename T>
void push_exp_precise(Sched& S, const T* x, T* y, T* ylo) {
    const adr_ctx* c = S.c;
    T* hi[2] = {static_cast<T*>(c->ws[4]), static_cast<T*>(c->ws[5])};
    T* lo[2] = {static_cast<T*>(c->ws[6]), static_cast<T*>(c->ws[7])};
    const T* in = x;
    const T* inlo = nullptr;
    for (int mu = 1; mu <= c->dim; ++mu) {
        const bool last = mu == c->dim;
        T* out = last ? y : hi[(mu - 1) % 2];
        T* outlo = last ? ylo : lo[(mu - 1) % 2];
        push_mode<T>(S, mu, FK_EXP_HALF_PRECISE, in, out, adr::EPI_STORE2, nullptr, 0.0, 0, outlo, inlo);
        in = out;
        inlo = outlo;
    }
}

template <typename T>
StencilArgs<T> stencil_base(const adr_ctx* c, const T* u);
template <typename T>
void push_stencil(Sched& S, StencilArgs<T> s, bool record_input = false);

// The stencil with zero (a - abar), no reaction and b = beta: F is then A u exactly (the
// constant-coefficient operator of Eq. (linop)), so out = cu u + sum cx X + cF A u.
template <typename T>
StencilArgs<T> linear_base(const adr_ctx* c, const T* u) {
    StencilArgs<T> s = stencil_base<T>(c, u);
    s.a = static_cast<const T*>(c->d_a0);
    for (int m = 0; m < 3; ++m) s.bmb[m] = 0.0;
    for (int i = 0; i < 4; ++i) s.r[i] = 0.0;
    return s;
}

double inv_factorial(int m) {
    double f = 1.0;
    for (int j = 2; j <= m; ++j) f *= j;
    return 1.0 / f;
}

// y = base + alpha phi_k(tau A) x (k = 1, 2) by exponentials only. With X = tau A / 2^s:
//   Taylor:   t = sum_{j=0}^{p} X^j x / (j+k)!  by Horner's rule, one stencil per term;
//             for k = 2 also phi_1(X) x = x + X phi_2(X) x.
//   Doubling: from the definitions of phi_1, phi_2,
//             phi_1(2X) = (e^X + I) phi_1(X) / 2,  phi_2(2X) = (phi_1(X) + (e^X + I) phi_2(X)) / 4.
//   Kept unnormalised, W1 = 2^i phi_1(2^i X) x and W2 = 4^i phi_2(2^i X) x obey
//             W1 <- e^{2^i X} W1 + W1,  W2 <- e^{2^i X} W2 + (W2 + 2^i W1),
//   so each level is exponential actions with plain axpy epilogues; at the end
//   phi_1(tau A) x = W1 / 2^s and phi_2(tau A) x = W2 / 4^s.
template <typename T>
void push_phi_doubling(Sched& S, int k, const T* x, T* y, const T* base, double alpha) {
    const adr_ctx* c = S.c;
    const int sh = c->dbl_s, p = c->dbl_p;
    const double c0 = std::ldexp(c->p.tau, -sh);
    T* W1 = static_cast<T*>(c->wsd[0]);
    T* W2 = static_cast<T*>(c->wsd[1]);
    T* Z = static_cast<T*>(c->wsd[2]);
    T* target = (k == 1) ? W1 : W2;
    const T* prev = x;
    for (int q = 0; q < p; ++q) {                          // coefficient j = p - 1 - q
        const int j = p - 1 - q;
        T* out = ((p - 1 - q) % 2 == 0) ? target : Z;
        auto st = linear_base<T>(c, prev);
        st.nx = 1; st.X[0] = x;
        st.nout = 1; st.out[0] = out;
        st.cx[0][0] = inv_factorial(j + k);
        st.cF[0] = (q == 0) ? c0 * inv_factorial(p + k) : c0;   // the first step starts from x / (p+k)!
        push_stencil(S, st);
        prev = out;
    }
    if (k == 2) {                                          // W1 = x + X W2
        auto st = linear_base<T>(c, W2);
        st.nx = 1; st.X[0] = x;
        st.nout = 1; st.out[0] = W1; st.cx[0][0] = 1.0; st.cF[0] = c0;
        push_stencil(S, st);
    }
    for (int i = 0; i < sh; ++i) {
        const int kind = kLevel0 + i;
        if (k == 2) {
            auto st = linear_base<T>(c, W2);               // Z = W2 + 2^i W1
            st.nx = 1; st.X[0] = W1;
            st.nout = 1; st.out[0] = Z; st.cu[0] = 1.0; st.cx[0][0] = std::ldexp(1.0, i);
            push_stencil(S, st);
            push_exp<T>(S, kind, W2, W2, Z, 1.0);
        }
        push_exp<T>(S, kind, W1, W1, W1, 1.0);
    }
    auto st = linear_base<T>(c, target);                   // y = base + alpha W / 2^(k s)
    st.nout = 1; st.out[0] = y;
    st.cu[0] = (base ? alpha : 1.0) * std::ldexp(1.0, -k * sh);
    if (base) { st.nx = 1; st.X[0] = base; st.cx[0][0] = 1.0; }
    push_stencil(S, st);
}

// y = phi_k(tau A) x through the eigenbasis (k = 0 gives e^{tau A}), optionally
// finished by y = base + alpha * (phi_k(tau A) x). Contexts on the doubling route apply
// phi_1, phi_2 by exponentials only (push_phi_doubling) and phi_0 with the dense e^{tau A}.
template <typename T>
void push_phi(Sched& S, int k, const T* x, T* y, const T* base = nullptr, double alpha = 0.0) {
    const adr_ctx* c = S.c;
    if (c->periodic) {   // multipliers d_pm[1], d_pm[3], d_pm[4]: phi_0, phi_1, phi_2 of tau s
        push_fourier<T>(S, k == 0 ? 1 : k == 1 ? 3 : 4, x, y, base, alpha);
        return;
    }
    if (c->phi_route == ADR_PHI_DOUBLING) {
        if (k == 0) push_exp<T>(S, FK_EXP_ONE, x, y, base, base ? alpha : 0.0);
        else push_phi_doubling<T>(S, k, x, y, base, alpha);
        return;
    }
    T* tmp[2] = {static_cast<T*>(c->ws[4]), static_cast<T*>(c->ws[5])};
    int flip = 0;
    const T* in = x;
    for (int mu = 1; mu <= c->dim; ++mu) {       // forward: V_mu^-1, phi_k on the last
        T* out = tmp[flip]; flip ^= 1;
        if (mu == c->dim) push_mode<T>(S, mu, FK_VINV, in, out, adr::EPI_PHI, nullptr, 0.0, k);
        else              push_mode<T>(S, mu, FK_VINV, in, out);
        in = out;
    }
    for (int mu = c->dim; mu >= 1; --mu) {       // back: V_mu
        T* out = (mu == 1) ? y : tmp[flip];
        if (mu != 1) flip ^= 1;
        const bool last = (mu == 1) && base;
        push_mode<T>(S, mu, FK_V, in, out, last ? adr::EPI_AXPY : adr::EPI_STORE, last ? base : nullptr, alpha);
        in = out;
    }
}

template <typename T>
StencilArgs<T> stencil_base(const adr_ctx* c, const T* u) {
    StencilArgs<T> s;
    s.u = u;
    s.err = c->d_err;
    s.a = static_cast<const T*>(c->d_a);
    s.apitch = c->apitch;
    s.dim = c->dim;
    s.n1 = c->n[0];
    s.n2 = c->n[1];
    s.n3 = c->dim == 3 ? c->n[2] : 1;
    s.neumann = c->p.bc_hi == ADR_BC_NEUMANN;
    s.adelta = c->p.form == ADR_FORM_ADELTA;
    for (int m = 0; m < c->dim; ++m) {
        const double h = s.neumann ? 1.0 / c->n[m] : 1.0 / (c->n[m] + 1);
        s.inv_h2[m] = 1.0 / (h * h);
        s.inv_2h[m] = 1.0 / (2.0 * h);
        s.bmb[m] = c->b[m] - c->beta[m];
        s.beta[m] = c->beta[m];
    }
    s.abar = c->abar;
    for (int i = 0; i < 4; ++i) s.r[i] = c->r[i];
    return s;
}

// Push a stencil op; on the mixed path its outputs (and, if asked, its input) get slots.
template <typename T>
void push_stencil(Sched& S, StencilArgs<T> s, bool record_input) {
    if (S.c->periodic) {   // the pseudospectral right-hand side (periodic.cu)
        const auto P = periodic_args<T>(S.c);
        Op op{[P, s](cudaStream_t st) { return adr::launch_periodic_rhs(P, s, st); }, OP_PERIODIC_RHS};
        op.launches = adr::periodic_rhs_launches(S.c->dim, s.nout);
        S.ops.push_back(op);
        return;
    }
    if (S.c->bs) {
        const auto a = batch_stencil_args(S.c, s);
        if constexpr (sizeof(T) == 4) {
            if (S.batch_mixed()) {   // compensated stencil: low parts in and out, max|out| per instance
                adr::BatchStencil2Args P;
                P.s = a;
                P.units = S.c->bs->d_sunits;
                P.nunits = S.c->bs->nsunits;
                P.u_lo = S.lo_of(s.u);
                for (int e = 0; e < s.nx; ++e) P.X_lo[e] = S.lo_of(s.X[e]);
                for (int j = 0; j < s.nout; ++j) {
                    P.out_lo[j] = S.lo_of(s.out[j]);
                    P.out_hs[j] = S.hs_of(s.out[j]);
                    P.amax[j] = S.produce(s.out[j]);
                }
                S.ops.push_back({[P](cudaStream_t st) { return adr::launch_batch_stencil2(P, st); }, OP_STENCIL});
                return;
            }
        }
        S.ops.push_back({[a](cudaStream_t st) { return adr::launch_batch_stencil(a, st); }, OP_STENCIL});
        return;
    }
    if (S.c->tc) {
        if (record_input) s.amax_u = S.produce(s.u);
        for (int j = 0; j < s.nout; ++j) s.amax[j] = S.produce(s.out[j]);
    }
    S.ops.push_back({[s](cudaStream_t st) { return adr::launch_stencil(s, st); }, OP_STENCIL});
}

// The step of a 2-D periodic context as stages kept in Fourier space from the state's transform
// to the stage result (see PeriodicStage); false for a scheme without that form (Lawson4 and
// stabilized Lawson2 keep more than one array between stages). d_pm: 0 e^{tau s/2}, 1 e^{tau s},
// 3 phi_1(tau s), 4 phi_2(tau s).
template <typename T>
bool push_fused_periodic_step(Sched& S, const adr_ctx* c, T* u) {
    if (!c->periodic || c->dim != 2) return false;
    constexpr int kEh = 0, kE1 = 1, kPhi1 = 3, kPhi2 = 4;
    const double tau = c->p.tau;
    T* B0 = static_cast<T*>(c->ws[0]);
    StageSpec a, b;
    switch (c->p.scheme) {
    case ADR_LAWSON_EULER:                       // u+ = E_1 (u + tau g(u))
        a.mu = kE1; a.cu = 1.0; a.mg = kE1; a.cgF = a.cg = tau;
        push_periodic_stage<T>(S, u, u, a);
        return true;
    case ADR_STABILIZED_LAWSON_EULER:            // u+ = u + tau E_1 F(u)
    case ADR_EXPONENTIAL_EULER:                  // u+ = u + tau phi_1 F(u)
        a.cu = 1.0; a.mg = c->p.scheme == ADR_EXPONENTIAL_EULER ? kPhi1 : kE1; a.cgF = tau;
        push_periodic_stage<T>(S, u, u, a);
        return true;
    case ADR_ETD2RK:                             // U = u + tau phi_1 F(u), Z = g(u)^;
    case ADR_ERK2P1: {                           // u+ = U + h phi_k (g(U)^ - Z)
        a.cu = 1.0; a.mg = kPhi1; a.cgF = tau;
        a.save = true; a.zu = 0.0; a.zF = 1.0; a.zg = 1.0;
        const bool etd = c->p.scheme == ADR_ETD2RK;
        const double h = etd ? tau : 0.5 * tau;  // ETD2RK: tau phi_2; erk2p1: tau/2 phi_1
        b.cu = 1.0; b.mg = etd ? kPhi2 : kPhi1; b.cgF = b.cg = h; b.cgz = -h;
        break;
    }
    case ADR_LAWSON2A:                           // U = E_h (u + tau/2 g(u)), Z = E_1 u^;
        a.mu = kEh; a.cu = 1.0; a.mg = kEh; a.cgF = a.cg = 0.5 * tau;
        a.save = true; a.ms = kE1;
        b.mg = kEh; b.cgF = b.cg = tau; b.cz = 1.0;   // u+ = Z + tau E_h g(U)^
        break;
    case ADR_LAWSON2B:                           // U = E_1 (u + tau g(u)), Z = E_1 (u^ + tau/2 g(u)^);
        a.mu = kE1; a.cu = 1.0; a.mg = kE1; a.cgF = a.cg = tau;
        a.save = true; a.ms = kE1; a.zF = a.zg = 0.5 * tau;
        b.cgF = b.cg = 0.5 * tau; b.cz = 1.0;          // u+ = Z + tau/2 g(U)^
        break;
    default:
        return false;
    }
    a.hand_on = b.take_over = true;            // stage b's input is stage a's result B0
    push_periodic_stage<T>(S, u, B0, a);
    push_periodic_stage<T>(S, B0, u, b);
    return true;
}

template <typename T>
std::vector<Op> build_step(const adr_ctx* c, T* u) {
    Sched S(c);
    S.bind_state(u);
    const double tau = c->p.tau;
    if (push_fused_periodic_step<T>(S, c, u)) return std::move(S.ops);
    T* B0 = static_cast<T*>(c->ws[0]);
    T* B1 = static_cast<T*>(c->ws[1]);
    T* B2 = static_cast<T*>(c->ws[2]);
    T* B3 = static_cast<T*>(c->ws[3]);
    switch (c->p.scheme) {
    case ADR_LAWSON_EULER: {
        auto s = stencil_base<T>(c, u);
        s.nout = 1; s.out[0] = B0; s.cu[0] = 1.0; s.cg[0] = tau;       // W = u + tau g(u)
        push_stencil(S, s);
        push_exp<T>(S, FK_EXP_ONE, B0, u);                               // u = e^{tau A} W
        break;
    }
    case ADR_ETD2RK: {
        auto s1 = stencil_base<T>(c, u);
        s1.nout = 2; s1.out[0] = B0; s1.cF[0] = 1.0;                    // F(u)
        s1.out[1] = B1; s1.cg[1] = 1.0;                                 // G0 = g(u)
        push_stencil(S, s1);
        push_phi<T>(S, 1, B0, B2, u, tau);                               // U = u + tau phi1 F
        auto s2 = stencil_base<T>(c, B2);
        s2.nx = 1; s2.X[0] = B1;
        s2.nout = 1; s2.out[0] = B0; s2.cg[0] = 1.0; s2.cx[0][0] = -1.0; // D = g(U) - G0
        push_stencil(S, s2);
        push_phi<T>(S, 2, B0, u, B2, tau);                               // u = U + tau phi2 D
        break;
    }
    case ADR_LAWSON4: {
        T* W = B0; T* X = B1; T* Eu = B2; T* ACC = B3;
        auto s1 = stencil_base<T>(c, u);
        s1.nout = 1; s1.out[0] = W; s1.cu[0] = 1.0; s1.cg[0] = 0.5 * tau;       // u + tau/2 k1
        push_stencil(S, s1, /*record_input=*/true);
        push_exp<T>(S, FK_EXP_HALF, W, X);                                        // U2
        push_exp<T>(S, FK_EXP_HALF, u, Eu);                                       // Eu
        auto s2 = stencil_base<T>(c, X);
        s2.nx = 1; s2.X[0] = Eu;
        s2.nout = 2;
        s2.out[0] = W; s2.cx[0][0] = 1.0; s2.cg[0] = 0.5 * tau;                  // U3 = Eu + tau/2 k2
        s2.out[1] = ACC; s2.cx[1][0] = 2.0 / 3.0; s2.cu[1] = 1.0 / 3.0; s2.cg[1] = tau / 3.0;
        push_stencil(S, s2);
        auto s3 = stencil_base<T>(c, W);
        s3.nx = 2; s3.X[0] = Eu; s3.X[1] = ACC;
        s3.nout = 2;
        s3.out[0] = X; s3.cx[0][0] = 1.0; s3.cg[0] = tau;                         // Eu + tau k3
        s3.out[1] = ACC; s3.cx[1][1] = 1.0; s3.cg[1] = tau / 3.0;                 // ACC += tau/3 k3
        push_stencil(S, s3);
        // U4 feeds the one stencil whose output no later exponential smooths (u+ = ... +
        // tau/6 g(U4)); on the mixed path it is kept as a double-float pair W + Wlo so that
        // FP32 rounding of U4 is not amplified by the 1/h^2 of the stencil.
        T* Wlo = c->tc ? static_cast<T*>(c->ws[8]) : nullptr;
        if (c->tc) push_exp_precise<T>(S, X, W, Wlo);                            // U4 (double-float)
        else       push_exp<T>(S, FK_EXP_HALF, X, W);                            // U4
        push_exp<T>(S, FK_EXP_HALF, ACC, X);                                      // E ACC
        auto s4 = stencil_base<T>(c, W);
        s4.u_lo = Wlo;
        s4.nx = 1; s4.X[0] = X;
        s4.nout = 1; s4.out[0] = u; s4.cx[0][0] = 1.0; s4.cg[0] = tau / 6.0;     // u+ = E ACC + tau/6 k4
        push_stencil(S, s4);
        break;
    }
    case ADR_EXPONENTIAL_EULER: {
        auto s = stencil_base<T>(c, u);
        s.nout = 1; s.out[0] = B0; s.cF[0] = 1.0;                       // F(u)
        push_stencil(S, s);
        push_phi<T>(S, 1, B0, u, u, tau);                                // u = u + tau phi1 F
        break;
    }
    case ADR_ERK2P1: {
        auto s1 = stencil_base<T>(c, u);
        s1.nout = 2; s1.out[0] = B0; s1.cF[0] = 1.0;                    // F(u)
        s1.out[1] = B1; s1.cg[1] = 1.0;                                 // G0 = g(u)
        push_stencil(S, s1);
        push_phi<T>(S, 1, B0, B2, u, tau);                               // U = u + tau phi1 F
        auto s2 = stencil_base<T>(c, B2);
        s2.nx = 1; s2.X[0] = B1;
        s2.nout = 1; s2.out[0] = B0; s2.cg[0] = 1.0; s2.cx[0][0] = -1.0; // D = g(U) - G0
        push_stencil(S, s2);
        push_phi<T>(S, 1, B0, u, B2, 0.5 * tau);                         // u = U + tau/2 phi1 D
        break;
    }
    case ADR_STABILIZED_LAWSON_EULER: {
        auto s = stencil_base<T>(c, u);
        s.nout = 1; s.out[0] = B0; s.cF[0] = 1.0;                       // F(u)
        push_stencil(S, s);
        push_exp<T>(S, FK_EXP_ONE, B0, u, u, tau);                       // u = u + tau e^{tau A} F
        break;
    }
    case ADR_LAWSON2A: {
        auto s1 = stencil_base<T>(c, u);
        s1.nout = 1; s1.out[0] = B0; s1.cu[0] = 1.0; s1.cg[0] = 0.5 * tau; // u + tau/2 g(u)
        push_stencil(S, s1);
        push_exp<T>(S, FK_EXP_HALF, B0, B1);                             // U = e^{tau A/2}(...)
        push_exp<T>(S, FK_EXP_ONE, u, B2);                               // e^{tau A} u
        auto s2 = stencil_base<T>(c, B1);
        s2.nout = 1; s2.out[0] = B0; s2.cg[0] = 1.0;                     // g(U)
        push_stencil(S, s2);
        push_exp<T>(S, FK_EXP_HALF, B0, u, B2, tau);                     // u = e^{tau A} u + tau e^{tau A/2} g(U)
        break;
    }
    case ADR_LAWSON2B: {
        auto s1 = stencil_base<T>(c, u);
        s1.nout = 2;
        s1.out[0] = B0; s1.cu[0] = 1.0; s1.cg[0] = tau;                  // u + tau g(u)
        s1.out[1] = B1; s1.cu[1] = 1.0; s1.cg[1] = 0.5 * tau;            // u + tau/2 g(u)
        push_stencil(S, s1);
        push_exp<T>(S, FK_EXP_ONE, B0, B2);                              // U = e^{tau A}(u + tau g(u))
        push_exp<T>(S, FK_EXP_ONE, B1, B3);                              // e^{tau A}(u + tau/2 g(u))
        auto s2 = stencil_base<T>(c, B2);
        s2.nx = 1; s2.X[0] = B3;
        s2.nout = 1; s2.out[0] = u; s2.cx[0][0] = 1.0; s2.cg[0] = 0.5 * tau; // u = ... + tau/2 g(U)
        push_stencil(S, s2);
        break;
    }
    case ADR_STABILIZED_LAWSON2: {
        const double al = adr::kLawsonAlpha;
        auto s1 = stencil_base<T>(c, u);
        s1.nout = 2; s1.out[0] = B0; s1.cF[0] = 1.0;                    // F(u)
        s1.out[1] = B1; s1.cg[1] = 1.0;                                 // G0 = g(u)
        push_stencil(S, s1);
        push_exp<T>(S, FK_EXP_ALPHA, B0, B2, u, al * tau);               // U = u + alpha tau e^{alpha tau A} F
        push_exp<T>(S, FK_EXP_HALF, B0, B3, u, tau);                     // u + tau e^{tau A/2} F
        auto s2 = stencil_base<T>(c, B2);
        s2.nx = 1; s2.X[0] = B1;
        s2.nout = 1; s2.out[0] = B0; s2.cg[0] = 1.0; s2.cx[0][0] = -1.0; // D = g(U) - G0
        push_stencil(S, s2);
        push_exp<T>(S, FK_EXP_ONE, B0, u, B3, tau / (2.0 * al));         // u = ... + tau/(2 alpha) e^{tau A} D
        break;
    }
    default:
        break;
    }
    if (S.overflow)   // more produced arrays than max-abs slots: refuse the schedule
        S.ops.push_back({[](cudaStream_t) { return cudaErrorInvalidValue; }, OP_MEMSET});
    return std::move(S.ops);
}

std::vector<Op> step_ops(const adr_ctx* c, void* u) {
    return c->fp64 ? build_step<double>(c, static_cast<double*>(u)) : build_step<float>(c, static_cast<float*>(u));
}

// NVTX range names of the op kinds (a profiler attributes the kernels an op launches to its range).
const char* op_name(int kind) {
    switch (kind) {
    case OP_MEMSET: return "max-abs slots: clear";
    case OP_AMAX: return "max-abs / low-part check";
    case OP_STENCIL: return "K1 stencil + stage combination";
    case OP_CONTRACT_SIMT: return "K2 mu-mode pass (FMA)";
    case OP_CONTRACT_TC: return "K2 mu-mode pass (tensor cores)";
    case OP_CONTRACT_TC_PRECISE: return "K2 mu-mode pass (tensor cores, double-float)";
    case OP_PERIODIC_RHS: return "periodic right-hand side (Fourier passes)";
    case OP_FOURIER_MULT: return "Fourier multiplier";
    case OP_PERIODIC_STAGE: return "periodic stage in Fourier space";
    default: return "op";
    }
}

// Enqueue ops directly (not under capture), each inside an NVTX range, the whole in one.
adr_status run_ops(adr_ctx* c, const std::vector<Op>& ops, const char* where) {
    nvtxRangePushA(where);
    for (const auto& op : ops) {
        nvtxRangePushA(op_name(op.kind));
        cudaError_t e = op(c->stream);
        nvtxRangePop();
        if (e != cudaSuccess) {
            nvtxRangePop();
            return cuda_fail(c, e, where);
        }
    }
    nvtxRangePop();
    return ADR_OK;
}

bool needs_phi(int scheme) {
    return scheme == ADR_ETD2RK || scheme == ADR_EXPONENTIAL_EULER || scheme == ADR_ERK2P1;
}

adr_status check_ready(adr_ctx* c) {
    if (!c) return ADR_ERR_ARG;
    if (!c->coeffs_set)
        return fail(c, ADR_ERR_STATE, c->bs ? "adr_set_coeffs has not been called for every instance"
                                            : "adr_set_coeffs has not been called");
    return ADR_OK;
}

}  // namespace

namespace {

// ------------------------------------------------------------------ batched contexts
constexpr int kCoef = 13;   // per instance: ih2[2] i2h[2] bmb[2] beta[2] abar r[4]

int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Copy src[off, off + len) (FP64 staging) to the same elements of a device array of the
// working precision.
cudaError_t upload_range(const adr_ctx* c, void* dst, const std::vector<double>& src, long long off, long long len) {
    if (len <= 0) return cudaSuccess;
    char* d = static_cast<char*>(dst) + off * static_cast<long long>(c->esize);
    if (c->fp64) return cudaMemcpy(d, src.data() + off, size_t(len) * 8, cudaMemcpyHostToDevice);
    std::vector<float> tmp(src.begin() + off, src.begin() + off + len);
    return cudaMemcpy(d, tmp.data(), size_t(len) * 4, cudaMemcpyHostToDevice);
}

template <typename T>
cudaError_t upload_instances(const adr_ctx* c) {
    const adr_batch_state& b = *c->bs;
    std::vector<adr::BatchInst<T>> h(b.B);
    for (int i = 0; i < b.B; ++i) {
        auto& d = h[i];
        const double* k = &b.coef[size_t(i) * kCoef];
        d.n1 = b.n1[i];
        d.n2 = b.n2[i];
        d.off = b.off[i];
        d.row0 = b.row0[i];
        d.a_off = b.a_off[i];
        d.apitch = b.apitch[i];
        for (int m = 0; m < 2; ++m) {
            d.ih2[m] = T(k[m]);
            d.i2h[m] = T(k[2 + m]);
            d.bmb[m] = T(k[4 + m]);
            d.beta[m] = T(k[6 + m]);
            d.zt_off[m] = b.zt_off[size_t(i) * 2 + m];
        }
        bool vec = (b.n1[i] % 4 == 0) && (b.n2[i] % 4 == 0) && (b.off[i] % 4 == 0);
        d.abar = T(k[8]);
        for (int j = 0; j < 4; ++j) d.r[j] = T(k[9 + j]);
        for (int r = 0; r < adr::kBatchRoles; ++r)
            for (int m = 0; m < 2; ++m) {
                d.f_off[r][m] = b.f_off[size_t(i) * 2 * adr::kBatchRoles + r * 2 + m];
                if (d.f_off[r][m] >= 0 && d.f_off[r][m] % 4 != 0) vec = false;
            }
        d.vec = vec ? 1 : 0;
    }
    return cudaMemcpy(b.d_inst, h.data(), h.size() * sizeof(adr::BatchInst<T>), cudaMemcpyHostToDevice);
}

// Upload everything (first time) or the regions of instance i (later changes).
cudaError_t batch_upload(adr_ctx* c, int i) {
    adr_batch_state& b = *c->bs;
    cudaError_t e = c->fp64 ? upload_instances<double>(c) : upload_instances<float>(c);
    if (e != cudaSuccess) return e;
    if (!b.uploaded) {
        e = upload_range(c, b.d_a, b.hA, 0, b.a_len);
        if (e == cudaSuccess) e = upload_range(c, b.d_f, b.hF, 0, b.f_len);
        if (e == cudaSuccess) e = upload_range(c, b.d_zt, b.hZt, 0, b.zt_len);
        if (e == cudaSuccess) b.uploaded = true;
        return e;
    }
    e = upload_range(c, b.d_a, b.hA, b.a_off[i], (long long)b.apitch[i] * (b.n2[i] + 2));
    for (int r = 0; r < adr::kBatchRoles && e == cudaSuccess; ++r)
        for (int m = 0; m < 2 && e == cudaSuccess; ++m) {
            const long long o = b.f_off[size_t(i) * 2 * adr::kBatchRoles + r * 2 + m];
            const long long nm = m == 0 ? b.n1[i] : b.n2[i];
            if (o >= 0) e = upload_range(c, b.d_f, b.hF, o, nm * nm);
        }
    for (int m = 0; m < 2 && e == cudaSuccess; ++m) {
        const long long o = b.zt_off[size_t(i) * 2 + m];
        const long long nm = m == 0 ? b.n1[i] : b.n2[i];
        if (o >= 0) e = upload_range(c, b.d_zt, b.hZt, o, nm);
    }
    return e;
}

// Work items of the instances `insts` with tile shape t: {instance, tile row, tile column, t}.
void append_items(const adr_batch_state& b, const std::vector<int>& insts, int t, std::vector<int4>& out) {
    const int edge = adr::batch_tile_edge(t);
    for (int i : insts)
        for (int ty = 0; ty < (b.n2[i] + edge - 1) / edge; ++ty)
            for (int tx = 0; tx < (b.n1[i] + edge - 1) / edge; ++tx) out.push_back(make_int4(i, ty, tx, t));
}

// Autotuner. Per instance size (n1, n2) and mode it times each candidate tile shape on the
// items of that size class and keeps the fastest; the full item list of a mode is then
// ordered by the measured cost per item, largest first (longest-processing-time order for
// the persistent CTAs that take items round robin); last it times the full list at 1-4
// CTAs per SM, and the stencil at 4, 8 and 16 CTAs per SM.
template <typename T>
adr_status batch_tune(adr_ctx* c) {
    adr_batch_state& b = *c->bs;
    const int sms = device_sms();
    std::vector<std::pair<std::pair<int, int>, std::vector<int>>> classes;
    for (int i = 0; i < b.B; ++i) {
        const std::pair<int, int> key(b.n1[i], b.n2[i]);
        auto it = classes.begin();
        while (it != classes.end() && it->first != key) ++it;
        if (it == classes.end()) classes.push_back({key, {i}});
        else it->second.push_back(i);
    }
    int role = 0;
    while (role < adr::kBatchRoles && !b.roles[role]) ++role;
    long long max_items = 0;
    for (int i = 0; i < b.B; ++i) max_items += (long long)((b.n1[i] + 31) / 32) * ((b.n2[i] + 31) / 32);
    int4* d_tmp = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&d_tmp), size_t(max_items) * sizeof(int4));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto cleanup = [&]() {
        if (d_tmp) cudaFree(d_tmp);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "autotuner set-up"); }
    // the fastest of 3 timed launches after 2 untimed ones
    auto best_of = [&](const std::function<cudaError_t(cudaStream_t)>& launch, float& ms) -> cudaError_t {
        ms = 1e30f;
        for (int r = 0; r < 5; ++r) {
            cudaError_t le = cudaEventRecord(e0, c->stream);
            if (le == cudaSuccess) le = launch(c->stream);
            if (le == cudaSuccess) le = cudaEventRecord(e1, c->stream);
            if (le == cudaSuccess) le = cudaEventSynchronize(e1);
            float t = 0.f;
            if (le == cudaSuccess) le = cudaEventElapsedTime(&t, e0, e1);
            if (le != cudaSuccess) return le;
            if (r >= 2 && t < ms) ms = t;
        }
        return cudaSuccess;
    };
    adr::BatchContractArgs<T> base;
    base.inst = static_cast<const adr::BatchInst<T>*>(b.d_inst);
    base.role = role;
    base.factors = static_cast<const T*>(b.d_f);
    base.zt = static_cast<const T*>(b.d_zt);
    base.aligned = aligned16(c->ws[0]) && aligned16(c->ws[1]);
    base.X = static_cast<const T*>(c->ws[0]);
    base.Y = static_cast<T*>(c->ws[1]);
    base.epi = adr::EPI_STORE;
    for (int mode = 1; mode <= 2 && e == cudaSuccess; ++mode) {
        std::vector<std::pair<double, int4>> all;
        for (const auto& cl : classes) {
            int best_t = b.tile_force >= 0 ? b.tile_force : adr::BT_64;
            float best_ms = 1e30f;
            for (int t = 0; t < adr::kBatchTiles && e == cudaSuccess; ++t) {
                if (b.tile_force >= 0 && t != b.tile_force) continue;
                std::vector<int4> items;
                append_items(b, cl.second, t, items);
                e = cudaMemcpy(d_tmp, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
                auto a = base;
                a.items = d_tmp;
                a.nitems = int(items.size());
                a.mode = mode;
                a.grid = std::min(int(items.size()), 2 * sms);
                float ms = 0.f;
                if (e == cudaSuccess) e = best_of([a](cudaStream_t s) { return adr::launch_batch_contract(a, s); }, ms);
                if (e == cudaSuccess && ms < best_ms) { best_ms = ms; best_t = t; }
            }
            std::vector<int4> items;
            append_items(b, cl.second, best_t, items);
            const double g = double(std::min(int(items.size()), 2 * sms));
            const double per_item = double(best_ms) * g / double(items.size());
            for (int i : cl.second) b.tile[mode - 1][i] = best_t;
            for (const auto& it : items) all.push_back({per_item, it});
        }
        if (e != cudaSuccess) break;
        std::stable_sort(all.begin(), all.end(), [](const std::pair<double, int4>& x, const std::pair<double, int4>& y) {
            return x.first > y.first;
        });
        std::vector<int4> items(all.size());
        for (size_t k = 0; k < all.size(); ++k) items[k] = all[k].second;
        if (b.d_items[mode - 1]) cudaFree(b.d_items[mode - 1]);
        b.d_items[mode - 1] = nullptr;
        e = cudaMalloc(reinterpret_cast<void**>(&b.d_items[mode - 1]), items.size() * sizeof(int4));
        if (e == cudaSuccess)
            e = cudaMemcpy(b.d_items[mode - 1], items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
        b.nitems[mode - 1] = int(items.size());
        float best_ms = 1e30f;
        b.grid[mode - 1] = std::min(b.nitems[mode - 1], 2 * sms);
        for (int per_sm = 1; per_sm <= 4 && e == cudaSuccess; ++per_sm) {
            auto a = base;
            a.items = b.d_items[mode - 1];
            a.nitems = b.nitems[mode - 1];
            a.mode = mode;
            a.grid = std::min(a.nitems, per_sm * sms);
            float ms = 0.f;
            e = best_of([a](cudaStream_t s) { return adr::launch_batch_contract(a, s); }, ms);
            if (e == cudaSuccess && ms < best_ms) { best_ms = ms; b.grid[mode - 1] = a.grid; }
        }
    }
    if (e == cudaSuccess) {
        adr::BatchStencilArgs<T> s;
        s.inst = static_cast<const adr::BatchInst<T>*>(b.d_inst);
        s.row_start = b.d_row_start;
        s.ninst = b.B;
        s.rows = b.rows;
        s.a = static_cast<const T*>(b.d_a);
        s.u = static_cast<const T*>(c->ws[0]);
        s.nout = 1;
        s.out[0] = static_cast<T*>(c->ws[1]);
        s.cg[0] = 1.0;
        float best_ms = 1e30f;
        b.sgrid = 8 * sms;
        for (int per_sm : {4, 8, 16}) {
            s.grid = per_sm * sms;
            float ms = 0.f;
            e = best_of([s](cudaStream_t st) { return adr::launch_batch_stencil(s, st); }, ms);
            if (e != cudaSuccess) break;
            if (ms < best_ms) { best_ms = ms; b.sgrid = s.grid; }
        }
    }
    cleanup();
    if (e != cudaSuccess) return cuda_fail(c, e, "autotuner");
    b.tuned = true;
    return ADR_OK;
}

// phi_k(z) for real z in FP64: the Taylor series for |z| < 1, the closed forms with expm1 elsewhere.
double phi_real(int k, double z) {
    if (k == 0) return std::exp(z);
    if (std::fabs(z) < 1.0) {
        double acc = 0.0;
        for (int j = 29; j >= 0; --j) acc = acc * z + inv_factorial(j + k);
        return acc;
    }
    const double em1 = std::expm1(z);
    return k == 1 ? em1 / z : (em1 - z) / (z * z);
}

// Mixed batched context, instance i: slice its factors for the tensor cores (batch_tc.cu)
// and upload them with their row scales; for the phi schemes also the double-float tables
// phi_k(tau (lambda_1[i1] + lambda_2[i2])), k = 0, 1, 2, at the instance's nodes.
cudaError_t batch_mixed_instance(adr_ctx* c, int i) {
    adr_batch_state& b = *c->bs;
    const adr::BatchTcInst& t = b.tci[size_t(i)];
    const int n[2] = {t.n1, t.n2};
    cudaError_t e = cudaSuccess;
    std::vector<uint8_t> img;
    std::vector<float> fsc;
    for (int r = 0; r < adr::kBatchRoles && e == cudaSuccess; ++r)
        for (int m = 0; m < 2 && e == cudaSuccess; ++m) {
            if (!b.roles[r]) continue;
            const double* M = &b.hF[size_t(b.f_off[size_t(i) * 2 * adr::kBatchRoles + r * 2 + m])];
            img.assign(adr::batch_tc_image_bytes(n[m], m + 1), 0);
            fsc.assign(size_t(n[m]), 0.0f);
            adr::make_batch_tc_factor(M, n[m], m + 1, img.data(), fsc.data());
            e = cudaMemcpy(b.d_img + t.img_off[r][m], img.data(), img.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(b.d_fsc + t.fsc_off[r][m], fsc.data(), fsc.size() * sizeof(float), cudaMemcpyHostToDevice);
        }
    if (e != cudaSuccess || !b.roles[adr::BR_V]) return e;
    const double* z1 = &b.hZt[size_t(b.zt_off[size_t(i) * 2])];
    const double* z2 = &b.hZt[size_t(b.zt_off[size_t(i) * 2 + 1])];
    std::vector<float2> tab(size_t(t.n1) * t.n2);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        for (int i2 = 0; i2 < t.n2; ++i2)
            for (int i1 = 0; i1 < t.n1; ++i1) {
                const double v = phi_real(k, z1[i1] + z2[i2]);
                const float hi = float(v);
                tab[size_t(i2) * t.n1 + i1] = make_float2(hi, float(v - double(hi)));
            }
        e = cudaMemcpy(b.d_phi[k] + t.off, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice);
    }
    return e;
}

// Mixed batched context, once every instance is set: the instance table and the work items of
// the tensor-core passes, instances in order of decreasing size (longest-processing-time order
// for the persistent CTAs that take items round robin). Mode 1: 64-row x2 tiles x 128 outputs
// along x1; mode 2: 128-position x1 tiles x 64 outputs along x2.
cudaError_t batch_mixed_plan(adr_ctx* c) {
    adr_batch_state& b = *c->bs;
    cudaError_t e = cudaMemcpy(b.d_tci, b.tci.data(), b.tci.size() * sizeof(adr::BatchTcInst), cudaMemcpyHostToDevice);
    std::vector<int> order(size_t(b.B));
    for (int i = 0; i < b.B; ++i) order[size_t(i)] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (long long)b.n1[x] * b.n2[x] * (b.n1[x] + b.n2[x]) > (long long)b.n1[y] * b.n2[y] * (b.n1[y] + b.n2[y]);
    });
    for (int mode = 1; mode <= 2 && e == cudaSuccess; ++mode) {
        std::vector<int4> items;
        for (int i : order) {
            const int n1 = b.n1[i], n2 = b.n2[i];
            const int npt = mode == 1 ? (n2 + 63) / 64 : (n1 + 127) / 128;
            const int nout = mode == 1 ? (n1 + 127) / 128 : (n2 + 63) / 64;
            for (int pt = 0; pt < npt; ++pt)
                for (int ot = 0; ot < nout; ++ot) items.push_back(make_int4(i, pt, ot, 0));
        }
        if (b.d_titems[mode - 1]) cudaFree(b.d_titems[mode - 1]);
        b.d_titems[mode - 1] = nullptr;
        e = cudaMalloc(reinterpret_cast<void**>(&b.d_titems[mode - 1]), items.size() * sizeof(int4));
        if (e == cudaSuccess)
            e = cudaMemcpy(b.d_titems[mode - 1], items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
        b.ntitems[mode - 1] = int(items.size());
        b.grid[mode - 1] = std::min(int(items.size()), device_sms());
    }
    // the compensated stencil marches down 16 rows of 32 x1 nodes per warp
    std::vector<int4> units;
    for (int i : order)
        for (int x0 = 0; x0 < b.n1[i]; x0 += 32)
            for (int r0 = 0; r0 < b.n2[i]; r0 += 16) units.push_back(make_int4(i, x0, r0, std::min(16, b.n2[i] - r0)));
    if (e == cudaSuccess) {
        if (b.d_sunits) cudaFree(b.d_sunits);
        b.d_sunits = nullptr;
        e = cudaMalloc(reinterpret_cast<void**>(&b.d_sunits), units.size() * sizeof(int4));
        if (e == cudaSuccess) e = cudaMemcpy(b.d_sunits, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice);
        b.nsunits = int(units.size());
    }
    b.sgrid = 8 * device_sms();
    return e;
}

adr_status create_batch(const adr_params* p, void* cuda_stream, adr_ctx** out) {
    if (p->dim != 2) return fail(nullptr, ADR_ERR_ARG, "a batched context is 2-D: dim must be 2");
    if (p->bc_hi != ADR_BC_DIRICHLET || p->form != ADR_FORM_FLUX)
        return fail(nullptr, ADR_ERR_UNSUPPORTED, "batched contexts are Dirichlet, flux form");
    if (!p->n_batch) return fail(nullptr, ADR_ERR_ARG, "n_batch is NULL");
    if (p->batch > (1 << 20)) return fail(nullptr, ADR_ERR_ARG, "batch must be <= 2^20");
    if (!(p->tau > 0.0) || !std::isfinite(p->tau)) return fail(nullptr, ADR_ERR_ARG, "tau must be positive");
    if (p->scheme < ADR_LAWSON_EULER || p->scheme > ADR_STABILIZED_LAWSON2) return fail(nullptr, ADR_ERR_ARG, "unknown scheme");
    if (p->precision == ADR_MIXED_TF32X3)
        return fail(nullptr, ADR_ERR_UNSUPPORTED, "ADR_MIXED_TF32X3 is not built; batched contexts run in ADR_FP64, "
                    "ADR_FP32 or ADR_MIXED_BF16X3");
    if (p->precision != ADR_FP64 && p->precision != ADR_FP32 && p->precision != ADR_MIXED_BF16X3)
        return fail(nullptr, ADR_ERR_ARG, "unknown precision");
    const bool mixed = p->precision == ADR_MIXED_BF16X3;
    int force = -1;
    if (p->batch_tile == 32) force = adr::BT_32;
    else if (p->batch_tile == 64) force = adr::BT_64;
    else if (p->batch_tile == 128) force = adr::BT_128;
    else if (p->batch_tile != 0) return fail(nullptr, ADR_ERR_ARG, "batch_tile must be 0, 32, 64 or 128");

    auto bs = std::make_unique<adr_batch_state>();
    adr_batch_state& b = *bs;
    b.B = p->batch;
    b.tile_force = force;
    b.mixed = mixed;
    switch (p->scheme) {
    case ADR_LAWSON_EULER:
    case ADR_STABILIZED_LAWSON_EULER:
    case ADR_LAWSON2B: b.roles[adr::BR_EXP_ONE] = true; break;
    case ADR_LAWSON4: b.roles[adr::BR_EXP_HALF] = true; break;
    case ADR_LAWSON2A: b.roles[adr::BR_EXP_HALF] = b.roles[adr::BR_EXP_ONE] = true; break;
    case ADR_STABILIZED_LAWSON2:
        b.roles[adr::BR_EXP_HALF] = b.roles[adr::BR_EXP_ONE] = b.roles[adr::BR_EXP_ALPHA] = true;
        break;
    default: b.roles[adr::BR_V] = b.roles[adr::BR_VINV] = true; break;   // the phi_k schemes
    }
    b.n1.resize(b.B); b.n2.resize(b.B); b.apitch.resize(b.B);
    b.off.resize(b.B); b.row0.resize(b.B); b.a_off.resize(b.B);
    b.f_off.assign(size_t(b.B) * 2 * adr::kBatchRoles, -1);
    b.zt_off.assign(size_t(b.B) * 2, -1);
    long long N = 0, img_len = 0, fsc_len = 0;
    for (int i = 0; i < b.B; ++i) {
        const int n1 = p->n_batch[2 * i], n2 = p->n_batch[2 * i + 1];
        if (n1 < 2 || n1 > 4096 || n2 < 2 || n2 > 4096)
            return fail(nullptr, ADR_ERR_ARG, "instance sizes must be in [2, 4096]");
        if (mixed && (n1 > 256 || n2 > 256))
            return fail(nullptr, ADR_ERR_ARG, "mixed batched instances must have n1, n2 <= 256 (exact accumulators)");
        b.n1[i] = n1; b.n2[i] = n2;
        b.off[i] = N; N += (long long)n1 * n2;
        b.row0[i] = b.rows; b.rows += n2;
        b.apitch[i] = ((n1 + 5) + 3) / 4 * 4;
        b.a_off[i] = b.a_len; b.a_len += (long long)b.apitch[i] * (n2 + 2);
        for (int r = 0; r < adr::kBatchRoles; ++r)
            for (int m = 0; m < 2; ++m) {
                if (!b.roles[r]) continue;
                const long long nm = m == 0 ? n1 : n2;
                b.f_off[size_t(i) * 2 * adr::kBatchRoles + r * 2 + m] = b.f_len;
                b.f_len += nm * nm;
            }
        if (b.roles[adr::BR_V])
            for (int m = 0; m < 2; ++m) {
                b.zt_off[size_t(i) * 2 + m] = b.zt_len;
                b.zt_len += ((m == 0 ? n1 : n2) + 3) / 4 * 4;
            }
        if (mixed) {
            adr::BatchTcInst t;
            t.n1 = n1;
            t.n2 = n2;
            t.off = b.off[i];
            t.vec = (n1 % 4 == 0 && b.off[i] % 4 == 0) ? 1 : 0;
            for (int r = 0; r < adr::kBatchRoles; ++r)
                for (int m = 0; m < 2; ++m) {
                    if (!b.roles[r]) continue;
                    const int nm = m == 0 ? n1 : n2;
                    t.img_off[r][m] = img_len;
                    img_len += (long long)adr::batch_tc_image_bytes(nm, m + 1);
                    t.fsc_off[r][m] = fsc_len;
                    fsc_len += (nm + 3) / 4 * 4;
                }
            b.tci.push_back(t);
        }
    }
    if (N > (1LL << 31) - 1) return fail(nullptr, ADR_ERR_ARG, "batch too large (more than 2^31 - 1 nodes)");
    b.hA.assign(size_t(b.a_len), 0.0);
    b.hF.assign(size_t(b.f_len), 0.0);
    b.hZt.assign(size_t(b.zt_len), 0.0);
    b.coef.assign(size_t(b.B) * kCoef, 0.0);
    b.kappa.assign(size_t(b.B) * 2, 0.0);
    b.set.assign(b.B, 0);
    b.tile[0].assign(b.B, 0);
    b.tile[1].assign(b.B, 0);

    std::unique_ptr<adr_ctx> c(new adr_ctx);
    c->p = *p;
    c->p.n_batch = nullptr;                // the sizes are copied above
    if (c->p.lambda <= 0.0) c->p.lambda = 1.0;
    if (c->p.kappa_tol <= 0.0) c->p.kappa_tol = 1e-2;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->dim = 2;
    c->n[0] = b.n1[0]; c->n[1] = b.n2[0]; c->n[2] = 1;
    c->N = size_t(N);
    c->nodes = 0;
    c->fp64 = (p->precision == ADR_FP64);
    c->esize = c->fp64 ? 8 : 4;
    c->tc = false;
    const size_t inst_bytes = c->fp64 ? sizeof(adr::BatchInst<double>) : sizeof(adr::BatchInst<float>);
    std::vector<long long> row_start(size_t(b.B) + 1);
    for (int i = 0; i < b.B; ++i) row_start[i] = b.row0[i];
    row_start[b.B] = b.rows;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&c->d_err), sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaMalloc(&c->ws[i], c->N * c->esize);
    if (e == cudaSuccess) e = cudaMalloc(&b.d_inst, size_t(b.B) * inst_bytes);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b.d_row_start), row_start.size() * sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemcpy(b.d_row_start, row_start.data(), row_start.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b.d_a, size_t(b.a_len) * c->esize);
    if (e == cudaSuccess) e = cudaMalloc(&b.d_f, size_t(b.f_len) * c->esize);
    if (e == cudaSuccess && b.zt_len > 0) e = cudaMalloc(&b.d_zt, size_t(b.zt_len) * c->esize);
    if (mixed && e == cudaSuccess) {
        // tensor-core images, row scales, double-float phi tables, low parts, per-instance slots
        e = cudaMalloc(reinterpret_cast<void**>(&b.d_img), size_t(img_len));
        if (e == cudaSuccess) e = cudaMemset(b.d_img, 0, size_t(img_len));
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b.d_fsc), size_t(fsc_len) * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(b.d_fsc, 0, size_t(fsc_len) * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&b.d_tci, size_t(b.B) * sizeof(adr::BatchTcInst));
        for (int k = 0; k < 3 && e == cudaSuccess && b.roles[adr::BR_V]; ++k)
            e = cudaMalloc(reinterpret_cast<void**>(&b.d_phi[k]), c->N * sizeof(float2));
        for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
            e = cudaMalloc(reinterpret_cast<void**>(&b.d_lo[k]), c->N * sizeof(float));
            if (e == cudaSuccess) e = cudaMemset(b.d_lo[k], 0, c->N * sizeof(float));
        }
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b.d_ulo), c->N * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(b.d_ulo, 0, c->N * sizeof(float));
        // NaN (all bits set) compares unequal to any state, so the first step starts with a zero low part
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b.d_uhs), c->N * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(b.d_uhs, 0xFF, c->N * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMalloc(reinterpret_cast<void**>(&b.d_bslots), size_t(kBatchSlots) * b.B * sizeof(unsigned));
    }
    c->bs = std::move(bs);
    if (e != cudaSuccess) {
        const std::string msg = std::string("batched context: ") + cudaGetErrorString(e);
        adr_destroy(c.release());
        return fail(nullptr, ADR_ERR_ALLOC, msg);
    }
    *out = c.release();
    return ADR_OK;
}

adr_status batch_set_coeffs(adr_ctx* c, int i, const double* a_nodes, const double bvec[3], const double r_poly[4]) {
    adr_batch_state& b = *c->bs;
    if (i < 0 || i >= b.B) return fail(c, ADR_ERR_ARG, "instance out of range");
    if (!a_nodes || !bvec || !r_poly) return fail(c, ADR_ERR_ARG, "NULL coefficient pointer");
    const int n[3] = {b.n1[i], b.n2[i], 1};
    const size_t nodes = size_t(n[0] + 2) * (n[1] + 2);
    for (size_t k = 0; k < nodes; ++k)
        if (!std::isfinite(a_nodes[k])) return fail(c, ADR_ERR_ARG, "a_nodes has a non-finite value");
    drop_graph(c);
    c->coeffs_set = false;
    // Eq. (amaxbeta), per instance
    const double abar = c->p.abar_override > 0 ? c->p.abar_override : c->p.lambda * adr::nodal_max(a_nodes, nodes);
    if (!(abar > 0)) return fail(c, ADR_ERR_ARG, "lambda * a_max must be positive");
    double beta[2];
    for (int m = 0; m < 2; ++m) beta[m] = bvec[m] + adr::mean_face_jump(a_nodes, 2, n, m + 1);
    for (int j2 = 0; j2 < n[1] + 2; ++j2)
        for (int j1 = 0; j1 < n[0] + 2; ++j1)
            b.hA[size_t(b.a_off[i] + (long long)j2 * b.apitch[i] + j1 + 3)] = a_nodes[size_t(j2) * (n[0] + 2) + j1] - abar;
    double* k = &b.coef[size_t(i) * kCoef];
    for (int m = 0; m < 2; ++m) {
        const double h = 1.0 / (n[m] + 1);
        k[m] = 1.0 / (h * h);
        k[2 + m] = 1.0 / (2.0 * h);
        k[4 + m] = bvec[m] - beta[m];
        k[6 + m] = beta[m];
    }
    k[8] = abar;
    for (int j = 0; j < 4; ++j) k[9 + j] = r_poly[j];
    // factors of the scheme, on the host in FP64
    for (int m = 0; m < 2; ++m) {
        const adr::Factor1D f = adr::make_factor(n[m], abar, beta[m]);
        const long long nm = n[m];
        for (int ci = 0; ci < 3; ++ci) {
            const int role = ci == 0 ? adr::BR_EXP_HALF : ci == 1 ? adr::BR_EXP_ONE : adr::BR_EXP_ALPHA;
            if (!b.roles[role]) continue;
            std::vector<double> sA = adr::factor_dense(f);
            for (auto& v : sA) v *= (ci == 0 ? 0.5 : ci == 1 ? 1.0 : adr::kLawsonAlpha) * c->p.tau;
            std::vector<double> E;
            try {
                E = adr::expm_pade13(sA, n[m]);
            } catch (const std::exception& ex) {
                return fail(c, ADR_ERR_ARG, std::string("expm: ") + ex.what());
            }
            std::copy(E.begin(), E.end(), b.hF.begin() + b.f_off[size_t(i) * 2 * adr::kBatchRoles + role * 2 + m]);
        }
        if (b.roles[adr::BR_V]) {
            const adr::Eigen1D eg = adr::eigen_closed_form(f);
            if (!eg.real) {
                char buf[128];
                std::snprintf(buf, sizeof buf, "instance %d: cell Peclet number >= 1: A_mu has no real eigenbasis", i);
                return fail(c, ADR_ERR_COMPLEX_SPECTRUM, buf);
            }
            b.kappa[size_t(i) * 2 + m] = eg.kappa;
            std::copy(eg.V.begin(), eg.V.end(), b.hF.begin() + b.f_off[size_t(i) * 2 * adr::kBatchRoles + adr::BR_V * 2 + m]);
            std::copy(eg.Vinv.begin(), eg.Vinv.end(), b.hF.begin() + b.f_off[size_t(i) * 2 * adr::kBatchRoles + adr::BR_VINV * 2 + m]);
            for (long long j = 0; j < nm; ++j) b.hZt[size_t(b.zt_off[size_t(i) * 2 + m] + j)] = c->p.tau * eg.lam[size_t(j)];
        }
    }
    if (b.mixed) {
        const cudaError_t me = batch_mixed_instance(c, i);
        if (me != cudaSuccess) return cuda_fail(c, me, "upload mixed batch instance");
    }
    if (b.roles[adr::BR_V]) {
        const double kp = b.kappa[size_t(i) * 2] * b.kappa[size_t(i) * 2 + 1];
        // the unit of the working precision: FP64, FP32, or the 40-bit state slices of the mixed path
        const double unit = c->fp64 ? std::ldexp(1.0, -53) : b.mixed ? std::ldexp(1.0, -40) : std::ldexp(1.0, -24);
        if (kp * unit > c->p.kappa_tol) {
            char buf[192];
            std::snprintf(buf, sizeof buf, "instance %d: eigen route ill-conditioned: prod kappa * u = %.3e > kappa_tol %.3e",
                          i, kp * unit, c->p.kappa_tol);
            return fail(c, ADR_ERR_ILL_CONDITIONED, buf);
        }
    }
    if (!b.set[i]) { b.set[i] = 1; ++b.nset; }
    if (b.nset < b.B) return ADR_OK;
    cudaError_t e = batch_upload(c, i);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload batch");
    if (b.mixed) {
        if (!b.tuned) {
            e = batch_mixed_plan(c);
            if (e != cudaSuccess) return cuda_fail(c, e, "mixed batch plan");
            b.tuned = true;
        }
        c->coeffs_set = true;
        return ADR_OK;
    }
    if (!b.tuned) {
        const adr_status st = c->fp64 ? batch_tune<double>(c) : batch_tune<float>(c);
        if (st != ADR_OK) return st;
    }
    c->coeffs_set = true;
    return ADR_OK;
}

}  // namespace

namespace {

// C = E E for a row-major n x n matrix.
std::vector<double> square_matrix(const std::vector<double>& E, int n) {
    std::vector<double> C(size_t(n) * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const double e = E[size_t(i) * n + k];
            if (e == 0.0) continue;
            const double* row = &E[size_t(k) * n];
            double* out = &C[size_t(i) * n];
            for (int j = 0; j < n; ++j) out[j] += e * row[j];
        }
    return C;
}

// The phi doubling route (see adr_phi_route in adr.h): s halvings so that
// tau ||A||_1 / 2^s <= 1/2 (||A||_1 <= sum_mu ||A_mu||_1 for the Kronecker sum), p = 13 Taylor
// terms (the remainder 0.5^14 / 15! is below 5e-17), the level factors e^{2^i X_mu} with
// X_mu = tau A_mu / 2^s (Pade-13 for i = 0, then repeated squaring), a zero coefficient array
// for the constant-coefficient stencil, and three state-sized work arrays.
adr_status setup_doubling(adr_ctx* c) {
    double norm = 0.0;   // sum over mu of the largest absolute row sum of A_mu (Neumann rows included)
    for (int m = 0; m < c->dim; ++m) {
        const std::vector<double> A = adr::factor_dense(c->f[m]);
        double rmax = 0.0;
        for (int i = 0; i < c->n[m]; ++i) {
            double r = 0.0;
            for (int j = 0; j < c->n[m]; ++j) r += std::fabs(A[size_t(i) * c->n[m] + j]);
            rmax = std::max(rmax, r);
        }
        norm += rmax;
    }
    const double x = c->p.tau * norm;
    int sh = 0;
    while (x > std::ldexp(0.5, sh)) ++sh;
    if (sh > kMaxLevels) return fail(c, ADR_ERR_ARG, "tau ||A|| too large for the phi doubling route");
    c->dbl_s = sh;
    c->dbl_p = 13;
    const double c0 = std::ldexp(c->p.tau, -sh);
    struct Cached { int n; double beta; std::vector<std::vector<double>> E; };
    std::vector<Cached> cache;
    cudaError_t e = cudaSuccess;
    for (int m = 0; m < c->dim && e == cudaSuccess; ++m) {
        const std::vector<std::vector<double>>* levels = nullptr;
        for (const auto& hit : cache)
            if (hit.n == c->n[m] && hit.beta == c->beta[m]) levels = &hit.E;
        if (!levels) {
            Cached cc{c->n[m], c->beta[m], {}};
            std::vector<double> A = adr::factor_dense(c->f[m]);
            for (auto& v : A) v *= c0;
            try {
                cc.E.push_back(adr::expm_pade13(A, c->n[m]));
            } catch (const std::exception& ex) {
                return fail(c, ADR_ERR_ARG, std::string("expm: ") + ex.what());
            }
            for (int i = 1; i < sh; ++i) cc.E.push_back(square_matrix(cc.E.back(), c->n[m]));
            cache.push_back(std::move(cc));
            levels = &cache.back().E;
        }
        for (int i = 0; i < sh && e == cudaSuccess; ++i) {
            e = upload(c, &c->d_El[i][m], (*levels)[size_t(i)]);
            if (e == cudaSuccess && c->tc) e = upload_tc(c, kLevel0 + i, m, (*levels)[size_t(i)]);
        }
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "upload doubling factors");
    const size_t abytes = size_t(c->apitch) * (c->n[1] + 2) * (c->dim == 3 ? c->n[2] + 2 : 1) * c->esize;
    if (!c->d_a0) {
        e = cudaMalloc(&c->d_a0, abytes);
        if (e == cudaSuccess) e = cudaMemset(c->d_a0, 0, abytes);
    }
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        if (!c->wsd[i]) e = cudaMalloc(&c->wsd[i], c->N * c->esize);
    if (e != cudaSuccess) return fail(c, ADR_ERR_ALLOC, std::string("doubling route: ") + cudaGetErrorString(e));
    return ADR_OK;
}

// ------------------------------------------------------------ periodic Fourier contexts
bool power_of_two(int n) { return n >= 2 && (n & (n - 1)) == 0; }

// phi_k(z), k = 0, 1, 2, of a complex argument from the definitions e^z, (e^z - 1) / z,
// (e^z - 1 - z) / z^2; for |z| < 1 the power series sum_j z^j / (j + k)! (30 terms, Horner),
// which avoids the cancellation of the closed forms near 0.
std::complex<double> phi_complex(int k, std::complex<double> z) {
    if (k == 0) return std::exp(z);
    if (std::abs(z) < 1.0) {
        std::complex<double> acc = 0.0;
        for (int j = 29; j >= 0; --j) acc = acc * z + inv_factorial(j + k);
        return acc;
    }
    // e^z - 1 = expm1(x) e^{iy} + (e^{iy} - 1), with cos y - 1 = -2 sin^2(y/2)
    const double x = z.real(), y = z.imag(), sh = std::sin(0.5 * y);
    const std::complex<double> em1 =
        std::expm1(x) * std::complex<double>(std::cos(y), std::sin(y)) + std::complex<double>(-2.0 * sh * sh, std::sin(y));
    return k == 1 ? em1 / z : (em1 - z) / (z * z);
}

// Wavenumbers of n Fourier modes on a period of length L in FFT order (j, then j - n for
// j > n/2), the Nyquist mode j = n/2 set to 0: the first derivative of the interpolant of
// real data has no real Nyquist component.
std::vector<double> wavenumbers(int n, double L) {
    std::vector<double> k(static_cast<size_t>(n));
    for (int j = 0; j < n; ++j) k[size_t(j)] = (2.0 * M_PI / L) * (j < n / 2 ? j : j == n / 2 ? 0 : j - n);
    return k;
}

adr_status create_periodic(const adr_params* p, void* cuda_stream, adr_ctx** out) {
    if (p->periodic != 1) return fail(nullptr, ADR_ERR_ARG, "periodic must be 0 or 1");
    if (p->batch != 0) return fail(nullptr, ADR_ERR_UNSUPPORTED, "periodic contexts are single grids");
    if (p->dim != 2 && p->dim != 3) return fail(nullptr, ADR_ERR_ARG, "dim must be 2 or 3");
    for (int m = 0; m < p->dim; ++m)
        if (!power_of_two(p->n[m]) || p->n[m] > (m == 0 ? 4096 : 1024) ||
            !adr::periodic_line_fits(p->n[m], m, p->dim, p->precision == ADR_FP64))
            return fail(nullptr, ADR_ERR_ARG,
                        "periodic contexts need n a power of two in [2, 4096] along x1 and [2, 1024] along the other axes");
    if (!(p->tau > 0.0) || !std::isfinite(p->tau)) return fail(nullptr, ADR_ERR_ARG, "tau must be positive");
    if (!(p->length > 0.0) || !std::isfinite(p->length)) return fail(nullptr, ADR_ERR_ARG, "length must be positive");
    if (p->scheme < ADR_LAWSON_EULER || p->scheme > ADR_STABILIZED_LAWSON2) return fail(nullptr, ADR_ERR_ARG, "unknown scheme");
    if (p->precision != ADR_FP64 && p->precision != ADR_FP32)
        return fail(nullptr, ADR_ERR_UNSUPPORTED, "periodic contexts run in ADR_FP64 or ADR_FP32");
    if (p->phi_route != ADR_PHI_AUTO && p->phi_route != ADR_PHI_FOURIER)
        return fail(nullptr, ADR_ERR_ARG, "periodic contexts apply phi_k as Fourier multipliers");
    if (p->bc_hi != ADR_BC_DIRICHLET) return fail(nullptr, ADR_ERR_ARG, "bc_hi does not apply to periodic contexts");
    if (p->form != ADR_FORM_FLUX && p->form != ADR_FORM_ADELTA) return fail(nullptr, ADR_ERR_ARG, "unknown form");
    size_t N = 1;
    for (int m = 0; m < p->dim; ++m) N *= size_t(p->n[m]);
    if (N > (size_t(1) << 31) - 1) return fail(nullptr, ADR_ERR_ARG, "grid too large");

    std::unique_ptr<adr_ctx> c(new adr_ctx);
    c->p = *p;
    if (c->p.lambda <= 0.0) c->p.lambda = 1.0;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->periodic = true;
    c->dim = p->dim;
    for (int m = 0; m < 3; ++m) c->n[m] = (m < p->dim) ? p->n[m] : 1;
    c->N = N;
    c->nodes = N;
    c->fp64 = (p->precision == ADR_FP64);
    c->esize = c->fp64 ? 8 : 4;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&c->d_err), sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaMalloc(&c->ws[i], N * c->esize);
    for (int i = 0; i <= c->dim && e == cudaSuccess; ++i) e = cudaMalloc(&c->d_pc[i], 2 * N * c->esize);
    if (e == cudaSuccess && p->form == ADR_FORM_ADELTA) e = cudaMalloc(&c->d_pdif, N * c->esize);
    if (e == cudaSuccess && p->dim == 2) e = cudaMalloc(&c->d_pcn, 2 * N * c->esize);
    if (e == cudaSuccess && p->dim == 2) e = cudaMalloc(&c->d_pz, 2 * N * c->esize);
    if (e == cudaSuccess) e = adr::periodic_prepare(c->fp64);
    if (e != cudaSuccess) {
        adr_destroy(c.release());
        return fail(nullptr, ADR_ERR_ALLOC, std::string("periodic context: ") + cudaGetErrorString(e));
    }
    for (int m = 0; m < c->dim && e == cudaSuccess; ++m) {
        const int n = c->n[m];
        std::vector<double> tw(static_cast<size_t>(n));   // e^{-2 pi i j / n}, j < n/2, interleaved (re, im)
        for (int j = 0; j < n / 2; ++j) {
            tw[2 * size_t(j)] = std::cos(2.0 * M_PI * j / n);
            tw[2 * size_t(j) + 1] = -std::sin(2.0 * M_PI * j / n);
        }
        e = upload(c.get(), &c->d_ptw[m], tw);
        if (e == cudaSuccess) e = upload(c.get(), &c->d_pk[m], wavenumbers(n, p->length));
    }
    if (e != cudaSuccess) {
        adr_destroy(c.release());
        return fail(nullptr, ADR_ERR_ALLOC, std::string("periodic tables: ") + cudaGetErrorString(e));
    }
    *out = c.release();
    return ADR_OK;
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

adr_status adr_create(const adr_params* p, void* cuda_stream, adr_ctx** out) {
    if (!out) return fail(nullptr, ADR_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, ADR_ERR_ARG, "params is NULL");
    if (p->batch < 0) return fail(nullptr, ADR_ERR_ARG, "batch must be >= 0");
    if (p->periodic) return create_periodic(p, cuda_stream, out);
    if (p->batch > 0) return create_batch(p, cuda_stream, out);
    if (p->dim != 2 && p->dim != 3) return fail(nullptr, ADR_ERR_ARG, "dim must be 2 or 3");
    for (int m = 0; m < p->dim; ++m)
        if (p->n[m] < 2 || p->n[m] > 4096) return fail(nullptr, ADR_ERR_ARG, "n must be in [2, 4096]");
    if (!(p->tau > 0.0) || !std::isfinite(p->tau)) return fail(nullptr, ADR_ERR_ARG, "tau must be positive");
    if (p->scheme < ADR_LAWSON_EULER || p->scheme > ADR_STABILIZED_LAWSON2) return fail(nullptr, ADR_ERR_ARG, "unknown scheme");
    if (p->precision == ADR_MIXED_TF32X3)
        return fail(nullptr, ADR_ERR_UNSUPPORTED, "ADR_MIXED_TF32X3 is not implemented");
    if (p->phi_route < ADR_PHI_AUTO || p->phi_route > ADR_PHI_DOUBLING) return fail(nullptr, ADR_ERR_ARG, "unknown phi route");
    if (p->bc_hi != ADR_BC_DIRICHLET && p->bc_hi != ADR_BC_NEUMANN) return fail(nullptr, ADR_ERR_ARG, "unknown bc_hi");
    if (p->form != ADR_FORM_FLUX && p->form != ADR_FORM_ADELTA) return fail(nullptr, ADR_ERR_ARG, "unknown form");
    if (p->bc_hi == ADR_BC_NEUMANN && p->form != ADR_FORM_ADELTA)
        return fail(nullptr, ADR_ERR_UNSUPPORTED, "Neumann faces are implemented for the a Lap u form");
    if (p->precision != ADR_FP64 && p->precision != ADR_FP32 && p->precision != ADR_MIXED_BF16X3)
        return fail(nullptr, ADR_ERR_ARG, "unknown precision");
    if (p->precision == ADR_MIXED_BF16X3)
        for (int m = 0; m < p->dim; ++m)
            if (p->n[m] > 512)
                return fail(nullptr, ADR_ERR_ARG, "ADR_MIXED_BF16X3 supports n <= 512 per direction");
    size_t N = 1, nodes = 1;
    for (int m = 0; m < p->dim; ++m) { N *= size_t(p->n[m]); nodes *= size_t(p->n[m] + 2); }
    if (N > (size_t(1) << 31) - 1) return fail(nullptr, ADR_ERR_ARG, "grid too large");

    std::unique_ptr<adr_ctx> c(new adr_ctx);
    c->p = *p;
    if (c->p.lambda <= 0.0) c->p.lambda = 1.0;
    if (c->p.kappa_tol <= 0.0) c->p.kappa_tol = 1e-2;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->dim = p->dim;
    for (int m = 0; m < 3; ++m) c->n[m] = (m < p->dim) ? p->n[m] : 1;
    c->N = N;
    c->nodes = nodes;
    c->fp64 = (p->precision == ADR_FP64);
    c->esize = c->fp64 ? 8 : 4;
    c->tc = (p->precision == ADR_MIXED_BF16X3);
    {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&c->d_err), sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
        if (e == cudaSuccess && c->tc) e = cudaMalloc(reinterpret_cast<void**>(&c->d_slots), kSlots * sizeof(unsigned));
        if (e != cudaSuccess) {
            adr_destroy(c.release());
            return fail(nullptr, ADR_ERR_ALLOC, std::string("context: ") + cudaGetErrorString(e));
        }
    }
    for (int i = 0; i < 9; ++i) {
        if (i >= 6 && !c->tc) continue;   // low parts exist on the mixed path only
        cudaError_t e = cudaMalloc(&c->ws[i], N * c->esize);
        if (e != cudaSuccess) {
            adr_destroy(c.release());
            return fail(nullptr, ADR_ERR_ALLOC, std::string("workspace: ") + cudaGetErrorString(e));
        }
    }
    *out = c.release();
    return ADR_OK;
}

adr_status adr_set_coeffs(adr_ctx* c, int instance, const double* a_nodes, const double b[3], const double r_poly[4]) {
    if (!c) return ADR_ERR_ARG;
    if (c->bs) return batch_set_coeffs(c, instance, a_nodes, b, r_poly);
    if (c->periodic) return fail(c, ADR_ERR_ARG, "periodic contexts take adr_set_coeffs_periodic");
    if (instance != 0) return fail(c, ADR_ERR_ARG, "instance must be 0 for a single-grid context");
    if (!a_nodes || !b || !r_poly) return fail(c, ADR_ERR_ARG, "NULL coefficient pointer");
    for (size_t i = 0; i < c->nodes; ++i)
        if (!std::isfinite(a_nodes[i])) return fail(c, ADR_ERR_ARG, "a_nodes has a non-finite value");
    drop_graph(c);
    c->coeffs_set = false;
    for (int m = 0; m < 3; ++m) c->b[m] = (m < c->dim) ? b[m] : 0.0;
    for (int i = 0; i < 4; ++i) c->r[i] = r_poly[i];
    // Eq. (amaxbeta)
    const bool neumann = c->p.bc_hi == ADR_BC_NEUMANN;
    double amax = adr::nodal_max(a_nodes, c->nodes);
    if (neumann) {   // the ring beyond x_mu = 1 lies outside the domain: max over j_mu <= n_mu
        amax = -INFINITY;
        const int N1 = c->n[0] + 2, N2 = c->n[1] + 2;
        const int J3 = c->dim == 3 ? c->n[2] + 1 : 1;
        for (int j3 = 0; j3 < J3; ++j3)
            for (int j2 = 0; j2 <= c->n[1]; ++j2)
                for (int j1 = 0; j1 <= c->n[0]; ++j1)
                    amax = std::max(amax, a_nodes[(size_t(j3) * N2 + j2) * N1 + j1]);
    }
    c->abar = c->p.abar_override > 0 ? c->p.abar_override : c->p.lambda * amax;
    if (!(c->abar > 0)) return fail(c, ADR_ERR_ARG, "lambda * a_max must be positive");
    for (int m = 0; m < c->dim; ++m)   // Eq. (amaxbeta); the a Lap u form of Eq. (adr3dstab) has beta = b
        c->beta[m] = c->b[m] + (c->p.form == ADR_FORM_ADELTA ? 0.0 : adr::mean_face_jump(a_nodes, c->dim, c->n, m + 1));

    // device copy of (a - abar) with padded rows: interior x1 nodes start 16-byte aligned
    const int N1 = c->n[0] + 2, N2 = c->n[1] + 2, N3 = c->dim == 3 ? c->n[2] + 2 : 1;
    c->apitch = ((c->n[0] + 5) + 3) / 4 * 4;
    std::vector<double> amb(size_t(c->apitch) * N2 * N3, 0.0);
    for (int j3 = 0; j3 < N3; ++j3)
        for (int j2 = 0; j2 < N2; ++j2)
            for (int j1 = 0; j1 < N1; ++j1)
                amb[(size_t(j3) * N2 + j2) * c->apitch + j1 + 3] =
                    a_nodes[(size_t(j3) * N2 + j2) * N1 + j1] - c->abar;
    if (c->d_a) { void* q = c->d_a; free_dev(q); c->d_a = nullptr; }
    cudaError_t e = upload(c, &c->d_a, amb);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload a");

    c->eig_real = true;
    struct CachedE { int n; double beta, c; std::vector<double> E; };
    std::vector<CachedE> cache;
    cache.reserve(9);
    for (int m = 0; m < c->dim; ++m) {
        c->f[m] = adr::make_factor(c->n[m], c->abar, c->beta[m], neumann);
        const auto A = adr::factor_dense(c->f[m]);
        for (int ci = 0; ci < 3; ++ci) {
            if (ci == 2 && c->p.scheme != ADR_STABILIZED_LAWSON2) continue;   // e^{alpha tau A_mu}
            const double cc = ci == 0 ? 0.5 : ci == 1 ? 1.0 : adr::kLawsonAlpha;
            // directions with the same (n, beta) share one host computation of e^{c tau A_mu}
            const std::vector<double>* E = nullptr;
            for (const auto& hit : cache)
                if (hit.n == c->n[m] && hit.beta == c->beta[m] && hit.c == cc) E = &hit.E;
            if (!E) {
                std::vector<double> sA(A);
                for (auto& v : sA) v *= cc * c->p.tau;
                try {
                    cache.push_back({c->n[m], c->beta[m], cc, adr::expm_pade13(sA, c->n[m])});
                } catch (const std::exception& ex) {
                    return fail(c, ADR_ERR_ARG, std::string("expm: ") + ex.what());
                }
                E = &cache.back().E;
            }
            e = upload(c, &c->d_E[ci][m], *E);
            if (e != cudaSuccess) return cuda_fail(c, e, "upload E");
            if (c->tc) {
                e = upload_tc(c, ci == 2 ? FK_EXP_ALPHA : ci, m, *E);
                if (e == cudaSuccess && ci == 0) e = upload_tc(c, FK_EXP_HALF_PRECISE, m, *E);
                if (e != cudaSuccess) return cuda_fail(c, e, "upload sliced E");
            }
        }
        const adr::Eigen1D eg = adr::eigen_closed_form(c->f[m]);
        c->kappa[m] = eg.real ? eg.kappa : 0.0;
        if (!eg.real) { c->eig_real = false; continue; }
        e = upload(c, &c->d_V[m], eg.V);
        if (e == cudaSuccess) e = upload(c, &c->d_Vi[m], eg.Vinv);
        if (e == cudaSuccess && !c->d_lam[m]) e = cudaMalloc(reinterpret_cast<void**>(&c->d_lam[m]), c->n[m] * sizeof(double));
        if (e == cudaSuccess) e = cudaMemcpy(c->d_lam[m], eg.lam.data(), c->n[m] * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && c->tc) e = upload_tc(c, FK_V, m, eg.V);
        if (e == cudaSuccess && c->tc) e = upload_tc(c, FK_VINV, m, eg.Vinv);
        if (e == cudaSuccess && c->tc) {
            std::vector<float> zt(c->n[m]);
            for (int j = 0; j < c->n[m]; ++j) zt[j] = static_cast<float>(c->p.tau * eg.lam[j]);
            if (!c->d_zt[m]) e = cudaMalloc(reinterpret_cast<void**>(&c->d_zt[m]), zt.size() * sizeof(float));
            if (e == cudaSuccess) e = cudaMemcpy(c->d_zt[m], zt.data(), zt.size() * sizeof(float), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "upload eigenpairs");
    }
    c->phi_route = 0;
    if (needs_phi(c->p.scheme)) {
        double kp = 1.0;
        for (int m = 0; m < c->dim; ++m) kp *= c->kappa[m];
        const double unit = c->fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
        const bool guard_ok = c->eig_real && kp * unit <= c->p.kappa_tol;
        if (c->p.phi_route == ADR_PHI_EIGEN && !c->eig_real)
            return fail(c, ADR_ERR_COMPLEX_SPECTRUM,
                        "no closed-form real eigenbasis of A_mu (cell Peclet number >= 1, or a Neumann face)");
        if (c->p.phi_route == ADR_PHI_EIGEN && !guard_ok) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "eigen route ill-conditioned: prod kappa * u = %.3e > kappa_tol %.3e",
                          kp * unit, c->p.kappa_tol);
            return fail(c, ADR_ERR_ILL_CONDITIONED, buf);
        }
        if (c->p.phi_route == ADR_PHI_DOUBLING || !guard_ok) {
            const adr_status st = setup_doubling(c);
            if (st != ADR_OK) return st;
            c->phi_route = ADR_PHI_DOUBLING;
        } else {
            c->phi_route = ADR_PHI_EIGEN;
        }
    }
    c->coeffs_set = true;
    return ADR_OK;
}

adr_status adr_set_coeffs_periodic(adr_ctx* c, const double* a_diag, const double* b_field, const double r_poly[4]) {
    if (!c) return ADR_ERR_ARG;
    if (!c->periodic) return fail(c, ADR_ERR_ARG, "adr_set_coeffs_periodic needs a periodic context");
    if (!a_diag || !b_field || !r_poly) return fail(c, ADR_ERR_ARG, "NULL coefficient pointer");
    const size_t N = c->N;
    const int d = c->dim;
    for (size_t i = 0; i < size_t(d) * N; ++i)
        if (!std::isfinite(a_diag[i]) || !std::isfinite(b_field[i]))
            return fail(c, ADR_ERR_ARG, "a_diag or b_field has a non-finite value");
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(r_poly[i])) return fail(c, ADR_ERR_ARG, "r_poly has a non-finite value");
    drop_graph(c);
    c->coeffs_set = false;
    for (int i = 0; i < 4; ++i) c->r[i] = r_poly[i];
    // Eq. (amaxbeta): a^max_mu = lambda max a_mumu, beta_mu = mean of b_mu (the mean of d_mu a_mumu
    // over a period is zero)
    double amax[3] = {0, 0, 0};
    c->abar = 0.0;
    for (int m = 0; m < d; ++m) {
        const double* a = a_diag + size_t(m) * N;
        const double* b = b_field + size_t(m) * N;
        amax[m] = c->p.abar_override > 0 ? c->p.abar_override : c->p.lambda * adr::nodal_max(a, N);
        if (!(amax[m] > 0)) return fail(c, ADR_ERR_ARG, "lambda * a_max must be positive");
        double sum = 0.0;
        for (size_t i = 0; i < N; ++i) sum += b[i];
        c->b[m] = c->beta[m] = sum / double(N);
        c->abar = std::max(c->abar, amax[m]);
        c->kappa[m] = 1.0;   // the Fourier basis is unitary
        cudaError_t e = upload(c, &c->d_pa[m], std::vector<double>(a, a + N));
        if (e == cudaSuccess) e = upload(c, &c->d_pb[m], std::vector<double>(b, b + N));
        if (e != cudaSuccess) return cuda_fail(c, e, "upload a, b");
    }
    // symbol s = sum_mu (-a^max_mu k_mu^2 + i beta_mu k_mu) and the multipliers of tau s
    std::vector<double> k[3];
    for (int m = 0; m < d; ++m) k[m] = wavenumbers(c->n[m], c->p.length);
    std::vector<double> sym(2 * N), mult[5];
    for (auto& v : mult) v.resize(2 * N);
    const double cexp[3] = {0.5, 1.0, adr::kLawsonAlpha};
    for (size_t i = 0; i < N; ++i) {
        size_t r = i;
        std::complex<double> sv = 0.0;
        for (int m = 0; m < d; ++m) {
            const double km = k[m][r % size_t(c->n[m])];
            r /= size_t(c->n[m]);
            sv += std::complex<double>(-amax[m] * km * km, c->beta[m] * km);
        }
        sym[2 * i] = sv.real();
        sym[2 * i + 1] = sv.imag();
        const std::complex<double> z = c->p.tau * sv;
        std::complex<double> v[5];
        for (int q = 0; q < 3; ++q) v[q] = std::exp(cexp[q] * z);
        v[3] = phi_complex(1, z);
        v[4] = phi_complex(2, z);
        for (int q = 0; q < 5; ++q) {
            mult[q][2 * i] = v[q].real();
            mult[q][2 * i + 1] = v[q].imag();
        }
    }
    cudaError_t e = upload(c, &c->d_psym, sym);
    for (int q = 0; q < 5 && e == cudaSuccess; ++q) e = upload(c, &c->d_pm[q], mult[q]);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload Fourier multipliers");
    c->phi_route = needs_phi(c->p.scheme) ? ADR_PHI_FOURIER : 0;
    c->coeffs_set = true;
    return ADR_OK;
}

adr_status adr_step(adr_ctx* c, void* u, double t) {
    (void)t;
    adr_status st = check_ready(c);
    if (st != ADR_OK) return st;
    if (!u) return fail(c, ADR_ERR_ARG, "u is NULL");
    return run_ops(c, step_ops(c, u), "adr_step");
}

adr_status adr_integrate(adr_ctx* c, void* u, double t0, double T, int m) {
    adr_status st = check_ready(c);
    if (st != ADR_OK) return st;
    if (!u) return fail(c, ADR_ERR_ARG, "u is NULL");
    if (m < 0) return fail(c, ADR_ERR_ARG, "m must be >= 0");
    if (T > 0 && std::fabs(t0 + m * c->p.tau - T) > 1e-9 * std::max(1.0, std::fabs(T)))
        return fail(c, ADR_ERR_ARG, "T != t0 + m * tau");
    if (m == 0) return ADR_OK;
    if (c->stream == nullptr) {   // the legacy stream cannot be captured: replay directly
        const auto ops = step_ops(c, u);
        for (int i = 0; i < m; ++i) {
            st = run_ops(c, ops, "adr_integrate");
            if (st != ADR_OK) return st;
        }
        return ADR_OK;
    }
    if (c->graph_u != u) {
        // two graphs of the same step: one step, and kGraphSteps steps back to back (one replay
        // then covers several steps, which matters where a step is a few microseconds)
        drop_graph(c);
        const auto ops = step_ops(c, u);
        auto capture = [&](int steps, cudaGraph_t* g, cudaGraphExec_t* x) -> adr_status {
            cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
            cudaError_t le = cudaSuccess;
            for (int k = 0; k < steps && le == cudaSuccess; ++k)
                for (const auto& op : ops) {
                    le = op(c->stream);
                    if (le != cudaSuccess) break;
                }
            e = cudaStreamEndCapture(c->stream, g);
            if (le != cudaSuccess) { drop_graph(c); return cuda_fail(c, le, "capture launch"); }
            if (e != cudaSuccess) { drop_graph(c); return cuda_fail(c, e, "end capture"); }
            e = cudaGraphInstantiate(x, *g, 0);
            if (e != cudaSuccess) { drop_graph(c); return cuda_fail(c, e, "instantiate graph"); }
            return ADR_OK;
        };
        st = capture(1, &c->graph, &c->gexec);
        if (st == ADR_OK) st = capture(kGraphSteps, &c->graph_k, &c->gexec_k);
        if (st != ADR_OK) return st;
        c->graph_u = u;
    }
    nvtxRangePushA("adr_integrate: graph replays");
    for (int left = m; left > 0;) {
        const bool many = left >= kGraphSteps;
        cudaError_t e = cudaGraphLaunch(many ? c->gexec_k : c->gexec, c->stream);
        if (e != cudaSuccess) {
            nvtxRangePop();
            return cuda_fail(c, e, "graph launch");
        }
        left -= many ? kGraphSteps : 1;
    }
    nvtxRangePop();
    return ADR_OK;
}

adr_status adr_integrate_host(adr_ctx* c, void* u_host, double t0, double T, int m) {
    adr_status st = check_ready(c);
    if (st != ADR_OK) return st;
    if (!u_host) return fail(c, ADR_ERR_ARG, "u_host is NULL");
    const size_t bytes = c->N * c->esize;
    cudaError_t e = cudaSuccess;
    if (!c->d_host_state) {
        e = cudaMalloc(&c->d_host_state, bytes);
        if (e != cudaSuccess) return fail(c, ADR_ERR_ALLOC, std::string("state buffer: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(c->d_host_state, u_host, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "H2D");
    st = adr_integrate(c, c->d_host_state, t0, T, m);
    if (st != ADR_OK) return st;
    e = cudaMemcpyAsync(u_host, c->d_host_state, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "D2H");
    return adr_synchronize(c);
}

adr_status adr_eval_rhs(adr_ctx* c, const void* u, void* F_out, void* g_out) {
    adr_status st = check_ready(c);
    if (st != ADR_OK) return st;
    if (!u || (!F_out && !g_out)) return fail(c, ADR_ERR_ARG, "NULL array");
    if (u == F_out || u == g_out) return fail(c, ADR_ERR_ARG, "output aliases input");
    Sched S(c);
    auto fill = [&](auto* uu, auto* F, auto* g) {
        auto s = stencil_base(c, uu);
        if (F) { s.out[s.nout] = F; s.cF[s.nout] = 1.0; ++s.nout; }
        if (g) { s.out[s.nout] = g; s.cg[s.nout] = 1.0; ++s.nout; }
        push_stencil(S, s);
    };
    if (c->fp64) fill(static_cast<const double*>(u), static_cast<double*>(F_out), static_cast<double*>(g_out));
    else         fill(static_cast<const float*>(u), static_cast<float*>(F_out), static_cast<float*>(g_out));
    return run_ops(c, S.ops, "adr_eval_rhs");
}

adr_status adr_apply_exp(adr_ctx* c, double cc, const void* v, void* y) {
    adr_status st = check_ready(c);
    if (st != ADR_OK) return st;
    if (!v || !y || v == y) return fail(c, ADR_ERR_ARG, "NULL or aliased array");
    int ci = -1;
    if (cc == 0.5) ci = 0;
    if (cc == 1.0) ci = 1;
    if (ci < 0) return fail(c, ADR_ERR_ARG, "c must be 0.5 or 1");
    if (c->bs && !c->bs->roles[ci])
        return fail(c, ADR_ERR_STATE, "this batched context's scheme does not build e^{c tau A} for this c");
    Sched S(c);
    if (c->fp64) push_exp<double>(S, ci, static_cast<const double*>(v), static_cast<double*>(y));
    else         push_exp<float>(S, ci, static_cast<const float*>(v), static_cast<float*>(y));
    return run_ops(c, S.ops, "adr_apply_exp");
}

adr_status adr_apply_phi(adr_ctx* c, int k, const void* v, void* y) {
    adr_status st = check_ready(c);
    if (st != ADR_OK) return st;
    if (!v || !y || v == y) return fail(c, ADR_ERR_ARG, "NULL or aliased array");
    if (k < 0 || k > 2) return fail(c, ADR_ERR_ARG, "k must be 0, 1 or 2");
    if (c->bs && !c->bs->roles[FK_V])
        return fail(c, ADR_ERR_STATE, "this batched context's scheme does not build the eigenbasis");
    if (!c->bs && !c->periodic && c->phi_route != ADR_PHI_DOUBLING && !c->eig_real)
        return fail(c, ADR_ERR_COMPLEX_SPECTRUM, "A_mu has no real eigenbasis");
    Sched S(c);
    if (c->fp64) push_phi<double>(S, k, static_cast<const double*>(v), static_cast<double*>(y));
    else         push_phi<float>(S, k, static_cast<const float*>(v), static_cast<float*>(y));
    return run_ops(c, S.ops, "adr_apply_phi");
}

adr_status adr_profile_step(adr_ctx* c, void* u, int max_ops, float* ms, int* kind, int* n_ops) {
    adr_status st = check_ready(c);
    if (st != ADR_OK) return st;
    if (!u || !ms || !kind || !n_ops || max_ops <= 0) return fail(c, ADR_ERR_ARG, "NULL argument");
    const auto ops = step_ops(c, u);
    if (int(ops.size()) > max_ops) return fail(c, ADR_ERR_ARG, "max_ops too small");
    std::vector<cudaEvent_t> ev(ops.size() + 1);
    for (auto& e : ev) cudaEventCreate(&e);
    cudaError_t e = cudaEventRecord(ev[0], c->stream);
    for (size_t i = 0; i < ops.size() && e == cudaSuccess; ++i) {
        e = ops[i](c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[i + 1], c->stream);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev.back());
    for (size_t i = 0; i < ops.size() && e == cudaSuccess; ++i) {
        e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
        kind[i] = ops[i].kind;
    }
    for (auto& x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_fail(c, e, "adr_profile_step");
    *n_ops = int(ops.size());
    return ADR_OK;
}

adr_status adr_synchronize(adr_ctx* c) {
    if (!c) return ADR_ERR_ARG;
    cudaError_t e = c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
    int err = 0;
    e = cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read error word");
    if (err != 0) {
        cudaMemset(c->d_err, 0, sizeof(int));
        char buf[96];
        std::snprintf(buf, sizeof buf, "a bounded device wait timed out (code 0x%x)", err);
        return fail(c, ADR_ERR_TIMEOUT, buf);
    }
    return ADR_OK;
}

adr_status adr_test_bounded_wait(adr_ctx* c, double limit_ms) {
    if (!c) return ADR_ERR_ARG;
    if (!(limit_ms > 0.0) || limit_ms > 1000.0) return fail(c, ADR_ERR_ARG, "limit_ms must be in (0, 1000]");
    const cudaError_t e = adr::launch_wait_probe(c->d_err, limit_ms, c->stream);
    return e == cudaSuccess ? ADR_OK : cuda_fail(c, e, "adr_test_bounded_wait");
}

adr_status adr_get_info(const adr_ctx* c, double kappa[3], double* abar, double beta[3]) {
    if (!c) return ADR_ERR_ARG;
    if (c->bs) {
        // the largest kappa per direction over the instances; a_max and beta of instance 0
        const adr_batch_state& b = *c->bs;
        if (kappa) {
            kappa[0] = kappa[1] = kappa[2] = 0.0;
            for (int i = 0; i < b.B; ++i)
                for (int m = 0; m < 2; ++m) kappa[m] = std::max(kappa[m], b.kappa[size_t(i) * 2 + m]);
        }
        return adr_get_instance_info(c, 0, nullptr, abar, beta);
    }
    if (kappa) for (int m = 0; m < 3; ++m) kappa[m] = c->kappa[m];
    if (abar) *abar = c->abar;
    if (beta) for (int m = 0; m < 3; ++m) beta[m] = c->beta[m];
    return ADR_OK;
}

adr_status adr_get_instance_info(const adr_ctx* c, int instance, double kappa[3], double* abar, double beta[3]) {
    if (!c) return ADR_ERR_ARG;
    if (!c->bs) {
        if (instance != 0) return ADR_ERR_ARG;
        return adr_get_info(c, kappa, abar, beta);
    }
    const adr_batch_state& b = *c->bs;
    if (instance < 0 || instance >= b.B) return ADR_ERR_ARG;
    if (!b.set[instance]) return ADR_ERR_STATE;
    const double* k = &b.coef[size_t(instance) * kCoef];
    if (kappa) { kappa[0] = b.kappa[size_t(instance) * 2]; kappa[1] = b.kappa[size_t(instance) * 2 + 1]; kappa[2] = 0.0; }
    if (abar) *abar = k[8];
    if (beta) { beta[0] = k[6]; beta[1] = k[7]; beta[2] = 0.0; }
    return ADR_OK;
}

adr_status adr_get_batch_plan(const adr_ctx* c, int mode, int* tile_edge, int* grid) {
    if (!c || !c->bs || (mode != 1 && mode != 2)) return ADR_ERR_ARG;
    const adr_batch_state& b = *c->bs;
    if (!b.tuned) return ADR_ERR_STATE;
    if (tile_edge)
        for (int i = 0; i < b.B; ++i)   // mixed: the tensor-core tiles' output extent (128 along x1, 64 along x2)
            tile_edge[i] = b.mixed ? (mode == 1 ? 128 : 64) : adr::batch_tile_edge(b.tile[mode - 1][i]);
    if (grid) *grid = b.grid[mode - 1];
    return ADR_OK;
}

int adr_phi_route_used(const adr_ctx* c, int* halvings, int* terms) {
    if (!c) return 0;
    if (halvings) *halvings = c->phi_route == ADR_PHI_DOUBLING ? c->dbl_s : 0;
    if (terms) *terms = c->phi_route == ADR_PHI_DOUBLING ? c->dbl_p : 0;
    return c->phi_route;
}

adr_status adr_tc_factor_slices(const adr_ctx* c, int* slices) {
    if (!c || !slices) return ADR_ERR_ARG;
    *slices = 0;
    if (!c->tc || c->bs || c->periodic || !c->coeffs_set) return ADR_OK;
    *slices = 4;   // every standard image of the TMA-fed kernel (contract_tma.cu)
    return ADR_OK;
}

int adr_kernels_per_step(const adr_ctx* c) {
    if (!c) return -1;
    if (c->coeffs_set || c->periodic) {   // count the kernels of the schedule itself (the address is never used)
        static double dummy[1];
        int n = 0;
        for (const auto& op : step_ops(c, dummy))
            if (op.kind != OP_MEMSET) n += op.launches;
        return n;
    }
    const int d = c->dim;
    switch (c->p.scheme) {
    case ADR_LAWSON_EULER: return 1 + d;
    case ADR_ETD2RK: return 2 + 4 * d;
    case ADR_LAWSON4: return 4 + 4 * d;
    case ADR_EXPONENTIAL_EULER: return 1 + 2 * d;
    case ADR_ERK2P1: return 2 + 4 * d;
    case ADR_STABILIZED_LAWSON_EULER: return 1 + d;
    case ADR_LAWSON2A: return 2 + 3 * d;
    case ADR_LAWSON2B: return 2 + 2 * d;
    case ADR_STABILIZED_LAWSON2: return 2 + 3 * d;
    default: return -1;
    }
}

const char* adr_last_error(const adr_ctx* c) {
    return c ? c->err.c_str() : g_create_error.c_str();
}

void adr_destroy(adr_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    drop_graph(c);
    for (auto& row : c->d_El) for (auto& q : row) free_dev(q);
    free_dev(c->d_a0);
    for (auto& q : c->wsd) free_dev(q);
    if (c->bs) {
        adr_batch_state& b = *c->bs;
        free_dev(b.d_inst);
        free_dev(b.d_a);
        free_dev(b.d_f);
        { void* q = b.d_row_start; free_dev(q); b.d_row_start = nullptr; }
        free_dev(b.d_zt);
        for (auto& it : b.d_items) { void* q = it; free_dev(q); it = nullptr; }
        for (auto& it : b.d_titems) { void* q = it; free_dev(q); it = nullptr; }
        { void* q = b.d_sunits; free_dev(q); b.d_sunits = nullptr; }
        { void* q = b.d_img; free_dev(q); b.d_img = nullptr; }
        { void* q = b.d_fsc; free_dev(q); b.d_fsc = nullptr; }
        free_dev(b.d_tci);
        for (auto& t : b.d_phi) { void* q = t; free_dev(q); t = nullptr; }
        for (auto& t : b.d_lo) { void* q = t; free_dev(q); t = nullptr; }
        { void* q = b.d_ulo; free_dev(q); b.d_ulo = nullptr; }
        { void* q = b.d_uhs; free_dev(q); b.d_uhs = nullptr; }
        { void* q = b.d_bslots; free_dev(q); b.d_bslots = nullptr; }
    }
    free_dev(c->d_a);
    for (auto& row : c->d_E) for (auto& p : row) free_dev(p);
    for (auto& p : c->d_V) free_dev(p);
    for (auto& p : c->d_Vi) free_dev(p);
    for (auto& p : c->d_lam) { void* q = p; free_dev(q); p = nullptr; }
    for (auto& p : c->ws) free_dev(p);
    free_dev(c->d_host_state);
    for (auto& q : c->d_pc) free_dev(q);
    for (auto& q : c->d_ptw) free_dev(q);
    for (auto& q : c->d_pk) free_dev(q);
    for (auto& q : c->d_pa) free_dev(q);
    for (auto& q : c->d_pb) free_dev(q);
    free_dev(c->d_psym);
    for (auto& q : c->d_pm) free_dev(q);
    free_dev(c->d_pdif);
    free_dev(c->d_pcn);
    free_dev(c->d_pz);
    for (auto& row : c->d_img) for (auto& p : row) { void* q = p; free_dev(q); p = nullptr; }  // 5 kinds
    for (auto& row : c->d_fsc) for (auto& p : row) { void* q = p; free_dev(q); p = nullptr; }
    for (auto& row : c->d_img2) for (auto& p : row) { void* q = p; free_dev(q); p = nullptr; }
    for (auto& row : c->d_fsc2) for (auto& p : row) { void* q = p; free_dev(q); p = nullptr; }
    for (auto& p : c->d_zt) { void* q = p; free_dev(q); p = nullptr; }
    { void* q = c->d_slots; free_dev(q); c->d_slots = nullptr; }
    { void* q = c->d_err; free_dev(q); c->d_err = nullptr; }
    delete c;
}

}  // extern "C"
