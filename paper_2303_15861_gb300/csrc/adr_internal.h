// Internal declarations shared by the translation units of libadr.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

namespace adr {

// ------------------------------------------------------------------ host setup (FP64)
// 1-D factor A_mu of the Kronecker sum: tridiagonal Toeplitz discretisation of
// a_max d_mumu + beta_mu d_mu on n interior nodes (Section 5.2).
struct Factor1D {
    int n = 0;
    double h = 0, sub = 0, diag = 0, sup = 0;  // coefficients of u_{i-1}, u_i, u_{i+1}
    bool neumann = false;                      // homogeneous Neumann end at x = 1 (last row)
};

Factor1D make_factor(int n, double abar, double beta, bool neumann_hi = false);
std::vector<double> factor_dense(const Factor1D& f);                   // row-major n*n
std::vector<double> expm_pade13(const std::vector<double>& A, int n);  // e^A, row-major

// Closed-form eigenpairs of the tridiagonal Toeplitz factor (real when sub*sup > 0):
// lambda_j = diag + 2 sqrt(sub*sup) cos(j pi/(n+1)),
// V[i][j] = rho^{i-c} sin(i j pi/(n+1)), rho = sqrt(sub/sup), c = (n+1)/2,
// Vinv[j][i] = 2/(n+1) sin(i j pi/(n+1)) rho^{c-i}  (1-based i, j).
struct Eigen1D {
    bool real = false;
    double kappa = 0;                 // 2-norm condition number of V (= of the diagonal scaling)
    std::vector<double> lam, V, Vinv;  // n, n*n, n*n (row-major)
};
Eigen1D eigen_closed_form(const Factor1D& f);

// a_max and beta of Eq. (amaxbeta) from the nodal a (incl. boundary ring).
double nodal_max(const double* a, size_t count);
double mean_face_jump(const double* a, int dim, const int* n, int mu);  // mu = 1..dim

// ------------------------------------------------------------------ kernel arguments
constexpr int kMaxExtra = 3;
constexpr int kMaxOut = 2;

// The state coefficients of one stage output (cu for the stencil's input, cx for the extra
// inputs) in the working precision T. Where they sum to one, an affine combination of states
// such as Lawson4's 2/3 Eu + 1/3 U2, the smallest nonzero one is replaced by one minus the
// others when that difference is exact in T, so the rounded coefficients still sum to one:
// 2/3 and 1/3 rounded to FP32 one by one sum to 1 + 3e-8, a gain that every time step would
// apply to the whole state. Only below double precision: the sum of the others is then exact
// in double, and in FP64 the rounding of the coefficients (1e-16) does not matter.
template <typename T>
inline void state_coefs(double cu, const double* cx, T& tu, T* tx) {
    tu = T(cu);
    double sum = cu;
    for (int e = 0; e < kMaxExtra; ++e) {
        tx[e] = T(cx[e]);
        sum += cx[e];
    }
    if (sizeof(T) >= sizeof(double)) return;
    if (!(sum > 1.0 - 1e-12 && sum < 1.0 + 1e-12)) return;
    int k = -2;                      // -1: cu; e >= 0: cx[e]
    double mag = 0.0;
    if (cu != 0.0) { k = -1; mag = cu < 0 ? -cu : cu; }
    for (int e = 0; e < kMaxExtra; ++e) {
        const double m = cx[e] < 0 ? -cx[e] : cx[e];
        if (cx[e] != 0.0 && (k == -2 || m < mag)) { k = e; mag = m; }
    }
    if (k == -2) return;
    double rest = (k == -1) ? 0.0 : double(tu);   // the others as T values (exact in double)
    for (int e = 0; e < kMaxExtra; ++e)
        if (e != k) rest += double(tx[e]);
    const T adj = T(1.0 - rest);
    if (double(adj) + rest != 1.0) return;           // not exact in T: keep the rounded values
    if (k == -1) tu = adj;
    else tx[k] = adj;
}

// K1: variable-coefficient stencil with a fused stage-combination epilogue.
//   g   = div_h((a - abar) grad_h u) + (b - beta) . grad_h u + r(u)
//   F   = g + A_h u,  A_h u = abar lap_h u + beta . grad_h u
//   out_j = cu[j] u + sum_i cx[j][i] X_i + cg[j] g + cF[j] F
template <typename T>
struct StencilArgs {
    const T* u = nullptr;
    const T* u_lo = nullptr;         // optional low part: the state is u + u_lo (FP32 only)
    const T* a = nullptr;            // nodal (a - abar) with the boundary ring, padded rows:
                                     // node (j1, j2, j3) in 0..n+1 at
                                     // (j3 * (n2 + 2) + j2) * apitch + j1 + 3
    int apitch = 0;                  // row pitch of a: multiple of 4, >= n1 + 5
    int dim = 3, n1 = 1, n2 = 1, n3 = 1;
    bool neumann = false;            // homogeneous Neumann faces at x_mu = 1: mirror ghosts
    bool adelta = false;             // (a - abar) Lap u instead of div((a - abar) grad u)
    double inv_h2[3] = {0, 0, 0}, inv_2h[3] = {0, 0, 0};
    double bmb[3] = {0, 0, 0};       // b - beta
    double beta[3] = {0, 0, 0};
    double abar = 0;
    double r[4] = {0, 0, 0, 0};
    const T* X[kMaxExtra] = {nullptr, nullptr, nullptr};
    int nx = 0;
    T* out[kMaxOut] = {nullptr, nullptr};
    int nout = 0;
    double cu[kMaxOut] = {0, 0};
    double cx[kMaxOut][kMaxExtra] = {{0, 0, 0}, {0, 0, 0}};
    double cg[kMaxOut] = {0, 0};
    double cF[kMaxOut] = {0, 0};
    unsigned* amax[kMaxOut] = {nullptr, nullptr};  // optional max|out_j| (float bits)
    unsigned* amax_u = nullptr;                      // optional max|u| over the interior
    int* err = nullptr;                              // device error word (bounded waits of the TMA form)
};

// K2 (SIMT): strided batched contraction C[b] = A[b] * B[b] with a fused epilogue.
// Element (m,k) of A[b] is A[b*sab + m*sam + k*sak]; likewise B (k,n), C (m,n).
// The linear offset of a C element is its index in the state array, which the phi
// epilogue decodes into (i1, i2, i3).
enum Epilogue { EPI_STORE = 0, EPI_PHI = 1, EPI_AXPY = 2, EPI_STORE2 = 3 /* hi + lo pair */ };

template <typename T>
struct ContractArgs {
    const T* A = nullptr;
    const T* B = nullptr;
    T* C = nullptr;
    long long sam = 0, sak = 0, sbk = 0, sbn = 0, scm = 0, scn = 0;
    long long sab = 0, sbb = 0, scb = 0;
    int M = 0, N = 0, K = 0, batch = 1;
    int epi = EPI_STORE;
    const T* base = nullptr;  // EPI_AXPY: C = base + alpha * acc
    double alpha = 0;
    int phik = 1;             // EPI_PHI: C = phi_k(ctau * (l1[i1]+l2[i2]+l3[i3])) * acc
    double ctau = 0;
    const double* lam[3] = {nullptr, nullptr, nullptr};
    int n1 = 1, n2 = 1;
};

// K2 (tensor cores, mixed precision): see contract_tc.cu for the exact-slice split.
// The factor M (n x n) is passed as a pre-sliced, pre-swizzled image: for output tile
// o (128 rows) and K chunk c (64 columns), four 16 KB tiles F0, F1, 2^-8 F1, 2^-8 F2.
struct TcArgs {
    const float* X = nullptr;
    const float* Xlo = nullptr;      // precise: optional low part of a double-float input
    float* Y = nullptr;
    float* Ylo = nullptr;            // EPI_STORE2: low part of the double-float result
    const uint8_t* fimg = nullptr;   // factor image (tc_factor_image_bytes(n) bytes)
    const float* fscale = nullptr;   // per output row i: 2^(e_i - 7)
    int n = 0;                       // extent of the contracted direction
    long long Q = 1;                 // product of the faster extents (1 for mode 1)
    long long npos = 0;              // positions P*Q (mode >= 2) or fibres P (mode 1)
    int nK = 0, nOut = 0;            // K chunks of 64, output tiles of 128
    long long ntiles = 0;
    bool state_is_a = true;          // modes >= 2: true; mode 1: false
    bool precise = false;            // four slices per operand, ten MMAs, double-float result
    bool vec4 = false;               // mode 1: X rows 16-byte aligned (n % 4 == 0)
    int epi = EPI_STORE;
    const float* base = nullptr;
    float alpha = 0.f;
    int phik = 1;
    // EPI_PHI (modes >= 2): z = zmu[i] + zq_a[q % na] + zq_b[q / na] + zp[p], with
    // tau*lambda tables (FP32) of the contracted direction and of the others
    const float* zmu = nullptr;
    const float* zq_a = nullptr;
    const float* zq_b = nullptr;
    const float* zp = nullptr;
    int na = 1;
    const unsigned* amax_in = nullptr;                  // max|X| (float bits)
    unsigned* amax_out = nullptr;                       // max|Y| accumulator (float bits)
    int* err = nullptr;                                 // bounded-wait timeout flags
};

// The TMA-fed form (contract_tma.cu): the same arguments plus tensor maps of the FP32 state
// (and of its low part), encoded at launch; position tiles are (p, 128 consecutive q).
struct TmaArgs : TcArgs {
    alignas(64) CUtensorMap map_x;
    alignas(64) CUtensorMap map_xlo;
    long long nqt = 1;          // position tiles per p: ceil(Q / 128) (modes >= 2)
    bool has_lo = false;
};
bool tma_supported(int n, long long Q, const void* x, const void* xlo);
cudaError_t launch_contract_tma(TmaArgs a, long long P, cudaStream_t s);

// Host: slice an FP64 factor into the tensor-core image, with output tiles of `rows` rows
// and K chunks of `chunk` (64: 128-byte swizzle, contract_tc.cu; 32: 64-byte swizzle,
// contract_tma.cu); slices F0, F1, 2^-8 F1, 2^-8 F2 (chunk 64, standard) or F0..F3 (chunk 32,
// and chunk 64 precise).
struct TcFactor {
    std::vector<uint8_t> img;
    std::vector<float> fscale;
};
TcFactor make_tc_factor(const std::vector<double>& M, int n, int rows, bool precise, int chunk = 64);
int tc_out_rows(bool state_is_a, bool precise);   // rows of an output tile of a kernel variant
int tc_pos_rows(bool state_is_a, bool precise);   // rows of a position / fibre tile

cudaError_t launch_contract_tc(const TcArgs& a, cudaStream_t s);
cudaError_t launch_amax(const float* x, size_t n, unsigned* slot, cudaStream_t s);

cudaError_t launch_stencil(const StencilArgs<double>& a, cudaStream_t s);
cudaError_t launch_stencil(const StencilArgs<float>& a, cudaStream_t s);
cudaError_t launch_contract(const ContractArgs<double>& a, cudaStream_t s);
cudaError_t launch_contract(const ContractArgs<float>& a, cudaStream_t s);
cudaError_t launch_convert_f64_to_f32(const double* in, float* out, size_t n, cudaStream_t s);

// ---------------------------------------------------------------- batched 2-D instances
// Many independent 2-D problems of uneven size advance together: every state-sized array
// of a batched context packs the instances one after another (instance i at element
// offset off, n2 rows of n1), and each stage is one persistent launch over all of them.
template <typename T>
struct BatchInst {
    int n1 = 0, n2 = 0;
    long long off = 0;             // element offset of the instance in every packed state array
    long long row0 = 0;            // first row of the instance in the concatenated row list
    long long a_off = 0;           // offset of its padded (a - abar), layout as StencilArgs::a
    int apitch = 0;
    T ih2[2] = {0, 0}, i2h[2] = {0, 0}, bmb[2] = {0, 0}, beta[2] = {0, 0};
    T abar = 0, r[4] = {0, 0, 0, 0};
    long long f_off[5][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}};  // factor role x direction
    long long zt_off[2] = {-1, -1};                                    // tau * eigenvalues per direction
    int vec = 0;                   // n1, n2, off and factor offsets multiples of 4 (16-byte rows)
};

// Factor roles of a batched context (the same numbering as the single-grid factor kinds).
enum BatchRole { BR_EXP_HALF = 0, BR_EXP_ONE = 1, BR_V = 2, BR_VINV = 3, BR_EXP_ALPHA = 4 };
constexpr int kBatchRoles = 5;
// alpha of the stabilized second-order Lawson scheme (Appendix)
constexpr double kLawsonAlpha = 0.327;

// One stencil stage over all instances: packed arrays, per-instance coefficients from
// `inst`, the stage combination (cu, cx, cg, cF) shared by all instances. Work unit: one
// row (i2) of one instance, found through the row prefix `row_start` (ninst + 1 entries).
template <typename T>
struct BatchStencilArgs {
    const BatchInst<T>* inst = nullptr;
    const long long* row_start = nullptr;
    int ninst = 0;
    long long rows = 0;
    const T* a = nullptr;          // all instances' padded (a - abar)
    const T* u = nullptr;
    const T* X[kMaxExtra] = {nullptr, nullptr, nullptr};
    int nx = 0;
    T* out[kMaxOut] = {nullptr, nullptr};
    int nout = 0;
    double cu[kMaxOut] = {0, 0};
    double cx[kMaxOut][kMaxExtra] = {{0, 0, 0}, {0, 0, 0}};
    double cg[kMaxOut] = {0, 0};
    double cF[kMaxOut] = {0, 0};
    int grid = 0;                  // persistent CTAs (0: the launcher picks)
};

// Tile shapes of the batched contraction (256 threads each): 32x32, 64x64, 128x128.
enum BatchTile { BT_32 = 0, BT_64 = 1, BT_128 = 2 };
constexpr int kBatchTiles = 3;
inline int batch_tile_edge(int t) { return t == BT_32 ? 32 : t == BT_64 ? 64 : 128; }

// One mu-mode pass over all instances. items[i] = {instance, tile row, tile column, tile
// shape}; mode 1: Y_i = X_i M_i^T (rows of x1), mode 2: Y_i = M_i X_i. Epilogues as
// ContractArgs, with the phi argument tau (lambda_1[i1] + lambda_2[i2]) of each instance.
template <typename T>
struct BatchContractArgs {
    const BatchInst<T>* inst = nullptr;
    const int4* items = nullptr;
    int nitems = 0;
    int mode = 1;
    int role = BR_VINV;
    const T* factors = nullptr;    // all instances' dense factors
    const T* zt = nullptr;         // all instances' tau * eigenvalues (working precision)
    const T* X = nullptr;
    T* Y = nullptr;
    int epi = EPI_STORE;
    const T* base = nullptr;
    double alpha = 0;
    int phik = 1;
    bool aligned = false;          // X, Y (and base) 16-byte aligned: vector loads where vec
    int grid = 0;
};

cudaError_t launch_batch_stencil(const BatchStencilArgs<double>& a, cudaStream_t s);
cudaError_t launch_batch_stencil(const BatchStencilArgs<float>& a, cudaStream_t s);
cudaError_t launch_batch_contract(const BatchContractArgs<double>& a, cudaStream_t s);
cudaError_t launch_batch_contract(const BatchContractArgs<float>& a, cudaStream_t s);

// ------------------------------------------------ batched 2-D instances, mixed precision
// The batched workload's eigenbases are ill-scaled (kappa(V_mu) up to 2e2 per direction) and
// ETD2RK at lambda = 1 amplifies a perturbation about a hundredfold over its 30 steps, so an
// FP32 state or FP32 rounding between the passes of a phi action leaves up to 3e-4 on the worst
// instances. The mixed batched path therefore carries every state-like array as a compensated
// FP32 pair (hi + lo), slices it into five exact BF16 slices against a per-instance scale, and
// runs the mu-mode products on the tensor cores (batch_tc.cu); the stencil forms its one-sided
// differences from both parts (batch_stencil2_kernel, batch2d.cu).

// Per instance (batch_tc.cu): sizes, packed offset, and the offsets of its sliced factor
// images (bytes into the image buffer), row scales and double-float phi tables.
struct BatchTcInst {
    int n1 = 0, n2 = 0;
    long long off = 0;                                   // element offset in every packed array
    long long img_off[5][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}};  // role x direction
    long long fsc_off[5][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}};
    int vec = 0;                                         // n1 and off multiples of 4 (16-byte rows)
};

// One mu-mode pass over every instance on the tensor cores. items[i] = {instance, position
// tile, output tile, 0}: mode 1 (Y_i = X_i M^T, K = n1): 64 rows (x2 fibres) x 128 outputs;
// mode 2 (Y_i = M X_i, K = n2): 128 positions (x1) x 64 outputs. Inputs and outputs are
// double-float pairs (a NULL low part reads as zero / is not written).
//   EPI_STORE: Y (+ Ylo) = the product;  EPI_PHI (mode 2): times the double-float table
//   phi = (hi, lo) pairs, one per node of the instance;  EPI_AXPY: base (+ base_lo) + alpha
//   times the product. Yhs, when set, receives a copy of the high part. amax_in[i] is the
//   max|X| of instance i (float bits), amax_out[i] accumulates max|Y|.
struct BatchTcArgs {
    const BatchTcInst* inst = nullptr;
    const int4* items = nullptr;
    int nitems = 0;
    int mode = 1;
    int role = 0;
    const uint8_t* fimg = nullptr;
    const float* fscale = nullptr;
    const float* X = nullptr;
    const float* Xlo = nullptr;
    float* Y = nullptr;
    float* Ylo = nullptr;
    float* Yhs = nullptr;
    int epi = EPI_STORE;
    const float* base = nullptr;
    const float* base_lo = nullptr;
    double alpha = 0;
    const float2* phi = nullptr;
    const unsigned* amax_in = nullptr;
    unsigned* amax_out = nullptr;
    int* err = nullptr;
    int grid = 0;
};
cudaError_t launch_batch_tc(const BatchTcArgs& a, cudaStream_t s);
// Bytes of the sliced image of an n x n factor in a pass of the given mode, and the host
// slicing: per (output tile, K chunk of 32), seven 64-byte-swizzled K-major BF16 tiles
// F0, F1, F2, F3, 2^-8 F1, 2^-8 F2, 2^-8 F3 of 64 (mode 2) or 128 (mode 1) rows; row i of
// the factor is 2^(e_i-7) sum_j 2^(-8j) F_j with integer |F_j| <= 128.
constexpr int kBatchTcRows1 = 128;         // output rows of a mode-1 factor tile (UMMA M)
constexpr int kBatchTcRows2 = 64;          // output rows of a mode-2 factor tile (UMMA N)
constexpr int kBatchTcChunk = 32;          // K per tile
constexpr int kBatchTcFactorTiles = 7;     // F0, F1, F2, F3, 2^-8 F1, 2^-8 F2, 2^-8 F3
size_t batch_tc_image_bytes(int n, int mode);
void make_batch_tc_factor(const double* M, int n, int mode, uint8_t* img, float* fscale);   // host_setup.cpp

// The compensated stage stencil of a mixed batched context: as BatchStencilArgs, with
// optional low parts of u and of the extra inputs, and per output an optional low part
// (the combination in double-float arithmetic), an optional copy of the high part (hs) and
// an optional per-instance max|out| (amax[j][instance], float bits).
struct BatchStencil2Args {
    BatchStencilArgs<float> s;
    const float* u_lo = nullptr;
    const float* X_lo[kMaxExtra] = {nullptr, nullptr, nullptr};
    float* out_lo[kMaxOut] = {nullptr, nullptr};
    float* out_hs[kMaxOut] = {nullptr, nullptr};
    unsigned* amax[kMaxOut] = {nullptr, nullptr};
    // optional marching form: units {instance, first x1 node, first row, rows}, one warp each
    // (32 x1 nodes); without them one warp per row of an instance
    const int4* units = nullptr;
    int nunits = 0;
};
cudaError_t launch_batch_stencil2(const BatchStencil2Args& a, cudaStream_t s);
// lo[i] = (u[i] == hs[i]) ? lo[i] : 0 over n elements: the low part of the state survives
// only where the caller's array still holds the high part the library wrote last.
cudaError_t launch_batch_keep_lo(const float* u, const float* hs, float* lo, long long n, cudaStream_t s);
// amax[i] = max |x| over instance i (float bits; atomicMax, so zero the slots first).
cudaError_t launch_batch_amax(const BatchStencilArgs<float>& geom, const float* x, unsigned* amax, cudaStream_t s);

// A kernel that waits on an mbarrier nothing arrives on, gives up after limit_ms and sets a code
// in err (wait_check.cu).
cudaError_t launch_wait_probe(int* err, double limit_ms, cudaStream_t s);

// ---------------------------------------------------------------- periodic Fourier contexts
// The pseudospectral form of the paper's two-dimensional experiment (Section 5.1): the state
// lives on n_1 x ... x n_d Fourier nodes (n_mu a power of two, <= 1024); derivatives and the
// matrix functions of A are applied to Fourier coefficients (periodic.cu).
template <typename T>
struct Cplx {
    T x, y;
};

template <typename T>
struct PeriodicArgs {
    int dim = 2;
    int n[3] = {1, 1, 1};
    long long N = 0;
    Cplx<T>* Cu = nullptr;                 // transform of the stage input
    Cplx<T>* C[3] = {nullptr, nullptr, nullptr};   // work: derivatives, fluxes, outputs (d of them)
    const Cplx<T>* tw[3] = {nullptr, nullptr, nullptr};   // e^{-2 pi i j / n_mu}, j < n_mu / 2
    const T* k[3] = {nullptr, nullptr, nullptr};          // wavenumbers (Nyquist 0)
    const T* a[3] = {nullptr, nullptr, nullptr};          // a_mumu at the nodes
    const T* b[3] = {nullptr, nullptr, nullptr};          // b_mu at the nodes
    const Cplx<T>* sym = nullptr;          // symbol of A at every Fourier point
    double r[4] = {0, 0, 0, 0};
    bool adelta = false;                   // a Lap u form: sum_mu a_mumu D_mu D_mu u + D_mu (b_mu u)
    T* dif = nullptr;                      // adelta: sum_mu a_mumu D_mu D_mu u at the nodes (work)
    Cplx<T>* CN = nullptr;                 // fused stages: the pointwise part of F, transformed (work)
};

// One fused stage of a 2-D periodic context, computed in Fourier space from the transform of x
// to the result y (real): with H = cgF F^(x) - cg s x^ (s the symbol of A; cgF = cg: the
// remainder g, cg = 0: F),
//     y = Re F^-1 ( Mu (cu x^) + Mg (H + cgz Z) + cz Z ),
// and, when Zs is set, Zs = Ms (zu x^ + zF F^(x) - zg s x^), where the multipliers Mu, Mg, Ms
// (NULL: the identity) are Fourier-space arrays and Z a Fourier-space array saved by an earlier
// stage (read before Zs is written, so a stage may read and save the same array). With E_h, E_1
// the multipliers e^{tau s/2}, e^{tau s}:
//   Lawson2a: U = E_h (u + tau/2 g(u)), Zs = E_1 u^; u+ = Re F^-1 (Z + tau E_h g(U)^).
//   Lawson2b: U = E_1 (u + tau g(u)), Zs = E_1 (u^ + tau/2 g(u)^); u+ = Re F^-1 (Z + tau/2 g(U)^).
//   Lawson-Euler u+ = E_1 (u + tau g(u)); stabilized Lawson-Euler u+ = u + tau E_1 F(u);
//   exponential Euler u+ = u + tau phi_1 F(u).
//   ETD2RK: U = u + tau phi_1 F(u), Zs = g(u)^; u+ = U + tau phi_2 (g(U)^ - Z); erk2p1 the
//   same with tau/2 phi_1 in the second stage.
template <typename T>
struct PeriodicStage {
    const T* x = nullptr;
    T* y = nullptr;
    const Cplx<T>* Mu = nullptr;
    const Cplx<T>* Mg = nullptr;
    const Cplx<T>* Ms = nullptr;
    const Cplx<T>* Z = nullptr;
    Cplx<T>* Zs = nullptr;
    double cu = 0, cgF = 0, cg = 0, cgz = 0, cz = 0;
    double zu = 1, zF = 0, zg = 0;
    // chaining: the last pass also transforms y along x1 for the next stage (whose x is this y),
    // and that stage then starts from the transform already in place (4 passes instead of 5)
    bool hand_on = false, take_over = false;
};

// Sets the shared-memory limits of the Fourier kernels of one precision (once, before any
// launch or stream capture).
cudaError_t periodic_prepare(bool fp64);
// Whether the lines of an axis (n points; axis 0 = x1, dim - 1 the pivot) fit the shared memory
// of the Fourier passes.
bool periodic_line_fits(int n, int axis, int dim, bool fp64);
// One stage: out_j = cu u + sum_e cx X_e + cg g(u) + cF F(u), F(u) = sum_mu D_mu(a_mumu D_mu u +
// b_mu u) + r(u), g = F - A u (the grid fields of s are not used; out_j must not alias u).
// Number of kernel launches:
int periodic_rhs_launches(int dim, int nout);
cudaError_t launch_periodic_rhs(const PeriodicArgs<double>& P, const StencilArgs<double>& s, cudaStream_t st);
cudaError_t launch_periodic_rhs(const PeriodicArgs<float>& P, const StencilArgs<float>& s, cudaStream_t st);
// y = base + alpha Re(IFFT(M FFT(x))) (y = Re(...) when base is null). Number of launches:
int periodic_multiplier_launches(int dim);
// Fused stages (2-D only; 5 launches). Number of launches (0: not available for dim):
int periodic_stage_launches(int dim, bool take_over);
cudaError_t launch_periodic_stage(const PeriodicArgs<double>& P, const PeriodicStage<double>& s, cudaStream_t st);
cudaError_t launch_periodic_stage(const PeriodicArgs<float>& P, const PeriodicStage<float>& s, cudaStream_t st);
cudaError_t launch_periodic_multiplier(const PeriodicArgs<double>& P, const Cplx<double>* M, const double* x, double* y,
                                       const double* base, double alpha, cudaStream_t st);
cudaError_t launch_periodic_multiplier(const PeriodicArgs<float>& P, const Cplx<float>* M, const float* x, float* y,
                                       const float* base, double alpha, cudaStream_t st);

}  // namespace adr
