/*
 * adr.h -- C ABI of libadr: exponential Runge--Kutta and Lawson time stepping for
 * semilinear advection-diffusion-reaction equations with an extracted constant-
 * coefficient operator, on one GB300 GPU.
 *
 * The problem (Eq. (adr), Section 3 of Caliari, Cassini, Einkemmer, Ostermann,
 * "Accelerating exponential integrators to efficiently solve semilinear
 * advection-diffusion-reaction equations"):
 *
 *     u_t = div(a(x) grad u) + b . grad u + r(u)   on (0,1)^d, d in {2,3},
 *
 * homogeneous Dirichlet boundary, second-order centred finite differences on n_mu
 * interior nodes per direction (x_i = i h_mu, h_mu = 1/(n_mu+1)), rewritten as
 * u' = A u + g(u) with (Eqs. (linop), (nonlin), (amaxbeta))
 *
 *     A = lambda a_max sum_mu d_mumu + beta . grad,     a_max = max a,
 *     beta_mu = |Omega|^-1 int (b_mu + d_mu a) dx,      g = F(u) - A u.
 *
 * The discrete A is the Kronecker sum A_3 (+) A_2 (+) A_1 of tridiagonal 1-D
 * factors (Section 5.2); e^{c tau A} is applied by mu-mode products with the dense
 * factors e^{c tau A_mu} (Section 1), phi_k(tau A) by mu-mode products with the
 * eigenvector matrices V_mu^-1, a pointwise phi_k(tau(l1+l2+l3)) scaling, and V_mu.
 *
 * Conventions for every entry point
 *   - Arrays are C-ordered with x1 varying fastest: a 3-D state is n3*n2*n1
 *     elements, element (i1,i2,i3) at i1 + n1*(i2 + n2*i3); interior nodes only.
 *   - State arrays live on the device of the context, are owned by the caller, and
 *     hold double (ADR_FP64) or float (all other precisions).
 *   - Calls are ordered on the stream given to adr_create and return after
 *     enqueueing, except where stated. The library owns its factors and workspace
 *     and frees them in adr_destroy.
 *   - Errors: every call returns an adr_status; arguments are validated on the host
 *     before any launch; the message of the last failure is kept per context
 *     (adr_last_error). Nothing throws across the ABI.
 */
#ifndef ADR_H
#define ADR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adr_ctx adr_ctx; /* opaque, library-owned */

typedef enum {
    ADR_OK = 0,
    ADR_ERR_ARG = 1,              /* invalid argument (sizes, pointers, enums)          */
    ADR_ERR_ALLOC = 2,            /* device or host allocation failed                   */
    ADR_ERR_CUDA = 3,             /* a CUDA runtime call failed                         */
    ADR_ERR_ILL_CONDITIONED = 4,  /* prod_mu kappa(V_mu) * eps exceeds kappa_tol        */
    ADR_ERR_COMPLEX_SPECTRUM = 5, /* s*p <= 0 (cell Peclet >= 1): no real eigenbasis     */
    ADR_ERR_TIMEOUT = 6,          /* a bounded device wait gave up                      */
    ADR_ERR_STATE = 7,            /* call out of order (e.g. step before set_coeffs)    */
    ADR_ERR_UNSUPPORTED = 8       /* valid request the library does not implement       */
} adr_status;

typedef enum {
    ADR_FP64 = 0,          /* FP64 state, stencil and contractions (FP64 FMA)            */
    ADR_FP32 = 1,          /* FP32 state, stencil and contractions (FP32 FMA)            */
    ADR_MIXED_TF32X3 = 2,  /* reserved: not implemented (returns ADR_ERR_UNSUPPORTED)    */
    ADR_MIXED_BF16X3 = 3   /* FP32 state and stencil; mu-mode contractions on the tensor
                              cores from four BF16 slices per operand (ten products) into
                              exact FP32 accumulators; factors and phi near 0 in FP64.
                              Batched contexts: the state is a compensated FP32 pair (the
                              caller's array holds the high part), five state slices and
                              fourteen products per multiply-add (see adr_create)        */
} adr_precision;

typedef enum {
    ADR_LAWSON_EULER = 0,  /* u+ = e^{tau A}(u + tau g(u))                 (Appendix)     */
    ADR_ETD2RK = 1,        /* exponential RK2 with phi_2, c2 = 1           (Appendix)     */
    ADR_LAWSON4 = 2,       /* Lawson's construction on classical RK4 (Section 1)          */
    ADR_EXPONENTIAL_EULER = 3,        /* u+ = u + tau phi_1(tau A) F(u)    (Appendix)     */
    ADR_ERK2P1 = 4,                   /* exponential RK2, phi_1 only, c2 = 1 (Appendix)   */
    ADR_STABILIZED_LAWSON_EULER = 5,  /* u+ = u + tau e^{tau A} F(u)       (Appendix)     */
    ADR_LAWSON2A = 6,                 /* second-order Lawson, midpoint form (Appendix)    */
    ADR_LAWSON2B = 7,                 /* second-order Lawson, trapezoidal form (Appendix) */
    ADR_STABILIZED_LAWSON2 = 8        /* stabilized second-order Lawson, alpha = 0.327
                                         (Appendix)                                       */
} adr_scheme;

typedef struct {
    int dim;               /* 2 or 3                                                     */
    int n[3];              /* interior points per direction, x1 first; n[2] unused if 2-D */
    double lambda;         /* lambda of Eq. (linop); <= 0 selects 1                     */
    double abar_override;  /* > 0: use this value as lambda*a_max instead of the nodal max */
    double tau;            /* time step (> 0)                                            */
    int scheme;            /* adr_scheme                                                 */
    int precision;         /* adr_precision                                              */
    double kappa_tol;      /* eigen route guard: fail with ADR_ERR_ILL_CONDITIONED when
                              prod_mu kappa(V_mu) * unit roundoff > kappa_tol; <= 0 selects
                              1e-2. Only schemes that need phi_k (ADR_ETD2RK,
                              ADR_EXPONENTIAL_EULER, ADR_ERK2P1) check it.               */
    int batch;             /* 0: one grid (dim, n). > 0: that many independent 2-D
                              instances of uneven size in one context (dim must be 2;
                              ADR_FP64, ADR_FP32 or ADR_MIXED_BF16X3, the last with
                              n1, n2 <= 256 per instance)                                 */
    const int* n_batch;    /* batch > 0: host, 2*batch ints (n1, n2) of instance i at
                              [2i], [2i+1]; copied by adr_create                          */
    int batch_tile;        /* batch > 0, FP64 / FP32: 0 = tile shapes and grid chosen by
                              the autotuner; 32, 64 or 128 = that square tile for every
                              instance (mixed batched contexts have one tiling)           */
    int phi_route;         /* adr_phi_route: how phi_k(tau A) is applied (single grids)     */
    int bc_hi;             /* adr_bc: the boundary condition on the faces x_mu = 1          */
    int form;              /* adr_form: the diffusion term                                  */
    int periodic;          /* 1: periodic Fourier pseudospectral context (see below)        */
    double length;         /* periodic: side of the periodic box (all directions)           */
} adr_params;

/* Periodic Fourier pseudospectral contexts (periodic = 1; the discretisation of the paper's
 * two-dimensional experiment, Section 5.1, Eq. (ad2d)):
 *     u_t = div(a grad u) + div(b u) + r(u)
 * or, with form = ADR_FORM_ADELTA (the one-dimensional linear experiment of Section 4, Eq.
 * (adlinearzero)), u_t = sum_mu a_mumu d_mumu u + div(b u) + r(u)
 * on a periodic box of side `length` with a diagonal diffusion tensor a = diag(a_11, ..., a_dd)
 * and a velocity field b(x), both given at the nodes x_j = x0 + j length / n_mu. Derivatives
 * are spectral (Nyquist wavenumber 0); A = lambda sum_mu a_mumu^max D_mu^2 + beta . D with
 * a^max the nodal maxima and beta_mu the mean of b_mu (Eqs. (linop), (amaxbeta)). A is
 * diagonal in Fourier space, so e^{c tau A} and phi_k(tau A) are multipliers on the Fourier
 * coefficients (ADR_PHI_FOURIER). n_mu must be powers of two in [2, 4096] along x1 and
 * [2, 1024] along the other axes (a one-dimensional problem runs on n x 2 nodes, constant along
 * x2); ADR_FP64 or ADR_FP32; single grids; bc_hi at its default. The coefficients are set with
 * adr_set_coeffs_periodic; all other entry points work as for finite-difference contexts. */
adr_status adr_set_coeffs_periodic(adr_ctx* ctx, const double* a_diag, const double* b_field,
                                   const double r_poly[4]);
/*   a_diag:  host, dim arrays of N doubles, a_11 then a_22 (then a_33), x1 fastest.
 *   b_field: host, dim arrays of N doubles, b_1 then b_2 (then b_3).
 *   r_poly:  host, 4 doubles, r(u) = r0 + r1 u + r2 u^2 + r3 u^3.
 * Computes a^max, beta, the symbol of A and the Fourier multipliers e^{c tau s} (c = 1/2, 1,
 * alpha), phi_1(tau s), phi_2(tau s) on the host in FP64 and uploads them. Synchronous. */

/* Boundary conditions on the faces x_mu = 1 (the faces x_mu = 0 are always homogeneous
 * Dirichlet). ADR_BC_NEUMANN: homogeneous Neumann, as in the paper's three-dimensional
 * experiment (Section 5.2, Eq. (adr3d)); the grid is then x_i = i/n, i = 1..n (x_n = 1 is
 * an unknown, its ghost mirrors u_{n-1}), and a_nodes still covers j = 0..n+1 (the ring
 * beyond x = 1 is not used). Only with ADR_FORM_ADELTA; single-grid contexts only. */
typedef enum { ADR_BC_DIRICHLET = 0, ADR_BC_NEUMANN = 1 } adr_bc;

/* The diffusion term: ADR_FORM_FLUX div(a grad u) with arithmetic-mean face coefficients
 * (Eq. (adr)); ADR_FORM_ADELTA a(x) Lap u (Eq. (adr3d)), for which beta = b. */
typedef enum { ADR_FORM_FLUX = 0, ADR_FORM_ADELTA = 1 } adr_form;

/* Routes for phi_k(tau A) v.
 *   ADR_PHI_EIGEN: mu-mode products with V_mu^-1, the pointwise phi_k(tau(l1+l2+l3)), V_mu
 *     (closed-form eigenpairs). Needs a real spectrum and passes the kappa guard.
 *   ADR_PHI_DOUBLING: exponentials only, for any conditioning of the eigenbasis. With
 *     X = tau A / 2^s (s halvings so that ||X||_1 <= 1/2), a Taylor sum of phi_k(X) v through
 *     the constant-coefficient stencil of A, then s doublings that follow from the phi
 *     definitions, phi_1(2X) = (e^X + I) phi_1(X) / 2 and
 *     phi_2(2X) = (phi_1(X) + (e^X + I) phi_2(X)) / 4, each applying e^{2^i X} by mu-mode
 *     products with dense factors. Per phi_1 action: s exponential actions and 14 stencil
 *     applications. Per phi_2 action: 2s exponential actions and s + 15 stencil applications.
 *     Single-grid contexts only; batched contexts use the eigen route.
 *   ADR_PHI_AUTO: the eigen route when it is available and passes the kappa guard, the
 *     doubling route otherwise. */
typedef enum { ADR_PHI_AUTO = 0, ADR_PHI_EIGEN = 1, ADR_PHI_DOUBLING = 2,
               ADR_PHI_FOURIER = 3 /* periodic contexts: multipliers on Fourier coefficients */ } adr_phi_route;

/* Create a context for one grid, or for a batch of independent 2-D instances.
 * cuda_stream is a cudaStream_t (NULL = legacy default stream) on the current device.
 * Validates params, allocates the device workspace. The factors are built by
 * adr_set_coeffs. On failure *out is NULL.
 *
 * Batched contexts. Every state-sized array (the state u of adr_step / adr_integrate,
 * the inputs and outputs of the building blocks) packs the instances one after another:
 * instance i occupies n1_i*n2_i elements (x1 fastest) starting at element
 * sum_{j<i} n1_j*n2_j. Every stage of a step is one persistent kernel launch over all
 * instances. All instances share tau and the scheme.
 *
 * Mixed batched contexts (ADR_MIXED_BF16X3) carry the state as a compensated FP32 pair: the
 * caller's FP32 array is the high part, and the library keeps the low part and a copy of the
 * high part it last wrote. Every step first keeps the low part only where the caller's array
 * still equals that copy: consecutive adr_step / adr_integrate calls on the same array continue
 * the compensated state, and elements the caller has overwritten start from a zero low part.
 * The contractions run on the tensor cores with five integer BF16 slices of the pair against
 * four of each factor row (fourteen products, exact accumulators for n <= 256); intermediates
 * between the passes of a phi action are pairs; phi_k comes from a double-float table; the
 * stencil forms its differences from both parts. This holds the batched ETD2RK workload to
 * 1e-5 of the FP64 oracle on instances where an FP32 state does not. */
adr_status adr_create(const adr_params* p, void* cuda_stream, adr_ctx** out);

/* Set the coefficients of Eq. (adr) of one instance (0 for a single-grid context,
 * 0..batch-1 for a batched one).
 *   a_nodes: host, (n3+2)*(n2+2)*(n1+2) doubles (2-D: (n2+2)*(n1+2)), the diffusion
 *            coefficient at every node including the boundary ring, x1 fastest.
 *   b:       host, 3 doubles, constant velocity (b3 ignored in 2-D).
 *   r_poly:  host, 4 doubles, reaction r(u) = r0 + r1 u + r2 u^2 + r3 u^3.
 * Computes a_max, beta (Eq. (amaxbeta)) and, on the host in FP64, the factors
 * e^{c tau A_mu} (Pade-13 scaling and squaring) and the closed-form eigenpairs of
 * A_mu; uploads them. Synchronous with respect to the host data (it may be freed on
 * return). Returns ADR_ERR_COMPLEX_SPECTRUM / ADR_ERR_ILL_CONDITIONED for ADR_ETD2RK
 * when the eigen route is unavailable or fails the kappa guard.
 * Batched contexts build only the factors their scheme uses (e^{tau A_mu} for
 * ADR_LAWSON_EULER, e^{tau A_mu / 2} for ADR_LAWSON4, the eigenpairs for ADR_ETD2RK).
 * Steps are refused (ADR_ERR_STATE) until every instance is set. The call that sets
 * the last unset instance uploads the batch and runs the autotuner: it times candidate
 * tile shapes per instance size and grid sizes on the context stream, synchronously.
 * It must not be made while the stream is being captured. */
adr_status adr_set_coeffs(adr_ctx* ctx, int instance, const double* a_nodes,
                          const double b[3], const double r_poly[4]);

/* One time step of the context's scheme, in place on the device state u_dev.
 * t is the time of the step's start (the reaction is autonomous; t is recorded only). */
adr_status adr_step(adr_ctx* ctx, void* u_dev, double t);

/* m steps from t0 with step tau (T must equal t0 + m*tau up to 1e-9 relative, or be
 * <= 0 to skip the check). The step is captured once into a CUDA graph per state
 * pointer and replayed m times on the context stream. Asynchronous. */
adr_status adr_integrate(adr_ctx* ctx, void* u_dev, double t0, double T, int m);

/* End-to-end variant of adr_integrate on a HOST state: copies u_host (pinned or
 * pageable, dtype of the precision) to a library-owned device buffer, integrates m
 * steps, copies the result back into u_host and synchronises the stream. */
adr_status adr_integrate_host(adr_ctx* ctx, void* u_host, double t0, double T, int m);

/* Building blocks of a step, exposed for verification. Inputs and outputs are
 * device arrays of the state's dtype and size; none may alias another.
 *   adr_eval_rhs:  F_out = F(u) (may be NULL), g_out = F(u) - A u (may be NULL).
 *   adr_apply_exp: y = e^{c tau A} v for c in {0.5, 1}.
 *   adr_apply_phi: y = phi_k(tau A) v for k in {0, 1, 2} through the eigenbasis. */
adr_status adr_eval_rhs(adr_ctx* ctx, const void* u_dev, void* F_out, void* g_out);
adr_status adr_apply_exp(adr_ctx* ctx, double c, const void* v_dev, void* y_dev);
adr_status adr_apply_phi(adr_ctx* ctx, int k, const void* v_dev, void* y_dev);

/* Wait for the context's stream and report device-side failures: returns
 * ADR_ERR_TIMEOUT (and clears the flag) when a bounded wait inside a tensor-core
 * kernel gave up since the last call. */
adr_status adr_synchronize(adr_ctx* ctx);

/* The failure path of the bounded device waits, exercised on purpose: enqueues on the context's
 * stream a kernel that waits on an mbarrier nothing arrives on, gives up after limit_ms
 * (in (0, 1000]; cycles at the maximum SM clock) and records a code in the context's error
 * word. The next adr_synchronize returns ADR_ERR_TIMEOUT and clears the word; the context stays
 * usable. The kernels' own waits take the same path with a limit of about 2 s. */
adr_status adr_test_bounded_wait(adr_ctx* ctx, double limit_ms);

/* Host-side facts of the current operator: kappa(V_mu) per direction (0 when the
 * spectrum is complex), lambda*a_max, and beta. Any pointer may be NULL. Periodic
 * contexts: kappa = 1 (the Fourier basis is unitary), the largest lambda*a_mumu^max. */
adr_status adr_get_info(const adr_ctx* ctx, double kappa[3], double* abar, double beta[3]);

/* The same facts for one instance of a batched context (instance 0 of a single-grid
 * context gives adr_get_info's values). ADR_ERR_STATE if the instance is not set. */
adr_status adr_get_instance_info(const adr_ctx* ctx, int instance, double kappa[3], double* abar,
                                 double beta[3]);

/* The contraction schedule of a batched context, as chosen by the autotuner (or forced
 * by batch_tile), for mode 1 (contraction along x1) or mode 2: the tile edge (32, 64 or
 * 128) of every instance in tile_edge[0..batch-1] (may be NULL) and the number of
 * persistent CTAs of the launch in *grid (may be NULL). Mixed batched contexts report their
 * tensor-core tiles' output extent: 128 in mode 1, 64 in mode 2. ADR_ERR_STATE before every
 * instance is set; ADR_ERR_ARG for a single-grid context. */
adr_status adr_get_batch_plan(const adr_ctx* ctx, int mode, int* tile_edge, int* grid);

/* One adr_step with a CUDA event recorded on the context stream around every enqueued
 * operation (no graph). Writes, for the i-th operation, its duration in ms[i] and its kind
 * in kind[i] (0 memset, 1 max-abs reduction, 2 stencil, 3 SIMT contraction,
 * 4 tensor-core contraction, 5 tensor-core contraction in the precise four-slice
 * configuration; periodic contexts: 6 pseudospectral right-hand side, 7 Fourier multiplier,
 * 8 whole stage kept in Fourier space (2-D Lawson2a and Lawson-Euler), each several kernels:
 * FFTs and pointwise passes) and the count in *n_ops. Synchronous. ADR_ERR_ARG if the step
 * has more than max_ops operations. */
adr_status adr_profile_step(adr_ctx* ctx, void* u_dev, int max_ops, float* ms, int* kind, int* n_ops);

/* The FP64 mu-mode chain y = v x_1 M_1 x_2 M_2 (x_3 M_3) -- with M_mu = e^{c tau A_mu} this is
 * e^{c tau A} v -- for callers that must not allocate device memory: a host application that
 * reserves all of its device memory up front in its own pool, or a pipeline in which a
 * cudaMalloc would synchronise the device. The paper has no counterpart; it exists for
 * such callers. It allocates nothing (no cudaMalloc / cudaFree, no allocating library
 * call) and needs no context:
 *   dim:      2 or 3; n: interior points per direction, x1 first;
 *   factors:  host array of dim device pointers, factor mu row-major n_mu x n_mu (FP64);
 *   v_dev, y_dev: device arrays of n1*n2(*n3) doubles, x1 fastest; must not alias;
 *   cuda_stream:  cudaStream_t of the launches (NULL = legacy stream). Asynchronous.
 * The intermediates live in a library-owned static device array of 2 x 1,048,576 doubles
 * (16 MiB, held on every GPU that loads the library until the process exits): grids with
 * more than 1,048,576 points return ADR_ERR_ARG. All calls share that array, so calls that
 * overlap on the GPU race with each other. The first call on a device looks up the array's
 * address (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture. Returns ADR_ERR_ARG for invalid arguments, ADR_ERR_CUDA if a CUDA call
 * or launch fails; no message is kept (adr_last_error does not cover this call). */
adr_status adr_mumode_apply_static(int dim, const int n[3], const double* const factors[3],
                                   const double* v_dev, double* y_dev, void* cuda_stream);

/* Table 1 and Theorems 2.1-2.7: the smallest lambda in [0, 1] for which the scheme is
 * unconditionally stable on the model problem, i.e. |Phi(z, lambda)| <= 1 for all z <= 0,
 * where Phi is one step of the scheme on u' = lambda z u + (1 - lambda) z u from u = 1.
 * Computed on the host by bisection over lambda, with z on a logarithmic grid down to -1e9.
 * ADR_ERR_ARG for an unknown scheme. */
adr_status adr_stability_bound(int scheme, double* lambda_min);

/* The lambda scan of Section 3 (choice of lambda): integrate a SMALL problem (params p,
 * coefficients and host initial state u0_host of N doubles as in adr_set_coeffs) for m
 * steps with each candidate lambda (lambdas[0..n_lambdas-1], or, when lambdas is NULL,
 * n_lambdas values evenly spaced from adr_stability_bound(p->scheme) to 1), and measure the
 * relative error against a reference (norm 0: l2; norm 1: the maximum norm, as the paper's
 * Section 5 measures errors): the same semidiscrete problem integrated by
 * Lawson4 in FP64 with step tau / ref_substeps (<= 0 selects 8). Writes the errors
 * (INFINITY where a lambda is refused) and the lambda with the smallest error. Runs on
 * cuda_stream and synchronises it; allocates its own device buffers. Finite-difference
 * single grids only (ADR_ERR_ARG for batched or periodic params; see adr_lambda_scan_periodic)
 * and for a norm other than 0 or 1. */
adr_status adr_lambda_scan(const adr_params* p, const double* a_nodes, const double b[3],
                           const double r_poly[4], const double* u0_host, int m, int n_lambdas,
                           const double* lambdas, int ref_substeps, int norm, void* cuda_stream,
                           double* errors, double* best_lambda);

/* The same scan for a periodic Fourier problem (p->periodic = 1; coefficients as in
 * adr_set_coeffs_periodic). With the paper's two-dimensional experiment on 2^6 modes and
 * 2^8 steps this is the scan behind the lambda values of Section 5.1. */
adr_status adr_lambda_scan_periodic(const adr_params* p, const double* a_diag, const double* b_field,
                                    const double r_poly[4], const double* u0_host, int m, int n_lambdas,
                                    const double* lambdas, int ref_substeps, int norm, void* cuda_stream,
                                    double* errors, double* best_lambda);

/* Measured arithmetic peak of the current device, for rooflines: independent FMA chains in
 * registers on every SM (8 blocks of 256 threads per SM), `iters` x 128 FMAs per thread, timed
 * with CUDA events on a private stream after one shorter warm-up launch. Writes 2 x FMAs / time
 * in TFLOP/s. kind: ADR_PEAK_FP64_FMA or ADR_PEAK_FP32_FMA. Synchronous; allocates 8 bytes.
 * ADR_ERR_ARG for an unknown kind, iters outside [1, 2^20] or a NULL pointer. */
typedef enum { ADR_PEAK_FP64_FMA = 0, ADR_PEAK_FP32_FMA = 1 } adr_peak_kind;
adr_status adr_measure_peak(int kind, int iters, double* tflops);

/* Number of kernels one adr_step launches (for launch accounting; memsets not counted). */
int adr_kernels_per_step(const adr_ctx* ctx);

/* Mixed-precision contexts after adr_set_coeffs: the number of slices (4) in which the standard
 * tensor-core images of the TMA-fed contraction write a factor; 0 for FP64 and FP32 contexts,
 * periodic and batched contexts, and before adr_set_coeffs. The exact-slice split of the
 * mu-mode products (Section 1) writes each factor row as 2^(e_i-7) sum_j 2^(-8j) f_j with
 * integer slices: four slices make a 32-bit factor, and the standard contraction then issues
 * ten BF16 products per multiply-add (every pair of state slice i and factor slice j with
 * i + j <= 3) into four TMEM accumulators D0..D3, one per weight 2^(-8(i+j)), each exact in
 * FP32. *slices must not be NULL. */
adr_status adr_tc_factor_slices(const adr_ctx* ctx, int* slices);

/* The phi route a context uses after adr_set_coeffs (ADR_PHI_EIGEN or ADR_PHI_DOUBLING; 0
 * when its scheme needs no phi_k or before adr_set_coeffs), and for the doubling route the
 * number of halvings s and of Taylor terms in *halvings, *terms (either may be NULL). */
int adr_phi_route_used(const adr_ctx* ctx, int* halvings, int* terms);

/* Message of the last failed call on ctx (or of the last failed adr_create when ctx
 * is NULL). Valid until the next call on the same context. */
const char* adr_last_error(const adr_ctx* ctx);

/* Free the context and all library-owned device memory (synchronises its stream). */
void adr_destroy(adr_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* ADR_H */
