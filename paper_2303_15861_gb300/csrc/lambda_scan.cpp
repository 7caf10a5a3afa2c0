// Choice of lambda (Section 3): the Table 1 stability bounds of the schemes and the
// parameter scan the paper recommends, which runs the small problem for admissible
// values of lambda and keeps the one with the smallest error.
//
// Stability function Phi(z, lambda) of a scheme: one step from u = 1 of the test equation
// u' = lambda z u + (1 - lambda) z u, split as A = lambda z and g(u) = (1 - lambda) z u
// (Section 2; z = tau times an eigenvalue of the diffusion operator, z <= 0). The scheme
// is unconditionally stable for lambda when |Phi(z, lambda)| <= 1 for all z <= 0.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/adr.h"
#include "adr_internal.h"

namespace {

// phi_1 and phi_2 of a real argument: closed forms with expm1, the Taylor series near 0.
double phi1(double x) {
    if (std::fabs(x) < 1e-3) return 1.0 + x / 2.0 + x * x / 6.0 + x * x * x / 24.0;
    return std::expm1(x) / x;
}
double phi2(double x) {
    if (std::fabs(x) < 1e-2) return 0.5 + x / 6.0 + x * x / 24.0 + x * x * x / 120.0 + x * x * x * x / 720.0;
    return (std::expm1(x) - x) / (x * x);
}

// Phi(z, lambda) for each scheme, written as one step of the scheme on the test equation.
double stability(int scheme, double z, double lam) {
    const double a = lam * z, w = (1.0 - lam) * z;   // A and the slope of g
    switch (scheme) {
    case ADR_LAWSON_EULER:                  // e^{a}(1 + w)
        return std::exp(a) * (1.0 + w);
    case ADR_ETD2RK: {                      // erk2p2, c2 = 1
        const double U = 1.0 + z * phi1(a);
        return 1.0 + z * phi1(a) + (w * U - w) * phi2(a);
    }
    case ADR_LAWSON4: {                     // E = e^{a/2}; stages of Lawson4
        const double E = std::exp(a / 2.0);
        const double k1 = w, U2 = E * (1.0 + k1 / 2.0), k2 = w * U2;
        const double U3 = E + k2 / 2.0, k3 = w * U3;
        const double U4 = E * (E + k3), k4 = w * U4;
        return E * (E * (1.0 + k1 / 6.0) + (k2 + k3) / 3.0) + k4 / 6.0;
    }
    case ADR_EXPONENTIAL_EULER:             // 1 + z phi_1(a)
        return 1.0 + z * phi1(a);
    case ADR_ERK2P1: {                      // c2 = 1, phi_1 only
        const double U = 1.0 + z * phi1(a);
        return 1.0 + z * phi1(a) + 0.5 * (w * U - w) * phi1(a);
    }
    case ADR_STABILIZED_LAWSON_EULER:       // 1 + z e^{a}
        return 1.0 + z * std::exp(a);
    case ADR_LAWSON2A: {
        const double U = std::exp(a / 2.0) * (1.0 + w / 2.0);
        return std::exp(a) + std::exp(a / 2.0) * w * U;
    }
    case ADR_LAWSON2B: {
        const double U = std::exp(a) * (1.0 + w);
        return std::exp(a) * (1.0 + w / 2.0) + w * U / 2.0;
    }
    case ADR_STABILIZED_LAWSON2: {
        const double al = adr::kLawsonAlpha;
        const double U = 1.0 + al * z * std::exp(al * a);
        return 1.0 + z * std::exp(a / 2.0) + std::exp(a) * (w * U - w) / (2.0 * al);
    }
    default:
        return NAN;
    }
}

// max over z <= 0 of |Phi(z, lambda)|, on z = -10^t for t in [-4, 9] (4001 points) and 0.
double max_abs_phi(int scheme, double lam) {
    double m = std::fabs(stability(scheme, 0.0, lam));
    for (int i = 0; i <= 4000; ++i) {
        const double z = -std::pow(10.0, -4.0 + 13.0 * i / 4000.0);
        const double v = std::fabs(stability(scheme, z, lam));
        if (!(v <= m)) m = v;   // also catches NaN
    }
    return m;
}

}  // namespace

extern "C" adr_status adr_stability_bound(int scheme, double* lambda_min) {
    if (!lambda_min) return ADR_ERR_ARG;
    if (scheme < ADR_LAWSON_EULER || scheme > ADR_STABILIZED_LAWSON2) return ADR_ERR_ARG;
    auto stable = [&](double lam) { return max_abs_phi(scheme, lam) <= 1.0 + 1e-12; };
    if (!stable(1.0)) return ADR_ERR_UNSUPPORTED;
    double lo = 0.0, hi = 1.0;
    if (stable(lo)) { *lambda_min = 0.0; return ADR_OK; }
    for (int it = 0; it < 60; ++it) {       // stable for lambda in [bound, 1]
        const double mid = 0.5 * (lo + hi);
        if (stable(mid)) hi = mid; else lo = mid;
    }
    *lambda_min = hi;
    return ADR_OK;
}

namespace {

// The scan itself: `setup` gives a context its coefficients (grid or periodic form).
template <typename Setup>
adr_status scan(const adr_params* p, Setup setup, const double* u0_host, int m, int n_lambdas, const double* lambdas,
                int ref_substeps, int norm, void* cuda_stream, double* errors, double* best_lambda) {
    if (!u0_host || !errors || !best_lambda || (norm != 0 && norm != 1)) return ADR_ERR_ARG;
    if (m < 1 || n_lambdas < 1 || p->batch != 0 || (p->dim != 2 && p->dim != 3)) return ADR_ERR_ARG;
    if (ref_substeps <= 0) ref_substeps = 8;
    size_t N = 1;
    for (int d = 0; d < p->dim; ++d) {
        if (p->n[d] < 2) return ADR_ERR_ARG;
        N *= static_cast<size_t>(p->n[d]);
    }
    std::vector<double> cand(static_cast<size_t>(n_lambdas));
    if (lambdas) {
        for (int i = 0; i < n_lambdas; ++i) cand[static_cast<size_t>(i)] = lambdas[i];
    } else {
        double lo = 0.0;
        const adr_status st = adr_stability_bound(p->scheme, &lo);
        if (st != ADR_OK) return st;
        for (int i = 0; i < n_lambdas; ++i)
            cand[static_cast<size_t>(i)] = n_lambdas == 1 ? 1.0 : lo + (1.0 - lo) * i / double(n_lambdas - 1);
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const bool fp64 = p->precision == ADR_FP64;
    const size_t esize = fp64 ? 8 : 4;
    void* d_u = nullptr;
    void* d_ref = nullptr;
    cudaError_t e = cudaMalloc(&d_u, N * esize);
    if (e == cudaSuccess) e = cudaMalloc(&d_ref, N * sizeof(double));
    auto cleanup = [&]() {
        if (d_u) cudaFree(d_u);
        if (d_ref) cudaFree(d_ref);
    };
    if (e != cudaSuccess) { cleanup(); return ADR_ERR_ALLOC; }

    // reference: the same semidiscrete problem, Lawson4 in FP64 at tau / ref_substeps
    std::vector<double> ref(N), got(N);
    {
        adr_params q = *p;
        q.scheme = ADR_LAWSON4;
        q.precision = ADR_FP64;
        q.lambda = 1.0;
        q.tau = p->tau / ref_substeps;
        adr_ctx* c = nullptr;
        adr_status st = adr_create(&q, cuda_stream, &c);
        if (st == ADR_OK) st = setup(c);
        if (st == ADR_OK && cudaMemcpyAsync(d_ref, u0_host, N * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
            st = ADR_ERR_CUDA;
        if (st == ADR_OK) st = adr_integrate(c, d_ref, 0.0, 0.0, m * ref_substeps);
        if (st == ADR_OK && cudaMemcpyAsync(ref.data(), d_ref, N * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            st = ADR_ERR_CUDA;
        if (st == ADR_OK) st = adr_synchronize(c);
        adr_destroy(c);
        if (st != ADR_OK) { cleanup(); return st; }
    }
    double rnorm = 0.0;   // norm 0: l2, norm 1: max
    for (double v : ref) rnorm = norm ? std::max(rnorm, std::fabs(v)) : rnorm + v * v;
    if (!norm) rnorm = std::sqrt(rnorm);

    std::vector<float> f32(N);
    int best = -1;
    for (int i = 0; i < n_lambdas; ++i) {
        adr_params q = *p;
        q.lambda = cand[static_cast<size_t>(i)];
        adr_ctx* c = nullptr;
        adr_status st = adr_create(&q, cuda_stream, &c);
        if (st == ADR_OK) st = setup(c);
        if (st == ADR_OK) {
            if (fp64) {
                if (cudaMemcpyAsync(d_u, u0_host, N * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) st = ADR_ERR_CUDA;
            } else {
                for (size_t k = 0; k < N; ++k) f32[k] = float(u0_host[k]);
                if (cudaMemcpyAsync(d_u, f32.data(), N * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) st = ADR_ERR_CUDA;
            }
        }
        if (st == ADR_OK) st = adr_integrate(c, d_u, 0.0, 0.0, m);
        if (st == ADR_OK) {
            const cudaError_t ce = fp64 ? cudaMemcpyAsync(got.data(), d_u, N * 8, cudaMemcpyDeviceToHost, s)
                                        : cudaMemcpyAsync(f32.data(), d_u, N * 4, cudaMemcpyDeviceToHost, s);
            if (ce != cudaSuccess) st = ADR_ERR_CUDA;
        }
        if (st == ADR_OK) st = adr_synchronize(c);
        adr_destroy(c);
        if (st != ADR_OK) {
            errors[i] = INFINITY;   // this lambda is not usable (e.g. refused by a guard)
            continue;
        }
        if (!fp64)
            for (size_t k = 0; k < N; ++k) got[k] = f32[k];
        double d = 0.0;
        for (size_t k = 0; k < N; ++k)
            d = norm ? std::max(d, std::fabs(got[k] - ref[k])) : d + (got[k] - ref[k]) * (got[k] - ref[k]);
        if (!norm) d = std::sqrt(d);
        errors[i] = rnorm > 0 ? d / rnorm : d;
        if (!std::isfinite(errors[i])) errors[i] = INFINITY;
        if (best < 0 || errors[i] < errors[best]) best = i;
    }
    cleanup();
    if (best < 0 || !std::isfinite(errors[best])) return ADR_ERR_STATE;
    *best_lambda = cand[static_cast<size_t>(best)];
    return ADR_OK;
}

}  // namespace

extern "C" adr_status adr_lambda_scan(const adr_params* p, const double* a_nodes, const double b[3],
                                      const double r_poly[4], const double* u0_host, int m, int n_lambdas,
                                      const double* lambdas, int ref_substeps, int norm, void* cuda_stream,
                                      double* errors, double* best_lambda) {
    if (!p || !a_nodes || !b || !r_poly || p->periodic) return ADR_ERR_ARG;
    return scan(p, [&](adr_ctx* c) { return adr_set_coeffs(c, 0, a_nodes, b, r_poly); }, u0_host, m, n_lambdas,
                lambdas, ref_substeps, norm, cuda_stream, errors, best_lambda);
}

extern "C" adr_status adr_lambda_scan_periodic(const adr_params* p, const double* a_diag, const double* b_field,
                                               const double r_poly[4], const double* u0_host, int m, int n_lambdas,
                                               const double* lambdas, int ref_substeps, int norm, void* cuda_stream,
                                               double* errors, double* best_lambda) {
    if (!p || !a_diag || !b_field || !r_poly || p->periodic != 1) return ADR_ERR_ARG;
    return scan(p, [&](adr_ctx* c) { return adr_set_coeffs_periodic(c, a_diag, b_field, r_poly); }, u0_host, m,
                n_lambdas, lambdas, ref_substeps, norm, cuda_stream, errors, best_lambda);
}
