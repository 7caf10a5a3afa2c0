// phi_k(z) on the device (k = 0, 1, 2): phi_0 = exp, phi_1(z) = (e^z - 1)/z,
// phi_2(z) = (phi_1(z) - 1)/z (Section 1; Theorem 2.4). Near zero (|z| < 1) the
// Taylor series sum_j z^j/(j+k)! is summed in FP64, which avoids the cancellation
// of the closed forms at the removable singularity; elsewhere the closed forms with
// expm1 in the working precision.
#pragma once

namespace adr {

// 1/m! for the series coefficients, evaluated by the compiler.
constexpr double inv_factorial(int m) {
    double f = 1.0;
    for (int j = 2; j <= m; ++j) f *= j;
    return 1.0 / f;
}

// sum_{j=0}^{19} z^j / (j+K)! by Horner's rule, FP64 (|z| < 1: the first omitted term is
// below 1/20! = 4e-19). Multiplications only: FP64 division is slow on this GPU.
template <int K>
__device__ __forceinline__ double phi_series_k(double z) {
    double s = inv_factorial(19 + K);
#pragma unroll
    for (int j = 18; j >= 0; --j) s = fma(s, z, inv_factorial(j + K));
    return s;
}

__device__ __forceinline__ double phi_series(int k, double z) {
    return k == 1 ? phi_series_k<1>(z) : k == 2 ? phi_series_k<2>(z) : phi_series_k<0>(z);
}

__device__ __forceinline__ double phi_eval(int k, double z) {
    if (k == 0) return exp(z);
    if (fabs(z) < 1.0) return phi_series(k, z);
    const double e = expm1(z);
    return k == 1 ? e / z : (e - z) / (z * z);
}

__device__ __forceinline__ float phi_eval(int k, float z) {
    if (k == 0) return expf(z);
    if (fabsf(z) < 1.0f) return float(phi_series(k, double(z)));   // FP64 near zero
    const float e = expm1f(z);
    return k == 1 ? e / z : (e - z) / (z * z);
}

}  // namespace adr
