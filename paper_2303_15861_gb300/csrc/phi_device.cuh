// phi_k(z) on the device (k = 0, 1, 2): phi_0 = exp, phi_1(z) = (e^z - 1)/z,
// phi_2(z) = (phi_1(z) - 1)/z (Section 1; Theorem 2.4). Near zero (|z| < 1) the
// Taylor series sum_j z^j/(j+k)! is summed in FP64, which avoids the cancellation
// of the closed forms at the removable singularity; elsewhere the closed forms with
// expm1 in the working precision.
#pragma once

namespace adr {

__device__ __forceinline__ double phi_series(int k, double z) {
    double fact = 1.0;
    for (int j = 2; j <= k; ++j) fact *= j;
    double term = 1.0 / fact, sum = 0.0;
    for (int j = 0; j < 22; ++j) {   // |z| < 1: the 22nd term is below 1e-21
        sum += term;
        term *= z / double(j + k + 1);
    }
    return sum;
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
