// Host-side operator setup in FP64: the 1-D factors A_mu of the extracted operator,
// their exponentials and their closed-form eigenpairs (Sections 3 and 5.2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "adr_internal.h"

namespace adr {

Factor1D make_factor(int n, double abar, double beta, bool neumann_hi) {
    // Centred second differences of abar*u'' and first differences of beta*u'
    // with Dirichlet ghosts (Section 5.2); Eq. (linop) restricted to one direction. With a
    // homogeneous Neumann end at x = 1 (Eq. (adr3d)) the grid is x_i = i/n, i = 1..n, and
    // the mirror ghost u_{n+1} = u_{n-1} makes the last row abar (2 u_{n-1} - 2 u_n) / h^2.
    Factor1D f;
    f.n = n;
    f.neumann = neumann_hi;
    f.h = neumann_hi ? 1.0 / n : 1.0 / (n + 1);
    const double d2 = abar / (f.h * f.h);
    const double d1 = beta / (2.0 * f.h);
    f.sub = d2 - d1;
    f.diag = -2.0 * d2;
    f.sup = d2 + d1;
    return f;
}

std::vector<double> factor_dense(const Factor1D& f) {
    const int n = f.n;
    std::vector<double> A(size_t(n) * n, 0.0);
    for (int i = 0; i < n; ++i) {
        A[size_t(i) * n + i] = f.diag;
        if (i + 1 < n) A[size_t(i) * n + i + 1] = f.sup;
        if (i > 0) A[size_t(i) * n + i - 1] = f.sub;
    }
    if (f.neumann && n >= 2) A[size_t(n - 1) * n + n - 2] = -f.diag;   // 2 abar / h^2, no advection
    return A;
}

namespace {

// C = A * B for row-major n*n matrices (i-k-j order so the inner loop vectorises).
void matmul(const std::vector<double>& A, const std::vector<double>& B, std::vector<double>& C, int n) {
    std::fill(C.begin(), C.end(), 0.0);
    for (int i = 0; i < n; ++i) {
        double* c = &C[size_t(i) * n];
        for (int k = 0; k < n; ++k) {
            const double a = A[size_t(i) * n + k];
            if (a == 0.0) continue;
            const double* b = &B[size_t(k) * n];
            for (int j = 0; j < n; ++j) c[j] += a * b[j];
        }
    }
}

// Solve P X = Q (n*n, n right-hand sides) by Gaussian elimination with partial pivoting.
std::vector<double> solve(std::vector<double> P, std::vector<double> Q, int n) {
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double best = std::fabs(P[size_t(col) * n + col]);
        for (int r = col + 1; r < n; ++r) {
            const double v = std::fabs(P[size_t(r) * n + col]);
            if (v > best) { best = v; piv = r; }
        }
        if (best == 0.0) throw std::runtime_error("singular Pade denominator");
        if (piv != col) {
            for (int j = 0; j < n; ++j) {
                std::swap(P[size_t(col) * n + j], P[size_t(piv) * n + j]);
                std::swap(Q[size_t(col) * n + j], Q[size_t(piv) * n + j]);
            }
        }
        const double inv = 1.0 / P[size_t(col) * n + col];
        for (int r = col + 1; r < n; ++r) {
            const double f = P[size_t(r) * n + col] * inv;
            if (f == 0.0) continue;
            for (int j = col; j < n; ++j) P[size_t(r) * n + j] -= f * P[size_t(col) * n + j];
            for (int j = 0; j < n; ++j) Q[size_t(r) * n + j] -= f * Q[size_t(col) * n + j];
        }
    }
    for (int col = n - 1; col >= 0; --col) {
        const double inv = 1.0 / P[size_t(col) * n + col];
        for (int j = 0; j < n; ++j) Q[size_t(col) * n + j] *= inv;
        for (int r = 0; r < col; ++r) {
            const double f = P[size_t(r) * n + col];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) Q[size_t(r) * n + j] -= f * Q[size_t(col) * n + j];
        }
    }
    return Q;
}

}  // namespace

std::vector<double> expm_pade13(const std::vector<double>& Ain, int n) {
    // Scaling and squaring with the diagonal [13/13] Pade approximant (Higham 2005).
    // Numerator coefficients c_j = (2m-j)! m! / ((2m)! j! (m-j)!), generated by the
    // ratio c_{j+1}/c_j = (m-j) / ((2m-j)(j+1)).
    const int m = 13;
    double c[m + 1];
    c[0] = 1.0;
    for (int j = 0; j < m; ++j) c[j + 1] = c[j] * double(m - j) / (double(2 * m - j) * double(j + 1));
    const double theta13 = 5.371920351148152;  // 1-norm threshold for degree 13

    double norm1 = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += std::fabs(Ain[size_t(i) * n + j]);
        norm1 = std::max(norm1, s);
    }
    int sq = 0;
    if (norm1 > theta13) sq = int(std::ceil(std::log2(norm1 / theta13)));
    const double scale = std::ldexp(1.0, -sq);
    std::vector<double> A(Ain);
    for (auto& v : A) v *= scale;

    const size_t nn = size_t(n) * n;
    std::vector<double> A2(nn), A4(nn), A6(nn), T1(nn), T2(nn), U(nn), V(nn);
    matmul(A, A, A2, n);
    matmul(A2, A2, A4, n);
    matmul(A4, A2, A6, n);
    for (size_t e = 0; e < nn; ++e) T1[e] = c[13] * A6[e] + c[11] * A4[e] + c[9] * A2[e];
    matmul(A6, T1, T2, n);
    for (size_t e = 0; e < nn; ++e) T2[e] += c[7] * A6[e] + c[5] * A4[e] + c[3] * A2[e];
    for (int i = 0; i < n; ++i) T2[size_t(i) * n + i] += c[1];
    matmul(A, T2, U, n);
    for (size_t e = 0; e < nn; ++e) T1[e] = c[12] * A6[e] + c[10] * A4[e] + c[8] * A2[e];
    matmul(A6, T1, V, n);
    for (size_t e = 0; e < nn; ++e) V[e] += c[6] * A6[e] + c[4] * A4[e] + c[2] * A2[e];
    for (int i = 0; i < n; ++i) V[size_t(i) * n + i] += c[0];

    std::vector<double> P(nn), Q(nn);
    for (size_t e = 0; e < nn; ++e) { P[e] = V[e] - U[e]; Q[e] = V[e] + U[e]; }
    std::vector<double> R = solve(P, Q, n);
    for (int s = 0; s < sq; ++s) {
        matmul(R, R, T1, n);
        R.swap(T1);
    }
    return R;
}

Eigen1D eigen_closed_form(const Factor1D& f) {
    Eigen1D e;
    const int n = f.n;
    if (f.neumann) return e;    // not Toeplitz: no closed form (the exponential-only routes remain)
    const double sp = f.sub * f.sup;
    if (!(sp > 0.0)) return e;  // complex (or defective) spectrum
    e.real = true;
    const double root = std::sqrt(sp) * (f.sup > 0 ? 1.0 : -1.0);
    const double rho = std::sqrt(f.sub / f.sup);
    const double lrho = std::log(rho);
    const double cmid = 0.5 * (n + 1);
    const double pi = 3.14159265358979323846;
    e.lam.resize(n);
    e.V.resize(size_t(n) * n);
    e.Vinv.resize(size_t(n) * n);
    for (int j = 1; j <= n; ++j) e.lam[j - 1] = f.diag + 2.0 * root * std::cos(j * pi / (n + 1));
    const long period = 2L * (n + 1);
    for (int i = 1; i <= n; ++i) {
        const double di = std::exp((i - cmid) * lrho);
        for (int j = 1; j <= n; ++j) {
            // sin(i j pi/(n+1)) with the argument reduced modulo 2 pi exactly in integers
            const long r = (long(i) * j) % period;
            const double sn = std::sin(r * pi / (n + 1));
            e.V[size_t(i - 1) * n + (j - 1)] = di * sn;
            e.Vinv[size_t(j - 1) * n + (i - 1)] = (2.0 / (n + 1)) * sn / di;
        }
    }
    e.kappa = std::exp(std::fabs(lrho) * (n - 1));
    return e;
}

namespace {
uint16_t bf16_bits_exact(double v) {
    // v has at most 8 significant bits (an integer slice, possibly times 2^-8), so the
    // upper half of its FP32 pattern is its exact BF16 pattern.
    const float f = static_cast<float>(v);
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    return static_cast<uint16_t>(u >> 16);
}
}  // namespace

TcFactor make_tc_factor(const std::vector<double>& M, int n, int rows, bool precise, int chunk) {
    // Each row i of M (an output index) is written as 2^(e_i-7) sum_j 2^(-8j) f_j with
    // integer slices |f_j| <= 128 and max_k |M[i][k]| < 2^e_i. The image stores, per
    // (output tile of `rows` rows, K chunk of 64), four slice tiles in the 128-byte-swizzled
    // K-major layout the tensor cores read (8-row groups of 1024 B; 16-byte chunk j of row r
    // at position j ^ (r mod 8)): F0, F1, 2^-8 F1, 2^-8 F2 (standard) or F0, F1, F2, F3
    // (precise). With chunks of 32 the tiles use the 64-byte swizzle (8-row groups of 512 B;
    // chunk j of row r at position j ^ ((r / 2) mod 4)), and every image holds F0, F1, F2, F3:
    // that kernel runs the ten-product split in every pass.
    const int tile = rows * chunk * 2;
    const int nK = (n + chunk - 1) / chunk, nOut = (n + rows - 1) / rows;
    const int nq = 4;
    TcFactor out;
    out.img.assign(size_t(nOut) * nK * nq * tile, 0);
    out.fscale.assign(size_t(nOut) * rows, 0.0f);
    std::vector<double> slices(size_t(n) * n * 4, 0.0);
    for (int i = 0; i < n; ++i) {
        double rmax = 0.0;
        for (int k = 0; k < n; ++k) rmax = std::max(rmax, std::fabs(M[size_t(i) * n + k]));
        int e = 0;
        if (rmax > 0.0) std::frexp(rmax, &e);   // rmax < 2^e
        out.fscale[i] = static_cast<float>(std::ldexp(1.0, e - 7));
        for (int k = 0; k < n; ++k) {
            const double y = std::ldexp(M[size_t(i) * n + k], 7 - e);
            const double f0 = std::nearbyint(y);
            const double y1 = (y - f0) * 256.0;
            const double f1 = std::nearbyint(y1);
            const double y2 = (y1 - f1) * 256.0;
            const double f2 = std::nearbyint(y2);
            const double f3 = std::nearbyint((y2 - f2) * 256.0);
            double* sl = &slices[(size_t(i) * n + k) * 4];
            if (precise || chunk == 32) {
                sl[0] = f0; sl[1] = f1; sl[2] = f2; sl[3] = f3;
            } else {
                sl[0] = f0; sl[1] = f1; sl[2] = f1 / 256.0; sl[3] = f2 / 256.0;
            }
        }
    }
    for (int ot = 0; ot < nOut; ++ot)
        for (int c = 0; c < nK; ++c)
            for (int q = 0; q < nq; ++q) {
                uint8_t* t = &out.img[((size_t(ot) * nK + c) * nq + q) * tile];
                for (int r = 0; r < rows; ++r) {
                    const int i = ot * rows + r;
                    if (i >= n) continue;
                    for (int j = 0; j < chunk / 8; ++j)
                        for (int e2 = 0; e2 < 8; ++e2) {
                            const int k = c * chunk + 8 * j + e2;
                            if (k >= n) continue;
                            const uint16_t b = bf16_bits_exact(slices[(size_t(i) * n + k) * 4 + q]);
                            const size_t off = chunk == 64
                                ? size_t((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4) + 2 * e2)
                                : size_t((r >> 3) * 512 + (r & 7) * 64 + ((j ^ ((r >> 1) & 3)) << 4) + 2 * e2);
                            t[off] = uint8_t(b & 0xFF);
                            t[off + 1] = uint8_t(b >> 8);
                        }
                }
            }
    return out;
}

double nodal_max(const double* a, size_t count) {
    double m = -INFINITY;
    for (size_t i = 0; i < count; ++i) m = std::max(m, a[i]);
    return m;
}

double mean_face_jump(const double* a, int dim, const int* n, int mu) {
    // (1/|Omega|) int d_mu a dx = mean over the face of a(x_mu = 1) - a(x_mu = 0),
    // with trapezoidal weights over the transverse boundary-inclusive nodes.
    const int N1 = n[0] + 2, N2 = n[1] + 2, N3 = dim == 3 ? n[2] + 2 : 1;
    auto at = [&](int i1, int i2, int i3) { return a[size_t(i1) + size_t(N1) * (size_t(i2) + size_t(N2) * i3)]; };
    auto w = [](int i, int len) { return (i == 0 || i == len - 1) ? 0.5 / (len - 1) : 1.0 / (len - 1); };
    double acc = 0.0;
    if (dim == 2) {
        if (mu == 1) for (int i2 = 0; i2 < N2; ++i2) acc += w(i2, N2) * (at(N1 - 1, i2, 0) - at(0, i2, 0));
        else         for (int i1 = 0; i1 < N1; ++i1) acc += w(i1, N1) * (at(i1, N2 - 1, 0) - at(i1, 0, 0));
        return acc;
    }
    if (mu == 1) {
        for (int i3 = 0; i3 < N3; ++i3)
            for (int i2 = 0; i2 < N2; ++i2) acc += w(i3, N3) * w(i2, N2) * (at(N1 - 1, i2, i3) - at(0, i2, i3));
    } else if (mu == 2) {
        for (int i3 = 0; i3 < N3; ++i3)
            for (int i1 = 0; i1 < N1; ++i1) acc += w(i3, N3) * w(i1, N1) * (at(i1, N2 - 1, i3) - at(i1, 0, i3));
    } else {
        for (int i2 = 0; i2 < N2; ++i2)
            for (int i1 = 0; i1 < N1; ++i1) acc += w(i2, N2) * w(i1, N1) * (at(i1, i2, N3 - 1) - at(i1, i2, 0));
    }
    return acc;
}

// ------------------------------------------------------------------ host: factor images
size_t batch_tc_image_bytes(int n, int mode) {
    const int rows = mode == 2 ? kBatchTcRows2 : kBatchTcRows1;
    const size_t nOut = size_t((n + rows - 1) / rows), nK = size_t((n + kBatchTcChunk - 1) / kBatchTcChunk);
    return nOut * nK * kBatchTcFactorTiles * size_t(rows) * kBatchTcChunk * 2;
}

void make_batch_tc_factor(const double* M, int n, int mode, uint8_t* img, float* fscale) {
    // Row i (an output index) of M is 2^(e_i-7) sum_j 2^(-8j) F_j with max_k |M[i][k]| < 2^e_i and
    // integer slices |F_j| <= 128 (rounded to nearest, so the remainder of each step is at most
    // half a unit of its slice). Per (output tile, K chunk of 32): tiles F0, F1, F2, F3,
    // 2^-8 F1, 2^-8 F2, 2^-8 F3 of `rows` rows in the 64-byte-swizzled K-major layout (8-row
    // groups of 512 B; the 16-byte chunk j of row r at position j ^ ((r / 2) mod 4)).
    const int rows = mode == 2 ? kBatchTcRows2 : kBatchTcRows1;
    const int tile = rows * kBatchTcChunk * 2;
    const int nK = (n + kBatchTcChunk - 1) / kBatchTcChunk;
    std::memset(img, 0, batch_tc_image_bytes(n, mode));
    for (int i = 0; i < n; ++i) {
        double rmax = 0.0;
        for (int k = 0; k < n; ++k) rmax = std::fmax(rmax, std::fabs(M[size_t(i) * n + k]));
        int e = 0;
        if (rmax > 0.0) std::frexp(rmax, &e);
        fscale[i] = static_cast<float>(std::ldexp(1.0, e - 7));
        const int ot = i / rows, r = i % rows;
        for (int k = 0; k < n; ++k) {
            double y = std::ldexp(M[size_t(i) * n + k], 7 - e);
            double f[4];
            for (int q = 0; q < 4; ++q) {
                f[q] = std::nearbyint(y);
                y = (y - f[q]) * 256.0;
            }
            const double vals[kBatchTcFactorTiles] = {f[0], f[1], f[2], f[3], f[1] / 256.0, f[2] / 256.0, f[3] / 256.0};
            const int c = k / kBatchTcChunk, kk = k % kBatchTcChunk, j = kk / 8, e2 = kk % 8;
            const size_t off = size_t((r >> 3) * 512 + (r & 7) * 64 + ((j ^ ((r >> 1) & 3)) << 4) + 2 * e2);
            for (int q = 0; q < kBatchTcFactorTiles; ++q) {
                // integers up to 128 (and their 2^-8 multiples) are exact in BF16: the upper half
                // of the FP32 pattern
                const float fv = static_cast<float>(vals[q]);
                uint32_t bits;
                std::memcpy(&bits, &fv, 4);
                const uint16_t b = uint16_t(bits >> 16);
                uint8_t* t = img + ((size_t(ot) * nK + c) * kBatchTcFactorTiles + q) * tile;
                t[off] = uint8_t(b & 0xFF);
                t[off + 1] = uint8_t(b >> 8);
            }
        }
    }
}

}  // namespace adr
