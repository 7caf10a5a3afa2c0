"""Accuracy of the 1-D exponential factors e^{c tau A_mu} (Section 1, Section 5.2) on both sides,
against an exact reference (no GPU).

The library's host set-up (expm_pade13 in csrc/host_setup.cpp) and the oracle (its own Pade-13)
both use [13/13] Pade scaling and squaring (Higham 2005). For the 256^3 workload
||c tau A_mu||_1 is about 500, so both square nine times, and their factors carry errors of a few
1e-14 of the largest entry. The reference here is the closed-form eigendecomposition of the
tridiagonal Toeplitz A_mu (lambda_j = d + 2 sqrt(s p) cos(j pi / (n+1)),
V_ij = (s/p)^((i-1)/2) sin(i j pi / (n+1)), V^-1 = 2/(n+1) S D^-1), evaluated in numpy's
extended precision (long double) from the FP64 entries of A_mu: it is exact to about 1e-18
where kappa(V) is small, as here (cell Peclet 0.013).

This fixes the accuracy the FP64 runs can have. A time step applies the factors of three
directions four times (Lawson4), so after the 40 steps of the 256^3 workload two FP64 paths
whose factors differ by delta can differ by up to 480 delta: with delta = 5e-14 that is
2.4e-11, and the FP64 GPU path and the oracle differ by 1.2e-11 there. Compiled here with g++
against host_setup.cpp."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import adr_oracle as O
from paper_2303_15861_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2303_15861_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "adr_internal.h"
int main(int argc, char** argv) {
    const int n = std::atoi(argv[1]);
    const double abar = std::strtod(argv[2], nullptr), beta = std::strtod(argv[3], nullptr);
    const double ctau = std::strtod(argv[4], nullptr);
    std::vector<double> A = adr::factor_dense(adr::make_factor(n, abar, beta));
    for (auto& v : A) v *= ctau;
    const std::vector<double> E = adr::expm_pade13(A, n);
    std::FILE* o = std::fopen(argv[5], "wb");
    std::fwrite(E.data(), 8, E.size(), o);
    std::fclose(o);
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("expm")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([gxx, "-std=c++17", "-O1", f"-I{CSRC}", f"-I{CUDA_INC}", str(src),
                    os.path.join(CSRC, "host_setup.cpp"), "-o", str(exe)], check=True, capture_output=True)
    return d, exe


def exact_factor(A, ctau):
    """e^{ctau A} of a tridiagonal Toeplitz A from its closed-form eigenpairs, in long double."""
    n = A.shape[0]
    LD = np.longdouble
    pi = LD("3.14159265358979323846264338327950288")
    sub, sup, diag = LD(A[1, 0]), LD(A[0, 1]), LD(A[0, 0])
    i = np.arange(1, n + 1, dtype=LD)
    S = np.sin(np.outer(i, i) * pi / (n + 1))
    lam = diag + 2 * np.sqrt(sub * sup) * np.cos(i * pi / (n + 1))
    D = np.sqrt(sub / sup) ** (i - 1)
    return ((D[:, None] * S) * np.exp(LD(ctau) * lam)[None, :]) @ ((2 / LD(n + 1)) * S / D[None, :])


@pytest.mark.parametrize("case", ["256^3 lawson4 e^{tau A/2}", "128^3 etd2rk e^{tau A}"])
def test_both_pade_factors_match_the_exact_factor(harness, case):
    w, c = (W.config3(), 0.5) if case.startswith("256") else (W.config2(), 1.0)
    prob = O.ADRProblem(w.dims, w.a_nodes, w.b, w.r_poly)
    A = prob.factor(1)
    n = A.shape[0]
    d, exe = harness
    out = d / "E.bin"
    subprocess.run([str(exe), str(n), repr(float(prob.abar)), repr(float(prob.beta[0])), repr(float(c * w.tau)),
                    str(out)], check=True)
    E_lib = np.fromfile(out).reshape(n, n)
    E_orc = O.expm(c * w.tau * A)
    E_ex = exact_factor(A, c * w.tau)
    scale = float(np.abs(E_ex).max())
    err_lib = float(np.abs(E_lib.astype(np.longdouble) - E_ex).max()) / scale
    err_orc = float(np.abs(E_orc.astype(np.longdouble) - E_ex).max()) / scale
    print(f"{case}: library Pade {err_lib:.2e}, oracle Pade {err_orc:.2e} of the largest entry")
    assert err_lib < 1e-13 and err_orc < 1e-13
