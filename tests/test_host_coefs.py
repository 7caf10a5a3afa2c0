"""Host logic of the stage coefficients (no GPU): `state_coefs` in csrc/adr_internal.h writes the
state coefficients of a stage output in the working precision so that an affine combination of
states (coefficients summing to one, like Lawson4's 2/3 Eu + 1/3 U2) still sums to exactly one.
Rounded one by one, 2/3 and 1/3 sum to 1 + 3e-8 in FP32, a gain every time step would apply to
the whole state. Compiled here with g++ against the header alone."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2303_15861_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

CASES = [  # cu, cx[0..2]
    (1.0 / 3.0, (2.0 / 3.0, 0.0, 0.0)),
    (2.0 / 3.0, (1.0 / 3.0, 0.0, 0.0)),
    (1.0, (0.0, 0.0, 0.0)),
    (0.5, (0.25, 0.25, 0.0)),
    (0.1, (0.2, 0.7, 0.0)),
    (-1.0, (2.0, 0.0, 0.0)),
    (1.0, (1.0, 0.0, 0.0)),          # sum 2: not affine, left as rounded
    (0.0, (0.0, 0.0, 0.0)),          # no state term
    (1.0 / 3.0, (1.0 / 3.0, 0.0, 0.0)),   # sum 2/3: not affine
]

SRC = r"""
#include <cstdio>
#include "adr_internal.h"
int main() {
    const double cases[][4] = {%s};
    for (const auto& c : cases) {
        float tu, tx[adr::kMaxExtra];
        adr::state_coefs<float>(c[0], c + 1, tu, tx);
        double du, dx[adr::kMaxExtra];
        adr::state_coefs<double>(c[0], c + 1, du, dx);
        std::printf("%%a %%a %%a %%a %%a %%a %%a %%a\n", tu, tx[0], tx[1], tx[2], du, dx[0], dx[1], dx[2]);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("coefs")
    rows = ", ".join("{%r, %r, %r, %r}" % (cu, *cx) for cu, cx in CASES)
    src = d / "coefs.cpp"
    src.write_text(SRC % rows)
    exe = d / "coefs"
    subprocess.run([gxx, "-std=c++17", "-O1", f"-I{CSRC}", f"-I{CUDA_INC}", str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    return [[float.fromhex(v) for v in line.split()] for line in out if line.strip()]


def f32(x):
    return struct.unpack("f", struct.pack("f", x))[0]


def test_affine_combinations_sum_to_one_in_the_working_precision(results):
    for (cu, cx), vals in zip(CASES, results):
        tu, tx = vals[0], vals[1:4]
        du, dx = vals[4], vals[5:8]
        affine = abs(cu + sum(cx) - 1.0) < 1e-12 and (cu != 0.0 or any(cx))
        # sums in exact arithmetic of the rounded values
        s32 = np.float64(tu) + sum(np.float64(v) for v in tx)
        if affine:
            assert s32 == 1.0, (cu, cx, tu, tx)
        # FP64 coefficients are only rounded
        assert du == cu and dx == list(cx), (cu, cx, du, dx)
        # every coefficient stays within one FP32 ulp of its own rounding
        for got, want in zip([tu, *tx], [cu, *cx]):
            w = f32(want)
            assert abs(got - w) <= abs(np.spacing(np.float32(w))) * 1.0, (want, got)


def test_lawson4_combination_before_and_after(results):
    """2/3 and 1/3 rounded one by one sum to 1 + 2^-25 in FP32; the helper makes it one."""
    assert np.float64(f32(1.0 / 3.0)) + np.float64(f32(2.0 / 3.0)) == 1.0 + 2.0 ** -25
    tu, tx0 = results[0][0], results[0][1]
    assert tx0 == f32(2.0 / 3.0) and np.float64(tu) + np.float64(tx0) == 1.0


def test_non_affine_coefficients_are_only_rounded(results):
    for (cu, cx), vals in zip(CASES[6:], results[6:]):
        assert vals[0] == f32(cu) and vals[1:4] == [f32(v) for v in cx]
