"""Host slicing of the factors for the batched tensor-core contraction (no GPU):
`make_batch_tc_factor` (csrc/host_setup.cpp) writes each factor row i as
2^(e_i - 7) (F0 + 2^-8 F1 + 2^-16 F2 + 2^-24 F3) with integer slices |F_j| <= 128, into tiles of
64 (mode 2) or 128 (mode 1) rows per output tile and 32 K columns per chunk, seven tiles per
(output tile, chunk): F0, F1, F2, F3, 2^-8 F1, 2^-8 F2, 2^-8 F3, each 64-byte-swizzled K-major
BF16 (8-row groups of 512 bytes; 16-byte chunk j of row r at position j ^ ((r / 2) mod 4)).
This test decodes the bytes with that rule, written out here, and checks that the slices are
exact BF16 integers (or their 2^-8 multiples), that they rebuild every entry of the factor to
within half a unit of the last slice (2^-31 of the row maximum), and that every byte outside
the factor is zero. Compiled here with g++ against host_setup.cpp."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2303_15861_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "adr_internal.h"
int main(int argc, char** argv) {
    int n = 0, mode = 0;
    std::FILE* f = std::fopen(argv[1], "rb");
    std::fread(&n, 4, 1, f);
    std::fread(&mode, 4, 1, f);
    std::vector<double> M(size_t(n) * n);
    std::fread(M.data(), 8, M.size(), f);
    std::fclose(f);
    std::vector<uint8_t> img(adr::batch_tc_image_bytes(n, mode));
    std::vector<float> fsc(n);
    adr::make_batch_tc_factor(M.data(), n, mode, img.data(), fsc.data());
    std::FILE* o = std::fopen(argv[2], "wb");
    std::fwrite(fsc.data(), 4, fsc.size(), o);
    std::fwrite(img.data(), 1, img.size(), o);
    std::fclose(o);
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("slices")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([gxx, "-std=c++17", "-O1", f"-I{CSRC}", f"-I{CUDA_INC}", str(src),
                    os.path.join(CSRC, "host_setup.cpp"), "-o", str(exe)], check=True, capture_output=True)
    return d, exe


def run(harness, M, mode):
    d, exe = harness
    n = M.shape[0]
    inp, out = d / "in.bin", d / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.array([n, mode], dtype=np.int32).tobytes())
        f.write(np.ascontiguousarray(M, dtype=np.float64).tobytes())
    subprocess.run([str(exe), str(inp), str(out)], check=True)
    raw = open(out, "rb").read()
    fsc = np.frombuffer(raw[:4 * n], dtype=np.float32)
    img = np.frombuffer(raw[4 * n:], dtype=np.uint8)
    return fsc, img


def bf16_to_float(lo, hi):
    bits = (hi.astype(np.uint32) << 24) | (lo.astype(np.uint32) << 16)
    return bits.view(np.float32).astype(np.float64)


def decode(img, n, mode):
    """slices[q, i, k] for the seven tiles q, and a mask of the bytes that belong to the factor."""
    rows, chunk, tiles = (64 if mode == 2 else 128), 32, 7
    n_k, n_out = -(-n // chunk), -(-n // rows)
    tile = rows * chunk * 2
    assert img.size == n_out * n_k * tiles * tile
    used = np.zeros(img.size, dtype=bool)
    out = np.zeros((tiles, n, n))
    for i in range(n):
        ot, r = divmod(i, rows)
        for k in range(n):
            c, kk = divmod(k, chunk)
            j, e2 = divmod(kk, 8)
            off = (r >> 3) * 512 + (r & 7) * 64 + ((j ^ ((r >> 1) & 3)) << 4) + 2 * e2
            for q in range(tiles):
                base = ((ot * n_k + c) * tiles + q) * tile + off
                out[q, i, k] = bf16_to_float(img[base:base + 1], img[base + 1:base + 2])[0]
                used[base:base + 2] = True
    return out, used


@pytest.mark.parametrize("n,mode", [(45, 2), (45, 1), (130, 2), (70, 1)])
def test_batch_factor_slices_rebuild_the_factor(harness, n, mode):
    rng = np.random.default_rng(n + mode)
    # rows of very different scales, entries spanning six orders within a row
    M = rng.standard_normal((n, n)) * 10.0 ** rng.uniform(-6, 0, size=(n, n)) * 10.0 ** rng.uniform(-3, 3, size=(n, 1))
    M[3] = 0.0                                    # an all-zero row
    fsc, img = run(harness, M, mode)
    sl, used = decode(img, n, mode)
    assert np.all(img[~used] == 0), "bytes outside the factor must be zero"
    F = sl[:4]
    assert np.all(F == np.round(F)) and np.all(np.abs(F) <= 128)
    assert np.array_equal(sl[4:], F[1:] / 256.0)
    rmax = np.abs(M).max(axis=1)
    e = np.array([np.frexp(x)[1] if x > 0 else 0 for x in rmax])
    assert np.array_equal(fsc.astype(np.float64), np.ldexp(1.0, e - 7))
    rebuilt = np.ldexp(1.0, e - 7)[:, None] * (F[0] + F[1] / 256.0 + F[2] / 65536.0 + F[3] / 16777216.0)
    bound = np.ldexp(1.0, e - 32)[:, None]       # half a unit of the last slice
    assert np.all(np.abs(rebuilt - M) <= bound * (1 + 1e-12))
    assert np.all(rebuilt[3] == 0.0)
