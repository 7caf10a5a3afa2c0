"""The exact-slice split of the tensor-core contraction, restated in numpy (no GPU), and the
claims its design rests on:

  * x = 2^(es-7) sum_{j<4} 2^(-8j) s_j with integer slices |s_j| <= 128, each exactly a BF16
    value, reconstructs x to 2^-32 of the scale 2^es (round-to-nearest slices);
  * D0 = S0.F0, D1 = S0.F1 + S1.F0, D2 = S0.F2 + S1.F1 + S2.F0,
    D3 = S0.F3 + S1.F2 + S2.F1 + S3.F0 have integer terms of magnitude at most 2^14; for
    K <= 256 all four stay within 2^24 even in the worst case (D0 and D1 for K <= 512), so FP32
    holds them exactly; for real residual slices D2 and D3 stay far below it at K = 512 too;
  * D0 + 2^-8 D1 + 2^-16 D2 + 2^-24 D3, scaled back, equals the dot product of the operands'
    values to the products left out (below 2^-32 of the scales) plus the representation error.
"""
import numpy as np

rng = np.random.default_rng(20230315)


def slices(x, scale_exp):
    """Four integer slices of x against the scale 2^scale_exp (|x| < 2^scale_exp)."""
    y = np.ldexp(x, 7 - scale_exp)
    out = []
    for _ in range(4):
        s = np.rint(y)
        out.append(s)
        y = (y - s) * 256.0
    return out


def is_bf16(v):
    """Exactly representable in BF16 (8 significant bits, wide exponent)."""
    v = np.asarray(v, dtype=np.float64)
    m, _ = np.frexp(v)
    return np.all(np.rint(m * 256.0) == m * 256.0)


def test_slices_are_bf16_integers_and_reconstruct_to_2_to_the_minus_32():
    x = rng.standard_normal(100_000) * np.exp(rng.uniform(-20, 0, 100_000))
    es = int(np.frexp(np.abs(x).max())[1])
    s = slices(x, es)
    for sj in s:
        assert np.all(np.abs(sj) <= 128) and np.all(sj == np.rint(sj)) and is_bf16(sj)
    rec = np.ldexp(sum(np.ldexp(sj, -8 * j) for j, sj in enumerate(s)), es - 7)
    assert np.max(np.abs(rec - x)) <= np.ldexp(1.0, es) * 2.0 ** -32
    # the low slices keep their values to the last bit of FP32 inputs: FP32 x are exact
    x32 = x.astype(np.float32).astype(np.float64)
    s32 = slices(x32, es)
    rec32 = np.ldexp(sum(np.ldexp(sj, -8 * j) for j, sj in enumerate(s32)), es - 7)
    assert np.max(np.abs(rec32 - x32)) <= np.ldexp(1.0, es) * 2.0 ** -32


def accumulators(S, F):
    """D0..D3 for slices S[j][k] (state) and F[j][i, k] (factor rows)."""
    D = [F[0] @ S[0],
         F[1] @ S[0] + F[0] @ S[1],
         F[2] @ S[0] + F[1] @ S[1] + F[0] @ S[2],
         F[3] @ S[0] + F[2] @ S[1] + F[1] @ S[2] + F[0] @ S[3]]
    return D


def test_accumulators_stay_exact_in_fp32():
    # worst case: every product at 2^14 with one sign; D_k has k + 1 products per k
    for K, exact in ((256, (0, 1, 2, 3)), (512, (0, 1))):
        D = accumulators([np.full(K, 128.0)] * 4, [np.full((1, K), 128.0)] * 4)
        for k in exact:
            assert np.all(np.abs(D[k]) <= 2 ** 24), (K, k)
    # K = 512 with real residual slices: all four far below 2^24, integers, exact in FP32
    K = 512
    x = rng.uniform(-1, 1, K) * (1 - 2 ** -20)
    f = rng.uniform(-1, 1, (64, K)) * (1 - 2 ** -20)
    for d in accumulators(slices(x, 0), slices(f, 0)):
        assert np.all(d == np.rint(d)) and np.all(np.abs(d) < 2 ** 24)
        assert np.all(d.astype(np.float32).astype(np.float64) == d)


def test_combined_product_matches_the_dot_product():
    K = 256
    x = rng.standard_normal(K)
    f = np.abs(rng.standard_normal((128, K)))             # a positive, heat-kernel-like factor
    es = int(np.frexp(np.abs(x).max())[1])
    ei = np.frexp(np.abs(f).max(axis=1))[1]
    S = slices(x, es)
    F = [np.stack(c) for c in zip(*[slices(f[i], int(ei[i])) for i in range(f.shape[0])])]
    D = accumulators(S, F)
    comb = D[0] + np.ldexp(D[1], -8) + np.ldexp(D[2], -16) + np.ldexp(D[3], -24)
    got = np.ldexp(comb, es - 7) * np.ldexp(1.0, ei - 7)
    ref = f @ x
    scale = np.ldexp(1.0, es) * np.ldexp(1.0, ei) * K
    assert np.max(np.abs(got - ref) / scale) < 2.0 ** -30
    # leaving out the 2^-24 cross products (the seven-product form) loses about 2^-24 of scale
    D3_part = F[3] @ S[0]
    comb7 = D[0] + np.ldexp(D[1], -8) + np.ldexp(D[2], -16) + np.ldexp(D3_part, -24)
    got7 = np.ldexp(comb7, es - 7) * np.ldexp(1.0, ei - 7)
    assert np.max(np.abs(got7 - ref) / scale) > np.max(np.abs(got - ref) / scale)
