"""The tensor-core products of the mixed-precision factorisation (step a2), checked alone.

C -= A B^T through the C ABI (exa_gemm_update) against the FP64 product, with
bounds that follow from each kind's arithmetic:
  T3: three TF32 products (hi/lo halves rounded to nearest, ~22 bits) and FP32
      accumulation over k terms: |err_ij| <= 2^-19 sum_k |A_ik B_jk| is generous.
  OZ: five 7-bit digits per value relative to the row maximum, exact integer
      accumulation: |err_ij| <= k * 2^-33 * max_k|A_ik| * max_k|B_jk|.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1908_06936_gb300 as exa

    c = exa.Context()
    yield c
    c.close()


def operands(m, n, k, seed, spread):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-spread, spread, (m, 1))
    B = rng.standard_normal((n, k)) * 10.0 ** rng.uniform(-spread, spread, (n, 1))
    # some exact zeros and a zero row
    A[3, :] = 0.0
    A[rng.integers(0, m, 20), rng.integers(0, k, 20)] = 0.0
    return A, B


def run(ctx, kind, A, B, C0, store):
    import torch
    import paper_1908_06936_gb300 as exa

    m, k = A.shape
    n = B.shape[0]
    dA = torch.as_tensor(A, device="cuda")
    dB = torch.as_tensor(B, device="cuda")
    # column-major C (m x n, ldc = m) held as a row-major (n, m) buffer
    dC = torch.as_tensor(np.ascontiguousarray(C0.T), device="cuda")
    ctx.check(exa.exa_gemm_update(ctx.handle, kind, m, n, k, dA, dB, dC, m, store))
    return dC.cpu().numpy().T


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (256, 384, 256), (384, 128, 512), (128, 256, 128)])
@pytest.mark.parametrize("store", [0, 1])
def test_t3_product(ctx, m, n, k, store):
    import paper_1908_06936_gb300 as exa

    A, B = operands(m, n, k, seed=m + n + k, spread=2)
    C0 = np.random.default_rng(1).standard_normal((m, n))
    got = run(ctx, exa.EXA_GEMM_T3, A, B, C0, store)
    ref = A @ B.T if store else C0 - A @ B.T
    bound = 2.0 ** -19 * (np.abs(A) @ np.abs(B).T) + 1e-300
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))


# (128, 32), (256, 96), (384, 32): odd column-tile counts (single CTAs); (128, 256), (256, 64),
# (2048, 512): CTA pairs sharing the A digits, the last with 128 tile pairs over 76 pairs of CTAs
@pytest.mark.parametrize("m,n,k", [(128, 32, 64), (256, 96, 256), (128, 256, 128), (384, 32, 192), (256, 64, 512),
                                   (2048, 512, 512)])
@pytest.mark.parametrize("store", [0, 1])
def test_oz_product(ctx, m, n, k, store):
    import paper_1908_06936_gb300 as exa

    A, B = operands(m, n, k, seed=7 * m + n + k, spread=3)
    C0 = np.random.default_rng(2).standard_normal((m, n))
    got = run(ctx, exa.EXA_GEMM_OZ, A, B, C0, store)
    ref = A @ B.T if store else C0 - A @ B.T
    bound = k * 2.0 ** -33 * np.outer(np.abs(A).max(1), np.abs(B).max(1)) + 4e-16 * np.abs(ref) + 1e-300
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))


def test_oz_exact_on_short_integers(ctx):
    # values that are exactly representable in the digits: the product must be exact
    import paper_1908_06936_gb300 as exa

    rng = np.random.default_rng(5)
    A = rng.integers(-127, 128, (128, 256)).astype(np.float64) / 128.0
    B = rng.integers(-127, 128, (32, 256)).astype(np.float64) / 256.0
    got = run(ctx, exa.EXA_GEMM_OZ, A, B, np.zeros((128, 32)), 1)
    assert np.array_equal(got, A @ B.T)


def test_bad_shapes(ctx):
    import torch
    import paper_1908_06936_gb300 as exa

    a = torch.zeros(100 * 64, dtype=torch.float64, device="cuda")
    b = torch.zeros(128 * 64, dtype=torch.float64, device="cuda")
    c = torch.zeros(128 * 128, dtype=torch.float64, device="cuda")
    assert exa.exa_gemm_update(ctx.handle, exa.EXA_GEMM_T3, 100, 128, 64, a, b, c, 128, 0) == exa.EXA_ERR_ARG


@pytest.mark.parametrize("m,n,k", [(256, 256, 64), (512, 768, 256), (768, 256, 512), (1024, 1024, 512)])
@pytest.mark.parametrize("store", [0, 1])
def test_t3_pair_product(ctx, m, n, k, store):
    # the CTA-pair kernel (256 x 256 tiles, tcgen05 .cta_group::2) computes the same
    # three-product TF32 arithmetic: same bound, and the single-CTA kernel's result to FP32 rounding
    import paper_1908_06936_gb300 as exa

    A, B = operands(m, n, k, seed=3 * m + n + k, spread=2)
    C0 = np.random.default_rng(3).standard_normal((m, n))
    got = run(ctx, exa.EXA_GEMM_T3_PAIR, A, B, C0, store)
    ref = A @ B.T if store else C0 - A @ B.T
    bound = 2.0 ** -19 * (np.abs(A) @ np.abs(B).T) + 1e-300
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))
    single = run(ctx, exa.EXA_GEMM_T3, A, B, C0, store)
    assert np.all(np.abs(got - single) <= 2.0 ** -22 * (np.abs(A) @ np.abs(B).T) + 1e-300)


@pytest.mark.parametrize("m,n,k", [(256, 256, 576), (512, 768, 1024), (768, 512, 768)])
@pytest.mark.parametrize("store", [0, 1])
def test_t3_pair_two_operand_pairs(ctx, m, n, k, store):
    # k > 512 on CTA pairs: columns 512.. are a second operand pair reduced into the same
    # accumulator (the two-panel pass of the factorisation); same three-product bound, and
    # within the sum of two such bounds of two separate passes (the FP32 partial sums
    # round differently when 1024 terms share one accumulator)
    import paper_1908_06936_gb300 as exa

    A, B = operands(m, n, k, seed=7 * m + n + k, spread=2)
    C0 = np.random.default_rng(5).standard_normal((m, n))
    got = run(ctx, exa.EXA_GEMM_T3_PAIR, A, B, C0, store)
    ref = A @ B.T if store else C0 - A @ B.T
    bound = 2.0 ** -19 * (np.abs(A) @ np.abs(B).T) + 1e-300
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))
    first = run(ctx, exa.EXA_GEMM_T3_PAIR, np.ascontiguousarray(A[:, :512]), np.ascontiguousarray(B[:, :512]), C0,
                store)
    two = run(ctx, exa.EXA_GEMM_T3_PAIR, np.ascontiguousarray(A[:, 512:]), np.ascontiguousarray(B[:, 512:]),
              first if not store else np.zeros_like(C0), 0 if not store else 1)
    two = two if not store else first + two
    assert np.all(np.abs(got - two) <= 2.0 ** -18 * (np.abs(A) @ np.abs(B).T) + 1e-300)


def test_t3_pair_k_limit(ctx):
    import torch
    import paper_1908_06936_gb300 as exa

    c = torch.zeros(256 * 256, dtype=torch.float64, device="cuda")
    for kind, k in ((exa.EXA_GEMM_T3_PAIR, 1088), (exa.EXA_GEMM_T3, 576), (exa.EXA_GEMM_OZ, 576)):
        a = torch.zeros(256 * k, dtype=torch.float64, device="cuda")
        assert exa.exa_gemm_update(ctx.handle, kind, 256, 256, k, a, a, c, 256, 0) == exa.EXA_ERR_ARG
