"""The tcgen05 BF16 GEMM (TMA, 128-byte swizzle, TMEM accumulator) against the exact products of
the same BF16-rounded operands, accumulated in FP64: FP32 accumulation over K terms bounds the
difference by ~K * 2^-24 * sum |a_k b_k|."""
import numpy as np
import pytest

from paper_1709_09763_gb300 import native

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1709_09763_gb300 import build
    build.build()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 49, 256), (1000, 256, 32), (256, 256, 1024),
                                   (130, 130, 136), (1, 1, 8)])
def test_gemm_bf16_matches_exact_products(M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.normal(0, 1, (M, K))
    B = rng.normal(0, 1, (N, K))
    C = native.gemm_bf16(A, B)
    a = native.bf16_value(native.bf16_bits(A)).astype(np.float64)
    b = native.bf16_value(native.bf16_bits(B)).astype(np.float64)
    ref = a @ b.T
    bound = K * 2.0 ** -23 * (np.abs(a) @ np.abs(b).T) + 1e-30
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
