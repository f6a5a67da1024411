"""Tensor-core (tcgen05) GEMM tile against an exact CPU product.

Inputs are BF16 values; their products are exact in FP32 and the reference
accumulates them in FP64, so the only difference is the FP32 accumulation
order: |C - ref| <= K * 2^-24 * sum_k |a_k b_k|."""
import numpy as np
import pytest
import torch

from paper_2408_03452_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03452_gb300 import build, tpfa
    build.build()
    return tpfa


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (128, 64, 64), (300, 32, 48), (1000, 128, 256),
                                   (77, 16, 32)])
def test_tc_gemm_matches_exact_product(tp, M, N, K):
    a = synth.uniform_field(M * K, 1).reshape(M, K)
    b = synth.uniform_field(N * K, 2).reshape(N, K)
    A = torch.from_numpy(a).to(torch.bfloat16)
    Bt = torch.from_numpy(b).to(torch.bfloat16)
    C = tp.tc_gemm_bf16(A.cuda(), Bt.cuda()).cpu().numpy().astype(np.float64)
    a16 = A.to(torch.float64).numpy()
    b16 = Bt.to(torch.float64).numpy()
    ref = a16 @ b16.T
    bound = K * 2.0 ** -24 * (np.abs(a16) @ np.abs(b16).T) + 1e-30
    assert np.all(np.abs(C - ref) <= bound), np.abs(C - ref).max()
