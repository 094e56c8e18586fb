"""The tcgen05 tensor-core building block (BF16 x BF16 -> FP32 in tensor memory)
against an FP64 matrix product of the same BF16 inputs."""
import numpy as np
import pytest

import paper_2607_02721_b300 as csgs
from paper_2607_02721_b300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build.build()
    c = csgs.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("K,N", [(16, 16), (64, 256), (128, 64), (32, 128)])
def test_tc_gemm_matches_fp64(ctx, K, N):
    import torch

    g = torch.Generator().manual_seed(K * 1000 + N)
    A = torch.randn(128, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = ctx.debug_tc_gemm(A.cuda(), B.cuda()).cpu().numpy().astype(np.float64)
    a, b = A.double().numpy(), B.double().numpy()
    ref = a @ b.T
    scale = np.abs(a) @ np.abs(b).T
    assert np.all(np.abs(C - ref) <= 1e-6 * scale + 1e-12)
