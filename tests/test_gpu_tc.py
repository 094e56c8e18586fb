"""The tcgen05 tensor-core building block (BF16 x BF16 -> FP32 in tensor memory)
against an FP64 matrix product of the same BF16 inputs, and the failure path of its
bounded completion wait."""
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


@pytest.mark.parametrize("K,N", [(16, 16), (64, 256), (128, 64), (128, 256), (32, 128)])
def test_tc_gemm_mn_major_matches_fp64(ctx, K, N):
    """The MN-major operand layout (A^T B with A [K][128], B [K][N] copied into shared
    memory as they are) against the FP64 product."""
    import torch

    g = torch.Generator().manual_seed(K * 1000 + N + 7)
    At = torch.randn(K, 128, generator=g).to(torch.bfloat16)
    Bt = torch.randn(K, N, generator=g).to(torch.bfloat16)
    C = ctx.debug_tc_gemm_mn(At.cuda(), Bt.cuda()).cpu().numpy().astype(np.float64)
    a, b = At.double().numpy(), Bt.double().numpy()
    ref = a.T @ b
    scale = np.abs(a).T @ np.abs(b)
    assert np.all(np.abs(C - ref) <= 1e-6 * scale + 1e-12), float(np.abs(C - ref).max())


def _check_product(C, A, B):
    a, b = A.double().numpy(), B.double().numpy()
    scale = np.abs(a) @ np.abs(b).T
    assert np.all(np.abs(C - a @ b.T) <= 1e-6 * scale + 1e-12)


def test_wait_budget_expiry_reports_timeout_and_context_survives(ctx):
    """A completion wait whose budget runs out (budget 0: one non-blocking test, taken
    before the 8-MMA chain can finish) reports CSGS_E_TIMEOUT; the kernel drains the
    chain before freeing its tensor memory, so the same context then computes a correct
    product, with the default and with an explicit generous budget."""
    import torch

    g = torch.Generator().manual_seed(7)
    A = torch.randn(128, 128, generator=g).to(torch.bfloat16)
    B = torch.randn(256, 128, generator=g).to(torch.bfloat16)
    Ad, Bd = A.cuda(), B.cuda()
    for _ in range(2):
        with pytest.raises(csgs.CsgsError) as e:
            ctx.debug_tc_gemm_wait(Ad, Bd, 0)
        assert e.value.status == csgs.CSGS_E_TIMEOUT
        _check_product(ctx.debug_tc_gemm(Ad, Bd).cpu().numpy().astype(np.float64), A, B)
    _check_product(ctx.debug_tc_gemm_wait(Ad, Bd, 2_000_000_000).cpu().numpy().astype(np.float64), A, B)
    with pytest.raises(csgs.CsgsError) as e:
        ctx.debug_tc_gemm_wait(Ad, Bd, -1)
    assert e.value.status == csgs.CSGS_E_INVAL
