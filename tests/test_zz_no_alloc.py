"""The allocation-free sampler entry point (csgs_sample_coreset_noalloc).

It serves callers that cannot allocate device memory (a host framework that owns all
GPU memory through its own pool, runtimes that forbid allocation after start-up,
callers without a csgs_ctx).  Its scratch is one fixed device array shared by every
call, so the test makes two calls in a row - a large draw, then a smaller one with
another seed - and checks each against the context-based entry point bit for bit
(same indices, same float32 weights, same count).  It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import paper_2607_02721_b300 as csgs
from paper_2607_02721_b300 import build

pytestmark = pytest.mark.gpu


def test_noalloc_sampler_matches_context_sampler_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build.build()
    L = csgs.lib()
    ctx = csgs.Context(0)
    rng = np.random.default_rng(5)
    n = 50_000
    s = rng.random(n) ** 4
    s[rng.random(n) < 0.3] = 0.0
    p = torch.tensor(s / s.sum(), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for m, seed in ((20_000, 1), (3_000, 99)):
        idx_ref, w_ref = ctx.sample_coreset_p(p, m, seed)
        torch.cuda.synchronize()
        idx = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        w = torch.full((m,), -1.0, dtype=torch.float32, device="cuda")
        nd = ctypes.c_int64(-1)
        r = L.csgs_sample_coreset_noalloc(ctypes.c_void_p(p.data_ptr()), n, m, seed, ctypes.c_void_p(idx.data_ptr()),
                                          ctypes.c_void_p(w.data_ptr()), ctypes.byref(nd),
                                          ctypes.c_void_p(stream.cuda_stream))
        assert r == csgs.CSGS_OK
        assert nd.value == idx_ref.numel()
        k = nd.value
        assert torch.equal(idx[:k], idx_ref)
        assert torch.equal(w[:k], w_ref)
    # sizes beyond the fixed scratch are rejected
    big = csgs.CSGS_NOALLOC_MAX_N + 1
    r = L.csgs_sample_coreset_noalloc(ctypes.c_void_p(p.data_ptr()), big, 10, 0, ctypes.c_void_p(idx.data_ptr()),
                                      ctypes.c_void_p(w.data_ptr()), ctypes.byref(nd), None)
    assert r == csgs.CSGS_E_INVAL
    ctx.close()
