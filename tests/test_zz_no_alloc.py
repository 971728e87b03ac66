"""krr_gather_noalloc: grouping rows by partition without any device
allocation, for callers that cannot call cudaMalloc (their GPU memory belongs
to another allocator, or their request loop must not allocate because
cudaMalloc/cudaFree can synchronise the device).  Called through the C ABI and
compared with the grouping krr_partition produces, on two calls in a row."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1805_00569_gb300 as K

pytestmark = pytest.mark.gpu


def _mixture(n, d, k, seed):
    rng = np.random.default_rng(seed)
    C = 4.0 * rng.standard_normal((k, d))
    X = C[rng.integers(0, k, n)] + rng.standard_normal((n, d))
    return X, rng.choice(n, k, replace=False).astype(np.int64)


def test_gather_noalloc_matches_partition_grouping():
    lib = K.load()
    fn = lib.krr_gather_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    ctx = K.krr_ctx_create(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        # two calls in a row; the second is smaller, so stale scratch would show
        for n, d, k, seed in [(9000, 6, 11, 1), (1500, 3, 4, 2)]:
            X, init = _mixture(n, d, k, seed)
            Xd = torch.as_tensor(X).cuda()
            assign, _, perm, offsets, _ = K.krr_partition(ctx, Xd, None, K.KRR_PART_KMEANS, k, iters=5,
                                                          init_idx=torch.as_tensor(init).cuda())
            perm2 = torch.full((n,), -1, dtype=torch.int64, device="cuda")
            off2 = torch.full((k + 1,), -1, dtype=torch.int64, device="cuda")
            rc = fn(stream, assign.data_ptr(), n, k, perm2.data_ptr(), off2.data_ptr())
            assert rc == K.KRR_OK
            torch.cuda.synchronize()
            assert torch.equal(perm2, perm)
            assert torch.equal(off2, offsets)
        # beyond the fixed scratch: rejected before anything is enqueued
        big_n = 1024 * 524288 // 8 + 1
        assert fn(stream, assign.data_ptr(), big_n, 8, perm2.data_ptr(), off2.data_ptr()) == K.KRR_ERR_ARG
        assert fn(stream, assign.data_ptr(), 10, 20000, perm2.data_ptr(), off2.data_ptr()) == K.KRR_ERR_ARG
    finally:
        ctx.close()
