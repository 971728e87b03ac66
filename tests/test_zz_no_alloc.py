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


def _noalloc():
    fn = K.load().krr_gather_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _stable_grouping(a, p):
    """Rows grouped by partition, ascending row order inside a partition, from
    numpy's stable sort; rows whose partition lies outside [0, p) are left out."""
    a = np.asarray(a, np.int64)
    ok = (a >= 0) & (a < p)
    rows = np.nonzero(ok)[0]
    perm = rows[np.argsort(a[rows], kind="stable")]
    offsets = np.concatenate([[0], np.cumsum(np.bincount(a[rows], minlength=p))])
    return perm, offsets


@pytest.mark.parametrize("n,p", [(5000, 12288), (1024 * 1024, 512)])
def test_gather_noalloc_at_its_limits(n, p):
    """The widest partition count the scratch takes (p = 12288: 96 KiB of
    per-partition totals in shared memory) and a request that fills the
    scratch exactly (ceil(n / 1024) * p == 524288)."""
    fn = _noalloc()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    a = np.random.default_rng(n + p).integers(0, p, n).astype(np.int32)
    ad = torch.as_tensor(a).cuda()
    perm = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    off = torch.full((p + 1,), -1, dtype=torch.int64, device="cuda")
    assert fn(stream, ad.data_ptr(), n, p, perm.data_ptr(), off.data_ptr()) == K.KRR_OK
    torch.cuda.synchronize()
    eperm, eoff = _stable_grouping(a, p)
    assert np.array_equal(perm.cpu().numpy(), eperm)
    assert np.array_equal(off.cpu().numpy(), eoff)


def test_gather_noalloc_skips_out_of_range_partitions():
    """Entries outside [0, p) are skipped on the device (no write outside the
    per-partition counts): their rows land in no partition and offsets[p]
    falls short of n by their number, which is how a caller detects them."""
    fn = _noalloc()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n, p = 3000, 5
    a = np.random.default_rng(4).integers(0, p, n).astype(np.int32)
    a[[0, 17, 1023, 1024, 2999]] = [-1, p, 2**31 - 1, -(2**31), 7]
    ad = torch.as_tensor(a).cuda()
    perm = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    off = torch.full((p + 1,), -1, dtype=torch.int64, device="cuda")
    assert fn(stream, ad.data_ptr(), n, p, perm.data_ptr(), off.data_ptr()) == K.KRR_OK
    torch.cuda.synchronize()
    eperm, eoff = _stable_grouping(a, p)
    o = off.cpu().numpy()
    assert np.array_equal(o, eoff) and o[p] == n - 5
    assert np.array_equal(perm.cpu().numpy()[:o[p]], eperm)
    assert np.all(perm.cpu().numpy()[o[p]:] == -1)
