"""Bounded device waits end, report KRR_ERR_TIMEOUT, and leave the context
usable.  No GPU fault is involved: the library's own self-check kernel waits
on an mbarrier that nothing ever completes (with a 4 KB bulk copy of its own
in flight, as the pipelined kernels have when a producer fails to deliver),
the deadline ends the wait, the copy is drained, and the kernel exits.  The
same context then runs a fit, prediction and selection that still match the
FP64 oracle."""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_1805_00569_gb300 as K
from paper_1805_00569_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_the_context_stays_usable():
    ctx = K.krr_ctx_create(0)
    try:
        for limit in (0.002, 0.05):
            t0 = time.perf_counter()
            rc = K.krr_ctx_wait_probe(ctx, limit)
            took = time.perf_counter() - t0
            assert rc == K.KRR_ERR_TIMEOUT, K.STATUS_NAMES.get(rc, rc)
            assert took >= limit and took < limit + 5.0
        assert K.krr_ctx_wait_probe(ctx, 0.0) == K.KRR_ERR_ARG
        w = synth.bkrr2(seed=21, n=700, t=90, d=9, p=2, sigmas=(3.0,), lambdas=(1e-4,))
        dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt)
        _, _, perm, offsets, _ = K.krr_partition(ctx, dev(w["X"]), None, K.KRR_PART_RANDOM, 2, seed=w["part_seed"])
        model, status, _ = K.krr_fit_batch(ctx, dev(w["X"]), dev(w["y"]), perm, offsets, w["sigmas"], w["lambdas"],
                                           "tf32")
        yhat = K.krr_predict(ctx, model, dev(w["Xt"])).cpu().numpy()
        model.free()
        assert np.all(status.cpu().numpy() == K.KRR_OK)
        operm, ooff, _ = oracle.partition_random(700, 2, w["part_seed"])
        al, _, _ = oracle.fit_batch(w["X"], w["y"], operm, ooff, w["sigmas"], w["lambdas"])
        oy = oracle.predict_all(w["X"], operm, ooff, al, w["sigmas"], w["lambdas"], w["Xt"])
        for r in range(2):
            assert np.max(np.abs(yhat[r] - oy[r])) / np.max(np.abs(oy[r])) <= 1e-6
    finally:
        ctx.close()
