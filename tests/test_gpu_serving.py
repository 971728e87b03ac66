"""Serving loop on the device: every request's prediction is bit-identical
whether it runs alone or in a mix of concurrently admitted requests (fixed
tile shapes, panel width and reduction orders; no atomics in any reduction),
matches the FP64 oracle within 1e-6 relative, and repeat requests are served
from resident models."""
import numpy as np
import pytest

import oracle
from paper_1805_00569_gb300 import KRR_OK, synth
from paper_1805_00569_gb300.serving import GpuExecutor, Scheduler, latency_summary, make_stream_requests

pytestmark = pytest.mark.gpu

TOL = 1e-6


def requests(count=14):
    st = synth.serve_stream(seed=11, requests=count, rate=1000.0, n_lo=130, n_hi=1800, t=64, repeat_frac=0.3)
    return make_stream_requests(st, count, lambda seed, n, d, t: synth.serve_request_data(seed, n, d, t), t=64)


def serve(reqs, slots, max_batch=1):
    ex = GpuExecutor(slots, prec="tf32", resident_bytes=1 << 30)
    try:
        s = Scheduler(ex, slots, 120 << 30, resident=ex.is_resident, reserved=ex.resident_bytes, t_rows=64,
                      max_batch=max_batch)
        return s.run(reqs, realtime=False), s
    finally:
        ex.close()


def rel(a, b):
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a))) if den == 0 else float(np.max(np.abs(a - b)) / den)


@pytest.fixture(scope="module")
def mix():
    rq = requests()
    res, s = serve(rq, slots=4)
    return rq, res, s


def test_mix_overlaps_and_completes(mix):
    rq, res, s = mix
    assert [r.status for r in res] == [KRR_OK] * len(rq)
    assert s.peak_concurrency > 1
    assert latency_summary(res)["completed"] == len(rq)


def test_alone_equals_mix_bitwise(mix):
    rq, res, _ = mix
    by_key = {r.key: r for r in rq if not r.predict_only}
    for r, out in zip(rq, res):
        alone_reqs = [r] if not r.predict_only else [by_key[r.key], r]
        alone, _ = serve(alone_reqs, slots=1)
        assert alone[-1].status == KRR_OK
        if r.predict_only:
            assert alone[-1].resident_hit
        assert np.array_equal(alone[-1].yhat, out.yhat), "request %d differs alone vs in the mix" % r.rid


def test_mix_matches_oracle(mix):
    rq, res, _ = mix
    for r, out in zip(rq, res):
        X, y, Xt = r.payload["X"], r.payload["y"], r.payload["Xt"]
        alpha, _, rc = oracle.fit(X, y, r.sigma, r.lam)
        assert rc == 0
        ref = oracle.predict(X, alpha, Xt, r.sigma)
        e = rel(out.yhat, ref)
        assert e <= TOL, "request %d (n=%d d=%d sigma=%.3g lambda=%.3g): rel err %.3e" % (
            r.rid, r.n, r.d, r.sigma, r.lam, e)


def test_packed_batches_equal_the_unpacked_mix_bitwise(mix):
    """Waiting fits of one feature count packed into one krr_fit_jobs call
    (one problem per partition, each with its own sigma and lambda) give
    every request the same bits as serving it on its own fit."""
    rq, res, _ = mix
    bres, s = serve(rq, slots=2, max_batch=4)
    assert s.batches > 0
    assert [r.status for r in bres] == [KRR_OK] * len(rq)
    for r, a, b in zip(rq, res, bres):
        assert np.array_equal(a.yhat, b.yhat), "request %d differs packed vs on its own" % r.rid
