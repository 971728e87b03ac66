"""Host logic of the serving loop: admission by slots and HBM budget, first
come first served order, rejection of requests that can never fit, failure
isolation, resident-model footprints and the latency summary.  A fake executor
stands in for the device, so this runs without a GPU."""
import threading
import time

import numpy as np

from paper_1805_00569_gb300 import KRR_ERR_BUDGET, KRR_ERR_NOT_SPD, KRR_OK, synth
from paper_1805_00569_gb300.serving import (Request, Scheduler, fit_footprint_bytes, latency_summary,
                                            make_stream_requests, model_bytes)


class FakeExec:
    """Sleeps in proportion to n and records the live footprint sum."""

    def __init__(self, sched_ref, fail_rids=()):
        self.sched_ref = sched_ref
        self.lock = threading.Lock()
        self.live = 0
        self.max_live = 0
        self.max_bytes = 0
        self.order = []
        self.fail = set(fail_rids)

    def __call__(self, slot, r):
        s = self.sched_ref[0]
        with self.lock:
            self.live += 1
            self.max_live = max(self.max_live, self.live)
            self.max_bytes = max(self.max_bytes, s.in_use)
            self.order.append(r.rid)
        try:
            time.sleep(0.002 + r.n * 2e-7)
            if r.rid in self.fail:
                raise RuntimeError("injected failure")
            return np.full(4, float(r.rid)), KRR_OK, False
        finally:
            with self.lock:
                self.live -= 1


def reqs(ns, d=32, arrival_gap=0.0):
    return [Request(i, i * arrival_gap, "k%d" % i, n, d, 1.0, 1e-4) for i, n in enumerate(ns)]


def run(ns, slots, budget, fail=(), realtime=False, gap=0.0):
    ref = [None]
    ex = FakeExec(ref, fail)
    s = Scheduler(ex, slots, budget)
    ref[0] = s
    res = s.run(reqs(ns, arrival_gap=gap), realtime=realtime)
    return s, ex, res


def test_slots_bound_concurrency():
    s, ex, res = run([1000] * 24, slots=3, budget=1 << 50)
    assert len(res) == 24 and all(r.status == KRR_OK for r in res)
    assert ex.max_live <= 3 and s.peak_concurrency == 3


def test_budget_bounds_bytes_in_use():
    one = fit_footprint_bytes(8000, 32, 256)
    s, ex, res = run([8000] * 10, slots=8, budget=int(2.5 * one))
    assert all(r.status == KRR_OK for r in res)
    assert s.peak_in_use <= 2.5 * one and s.peak_concurrency == 2 and ex.max_live <= 2


def test_fcfs_large_request_not_starved():
    # a request that fits only alone waits for the running ones, and those
    # behind it wait for it: starts follow arrival order
    one = fit_footprint_bytes(2000, 32, 256)
    big = fit_footprint_bytes(16000, 32, 256)
    ns = [2000, 2000, 16000, 2000, 2000, 2000]
    s, ex, res = run(ns, slots=4, budget=big + one // 2)
    assert ex.order == list(range(len(ns)))
    starts = [r.start for r in res]
    assert starts[3] >= res[2].start


def test_oversized_rejected_others_served():
    small = fit_footprint_bytes(1000, 32, 256)
    s, ex, res = run([1000, 200000, 1000], slots=2, budget=3 * small)
    assert [r.status for r in res] == [KRR_OK, KRR_ERR_BUDGET, KRR_OK]
    assert 1 not in ex.order


def test_failure_frees_slot():
    s, ex, res = run([500] * 6, slots=1, budget=1 << 50, fail=(2,))
    st = [r.status for r in res]
    assert st[2] != KRR_OK and st.count(KRR_OK) == 5
    assert s.in_use == 0 and s.active == 0 and len(s.free_slots) == 1


def test_resident_predict_footprint_and_reserved():
    calls = []
    s = Scheduler(lambda slot, r: (None, KRR_OK, True), 2, 1 << 40, resident=lambda r: True,
                  reserved=lambda: calls.append(1) or 123)
    r_fit = Request(0, 0.0, "a", 16384, 90, 1.0, 1e-4)
    r_pred = Request(1, 0.0, "a", 16384, 90, 1.0, 1e-4, predict_only=True)
    assert s.footprint(r_pred) < s.footprint(r_fit) // 50
    s.run([r_fit, r_pred], realtime=False)
    assert calls  # reserved bytes consulted at admission


def test_realtime_arrivals_respected():
    s, ex, res = run([200] * 5, slots=5, budget=1 << 50, realtime=True, gap=0.02)
    for r in res:
        assert r.start + 1e-3 >= r.arrival
    assert res[-1].start >= 0.08 - 1e-3


def test_latency_summary_and_status_filter():
    from paper_1805_00569_gb300.serving import Result
    rs = [Result(i, 0.0, 0.0, (i + 1) * 1e-3, None, KRR_OK, False) for i in range(100)]
    rs.append(Result(100, 0.0, 0.0, 5.0, None, KRR_ERR_NOT_SPD, False))
    out = latency_summary(rs)
    assert out["completed"] == 100
    assert abs(out["p50_ms"] - 50.5) < 1e-9 and abs(out["p99_ms"] - 99.01) < 1e-9


def test_footprint_monotone_and_model_bytes():
    prev = 0
    for n in (1, 128, 129, 1000, 4096, 16384):  # grows with the tile count (1, 1, 2, 8, 32, 128)
        f = fit_footprint_bytes(n, 90, 256)
        assert f >= prev and (n == 128) == (f == prev)
        prev = f
        assert model_bytes(n, 90) < f
    # kernel store of a 16384-row request: 2 * 8256 tiles of 64 KiB dominate
    assert fit_footprint_bytes(16384, 90, 256) > 2 * 8256 * 65536


def test_stream_requests_shapes_and_repeats():
    st = synth.serve_stream(seed=4, requests=60)
    rq = make_stream_requests(st, 60, lambda seed, n, d, t: synth.serve_request_data(seed, n, d, t), t=16)
    assert len(rq) == 60
    fits = {r.key: r for r in rq if not r.predict_only}
    for r in rq:
        assert 512 <= r.n <= 16384 and r.d in (8, 32, 90)
        assert r.payload["Xt"].shape == (16, r.d)
        if r.predict_only:
            b = fits[r.key]
            assert b.rid < r.rid and r.payload["X"] is b.payload["X"]
    assert any(r.predict_only for r in rq)
    assert np.all(np.diff([r.arrival for r in rq]) > 0)


class FakeBatchExec(FakeExec):
    """FakeExec with a packed-batch entry point that records each batch."""

    def __init__(self, sched_ref):
        super().__init__(sched_ref)
        self.batches = []

    def batch(self, slot, rs):
        with self.lock:
            self.batches.append([(r.rid, r.d) for r in rs])
        time.sleep(0.002)
        return [(np.full(4, float(r.rid)), KRR_OK, False) for r in rs]


def test_batches_pack_waiting_fits_of_one_feature_count():
    ds = [8, 32, 8, 90, 8, 32, 8, 8, 32, 90, 8, 8]
    rq = [Request(i, 0.0, "k%d" % i, 500 + 10 * i, d, 1.0, 1e-4) for i, d in enumerate(ds)]
    ref = [None]
    ex = FakeBatchExec(ref)
    s = Scheduler(ex, 1, 1 << 50, max_batch=3)
    ref[0] = s
    res = s.run(rq, realtime=False)
    assert sorted(r.rid for r in res) == list(range(len(ds))) and all(r.status == KRR_OK for r in res)
    assert all(np.array_equal(r.yhat, np.full(4, float(r.rid))) for r in res)
    seen = []
    for b in ex.batches:
        assert 1 <= len(b) <= 3 and len({d for _, d in b}) == 1
        # the oldest request not yet served leads every batch
        assert b[0][0] == min(rid for rid in range(len(ds)) if rid not in seen)
        seen += [rid for rid, _ in b]
    assert sorted(seen) == list(range(len(ds)))
    assert s.batches >= 3 and s.batched_requests >= 7


def test_batches_respect_the_budget():
    fp = fit_footprint_bytes(4000, 32, 256)
    rq = [Request(i, 0.0, "k%d" % i, 4000, 32, 1.0, 1e-4) for i in range(6)]
    ref = [None]
    ex = FakeBatchExec(ref)
    s = Scheduler(ex, 2, 2 * fp + fp // 2, max_batch=4)
    ref[0] = s
    res = s.run(rq, realtime=False)
    assert all(r.status == KRR_OK for r in res) and len(res) == 6
    assert all(len(b) <= 2 for b in ex.batches)
    assert s.peak_in_use <= 2 * fp + fp // 2
