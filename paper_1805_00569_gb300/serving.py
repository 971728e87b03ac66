"""Serving form of the KRR hot path: a request loop with continuous admission.

Requests (fit + predict of one KRR problem, or predict-only against a model
kept resident from an earlier fit) arrive over time.  A dispatcher admits the
oldest waiting request as soon as a worker slot is free and the HBM budget
holds its estimated footprint; each slot owns a CUDA stream and a libkrr
context, so requests admitted while others are running overlap on the device.
Fitted models stay resident (least recently used evicted first) so repeat
predictions run only the fused predict kernel.  Each request's work depends
only on its own inputs and every kernel reduces in a fixed order, so a result
is bit-identical whether the request runs alone or in a mix.

The scheduling core (``Scheduler``) takes an executor callable and knows
nothing about GPUs; ``GpuExecutor`` is the libkrr executor.
"""
from __future__ import annotations

import collections
import heapq
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import KRR_ERR_BUDGET, KRR_ERR_CUDA, KRR_OK

TILE = 128


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds from the start of the stream
    key: str                       # identity of the training data (resident-model cache key)
    n: int
    d: int
    sigma: float
    lam: float
    predict_only: bool = False
    payload: dict = field(default_factory=dict)   # X, y, Xt (numpy) as needed


@dataclass
class Result:
    rid: int
    arrival: float
    start: float
    done: float
    yhat: np.ndarray | None
    status: int
    resident_hit: bool
    error: str | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def fit_footprint_bytes(n: int, d: int, t: int) -> int:
    """Device bytes one single-partition fit + predict needs at its peak
    (kernel store hi/lo, factor, inverses, refinement vectors and slots, the
    gathered rows and their slices, the test rows): mirrors libkrr's own
    allocation for p = 1, one sigma, one lambda."""
    T = (n + TILE - 1) // TILE
    tiles = T * (T + 1) // 2
    tile_b = TILE * TILE * 4
    rows = T * TILE
    dp = (d + 15) // 16 * 16
    dz = (d + 31) // 32 * 32
    # kernel store hi/lo, factor, FP16 factor copy, lo parts of a three-pass
    # factor, diagonal inverses, refinement vectors, matvec slots, row sums
    work = (2 * tiles * tile_b + tiles * tile_b + tiles * TILE * TILE * 2 + tiles * tile_b + T * tile_b
            + 7 * rows * 8 + T * T * TILE * 8 + T * T * 9 * TILE * 4)
    model = rows * d * 8 + 2 * rows * dp * 4 + rows * 8 + rows * 8 + rows * (10 * dz + 4)
    test = t * d * 8 + (t + 256) * (10 * dz + 12) + t * 8
    return int(work + model + test + (64 << 20))


def model_bytes(n: int, d: int) -> int:
    T = (n + TILE - 1) // TILE
    rows = T * TILE
    dp = (d + 15) // 16 * 16
    dz = (d + 31) // 32 * 32
    return int(rows * d * 8 + 2 * rows * dp * 4 + 2 * rows * 8 + rows * (10 * dz + 4))


class Scheduler:
    """Continuous admission of requests into `slots` workers under an HBM
    budget.  `execute(slot, request) -> (yhat, status, resident_hit)` runs a
    request on a slot; `resident(request) -> bool` says whether a predict-only
    request's model is resident (its footprint is then only the test rows);
    `reserved() -> bytes` is memory held outside running requests (resident
    models), charged against the budget too.  Admission is first come, first
    served: a request that does not fit yet blocks the ones behind it, so a
    large request is never starved by a run of small ones."""

    def __init__(self, execute, slots: int, budget_bytes: int, resident=None, t_rows: int = 256,
                 clock=time.perf_counter, reserved=None):
        self.execute = execute
        self.reserved = reserved or (lambda: 0)
        self.slots = slots
        self.budget = budget_bytes
        self.resident = resident or (lambda r: False)
        self.t_rows = t_rows
        self.clock = clock
        self.lock = threading.Condition()
        self.free_slots = list(range(slots))
        self.in_use = 0
        self.peak_in_use = 0
        self.peak_concurrency = 0
        self.active = 0
        self.results: list[Result] = []

    def footprint(self, r: Request) -> int:
        if r.predict_only and self.resident(r):
            return self.t_rows * r.d * 8 * 3 + (16 << 20)
        return fit_footprint_bytes(r.n, r.d, self.t_rows)

    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Replay `requests` (sorted by arrival).  realtime: wait for each
        arrival time; otherwise every request is queued at the start (its
        latency then counts from the start)."""
        t0 = self.clock()
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting: list[tuple[float, int, Request]] = []
        threads = []

        def worker(slot: int, req: Request, need: int, start: float):
            err = None
            try:
                yhat, status, hit = self.execute(slot, req)
            except Exception as e:  # a failed request frees its slot and reports its status
                yhat, status, hit, err = None, getattr(e, "status", KRR_ERR_CUDA), False, repr(e)
            done = self.clock() - t0
            with self.lock:
                self.results.append(Result(req.rid, req.arrival if realtime else 0.0, start, done, yhat, status,
                                           hit, err))
                self.in_use -= need
                self.active -= 1
                self.free_slots.append(slot)
                self.lock.notify_all()

        while pending or waiting:
            now = self.clock() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                heapq.heappush(waiting, (r.arrival, r.rid, r))
            with self.lock:
                while waiting:
                    req = waiting[0][2]
                    need = self.footprint(req)
                    if need > self.budget:  # can never fit: reject
                        heapq.heappop(waiting)
                        self.results.append(Result(req.rid, req.arrival if realtime else 0.0, now, now, None,
                                                   KRR_ERR_BUDGET, False))
                        continue
                    if not self.free_slots or self.in_use + self.reserved() + need > self.budget:
                        break
                    heapq.heappop(waiting)
                    slot = self.free_slots.pop()
                    self.in_use += need
                    self.peak_in_use = max(self.peak_in_use, self.in_use + self.reserved())
                    self.active += 1
                    self.peak_concurrency = max(self.peak_concurrency, self.active)
                    th = threading.Thread(target=worker, args=(slot, req, need, self.clock() - t0), daemon=True)
                    threads.append(th)
                    th.start()
                if pending and realtime:
                    timeout = max(0.0, pending[0].arrival - (self.clock() - t0))
                    self.lock.wait(timeout=min(timeout, 0.05))
                elif waiting:
                    self.lock.wait(timeout=0.05)
        for th in threads:
            th.join()
        return sorted(self.results, key=lambda r: r.rid)


def latency_summary(results: list[Result]) -> dict:
    lat = np.array([r.latency for r in results if r.status == KRR_OK])
    failed = collections.Counter(int(r.status) for r in results if r.status != KRR_OK)
    errors = sorted({r.error for r in results if r.error})[:3]
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "completed": 0, "failed": dict(failed), "errors": errors}
    span = max(r.done for r in results) - min(r.arrival for r in results)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "completed": int(lat.size),
            "requests_per_s": float(lat.size / span) if span > 0 else None,
            "failed": dict(failed), "errors": errors}


class GpuExecutor:
    """libkrr executor: one CUDA stream and context per slot.  The scheduler
    runs at most one request per slot at a time, so each context is only ever
    called from one thread at a time.  Fitted models stay resident in an LRU
    cache bounded by `resident_bytes`; a predict-only request uses the
    resident model from its own slot's context (a model may be read by any
    context on its device once its fit has completed).  An evicted model is
    freed later by its owning slot, and never while a request holds it."""

    def __init__(self, slots: int, prec: str = "tf32", device: int = 0, resident_bytes: int = 8 << 30,
                 panel_width: int = 8):
        import torch

        import paper_1805_00569_gb300 as K
        self.K = K
        self.torch = torch
        self.prec = prec
        self.device = device
        torch.cuda.set_device(device)
        self.streams = [torch.cuda.Stream(device) for _ in range(slots)]
        self.ctx = [K.krr_ctx_create(device, s) for s in self.streams]
        for c in self.ctx:  # a fixed panel width: the factor's bits do not depend on timing
            K.krr_ctx_set_panel_width(c, panel_width)
        self.cache: collections.OrderedDict[str, list] = collections.OrderedDict()  # key -> [model, owner, bytes, pins]
        self.cache_bytes = 0
        self.resident_limit = resident_bytes
        self.to_free: list[list] = [[] for _ in range(slots)]
        self.lock = threading.Lock()

    def is_resident(self, r: Request) -> bool:
        with self.lock:
            return r.key in self.cache

    def resident_bytes(self) -> int:
        with self.lock:
            return self.cache_bytes + sum(m[2] for lst in self.to_free for m in lst)

    def _evict_locked(self):
        for key in list(self.cache.keys()):
            if self.cache_bytes <= self.resident_limit:
                break
            ent = self.cache[key]
            if ent[3] > 0:
                continue
            del self.cache[key]
            self.cache_bytes -= ent[2]
            self.to_free[ent[1]].append(ent)

    def _free_pending(self, slot: int):
        with self.lock:
            lst, self.to_free[slot] = self.to_free[slot], []
        for ent in lst:
            self.K.krr_model_free(self.ctx[slot], ent[0])

    def __call__(self, slot: int, r: Request):
        torch, K = self.torch, self.K
        stream = self.streams[slot]
        ctx = self.ctx[slot]
        self._free_pending(slot)
        with torch.cuda.stream(stream):
            Xt = torch.from_numpy(np.ascontiguousarray(r.payload["Xt"])).to("cuda")
            if r.predict_only:
                with self.lock:
                    ent = self.cache.get(r.key)
                    if ent is not None:
                        self.cache.move_to_end(r.key)
                        ent[3] += 1
                if ent is not None:
                    try:
                        out = K.krr_predict(ctx, ent[0], Xt).cpu().numpy()[0]
                        stream.synchronize()
                    finally:
                        with self.lock:
                            ent[3] -= 1
                    return out, KRR_OK, True
                if "X" not in r.payload:  # evicted and no training data with the request
                    return None, KRR_ERR_BUDGET, False
            X = torch.from_numpy(np.ascontiguousarray(r.payload["X"])).to("cuda")
            y = torch.from_numpy(np.ascontiguousarray(r.payload["y"])).to("cuda")
            n = X.shape[0]
            perm = torch.arange(n, dtype=torch.int64, device="cuda")
            offsets = torch.tensor([0, n], dtype=torch.int64, device="cuda")
            model, status, _ = K.krr_fit_batch(ctx, X, y, perm, offsets, [r.sigma], [r.lam], self.prec)
            out = K.krr_predict(ctx, model, Xt).cpu().numpy()[0]
            st = int(status.cpu()[0])
            stream.synchronize()
        with self.lock:
            old = self.cache.pop(r.key, None)
            if old is not None:
                self.cache_bytes -= old[2]
                self.to_free[old[1]].append(old)
            self.cache[r.key] = [model, slot, model_bytes(r.n, r.d), 0]
            self.cache_bytes += model_bytes(r.n, r.d)
            self._evict_locked()
        return out, st, False

    def close(self):
        with self.lock:
            for ent in self.cache.values():
                self.to_free[ent[1]].append(ent)
            self.cache.clear()
            self.cache_bytes = 0
        for s in range(len(self.ctx)):
            self._free_pending(s)
        for s in self.streams:
            s.synchronize()
        for c in self.ctx:
            c.close()


def make_stream_requests(stream: dict, count: int, data_fn, t: int = 256, bank: int = 0) -> list[Request]:
    """Requests from a synthetic serving stream (arrival times and shapes);
    `data_fn(seed, n, d, t)` returns X, y, Xt and the mixture's parameters.  A
    repeat request predicts new test rows, drawn from the mixture of an
    earlier request, with that request's model; it carries that request's
    training rows too, so it refits if the model has been evicted.

    bank > 0: instead of one data set per request, `bank` mixtures per
    feature count are drawn once at the stream's largest n, and a request
    takes the first n (shuffled) rows of the one its data seed picks -- the
    same shapes, sigma, lambda and arrivals, without drawing gigabytes of rows
    for a long stream."""
    from .synth import serve_repeat_rows
    reqs = []
    fitted = []
    n_max = int(max(stream["n"][:count])) if count else 0
    banked: dict = {}
    for i in range(count):
        if stream["repeat"][i] and fitted:
            j = fitted[(i * 7919) % len(fitted)]
            base = reqs[j]
            Xt = serve_repeat_rows(base.payload["mix"], int(stream["data_seed"][i]), t)
            reqs.append(Request(i, float(stream["arrival"][i]), base.key, base.n, base.d, base.sigma, base.lam,
                                True, {"X": base.payload["X"], "y": base.payload["y"], "Xt": Xt}))
            continue
        n, d = int(stream["n"][i]), int(stream["d"][i])
        if bank > 0:
            b = int(stream["data_seed"][i] % bank)
            if (d, b) not in banked:
                banked[(d, b)] = data_fn(1000003 * d + b, n_max, d, t)
            src = banked[(d, b)]
            data = dict(X=src["X"][:n], y=src["y"][:n], Xt=src["Xt"], yt=src["yt"], mix=src["mix"])
        else:
            data = data_fn(int(stream["data_seed"][i]), n, d, t)
        reqs.append(Request(i, float(stream["arrival"][i]), "req%d" % i, n, d, float(stream["sigma"][i]),
                            float(stream["lam"][i]), False, data))
        fitted.append(i)
    return reqs
