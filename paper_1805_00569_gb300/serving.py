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
    model = rows * d * 8 + 2 * rows * dp * 4 + rows * 8 + rows * 16 + rows * (10 * dz + 4)
    test = t * d * 8 + (t + 256) * (10 * dz + 12) + t * 8
    return int(work + model + test + (64 << 20))


def model_bytes(n: int, d: int) -> int:
    T = (n + TILE - 1) // TILE
    rows = T * TILE
    dp = (d + 15) // 16 * 16
    dz = (d + 31) // 32 * 32
    return int(rows * d * 8 + 2 * rows * dp * 4 + 3 * rows * 8 + rows * (10 * dz + 4))


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
                 clock=time.perf_counter, reserved=None, max_batch: int = 1):
        self.execute = execute
        # max_batch > 1: the oldest waiting fit takes later waiting fits with
        # the same feature count into the same slot, run as one packed fit by
        # execute.batch(slot, requests) -> [(yhat, status, resident_hit)]
        self.max_batch = max_batch if hasattr(execute, "batch") else 1
        self.batches = 0
        self.batched_requests = 0
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

        def worker(slot: int, batch: list, need: int, start: float):
            outs = None
            err = None
            try:
                if len(batch) == 1 and self.max_batch == 1:
                    outs = [self.execute(slot, batch[0])]
                else:
                    outs = self.execute.batch(slot, batch)
            except Exception as e:  # a failed request frees its slot and reports its status
                err = repr(e)
                outs = [(None, getattr(e, "status", KRR_ERR_CUDA), False)] * len(batch)
            done = self.clock() - t0
            with self.lock:
                for req, (yhat, status, hit) in zip(batch, outs):
                    self.results.append(Result(req.rid, req.arrival if realtime else 0.0, start, done, yhat, status,
                                               hit, err))
                self.in_use -= need
                self.active -= len(batch)
                self.free_slots.append(slot)
                self.lock.notify_all()

        def batchable(r: Request) -> bool:  # a fit (a predict-only request whose model is gone refits)
            return not (r.predict_only and self.resident(r))

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
                    batch = [req]
                    if self.max_batch > 1 and batchable(req):
                        keep = []
                        for item in sorted(waiting):
                            r2 = item[2]
                            if (len(batch) < self.max_batch and r2.d == req.d and batchable(r2)
                                    and self.footprint(r2) + need + self.in_use + self.reserved() <= self.budget):
                                batch.append(r2)
                                need += self.footprint(r2)
                            else:
                                keep.append(item)
                        waiting[:] = keep
                        heapq.heapify(waiting)
                        if len(batch) > 1:
                            self.batches += 1
                            self.batched_requests += len(batch)
                    slot = self.free_slots.pop()
                    self.in_use += need
                    self.peak_in_use = max(self.peak_in_use, self.in_use + self.reserved())
                    self.active += len(batch)
                    self.peak_concurrency = max(self.peak_concurrency, self.active)
                    th = threading.Thread(target=worker, args=(slot, batch, need, self.clock() - t0), daemon=True)
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


class _Shared:
    """A fitted model held by one or more resident-cache entries (a packed
    fit holds every request of its batch); freed by its owning slot once the
    last entry is evicted."""

    def __init__(self, model, owner: int, refs: int):
        self.model, self.owner, self.refs = model, owner, refs
        self.bytes = 0  # device bytes of all its requests' models


class GpuExecutor:
    """libkrr executor: one CUDA stream and context per slot.  The scheduler
    runs at most one request (or one packed batch) per slot at a time, so each
    context is only ever called from one thread at a time.  Fitted models stay
    resident in an LRU cache bounded by `resident_bytes`; a predict-only
    request uses the resident model from its own slot's context (a model may
    be read by any context on its device once its fit has completed).  An
    evicted model is freed later by its owning slot, and never while a request
    holds it.  `batch` runs several waiting fits of the same feature count as
    one krr_fit_jobs call (one problem per partition, each with its own sigma
    and lambda) and one routed prediction."""

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
        # key -> [shared model, partition (None: the whole model is the request's), bytes, pins]
        self.cache: collections.OrderedDict[str, list] = collections.OrderedDict()
        self.cache_bytes = 0
        self.resident_limit = resident_bytes
        self.to_free: list[list] = [[] for _ in range(slots)]
        self.live: set = set()  # shared models not freed yet (cached or waiting for their owner)
        self.lock = threading.Lock()

    def is_resident(self, r: Request) -> bool:
        with self.lock:
            return r.key in self.cache

    def resident_bytes(self) -> int:
        with self.lock:
            return sum(sh.bytes for sh in self.live)

    def _drop_locked(self, ent):
        self.cache_bytes -= ent[2]
        sh = ent[0]
        sh.refs -= 1
        if sh.refs == 0:
            self.to_free[sh.owner].append(sh)

    def _evict_locked(self):
        for key in list(self.cache.keys()):
            if self.cache_bytes <= self.resident_limit:
                break
            ent = self.cache[key]
            if ent[3] > 0:
                continue
            del self.cache[key]
            self._drop_locked(ent)

    def _free_pending(self, slot: int):
        with self.lock:
            lst, self.to_free[slot] = self.to_free[slot], []
        for sh in lst:
            self.K.krr_model_free(self.ctx[slot], sh.model)
            with self.lock:
                self.live.discard(sh)

    def _insert(self, r: Request, sh: _Shared, part):
        with self.lock:
            old = self.cache.pop(r.key, None)
            if old is not None:
                self._drop_locked(old)
            self.cache[r.key] = [sh, part, model_bytes(r.n, r.d), 0]
            self.cache_bytes += model_bytes(r.n, r.d)
            sh.bytes += model_bytes(r.n, r.d)
            self.live.add(sh)
            self._evict_locked()

    def _predict_resident(self, slot: int, r: Request, Xt):
        """yhat of a predict-only request from its resident model, or None."""
        K, torch = self.K, self.torch
        with self.lock:
            ent = self.cache.get(r.key)
            if ent is not None:
                self.cache.move_to_end(r.key)
                ent[3] += 1
        if ent is None:
            return None
        try:
            if ent[1] is None:
                out = K.krr_predict(self.ctx[slot], ent[0].model, Xt).cpu().numpy()[0]
            else:
                route = torch.full((Xt.shape[0],), int(ent[1]), dtype=torch.int32, device="cuda")
                out = K.krr_predict(self.ctx[slot], ent[0].model, Xt, route=route).cpu().numpy()[0]
            self.streams[slot].synchronize()
        finally:
            with self.lock:
                ent[3] -= 1
        return out

    def __call__(self, slot: int, r: Request):
        torch, K = self.torch, self.K
        stream = self.streams[slot]
        ctx = self.ctx[slot]
        self._free_pending(slot)
        with torch.cuda.stream(stream):
            Xt = torch.from_numpy(np.ascontiguousarray(r.payload["Xt"])).to("cuda")
            if r.predict_only:
                out = self._predict_resident(slot, r, Xt)
                if out is not None:
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
        self._insert(r, _Shared(model, slot, 1), None)
        return out, st, False

    def batch(self, slot: int, reqs: list):
        """Several fits of one feature count in one packed fit and one routed
        prediction; a predict-only request whose model is resident is served
        from it (the scheduler only batches it when its model was evicted)."""
        torch, K = self.torch, self.K
        stream = self.streams[slot]
        ctx = self.ctx[slot]
        self._free_pending(slot)
        outs = [None] * len(reqs)
        fits = []
        with torch.cuda.stream(stream):
            for i, r in enumerate(reqs):
                if r.predict_only:
                    Xt = torch.from_numpy(np.ascontiguousarray(r.payload["Xt"])).to("cuda")
                    out = self._predict_resident(slot, r, Xt)
                    if out is not None:
                        outs[i] = (out, KRR_OK, True)
                        continue
                    if "X" not in r.payload:
                        outs[i] = (None, KRR_ERR_BUDGET, False)
                        continue
                fits.append(i)
            if fits:
                sizes = [reqs[i].payload["X"].shape[0] for i in fits]
                tsz = [reqs[i].payload["Xt"].shape[0] for i in fits]
                X = torch.from_numpy(np.ascontiguousarray(np.concatenate([reqs[i].payload["X"] for i in fits]))).to(
                    "cuda")
                y = torch.from_numpy(np.ascontiguousarray(np.concatenate([reqs[i].payload["y"] for i in fits]))).to(
                    "cuda")
                Xt = torch.from_numpy(np.ascontiguousarray(np.concatenate([reqs[i].payload["Xt"] for i in fits]))).to(
                    "cuda")
                off = torch.tensor(np.concatenate([[0], np.cumsum(sizes)]), dtype=torch.int64, device="cuda")
                perm = torch.arange(X.shape[0], dtype=torch.int64, device="cuda")
                route = torch.tensor(np.repeat(np.arange(len(fits)), tsz), dtype=torch.int32, device="cuda")
                model, status, _ = K.krr_fit_jobs(ctx, X, y, perm, off, [reqs[i].sigma for i in fits],
                                                  [reqs[i].lam for i in fits], self.prec)
                yh = K.krr_predict(ctx, model, Xt, route=route).cpu().numpy()[0]
                st = status.cpu().numpy()
                stream.synchronize()
                sh = _Shared(model, slot, len(fits))
                pos = np.concatenate([[0], np.cumsum(tsz)])
                for k, i in enumerate(fits):
                    outs[i] = (yh[pos[k]:pos[k + 1]].copy(), int(st[k]), False)
                    self._insert(reqs[i], sh, k)
        return outs

    def close(self):
        with self.lock:
            for ent in list(self.cache.values()):
                self._drop_locked(ent)
            self.cache.clear()
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
