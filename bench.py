"""Benchmark of the BKRR2 hot path on GB300: partition-solves per second.

One step = one pass of the whole hot path over one synthetic BKRR2 workload
(n = 65536 training and 8192 test rows, d = 90, p = 16 random equal
partitions, sigma in {1, 4, 16} x lambda in {1e-6, 1e-4}): random partition,
kernel build + TF32-factor Cholesky + FP64-level refinement of all 96
(partition, sigma, lambda) solves, all-model prediction of the 8192 test rows,
best-model selection.  Inputs are resident in HBM when a timed step starts;
L2 is flushed (512 MB write) before every timed step.  `e2e` repeats the
measurement through the same public calls with the inputs copied from pinned
host memory each step and the chosen model read back.

The default run also replays the serving stream (10000 fit + predict
requests, Poisson 200/s) through the serving loop and adds its latency and
capacity as the line's `serve` object.

Multi-GPU (torchrun): weak scaling -- one BKRR2 workload N times the one-GPU
size (N x 65536 training rows, N x 16 partitions, the same 8192 test rows),
identical on every rank; each rank fits the partitions LPT gives it and
predicts every test row with its models, and one all-gather of the scores
picks the global best model (kkrr2: the K-means block sums are exchanged every
round as well).  `--impl reference` times the FP64 CPU oracle on a bounded
sample of the same workload (it is the deliberately slow reference).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "KRR partition-solves/s & TFLOP/s vs plain FP64 at ≤1e-6 rel err; serve p50/p99"
UNIT = "partition-solves/s"
# arithmetic the path computes in, per factor precision: the factor's tensor-core
# passes, then refinement with double-float (~44-bit) kernel entries and FP64 vectors
DTYPE_LABEL = {"tf32": "fp16 1-pass / tf32x3 factor + df64 refinement",
               "bf16x3": "bf16x3 / tf32x3 factor + df64 refinement",
               "fp32": "tf32x3 factor + df64 refinement", "fp64": "f64"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="tf32", choices=["tf32", "bf16x3", "fp32", "fp64"])
    ap.add_argument("--panel", type=int, default=0, help="Cholesky outer panel width (0 = library default)")
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle solves in the CPU baseline (0 = auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true")
    ap.add_argument("--profile", action="store_true", help="print per-kernel-class times to stderr")
    ap.add_argument("--workload", default="bkrr2", choices=["bkrr2", "kkrr2", "bkrr2kb", "sweep", "dkrr", "serve"],
                    help="bkrr2: the headline configuration; kkrr2: K-means partitions (uneven, routed); "
                         "bkrr2kb: the bkrr2 data with K-balance partitions (routed); "
                         "sweep: 520000 rows, p = 128; dkrr: one partition of 2048 rows; serve: the request "
                         "stream (Poisson 200/s, n log-uniform in [512, 16384]) through the serving loop")
    ap.add_argument("--requests", type=int, default=10000, help="serve: requests replayed from the stream")
    ap.add_argument("--shard", action="store_true",
                    help="bkrr2/kkrr2: take the multi-GPU (LPT-sharded) step even on one GPU")
    ap.add_argument("--no-serve", action="store_true",
                    help="bkrr2 line without its serve object (the request stream through the serving loop)")
    ap.add_argument("--serve-batch", type=int, default=8,
                    help="serve: waiting fits of one feature count packed into one krr_fit_jobs call (1 = off)")
    ap.add_argument("--serve-bank", type=int, default=32,
                    help="serve: mixtures drawn per feature count; requests take row prefixes (0 = one per request)")
    ap.add_argument("--slots", type=int, default=16, help="serve: concurrent requests (one stream each)")
    ap.add_argument("--fp64-sample", type=int, default=24, help="serve: requests in the sequential FP64 sample")
    ap.add_argument("--precisions", default="",
                    help="comma list (fp64,fp32,tf32,bf16x3): time the workload once per factor precision and "
                         "report each in the line's precision_sweep object")
    ap.add_argument("--n", type=int, default=0, help="training rows (0 = the workload's; smaller: profiling cases)")
    ap.add_argument("--t", type=int, default=0, help="test rows (0 = the workload's)")
    ap.add_argument("--p", type=int, default=0, help="partitions (0 = the workload's)")
    return ap.parse_args()


# ---------------------------------------------------------------- CPU oracle sample
def _oracle_solve(args):
    """One full partition-solve pipeline of the oracle (kernel build, Cholesky,
    refinement, prediction of every test row, MSE)."""
    Xp, yp, Xt, yt, sigma, lam = args
    import oracle
    t0 = time.perf_counter()
    a, info, rc = oracle.fit(Xp, yp, sigma, lam)
    yh = oracle.predict(Xp, a, Xt, sigma)
    m = oracle.mse(yh, yt)
    return time.perf_counter() - t0, m, a, yh, float(info[0])


def sample_models(p: int, G: int, count: int):
    """(partition, grid point) of the solves the oracle recomputes: every
    partition in turn, grid points spread over the sigma x lambda grid."""
    return [(k % p, (k * 5 + 2) % G) for k in range(count)]


def _oracle_jobs(w, perm, offsets, count):
    jobs = []
    G = len(w["sigmas"]) * len(w["lambdas"])
    for j, g in sample_models(len(offsets) - 1, G, count):
        si, li = divmod(g, len(w["lambdas"]))
        rows = perm[offsets[j]:offsets[j + 1]]
        jobs.append((w["X"][rows], w["y"][rows], w["Xt"], w["yt"], w["sigmas"][si], w["lambdas"][li]))
    return jobs


def host_cpu(cpuinfo: str = "/proc/cpuinfo") -> dict:
    """nproc and the CPU model of the host that runs the oracle (the model
    name on x86, implementer and part codes on Arm)."""
    info = {"nproc": os.cpu_count(), "machine": platform.machine()}
    try:
        keys = {}
        with open(cpuinfo) as f:
            for line in f:
                k, _, v = line.partition(":")
                k, v = k.strip(), v.strip()
                if k in ("model name", "CPU implementer", "CPU part") and k not in keys:
                    keys[k] = v
        if "model name" in keys:
            info["model"] = keys["model name"]
        elif "CPU part" in keys:
            info["model"] = "implementer %s part %s" % (keys.get("CPU implementer", "?"), keys["CPU part"])
    except (OSError, UnicodeDecodeError):
        pass
    return info


def cpu_baseline(w, sample: int):
    import oracle
    oracle.build()
    perm, offsets, _ = oracle.partition_random(w["X"].shape[0], w["p"], w["part_seed"])
    jobs = _oracle_jobs(w, perm, offsets, sample)
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(processes=sample) as pool:
        res = pool.map(_oracle_solve, jobs)
    wall = time.perf_counter() - t0
    out = dict(value=sample / wall, unit=UNIT, cores=sample, kind="oracle", host=host_cpu(),
               sample="%d of the %d (partition, sigma, lambda) solves of %s, one process each: kernel build + "
                      "Cholesky + long-double refinement + prediction of all %d test rows + MSE; %.1f s wall"
                      % (sample, w["p"] * len(w["sigmas"]) * len(w["lambdas"]), w["workload"],
                         w["Xt"].shape[0], wall))
    refs = [dict(alpha=r[2], yhat=r[3], mse=r[1], kappa=r[4]) for r in res]
    return out, refs


def rel_err(a, b) -> float:
    """Max-norm relative error of a result vector against the oracle's."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = float(np.max(np.abs(b))) if b.size else 0.0
    num = float(np.max(np.abs(a - b))) if b.size else 0.0
    return num / den if den > 0 else num


def accuracy_vs_oracle(gpu: dict, refs: list, pairs: list) -> dict:
    """Per factor precision: the largest relative error of alpha, of the
    predictions of every test row and of the MSE over the sampled solves."""
    out = {}
    for prec, got in gpu.items():
        ea, ep, em = [], [], []
        for (jg, ref) in zip(pairs, refs):
            a, yh, m = got[jg]
            ea.append(rel_err(a, ref["alpha"]))
            ep.append(rel_err(yh, ref["yhat"]))
            em.append(abs(m - ref["mse"]) / ref["mse"])
        worst = int(np.argmax(ea))
        out[prec] = {"max_rel_err_alpha": max(ea), "max_rel_err_pred": max(ep), "max_rel_err_mse": max(em),
                     "worst_alpha_model": list(pairs[worst]),
                     "worst_alpha_kappa": refs[worst]["kappa"],
                     "failed_solves": got["failed"]}
    return out


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons; the summary keeps
    the samples taken inside the timed window (window(t0, t1), perf_counter
    times)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.win = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0:  # sampler running before timing starts
                time.sleep(0.01)
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def window(self, t0: float, t1: float):
        self.win = (t0, t1)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        parsed = []
        for ts, ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                parsed.append((ts, float(f[1]), float(f[2]), float(f[3]),
                               [nm for nm, v in zip(names, f[5:9]) if v.lower() == "active"]))
            except ValueError:
                continue
        inside = [x for x in parsed if self.win and self.win[0] - 0.05 <= x[0] <= self.win[1] + 0.05]
        use = inside or parsed
        sm = [x[1] for x in use]
        reasons = sorted({r for x in use for r in x[4]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max((x[2] for x in parsed), default=None),
                "power_w_max": max((x[3] for x in use), default=None),
                "reasons": reasons, "samples": len(parsed), "samples_in_timed_region": len(inside)}


# ---------------------------------------------------------------- our arm
SHARDED = ("bkrr2", "kkrr2")  # workloads whose partitions are split over ranks (weak scaling)


def make_workload(args, rank, world=1):
    """The synthetic workload of this rank.  bkrr2 / kkrr2 on N ranks: ONE
    workload N times the one-GPU size (N x the training rows and partitions,
    the same test rows), identical on every rank, whose partitions the ranks
    split by LPT -- the paper's weak-scaling setting.  Other workloads: an
    independent copy per rank."""
    from paper_1805_00569_gb300 import synth
    kw = {}
    if args.t:
        kw["t"] = args.t
    if args.workload == "bkrr2":
        kw["n"] = (args.n or 65536) * world
        kw["p"] = (args.p or 16) * world
        return synth.bkrr2(seed=1, **kw)
    if args.workload == "kkrr2":
        n1 = args.n or 262144
        kw["n"] = n1 * world
        kw["k"] = (args.p or 64) * world
        if n1 < 262144:  # keep the mixture's size range proportional
            kw["lo"] = max(16, int(500 * n1 / 262144))
            kw["hi"] = max(kw["lo"] + 1, int(16000 * n1 / 262144))
        return synth.kkrr2(seed=2, **kw)
    if args.n:
        kw["n"] = args.n
    if args.workload == "sweep":
        if args.p:
            kw["p"] = args.p
        return synth.sweep(seed=3 + rank, **kw)
    if args.workload == "bkrr2kb":
        if args.p:
            kw["p"] = args.p
        return synth.bkrr2_kbalance(seed=5 + rank, **kw)
    return synth.dkrr(seed=0 + rank, **kw)


def oracle_sample_size(args) -> int:
    """Solves the oracle recomputes in the CPU baseline (one process each)."""
    return args.cpu_sample or max(1, min(16, os.cpu_count() or 1))


def ctypes_int():
    return ctypes.c_int(0)


def solve_flops(m: int, d: int) -> float:
    """Algorithmic flops of one partition-solve: Cholesky m^3/3, kernel m^2 d,
    two triangular solves 2 m^2."""
    return m ** 3 / 3.0 + m * m * d + 2.0 * m * m


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1805_00569_gb300 as K
    from paper_1805_00569_gb300 import dist as kd, synth

    torch.cuda.set_device(local_rank)
    w = make_workload(args, rank, world)
    sharded = (world > 1 or args.shard) and args.workload in SHARDED
    n, d = w["X"].shape
    t = w["Xt"].shape[0]
    p = w["p"]
    kmeans = args.workload in ("kkrr2", "bkrr2kb")  # routed prediction and selection
    pmode = K.KRR_PART_KBALANCE if args.workload == "bkrr2kb" else K.KRR_PART_KMEANS
    S, L = w["sigmas"], w["lambdas"]
    G = len(S) * len(L)
    nsolve = p * G
    stream = torch.cuda.current_stream()
    ctx = K.krr_ctx_create(local_rank, stream)
    if args.panel:
        K.krr_ctx_set_panel_width(ctx, args.panel)
    dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt)
    X, y, Xt, yt = dev(w["X"]), dev(w["y"]), dev(w["Xt"]), dev(w["yt"])
    yhat_buf = torch.empty((nsolve, t), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    init_idx = dev(w["init_idx"], torch.int64) if kmeans else None
    if kmeans:
        yhat_buf = torch.empty((G, t), dtype=torch.float64, device="cuda")

    last_offsets = [None]
    last_route = [None]

    owned_sizes = [None]

    def step_sharded(Xd, yd, Xtd, ytd, prec):
        """One step of the partitions this rank owns (LPT on m^3) of the one
        workload all ranks share; exchanges: the K-means block sums per round
        (kkrr2), then the scores."""
        if kmeans:
            C, a = kd.kmeans_sharded(kd.gpu_kmeans_ops(ctx), Xd, Xd[init_idx].clone(), w["iters"])
            perm, offsets = K.krr_group_rows(ctx, a, p)
            route = K.krr_kmeans_assign(ctx, Xtd, C)
            last_route[0] = route
        else:
            _, _, perm, offsets, _ = K.krr_partition(ctx, Xd, None, K.KRR_PART_RANDOM, p, seed=w["part_seed"])
        off = offsets.cpu()
        sizes = np.diff(off.numpy())
        owned = kd.lpt_assign([float(m) ** 3 for m in sizes], world)[rank]
        owned_sizes[0] = sizes[owned]
        sub, soff = kd.partition_subset(perm, off, owned)
        model, status, _ = K.krr_fit_batch(ctx, Xd, yd, sub, soff.to(Xd.device), S, L, prec)
        if kmeans:
            lmap = torch.full((p,), -1, dtype=torch.int32, device=Xd.device)
            lmap[torch.as_tensor(owned, dtype=torch.int64, device=Xd.device)] = torch.arange(
                len(owned), dtype=torch.int32, device=Xd.device)
            lroute = lmap[route.long()]
            rows = torch.nonzero(lroute >= 0).flatten()
            sse = torch.zeros(G, dtype=torch.float64, device=Xd.device)
            if rows.numel():
                yh = K.krr_predict(ctx, model, Xtd[rows], route=lroute[rows])
                m_loc, _ = K.krr_select(ctx, yh, ytd[rows], len(owned), G, K.KRR_SEL_ROUTED)
                sse = m_loc * rows.numel()
            mse = kd.sum_over_ranks(sse) / Xtd.shape[0]
            best = torch.tensor([kd.best_of(mse.cpu())[0]], dtype=torch.int32)
        else:
            yh = K.krr_predict(ctx, model, Xtd, out=yhat_buf[:len(owned) * G])
            m_loc, _ = K.krr_select(ctx, yh, ytd, len(owned), G, K.KRR_SEL_PER_MODEL)
            mse = kd.gather_scores(m_loc, [j * G + g for j in owned for g in range(G)], p * G)
            best = torch.tensor([kd.best_of(mse)[0]], dtype=torch.int32)
        model.free()
        last_offsets[0] = offsets
        return mse, best, status

    def step(Xd, yd, Xtd, ytd, prec):
        if sharded:
            return step_sharded(Xd, yd, Xtd, ytd, prec)
        if kmeans:  # KKRR2 / K-balance BKRR2: clustered partitions, routed prediction and selection
            _, route, perm, offsets, _ = K.krr_partition(ctx, Xd, Xtd, pmode, p, iters=w["iters"],
                                                         init_idx=init_idx)
            last_route[0] = route
            model, status, _ = K.krr_fit_batch(ctx, Xd, yd, perm, offsets, S, L, prec)
            yh = K.krr_predict(ctx, model, Xtd, route=route, out=yhat_buf)
            mse, best = K.krr_select(ctx, yh, ytd, p, G, K.KRR_SEL_ROUTED)
        else:
            _, _, perm, offsets, _ = K.krr_partition(ctx, Xd, None, K.KRR_PART_RANDOM, p, seed=w["part_seed"])
            model, status, _ = K.krr_fit_batch(ctx, Xd, yd, perm, offsets, S, L, prec)
            yh = K.krr_predict(ctx, model, Xtd, out=yhat_buf)
            mse, best = K.krr_select(ctx, yh, ytd, p, G, K.KRR_SEL_PER_MODEL)
        model.free()
        last_offsets[0] = offsets
        return mse, best, status

    for _ in range(args.warmup):
        mse, best, status = step(X, y, Xt, yt, args.prec)
    torch.cuda.synchronize()
    bad = int((status != K.KRR_OK).sum().item())
    if args.profile:
        if kmeans:
            _, _, perm, offsets, _ = K.krr_partition(ctx, X, Xt, pmode, p, iters=w["iters"],
                                                     init_idx=init_idx)
        else:
            _, _, perm, offsets, _ = K.krr_partition(ctx, X, None, K.KRR_PART_RANDOM, p, seed=w["part_seed"])
        model, _, _ = K.krr_fit_batch(ctx, X, y, perm, offsets, S, L, args.prec)
        it, ka, rs = K.krr_model_stats(ctx, model)
        model.free()
        Wt = ctypes_int()
        sizes = np.diff(offsets.cpu().numpy())
        ctx.lib.krr_ctx_get_panel_width(ctx.handle, {"fp64": 0, "fp32": 1, "tf32": 2, "bf16x3": 3}[args.prec],
                                        int((sizes.max() + 127) // 128), ctypes.byref(Wt))
        sys.stderr.write("partition sizes: min %d max %d\n" % (sizes.min(), sizes.max()))
        sys.stderr.write("refinement iterations per (sigma, lambda): %s; panel width %d\n" % (
            [sorted(set(int(v) for v in it.view(p, G)[:, g].tolist())) for g in range(G)], Wt.value))

    # ---- device-timed steps (inputs resident)
    # ---- per-stage CUDA-event profile: separate (untimed) steps, so the
    # timed steps carry no per-launch events
    nprof = min(args.steps, 5)
    K.krr_ctx_set_profiling(ctx, True)
    for _ in range(nprof):
        flush.zero_()
        step(X, y, Xt, yt, args.prec)
    torch.cuda.synchronize()
    prof = K.krr_ctx_profile(ctx)
    K.krr_ctx_set_profiling(ctx, False)

    clocks = Clocks(local_rank)
    launches0 = ctx.lib.krr_launch_count()
    clocks.start()
    times = []
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    t_win0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mse, best, status = step(X, y, Xt, yt, args.prec)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clocks.window(t_win0, time.perf_counter())
    if world > 1:
        tdist.barrier()
    clk = clocks.stop()
    launches = ctx.lib.krr_launch_count() - launches0
    flush_launches = 0
    total_ms = kd.max_over_ranks(sum(times))
    if sharded:
        gbest, gmse = int(best[0]), float(mse[int(best[0])])
    else:
        gbest, gmse = kd.global_best(mse, rank * nsolve)

    # ---- end to end through the same calls, host inputs
    hX, hy, hXt, hyt = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
                        (w["X"], w["y"], w["Xt"], w["yt"]))
    dX, dy, dXt, dyt = (torch.empty_like(a, device="cuda") for a in (hX, hy, hXt, hyt))
    hbest = torch.empty(1, dtype=torch.int32).pin_memory()
    hmse = torch.empty(G if kmeans else nsolve, dtype=torch.float64).pin_memory()
    e2e_times = []
    for it in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for h, dd in ((hX, dX), (hy, dy), (hXt, dXt), (hyt, dyt)):
            dd.copy_(h, non_blocking=True)
        mse2, best2, _ = step(dX, dy, dXt, dyt, args.prec)
        hbest.copy_(best2, non_blocking=True)
        hmse.copy_(mse2, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = kd.max_over_ranks(sum(e2e_times))
    h2d = sum(a.numel() * a.element_size() for a in (hX, hy, hXt, hyt))
    d2h = hbest.numel() * 4 + hmse.numel() * 8

    # ---- plain FP64 path, one step, for the comparison the metric names
    sizes0 = np.diff(last_offsets[0].cpu().numpy())
    Wt = ctypes_int()
    ctx.lib.krr_ctx_get_panel_width(ctx.handle, {"fp64": 0, "fp32": 1, "tf32": 2, "bf16x3": 3}[args.prec],
                                    int((sizes0.max() + 127) // 128), ctypes.byref(Wt))
    panel_width = int(Wt.value)

    fp64 = None
    if not args.no_fp64_path and world == 1:
        torch.cuda.synchronize()
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, st64 = step(X, y, Xt, yt, "fp64")
        e1.record(stream)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": nsolve / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                "ok_solves": int((st64 == K.KRR_OK).sum().item())}

    # ---- untimed fits: factor class of every solve (roofline), and the
    # sampled models' alpha, predictions and MSE per precision (accuracy)
    pairs = sample_models(p, G, oracle_sample_size(args)) if (rank == 0 and not kmeans and world == 1) else []
    precs = [] if sharded else [args.prec] + ([q for q in ("fp64", "fp32", "tf32", "bf16x3") if q != args.prec]
                                              if (pairs and not args.no_cpu_baseline) else [])
    gpu_acc, classes = {}, None
    for pr in precs:
        if kmeans:
            _, _, perm, offsets, _ = K.krr_partition(ctx, X, Xt, pmode, p, iters=w["iters"], init_idx=init_idx)
        else:
            _, _, perm, offsets, _ = K.krr_partition(ctx, X, None, K.KRR_PART_RANDOM, p, seed=w["part_seed"])
        model, st, alpha = K.krr_fit_batch(ctx, X, y, perm, offsets, S, L, pr, want_alpha=bool(pairs))
        if pr == args.prec:
            classes = K.krr_model_factor_class(ctx, model).numpy()
        if pairs and world == 1 and not args.no_cpu_baseline:
            yh = K.krr_predict(ctx, model, Xt, out=yhat_buf)
            mse_g, _ = K.krr_select(ctx, yh, yt, p, G, K.KRR_SEL_PER_MODEL)
            al, off, yhn, msen = (alpha.cpu().numpy(), offsets.cpu().numpy(), yh.cpu().numpy(),
                                  mse_g.cpu().numpy())
            got = {"failed": int((st != K.KRR_OK).sum().item())}
            for j, g in pairs:
                mj = int(off[j + 1] - off[j])
                a0 = int(off[j]) * G + g * mj
                got[(j, g)] = (al[a0:a0 + mj].copy(), yhn[j * G + g].copy(), float(msen[j * G + g]))
            gpu_acc[pr] = got
        model.free()
    ctx.close()

    ms_per_step = total_ms / args.steps
    # solves of all ranks per step: the shared workload's p G when sharded,
    # else every rank's own p G
    all_solves = nsolve if sharded else world * nsolve
    value = all_solves * args.steps / (total_ms / 1e3)
    gsizes = np.diff(last_offsets[0].cpu().numpy())
    tflops = ((1 if sharded else world) * G * sum(solve_flops(int(m), d) for m in gsizes) * args.steps
              / (total_ms / 1e3) / 1e12)
    sizes = owned_sizes[0] if sharded else gsizes
    return dict(w=w, sizes=sizes, value=value, ms_per_step=ms_per_step, tflops=tflops, prof=prof, nprof=nprof,
                clocks=clk,
                panel_width=panel_width,
                launches=launches + flush_launches, e2e=dict(value=all_solves * args.steps / e2e_s, unit=UNIT,
                                                         h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
                fp64=fp64, best=gbest, best_mse=gmse, bad=bad, times=times, classes=classes,
                gpu_acc=gpu_acc, pairs=pairs,
                route_counts=(np.bincount(last_route[0].cpu().numpy(), minlength=p) if kmeans else None))


# DRAM bytes (read + write) per launch from one ncu capture, keyed by kernel
# class, workload and the SHA-256 (first 16 hex digits) of the source file
# that defines the kernel: a figure whose kernel source has changed since the
# capture is dropped (null), never reused.
TRAFFIC = {
    # predict_oz_kernel, full-size BKRR2 launch: ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum
    # (one pass) -k regex:predict_oz -s 1 -c 1 on "bench.py --steps 1 --warmup 1 --no-cpu-baseline
    # --no-fp64-path --no-serve --panel 8": 74953216 read + 4427520 written
    ("predict", "bkrr2_n65536_t8192_d90_p16", "04a37c04cba64e92"): 79380736,
}
KERNEL_SOURCE = {"predict": "predict_oz.cu", "kbuild": "predict_oz.cu", "update": "chol.cu", "potrf": "chol.cu",
                 "trsm": "chol.cu", "matvec": "pcg.cu", "precond": "pcg.cu", "partition": "partition.cu"}
MUFU_PER_CLK_SM = 16      # nominal ex2 results per clock per SM
FP64_PEAK_TFLOPS = 1.25   # nominal FP64 rate of GB300 (no FP64 tensor path)


def _source_sha(kind: str) -> str | None:
    import hashlib
    f = KERNEL_SOURCE.get(kind)
    if f is None:
        return None
    try:
        with open(os.path.join(ROOT, "paper_1805_00569_gb300", "csrc", f), "rb") as fh:
            return hashlib.sha256(fh.read()).hexdigest()[:16]
    except OSError:
        return None


def _class_peak(cls: int, peaks: dict) -> float:
    """Tensor-core peak (TFLOP/s) of the precision a factor class runs at:
    one FP16 pass and three BF16 passes at the BF16 rate, three TF32 passes
    at the TF32 rate (measured BF16 x nominal 1.1/2.25), FP64 at the nominal
    FP64 rate (the algorithmic m^3/3 flops are charged against it, so
    three-pass classes pay for their extra passes)."""
    bf16 = peaks.get("bf16_tflops", 1885.0)
    if cls in (1, 2):
        return bf16
    if cls in (3, 4):
        return bf16 * 1.1 / 2.25
    return FP64_PEAK_TFLOPS


def factor_flops(m: int):
    """Algorithmic flops of the blocked Cholesky of one m x m solve (128-wide
    tiles): total m^3/3, split into the diagonal-tile factorisations, the
    panel solves and the trailing updates."""
    T = (m + 127) // 128
    tot = m ** 3 / 3.0
    potrf = T * 128 ** 3 / 3.0
    trsm = T * (T - 1) / 2.0 * 128 ** 3
    return tot, potrf, trsm, max(tot - potrf - trsm, 0.0)


def stage_rooflines(res, peaks) -> dict:
    """Each stage's measured time per step against the section 8(d) work of
    the method (not of its implementation) and the roofline that bounds it."""
    prof, nprof = res["prof"], max(res["nprof"], 1)
    w = res["w"]
    n, d = w["X"].shape
    t = w["Xt"].shape[0]
    ns, nl = len(w["sigmas"]), len(w["lambdas"])
    G = ns * nl
    sizes = [int(v) for v in res["sizes"]]
    clock = (res["clocks"] or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    hbm = peaks.get("hbm_gbs", 6779.4)
    bf16 = peaks.get("bf16_tflops", 1885.0)
    mufu = 152 * MUFU_PER_CLK_SM * clock * 1e6 / 1e9  # G exp / s
    ms = {k: v[0] / nprof for k, v in prof.items()}
    out = {}
    routed = w["workload"].startswith(("kkrr2", "bkrr2kb"))
    # a10 prediction: distances 2d flops per pair (tensor), one exponential per
    # pair and sigma (MUFU), 2 flops per pair and model (contraction); bytes:
    # the test and training rows once, (t + m) d 8 per partition
    if ms.get("predict", 0) > 0:
        if routed and res.get("route_counts") is not None:
            pairs = float(sum(int(c) * m for c, m in zip(res["route_counts"], sizes)))
        else:
            pairs = float(t) * sum(sizes)
        sec = ms["predict"] / 1e3
        f_t = pairs * 2 * d / sec / 1e12 / bf16
        f_m = pairs * ns / sec / 1e9 / mufu
        byts = (len(sizes) * t + n) * d * 8.0
        f_h = byts / sec / 1e9 / hbm
        fr = {"tensor": f_t, "mufu": f_m, "hbm": f_h}
        out["predict"] = {"ms": ms["predict"], "pairs": pairs, "tensor_frac": f_t, "mufu_frac": f_m, "hbm_frac": f_h,
                          "binding": max(fr, key=fr.get), "frac": max(fr.values()),
                          # the implementation's own work: double-float FP32 operations per pair
                          "impl_fp32_ops_per_pair": 22 + ns * (7 + 41) + G * 12,
                          "impl_alu_frac": pairs * (22 + ns * (7 + 41) + G * 12) / sec / 1e12
                          / (152 * 128 * clock * 1e6 / 1e12)}
    # a7 Cholesky: m^3/3 per solve at the rate of the precision each solve used
    fk = [k for k in ("potrf", "trsm", "update") if ms.get(k, 0) > 0]
    cls = res.get("classes")
    if fk and cls is not None:
        need = 0.0
        upd_need = 0.0
        for s_i, c in enumerate(cls):
            m = sizes[s_i // G]
            tot, _, _, upd = factor_flops(m)
            need += tot / (_class_peak(int(c), peaks) * 1e12)
            upd_need += upd / (_class_peak(int(c), peaks) * 1e12)
        sec = sum(ms[k] for k in fk) / 1e3
        out["factor"] = {"ms": sec * 1e3, "flops": float(sum(factor_flops(sizes[i // G])[0] for i in range(len(cls)))),
                         "classes": {str(c): int((cls == c).sum()) for c in sorted(set(int(x) for x in cls))},
                         "frac": need / sec, "ms_at_peak": need * 1e3,
                         "update_frac": upd_need / (ms["update"] / 1e3) if ms.get("update", 0) > 0 else None}
    # a6 kernel build: tensor (m^2 d flops per partition, distances once), MUFU
    # (m^2/2 exponentials per partition and sigma), HBM (4 bytes per stored
    # kernel entry: m^2/2 per partition and sigma)
    if ms.get("kbuild", 0) > 0:
        sec = ms["kbuild"] / 1e3
        ent = sum(m * m / 2.0 for m in sizes) * ns
        f_t = sum(m * m * d for m in sizes) / sec / 1e12 / bf16
        f_m = ent / sec / 1e9 / mufu
        f_h = ent * 4 / sec / 1e9 / hbm
        fr = {"tensor": f_t, "mufu": f_m, "hbm": f_h}
        out["kbuild"] = {"ms": ms["kbuild"], "tensor_frac": f_t, "mufu_frac": f_m, "hbm_frac": f_h,
                         "binding": max(fr, key=fr.get), "frac": max(fr.values())}
    # a3/a4 K-means: per round the FP32 copy of X read and the assignment
    # written, the FP64 rows read by the centre update, plus the final pass
    if routed and ms.get("partition", 0) > 0:
        iters = int(w.get("iters", 0))
        dpad = (d + 7) // 8 * 8
        byts = (iters + 1) * (n * dpad * 4 + 4 * n) + iters * n * d * 8
        sec = ms["partition"] / 1e3
        out["kmeans"] = {"ms": ms["partition"], "bytes": byts, "hbm_frac": byts / sec / 1e9 / hbm,
                         "frac": byts / sec / 1e9 / hbm, "binding": "hbm"}
    return out


def roofline(res, stages, peaks):
    """Roofline object of the kernel class with the largest share of device
    time, from its section 8(d) stage figures."""
    prof, nprof = res["prof"], max(res["nprof"], 1)
    dom = max(prof, key=lambda k: prof[k][0])
    ms, launches = prof[dom]
    w = res["w"]
    hbm = peaks.get("hbm_gbs", 6779.4)
    bf16 = peaks.get("bf16_tflops", 1885.0)
    clock = (res["clocks"] or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    out = {"kernel": dom, "launches": launches, "avg_launch_ms": ms / max(launches, 1),
           "share": ms / sum(v[0] for v in prof.values())}
    per = ms / nprof / 1e3  # seconds per step
    if dom == "predict" and "predict" in stages:
        st = stages["predict"]
        b = st["binding"]
        if b == "tensor":
            out.update(bound="tensor", achieved=st["tensor_frac"] * bf16, peak=bf16, unit="TFLOP/s",
                       peak_note="BF16 dense burst, of measured; 2d flops per (test, training) pair")
        elif b == "hbm":
            out.update(bound="hbm", achieved=st["hbm_frac"] * hbm, peak=hbm, unit="GB/s",
                       peak_note="copy bandwidth, of measured; (t + m) d 8 bytes per partition")
        else:
            mufu = 152 * MUFU_PER_CLK_SM * clock * 1e6 / 1e9
            out.update(bound="alu", achieved=st["mufu_frac"] * mufu, peak=mufu, unit="Gexp/s",
                       peak_note="MUFU ex2 rate, nominal 16 per clock per SM x 152 SMs x sampled SM clock; one "
                                 "exponential per (test, training) pair and sigma")
        out.update(stage_fracs={"tensor": st["tensor_frac"], "mufu": st["mufu_frac"], "hbm": st["hbm_frac"]},
                   impl_alu_frac=st["impl_alu_frac"],
                   impl_note="impl_alu_frac: the kernel's designed double-float FP32 operations "
                             "(%d per pair) against 152 x 128 FP32 lanes x clock" % st["impl_fp32_ops_per_pair"])
    elif dom in ("update", "potrf", "trsm") and "factor" in stages:
        st = stages["factor"]
        cls = res["classes"]
        G = len(w["sigmas"]) * len(w["lambdas"])
        sizes = [int(v) for v in res["sizes"]]
        idx = {"potrf": 1, "trsm": 2, "update": 3}[dom]
        flops = sum(factor_flops(sizes[i // G])[idx] for i in range(len(cls)))
        need = sum(factor_flops(sizes[i // G])[idx] / (_class_peak(int(c), peaks) * 1e12) for i, c in enumerate(cls))
        achieved = flops / per / 1e12
        out.update(bound="tensor", achieved=achieved, peak=achieved / (need / per), unit="TFLOP/s",
                   peak_note="per solve the tensor peak of its factor class (FP16/BF16 = BF16 burst, of measured; "
                             "three-pass TF32 = BF16 x 1.1/2.25); peak = the flop-weighted harmonic mean")
    elif dom == "kbuild" and "kbuild" in stages:
        st = stages["kbuild"]
        out.update(bound="hbm", achieved=st["hbm_frac"] * hbm, peak=hbm, unit="GB/s",
                   peak_note="copy bandwidth, of measured; 4 bytes per stored kernel entry (m^2/2 per sigma)",
                   stage_fracs={"tensor": st["tensor_frac"], "mufu": st["mufu_frac"], "hbm": st["hbm_frac"]})
    elif dom == "partition" and "kmeans" in stages:
        st = stages["kmeans"]
        out.update(bound="hbm", achieved=st["hbm_frac"] * hbm, peak=hbm, unit="GB/s",
                   peak_note="copy bandwidth, of measured")
    else:
        out.update(bound="hbm", achieved=None, peak=hbm, unit="GB/s", peak_note="no section 8(d) figure")
    out["frac"] = (out["achieved"] / out["peak"]) if out.get("achieved") is not None else None
    out["traffic"] = TRAFFIC.get((dom, w["workload"], _source_sha(dom)))
    if out["traffic"] is not None:
        out["traffic_unit"] = "bytes per launch (DRAM read + write)"
    return out


def run_serve(args, rank, world, local_rank):
    """Serving stream: `--requests` fit+predict requests (a fraction are
    repeat predicts of an earlier model) replayed through the serving loop,
    once at their Poisson arrival times (latency at the offered load) and once
    with every request queued at the start (capacity).  A step is one request;
    every request's time includes its host->device copies and the read-back
    of its predictions."""
    import torch
    from paper_1805_00569_gb300 import synth
    from paper_1805_00569_gb300.serving import GpuExecutor, Scheduler, latency_summary, make_stream_requests

    torch.cuda.set_device(local_rank)
    data = lambda seed, n, d, t: synth.serve_request_data(seed, n, d, t)
    st = synth.serve_stream(seed=4 + rank, requests=args.requests)
    t = int(st["t"])
    reqs = make_stream_requests(st, args.requests, data, t=t, bank=args.serve_bank)
    warm = make_stream_requests(synth.serve_stream(seed=1000 + rank, requests=max(args.warmup, 1) * 8),
                                max(args.warmup, 1) * 8, data, t=t)
    budget = 120 << 30

    def replay(rq, slots, prec, realtime):
        ex = GpuExecutor(slots, prec=prec, device=local_rank, resident_bytes=16 << 30)
        mb = args.serve_batch if prec != "fp64" else 1
        try:
            Scheduler(ex, slots, budget, resident=ex.is_resident, reserved=ex.resident_bytes, t_rows=t,
                      max_batch=mb).run(warm[:2 * slots] if prec != "fp64" else warm[:1], realtime=False)
            sc = Scheduler(ex, slots, budget, resident=ex.is_resident, reserved=ex.resident_bytes, t_rows=t,
                           max_batch=mb)
            torch.cuda.synchronize()
            res = sc.run(rq, realtime=realtime)
            torch.cuda.synchronize()
            return res, sc
        finally:
            ex.close()

    import paper_1805_00569_gb300 as K
    launches0 = K.load().krr_launch_count()
    clocks = Clocks(local_rank)
    clocks.start()
    t_live0 = time.perf_counter()
    live, sc_live = replay(reqs, args.slots, args.prec, True)
    cap, sc_cap = replay(reqs, args.slots, args.prec, False)
    clocks.window(t_live0, time.perf_counter())
    clk = clocks.stop()
    launches = K.load().krr_launch_count() - launches0
    span = max(r.done for r in cap) - min(r.start for r in cap)
    ok = sum(r.status == K.KRR_OK for r in cap)
    fits = sum(1 for r in cap if not r.resident_hit)
    seq = None
    if not args.no_fp64_path:
        sample = reqs[:args.fp64_sample]
        r64, _ = replay(sample, 1, "fp64", False)
        span64 = max(r.done for r in r64) - min(r.start for r in r64)
        seq = {"value": len(sample) / span64, "unit": "requests/s", "requests": len(sample),
               "note": "plain FP64 path, one request at a time, first %d requests of the stream" % len(sample)}
    by_id = {r.rid: r for r in reqs}  # a resident hit copies only its test rows
    h2d = sum(by_id[r.rid].payload["Xt"].nbytes + (0 if r.resident_hit else by_id[r.rid].payload["X"].nbytes
                                                   + by_id[r.rid].payload["y"].nbytes) for r in cap) / len(cap)
    return dict(value=ok / span, span=span, ok=ok, fits=fits, live=latency_summary(live),
                cap=latency_summary(cap), peak_conc=(sc_live.peak_concurrency, sc_cap.peak_concurrency),
                packed=({"batches": sc_live.batches, "requests": sc_live.batched_requests},
                        {"batches": sc_cap.batches, "requests": sc_cap.batched_requests}),
                peak_bytes=(sc_live.peak_in_use, sc_cap.peak_in_use), seq=seq, clocks=clk, launches=launches,
                h2d=h2d, offered=float(len(reqs) / st["arrival"][len(reqs) - 1]))


def main_serve(args, rank, world, local_rank):
    res = run_serve(args, rank, world, local_rank)
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": res["value"], "unit": "requests/s", "n_gpus": world, "steps": args.requests,
        "warmup": args.warmup, "ms_per_step": 1e3 * res["span"] / args.requests, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_LABEL.get(args.prec, args.prec),
        "data": "synthetic",
        "config": {"workload": "serve: %d requests, Poisson %.0f/s, n log-uniform [512, 16384], d in {8, 32, 90}, "
                               "256 test rows each, repeat predicts 20%%" % (args.requests, res["offered"]),
                   "slots": args.slots, "hbm_budget_gb": 120, "prec": args.prec,
                   "l2": "inputs of concurrent requests exceed L2; no flush between requests"},
        "serve": {"offered_rps": res["offered"], "at_offered_load": res["live"], "saturated": res["cap"],
                  "peak_concurrency": res["peak_conc"], "peak_admitted_bytes": res["peak_bytes"],
                  "fits": res["fits"], "max_batch": args.serve_batch,
                  "packed_batches": {"at_offered_load": res["packed"][0], "saturated": res["packed"][1]}},
        "fp64_sequential": res["seq"],
        "roofline": None, "roofline_note": "concurrent streams: per-kernel durations overlap; see the bkrr2 line",
        "cpu_baseline": None,
        "e2e": {"value": res["value"], "unit": "requests/s", "h2d_bytes_per_step": res["h2d"],
                "d2h_bytes_per_step": 256 * 8},
        "clocks": res["clocks"], "gpu_launches": res["launches"],
    }))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "serve":
        return main_serve(args, rank, world, local_rank)
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    sweep = None
    if args.precisions:
        sweep = {}
        for pr in [x.strip() for x in args.precisions.split(",") if x.strip()]:
            a2 = argparse.Namespace(**vars(args))
            a2.prec, a2.no_fp64_path = pr, True
            a2.steps = max(1, min(args.steps, 3)) if pr == "fp64" else args.steps
            r2 = run_ours(a2, rank, world, local_rank)
            sweep[pr] = {"value": r2["value"], "unit": UNIT, "ms_per_step": r2["ms_per_step"],
                         "failed_solves": r2["bad"], "tflops": r2["tflops"],
                         "stages_ms_per_step": {k: v[0] / r2["nprof"] for k, v in r2["prof"].items()}}
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()
    if rank != 0:
        return
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        peaks = {}
    stages = stage_rooflines(res, peaks)
    roof = roofline(res, stages, peaks)
    cpu, accuracy = None, None
    if world == 1 and not args.no_cpu_baseline:
        cpu, refs = cpu_baseline(res["w"], oracle_sample_size(args))
        if res["gpu_acc"]:
            accuracy = accuracy_vs_oracle(res["gpu_acc"], refs, res["pairs"])
    if args.profile:
        sys.stderr.write(json.dumps({k: [round(v[0], 3), v[1]] for k, v in res["prof"].items()}) + "\n")
        sys.stderr.write("step ms: %s\n" % [round(x, 2) for x in res["times"]])
    w = res["w"]
    line = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_LABEL.get(args.prec, "f64"),
        "data": "synthetic",
        "config": {"workload": w["workload"], "sigmas": w["sigmas"], "lambdas": w["lambdas"], "prec": args.prec,
                   "solves_per_step_per_gpu": w["p"] * len(w["sigmas"]) * len(w["lambdas"]) // (
                       world if args.workload in SHARDED else 1),
                   "parallelism": ("one workload, partitions split over GPUs by LPT on m^3 (weak scaling: "
                                   "%dx the one-GPU training rows and partitions)" % world
                                   if world > 1 and args.workload in SHARDED else
                                   "independent workloads per GPU" if world > 1 else "single GPU"),
                   "panel_width": res["panel_width"],
                   "l2": "flushed (512 MB write) before every timed step"},
        "tflops": res["tflops"], "roofline": roof, "cpu_baseline": cpu, "e2e": res["e2e"],
        "clocks": res["clocks"], "gpu_launches": res["launches"], "fp64_path": res["fp64"],
        "failed_solves": res["bad"], "best_model": res["best"], "best_mse": res["best_mse"],
        "stages_ms_per_step": {k: v[0] / res["nprof"] for k, v in res["prof"].items()},
        "stage_roofline": stages,
        "accuracy_vs_oracle": accuracy,
    }
    if accuracy is not None:
        line["accuracy_note"] = ("max-norm relative errors against the FP64 oracle on the %d sampled solves of the "
                                 "CPU baseline (alpha, predictions of all %d test rows, MSE), per factor precision; "
                                 "the plain FP64 path's 1e-10 bar applies where kappa * 2^-53 <= 1e-11"
                                 % (len(res["pairs"]), w["Xt"].shape[0]))
    if sweep is not None:
        line["precision_sweep"] = sweep
    if world == 1 and args.workload == "bkrr2" and not args.no_serve:
        sv = run_serve(args, rank, world, local_rank)
        line["serve"] = serve_object(args, sv)
        line["serve"]["fp64_sequential"] = sv["seq"]
        line["serve"]["clocks"] = sv["clocks"]
        line["serve"]["gpu_launches"] = sv["launches"]
    print(json.dumps(line))


def serve_object(args, res) -> dict:
    """The request stream's figures: latency at the offered load, capacity
    with every request queued at once, completions and admission peaks."""
    return {"workload": "serve: %d requests, Poisson %.0f/s offered, n log-uniform [512, 16384], d in {8, 32, 90}, "
                        "sigma log-uniform [0.5, 16], lambda log-uniform [1e-7, 1e-3], 256 test rows each, repeat "
                        "predicts 20%%, %s" % (args.requests, res["offered"],
                                               "row prefixes of %d mixtures per d" % args.serve_bank
                                               if args.serve_bank else "one mixture per request"),
            "slots": args.slots, "hbm_budget_gb": 120, "prec": args.prec,
            "offered_rps": res["offered"], "p50_ms": res["live"]["p50_ms"], "p99_ms": res["live"]["p99_ms"],
            "completed": res["live"]["completed"], "requests": args.requests,
            "at_offered_load": res["live"], "saturated": res["cap"], "saturated_rps": res["value"],
            "peak_concurrency": res["peak_conc"], "peak_admitted_bytes": res["peak_bytes"], "fits": res["fits"],
            "max_batch": args.serve_batch,
            "packed_batches": {"at_offered_load": res["packed"][0], "saturated": res["packed"][1]},
            "e2e_note": "every request's latency includes its host-to-device copies and the read-back of its "
                        "predictions"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_1805_00569_gb300 import synth
    w = synth.bkrr2(seed=1)
    sample = args.cpu_sample or max(1, min(16, os.cpu_count() or 1))
    vals = []
    for i in range(args.warmup + args.steps):
        r, _ = cpu_baseline(w, sample)
        if i >= args.warmup:
            vals.append(sample / r["value"])
    wall = sum(vals)
    value = sample * args.steps / wall
    cpu = dict(value=value, unit=UNIT, cores=sample, kind="oracle", host=host_cpu(),
               sample="per step %d of the 96 solves of %s (kernel build + Cholesky + refinement + predict + MSE), "
                      "one process each" % (sample, w["workload"]))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["workload"], "sigmas": w["sigmas"], "lambdas": w["lambdas"], "prec": "fp64"},
        "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
