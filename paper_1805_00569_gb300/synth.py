"""Seeded synthetic workloads shaped like the paper's experiments.

This module only draws random inputs; it holds none of the method's
arithmetic, and it is the one piece of code that both the CUDA path's tests
and the FP64 oracle consume.  The paper measures on the Million Song Dataset
(d = 90; Sec. 5.1) and three smaller regression sets, none of which are
available here: these generators stand in for them with the shapes listed
below.  Every array is float64, row-major.

workload            n train  n test  d   structure
dkrr_2048           2048     512     16  X ~ N(0, I); y = sin(x1+x2+x3+x4) + 0.1 e
bkrr2_65536         65536    8192    90  X ~ N(0,1) * U(0.5, 2) per column; y = tanh(w.x/sqrt d) + 0.05 e
kkrr2_262144        262144   16384   90  64-component Gaussian mixture, centres N(0, 25 I), unit spread,
                                         Dirichlet(0.5) weights clipped to [500, 16000] rows;
                                         y = w_c.x/sqrt d + b_c + sin||x|| + 0.05 e
sweep_520000        520000   51630   90  Student-t(5) features, standardised; tanh target as above
bkrr2kb_65536       65536    8192    90  the bkrr2 data; K-balance partitions (K-means from p random rows, 20 rounds)
serve stream        10000 requests, Poisson 200/s; n log-U[512, 16384], d in {8, 32, 90},
                    sigma log-U[0.5, 16], lambda log-U[1e-7, 1e-3], 256 test rows, mixture features

``scale`` shrinks n and t (and the partition counts where noted) while keeping
the distributions, for parity tests that must finish on the CPU oracle.
"""
from __future__ import annotations

import numpy as np


def _rows(n: float) -> int:
    return max(1, int(round(n)))


def dkrr(seed: int = 0, n: int = 2048, t: int = 512, d: int = 16):
    """Plain DKRR workload (single partition, sigma = 2, lambda = 1e-4)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    Xt = rng.standard_normal((t, d))
    k = min(4, d)
    y = np.sin(X[:, :k].sum(1)) + 0.1 * rng.standard_normal(n)
    yt = np.sin(Xt[:, :k].sum(1)) + 0.1 * rng.standard_normal(t)
    return dict(X=X, y=y, Xt=Xt, yt=yt, sigmas=[2.0], lambdas=[1e-4], p=1,
                workload="dkrr_n%d_t%d_d%d" % (n, t, d))


def bkrr2(seed: int = 1, n: int = 65536, t: int = 8192, d: int = 90, p: int = 16,
          sigmas=(1.0, 4.0, 16.0), lambdas=(1e-6, 1e-4)):
    """BKRR2 with random equal partitions (p parts of n/p rows)."""
    rng = np.random.default_rng(seed)
    col = rng.uniform(0.5, 2.0, d)
    w = rng.standard_normal(d)
    X = rng.standard_normal((n, d)) * col
    Xt = rng.standard_normal((t, d)) * col
    y = np.tanh(X @ w / np.sqrt(d)) + 0.05 * rng.standard_normal(n)
    yt = np.tanh(Xt @ w / np.sqrt(d)) + 0.05 * rng.standard_normal(t)
    return dict(X=X, y=y, Xt=Xt, yt=yt, sigmas=list(sigmas), lambdas=list(lambdas), p=p,
                part_seed=int(rng.integers(0, 2**63)),
                workload="bkrr2_n%d_t%d_d%d_p%d" % (n, t, d, p))


def bkrr2_kbalance(seed: int = 5, n: int = 65536, t: int = 8192, d: int = 90, p: int = 16, iters: int = 20,
                   sigmas=(1.0, 4.0, 16.0), lambdas=(1e-6, 1e-4)):
    """The BKRR2 shapes with the paper's own partitioner: K-balance over
    K-means centres that start at p random training rows."""
    w = bkrr2(seed=seed, n=n, t=t, d=d, p=p, sigmas=sigmas, lambdas=lambdas)
    rng = np.random.default_rng(seed + 1000)
    w.update(init_idx=rng.choice(n, size=p, replace=False).astype(np.int64), iters=iters,
             workload="bkrr2kb_n%d_t%d_d%d_p%d" % (n, t, d, p))
    return w


def _mixture_sizes(rng, n: int, k: int, lo: int, hi: int):
    """Dirichlet(0.5) component sizes clipped to [lo, hi] and rescaled to n."""
    w = rng.dirichlet(np.full(k, 0.5))
    sizes = np.clip(np.round(w * n), lo, hi).astype(np.int64)
    for _ in range(200):
        diff = n - int(sizes.sum())
        if diff == 0:
            break
        free = (sizes < hi) if diff > 0 else (sizes > lo)
        idx = np.nonzero(free)[0]
        if idx.size == 0:
            break
        step = np.sign(diff) * max(1, abs(diff) // idx.size)
        sizes[idx] = np.clip(sizes[idx] + step, lo, hi)
    diff = n - int(sizes.sum())
    if diff != 0:  # exact fix-up on the largest component
        sizes[int(np.argmax(sizes))] += diff
    return sizes


def _mixture(rng, n: int, t: int, d: int, k: int, lo: int, hi: int, params: dict | None = None):
    centres = 5.0 * rng.standard_normal((k, d))
    W = rng.standard_normal((k, d))
    b = rng.standard_normal(k)
    sizes = _mixture_sizes(rng, n, k, lo, hi)
    comp = np.repeat(np.arange(k), sizes)
    rng.shuffle(comp)
    X = centres[comp] + rng.standard_normal((n, d))
    tw = sizes / sizes.sum()
    comp_t = rng.choice(k, size=t, p=tw)
    Xt = centres[comp_t] + rng.standard_normal((t, d))

    def target(Z, c):
        return (np.einsum("ij,ij->i", Z, W[c]) / np.sqrt(d) + b[c]
                + np.sin(np.linalg.norm(Z, axis=1)))
    y = target(X, comp) + 0.05 * rng.standard_normal(n)
    yt = target(Xt, comp_t) + 0.05 * rng.standard_normal(t)
    if params is not None:
        params.update(centres=centres, weights=tw)
    return X, y, Xt, yt, sizes


def kkrr2(seed: int = 2, n: int = 262144, t: int = 16384, d: int = 90, k: int = 64,
          iters: int = 20, lo: int = 500, hi: int = 16000,
          sigmas=(1.0, 4.0, 16.0), lambdas=(1e-6, 1e-4)):
    """KKRR2 with K-means partitions of a Gaussian mixture (uneven sizes)."""
    rng = np.random.default_rng(seed)
    X, y, Xt, yt, sizes = _mixture(rng, n, t, d, k, lo, hi)
    init_idx = rng.choice(n, size=k, replace=False).astype(np.int64)
    return dict(X=X, y=y, Xt=Xt, yt=yt, sigmas=list(sigmas), lambdas=list(lambdas), p=k,
                init_idx=init_idx, iters=iters, mixture_sizes=sizes,
                workload="kkrr2_n%d_t%d_d%d_k%d" % (n, t, d, k))


def sweep(seed: int = 3, n: int = 520000, t: int = 51630, d: int = 90, p: int = 128,
          sigma: float = 4.0, lam: float = 1e-4):
    """Heavy-tailed BKRR2 workload (Student-t with 5 degrees of freedom)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(d)
    scale = np.sqrt(5.0 / 3.0)  # standard deviation of t(5)
    X = rng.standard_t(5, (n, d)) / scale
    Xt = rng.standard_t(5, (t, d)) / scale
    y = np.tanh(X @ w / np.sqrt(d)) + 0.05 * rng.standard_normal(n)
    yt = np.tanh(Xt @ w / np.sqrt(d)) + 0.05 * rng.standard_normal(t)
    return dict(X=X, y=y, Xt=Xt, yt=yt, sigmas=[sigma], lambdas=[lam], p=p,
                part_seed=int(rng.integers(0, 2**63)),
                workload="sweep_n%d_t%d_d%d_p%d" % (n, t, d, p))


def serve_stream(seed: int = 4, requests: int = 10000, rate: float = 200.0,
                 n_lo: int = 512, n_hi: int = 16384, dims=(8, 32, 90), t: int = 256,
                 repeat_frac: float = 0.2):
    """Request stream: arrival times and per-request shapes/parameters.
    Arrays themselves are drawn lazily by ``serve_request_data``."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, requests)
    arrival = np.cumsum(gaps)
    n = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), requests)).astype(np.int64)
    d = rng.choice(np.asarray(dims), requests)
    sigma = np.exp(rng.uniform(np.log(0.5), np.log(16.0), requests))
    lam = np.exp(rng.uniform(np.log(1e-7), np.log(1e-3), requests))
    repeat = rng.uniform(size=requests) < repeat_frac
    data_seed = rng.integers(0, 2**63, requests)
    return dict(arrival=arrival, n=n, d=d, sigma=sigma, lam=lam, t=t, repeat=repeat,
                data_seed=data_seed)


def serve_request_data(data_seed: int, n: int, d: int, t: int, k: int = 8):
    """Mixture features and the mixture target for one serving request."""
    rng = np.random.default_rng(int(data_seed))
    mix = {}
    X, y, Xt, yt, _ = _mixture(rng, int(n), int(t), int(d), k, 1, int(n), mix)
    return dict(X=X, y=y, Xt=Xt, yt=yt, mix=mix)


def serve_repeat_rows(mix: dict, seed: int, t: int):
    """New test rows from the mixture of an earlier request (a repeat predict)."""
    rng = np.random.default_rng(int(seed))
    c = rng.choice(mix["centres"].shape[0], size=int(t), p=mix["weights"])
    return mix["centres"][c] + rng.standard_normal((int(t), mix["centres"].shape[1]))
