"""FP64 CPU oracle for the partitioned kernel ridge regression hot path.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA product
path never does, and the two share no code.

The arithmetic lives in ``krr_oracle.c`` (plain C, FP64, no fused multiply-add,
long-double refinement residuals).  This module compiles it with gcc on first
use and exposes thin numpy wrappers plus the paper's pipelines composed from
them:

* ``partition_random``  -- Alg. DC-KRR, its partitioning step (shuffle, even scatter).
* ``kmeans`` / ``assign`` -- Alg. 2 (plain K-means) and the KKRR2 routing rule.
* ``kbalance_assign`` / ``partition_kbalance`` -- Alg. K-balance Clustering
                           (the BKRR partitioner).
* ``fit``               -- Alg. 1 / the training step of Alg. BKRR2 for one
                           partition and one (sigma, lambda): Eq. 6 solved by
                           Cholesky (Sec. 5.4) plus refinement.
* ``predict``           -- Eq. 7.
* ``select``            -- Eq. 3 and the model choice of Alg. BKRR2
                           (routed), best-of-p per-model MSE, the DC-KRR
                           average (Alg. DC-KRR) and the BKRR3
                           per-point choice (Alg. BKRR3).

Grid index g = i_sigma * |Lambda| + i_lambda; model index = partition * G + g.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "krr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libkrr_oracle.so")
_lock = threading.Lock()
_lib = None

KIND_GAUSSIAN = 0
KIND_LINEAR = 1


def build(force: bool = False) -> str:
    """Compile krr_oracle.c into oracle/_build/libkrr_oracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, f64, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_perm_index.argtypes = [i64, i64, u64]
            lib.orc_perm_index.restype = i64
            lib.orc_partition_random.argtypes = [i64, i32, u64, P, P, P]
            lib.orc_assign.argtypes = [P, i64, i32, P, i32, P]
            lib.orc_update_centres.argtypes = [P, i64, i32, P, i32, P]
            lib.orc_block_sums.argtypes = [P, i64, i32, P, i32, P, P]
            lib.orc_tree_combine.argtypes = [P, P, i64, i32, i32, P]
            lib.orc_kmeans.argtypes = [P, i64, i32, i32, P, i32, P, P, P]
            lib.orc_kmeans.restype = i32
            lib.orc_gather_stable.argtypes = [P, i64, i32, P, P]
            lib.orc_kbalance_assign.argtypes = [P, i64, i32, P, i32, i64, P, P]
            lib.orc_kernel_matrix.argtypes = [P, i64, P, i64, i32, i32, f64, P]
            lib.orc_solve_spd.argtypes = [P, i64, P, P, f64, P]
            lib.orc_solve_spd.restype = ctypes.c_int
            lib.orc_krr_fit.argtypes = [P, P, i64, i32, i32, f64, f64, P, P]
            lib.orc_krr_fit.restype = ctypes.c_int
            lib.orc_krr_predict.argtypes = [P, P, i64, i32, i32, f64, P, i64, P, P]
            lib.orc_mse.argtypes = [P, P, i64]
            lib.orc_mse.restype = f64
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- generator
def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al., SC'11): four 32-bit counter words and two
    32-bit key words in, four 32-bit words out."""
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def perm_index(i: int, n: int, seed: int) -> int:
    return int(_load().orc_perm_index(int(i), int(n), int(seed) & (2**64 - 1)))


# ---------------------------------------------------------------- partition
def partition_random(n: int, p: int, seed: int):
    """The partitioning step of Alg. DC-KRR: returns (perm, offsets, assign)."""
    perm = np.zeros(n, np.int64)
    offsets = np.zeros(p + 1, np.int64)
    assign = np.zeros(n, np.int32)
    _load().orc_partition_random(n, p, int(seed) & (2**64 - 1), _p(perm), _p(offsets), _p(assign))
    return perm, offsets, assign


def assign(X, C):
    """Alg. 2 step 4 / KKRR2 routing: nearest centre, lowest index on ties."""
    X = _c(X, np.float64)
    C = _c(C, np.float64)
    out = np.zeros(X.shape[0], np.int32)
    _load().orc_assign(_p(X), X.shape[0], X.shape[1], _p(C), C.shape[0], _p(out))
    return out


def update_centres(X, c, C_prev):
    """Alg. 2 step 6 in the canonical summation order; empty clusters keep
    their previous centre."""
    X = _c(X, np.float64)
    c = _c(c, np.int32)
    C = np.array(C_prev, dtype=np.float64, copy=True, order="C")
    _load().orc_update_centres(_p(X), X.shape[0], X.shape[1], _p(c), C.shape[0], _p(C))
    return C


def block_sums(X, c, k: int):
    """First half of Alg. 2 step 6 in the canonical order: per block of 1024
    consecutive rows (from row 0 of X), every centre's member sum in
    ascending row order and its member count.  Returns (sums [nblk, k, d],
    counts [nblk, k])."""
    X = _c(X, np.float64)
    c = _c(c, np.int32)
    nblk = -(-X.shape[0] // 1024)
    part = np.zeros((nblk, k, X.shape[1]), np.float64)
    cnt = np.zeros((nblk, k), np.int64)
    _load().orc_block_sums(_p(X), X.shape[0], X.shape[1], _p(c), k, _p(part), _p(cnt))
    return part, cnt


def tree_combine(sums, counts, C_prev):
    """Second half of Alg. 2 step 6: the pairwise tree over the block sums in
    block order, one division by the member count; empty clusters keep
    their previous centre."""
    part = np.array(sums, dtype=np.float64, copy=True, order="C")
    cnt = _c(counts, np.int64)
    C = np.array(C_prev, dtype=np.float64, copy=True, order="C")
    _load().orc_tree_combine(_p(part), _p(cnt), part.shape[0], C.shape[0], C.shape[1], _p(C))
    return C


def kmeans(X, k: int, init_idx, iters: int):
    """Alg. 2: returns (centres, final assignment, per-round change counts)."""
    X = _c(X, np.float64)
    init_idx = _c(init_idx, np.int64)
    C = np.zeros((k, X.shape[1]), np.float64)
    c = np.zeros(X.shape[0], np.int32)
    delta = np.zeros(max(iters, 1), np.int64)
    r = _load().orc_kmeans(_p(X), X.shape[0], X.shape[1], k, _p(init_idx), iters, _p(C), _p(c), _p(delta))
    return C, c, delta[:r]


def gather_stable(assign_, p: int):
    """Group rows by partition, ascending row index inside each partition."""
    a = _c(assign_, np.int32)
    perm = np.zeros(a.shape[0], np.int64)
    offsets = np.zeros(p + 1, np.int64)
    _load().orc_gather_stable(_p(a), a.shape[0], p, _p(perm), _p(offsets))
    return perm, offsets


def partition_kmeans(X, Xt, k: int, init_idx, iters: int):
    """KKRR2 partition: K-means, final assignment, stable grouping, routing."""
    C, c, delta = kmeans(X, k, init_idx, iters)
    perm, offsets = gather_stable(c, k)
    route = assign(Xt, C) if Xt is not None else None
    return perm, offsets, c, route, C, delta


def kbalance_assign(X, C, cap: int):
    """Alg. K-balance Clustering, per-sample loop: every sample in index
    order takes its nearest centre among those holding fewer than `cap`
    samples.  Returns (assignment, counts)."""
    X = _c(X, np.float64)
    C = _c(C, np.float64)
    out = np.zeros(X.shape[0], np.int32)
    cs = np.zeros(C.shape[0], np.int64)
    _load().orc_kbalance_assign(_p(X), X.shape[0], X.shape[1], _p(C), C.shape[0], int(cap), _p(out), _p(cs))
    return out, cs


def partition_kbalance(X, Xt, p: int, init_idx, iters: int):
    """BKRR / BKRR2 partition (Alg. K-balance Clustering): K-means centres
    (Alg. 2, as in partition_kmeans), the balanced per-sample assignment with
    cap = ceil(n / p), the centres recomputed as the means of the balanced
    parts (the listing's final averaging; empty parts keep their centre),
    stable grouping, and nearest-centre routing of the test rows with the
    recomputed centres."""
    X = _c(X, np.float64)
    C, _, _ = kmeans(X, p, init_idx, iters)
    cap = -(-X.shape[0] // p)
    c, cs = kbalance_assign(X, C, cap)
    C2 = update_centres(X, c, C)
    perm, offsets = gather_stable(c, p)
    route = assign(Xt, C2) if Xt is not None else None
    return perm, offsets, c, route, C2, cs


# ---------------------------------------------------------------- kernels
def kernel_matrix(A, B, sigma: float, kind: int = KIND_GAUSSIAN):
    """Table 1 kernel matrix K[i, j] = Phi(A_i, B_j)."""
    A = _c(A, np.float64)
    B = _c(B, np.float64)
    K = np.zeros((A.shape[0], B.shape[0]), np.float64)
    _load().orc_kernel_matrix(_p(A), A.shape[0], _p(B), B.shape[0], A.shape[1], kind, float(sigma), _p(K))
    return K


def solve_spd(A, y, lambda_m: float):
    """Cholesky solve of an SPD system plus long-double refinement.
    Returns (x, info, rc); info = (condition estimate, scaled residual, steps)."""
    A = _c(A, np.float64)
    y = _c(y, np.float64)
    x = np.zeros_like(y)
    info = np.zeros(3, np.float64)
    rc = _load().orc_solve_spd(_p(A), A.shape[0], _p(y), _p(x), float(lambda_m), _p(info))
    return x, info, rc


def fit(Xp, yp, sigma: float, lam: float, kind: int = KIND_GAUSSIAN):
    """Eq. 6 for one partition: (K + lambda m I) alpha = y, m = len(yp).
    Returns (alpha, info, rc)."""
    Xp = _c(Xp, np.float64)
    yp = _c(yp, np.float64)
    m = Xp.shape[0]
    alpha = np.zeros(m, np.float64)
    info = np.zeros(3, np.float64)
    rc = _load().orc_krr_fit(_p(Xp), _p(yp), m, Xp.shape[1] if Xp.ndim == 2 else 0, kind,
                             float(sigma), float(lam), _p(alpha), _p(info))
    return alpha, info, rc


def predict(Xp, alpha, Xt, sigma: float, kind: int = KIND_GAUSSIAN, with_cancel: bool = False):
    """Eq. 7 for one model over test rows Xt."""
    Xp = _c(Xp, np.float64)
    alpha = _c(alpha, np.float64)
    Xt = _c(Xt, np.float64)
    t = Xt.shape[0]
    yhat = np.zeros(t, np.float64)
    cancel = np.zeros(t, np.float64) if with_cancel else None
    _load().orc_krr_predict(_p(Xp), _p(alpha), Xp.shape[0], Xt.shape[1], kind, float(sigma), _p(Xt), t,
                            _p(yhat), _p(cancel) if with_cancel else None)
    return (yhat, cancel) if with_cancel else yhat


def mse(yhat, y) -> float:
    """Eq. 3."""
    a = _c(yhat, np.float64)
    b = _c(y, np.float64)
    return float(_load().orc_mse(_p(a), _p(b), a.shape[0]))


# ---------------------------------------------------------------- pipelines
SEL_PER_MODEL, SEL_ROUTED, SEL_AVERAGE, SEL_ORACLE = 0, 1, 2, 3


def fit_batch(X, y, perm, offsets, sigmas, lambdas, kind: int = KIND_GAUSSIAN):
    """Every (partition, sigma, lambda) solve.  Returns alphas[p][g] (arrays),
    infos[p][g], rcs[p][g]."""
    X = _c(X, np.float64)
    y = _c(y, np.float64)
    P = len(offsets) - 1
    alphas, infos, rcs = [], [], []
    for j in range(P):
        rows = perm[offsets[j]:offsets[j + 1]]
        Xp, yp = X[rows], y[rows]
        a_row, i_row, r_row = [], [], []
        for s in sigmas:
            for lam in lambdas:
                a, info, rc = fit(Xp, yp, s, lam, kind)
                a_row.append(a)
                i_row.append(info)
                r_row.append(rc)
        alphas.append(a_row)
        infos.append(i_row)
        rcs.append(r_row)
    return alphas, infos, rcs


def predict_all(X, perm, offsets, alphas, sigmas, lambdas, Xt, route=None, kind: int = KIND_GAUSSIAN):
    """All-models form: yhat[p*G + g, j] for every test row j.  Routed form
    (route given): yhat[g, j] from the model of partition route[j]."""
    X = _c(X, np.float64)
    Xt = _c(Xt, np.float64)
    P = len(offsets) - 1
    G = len(sigmas) * len(lambdas)
    t = Xt.shape[0]
    if route is None:
        out = np.zeros((P * G, t), np.float64)
    else:
        out = np.zeros((G, t), np.float64)
    for j in range(P):
        Xp = X[perm[offsets[j]:offsets[j + 1]]]
        if route is None:
            cols = np.arange(t)
        else:
            cols = np.nonzero(np.asarray(route) == j)[0]
        if cols.size == 0:
            continue
        for si, s in enumerate(sigmas):
            for li in range(len(lambdas)):
                g = si * len(lambdas) + li
                yh = predict(Xp, alphas[j][g], Xt[cols], s, kind)
                if route is None:
                    out[j * G + g, cols] = yh
                else:
                    out[g, cols] = yh
    return out


def select(yhat, yt, mode: int, n_partitions: int = 1, G: int = 1):
    """Model choice.  Returns (mse array, best index).

    SEL_PER_MODEL: yhat[model, t]; one MSE per model, best = lowest MSE.
    SEL_ROUTED:    yhat[g, t] holds each test point's routed prediction; one
                   MSE per grid point (Alg. BKRR2), best grid point.
    SEL_AVERAGE:   yhat[model, t]; per grid point the average over partitions
                   (Alg. DC-KRR) is scored.
    SEL_ORACLE:    yhat[model, t]; per grid point each test point takes the
                   partition whose prediction is closest to its label
                   (Alg. BKRR3, lowest partition on ties).
    Ties in the best index go to the lowest index (strict <)."""
    yhat = np.asarray(yhat, np.float64)
    yt = _c(yt, np.float64)
    if mode in (SEL_PER_MODEL, SEL_ROUTED):
        mses = np.array([mse(yhat[i], yt) for i in range(yhat.shape[0])])
    elif mode == SEL_AVERAGE:
        mses = np.zeros(G)
        for g in range(G):
            acc = np.zeros(yt.shape[0])
            for j in range(n_partitions):
                acc = acc + yhat[j * G + g]
            mses[g] = mse(acc / n_partitions, yt)
    elif mode == SEL_ORACLE:
        mses = np.zeros(G)
        for g in range(G):
            chosen = np.zeros(yt.shape[0])
            for q in range(yt.shape[0]):
                best_e, best_v = np.inf, 0.0
                for j in range(n_partitions):
                    v = yhat[j * G + g, q]
                    e = (v - yt[q]) * (v - yt[q])
                    if e < best_e:
                        best_e, best_v = e, v
                chosen[q] = best_v
            mses[g] = mse(chosen, yt)
    else:
        raise ValueError("unknown selection mode")
    best = 0
    for i in range(1, mses.shape[0]):
        if mses[i] < mses[best]:
            best = i
    return mses, best
