"""CPU model of the FP32 screen of the K-means assignment kernels (Alg. 2,
assignment step).  The kernels take every centre's squared distance in FP32,
keep the centres whose distance lies within a rigorous error bound of the best
upper bound, and let FP64 distances in the definition's order decide among
them.  Bit-exact assignments need the FP64 argmin (strict <, lowest index) to
be among the candidates for every row, at every feature scale.  This test
redoes the screen's arithmetic in numpy FP32 (IEEE, subnormals kept, the
fused multiply-add as an exact product rounded once) and checks that property
and the bound itself, from FP32 subnormals to beyond the FP32 range."""
import numpy as np
import pytest

F32 = np.float32


def _fma32(a, b, c):
    # a*b is exact in FP64 for FP32 a, b; the sum is rounded (once to FP64,
    # then to FP32: a double rounding only on exact FP32 midpoints)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def _screen(X, C):
    """Candidates per row (bool [n, k]) and |d32 - d64| <= bound where finite."""
    n, d = X.shape
    k = C.shape[0]
    with np.errstate(over="ignore", invalid="ignore", under="ignore"):
        x32, c32 = X.astype(F32), C.astype(F32)
        xn = np.zeros(n, F32)
        for f in range(d):
            xn = _fma32(x32[:, f], x32[:, f], xn)
        cn = np.zeros(k, F32)
        for f in range(d):
            cn = _fma32(c32[:, f], c32[:, f], cn)
        acc = np.zeros((n, k), F32)
        for f in range(d):
            t = (x32[:, f][:, None] - c32[:, f][None, :]).astype(F32)
            acc = _fma32(t, t, acc)
        bscale = F32(d + 16) * F32(5.9604644775390625e-8) * F32(1.27) * F32(2.0)
        babs = np.array([4 * d + 64], np.int32).view(F32)[0]  # (4 d + 64) 2^-149
        bnd = (bscale * (xn[:, None] + cn[None, :])).astype(F32) + babs
        ub = (acc + bnd).astype(F32)
        best_hi = np.where(np.isnan(ub), np.inf, ub).min(axis=1)
        cand = ((acc - bnd).astype(F32) <= best_hi[:, None]) | ~(np.abs(ub) < np.inf)
    # FP64 distances in the definition's order (features ascending, unfused)
    d64 = np.zeros((n, k))
    for f in range(d):
        t = X[:, f][:, None] - C[:, f][None, :]
        d64 = d64 + t * t
    return cand, acc, bnd, d64


def _argmin_strict(d64):
    out = np.zeros(d64.shape[0], np.int64)
    for i, row in enumerate(d64):
        best, arg = np.inf, 0
        for j, v in enumerate(row):
            if v < best:
                best, arg = v, j
        out[i] = arg
    return out


@pytest.mark.parametrize("scale", [1e-44, 1e-40, 1e-30, 1e-22, 1e-20, 1e-19, 1e-10, 1.0, 1e15, 1e18, 1e19,
                                   1e25, 1e40])
@pytest.mark.parametrize("d", [3, 90])
def test_fp64_argmin_is_always_a_candidate(scale, d):
    rng = np.random.default_rng(d * 7 + int(np.log10(scale) + 50))
    k = 16
    C = 4.0 * rng.standard_normal((k, d))
    X = C[rng.integers(0, k, 300)] + rng.standard_normal((300, d))
    # near ties: rows half-way between two centres, and rows on a centre
    X[:20] = 0.5 * (C[rng.integers(0, k, 20)] + C[rng.integers(0, k, 20)])
    X[20:30] = C[rng.integers(0, k, 10)]
    X, C = X * scale, C * scale
    cand, acc, bnd, d64 = _screen(X, C)
    arg = _argmin_strict(d64)
    assert cand[np.arange(len(arg)), arg].all()
    fin = np.isfinite(acc) & np.isfinite(bnd) & np.isfinite(d64)
    assert np.all(np.abs(acc[fin].astype(np.float64) - d64[fin]) <= bnd[fin].astype(np.float64))


def test_screen_keeps_pruning_in_the_normal_range():
    """At ordinary scales the bound is tight enough that most rows need no
    FP64 recheck (a single candidate)."""
    rng = np.random.default_rng(3)
    C = 4.0 * rng.standard_normal((16, 90))
    X = C[rng.integers(0, 16, 400)] + rng.standard_normal((400, 90))
    cand, _, _, _ = _screen(X, C)
    assert (cand.sum(axis=1) == 1).mean() > 0.95
