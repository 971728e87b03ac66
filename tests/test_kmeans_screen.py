"""CPU model of the FP32 screen of the K-means assignment kernels (Alg. 2,
assignment step), in each summation form the kernels use (the difference
form of the general kernel; the Gram form of the tiled screen and of the
recheck, each in its own order).  The kernels take every centre's squared
distance in FP32,
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


def _lane_tree(parts):
    """Sum of 32 lane partials [32, ...] by the butterfly the kernels use
    (stage o: lane l adds lane l ^ o, o = 16, 8, 4, 2, 1)."""
    v = parts
    for o in (16, 8, 4, 2, 1):
        v = np.stack([(v[l] + v[l ^ o]).astype(F32) for l in range(32)])
    return v[0]


def _lane_partials(a, b, d):
    """Per-lane FMA chains over features f = lane, lane + 32, ... of a * b
    (a [d, ...], b [d, ...]): [32, ...] partials."""
    out = []
    for lane in range(32):
        acc = np.zeros(np.broadcast(a[0], b[0]).shape, F32)
        for f in range(lane, d, 32):
            acc = _fma32(a[f], b[f], acc)
        out.append(acc)
    return np.stack(out)


def _screen(X, C, form="diff"):
    """Candidates per row (bool [n, k]) and |d32 - d64| <= bound where finite.

    form: "diff" -- sum over features of (x - c)^2 (the general kernel);
    "screen" -- Gram form rn(rn(|x|^2 + |c|^2) - 2 x.c), |x|^2 as two
    half-feature chains added, |c|^2 by lane partials and the butterfly,
    x.c one chain in feature order (the tiled screening kernel);
    "recheck" -- the same Gram form with |x|^2 and x.c as lane partials and
    the butterfly (the recheck kernel)."""
    n, d = X.shape
    k = C.shape[0]
    with np.errstate(over="ignore", invalid="ignore", under="ignore"):
        x32, c32 = X.astype(F32), C.astype(F32)
        xT, cT = x32.T, c32.T
        if form == "screen":
            dp = (d + 7) // 8 * 8
            h0 = np.zeros(n, F32)
            h1 = np.zeros(n, F32)
            for f in range(min(d, dp // 2)):
                h0 = _fma32(xT[f], xT[f], h0)
            for f in range(dp // 2, d):
                h1 = _fma32(xT[f], xT[f], h1)
            xn = (h0 + h1).astype(F32)
        elif form == "recheck":
            xn = _lane_tree(_lane_partials(xT, xT, d))
        else:
            xn = np.zeros(n, F32)
            for f in range(d):
                xn = _fma32(xT[f], xT[f], xn)
        if form == "diff":
            cn = np.zeros(k, F32)
            for f in range(d):
                cn = _fma32(cT[f], cT[f], cn)
        else:
            cn = _lane_tree(_lane_partials(cT, cT, d))
        if form == "diff":
            acc = np.zeros((n, k), F32)
            for f in range(d):
                t = (x32[:, f][:, None] - c32[:, f][None, :]).astype(F32)
                acc = _fma32(t, t, acc)
        else:
            if form == "screen":
                dot = np.zeros((n, k), F32)
                for f in range(d):
                    dot = _fma32(xT[f][:, None], cT[f][None, :], dot)
            else:
                dot = _lane_tree(_lane_partials(xT[:, :, None], cT[:, None, :], d))
            s = (xn[:, None] + cn[None, :]).astype(F32)
            acc = _fma32(np.full_like(dot, -2.0), dot, s)
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
@pytest.mark.parametrize("form", ["diff", "screen", "recheck"])
def test_fp64_argmin_is_always_a_candidate(scale, d, form):
    rng = np.random.default_rng(d * 7 + int(np.log10(scale) + 50))
    k = 16
    C = 4.0 * rng.standard_normal((k, d))
    X = C[rng.integers(0, k, 300)] + rng.standard_normal((300, d))
    # near ties: rows half-way between two centres, and rows on a centre
    X[:20] = 0.5 * (C[rng.integers(0, k, 20)] + C[rng.integers(0, k, 20)])
    X[20:30] = C[rng.integers(0, k, 10)]
    X, C = X * scale, C * scale
    cand, acc, bnd, d64 = _screen(X, C, form)
    arg = _argmin_strict(d64)
    assert cand[np.arange(len(arg)), arg].all()
    fin = np.isfinite(acc) & np.isfinite(bnd) & np.isfinite(d64)
    assert np.all(np.abs(acc[fin].astype(np.float64) - d64[fin]) <= bnd[fin].astype(np.float64))


@pytest.mark.parametrize("form", ["diff", "screen"])
def test_screen_keeps_pruning_in_the_normal_range(form):
    """At ordinary scales the bound is tight enough that most rows need no
    FP64 recheck (a single candidate)."""
    rng = np.random.default_rng(3)
    C = 4.0 * rng.standard_normal((16, 90))
    X = C[rng.integers(0, 16, 400)] + rng.standard_normal((400, 90))
    cand, _, _, _ = _screen(X, C, form)
    assert (cand.sum(axis=1) == 1).mean() > 0.95
