"""Parity of the sm_103a path (called through the C ABI) with the FP64 oracle.

Bars: partition assignments, permutations and centres bit-exact; alpha,
predictions and MSE within 1e-6 relative (max-norm per model) for the refined
precisions (FP32, TF32) and 1e-10 for the plain FP64 path where the
condition estimate times the FP64 unit roundoff stays below 1e-11.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1805_00569_gb300 as K
from paper_1805_00569_gb300 import synth

pytestmark = pytest.mark.gpu

REFINED_TOL = 1e-6
FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = K.krr_ctx_create(0)
    yield c
    c.close()


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.max(np.abs(b))
    return 0.0 if den == 0 and np.max(np.abs(a)) == 0 else float(np.max(np.abs(a - b)) / den)


def tol_for(prec, kappa):
    if prec == "fp64":
        return FP64_TOL if kappa * 2.0 ** -53 <= 1e-11 else None
    return REFINED_TOL


def split_alpha(alpha, offsets, G):
    """Caller layout of krr_fit_batch's alpha -> alphas[j][g]."""
    out = []
    for j in range(len(offsets) - 1):
        m = offsets[j + 1] - offsets[j]
        blk = alpha[offsets[j] * G:offsets[j + 1] * G]
        out.append([blk[g * m:(g + 1) * m] for g in range(G)])
    return out


# ------------------------------------------------------------------ partitions
@pytest.mark.parametrize("n,p,seed", [(1, 1, 3), (1000, 7, 12345), (65536, 16, 2**63 + 5), (4097, 128, 9)])
def test_random_partition_bit_exact(ctx, n, p, seed):
    X = np.random.default_rng(0).standard_normal((n, 3))
    assign, _, perm, offsets, _ = K.krr_partition(ctx, cuda(X), None, K.KRR_PART_RANDOM, p, seed=seed)
    operm, ooff, oassign = oracle.partition_random(n, p, seed)
    assert np.array_equal(perm.cpu().numpy(), operm)
    assert np.array_equal(offsets.cpu().numpy(), ooff)
    assert np.array_equal(assign.cpu().numpy(), oassign)


def _mixture(n, t, d, k, seed):
    rng = np.random.default_rng(seed)
    C = 4.0 * rng.standard_normal((k, d))
    X = C[rng.integers(0, k, n)] + rng.standard_normal((n, d))
    Xt = C[rng.integers(0, k, t)] + rng.standard_normal((t, d))
    return X, Xt, rng.choice(n, k, replace=False).astype(np.int64)


@pytest.mark.parametrize("n,t,d,k,iters", [(5000, 700, 12, 8, 10), (3333, 129, 90, 16, 5), (2500, 1, 3, 5, 0),
                                           # the screen's centre tiles: 2 and 4 tiles of 64 (k = 256 its limit)
                                           (4000, 100, 20, 100, 3), (3000, 30, 5, 256, 2),
                                           # the general kernel: d > 96, k > 256
                                           (3000, 50, 100, 12, 3), (4000, 40, 8, 300, 2)])
def test_kmeans_partition_bit_exact(ctx, n, t, d, k, iters):
    X, Xt, init = _mixture(n, t, d, k, n)
    assign, route, perm, offsets, centers = K.krr_partition(ctx, cuda(X), cuda(Xt), K.KRR_PART_KMEANS, k,
                                                            iters=iters, init_idx=cuda(init, torch.int64))
    operm, ooff, oassign, oroute, oC, _ = oracle.partition_kmeans(X, Xt, k, init, iters)
    assert np.array_equal(assign.cpu().numpy(), oassign)
    assert np.array_equal(route.cpu().numpy(), oroute)
    assert np.array_equal(perm.cpu().numpy(), operm)
    assert np.array_equal(offsets.cpu().numpy(), ooff)
    assert np.array_equal(centers.cpu().numpy().view(np.uint64), oC.view(np.uint64))


@pytest.mark.parametrize("scale", [1e-40, 1e-20, 1e18, 1e25, 1e40])
@pytest.mark.parametrize("mode", ["kmeans", "kbalance"])
def test_partition_bit_exact_at_extreme_feature_scales(ctx, scale, mode):
    """Alg. 2 assignments stay the FP64 argmin when the FP32 screen leaves its
    normal range: squared features in FP32 subnormals (1e-20), features that
    are FP32 subnormals themselves (1e-40), squared distances that overflow
    FP32 (1e18, 1e25) and features beyond the FP32 range (1e40).  Assignments,
    routes, groupings and centres bit-exact with the oracle."""
    n, t, d, k, iters = 3000, 200, 90, 16, 4
    X, Xt, init = _mixture(n, t, d, k, 77)
    X, Xt = X * scale, Xt * scale
    pm = K.KRR_PART_KMEANS if mode == "kmeans" else K.KRR_PART_KBALANCE
    assign, route, perm, offsets, centers = K.krr_partition(ctx, cuda(X), cuda(Xt), pm, k, iters=iters,
                                                            init_idx=cuda(init, torch.int64))
    fn = oracle.partition_kmeans if mode == "kmeans" else oracle.partition_kbalance
    operm, ooff, oassign, oroute, oC, _ = fn(X, Xt, k, init, iters)
    assert np.array_equal(assign.cpu().numpy(), oassign)
    assert np.array_equal(route.cpu().numpy(), oroute)
    assert np.array_equal(perm.cpu().numpy(), operm)
    assert np.array_equal(offsets.cpu().numpy(), ooff)
    assert np.array_equal(centers.cpu().numpy().view(np.uint64), oC.view(np.uint64))


@pytest.mark.parametrize("n,t,d,k,iters", [(5000, 700, 12, 8, 10), (3333, 129, 90, 16, 5), (2500, 1, 3, 5, 0),
                                           (4096, 64, 7, 32, 3), (70000, 300, 90, 16, 4)])
def test_kbalance_partition_bit_exact(ctx, n, t, d, k, iters):
    """Alg. K-balance Clustering (the BKRR partitioner): K-means centres, the
    balanced sequential assignment replayed on the GPU in rounds, the means
    of the balanced parts and the routes, all bit-exact with the oracle."""
    X, Xt, init = _mixture(n, t, d, k, n)
    assign, route, perm, offsets, centers = K.krr_partition(ctx, cuda(X), cuda(Xt), K.KRR_PART_KBALANCE, k,
                                                            iters=iters, init_idx=cuda(init, torch.int64))
    operm, ooff, oassign, oroute, oC, ocs = oracle.partition_kbalance(X, Xt, k, init, iters)
    assert np.array_equal(assign.cpu().numpy(), oassign)
    assert np.array_equal(route.cpu().numpy(), oroute)
    assert np.array_equal(perm.cpu().numpy(), operm)
    assert np.array_equal(offsets.cpu().numpy(), ooff)
    assert np.array_equal(centers.cpu().numpy().view(np.uint64), oC.view(np.uint64))
    sizes = np.diff(offsets.cpu().numpy())
    assert sizes.max() <= -(-n // k)
    if n % k == 0:
        assert np.all(sizes == n // k)


def test_kbalance_exact_ties(ctx):
    """Integer points and duplicated centres: equal distances go to the lower
    open index, and a centre that fills passes its later ties to the next one."""
    X = np.array([[float(i % 5), float(i % 3)] for i in range(60)])
    init = np.array([0, 15, 0, 7], np.int64)  # centres 0 and 2 coincide
    for iters in (0, 2):
        assign, route, perm, offsets, centers = K.krr_partition(ctx, cuda(X), None, K.KRR_PART_KBALANCE, 4,
                                                                iters=iters, init_idx=cuda(init, torch.int64))
        operm, ooff, oassign, _, oC, _ = oracle.partition_kbalance(X, None, 4, init, iters)
        assert np.array_equal(assign.cpu().numpy(), oassign)
        assert np.array_equal(offsets.cpu().numpy(), ooff)
        assert np.array_equal(centers.cpu().numpy().view(np.uint64), oC.view(np.uint64))
        assert np.diff(ooff).max() <= 15


def test_kmeans_exact_ties_and_empty_cluster(ctx):
    """Integer points equidistant from two centres go to the lower index; a
    duplicated initial centre loses every tie, so with no update round it owns
    no rows; with updates the result still equals the definition bit for bit."""
    g = np.arange(-6, 7, dtype=np.float64)
    X = np.array([[a, b] for a in g for b in g])  # 169 integer grid points
    init = np.array([0, 168, 84, 0], np.int64)  # centre 3 duplicates centre 0
    Xt = np.array([[0.0, 0.0], [-6.0, -6.0], [6.0, 6.0]])
    for iters in (0, 4):
        assign, route, perm, offsets, centers = K.krr_partition(ctx, cuda(X), cuda(Xt), K.KRR_PART_KMEANS, 4,
                                                                iters=iters, init_idx=cuda(init, torch.int64))
        operm, ooff, oassign, oroute, oC, _ = oracle.partition_kmeans(X, Xt, 4, init, iters)
        assert np.array_equal(assign.cpu().numpy(), oassign)
        assert np.array_equal(route.cpu().numpy(), oroute)
        assert np.array_equal(perm.cpu().numpy(), operm)
        assert np.array_equal(offsets.cpu().numpy(), ooff)
        assert np.array_equal(centers.cpu().numpy().view(np.uint64), oC.view(np.uint64))
        if iters == 0:
            assert ooff[4] - ooff[3] == 0  # the duplicate centre owns no rows


def test_kmeans_centre_sum_order_bit_exact(ctx):
    """A centre whose value depends on the summation order: 2^53 absorbs the
    ones of its own 1024-row block, the next block's ones survive, and -2^53
    in the third block cancels; the canonical block-tree order gives 1024 / 3000
    (the exact mean would be 2047 / 3000, one ascending pass 0)."""
    n = 3000
    X = np.zeros((n, 2))
    X[0, 0] = 2.0**53
    X[1:2048, 0] = 1.0
    X[2048, 0] = -(2.0**53)
    X[:, 1] = np.arange(n) % 7
    Xt = np.array([[0.0, 0.0], [5.0, 1.0]])
    init = np.array([5], np.int64)
    for iters in (1, 3):
        assign, route, perm, offsets, centers = K.krr_partition(ctx, cuda(X), cuda(Xt), K.KRR_PART_KMEANS, 1,
                                                                iters=iters, init_idx=cuda(init, torch.int64))
        operm, ooff, oassign, oroute, oC, _ = oracle.partition_kmeans(X, Xt, 1, init, iters)
        got = centers.cpu().numpy()
        assert got[0, 0] == 1024.0 / 3000.0
        assert np.array_equal(got.view(np.uint64), oC.view(np.uint64))
        assert np.array_equal(assign.cpu().numpy(), oassign) and np.array_equal(perm.cpu().numpy(), operm)


# ------------------------------------------------------------------ fit / predict / select
def _case(seed=7, n=950, d=13, t=333):
    rng = np.random.default_rng(seed)
    col = rng.uniform(0.5, 1.5, d)
    X = rng.standard_normal((n, d)) * col
    Xt = rng.standard_normal((t, d)) * col
    w = rng.standard_normal(d)
    y = np.tanh(X @ w / np.sqrt(d)) + 0.05 * rng.standard_normal(n)
    yt = np.tanh(Xt @ w / np.sqrt(d)) + 0.05 * rng.standard_normal(t)
    perm = rng.permutation(n).astype(np.int64)
    offsets = np.array([0, 300, 817, n], np.int64)  # 300, 517, 133 rows: ragged tiles
    return X, y, Xt, yt, perm, offsets


SIG = [0.8, 3.0]
LAM = [1e-5, 1e-3]


@pytest.fixture(scope="module")
def oracle_case():
    X, y, Xt, yt, perm, offsets = _case()
    al, infos, rcs = oracle.fit_batch(X, y, perm, offsets, SIG, LAM)
    yall = oracle.predict_all(X, perm, offsets, al, SIG, LAM, Xt)
    return dict(X=X, y=y, Xt=Xt, yt=yt, perm=perm, offsets=offsets, alphas=al, infos=infos, rcs=rcs, yall=yall)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16x3"])
def test_fit_predict_select_parity(ctx, oracle_case, prec):
    c = oracle_case
    G = len(SIG) * len(LAM)
    model, status, alpha = K.krr_fit_batch(ctx, cuda(c["X"]), cuda(c["y"]), cuda(c["perm"], torch.int64),
                                           cuda(c["offsets"], torch.int64), SIG, LAM, prec, want_alpha=True)
    try:
        assert np.all(status.cpu().numpy() == K.KRR_OK), status
        galpha = split_alpha(alpha.cpu().numpy(), c["offsets"], G)
        worst = 0.0
        for j in range(3):
            for g in range(G):
                kappa = c["infos"][j][g][0]
                tol = tol_for(prec, kappa)
                e = rel(galpha[j][g], c["alphas"][j][g])
                worst = max(worst, e)
                if tol is not None:
                    assert e <= tol, (prec, j, g, e, kappa)
        yhat = K.krr_predict(ctx, model, cuda(c["Xt"])).cpu().numpy()
        for row in range(3 * G):
            kappa = c["infos"][row // G][row % G][0]
            tol = tol_for(prec, kappa)
            if tol is not None:
                assert rel(yhat[row], c["yall"][row]) <= tol, (prec, row)
        for mode in (K.KRR_SEL_PER_MODEL, K.KRR_SEL_AVERAGE, K.KRR_SEL_ORACLE):
            mse, best = K.krr_select(ctx, cuda(yhat), cuda(c["yt"]), 3, G, mode)
            omse, obest = oracle.select(c["yall"], c["yt"], mode, 3, G)
            np.testing.assert_allclose(mse.cpu().numpy(), omse, rtol=REFINED_TOL if prec != "fp64" else 1e-9)
            b = int(best.cpu()[0])
            assert omse[b] <= omse[obest] * (1 + REFINED_TOL)
        it, kap, res = K.krr_model_stats(ctx, model)
        assert np.all(it.numpy() >= 1)
        # ||K + lambda m I||_inf / (lambda m): FP64 matrix-vector product on
        # the FP64 path, FP32 row sums of the stored tiles otherwise
        okap = np.array([c["infos"][j][g][0] for j in range(3) for g in range(G)])
        np.testing.assert_allclose(kap.numpy(), okap, rtol=1e-12 if prec == "fp64" else 1e-5)
    finally:
        model.free()


@pytest.mark.parametrize("lam", [1e5, 1e8])
def test_large_lambda_m_leaves_the_fp16_factor(ctx, lam):
    """A one-pass solve keeps its factor in FP16 only while 1 + lambda m <=
    2^24 (|L_ij| <= sqrt(A_jj)); beyond that (lambda m = 3e7 and 3e10 here;
    sqrt(3e10) would overflow FP16) it is factored in the three-pass class,
    and the result still matches the oracle."""
    X, y, Xt, yt, perm, offsets = _case()
    model, status, alpha = K.krr_fit_batch(ctx, cuda(X), cuda(y), cuda(perm, torch.int64), cuda(offsets, torch.int64),
                                           [2.0], [lam], "tf32", want_alpha=True)
    try:
        assert np.all(status.cpu().numpy() == K.KRR_OK)
        ga = alpha.cpu().numpy()
        for j in range(3):
            rows = perm[offsets[j]:offsets[j + 1]]
            oa, info, rc = oracle.fit(X[rows], y[rows], 2.0, lam)
            assert rc == 0
            assert rel(split_alpha(ga, offsets, 1)[j][0], oa) <= REFINED_TOL
    finally:
        model.free()


def test_linear_kernel_fp64_matches_oracle_and_primal_ridge(ctx):
    """Table 1's linear kernel (FP64 path): alpha and predictions match the
    oracle's linear fit, the predictions equal primal ridge regression
    (Eq. 2: yhat = Xt w, w = (X^T X + lambda m I)^-1 X^T y per partition), the
    condition estimates use |K|, and the other precisions are refused."""
    X, y, Xt, yt, perm, offsets = _case()
    d = X.shape[1]
    lams = [1e-3, 1e-1]
    K.krr_ctx_set_kernel(ctx, K.KRR_KERNEL_LINEAR)
    try:
        with pytest.raises(K.KrrError):
            K.krr_fit_batch(ctx, cuda(X), cuda(y), cuda(perm, torch.int64), cuda(offsets, torch.int64), [1.0], lams,
                            "tf32")
        model, status, alpha = K.krr_fit_batch(ctx, cuda(X), cuda(y), cuda(perm, torch.int64),
                                               cuda(offsets, torch.int64), [1.0], lams, "fp64", want_alpha=True)
    finally:
        K.krr_ctx_set_kernel(ctx, K.KRR_KERNEL_GAUSSIAN)
    try:
        assert np.all(status.cpu().numpy() == K.KRR_OK)
        ga = split_alpha(alpha.cpu().numpy(), offsets, 2)
        yhat = K.krr_predict(ctx, model, cuda(Xt)).cpu().numpy()
        _, kap, _ = K.krr_model_stats(ctx, model)
        for j in range(3):
            rows = perm[offsets[j]:offsets[j + 1]]
            m = len(rows)
            for g, lam in enumerate(lams):
                oa, info, rc = oracle.fit(X[rows], y[rows], 1.0, lam, oracle.KIND_LINEAR)
                assert rc == 0
                assert rel(ga[j][g], oa) <= FP64_TOL, (j, g)
                Xp = X[rows]
                w = np.linalg.solve(Xp.T @ Xp + lam * m * np.eye(d), Xp.T @ y[rows])
                assert rel(yhat[j * 2 + g], Xt @ w) <= 1e-9, (j, g)
                assert kap.numpy()[j * 2 + g] == pytest.approx(info[0], rel=1e-6)
    finally:
        model.free()


def test_routed_predict_parity(ctx):
    X, Xt, init = _mixture(1400, 300, 7, 5, 31)
    y = np.sin(X.sum(1)) + 0.05 * np.random.default_rng(1).standard_normal(1400)
    yt = np.sin(Xt.sum(1))
    assign, route, perm, offsets, centers = K.krr_partition(ctx, cuda(X), cuda(Xt), K.KRR_PART_KMEANS, 5, iters=6,
                                                            init_idx=cuda(init, torch.int64))
    operm, ooff, _, oroute, _, _ = oracle.partition_kmeans(X, Xt, 5, init, 6)
    assert np.array_equal(perm.cpu().numpy(), operm) and np.array_equal(route.cpu().numpy(), oroute)
    sig, lam = [2.0, 5.0], [1e-4]
    model, status, _ = K.krr_fit_batch(ctx, cuda(X), cuda(y), perm, offsets, sig, lam, "tf32")
    try:
        assert np.all(status.cpu().numpy() == K.KRR_OK)
        yr = K.krr_predict(ctx, model, cuda(Xt), route=route).cpu().numpy()
        al, infos, _ = oracle.fit_batch(X, y, operm, ooff, sig, lam)
        oyr = oracle.predict_all(X, operm, ooff, al, sig, lam, Xt, route=oroute)
        for g in range(2):
            assert rel(yr[g], oyr[g]) <= REFINED_TOL
        mse, best = K.krr_select(ctx, cuda(yr), cuda(yt), 5, 2, K.KRR_SEL_ROUTED)
        omse, _ = oracle.select(oyr, yt, oracle.SEL_ROUTED)
        np.testing.assert_allclose(mse.cpu().numpy(), omse, rtol=REFINED_TOL)
        # a route outside [0, p) is skipped on the device: that row predicts 0,
        # every other row exactly as before
        bad = route.clone()
        bad[[0, 7, 299]] = torch.tensor([-1, 5, 2**31 - 1], dtype=torch.int32, device="cuda")
        yb = K.krr_predict(ctx, model, cuda(Xt), route=bad).cpu().numpy()
        keep = np.ones(300, bool)
        keep[[0, 7, 299]] = False
        assert np.all(yb[:, ~keep] == 0.0)
        assert np.array_equal(yb[:, keep], yr[:, keep])
    finally:
        model.free()


def test_select_hand_values_two_partitions_two_grid_points(ctx):
    """krr_select on the hand-worked p = 2, G = 2 case of the oracle pins
    (tests/golden/select_p2_g2_hand.txt): DC-KRR averaging over partitions
    and the BKRR3 per-point choice, model index j*G + g."""
    from test_oracle_pins import _select_hand_fixture
    yhat, yt, want = _select_hand_fixture()
    for name, mode in (("per_model", K.KRR_SEL_PER_MODEL), ("average", K.KRR_SEL_AVERAGE),
                       ("oracle", K.KRR_SEL_ORACLE)):
        mse, best = K.krr_select(ctx, cuda(yhat), cuda(yt), 2, 2, mode)
        np.testing.assert_allclose(mse.cpu().numpy(), want[name][0], rtol=1e-15, atol=0)
        assert int(best.cpu()[0]) == want[name][1], name


def test_dkrr_fp64_full_size(ctx):
    """The plain DKRR workload (n = 2048, one partition) on the FP64 path."""
    w = synth.dkrr(seed=0)
    n = w["X"].shape[0]
    perm = np.arange(n, dtype=np.int64)
    off = np.array([0, n], np.int64)
    model, status, alpha = K.krr_fit_batch(ctx, cuda(w["X"]), cuda(w["y"]), cuda(perm, torch.int64),
                                           cuda(off, torch.int64), w["sigmas"], w["lambdas"], "fp64",
                                           want_alpha=True)
    try:
        assert int(status.cpu()[0]) == K.KRR_OK
        oa, info, rc = oracle.fit(w["X"], w["y"], w["sigmas"][0], w["lambdas"][0])
        assert rc == 0 and info[0] * 2.0 ** -53 <= 1e-11
        assert rel(alpha.cpu().numpy(), oa) <= FP64_TOL
        yh = K.krr_predict(ctx, model, cuda(w["Xt"])).cpu().numpy()[0]
        oyh = oracle.predict(w["X"], oa, w["Xt"], w["sigmas"][0])
        assert rel(yh, oyh) <= FP64_TOL
        mse, _ = K.krr_select(ctx, cuda(yh[None, :]), cuda(w["yt"]), 1, 1, K.KRR_SEL_PER_MODEL)
        assert abs(float(mse.cpu()[0]) - oracle.mse(oyh, w["yt"])) <= 1e-9 * oracle.mse(oyh, w["yt"])
    finally:
        model.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16x3"])
def test_bkrr2_full_size_sampled(ctx, prec):
    """The BKRR2 workload at full size (n = 65536, p = 16 x 4096, 3 sigma x 2
    lambda) in the benchmark's launch configuration; the oracle recomputes two
    of the 96 solves (the worst conditioned and a mid one) and their
    predictions on a sample of test rows."""
    w = synth.bkrr2()
    X, y, Xt, yt = w["X"], w["y"], w["Xt"], w["yt"]
    dX = cuda(X)
    assign, _, perm, offsets, _ = K.krr_partition(ctx, dX, None, K.KRR_PART_RANDOM, 16, seed=w["part_seed"])
    model, status, alpha = K.krr_fit_batch(ctx, dX, cuda(y), perm, offsets, w["sigmas"], w["lambdas"], prec,
                                           want_alpha=True)
    try:
        st = status.cpu().numpy()
        assert np.all(st == K.KRR_OK), st
        G = 6
        operm, ooff, _ = oracle.partition_random(65536, 16, w["part_seed"])
        assert np.array_equal(perm.cpu().numpy(), operm)
        galpha = split_alpha(alpha.cpu().numpy(), ooff, G)
        sample = np.random.default_rng(5).choice(Xt.shape[0], 256, replace=False)
        yhat = K.krr_predict(ctx, model, cuda(Xt[sample])).cpu().numpy()
        for j, si, li in [(0, 2, 0), (9, 1, 1)]:  # (sigma 16, lambda 1e-6) and (sigma 4, lambda 1e-4)
            rows = operm[ooff[j]:ooff[j + 1]]
            oa, info, rc = oracle.fit(X[rows], y[rows], w["sigmas"][si], w["lambdas"][li])
            g = si * 2 + li
            assert rc == 0
            # the FP64 path's 1e-10 bar holds where kappa u_64 <= 1e-11; beyond
            # it (sigma 16, lambda 1e-6: kappa ~ 1e6) the refined bar applies
            tol = tol_for(prec, info[0]) or REFINED_TOL
            assert rel(galpha[j][g], oa) <= tol, (j, g, info)
            oyh = oracle.predict(X[rows], oa, Xt[sample], w["sigmas"][si])
            assert rel(yhat[j * G + g], oyh) <= tol
            gm = np.mean((yhat[j * G + g] - yt[sample]) ** 2)
            assert abs(gm - oracle.mse(oyh, yt[sample])) <= tol * oracle.mse(oyh, yt[sample])
        if prec == "tf32":
            # one-pass solves (FP16 factor store, several panels of 8 tiles):
            # their factor must still precondition well
            it, kap, _ = K.krr_model_stats(ctx, model)
            one_pass = kap.numpy() * 2.0 ** -11 <= 32
            assert one_pass.sum() >= 48, kap.numpy()
            assert np.all(it.numpy()[one_pass] <= 10), it.numpy()[one_pass]
    finally:
        model.free()


def _reference_solve_large(X, y, sigma, lam):
    """Eq. 6 for one large partition: the oracle's FP64 kernel matrix (direct
    differences, built in row blocks on all host cores), a LAPACK Cholesky
    solve as the factor step, then FP64 refinement steps with residuals
    formed from the same matrix."""
    import concurrent.futures as cf
    import scipy.linalg as sla
    m = X.shape[0]
    A = np.empty((m, m))
    blk = 512
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        def fill(r0):
            A[r0:r0 + blk] = oracle.kernel_matrix(X[r0:r0 + blk], X, sigma)
        list(ex.map(fill, range(0, m, blk)))
    A[np.diag_indices(m)] += lam * m
    c = sla.cho_factor(A, lower=True, overwrite_a=False, check_finite=False)
    a = sla.cho_solve(c, y, check_finite=False)
    for _ in range(3):
        a = a + sla.cho_solve(c, y - A @ a, check_finite=False)
    return a, A


def test_top_of_the_condition_range(ctx):
    """One partition of n = 16384 BKRR2-shaped rows (d = 90) at sigma = 16,
    lambda = 1e-7: kappa_est ~ 1e7, the top of the serving range.  The TF32
    request escalates to the FP32-class factor, which preconditions the
    refinement; alpha and the predictions stay within 1e-6 of the reference."""
    w = synth.bkrr2(seed=31, n=16384, t=512, p=1, sigmas=(16.0,), lambdas=(1e-7,))
    X, y, Xt = w["X"], w["y"], w["Xt"]
    n = X.shape[0]
    perm = np.arange(n, dtype=np.int64)
    off = np.array([0, n], np.int64)
    model, status, alpha = K.krr_fit_batch(ctx, cuda(X), cuda(y), cuda(perm, torch.int64), cuda(off, torch.int64),
                                           [16.0], [1e-7], "tf32", want_alpha=True)
    try:
        assert int(status.cpu()[0]) == K.KRR_OK
        it, kap, res = K.krr_model_stats(ctx, model)
        assert kap[0] > 1e6, kap
        yh = K.krr_predict(ctx, model, cuda(Xt)).cpu().numpy()[0]
        ra, A = _reference_solve_large(X, y, 16.0, 1e-7)
        assert np.max(np.abs(A @ ra - y)) <= 1e-12 * (np.max(np.abs(A).sum(1)) * np.max(np.abs(ra)) + 1.0)
        del A
        assert rel(alpha.cpu().numpy(), ra) <= REFINED_TOL
        sample = np.arange(0, Xt.shape[0], 4)
        oyh = oracle.predict(X, ra, Xt[sample], 16.0)
        assert rel(yh[sample], oyh) <= REFINED_TOL
    finally:
        model.free()


def test_kkrr2_full_size_sampled(ctx):
    """The KKRR2 workload at full size (n = 262144, k = 64, 20 rounds, uneven
    partitions, 3 sigma x 2 lambda) as the benchmark runs it: partitions,
    routes and centres bit-exact against the oracle's K-means; three
    partitions (the two smallest non-empty ones and a mid-sized one) refitted
    by the oracle for the worst-conditioned and a mid model, and their routed
    predictions compared on every test row routed to them."""
    w = synth.kkrr2()
    X, y, Xt, yt = w["X"], w["y"], w["Xt"], w["yt"]
    k, iters, init = w["p"], w["iters"], w["init_idx"]
    assign, route, perm, offsets, centers = K.krr_partition(ctx, cuda(X), cuda(Xt), K.KRR_PART_KMEANS, k,
                                                            iters=iters, init_idx=cuda(init, torch.int64))
    operm, ooff, oassign, oroute, ocent, _ = oracle.partition_kmeans(X, Xt, k, init, iters)
    assert np.array_equal(assign.cpu().numpy(), oassign)
    assert np.array_equal(perm.cpu().numpy(), operm) and np.array_equal(offsets.cpu().numpy(), ooff)
    assert np.array_equal(route.cpu().numpy(), oroute)
    assert np.array_equal(centers.cpu().numpy(), ocent)
    model, status, alpha = K.krr_fit_batch(ctx, cuda(X), cuda(y), perm, offsets, w["sigmas"], w["lambdas"], "tf32",
                                           want_alpha=True)
    try:
        G = 6
        st = status.cpu().numpy()
        assert np.all(st == K.KRR_OK), np.unique(st, return_counts=True)
        yr = K.krr_predict(ctx, model, cuda(Xt), route=route).cpu().numpy()
        galpha = split_alpha(alpha.cpu().numpy(), ooff, G)
        sizes = np.diff(ooff)
        nonempty = np.nonzero(sizes > 0)[0]
        order = nonempty[np.argsort(sizes[nonempty], kind="stable")]
        mid = nonempty[np.argmin(np.abs(sizes[nonempty] - 2000))]
        for j in [int(order[0]), int(order[1]), int(mid)]:
            rows = operm[ooff[j]:ooff[j + 1]]
            test_rows = np.nonzero(oroute == j)[0]
            for si, li in [(2, 0), (1, 1)]:  # (sigma 16, lambda 1e-6), (sigma 4, lambda 1e-4)
                g = si * 2 + li
                oa, info, rc = oracle.fit(X[rows], y[rows], w["sigmas"][si], w["lambdas"][li])
                assert rc == 0
                assert rel(galpha[j][g], oa) <= REFINED_TOL, (j, g, sizes[j], info)
                if test_rows.size:
                    oyh = oracle.predict(X[rows], oa, Xt[test_rows], w["sigmas"][si])
                    assert rel(yr[g][test_rows], oyh) <= REFINED_TOL, (j, g)
    finally:
        model.free()


def test_sweep_full_size_sampled(ctx):
    """The precision-sweep workload at full size (n = 520000, p = 128
    partitions of 4062/4063 rows, heavy-tailed features) in every refined
    precision: the partition bit-exact, two solves and their predictions on a
    sample of test rows within 1e-6 of the oracle."""
    w = synth.sweep()
    X, y, Xt = w["X"], w["y"], w["Xt"]
    dX = cuda(X)
    _, _, perm, offsets, _ = K.krr_partition(ctx, dX, None, K.KRR_PART_RANDOM, 128, seed=w["part_seed"])
    operm, ooff, _ = oracle.partition_random(X.shape[0], 128, w["part_seed"])
    assert np.array_equal(perm.cpu().numpy(), operm) and np.array_equal(offsets.cpu().numpy(), ooff)
    sample = np.random.default_rng(8).choice(Xt.shape[0], 192, replace=False)
    picks = [0, 127]  # a 4063-row and a 4062-row partition
    refs = {}
    for j in picks:
        rows = operm[ooff[j]:ooff[j + 1]]
        oa, _, rc = oracle.fit(X[rows], y[rows], w["sigmas"][0], w["lambdas"][0])
        assert rc == 0
        refs[j] = (oa, oracle.predict(X[rows], oa, Xt[sample], w["sigmas"][0]))
    for prec in ("tf32", "bf16x3", "fp32"):
        model, status, alpha = K.krr_fit_batch(ctx, dX, cuda(y), perm, offsets, w["sigmas"], w["lambdas"], prec,
                                               want_alpha=True)
        try:
            assert np.all(status.cpu().numpy() == K.KRR_OK)
            galpha = split_alpha(alpha.cpu().numpy(), ooff, 1)
            yhat = K.krr_predict(ctx, model, cuda(Xt[sample])).cpu().numpy()
            for j in picks:
                assert rel(galpha[j][0], refs[j][0]) <= REFINED_TOL, (prec, j)
                assert rel(yhat[j], refs[j][1]) <= REFINED_TOL, (prec, j)
        finally:
            model.free()


# ------------------------------------------------------------------ edge cases and errors
def test_single_row_and_empty_partitions(ctx):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((130, 4))
    y = rng.standard_normal(130)
    perm = np.arange(130, dtype=np.int64)
    off = np.array([0, 1, 1, 130], np.int64)  # sizes 1, 0, 129
    model, status, alpha = K.krr_fit_batch(ctx, cuda(X), cuda(y), cuda(perm, torch.int64), cuda(off, torch.int64),
                                           [1.5], [1e-3], "tf32", want_alpha=True)
    try:
        st = status.cpu().numpy()
        assert st[0] == K.KRR_OK and st[2] == K.KRR_OK
        a = alpha.cpu().numpy()
        assert abs(a[0] - y[0] / (1 + 1e-3)) <= 1e-15 * abs(y[0])
        oa, _, _ = oracle.fit(X[1:], y[1:], 1.5, 1e-3)
        assert rel(a[1:], oa) <= REFINED_TOL
        Xt = rng.standard_normal((70, 4))
        yh = K.krr_predict(ctx, model, cuda(Xt)).cpu().numpy()
        assert np.all(yh[1] == 0.0)  # the empty partition predicts 0
        assert rel(yh[2], oracle.predict(X[1:], oa, Xt, 1.5)) <= REFINED_TOL
    finally:
        model.free()


@pytest.mark.parametrize("d", [20, 100])  # exact slice-Gram kernel; double-float fallback (d > 96)
@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_far_test_rows_keep_relative_accuracy(ctx, d, prec):
    """Test rows far from every training row at a small sigma: their Eq. 7
    sums (~e^-300) lie far below the FP32 exponent range of the double-float
    exponential, yet each must match the oracle to 1e-6 relative, row by row;
    near rows in the same launch keep their accuracy too."""
    rng = np.random.default_rng(17)
    n, sigma, lam = 300, 0.5, 1e-3
    X = rng.standard_normal((n, d))
    y = rng.standard_normal(n)
    src = rng.integers(0, n, 96)
    push = np.sqrt(np.linspace(2.0, 280.0, 96) / d)  # squared distance to the source row: 2 .. 280
    dirs = rng.standard_normal((96, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    Xt = X[src] + dirs * push[:, None] * np.sqrt(d)
    perm = np.arange(n, dtype=np.int64)
    off = np.array([0, 140, n], np.int64)  # two partitions: the shift is per (row, partition)
    model, status, alpha = K.krr_fit_batch(ctx, cuda(X), cuda(y), cuda(perm, torch.int64), cuda(off, torch.int64),
                                           [sigma], [lam], prec, want_alpha=True)
    try:
        assert np.all(status.cpu().numpy() == K.KRR_OK)
        a = alpha.cpu().numpy()
        yh = K.krr_predict(ctx, model, cuda(Xt)).cpu().numpy()
        for j in range(2):
            Xj, aj = X[off[j]:off[j + 1]], a[off[j]:off[j + 1]]
            ref = oracle.predict(Xj, aj, Xt, sigma)
            live = np.abs(ref) > 1e-290  # away from FP64 subnormals
            assert live.sum() > 20 and np.min(np.abs(ref[live])) < 1e-100
            err = np.abs(yh[j][live] - ref[live]) / np.abs(ref[live])
            assert err.max() <= REFINED_TOL, "partition %d: worst row rel err %.3e" % (j, err.max())
            assert np.all(yh[j][~live] == 0.0) or np.max(np.abs(yh[j][~live])) < 1e-280
    finally:
        model.free()


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_indefinite_system_is_reported_per_solve(ctx, prec):
    """A negative shift makes K + lambda m I indefinite: that solve reports
    NOT_SPD (or NO_CONVERGE), the batch itself succeeds."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((200, 3)) * 0.01  # nearly identical rows: K ~ 1 1^T, eigenvalues ~ 0
    y = rng.standard_normal(200)
    perm = np.arange(200, dtype=np.int64)
    off = np.array([0, 200], np.int64)
    model, status, _ = K.krr_fit_batch(ctx, cuda(X), cuda(y), cuda(perm, torch.int64), cuda(off, torch.int64),
                                       [1.0], [-0.5 / 200, 1e-2], prec)
    try:
        st = status.cpu().numpy()
        assert st[0] in (K.KRR_ERR_NOT_SPD, K.KRR_ERR_NO_CONVERGE), st
        assert st[1] == K.KRR_OK
    finally:
        model.free()


def test_budget_and_argument_errors(ctx):
    rng = np.random.default_rng(5)
    X = cuda(rng.standard_normal((600, 5)))
    y = cuda(rng.standard_normal(600))
    perm = cuda(np.arange(600), torch.int64)
    off = cuda(np.array([0, 600]), torch.int64)
    small = K.krr_ctx_create(0, hbm_budget_bytes=1 << 20)
    with pytest.raises(K.KrrError) as e:
        K.krr_fit_batch(small, X, y, perm, off, [1.0], [1e-3], "tf32")
    assert e.value.status == K.KRR_ERR_BUDGET
    assert small.bytes_in_use() == 0
    small.close()
    with pytest.raises(K.KrrError) as e:
        K.krr_fit_batch(ctx, X, y, perm, off, [0.0], [1e-3], "tf32")
    assert e.value.status == K.KRR_ERR_ARG
    for bad_off in ([0, 601], [1, 600], [0, 400, 300]):  # beyond n, not from 0, decreasing
        bad = cuda(np.array(bad_off), torch.int64)
        with pytest.raises(K.KrrError) as e:
            K.krr_fit_batch(ctx, X, y, perm, bad, [1.0], [1e-3], "tf32")
        assert e.value.status == K.KRR_ERR_ARG
    with pytest.raises(K.KrrError) as e:
        K.krr_partition(ctx, X, None, K.KRR_PART_RANDOM, 0)
    assert e.value.status == K.KRR_ERR_ARG


def test_kmeans_steps_and_partition_subset_fit(ctx):
    """The multi-process building blocks on one GPU: Alg. 2 driven through
    krr_kmeans_assign / krr_kmeans_block_sums / krr_kmeans_combine (the
    per-round exchange of the sharded K-means, here with one rank) gives the
    centres and assignments of krr_partition(KMEANS) bit for bit; and a fit of
    a subset of the partitions against the full X (as a rank fits the ones
    LPT gave it) gives those partitions' alphas of the full fit."""
    from paper_1805_00569_gb300 import dist as kd
    n, t, d, k, iters = 5000, 300, 11, 7, 6
    X, Xt, init = _mixture(n, t, d, k, 5)
    dX = cuda(X)
    assign, route, perm, offsets, centers = K.krr_partition(ctx, dX, cuda(Xt), K.KRR_PART_KMEANS, k, iters=iters,
                                                            init_idx=cuda(init, torch.int64))
    C, a = kd.kmeans_sharded(kd.gpu_kmeans_ops(ctx), dX, dX[cuda(init, torch.int64)].clone(), iters)
    assert torch.equal(a, assign)
    assert np.array_equal(C.cpu().numpy().view(np.uint64), centers.cpu().numpy().view(np.uint64))
    y = np.sin(X[:, 0]) + 0.1 * X[:, 1]
    sig, lam = [3.0], [1e-4]
    full, st, al_full = K.krr_fit_batch(ctx, dX, cuda(y), perm, offsets, sig, lam, "fp64", want_alpha=True)
    owned = kd.lpt_assign(np.diff(offsets.cpu().numpy()) ** 3, 2)[1]
    sub, soff = kd.partition_subset(perm, offsets.cpu(), owned)
    part, st2, al_sub = K.krr_fit_batch(ctx, dX, cuda(y), sub, soff.cuda(), sig, lam, "fp64", want_alpha=True)
    try:
        assert np.all(st.cpu().numpy() == K.KRR_OK) and np.all(st2.cpu().numpy() == K.KRR_OK)
        off = offsets.cpu().numpy()
        so = soff.cpu().numpy()
        af, asb = al_full.cpu().numpy(), al_sub.cpu().numpy()
        for i, j in enumerate(owned):
            assert np.array_equal(asb[so[i]:so[i + 1]], af[off[j]:off[j + 1]])
        yf = K.krr_predict(ctx, full, cuda(Xt)).cpu().numpy()
        ys = K.krr_predict(ctx, part, cuda(Xt)).cpu().numpy()
        for i, j in enumerate(owned):
            assert np.array_equal(ys[i], yf[j])
    finally:
        full.free()
        part.free()


def _serve_request_5943():
    """Request 5943 of the serving stream (seed 4): n = 589, d = 8,
    sigma ~ 12, lambda ~ 1.4e-7 (kappa_est ~ 5e6), rows as the benchmark's
    stream draws them (row prefix of its feature count's mixture bank)."""
    st = synth.serve_stream(seed=4, requests=10000)
    i = 5943
    n, d = int(st["n"][i]), int(st["d"][i])
    b = int(st["data_seed"][i] % 32)
    src = synth.serve_request_data(1000003 * d + b, int(max(st["n"])), d, 256)
    return src["X"][:n], src["y"][:n], src["Xt"], float(st["sigma"][i]), float(st["lam"][i])


def test_fp64_fallback_for_an_unconverged_solve():
    """A served request whose FP32-class factor broke down (the shifted
    refactorisation then preconditions too poorly for the refinement to
    converge in 80 iterations) is solved again on the plain FP64 path: status
    OK, factor class 0, alpha and predictions within the refined bar."""
    X, y, Xt, sigma, lam = _serve_request_5943()
    n = X.shape[0]
    perm = cuda(np.arange(n, dtype=np.int64), torch.int64)
    off = cuda(np.array([0, n], np.int64), torch.int64)
    out = {}
    for on in (False, True):
        c = K.krr_ctx_create(0)
        K.krr_ctx_set_panel_width(c, 8)
        K.krr_ctx_set_fp64_fallback(c, on)
        model, status, alpha = K.krr_fit_batch(c, cuda(X), cuda(y), perm, off, [sigma], [lam], "tf32",
                                               want_alpha=True)
        out[on] = (int(status.cpu()[0]), int(K.krr_model_factor_class(c, model)[0]), alpha.cpu().numpy(),
                   K.krr_predict(c, model, cuda(Xt)).cpu().numpy()[0])
        model.free()
        c.close()
    st_on, cls_on, a_on, y_on = out[True]
    assert st_on == K.KRR_OK
    if out[False][0] == K.KRR_ERR_NO_CONVERGE:
        assert cls_on == 0
    oa, info, rc = oracle.fit(X, y, sigma, lam)
    assert rc == 0 and info[0] > 1e6
    assert rel(a_on, oa) <= REFINED_TOL
    assert rel(y_on, oracle.predict(X, oa, Xt, sigma)) <= REFINED_TOL


def test_fit_jobs_packs_independent_problems():
    """krr_fit_jobs: five independent problems of uneven sizes (a one-row one
    included), each with its own sigma and lambda, in one batched fit; each
    alpha and each routed prediction within the refined bar of the oracle's
    solve of that problem alone, and the same bits as fitting it alone."""
    rng = np.random.default_rng(71)
    d = 20
    sizes = [300, 1000, 129, 2000, 1]
    sig = [0.7, 3.0, 12.0, 5.0, 2.0]
    lam = [1e-3, 1e-6, 1e-4, 1e-7, 1e-2]
    Xs = [rng.standard_normal((m, d)) * 1.5 for m in sizes]
    ys = [np.sin(Xj[:, 0]) + 0.1 * Xj[:, 1] for Xj in Xs]
    Xts = [rng.standard_normal((37, d)) * 1.5 for _ in sizes]
    X, y, Xt = np.concatenate(Xs), np.concatenate(ys), np.concatenate(Xts)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    route = np.repeat(np.arange(len(sizes)), 37).astype(np.int32)
    c = K.krr_ctx_create(0)
    K.krr_ctx_set_panel_width(c, 8)
    try:
        model, st, al = K.krr_fit_jobs(c, cuda(X), cuda(y), cuda(np.arange(X.shape[0]), torch.int64),
                                       cuda(off, torch.int64), sig, lam, "tf32", want_alpha=True)
        assert np.all(st.cpu().numpy() == K.KRR_OK)
        yh = K.krr_predict(c, model, cuda(Xt), route=cuda(route, torch.int32)).cpu().numpy()[0]
        al = al.cpu().numpy()
        model.free()
        for j, m in enumerate(sizes):
            oa, info, rc = oracle.fit(Xs[j], ys[j], sig[j], lam[j])
            assert rc == 0
            assert rel(al[off[j]:off[j + 1]], oa) <= REFINED_TOL, j
            assert rel(yh[37 * j:37 * (j + 1)], oracle.predict(Xs[j], oa, Xts[j], sig[j])) <= REFINED_TOL, j
            alone, st1, a1 = K.krr_fit_jobs(c, cuda(Xs[j]), cuda(ys[j]), cuda(np.arange(m), torch.int64),
                                            cuda(np.array([0, m]), torch.int64), [sig[j]], [lam[j]], "tf32",
                                            want_alpha=True)
            y1 = K.krr_predict(c, alone, cuda(Xts[j]), route=cuda(np.zeros(37, np.int32), torch.int32))
            assert np.array_equal(a1.cpu().numpy(), al[off[j]:off[j + 1]]), j
            assert np.array_equal(y1.cpu().numpy()[0], yh[37 * j:37 * (j + 1)]), j
            alone.free()
        with pytest.raises(K.KrrError) as e:
            K.krr_fit_jobs(c, cuda(X), cuda(y), cuda(np.arange(X.shape[0]), torch.int64), cuda(off, torch.int64),
                           sig, lam, "fp64")
        assert e.value.status == K.KRR_ERR_UNSUPPORTED
    finally:
        c.close()
