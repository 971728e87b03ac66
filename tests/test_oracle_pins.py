"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, brute force, invariants, published test vectors).  None of
these checks re-types an oracle formula; each would fail for a dropped term,
a wrong sign or index, or a transposed operand in the oracle."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------- generator pins
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors."""
    rows = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(v, 16) for v in line.split()]
            out = oracle.philox4x32_10(w[0:4], w[4:6])
            assert [int(v) for v in out] == w[6:10]
            rows += 1
    assert rows == 3


@pytest.mark.parametrize("n,p", [(1, 1), (2, 1), (17, 4), (1000, 7), (4096, 16), (65, 64)])
def test_random_partition_is_even_bijection(n, p):
    """The partitioning of Alg. DC-KRR: a shuffle (a bijection) cut into p even parts,
    the larger parts first."""
    perm, offsets, assign = oracle.partition_random(n, p, 99)
    assert np.array_equal(np.sort(perm), np.arange(n))
    sizes = np.diff(offsets)
    assert sizes.sum() == n and sizes.max() - sizes.min() <= 1
    assert np.all(np.diff(sizes) <= 0)
    for j in range(p):
        assert np.all(assign[perm[offsets[j]:offsets[j + 1]]] == j)


def test_random_partition_depends_on_seed():
    a, _, _ = oracle.partition_random(500, 4, 1)
    b, _, _ = oracle.partition_random(500, 4, 2)
    assert not np.array_equal(a, b)
    c, _, _ = oracle.partition_random(500, 4, 1)
    assert np.array_equal(a, c)


# ----------------------------------------------------------- kernel pins
def test_gaussian_kernel_hand_values():
    """Table 1 Gaussian kernel against hand-computed values."""
    with open(os.path.join(GOLDEN, "gaussian_kernel_hand.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            s, a, b, v = [f.strip() for f in line.split("|")]
            A = np.array([[float(x) for x in a.split(",")]])
            B = np.array([[float(x) for x in b.split(",")]])
            K = oracle.kernel_matrix(A, B, float(s))
            assert abs(K[0, 0] - float(v)) <= 2e-16 * max(1.0, float(v))


def test_linear_kernel_hand_value():
    A = np.array([[1.0, 2.0, 3.0]])
    B = np.array([[4.0, -5.0, 6.0]])
    assert oracle.kernel_matrix(A, B, 1.0, oracle.KIND_LINEAR)[0, 0] == 12.0


def test_kernel_matrix_structure():
    """K symmetric, unit diagonal, entries in (0, 1]."""
    rng = np.random.default_rng(0)
    X = rng.standard_normal((40, 7))
    K = oracle.kernel_matrix(X, X, 1.7)
    assert np.array_equal(K, K.T)
    assert np.all(np.diag(K) == 1.0)
    assert np.all(K > 0) and np.all(K <= 1.0)
    # direct-difference brute force in exact rational arithmetic of the squared distance
    i, j = 3, 17
    dd = math.fsum((float(a) - float(b)) ** 2 for a, b in zip(X[i], X[j]))
    assert abs(K[i, j] - math.exp(-dd / (2 * 1.7 ** 2))) <= 1e-15


# ----------------------------------------------------------- solve pins
def _data(m, d, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, d))
    y = np.sin(X[:, 0]) + 0.1 * rng.standard_normal(m)
    return X, y


@pytest.mark.parametrize("m,sigma,lam", [(8, 1.0, 1e-3), (33, 2.0, 1e-4), (64, 3.0, 1e-2)])
def test_solve_matches_high_precision_inverse(m, sigma, lam):
    """Eq. 6 against an explicit inverse in 40-digit arithmetic (m <= 64)."""
    mpmath = pytest.importorskip("mpmath")
    X, y = _data(m, 5, m)
    alpha, info, rc = oracle.fit(X, y, sigma, lam)
    assert rc == 0
    K = oracle.kernel_matrix(X, X, sigma)
    mpmath.mp.dps = 40
    A = mpmath.matrix(K.tolist())
    for i in range(m):
        A[i, i] += mpmath.mpf(lam) * m
    exact = (A ** -1) * mpmath.matrix(y.tolist())
    exact = np.array([float(v) for v in exact])
    assert np.max(np.abs(alpha - exact)) <= 1e-13 * np.max(np.abs(exact))


def test_sigma_to_zero_closed_form():
    """sigma -> 0: off-diagonal kernel entries underflow to 0, so K = I and
    alpha = y / (1 + lambda m); predictions of unseen points vanish."""
    X, y = _data(50, 5, 3)
    lam = 1e-3
    alpha, _, rc = oracle.fit(X, y, 1e-3, lam)
    assert rc == 0
    np.testing.assert_allclose(alpha, y / (1 + lam * 50), rtol=1e-15, atol=0)
    Xt = np.random.default_rng(9).standard_normal((5, 5))
    assert np.all(oracle.predict(X, alpha, Xt, 1e-3) == 0.0)


def test_sigma_to_infinity_sherman_morrison():
    """sigma -> inf: K -> 1 1^T and (1 1^T + c I) alpha = y has the
    Sherman-Morrison solution alpha = (y - 1 (1^T y) / (c + m)) / c, c = lambda m."""
    m, lam = 40, 0.05
    X, y = _data(m, 4, 5)
    alpha, _, rc = oracle.fit(X, y, 1e6, lam)
    assert rc == 0
    c = lam * m
    sm = (y - np.sum(y) / (c + m)) / c
    np.testing.assert_allclose(alpha, sm, rtol=0, atol=1e-8 * np.abs(sm).max())


def test_linear_kernel_equals_primal_ridge():
    """Linear kernel (Table 1) KRR predictions equal the ridge regression
    (Eq. 2) closed form xhat^T (X^T X + lambda m I_d)^{-1} X^T y."""
    m, d, lam = 120, 6, 1e-2
    X, y = _data(m, d, 11)
    Xt = np.random.default_rng(12).standard_normal((9, d))
    alpha, _, rc = oracle.fit(X, y, 1.0, lam, oracle.KIND_LINEAR)
    assert rc == 0
    yh = oracle.predict(X, alpha, Xt, 1.0, oracle.KIND_LINEAR)
    w = np.linalg.solve(X.T @ X + lam * m * np.eye(d), X.T @ y)
    np.testing.assert_allclose(yh, Xt @ w, rtol=1e-10, atol=1e-12)


def test_residual_and_library_cross_check():
    """Backward error <= 1e-12 and agreement with scipy's Cholesky solve."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    X, y = _data(300, 8, 21)
    sigma, lam = 2.5, 1e-5
    alpha, info, rc = oracle.fit(X, y, sigma, lam)
    assert rc == 0
    A = oracle.kernel_matrix(X, X, sigma) + lam * 300 * np.eye(300)
    r = A @ alpha - y
    assert np.abs(r).max() <= 1e-12 * (np.abs(A).sum(1).max() * np.abs(alpha).max() + np.abs(y).max())
    ref = scipy_linalg.cho_solve(scipy_linalg.cho_factor(A, lower=True), y)
    kappa = np.linalg.cond(A)
    assert np.abs(alpha - ref).max() <= 1e-15 * kappa * np.abs(ref).max() * 10
    assert info[0] >= kappa * 0.999  # Gershgorin estimate bounds kappa from above


def test_not_spd_reported():
    """A negative shift makes K + lambda m I indefinite: the solve reports it."""
    X, y = _data(20, 3, 2)
    _, _, rc = oracle.fit(X, y, 1e-3, -2.0 / 20)
    assert rc == 1


def test_single_row_partition():
    X = np.array([[0.3, -0.2]])
    y = np.array([2.0])
    alpha, _, rc = oracle.fit(X, y, 1.0, 0.5)
    assert rc == 0 and abs(alpha[0] - 2.0 / 1.5) < 1e-16


# ----------------------------------------------------------- predict / MSE pins
def test_mse_hand_value():
    assert oracle.mse(np.array([1.0, 2.0, 3.0]), np.array([1.0, 1.0, 1.0])) == 5.0 / 3.0


def test_predict_on_training_rows_reproduces_fit():
    """Eq. 7 at the training rows gives K alpha = y - lambda m alpha."""
    X, y = _data(60, 4, 8)
    lam = 1e-3
    alpha, _, _ = oracle.fit(X, y, 1.5, lam)
    yh = oracle.predict(X, alpha, X, 1.5)
    np.testing.assert_allclose(yh, y - lam * 60 * alpha, rtol=0, atol=1e-12)


# ----------------------------------------------------------- K-means pins
def test_assign_brute_force_and_ties():
    """Alg. 2 step 4: the nearest centre; exact ties go to the lower index."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((500, 6))
    C = rng.standard_normal((9, 6))
    got = oracle.assign(X, C)
    dist = ((X[:, None, :] - C[None, :, :]) ** 2).sum(-1)
    assert np.array_equal(got, np.argmin(dist, axis=1))
    # exact ties: centres at (+-1, 0), points on the perpendicular bisector
    C2 = np.array([[1.0, 0.0], [-1.0, 0.0], [1.0, 0.0]])
    P = np.array([[0.0, 0.5], [0.0, -3.0], [2.0, 0.0]])
    assert list(oracle.assign(P, C2)) == [0, 0, 0]
    C3 = np.array([[5.0, 5.0], [-1.0, 0.0], [1.0, 0.0]])
    assert list(oracle.assign(P, C3)) == [1, 1, 2]


def test_kmeans_objective_non_increasing_and_fixed_point():
    rng = np.random.default_rng(5)
    X = np.concatenate([rng.standard_normal((300, 3)) + 6 * rng.standard_normal(3) for _ in range(5)])
    init = rng.choice(len(X), 5, replace=False)
    prev = np.inf
    for r in range(1, 8):
        C, c, delta = oracle.kmeans(X, 5, init, r)
        obj = ((X - C[c]) ** 2).sum()
        assert obj <= prev * (1 + 1e-12)
        prev = obj
        dist = ((X[:, None, :] - C[None, :, :]) ** 2).sum(-1)
        assert np.array_equal(c, np.argmin(dist, axis=1))
    assert delta[0] == len(X)  # first round: every point is new


def test_kmeans_single_cluster_is_mean():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((3000, 4)) * 10
    C, c, delta = oracle.kmeans(X, 1, [17], 3)
    exact = np.array([math.fsum(X[:, f]) / 3000 for f in range(4)])
    np.testing.assert_allclose(C[0], exact, rtol=1e-14, atol=1e-14)
    assert np.all(c == 0) and list(delta) == [3000, 0]


def test_centre_sum_order_is_the_canonical_block_tree():
    """The centre step's summation order decides bit-exactness (the order the
    paper leaves open, Alg. 2 centre step): rows in blocks of 1024, each block
    summed in ascending row order, block sums combined pairwise in block order.
    Hand-worked case, one cluster, 3000 rows, feature 0:
      block 0 = [2^53, 1 x 1023]: 2^53 + 1 ties to even, so s0 = 2^53;
      block 1 = [1 x 1024]: s1 = 1024;  block 2 = [-2^53, 0 x 951]: s2 = -2^53;
      (s0 + s1) + s2 = 1024, while the exact sum is 2047 and a single
      ascending pass gives 0.  Feature 1 (rows of cluster 1 only, every
      other row) checks that a block sums only its own cluster's rows."""
    n = 3000
    X = np.zeros((n, 2))
    X[0, 0] = 2.0**53
    X[1:2048, 0] = 1.0
    X[2048, 0] = -(2.0**53)
    c = np.zeros(n, np.int32)
    c[1::2] = 1
    X[1::2, 1] = 3.0  # cluster 1: 1500 rows of 3 in feature 1
    C = oracle.update_centres(X, c, np.zeros((2, 2)))
    # cluster 0 (even rows): block 0 = 2^53 + 511 ones -> 2^53; block 1: 512 ones;
    # block 2: -2^53 (row 2048 is even) -> (2^53 + 512) - 2^53 = 512, over 1500 rows
    assert C[0, 0] == 512.0 / 1500.0
    # cluster 1 (odd rows): 512 + 512 ones in blocks 0 and 1, row 2049 onwards zeros
    assert C[1, 0] == 1024.0 / 1500.0
    assert C[1, 1] == 3.0 and C[0, 1] == 0.0
    C1 = oracle.update_centres(X, np.zeros(n, np.int32), np.zeros((1, 2)))
    assert C1[0, 0] == 1024.0 / 3000.0


def test_kmeans_empty_cluster_keeps_centre():
    X = np.array([[0.0], [0.1], [0.2], [10.0]])
    C0 = np.array([[0.0], [10.0], [100.0]])
    C = oracle.update_centres(X, np.array([0, 0, 0, 1], np.int32), C0)
    assert C[2, 0] == 100.0 and C[1, 0] == 10.0
    assert abs(C[0, 0] - 0.1) < 1e-16


def test_gather_stable():
    rng = np.random.default_rng(7)
    a = rng.integers(0, 6, 777).astype(np.int32)
    perm, offsets = oracle.gather_stable(a, 6)
    assert np.array_equal(perm, np.argsort(a, kind="stable"))
    assert np.array_equal(np.diff(offsets), np.bincount(a, minlength=6))


# ----------------------------------------------------------- selection pins
def test_select_hand_values_and_ties():
    yt = np.array([0.0, 0.0])
    yhat = np.array([[1.0, 1.0], [0.0, 1.0], [1.0, 0.0], [2.0, 0.0]])
    mses, best = oracle.select(yhat, yt, oracle.SEL_PER_MODEL)
    assert list(mses) == [1.0, 0.5, 0.5, 2.0] and best == 1


def _select_hand_fixture():
    """tests/golden/select_p2_g2_hand.txt: yhat rows, labels, and the
    hand-worked MSEs (as fractions) and best index of each mode."""
    from fractions import Fraction
    rows, yt, want = [], None, {}
    with open(os.path.join(GOLDEN, "select_p2_g2_hand.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            parts = [x.strip() for x in line.split("|")]
            if parts[0] == "yt":
                yt = np.array([float(v) for v in parts[1].split(",")])
            elif parts[0].startswith("model"):
                rows.append([float(v) for v in parts[1].split(",")])
            else:
                vals = [float(Fraction(v)) for v in parts[1].split(",")]
                want[parts[0]] = (np.array(vals), int(parts[2].split()[1]))
    return np.array(rows), yt, want


def test_select_hand_values_two_partitions_two_grid_points():
    """p = 2, G = 2: the DC-KRR average (Alg. DC-KRR) divides by p and the
    BKRR3 choice (Alg. BKRR3) takes models j*G + g; hand-worked values."""
    yhat, yt, want = _select_hand_fixture()
    for name, mode in (("per_model", oracle.SEL_PER_MODEL), ("average", oracle.SEL_AVERAGE),
                       ("oracle", oracle.SEL_ORACLE)):
        mses, best = oracle.select(yhat, yt, mode, 2, 2)
        np.testing.assert_allclose(mses, want[name][0], rtol=1e-15, atol=0)
        assert best == want[name][1], name


def test_single_partition_modes_agree_with_dkrr():
    """p = 1: random, K-means, routed, per-model and averaged selection all
    reduce to Alg. 1 (DKRR)."""
    rng = np.random.default_rng(8)
    X = rng.standard_normal((80, 3))
    y = np.cos(X[:, 0])
    Xt = rng.standard_normal((20, 3))
    yt = np.cos(Xt[:, 0])
    sig, lams = [1.0, 2.0], [1e-3]
    a_dkrr = [oracle.fit(X, y, s, lams[0])[0] for s in sig]
    ref = [oracle.mse(oracle.predict(X, a, Xt, s), yt) for a, s in zip(a_dkrr, sig)]
    perm, off, _ = oracle.partition_random(80, 1, 5)
    al, _, _ = oracle.fit_batch(X, y, np.sort(perm), off, sig, lams)
    yh = oracle.predict_all(X, np.sort(perm), off, al, sig, lams, Xt)
    for mode in (oracle.SEL_PER_MODEL, oracle.SEL_AVERAGE, oracle.SEL_ORACLE):
        mses, best = oracle.select(yh, yt, mode, 1, 2)
        np.testing.assert_allclose(mses, ref, rtol=1e-12)
    yr = oracle.predict_all(X, np.sort(perm), off, al, sig, lams, Xt, route=np.zeros(20, np.int32))
    mses, _ = oracle.select(yr, yt, oracle.SEL_ROUTED)
    np.testing.assert_allclose(mses, ref, rtol=1e-12)


def test_bkrr3_lower_bound():
    """The per-point best model (BKRR3) never scores worse than routing or
    than any single partition's model."""
    rng = np.random.default_rng(10)
    X = rng.standard_normal((240, 3)) * 2
    y = np.sin(X.sum(1))
    Xt = rng.standard_normal((50, 3)) * 2
    yt = np.sin(Xt.sum(1))
    C, c, _ = oracle.kmeans(X, 4, [0, 1, 2, 3], 10)
    perm, off = oracle.gather_stable(c, 4)
    route = oracle.assign(Xt, C)
    sig, lams = [1.0], [1e-3]
    al, _, _ = oracle.fit_batch(X, y, perm, off, sig, lams)
    yall = oracle.predict_all(X, perm, off, al, sig, lams, Xt)
    yr = oracle.predict_all(X, perm, off, al, sig, lams, Xt, route=route)
    m3, _ = oracle.select(yall, yt, oracle.SEL_ORACLE, 4, 1)
    m2, _ = oracle.select(yr, yt, oracle.SEL_ROUTED)
    mp, _ = oracle.select(yall, yt, oracle.SEL_PER_MODEL)
    assert m3[0] <= m2[0] and m3[0] <= mp.min()


# ---------------------------------------------------------------- K-balance
def _kbalance_listing(X, C, cap):
    """The K-balance listing transcribed literally (Euclidean distances with
    the square root, mindis / minind, the count test against the cap), for
    brute-force comparison on small inputs."""
    n, p = X.shape[0], C.shape[0]
    cs = [0] * p
    out = []
    for i in range(n):
        mindis, minind = math.inf, None
        for j in range(p):
            dist = math.sqrt(sum((float(a) - float(b)) ** 2 for a, b in zip(X[i], C[j])))
            if dist < mindis and cs[j] < cap:
                mindis, minind = dist, j
        cs[minind] += 1
        out.append(minind)
    return np.array(out, np.int32), np.array(cs, np.int64)


@pytest.mark.parametrize("n,p,d,seed", [(40, 3, 2, 1), (97, 7, 5, 2), (64, 8, 3, 3), (33, 1, 4, 4)])
def test_kbalance_matches_the_listing_brute_force(n, p, d, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    C = rng.standard_normal((p, d)) * 0.5
    cap = -(-n // p)
    c, cs = oracle.kbalance_assign(X, C, cap)
    bc, bcs = _kbalance_listing(X, C, cap)
    assert np.array_equal(c, bc) and np.array_equal(cs, bcs)
    assert cs.sum() == n and cs.max() <= cap
    if n % p == 0:
        assert np.all(cs == n // p)  # p caps of n / p hold exactly n samples


def test_kbalance_greedy_invariant():
    """Every sample sits at its nearest centre among those still open when it
    was placed: any strictly nearer centre had already reached the cap."""
    rng = np.random.default_rng(11)
    X = rng.standard_normal((500, 4))
    C = rng.standard_normal((6, 4))
    cap = -(-500 // 6)
    c, _ = oracle.kbalance_assign(X, C, cap)
    D = ((X[:, None, :] - C[None, :, :]) ** 2).sum(-1)
    filled = np.zeros(6, np.int64)
    for i in range(500):
        for j in range(6):
            if D[i, j] < D[i, c[i]]:
                assert filled[j] == cap, (i, j)
        filled[c[i]] += 1


def test_kbalance_equals_nearest_centre_when_nothing_fills():
    """Well separated clusters of at most cap samples: no centre ever fills,
    so the balanced loop is the plain assignment step (Alg. 2)."""
    rng = np.random.default_rng(5)
    centres = np.array([[0.0, 0.0], [50.0, 0.0], [0.0, 50.0], [50.0, 50.0]])
    X = np.concatenate([c + rng.standard_normal((25, 2)) for c in centres])[rng.permutation(100)]
    c, cs = oracle.kbalance_assign(X, centres, 25)
    assert np.array_equal(c, oracle.assign(X, centres))
    assert np.all(cs == 25)


def test_partition_kbalance_parts_and_routes():
    rng = np.random.default_rng(9)
    X = np.concatenate([rng.standard_normal((70, 3)) + 6 * k for k in range(3)])
    Xt = rng.standard_normal((20, 3)) * 6
    perm, offsets, c, route, C2, cs = oracle.partition_kbalance(X, Xt, 4, np.array([0, 70, 140, 5]), 5)
    sizes = np.diff(offsets)
    assert sizes.sum() == 210 and sizes.max() <= 53 and np.array_equal(sizes, cs)
    for j in range(4):
        rows = perm[offsets[j]:offsets[j + 1]]
        assert np.all(c[rows] == j) and np.all(np.diff(rows) > 0)
        if len(rows):
            np.testing.assert_allclose(C2[j], X[rows].mean(0), rtol=1e-12, atol=1e-12)
    assert np.array_equal(route, oracle.assign(Xt, C2))
