"""CPU check of the round structure the GPU uses to replay Alg. K-balance
Clustering exactly: every unplaced row takes its nearest open centre, the
first row that would overflow its centre ends the round, the rows before it
are placed and every full centre closes.  A numpy model of those rounds
(the same steps as the kernels, in numpy) must reproduce the oracle's
sequential loop, including rounds in which several centres fill at once."""
import numpy as np
import pytest

import oracle


def _rounds(D, cap):
    n, p = D.shape
    open_ = np.ones(p, bool)
    cs = np.zeros(p, np.int64)
    choice = np.zeros(n, np.int64)
    assign = np.full(n, -1)
    start, rounds = 0, 0
    while start < n:
        redo = np.arange(start, n) if rounds == 0 else np.arange(start, n)[~open_[choice[start:]]]
        for i in redo:
            Dm = np.where(open_, D[i], np.inf)
            choice[i] = int(np.flatnonzero(open_)[0]) if not np.isfinite(Dm.min()) else int(np.argmin(Dm))
        stop = n
        for j in np.flatnonzero(open_):  # the (rem_j + 1)-th row of the round choosing j
            hits = np.flatnonzero(choice[start:] == j)
            rem = cap - cs[j]
            if len(hits) > rem:
                stop = min(stop, start + int(hits[rem]))
        assert stop > start
        assign[start:stop] = choice[start:stop]
        np.add.at(cs, choice[start:stop], 1)
        open_ &= cs < cap
        start = stop
        rounds += 1
    return assign, cs, rounds


@pytest.mark.parametrize("n,p,d,seed", [(600, 7, 5, 1), (512, 16, 3, 2), (1000, 32, 2, 5), (37, 37, 2, 6),
                                        (300, 1, 3, 7)])
def test_round_replay_equals_the_sequential_loop(n, p, d, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    C = rng.standard_normal((p, d)) * 0.3
    cap = -(-n // p)
    D = ((X[:, None, :] - C[None, :, :]) ** 2).sum(-1)
    a, cs, rounds = _rounds(D, cap)
    oa, ocs = oracle.kbalance_assign(X, C, cap)
    assert np.array_equal(a, oa) and np.array_equal(cs, ocs)
    assert rounds <= p
