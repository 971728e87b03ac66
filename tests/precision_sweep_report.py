"""Precision sweep report: error of every factor precision against the FP64
oracle, per partition, on the sweep workload (520000 rows, p = 128 random
partitions of 4062/4063 rows, Student-t(5) features, sigma 4, lambda 1e-4).

Needs a GPU: python tests/precision_sweep_report.py [partitions]
Prints one markdown table row per (precision, sampled partition) with the
max-norm relative error of alpha and of the predictions of 256 sampled test
rows, the refinement iterations and the solve status."""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _oracle(args):
    Xp, yp, Xt, sigma, lam = args
    import oracle
    a, info, rc = oracle.fit(Xp, yp, sigma, lam)
    return a, oracle.predict(Xp, a, Xt, sigma), rc


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def main():
    npart = int(sys.argv[1]) if len(sys.argv) > 1 else 8
    import oracle
    from paper_1805_00569_gb300 import synth
    oracle.build()
    w = synth.sweep()
    X, y, Xt = w["X"], w["y"], w["Xt"]
    sigma, lam = w["sigmas"][0], w["lambdas"][0]
    operm, ooff, _ = oracle.partition_random(X.shape[0], w["p"], w["part_seed"])
    picks = np.linspace(0, w["p"] - 1, npart).astype(int)
    sample = np.random.default_rng(8).choice(Xt.shape[0], 256, replace=False)
    jobs = [(X[operm[ooff[j]:ooff[j + 1]]], y[operm[ooff[j]:ooff[j + 1]]], Xt[sample], sigma, lam) for j in picks]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:  # before any GPU call
        refs = pool.map(_oracle, jobs)
    import torch
    import paper_1805_00569_gb300 as K
    ctx = K.krr_ctx_create(0)
    dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt)
    dX, dy = dev(X), dev(y)
    _, _, perm, offsets, _ = K.krr_partition(ctx, dX, None, K.KRR_PART_RANDOM, w["p"], seed=w["part_seed"])
    assert np.array_equal(perm.cpu().numpy(), operm)
    print("| precision | partition | rows | rel err alpha | rel err predictions | iterations | status |")
    print("|---|---|---|---|---|---|---|")
    for prec in ("fp64", "fp32", "tf32", "bf16x3"):
        model, status, alpha = K.krr_fit_batch(ctx, dX, dy, perm, offsets, [sigma], [lam], prec, want_alpha=True)
        st = status.cpu().numpy()
        it, _, _ = K.krr_model_stats(ctx, model)
        al = alpha.cpu().numpy()
        yh = K.krr_predict(ctx, model, dev(Xt[sample])).cpu().numpy()
        for (j, (oa, oyh, rc)) in zip(picks, refs):
            a = al[ooff[j]:ooff[j + 1]]
            print("| %s | %d | %d | %.2e | %.2e | %d | %d |" % (prec, j, ooff[j + 1] - ooff[j], rel(a, oa),
                                                            rel(yh[j], oyh), int(it[j]), int(st[j])))
        model.free()


if __name__ == "__main__":
    main()
