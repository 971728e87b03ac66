"""CPU model of the prediction's far-term path (Eq. 7 terms far below a test
row's largest): the kernel forms such a term in FP32 as
  x_f = rn32(D_hi * c_hi + s_hi)      (one FMA; D = D_hi + D_lo the squared
                                        distance, c = -1/(2 sigma^2) as c_hi + c_lo,
                                        s = -K ln2 the row's range shift)
  k_f = ex2.approx(rn32(x_f * log2 e))  (relative error <= 2^-22)
and its comment bounds the argument error by 2^-22 (|D c| + |s| + 1), so the
term is within about 2e-4 relative while |D c| and |s| stay under 800.  This
test redoes that arithmetic in numpy (FP32 roundings emulated exactly) and
checks the bound against the exponential of the exact argument, over the
arguments the far path takes (x + s below -20)."""
import numpy as np

F32 = np.float32
LOG2E32 = F32(1.44269504088896341)


def _rn32(x):
    return np.asarray(x, np.float64).astype(F32).astype(np.float64)


def _far_term(D, c, s):
    """(model of the kernel's FP32 far term, exact value) for float64 inputs."""
    D_hi = _rn32(D)
    c_hi = _rn32(c)
    s_hi = _rn32(s)
    xf = _rn32(D_hi * c_hi + s_hi)             # the product of two FP32 values is exact in FP64
    y = _rn32(xf * np.float64(LOG2E32))
    kf = np.exp2(y)                            # ex2.approx: within 2^-22 relative of this
    exact = np.exp(D * c + s)
    return kf, exact, D * c


def test_far_term_error_bound():
    rng = np.random.default_rng(5)
    n = 200000
    sigma = np.exp(rng.uniform(np.log(0.3), np.log(30.0), n))
    c = -1.0 / (2.0 * sigma * sigma)
    x = -rng.uniform(0.0, 800.0, n)            # D c
    D = x / c
    # row shift s = -K ln2 with K = ceil((x_max + 1/64) / ln2), x_max >= x + 20
    xmax = np.minimum(x + rng.uniform(20.0, 60.0, n), 0.0)
    K = np.where(xmax < -20.0, np.ceil((xmax + 1.0 / 64.0) / np.log(2.0)), 0.0)
    s = -K * np.log(2.0)
    far = (x + s) < -20.0
    kf, exact, xc = _far_term(D[far], c[far], s[far])
    ok = exact > 1e-37                          # kept terms (FP32 normal range)
    rel = np.abs(kf[ok] / exact[ok] - 1.0)
    bound = 2.0 ** -22 * (np.abs(xc[ok]) + np.abs(s[far][ok]) + 1.0) + 2.0 ** -22
    assert np.all(rel <= bound)
    assert rel.max() <= 2e-4 * 2.0               # |x|, |s| < 800: about 2e-4
    # relative to the row's largest term (e^(x_max + s) >= 1/2 after the
    # shift) a far term's error stays below 4e-13
    assert np.all(np.abs(kf[ok] - exact[ok]) <= 4e-13 * 2.0)
