/*
 * krr_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the
 * partitioned kernel ridge regression hot path of You, Demmel, Hsieh and
 * Vuduc, "Accurate, Fast and Scalable Kernel Ridge Regression on Parallel and
 * Distributed Systems" (ICS'18).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  The CUDA product path
 * never calls it and shares no code, header, table or constant with it.
 *
 * Every routine is written from the paper's definitions, in the paper's
 * order, with no blocking, fusion or reordering beyond what the definition
 * states.  Compile with -O2 -ffp-contract=off so no multiply-add is fused.
 *
 * Readings of the paper where it is silent or ambiguous (each repeated next
 * to the code that takes it):
 *   R1  lambda is scaled by the partition's own size m (Alg. DC-KRR and
 *       Alg. BKRR2 solve (K + lambda m I) alpha = y with m = n/p).
 *   R2  K-means centres start at caller-given training rows (Alg. 2 says
 *       "randomly"; the random draw is an input).
 *   R3  argmin over squared distances, strict "<", so the lowest index wins a
 *       tie (Alg. K-balance compares "dist < mindis").
 *   R4  an empty cluster keeps its previous centre (Alg. 2 step 6 divides by
 *       zero otherwise).
 *   R5  Alg. 2 loops while delta/n > threshold; threshold = 0 with a cap of
 *       `iters` assign+update rounds.  A final assignment of training and test
 *       points with the final centres defines partitions and routing (KKRR2,
 *       Sec. 4.2: a test point uses the model of its closest centre).
 *   R6  centre sums follow one canonical order: blocks of 1024 consecutive
 *       training indices summed in ascending index, block partial sums
 *       combined by a pairwise tree in block order, then one division.
 *   R7  random partitions: a seeded bijection shuffles the rows (Alg. DC-KRR
 *       "shuffle M by rows"), the shuffled order is cut into p consecutive
 *       parts, the first (n mod p) parts one row longer.
 *   R8  grid index g = i_sigma * |Lambda| + i_lambda; model index
 *       = partition * G + g.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Counter-based generator: Philox4x32-10, Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 4.
 * Round: (L0,R0,L1,R1) -> using two 32x32->64 products with the multipliers
 * M0, M1 and a key schedule bumped by the Weyl constants W0, W1.
 * ---------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------
 * Seeded bijection of [0, n) (reading R7): a balanced Feistel network over
 * 2^(2h) >= n values whose round function is Philox4x32-10, restricted to
 * [0, n) by cycle walking (Black and Rogaway, "Ciphers with arbitrary finite
 * domains", CT-RSA 2002, Sec. 2).
 * ---------------------------------------------------------------------- */
#define FEISTEL_ROUNDS 8

static int feistel_half_bits(int64_t n)
{
    int b = 2;
    while (b < 62 && ((int64_t)1 << b) < n) b += 2;
    return b / 2;
}

static uint64_t feistel_encrypt(uint64_t x, int h, uint64_t seed)
{
    uint64_t mask = ((uint64_t)1 << h) - 1;
    uint64_t left = x >> h, right = x & mask;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t r = 0; r < FEISTEL_ROUNDS; ++r) {
        uint32_t ctr[4] = {(uint32_t)right, (uint32_t)(right >> 32), r, 0u};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        uint64_t f = ((uint64_t)out[1] << 32 | out[0]) & mask;
        uint64_t new_right = left ^ f;
        left = right;
        right = new_right;
    }
    return (left << h) | right;
}

int64_t orc_perm_index(int64_t i, int64_t n, uint64_t seed)
{
    int h = feistel_half_bits(n);
    uint64_t x = (uint64_t)i;
    do {
        x = feistel_encrypt(x, h, seed);
    } while (x >= (uint64_t)n);
    return (int64_t)x;
}

/* Random equal partition (Alg. DC-KRR: shuffle rows, scatter evenly; R7).
 * perm[k] = original row index at shuffled position k; part j owns shuffled
 * positions [offsets[j], offsets[j+1]); assign[row] = its part. */
void orc_partition_random(int64_t n, int32_t p, uint64_t seed,
                          int64_t *perm, int64_t *offsets, int32_t *assign)
{
    int64_t base = n / p, extra = n % p;
    offsets[0] = 0;
    for (int32_t j = 0; j < p; ++j)
        offsets[j + 1] = offsets[j] + base + (j < extra ? 1 : 0);
    for (int64_t k = 0; k < n; ++k)
        perm[k] = orc_perm_index(k, n, seed);
    for (int32_t j = 0; j < p; ++j)
        for (int64_t k = offsets[j]; k < offsets[j + 1]; ++k)
            assign[perm[k]] = j;
}

/* ------------------------------------------------------------------------
 * K-means (Alg. 2) with readings R2-R6.
 * ---------------------------------------------------------------------- */

/* Squared Euclidean distance, features summed in ascending order. */
static double sqdist(const double *a, const double *b, int32_t d)
{
    double s = 0.0;
    for (int32_t f = 0; f < d; ++f) {
        double diff = a[f] - b[f];
        s = s + diff * diff;
    }
    return s;
}

/* Alg. 2 step 4: c_i = argmin_j ||x_i - CT_j|| (R3: strict <). */
void orc_assign(const double *X, int64_t n, int32_t d, const double *CT,
                int32_t k, int32_t *c)
{
    for (int64_t i = 0; i < n; ++i) {
        double best = INFINITY;
        int32_t arg = 0;
        for (int32_t j = 0; j < k; ++j) {
            double dist = sqdist(X + i * d, CT + (int64_t)j * d, d);
            if (dist < best) {
                best = dist;
                arg = j;
            }
        }
        c[i] = arg;
    }
}

#define CANON_BLOCK 1024

/* Alg. 2 step 6, first half (R6): per block of CANON_BLOCK consecutive rows
 * starting at row 0 of X, each centre's member sum taken in ascending row
 * order from 0, and its member count.  part [nblk][k][d], cnt [nblk][k]. */
void orc_block_sums(const double *X, int64_t n, int32_t d, const int32_t *c, int32_t k,
                    double *part, int64_t *cnt)
{
    int64_t nblk = (n + CANON_BLOCK - 1) / CANON_BLOCK;
    for (int64_t e = 0; e < nblk * (int64_t)k * d; ++e) part[e] = 0.0;
    for (int64_t e = 0; e < nblk * (int64_t)k; ++e) cnt[e] = 0;
    for (int64_t b = 0; b < nblk; ++b) {
        double *S = part + b * (int64_t)k * d;
        int64_t hi = (b + 1) * CANON_BLOCK < n ? (b + 1) * CANON_BLOCK : n;
        for (int64_t i = b * CANON_BLOCK; i < hi; ++i) {
            int32_t j = c[i];
            cnt[b * k + j] += 1;
            for (int32_t f = 0; f < d; ++f)
                S[(int64_t)j * d + f] = S[(int64_t)j * d + f] + X[i * d + f];
        }
    }
}

/* Alg. 2 step 6, second half (R4, R6): the block sums combined by a pairwise
 * tree over blocks, level by level in block order (an odd last block carried
 * up), then one division by the centre's member count; a centre with no
 * members keeps its entry of CT.  part is overwritten. */
void orc_tree_combine(double *part, const int64_t *cnt, int64_t nblk, int32_t k, int32_t d, double *CT)
{
    if (nblk == 0) return;
    int64_t len = nblk;
    while (len > 1) {
        int64_t half = (len + 1) / 2;
        for (int64_t q = 0; q < half; ++q) {
            double *dst = part + q * (int64_t)k * d;
            double *a = part + (2 * q) * (int64_t)k * d;
            if (2 * q + 1 < len) {
                double *b2 = part + (2 * q + 1) * (int64_t)k * d;
                for (int64_t e = 0; e < (int64_t)k * d; ++e) dst[e] = a[e] + b2[e];
            } else if (dst != a) {
                for (int64_t e = 0; e < (int64_t)k * d; ++e) dst[e] = a[e];
            }
        }
        len = half;
    }
    for (int32_t j = 0; j < k; ++j) {
        int64_t m = 0;
        for (int64_t b = 0; b < nblk; ++b) m += cnt[b * k + j];
        if (m == 0) continue; /* R4 */
        for (int32_t f = 0; f < d; ++f)
            CT[(int64_t)j * d + f] = part[(int64_t)j * d + f] / (double)m;
    }
}

/* Alg. 2 step 6 with R4 and R6: CT_j = (sum of members) / (member count). */
void orc_update_centres(const double *X, int64_t n, int32_t d,
                        const int32_t *c, int32_t k, double *CT)
{
    int64_t nblk = (n + CANON_BLOCK - 1) / CANON_BLOCK;
    if (nblk == 0) return;
    double *part = (double *)calloc((size_t)nblk * k * d, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)nblk * k, sizeof(int64_t));
    orc_block_sums(X, n, d, c, k, part, cnt);
    orc_tree_combine(part, cnt, nblk, k, d, CT);
    free(part);
    free(cnt);
}

/* Alg. 2 in full (R2, R5).  Returns the number of assign+update rounds run;
 * delta[r] receives the change count of round r (first round: every point
 * counts as changed).  The final assignment uses the final centres. */
int32_t orc_kmeans(const double *X, int64_t n, int32_t d, int32_t k,
                   const int64_t *init_idx, int32_t iters, double *CT,
                   int32_t *c, int64_t *delta)
{
    for (int32_t j = 0; j < k; ++j)
        memcpy(CT + (int64_t)j * d, X + init_idx[j] * d, sizeof(double) * d);
    int32_t *prev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) prev[i] = -1;
    int32_t rounds = 0;
    while (rounds < iters) {
        orc_assign(X, n, d, CT, k, c);
        int64_t dl = 0;
        for (int64_t i = 0; i < n; ++i)
            if (c[i] != prev[i]) ++dl;
        memcpy(prev, c, sizeof(int32_t) * (size_t)n);
        orc_update_centres(X, n, d, c, k, CT);
        if (delta) delta[rounds] = dl;
        ++rounds;
        if (dl == 0) break; /* delta/n > 0 fails: Alg. 2 step 7 stops */
    }
    orc_assign(X, n, d, CT, k, c);
    free(prev);
    return rounds;
}

/* Alg. K-balance Clustering, the per-sample loop: samples in index order,
 * each takes the nearest centre that is not yet full (strict <, so the lowest
 * index wins ties), with the counts starting at zero and the cap
 * ceil(n / p) (the reading of balanced = n / p; the total capacity covers n).
 * Distances are the squared Euclidean distances of the assignment step
 * (sqdist).  A sample whose open centres are all at infinite distance takes
 * the lowest open centre (the reading of the listing's minind = 0).  CS
 * receives the final counts. */
void orc_kbalance_assign(const double *X, int64_t n, int32_t d, const double *CT,
                         int32_t p, int64_t cap, int32_t *c, int64_t *CS)
{
    for (int32_t j = 0; j < p; ++j) CS[j] = 0;
    for (int64_t i = 0; i < n; ++i) {
        double best = INFINITY;
        int32_t arg = -1;
        for (int32_t j = 0; j < p; ++j) {
            if (CS[j] >= cap) continue;
            if (arg < 0) arg = j;
            double dist = sqdist(X + i * d, CT + (int64_t)j * d, d);
            if (dist < best) {
                best = dist;
                arg = j;
            }
        }
        c[i] = arg;
        CS[arg] += 1;
    }
}

/* Group rows by partition, keeping ascending row index inside a partition
 * (the scatter of the KKRR pipeline).  perm/offsets as in the random case. */
void orc_gather_stable(const int32_t *assign, int64_t n, int32_t p,
                       int64_t *perm, int64_t *offsets)
{
    for (int32_t j = 0; j <= p; ++j) offsets[j] = 0;
    for (int64_t i = 0; i < n; ++i) offsets[assign[i] + 1] += 1;
    for (int32_t j = 0; j < p; ++j) offsets[j + 1] += offsets[j];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)p);
    for (int32_t j = 0; j < p; ++j) fill[j] = offsets[j];
    for (int64_t i = 0; i < n; ++i) perm[fill[assign[i]]++] = i;
    free(fill);
}

/* ------------------------------------------------------------------------
 * Kernels (Table 1).  kind 0 = Gaussian exp(-||a-b||^2 / (2 sigma^2)),
 * kind 1 = linear a^T b.  The Gaussian distance is taken by direct
 * differences; the diagonal of a training kernel matrix is exactly 1.
 * ---------------------------------------------------------------------- */
static double kernel_value(const double *a, const double *b, int32_t d,
                           int32_t kind, double sigma)
{
    if (kind == 1) {
        double s = 0.0;
        for (int32_t f = 0; f < d; ++f) s = s + a[f] * b[f];
        return s;
    }
    return exp(-sqdist(a, b, d) / (2.0 * sigma * sigma));
}

void orc_kernel_matrix(const double *A, int64_t ma, const double *B,
                       int64_t mb, int32_t d, int32_t kind, double sigma,
                       double *K)
{
    for (int64_t i = 0; i < ma; ++i)
        for (int64_t j = 0; j < mb; ++j)
            K[i * mb + j] = kernel_value(A + i * d, B + j * d, d, kind, sigma);
}

/* ------------------------------------------------------------------------
 * KRR solve (Eq. 6 with R1): (K + lambda m I) alpha = y.
 * Unblocked Cholesky A = L L^T (the paper's choice of solver, Sec. 5.4),
 * two triangular solves, then iterative refinement whose residual is
 * accumulated in long double.  Returns 0 on success, 1 if a pivot is not
 * positive (A not SPD in floating point).
 * info[0] = Gershgorin condition estimate (max row sum of |A|) / (lambda m)
 * info[1] = final scaled residual ||r||_inf / (||A||_inf ||alpha||_inf + ||y||_inf)
 * info[2] = refinement steps taken
 * ---------------------------------------------------------------------- */
static int cholesky_lower(double *L, int64_t m)
{
    /* L holds A (full, row-major) on entry; lower triangle of L on exit. */
    for (int64_t j = 0; j < m; ++j) {
        double s = L[j * m + j];
        for (int64_t k = 0; k < j; ++k) s = s - L[j * m + k] * L[j * m + k];
        if (!(s > 0.0)) return 1;
        double ljj = sqrt(s);
        L[j * m + j] = ljj;
        for (int64_t i = j + 1; i < m; ++i) {
            double t = L[i * m + j];
            for (int64_t k = 0; k < j; ++k) t = t - L[i * m + k] * L[j * m + k];
            L[i * m + j] = t / ljj;
        }
    }
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = i + 1; j < m; ++j) L[i * m + j] = 0.0;
    return 0;
}

static void cholesky_solve(const double *L, int64_t m, const double *b,
                           double *x)
{
    for (int64_t i = 0; i < m; ++i) { /* L z = b */
        double s = b[i];
        for (int64_t k = 0; k < i; ++k) s = s - L[i * m + k] * x[k];
        x[i] = s / L[i * m + i];
    }
    for (int64_t i = m - 1; i >= 0; --i) { /* L^T x = z */
        double s = x[i];
        for (int64_t k = i + 1; k < m; ++k) s = s - L[k * m + i] * x[k];
        x[i] = s / L[i * m + i];
    }
}

int orc_solve_spd(const double *A, int64_t m, const double *y, double *alpha,
                  double lambda_m, double *info)
{
    double *L = (double *)malloc(sizeof(double) * (size_t)(m * m > 0 ? m * m : 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *c = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    memcpy(L, A, sizeof(double) * (size_t)(m * m));
    double anorm = 0.0, ynorm = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double rs = 0.0;
        for (int64_t j = 0; j < m; ++j) rs = rs + fabs(A[i * m + j]);
        if (rs > anorm) anorm = rs;
        if (fabs(y[i]) > ynorm) ynorm = fabs(y[i]);
    }
    if (info) {
        info[0] = lambda_m > 0.0 ? anorm / lambda_m : INFINITY;
        info[1] = 0.0;
        info[2] = 0.0;
    }
    int bad = cholesky_lower(L, m);
    if (bad) {
        free(L); free(r); free(c);
        return 1;
    }
    cholesky_solve(L, m, y, alpha);
    double prev = INFINITY, scaled = 0.0;
    int steps = 0;
    for (int it = 0; it < 10; ++it) {
        double rmax = 0.0, amax = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            long double s = (long double)y[i];
            for (int64_t j = 0; j < m; ++j)
                s -= (long double)A[i * m + j] * (long double)alpha[j];
            r[i] = (double)s;
            if (fabs(r[i]) > rmax) rmax = fabs(r[i]);
            if (fabs(alpha[i]) > amax) amax = fabs(alpha[i]);
        }
        scaled = rmax / (anorm * amax + ynorm + 1e-300);
        if (it >= 2 && !(scaled < 0.5 * prev)) break;
        prev = scaled;
        cholesky_solve(L, m, r, c);
        for (int64_t i = 0; i < m; ++i) alpha[i] = alpha[i] + c[i];
        ++steps;
    }
    if (info) {
        info[1] = scaled;
        info[2] = (double)steps;
    }
    free(L); free(r); free(c);
    return 0;
}

/* Build K + lambda m I for one partition and solve it (Alg. 1 / the
 * training step of Alg. BKRR2 for one (lambda, sigma)). */
int orc_krr_fit(const double *Xp, const double *yp, int64_t m, int32_t d,
                int32_t kind, double sigma, double lambda, double *alpha,
                double *info)
{
    if (m == 0) return 0;
    double *A = (double *)malloc(sizeof(double) * (size_t)(m * m));
    orc_kernel_matrix(Xp, m, Xp, m, d, kind, sigma, A);
    double lm = lambda * (double)m; /* R1 */
    for (int64_t i = 0; i < m; ++i) A[i * m + i] = A[i * m + i] + lm;
    int rc = orc_solve_spd(A, m, yp, alpha, lm, info);
    free(A);
    return rc;
}

/* Eq. 7: yhat_j = sum_i alpha_i Phi(x_i, xhat_j); cancel_j =
 * sum_i |alpha_i Phi(x_i, xhat_j)| / |yhat_j| (cancellation factor). */
void orc_krr_predict(const double *Xp, const double *alpha, int64_t m,
                     int32_t d, int32_t kind, double sigma, const double *Xt,
                     int64_t t, double *yhat, double *cancel)
{
    for (int64_t j = 0; j < t; ++j) {
        double s = 0.0, a = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            double term = alpha[i] * kernel_value(Xp + i * d, Xt + j * d, d, kind, sigma);
            s = s + term;
            a = a + fabs(term);
        }
        yhat[j] = s;
        if (cancel) cancel[j] = a / fabs(s);
    }
}

/* Eq. 3: MSE = (1/k) sum (yhat - y)^2. */
double orc_mse(const double *yhat, const double *y, int64_t k)
{
    double s = 0.0;
    for (int64_t j = 0; j < k; ++j) {
        double e = yhat[j] - y[j];
        s = s + e * e;
    }
    return k > 0 ? s / (double)k : 0.0;
}
