// partition.cu -- partitioning kernels (Alg. DC-KRR's partitioning; Alg. 2 plain
// K-means; KKRR2 nearest-centre routing, Sec. 4.2).
//
// * random_perm: seeded bijection of [0, n) -- a balanced Feistel network over
//   2^(2h) >= n values with Philox4x32-10 as round function, restricted to
//   [0, n) by cycle walking (Black & Rogaway, CT-RSA 2002).  Shuffled position
//   k holds row perm[k]; positions are cut into p consecutive parts, the first
//   n mod p one row longer.
// * kmeans_assign: nearest centre with ties to the lowest index.  Distances are
//   first taken in FP32 with a rigorous error bound; only when two or more
//   centres fall inside the bound is the distance recomputed in FP64 in the
//   definition's order (features ascending, no fused multiply-add), so the
//   chosen index equals the FP64 argmin bit for bit.
// * kmeans_block_sums / kmeans_tree_divide: centre means in one canonical
//   order -- blocks of 1024 consecutive rows summed in ascending row order,
//   block sums combined level by level by a pairwise tree in block order, one
//   division by the member count; an empty cluster keeps its centre.
// * gather: stable grouping of rows by partition (ascending row inside a
//   partition), via per-block counts, a scan and an ordered scatter.
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace krr {

// ------------------------------------------------------------ random shuffle
__device__ __forceinline__ uint64_t feistel(uint64_t x, int h, uint32_t k0, uint32_t k1) {
    const uint64_t mask = (h >= 64) ? ~0ull : ((1ull << h) - 1);
    uint64_t L = x >> h, R = x & mask;
    for (uint32_t r = 0; r < 8; ++r) {
        u32x4 c;
        c.x = (uint32_t)R;
        c.y = (uint32_t)(R >> 32);
        c.z = r;
        c.w = 0u;
        u32x4 o = philox4x32_10(c, k0, k1);
        uint64_t f = (((uint64_t)o.y << 32) | o.x) & mask;
        uint64_t nr = L ^ f;
        L = R;
        R = nr;
    }
    return (L << h) | R;
}

__global__ void random_perm_kernel(int64_t n, int32_t p, int h, uint32_t k0, uint32_t k1, int64_t *perm,
                                   int32_t *assign) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint64_t x = (uint64_t)k;
    do {
        x = feistel(x, h, k0, k1);
    } while (x >= (uint64_t)n);
    perm[k] = (int64_t)x;
    int64_t base = n / p, extra = n % p;
    int64_t big = extra * (base + 1);
    int32_t part = (k < big) ? (int32_t)(k / (base + 1)) : (int32_t)(extra + (k - big) / base);
    assign[x] = part;
}

__global__ void random_offsets_kernel(int64_t n, int32_t p, int64_t *offsets, int32_t *route, int64_t t) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t base = n / p, extra = n % p;
    if (i <= p) offsets[i] = i * base + (i < extra ? i : extra);
    if (route && i < t) route[i] = 0;
    for (int64_t q = i + (int64_t)gridDim.x * blockDim.x; route && q < t; q += (int64_t)gridDim.x * blockDim.x)
        route[q] = 0;
}

// ------------------------------------------------------------ K-means assign
constexpr int ASSIGN_THREADS = 128;

// (4 d + 64) 2^-149: the subnormal with that integer significand (exact)
__device__ __forceinline__ float assign_abs_bound(int d) { return __int_as_float(4 * d + 64); }
// Centre with FP32 distance acc and error bound bnd may be the nearest given
// the best upper bound best_hi; an overflowed or NaN distance always may.
__device__ __forceinline__ bool assign_candidate(float acc, float bnd, float best_hi) {
    const float ub = acc + bnd;
    return acc - bnd <= best_hi || !(fabsf(ub) < INFINITY);
}

// One thread per point.  X32: FP32 copy of the rows (converted once per
// K-means run: on GB300 the FP64 -> FP32 conversion runs on the slow FP64
// pipe); C32 / C64: FP32 and FP64 centres.  The FP32 distance of every centre
// carries the bound
//   |d32 - d64| <= (d + 16) 2^-24 1.27 * 2 (||x||^2 + ||c||^2) + (4 d + 64) 2^-149
// The relative part covers the rounding of the inputs, the differences, the
// squares and the sum in the normal range (the factor 2 bounds
// sum (|x|+|c|)^2); the absolute part covers FP32 subnormals, where rounding
// is absolute (at most 2^-150 per input conversion and per accumulation step;
// subnormal differences are exact), so tiny features keep a valid bound.
// An overflowed or NaN distance (huge features) is always a candidate, and
// with no finite upper bound every centre is one.  Centres within the bound
// of the best upper bound are candidates; with two or more, the FP64
// distances in the definition's order decide (strict <, lowest index; index 0
// when no FP64 distance is finite, as the definition's loop leaves it).
__global__ void __launch_bounds__(ASSIGN_THREADS)
kmeans_assign_kernel(const float *__restrict__ X32, const double *__restrict__ X, int64_t n, int32_t d,
                     const double *__restrict__ C64, const float *__restrict__ C32, int32_t k,
                     const int32_t *__restrict__ prev, int32_t *__restrict__ out, unsigned long long *delta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sC = reinterpret_cast<float *>(smem_raw);   // [k][d]
    float *sCn = sC + (size_t)k * d;                     // [k] ||c||^2
    float *sX = sCn + k;                                 // [d][ASSIGN_THREADS]
    for (int e = threadIdx.x; e < k * d; e += blockDim.x) sC[e] = C32[e];
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x;
    const int nrow = (int)((n - i0) < (int64_t)blockDim.x ? (n - i0) : (int64_t)blockDim.x);
    for (int e = threadIdx.x; e < nrow * d; e += blockDim.x) {
        const int r = e / d, f = e % d;
        sX[f * ASSIGN_THREADS + r] = X32[(i0 + r) * d + f];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        float s = 0.f;
        for (int f = 0; f < d; ++f) s = fmaf(sC[j * d + f], sC[j * d + f], s);
        sCn[j] = s;
    }
    __syncthreads();
    const int r = threadIdx.x;
    if (r >= nrow) return;
    const int64_t i = i0 + r;
    float xn = 0.f;
    for (int f = 0; f < d; ++f) xn = fmaf(sX[f * ASSIGN_THREADS + r], sX[f * ASSIGN_THREADS + r], xn);
    const float bscale = (float)(d + 16) * 5.9604644775390625e-8f * 1.27f * 2.0f;
    const float babs = assign_abs_bound(d);
    float best_hi = INFINITY;
#pragma unroll 1
    for (int j = 0; j < k; ++j) {
        const float *c = sC + j * d;
        float acc = 0.f;
        for (int f = 0; f < d; ++f) {
            const float t = sX[f * ASSIGN_THREADS + r] - c[f];
            acc = fmaf(t, t, acc);
        }
        best_hi = fminf(best_hi, acc + (bscale * (xn + sCn[j]) + babs));
    }
    int ncand = 0, first = -1;
#pragma unroll 1
    for (int j = 0; j < k; ++j) {
        const float *c = sC + j * d;
        float acc = 0.f;
        for (int f = 0; f < d; ++f) {
            const float t = sX[f * ASSIGN_THREADS + r] - c[f];
            acc = fmaf(t, t, acc);
        }
        if (assign_candidate(acc, bscale * (xn + sCn[j]) + babs, best_hi)) {
            if (ncand == 0) first = j;
            ++ncand;
        }
    }
    int arg = first;
    if (ncand > 1) {
        const double *x = X + i * d;
        double best = INFINITY;
#pragma unroll 1
        for (int j = 0; j < k; ++j) {
            const float *c = sC + j * d;
            float acc = 0.f;
            for (int f = 0; f < d; ++f) {
                const float t = sX[f * ASSIGN_THREADS + r] - c[f];
                acc = fmaf(t, t, acc);
            }
            if (!assign_candidate(acc, bscale * (xn + sCn[j]) + babs, best_hi)) continue;
            const double *c64 = C64 + (size_t)j * d;
            double s = 0.0;
            for (int f = 0; f < d; ++f) {
                const double t = __dsub_rn(x[f], c64[f]);
                s = __dadd_rn(s, __dmul_rn(t, t));
            }
            if (s < best) {
                best = s;
                arg = j;
            }
        }
        if (!(best < INFINITY)) arg = 0;
    }
    out[i] = arg;
    if (delta && (prev == nullptr || prev[i] != arg)) atomicAdd(delta, 1ull);
}

// Same assignment, organised for throughput in two kernels.
//
// Screen (kmeans_screen_kernel): a CTA takes 128 rows and every centre, 64
// at a time; thread (rg, cg) forms the FP32 Gram products of 8 rows x 4
// centres from shared copies of the rows ([feature][row]) and centres
// ([feature][centre]), one fused multiply-add per row, centre and feature.
// The screening distance is the Gram form
//   d32 = rn(rn(||x||^2 + ||c||^2) - 2 x.c)
// with ||x||^2, ||c||^2 and x.c each an FP32 sum of products (in any order:
// a sum of d terms in any order is off by at most (d - 1) 2^-24 times the sum
// of their magnitudes).  The bound used above also holds for it: the three sums
// and the two final roundings contribute at most (2d + 3) 2^-24 (||x||^2 +
// ||c||^2) in the normal range, the FP32 rounding of the inputs 4 2^-24 of
// the same, so (2d + 7) 2^-24 (...) <= (d + 16) 2^-24 1.27 * 2 (...); in the
// subnormal range each of the 4d + 2 roundings is off by at most 2^-150,
// within (4d + 64) 2^-149.  Every row with one candidate takes it; a row
// with several goes to a list.
//
// Recheck (kmeans_recheck_kernel): one warp per listed row.  Its lanes form
// the same screening distances of their centres and the candidates among
// them; a single candidate is the nearest.  Several go, as (row, centre)
// pairs in ascending centre order, to kmeans_pair_dist_kernel (one thread per
// pair: the FP64 distance in the definition's order, feature by feature,
// rounding each step -- a divergent FP64 instruction costs the same issue
// slot with one lane as with 32, so the pairs of many rows fill the lanes)
// and kmeans_pair_pick_kernel (one thread per row: the nearest by FP64
// distance, strict <, lowest index; index 0 when no FP64 distance is
// finite).  A row whose pairs do not fit the pair buffer is decided by its
// warp the same way.  A row's
// candidates are a superset of the centres that can be nearest under the
// definition, so the result is the definition's whatever the list order.
constexpr int SCR_THREADS = 256;
constexpr int SCR_ROWS = 128;            // rows per CTA
constexpr int SCR_CT = 64;               // centres per tile
constexpr int SCR_XL = SCR_ROWS + 4;     // row stride of the [feature][row] copy (16-byte rows)
constexpr int SCR_CL = SCR_CT + 4;       // row stride of the [feature][centre] copy
constexpr int SCR_KMAX = 256;            // centres the screen keeps in shared memory

static size_t screen_smem(int dp, int kt) {
    return ((size_t)dp * SCR_XL + (size_t)dp * SCR_CL + SCR_ROWS + kt + (size_t)SCR_ROWS * (kt + 1)) * sizeof(float);
}

template <int DP>
__global__ void __launch_bounds__(SCR_THREADS)
kmeans_screen_kernel(const float *__restrict__ X32, int64_t n, int32_t d, const float *__restrict__ C32,
                     const float *__restrict__ cn32, int32_t k, int32_t kt, const int32_t *__restrict__ prev,
                     int32_t *__restrict__ out, int32_t *__restrict__ list, unsigned int *__restrict__ nlist,
                     unsigned long long *delta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *xs = reinterpret_cast<float *>(smem_raw);  // [DP][SCR_XL]
    float *cs = xs + DP * SCR_XL;                      // [DP][SCR_CL]
    float *xn = cs + DP * SCR_CL;                      // [SCR_ROWS] ||x||^2
    float *cn = xn + SCR_ROWS;                         // [kt] ||c||^2
    float *dist = cn + kt;                             // [SCR_ROWS][kt + 1] screening distances
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * SCR_ROWS;
    const int nrow = (int)min((int64_t)SCR_ROWS, n - i0);
    {
        // the tile's rows: warp w takes rows w, w + 8, ..., its lanes the
        // features lane, lane + 32, lane + 64; all loads issued before the
        // first shared store
        constexpr int NQ = (DP + 31) / 32, NR = SCR_ROWS / (SCR_THREADS / 32);
        const int w = tid >> 5, lane = tid & 31;
        float v[NR][NQ];
#pragma unroll
        for (int u = 0; u < NR; ++u)
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int r = w + u * (SCR_THREADS / 32), f = lane + 32 * q;
                v[u][q] = (r < nrow && f < d) ? X32[(i0 + r) * d + f] : 0.f;
            }
#pragma unroll
        for (int u = 0; u < NR; ++u)
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int r = w + u * (SCR_THREADS / 32), f = lane + 32 * q;
                if (f < DP) xs[f * SCR_XL + r] = v[u][q];
            }
    }
    for (int j = tid; j < kt; j += SCR_THREADS) cn[j] = cn32[j];
    __syncthreads();
    {
        // ||x||^2: warp w takes rows 16 w .. 16 w + 15, two lanes per row (the
        // two halves of the features, then their sum)
        const int rr = (tid >> 5) * 16 + (tid & 15), h = (tid >> 4) & 1;
        float sx = 0.f;
#pragma unroll 8
        for (int f = h * (DP / 2); f < (h + 1) * (DP / 2); ++f) sx = fmaf(xs[f * SCR_XL + rr], xs[f * SCR_XL + rr], sx);
        sx += __shfl_xor_sync(0xffffffffu, sx, 16);
        if (h == 0) xn[rr] = sx;
    }
    const int rg = tid >> 4, cg = tid & 15;  // rows 8 rg .. 8 rg + 7, centres 4 cg .. 4 cg + 3 of the tile
    const int DL = kt + 1;
    for (int c0 = 0; c0 < kt; c0 += SCR_CT) {
        __syncthreads();  // the previous tile's products are done with cs
        {
            constexpr int NC = SCR_CT * DP / SCR_THREADS;
            float v[NC];
#pragma unroll
            for (int u = 0; u < NC; ++u) {
                const int e = tid + u * SCR_THREADS, jj = e / DP, f = e % DP;
                v[u] = (c0 + jj < k && f < d) ? C32[(size_t)(c0 + jj) * d + f] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < NC; ++u) {
                const int e = tid + u * SCR_THREADS, jj = e / DP, f = e % DP;
                cs[f * SCR_CL + jj] = v[u];
            }
        }
        __syncthreads();
        float acc[8][4] = {};
#pragma unroll 4
        for (int f = 0; f < DP; ++f) {
            const float4 a0 = *reinterpret_cast<const float4 *>(xs + f * SCR_XL + rg * 8);
            const float4 a1 = *reinterpret_cast<const float4 *>(xs + f * SCR_XL + rg * 8 + 4);
            const float4 b = *reinterpret_cast<const float4 *>(cs + f * SCR_CL + cg * 4);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int r = rg * 8 + u, j = c0 + cg * 4 + v;
                dist[r * DL + j] = __fmaf_rn(-2.0f, acc[u][v], __fadd_rn(xn[r], cn[j]));
            }
    }
    __syncthreads();
    // per row: two threads (lanes l and l + 16 of a warp), each over half the
    // centres; the best upper bound is a minimum (any order), the candidates
    // a count and the first of them
    const int r = (tid >> 5) * 16 + (tid & 15), h = (tid >> 4) & 1;
    const bool live = r < nrow;
    const float bscale = (float)(d + 16) * 5.9604644775390625e-8f * 1.27f * 2.0f;
    const float babs = assign_abs_bound(d);
    const int kh = (k + 1) / 2, j0 = h * kh, j1 = h ? k : kh;
    float best_hi = INFINITY;
    if (live)
        for (int j = j0; j < j1; ++j) best_hi = fminf(best_hi, dist[r * DL + j] + (bscale * (xn[r] + cn[j]) + babs));
    best_hi = fminf(best_hi, __shfl_xor_sync(0xffffffffu, best_hi, 16));
    int ncand = 0, first = -1;
    if (live)
        for (int j = j0; j < j1; ++j)
            if (assign_candidate(dist[r * DL + j], bscale * (xn[r] + cn[j]) + babs, best_hi)) {
                if (ncand == 0) first = j;
                ++ncand;
            }
    const int ncand_o = __shfl_xor_sync(0xffffffffu, ncand, 16);
    const int first_o = __shfl_xor_sync(0xffffffffu, first, 16);
    int arg = -1;
    if (live && h == 0) {
        const int nc = ncand + ncand_o;
        if (nc == 1) {
            arg = ncand == 1 ? first : first_o;
            out[i0 + r] = arg;
        } else {
            list[atomicAdd(nlist, 1u)] = (int32_t)(i0 + r);  // decided by the recheck
        }
    }
    if (delta) {  // one atomic per warp: the counter is a single address
        const bool changed = arg >= 0 && (prev == nullptr || prev[i0 + r] != arg);
        const unsigned vote = __ballot_sync(0xffffffffu, changed);
        if ((tid & 31) == 0 && vote) atomicAdd(delta, (unsigned long long)__popc(vote));
    }
}

// ||c||^2 of every centre (0 for the padding up to kt): one warp per centre
__global__ void centre_norms_kernel(const float *__restrict__ C32, int32_t k, int32_t d, int32_t kt,
                                    float *__restrict__ cn32) {
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= kt) return;
    float s = 0.f;
    if (j < k)
        for (int f = lane; f < d; f += 32) s = fmaf(C32[(size_t)j * d + f], C32[(size_t)j * d + f], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) cn32[j] = s;
}

constexpr int RCK_WARPS = 8;                  // warps (rows in flight) per CTA
constexpr int RCK_CH = SCR_KMAX / 32;         // 32-centre chunks
__global__ void __launch_bounds__(RCK_WARPS * 32)
kmeans_recheck_kernel(const float *__restrict__ X32, const double *__restrict__ X, int32_t d,
                      const float *__restrict__ C32, const double *__restrict__ C64, const float *__restrict__ cn32,
                      int32_t k, const int32_t *__restrict__ list, const unsigned int *__restrict__ nlist,
                      const int32_t *__restrict__ prev, int32_t *__restrict__ out, unsigned long long *delta,
                      int32_t *__restrict__ pstart, int32_t *__restrict__ pcnt, int32_t *__restrict__ prow,
                      int32_t *__restrict__ pj, unsigned int *__restrict__ npairs, int64_t pcap) {
    __shared__ double xsh[RCK_WARPS][96];  // the row in FP64 (d <= 96 on this path)
    __shared__ float dsh[RCK_WARPS][SCR_KMAX], bsh[RCK_WARPS][SCR_KMAX];  // screening distance, bound per centre
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * RCK_WARPS;
    const int64_t cnt = *nlist;
    const float bscale = (float)(d + 16) * 5.9604644775390625e-8f * 1.27f * 2.0f;
    const float babs = assign_abs_bound(d);
    for (int64_t w = (int64_t)blockIdx.x * RCK_WARPS + wid; w < cnt; w += warps) {
        const int64_t i = list[w];
        // the row: FP32 features f = lane + 32 q in registers, FP64 in shared memory
        float xv[3];
        float xn = 0.f;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int f = lane + 32 * q;
            xv[q] = f < d ? X32[i * d + f] : 0.f;
            xn = fmaf(xv[q], xv[q], xn);
            if (f < d) xsh[wid][f] = X[i * d + f];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) xn += __shfl_xor_sync(0xffffffffu, xn, o);
        __syncwarp();
        // screening distance and bound of every centre (lane jj writes centre ch 32 + jj)
        float lbest = INFINITY;
#pragma unroll 1
        for (int ch = 0; ch * 32 < k; ++ch) {
            for (int jj0 = 0; jj0 < 32 && ch * 32 + jj0 < k; jj0 += 8) {
                // the features of 8 centres, all loads issued first
                float cv[8][3];
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const int j = ch * 32 + jj0 + u, f = lane + 32 * q;
                        cv[u][q] = (j < k && f < d) ? C32[(size_t)j * d + f] : 0.f;
                    }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int jj = jj0 + u, j = ch * 32 + jj;
                    float p = 0.f;
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        if (lane + 32 * q < d) p = fmaf(xv[q], cv[u][q], p);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
                    if (j < k && lane == jj) {
                        const float dj = __fmaf_rn(-2.0f, p, __fadd_rn(xn, cn32[j]));
                        const float bj = bscale * (xn + cn32[j]) + babs;
                        dsh[wid][j] = dj;
                        bsh[wid][j] = bj;
                        lbest = fminf(lbest, dj + bj);
                    }
                }
            }
        }
        float best_hi = lbest;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best_hi = fminf(best_hi, __shfl_xor_sync(0xffffffffu, best_hi, o));
        __syncwarp();  // dsh, bsh written
        unsigned mask[RCK_CH];
        int ncand = 0;
#pragma unroll
        for (int ch = 0; ch < RCK_CH; ++ch) {
            const int j = ch * 32 + lane;
            mask[ch] = __ballot_sync(0xffffffffu, j < k && assign_candidate(dsh[wid][j], bsh[wid][j], best_hi));
            ncand += __popc(mask[ch]);
        }
        // candidate c in ascending index order
        auto cand_index = [&](int c) {
            int j = -1, rem = c;
#pragma unroll
            for (int ch = 0; ch < RCK_CH; ++ch) {
                const int pc = __popc(mask[ch]);
                if (j < 0 && rem < pc) {
                    unsigned m = mask[ch];
                    for (int u = 0; u < rem; ++u) m &= m - 1;  // drop the rem lowest candidates
                    j = ch * 32 + __ffs(m) - 1;
                }
                if (j < 0) rem -= pc;
            }
            return j;
        };
        if (ncand == 1) {  // one candidate: it is the nearest (its bound is finite)
            if (lane == 0) {
                const int arg = cand_index(0);
                pcnt[w] = 0;
                out[i] = arg;
                if (delta && (prev == nullptr || prev[i] != arg)) atomicAdd(delta, 1ull);
            }
            __syncwarp();
            continue;
        }
        // several: the (row, candidate) pairs go to the pair kernels, one
        // FP64 distance per thread, when the pair buffer has room
        unsigned int pos = 0;
        if (lane == 0) pos = atomicAdd(npairs, (unsigned int)ncand);
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if ((int64_t)pos + ncand <= pcap) {
            for (int c = lane; c < ncand; c += 32) {
                pj[pos + c] = cand_index(c);
                prow[pos + c] = (int32_t)i;
            }
            if (lane == 0) {
                pstart[w] = (int32_t)pos;
                pcnt[w] = ncand;
            }
            __syncwarp();
            continue;
        }
        // decided here; reserved slots inside the buffer are marked unused
        for (int64_t q = (int64_t)pos + lane; q < min((int64_t)pos + ncand, pcap); q += 32) prow[q] = -1;
        if (lane == 0) pcnt[w] = 0;
        // candidate c goes to lane c % 32: FP64 distance in the definition's
        // order, the lane keeping its smallest (strict <)
        double best = INFINITY;
        int barg = k;
        for (int c0 = 0; c0 < ncand; c0 += 32) {
            const int c = c0 + lane;
            const int j = c < ncand ? cand_index(c) : -1;
            if (j >= 0) {
                const double *c64 = C64 + (size_t)j * d;
                double sd = 0.0;
#pragma unroll 8
                for (int f = 0; f < d; ++f) {
                    const double t = __dsub_rn(xsh[wid][f], c64[f]);
                    sd = __dadd_rn(sd, __dmul_rn(t, t));
                }
                if (sd < best) {
                    best = sd;
                    barg = j;
                }
            }
        }
        // smallest finite distance over the lanes, lowest index on equal distances
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oa = __shfl_xor_sync(0xffffffffu, barg, o);
            if (ob < best || (ob == best && oa < barg)) {
                best = ob;
                barg = oa;
            }
        }
        const int arg = best < INFINITY ? barg : 0;
        if (lane == 0) {
            out[i] = arg;
            if (delta && (prev == nullptr || prev[i] != arg)) atomicAdd(delta, 1ull);
        }
        __syncwarp();  // xsh is reused by the warp's next row
    }
}

// FP64 distance of every (row, candidate) pair in the definition's order
__global__ void kmeans_pair_dist_kernel(const double *__restrict__ X, const double *__restrict__ C64, int32_t d,
                                        const int32_t *__restrict__ prow, const int32_t *__restrict__ pj,
                                        const unsigned int *__restrict__ npairs, int64_t pcap,
                                        double *__restrict__ pd) {
    const int64_t np = min((int64_t)*npairs, pcap);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
        if (prow[q] < 0) continue;  // slot of a row decided by its recheck warp
        const double *xr = X + (int64_t)prow[q] * d, *c64 = C64 + (int64_t)pj[q] * d;
        double sd = 0.0;
#pragma unroll 8
        for (int f = 0; f < d; ++f) {
            const double t = __dsub_rn(xr[f], c64[f]);
            sd = __dadd_rn(sd, __dmul_rn(t, t));
        }
        pd[q] = sd;
    }
}

// the nearest candidate of every listed row whose pairs were handed over:
// smallest finite FP64 distance, the first (lowest index) on equal distances;
// index 0 when none is finite
__global__ void kmeans_pair_pick_kernel(const int32_t *__restrict__ list, const unsigned int *__restrict__ nlist,
                                        const int32_t *__restrict__ pstart, const int32_t *__restrict__ pcnt,
                                        const int32_t *__restrict__ pj, const double *__restrict__ pd,
                                        const int32_t *__restrict__ prev, int32_t *__restrict__ out,
                                        unsigned long long *delta) {
    const int64_t cnt = *nlist;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < cnt; w += (int64_t)gridDim.x * blockDim.x) {
        const int c = pcnt[w];
        if (c == 0) continue;
        const int64_t p0 = pstart[w];
        double best = INFINITY;
        int arg = 0;
        for (int q = 0; q < c; ++q)
            if (pd[p0 + q] < best) {
                best = pd[p0 + q];
                arg = pj[p0 + q];
            }
        const int64_t i = list[w];
        out[i] = arg;
        if (delta && (prev == nullptr || prev[i] != arg)) atomicAdd(delta, 1ull);
    }
}

__global__ void to_float_kernel(const double *__restrict__ a, float *__restrict__ b, int64_t cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) b[i] = __double2float_rn(a[i]);
}

__global__ void init_centres_kernel(const double *__restrict__ X, int32_t d, const int64_t *__restrict__ idx,
                                    int32_t k, double *__restrict__ C) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)k * d) return;
    int j = (int)(e / d), f = (int)(e % d);
    C[e] = X[idx[j] * d + f];
}

// ------------------------------------------------------------ K-means update
constexpr int CANON = 1024;

// grid = number of 1024-row blocks; partial [nblk][k][d] FP64, counts [nblk][k]
// Centre sums of one block of CANON consecutive rows in the canonical order
// (each centre's rows added in ascending row order, starting from 0).  A
// stable counting sort groups the block's rows by centre (warp 0 places 32
// rows at a time with match/popc ranks); then thread (feature chunk, centre
// group, lane) sums its centres' rows for one feature in a register, loads
// issued four rows ahead of the additions.  blockDim = 32 * ceil(d/32) * CG.
__global__ void kmeans_block_sums_kernel(const double *__restrict__ X, int64_t n, int32_t d,
                                         const int32_t *__restrict__ c, int32_t k, int32_t cg_count,
                                         double *__restrict__ partial, long long *__restrict__ counts) {
    extern __shared__ unsigned char smem_raw[];
    int32_t *sc = reinterpret_cast<int32_t *>(smem_raw);  // [CANON] centre of each row
    int32_t *order = sc + CANON;                          // [CANON] rows grouped by centre
    int32_t *start = order + CANON;                       // [k + 1]
    int32_t *cursor = start + k + 1;                      // [k]
    const int64_t b = blockIdx.x;
    const int64_t lo = b * CANON;
    const int len = (int)(min(n, lo + CANON) - lo);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < k; j += blockDim.x) cursor[j] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const int j = c[lo + i];
        sc[i] = j;
        atomicAdd(&cursor[j], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int j = 0; j < k; ++j) {
            start[j] = run;
            run += cursor[j];
            cursor[j] = start[j];
        }
        start[k] = run;
    }
    __syncthreads();
    if (warp == 0) {
        for (int base = 0; base < len; base += 32) {
            const int i = base + lane;
            const bool valid = i < len;
            const int j = valid ? sc[i] : -1 - lane;  // invalid lanes match nobody
            const unsigned mask = __match_any_sync(0xffffffffu, j);
            const int leader = __ffs(mask) - 1;
            int pos = 0;
            if (valid) pos = cursor[j] + __popc(mask & ((1u << lane) - 1u));
            __syncwarp();
            if (valid) {
                order[pos] = i;
                if (lane == leader) cursor[j] += __popc(mask);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) counts[b * k + j] = start[j + 1] - start[j];
    const int fc = warp / cg_count, cg = warp % cg_count;
    const int f = fc * 32 + lane;
    if (f >= d) return;
    double *P = partial + b * (int64_t)k * d;
    const double *Xb = X + lo * d + f;
    for (int j = cg; j < k; j += cg_count) {
        double acc = 0.0;
        int r = start[j];
        const int e = start[j + 1];
        for (; r + 4 <= e; r += 4) {
            const double v0 = Xb[(int64_t)order[r] * d], v1 = Xb[(int64_t)order[r + 1] * d];
            const double v2 = Xb[(int64_t)order[r + 2] * d], v3 = Xb[(int64_t)order[r + 3] * d];
            acc = __dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(acc, v0), v1), v2), v3);
        }
        for (; r < e; ++r) acc = __dadd_rn(acc, Xb[(int64_t)order[r] * d]);
        P[(size_t)j * d + f] = acc;
    }
}

// Pairwise tree over the block sums (level by level: element q of a level is
// element 2q + element 2q + 1 of the one below, an odd last element carried
// up unchanged), then one division by the centre's count.  A CTA takes TE
// consecutive (centre, feature) entries and keeps both levels of the tree in
// shared memory (ping-pong), so every addition reads shared memory.
constexpr int TREE_THREADS = 256;
constexpr int TREE_MAXTE = 32;                  // entries per CTA at most
constexpr int TREE_MAXC = TREE_MAXTE + 1;       // centres those entries can span
__global__ void kmeans_tree_divide_kernel(const double *__restrict__ partial, const long long *__restrict__ counts,
                                          int64_t nblk, int32_t k, int32_t d, int32_t te, double *__restrict__ C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *buf0 = reinterpret_cast<double *>(smem_raw);  // [nblk][te]
    double *buf1 = buf0 + nblk * te;
    const int64_t kd = (int64_t)k * d;
    const int64_t e0 = (int64_t)blockIdx.x * te;
    const int ne = (int)min((int64_t)te, kd - e0);
    for (int64_t x0 = 0; x0 < nblk * te; x0 += 8 * (int64_t)blockDim.x) {
        double v[8];  // eight loads in flight per thread
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t x = x0 + threadIdx.x + u * (int64_t)blockDim.x;
            const int64_t b = x / te;
            const int c = (int)(x % te);
            v[u] = (x < nblk * te && c < ne) ? partial[b * kd + e0 + c] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t x = x0 + threadIdx.x + u * (int64_t)blockDim.x;
            if (x < nblk * te) buf0[x] = v[u];
        }
    }
    // the row counts of the centres this CTA's entries belong to (integer sums:
    // any order), one warp per centre, lanes striding over the blocks
    __shared__ long long ctot[TREE_MAXC];
    const int j0 = (int)(e0 / d), nj = (int)((e0 + ne - 1) / d) - j0 + 1;
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int jj = warp; jj < nj; jj += (int)(blockDim.x >> 5)) {
            long long sacc = 0;
            for (int64_t b0 = lane; b0 < nblk; b0 += 32 * 8) {
                long long v[8];  // eight loads in flight per lane
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int64_t b = b0 + 32 * u;
                    v[u] = b < nblk ? counts[b * k + j0 + jj] : 0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) sacc += v[u];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
            if (lane == 0) ctot[jj] = sacc;
        }
    }
    __syncthreads();
    double *src = buf0, *dst = buf1;
    int64_t len = nblk;
    while (len > 1) {
        const int64_t half = (len + 1) / 2;
        for (int64_t x = threadIdx.x; x < half * te; x += blockDim.x) {
            const int64_t q = x / te;
            const int c = (int)(x % te);
            const double a = src[(2 * q) * te + c];
            dst[x] = (2 * q + 1 < len) ? __dadd_rn(a, src[(2 * q + 1) * te + c]) : a;
        }
        __syncthreads();
        double *tmp = src;
        src = dst;
        dst = tmp;
        len = half;
    }
    for (int c = threadIdx.x; c < ne; c += blockDim.x) {
        const int64_t e = e0 + c;
        const long long cnt = ctot[(int)(e / d) - j0];
        if (cnt > 0) C[e] = __ddiv_rn(src[c], (double)cnt);
    }
}

// ------------------------------------------------------------ stable gather
__global__ void gather_count_kernel(const int32_t *__restrict__ a, int64_t n, int32_t p,
                                    long long *__restrict__ bcount) {
    extern __shared__ unsigned char smem_raw[];
    int *h = reinterpret_cast<int *>(smem_raw);
    for (int j = threadIdx.x; j < p; j += blockDim.x) h[j] = 0;
    __syncthreads();
    int64_t lo = (int64_t)blockIdx.x * CANON, hi = min(n, lo + CANON);
    // a partition index outside [0, p) is counted nowhere (the scatter places
    // only rows with an index in range, so offsets[p] then falls short of n)
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int32_t v = a[i];
        if ((uint32_t)v < (uint32_t)p) atomicAdd(&h[v], 1);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += blockDim.x) bcount[(int64_t)blockIdx.x * p + j] = h[j];
}

// Offsets and per-block starting positions, one CTA (1024 threads = 32
// warps): warp w takes partitions w, w + 32, ...; its lanes walk the
// partition's block counts 32 blocks at a time (warp sums for the total, then
// warp scans for the block starts), so a large block count costs nblk / 32
// steps per partition instead of nblk.  Between the passes one scan over the
// partitions turns the totals into the partition starts.
__global__ void gather_scan_kernel(long long *__restrict__ bcount, int64_t nblk, int32_t p,
                                   int64_t *__restrict__ offsets) {
    extern __shared__ unsigned char smem_raw[];
    long long *tot = reinterpret_cast<long long *>(smem_raw);  // [p]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = warp; j < p; j += nw) {
        long long run = 0;
        for (int64_t b0 = 0; b0 < nblk; b0 += 32) {
            const int64_t b = b0 + lane;
            run += b < nblk ? bcount[b * p + j] : 0;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) run += __shfl_xor_sync(0xffffffffu, run, off);
        if (lane == 0) tot[j] = run;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int j = 0; j < p; ++j) {
            const long long c = tot[j];
            tot[j] = run;
            offsets[j] = run;
            run += c;
        }
        offsets[p] = run;
    }
    __syncthreads();
    for (int j = warp; j < p; j += nw) {
        long long base = tot[j];
        for (int64_t b0 = 0; b0 < nblk; b0 += 32) {
            const int64_t b = b0 + lane;
            const long long c = b < nblk ? bcount[b * p + j] : 0;
            long long incl = c;  // inclusive scan over the 32 blocks of this step
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const long long v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            if (b < nblk) bcount[b * p + j] = base + incl - c;
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

__global__ void gather_scatter_kernel(const int32_t *__restrict__ a, int64_t n, int32_t p,
                                      const long long *__restrict__ bstart, int64_t *__restrict__ perm) {
    extern __shared__ unsigned char smem_raw[];
    int32_t *sa = reinterpret_cast<int32_t *>(smem_raw);
    int64_t lo = (int64_t)blockIdx.x * CANON, hi = min(n, lo + CANON);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) sa[i - lo] = a[i];
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        long long pos = bstart[(int64_t)blockIdx.x * p + j];
        for (int64_t i = lo; i < hi; ++i)
            if (sa[i - lo] == j) perm[pos++] = i;
    }
}

// ------------------------------------------------------------ host drivers
// ------------------------------------------------------------ K-balance
// Alg. K-balance Clustering replayed exactly in rounds.  D holds the squared
// FP64 distance of every (row, centre) pair in the definition's order
// (ascending feature, unfused operations, as the assignment step's FP64
// recheck).  A round: every unplaced row takes its nearest open centre
// (strict <, lowest index); the first row whose centre already holds its
// remaining capacity of earlier rows of the round is the overflow row; the
// rows before it are placed exactly as the sequential loop places them (no
// centre overflows before it), every centre that is now full closes (the
// overflowing one among them), and the next round starts at the overflow
// row.  Every round but the last closes a centre, so there are at most p
// rounds; after the first, only the rows whose choice has closed look again.
constexpr int KB_ROWS = 64;     // rows per CTA of the distance kernel
constexpr int KB_BLK = 1024;    // rows per counting block

__global__ void __launch_bounds__(KB_ROWS)
kb_dist_kernel(const double *__restrict__ X, int64_t n, int32_t d, const double *__restrict__ C, int32_t p,
               double *__restrict__ D) {
    extern __shared__ double kb_sx[];  // [d][KB_ROWS]
    const int64_t i0 = (int64_t)blockIdx.x * KB_ROWS;
    const int nrow = (int)((n - i0) < (int64_t)KB_ROWS ? (n - i0) : (int64_t)KB_ROWS);
    for (int e = threadIdx.x; e < nrow * d; e += KB_ROWS) {
        const int r = e / d, f = e % d;
        kb_sx[f * KB_ROWS + r] = X[(i0 + r) * d + f];
    }
    __syncthreads();
    const int r = threadIdx.x;
    if (r >= nrow) return;
    for (int j = 0; j < p; ++j) {
        const double *c = C + (size_t)j * d;
        double s = 0.0;
        for (int f = 0; f < d; ++f) {
            const double t = __dsub_rn(kb_sx[f * KB_ROWS + r], __ldg(c + f));
            s = __dadd_rn(s, __dmul_rn(t, t));
        }
        D[(i0 + r) * p + j] = s;
    }
}

// choice[i] for rows [start, n): nearest open centre; after the first round
// only the rows whose choice has closed look again
__global__ void kb_choose_kernel(const double *__restrict__ D, int64_t n, int32_t p, int64_t start,
                                 const int32_t *__restrict__ open, int first, int32_t *__restrict__ choice) {
    extern __shared__ int32_t kb_open[];  // [p]
    for (int j = threadIdx.x; j < p; j += blockDim.x) kb_open[j] = open[j];
    __syncthreads();
    const int64_t i = start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!first && kb_open[choice[i]]) return;  // its nearest open centre is unchanged
    int arg = -1;
    double best = INFINITY;
    for (int j = 0; j < p; ++j) {
        if (!kb_open[j]) continue;
        if (arg < 0) arg = j;
        const double v = D[i * p + j];
        if (v < best) {
            best = v;
            arg = j;
        }
    }
    choice[i] = arg < 0 ? 0 : arg;  // some centre is always open while rows remain (p cap >= n)
}

// per block of KB_BLK rows of [start, n): how many rows chose each centre
__global__ void kb_count_kernel(const int32_t *__restrict__ choice, int64_t n, int32_t p, int64_t start,
                                int32_t *__restrict__ bcnt) {
    extern __shared__ int32_t kb_c[];  // [p]
    for (int j = threadIdx.x; j < p; j += blockDim.x) kb_c[j] = 0;
    __syncthreads();
    const int64_t i0 = start + (int64_t)blockIdx.x * KB_BLK;
    const int64_t hi = i0 + KB_BLK < n ? i0 + KB_BLK : n;
    for (int64_t i = i0 + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&kb_c[choice[i]], 1);
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += blockDim.x) bcnt[(int64_t)blockIdx.x * p + j] = kb_c[j];
}

// one warp per centre j: the row at which j's count in the round would pass
// its remaining capacity cap - cs[j] (n when it does not)
__global__ void kb_find_kernel(const int32_t *__restrict__ bcnt, int64_t nblk, int32_t p,
                               const unsigned long long *__restrict__ cs, int64_t cap,
                               const int32_t *__restrict__ choice, int64_t n, int64_t start,
                               long long *__restrict__ ovf) {
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= p) return;
    const int64_t rem = cap - (int64_t)cs[j];
    int64_t cum = 0;
    long long res = n;
    for (int64_t b = 0; b < nblk; ++b) {
        const int c = bcnt[b * p + j];
        if (cum + c > rem) {
            int64_t need = rem - cum + 1;  // the need-th row of block b that chose j
            const int64_t i0 = start + b * KB_BLK, hi = i0 + KB_BLK < n ? i0 + KB_BLK : n;
            for (int64_t base = i0; base < hi; base += 32) {
                const int64_t i = base + lane;
                unsigned mask = __ballot_sync(0xffffffffu, i < hi && choice[i] == j);
                const int cnt = __popc(mask);
                if (need <= cnt) {
                    for (int64_t q = 1; q < need; ++q) mask &= mask - 1;
                    res = base + __ffs(mask) - 1;
                    break;
                }
                need -= cnt;
            }
            break;
        }
        cum += c;
    }
    if (lane == 0) ovf[j] = res;
}

// place rows [start, stop): assign = choice, and add them to the counts
__global__ void kb_accept_kernel(const int32_t *__restrict__ choice, int64_t start, int64_t stop, int32_t p,
                                 int32_t *__restrict__ assign, unsigned long long *__restrict__ cs) {
    extern __shared__ int32_t kb_a[];  // [p]
    for (int j = threadIdx.x; j < p; j += blockDim.x) kb_a[j] = 0;
    __syncthreads();
    for (int64_t i = start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < stop;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = choice[i];
        assign[i] = c;
        atomicAdd(&kb_a[c], 1);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += blockDim.x)
        if (kb_a[j]) atomicAdd(&cs[j], (unsigned long long)kb_a[j]);
}

__global__ void kb_fill_kernel(int32_t *__restrict__ a, int32_t p, int32_t v) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p; j += gridDim.x * blockDim.x) a[j] = v;
}

// close every centre that holds cap rows
__global__ void kb_close_kernel(int32_t *__restrict__ open, const unsigned long long *__restrict__ cs, int32_t p,
                                int64_t cap) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p; j += gridDim.x * blockDim.x)
        if ((int64_t)cs[j] >= cap) open[j] = 0;
}

static inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

krr_status run_gather(Ctx *ctx, const int32_t *assign, int64_t n, int32_t p, int64_t *perm, int64_t *offsets) {
    cudaStream_t st = ctx->stream;
    int64_t nblk = (n + CANON - 1) / CANON;
    long long *bcount = nullptr;
    size_t bytes = (size_t)std::max<int64_t>(nblk, 1) * p * sizeof(long long);
    KRR_CUDA_TRY(ctx, ctx_malloc(ctx, (void **)&bcount, bytes));
    if (nblk > 0) {
        KRR_LAUNCHED(), gather_count_kernel<<<(unsigned)nblk, 256, p * sizeof(int), st>>>(assign, n, p, bcount);
    }
    KRR_CUDA_TRY(ctx, allow_max_dyn_smem(gather_scan_kernel));
    KRR_LAUNCHED(), gather_scan_kernel<<<1, 1024, (size_t)p * sizeof(long long), st>>>(bcount, nblk, p, offsets);
    if (nblk > 0) {
        KRR_LAUNCHED(), gather_scatter_kernel<<<(unsigned)nblk, 128, CANON * sizeof(int32_t), st>>>(assign, n, p, bcount, perm);
    }
    cudaError_t e = cudaGetLastError();
    ctx_free(ctx, bcount, bytes);
    KRR_CUDA_TRY(ctx, e);
    return KRR_OK;
}

static int feistel_half_bits(int64_t n) {
    int b = 2;
    while (b < 62 && ((int64_t)1 << b) < n) b += 2;
    return b / 2;
}

krr_status run_partition_random(Ctx *ctx, int64_t n, int32_t p, uint64_t seed, int32_t *assign, int64_t *perm,
                                int64_t *offsets, int32_t *route, int64_t t) {
    cudaStream_t st = ctx->stream;
    int h = feistel_half_bits(n);
    if (n > 0)
        KRR_LAUNCHED(), random_perm_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, p, h, (uint32_t)seed, (uint32_t)(seed >> 32), perm,
                                                             assign);
    int64_t cover = std::max<int64_t>((int64_t)p + 1, route ? t : 0);
    KRR_LAUNCHED(), random_offsets_kernel<<<std::min<unsigned>(grid_for(cover, 256), 4096u), 256, 0, st>>>(n, p, offsets, route, t);
    KRR_CUDA_TRY(ctx, cudaGetLastError());
    return KRR_OK;
}

krr_status run_assign(Ctx *ctx, const float *X32, const double *X, int64_t n, int32_t d, const double *C64,
                      const float *C32, int32_t k, const int32_t *prev, int32_t *out, unsigned long long *delta) {
    if (n == 0) return KRR_OK;
    const int dp = (d + 7) / 8 * 8, kt = (k + SCR_CT - 1) / SCR_CT * SCR_CT;
    if (dp <= 96 && k <= SCR_KMAX) {
        // screen, then the FP64 recheck of the rows with several candidates
        cudaStream_t st = ctx->stream;
        int32_t *list = nullptr;
        const int64_t nl = (n + 63) / 64 * 64;
        const int64_t pcap = 4 * nl;  // (row, candidate) pairs handed to the pair kernels
        // the listed rows; two counts; ||c||^2 per centre; per listed row the
        // first pair and the pair count; per pair the row, the centre and the
        // FP64 distance
        const int64_t o_cnt = nl, o_cn = nl + 64, o_ps = o_cn + (kt + 63) / 64 * 64, o_pc = o_ps + nl,
                      o_pr = o_pc + nl, o_pj = o_pr + pcap, o_pd = o_pj + pcap;  // in int32 units
        const size_t bl = ((size_t)o_pd + 2 * (size_t)pcap) * sizeof(int32_t);
        KRR_CUDA_TRY(ctx, ctx_malloc(ctx, (void **)&list, bl));
        unsigned int *nlist = reinterpret_cast<unsigned int *>(list + o_cnt);
        unsigned int *npairs = nlist + 1;
        float *cn32 = reinterpret_cast<float *>(list + o_cn);
        int32_t *pstart = list + o_ps, *pcnt = list + o_pc, *prow = list + o_pr, *pj = list + o_pj;
        double *pd = reinterpret_cast<double *>(list + o_pd);
        cudaError_t e = cudaMemsetAsync(nlist, 0, 2 * sizeof(unsigned int), st);
        if (e == cudaSuccess) {
            KRR_LAUNCHED(), centre_norms_kernel<<<(unsigned)((kt * 32 + 255) / 256), 256, 0, st>>>(C32, k, d, kt, cn32);
            e = cudaGetLastError();
        }
        const size_t sm = screen_smem(dp, kt);
        auto launch = [&](auto kern) {
            cudaError_t r = allow_max_dyn_smem(kern);
            if (r == cudaSuccess) {
                KRR_LAUNCHED(), kern<<<grid_for(n, SCR_ROWS), SCR_THREADS, sm, st>>>(X32, n, d, C32, cn32, k, kt,
                                                                                      prev, out, list, nlist, delta);
                r = cudaGetLastError();
            }
            return r;
        };
        if (e == cudaSuccess) {
            switch (dp) {
                case 8: e = launch(kmeans_screen_kernel<8>); break;
                case 16: e = launch(kmeans_screen_kernel<16>); break;
                case 24: e = launch(kmeans_screen_kernel<24>); break;
                case 32: e = launch(kmeans_screen_kernel<32>); break;
                case 40: e = launch(kmeans_screen_kernel<40>); break;
                case 48: e = launch(kmeans_screen_kernel<48>); break;
                case 56: e = launch(kmeans_screen_kernel<56>); break;
                case 64: e = launch(kmeans_screen_kernel<64>); break;
                case 72: e = launch(kmeans_screen_kernel<72>); break;
                case 80: e = launch(kmeans_screen_kernel<80>); break;
                case 88: e = launch(kmeans_screen_kernel<88>); break;
                default: e = launch(kmeans_screen_kernel<96>); break;
            }
        }
        if (e == cudaSuccess) {
            const int64_t g = std::min<int64_t>((n + RCK_WARPS - 1) / RCK_WARPS, 152 * 8);
            KRR_LAUNCHED(), kmeans_recheck_kernel<<<(unsigned)std::max<int64_t>(g, 1), RCK_WARPS * 32, 0, st>>>(
                X32, X, d, C32, C64, cn32, k, list, nlist, prev, out, delta, pstart, pcnt, prow, pj, npairs, pcap);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            KRR_LAUNCHED(), kmeans_pair_dist_kernel<<<152 * 4, 256, 0, st>>>(X, C64, d, prow, pj, npairs, pcap, pd);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            const unsigned gp = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 4));
            KRR_LAUNCHED(), kmeans_pair_pick_kernel<<<gp, 256, 0, st>>>(list, nlist, pstart, pcnt, pj, pd, prev, out,
                                                                         delta);
            e = cudaGetLastError();
        }
        ctx_free(ctx, list, bl);
        if (e != cudaSuccess) {
            ctx->last_error = std::string("kmeans assign: ") + cudaGetErrorString(e);
            return KRR_ERR_CUDA;
        }
        return KRR_OK;
    }
    size_t sm = ((size_t)k * d + k + (size_t)d * ASSIGN_THREADS) * sizeof(float) + 16;
    if (sm > 200 * 1024) {
        ctx->last_error = "kmeans: k*d too large for the shared-memory centre copy";
        return KRR_ERR_UNSUPPORTED;
    }
    if (sm > 48 * 1024)
        KRR_CUDA_TRY(ctx, allow_max_dyn_smem(kmeans_assign_kernel));
    KRR_LAUNCHED(), kmeans_assign_kernel<<<grid_for(n, ASSIGN_THREADS), ASSIGN_THREADS, sm, ctx->stream>>>(
        X32, X, n, d, C64, C32, k, prev, out, delta);
    KRR_CUDA_TRY(ctx, cudaGetLastError());
    return KRR_OK;
}

krr_status run_update(Ctx *ctx, const double *X, int64_t n, int32_t d, const int32_t *c, int32_t k, double *C,
                      double *partial, long long *counts) {
    int64_t nblk = (n + CANON - 1) / CANON;
    if (nblk == 0) return KRR_OK;
    const size_t sm = (2 * (size_t)CANON + 2 * (size_t)k + 1) * sizeof(int32_t);
    const int fcs = (d + 31) / 32;
    if (fcs > 32) {
        ctx->last_error = "kmeans: more than 1024 features";
        return KRR_ERR_UNSUPPORTED;
    }
    const int cgs = std::max(1, std::min(8, 32 / fcs));  // centre groups: up to 1024 threads
    KRR_CUDA_TRY(ctx, allow_max_dyn_smem(kmeans_block_sums_kernel));
    KRR_LAUNCHED(), kmeans_block_sums_kernel<<<(unsigned)nblk, 32 * fcs * cgs, sm, ctx->stream>>>(
        X, n, d, c, k, cgs, partial, counts);
    int te = TREE_MAXTE;  // entries per CTA: both tree levels within ~128 KiB of shared memory
    while (te > 1 && 2 * (size_t)nblk * te * sizeof(double) > 128 * 1024) te /= 2;
    if (2 * (size_t)nblk * te * sizeof(double) > 200 * 1024) {
        ctx->last_error = "kmeans: too many row blocks for the shared-memory centre tree";
        return KRR_ERR_UNSUPPORTED;
    }
    KRR_CUDA_TRY(ctx, allow_max_dyn_smem(kmeans_tree_divide_kernel));
    KRR_LAUNCHED(), kmeans_tree_divide_kernel<<<(unsigned)(((int64_t)k * d + te - 1) / te), TREE_THREADS,
                                                2 * (size_t)nblk * te * sizeof(double), ctx->stream>>>(
        partial, counts, nblk, k, d, te, C);
    KRR_CUDA_TRY(ctx, cudaGetLastError());
    return KRR_OK;
}

// ---- Alg. 2 steps as separate calls (ranks that hold different row blocks
// exchange the block sums between the two halves of the centre update)

// assignment step of rows X [n x d] to the FP64 centres C [k x d]
krr_status run_kmeans_assign_rows(Ctx *ctx, const double *X, int64_t n, int32_t d, const double *C, int32_t k,
                                  int32_t *assign) {
    if (n == 0) return KRR_OK;
    cudaStream_t st = ctx->stream;
    float *X32 = nullptr, *C32 = nullptr;
    const size_t bx = (size_t)n * d * sizeof(float), bc = (size_t)k * d * sizeof(float);
    KRR_CUDA_TRY(ctx, ctx_malloc(ctx, (void **)&X32, bx));
    cudaError_t e = ctx_malloc(ctx, (void **)&C32, bc);
    if (e != cudaSuccess) {
        ctx_free(ctx, X32, bx);
        KRR_CUDA_TRY(ctx, e);
    }
    KRR_LAUNCHED(), to_float_kernel<<<grid_for(n * d, 256), 256, 0, st>>>(X, X32, n * d);
    KRR_LAUNCHED(), to_float_kernel<<<grid_for((int64_t)k * d, 256), 256, 0, st>>>(C, C32, (int64_t)k * d);
    krr_status rc = run_assign(ctx, X32, X, n, d, C, C32, k, nullptr, assign, nullptr);
    ctx_free(ctx, C32, bc);
    ctx_free(ctx, X32, bx);
    return rc;
}

// first half of the centre update: per block of 1024 rows of X (X starts at
// a block boundary of the row numbering), sums [nblk][k][d] and counts [nblk][k]
krr_status run_kmeans_block_sums(Ctx *ctx, const double *X, int64_t n, int32_t d, const int32_t *c, int32_t k,
                                 double *partial, long long *counts) {
    int64_t nblk = (n + CANON - 1) / CANON;
    if (nblk == 0) return KRR_OK;
    const size_t sm = (2 * (size_t)CANON + 2 * (size_t)k + 1) * sizeof(int32_t);
    const int fcs = (d + 31) / 32;
    if (fcs > 32) {
        ctx->last_error = "kmeans: more than 1024 features";
        return KRR_ERR_UNSUPPORTED;
    }
    const int cgs = std::max(1, std::min(8, 32 / fcs));
    KRR_CUDA_TRY(ctx, allow_max_dyn_smem(kmeans_block_sums_kernel));
    KRR_LAUNCHED(), kmeans_block_sums_kernel<<<(unsigned)nblk, 32 * fcs * cgs, sm, ctx->stream>>>(
        X, n, d, c, k, cgs, partial, counts);
    KRR_CUDA_TRY(ctx, cudaGetLastError());
    return KRR_OK;
}

// second half: the pairwise tree over all nblk block sums, one division per
// centre; empty centres keep C
krr_status run_kmeans_combine(Ctx *ctx, const double *partial, const long long *counts, int64_t nblk, int32_t k,
                              int32_t d, double *C) {
    if (nblk == 0) return KRR_OK;
    int te = 32;
    while (te > 1 && 2 * (size_t)nblk * te * sizeof(double) > 128 * 1024) te /= 2;
    if (2 * (size_t)nblk * te * sizeof(double) > 200 * 1024) {
        ctx->last_error = "kmeans: too many row blocks for the shared-memory centre tree";
        return KRR_ERR_UNSUPPORTED;
    }
    KRR_CUDA_TRY(ctx, allow_max_dyn_smem(kmeans_tree_divide_kernel));
    KRR_LAUNCHED(), kmeans_tree_divide_kernel<<<(unsigned)(((int64_t)k * d + te - 1) / te), TREE_THREADS,
                                                2 * (size_t)nblk * te * sizeof(double), ctx->stream>>>(
        partial, counts, nblk, k, d, te, C);
    KRR_CUDA_TRY(ctx, cudaGetLastError());
    return KRR_OK;
}

// Alg. K-balance Clustering's balanced assignment of the n rows to the p
// centres C (cap = ceil(n / p)); see the kernels above.
krr_status run_kbalance(Ctx *ctx, const double *X, int64_t n, int32_t d, const double *C, int32_t p,
                        int32_t *assign) {
    if (n == 0) return KRR_OK;
    cudaStream_t st = ctx->stream;
    const int64_t cap = (n + p - 1) / p;
    const int64_t nblk_max = (n + KB_BLK - 1) / KB_BLK;
    const size_t b_d = (size_t)n * p * sizeof(double), b_ch = (size_t)n * sizeof(int32_t),
                 b_open = (size_t)p * sizeof(int32_t), b_cs = (size_t)p * sizeof(unsigned long long),
                 b_bc = (size_t)nblk_max * p * sizeof(int32_t), b_ovf = (size_t)p * sizeof(long long);
    const size_t sm_d = (size_t)d * KB_ROWS * sizeof(double);
    if (sm_d > 200 * 1024) {
        ctx->last_error = "kbalance: more than 400 features";
        return KRR_ERR_UNSUPPORTED;
    }
    double *D = nullptr;
    int32_t *choice = nullptr, *open = nullptr, *bcnt = nullptr;
    unsigned long long *cs = nullptr;
    long long *ovf = nullptr;
    std::vector<long long> hovf(p);
    krr_status rc = KRR_OK;
    int64_t start = 0;
#define KB_ALLOC(ptr, bytes)                                                  \
    do {                                                                      \
        cudaError_t _e = ctx_malloc(ctx, (void **)&(ptr), (bytes));           \
        if (_e != cudaSuccess) {                                              \
            ctx->last_error = std::string("kbalance workspace: ") + cudaGetErrorString(_e); \
            rc = (_e == cudaErrorMemoryAllocation) ? KRR_ERR_OOM : KRR_ERR_BUDGET; \
            goto done;                                                        \
        }                                                                     \
    } while (0)
    KB_ALLOC(D, b_d);
    KB_ALLOC(choice, b_ch);
    KB_ALLOC(open, b_open);
    KB_ALLOC(cs, b_cs);
    KB_ALLOC(bcnt, b_bc);
    KB_ALLOC(ovf, b_ovf);
    if (sm_d > 48 * 1024 && allow_max_dyn_smem(kb_dist_kernel) != cudaSuccess) {
        rc = KRR_ERR_CUDA;
        goto done;
    }
    KRR_LAUNCHED(), kb_dist_kernel<<<grid_for(n, KB_ROWS), KB_ROWS, sm_d, st>>>(X, n, d, C, p, D);
    KRR_LAUNCHED(), kb_fill_kernel<<<grid_for(p, 256), 256, 0, st>>>(open, p, 1);
    cudaMemsetAsync(cs, 0, b_cs, st);
    for (int round = 0; round <= p && start < n; ++round) {
        KRR_LAUNCHED(), kb_choose_kernel<<<grid_for(n - start, 256), 256, b_open, st>>>(D, n, p, start, open,
                                                                                       round == 0, choice);
        const int64_t nblk = (n - start + KB_BLK - 1) / KB_BLK;
        KRR_LAUNCHED(), kb_count_kernel<<<(unsigned)nblk, 256, b_open, st>>>(choice, n, p, start, bcnt);
        KRR_LAUNCHED(), kb_find_kernel<<<grid_for((int64_t)p * 32, 256), 256, 0, st>>>(bcnt, nblk, p, cs, cap, choice,
                                                                                      n, start, ovf);
        cudaError_t e = cudaMemcpyAsync(hovf.data(), ovf, b_ovf, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            ctx->last_error = std::string("kbalance: ") + cudaGetErrorString(e);
            rc = KRR_ERR_CUDA;
            goto done;
        }
        int64_t stop = n;
        for (int32_t j = 0; j < p; ++j) stop = std::min<int64_t>(stop, hovf[j]);
        if (stop <= start) {  // cannot happen: every open centre has room for at least one row
            ctx->last_error = "kbalance: no progress in a round";
            rc = KRR_ERR_CUDA;
            goto done;
        }
        KRR_LAUNCHED(), kb_accept_kernel<<<std::min<unsigned>(grid_for(stop - start, 256), 1024u), 256, b_open, st>>>(
            choice, start, stop, p, assign, cs);
        start = stop;
        KRR_LAUNCHED(), kb_close_kernel<<<grid_for(p, 256), 256, 0, st>>>(open, cs, p, cap);
    }
    if (start < n) {
        ctx->last_error = "kbalance: rows left after p rounds";
        rc = KRR_ERR_CUDA;
        goto done;
    }
    {
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // workspace is freed below
        if (e != cudaSuccess) {
            ctx->last_error = std::string("kbalance: ") + cudaGetErrorString(e);
            rc = KRR_ERR_CUDA;
        }
    }
done:
#undef KB_ALLOC
    if (ovf) ctx_free(ctx, ovf, b_ovf);
    if (bcnt) ctx_free(ctx, bcnt, b_bc);
    if (cs) ctx_free(ctx, cs, b_cs);
    if (open) ctx_free(ctx, open, b_open);
    if (choice) ctx_free(ctx, choice, b_ch);
    if (D) ctx_free(ctx, D, b_d);
    return rc;
}

krr_status run_partition_kmeans(Ctx *ctx, const double *X, int64_t n, int32_t d, const double *Xt, int64_t t,
                                int32_t k, int32_t iters, const int64_t *init_idx, int32_t *assign, int32_t *route,
                                int64_t *perm, int64_t *offsets, double *C, bool kbalance) {
    cudaStream_t st = ctx->stream;
    int64_t nblk = (n + CANON - 1) / CANON;
    float *C32 = nullptr;
    double *partial = nullptr;
    long long *counts = nullptr;
    int32_t *prev = nullptr;
    unsigned long long *delta = nullptr;
    float *X32 = nullptr, *Xt32 = nullptr;
    size_t b_x32 = (size_t)std::max<int64_t>(n, 1) * d * sizeof(float);
    size_t b_xt32 = (size_t)std::max<int64_t>(t, 1) * d * sizeof(float);
    size_t b_c32 = (size_t)k * d * sizeof(float);
    size_t b_part = (size_t)std::max<int64_t>(nblk, 1) * k * d * sizeof(double);
    size_t b_cnt = (size_t)std::max<int64_t>(nblk, 1) * k * sizeof(long long);
    size_t b_prev = (size_t)std::max<int64_t>(n, 1) * sizeof(int32_t);
    size_t b_delta = (size_t)std::max(iters, 1) * sizeof(unsigned long long);
    krr_status rc = KRR_OK;
#define KM_ALLOC(ptr, bytes)                                                  \
    do {                                                                      \
        cudaError_t _e = ctx_malloc(ctx, (void **)&(ptr), (bytes));           \
        if (_e != cudaSuccess) {                                              \
            ctx->last_error = std::string("kmeans workspace: ") + cudaGetErrorString(_e); \
            rc = (_e == cudaErrorMemoryAllocation) ? KRR_ERR_OOM : KRR_ERR_BUDGET; \
            goto done;                                                        \
        }                                                                     \
    } while (0)
    KM_ALLOC(C32, b_c32);
    KM_ALLOC(partial, b_part);
    KM_ALLOC(counts, b_cnt);
    KM_ALLOC(prev, b_prev);
    KM_ALLOC(delta, b_delta);
    KM_ALLOC(X32, b_x32);
    if (route && t > 0) KM_ALLOC(Xt32, b_xt32);
    {
        if (n > 0) KRR_LAUNCHED(), to_float_kernel<<<grid_for(n * d, 256), 256, 0, st>>>(X, X32, n * d);
        if (Xt32) KRR_LAUNCHED(), to_float_kernel<<<grid_for(t * d, 256), 256, 0, st>>>(Xt, Xt32, t * d);
        cudaMemsetAsync(delta, 0, b_delta, st);
        KRR_LAUNCHED(), init_centres_kernel<<<grid_for((int64_t)k * d, 256), 256, 0, st>>>(X, d, init_idx, k, C);
        for (int it = 0; it < iters; ++it) {
            KRR_LAUNCHED(), to_float_kernel<<<grid_for((int64_t)k * d, 256), 256, 0, st>>>(C, C32, (int64_t)k * d);
            rc = run_assign(ctx, X32, X, n, d, C, C32, k, it == 0 ? nullptr : prev, assign, delta + it);
            if (rc != KRR_OK) goto done;
            rc = run_update(ctx, X, n, d, assign, k, C, partial, counts);
            if (rc != KRR_OK) goto done;
            cudaMemcpyAsync(prev, assign, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
        }
        if (kbalance) {
            // Alg. K-balance Clustering: the balanced assignment to the K-means
            // centres, then the centres as the means of the balanced parts
            rc = run_kbalance(ctx, X, n, d, C, k, assign);
            if (rc != KRR_OK) goto done;
            rc = run_update(ctx, X, n, d, assign, k, C, partial, counts);
            if (rc != KRR_OK) goto done;
            KRR_LAUNCHED(), to_float_kernel<<<grid_for((int64_t)k * d, 256), 256, 0, st>>>(C, C32, (int64_t)k * d);
        } else {
            KRR_LAUNCHED(), to_float_kernel<<<grid_for((int64_t)k * d, 256), 256, 0, st>>>(C, C32, (int64_t)k * d);
            rc = run_assign(ctx, X32, X, n, d, C, C32, k, nullptr, assign, nullptr);
            if (rc != KRR_OK) goto done;
        }
        if (route && t > 0) {
            rc = run_assign(ctx, Xt32, Xt, t, d, C, C32, k, nullptr, route, nullptr);
            if (rc != KRR_OK) goto done;
        }
        rc = run_gather(ctx, assign, n, k, perm, offsets);
        if (rc != KRR_OK) goto done;
        cudaError_t e = cudaStreamSynchronize(st);  // workspace is freed below
        if (e != cudaSuccess) {
            ctx->last_error = std::string("kmeans: ") + cudaGetErrorString(e);
            rc = KRR_ERR_CUDA;
        }
    }
done:
#undef KM_ALLOC
    if (Xt32) ctx_free(ctx, Xt32, b_xt32);
    if (X32) ctx_free(ctx, X32, b_x32);
    if (delta) ctx_free(ctx, delta, b_delta);
    if (prev) ctx_free(ctx, prev, b_prev);
    if (counts) ctx_free(ctx, counts, b_cnt);
    if (partial) ctx_free(ctx, partial, b_part);
    if (C32) ctx_free(ctx, C32, b_c32);
    return rc;
}

}  // namespace krr
