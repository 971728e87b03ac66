// partition.cu -- partitioning kernels (Alg. DC-KRR lines 1-5; Alg. 2 plain
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

// One thread per point.  X32: FP32 copy of the rows (converted once per
// K-means run: on GB300 the FP64 -> FP32 conversion runs on the slow FP64
// pipe); C32 / C64: FP32 and FP64 centres.  The FP32 distance of every centre
// carries the bound |d32 - d64| <= (d + 16) 2^-24 1.27 * 2 (||x||^2 + ||c||^2)
// (rounding of the inputs, the differences, the squares and the sum; the
// factor 2 bounds sum (|x|+|c|)^2).  Centres within the bound of the best
// upper bound are candidates; with two or more, the FP64 distances in the
// definition's order decide (strict <, lowest index).
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
    float best_hi = INFINITY;
#pragma unroll 1
    for (int j = 0; j < k; ++j) {
        const float *c = sC + j * d;
        float acc = 0.f;
        for (int f = 0; f < d; ++f) {
            const float t = sX[f * ASSIGN_THREADS + r] - c[f];
            acc = fmaf(t, t, acc);
        }
        best_hi = fminf(best_hi, acc + bscale * (xn + sCn[j]));
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
        if (acc - bscale * (xn + sCn[j]) <= best_hi) {
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
            if (acc - bscale * (xn + sCn[j]) > best_hi) continue;
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
    }
    out[i] = arg;
    if (delta && (prev == nullptr || prev[i] != arg)) atomicAdd(delta, 1ull);
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
__global__ void kmeans_block_sums_kernel(const double *__restrict__ X, int64_t n, int32_t d,
                                         const int32_t *__restrict__ c, int32_t k, double *__restrict__ partial,
                                         long long *__restrict__ counts) {
    extern __shared__ unsigned char smem_raw[];
    double *S = reinterpret_cast<double *>(smem_raw);  // k*d
    int32_t *sc = reinterpret_cast<int32_t *>(S + (size_t)k * d);
    int64_t b = blockIdx.x;
    int64_t lo = b * CANON, hi = min(n, lo + CANON);
    for (int e = threadIdx.x; e < k * d; e += blockDim.x) S[e] = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) sc[i - lo] = c[i];
    __syncthreads();
    for (int f = threadIdx.x; f < d; f += blockDim.x) {
        for (int64_t i = lo; i < hi; ++i) {
            int j = sc[i - lo];
            S[(size_t)j * d + f] = __dadd_rn(S[(size_t)j * d + f], X[i * d + f]);
        }
    }
    __syncthreads();
    double *P = partial + b * (int64_t)k * d;
    for (int e = threadIdx.x; e < k * d; e += blockDim.x) P[e] = S[e];
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        long long cnt = 0;
        for (int64_t i = lo; i < hi; ++i) cnt += (sc[i - lo] == j);
        counts[b * k + j] = cnt;
    }
}

// thread per (cluster, feature): pairwise tree over blocks in place, then divide
__global__ void kmeans_tree_divide_kernel(double *__restrict__ partial, const long long *__restrict__ counts,
                                          int64_t nblk, int32_t k, int32_t d, double *__restrict__ C) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)k * d) return;
    int j = (int)(e / d);
    const int64_t stride = (int64_t)k * d;
    int64_t len = nblk;
    while (len > 1) {
        int64_t half = (len + 1) / 2;
        for (int64_t q = 0; q < half; ++q) {
            double a = partial[(2 * q) * stride + e];
            double v = (2 * q + 1 < len) ? __dadd_rn(a, partial[(2 * q + 1) * stride + e]) : a;
            partial[q * stride + e] = v;
        }
        len = half;
    }
    long long cnt = 0;
    for (int64_t b = 0; b < nblk; ++b) cnt += counts[b * k + j];
    if (cnt > 0) C[e] = __ddiv_rn(partial[e], (double)cnt);
}

// ------------------------------------------------------------ stable gather
__global__ void gather_count_kernel(const int32_t *__restrict__ a, int64_t n, int32_t p,
                                    long long *__restrict__ bcount) {
    extern __shared__ unsigned char smem_raw[];
    int *h = reinterpret_cast<int *>(smem_raw);
    for (int j = threadIdx.x; j < p; j += blockDim.x) h[j] = 0;
    __syncthreads();
    int64_t lo = (int64_t)blockIdx.x * CANON, hi = min(n, lo + CANON);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&h[a[i]], 1);
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += blockDim.x) bcount[(int64_t)blockIdx.x * p + j] = h[j];
}

// one thread per partition: offsets and per-block starting positions
__global__ void gather_scan_kernel(long long *__restrict__ bcount, int64_t nblk, int32_t p,
                                   int64_t *__restrict__ offsets) {
    __shared__ long long tot_sh[1];
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        long long run = 0;
        for (int j = 0; j < p; ++j) {
            offsets[j] = run;
            for (int64_t b = 0; b < nblk; ++b) {
                long long c = bcount[b * p + j];
                bcount[b * p + j] = run;
                run += c;
            }
        }
        offsets[p] = run;
        tot_sh[0] = run;
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
    KRR_LAUNCHED(), gather_scan_kernel<<<1, 32, 0, st>>>(bcount, nblk, p, offsets);
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
    size_t sm = (size_t)k * d * sizeof(double) + CANON * sizeof(int32_t);
    if (sm > 200 * 1024) {
        ctx->last_error = "kmeans: k*d too large for the shared-memory block sums";
        return KRR_ERR_UNSUPPORTED;
    }
    if (sm > 48 * 1024)
        KRR_CUDA_TRY(ctx, allow_max_dyn_smem(kmeans_block_sums_kernel));
    KRR_LAUNCHED(), kmeans_block_sums_kernel<<<(unsigned)nblk, 128, sm, ctx->stream>>>(X, n, d, c, k, partial, counts);
    KRR_LAUNCHED(), kmeans_tree_divide_kernel<<<grid_for((int64_t)k * d, 128), 128, 0, ctx->stream>>>(partial, counts, nblk, k, d,
                                                                                     C);
    KRR_CUDA_TRY(ctx, cudaGetLastError());
    return KRR_OK;
}

krr_status run_partition_kmeans(Ctx *ctx, const double *X, int64_t n, int32_t d, const double *Xt, int64_t t,
                                int32_t k, int32_t iters, const int64_t *init_idx, int32_t *assign, int32_t *route,
                                int64_t *perm, int64_t *offsets, double *C) {
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
        KRR_LAUNCHED(), to_float_kernel<<<grid_for((int64_t)k * d, 256), 256, 0, st>>>(C, C32, (int64_t)k * d);
        rc = run_assign(ctx, X32, X, n, d, C, C32, k, nullptr, assign, nullptr);
        if (rc != KRR_OK) goto done;
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
