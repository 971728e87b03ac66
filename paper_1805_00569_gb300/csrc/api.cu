// api.cu -- the C ABI of libkrr (declared in include/krr.h): context and
// budget, model lifetime, and the orchestration of the hot path
//   krr_partition -> krr_fit_batch -> krr_predict -> krr_select.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <set>

#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

struct krr_ctx {
    krr::Ctx c;
};
struct krr_model {
    krr::Model m;
};

namespace krr {

std::atomic<long long> g_launch_count{0};

// ---- defined in the other translation units
krr_status run_partition_random(Ctx *, int64_t, int32_t, uint64_t, int32_t *, int64_t *, int64_t *, int32_t *,
                                int64_t);
krr_status run_partition_kmeans(Ctx *, const double *, int64_t, int32_t, const double *, int64_t, int32_t, int32_t,
                                const int64_t *, int32_t *, int32_t *, int64_t *, int64_t *, double *, bool);
krr_status run_gather(Ctx *, const int32_t *, int64_t, int32_t, int64_t *, int64_t *);
krr_status run_kmeans_assign_rows(Ctx *, const double *, int64_t, int32_t, const double *, int32_t, int32_t *);
krr_status run_kmeans_block_sums(Ctx *, const double *, int64_t, int32_t, const int32_t *, int32_t, double *,
                                 long long *);
krr_status run_kmeans_combine(Ctx *, const double *, const long long *, int64_t, int32_t, int32_t, double *);
void launch_stage(cudaStream_t, const double *, const double *, const int64_t *, const Model &, double *);
void launch_kbuild_df(cudaStream_t, const Model &, int64_t, float *, float *, float *);
void launch_kbuild_fp64(cudaStream_t, const Model &, int64_t, double *, double *);
void launch_k64_abs_rowsums(cudaStream_t, const Model &, int64_t, const double *, float *, float *, const int64_t *,
                            int64_t);
struct CholLaunch {
    int kind;
    int K0, W;
    int64_t pre;
    int64_t tasks;
    int tc;
};
void build_chol_plan(const std::vector<int> &, const std::vector<int> &, int, std::vector<CholLaunch> &,
                     std::vector<int64_t> &);
cudaError_t run_chol_plan(cudaStream_t, const std::vector<CholLaunch> &, const int64_t *, void *, void *, bool,
                          const SolveDesc *, int, int32_t *, int, const CUtensorMap *, const CUtensorMap *, __half *,
                          const CUtensorMap *, float *, const CUtensorMap *, const float *, const CUtensorMap *, int *,
                          Prof *);
bool make_tile_tmap(CUtensorMap *, float *, int64_t);
bool make_tile_tmap16(CUtensorMap *, __half *, int64_t);
size_t pcg_state_size();
size_t precond_smem_bytes(bool, int);
cudaError_t run_pcg(cudaStream_t, const Model &, const PcgBuffers &, const float *, const float *, const double *,
                    const void *, const void *, bool, int, double, double, int, const int32_t *, unsigned int *, int,
                    Prof *);
cudaError_t run_pcg_norms(cudaStream_t, const Model &, const PcgBuffers &, const float *, const float *,
                          const double *, bool, Prof *);
void launch_predict(cudaStream_t, const Model &, const double *, int64_t, const int64_t *, const int64_t *, int64_t,
                    int, double *);
void launch_select(cudaStream_t, const double *, const double *, int64_t, int, int, int, double *, int32_t *);
int oz_dpz(int d);
bool oz_supported(int d);
void launch_oz_slice(cudaStream_t, const double *, int, const int64_t *, int64_t, int64_t, void *, int32_t *, float2 *);
bool make_slice_tmap(CUtensorMap *, void *, int64_t, int, int);
cudaError_t launch_kbuild_oz(cudaStream_t, const Model &, int64_t, float *, float *, float *, float *, float *,
                             const int64_t *, int64_t, int *, bool, const float2 *);
cudaError_t launch_predict_oz(cudaStream_t, const Model &, const CUtensorMap &, const double *, int64_t,
                              const int64_t *, const int64_t *, int, void *, int32_t *, float2 *, int64_t, double *,
                              int *);

// ---- kernel attributes
cudaError_t allow_max_dyn_smem_fn(const void *fn) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (done.count({fn, dev})) return cudaSuccess;
    }
    int optin = 0;
    cudaFuncAttributes fa;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - (int)fa.sharedSizeBytes)) != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lk(mu);
    done.insert({fn, dev});
    return cudaSuccess;
}

// ---- budgeted stream-ordered allocation
cudaError_t ctx_malloc(Ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    if (c->budget && c->used + bytes > c->budget) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, c->pool, c->stream);
    if (e == cudaSuccess) c->used += bytes;
    return e;
}
void ctx_free(Ctx *c, void *p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    cudaFreeAsync(p, c->stream);
    c->used -= std::min(c->used, bytes);
}

// ---- small kernels of the fit
__global__ void fill_rhs_kernel(const SolveDesc *__restrict__ solves, const PartDesc *__restrict__ parts,
                                const double *__restrict__ yg, double *__restrict__ y) {
    const SolveDesc S = solves[blockIdx.x];
    const PartDesc P = parts[S.part];
    for (int e = threadIdx.x; e < S.T * KRR_TILE; e += blockDim.x) y[S.vec0 + e] = yg[P.prow0 + e];
}
__global__ void export_kernel(const SolveDesc *__restrict__ solves, const PartDesc *__restrict__ parts, int G,
                              const double *__restrict__ x, const PcgState *__restrict__ state,
                              int32_t *__restrict__ status, double *__restrict__ alpha_out) {
    const int s = blockIdx.x;
    const SolveDesc S = solves[s];
    const PartDesc P = parts[S.part];
    if (threadIdx.x == 0 && status) status[s] = state[s].status;
    if (alpha_out) {
        const int g = s % G;
        double *dst = alpha_out + P.row0 * G + (int64_t)g * S.m;
        for (int e = threadIdx.x; e < S.m; e += blockDim.x) dst[e] = x[S.vec0 + e];
    }
}
// refill the factor tiles of the listed solves with K_hi + (lambda m + shift) I
__global__ void reform_kernel(const SolveDesc *__restrict__ sub, const int64_t *__restrict__ pre, int nsub,
                              const float *__restrict__ Kh, float *__restrict__ A, float shift) {
    int lo = 0, hi = nsub - 1;
    const int64_t b = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const SolveDesc S = sub[lo];
    const int64_t lt = b - pre[lo];
    int ti, tj;
    tri_decode(lt, ti, tj);
    const float *src = Kh + (S.ktile0 + lt) * KRR_TILE_ELEMS;
    float *dst = A + (S.ltile0 + lt) * KRR_TILE_ELEMS;
    for (int e = threadIdx.x; e < KRR_TILE_ELEMS; e += blockDim.x) {
        const int r = e >> 7, c = e & 127;
        const int gr = ti * KRR_TILE + r, gc = tj * KRR_TILE + c;
        dst[e] = src[e] + ((gr == gc && gr < S.m) ? (float)S.lambda_m + shift : 0.f);
    }
}

// A wait that nothing completes while a bulk copy of the CTA's own is in
// flight: the deadline path of the pipelined kernels in miniature.  Every
// thread waits on bars[1], which never gets an arrival, until limit_ns
// passes; then the CTA waits (bounded) for its copy on bars[0] to land before
// it exits, and thread 0 reports the sum of the landed data (-1 if the
// never-completed wait returned as completed).
__global__ void wait_probe_kernel(const float4 *__restrict__ src, float *__restrict__ sum_out, int *err,
                                  uint64_t limit_ns) {
    __shared__ __align__(128) float4 buf[256];  // 4 KB landing zone of the copy
    __shared__ __align__(8) uint64_t bars[2];
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bars[0], (uint32_t)sizeof(buf));
        bulk_g2s(buf, src, (uint32_t)sizeof(buf), &bars[0]);
    }
    const bool got = mbar_wait_until(&bars[1], 0, err, limit_ns, KRR_ERR_TIMEOUT);
    const bool landed = mbar_wait_until(&bars[0], 0, err, KRR_WAIT_LIMIT_NS, KRR_ERR_TIMEOUT);
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; landed && i < 256; ++i) s += (buf[i].x + buf[i].y) + (buf[i].z + buf[i].w);
        sum_out[0] = got ? -1.f : (landed ? s : -2.f);
    }
}

// alpha as double-float pairs, formed once per fit: the prediction's
// contraction then runs with no FP64 instruction (GB300's FP64 pipe runs at
// 1/64 of the FP32 rate)
__global__ void alpha_pairs_kernel(const double *__restrict__ a, float2 *__restrict__ a2, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = a[i];
    const float h = __double2float_rn(v);
    a2[i] = make_float2(h, __double2float_rn(v - (double)h));
}

struct DevBuf {
    Ctx *c;
    std::vector<std::pair<void *, size_t>> list;
    explicit DevBuf(Ctx *c_) : c(c_) {}
    template <typename T>
    cudaError_t get(T **p, size_t bytes) {
        cudaError_t e = ctx_malloc(c, (void **)p, bytes);
        if (e == cudaSuccess) list.push_back({(void *)*p, bytes});
        return e;
    }
    ~DevBuf() {
        for (auto &a : list) ctx_free(c, a.first, a.second);
    }
};

static krr_status fail(Ctx *c, krr_status s, const std::string &msg) {
    c->last_error = msg;
    return s;
}

static void free_model(Ctx *c, Model &M) {
    for (auto &a : M.allocs) ctx_free(c, a.first, a.second);
    M.allocs.clear();
}

template <typename T>
static cudaError_t model_alloc(Ctx *c, Model &M, T **p, size_t bytes) {
    cudaError_t e = ctx_malloc(c, (void **)p, bytes);
    if (e == cudaSuccess) M.allocs.push_back({(void *)*p, bytes});
    return e;
}

}  // namespace krr

using namespace krr;

#define API_TRY(ctxp, expr)                                                                  \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess) {                                                             \
            (ctxp)->last_error = std::string(#expr) + ": " + cudaGetErrorString(_e);        \
            return (_e == cudaErrorMemoryAllocation)                                         \
                       ? ((ctxp)->budget ? KRR_ERR_BUDGET : KRR_ERR_OOM)                    \
                       : KRR_ERR_CUDA;                                                       \
        }                                                                                    \
    } while (0)

extern "C" {

krr_status krr_ctx_create(krr_ctx **out, int device, void *cuda_stream, size_t hbm_budget_bytes) {
    if (!out) return KRR_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return KRR_ERR_ARG;
    krr_ctx *k = new (std::nothrow) krr_ctx();
    if (!k) return KRR_ERR_OOM;
    k->c.device = device;
    k->c.stream = (cudaStream_t)cuda_stream;
    k->c.budget = hbm_budget_bytes;
    // A private pool whose freed blocks stay mapped (release threshold: never):
    // with the default threshold a stream synchronisation returns freed memory
    // to the driver and the next fit maps it again, which costs milliseconds.
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    uint64_t keep = UINT64_MAX;
    if (cudaSetDevice(device) != cudaSuccess || cudaMemPoolCreate(&k->c.pool, &pp) != cudaSuccess ||
        cudaMemPoolSetAttribute(k->c.pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
        cudaMalloc(&k->c.d_err, sizeof(int)) != cudaSuccess || cudaMemset(k->c.d_err, 0, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&k->c.h_flag, sizeof(unsigned int)) != cudaSuccess) {
        if (k->c.pool) cudaMemPoolDestroy(k->c.pool);
        delete k;
        return KRR_ERR_CUDA;
    }
    *out = k;
    return KRR_OK;
}

krr_status krr_ctx_destroy(krr_ctx *ctx) {
    if (!ctx) return KRR_ERR_ARG;
    cudaStreamSynchronize(ctx->c.stream);
    for (auto e : ctx->c.prof.pool) cudaEventDestroy(e);
    cudaFree(ctx->c.d_err);
    cudaFreeHost(ctx->c.h_flag);
    // blocks still held by live models keep the pool's memory until they are freed
    cudaMemPoolDestroy(ctx->c.pool);
    delete ctx;
    return KRR_OK;
}

long long krr_launch_count(void) { return g_launch_count.load(); }

const char *krr_last_error(const krr_ctx *ctx) { return ctx ? ctx->c.last_error.c_str() : "null context"; }

size_t krr_ctx_bytes_in_use(const krr_ctx *ctx) { return ctx ? ctx->c.used : 0; }

// Per-kernel-class timing (not part of krr.h's core path; used by benchmarks).
krr_status krr_ctx_set_profiling(krr_ctx *ctx, int on) {
    if (!ctx) return KRR_ERR_ARG;
    ctx->c.prof.on = on != 0;
    ctx->c.prof.reset();
    return KRR_OK;
}
krr_status krr_ctx_profile(krr_ctx *ctx, int kind, double *total_ms, long long *launches) {
    if (!ctx || kind < 0 || kind >= PROF_NKINDS) return KRR_ERR_ARG;
    cudaStreamSynchronize(ctx->c.stream);
    ctx->c.prof.collect();
    if (total_ms) *total_ms = ctx->c.prof.total_ms[kind];
    if (launches) *launches = ctx->c.prof.launches[kind];
    return KRR_OK;
}
krr_status krr_ctx_get_panel_width(const krr_ctx *ctx, int prec, int max_tiles, int *W) {
    if (!ctx || !W) return KRR_ERR_ARG;
    auto it = ctx->c.tuned_W.find(std::make_pair(prec, max_tiles));
    *W = ctx->c.chol_W > 0 ? ctx->c.chol_W : (it == ctx->c.tuned_W.end() ? 0 : it->second);
    return KRR_OK;
}

krr_status krr_ctx_set_target_error(krr_ctx *ctx, double rel) {
    if (!ctx || !(rel >= 0.0) || rel > 1e-2) return KRR_ERR_ARG;
    ctx->c.target_err = rel;
    return KRR_OK;
}

krr_status krr_ctx_set_fp64_fallback(krr_ctx *ctx, int on) {
    if (!ctx) return KRR_ERR_ARG;
    ctx->c.fp64_fallback = on != 0;
    return KRR_OK;
}

krr_status krr_ctx_set_escalation(krr_ctx *ctx, double kappa_u) {
    if (!ctx || !(kappa_u >= 0.0)) return KRR_ERR_ARG;
    ctx->c.escalate = kappa_u;
    return KRR_OK;
}

krr_status krr_group_rows(krr_ctx *ctx, const int32_t *assign, int64_t n, int32_t p, int64_t *perm,
                          int64_t *offsets) {
    if (!ctx) return KRR_ERR_ARG;
    Ctx *c = &ctx->c;
    if (n < 0 || p <= 0 || !offsets || (n > 0 && (!assign || !perm)))
        return fail(c, KRR_ERR_ARG, "krr_group_rows: invalid argument");
    if ((int64_t)p * 4 > 48 * 1024) return fail(c, KRR_ERR_ARG, "krr_group_rows: p above 12288");
    cudaSetDevice(c->device);
    ProfScope ps(c->prof.on ? &c->prof : nullptr, PROF_PARTITION, c->stream);
    return run_gather(c, assign, n, p, perm, offsets);
}

krr_status krr_kmeans_assign(krr_ctx *ctx, const double *X, int64_t n, int32_t d, const double *C, int32_t k,
                             int32_t *assign) {
    if (!ctx) return KRR_ERR_ARG;
    Ctx *c = &ctx->c;
    if (n < 0 || d <= 0 || k <= 0 || !C || (n > 0 && (!X || !assign)))
        return fail(c, KRR_ERR_ARG, "krr_kmeans_assign: invalid argument");
    cudaSetDevice(c->device);
    ProfScope ps(c->prof.on ? &c->prof : nullptr, PROF_PARTITION, c->stream);
    return run_kmeans_assign_rows(c, X, n, d, C, k, assign);
}

krr_status krr_kmeans_block_sums(krr_ctx *ctx, const double *X, int64_t n, int32_t d, const int32_t *assign,
                                 int32_t k, double *sums, int64_t *counts) {
    if (!ctx) return KRR_ERR_ARG;
    Ctx *c = &ctx->c;
    if (n < 0 || d <= 0 || k <= 0 || (n > 0 && (!X || !assign || !sums || !counts)))
        return fail(c, KRR_ERR_ARG, "krr_kmeans_block_sums: invalid argument");
    cudaSetDevice(c->device);
    ProfScope ps(c->prof.on ? &c->prof : nullptr, PROF_PARTITION, c->stream);
    return run_kmeans_block_sums(c, X, n, d, assign, k, sums, reinterpret_cast<long long *>(counts));
}

krr_status krr_kmeans_combine(krr_ctx *ctx, const double *sums, const int64_t *counts, int64_t nblk, int32_t k,
                              int32_t d, double *C) {
    if (!ctx) return KRR_ERR_ARG;
    Ctx *c = &ctx->c;
    if (nblk < 0 || d <= 0 || k <= 0 || !C || (nblk > 0 && (!sums || !counts)))
        return fail(c, KRR_ERR_ARG, "krr_kmeans_combine: invalid argument");
    cudaSetDevice(c->device);
    ProfScope ps(c->prof.on ? &c->prof : nullptr, PROF_PARTITION, c->stream);
    return run_kmeans_combine(c, sums, reinterpret_cast<const long long *>(counts), nblk, k, d, C);
}

krr_status krr_ctx_wait_probe(krr_ctx *ctx, double seconds) {
    if (!ctx) return KRR_ERR_ARG;
    Ctx *c = &ctx->c;
    if (!(seconds >= 1e-6 && seconds <= 10.0)) return fail(c, KRR_ERR_ARG, "krr_ctx_wait_probe: seconds outside [1e-6, 10]");
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    const size_t bytes = 4096 + 256;
    void *buf = nullptr;
    API_TRY(c, ctx_malloc(c, &buf, bytes));
    float ones[1024];
    for (int i = 0; i < 1024; ++i) ones[i] = 1.0f;
    float sum = 0.f;
    int herr = 0;
    cudaError_t e = cudaMemsetAsync(c->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf, ones, sizeof(ones), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        KRR_LAUNCHED(), wait_probe_kernel<<<1, 128, 0, st>>>((const float4 *)buf, (float *)((char *)buf + 4096),
                                                              c->d_err, (uint64_t)(seconds * 1e9));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sum, (char *)buf + 4096, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    ctx_free(c, buf, bytes);
    API_TRY(c, e);
    if (sum != 1024.0f) return fail(c, KRR_ERR_CUDA, "krr_ctx_wait_probe: the copy in flight did not land intact");
    if (herr != KRR_ERR_TIMEOUT) return fail(c, KRR_ERR_CUDA, "krr_ctx_wait_probe: the wait did not report expiry");
    return fail(c, KRR_ERR_TIMEOUT, "krr_ctx_wait_probe: the bounded wait expired as designed");
}

krr_status krr_ctx_set_kernel(krr_ctx *ctx, krr_kernel kind) {
    if (!ctx || (kind != KRR_KERNEL_GAUSSIAN && kind != KRR_KERNEL_LINEAR)) return KRR_ERR_ARG;
    ctx->c.kernel = kind;
    return KRR_OK;
}

krr_status krr_ctx_set_panel_width(krr_ctx *ctx, int W) {
    if (!ctx || W < 0 || W > 64) return KRR_ERR_ARG;
    ctx->c.chol_W = W;
    return KRR_OK;
}

krr_status krr_partition(krr_ctx *ctx, const double *X, int64_t n, int32_t d, const double *Xt, int64_t t,
                         krr_part_mode mode, int32_t p, int32_t iters, uint64_t seed, const int64_t *init_idx,
                         int32_t *assign, int32_t *route, int64_t *perm, int64_t *offsets, double *centers) {
    if (!ctx) return KRR_ERR_ARG;
    Ctx *c = &ctx->c;
    if (n < 0 || d <= 0 || p <= 0 || t < 0 || !assign || !perm || !offsets || (n > 0 && !X) ||
        (t > 0 && route && !Xt))
        return fail(c, KRR_ERR_ARG, "krr_partition: invalid argument");
    if (p > n && n > 0 && mode != KRR_PART_RANDOM) return fail(c, KRR_ERR_ARG, "krr_partition: p > n");
    cudaSetDevice(c->device);
    ProfScope ps(&c->prof, PROF_PARTITION, c->stream);
    if (mode == KRR_PART_RANDOM) return run_partition_random(c, n, p, seed, assign, perm, offsets, route, t);
    if (mode == KRR_PART_KMEANS || mode == KRR_PART_KBALANCE) {
        if (!init_idx || !centers || iters < 0)
            return fail(c, KRR_ERR_ARG, "krr_partition: K-means and K-balance need init_idx and centers");
        return run_partition_kmeans(c, X, n, d, Xt, t, p, iters, init_idx, assign, route, perm, offsets, centers,
                                    mode == KRR_PART_KBALANCE);
    }
    return fail(c, KRR_ERR_ARG, "krr_partition: unknown mode");
}

// The fit of krr_fit_batch (a sigma x lambda grid shared by all partitions)
// and of krr_fit_jobs (per_part: one sigma and one lambda per partition, given
// in sigmas[p] / lambdas[p], with ns = nl = 1).
static krr_status fit_impl(krr_ctx *ctx, const double *X, const double *y, int64_t n, int32_t d,
                           const int64_t *perm, const int64_t *offsets, int32_t p, const double *sigmas, int32_t ns,
                           const double *lambdas, int32_t nl, krr_prec prec, krr_model **out,
                           int32_t *solve_status, double *alpha, bool per_part) {
    if (!ctx) return KRR_ERR_ARG;
    Ctx *c = &ctx->c;
    if (!out || !X || !y || !perm || !offsets || !sigmas || !lambdas || n <= 0 || d <= 0 || p <= 0 || ns <= 0 ||
        nl <= 0 || ns > 8 || nl > 8 || (prec != KRR_PREC_FP64 && prec != KRR_PREC_FP32 && prec != KRR_PREC_TF32 && prec != KRR_PREC_BF16X3))
        return fail(c, KRR_ERR_ARG, "krr_fit_batch: invalid argument (1 <= ns, nl <= 8)");
    const int nsv = per_part ? p : ns, nlv = per_part ? p : nl;  // values given
    for (int i = 0; i < nsv; ++i)
        if (!(sigmas[i] > 0.0) || !std::isfinite(sigmas[i]))
            return fail(c, KRR_ERR_ARG, "krr_fit_batch: sigma must be positive and finite");
    for (int i = 0; i < nlv; ++i)
        if (!std::isfinite(lambdas[i])) return fail(c, KRR_ERR_ARG, "krr_fit_batch: lambda must be finite");
    if (per_part && (prec == KRR_PREC_FP64 || !oz_supported(d) || c->kernel != KRR_KERNEL_GAUSSIAN))
        return fail(c, KRR_ERR_UNSUPPORTED,
                    "krr_fit_jobs: needs a refined precision, the Gaussian kernel and d <= 96");
    *out = nullptr;
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    const bool fp64 = prec == KRR_PREC_FP64;
    const bool tf32 = prec == KRR_PREC_TF32;
    const bool bf16x3 = prec == KRR_PREC_BF16X3;
    Prof *prof = c->prof.on ? &c->prof : nullptr;

    // partition sizes on the host
    std::vector<int64_t> off(p + 1);
    API_TRY(c, cudaMemcpyAsync(off.data(), offsets, sizeof(int64_t) * (p + 1), cudaMemcpyDeviceToHost, st));
    API_TRY(c, cudaStreamSynchronize(st));
    if (off[0] != 0 || off[p] > n) return fail(c, KRR_ERR_ARG, "krr_fit_batch: offsets must run from 0 to at most n");
    for (int j = 0; j < p; ++j)
        if (off[j + 1] < off[j]) return fail(c, KRR_ERR_ARG, "krr_fit_batch: offsets must be non-decreasing");

    if (c->kernel == KRR_KERNEL_LINEAR && !fp64)
        return fail(c, KRR_ERR_UNSUPPORTED, "krr_fit_batch: the linear kernel needs KRR_PREC_FP64");
    krr_model *km = new (std::nothrow) krr_model();
    if (!km) return KRR_ERR_OOM;
    Model &M = km->m;
    M.kind = c->kernel;
    M.d = d;
    M.dp = ((d + 15) / 16) * 16;
    M.p = p;
    M.nsig = ns;
    M.nlam = nl;
    M.prec = prec;
    M.n = n;
    M.sigmas.assign(sigmas, sigmas + nsv);
    M.lambdas.assign(lambdas, lambdas + nlv);
    M.per_part = per_part;
    const int G = ns * nl;
    int64_t prow = 0, ktot = 0;
    int maxT = 0;
    for (int j = 0; j < p; ++j) {
        PartDesc P;
        P.m = (int32_t)(off[j + 1] - off[j]);
        P.T = (P.m + KRR_TILE - 1) / KRR_TILE;
        P.row0 = off[j];
        P.prow0 = prow;
        P.ktile0 = ktot;
        prow += (int64_t)P.T * KRR_TILE;
        ktot += tri(P.T);
        maxT = std::max(maxT, P.T);
        M.parts.push_back(P);
    }
    M.prows = prow;
    int64_t ltiles = 0, dtiles = 0, vec = 0, scratch = 0;
    std::vector<GroupDesc> groups;
    std::vector<int64_t> gpre;
    for (int j = 0; j < p; ++j) {
        const PartDesc &P = M.parts[j];
        for (int is = 0; is < ns; ++is) {
            GroupDesc Gd;
            Gd.part = j;
            Gd.isig = is;
            Gd.T = P.T;
            Gd.nlam = nl;
            Gd.ktile0 = (int64_t)is * ktot + P.ktile0;
            Gd.solve0 = (int64_t)j * G + is * nl;
            Gd.scratch0 = scratch;
            scratch += (int64_t)nl * P.T * P.T * KRR_TILE;
            gpre.push_back(groups.empty() ? 0 : gpre.back() + tri(groups.back().T));
            groups.push_back(Gd);
            for (int il = 0; il < nl; ++il) {
                SolveDesc S;
                S.part = j;
                S.isig = is;
                S.ilam = il;
                S.T = P.T;
                S.m = P.m;
                S.grp = j * ns + is;
                S.cls = 0;
                S.pad0 = 0;
                S.lotile0 = -1;
                S.ltile0 = ltiles;
                S.dtile0 = dtiles;
                S.ktile0 = Gd.ktile0;
                S.vec0 = vec;
                S.lambda_m = (per_part ? lambdas[j] : lambdas[il]) * (double)P.m;
                ltiles += tri(P.T);
                dtiles += P.T;
                vec += (int64_t)P.T * KRR_TILE;
                M.solves.push_back(S);
            }
        }
    }
    const int64_t gtiles = groups.empty() ? 0 : gpre.back() + tri(groups.back().T);
    M.nvec = vec;
    const int nsolve = (int)M.solves.size();
    const size_t esz = fp64 ? 8 : 4;
    if (precond_smem_bytes(fp64, maxT) > 200 * 1024) {
        delete km;
        return fail(c, KRR_ERR_UNSUPPORTED, "krr_fit_batch: partition too large for the preconditioner (m <= " +
                                                std::to_string(fp64 ? 24000 : 48000) + ")");
    }

    // ---- budget check before any allocation
    int64_t rs_slots = 0;  // row-sum tile slots of the exact-Gram tile build: sum of T^2
    for (const PartDesc &P : M.parts) rs_slots += (int64_t)P.T * P.T;
    const size_t tileb = (size_t)KRR_TILE_ELEMS * esz;
    size_t model_bytes = (size_t)prow * d * 8 + 2 * (size_t)prow * M.dp * 4 + (size_t)prow * 8 + (size_t)vec * 16 +
                         (size_t)prow * (10 * (size_t)((d + 31) / 32 * 32) + 4) +
                         sizeof(PartDesc) * p + sizeof(SolveDesc) * nsolve + 8 * 256;
    size_t work_bytes = (size_t)prow * 8 + (fp64 ? 1 : 2) * (size_t)ns * ktot * tileb + (size_t)ltiles * tileb +
                        (size_t)dtiles * tileb + 6 * (size_t)vec * 8 + (size_t)scratch * 8 +
                        (tf32 ? (size_t)ltiles * KRR_TILE_ELEMS * 2 : 0) + (fp64 ? 0 : (size_t)ltiles * tileb) +
                        (fp64 ? 0 : (size_t)ns * rs_slots * 9 * KRR_TILE * sizeof(float)) +
                        pcg_state_size() * nsolve + sizeof(GroupDesc) * groups.size() + 8 * gpre.size() +
                        8 * nsolve + 64 * 1024 * 1024;
    if (c->budget && c->used + model_bytes + work_bytes > c->budget) {
        delete km;
        return fail(c, KRR_ERR_BUDGET, "krr_fit_batch: needs " + std::to_string(model_bytes + work_bytes) +
                                           " bytes, budget leaves " + std::to_string(c->budget - c->used));
    }

    auto bail = [&](krr_status s, const std::string &msg) {
        free_model(c, M);
        delete km;
        return fail(c, s, msg);
    };
#define FIT_TRY(expr)                                                                        \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess)                                                               \
            return bail(_e == cudaErrorMemoryAllocation ? KRR_ERR_OOM : KRR_ERR_CUDA,       \
                        std::string(#expr) + ": " + cudaGetErrorString(_e));                 \
    } while (0)

    FIT_TRY(model_alloc(c, M, &M.X64, (size_t)prow * d * 8));
    FIT_TRY(model_alloc(c, M, &M.Xh, (size_t)prow * M.dp * 4));
    FIT_TRY(model_alloc(c, M, &M.Xl, (size_t)prow * M.dp * 4));
    FIT_TRY(model_alloc(c, M, &M.nrm, (size_t)prow * 8));
    FIT_TRY(model_alloc(c, M, &M.alpha, (size_t)vec * 8));
    FIT_TRY(model_alloc(c, M, &M.d_parts, sizeof(PartDesc) * p));
    FIT_TRY(model_alloc(c, M, &M.d_solves, sizeof(SolveDesc) * nsolve));
    std::vector<float2> hcpart;  // per_part: -1 / (2 sigma_j^2) as df
    if (per_part) {
        for (int j = 0; j < p; ++j) {
            const double cv = -1.0 / (2.0 * sigmas[j] * sigmas[j]);
            hcpart.push_back(make_float2((float)cv, (float)(cv - (double)(float)cv)));
        }
        FIT_TRY(model_alloc(c, M, &M.d_cpart, sizeof(float2) * p));
        FIT_TRY(cudaMemcpyAsync(M.d_cpart, hcpart.data(), sizeof(float2) * p, cudaMemcpyHostToDevice, st));
    }
    FIT_TRY(cudaMemcpyAsync(M.d_parts, M.parts.data(), sizeof(PartDesc) * p, cudaMemcpyHostToDevice, st));
    FIT_TRY(cudaMemcpyAsync(M.d_solves, M.solves.data(), sizeof(SolveDesc) * nsolve, cudaMemcpyHostToDevice, st));

    {
        DevBuf W(c);
        double *yg = nullptr, *r = nullptr, *z = nullptr, *pv = nullptr, *q = nullptr, *yv = nullptr;
        float2 *pdf = nullptr, *slots = nullptr;
        void *Kst = nullptr, *Ast = nullptr, *Zst = nullptr;
        PcgState *state = nullptr;
        unsigned int *nactive = nullptr;
        GroupDesc *d_groups = nullptr;
        int64_t *d_gpre = nullptr;
        int32_t *flags = nullptr;
        FIT_TRY(W.get(&yg, (size_t)prow * 8));
        FIT_TRY(W.get(&Kst, (fp64 ? 1 : 2) * (size_t)ns * ktot * tileb));
        FIT_TRY(W.get(&Ast, (size_t)ltiles * tileb));
        FIT_TRY(W.get(&Zst, (size_t)dtiles * tileb));
        __half *A16 = nullptr;  // FP16 copies of the L tiles of one-pass (class 1) solves
        if (tf32) FIT_TRY(W.get(&A16, (size_t)ltiles * KRR_TILE_ELEMS * sizeof(__half)));
        FIT_TRY(W.get(&r, (size_t)vec * 8));
        FIT_TRY(W.get(&z, (size_t)vec * 8));
        FIT_TRY(W.get(&pv, (size_t)vec * 8));
        FIT_TRY(W.get(&pdf, (size_t)vec * 8));
        FIT_TRY(W.get(&q, (size_t)vec * 8));
        FIT_TRY(W.get(&yv, (size_t)vec * 8));
        FIT_TRY(W.get(&slots, (size_t)scratch * 8));
        FIT_TRY(W.get((unsigned char **)&state, pcg_state_size() * nsolve));
        FIT_TRY(W.get(&nactive, sizeof(unsigned int)));
        FIT_TRY(W.get(&d_groups, sizeof(GroupDesc) * groups.size()));
        FIT_TRY(W.get(&d_gpre, sizeof(int64_t) * gpre.size()));
        FIT_TRY(W.get(&flags, sizeof(int32_t) * nsolve));
        int32_t *d_order = nullptr;
        FIT_TRY(W.get(&d_order, sizeof(int32_t) * nsolve));
        {
            std::vector<int32_t> order(nsolve);
            for (int s = 0; s < nsolve; ++s) order[s] = s;
            std::stable_sort(order.begin(), order.end(),
                             [&](int32_t a, int32_t b) { return M.solves[a].T > M.solves[b].T; });
            FIT_TRY(cudaMemcpyAsync(d_order, order.data(), sizeof(int32_t) * nsolve, cudaMemcpyHostToDevice, st));
            FIT_TRY(cudaStreamSynchronize(st));  // the host vector goes out of scope
        }
        FIT_TRY(cudaMemcpyAsync(d_groups, groups.data(), sizeof(GroupDesc) * groups.size(), cudaMemcpyHostToDevice,
                                st));
        FIT_TRY(cudaMemcpyAsync(d_gpre, gpre.data(), sizeof(int64_t) * gpre.size(), cudaMemcpyHostToDevice, st));
        FIT_TRY(cudaMemsetAsync(flags, 0, sizeof(int32_t) * nsolve, st));
        FIT_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));

        // stage + kernel build
        {
            ProfScope ps(prof, PROF_STAGE, st);
            launch_stage(st, X, y, perm, M, yg);
            if (!fp64 && oz_supported(d)) {
                M.dpz = oz_dpz(d);
                FIT_TRY(model_alloc(c, M, (unsigned char **)&M.ozS, (size_t)5 * prow * M.dpz * 2));
                FIT_TRY(model_alloc(c, M, &M.ozex, (size_t)prow * 4));
                launch_oz_slice(st, M.X64, d, nullptr, prow, prow, M.ozS, M.ozex, nullptr);
                if (!make_slice_tmap(&M.oz_tmB, M.ozS, (int64_t)5 * prow, M.dpz, 64))
                    return bail(KRR_ERR_CUDA, "krr_fit_batch: slice tensor map encoding failed");
            }
        }
        float *Kh = nullptr, *Kl = nullptr;
        double *K64 = nullptr;
        // row sums of K left by the exact-Gram tile build, for ||A||_inf
        float *rsR = nullptr, *rsC = nullptr;
        int64_t *d_rsoff = nullptr, rstot = 0;
        // (the FP64 path takes them from the stored tiles for the linear
        // kernel, whose entries can be negative: ||A||_inf needs |K|)
        if ((!fp64 && M.ozS) || (fp64 && M.kind == KRR_KERNEL_LINEAR)) {
            std::vector<int64_t> rsoff(p);
            for (int j = 0; j < p; ++j) {
                rsoff[j] = rstot;
                rstot += (int64_t)M.parts[j].T * M.parts[j].T;
            }
            if (rstot > 0) {
                FIT_TRY(W.get(&rsR, (size_t)ns * rstot * 8 * KRR_TILE * sizeof(float)));
                FIT_TRY(W.get(&rsC, (size_t)ns * rstot * KRR_TILE * sizeof(float)));
                FIT_TRY(W.get(&d_rsoff, sizeof(int64_t) * p));
                FIT_TRY(cudaMemcpyAsync(d_rsoff, rsoff.data(), sizeof(int64_t) * p, cudaMemcpyHostToDevice, st));
                FIT_TRY(cudaStreamSynchronize(st));  // the host vector goes out of scope
            }
        }
        {
            ProfScope ps(prof, PROF_KBUILD, st);
            if (fp64) {
                K64 = (double *)Kst;
                launch_kbuild_fp64(st, M, ktot, K64, (double *)Ast);
                if (rsR) launch_k64_abs_rowsums(st, M, ktot, K64, rsR, rsC, d_rsoff, rstot);
            } else {
                Kh = (float *)Kst;
                Kl = Kh + (size_t)ns * ktot * KRR_TILE_ELEMS;
                if (M.ozS) {
                    // no factor tiles: the factorisation's first touch reads K_hi (Kfirst below)
                    FIT_TRY(launch_kbuild_oz(st, M, ktot, Kh, Kl, (float *)Ast, rsR, rsC, d_rsoff, rstot,
                                             c->d_err, false, M.d_cpart));
                } else {
                    launch_kbuild_df(st, M, ktot, Kh, Kl, (float *)Ast);
                }
            }
        }
        FIT_TRY(cudaGetLastError());

        // condition estimates before factorising: ||K + lambda m I||_inf per solve
        // (the first refinement phase), read back to choose each solve's factor
        KRR_LAUNCHED(), fill_rhs_kernel<<<nsolve, 256, 0, st>>>(M.d_solves, M.d_parts, yg, yv);
        PcgBuffers B;
        B.x = M.alpha;
        B.r = r;
        B.z = z;
        B.p = pv;
        B.q = q;
        B.y = yv;
        B.pdf = pdf;
        B.slots = slots;
        B.state = state;
        B.nactive = nactive;
        B.d_groups = d_groups;
        B.d_gpre = d_gpre;
        B.ng = (int)groups.size();
        B.gtiles = gtiles;
        B.maxT = maxT;
        B.L16 = A16;
        B.order = d_order;
        B.rsR = rsR;
        B.rsC = rsC;
        B.rsoff = d_rsoff;
        B.rstot = rstot;
        FIT_TRY(run_pcg_norms(st, M, B, Kh, Kl, K64, fp64, prof));
        std::vector<PcgState> hs0(nsolve);
        FIT_TRY(cudaMemcpyAsync(hs0.data(), state, sizeof(PcgState) * nsolve, cudaMemcpyDeviceToHost, st));
        FIT_TRY(cudaStreamSynchronize(st));

        // factor class per solve: FP64 path -> FP64; FP32 -> 3-pass TF32; TF32 ->
        // one FP16 pass unless kappa_est * 2^-11 exceeds the escalation threshold;
        // BF16x3 -> 3-pass BF16 unless kappa_est * 2^-16 exceeds it (then 3-pass TF32)
        CUtensorMap tmap, tmapZ, tmap16, tmapK;
        memset(&tmap, 0, sizeof(tmap));
        memset(&tmapZ, 0, sizeof(tmapZ));
        memset(&tmap16, 0, sizeof(tmap16));
        memset(&tmapK, 0, sizeof(tmapK));
        if (!fp64 && (!make_tile_tmap(&tmap, (float *)Ast, ltiles) || !make_tile_tmap(&tmapZ, (float *)Zst, dtiles) ||
                      (A16 && !make_tile_tmap16(&tmap16, A16, ltiles))))
            return bail(KRR_ERR_CUDA, "krr_fit_batch: cuTensorMapEncodeTiled unavailable or failed");
        // the exact-Gram tile build stores no factor tiles: each factor tile's
        // first touch in the factorisation reads K_hi and adds lambda m
        const float *Kfirst = (!fp64 && M.ozS) ? Kh : nullptr;
        if (Kfirst && !make_tile_tmap(&tmapK, Kh, (int64_t)ns * ktot))
            return bail(KRR_ERR_CUDA, "krr_fit_batch: cuTensorMapEncodeTiled failed");
        const int base_cls = fp64 ? 0 : (tf32 ? 1 : (bf16x3 ? 2 : 3));
        std::vector<int> cls(nsolve, base_cls);  // update class per solve
        M.st_class.assign(nsolve, 0);
        if ((tf32 || bf16x3) && c->escalate > 0.0)
            for (int s = 0; s < nsolve; ++s) {
                const double lm = M.solves[s].lambda_m;
                const double kap = lm > 0.0 ? hs0[s].anorm / lm : INFINITY;
                if (kap * std::ldexp(1.0, tf32 ? -11 : -16) > c->escalate) cls[s] = 3;
            }
        // FP16 range: |L_ij| <= sqrt(A_jj) = sqrt(1 + lambda m) must stay far below 65504
        if (tf32)
            for (int s = 0; s < nsolve; ++s)
                if (cls[s] == 1 && !(1.0 + M.solves[s].lambda_m <= 16777216.0)) cls[s] = 3;
        int64_t lotiles = 0;  // lo parts of class-3 L tiles, written by the panel solves
        for (int s = 0; s < nsolve; ++s) {
            M.st_class[s] = cls[s];
            M.solves[s].cls = cls[s];
            M.solves[s].lotile0 = -1;
            if (cls[s] == 3) {
                M.solves[s].lotile0 = lotiles;
                lotiles += tri(M.solves[s].T);
            }
        }
        float *Alo = nullptr;
        CUtensorMap tmapLo;
        memset(&tmapLo, 0, sizeof(tmapLo));
        if (lotiles > 0) {
            FIT_TRY(W.get(&Alo, (size_t)lotiles * KRR_TILE_ELEMS * sizeof(float)));
            if (!make_tile_tmap(&tmapLo, Alo, lotiles))
                return bail(KRR_ERR_CUDA, "krr_fit_batch: cuTensorMapEncodeTiled failed");
        }
        FIT_TRY(cudaMemcpyAsync(M.d_solves, M.solves.data(), sizeof(SolveDesc) * nsolve, cudaMemcpyHostToDevice, st));

        // one joint schedule: shared diagonal factorisations and panel solves,
        // one update launch per class; outer panel width W explicit, cached per
        // (precision, largest tile count), or tuned now by timing each candidate
        // on these matrices (restored from K_hi between trials)
        std::vector<int> Ts(nsolve);
        for (int s = 0; s < nsolve; ++s) Ts[s] = M.solves[s].T;
        const int tcmode = base_cls;  // tensor-core mode of the factor (0: SIMT FP64)
        int Wp = c->chol_W;
        const std::pair<int, int> key((int)prec, maxT);
        if (Wp <= 0 && c->tuned_W.count(key)) Wp = c->tuned_W[key];
        if (Wp <= 0 && (fp64 || maxT < 4)) Wp = 1;
        std::vector<int32_t> hflags(nsolve, 0);
        {
            DevBuf CB(c);
            if (Wp <= 0) {
                std::vector<int64_t> rpre(nsolve + 1, 0);
                for (int s = 0; s < nsolve; ++s) rpre[s + 1] = rpre[s] + tri(M.solves[s].T);
                int64_t *d_rpre = nullptr;
                FIT_TRY(CB.get(&d_rpre, sizeof(int64_t) * (nsolve + 1)));
                FIT_TRY(cudaMemcpyAsync(d_rpre, rpre.data(), sizeof(int64_t) * (nsolve + 1), cudaMemcpyHostToDevice,
                                        st));
                cudaEvent_t e0, e1;
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                float best_ms = 1e30f;
                int best_W = 1;
                const int cands[4] = {1, 2, 4, 8};
                for (int ci = 0; ci < 4; ++ci) {
                    const int Wc = cands[ci];
                    if (Wc > maxT) break;
                    std::vector<CholLaunch> tplan;
                    std::vector<int64_t> tpre;
                    build_chol_plan(Ts, cls, Wc, tplan, tpre);
                    int64_t *d_tplan = nullptr;
                    FIT_TRY(CB.get(&d_tplan, sizeof(int64_t) * std::max<size_t>(tpre.size(), 1)));
                    FIT_TRY(cudaMemcpyAsync(d_tplan, tpre.data(), sizeof(int64_t) * tpre.size(),
                                            cudaMemcpyHostToDevice, st));
                    KRR_LAUNCHED(), reform_kernel<<<(unsigned)rpre[nsolve], 256, 0, st>>>(M.d_solves, d_rpre, nsolve,
                                                                                         Kh, (float *)Ast, 0.f);
                    cudaEventRecord(e0, st);
                    FIT_TRY(run_chol_plan(st, tplan, d_tplan, Ast, Zst, false, M.d_solves, nsolve, flags, tcmode,
                                          &tmap, &tmapZ, A16, &tmap16, Alo, &tmapLo, Kfirst, &tmapK, c->d_err,
                                          nullptr));
                    cudaEventRecord(e1, st);
                    FIT_TRY(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best_ms) {
                        best_ms = ms;
                        best_W = Wc;
                    }
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                Wp = best_W;
                c->tuned_W[key] = best_W;
                KRR_LAUNCHED(), reform_kernel<<<(unsigned)rpre[nsolve], 256, 0, st>>>(M.d_solves, d_rpre, nsolve, Kh,
                                                                                     (float *)Ast, 0.f);
                FIT_TRY(cudaMemsetAsync(flags, 0, sizeof(int32_t) * nsolve, st));
            }
            std::vector<CholLaunch> plan;
            std::vector<int64_t> pre;
            build_chol_plan(Ts, cls, Wp, plan, pre);
            int64_t *d_plan = nullptr;
            FIT_TRY(CB.get(&d_plan, sizeof(int64_t) * std::max<size_t>(pre.size(), 1)));
            if (!pre.empty())
                FIT_TRY(cudaMemcpyAsync(d_plan, pre.data(), sizeof(int64_t) * pre.size(), cudaMemcpyHostToDevice, st));
            FIT_TRY(run_chol_plan(st, plan, d_plan, Ast, Zst, fp64, M.d_solves, nsolve, flags, tcmode, &tmap, &tmapZ,
                                  A16, &tmap16, Alo, &tmapLo, Kfirst, &tmapK, c->d_err, prof));
            FIT_TRY(cudaMemcpyAsync(hflags.data(), flags, sizeof(int32_t) * nsolve, cudaMemcpyDeviceToHost, st));
            FIT_TRY(cudaStreamSynchronize(st));
        }

        // breakdown of a low-precision factor: refactor those solves in the
        // 3-pass mode with a growing diagonal shift (it only changes the preconditioner)
        if (!fp64) {
            for (int attempt = 0; attempt < 3; ++attempt) {
                std::vector<int> failed;
                for (int s = 0; s < nsolve; ++s)
                    if (hflags[s]) failed.push_back(s);
                if (failed.empty()) break;
                DevBuf R(c);
                const int nsub = (int)failed.size();
                std::vector<SolveDesc> sub(nsub);
                std::vector<int64_t> rpre(nsub + 1, 0);
                for (int i = 0; i < nsub; ++i) {
                    sub[i] = M.solves[failed[i]];
                    sub[i].cls = 4;  // refactored in 3 passes split in shared memory, L in the FP32 store
                    rpre[i + 1] = rpre[i] + tri(sub[i].T);
                }
                SolveDesc *d_sub = nullptr;
                int64_t *d_rpre = nullptr;
                int32_t *rflags = nullptr;
                FIT_TRY(R.get(&d_sub, sizeof(SolveDesc) * nsub));
                FIT_TRY(R.get(&d_rpre, sizeof(int64_t) * (nsub + 1)));
                FIT_TRY(R.get(&rflags, sizeof(int32_t) * nsub));
                FIT_TRY(cudaMemcpyAsync(d_sub, sub.data(), sizeof(SolveDesc) * nsub, cudaMemcpyHostToDevice, st));
                FIT_TRY(cudaMemcpyAsync(d_rpre, rpre.data(), sizeof(int64_t) * (nsub + 1), cudaMemcpyHostToDevice,
                                        st));
                FIT_TRY(cudaMemsetAsync(rflags, 0, sizeof(int32_t) * nsub, st));
                const float shift = (float)(std::pow(10.0, attempt) * 1e-4 * 0.5 * (double)sub[0].m + 1e-6);
                KRR_LAUNCHED(), reform_kernel<<<(unsigned)rpre[nsub], 256, 0, st>>>(d_sub, d_rpre, nsub, Kh,
                                                                                   (float *)Ast, shift);
                std::vector<int> rT(nsub);
                for (int i = 0; i < nsub; ++i) rT[i] = sub[i].T;
                std::vector<CholLaunch> rplan;
                std::vector<int64_t> rp;
                build_chol_plan(rT, std::vector<int>(nsub, 4), 1, rplan, rp);
                int64_t *d_rplan = nullptr;
                FIT_TRY(R.get(&d_rplan, sizeof(int64_t) * std::max<size_t>(rp.size(), 1)));
                FIT_TRY(cudaMemcpyAsync(d_rplan, rp.data(), sizeof(int64_t) * rp.size(), cudaMemcpyHostToDevice,
                                        st));
                FIT_TRY(run_chol_plan(st, rplan, d_rplan, Ast, Zst, false, d_sub, nsub, rflags, 3, &tmap, &tmapZ,
                                      A16, &tmap16, Alo, &tmapLo, nullptr, nullptr, c->d_err, prof));
                std::vector<int32_t> hr(nsub);
                FIT_TRY(cudaMemcpyAsync(hr.data(), rflags, sizeof(int32_t) * nsub, cudaMemcpyDeviceToHost, st));
                FIT_TRY(cudaStreamSynchronize(st));
                for (int i = 0; i < nsub; ++i) {
                    hflags[failed[i]] = hr[i];
                    if (!hr[i]) M.st_class[failed[i]] = 4;
                }
            }
        }
        FIT_TRY(cudaMemcpyAsync(flags, hflags.data(), sizeof(int32_t) * nsolve, cudaMemcpyHostToDevice, st));
        if (!fp64) {  // the preconditioner reads each solve's L where its final class left it
            bool changed = false;
            for (int s = 0; s < nsolve; ++s)
                if (M.solves[s].cls != M.st_class[s]) {
                    M.solves[s].cls = M.st_class[s];
                    changed = true;
                }
            if (changed)
                FIT_TRY(cudaMemcpyAsync(M.d_solves, M.solves.data(), sizeof(SolveDesc) * nsolve,
                                        cudaMemcpyHostToDevice, st));
        }

        // refinement: stop at the FP64-class floor, or earlier once
        // kappa_est * residual meets the context's forward-error target (refined precisions)
        const double tau = fp64 ? std::ldexp(1.0, -50) : std::ldexp(1.0, -46);
        const double target = fp64 ? 0.0 : c->target_err;
        FIT_TRY(run_pcg(st, M, B, Kh, Kl, K64, Ast, Zst, fp64, maxT, tau, target, 80, flags, c->h_flag, 2, prof));
        KRR_LAUNCHED(), export_kernel<<<nsolve, 256, 0, st>>>(M.d_solves, M.d_parts, G, M.alpha, state, solve_status, alpha);
        FIT_TRY(cudaGetLastError());
        int herr = 0;
        std::vector<PcgState> hs(nsolve);
        FIT_TRY(cudaMemcpyAsync(hs.data(), state, sizeof(PcgState) * nsolve, cudaMemcpyDeviceToHost, st));
        FIT_TRY(cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        FIT_TRY(cudaStreamSynchronize(st));
        M.st_iters.resize(nsolve);
        M.st_status.resize(nsolve);
        M.st_kappa.resize(nsolve);
        M.st_resid.resize(nsolve);
        for (int s = 0; s < nsolve; ++s) {
            M.st_iters[s] = hs[s].iters;
            M.st_status[s] = hs[s].status;
            M.st_kappa[s] = M.solves[s].lambda_m > 0 ? hs[s].anorm / M.solves[s].lambda_m : INFINITY;
            M.st_resid[s] = hs[s].resid;
        }
        if (herr != 0) return bail(KRR_ERR_TIMEOUT, "krr_fit_batch: a bounded device wait expired");
        // kernel stores (Kh/Kl, K64) could stay for later refinement; they are released here
        (void)Zst;
    }
    // FP64 fallback: a refined-precision solve whose low-precision factor was
    // too poor a preconditioner to converge (condition estimates near the
    // reciprocal of the factor's unit roundoff) is solved again on the plain
    // FP64 path -- FP64 kernel, FP64 Cholesky, FP64 refinement -- with the
    // work buffers of the batch already released; its alpha replaces the
    // unconverged one and its factor class reads 0.
    if (!fp64 && c->fp64_fallback) {
        for (int s = 0; s < nsolve; ++s) {
            if (M.st_status[s] != KRR_ERR_NO_CONVERGE) continue;
            const SolveDesc &S = M.solves[s];
            if (S.m == 0) continue;
            int64_t *d_off = nullptr;
            int32_t *d_st = nullptr;
            const int64_t hoff[2] = {0, (int64_t)S.m};
            krr_model *sub = nullptr;
            int32_t hst = KRR_ERR_NO_CONVERGE;
            const double sg = M.sigmas[per_part ? S.part : S.isig], lm = M.lambdas[per_part ? S.part : S.ilam];
            if (ctx_malloc(c, (void **)&d_off, 16) != cudaSuccess) break;
            if (ctx_malloc(c, (void **)&d_st, 4) != cudaSuccess) {
                ctx_free(c, d_off, 16);
                break;
            }
            const int prev_kernel = c->kernel;
            c->kernel = M.kind;
            krr_status rc = cudaMemcpyAsync(d_off, hoff, 16, cudaMemcpyHostToDevice, st) == cudaSuccess
                                ? krr_fit_batch(ctx, X, y, n, d, perm + M.parts[S.part].row0, d_off, 1, &sg, 1, &lm, 1,
                                                KRR_PREC_FP64, &sub, d_st, nullptr)
                                : KRR_ERR_CUDA;
            c->kernel = prev_kernel;
            if (rc == KRR_OK && cudaMemcpyAsync(&hst, d_st, 4, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                cudaStreamSynchronize(st) == cudaSuccess && hst == KRR_OK &&
                cudaMemcpyAsync(M.alpha + S.vec0, sub->m.alpha, (size_t)S.T * KRR_TILE * 8, cudaMemcpyDeviceToDevice,
                                st) == cudaSuccess) {
                M.st_status[s] = KRR_OK;
                M.st_iters[s] += sub->m.st_iters[0];
                M.st_resid[s] = sub->m.st_resid[0];
                M.st_class[s] = 0;
                const int32_t ok = KRR_OK;
                if (solve_status) cudaMemcpyAsync(solve_status + s, &ok, 4, cudaMemcpyHostToDevice, st);
                if (alpha)
                    cudaMemcpyAsync(alpha + M.parts[S.part].row0 * G + (int64_t)(s % G) * S.m, sub->m.alpha,
                                    (size_t)S.m * 8, cudaMemcpyDeviceToDevice, st);
                cudaStreamSynchronize(st);  // host sources above are on this stack frame
            }
            if (sub) {
                free_model(c, sub->m);
                delete sub;
            }
            ctx_free(c, d_st, 4);
            ctx_free(c, d_off, 16);
        }
    }
    if (M.ozS) {
        cudaError_t e = model_alloc(c, M, &M.alpha2, (size_t)M.nvec * sizeof(float2));
        if (e == cudaSuccess) {
            KRR_LAUNCHED(), alpha_pairs_kernel<<<(unsigned)((M.nvec + 255) / 256), 256, 0, st>>>(M.alpha, M.alpha2,
                                                                                               M.nvec);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess)
            return bail(e == cudaErrorMemoryAllocation ? KRR_ERR_OOM : KRR_ERR_CUDA,
                        std::string("krr_fit_batch: alpha pairs: ") + cudaGetErrorString(e));
    }
#undef FIT_TRY
    *out = km;
    return KRR_OK;
}

krr_status krr_fit_batch(krr_ctx *ctx, const double *X, const double *y, int64_t n, int32_t d,
                         const int64_t *perm, const int64_t *offsets, int32_t p, const double *sigmas, int32_t ns,
                         const double *lambdas, int32_t nl, krr_prec prec, krr_model **out,
                         int32_t *solve_status, double *alpha) {
    return fit_impl(ctx, X, y, n, d, perm, offsets, p, sigmas, ns, lambdas, nl, prec, out, solve_status, alpha,
                    false);
}

krr_status krr_fit_jobs(krr_ctx *ctx, const double *X, const double *y, int64_t n, int32_t d,
                        const int64_t *perm, const int64_t *offsets, int32_t p, const double *sigmas,
                        const double *lambdas, krr_prec prec, krr_model **out, int32_t *solve_status,
                        double *alpha) {
    return fit_impl(ctx, X, y, n, d, perm, offsets, p, sigmas, 1, lambdas, 1, prec, out, solve_status, alpha, true);
}

krr_status krr_predict(krr_ctx *ctx, const krr_model *model, const double *Xt, int64_t t, const int32_t *route,
                       double *yhat) {
    if (!ctx) return KRR_ERR_ARG;
    Ctx *c = &ctx->c;
    if (!model || t < 0 || (t > 0 && (!Xt || !yhat))) return fail(c, KRR_ERR_ARG, "krr_predict: invalid argument");
    const Model &M = model->m;
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    Prof *prof = c->prof.on ? &c->prof : nullptr;
    const int G = M.nsig * M.nlam;
    if (t == 0) return KRR_OK;
    const bool oz = M.ozS != nullptr;
    // routed: group the test rows by partition (stable) first
    int64_t *tperm = nullptr, *toff = nullptr;
    if (route) {
        API_TRY(c, ctx_malloc(c, (void **)&tperm, (size_t)t * 8));
        cudaError_t e = ctx_malloc(c, (void **)&toff, (size_t)(M.p + 1) * 8);
        if (e != cudaSuccess) {
            ctx_free(c, tperm, (size_t)t * 8);
            API_TRY(c, e);
        }
        // a route value outside [0, p) places its row nowhere: zeroed positions
        // keep every grouped index a valid row, and such rows predict 0
        cudaError_t ez = cudaMemsetAsync(tperm, 0, (size_t)t * 8, st);
        krr_status rc = ez == cudaSuccess ? run_gather(c, route, t, M.p, tperm, toff) : KRR_ERR_CUDA;
        if (rc != KRR_OK) {
            ctx_free(c, toff, (size_t)(M.p + 1) * 8);
            ctx_free(c, tperm, (size_t)t * 8);
            return rc;
        }
        API_TRY(c, cudaMemsetAsync(yhat, 0, sizeof(double) * (size_t)G * t, st));
    }
    cudaError_t err = cudaSuccess;
    if (oz) {
        const int64_t t_rows = (t + 127) / 128 * 128 + 128;
        const size_t b_sl = (size_t)5 * t_rows * M.dpz * 2, b_ex = (size_t)t_rows * 4, b_nr = (size_t)t_rows * 8;
        void *sl = nullptr;
        int32_t *tex = nullptr;
        float2 *tnr = nullptr;
        err = ctx_malloc(c, &sl, b_sl);
        if (err == cudaSuccess) err = ctx_malloc(c, (void **)&tex, b_ex);
        if (err == cudaSuccess) err = ctx_malloc(c, (void **)&tnr, b_nr);
        if (err == cudaSuccess) {
            ProfScope ps(prof, PROF_PREDICT, st);
            err = launch_predict_oz(st, M, M.oz_tmB, Xt, t, toff, tperm, route ? 1 : 0, sl, tex, tnr, t_rows, yhat,
                                    c->d_err);
        }
        if (tnr) ctx_free(c, tnr, b_nr);
        if (tex) ctx_free(c, tex, b_ex);
        if (sl) ctx_free(c, sl, b_sl);
    } else {
        ProfScope ps(prof, PROF_PREDICT, st);
        launch_predict(st, M, Xt, t, toff, tperm, t, route ? 1 : 0, yhat);
        err = cudaGetLastError();
    }
    if (toff) ctx_free(c, toff, (size_t)(M.p + 1) * 8);
    if (tperm) ctx_free(c, tperm, (size_t)t * 8);
    API_TRY(c, err);
    return KRR_OK;
}

krr_status krr_select(krr_ctx *ctx, const double *yhat, const double *yt, int64_t t, int32_t p, int32_t G,
                      krr_sel mode, double *mse, int32_t *best) {
    if (!ctx) return KRR_ERR_ARG;
    Ctx *c = &ctx->c;
    if (!yhat || !yt || !mse || !best || t <= 0 || p <= 0 || G <= 0 || (int)mode < 0 || (int)mode > 3)
        return fail(c, KRR_ERR_ARG, "krr_select: invalid argument");
    cudaSetDevice(c->device);
    ProfScope ps(c->prof.on ? &c->prof : nullptr, PROF_SELECT, c->stream);
    launch_select(c->stream, yhat, yt, t, p, G, (int)mode, mse, best);
    API_TRY(c, cudaGetLastError());
    return KRR_OK;
}

krr_status krr_model_stats(krr_ctx *ctx, const krr_model *model, int32_t *iters, double *kappa_est,
                           double *resid) {
    if (!ctx || !model) return KRR_ERR_ARG;
    const Model &M = model->m;
    const size_t n = M.st_iters.size();
    if (iters) std::copy(M.st_iters.begin(), M.st_iters.end(), iters);
    if (kappa_est) std::copy(M.st_kappa.begin(), M.st_kappa.begin() + n, kappa_est);
    if (resid) std::copy(M.st_resid.begin(), M.st_resid.begin() + n, resid);
    return KRR_OK;
}

krr_status krr_model_factor_class(krr_ctx *ctx, const krr_model *model, int32_t *cls) {
    if (!ctx || !model || !cls) return KRR_ERR_ARG;
    const Model &M = model->m;
    std::copy(M.st_class.begin(), M.st_class.end(), cls);
    return KRR_OK;
}

krr_status krr_model_free(krr_ctx *ctx, krr_model *model) {
    if (!ctx || !model) return KRR_ERR_ARG;
    free_model(&ctx->c, model->m);
    delete model;
    return KRR_OK;
}

}  // extern "C"
