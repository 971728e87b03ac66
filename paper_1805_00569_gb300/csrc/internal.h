// internal.h -- host/device structures of libkrr shared by the .cu files.
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>
#include <atomic>
#include <map>

#include "../../include/krr.h"

namespace krr {

// Kernels launched through the library (process-wide, for launch accounting).
extern std::atomic<long long> g_launch_count;

// Lets a kernel launch with as much dynamic shared memory as the device's
// opt-in limit leaves beside its static shared memory.  The value never varies,
// so host threads launching the same kernel at once (one context each) can
// never lower the limit under another's launch.  Set once per (kernel, device).
cudaError_t allow_max_dyn_smem_fn(const void *fn);
template <typename F>
inline cudaError_t allow_max_dyn_smem(F *fn) {
    return allow_max_dyn_smem_fn(reinterpret_cast<const void *>(fn));
}
#define KRR_LAUNCHED() (::krr::g_launch_count.fetch_add(1, std::memory_order_relaxed))

constexpr int TILE = 128;
constexpr int64_t TILE_ELEMS = (int64_t)TILE * TILE;

// One partition of the training set after gathering.
struct PartDesc {
    int32_t m;       // rows
    int32_t T;       // tiles per edge, ceil(m / TILE) (0 when m == 0)
    int64_t row0;    // first row in the gathered (unpadded) order
    int64_t prow0;   // first row in the padded, tile-aligned order
    int64_t ktile0;  // first tile of this partition inside one sigma's kernel store
};

// One (partition, sigma, lambda) solve.
struct SolveDesc {
    int32_t part, isig, ilam, T;
    int32_t m, grp;   // grp = partition * nsig + isig (kernel-store group)
    int32_t cls;      // factor class: 0 FP64, 1 one pass (FP16 factor store), 2 BF16x3,
                      // 3 TF32x3 on operands split by the panel solve, 4 TF32x3 split in shared memory
    int32_t pad0;
    int64_t ltile0;   // first tile in the factor store (lower tiles, row-major triangle order)
    int64_t lotile0;  // class 3: first tile of its L lo parts in the lo store (else -1)
    int64_t dtile0;   // first tile in the diagonal-inverse store
    int64_t ktile0;   // first tile of the (partition, sigma) kernel store
    int64_t vec0;     // first element in the per-solve padded vectors
    double lambda_m;  // lambda * m (Eq. 6 with the partition's own size)
};

// Kernel-store group (partition, sigma): the matrix-vector products of the
// refinement run per group with every lambda as a right-hand side.
struct GroupDesc {
    int32_t part, isig, T, nlam;
    int64_t ktile0;
    int64_t solve0;   // first solve of this group; solves solve0 .. solve0+nlam-1
    int64_t scratch0; // first element of this group's matvec partial buffer
};

// Per-solve state of the conjugate-gradient refinement.
struct PcgState {
    double rz, anorm, ymax, resid;
    int32_t active, iters, status, pad;
};

// device buffers of the refinement, shared by the library and the refinement kernels
struct PcgBuffers {
    double *x, *r, *z, *p, *q, *y;
    float2 *pdf, *slots;  // the direction as double-float pairs; matvec partials
    PcgState *state;
    unsigned int *nactive;
    GroupDesc *d_groups;
    int64_t *d_gpre;
    int ng;
    int64_t gtiles;
    int maxT;
    const void *L16;  // FP16 factor store of class-1 solves (null without them)
    int32_t *order;   // solve indices by tile count, largest first (preconditioner CTA order)
    const float *rsR, *rsC;  // row sums of K from the kernel-tile build (null: none)
    const int64_t *rsoff;
    int64_t rstot;
};

// Optional per-kernel timing with CUDA events on the launching stream.
enum ProfKind {
    PROF_PARTITION = 0, PROF_STAGE, PROF_KBUILD, PROF_POTRF, PROF_TRSM, PROF_UPDATE, PROF_MATVEC,
    PROF_PRECOND, PROF_PCGVEC, PROF_PREDICT, PROF_SELECT, PROF_NKINDS
};
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<int> kinds;  // kind of event pair i (events 2i, 2i+1)
    size_t used = 0;         // pairs in use
    double total_ms[PROF_NKINDS] = {0};
    long long launches[PROF_NKINDS] = {0};
    int begin(cudaStream_t st) {
        if (!on) return -1;
        if (2 * used + 2 > pool.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            pool.push_back(a);
            pool.push_back(b);
            kinds.push_back(0);
        }
        cudaEventRecord(pool[2 * used], st);
        return (int)used++;
    }
    void end(int idx, int kind, cudaStream_t st) {
        if (idx < 0) return;
        kinds[idx] = kind;
        cudaEventRecord(pool[2 * idx + 1], st);
    }
    // fold recorded pairs into the totals (caller synchronised the stream)
    void collect() {
        for (size_t i = 0; i < used; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pool[2 * i], pool[2 * i + 1]) == cudaSuccess) {
                total_ms[kinds[i]] += ms;
                launches[kinds[i]] += 1;
            }
        }
        used = 0;
    }
    void reset() {
        used = 0;
        for (int k = 0; k < PROF_NKINDS; ++k) {
            total_ms[k] = 0;
            launches[k] = 0;
        }
    }
};
struct ProfScope {
    Prof *p;
    int idx, kind;
    cudaStream_t st;
    ProfScope(Prof *p_, int kind_, cudaStream_t st_) : p(p_), idx(-1), kind(kind_), st(st_) {
        if (p) idx = p->begin(st);
    }
    ~ProfScope() {
        if (p) p->end(idx, kind, st);
    }
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0, used = 0;
    std::string last_error;
    cudaMemPool_t pool = nullptr;  // this context's stream-ordered pool (freed blocks stay mapped)
    int *d_err = nullptr;      // device error word (timeouts inside kernels)
    unsigned int *h_flag = nullptr;  // pinned host word for polling
    Prof prof;
    int chol_W = 0;            // outer panel width (0 = tuned on first use)
    double target_err = 1e-7;  // refinement stops once kappa_est * backward error <= this
    double escalate = 32.0;    // TF32: factor a solve in 3 passes when kappa_est * 2^-11 exceeds this
    int kernel = KRR_KERNEL_GAUSSIAN;  // Table 1 kernel of the next fits
    bool fp64_fallback = true;  // re-solve unconverged refined-precision solves on the FP64 path
    std::map<std::pair<int, int>, int> tuned_W;  // (precision, max tiles) -> tuned panel width
};

struct Model {
    int32_t d = 0, dp = 0, p = 0, nsig = 0, nlam = 0, prec = 0;
    int32_t kind = KRR_KERNEL_GAUSSIAN;  // Table 1 kernel
    int64_t n = 0, prows = 0, nvec = 0;
    std::vector<double> sigmas, lambdas;
    std::vector<PartDesc> parts;
    std::vector<SolveDesc> solves;
    PartDesc *d_parts = nullptr;
    SolveDesc *d_solves = nullptr;
    double *X64 = nullptr;     // gathered rows, padded order, FP64 [prows x d]
    float *Xh = nullptr;       // hi part FP32 [prows x dp]
    float *Xl = nullptr;       // lo part FP32 [prows x dp]
    float2 *nrm = nullptr;     // squared norms as (hi, lo) [prows]
    double *alpha = nullptr;   // per-solve coefficients, padded [nvec]
    float2 *alpha2 = nullptr;  // the same as double-float pairs (hi, lo) for the exact-Gram prediction
    void *ozS = nullptr;       // integer bf16 slices of the padded rows [5][prows][dpz] (tensor-core predict)
    int32_t *ozex = nullptr;   // per-row slice exponent [prows]
    int32_t dpz = 0;           // features padded to the slice K chunk
    CUtensorMap oz_tmB;        // TMA view of ozS for the training-row operand
    bool per_part = false;     // one (sigma, lambda) per partition (krr_fit_jobs): sigmas/lambdas have p entries
    float2 *d_cpart = nullptr; // per_part: -1 / (2 sigma_j^2) as df per partition
    std::vector<int32_t> st_iters, st_status, st_class;  // per-solve refinement statistics, factor class
    std::vector<double> st_kappa, st_resid;
    std::vector<std::pair<void *, size_t>> allocs;
};

// allocation through the context budget
cudaError_t ctx_malloc(Ctx *c, void **p, size_t bytes);
void ctx_free(Ctx *c, void *p, size_t bytes);

inline int64_t tri(int64_t T) { return T * (T + 1) / 2; }

}  // namespace krr

#define KRR_CUDA_TRY(ctx, expr)                                                        \
    do {                                                                               \
        cudaError_t _e = (expr);                                                       \
        if (_e != cudaSuccess) {                                                       \
            (ctx)->last_error = std::string(#expr) + ": " + cudaGetErrorString(_e);    \
            return _e == cudaErrorMemoryAllocation ? KRR_ERR_OOM : KRR_ERR_CUDA;       \
        }                                                                              \
    } while (0)
