// chol.cu -- batched blocked Cholesky over uneven partitions (Eq. 6 solved
// by Cholesky as in Sec. 5.4, every (partition, sigma, lambda) matrix at once).
//
// Each matrix is a lower-triangular array of 128 x 128 tiles (see kbuild.cu).
// A blocked right-looking factorisation with outer panel width W tiles runs
// as a host-side schedule of three batched kernels:
//   potrf  -- diagonal tile L_kk = chol(A_kk) in shared memory, plus the
//             in-place inverse Z_kk = L_kk^-1 (kept: it turns the panel
//             solve into a product and is the diagonal block of the
//             preconditioner in the refinement);
//   trsm   -- L_ik = A_ik Z_kk^T for every tile below the diagonal;
//   update -- A_ij -= sum_k L_ik L_jk^T, either for the trailing submatrix
//             (TRAIL: K range [K0, K0+W), tiles K0+W <= j <= i) or for one
//             block column inside a panel (COLUMN: tiles i >= c, K range
//             [K0, c)).
// Work lists: a launch covers tasks of every solve; an exclusive prefix over
// solves of the per-solve task counts (built on the host for the whole
// schedule) maps blockIdx.x to (solve, local task) by binary search, so
// uneven partitions need no padding launches.
//
// Trailing-update arithmetic by precision: FP64 and FP32 run a SIMT GEMM tile;
// TF32 runs on the tcgen05 tensor cores: one elected thread streams the
// operand tiles with 2-D TMA loads (128-byte swizzle) through a 3-stage
// mbarrier ring, one elected thread issues kind::tf32 MMAs (M = N = 128,
// K = 8) into a 128-column FP32 accumulator in tensor memory, and all four
// warps read it back with tcgen05.ld for the A_ij -= C epilogue.
#include "common.cuh"
#include "internal.h"

namespace krr {

enum { UPD_TRAIL = 0, UPD_COLUMN = 1, UPD_TRSM = 2 };

__device__ __forceinline__ int find_solve(const int64_t *pre, int n, int64_t b) {
    int lo = 0, hi = n - 1;  // last s with pre[s] <= b
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Task (s, local) -> destination tile (i, j) and K range [kb, ke) of panels.
struct TaskGeom { int i, j, kb, ke; };
__device__ __forceinline__ TaskGeom decode_task(int mode, int64_t local, int K0, int W) {
    TaskGeom g;
    if (mode == UPD_TRAIL) {
        int ii, jj;
        tri_decode(local, ii, jj);
        g.i = K0 + W + ii;
        g.j = K0 + W + jj;
        g.kb = K0;
        g.ke = K0 + W;
    } else if (mode == UPD_COLUMN) {  // column c = W here, K range [K0, c)
        g.i = W + (int)local;
        g.j = W;
        g.kb = K0;
        g.ke = W;
    } else {  // TRSM: panel column K0, rows below
        g.i = K0 + 1 + (int)local;
        g.j = K0;
        g.kb = K0;
        g.ke = K0 + 1;
    }
    return g;
}

// ---------------------------------------------------------------- potrf
// 512 threads; row r handled by the 4 threads 4r .. 4r+3.
template <typename T>
__global__ void __launch_bounds__(512) potrf_tile_kernel(T *__restrict__ A, T *__restrict__ Z,
                                                         const SolveDesc *__restrict__ solves,
                                                         const int64_t *__restrict__ pre, int nsolve, int k,
                                                         int32_t *__restrict__ flags) {
    extern __shared__ __align__(16) unsigned char po_dyn[];
    T *sm = reinterpret_cast<T *>(po_dyn);  // [128][129]
    const int s = find_solve(pre, nsolve, blockIdx.x);
    const SolveDesc S = solves[s];
    const int64_t tile = S.ltile0 + (int64_t)k * (k + 1) / 2 + k;
    T *g = A + tile * KRR_TILE_ELEMS;
    for (int e = threadIdx.x; e < KRR_TILE_ELEMS; e += blockDim.x) sm[(e >> 7) * 129 + (e & 127)] = g[e];
    __syncthreads();
    const int r = threadIdx.x >> 2, part = threadIdx.x & 3;
    bool bad = false;
    for (int c = 0; c < KRR_TILE; ++c) {
        T piv = sm[c * 129 + c];
        if (!(piv > T(0))) {  // not positive: record and continue without NaNs
            bad = true;
            piv = T(1);
            __syncthreads();
            if (threadIdx.x == 0) sm[c * 129 + c] = T(1);
            __syncthreads();
        }
        const T inv = T(1) / piv;
        if (r > c) {
            const T lrc = sm[r * 129 + c] * inv;
            for (int q = c + 1 + part; q <= r; q += 4) sm[r * 129 + q] -= lrc * sm[q * 129 + c];
        }
        __syncthreads();
    }
    if (bad && threadIdx.x == 0) flags[s] = 1;
    // L: column c scaled by 1/sqrt(pivot c)
    for (int e = threadIdx.x; e < KRR_TILE_ELEMS; e += blockDim.x) {
        const int rr = e >> 7, cc = e & 127;
        T v;
        if (rr > cc) v = sm[rr * 129 + cc] / sqrt(sm[cc * 129 + cc]);
        else if (rr == cc) v = sqrt(sm[cc * 129 + cc]);
        else v = T(0);
        g[e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < KRR_TILE_ELEMS; e += blockDim.x) sm[(e >> 7) * 129 + (e & 127)] = g[e];
    __syncthreads();
    // in-place inverse of the lower-triangular L, columns right to left:
    // Z_jj = 1 / L_jj, Z_rj = -(sum_{q=j+1..r} Z_rq L_qj) Z_jj
    for (int j = KRR_TILE - 1; j >= 0; --j) {
        const T zjj = T(1) / sm[j * 129 + j];
        T acc = T(0);
        if (r > j)
            for (int q = j + 1 + part; q <= r; q += 4) acc += sm[r * 129 + q] * sm[q * 129 + j];
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        __syncthreads();
        if (part == 0) {
            if (r > j) sm[r * 129 + j] = -acc * zjj;
            else if (r == j) sm[j * 129 + j] = zjj;
        }
        __syncthreads();
    }
    T *z = Z + (S.dtile0 + k) * KRR_TILE_ELEMS;
    for (int e = threadIdx.x; e < KRR_TILE_ELEMS; e += blockDim.x) {
        const int rr = e >> 7, cc = e & 127;
        z[e] = (rr >= cc) ? sm[rr * 129 + cc] : T(0);
    }
}

// ---------------------------------------------------------------- SIMT GEMM tile
// UPD_TRAIL / UPD_COLUMN: A_ij -= sum_{k in [kb,ke)} L_ik L_jk^T
// UPD_TRSM:               A_ik  = A_ik Z_kk^T
template <typename T>
struct SimtCfg { static constexpr int KC = 32; };
template <>
struct SimtCfg<double> { static constexpr int KC = 16; };

template <typename T>
__global__ void __launch_bounds__(256) gemm_tile_simt_kernel(T *__restrict__ A, const T *__restrict__ Z,
                                                             const SolveDesc *__restrict__ solves,
                                                             const int64_t *__restrict__ pre, int nsolve, int mode,
                                                             int K0, int W) {
    constexpr int KC = SimtCfg<T>::KC;
    __shared__ __align__(16) T sA[KC][KRR_TILE + 4];
    __shared__ __align__(16) T sB[KC][KRR_TILE + 4];
    const int s = find_solve(pre, nsolve, blockIdx.x);
    const SolveDesc S = solves[s];
    const TaskGeom g = decode_task(mode, (int64_t)blockIdx.x - pre[s], K0, W);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
    for (int kt = g.kb; kt < g.ke; ++kt) {
        const T *ta = A + (S.ltile0 + (int64_t)g.i * (g.i + 1) / 2 + kt) * KRR_TILE_ELEMS;
        const T *tb = (mode == UPD_TRSM) ? Z + (S.dtile0 + kt) * KRR_TILE_ELEMS
                                         : A + (S.ltile0 + (int64_t)g.j * (g.j + 1) / 2 + kt) * KRR_TILE_ELEMS;
        for (int c0 = 0; c0 < KRR_TILE; c0 += KC) {
            __syncthreads();
            for (int e = threadIdx.x; e < KC * KRR_TILE; e += 256) {
                const int row = e / KC, cc = e % KC;
                sA[cc][row] = ta[row * KRR_TILE + c0 + cc];
                sB[cc][row] = tb[row * KRR_TILE + c0 + cc];
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < KC; ++kk) {
                T a[8], b[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    a[i] = sA[kk][ty * 8 + i];
                    b[i] = sB[kk][tx * 8 + i];
                }
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
        }
    }
    __syncthreads();  // TRSM writes the tile it has just read
    T *dst = A + (S.ltile0 + (int64_t)g.i * (g.i + 1) / 2 + g.j) * KRR_TILE_ELEMS;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        T *row = dst + (int64_t)(ty * 8 + i) * KRR_TILE + tx * 8;
#pragma unroll
        for (int j = 0; j < 8; ++j) row[j] = (mode == UPD_TRSM) ? acc[i][j] : row[j] - acc[i][j];
    }
}

// ---------------------------------------------------------------- tcgen05 TF32
constexpr int TC_STAGES = 3;
constexpr int TC_CHUNK = 32;                                     // floats of K per stage (128 bytes)
constexpr uint32_t TC_STAGE_BYTES = 2u * KRR_TILE * TC_CHUNK * 4;  // A + B, 32 KB
constexpr uint32_t TC_IDESC = make_idesc(2u /*TF32*/, 128u, 128u);
constexpr size_t TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// wait with a ~2 s deadline; on expiry set *err and return false
__device__ __forceinline__ bool mbar_wait_deadline(uint64_t *bar, uint32_t parity, int *err) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 256; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 2000000000ull) {
            atomicExch(err, KRR_ERR_TIMEOUT);
            return false;
        }
    }
}

__global__ void __launch_bounds__(128, 1)
update_tf32_kernel(const __grid_constant__ CUtensorMap tmap, float *__restrict__ A,
                   const SolveDesc *__restrict__ solves, const int64_t *__restrict__ pre, int nsolve, int mode,
                   int K0, int W, int *__restrict__ err) {
    extern __shared__ unsigned char tc_dyn[];
    const uint32_t base = smem_u32(tc_dyn);
    unsigned char *buf = tc_dyn + (((base + 1023u) & ~1023u) - base);  // 1024-aligned stage ring
    uint64_t *full = reinterpret_cast<uint64_t *>(buf + TC_STAGES * TC_STAGE_BYTES);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *done = empty + TC_STAGES;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int s = find_solve(pre, nsolve, blockIdx.x);
    const SolveDesc S = solves[s];
    const TaskGeom g = decode_task(mode, (int64_t)blockIdx.x - pre[s], K0, W);
    const int nchunks = (g.ke - g.kb) * (KRR_TILE / TC_CHUNK);

    if (threadIdx.x == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(done, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tslot, 128);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (threadIdx.x == 0) {  // TMA producer
        for (int q = 0; q < nchunks; ++q) {
            const int st = q % TC_STAGES, use = q / TC_STAGES;
            if (use > 0 && !mbar_wait_deadline(&empty[st], (use - 1) & 1, err)) break;
            unsigned char *sa = buf + st * TC_STAGE_BYTES;
            unsigned char *sb = sa + TC_STAGE_BYTES / 2;
            const int kt = g.kb + q / (KRR_TILE / TC_CHUNK);
            const int x = (q % (KRR_TILE / TC_CHUNK)) * TC_CHUNK;
            const int ya = (int)((S.ltile0 + (int64_t)g.i * (g.i + 1) / 2 + kt) * KRR_TILE);
            const int yb = (int)((S.ltile0 + (int64_t)g.j * (g.j + 1) / 2 + kt) * KRR_TILE);
            mbar_arrive_expect_tx(&full[st], TC_STAGE_BYTES);
            tma_load_2d(sa, &tmap, x, ya, &full[st]);
            tma_load_2d(sb, &tmap, x, yb, &full[st]);
        }
    } else if (threadIdx.x == 32) {  // MMA issuer
        bool ok = true;
        for (int q = 0; q < nchunks && ok; ++q) {
            const int st = q % TC_STAGES, use = q / TC_STAGES;
            if (!mbar_wait_deadline(&full[st], use & 1, err)) {
                ok = false;
                break;
            }
            tc_fence_after();
            unsigned char *sa = buf + st * TC_STAGE_BYTES;
            unsigned char *sb = sa + TC_STAGE_BYTES / 2;
            const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sb);
#pragma unroll
            for (int kk = 0; kk < TC_CHUNK / 8; ++kk)  // K = 8 TF32 = 32 bytes per MMA
                tc_mma_tf32(tmem, da + 2 * kk, db + 2 * kk, TC_IDESC, (q > 0 || kk > 0) ? 1u : 0u);
            tc_commit(&empty[st]);
        }
        tc_commit(done);
    }
    __syncwarp();
    const bool have = mbar_wait_deadline(done, 0, err);
    tc_fence_after();
    if (have && *err == 0) {
        const int r = warp * 32 + lane;
        float *dst = A + (S.ltile0 + (int64_t)g.i * (g.i + 1) / 2 + g.j) * KRR_TILE_ELEMS + (int64_t)r * KRR_TILE;
#pragma unroll 1
        for (int cb = 0; cb < KRR_TILE / 32; ++cb) {
            float v[32];
            tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32), v);
            float4 *d4 = reinterpret_cast<float4 *>(dst + cb * 32);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float4 o = d4[q];
                o.x -= v[4 * q + 0];
                o.y -= v[4 * q + 1];
                o.z -= v[4 * q + 2];
                o.w -= v[4 * q + 3];
                d4[q] = o;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

// ---------------------------------------------------------------- host side
typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                    CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                    CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_encodeTiled)p;
    }
    return fn;
}

// 2-D view of a float tile store: rows of 128 floats, box 32 x 128, 128B swizzle
bool make_tile_tmap(CUtensorMap *map, float *store, int64_t ntiles) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)KRR_TILE, (cuuint64_t)(ntiles * KRR_TILE)};
    cuuint64_t strides[1] = {(cuuint64_t)KRR_TILE * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)TC_CHUNK, (cuuint32_t)KRR_TILE};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, store, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// One launch of the factorisation schedule.
struct CholLaunch {
    int kind;      // 0 potrf, 1 trsm, 2 update-trail, 3 update-column
    int K0, W;     // step parameters (see decode_task)
    int64_t pre;   // offset of this launch's prefix array in the plan buffer
    int64_t tasks; // total CTAs
};

// Build the schedule for a batch of solves with tile counts T[s].
void build_chol_plan(const std::vector<int> &T, int W, std::vector<CholLaunch> &plan, std::vector<int64_t> &pre) {
    const int ns = (int)T.size();
    int Tmax = 0;
    for (int t : T) Tmax = std::max(Tmax, t);
    plan.clear();
    pre.clear();
    auto add = [&](int kind, int K0, int Wp, auto count) {
        CholLaunch L;
        L.kind = kind;
        L.K0 = K0;
        L.W = Wp;
        L.pre = (int64_t)pre.size();
        int64_t run = 0;
        for (int s = 0; s < ns; ++s) {
            pre.push_back(run);
            run += count(T[s]);
        }
        pre.push_back(run);
        L.tasks = run;
        if (run > 0) plan.push_back(L); else pre.resize(L.pre);
    };
    for (int K0 = 0; K0 < Tmax; K0 += W) {
        const int Wb = std::min(W, Tmax - K0);
        for (int c = K0; c < K0 + Wb; ++c) {
            if (c > K0)
                add(3, K0, c, [&](int t) -> int64_t { return t > c ? (int64_t)(t - c) : 0; });
            add(0, c, 0, [&](int t) -> int64_t { return t > c ? 1 : 0; });
            add(1, c, 0, [&](int t) -> int64_t { return t > c + 1 ? (int64_t)(t - c - 1) : 0; });
        }
        add(2, K0, Wb, [&](int t) -> int64_t {
            int64_t r = (int64_t)t - K0 - Wb;
            return r > 0 ? r * (r + 1) / 2 : 0;
        });
    }
}

template <typename T>
cudaError_t run_chol_plan_t(cudaStream_t st, const std::vector<CholLaunch> &plan, const int64_t *d_pre, T *A, T *Z,
                            const SolveDesc *d_solves, int nsolve, int32_t *flags, bool tf32, const CUtensorMap *tmap,
                            int *d_err, Prof *prof) {
    const size_t po_sm = (size_t)KRR_TILE * 129 * sizeof(T);
    cudaFuncSetAttribute(potrf_tile_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)po_sm);
    for (const CholLaunch &L : plan) {
        const unsigned grid = (unsigned)L.tasks;
        const int64_t *p = d_pre + L.pre;
        ProfScope ps(prof, L.kind == 0 ? PROF_POTRF : (L.kind == 1 ? PROF_TRSM : PROF_UPDATE), st);
        if (L.kind == 0) {
            KRR_LAUNCHED(), potrf_tile_kernel<T><<<grid, 512, po_sm, st>>>(A, Z, d_solves, p, nsolve, L.K0, flags);
        } else if (L.kind == 1) {
            KRR_LAUNCHED(), gemm_tile_simt_kernel<T><<<grid, 256, 0, st>>>(A, Z, d_solves, p, nsolve, UPD_TRSM, L.K0, 0);
        } else {
            const int mode = (L.kind == 2) ? UPD_TRAIL : UPD_COLUMN;
            if constexpr (sizeof(T) == 4) {
                if (tf32) {
                    KRR_LAUNCHED(), update_tf32_kernel<<<grid, 128, TC_SMEM, st>>>(*tmap, reinterpret_cast<float *>(A), d_solves, p,
                                                                   nsolve, mode, L.K0, L.W, d_err);
                    continue;
                }
            }
            KRR_LAUNCHED(), gemm_tile_simt_kernel<T><<<grid, 256, 0, st>>>(A, Z, d_solves, p, nsolve, mode, L.K0, L.W);
        }
    }
    return cudaGetLastError();
}

cudaError_t run_chol_plan(cudaStream_t st, const std::vector<CholLaunch> &plan, const int64_t *d_pre, void *A, void *Z,
                          bool fp64, const SolveDesc *d_solves, int nsolve, int32_t *flags, bool tf32,
                          const CUtensorMap *tmap, int *d_err, Prof *prof) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(update_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
        attr = true;
    }
    if (fp64)
        return run_chol_plan_t<double>(st, plan, d_pre, (double *)A, (double *)Z, d_solves, nsolve, flags, false,
                                       tmap, d_err, prof);
    return run_chol_plan_t<float>(st, plan, d_pre, (float *)A, (float *)Z, d_solves, nsolve, flags, tf32, tmap,
                                  d_err, prof);
}

}  // namespace krr
