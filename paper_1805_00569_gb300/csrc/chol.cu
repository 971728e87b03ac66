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
// TF32 and FP32 run on the tcgen05 tensor cores (tile_mma_kernel): TF32 as one
// kind::tf32 pass, FP32 as three passes over a hi/lo split; the panel solve
// L_ik = A_ik Z_kk^T always runs as three passes (an FP32-class product).
#include <algorithm>

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

// Blocked FP32 version.  For each 32-column block b: warp 0 factors the
// 32 x 32 diagonal block in shared memory (lane i owns row i), the rows below
// solve against it in place (one thread per row), and the trailing part is
// updated block-parallel.  At the end warps 0..3 invert the four diagonal
// blocks in parallel (lane j owns column j) and the off-diagonal blocks of
// the tile inverse follow by block products.  Every serial phase is a compact
// rolled loop: the kernel runs once per tile and column, so straight-line
// unrolled code would be fetched from L2 on every SM.
constexpr int PB = 32;

__global__ void __launch_bounds__(256) potrf_tile_blocked_kernel(float *__restrict__ A, float *__restrict__ Z,
                                                                 const SolveDesc *__restrict__ solves,
                                                                 const int64_t *__restrict__ pre, int nsolve, int k,
                                                                 int32_t *__restrict__ flags) {
    extern __shared__ __align__(16) unsigned char po_dyn[];
    float *L = reinterpret_cast<float *>(po_dyn);  // [128][129]
    float *Zs = L + KRR_TILE * 129;                // [128][129]
    float *T = Zs + KRR_TILE * 129;                // [96][33] scratch
    __shared__ int bad_sh;
    const int s = find_solve(pre, nsolve, blockIdx.x);
    const SolveDesc S = solves[s];
    const int64_t tile = S.ltile0 + (int64_t)k * (k + 1) / 2 + k;
    float *g = A + tile * KRR_TILE_ELEMS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) bad_sh = 0;
    for (int e = threadIdx.x; e < KRR_TILE_ELEMS; e += blockDim.x) {
        const int rr = e >> 7, cc = e & 127;
        L[rr * 129 + cc] = g[e];
        if (cc / PB > rr / PB) Zs[rr * 129 + cc] = 0.f;  // strictly upper blocks of Z
    }
    __syncthreads();
#pragma unroll 1
    for (int b = 0; b < KRR_TILE / PB; ++b) {
        const int rb = b * PB;
        if (warp == 0) {  // diagonal block, right-looking, lane = row
            float *D = L + rb * 129 + rb;
#pragma unroll 1
            for (int c = 0; c < PB; ++c) {
                float dg = D[c * 129 + c];
                if (!(dg > 0.f)) {
                    dg = 1.f;
                    if (lane == 0) bad_sh = 1;
                }
                const float dc = sqrtf(dg);
                __syncwarp();
                if (lane > c) D[lane * 129 + c] /= dc;
                __syncwarp();
                if (lane == c) D[c * 129 + c] = dc;
                if (lane > c) {
                    const float lc = D[lane * 129 + c];
#pragma unroll 1
                    for (int j = c + 1; j <= lane; ++j) D[lane * 129 + j] -= lc * D[j * 129 + c];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // rows below: x L_bb^T = a, solved in place, one thread per row
        const int r = rb + PB + threadIdx.x;
        if (r < KRR_TILE) {
            float *x = L + r * 129 + rb;
            const float *D = L + rb * 129 + rb;
#pragma unroll 1
            for (int c = 0; c < PB; ++c) {
                float v = x[c];
#pragma unroll 4
                for (int q = 0; q < c; ++q) v -= x[q] * D[c * 129 + q];
                x[c] = v / D[c * 129 + c];
            }
        }
        __syncthreads();
        // trailing update of rows/cols >= rb + 32 (lower part), 2 x 2 per thread
        const int n2 = KRR_TILE - rb - PB;
        if (n2 > 0) {
            const int nb2 = n2 / 2;
            for (int e = threadIdx.x; e < nb2 * nb2; e += blockDim.x) {
                const int bi = e / nb2, bj = e % nb2;
                if (bj > bi) continue;
                const int r0 = rb + PB + 2 * bi, q0 = rb + PB + 2 * bj;
                float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
#pragma unroll 8
                for (int kk = 0; kk < PB; ++kk) {
                    const float a0 = L[r0 * 129 + rb + kk], a1 = L[(r0 + 1) * 129 + rb + kk];
                    const float b0 = L[q0 * 129 + rb + kk], b1 = L[(q0 + 1) * 129 + rb + kk];
                    s00 = fmaf(a0, b0, s00);
                    s01 = fmaf(a0, b1, s01);
                    s10 = fmaf(a1, b0, s10);
                    s11 = fmaf(a1, b1, s11);
                }
                L[r0 * 129 + q0] -= s00;
                L[(r0 + 1) * 129 + q0] -= s10;
                L[(r0 + 1) * 129 + q0 + 1] -= s11;
                if (bi != bj) L[r0 * 129 + q0 + 1] -= s01;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && bad_sh) flags[s] = 1;
    for (int e = threadIdx.x; e < KRR_TILE_ELEMS; e += blockDim.x) {
        const int rr = e >> 7, cc = e & 127;
        g[e] = (rr >= cc) ? L[rr * 129 + cc] : 0.f;
    }
    // diagonal blocks of the inverse: warp w inverts block w, lane j = column j
    if (warp < KRR_TILE / PB) {
        const int rb = warp * PB;
        const float *D = L + rb * 129 + rb;
        float *Zb = Zs + rb * 129 + rb;
#pragma unroll 1
        for (int i = 0; i < PB; ++i) {
            float v = (i == lane) ? 1.f : 0.f;
#pragma unroll 4
            for (int q = lane; q < i; ++q) v -= D[i * 129 + q] * Zb[q * 129 + lane];
            Zb[i * 129 + lane] = (i >= lane) ? v / D[i * 129 + i] : 0.f;
        }
    }
    __syncthreads();
    // off-diagonal blocks of Z by distance d: Z_ij = -Z_ii sum_{q=j}^{i-1} L_iq Z_qj
#pragma unroll 1
    for (int d = 1; d < KRR_TILE / PB; ++d) {
        const int nblk = KRR_TILE / PB - d;
        for (int e = threadIdx.x; e < nblk * PB * PB; e += blockDim.x) {
            const int jb = e / (PB * PB), rr = (e / PB) % PB, cc = e % PB;
            const int ib = jb + d;
            float v = 0.f;
            for (int qb = jb; qb < ib; ++qb)
#pragma unroll 8
                for (int q = 0; q < PB; ++q)
                    v = fmaf(L[(ib * PB + rr) * 129 + qb * PB + q], Zs[(qb * PB + q) * 129 + jb * PB + cc], v);
            T[(jb * PB + rr) * 33 + cc] = v;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nblk * PB * PB; e += blockDim.x) {
            const int jb = e / (PB * PB), rr = (e / PB) % PB, cc = e % PB;
            const int ib = jb + d;
            float v = 0.f;
#pragma unroll 4
            for (int q = 0; q <= rr; ++q)
                v = fmaf(Zs[(ib * PB + rr) * 129 + ib * PB + q], T[(jb * PB + q) * 33 + cc], v);
            Zs[(ib * PB + rr) * 129 + jb * PB + cc] = -v;
        }
        __syncthreads();
    }
    float *z = Z + (S.dtile0 + k) * KRR_TILE_ELEMS;
    for (int e = threadIdx.x; e < KRR_TILE_ELEMS; e += blockDim.x) {
        const int rr = e >> 7, cc = e & 127;
        z[e] = (rr >= cc) ? Zs[rr * 129 + cc] : 0.f;
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
// One CTA per task, 192 threads: warp 0 lane 0 streams the operand tiles with
// 2-D TMA loads (128-byte swizzle) through an mbarrier ring; warp 1 lane 0
// issues the MMAs into a 128 x 128 FP32 accumulator in tensor memory; warps
// 2..5 read it back (tcgen05.ld) for the epilogue (A_ij -= C, or A_ik = C for
// the panel solve).  X3 = false: one kind::tf32 MMA per K step (the tensor
// core reads the top 19 bits of each FP32 operand).  X3 = true: warps 2..5
// also split each landed stage into hi = x with the low 13 mantissa bits
// cleared and lo = x - hi (exact), and three MMAs per K step form
// hi*hi + hi*lo + lo*hi: FP32-class products on the tensor cores.
constexpr int TC_CHUNK = 32;                                       // floats of K per stage (128 bytes)
constexpr uint32_t TC_HALF = (uint32_t)KRR_TILE * TC_CHUNK * 4;     // one operand tile chunk, 16 KB
constexpr uint32_t TC_IDESC = make_idesc(2u /*TF32*/, 128u, 128u);
template <bool X3> struct TcCfg {
    static constexpr int STAGES = X3 ? 2 : 3;
    static constexpr uint32_t STAGE_BYTES = (X3 ? 4u : 2u) * TC_HALF;  // A, B (+ A_lo, B_lo)
    static constexpr size_t SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};

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

template <bool X3>
__global__ void __launch_bounds__(192, 1)
tile_mma_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmapZ,
                float *__restrict__ A, const SolveDesc *__restrict__ solves, const int64_t *__restrict__ pre,
                int nsolve, int mode, int K0, int W, int *__restrict__ err) {
    using Cfg = TcCfg<X3>;
    extern __shared__ unsigned char tc_dyn[];
    const uint32_t base = smem_u32(tc_dyn);
    unsigned char *buf = tc_dyn + (((base + 1023u) & ~1023u) - base);  // 1024-aligned stage ring
    uint64_t *full = reinterpret_cast<uint64_t *>(buf + Cfg::STAGES * Cfg::STAGE_BYTES);
    uint64_t *empty = full + Cfg::STAGES;
    uint64_t *split = empty + Cfg::STAGES;
    uint64_t *done = split + Cfg::STAGES;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int s = find_solve(pre, nsolve, blockIdx.x);
    const SolveDesc S = solves[s];
    const TaskGeom g = decode_task(mode, (int64_t)blockIdx.x - pre[s], K0, W);
    const int nchunks = (g.ke - g.kb) * (KRR_TILE / TC_CHUNK);

    if (threadIdx.x == 0) {
        for (int i = 0; i < Cfg::STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
            mbar_init(&split[i], 4);
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
            const int st = q % Cfg::STAGES, use = q / Cfg::STAGES;
            if (use > 0 && !mbar_wait_deadline(&empty[st], (use - 1) & 1, err)) break;
            unsigned char *sa = buf + st * Cfg::STAGE_BYTES;
            unsigned char *sb = sa + TC_HALF;
            const int kt = g.kb + q / (KRR_TILE / TC_CHUNK);
            const int x = (q % (KRR_TILE / TC_CHUNK)) * TC_CHUNK;
            const int ya = (int)((S.ltile0 + (int64_t)g.i * (g.i + 1) / 2 + kt) * KRR_TILE);
            mbar_arrive_expect_tx(&full[st], 2 * TC_HALF);
            tma_load_2d(sa, &tmap, x, ya, &full[st]);
            if (mode == UPD_TRSM) {
                tma_load_2d(sb, &tmapZ, x, (int)((S.dtile0 + kt) * KRR_TILE), &full[st]);
            } else {
                const int yb = (int)((S.ltile0 + (int64_t)g.j * (g.j + 1) / 2 + kt) * KRR_TILE);
                tma_load_2d(sb, &tmap, x, yb, &full[st]);
            }
        }
    } else if (threadIdx.x == 32) {  // MMA issuer
        bool ok = true;
        for (int q = 0; q < nchunks && ok; ++q) {
            const int st = q % Cfg::STAGES, use = q / Cfg::STAGES;
            if (!mbar_wait_deadline(X3 ? &split[st] : &full[st], use & 1, err)) {
                ok = false;
                break;
            }
            tc_fence_after();
            unsigned char *sa = buf + st * Cfg::STAGE_BYTES;
            unsigned char *sb = sa + TC_HALF;
            const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sb);
#pragma unroll
            for (int kk = 0; kk < TC_CHUNK / 8; ++kk) {  // K = 8 TF32 = 32 bytes per MMA
                const uint32_t acc0 = (q > 0 || kk > 0) ? 1u : 0u;
                tc_mma_tf32(tmem, da + 2 * kk, db + 2 * kk, TC_IDESC, acc0);
                if (X3) {
                    const uint64_t dal = smem_desc_sw128(sa + 2 * TC_HALF), dbl = smem_desc_sw128(sb + 2 * TC_HALF);
                    tc_mma_tf32(tmem, da + 2 * kk, dbl + 2 * kk, TC_IDESC, 1u);
                    tc_mma_tf32(tmem, dal + 2 * kk, db + 2 * kk, TC_IDESC, 1u);
                }
            }
            tc_commit(&empty[st]);
        }
        tc_commit(done);
    } else if (warp >= 2 && X3) {  // split landed stages into hi / lo
        const int t = threadIdx.x - 64;  // 0..127
        for (int q = 0; q < nchunks; ++q) {
            const int st = q % Cfg::STAGES, use = q / Cfg::STAGES;
            if (!mbar_wait_deadline(&full[st], use & 1, err)) break;
            float4 *hi = reinterpret_cast<float4 *>(buf + st * Cfg::STAGE_BYTES);
            float4 *lo = reinterpret_cast<float4 *>(buf + st * Cfg::STAGE_BYTES + 2 * TC_HALF);
#pragma unroll 4
            for (int e = t; e < (int)(2 * TC_HALF / 16); e += 128) {
                float4 v = hi[e], h, l;
                h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
                h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
                h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
                h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
                l.x = v.x - h.x;
                l.y = v.y - h.y;
                l.z = v.z - h.z;
                l.w = v.w - h.w;
                hi[e] = h;
                lo[e] = l;
            }
            fence_proxy_async_smem();  // generic-proxy writes -> visible to the tensor core
            __syncwarp();
            if (lane == 0) mbar_arrive(&split[st]);
        }
    }
    __syncwarp();
    if (warp >= 2) {  // epilogue
        const bool have = mbar_wait_deadline(done, 0, err);
        tc_fence_after();
        if (have && *err == 0) {
            const int quad = warp & 3;
            const int r = quad * 32 + lane;
            float *dst =
                A + (S.ltile0 + (int64_t)g.i * (g.i + 1) / 2 + g.j) * KRR_TILE_ELEMS + (int64_t)r * KRR_TILE;
#pragma unroll 1
            for (int cb = 0; cb < KRR_TILE / 32; ++cb) {
                float v[32];
                tmem_ld_32x32b_x32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cb * 32), v);
                float4 *d4 = reinterpret_cast<float4 *>(dst + cb * 32);
                if (mode == UPD_TRSM) {
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq)
                        d4[qq] = make_float4(v[4 * qq], v[4 * qq + 1], v[4 * qq + 2], v[4 * qq + 3]);
                } else {
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        float4 o = d4[qq];
                        o.x -= v[4 * qq + 0];
                        o.y -= v[4 * qq + 1];
                        o.z -= v[4 * qq + 2];
                        o.w -= v[4 * qq + 3];
                        d4[qq] = o;
                    }
                }
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
    if (ntiles <= 0) ntiles = 1;
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
    int tc;        // update arithmetic: 0 SIMT, 1 TF32 one pass, 3 three passes
};

// Build the schedule for a batch of solves with tile counts T[s] and update
// classes cls[s] (0 SIMT, 1 TF32, 3 three-pass): the diagonal factorisations
// and panel solves of all solves share their launches; each update step is
// one launch per class present.
void build_chol_plan(const std::vector<int> &T, const std::vector<int> &cls, int W, std::vector<CholLaunch> &plan,
                     std::vector<int64_t> &pre) {
    const int ns = (int)T.size();
    int Tmax = 0;
    for (int t : T) Tmax = std::max(Tmax, t);
    std::vector<int> classes;
    for (int s = 0; s < ns; ++s)
        if (std::find(classes.begin(), classes.end(), cls[s]) == classes.end()) classes.push_back(cls[s]);
    std::sort(classes.begin(), classes.end());
    plan.clear();
    pre.clear();
    auto add = [&](int kind, int K0, int Wp, int tc, auto count) {
        CholLaunch L;
        L.kind = kind;
        L.K0 = K0;
        L.W = Wp;
        L.tc = tc;
        L.pre = (int64_t)pre.size();
        int64_t run = 0;
        for (int s = 0; s < ns; ++s) {
            pre.push_back(run);
            if (kind < 2 || cls[s] == tc) run += count(T[s]);
        }
        pre.push_back(run);
        L.tasks = run;
        if (run > 0) plan.push_back(L); else pre.resize(L.pre);
    };
    for (int K0 = 0; K0 < Tmax; K0 += W) {
        const int Wb = std::min(W, Tmax - K0);
        for (int c = K0; c < K0 + Wb; ++c) {
            if (c > K0)
                for (int tc : classes)
                    add(3, K0, c, tc, [&](int t) -> int64_t { return t > c ? (int64_t)(t - c) : 0; });
            add(0, c, 0, 0, [&](int t) -> int64_t { return t > c ? 1 : 0; });
            add(1, c, 0, 0, [&](int t) -> int64_t { return t > c + 1 ? (int64_t)(t - c - 1) : 0; });
        }
        for (int tc : classes)
            add(2, K0, Wb, tc, [&](int t) -> int64_t {
                int64_t r = (int64_t)t - K0 - Wb;
                return r > 0 ? r * (r + 1) / 2 : 0;
            });
    }
}

template <typename T>
cudaError_t run_chol_plan_t(cudaStream_t st, const std::vector<CholLaunch> &plan, const int64_t *d_pre, T *A, T *Z,
                            const SolveDesc *d_solves, int nsolve, int32_t *flags, int tc, const CUtensorMap *tmap,
                            const CUtensorMap *tmapZ, int *d_err, Prof *prof) {
    const size_t po_sm = (size_t)KRR_TILE * 129 * sizeof(T);
    cudaFuncSetAttribute(potrf_tile_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)po_sm);
    const size_t po_blk_sm = (2 * (size_t)KRR_TILE * 129 + 96 * 33) * sizeof(float);
    cudaFuncSetAttribute(potrf_tile_blocked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)po_blk_sm);
    for (const CholLaunch &L : plan) {
        const unsigned grid = (unsigned)L.tasks;
        const int64_t *p = d_pre + L.pre;
        ProfScope ps(prof, L.kind == 0 ? PROF_POTRF : (L.kind == 1 ? PROF_TRSM : PROF_UPDATE), st);
        if (L.kind == 0) {
            if constexpr (sizeof(T) == 4)
                KRR_LAUNCHED(), potrf_tile_blocked_kernel<<<grid, 256, po_blk_sm, st>>>(
                    reinterpret_cast<float *>(A), reinterpret_cast<float *>(Z), d_solves, p, nsolve, L.K0, flags);
            else
                KRR_LAUNCHED(), potrf_tile_kernel<T><<<grid, 512, po_sm, st>>>(A, Z, d_solves, p, nsolve, L.K0,
                                                                               flags);
            continue;
        }
        const int mode = L.kind == 1 ? UPD_TRSM : (L.kind == 2 ? UPD_TRAIL : UPD_COLUMN);
        const int W = L.kind == 1 ? 0 : L.W;
        if constexpr (sizeof(T) == 4) {
            // tensor cores: the panel solve always FP32-class (3 passes); the
            // trailing updates 1 pass (TF32) or 3 passes (FP32), per launch class
            if (tc != 0) {
                const bool x3 = (L.kind == 1) || L.tc == 3;
                if (x3)
                    KRR_LAUNCHED(), tile_mma_kernel<true><<<grid, 192, TcCfg<true>::SMEM, st>>>(
                        *tmap, *tmapZ, reinterpret_cast<float *>(A), d_solves, p, nsolve, mode, L.K0, W, d_err);
                else
                    KRR_LAUNCHED(), tile_mma_kernel<false><<<grid, 192, TcCfg<false>::SMEM, st>>>(
                        *tmap, *tmapZ, reinterpret_cast<float *>(A), d_solves, p, nsolve, mode, L.K0, W, d_err);
                continue;
            }
        }
        KRR_LAUNCHED(), gemm_tile_simt_kernel<T><<<grid, 256, 0, st>>>(A, Z, d_solves, p, nsolve, mode, L.K0, W);
    }
    return cudaGetLastError();
}

// tc: 0 = SIMT trailing updates, 1 = TF32 (1 pass), 3 = FP32-class (3 passes)
cudaError_t run_chol_plan(cudaStream_t st, const std::vector<CholLaunch> &plan, const int64_t *d_pre, void *A, void *Z,
                          bool fp64, const SolveDesc *d_solves, int nsolve, int32_t *flags, int tc,
                          const CUtensorMap *tmap, const CUtensorMap *tmapZ, int *d_err, Prof *prof) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tile_mma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcCfg<false>::SMEM);
        cudaFuncSetAttribute(tile_mma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcCfg<true>::SMEM);
        attr = true;
    }
    if (fp64)
        return run_chol_plan_t<double>(st, plan, d_pre, (double *)A, (double *)Z, d_solves, nsolve, flags, 0, tmap,
                                       tmapZ, d_err, prof);
    return run_chol_plan_t<float>(st, plan, d_pre, (float *)A, (float *)Z, d_solves, nsolve, flags, tc, tmap, tmapZ,
                                  d_err, prof);
}

}  // namespace krr
