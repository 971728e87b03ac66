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

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

namespace krr {

enum { UPD_TRAIL = 0, UPD_COLUMN = 1, UPD_TRSM = 2 };

// Programmatic dependent launch: the factorisation's launches form one long
// dependent chain, so each kernel lets the next one be scheduled early
// (launch_dependents) and waits for its predecessor's results (wait) only
// after its own set-up; a kernel is scheduled early only once every CTA of
// its predecessor is resident, and the wait is a hardware dependency.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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
// Cholesky factor L and inverse Z = L^-1 of one 128 x 128 diagonal tile in a
// single right-looking sweep with the tile held in registers (the FP64 path;
// FP32 factors use potrf_blocked_kernel below).  512 threads:
// thread (rg = tid / 16, cg = tid % 16) owns the 4 x 8 block of rows
// 4 rg .. 4 rg + 3 and columns 8 cg .. 8 cg + 7, so a step reads 4 row and 8
// column values of the broadcast vector for its 32 updates.  An entry (i, j)
// holds A_ij until column j is eliminated and from then on the entry X_ij of
// the inverse being formed, so every step is one broadcast and one rank-1
// update of the same registers.  Step q:
//   publish  b[i] = A_iq (i > q, unscaled column q), b[q] = A_qq + 1,
//            b[j] = X~_qj (j < q, row q of the inverse before its scaling),
//            and the pivot's rl = 1 / sqrt(A_qq);
//   L(:, q) = b(:) rl (L_qq = A_qq rl);
//   update   every row i > q: v_ij -= (b[i] rl^2) b[j]
// For j > q this is A_ij -= L_iq L_jq; for j < q it is X_ij -= L_iq X_qj with
// X_qj = X~_qj rl; for j = q the entry turns into X_iq = -L_iq / L_qq, which
// the shifted b[q] produces from A_iq in the same fused multiply-add.  Row q
// of the inverse is final once scaled by rl (X_qq = rl).  The step loop is
// rolled (the kernel runs once per tile column, so a straight-line body would
// be fetched from L2 on every SM); the 4 x 8 update is unrolled.
template <typename T>
__device__ __forceinline__ T potrf_rsqrt(T x);
template <>
__device__ __forceinline__ float potrf_rsqrt<float>(float x) {
    const float r = rsqrtf(x);
    return r * fmaf(-0.5f * x * r, r, 1.5f);  // one Newton step
}
template <>
__device__ __forceinline__ double potrf_rsqrt<double>(double x) { return 1.0 / sqrt(x); }

// padded broadcast index: 4 extra words per 32 columns, so the 8-lane phases
// of a warp's 16-byte loads of 8-column groups hit distinct banks
__device__ __forceinline__ int po_idx(int c) { return c + ((c >> 5) << 2); }

template <typename T> struct PoVec;
template <> struct PoVec<float> { using V = float4; static constexpr int N = 4; };
template <> struct PoVec<double> { using V = double2; static constexpr int N = 2; };
template <typename T, typename V>
__device__ __forceinline__ void po_unpack(const V &w, T *dst) {
    if constexpr (sizeof(V) / sizeof(T) == 4) {
        dst[0] = w.x; dst[1] = w.y; dst[2] = w.z; dst[3] = w.w;
    } else {
        dst[0] = w.x; dst[1] = w.y;
    }
}

template <typename T>
__global__ void __launch_bounds__(512, 1) potrf_tile_kernel(T *__restrict__ A, T *__restrict__ Z,
                                                            const SolveDesc *__restrict__ solves,
                                                            const int64_t *__restrict__ pre, int nsolve, int k,
                                                            int32_t *__restrict__ flags) {
    using V = typename PoVec<T>::V;
    constexpr int VN = PoVec<T>::N;
    extern __shared__ __align__(16) unsigned char po_dyn[];
    T *Ls = reinterpret_cast<T *>(po_dyn);  // [128][129] the factor, column by column
    __shared__ __align__(16) T bsh[2][KRR_TILE + 16];
    __shared__ T psh[2][2];  // (pivot, 1 / sqrt(pivot))
    __shared__ int bad_sh;
    pdl_launch_dependents();
    pdl_wait();  // the column update of this diagonal tile has completed
    const int s = find_solve(pre, nsolve, blockIdx.x);
    const SolveDesc S = solves[s];
    const int64_t tile = S.ltile0 + (int64_t)k * (k + 1) / 2 + k;
    T *g = A + tile * KRR_TILE_ELEMS;
    const int rg = threadIdx.x >> 4, cg = threadIdx.x & 15;
    const int r0 = rg * 4, c0 = cg * 8;
    T v[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const V *src = reinterpret_cast<const V *>(g + (r0 + r) * KRR_TILE + c0);
#pragma unroll
        for (int m = 0; m < 8 / VN; ++m) po_unpack<T>(src[m], &v[r][VN * m]);
    }
    if (threadIdx.x == 0) bad_sh = 0;
#pragma unroll 1
    for (int q = 0; q < KRR_TILE; ++q) {
        T *b = bsh[q & 1];
        if (cg == (q >> 3) && r0 + 3 >= q) {  // column q of A, rows >= q
            T col[4];
            switch (q & 7) {
#define KRR_COL(c) \
    case c: col[0] = v[0][c]; col[1] = v[1][c]; col[2] = v[2][c]; col[3] = v[3][c]; break;
                KRR_COL(0) KRR_COL(1) KRR_COL(2) KRR_COL(3) KRR_COL(4) KRR_COL(5) KRR_COL(6) KRR_COL(7)
#undef KRR_COL
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r0 + r == q) {
                    T pv = col[r];
                    if (!(pv > T(0))) {  // not positive: record, continue with 1 (no NaNs)
                        bad_sh = 1;
                        pv = T(1);
                    }
                    psh[q & 1][0] = pv;
                    psh[q & 1][1] = potrf_rsqrt<T>(pv);
                    b[po_idx(q)] = pv + T(1);
                } else if (r0 + r > q) {
                    b[po_idx(r0 + r)] = col[r];
                }
            }
        }
        if (rg == (q >> 2)) {  // row q of the inverse, before scaling
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (r0 + r == q) {
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c0 + c < q) b[po_idx(c0 + c)] = v[r][c];
                }
        }
        __syncthreads();
        const T rl = psh[q & 1][1];
        if (threadIdx.x < KRR_TILE && (int)threadIdx.x >= q)
            Ls[threadIdx.x * 129 + q] =
                ((int)threadIdx.x == q) ? psh[q & 1][0] * rl : b[po_idx(threadIdx.x)] * rl;
        if (r0 + 3 >= q) {
            const T inv = rl * rl;
            T rb[4], cb[8];
            const T *br = b + po_idx(r0), *bc = b + po_idx(c0);  // contiguous: no 32-column crossing
            po_unpack<T>(*reinterpret_cast<const V *>(br), rb);
            if constexpr (VN == 2) po_unpack<T>(*reinterpret_cast<const V *>(br + 2), rb + 2);
#pragma unroll
            for (int m = 0; m < 8 / VN; ++m) po_unpack<T>(*reinterpret_cast<const V *>(bc + VN * m), cb + VN * m);
            // rows <= q take a zero multiplier (x + 0 b = x exactly): no divergence
            T ci[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) ci[r] = (r0 + r > q) ? -rb[r] * inv : T(0);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) v[r][c] = fma(ci[r], cb[c], v[r][c]);
            if (rg == (q >> 2)) {  // row q of the inverse: scale by rl
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (r0 + r == q) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            if (c0 + c < q) v[r][c] *= rl;
                            else if (c0 + c == q) v[r][c] = rl;
                        }
                    }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && bad_sh) flags[s] = 1;
    for (int e = threadIdx.x; e < KRR_TILE_ELEMS; e += blockDim.x) {
        const int rr = e >> 7, cc = e & 127;
        g[e] = (rr >= cc) ? Ls[rr * 129 + cc] : T(0);
    }
    T *z = Z + (S.dtile0 + k) * KRR_TILE_ELEMS;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        T w[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) w[c] = (c0 + c <= r0 + r) ? v[r][c] : T(0);
        V *dst = reinterpret_cast<V *>(z + (r0 + r) * KRR_TILE + c0);
#pragma unroll
        for (int m = 0; m < 8 / VN; ++m) {
            V o;
            if constexpr (VN == 4) {
                o.x = w[4 * m]; o.y = w[4 * m + 1]; o.z = w[4 * m + 2]; o.w = w[4 * m + 3];
            } else {
                o.x = w[2 * m]; o.y = w[2 * m + 1];
            }
            dst[m] = o;
        }
    }
}

// ---------------------------------------------------------------- potrf, blocked (FP32)
// The same factor L and inverse Z of one FP32 diagonal tile, blocked by 32
// columns so that block barriers come per block, not per column.  For each
// 32-column block kb (rows and columns [o, o + 32), o = 32 kb):
//   A. the previous block's rank-32 update of this block's 32 x 32 diagonal
//      block only (lookahead: the rest of that update is not needed yet).
//   B. warp 0 factors the diagonal block and inverts it in registers (lane i
//      holds row i; values travel by shuffle, no block barrier).  Meanwhile
//      the warps on the other three schedulers finish the previous block's
//      rank-32 update of the lower trailing part, copy the block's columns
//      below the diagonal block, transposed, into Pt, and form
//      T = L_kb,<o Z_<o,<o, the first half of the blocked triangular inverse
//        Z_kb,jb = -Z_kb,kb sum_{m in blocks [jb, kb)} L_kb,m Z_m,jb.
//   C. the rows below solve against the block's inverse,
//      L_r,kb = A_r,kb Z_kb,kb^T (into Pn, which the next block's updates
//      read), while Z_kb,<o = -Z_kb,kb T completes the inverse's block row.
// The products run as 4 x 4 register tiles from 16-byte shared loads of the
// transposed panel (two loads per 16 fused multiply-adds).  Eleven block
// barriers instead of one per column.  Shared memory: the tile (padded rows:
// lanes reading a column hit distinct banks), Z, the transposed panel Pt,
// the solved panel Pn, the diagonal block's inverse transposed (Zt), its L
// rows (Lb) and T.
constexpr int PO_B = 32;               // block width
constexpr int PO_LD = KRR_TILE + 1;    // padded row stride of the tile
constexpr int PO_ZL = KRR_TILE + 4;    // row stride of Z (16-byte rows: T reads four Z columns at once)
constexpr int PO_PT = KRR_TILE + 4;    // row stride of Pt (16-byte rows)
constexpr int PO_ZT = PO_B + 4;        // row stride of Zt
constexpr int PO_TT = KRR_TILE - PO_B + 4;  // row stride of T
constexpr size_t PO_BLOCKED_SMEM =
    ((size_t)KRR_TILE * (PO_LD + PO_ZL) + (size_t)PO_B * (2 * PO_PT + 2 * PO_ZT + PO_TT)) * sizeof(float);

__device__ __forceinline__ void po_tri_decode(int t, int &a, int &b) {  // t = a (a + 1) / 2 + b, b <= a
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    a = r;
    b = t - r * (r + 1) / 2;
}

// Rank-32 update of the 4 x 4 tile (a, b), b <= a, of the tile's lower part
// from row and column `base` on, by the solved panel Pn (Pn[kk][r] = L_r,kk of
// the previous block): A -= L L^T there (upper entries of a diagonal tile kept).
__device__ __forceinline__ void po_rank32_tile(float *__restrict__ Ls, const float *__restrict__ Pn, int base,
                                               int a, int b) {
    const int r0 = base + 4 * a, c0 = base + 4 * b;
    float acc[4][4] = {};
#pragma unroll 4
    for (int kk = 0; kk < PO_B; ++kk) {
        const float4 x = *reinterpret_cast<const float4 *>(Pn + kk * PO_PT + r0);
        const float4 y = *reinterpret_cast<const float4 *>(Pn + kk * PO_PT + c0);
        const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xv[u], yv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
            if (a != b || v <= u) Ls[(r0 + u) * PO_LD + c0 + v] -= acc[u][v];
}

__global__ void __launch_bounds__(512, 1) potrf_blocked_kernel(float *__restrict__ A, float *__restrict__ Z,
                                                               const float *__restrict__ Kfirst,
                                                               const SolveDesc *__restrict__ solves,
                                                               const int64_t *__restrict__ pre, int nsolve, int k,
                                                               int32_t *__restrict__ flags) {
    extern __shared__ __align__(16) unsigned char po_dyn[];
    float *Ls = reinterpret_cast<float *>(po_dyn);  // [128][PO_LD]: A, becoming L
    float *Zs = Ls + KRR_TILE * PO_LD;              // [128][PO_ZL]: Z
    float *Pt = Zs + KRR_TILE * PO_ZL;              // [32][PO_PT]: Pt[kk][r] = (A or L)_r,o+kk
    float *Zt = Pt + PO_B * PO_PT;                  // [32][PO_ZT]: Zt[kk][c] = Z_o+c,o+kk
    float *Ts = Zt + PO_B * PO_ZT;                  // [32][PO_TT]: T of the blocked inverse
    float *Pn = Ts + PO_B * PO_TT;                  // [32][PO_PT]: Pn[c][r] = L_r,o+c (the solved panel)
    float *Lb = Pn + PO_B * PO_PT;                  // [32][PO_ZT]: the diagonal block's L rows, 1 / L_ii
    __shared__ int bad_sh;
    pdl_launch_dependents();
    pdl_wait();  // the column update of this diagonal tile has completed
    const int s = find_solve(pre, nsolve, blockIdx.x);
    const SolveDesc S = solves[s];
    const int64_t tile = S.ltile0 + (int64_t)k * (k + 1) / 2 + k;
    float *g = A + tile * KRR_TILE_ELEMS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) bad_sh = 0;
    // the first diagonal tile's first touch reads the kernel store: K_00 + lambda m I
    const bool kf = Kfirst != nullptr && k == 0;
    const float *src = kf ? Kfirst + S.ktile0 * KRR_TILE_ELEMS : g;
    const float lm = (float)S.lambda_m;
    {
        // the tile in 16-byte loads, all issued before any is used
        constexpr int NV = KRR_TILE_ELEMS / 4 / 512;  // float4 per thread
        float4 v[NV];
#pragma unroll
        for (int u = 0; u < NV; ++u) v[u] = reinterpret_cast<const float4 *>(src)[tid + u * 512];
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int e = (tid + u * 512) * 4, r = e >> 7, c = e & 127;
            const float w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                Ls[r * PO_LD + c + q] = c + q <= r ? (kf && r == c + q && r < S.m ? w[q] + lm : w[q]) : 0.f;
                Zs[r * PO_ZL + c + q] = 0.f;
            }
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int kb = 0; kb < KRR_TILE / PO_B; ++kb) {
        const int o = kb * PO_B;
        const int b0 = o + PO_B;             // first row below the block
        const int nr = KRR_TILE - b0;        // rows below the block
        // ---- A (lookahead): the previous block's rank-32 update of this
        // block's diagonal block only (the 36 lower 4 x 4 tiles); the rest of
        // that update runs beside warp 0's phase below
        if (kb > 0) {
            if (tid < 36) {
                int a, b;
                po_tri_decode(tid, a, b);
                po_rank32_tile(Ls, Pn, o, a, b);
            }
            __syncthreads();
        }
        // ---- B: the diagonal block (warp 0); the rest of the previous
        // block's update, then Pt and T (warps on the other schedulers)
        if (warp == 0) {
            // factor: step q scales column q by 1 / sqrt(pivot) and updates
            // the columns right of it; entries right of a lane's diagonal
            // collect values that are never read (their multiplier is 0 by
            // the time they are)
            float d[PO_B];
#pragma unroll
            for (int j = 0; j < PO_B; ++j) d[j] = j <= lane ? Ls[(o + lane) * PO_LD + o + j] : 0.f;
            float dinv = 0.f;  // 1 / L_ii of this lane's row
            bool bad = false;
#pragma unroll
            for (int q = 0; q < PO_B; ++q) {
                float pv = __shfl_sync(0xffffffffu, d[q], q);
                if (!(pv > 0.f)) {  // not positive: record, continue with 1 (no NaNs)
                    bad = true;
                    pv = 1.f;
                }
                // MUFU reciprocal square root (2 ulp): the pivot's rounding is
                // far below the factor classes' own (11-bit to FP32-class) errors
                const float rl = rsqrtf(pv);
                const float l = lane > q ? d[q] * rl : (lane == q ? pv * rl : 0.f);
                if (lane == q) dinv = rl;
                d[q] = l;
#pragma unroll
                for (int j = q + 1; j < PO_B; ++j) d[j] = fmaf(-l, __shfl_sync(0xffffffffu, l, j), d[j]);
            }
            // the block's L rows go to shared memory first (16-byte rows in
            // Lb): the inverse reads row i of L there with broadcast loads
#pragma unroll
            for (int j = 0; j < PO_B; ++j) {
                if (j <= lane) Ls[(o + lane) * PO_LD + o + j] = d[j];
                Lb[lane * PO_ZT + j] = j <= lane ? d[j] : 0.f;
            }
            Lb[lane * PO_ZT + PO_B] = dinv;  // spare column: 1 / L_ii
            __syncwarp();
            // inverse of the block: lane j forms column j, four rows at a time:
            // their sums over the columns before the group are independent of
            // each other, then the group's own 4 x 4 triangle in row order
            float z[PO_B];
#pragma unroll
            for (int i0 = 0; i0 < PO_B; i0 += 4) {
                float sg[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float *li = Lb + (i0 + u) * PO_ZT;
                    float a0 = 0.f, a1 = 0.f;
#pragma unroll
                    for (int k4 = 0; k4 < i0; k4 += 4) {
                        const float4 lv = *reinterpret_cast<const float4 *>(li + k4);
                        a0 = fmaf(lv.x, z[k4], fmaf(lv.y, z[k4 + 1], a0));
                        a1 = fmaf(lv.z, z[k4 + 2], fmaf(lv.w, z[k4 + 3], a1));
                    }
                    sg[u] = a0 + a1;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u;
                    const float *li = Lb + i * PO_ZT;
                    float acc = sg[u];
#pragma unroll
                    for (int v = 0; v < u; ++v) acc = fmaf(li[i0 + v], z[i0 + v], acc);
                    const float inv_ii = li[PO_B];
                    z[i] = lane == i ? inv_ii : (lane < i ? -acc * inv_ii : 0.f);
                }
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < PO_B; ++i) {
                Zs[(o + i) * PO_ZL + o + lane] = i >= lane ? z[i] : 0.f;
                Zt[lane * PO_ZT + i] = i >= lane ? z[i] : 0.f;  // Zt[kk = lane][c = i] = Z_o+i,o+lane
            }
            if (bad && lane == 0) bad_sh = 1;
        } else if ((warp & 3) != 0) {
            // the 12 warps on the other three schedulers (warps 4, 8, 12 share
            // warp 0's scheduler and stay idle: its serial chain keeps the issue slots)
            const int t2 = (warp - 1 - (warp >> 2)) * 32 + lane;  // 0..383
            constexpr int NB = 12 * 32;
            if (kb > 0) {
                // the previous block's update of rows and columns >= o outside
                // this block's diagonal block: lower 4 x 4 tiles (a, b), a >= 8
                const int RT = (KRR_TILE - o) / 4;
                for (int t = 36 + t2; t < RT * (RT + 1) / 2; t += NB) {
                    int a, b;
                    po_tri_decode(t, a, b);
                    po_rank32_tile(Ls, Pn, o, a, b);
                }
                asm volatile("bar.sync 2, 384;" ::: "memory");  // these 12 warps: the panel columns are final
            }
            // Pt[kk][r] = A_r,o+kk for the rows below the block
            for (int e = t2; e < nr * PO_B; e += NB) {
                const int kk = e / nr, r = b0 + (e - kk * nr);
                Pt[kk * PO_PT + r] = Ls[r * PO_LD + o + kk];
            }
            // T_i,c = sum_{m < o} L_o+i,m Z_m,c for c < o (Z_m,c = 0 for m < c), 4 x 4
            // tiles, one 16-byte load of Z per step: few shared loads beside warp 0's chain
            const int ntt = (PO_B / 4) * (o / 4);
            for (int t = t2; t < ntt; t += NB) {
                const int i0 = (t / (o / 4)) * 4, c0 = (t % (o / 4)) * 4;
                float acc[4][4] = {};
                for (int m = c0; m < o; ++m) {
                    const float4 zz = *reinterpret_cast<const float4 *>(Zs + m * PO_ZL + c0);
                    const float zv[4] = {zz.x, zz.y, zz.z, zz.w};
                    float lv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) lv[u] = Ls[(o + i0 + u) * PO_LD + m];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(lv[u], zv[v], acc[u][v]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    *reinterpret_cast<float4 *>(Ts + (i0 + u) * PO_TT + c0) =
                        make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
            }
        }
        __syncthreads();
        // ---- C: rows below and the inverse's block row, as one list of 4 x 4 tiles:
        // tiles [0, np) solve rows below into Pn (transposed, like Pt), tiles
        // [np, np + nz) form Z_kb,<o = -Z_kb,kb T
        const int np = (nr / 4) * (PO_B / 4), nz = (PO_B / 4) * (o / 4);
        for (int t = tid; t < np + nz; t += blockDim.x) {
            float acc[4][4] = {};
            if (t < np) {
                const int r0 = b0 + (t >> 3) * 4, c0 = (t & 7) * 4;
#pragma unroll 4
                for (int kk = 0; kk < PO_B; ++kk) {  // Z_o+c,o+kk = 0 for kk > c
                    const float4 a = *reinterpret_cast<const float4 *>(Pt + kk * PO_PT + r0);
                    const float4 zz = *reinterpret_cast<const float4 *>(Zt + kk * PO_ZT + c0);
                    const float av[4] = {a.x, a.y, a.z, a.w}, zv[4] = {zz.x, zz.y, zz.z, zz.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], zv[v], acc[u][v]);
                }
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    *reinterpret_cast<float4 *>(Pn + (c0 + v) * PO_PT + r0) =
                        make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
            } else {
                const int tz = t - np;
                const int i0 = (tz / (o / 4)) * 4, c0 = (tz % (o / 4)) * 4;
#pragma unroll 4
                for (int kk = 0; kk < PO_B; ++kk) {  // Z_o+i,o+kk = 0 for kk > i
                    const float4 tt = *reinterpret_cast<const float4 *>(Ts + kk * PO_TT + c0);
                    const float tv[4] = {tt.x, tt.y, tt.z, tt.w};
                    float zv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) zv[u] = Zs[(o + i0 + u) * PO_ZL + o + kk];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(zv[u], tv[v], acc[u][v]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) Zs[(o + i0 + u) * PO_ZL + c0 + v] = -acc[u][v];
            }
        }
        if (nr == 0) break;  // the last block has nothing below it
        __syncthreads();
        // the solved panel into the tile: L_r,o+c = Pn[c][r]
        for (int e = tid; e < nr * PO_B; e += blockDim.x) {
            const int c = e / nr, r = b0 + (e - c * nr);
            Ls[r * PO_LD + o + c] = Pn[c * PO_PT + r];
        }
        // (the update by this block's panel starts at the next block's step A)
    }
    __syncthreads();
    // the solve's descriptor again (not held in registers across the blocks)
    const int s2 = find_solve(pre, nsolve, blockIdx.x);
    if (tid == 0 && bad_sh) flags[s2] = 1;
    g = A + (solves[s2].ltile0 + (int64_t)k * (k + 1) / 2 + k) * KRR_TILE_ELEMS;
    float *z = Z + (solves[s2].dtile0 + k) * KRR_TILE_ELEMS;
    for (int e4 = tid; e4 < KRR_TILE_ELEMS / 4; e4 += blockDim.x) {
        const int e = e4 * 4, r = e >> 7, c = e & 127;
        const float *lr = Ls + r * PO_LD + c, *zr = Zs + r * PO_ZL + c;
        reinterpret_cast<float4 *>(g)[e4] =
            make_float4(c <= r ? lr[0] : 0.f, c + 1 <= r ? lr[1] : 0.f, c + 2 <= r ? lr[2] : 0.f,
                        c + 3 <= r ? lr[3] : 0.f);
        reinterpret_cast<float4 *>(z)[e4] = make_float4(zr[0], zr[1], zr[2], zr[3]);
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
// Persistent: each CTA takes tasks blockIdx.x, blockIdx.x + gridDim.x, ... of
// one launch (a task is one 128 x 128 output tile).  Warp 0 lane 0 streams the
// operand tiles of all its tasks with 2-D TMA loads (128-byte swizzle) through
// an mbarrier ring; warp 1 lane 0 issues the MMAs of task t into one of two
// 128-column FP32 accumulators in tensor memory (t % 2); warps 2..5 read the
// other one back (tcgen05.ld) for the epilogue of the previous task, so loads,
// MMAs and epilogues of consecutive tasks overlap and the per-CTA setup is
// paid once per launch.  Update epilogue: the destination tile A_ij lands in
// shared memory by TMA while the task's MMAs run, A_ij -= C is formed there
// (128-byte swizzle: conflict-free row access) and the tile leaves by TMA
// store; the panel solve (A_ik = C, no read) stores directly.
// TC_TF32: one kind::tf32 MMA per K step (the tensor core reads the top 19
// bits of each FP32 operand).  TC_F16: one kind::f16 MMA per K step on the
// FP16 copy of the panel (the same 11-bit significand as TF32 at twice the
// rate and half the operand bytes); the panel solve of a class-1 solve writes
// its L tiles in FP16 for this.  TC_BF16X3: warps 6..9 convert each landed FP32
// stage into BF16 hi = rn(x) and lo = rn(x - hi) operands and three kind::f16
// MMAs per K step form hi*hi + hi*lo + lo*hi (~16-bit products at the BF16
// rate).  TC_TF32X3P: the three-pass form on operands split once, by the
// panel solve that wrote them: x (FP32 store; the tensor core reads its top
// 19 bits, hi) and lo = x - hi (FP32 side store); TMA lands x and lo, no
// split warps.  TC_TF32X3: warps 6..9 split each landed stage
// into hi = x rounded to the nearest TF32 value and lo = x - hi (exact), and
// three MMAs per K step form hi*hi + hi*lo + lo*hi: FP32-class products on
// the tensor cores.  TC_TRSM (the panel solve) splits the same way and takes
// three passes for every solve: a one-pass panel solve for the one-pass
// (class 1) solves, whose L tiles are kept in FP16, was measured to cost
// more refinement iterations than it saves.
constexpr int TC_CHUNK = 32;                                       // floats of K per stage (128 bytes)
constexpr uint32_t TC_HALF = (uint32_t)KRR_TILE * TC_CHUNK * 4;     // one operand tile chunk, 16 KB
constexpr uint32_t TC_IDESC = make_idesc(2u /*TF32*/, 128u, 128u);
constexpr uint32_t TC_IDESC_BF16 = make_idesc(1u /*BF16*/, 128u, 128u);
constexpr uint32_t TC_IDESC_F16 = make_idesc(0u /*F16*/, 128u, 128u);
constexpr uint32_t TC_BHALF = (uint32_t)KRR_TILE * TC_CHUNK * 2;  // one BF16 operand chunk, 8 KB

// Shared-memory descriptor, K-major operand with the 64-byte swizzle (8-row x
// 64-byte atoms, 512 bytes apart along M/N): the BF16 hi/lo operands.
__device__ __forceinline__ uint64_t smem_desc_sw64_tc(const void *p) {
    uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr & 0x3FFFFull) >> 4;
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}
// MODE: TC_TF32 one pass; TC_TF32X3 three TF32 passes on hi/lo splits;
// TC_BF16X3 three BF16 passes (kind::f16) on hi/lo BF16 splits; TC_F16 one
// kind::f16 pass on FP16 operands (64 halves = 128 bytes of K per stage);
// TC_TF32X3P three TF32 passes on operands split by the panel solve; TC_TRSM
// the panel solve (TC_TF32X3 arithmetic, no destination tile buffer, so a
// deeper ring)
enum { TC_TF32 = 0, TC_TF32X3 = 1, TC_BF16X3 = 2, TC_F16 = 3, TC_TF32X3P = 4, TC_TRSM = 5 };
template <int MODE> struct TcCfg {
    static constexpr bool SPLIT = MODE == TC_TF32X3 || MODE == TC_BF16X3 || MODE == TC_TRSM;  // split warps
    static constexpr bool PRE = MODE == TC_TF32X3P;                        // lo operands landed by TMA
    // operand ring depth: as many stages as fit beside the 64 KB destination
    // tile (the loads come from L2 at ~1-2 us latency; bytes in flight set the pace)
    static constexpr int STAGES = (MODE == TC_TRSM || PRE) ? 3 : (SPLIT ? 2 : (MODE == TC_F16 ? 5 : 3));
    // A, B as landed (FP32) + the hi/lo operands: FP32 A_lo, B_lo (TF32X3) or
    // BF16 A_hi, A_lo, B_hi, B_lo (BF16X3, 8 KB each)
    static constexpr uint32_t STAGE_BYTES = (SPLIT || PRE ? 4u : 2u) * TC_HALF;
    static constexpr int THREADS = SPLIT ? 320 : 192;
    // destination tile of the update epilogue, in 32-column boxes of 16 KB:
    // the whole tile, or half of it at a time for the pre-split three-pass
    // mode (whose 64 KB stages need the room); none for the panel solve
    static constexpr uint32_t CBUF = MODE == TC_TRSM ? 0u : (uint32_t)KRR_TILE * KRR_TILE * 4 / (PRE ? 2 : 1);
    static constexpr size_t SMEM = STAGES * STAGE_BYTES + CBUF + 1024 + 256;
    static_assert(SMEM <= 232448, "tile kernel shared memory");
};

// wait with the library's deadline; on expiry set *err and return false
__device__ __forceinline__ bool mbar_wait_deadline(uint64_t *bar, uint32_t parity, int *err) {
    return mbar_wait_until(bar, parity, err, KRR_WAIT_LIMIT_NS, KRR_ERR_TIMEOUT);
}

template <int MODE>
__global__ void __launch_bounds__(TcCfg<MODE>::THREADS, 1)
tile_mma_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmapZ,
                const __grid_constant__ CUtensorMap tmapLo, const __grid_constant__ CUtensorMap tmapC,
                const __grid_constant__ CUtensorMap tmapK,
                float *__restrict__ A, __half *__restrict__ A16,
                float *__restrict__ Alo, const SolveDesc *__restrict__ solves, const int64_t *__restrict__ pre,
                int nsolve, int64_t ntasks, int mode, int K0, int W, int first, int *__restrict__ err) {
    using Cfg = TcCfg<MODE>;
    constexpr bool X3 = Cfg::SPLIT;                              // split warps
    constexpr bool X3MMA = MODE == TC_TF32X3 || MODE == TC_TF32X3P || MODE == TC_TRSM;  // three TF32 passes
    // elements of K per stage: 32 floats or 64 halves (128 bytes either way)
    constexpr int KEL = MODE == TC_F16 ? 2 * TC_CHUNK : TC_CHUNK;
    constexpr int KCH = KRR_TILE / KEL;  // chunks per K tile
    extern __shared__ unsigned char tc_dyn[];
    const uint32_t base = smem_u32(tc_dyn);
    unsigned char *buf = tc_dyn + (((base + 1023u) & ~1023u) - base);  // 1024-aligned stage ring
    // destination tile of the update epilogue: four 32-column boxes (16 KB,
    // 128-byte swizzle) as the FP32 tile map lands and stores them
    unsigned char *cbuf = buf + Cfg::STAGES * Cfg::STAGE_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(cbuf + Cfg::CBUF);
    uint64_t *empty = full + Cfg::STAGES;
    uint64_t *split = empty + Cfg::STAGES;
    uint64_t *tfull = split + Cfg::STAGES;  // accumulator b ready for the epilogue
    uint64_t *tempty = tfull + 2;           // accumulator b read back by the 4 epilogue warps
    uint64_t *cfull = tempty + 2;           // destination tile landed in cbuf
    uint32_t *tslot = reinterpret_cast<uint32_t *>(cfull + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // task geometry: the solve by binary search, then the tile of that solve
    auto task = [&](int64_t b, SolveDesc &S, TaskGeom &g) {
        const int s = find_solve(pre, nsolve, b);
        S = solves[s];
        g = decode_task(mode, b - pre[s], K0, W);
    };
    auto dst_tile = [&](const SolveDesc &S, const TaskGeom &g) {
        return A + (S.ltile0 + (int64_t)g.i * (g.i + 1) / 2 + g.j) * KRR_TILE_ELEMS;
    };

    if (threadIdx.x == 0) {
        for (int i = 0; i < Cfg::STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
            mbar_init(&split[i], 4);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(cfull, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tslot, 256);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    pdl_launch_dependents();
    pdl_wait();  // the previous launch of the factorisation has completed

    if (threadIdx.x == 0) {  // TMA producer
        int64_t q = 0;       // chunk counter across this CTA's tasks
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ntasks && ok; t += gridDim.x) {
            SolveDesc S;
            TaskGeom g;
            task(t, S, g);
            const int nch = (g.ke - g.kb) * KCH;
            for (int c = 0; c < nch; ++c, ++q) {
                const int st = (int)(q % Cfg::STAGES);
                const int64_t use = q / Cfg::STAGES;
                if (use > 0 && !mbar_wait_deadline(&empty[st], (uint32_t)((use - 1) & 1), err)) {
                    ok = false;
                    break;
                }
                unsigned char *sa = buf + st * Cfg::STAGE_BYTES;
                unsigned char *sb = sa + TC_HALF;
                const int kt = g.kb + c / KCH;
                const int x = (c % KCH) * KEL;
                // first touch of a panel tile (K0 = 0): A_i0 is K_i0 of the kernel store
                const bool kfirst = first && mode == UPD_TRSM;
                const int ya =
                    (int)(((kfirst ? S.ktile0 : S.ltile0) + (int64_t)g.i * (g.i + 1) / 2 + kt) * KRR_TILE);
                mbar_arrive_expect_tx(&full[st], (Cfg::PRE ? 4 : 2) * TC_HALF);
                tma_load_2d(sa, kfirst ? &tmapK : &tmap, x, ya, &full[st]);
                if (mode == UPD_TRSM) {
                    tma_load_2d(sb, &tmapZ, x, (int)((S.dtile0 + kt) * KRR_TILE), &full[st]);
                } else {
                    const int yb = (int)((S.ltile0 + (int64_t)g.j * (g.j + 1) / 2 + kt) * KRR_TILE);
                    tma_load_2d(sb, &tmap, x, yb, &full[st]);
                }
                if constexpr (Cfg::PRE) {  // lo parts of both operands (updates only)
                    tma_load_2d(sa + 2 * TC_HALF, &tmapLo, x,
                                (int)((S.lotile0 + (int64_t)g.i * (g.i + 1) / 2 + kt) * KRR_TILE), &full[st]);
                    tma_load_2d(sa + 3 * TC_HALF, &tmapLo, x,
                                (int)((S.lotile0 + (int64_t)g.j * (g.j + 1) / 2 + kt) * KRR_TILE), &full[st]);
                }
            }
        }
    } else if (threadIdx.x == 32) {  // MMA issuer
        int64_t q = 0;
        int lt = 0;  // local task index
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ntasks && ok; t += gridDim.x, ++lt) {
            SolveDesc S;
            TaskGeom g;
            task(t, S, g);
            const int nch = (g.ke - g.kb) * KCH;
            const int b = lt & 1;
            if (lt >= 2 && !mbar_wait_deadline(&tempty[b], (uint32_t)(((lt >> 1) - 1) & 1), err)) break;
            tc_fence_after();
            const uint32_t acc = tmem + (uint32_t)(b * KRR_TILE);
            for (int c = 0; c < nch; ++c, ++q) {
                const int st = (int)(q % Cfg::STAGES);
                const int64_t use = q / Cfg::STAGES;
                if (!mbar_wait_deadline(X3 ? &split[st] : &full[st], (uint32_t)(use & 1), err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                unsigned char *sa = buf + st * Cfg::STAGE_BYTES;
                unsigned char *sb = sa + TC_HALF;
                if constexpr (MODE == TC_BF16X3) {
                    // BF16 hi/lo operands after the two FP32 chunks: A_hi, A_lo, B_hi, B_lo
                    unsigned char *sp = sa + 2 * TC_HALF;
                    const uint64_t dah = smem_desc_sw64_tc(sp), dal = smem_desc_sw64_tc(sp + TC_BHALF);
                    const uint64_t dbh = smem_desc_sw64_tc(sp + 2 * TC_BHALF), dbl = smem_desc_sw64_tc(sp + 3 * TC_BHALF);
#pragma unroll
                    for (int kk = 0; kk < TC_CHUNK / 16; ++kk) {  // K = 16 BF16 = 32 bytes per MMA
                        const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
                        tc_mma_f16(acc, dah + 2 * kk, dbh + 2 * kk, TC_IDESC_BF16, acc0);
                        tc_mma_f16(acc, dah + 2 * kk, dbl + 2 * kk, TC_IDESC_BF16, 1u);
                        tc_mma_f16(acc, dal + 2 * kk, dbh + 2 * kk, TC_IDESC_BF16, 1u);
                    }
                } else if constexpr (MODE == TC_F16) {
                    const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sb);
#pragma unroll
                    for (int kk = 0; kk < KEL / 16; ++kk) {  // K = 16 halves = 32 bytes per MMA
                        const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
                        tc_mma_f16(acc, da + 2 * kk, db + 2 * kk, TC_IDESC_F16, acc0);
                    }
                } else {
                    const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sb);
#pragma unroll
                    for (int kk = 0; kk < TC_CHUNK / 8; ++kk) {  // K = 8 TF32 = 32 bytes per MMA
                        const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
                        tc_mma_tf32(acc, da + 2 * kk, db + 2 * kk, TC_IDESC, acc0);
                        if (X3MMA) {
                            const uint64_t dal = smem_desc_sw128(sa + 2 * TC_HALF),
                                           dbl = smem_desc_sw128(sb + 2 * TC_HALF);
                            tc_mma_tf32(acc, da + 2 * kk, dbl + 2 * kk, TC_IDESC, 1u);
                            tc_mma_tf32(acc, dal + 2 * kk, db + 2 * kk, TC_IDESC, 1u);
                        }
                    }
                }
                tc_commit(&empty[st]);
            }
            if (ok) tc_commit(&tfull[b]);
        }
    } else if (X3 && warp >= 6) {  // split landed stages into hi / lo
        const int tsp = threadIdx.x - 192;  // 0..127
        int64_t q = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ntasks && ok; t += gridDim.x) {
            SolveDesc S;
            TaskGeom g;
            task(t, S, g);
            const int nch = (g.ke - g.kb) * KCH;
            for (int c = 0; c < nch; ++c, ++q) {
                const int st = (int)(q % Cfg::STAGES);
                const int64_t use = q / Cfg::STAGES;
                if (!mbar_wait_deadline(&full[st], (uint32_t)(use & 1), err)) {
                    ok = false;
                    break;
                }
                if constexpr (MODE == TC_BF16X3) {
                    // FP32 chunk (128-byte swizzle: 16-byte unit q of row r at q ^ (r % 8))
                    // -> BF16 hi = rn(x), lo = rn(x - hi) (64-byte swizzle: 16-byte unit c of
                    // row r at c ^ ((r % 8) >> 1)); operand o = 0 (A), 1 (B)
                    unsigned char *stage = buf + st * Cfg::STAGE_BYTES;
#pragma unroll 4
                    for (int e = tsp; e < 2 * KRR_TILE * (TC_CHUNK / 4); e += 128) {
                        const int o = e / (KRR_TILE * (TC_CHUNK / 4));
                        const int r = (e / (TC_CHUNK / 4)) % KRR_TILE, q = e % (TC_CHUNK / 4);
                        const float4 v = *reinterpret_cast<const float4 *>(
                            stage + o * TC_HALF + (r >> 3) * 1024 + (r & 7) * 128 + ((q ^ (r & 7)) << 4));
                        const __nv_bfloat16 h0 = __float2bfloat16_rn(v.x), h1 = __float2bfloat16_rn(v.y);
                        const __nv_bfloat16 h2 = __float2bfloat16_rn(v.z), h3 = __float2bfloat16_rn(v.w);
                        const __nv_bfloat16 l0 = __float2bfloat16_rn(v.x - __bfloat162float(h0));
                        const __nv_bfloat16 l1 = __float2bfloat16_rn(v.y - __bfloat162float(h1));
                        const __nv_bfloat16 l2 = __float2bfloat16_rn(v.z - __bfloat162float(h2));
                        const __nv_bfloat16 l3 = __float2bfloat16_rn(v.w - __bfloat162float(h3));
                        const uint32_t off = (uint32_t)(r >> 3) * 512 + (r & 7) * 64 +
                                             ((((uint32_t)q >> 1) ^ ((r & 7) >> 1)) << 4) + (q & 1) * 8;
                        unsigned char *ph = stage + 2 * TC_HALF + (2 * o) * TC_BHALF + off;
                        unsigned char *pl = ph + TC_BHALF;
                        *reinterpret_cast<__nv_bfloat162 *>(ph) = __halves2bfloat162(h0, h1);
                        *reinterpret_cast<__nv_bfloat162 *>(ph + 4) = __halves2bfloat162(h2, h3);
                        *reinterpret_cast<__nv_bfloat162 *>(pl) = __halves2bfloat162(l0, l1);
                        *reinterpret_cast<__nv_bfloat162 *>(pl + 4) = __halves2bfloat162(l2, l3);
                    }
                } else {
                    float4 *hi = reinterpret_cast<float4 *>(buf + st * Cfg::STAGE_BYTES);
                    float4 *lo = reinterpret_cast<float4 *>(buf + st * Cfg::STAGE_BYTES + 2 * TC_HALF);
#pragma unroll 4
                    for (int e = tsp; e < (int)(2 * TC_HALF / 16); e += 128) {
                        // hi = x rounded to the nearest TF32 value (the 13 low
                        // significand bits rounded half away from zero), lo = x - hi
                        float4 v = hi[e], h, l;
                        h.x = __uint_as_float((__float_as_uint(v.x) + 0x1000u) & 0xFFFFE000u);
                        h.y = __uint_as_float((__float_as_uint(v.y) + 0x1000u) & 0xFFFFE000u);
                        h.z = __uint_as_float((__float_as_uint(v.z) + 0x1000u) & 0xFFFFE000u);
                        h.w = __uint_as_float((__float_as_uint(v.w) + 0x1000u) & 0xFFFFE000u);
                        l.x = v.x - h.x;
                        l.y = v.y - h.y;
                        l.z = v.z - h.z;
                        l.w = v.w - h.w;
                        hi[e] = h;
                        lo[e] = l;
                    }
                }
                fence_proxy_async_smem();  // generic-proxy writes -> visible to the tensor core
                __syncwarp();
                if (lane == 0) mbar_arrive(&split[st]);
            }
        }
    } else if (warp >= 2 && warp < 6) {  // epilogue
        const int quad = warp & 3;
        const int r = quad * 32 + lane;
        // updates: the destination tile comes in by TMA (issued by thread 64 as
        // soon as the previous tile's store has read cbuf), A_ij -= C is formed
        // in shared memory and the tile goes back by TMA store; the panel
        // solve (no read of the destination) stores directly
        const bool tma_c = mode != UPD_TRSM && Cfg::CBUF > 0;
        constexpr uint32_t BOX = (uint32_t)KRR_TILE * 32 * 4;       // one 32-column box, 16 KB
        constexpr int CBOX = (int)(Cfg::CBUF / BOX);               // boxes held in cbuf
        constexpr int NH = CBOX > 0 ? (KRR_TILE / 32) / CBOX : 1;  // cbuf rounds per tile
        // the destination's first touch (K0 = 0) lands the kernel-store tile
        // instead: A_ij = K_ij + lambda m [i = j] before this update
        auto c_tile_y = [&](int64_t tt) {
            SolveDesc S2;
            TaskGeom g2;
            task(tt, S2, g2);
            return (int)(((first ? S2.ktile0 : S2.ltile0) + (int64_t)g2.i * (g2.i + 1) / 2 + g2.j) * KRR_TILE);
        };
        // round h of task tt: boxes h CBOX .. h CBOX + CBOX - 1 of its destination tile
        auto c_load = [&](int64_t tt, int h) {
            const int y = c_tile_y(tt);
            mbar_arrive_expect_tx(cfull, Cfg::CBUF);
            for (int k = 0; k < CBOX; ++k)
                tma_load_2d(cbuf + k * BOX, first ? &tmapK : &tmapC, (h * CBOX + k) * 32, y, cfull);
        };
        if (tma_c) {
            if (threadIdx.x == 64 && (int64_t)blockIdx.x < ntasks) c_load(blockIdx.x, 0);
            int lt = 0;
            uint32_t nround = 0;  // cbuf rounds consumed (cfull phases)
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntasks; t += gridDim.x, ++lt) {
                SolveDesc S;
                TaskGeom g;
                task(t, S, g);
                const int b = lt & 1;
                // after a timeout the warp keeps the loop and its barriers but
                // skips the work (the error word is set; the results are not used)
                bool got = ok && mbar_wait_deadline(&tfull[b], (uint32_t)((lt >> 1) & 1), err);
                if (got) tc_fence_after();
                for (int h = 0; h < NH; ++h, ++nround) {
                    got = got && mbar_wait_deadline(cfull, nround & 1, err);
                    if (got) {
#pragma unroll 1
                        for (int k = 0; k < CBOX; ++k) {
                            const int cb = h * CBOX + k;
                            float v[32];
                            tmem_ld_32x32b_x32(
                                tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * KRR_TILE + cb * 32), v);
                            // row r of the box: 16-byte unit q at q ^ (r % 8)
                            unsigned char *row = cbuf + k * BOX + r * 128;
                            if (first && g.i == g.j && (r >> 5) == cb && g.i * KRR_TILE + r < S.m) {
                                // first touch of a diagonal tile: its real diagonal gets lambda m
                                float *dd = reinterpret_cast<float *>(row + ((((r & 31) >> 2) ^ (r & 7)) << 4)) +
                                            (r & 3);
                                *dd += (float)S.lambda_m;
                            }
#pragma unroll
                            for (int qq = 0; qq < 8; ++qq) {
                                float4 *p4 = reinterpret_cast<float4 *>(row + ((qq ^ (r & 7)) << 4));
                                float4 o = *p4;
                                o.x -= v[4 * qq + 0];
                                o.y -= v[4 * qq + 1];
                                o.z -= v[4 * qq + 2];
                                o.w -= v[4 * qq + 3];
                                *p4 = o;
                            }
                        }
                    }
                    if (h == NH - 1) {  // the accumulator has been read back
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&tempty[b]);
                    }
                    fence_proxy_async_smem();  // cbuf writes -> visible to the TMA store
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    if (threadIdx.x == 64) {
                        const int y = (int)((S.ltile0 + (int64_t)g.i * (g.i + 1) / 2 + g.j) * KRR_TILE);
                        if (got)
                            for (int k = 0; k < CBOX; ++k) tma_store_2d(&tmapC, (h * CBOX + k) * 32, y, cbuf + k * BOX);
                        bulk_commit();
                        bulk_wait_read_all();  // cbuf may be refilled
                        if (got) {
                            if (h + 1 < NH) c_load(t, h + 1);
                            else if (t + gridDim.x < ntasks) c_load(t + gridDim.x, 0);
                        }
                    }
                }
                ok = got;
            }
            if (threadIdx.x == 64) bulk_wait_all();  // the stores have completed
        } else {  // the panel solve (TC_TRSM): A_ik = C, stored directly
            int lt = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntasks; t += gridDim.x, ++lt) {
                SolveDesc S;
                TaskGeom g;
                task(t, S, g);
                float *dst = dst_tile(S, g) + (int64_t)r * KRR_TILE;
                // a class-1 solve's panel solve writes its L tile in FP16 (operand of the one-pass updates)
                const bool half_out = S.cls == 1;
                __half *dst16 = half_out ? A16 + (dst_tile(S, g) - A) + (int64_t)r * KRR_TILE : nullptr;
                // a class-3 solve's panel solve also writes lo = x - hi (hi: x with
                // the low 13 mantissa bits cleared), the second operand of TC_TF32X3P
                const bool lo_out = S.cls == 3 && Alo != nullptr;
                float *dstlo = lo_out ? Alo + (S.lotile0 + (int64_t)g.i * (g.i + 1) / 2 + g.j) * KRR_TILE_ELEMS +
                                            (int64_t)r * KRR_TILE
                                      : nullptr;
                const int b = lt & 1;
                const bool got = ok && mbar_wait_deadline(&tfull[b], (uint32_t)((lt >> 1) & 1), err);
                ok = got;
                if (got) {
                    tc_fence_after();
    #pragma unroll 1
                    for (int cb = 0; cb < KRR_TILE / 32; ++cb) {
                        float v[32];
                        tmem_ld_32x32b_x32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * KRR_TILE + cb * 32),
                                           v);
                        if (half_out) {
                            uint4 *h4 = reinterpret_cast<uint4 *>(dst16 + cb * 32);
    #pragma unroll
                            for (int qq = 0; qq < 4; ++qq) {
                                uint4 o;
                                __half2 hh;
                                hh = __floats2half2_rn(v[8 * qq + 0], v[8 * qq + 1]);
                                o.x = *reinterpret_cast<uint32_t *>(&hh);
                                hh = __floats2half2_rn(v[8 * qq + 2], v[8 * qq + 3]);
                                o.y = *reinterpret_cast<uint32_t *>(&hh);
                                hh = __floats2half2_rn(v[8 * qq + 4], v[8 * qq + 5]);
                                o.z = *reinterpret_cast<uint32_t *>(&hh);
                                hh = __floats2half2_rn(v[8 * qq + 6], v[8 * qq + 7]);
                                o.w = *reinterpret_cast<uint32_t *>(&hh);
                                h4[qq] = o;
                            }
                        } else {
                            float4 *d4 = reinterpret_cast<float4 *>(dst + cb * 32);
    #pragma unroll
                            for (int qq = 0; qq < 8; ++qq)
                                d4[qq] = make_float4(v[4 * qq], v[4 * qq + 1], v[4 * qq + 2], v[4 * qq + 3]);
                            if (lo_out) {
                                float4 *l4 = reinterpret_cast<float4 *>(dstlo + cb * 32);
    #pragma unroll
                                for (int qq = 0; qq < 8; ++qq) {
                                    float4 o;
                                    o.x = v[4 * qq + 0] - __uint_as_float(__float_as_uint(v[4 * qq + 0]) & 0xFFFFE000u);
                                    o.y = v[4 * qq + 1] - __uint_as_float(__float_as_uint(v[4 * qq + 1]) & 0xFFFFE000u);
                                    o.z = v[4 * qq + 2] - __uint_as_float(__float_as_uint(v[4 * qq + 2]) & 0xFFFFE000u);
                                    o.w = v[4 * qq + 3] - __uint_as_float(__float_as_uint(v[4 * qq + 3]) & 0xFFFFE000u);
                                    l4[qq] = o;
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[b]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 256);
}

// ---------------------------------------------------------------- host side
typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                    CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                    CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
    static const PFN_encodeTiled fn = []() -> PFN_encodeTiled {  // thread-safe one-time lookup
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_encodeTiled)p;
        return nullptr;
    }();
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

// 2-D view of an FP16 tile store: rows of 128 halves, box 64 x 128, 128B swizzle
bool make_tile_tmap16(CUtensorMap *map, __half *store, int64_t ntiles) {
    if (ntiles <= 0) ntiles = 1;
    PFN_encodeTiled enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)KRR_TILE, (cuuint64_t)(ntiles * KRR_TILE)};
    cuuint64_t strides[1] = {(cuuint64_t)KRR_TILE * sizeof(__half)};
    cuuint32_t box[2] = {(cuuint32_t)(2 * TC_CHUNK), (cuuint32_t)KRR_TILE};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, store, dims, strides, box, es,
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
    int tc;        // update arithmetic: 0 SIMT, 1 one FP16 pass, 2 BF16x3, 3 TF32x3
};

// Build the schedule for a batch of solves with tile counts T[s] and update
// classes cls[s] (0 SIMT, 1 one FP16 pass, 2 BF16x3, 3 TF32x3 pre-split,
// 4 TF32x3 split in shared memory): the diagonal factorisations and panel
// solves of all solves share their launches; each update step is one launch
// per class present.
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

// launch with programmatic stream serialisation (see pdl_wait)
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                              cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename T>
cudaError_t run_chol_plan_t(cudaStream_t st, const std::vector<CholLaunch> &plan, const int64_t *d_pre, T *A, T *Z,
                            __half *A16, float *Alo, const SolveDesc *d_solves, int nsolve, int32_t *flags, int tc,
                            const CUtensorMap *tmap, const CUtensorMap *tmapZ, const CUtensorMap *tmap16,
                            const CUtensorMap *tmapLo, const float *Kfirst, const CUtensorMap *tmapK, int *d_err,
                            Prof *prof) {
    const size_t po_sm = (size_t)KRR_TILE * 129 * sizeof(T);
    if constexpr (sizeof(T) == 4) allow_max_dyn_smem(potrf_blocked_kernel);  // FP32 factors: blocked
    else allow_max_dyn_smem(potrf_tile_kernel<T>);                           // FP64 path
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    for (const CholLaunch &L : plan) {
        const unsigned grid = (unsigned)L.tasks;
        const int64_t *p = d_pre + L.pre;
        ProfScope ps(prof, L.kind == 0 ? PROF_POTRF : (L.kind == 1 ? PROF_TRSM : PROF_UPDATE), st);
        if (L.kind == 0) {
            KRR_LAUNCHED();
            cudaError_t e;
            if constexpr (sizeof(T) == 4)
                e = launch_pdl(potrf_blocked_kernel, grid, 512, PO_BLOCKED_SMEM, st, A, Z, Kfirst, d_solves, p,
                               nsolve, L.K0, flags);
            else
                e = launch_pdl(potrf_tile_kernel<T>, grid, 512, po_sm, st, A, Z, d_solves, p, nsolve, L.K0, flags);
            if (e != cudaSuccess) return e;
            continue;
        }
        const int mode = L.kind == 1 ? UPD_TRSM : (L.kind == 2 ? UPD_TRAIL : UPD_COLUMN);
        const int W = L.kind == 1 ? 0 : L.W;
        if constexpr (sizeof(T) == 4) {
            // tensor cores: the panel solve always FP32-class (3 TF32 passes,
            // split in shared memory); updates per class: 1 one FP16 pass
            // (operands from the FP16 copy of the panel), 2 BF16x3, 3 TF32x3 on
            // operands split by the panel solve, 4 TF32x3 split in shared memory
            if (tc != 0) {
                int m = TC_TRSM;
                if (L.kind != 1) {
                    m = TC_TF32X3;
                    if (L.tc == 1) m = TC_F16;
                    else if (L.tc == 2) m = TC_BF16X3;
                    else if (L.tc == 3) m = TC_TF32X3P;
                }
                if ((m == TC_F16 && (A16 == nullptr || tmap16 == nullptr)) ||
                    (m == TC_TF32X3P && (Alo == nullptr || tmapLo == nullptr)))
                    return cudaErrorInvalidValue;  // classes 1 and 3 need their side stores
                const unsigned pgrid = (unsigned)std::min<int64_t>(L.tasks, nsm);  // persistent: one CTA per SM
                float *Af = reinterpret_cast<float *>(A);
                const CUtensorMap &tmLo = tmapLo ? *tmapLo : *tmap;
                const CUtensorMap &tmK = tmapK ? *tmapK : *tmap;
                const int first = (Kfirst != nullptr && tmapK != nullptr && L.K0 == 0) ? 1 : 0;
                auto go = [&](auto kern, unsigned threads, size_t smem, const CUtensorMap &opmap) {
                    KRR_LAUNCHED();
                    return launch_pdl(kern, pgrid, threads, smem, st, opmap, *tmapZ, tmLo, *tmap, tmK, Af, A16, Alo,
                                      d_solves, p, nsolve, L.tasks, mode, L.K0, W, first, d_err);
                };
                cudaError_t err;
                if (m == TC_TRSM)
                    err = go(tile_mma_kernel<TC_TRSM>, TcCfg<TC_TRSM>::THREADS, TcCfg<TC_TRSM>::SMEM, *tmap);
                else if (m == TC_TF32X3)
                    err = go(tile_mma_kernel<TC_TF32X3>, TcCfg<TC_TF32X3>::THREADS, TcCfg<TC_TF32X3>::SMEM, *tmap);
                else if (m == TC_TF32X3P)
                    err = go(tile_mma_kernel<TC_TF32X3P>, TcCfg<TC_TF32X3P>::THREADS, TcCfg<TC_TF32X3P>::SMEM, *tmap);
                else if (m == TC_BF16X3)
                    err = go(tile_mma_kernel<TC_BF16X3>, TcCfg<TC_BF16X3>::THREADS, TcCfg<TC_BF16X3>::SMEM, *tmap);
                else
                    err = go(tile_mma_kernel<TC_F16>, TcCfg<TC_F16>::THREADS, TcCfg<TC_F16>::SMEM, *tmap16);
                if (err != cudaSuccess) return err;
                continue;
            }
        }
        KRR_LAUNCHED(), gemm_tile_simt_kernel<T><<<grid, 256, 0, st>>>(A, Z, d_solves, p, nsolve, mode, L.K0, W);
    }
    return cudaGetLastError();
}

// tc: 0 = SIMT trailing updates, else tensor cores (classes per launch).
// A16 / tmap16: the FP16 tile store (same tile indices as A) that class-1
// solves' panel solves write and their updates read; null without class 1.
// Alo / tmapLo: the lo parts of class-3 solves' L tiles (tile index
// S.lotile0 + i(i+1)/2 + j); null without class 3.
cudaError_t run_chol_plan(cudaStream_t st, const std::vector<CholLaunch> &plan, const int64_t *d_pre, void *A, void *Z,
                          bool fp64, const SolveDesc *d_solves, int nsolve, int32_t *flags, int tc,
                          const CUtensorMap *tmap, const CUtensorMap *tmapZ, __half *A16, const CUtensorMap *tmap16,
                          float *Alo, const CUtensorMap *tmapLo, const float *Kfirst, const CUtensorMap *tmapK,
                          int *d_err, Prof *prof) {
    allow_max_dyn_smem(tile_mma_kernel<TC_F16>);
    allow_max_dyn_smem(tile_mma_kernel<TC_TF32X3>);
    allow_max_dyn_smem(tile_mma_kernel<TC_TF32X3P>);
    allow_max_dyn_smem(tile_mma_kernel<TC_TRSM>);
    allow_max_dyn_smem(tile_mma_kernel<TC_BF16X3>);
    if (fp64)
        return run_chol_plan_t<double>(st, plan, d_pre, (double *)A, (double *)Z, nullptr, nullptr, d_solves, nsolve,
                                       flags, 0, tmap, tmapZ, nullptr, nullptr, nullptr, nullptr, d_err, prof);
    return run_chol_plan_t<float>(st, plan, d_pre, (float *)A, (float *)Z, A16, Alo, d_solves, nsolve, flags, tc,
                                  tmap, tmapZ, tmap16, tmapLo, Kfirst, tmapK, d_err, prof);
}

}  // namespace krr
