// pcg.cu -- refinement of every solve of Eq. 6 to FP64-level residuals.
//
// The low-precision Cholesky factor L (FP32 storage, TF32 or FP32 trailing
// updates) preconditions a conjugate-gradient iteration on the exact system
// (K + lambda m I) alpha = y.  Vectors and scalars are FP64; the residual
// products use the double-float kernel K_hi + K_lo (~1e-13 relative), so the
// attainable accuracy is that of the kernel, not of the factor.  With the
// plain FP64 path the same loop runs with the FP64 factor and FP64 kernel.
//
//   matvec      q = (K + lambda m I) p for every lambda of a (partition, sigma)
//               group: each lower tile contributes K_ij p_j to row block i and
//               K_ij^T p_i to row block j into a private slot; a second kernel
//               sums the slots of each row block in a fixed order, so results
//               do not depend on scheduling.
//   precond     z = L^-T L^-1 r by blocked substitution, one CTA per solve:
//               off-diagonal tiles as matrix-vector products, diagonal blocks
//               through the stored inverses Z_ii (no sequential 128-step
//               solves).
//   pcg_*       per-solve dot products (fixed-order reductions), updates,
//               stopping test ||r||_inf <= tau (||A||_inf ||x||_inf + ||y||_inf).
#include <type_traits>

#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

namespace krr {

// ---------------------------------------------------------------- matvec
__device__ __forceinline__ int find_group(const GroupDesc *gd, const int64_t *gpre, int ng, int64_t b) {
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (gpre[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// df butterfly sum over the 16 lanes that share (lane >> 4); identical in all of them
__device__ __forceinline__ df df_sum16(df v) {
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
        df o;
        o.hi = __shfl_xor_sync(0xffffffffu, v.hi, off);
        o.lo = __shfl_xor_sync(0xffffffffu, v.lo, off);
        v = ((threadIdx.x & off) == 0) ? df_add(v, o) : df_add(o, v);
    }
    return v;
}

// Tile products for every lambda of a group.  256 threads: thread (ty, tx)
// owns rows ty*8 .. ty*8+7 and columns tx*8 .. tx*8+7, taken four rows at a
// time.  Row partials are reduced across the 16 lanes of a half-warp by
// shuffles, column partials across ty through shared memory, both in
// double-float and in a fixed order.  Refined path: K = K_hi + K_lo; FP64
// path: K64 with FP64 arithmetic.  grid = sum over groups of tri(T).
template <bool DF>
__global__ void __launch_bounds__(256, 2)
matvec_tiles_kernel(const float *__restrict__ Kh, const float *__restrict__ Kl, const double *__restrict__ K64,
                    const GroupDesc *__restrict__ groups, const int64_t *__restrict__ gpre, int ng,
                    const SolveDesc *__restrict__ solves, const PcgState *__restrict__ state,
                    const float2 *__restrict__ pdf, float2 *__restrict__ slots) {
    constexpr int NL = 2;  // lambdas per pass
    __shared__ float2 sp_row[NL][KRR_TILE];   // p of the column block (df)
    __shared__ float2 sp_col[NL][KRR_TILE];   // p of the row block
    __shared__ float2 scol[NL][16][KRR_TILE]; // column partials per ty
    const int gi = find_group(groups, gpre, ng, blockIdx.x);
    const GroupDesc G = groups[gi];
    bool any = false;
    for (int l = 0; l < G.nlam; ++l) any |= state[G.solve0 + l].active != 0;
    if (!any) return;
    int ti, tj;
    tri_decode((int64_t)blockIdx.x - gpre[gi], ti, tj);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t tile = G.ktile0 + (int64_t)ti * (ti + 1) / 2 + tj;
    const int T = G.T;
    for (int l0 = 0; l0 < G.nlam; l0 += NL) {
        const int nl = min(NL, G.nlam - l0);
        __syncthreads();
        for (int e = threadIdx.x; e < nl * KRR_TILE; e += 256) {
            const int l = e >> 7, c = e & 127;
            const SolveDesc S = solves[G.solve0 + l0 + l];
            sp_row[l][c] = pdf[S.vec0 + (int64_t)tj * KRR_TILE + c];
            sp_col[l][c] = pdf[S.vec0 + (int64_t)ti * KRR_TILE + c];
        }
        __syncthreads();
        constexpr int RB = 2;  // rows per step
        using Acc = typename std::conditional<DF, df_acc, double>::type;
        Acc cacc[NL][8];
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if constexpr (DF) dfa_zero(cacc[l][j]);
                else cacc[l][j] = 0.0;
            }
#pragma unroll 1
        for (int h = 0; h < 8 / RB; ++h) {  // rows ty*8 + RB*h .. + RB-1
            using KT = typename std::conditional<DF, float, double>::type;
            KT kh[RB][8], kl[RB][8];
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int64_t off = tile * KRR_TILE_ELEMS + (int64_t)(ty * 8 + RB * h + i) * KRR_TILE + tx * 8;
                if constexpr (DF) {
                    const float4 a0 = __ldcs(reinterpret_cast<const float4 *>(Kh + off));
                    const float4 a1 = __ldcs(reinterpret_cast<const float4 *>(Kh + off) + 1);
                    const float4 b0 = __ldcs(reinterpret_cast<const float4 *>(Kl + off));
                    const float4 b1 = __ldcs(reinterpret_cast<const float4 *>(Kl + off) + 1);
                    kh[i][0] = a0.x; kh[i][1] = a0.y; kh[i][2] = a0.z; kh[i][3] = a0.w;
                    kh[i][4] = a1.x; kh[i][5] = a1.y; kh[i][6] = a1.z; kh[i][7] = a1.w;
                    kl[i][0] = b0.x; kl[i][1] = b0.y; kl[i][2] = b0.z; kl[i][3] = b0.w;
                    kl[i][4] = b1.x; kl[i][5] = b1.y; kl[i][6] = b1.z; kl[i][7] = b1.w;
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        kh[i][j] = K64[off + j];
                        kl[i][j] = 0.0;
                    }
                }
            }
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                if (l >= nl) break;
                float2 *base = slots + G.scratch0 + (int64_t)(l0 + l) * T * T * KRR_TILE;
#pragma unroll
                for (int i = 0; i < RB; ++i) {
                    const int r = ty * 8 + RB * h + i;
                    df rv;
                    if constexpr (DF) {
                        df_acc a;
                        dfa_zero(a);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float2 pj = sp_row[l][tx * 8 + j];
                            dfa_fma(a, kh[i][j], kl[i][j], pj.x, pj.y);
                        }
                        rv = df_sum16(dfa_value(a));
                    } else {
                        double a = 0.0;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float2 pj = sp_row[l][tx * 8 + j];
                            a = fma(kh[i][j], (double)pj.x + (double)pj.y, a);
                        }
                        rv = df_sum16(df_from_double(a));
                    }
                    if (tx == 0) base[((int64_t)ti * T + tj) * KRR_TILE + r] = make_float2(rv.hi, rv.lo);
                    const float2 pr = sp_col[l][r];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if constexpr (DF) dfa_fma(cacc[l][j], kh[i][j], kl[i][j], pr.x, pr.y);
                        else cacc[l][j] = fma(kh[i][j], (double)pr.x + (double)pr.y, cacc[l][j]);
                    }
                }
            }
        }
        if (ti != tj) {  // column partials -> slot (tj, ti)
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                if (l >= nl) break;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    df v;
                    if constexpr (DF) v = dfa_value(cacc[l][j]);
                    else v = df_from_double(cacc[l][j]);
                    scol[l][ty][tx * 8 + j] = make_float2(v.hi, v.lo);
                }
            }
            __syncthreads();
            {
                const int l = threadIdx.x >> 7, c = threadIdx.x & 127;
                if (l < nl) {
                    df s = df_make(scol[l][0][c].x, scol[l][0][c].y);
                    for (int u = 1; u < 16; ++u) s = df_add(s, df_make(scol[l][u][c].x, scol[l][u][c].y));
                    float2 *base = slots + G.scratch0 + (int64_t)(l0 + l) * T * T * KRR_TILE;
                    base[((int64_t)tj * T + ti) * KRR_TILE + c] = make_float2(s.hi, s.lo);
                }
            }
        }
    }
}

// q_a = sum_b slot(a, b) + lambda m p_a, the slots (double-float) summed in
// double-float in the fixed order b = 0 .. T-1; grid (solves, largest T),
// 128 threads: CTA (s, a) finishes row block a of solve s
__global__ void matvec_reduce_kernel(const GroupDesc *__restrict__ groups, const SolveDesc *__restrict__ solves,
                                     const PcgState *__restrict__ state, const double *__restrict__ pv,
                                     const float2 *__restrict__ slots, double *__restrict__ q) {
    const int s = blockIdx.x, a = blockIdx.y;
    if (!state[s].active) return;
    const SolveDesc S = solves[s];
    const GroupDesc G = groups[S.grp];
    const int T = G.T;
    if (a >= T) return;
    const int l = s - (int)G.solve0;
    const int c = threadIdx.x;
    const float2 *base = slots + G.scratch0 + (int64_t)l * T * T * KRR_TILE + (int64_t)a * T * KRR_TILE + c;
    df acc = df_make(0.f, 0.f);
    for (int b = 0; b < T; ++b) {
        const float2 v = base[(int64_t)b * KRR_TILE];
        acc = df_add(acc, df_make(v.x, v.y));
    }
    const int64_t e = (int64_t)a * KRR_TILE + c;
    const double pe = pv[S.vec0 + e];
    q[S.vec0 + e] = (e < S.m) ? df_to_double(acc) + S.lambda_m * pe : pe;
}

// ---------------------------------------------------------------- preconditioner
// z = L^-T L^-1 r for active solves; off-diagonal L tiles in Lst (FP32 or
// FP64) or, for one-pass (class 1) solves, in the FP16 store L16; diagonal
// blocks through the inverses Zst.  512 threads (16 warps).  v: working vector
// in shared memory (TT type); arithmetic in TT.  Off-diagonal tiles are
// processed two at a time with every load of both tiles issued before the
// arithmetic (streaming hint, no L1 allocation): one CTA per solve must keep
// ~100 KB in flight to approach its share of HBM.
// four consecutive elements of a tile row, loaded with one 8-byte (half), one
// 16-byte (float) or two 16-byte (double) streaming loads; kept as loaded
// (Raw) until use, so a batch of FP16 loads takes half the registers
struct V4f { float a, b, c, d; };
struct V4d { double a, b, c, d; };
template <typename LT> struct Raw;
template <> struct Raw<__half> { using type = uint2; using val = V4f; };
template <> struct Raw<float> { using type = float4; using val = V4f; };
template <> struct Raw<double> { using type = V4d; using val = V4d; };
__device__ __forceinline__ uint2 ldraw(const __half *p) { return __ldcs(reinterpret_cast<const uint2 *>(p)); }
__device__ __forceinline__ float4 ldraw(const float *p) { return __ldcs(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ V4d ldraw(const double *p) {
    const double2 v0 = __ldcs(reinterpret_cast<const double2 *>(p));
    const double2 v1 = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    return V4d{v0.x, v0.y, v1.x, v1.y};
}
__device__ __forceinline__ V4f val4(uint2 u) {
    const float2 x = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
    const float2 y = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    return V4f{x.x, x.y, y.x, y.y};
}
__device__ __forceinline__ V4f val4(float4 v) { return V4f{v.x, v.y, v.z, v.w}; }
__device__ __forceinline__ V4d val4(V4d v) { return v; }

// acc[u] += sum over tiles k and this lane's columns 4 lane .. 4 lane + 3 of
// t_k[row warp + 16u] * y_k (all loads of the batch issued before any use)
template <int NT, typename TT, typename LT>
__device__ __forceinline__ void rows_acc(const LT *const *t, const TT *const *y, int warp, int lane, TT (&acc)[8]) {
    typename Raw<LT>::type l[NT][8];
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
        for (int u = 0; u < 8; ++u) l[k][u] = ldraw(t[k] + (warp + 16 * u) * KRR_TILE + 4 * lane);
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        const TT a0 = y[k][4 * lane], a1 = y[k][4 * lane + 1], a2 = y[k][4 * lane + 2], a3 = y[k][4 * lane + 3];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const typename Raw<LT>::val e = val4(l[k][u]);
            acc[u] += e.a * a0 + e.b * a1 + e.c * a2 + e.d * a3;
        }
    }
}
// part[q] += sum over tiles k and this warp's rows rr of t_k[rr][4 lane + q] * w_k[rr]
template <int NT, typename TT, typename LT>
__device__ __forceinline__ void cols_acc(const LT *const *t, const TT *const *w, int warp, int lane, TT (&part)[4]) {
    typename Raw<LT>::type l[NT][8];
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
        for (int u = 0; u < 8; ++u) l[k][u] = ldraw(t[k] + (warp + 16 * u) * KRR_TILE + 4 * lane);
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const TT wr = w[k][warp + 16 * u];
            const typename Raw<LT>::val e = val4(l[k][u]);
            part[0] += e.a * wr;
            part[1] += e.b * wr;
            part[2] += e.c * wr;
            part[3] += e.d * wr;
        }
}

// v <- L^-T L^-1 v for one solve, off-diagonal tiles of type LT from Lst
template <typename TT, typename LT>
__device__ __forceinline__ void precond_solve(const LT *__restrict__ Lst, const TT *__restrict__ Zst,
                                              const SolveDesc &S, TT *v, TT *red, TT *tmp, int warp, int lane) {
    const int T = S.T;
    constexpr int NB = sizeof(LT) == 2 ? 4 : 2;  // tiles per batch of loads (~128 KB in flight per CTA)
    // forward: y_i = Z_ii (v_i - sum_{j<i} L_ij y_j); y overwrites v
    for (int i = 0; i < T; ++i) {
        TT acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = TT(0);
        const LT *row0 = Lst + (S.ltile0 + (int64_t)i * (i + 1) / 2) * KRR_TILE_ELEMS;
        int j = 0;
        for (; j + NB - 1 < i; j += NB) {
            const LT *tt[NB];
            const TT *yy[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                tt[k] = row0 + (int64_t)(j + k) * KRR_TILE_ELEMS;
                yy[k] = v + (j + k) * KRR_TILE;
            }
            rows_acc<NB>(tt, yy, warp, lane, acc);
        }
        for (; j < i; ++j) {
            const LT *tt[1] = {row0 + (int64_t)j * KRR_TILE_ELEMS};
            const TT *yy[1] = {v + j * KRR_TILE};
            rows_acc<1>(tt, yy, warp, lane, acc);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            TT a = acc[u];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
            if (lane == 0) tmp[warp + 16 * u] = v[i * KRR_TILE + warp + 16 * u] - a;
        }
        __syncthreads();
        {
            TT zr[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) zr[u] = TT(0);
            const TT *zt[1] = {Zst + (S.dtile0 + i) * KRR_TILE_ELEMS};
            const TT *zy[1] = {tmp};
            rows_acc<1>(zt, zy, warp, lane, zr);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                TT a = zr[u];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
                if (lane == 0) v[i * KRR_TILE + warp + 16 * u] = a;
            }
        }
        __syncthreads();
    }
    // backward, left-looking: w_i = Z_ii^T (y_i - sum_{j>i} L_ji^T w_j) for
    // i = T-1 .. 0; the tiles of block column i below the diagonal are
    // streamed with per-thread partial sums and one cross-warp reduction per
    // block column; w overwrites v
    for (int i = T - 1; i >= 0; --i) {
        TT part[4] = {TT(0), TT(0), TT(0), TT(0)};
        int j = i + 1;
        for (; j + NB - 1 < T; j += NB) {
            const LT *tt[NB];
            const TT *ww[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                tt[k] = Lst + (S.ltile0 + (int64_t)(j + k) * (j + k + 1) / 2 + i) * KRR_TILE_ELEMS;
                ww[k] = v + (j + k) * KRR_TILE;
            }
            cols_acc<NB>(tt, ww, warp, lane, part);
        }
        for (; j < T; ++j) {
            const LT *tt[1] = {Lst + (S.ltile0 + (int64_t)j * (j + 1) / 2 + i) * KRR_TILE_ELEMS};
            const TT *ww[1] = {v + j * KRR_TILE};
            cols_acc<1>(tt, ww, warp, lane, part);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) red[warp * KRR_TILE + 4 * lane + q] = part[q];
        __syncthreads();
        if (threadIdx.x < KRR_TILE) {
            TT a = TT(0);
            for (int w = 0; w < 16; ++w) a += red[w * KRR_TILE + threadIdx.x];
            tmp[threadIdx.x] = v[i * KRR_TILE + threadIdx.x] - a;
        }
        __syncthreads();
        {
            TT zp[4] = {TT(0), TT(0), TT(0), TT(0)};
            const TT *zt[1] = {Zst + (S.dtile0 + i) * KRR_TILE_ELEMS};
            const TT *zw[1] = {tmp};
            cols_acc<1>(zt, zw, warp, lane, zp);
#pragma unroll
            for (int q = 0; q < 4; ++q) red[warp * KRR_TILE + 4 * lane + q] = zp[q];
        }
        __syncthreads();
        if (threadIdx.x < KRR_TILE) {
            TT a = TT(0);
            for (int w = 0; w < 16; ++w) a += red[w * KRR_TILE + threadIdx.x];
            v[i * KRR_TILE + threadIdx.x] = a;
        }
        __syncthreads();
    }
}

template <typename TT>
__global__ void __launch_bounds__(512, 1)
precond_kernel(const TT *__restrict__ Lst, const __half *__restrict__ L16, const TT *__restrict__ Zst,
               const SolveDesc *__restrict__ solves, const int32_t *__restrict__ order,
               const PcgState *__restrict__ state, const double *__restrict__ r, double *__restrict__ z) {
    extern __shared__ __align__(16) unsigned char pc_dyn[];
    const int s = order[blockIdx.x];  // largest solves first: they set the launch's length
    if (!state[s].active) return;
    const SolveDesc S = solves[s];
    const int T = S.T, M = T * KRR_TILE;
    TT *v = reinterpret_cast<TT *>(pc_dyn);            // [M]
    TT *red = v + M;                                   // [2][16][128]
    TT *tmp = red + 32 * KRR_TILE;                     // [128]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < M; e += blockDim.x) v[e] = (TT)r[S.vec0 + e];
    __syncthreads();
    if constexpr (std::is_same<TT, float>::value) {
        if (S.cls == 1 && L16 != nullptr) precond_solve<float, __half>(L16, Zst, S, v, red, tmp, warp, lane);
        else precond_solve<float, float>(Lst, Zst, S, v, red, tmp, warp, lane);
    } else {
        precond_solve<TT, TT>(Lst, Zst, S, v, red, tmp, warp, lane);
    }
    for (int e = threadIdx.x; e < M; e += blockDim.x) z[S.vec0 + e] = (e < S.m) ? (double)v[e] : 0.0;
}

// ---------------------------------------------------------------- PCG vector steps
// block reduction helpers (256 threads, fixed order)
__device__ __forceinline__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}
__device__ __forceinline__ double block_max(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// phase 0: p = 1 on real rows (for ||A||_inf = max (A 1) since A >= 0), x = 0
__global__ void pcg_prepare_kernel(const SolveDesc *__restrict__ solves, PcgState *__restrict__ state,
                                   const int32_t *__restrict__ flags, double *__restrict__ x, double *__restrict__ p,
                                   float2 *__restrict__ pdf) {
    const int s = blockIdx.x;
    const SolveDesc S = solves[s];
    const int M = S.T * KRR_TILE;
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        x[S.vec0 + e] = 0.0;
        p[S.vec0 + e] = (e < S.m) ? 1.0 : 0.0;
        pdf[S.vec0 + e] = make_float2((e < S.m) ? 1.f : 0.f, 0.f);
    }
    if (threadIdx.x == 0) {
        PcgState st;
        st.rz = 0.0; st.anorm = 0.0; st.ymax = 0.0; st.resid = 0.0;
        const bool broken = flags && flags[s] != 0;  // factorisation failed for good
        st.active = (S.m > 0 && !broken) ? 1 : 0;
        st.iters = 0;
        st.status = broken ? KRR_ERR_NOT_SPD : KRR_OK;
        st.pad = 0;
        state[s] = st;
    }
}

// phase 1: anorm = max(q), ymax, r = y
__global__ void pcg_norms_kernel(const SolveDesc *__restrict__ solves, PcgState *__restrict__ state,
                                 const double *__restrict__ y, const double *__restrict__ q, double *__restrict__ r) {
    __shared__ double sh[256];
    const int s = blockIdx.x;
    const SolveDesc S = solves[s];
    const int M = S.T * KRR_TILE;
    double an = 0.0, ym = 0.0;
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const double yv = (e < S.m) ? y[S.vec0 + e] : 0.0;
        r[S.vec0 + e] = yv;
        if (e < S.m) {
            an = fmax(an, fabs(q[S.vec0 + e]));
            ym = fmax(ym, fabs(yv));
        }
    }
    an = block_max(an, sh);
    ym = block_max(ym, sh);
    if (threadIdx.x == 0) {
        state[s].anorm = an;
        state[s].ymax = ym;
    }
}

// the direction as a double-float pair for the matvec: hi = rn(v), lo = rn(v - hi)
__device__ __forceinline__ float2 split_df(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

// phase 2 (after the first preconditioner application): p = z, rz = r.z
__global__ void pcg_start_kernel(const SolveDesc *__restrict__ solves, PcgState *__restrict__ state,
                                 const double *__restrict__ r, const double *__restrict__ z, double *__restrict__ p,
                                 float2 *__restrict__ pdf) {
    __shared__ double sh[256];
    const int s = blockIdx.x;
    if (!state[s].active) return;
    const SolveDesc S = solves[s];
    const int M = S.T * KRR_TILE;
    double acc = 0.0;
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const double zv = z[S.vec0 + e];
        p[S.vec0 + e] = zv;
        pdf[S.vec0 + e] = split_df(zv);
        acc += r[S.vec0 + e] * zv;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) state[s].rz = acc;
}

// solves whose factorisation failed for good: NOT_SPD, skipped by the iterations
__global__ void pcg_apply_flags_kernel(PcgState *__restrict__ state, const int32_t *__restrict__ flags, int n) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n && flags && flags[s] != 0) {
        state[s].active = 0;
        state[s].status = KRR_ERR_NOT_SPD;
    }
}

// step 1: a = rz / p.q ; x += a p ; r -= a q ; stopping test
__global__ void pcg_step1_kernel(const SolveDesc *__restrict__ solves, PcgState *__restrict__ state,
                                 double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                                 const double *__restrict__ q, double tau_min, double target, int maxit,
                                 unsigned int *__restrict__ nactive) {
    __shared__ double sh[256];
    const int s = blockIdx.x;
    if (!state[s].active) return;
    const SolveDesc S = solves[s];
    const int M = S.T * KRR_TILE;
    double pq = 0.0;
    for (int e = threadIdx.x; e < M; e += blockDim.x) pq += p[S.vec0 + e] * q[S.vec0 + e];
    pq = block_sum(pq, sh);
    PcgState st = state[s];
    if (!(pq > 0.0)) {  // the system matrix is not positive definite (or breakdown)
        if (threadIdx.x == 0) {
            state[s].active = 0;
            state[s].status = (st.iters == 0) ? KRR_ERR_NOT_SPD : KRR_ERR_NO_CONVERGE;
        }
        return;
    }
    const double a = st.rz / pq;
    double rmax = 0.0, xmax = 0.0;
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const double xv = x[S.vec0 + e] + a * p[S.vec0 + e];
        const double rv = r[S.vec0 + e] - a * q[S.vec0 + e];
        x[S.vec0 + e] = xv;
        r[S.vec0 + e] = rv;
        rmax = fmax(rmax, fabs(rv));
        xmax = fmax(xmax, fabs(xv));
    }
    rmax = block_max(rmax, sh);
    xmax = block_max(xmax, sh);
    if (threadIdx.x == 0) {
        const double scale = st.anorm * xmax + st.ymax;
        const double rel = scale > 0.0 ? rmax / scale : 0.0;
        // forward error <= kappa * backward error: stop once the bound meets the target
        const double kappa = S.lambda_m > 0.0 ? st.anorm / S.lambda_m : 1e300;
        const double tau = fmax(tau_min, target / kappa);
        state[s].resid = rel;
        state[s].iters = st.iters + 1;
        if (rel <= tau) {
            state[s].active = 0;
            state[s].status = KRR_OK;
        } else if (st.iters + 1 >= maxit) {
            state[s].active = 0;
            state[s].status = KRR_ERR_NO_CONVERGE;
        } else {
            atomicAdd(nactive, 1u);
        }
    }
}

// step 2: rz' = r.z ; p = z + (rz'/rz) p
__global__ void pcg_step2_kernel(const SolveDesc *__restrict__ solves, PcgState *__restrict__ state,
                                 const double *__restrict__ r, const double *__restrict__ z, double *__restrict__ p,
                                 float2 *__restrict__ pdf) {
    __shared__ double sh[256];
    const int s = blockIdx.x;
    if (!state[s].active) return;
    const SolveDesc S = solves[s];
    const int M = S.T * KRR_TILE;
    double acc = 0.0;
    for (int e = threadIdx.x; e < M; e += blockDim.x) acc += r[S.vec0 + e] * z[S.vec0 + e];
    acc = block_sum(acc, sh);
    const double beta = acc / state[s].rz;
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const double pe = z[S.vec0 + e] + beta * p[S.vec0 + e];
        p[S.vec0 + e] = pe;
        pdf[S.vec0 + e] = split_df(pe);
    }
    __syncthreads();
    if (threadIdx.x == 0) state[s].rz = acc;
}

// ---------------------------------------------------------------- host

size_t pcg_state_size() { return sizeof(PcgState); }

// q = (K + lambda m I) p for every active solve; p in FP64 (B.p) and as
// double-float pairs (B.pdf), both written by the kernel that formed p
static void launch_matvec(cudaStream_t st, const Model &M, const PcgBuffers &B, const float *Kh, const float *Kl,
                          const double *K64, bool fp64, Prof *prof) {
    if (B.gtiles == 0) return;
    ProfScope ps(prof, PROF_MATVEC, st);
    if (fp64)
        KRR_LAUNCHED(), matvec_tiles_kernel<false><<<(unsigned)B.gtiles, 256, 0, st>>>(Kh, Kl, K64, B.d_groups, B.d_gpre, B.ng,
                                                                       M.d_solves, B.state, B.pdf, B.slots);
    else
        KRR_LAUNCHED(), matvec_tiles_kernel<true><<<(unsigned)B.gtiles, 256, 0, st>>>(Kh, Kl, K64, B.d_groups, B.d_gpre, B.ng,
                                                                      M.d_solves, B.state, B.pdf, B.slots);
    const dim3 rgrid((unsigned)M.solves.size(), (unsigned)B.maxT);
    KRR_LAUNCHED(), matvec_reduce_kernel<<<rgrid, KRR_TILE, 0, st>>>(B.d_groups, M.d_solves, B.state, B.p, B.slots, B.q);
}

static cudaError_t launch_precond(cudaStream_t st, const Model &M, const PcgBuffers &B, const void *L, const void *Z,
                                  bool fp64, int maxT, Prof *prof) {
    ProfScope ps(prof, PROF_PRECOND, st);
    const size_t esz = fp64 ? 8 : 4;
    const size_t sm = esz * ((size_t)maxT * KRR_TILE + 33 * KRR_TILE);
    if (fp64) {
        allow_max_dyn_smem(precond_kernel<double>);
        KRR_LAUNCHED(), precond_kernel<double><<<(unsigned)M.solves.size(), 512, sm, st>>>(
            (const double *)L, nullptr, (const double *)Z, M.d_solves, B.order, B.state, B.r, B.z);
    } else {
        allow_max_dyn_smem(precond_kernel<float>);
        KRR_LAUNCHED(), precond_kernel<float><<<(unsigned)M.solves.size(), 512, sm, st>>>(
            (const float *)L, (const __half *)B.L16, (const float *)Z, M.d_solves, B.order, B.state, B.r, B.z);
    }
    return cudaGetLastError();
}

size_t precond_smem_bytes(bool fp64, int maxT) {
    return (fp64 ? 8 : 4) * ((size_t)maxT * KRR_TILE + 33 * KRR_TILE);
}

// q = (K + lambda m I) 1 for every solve from the row sums the kernel-tile
// build left (FP32 partials, summed in FP64 in a fixed order: tiles b <= a of
// block row a, eight 16-column partials each, then the column sums of tiles
// (b > a, a));
// grid (groups, largest T), 128 threads
__global__ void rowsum_reduce_kernel(const GroupDesc *__restrict__ groups, const SolveDesc *__restrict__ solves,
                                     const float *__restrict__ rsR, const float *__restrict__ rsC,
                                     const int64_t *__restrict__ rsoff, int64_t rstot, double *__restrict__ q) {
    const GroupDesc G = groups[blockIdx.x];
    const int a = blockIdx.y, T = G.T, c = threadIdx.x;
    if (a >= T) return;
    const int64_t g0 = (int64_t)G.isig * rstot + rsoff[G.part];
    // the FP32 pieces (all >= 0) summed as a double-float (TwoSum into s,
    // compensation in cs): within ~2^-47 of the exact row sum, without FP64
    // instructions (GB300's FP64 pipe runs at 1/64 of FP32)
    float s = 0.f, cs = 0.f;
    auto add = [&](float v) {
        float t, e;
        two_sum(s, v, t, e);
        s = t;
        cs += e;
    };
    for (int b = 0; b <= a; ++b) {
        const int64_t sl = (g0 + (int64_t)a * T + b) * 8;
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = rsR[(sl + u) * KRR_TILE + c];
#pragma unroll
        for (int u = 0; u < 8; ++u) add(v[u]);
    }
    for (int b = a + 1; b < T; ++b) add(rsC[(g0 + (int64_t)a * T + b) * KRR_TILE + c]);
    const double sum = (double)s + (double)cs;
    const int e = a * KRR_TILE + c;
    for (int l = 0; l < G.nlam; ++l) {
        const SolveDesc S = solves[G.solve0 + l];
        q[S.vec0 + e] = (e < S.m) ? sum + S.lambda_m : 0.0;
    }
}

// Phase 1 of the refinement, also used before the factorisation: x = 0 and
// ||A||_inf = max(A 1) (A >= 0 entrywise), ||y||_inf, r = y per solve.  A 1
// comes from the kernel-tile build's row sums when it left them (B.rsR), else
// from one matrix-vector product.
cudaError_t run_pcg_norms(cudaStream_t st, const Model &M, const PcgBuffers &B, const float *Kh, const float *Kl,
                          const double *K64, bool fp64, Prof *prof) {
    const unsigned ns = (unsigned)M.solves.size();
    KRR_LAUNCHED(), pcg_prepare_kernel<<<ns, 256, 0, st>>>(M.d_solves, B.state, nullptr, B.x, B.p, B.pdf);
    if (B.rsR && B.ng > 0) {
        ProfScope ps(prof, PROF_MATVEC, st);
        KRR_LAUNCHED(), rowsum_reduce_kernel<<<dim3((unsigned)B.ng, (unsigned)B.maxT), KRR_TILE, 0, st>>>(
            B.d_groups, M.d_solves, B.rsR, B.rsC, B.rsoff, B.rstot, B.q);
    } else {
        launch_matvec(st, M, B, Kh, Kl, K64, fp64, prof);
    }
    KRR_LAUNCHED(), pcg_norms_kernel<<<ns, 256, 0, st>>>(M.d_solves, B.state, B.y, B.q, B.r);
    return cudaGetLastError();
}

// Phase 2: the iterations (state from run_pcg_norms; solves whose factor
// failed for good are marked NOT_SPD and skipped).
cudaError_t run_pcg(cudaStream_t st, const Model &M, const PcgBuffers &B, const float *Kh, const float *Kl,
                    const double *K64, const void *L, const void *Z, bool fp64, int maxT, double tau, double target,
                    int maxit, const int32_t *flags, unsigned int *h_nactive, int check_every, Prof *prof) {
    const unsigned ns = (unsigned)M.solves.size();
    KRR_LAUNCHED(), pcg_apply_flags_kernel<<<(ns + 127) / 128, 128, 0, st>>>(B.state, flags, (int)ns);
    cudaError_t e = launch_precond(st, M, B, L, Z, fp64, maxT, prof);
    if (e != cudaSuccess) return e;
    KRR_LAUNCHED(), pcg_start_kernel<<<ns, 256, 0, st>>>(M.d_solves, B.state, B.r, B.z, B.p, B.pdf);
    for (int it = 0; it < maxit; ++it) {
        cudaMemsetAsync(B.nactive, 0, sizeof(unsigned int), st);
        launch_matvec(st, M, B, Kh, Kl, K64, fp64, prof);
        KRR_LAUNCHED(), pcg_step1_kernel<<<ns, 256, 0, st>>>(M.d_solves, B.state, B.x, B.r, B.p, B.q, tau, target, maxit,
                                                              B.nactive);
        e = launch_precond(st, M, B, L, Z, fp64, maxT, prof);
        if (e != cudaSuccess) return e;
        KRR_LAUNCHED(), pcg_step2_kernel<<<ns, 256, 0, st>>>(M.d_solves, B.state, B.r, B.z, B.p, B.pdf);
        if (it % check_every == check_every - 1) {
            cudaMemcpyAsync(h_nactive, B.nactive, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return e;
            if (*h_nactive == 0) break;
        }
    }
    return cudaGetLastError();
}

}  // namespace krr
