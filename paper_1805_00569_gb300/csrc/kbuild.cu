// kbuild.cu -- staging of the gathered partitions and the Gaussian kernel tile
// builder (Table 1: K_ab = exp(-||x_a - x_b||^2 / (2 sigma^2)); the kernel
// step of Alg. BKRR2; the lambda m shift of Eq. 6 in its partitioned form).
//
// Layout in HBM.  Rows of partition j occupy padded rows [prow0, prow0 + 128 T)
// (T = ceil(m / 128)); padding rows are zero.  Every matrix is stored as its
// lower tiles (i >= j) of 128 x 128 elements, tile (i, j) at tile index
// i (i + 1) / 2 + j of its matrix, row-major inside the tile.  Padding turns
// the matrix into diag(K, I), so factor, solves and products need no ragged
// edge code: the padded unknowns are exactly zero.
//
// Refined precisions (FP32 / TF32 factor): one distance pass per tile feeds
// every sigma.  Distances use the Gram form ||a||^2 + ||b||^2 - 2 a.b with the
// dot product accumulated in double-float (hi*hi products exact), the
// exponential in double-float; the result is split into K_hi + K_lo (two FP32
// stores, ~1e-13 relative) for the refinement residuals, and K_hi + lambda m I
// is written once per lambda as the matrix the low-precision Cholesky factors.
// Plain FP64: direct differences and exp in FP64, one FP64 store per sigma and
// one FP64 factor matrix per (sigma, lambda).
#include "common.cuh"
#include "internal.h"

namespace krr {

// ------------------------------------------------------------------ staging
// block (32, 8): warp w handles one padded row; lanes stride over features.
__global__ void stage_rows_kernel(const double *__restrict__ X, const double *__restrict__ y,
                                  const int64_t *__restrict__ perm, const PartDesc *__restrict__ parts, int32_t d,
                                  int32_t dp, double *__restrict__ X64, float *__restrict__ Xh,
                                  float *__restrict__ Xl, float2 *__restrict__ nrm, double *__restrict__ yg) {
    const PartDesc P = parts[blockIdx.y];
    int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
    if (r >= (int64_t)P.T * KRR_TILE) return;
    int64_t prow = P.prow0 + r;
    bool real = r < P.m;
    int64_t src = real ? perm[P.row0 + r] : 0;
    df_acc acc;
    dfa_zero(acc);
    for (int f = threadIdx.x; f < dp; f += 32) {
        double v = (real && f < d) ? X[src * d + f] : 0.0;
        if (f < d) X64[prow * d + f] = v;
        float h = __double2float_rn(v);
        float l = __double2float_rn(v - (double)h);
        Xh[prow * dp + f] = h;
        Xl[prow * dp + f] = l;
        dfa_fma(acc, h, l, h, l);
    }
    // deterministic butterfly reduction of the df partial norms
    df v = dfa_value(acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        df o;
        o.hi = __shfl_xor_sync(0xffffffffu, v.hi, off);
        o.lo = __shfl_xor_sync(0xffffffffu, v.lo, off);
        // order the operands by lane so both partners compute the same sum
        v = ((threadIdx.x & off) == 0) ? df_add(v, o) : df_add(o, v);
    }
    if (threadIdx.x == 0) {
        nrm[prow] = make_float2(v.hi, v.lo);
        yg[prow] = real ? y[src] : 0.0;
    }
}

// ------------------------------------------------------------------ tile decode
__device__ __forceinline__ int find_part(const PartDesc *parts, int np, int64_t tile) {
    int lo = 0, hi = np - 1;
    while (lo < hi) {  // last partition whose ktile0 <= tile
        int mid = (lo + hi + 1) >> 1;
        if (parts[mid].ktile0 <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct KParams {
    int nsig, nlam;
    int kind;                     // Table 1 kernel (KRR_KERNEL_*)
    int64_t ktot;                 // tiles of one sigma's store
    float inv2s2_hi[8], inv2s2_lo[8];
    double inv2s2[8];
    double lam[8];
};

constexpr int KB_THREADS = 256;
constexpr int KC = 16;  // features per staging chunk

// Refined precisions: grid = ktot tiles.  Kh/Kl: [nsig][ktot] tiles.  A: factor
// stores, tile base given per solve (solve = part * nsig * nlam + isig * nlam + ilam).
__global__ void __launch_bounds__(KB_THREADS, 1)
kbuild_df_kernel(const float *__restrict__ Xh, const float *__restrict__ Xl, const float2 *__restrict__ nrm,
                 int32_t dp, const PartDesc *__restrict__ parts, int np, const SolveDesc *__restrict__ solves,
                 KParams kp, float *__restrict__ Kh, float *__restrict__ Kl, float *__restrict__ A) {
    __shared__ __align__(16) float sAh[KC][KRR_TILE];
    __shared__ __align__(16) float sAl[KC][KRR_TILE];
    __shared__ __align__(16) float sBh[KC][KRR_TILE];
    __shared__ __align__(16) float sBl[KC][KRR_TILE];
    __shared__ float2 sExp[256];
    exp_table_init(sExp);
    const int64_t tile = blockIdx.x;
    const int pj = find_part(parts, np, tile);
    const PartDesc P = parts[pj];
    int ti, tj;
    tri_decode(tile - P.ktile0, ti, tj);
    const int64_t ra = P.prow0 + (int64_t)ti * KRR_TILE;  // first padded row of the A side
    const int64_t rb = P.prow0 + (int64_t)tj * KRR_TILE;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    df_acc acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) dfa_zero(acc[i][j]);

    for (int f0 = 0; f0 < dp; f0 += KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < KC * KRR_TILE; e += KB_THREADS) {
            int r = e / KC, f = e % KC;
            bool ok = (f0 + f) < dp;
            sAh[f][r] = ok ? Xh[(ra + r) * dp + f0 + f] : 0.f;
            sAl[f][r] = ok ? Xl[(ra + r) * dp + f0 + f] : 0.f;
            sBh[f][r] = ok ? Xh[(rb + r) * dp + f0 + f] : 0.f;
            sBl[f][r] = ok ? Xl[(rb + r) * dp + f0 + f] : 0.f;
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < KC; ++kk) {
            float ah[8], al[8], bh[8], bl[8];
            *reinterpret_cast<float4 *>(&ah[0]) = *reinterpret_cast<const float4 *>(&sAh[kk][ty * 8]);
            *reinterpret_cast<float4 *>(&ah[4]) = *reinterpret_cast<const float4 *>(&sAh[kk][ty * 8 + 4]);
            *reinterpret_cast<float4 *>(&al[0]) = *reinterpret_cast<const float4 *>(&sAl[kk][ty * 8]);
            *reinterpret_cast<float4 *>(&al[4]) = *reinterpret_cast<const float4 *>(&sAl[kk][ty * 8 + 4]);
            *reinterpret_cast<float4 *>(&bh[0]) = *reinterpret_cast<const float4 *>(&sBh[kk][tx * 8]);
            *reinterpret_cast<float4 *>(&bh[4]) = *reinterpret_cast<const float4 *>(&sBh[kk][tx * 8 + 4]);
            *reinterpret_cast<float4 *>(&bl[0]) = *reinterpret_cast<const float4 *>(&sBl[kk][tx * 8]);
            *reinterpret_cast<float4 *>(&bl[4]) = *reinterpret_cast<const float4 *>(&sBl[kk][tx * 8 + 4]);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) dfa_fma(acc[i][j], ah[i], al[i], bh[j], bl[j]);
        }
    }

    // epilogue: distances into shared memory, then every sigma and lambda with
    // one thread per element (coalesced stores, no register-array indexing)
    extern __shared__ __align__(16) unsigned char kb_dyn[];
    float2 *sD = reinterpret_cast<float2 *>(kb_dyn);  // [128][129]
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float2 v = nrm[ra + ty * 8 + i];
        const df na = df_make(v.x, v.y);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float2 w = nrm[rb + tx * 8 + j];
            df g = dfa_value(acc[i][j]);
            df t = df_add(na, df_make(w.x, w.y));
            t = df_add(t, df_make(-2.f * g.hi, -2.f * g.lo));
            if (t.hi < 0.f) t = df_make(0.f, 0.f);
            sD[(ty * 8 + i) * (KRR_TILE + 1) + tx * 8 + j] = make_float2(t.hi, t.lo);
        }
    }
    __syncthreads();
    const int G = kp.nsig * kp.nlam;
    const int64_t s0 = (int64_t)pj * G;
    const int64_t lt = (int64_t)ti * (ti + 1) / 2 + tj;  // tile inside the matrix
#pragma unroll 1
    for (int e = threadIdx.x; e < KRR_TILE_ELEMS; e += KB_THREADS) {
        const int r = e >> 7, c = e & (KRR_TILE - 1);
        const int gr = ti * KRR_TILE + r, gc = tj * KRR_TILE + c;
        const float2 dv = sD[r * (KRR_TILE + 1) + c];
        const df D = df_make(dv.x, dv.y);
#pragma unroll 1
        for (int is = 0; is < kp.nsig; ++is) {
            df k;
            if (gr >= P.m || gc >= P.m) k = df_make(gr == gc ? 1.f : 0.f, 0.f);
            else if (gr == gc) k = df_make(1.f, 0.f);
            else k = df_exp_nonpos(df_mul(D, df_make(-kp.inv2s2_hi[is], -kp.inv2s2_lo[is])), sExp);
            const int64_t kt = (int64_t)is * kp.ktot + P.ktile0 + lt;
            Kh[kt * KRR_TILE_ELEMS + e] = k.hi;
            Kl[kt * KRR_TILE_ELEMS + e] = k.lo;
#pragma unroll 1
            for (int il = 0; il < kp.nlam; ++il) {
                const SolveDesc S = solves[s0 + is * kp.nlam + il];
                A[(S.ltile0 + lt) * KRR_TILE_ELEMS + e] =
                    k.hi + ((gr == gc && gr < P.m) ? (float)S.lambda_m : 0.f);
            }
        }
    }
}

// Plain FP64: direct differences, FP64 exp.  K64: [nsig][ktot] tiles (doubles).
constexpr int KC64 = 8;
__global__ void __launch_bounds__(KB_THREADS, 1)
kbuild_fp64_kernel(const double *__restrict__ X64, int32_t d, const PartDesc *__restrict__ parts, int np,
                   const SolveDesc *__restrict__ solves, KParams kp, double *__restrict__ K64,
                   double *__restrict__ A) {
    __shared__ __align__(16) double sA[KC64][KRR_TILE];
    __shared__ __align__(16) double sB[KC64][KRR_TILE];
    const int64_t tile = blockIdx.x;
    const int pj = find_part(parts, np, tile);
    const PartDesc P = parts[pj];
    int ti, tj;
    tri_decode(tile - P.ktile0, ti, tj);
    const int64_t ra = P.prow0 + (int64_t)ti * KRR_TILE;
    const int64_t rb = P.prow0 + (int64_t)tj * KRR_TILE;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
    for (int f0 = 0; f0 < d; f0 += KC64) {
        __syncthreads();
        for (int e = threadIdx.x; e < KC64 * KRR_TILE; e += KB_THREADS) {
            int r = e / KC64, f = e % KC64;
            bool ok = (f0 + f) < d;
            sA[f][r] = ok ? X64[(ra + r) * d + f0 + f] : 0.0;
            sB[f][r] = ok ? X64[(rb + r) * d + f0 + f] : 0.0;
        }
        __syncthreads();
        for (int kk = 0; kk < KC64; ++kk) {
            double a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                a[i] = sA[kk][ty * 8 + i];
                b[i] = sB[kk][tx * 8 + i];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (kp.kind == KRR_KERNEL_LINEAR) {  // the dot product x_a . x_b
                        acc[i][j] = fma(a[i], b[j], acc[i][j]);
                    } else {  // the squared distance
                        double t = a[i] - b[j];
                        acc[i][j] = fma(t, t, acc[i][j]);
                    }
                }
        }
    }
    extern __shared__ __align__(16) unsigned char kb_dyn[];
    double *sD = reinterpret_cast<double *>(kb_dyn);  // [128][129]
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) sD[(ty * 8 + i) * (KRR_TILE + 1) + tx * 8 + j] = acc[i][j];
    __syncthreads();
    const int G = kp.nsig * kp.nlam;
    const int64_t s0 = (int64_t)pj * G;
    const int64_t lt = (int64_t)ti * (ti + 1) / 2 + tj;
#pragma unroll 1
    for (int e = threadIdx.x; e < KRR_TILE_ELEMS; e += KB_THREADS) {
        const int r = e >> 7, c = e & (KRR_TILE - 1);
        const int gr = ti * KRR_TILE + r, gc = tj * KRR_TILE + c;
        const double D = sD[r * (KRR_TILE + 1) + c];
#pragma unroll 1
        for (int is = 0; is < kp.nsig; ++is) {
            double kv;
            if (gr >= P.m || gc >= P.m) kv = (gr == gc) ? 1.0 : 0.0;  // padding: an identity block
            else if (kp.kind == KRR_KERNEL_LINEAR) kv = D;                // x_a . x_b
            else if (gr == gc) kv = 1.0;
            else kv = exp(-D * kp.inv2s2[is]);
            const int64_t kt = (int64_t)is * kp.ktot + P.ktile0 + lt;
            K64[kt * KRR_TILE_ELEMS + e] = kv;
#pragma unroll 1
            for (int il = 0; il < kp.nlam; ++il) {
                const SolveDesc S = solves[s0 + is * kp.nlam + il];
                A[(S.ltile0 + lt) * KRR_TILE_ELEMS + e] = kv + ((gr == gc && gr < P.m) ? S.lambda_m : 0.0);
            }
        }
    }
}

// ||K + lambda m I||_inf for a kernel with signed entries (linear): per
// (sigma, tile) the row sums of |K| into the first of a tile's eight
// row-partial slots (the others stay zero) and, for an off-diagonal tile, the
// column sums of |K| -- the slots the exact-Gram tile build fills for the
// Gaussian kernel.  grid (tiles of every sigma), 128 threads.
__global__ void k64_abs_rowsum_kernel(const double *__restrict__ K64, const PartDesc *__restrict__ parts, int np,
                                      int64_t ktot, float *__restrict__ rsR, float *__restrict__ rsC,
                                      const int64_t *__restrict__ rsoff, int64_t rstot) {
    const int64_t g = blockIdx.x;  // sigma * ktot + tile
    const int is = (int)(g / ktot);
    const int64_t tile = g % ktot;
    const int pj = find_part(parts, np, tile);
    const PartDesc P = parts[pj];
    int ti, tj;
    tri_decode(tile - P.ktile0, ti, tj);
    const double *Kt = K64 + g * KRR_TILE_ELEMS;
    const int c = threadIdx.x;
    double cs = 0.0, rs = 0.0;
    for (int r = 0; r < KRR_TILE; ++r) cs += fabs(Kt[r * KRR_TILE + c]);  // column c
    for (int q = 0; q < KRR_TILE; ++q) rs += fabs(Kt[c * KRR_TILE + q]);  // row c
    const int64_t g0 = (int64_t)is * rstot + rsoff[pj];
    rsR[((g0 + (int64_t)ti * P.T + tj) * 8) * KRR_TILE + c] = (float)rs;
    if (ti != tj) rsC[(g0 + (int64_t)tj * P.T + ti) * KRR_TILE + c] = (float)cs;
}

// ------------------------------------------------------------------ host
void launch_stage(cudaStream_t st, const double *X, const double *y, const int64_t *perm, const Model &M,
                  double *yg) {
    int64_t maxrows = 0;
    for (auto &p : M.parts) maxrows = std::max<int64_t>(maxrows, (int64_t)p.T * KRR_TILE);
    if (maxrows == 0) return;
    dim3 blk(32, 8), grd((unsigned)((maxrows + 7) / 8), (unsigned)M.p);
    KRR_LAUNCHED(), stage_rows_kernel<<<grd, blk, 0, st>>>(X, y, perm, M.d_parts, M.d, M.dp, M.X64, M.Xh, M.Xl, M.nrm, yg);
}

void make_kparams(const Model &M, int64_t ktot, KParams &kp) {
    kp.kind = M.kind;
    kp.nsig = M.nsig;
    kp.nlam = M.nlam;
    kp.ktot = ktot;
    for (int i = 0; i < 8; ++i) {
        double v = i < M.nsig ? 1.0 / (2.0 * M.sigmas[i] * M.sigmas[i]) : 0.0;
        kp.inv2s2[i] = v;
        float h = (float)v;
        kp.inv2s2_hi[i] = h;
        kp.inv2s2_lo[i] = (float)(v - (double)h);
        kp.lam[i] = i < M.nlam ? M.lambdas[i] : 0.0;
    }
}

void launch_kbuild_df(cudaStream_t st, const Model &M, int64_t ktot, float *Kh, float *Kl, float *A) {
    if (ktot == 0) return;
    KParams kp;
    make_kparams(M, ktot, kp);
    const size_t sm = (size_t)KRR_TILE * (KRR_TILE + 1) * sizeof(float2);
    allow_max_dyn_smem(kbuild_df_kernel);
    KRR_LAUNCHED(), kbuild_df_kernel<<<(unsigned)ktot, KB_THREADS, sm, st>>>(M.Xh, M.Xl, M.nrm, M.dp, M.d_parts, M.p, M.d_solves, kp,
                                                            Kh, Kl, A);
}

void launch_k64_abs_rowsums(cudaStream_t st, const Model &M, int64_t ktot, const double *K64, float *rsR, float *rsC,
                            const int64_t *rsoff, int64_t rstot) {
    if (ktot == 0) return;
    cudaMemsetAsync(rsR, 0, (size_t)M.nsig * rstot * 8 * KRR_TILE * sizeof(float), st);
    KRR_LAUNCHED(), k64_abs_rowsum_kernel<<<(unsigned)((int64_t)M.nsig * ktot), KRR_TILE, 0, st>>>(
        K64, M.d_parts, M.p, ktot, rsR, rsC, rsoff, rstot);
}

void launch_kbuild_fp64(cudaStream_t st, const Model &M, int64_t ktot, double *K64, double *A) {
    if (ktot == 0) return;
    KParams kp;
    make_kparams(M, ktot, kp);
    const size_t sm = (size_t)KRR_TILE * (KRR_TILE + 1) * sizeof(double);
    allow_max_dyn_smem(kbuild_fp64_kernel);
    KRR_LAUNCHED(), kbuild_fp64_kernel<<<(unsigned)ktot, KB_THREADS, sm, st>>>(M.X64, M.d, M.d_parts, M.p, M.d_solves, kp, K64, A);
}

}  // namespace krr
