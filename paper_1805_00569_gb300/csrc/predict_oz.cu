// predict_oz.cu -- fused prediction (Eq. 7) with the distance Gram on the
// tcgen05 tensor cores, exactly.
//
// Every row x (FP64, d <= 96 features) is written as x = 2^e sum_s c_s 2^(-7-8s),
// s = 0..4, with integer slices |c_s| <= 128 (exact in bf16) and a residual
// below 2^(e-40).  The dot product of two rows is then
//   x_a . x_b = 2^(e_a+e_b-14) sum_L 2^(-8L) S_L,   S_L = sum_{s+t=L} C_a,s . C_b,t
// for L = 0..4 (the 15 slice products with s + t <= 4; the dropped terms are
// below 2^(e_a+e_b) * 96 * 2^-37).  Each S_L is an integer below 2^23, so the
// bf16 MMAs accumulate it exactly in FP32: no rounding happens on the tensor
// cores at all, and the distance ||a||^2 + ||b||^2 - 2 a.b is assembled in
// double-float (~1e-11 relative to the norms, the size of the dropped slice
// products; the kernel values need ~1e-10).
//
// Kernel layout, one CTA per (partition, 128 test rows):
//   warp 0, one thread: TMA producer -- the 5 slices of the next 64 training
//     rows (B operand, N = 64) and, per slice s, the 5 slices of the test rows
//     (A operand, M = 128) through a 3-stage ring; 64-byte swizzle, K chunks
//     of 32 features;
//   warp 1, one thread: MMA issuer -- 15 x (d/16) kind::f16 MMAs per chunk into
//     five 64-column FP32 accumulators in tensor memory;
//   warps 2..17: epilogue -- tcgen05.ld of the five levels (8 columns at a
//     time), distance, every sigma's double-float exponential and every
//     lambda's alpha contraction into double-float accumulators; each warp
//     owns one TMEM lane quadrant and one 16-column quarter of the chunk, and
//     the four quarter sums of a test row are combined in a fixed order at
//     the end.  K(test, train) is never stored.
// The kernel-tile build uses the same producer / MMA / 16-warp epilogue
// layout on the two 64-column chunks of each 128 x 128 tile, persistent over
// the tiles (one CTA per SM).
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace krr {

constexpr int OZ_SLICES = 5;
constexpr int OZ_M = 128;          // test rows per CTA
constexpr int OZ_N = 64;           // training rows per chunk
constexpr int OZ_KC = 32;          // features per K chunk (64 bytes of bf16)
constexpr int OZ_MAXKC = 3;        // d <= 96
constexpr int OZ_ASTAGES = 3;
constexpr int OZ_NSP = 4, OZ_NLP = 2;  // sigmas / lambdas per pass
constexpr int OZ_EPI_WARP0 = 2;    // warps 0, 1: TMA producer, MMA issuer

constexpr uint32_t OZ_A_CHUNK = OZ_M * 64;                 // bytes of one K chunk of one A slice
constexpr uint32_t OZ_B_CHUNK = OZ_N * 64;
constexpr uint32_t OZ_A_STAGE = OZ_MAXKC * OZ_A_CHUNK;     // 24 KB
constexpr uint32_t OZ_B_BYTES = OZ_SLICES * OZ_MAXKC * OZ_B_CHUNK;  // 60 KB
constexpr uint32_t OZ_IDESC = make_idesc(1u /*BF16*/, OZ_M, OZ_N);

struct OzChunkData {  // per training column of a chunk
    float nh[OZ_N], nl[OZ_N];
    int e[OZ_N];
    // alpha of (sigma, lambda) g as double-float, two columns per entry:
    // (hi, lo) of column 2k, then of column 2k + 1 (one 16-byte load per pair)
    float4 a2[OZ_NSP * OZ_NLP][OZ_N / 2];
};

constexpr uint32_t OZ_SBOX = (uint32_t)KRR_TILE * 32 * 4;  // one 32-column box of a 128-row FP32 tile, 16 KB

struct OzSmem {  // kernel-tile build CTA
    unsigned char a[OZ_ASTAGES][OZ_A_STAGE];   // 1024-aligned stage ring
    unsigned char b[OZ_B_BYTES];
    // one chunk (128 rows x 64 columns) of K_hi and of K_lo for the TMA
    // stores: [hi / lo][32-column box], 128-byte swizzle
    unsigned char stage[2][2][OZ_SBOX];
    float2 exptab[256];
    uint64_t a_full[OZ_ASTAGES], a_empty[OZ_ASTAGES];
    uint64_t b_full, b_empty, t_full, t_empty, s_free;
    uint32_t tmem;
    float2 cs[8];  // -1/(2 sigma^2) as df
};
static_assert(sizeof(OzSmem) + 1024 <= 232448, "kernel-tile build CTA exceeds the opt-in shared memory");

struct OzParams {
    int nsig, nlam, sig0, lam0, Gtot, nl_total;
    float c_hi[OZ_NSP], c_lo[OZ_NSP];  // -1 / (2 sigma^2) as df
    int kc;                              // K chunks of 32 features
    int64_t t_rows;                      // rows per slice in the test slice array
    const float2 *cpart;                 // per-partition -1 / (2 sigma_j^2) (one sigma per partition), or null
};

// Shared-memory descriptor, K-major operand with the 64-byte swizzle
// (8-row x 64-byte atoms, 512 bytes apart along M/N).
__device__ __forceinline__ uint64_t smem_desc_sw64(const void *p) {
    uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr & 0x3FFFFull) >> 4;
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;  // 64-byte swizzle
    return d;
}
__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ bool oz_wait(uint64_t *bar, uint32_t parity, int *err) {
    return mbar_wait_until(bar, parity, err, KRR_WAIT_LIMIT_NS, KRR_ERR_TIMEOUT);
}

// Squared distance ||a||^2 + ||b||^2 - 2 a.b from the five exact slice levels
// S_L of the scaled Gram G = S0 + 2^-8 S1 + 2^-16 S2 + 2^-24 S3 + 2^-32 S4:
// S0 + 2^-8 S1 exactly by TwoSum; the three lower levels (below 2^8 in size)
// in FP32, folded into the low part (rounding ~2^-17 absolute in G, below the
// size of the dropped slice products); then (na + nb) - 2^sc G with TwoSums on
// the high parts, the low parts summed in FP32 and one Fast2Sum to normalise.
// Clamped at 0 (rounding can leave a tiny negative for coincident rows).
__device__ __forceinline__ df oz_distance(float s0, float s1, float s2, float s3, float s4, df na, float nbh,
                                          float nbl, float scale) {
    float h, l;
    two_sum(s0, s1 * 0x1p-8f, h, l);
    l = __fadd_rn(l, __fmaf_rn(s2, 0x1p-16f, __fmaf_rn(s3, 0x1p-24f, s4 * 0x1p-32f)));
    float t1, e1, t2, e2;
    two_sum(na.hi, nbh, t1, e1);
    two_sum(t1, -h * scale, t2, e2);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(na.lo, nbl)), -l * scale);
    df D;
    fast_two_sum(t2, lo, D.hi, D.lo);
    if (D.hi < 0.f) D = df_make(0.f, 0.f);
    return D;
}

// ---------------------------------------------------------------- slicing
// Row r of the output takes source row map[r] (or r); rows >= nreal are zero.
// S: [5][nout][dpz] bf16; ex: exponent per row; nrm (optional): ||x||^2 as df.
//
// The slices of a feature x are the base-256 digits of v = x 2^(7 - e) (e:
// the exponent of the row's largest magnitude, |v| < 128), each the nearest
// integer (ties to even) to what the digits before it leave:
//   c_0 = rint(v), c_1 = rint((v - c_0) 256), ...
// every step exact (but the scaling, which can underflow to a signed zero).
// They are taken here in 64-bit integers from the double's bits: F = v 2^56
// (below 2^63), truncated towards zero with a sticky flag for the bits
// shifted out (their sign is x's), so a remainder exactly half-way is
// resolved as the exact value would be -- the same digits, and the same
// signed zeros, as the FP64 steps, without FP64 instructions (GB300's FP64
// pipe runs at 1/64 of FP32).

// nearest integer to R / 2^k, ties to even; dsign: sign of the part of the
// exact value below R's last place (0 when there is none)
__device__ __forceinline__ long long oz_digit(long long R, int k, int dsign) {
    const long long q = R >> k;
    const long long rem = R - q * (1ll << k);
    const long long half = 1ll << (k - 1);
    const bool up = rem > half || (rem == half && (dsign > 0 || (dsign == 0 && (q & 1))));
    return up ? q + 1 : q;
}

// the OZ_SLICES bf16 digits of a finite x for row exponent e
__device__ __forceinline__ void oz_digits(double x, int e, uint16_t *dig) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const bool neg = (b >> 63) != 0;
    const int E = (int)((b >> 52) & 0x7FF);
    unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (E) m |= 1ull << 52;
    const int sh = max(E, 1) - 1012 - e;  // F = m 2^sh
    // the FP64 steps scale x by 2^(7 - e) first: a result at or below 2^-1075
    // in magnitude rounds to a signed zero (v = m 2^(t - 1075)), whose digits
    // are that zero and then +0
    const int t = max(E, 1) + 7 - e;
    const bool vzero = m == 0 || (t <= 0 && (-t >= 53 || m <= (1ull << -t)));
    long long F = 0;
    bool sticky = false;
    if (!vzero) {
        if (sh >= 0) {
            F = (long long)(m << sh);
        } else if (sh > -64) {
            F = (long long)(m >> -sh);
            sticky = (m & ((1ull << -sh) - 1)) != 0;
        } else {
            sticky = true;
        }
    }
    const int dsign = sticky ? (neg ? -1 : 1) : 0;
    long long R = neg ? -F : F;
#pragma unroll
    for (int s = 0; s < OZ_SLICES; ++s) {
        const int k = 56 - 8 * s;
        const long long c = oz_digit(R, k, dsign);  // |c| <= 128
        // rint of a negative value above -1/2 is -0 (and of a negative zero at the first digit)
        const bool negz = c == 0 && (R < 0 || (R == 0 && dsign < 0) || (s == 0 && neg && vzero));
        uint32_t fb = __float_as_uint(__int_as_float(0x4B400000 + (int)c) - 12582912.0f);  // (float)c, exact
        if (negz) fb |= 0x80000000u;
        dig[s] = (uint16_t)(fb >> 16);  // bf16: at most 8 significant bits, exact
        R -= c * (1ll << k);
    }
}

__global__ void oz_slice_kernel(const double *__restrict__ X, int32_t d, int32_t dpz, const int64_t *__restrict__ map,
                                int64_t nreal, int64_t nout, __nv_bfloat16 *__restrict__ S, int32_t *__restrict__ ex,
                                float2 *__restrict__ nrm) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nout) return;
    const bool real = r < nreal;
    const double *x = X + (real ? (map ? map[r] : r) : 0) * d;
    unsigned long long mxb = 0;  // largest magnitude's bits
    bool finite = true;
    df_acc a;
    dfa_zero(a);
    if (real)
        for (int f = 0; f < d; ++f) {
            const double v = x[f];
            const unsigned long long ab = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
            finite = finite && ab < 0x7FF0000000000000ull;
            mxb = ab > mxb ? ab : mxb;
            const float h = __double2float_rn(v), l = __double2float_rn(v - (double)h);
            dfa_fma(a, h, l, h, l);
        }
    if (nrm) {
        const df v = dfa_value(a);
        nrm[r] = make_float2(v.hi, v.lo);
    }
    int e = 0;
    if (!finite) {  // the FP64 steps (a row with an infinite or NaN feature)
        double mx = 0.0;
        for (int f = 0; f < d; ++f) mx = fmax(mx, fabs(x[f]));
        if (mx > 0.0) frexp(mx, &e);
        ex[r] = e;
        for (int f = 0; f < dpz; ++f) {
            double v = f < d ? ldexp(x[f], 7 - e) : 0.0;
#pragma unroll
            for (int s = 0; s < OZ_SLICES; ++s) {
                const double c = rint(v);
                S[((int64_t)s * nout + r) * dpz + f] = __float2bfloat16_rn((float)c);
                v = (v - c) * 256.0;
            }
        }
        return;
    }
    if (mxb) {  // frexp's exponent of the largest magnitude: mx = f 2^e, f in [0.5, 1)
        const int E = (int)(mxb >> 52);
        const unsigned long long m = (mxb & 0xFFFFFFFFFFFFFull) | (E ? 1ull << 52 : 0ull);
        e = (64 - __clzll((long long)m)) + max(E, 1) - 1075;
    }
    ex[r] = e;
    // eight features at a time: one 16-byte store per slice (dpz is a multiple of 32)
    for (int f0 = 0; f0 < dpz; f0 += 8) {
        uint32_t pk[OZ_SLICES][4] = {};
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int f = f0 + u;
            uint16_t dg[OZ_SLICES];
            oz_digits((real && f < d) ? x[f] : 0.0, e, dg);
#pragma unroll
            for (int s = 0; s < OZ_SLICES; ++s) pk[s][u >> 1] |= (uint32_t)dg[s] << (16 * (u & 1));
        }
#pragma unroll
        for (int s = 0; s < OZ_SLICES; ++s)
            *reinterpret_cast<uint4 *>(S + ((int64_t)s * nout + r) * dpz + f0) =
                make_uint4(pk[s][0], pk[s][1], pk[s][2], pk[s][3]);
    }
}

// ---------------------------------------------------------------- predict
// Prediction CTA: 18 warps -- TMA producer, MMA issuer and 16 epilogue warps
// (4 TMEM lane quadrants x 4 column quarters of a 64-column chunk; the
// quarters' partial sums meet at the end in the fixed order
// (q0 + q1) + (q2 + q3)).
constexpr int OZP_EPI_WARPS = 16;
constexpr int OZP_EPI = OZP_EPI_WARPS * 32;                // epilogue threads
constexpr int OZP_THREADS = (OZ_EPI_WARP0 + OZP_EPI_WARPS) * 32;
constexpr int OZP_SUB = 8;                                 // columns per TMEM read
constexpr int OZP_COLS = 2;                                // columns whose exponentials interleave (4 measured no faster)
struct OzPSmem {
    unsigned char a[OZ_ASTAGES][OZ_A_STAGE];   // 1024-aligned stage ring
    unsigned char b[OZ_B_BYTES];
    OzChunkData cd[2];
    float2 exptab[256];
    float2 comb[2][OZ_NSP * OZ_NLP][OZ_M];       // quarter partial sums on their way to quarter 0
    int combk[2][OZ_NSP][OZ_M];                  // and their range shifts
    float2 shift[OZ_NSP][OZP_EPI];               // per epilogue thread: -K ln2 per sigma (df)
    float2 dist[OZP_EPI][OZP_SUB + 1];           // per epilogue thread: 8 distances (padded row)
    float qmin[2][4][OZ_M];                      // per chunk parity and column quarter: each row's D_min so far
    uint64_t a_full[OZ_ASTAGES], a_empty[OZ_ASTAGES];
    uint64_t b_full, b_empty, t_full, t_empty;
    uint32_t tmem;
};
static_assert(sizeof(OzPSmem) + 1024 <= 232448, "prediction CTA exceeds the opt-in shared memory");
__device__ __forceinline__ void epi_bar_p() { asm volatile("bar.sync 1, %0;" ::"n"(OZP_EPI) : "memory"); }
__device__ __forceinline__ void tmem_ld_32x32b_x8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
// Far terms of a prediction row.  A term whose exponent argument lies more
// than OZ_FAR below that of a training row already seen, x - x_max = (D -
// D_min) c < -OZ_FAR, is below e^-20 (2e-9) of the row's largest term (a
// nearer training row only makes it smaller).  D_min is the smallest distance
// this thread has seen, or that the row's other three column quarters had
// published by the end of the previous chunk (exchanged through shared
// memory across the chunk barrier, double-buffered, so every decision is the
// same in every run).  Such a term is formed in FP32: x + shift by
// one FMA on the high parts and ex2.approx (argument error below
// 2^-22 (|x| + |shift| + 1), so relative error below 2e-4 while |x| and the
// shift stay under 800; results below 2^-126 flush to 0, as the double-float
// exponential drops arguments below -87), and its product with alpha_hi is
// added to the accumulator's low part.  Per term that is an error below 4e-13
// of the largest term times |alpha|, under the double-float path's own
// rounding of the sum.  The test is per row (lane); a lane's other columns
// are queued and the warp runs them through the double-float path one per
// lane per round.
constexpr float OZ_FAR = 20.0f;
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// a (shift ka) + b (shift kb) at the larger shift; *k receives it
__device__ __forceinline__ df oz_combine(df a, int ka, df b, int kb, int *k) {
    const int km = max(ka, kb);
    if (ka != km) a = df_scale2(a, pow2_nonpos(ka - km));
    if (kb != km) b = df_scale2(b, pow2_nonpos(kb - km));
    *k = km;
    return df_add(a, b);
}

__global__ void __launch_bounds__(OZP_THREADS, 1)
predict_oz_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const PartDesc *__restrict__ parts, const SolveDesc *__restrict__ solves,
                  const float2 *__restrict__ alpha2, const int32_t *__restrict__ ex_train,
                  const float2 *__restrict__ nrm_train, const int32_t *__restrict__ ex_test,
                  const float2 *__restrict__ nrm_test, int64_t t, const int64_t *__restrict__ toff,
                  const int64_t *__restrict__ tidx, OzParams pp, int routed, int64_t prows,
                  double *__restrict__ out, int *__restrict__ err) {
    extern __shared__ unsigned char oz_dyn[];
    const uint32_t base = smem_u32(oz_dyn);
    OzPSmem &sm = *reinterpret_cast<OzPSmem *>(oz_dyn + (((base + 1023u) & ~1023u) - base));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.y;
    const PartDesc P = parts[j];
    const int64_t cnt = toff ? toff[j + 1] - toff[j] : t;
    const int64_t tstart = toff ? toff[j] : 0;
    const int64_t q0 = (int64_t)blockIdx.x * OZ_M;
    if (q0 >= cnt) return;
    const int nchunks = P.T * (KRR_TILE / OZ_N);
    const int G = pp.nsig * pp.nlam;

    if (threadIdx.x == 0) {
        for (int i = 0; i < OZ_ASTAGES; ++i) {
            mbar_init(&sm.a_full[i], 1);
            mbar_init(&sm.a_empty[i], 1);
        }
        mbar_init(&sm.b_full, 1);
        mbar_init(&sm.b_empty, 1);
        mbar_init(&sm.t_full, 1);
        mbar_init(&sm.t_empty, OZP_EPI_WARPS);
        fence_mbar_init();
    }
    exp_table_init(sm.exptab);
    if (warp == 0) {
        tmem_alloc(&sm.tmem, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;

    if (nchunks > 0 && threadIdx.x == 0) {
        // ---------------- TMA producer
        const uint32_t bbytes = (uint32_t)(OZ_SLICES * pp.kc) * OZ_B_CHUNK;
        const uint32_t abytes = (uint32_t)pp.kc * OZ_A_CHUNK;
        int ait = 0;
        for (int c = 0; c < nchunks; ++c) {
            if (c > 0 && !oz_wait(&sm.b_empty, (c - 1) & 1, err)) break;
            mbar_arrive_expect_tx(&sm.b_full, bbytes);
            const int brow = (int)(P.prow0 + (int64_t)c * OZ_N);
            for (int s = 0; s < OZ_SLICES; ++s)
                for (int kc = 0; kc < pp.kc; ++kc)
                    tma_load_2d(sm.b + (s * OZ_MAXKC + kc) * OZ_B_CHUNK, &tmB, kc * OZ_KC, (int)(s * prows) + brow,
                                &sm.b_full);
            bool ok = true;
            for (int s = 0; s < OZ_SLICES; ++s, ++ait) {
                const int st = ait % OZ_ASTAGES, use = ait / OZ_ASTAGES;
                if (use > 0 && !oz_wait(&sm.a_empty[st], (use - 1) & 1, err)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&sm.a_full[st], abytes);
                const int arow = (int)(s * pp.t_rows + tstart + q0);
                for (int kc = 0; kc < pp.kc; ++kc)
                    tma_load_2d(sm.a[st] + kc * OZ_A_CHUNK, &tmA, kc * OZ_KC, arow, &sm.a_full[st]);
            }
            if (!ok) break;
        }
    } else if (nchunks > 0 && threadIdx.x == 32) {
        // ---------------- MMA issuer
        int ait = 0;
        bool ok = true;
        for (int c = 0; c < nchunks && ok; ++c) {
            if (c > 0 && !oz_wait(&sm.t_empty, (c - 1) & 1, err)) break;
            if (!oz_wait(&sm.b_full, c & 1, err)) break;
            tc_fence_after();
            for (int s = 0; s < OZ_SLICES; ++s, ++ait) {
                const int st = ait % OZ_ASTAGES, use = ait / OZ_ASTAGES;
                if (!oz_wait(&sm.a_full[st], use & 1, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int tt = 0; tt + s < OZ_SLICES; ++tt) {
                    const uint32_t dcol = tmem + (uint32_t)((s + tt) * OZ_N);
                    for (int kk = 0; kk < 2 * pp.kc; ++kk) {
                        const uint64_t da = smem_desc_sw64(sm.a[st] + (kk >> 1) * OZ_A_CHUNK) + 2 * (kk & 1);
                        const uint64_t db =
                            smem_desc_sw64(sm.b + (tt * OZ_MAXKC + (kk >> 1)) * OZ_B_CHUNK) + 2 * (kk & 1);
                        tc_mma_f16(dcol, da, db, OZ_IDESC, (s > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                tc_commit(&sm.a_empty[st]);
            }
            tc_commit(&sm.b_empty);
            tc_commit(&sm.t_full);
        }
    } else if (warp >= OZ_EPI_WARP0) {
        // ---------------- epilogue
        const int ew = warp - OZ_EPI_WARP0;       // 0..15
        const int quad = warp & 3;                // TMEM lane quadrant of this warp
        const int quarter = ew >> 2;              // column quarter of the chunk
        const int row = quad * 32 + lane;         // test row inside the tile
        const int64_t grow = tstart + q0 + row;   // row in the (grouped) test slice array
        const bool live = q0 + row < cnt;
        const int eq = live ? ex_test[grow] : 0;
        const float2 nq2 = live ? nrm_test[grow] : make_float2(0.f, 0.f);
        const df nq = df_make(nq2.x, nq2.y);
        df_acc acc[OZ_NSP][OZ_NLP];
        int ksh[OZ_NSP];       // range shift of the accumulators per sigma (exp_row_shift)
        float shh[OZ_NSP];     // high part of the shift argument -K ln2 (far terms)
        float dmin = INFINITY;  // smallest distance to a real training row so far
        const int et = threadIdx.x - OZ_EPI_WARP0 * 32;  // 0..511
        // -1 / (2 sigma^2) per sigma slot: the launch's grid, or the partition's own sigma
        float chi[OZ_NSP], clo[OZ_NSP];
#pragma unroll
        for (int a = 0; a < OZ_NSP; ++a) {
            chi[a] = pp.c_hi[a];
            clo[a] = pp.c_lo[a];
        }
        if (pp.cpart) {
            const float2 cj = pp.cpart[j];
            chi[0] = cj.x;
            clo[0] = cj.y;
        }
#pragma unroll
        for (int a = 0; a < OZ_NSP; ++a) {
            ksh[a] = KRR_SHIFT_NONE;  // no term yet: the shift argument stays 0
            shh[a] = 0.f;
            sm.shift[a][et] = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < OZ_NLP; ++b) dfa_zero(acc[a][b]);
        }
        sm.qmin[0][quarter][row] = INFINITY;
        sm.qmin[1][quarter][row] = INFINITY;
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            OzChunkData &cd = sm.cd[c & 1];
            // training-side data of the chunk
            for (int e = et; e < OZ_N; e += OZP_EPI) {
                const int64_t pr = P.prow0 + (int64_t)c * OZ_N + e;
                const float2 v = nrm_train[pr];
                cd.nh[e] = v.x;
                cd.nl[e] = v.y;
                cd.e[e] = ex_train[pr];
            }
            for (int e = et; e < G * OZ_N; e += OZP_EPI) {
                const int g = e / OZ_N, col = e % OZ_N;
                const int is = g / pp.nlam, il = g % pp.nlam;
                const SolveDesc S =
                    solves[(int64_t)j * pp.Gtot + (int64_t)(pp.sig0 + is) * pp.nl_total + pp.lam0 + il];
                reinterpret_cast<float2 *>(&cd.a2[is * OZ_NLP + il][col >> 1])[col & 1] =
                    alpha2[S.vec0 + (int64_t)c * OZ_N + col];
            }
            epi_bar_p();
            // after a timeout the warp keeps the loop (and its barriers) but skips the work,
            // so no epilogue warp can be left waiting at a barrier for one that returned
            if (!ok || !oz_wait(&sm.t_full, c & 1, err)) {
                ok = false;
                continue;
            }
            tc_fence_after();
            // the row's nearest distance over all quarters as published after the previous chunk
            float dpub = INFINITY;
            if (c > 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) dpub = fminf(dpub, sm.qmin[(c - 1) & 1][q][row]);
            }
#pragma unroll 1
            for (int sub = 0; sub < (OZ_N / 4) / OZP_SUB; ++sub) {
                float lv[OZ_SLICES][OZP_SUB];
                const uint32_t col0 = (uint32_t)(quarter * (OZ_N / 4) + sub * OZP_SUB);
#pragma unroll
                for (int L = 0; L < OZ_SLICES; ++L)
                    tmem_ld_32x32b_x8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(L * OZ_N) + col0, lv[L]);
                tmem_wait_ld();
                if (sub == (OZ_N / 4) / OZP_SUB - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.t_empty);
                }
                // distances of the columns (static register indices), parked in shared memory
                float dm = INFINITY, dM = 0.f;
#pragma unroll
                for (int k = 0; k < OZP_SUB; ++k) {
                    const int col = (int)col0 + k;
                    const int sc = eq + cd.e[col] - 13;  // factor 2 of -2 a.b folded in
                    const df D = oz_distance(lv[0][k], lv[1][k], lv[2][k], lv[3][k], lv[4][k], nq, cd.nh[col],
                                             cd.nl[col], __int_as_float((127 + sc) << 23));
                    sm.dist[et][k] = make_float2(D.hi, D.lo);
                    if (c * OZ_N + col < P.m) dm = fminf(dm, D.hi);
                    dM = fmaxf(dM, D.hi);
                }
                // a closer training row raises the range shift: rescale by 2^(K_old - K_new)
                if (dm < dmin) {
                    dmin = dm;
#pragma unroll
                    for (int is = 0; is < OZ_NSP; ++is) {
                        const int kn = is < pp.nsig ? exp_row_shift(dmin * chi[is]) : 0;
                        if (is < pp.nsig && kn != ksh[is]) {
                            const float f = pow2_nonpos(ksh[is] - kn);
#pragma unroll
                            for (int il = 0; il < OZ_NLP; ++il) {
                                acc[is][il].s *= f;
                                acc[is][il].c *= f;
                            }
                            ksh[is] = kn;
                            const float2 sa = exp_shift_arg(kn);
                            sm.shift[is][et] = sa;
                            shh[is] = sa.x;
                        }
                    }
                }
                // a sigma's range shift is applied warp-wide when any row of the
                // warp has one: adding the zero shift of the other rows is exact
                // (x + 0 = x in double-float), so every row's value is what it
                // would be alone and the warp does not diverge
                unsigned wsh = 0;
#pragma unroll
                for (int is = 0; is < OZ_NSP; ++is)
                    wsh |= __any_sync(0xffffffffu, ksh[is] != 0) ? (1u << is) : 0u;
                // sigmas for which some lane has a far column in this group
                const float dfar = fminf(dmin, dpub);
                unsigned wfar = 0;
#pragma unroll
                for (int is = 0; is < OZ_NSP; ++is)
                    wfar |= __any_sync(0xffffffffu, is < pp.nsig && (dM - dfar) * chi[is] < -OZ_FAR) ? (1u << is)
                                                                                                       : 0u;
                // the other sigmas: OZP_COLS columns per iteration through the
                // double-float path (their exponentials are independent chains
                // the scheduler can interleave).  Padded training rows have
                // alpha = 0 exactly, so they need no test.
#pragma unroll 1
                for (int k = 0; k < OZP_SUB; k += OZP_COLS) {
                    const int col = (int)col0 + k;
                    df D[OZP_COLS];
#pragma unroll
                    for (int u = 0; u < OZP_COLS; ++u) {
                        const float2 dv = sm.dist[et][k + u];
                        D[u] = df_make(dv.x, dv.y);
                    }
#pragma unroll
                    for (int is = 0; is < OZ_NSP; ++is) {
                        if (is < pp.nsig && !((wfar >> is) & 1u)) {
                            const df cs = df_make(chi[is], clo[is]);
                            df kv[OZP_COLS];
#pragma unroll
                            for (int u = 0; u < OZP_COLS; ++u) {
                                df x = df_mul(D[u], cs);
                                if (wsh & (1u << is)) {
                                    const float2 sv = sm.shift[is][et];  // (0, 0) for an unshifted row
                                    x = df_add(x, df_make(sv.x, sv.y));
                                }
                                kv[u] = df_exp_nonpos<false>(x, sm.exptab);
                            }
#pragma unroll
                            for (int il = 0; il < OZ_NLP; ++il)
                                if (il < pp.nlam) {
#pragma unroll
                                    for (int u = 0; u < OZP_COLS; u += 2) {
                                        const float4 a = cd.a2[is * OZ_NLP + il][(col + u) >> 1];  // col is even
                                        dfa_fma(acc[is][il], kv[u].hi, kv[u].lo, a.x, a.y);
                                        dfa_fma(acc[is][il], kv[u + 1].hi, kv[u + 1].lo, a.z, a.w);
                                    }
                                }
                        }
                    }
                }
                // sigmas with far columns: each lane takes its own far columns
                // in FP32 and queues the others, which the warp then runs
                // through the double-float path one per lane per round, so
                // the rounds are the longest queue, not the columns any lane needs
#pragma unroll
                for (int is = 0; is < OZ_NSP; ++is) {
                    if (!((wfar >> is) & 1u)) continue;
                    unsigned nf = 0;  // this lane's columns that are not far
#pragma unroll
                    for (int k = 0; k < OZP_SUB; ++k) {
                        const float dh = sm.dist[et][k].x;
                        const bool far = (dh - dfar) * chi[is] < -OZ_FAR;  // false while D_min = inf
                        if (far) {
                            const float kf = ex2_approx(__fmaf_rn(dh, chi[is], shh[is]) * 1.44269504088896341f);
                            const int col = (int)col0 + k;
#pragma unroll
                            for (int il = 0; il < OZ_NLP; ++il)
                                if (il < pp.nlam) {
                                    const float4 a = cd.a2[is * OZ_NLP + il][col >> 1];
                                    acc[is][il].c = __fmaf_rn(kf, (k & 1) ? a.z : a.x, acc[is][il].c);
                                }
                        } else {
                            nf |= 1u << k;
                        }
                    }
                    const df cs = df_make(chi[is], clo[is]);
                    const float2 sv = sm.shift[is][et];  // (0, 0) for an unshifted row
                    while (__any_sync(0xffffffffu, nf != 0)) {
                        if (nf != 0) {
                            const int k = __ffs(nf) - 1;
                            nf &= nf - 1;
                            const float2 dv = sm.dist[et][k];
                            df x = df_mul(df_make(dv.x, dv.y), cs);
                            if (wsh & (1u << is)) x = df_add(x, df_make(sv.x, sv.y));
                            const df kv = df_exp_nonpos<false>(x, sm.exptab);
                            const int col = (int)col0 + k;
#pragma unroll
                            for (int il = 0; il < OZ_NLP; ++il)
                                if (il < pp.nlam) {
                                    const float4 a = cd.a2[is * OZ_NLP + il][col >> 1];
                                    if (k & 1) dfa_fma(acc[is][il], kv.hi, kv.lo, a.z, a.w);
                                    else dfa_fma(acc[is][il], kv.hi, kv.lo, a.x, a.y);
                                }
                        }
                    }
                }
            }
            sm.qmin[c & 1][quarter][row] = dmin;  // read by the row's other quarters after the next barrier
        }
        // combine the four column quarters of a row in a fixed order:
        // (q0 + q1) + (q2 + q3)
        df v[OZ_NSP][OZ_NLP];
        int kv[OZ_NSP];
#pragma unroll
        for (int is = 0; is < OZ_NSP; ++is) {
            kv[is] = ksh[is];
#pragma unroll
            for (int il = 0; il < OZ_NLP; ++il) v[is][il] = dfa_value(acc[is][il]);
        }
        epi_bar_p();
        if (quarter & 1) {  // quarters 1 and 3 hand their sums to 0 and 2
#pragma unroll
            for (int is = 0; is < OZ_NSP; ++is) {
                sm.combk[quarter >> 1][is][row] = kv[is];
#pragma unroll
                for (int il = 0; il < OZ_NLP; ++il)
                    sm.comb[quarter >> 1][is * OZ_NLP + il][row] = make_float2(v[is][il].hi, v[is][il].lo);
            }
        }
        epi_bar_p();
        if (!(quarter & 1)) {
#pragma unroll
            for (int is = 0; is < OZ_NSP; ++is) {
                const int kb = sm.combk[quarter >> 1][is][row];
                int km = kv[is];
#pragma unroll
                for (int il = 0; il < OZ_NLP; ++il) {
                    const float2 o = sm.comb[quarter >> 1][is * OZ_NLP + il][row];
                    v[is][il] = oz_combine(v[is][il], kv[is], df_make(o.x, o.y), kb, &km);
                }
                kv[is] = km;
            }
        }
        epi_bar_p();
        if (quarter == 2) {  // (q2 + q3) to quarter 0
#pragma unroll
            for (int is = 0; is < OZ_NSP; ++is) {
                sm.combk[0][is][row] = kv[is];
#pragma unroll
                for (int il = 0; il < OZ_NLP; ++il)
                    sm.comb[0][is * OZ_NLP + il][row] = make_float2(v[is][il].hi, v[is][il].lo);
            }
        }
        epi_bar_p();
        if (quarter == 0 && live) {
            const int64_t orow_t = toff ? (tidx ? tidx[grow] : grow) : (q0 + row);
#pragma unroll
            for (int is = 0; is < OZ_NSP; ++is)
#pragma unroll
                for (int il = 0; il < OZ_NLP; ++il) {
                    if (is < pp.nsig && il < pp.nlam) {
                        const float2 o = sm.comb[0][is * OZ_NLP + il][row];
                        int km;
                        const df r = oz_combine(v[is][il], kv[is], df_make(o.x, o.y), sm.combk[0][is][row], &km);
                        const int gm = (pp.sig0 + is) * pp.nl_total + pp.lam0 + il;
                        const int64_t orow = routed ? (int64_t)gm : (int64_t)j * pp.Gtot + gm;
                        out[orow * t + orow_t] = km == 0 ? df_to_double(r) : ldexp(df_to_double(r), km);
                    }
                }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------- kernel tiles
// Gaussian kernel tiles of the training partitions from the same exact slice
// Gram: persistent CTAs (one per SM) walk the lower tiles (i, j) of every
// partition; a tile's 128 x 128 Gram is formed as two 64-column chunks
// (A = rows of block i, B = rows of block j).  The epilogue writes, per sigma, K_hi + K_lo (df split) and, per
// lambda, K_hi + lambda m I into the factor store.  Diagonal entries are
// exactly 1; padding rows and columns form an identity block.
struct OzKParams {
    int nsig, nlam, np;
    float c_hi[8], c_lo[8];
    int kc;
    int64_t ktot;
    // row sums of K (for ||K + lambda m I||_inf): per (sigma, partition) a
    // T x T grid of tile slots; R holds tile (a, b <= a)'s row sums as eight
    // 16-column partials (2 chunks x 4 column quarters) of 128 floats, C
    // holds tile (b > a, a)'s column sums (128 floats) (null: skipped)
    float *rsR, *rsC;
    const int64_t *rsoff;  // per partition: first slot of its grid (sigma 0)
    int64_t rstot;         // slots per sigma (sum of T^2)
    int store_factor;      // also store K_hi + lambda m I per lambda (0: the factorisation reads K_hi itself)
    const float2 *cpart;   // per-partition -1 / (2 sigma_j^2) (one sigma per partition), or null
};

__device__ __forceinline__ int oz_find_part(const PartDesc *parts, int np, int64_t tile) {
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (parts[mid].ktile0 <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// the tile of one persistent iteration: partition, block row / column
struct OzTile {
    int pj, ti, tj;
    int64_t lt;  // tile index inside the partition
    PartDesc P;
};
__device__ __forceinline__ OzTile oz_tile_of(const PartDesc *__restrict__ parts, int np, int64_t tile) {
    OzTile t;
    t.pj = oz_find_part(parts, np, tile);
    t.P = parts[t.pj];
    t.lt = tile - t.P.ktile0;
    tri_decode(t.lt, t.ti, t.tj);
    return t;
}

__global__ void __launch_bounds__(OZP_THREADS, 1)
kbuild_oz_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ CUtensorMap tmKh, const __grid_constant__ CUtensorMap tmKl,
                 const __grid_constant__ CUtensorMap tmF, const PartDesc *__restrict__ parts,
                 const SolveDesc *__restrict__ solves,
                 const int32_t *__restrict__ ex, const float2 *__restrict__ nrm, OzKParams kp, int64_t prows,
                 float *__restrict__ Kh, float *__restrict__ Kl, float *__restrict__ A, int *__restrict__ err) {
    extern __shared__ unsigned char oz_dyn[];
    const uint32_t base = smem_u32(oz_dyn);
    OzSmem &sm = *reinterpret_cast<OzSmem *>(oz_dyn + (((base + 1023u) & ~1023u) - base));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int nchunks = KRR_TILE / OZ_N;  // 2 per tile
    if (threadIdx.x == 0) {  // static indices: the parameter block stays in the constant bank
#pragma unroll
        for (int i = 0; i < 8; ++i) sm.cs[i] = make_float2(kp.c_hi[i], kp.c_lo[i]);
    }

    if (threadIdx.x == 0) {
        for (int i = 0; i < OZ_ASTAGES; ++i) {
            mbar_init(&sm.a_full[i], 1);
            mbar_init(&sm.a_empty[i], 1);
        }
        mbar_init(&sm.b_full, 1);
        mbar_init(&sm.b_empty, 1);
        mbar_init(&sm.t_full, 1);
        mbar_init(&sm.t_empty, OZP_EPI_WARPS);
        mbar_init(&sm.s_free, 1 + (kp.rsR ? 2 : 0));  // the store thread, and the column-sum warps
        fence_mbar_init();
    }
    exp_table_init(sm.exptab);
    if (warp == 0) {
        tmem_alloc(&sm.tmem, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;

    // Persistent: every role walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
    // with running chunk counters (cg) for the barrier phases, so the slices
    // of the next tile stream in while the epilogue finishes the current one.
    if (threadIdx.x == 0) {
        const uint32_t bbytes = (uint32_t)(OZ_SLICES * kp.kc) * OZ_B_CHUNK;
        const uint32_t abytes = (uint32_t)kp.kc * OZ_A_CHUNK;
        int ait = 0;
        int64_t cg = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < kp.ktot && ok; tile += gridDim.x) {
            const OzTile tl = oz_tile_of(parts, kp.np, tile);
            const PartDesc &P = tl.P;
            const int ti = tl.ti, tj = tl.tj;
            for (int c = 0; c < nchunks && ok; ++c, ++cg) {
                if (cg > 0 && !oz_wait(&sm.b_empty, (uint32_t)((cg - 1) & 1), err)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&sm.b_full, bbytes);
                const int brow = (int)(P.prow0 + (int64_t)tj * KRR_TILE + c * OZ_N);
                for (int s = 0; s < OZ_SLICES; ++s)
                    for (int kc = 0; kc < kp.kc; ++kc)
                        tma_load_2d(sm.b + (s * OZ_MAXKC + kc) * OZ_B_CHUNK, &tmB, kc * OZ_KC,
                                    (int)(s * prows) + brow, &sm.b_full);
                for (int s = 0; s < OZ_SLICES; ++s, ++ait) {
                    const int st = ait % OZ_ASTAGES, use = ait / OZ_ASTAGES;
                    if (use > 0 && !oz_wait(&sm.a_empty[st], (use - 1) & 1, err)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&sm.a_full[st], abytes);
                    const int arow = (int)(s * prows + P.prow0 + (int64_t)ti * KRR_TILE);
                    for (int kc = 0; kc < kp.kc; ++kc)
                        tma_load_2d(sm.a[st] + kc * OZ_A_CHUNK, &tmA, kc * OZ_KC, arow, &sm.a_full[st]);
                }
            }
        }
    } else if (threadIdx.x == 32) {
        int ait = 0;
        int64_t cg = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < kp.ktot && ok; tile += gridDim.x) {
            for (int c = 0; c < nchunks && ok; ++c, ++cg) {
                if (cg > 0 && !oz_wait(&sm.t_empty, (uint32_t)((cg - 1) & 1), err)) {
                    ok = false;
                    break;
                }
                if (!oz_wait(&sm.b_full, (uint32_t)(cg & 1), err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int s = 0; s < OZ_SLICES; ++s, ++ait) {
                    const int st = ait % OZ_ASTAGES, use = ait / OZ_ASTAGES;
                    if (!oz_wait(&sm.a_full[st], use & 1, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int tt = 0; tt + s < OZ_SLICES; ++tt) {
                        const uint32_t dcol = tmem + (uint32_t)((s + tt) * OZ_N);
                        for (int kk = 0; kk < 2 * kp.kc; ++kk) {
                            const uint64_t da = smem_desc_sw64(sm.a[st] + (kk >> 1) * OZ_A_CHUNK) + 2 * (kk & 1);
                            const uint64_t db =
                                smem_desc_sw64(sm.b + (tt * OZ_MAXKC + (kk >> 1)) * OZ_B_CHUNK) + 2 * (kk & 1);
                            tc_mma_f16(dcol, da, db, OZ_IDESC, (s > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                    tc_commit(&sm.a_empty[st]);
                }
                if (!ok) break;
                tc_commit(&sm.b_empty);
                tc_commit(&sm.t_full);
            }
        }
    } else if (warp >= OZ_EPI_WARP0) {
        // Per chunk: the five levels of both 8-column subs are read from TMEM
        // (then the TMEM is released), distances formed; per sigma the values
        // go to the staging chunk (row r, 16-byte unit u at u ^ (r % 8)) and
        // one thread stores it by TMA to K_hi, K_lo and, as K_hi + lambda m I,
        // to every lambda's factor tile (diagonal tiles: the diagonal patched
        // in the staging copy between the stores).  Another sigma's values are
        // formed while the stores read the staging chunk.
        const int ew = warp - OZ_EPI_WARP0;    // 0..15
        const int quad = warp & 3, quarter = ew >> 2;
        const int r = quad * 32 + lane;            // row inside the tile
        const int et = threadIdx.x - OZ_EPI_WARP0 * 32;  // 0..511
        const int G = kp.nsig * kp.nlam;
        int64_t cg = 0;
        uint32_t round = 0;  // staging rounds (s_free phases)
        bool ok = true;
        // after a timeout the warp keeps walking the tiles (and the barriers)
        // but skips the work; the error word is set and the results unused
        for (int64_t tile = blockIdx.x; tile < kp.ktot; tile += gridDim.x) {
            const OzTile tl = oz_tile_of(parts, kp.np, tile);
            const PartDesc &P = tl.P;
            const int pj = tl.pj, ti = tl.ti, tj = tl.tj;
            const int64_t lt = tl.lt;
            const int gr = ti * KRR_TILE + r;          // row inside the partition
            const int64_t prow = P.prow0 + gr;
            const int er = ex[prow];
            const float2 nr2 = nrm[prow];
            const df nr = df_make(nr2.x, nr2.y);
            for (int c = 0; c < nchunks; ++c, ++cg) {
                const bool got = ok && oz_wait(&sm.t_full, (uint32_t)(cg & 1), err);
                ok = got;
                float dh[2][OZP_SUB], dl[2][OZP_SUB];
                if (got) {
                    tc_fence_after();
#pragma unroll
                    for (int sub = 0; sub < 2; ++sub) {
                        float lv[OZ_SLICES][OZP_SUB];
                        const uint32_t col0 = (uint32_t)(quarter * (OZ_N / 4) + sub * OZP_SUB);
#pragma unroll
                        for (int L = 0; L < OZ_SLICES; ++L)
                            tmem_ld_32x32b_x8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(L * OZ_N) + col0,
                                              lv[L]);
                        tmem_wait_ld();
                        const int cbase = c * OZ_N + (int)col0;  // column inside the tile
#pragma unroll
                        for (int k = 0; k < OZP_SUB; ++k) {
                            const int64_t pc = P.prow0 + (int64_t)tj * KRR_TILE + cbase + k;
                            const float2 nc2 = nrm[pc];
                            const int sc = er + ex[pc] - 13;
                            const df D = oz_distance(lv[0][k], lv[1][k], lv[2][k], lv[3][k], lv[4][k], nr, nc2.x,
                                                     nc2.y, __int_as_float((127 + sc) << 23));
                            dh[sub][k] = D.hi;
                            dl[sub][k] = D.lo;
                        }
                    }
                } else {
#pragma unroll
                    for (int sub = 0; sub < 2; ++sub)
#pragma unroll
                        for (int k = 0; k < OZP_SUB; ++k) dh[sub][k] = dl[sub][k] = 0.f;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.t_empty);  // the levels are in registers
#pragma unroll 1
                for (int is = 0; is < kp.nsig; ++is, ++round) {
                    const float2 cv = kp.cpart ? kp.cpart[pj] : sm.cs[is];
                    const df cs = df_make(cv.x, cv.y);
                    float hv[2][OZP_SUB], lw[2][OZP_SUB];
#pragma unroll
                    for (int sub = 0; sub < 2; ++sub)
#pragma unroll
                        for (int k = 0; k < OZP_SUB; ++k) {
                            const int gc = tj * KRR_TILE + c * OZ_N + quarter * (OZ_N / 4) + sub * OZP_SUB + k;
                            df kv;
                            if (gr >= P.m || gc >= P.m) kv = df_make(gr == gc ? 1.f : 0.f, 0.f);
                            else if (gr == gc) kv = df_make(1.f, 0.f);
                            else kv = df_exp_nonpos(df_mul(df_make(dh[sub][k], dl[sub][k]), cs), sm.exptab);
                            hv[sub][k] = kv.hi;
                            lw[sub][k] = kv.lo;
                        }
                    // the previous round's stores have read the staging chunk
                    if (round > 0 && !oz_wait(&sm.s_free, (round - 1) & 1, err)) ok = false;
#pragma unroll
                    for (int sub = 0; sub < 2; ++sub) {
                        const int col = quarter * (OZ_N / 4) + sub * OZP_SUB;  // in the chunk
                        const int box = col >> 5, u0 = (col & 31) >> 2;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t off = (uint32_t)r * 128u + ((uint32_t)((u0 + h) ^ (r & 7)) << 4);
                            *reinterpret_cast<float4 *>(sm.stage[0][box] + off) =
                                make_float4(hv[sub][4 * h], hv[sub][4 * h + 1], hv[sub][4 * h + 2], hv[sub][4 * h + 3]);
                            *reinterpret_cast<float4 *>(sm.stage[1][box] + off) =
                                make_float4(lw[sub][4 * h], lw[sub][4 * h + 1], lw[sub][4 * h + 2], lw[sub][4 * h + 3]);
                        }
                    }
                    fence_proxy_async_smem();
                    epi_bar_p();
                    const bool diag = ti == tj;
                    if (kp.rsR) {
                        const int64_t g0 = (int64_t)is * kp.rstot + kp.rsoff[pj];
                        // row sums: this thread's 16 columns of row r (registers)
                        float rs = 0.f;
#pragma unroll
                        for (int sub = 0; sub < 2; ++sub)
#pragma unroll
                            for (int k = 0; k < OZP_SUB; ++k) rs += hv[sub][k];
                        kp.rsR[((g0 + (int64_t)ti * P.T + tj) * 8 + c * 4 + quarter) * KRR_TILE + r] = rs;
                        // column sums of off-diagonal tiles (threads 128..191,
                        // column et - 128 of the chunk), from the staged K_hi
                        if (et >= KRR_TILE && et < 3 * KRR_TILE / 2) {
                            if (!diag) {
                                const int cc = et - KRR_TILE;  // column of the chunk
                                const uint32_t cu = (uint32_t)((cc & 31) >> 2), ce = (uint32_t)(cc & 3);
                                const unsigned char *bx = sm.stage[0][cc >> 5];
                                float cs[4] = {0.f, 0.f, 0.f, 0.f};  // four chains: rows r = 4 i + j
#pragma unroll 8
                                for (int rr = 0; rr < KRR_TILE; ++rr)
                                    cs[rr & 3] += *reinterpret_cast<const float *>(
                                        bx + (uint32_t)rr * 128u + ((cu ^ (uint32_t)(rr & 7)) << 4) + 4u * ce);
                                kp.rsC[(g0 + (int64_t)tj * P.T + ti) * KRR_TILE + c * OZ_N + cc] =
                                    (cs[0] + cs[1]) + (cs[2] + cs[3]);
                            }
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&sm.s_free);
                        }
                    }
                    const int y = (int)(((int64_t)is * kp.ktot + P.ktile0 + lt) * KRR_TILE);
                    if (et == 0) {
                        for (int bx = 0; bx < 2; ++bx) {
                            tma_store_2d(&tmKh, c * OZ_N + 32 * bx, y, sm.stage[0][bx]);
                            tma_store_2d(&tmKl, c * OZ_N + 32 * bx, y, sm.stage[1][bx]);
                        }
                        if (!diag && kp.store_factor)
                            for (int il = 0; il < kp.nlam; ++il) {
                                const int yf =
                                    (int)((solves[(int64_t)pj * G + is * kp.nlam + il].ltile0 + lt) * KRR_TILE);
                                for (int bx = 0; bx < 2; ++bx)
                                    tma_store_2d(&tmF, c * OZ_N + 32 * bx, yf, sm.stage[0][bx]);
                            }
                        bulk_commit();
                    }
                    if (diag && kp.store_factor) {  // factor tiles: K_hi + lambda m on the real diagonal
                        for (int il = 0; il < kp.nlam; ++il) {
                            if (et == 0) bulk_wait_read_all();
                            epi_bar_p();  // the staging copy is no longer being read
                            const int rr = c * OZ_N + et;  // diagonal entry (rr, rr) of this chunk
                            if (et < OZ_N && ti * KRR_TILE + rr < P.m) {
                                const float lm = (float)solves[(int64_t)pj * G + is * kp.nlam + il].lambda_m;
                                const int box = et >> 5, u = (et & 31) >> 2;
                                float *d = reinterpret_cast<float *>(sm.stage[0][box] + (uint32_t)rr * 128u +
                                                                     ((uint32_t)(u ^ (rr & 7)) << 4)) +
                                           (et & 3);
                                *d = 1.f + lm;
                            }
                            fence_proxy_async_smem();
                            epi_bar_p();
                            if (et == 0) {
                                const int yf =
                                    (int)((solves[(int64_t)pj * G + is * kp.nlam + il].ltile0 + lt) * KRR_TILE);
                                for (int bx = 0; bx < 2; ++bx)
                                    tma_store_2d(&tmF, c * OZ_N + 32 * bx, yf, sm.stage[0][bx]);
                                bulk_commit();
                            }
                        }
                    }
                    if (et == 0) {
                        bulk_wait_read_all();
                        mbar_arrive(&sm.s_free);
                    }
                }
            }
        }
        if (et == 0) bulk_wait_all();  // the stores have completed
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------- host
bool make_tile_tmap(CUtensorMap *, float *, int64_t);  // chol.cu: FP32 tile store, 32 x 128 boxes, 128B swizzle

typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                      const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                      CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                      CUtensorMapFloatOOBfill);
static PFN_encodeTiled_t oz_encode() {
    static const PFN_encodeTiled_t fn = []() -> PFN_encodeTiled_t {  // thread-safe one-time lookup
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_encodeTiled_t)p;
        return nullptr;
    }();
    return fn;
}

// 2-D view of a slice array [rows][dpz] bf16, box 32 x box_rows, 64-byte swizzle
bool make_slice_tmap(CUtensorMap *map, void *base, int64_t rows, int dpz, int box_rows) {
    PFN_encodeTiled_t enc = oz_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)dpz, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)dpz * 2};
    cuuint32_t box[2] = {(cuuint32_t)OZ_KC, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int oz_dpz(int d) { return ((d + OZ_KC - 1) / OZ_KC) * OZ_KC; }
bool oz_supported(int d) { return d <= OZ_MAXKC * OZ_KC; }

void launch_oz_slice(cudaStream_t st, const double *X, int d, const int64_t *map, int64_t nreal, int64_t nout,
                     void *S, int32_t *ex, float2 *nrm) {
    if (nout <= 0) return;
    KRR_LAUNCHED(), oz_slice_kernel<<<(unsigned)((nout + 127) / 128), 128, 0, st>>>(
        X, d, oz_dpz(d), map, nreal, nout, (__nv_bfloat16 *)S, ex, nrm);
}

size_t oz_smem_bytes() { return sizeof(OzSmem) + 1024; }
static size_t oz_psmem_bytes() { return sizeof(OzPSmem) + 1024; }

// Kernel tiles of every partition and sigma, plus (store_factor) the factor
// matrices K_hi + lambda m I; without them the factorisation's first touch of
// each factor tile reads K_hi and adds lambda m itself.
cudaError_t launch_kbuild_oz(cudaStream_t st, const Model &M, int64_t ktot, float *Kh, float *Kl, float *A,
                             float *rsR, float *rsC, const int64_t *rsoff, int64_t rstot, int *d_err,
                             bool store_factor, const float2 *cpart) {
    if (ktot == 0) return cudaSuccess;
    CUtensorMap tmA, tmKh, tmKl, tmF;
    if (!make_slice_tmap(&tmA, M.ozS, (int64_t)OZ_SLICES * M.prows, M.dpz, OZ_M)) return cudaErrorInvalidValue;
    int64_t ftiles = 0;  // tiles of the factor store
    for (const SolveDesc &S : M.solves) ftiles = std::max<int64_t>(ftiles, S.ltile0 + tri(S.T));
    if (!make_tile_tmap(&tmKh, Kh, (int64_t)M.nsig * ktot) || !make_tile_tmap(&tmKl, Kl, (int64_t)M.nsig * ktot) ||
        !make_tile_tmap(&tmF, A, ftiles))
        return cudaErrorInvalidValue;
    allow_max_dyn_smem(kbuild_oz_kernel);
    OzKParams kp;
    kp.nsig = M.nsig;
    kp.nlam = M.nlam;
    kp.np = M.p;
    kp.kc = M.dpz / OZ_KC;
    kp.ktot = ktot;
    kp.rsR = rsR;
    kp.rsC = rsC;
    kp.rsoff = rsoff;
    kp.rstot = rstot;
    kp.store_factor = store_factor ? 1 : 0;
    kp.cpart = cpart;
    for (int i = 0; i < 8; ++i) {
        const double c = i < M.nsig ? -1.0 / (2.0 * M.sigmas[i] * M.sigmas[i]) : 0.0;
        kp.c_hi[i] = (float)c;
        kp.c_lo[i] = (float)(c - (double)(float)c);
    }
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::min<int64_t>(ktot, nsm);  // persistent: one CTA per SM
    KRR_LAUNCHED(), kbuild_oz_kernel<<<grid, OZP_THREADS, oz_smem_bytes(), st>>>(
        tmA, M.oz_tmB, tmKh, tmKl, tmF, M.d_parts, M.d_solves, M.ozex, M.nrm, kp, M.prows, Kh, Kl, A, d_err);
    return cudaGetLastError();
}

// Slices the test rows (grouped by route when given), then launches one pass
// per (sigma subset, lambda subset).  Xt rows -> workspace owned by the caller.
cudaError_t launch_predict_oz(cudaStream_t st, const Model &M, const CUtensorMap &tmB, const double *Xt, int64_t t,
                              const int64_t *toff, const int64_t *tidx, int routed, void *tslices, int32_t *tex,
                              float2 *tnrm, int64_t t_rows, double *out, int *d_err) {
    // a model with one sigma per partition (krr_fit_jobs) reads its c from M.d_cpart
    const int dpz = oz_dpz(M.d);
    launch_oz_slice(st, Xt, M.d, tidx, t, t_rows, tslices, tex, tnrm);
    CUtensorMap tmA;
    if (!make_slice_tmap(&tmA, tslices, (int64_t)OZ_SLICES * t_rows, dpz, OZ_M)) return cudaErrorInvalidValue;
    allow_max_dyn_smem(predict_oz_kernel);
    for (int s0 = 0; s0 < M.nsig; s0 += OZ_NSP)
        for (int l0 = 0; l0 < M.nlam; l0 += OZ_NLP) {
            OzParams pp;
            pp.nsig = std::min(OZ_NSP, M.nsig - s0);
            pp.nlam = std::min(OZ_NLP, M.nlam - l0);
            pp.sig0 = s0;
            pp.lam0 = l0;
            pp.Gtot = M.nsig * M.nlam;
            pp.nl_total = M.nlam;
            pp.kc = dpz / OZ_KC;
            pp.t_rows = t_rows;
            pp.cpart = M.d_cpart;
            for (int i = 0; i < OZ_NSP; ++i) {
                const double c = i < pp.nsig ? -1.0 / (2.0 * M.sigmas[s0 + i] * M.sigmas[s0 + i]) : 0.0;
                pp.c_hi[i] = (float)c;
                pp.c_lo[i] = (float)(c - (double)(float)c);
            }
            // for the routed form the grouped rows start at toff[j]; the tile count bounds every
            // partition.  Test tiles run fastest: the CTAs in flight share two or three
            // partitions' training slices, which L2 then serves to every test tile
            dim3 grid((unsigned)((t + OZ_M - 1) / OZ_M), (unsigned)M.p);
            KRR_LAUNCHED(), predict_oz_kernel<<<grid, OZP_THREADS, oz_psmem_bytes(), st>>>(
                tmA, tmB, M.d_parts, M.d_solves, M.alpha2, M.ozex, M.nrm, tex, tnrm, t, toff, routed ? tidx : nullptr,
                pp, routed, M.prows, out, d_err);
        }
    return cudaGetLastError();
}

}  // namespace krr
