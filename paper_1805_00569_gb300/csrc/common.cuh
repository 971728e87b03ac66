// common.cuh -- device helpers shared by the sm_103a kernels of libkrr.
//
// * double-float ("df") arithmetic: a value is hi + lo, two FP32 numbers with
//   |lo| <= ulp(hi)/2.  Error-free transformations: TwoSum (Knuth, TAOCP vol. 2,
//   Sec. 4.2.2), Fast2Sum and TwoProduct via FMA (Dekker, "A floating-point
//   technique for extending the available precision", Numer. Math. 1971).
//   This gives ~44-bit arithmetic on the FP32 pipes, which on GB300 are 64x
//   faster than the FP64 pipe.
// * df exponential: table-driven reduction by ln2/256 (three-part constant,
//   256-entry df table of 2^(j/256)) and a short series (relative error ~7e-13
//   for arguments <= 0).
// * Philox4x32-10 (Salmon et al., SC'11) for the seeded row shuffle.
// * thin inline-PTX wrappers for mbarrier, cp.async.bulk(.tensor) and tcgen05.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "exp2_table.h"

#define KRR_TILE 128            // tile edge of every kernel/factor tile
#define KRR_TILE_ELEMS (KRR_TILE * KRR_TILE)

// ----------------------------------------------------------------- df
struct df { float hi, lo; };

__device__ __forceinline__ df df_make(float h, float l) { df r; r.hi = h; r.lo = l; return r; }

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ df df_add(df a, df b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    df r; fast_two_sum(s, e, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ df df_mul(df a, df b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    df r; fast_two_sum(p, e, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ df df_scale2(df a, float pow2) {  // exact scaling by a power of two
    return df_make(a.hi * pow2, a.lo * pow2);
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_from_double(double x) {
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return df_make(h, l);
}

// Accumulator that adds exact products of df numbers: acc += a*b, where the
// hi*hi product is kept exactly and the cross terms are rounded once.
struct df_acc { float s, c; };  // value = s + c (c unnormalised)
__device__ __forceinline__ void dfa_zero(df_acc &a) { a.s = 0.f; a.c = 0.f; }
__device__ __forceinline__ void dfa_fma(df_acc &acc, float ah, float al, float bh, float bl) {
    float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    float s, t;
    two_sum(acc.s, p, s, t);
    acc.s = s;
    acc.c = __fadd_rn(acc.c, __fadd_rn(t, e));
}
__device__ __forceinline__ df dfa_value(const df_acc &a) {
    df r; fast_two_sum(a.s, a.c, r.hi, r.lo);
    if (!(fabsf(a.s) >= fabsf(a.c))) two_sum(a.s, a.c, r.hi, r.lo);
    return r;
}

// exp(x) for df x <= 0; 0 below -87, where the FP32 hi part would be
// subnormal.  Method (table-driven, Tang-style): with n = round(x 256 / ln 2),
// x = n ln2/256 + r, |r| <= ln2/512, so exp(x) = 2^(n >> 8) 2^((n & 255)/256) exp(r).
// ln2/256 = C1 + C2 + C3 with C1 of 8 significant bits, so n C1 is exact for
// |n| < 2^15 and x.hi - n C1 is exact (Sterbenz); n C2 is split exactly into
// p2 + e2 by an FMA and x.hi - n C1 - p2 = s + u exactly by TwoSum, leaving
// r = s + rlo with the small terms rlo = u - e2 - n C3 + x.lo (|rlo| < 4e-6,
// rounded to ~1e-13 absolute).  Then
//   exp(r) = 1 + s + q(s) + rlo (1 + s + s^2/2 + rlo/2),  q = s^2/2 + s^3/6 + s^4/24,
// with q and the rlo term in FP32 (both below 1e-6 in size, so their rounding
// stays below 1e-13) and 1 + s exact as a double-float.  The 256 table values
// 2^(j/256) are double-float numbers (exp2_table.h, computed to 60 digits and
// rounded to hi + lo once), copied to shared memory by every CTA.  Relative
// error ~7e-13 for results above ~1e-30 (the lo part runs into FP32
// subnormals below that).
__device__ __forceinline__ void exp_table_init(float2 *tab) {
    for (int j = threadIdx.x; j < 256; j += blockDim.x) tab[j] = krr_exp2_tab[j];
}
// NORM = false returns the pair unnormalised (hi + lo with |lo| below a few
// ulps of hi, not necessarily hi = rn(hi + lo)): enough for a product that is
// accumulated at once, three operations cheaper.
template <bool NORM = true>
__device__ __forceinline__ df df_exp_nonpos(df x, const float2 *__restrict__ tab) {
    if (!(x.hi > -87.0f)) return df_make(0.f, 0.f);
    const float C1 = 0x1.62p-9f, C2 = 0x1.c85fep-18f, C3 = -0x1.718432p-43f;
    // n = x.hi 256 / ln2 rounded to an integer by the FMA into 1.5 2^23 (integers
    // there are spaced 1; |n| < 2^15), read back from the bits: no conversion
    const float rnd = __fmaf_rn(x.hi, 369.329930467574632284140718f, 0x1.8p23f);
    const float nf = __fsub_rn(rnd, 0x1.8p23f);
    const int n = __float_as_int(rnd) - 0x4B400000;
    const float t1 = __fmaf_rn(-nf, C1, x.hi);  // exact
    const float p2 = __fmul_rn(nf, C2);
    const float e2 = __fmaf_rn(nf, C2, -p2);     // n C2 = p2 + e2
    float s, u;
    two_sum(t1, -p2, s, u);
    const float rlo = __fadd_rn(__fadd_rn(u, -e2), __fmaf_rn(-nf, C3, x.lo));
    const float q = __fmul_rn(__fmul_rn(s, s), __fmaf_rn(s, __fmaf_rn(s, 1.0f / 24.0f, 1.0f / 6.0f), 0.5f));
    const float w = __fmaf_rn(0.5f, rlo, __fmaf_rn(s, __fmul_rn(0.5f, s), s));  // s + s^2/2 + rlo/2
    float eh, el;
    fast_two_sum(1.0f, s, eh, el);
    el = __fadd_rn(el, __fadd_rn(q, __fmaf_rn(rlo, w, rlo)));
    const float2 tv = tab[n & 255];
    const float p = __fmul_rn(tv.x, eh);
    float e = __fmaf_rn(tv.x, eh, -p);
    e = __fmaf_rn(tv.x, el, e);
    e = __fmaf_rn(tv.y, eh, e);
    float yh = p, yl = e;
    if (NORM) fast_two_sum(p, e, yh, yl);
    const float sc = __int_as_float((127 + (n >> 8)) << 23);  // 2^(n >> 8), n >> 8 in [-126, 0]
    return df_make(yh * sc, yl * sc);
}

// Exponent range of a prediction row.  The double-float exponential has the
// FP32 range (results below e^-87 are 0), while an Eq. 7 sum can be a
// meaningful number far below that (a test row far from every training row
// at a small sigma).  A row whose largest exponent argument so far, x_max =
// D_min * c (c = -1/(2 sigma^2)), is below -20 takes its terms as
// exp(x - K ln2) = exp(x) 2^-K with the integer
//   K = ceil((x_max + 1/64) / ln2) <= 0,
// so every shifted argument is <= -1/64 and the largest term is >= 1/2; the
// accumulated sum is scaled back by 2^K in FP64.  Rows with x_max >= -20
// keep K = 0 and the unshifted arithmetic; the terms the exponential drops
// (below e^-87) are then below e^-67 of the largest one.  K is clamped at
// KRR_SHIFT_NONE (2^-1100 is 0 in FP64, as is every term the clamp affects);
// KRR_SHIFT_NONE also marks a row that has seen no term yet.
#define KRR_SHIFT_NONE (-1100)
__device__ __forceinline__ int exp_row_shift(float xmax) {
    if (!(xmax < -20.f)) return 0;
    const float k = ceilf((xmax + 0.015625f) * 1.44269504088896341f);  // 1 / ln 2
    return k < (float)KRR_SHIFT_NONE ? KRR_SHIFT_NONE : (int)k;
}
// -K ln2 as a double-float, to be added to a shifted row's exponent arguments
__device__ __forceinline__ float2 exp_shift_arg(int k) {
    const double v = -(double)k * 0.69314718055994530942;
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}
// 2^e for e <= 0 as a float, 0 below the normal range (exact scaling otherwise)
__device__ __forceinline__ float pow2_nonpos(int e) { return e >= -126 ? __int_as_float((127 + e) << 23) : 0.f; }

// ----------------------------------------------------------------- Philox4x32-10
struct u32x4 { uint32_t x, y, z, w; };
__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        u32x4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// ----------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_time_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Every spin-wait of the library's kernels on an mbarrier gives up after this
// long (a producer that never completes must not hang the GPU).
#define KRR_WAIT_LIMIT_NS 2000000000ull
// Bounded wait for phase `parity` of *bar: polls until it completes or
// limit_ns of the global timer have passed; on expiry stores `code` in *err
// and returns false.  The caller then stops issuing work that depends on the
// barrier, still waits (bounded) for any bulk copy it has in flight, frees
// what it holds and returns.
__device__ __forceinline__ bool mbar_wait_until(uint64_t *bar, uint32_t parity, int *err, uint64_t limit_ns,
                                                int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_time_ns();
    for (;;) {
        for (int i = 0; i < 256; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_time_ns() - t0 > limit_ns) {
            if (err) atomicExch(err, code);
            return false;
        }
    }
}

// 1-D bulk copy global -> shared, completion counted on an mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Bulk prefetch of [src, src + bytes) into L2 (bytes a multiple of 16, src 16-byte aligned).
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// 2-D tiled TMA load.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// 2-D tiled TMA store of a shared-memory box (bulk-group completion).  The
// threads that wrote the box issue fence_proxy_async_smem and synchronise
// with the issuing thread first; x, y >= 0.
__device__ __forceinline__ void tma_store_2d(const void *tmap, int x, int y, const void *src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(tmap), "r"(x),
                 "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of every committed bulk store have been read
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed bulk store has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// tcgen05 (5th-generation tensor core, accumulator in tensor memory)
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D(tmem) (+)= A(smem desc) * B(smem desc)^T, kind::tf32 / kind::f16
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 32 lanes x 32 consecutive columns of FP32 from tensor memory.
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, K-major operand with the 128-byte swizzle
// (8-row x 128-byte atoms, atoms 1024 bytes apart along M/N).
__device__ __forceinline__ uint64_t smem_desc_sw128(const void *p) {
    uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr & 0x3FFFFull) >> 4;          // start address
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}
// Instruction descriptor: FP32 accumulate, A/B format code fmt (TF32 = 2 for
// kind::tf32, BF16 = 1 for kind::f16), both K-major, shape M x N.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// ----------------------------------------------------------------- misc
__device__ __forceinline__ int64_t tri_index(int64_t i, int64_t j) { return i * (i + 1) / 2 + j; }
// inverse of tri_index for idx < T(T+1)/2: row i (>= col j)
__device__ __forceinline__ void tri_decode(int64_t idx, int &i, int &j) {
    // FP32 estimate (no FP64 instructions: GB300's FP64 pipe runs at 1/64 of
    // the FP32 rate); the integer steps below correct it exactly
    int r = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
    while ((int64_t)(r + 1) * (r + 2) / 2 <= idx) ++r;
    while ((int64_t)r * (r + 1) / 2 > idx) --r;
    i = r;
    j = (int)(idx - (int64_t)r * (r + 1) / 2);
}
