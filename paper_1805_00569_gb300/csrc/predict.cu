// predict.cu -- fused prediction (Eq. 7: yhat = sum_i alpha_i Phi(x_i, xhat))
// and model scoring/choice (Eq. 3; the model choice of Alg. BKRR2; the
// averaging of Alg. DC-KRR; the per-point choice of Alg. BKRR3).
//
// Prediction never stores K(test, train).  A CTA owns (partition, 64 test
// rows) and walks the partition's training rows in chunks of 128:
//   1. double-float Gram tile (8 x 4 per thread) of the chunk against the
//      test rows, turned into distances ||a||^2 + ||b||^2 - 2 a.b;
//   2. distances through shared memory; 4 threads per test row then take, for
//      every sigma, the double-float exponential and, for every lambda, add
//      alpha * K into double-float accumulators;
//   3. after the last chunk the 4 partial sums of a test row are combined in
//      a fixed order.  One distance pass feeds all (sigma, lambda) models.
// Routed form: the test rows of partition j are listed (grouped by route) and
// each CTA predicts only its partition's rows.  The plain FP64 path computes
// the same thing with FP64 direct differences and FP64 exp.
#include "common.cuh"
#include "internal.h"

namespace krr {

constexpr int PT = 64;   // test rows per CTA
constexpr int PKC = 16;  // features per staging chunk

constexpr int PG = 16;  // (sigma, lambda) models per pass

struct PredParams {
    int kind;           // Table 1 kernel (KRR_KERNEL_*)
    int nsig, nlam;     // sigmas in this pass, lambdas
    int sig0, Gtot;     // first sigma of this pass, grid size of the model
    float c_hi[PG], c_lo[PG];  // -1 / (2 sigma^2) as df, for this pass
    double c64[PG];
};

// grid (p, ceil(tmax / 64)).  tstart/tcount per partition; tidx maps a
// grouped position to a test row (nullptr = identity).  out[row][q]: row =
// j*G+g (all-models) or g (routed, routed != 0).
__global__ void __launch_bounds__(256, 1)
predict_df_kernel(const float *__restrict__ Xh, const float *__restrict__ Xl, const float2 *__restrict__ nrm,
                  int32_t dp, const PartDesc *__restrict__ parts, const SolveDesc *__restrict__ solves,
                  const double *__restrict__ alpha, const double *__restrict__ Xt, int64_t t, int32_t d,
                  const int64_t *__restrict__ toff, const int64_t *__restrict__ tidx, PredParams pp, int routed,
                  double *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char pd_dyn[];
    float2 *sD = reinterpret_cast<float2 *>(pd_dyn);             // [128][PT]
    float2 *sAl = sD + KRR_TILE * PT;                             // [PG][128] alpha as df
    float *sTh = reinterpret_cast<float *>(sAl + PG * KRR_TILE);  // [PKC][PT]
    float *sTl = sTh + PKC * PT;
    float *sXh = sTl + PKC * PT;  // [PKC][128]
    float *sXl = sXh + PKC * KRR_TILE;
    float2 *sTn = reinterpret_cast<float2 *>(sXl + PKC * KRR_TILE);  // [PT] test norms
    int64_t *sRow = reinterpret_cast<int64_t *>(sTn + PT);           // [PT] test row ids
    float2 *sY = reinterpret_cast<float2 *>(sRow + PT);               // [PG][256] df accumulators
    float2 *sExp = sY + PG * 256;                                     // [256] 2^(j/256) table
    float2 *sS = sExp + 256;                                          // [PG][256] -K ln2 per sigma (df)
    int *sK = reinterpret_cast<int *>(sS + PG * 256);                 // [PG][256] range shift per sigma
    exp_table_init(sExp);

    const int j = blockIdx.x;
    const PartDesc P = parts[j];
    const int64_t cnt = toff ? toff[j + 1] - toff[j] : t;
    const int64_t q0 = (int64_t)blockIdx.y * PT;
    if (q0 >= cnt) return;
    const int G = pp.nsig * pp.nlam;  // models of this pass
    const int nq = (int)((cnt - q0) < PT ? (cnt - q0) : PT);
    for (int g = 0; g < G; ++g) sY[g * 256 + threadIdx.x] = make_float2(0.f, 0.f);
    for (int is = 0; is < pp.nsig; ++is) {
        sK[is * 256 + threadIdx.x] = KRR_SHIFT_NONE;  // no term yet: the shift argument stays 0
        sS[is * 256 + threadIdx.x] = make_float2(0.f, 0.f);
    }
    float dmin = INFINITY;  // smallest distance of this thread's test row to a real training row
    if (threadIdx.x < PT) {
        int64_t pos = (toff ? toff[j] : 0) + q0 + threadIdx.x;
        sRow[threadIdx.x] = (threadIdx.x < nq) ? (tidx ? tidx[pos] : pos) : -1;
    }
    __syncthreads();
    // test norms (df), one thread per test row
    if (threadIdx.x < PT) {
        df_acc a;
        dfa_zero(a);
        const int64_t row = sRow[threadIdx.x];
        if (row >= 0)
            for (int f = 0; f < d; ++f) {
                const double v = Xt[row * d + f];
                const float h = __double2float_rn(v), l = __double2float_rn(v - (double)h);
                dfa_fma(a, h, l, h, l);
            }
        const df v = dfa_value(a);
        sTn[threadIdx.x] = make_float2(v.hi, v.lo);
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // Gram mapping: rows ty*8.., cols tx*4..
    const int qc = threadIdx.x >> 2, part = threadIdx.x & 3;  // exp mapping: test col qc, rows part*32..
    for (int ch = 0; ch < P.T; ++ch) {
        const int64_t prow = P.prow0 + (int64_t)ch * KRR_TILE;
        df_acc acc[8][4];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) dfa_zero(acc[a][b]);
        for (int f0 = 0; f0 < dp; f0 += PKC) {
            __syncthreads();
            for (int e = threadIdx.x; e < PKC * KRR_TILE; e += 256) {
                const int r = e / PKC, f = e % PKC;
                const bool ok = f0 + f < dp;
                sXh[f * KRR_TILE + r] = ok ? Xh[(prow + r) * dp + f0 + f] : 0.f;
                sXl[f * KRR_TILE + r] = ok ? Xl[(prow + r) * dp + f0 + f] : 0.f;
            }
            for (int e = threadIdx.x; e < PKC * PT; e += 256) {
                const int c = e / PKC, f = e % PKC;
                const int64_t row = sRow[c];
                double v = (row >= 0 && f0 + f < d) ? Xt[row * d + f0 + f] : 0.0;
                const float h = __double2float_rn(v);
                sTh[f * PT + c] = h;
                sTl[f * PT + c] = __double2float_rn(v - (double)h);
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < PKC; ++kk) {
                float ah[8], al[8], bh[4], bl[4];
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    ah[a] = sXh[kk * KRR_TILE + ty * 8 + a];
                    al[a] = sXl[kk * KRR_TILE + ty * 8 + a];
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    bh[b] = sTh[kk * PT + tx * 4 + b];
                    bl[b] = sTl[kk * PT + tx * 4 + b];
                }
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) dfa_fma(acc[a][b], ah[a], al[a], bh[b], bl[b]);
            }
        }
        __syncthreads();
        // distances -> shared; alpha chunk -> shared
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const float2 na = nrm[prow + ty * 8 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float2 nb = sTn[tx * 4 + b];
                df gv = dfa_value(acc[a][b]);
                df D = df_add(df_make(na.x, na.y), df_make(nb.x, nb.y));
                D = df_add(D, df_make(-2.f * gv.hi, -2.f * gv.lo));
                if (D.hi < 0.f) D = df_make(0.f, 0.f);
                sD[(ty * 8 + a) * PT + tx * 4 + b] = make_float2(D.hi, D.lo);
            }
        }
        for (int e = threadIdx.x; e < G * KRR_TILE; e += 256) {
            const int g = e >> 7, r = e & 127;
            const SolveDesc S = solves[(int64_t)j * pp.Gtot + pp.sig0 * pp.nlam + g];
            const double av = alpha[S.vec0 + (int64_t)ch * KRR_TILE + r];
            const float h = __double2float_rn(av);
            sAl[g * KRR_TILE + r] = make_float2(h, __double2float_rn(av - (double)h));
        }
        __syncthreads();
        // range shift (exp_row_shift): the chunk's smallest distance of the test
        // row, the same in its 4 threads; a closer row rescales by 2^(K_old - K_new)
        float dm = INFINITY;
        for (int rr = 0; rr < 32; ++rr) {
            const int r = part * 32 + rr;
            if ((int64_t)ch * KRR_TILE + r >= P.m) break;
            dm = fminf(dm, sD[r * PT + qc].x);
        }
        dm = fminf(dm, __shfl_xor_sync(0xffffffffu, dm, 1));
        dm = fminf(dm, __shfl_xor_sync(0xffffffffu, dm, 2));
        if (dm < dmin) {
            dmin = dm;
            for (int is = 0; is < pp.nsig; ++is) {
                const int ko = sK[is * 256 + threadIdx.x], kn = exp_row_shift(dmin * pp.c_hi[is]);
                if (kn != ko) {
                    const float f = pow2_nonpos(ko - kn);
                    for (int il = 0; il < pp.nlam; ++il) {
                        float2 &y = sY[(is * pp.nlam + il) * 256 + threadIdx.x];
                        y = make_float2(y.x * f, y.y * f);
                    }
                    sK[is * 256 + threadIdx.x] = kn;
                    sS[is * 256 + threadIdx.x] = exp_shift_arg(kn);
                }
            }
        }
        // exp + contraction: thread (qc, part) takes rows part*32 .. part*32+31
#pragma unroll 1
        for (int rr = 0; rr < 32; ++rr) {
            const int r = part * 32 + rr;
            if ((int64_t)ch * KRR_TILE + r >= P.m) break;
            const float2 dv = sD[r * PT + qc];
            const df D = df_make(dv.x, dv.y);
#pragma unroll 1
            for (int is = 0; is < pp.nsig; ++is) {
                df x = df_mul(D, df_make(pp.c_hi[is], pp.c_lo[is]));
                if (sK[is * 256 + threadIdx.x] != 0) {
                    const float2 sv = sS[is * 256 + threadIdx.x];
                    x = df_add(x, df_make(sv.x, sv.y));
                }
                const df k = df_exp_nonpos(x, sExp);
#pragma unroll 1
                for (int il = 0; il < pp.nlam; ++il) {
                    const int g = is * pp.nlam + il;
                    const float2 a = sAl[g * KRR_TILE + r];
                    float2 *slot = &sY[g * 256 + threadIdx.x];
                    df_acc y;
                    y.s = slot->x;
                    y.c = slot->y;
                    dfa_fma(y, k.hi, k.lo, a.x, a.y);
                    *slot = make_float2(y.s, y.c);
                }
            }
        }
    }
    // combine the 4 partial sums of each test row (fixed order) and store
    __syncthreads();
#pragma unroll 1
    for (int g = 0; g < G; ++g) {
        const float2 sv = sY[g * 256 + threadIdx.x];
        df_acc ya;
        ya.s = sv.x;
        ya.c = sv.y;
        df v = dfa_value(ya);
        df o;
        o.hi = __shfl_xor_sync(0xffffffffu, v.hi, 1);
        o.lo = __shfl_xor_sync(0xffffffffu, v.lo, 1);
        v = (part & 1) ? df_add(o, v) : df_add(v, o);
        o.hi = __shfl_xor_sync(0xffffffffu, v.hi, 2);
        o.lo = __shfl_xor_sync(0xffffffffu, v.lo, 2);
        v = (part & 2) ? df_add(o, v) : df_add(v, o);
        if (part == 0 && qc < nq) {
            const int64_t row = sRow[qc];
            const int gm = pp.sig0 * pp.nlam + g;
            const int64_t orow = routed ? (int64_t)gm : (int64_t)j * pp.Gtot + gm;
            const int k = sK[(g / pp.nlam) * 256 + threadIdx.x];  // the same in the row's 4 threads
            out[orow * t + row] = k == 0 ? df_to_double(v) : ldexp(df_to_double(v), k);
        }
    }
}

// Plain FP64 path: direct differences, FP64 exp; 4 threads per test row.
__global__ void __launch_bounds__(256)
predict_fp64_kernel(const double *__restrict__ X64, int32_t d, const PartDesc *__restrict__ parts,
                    const SolveDesc *__restrict__ solves, const double *__restrict__ alpha,
                    const double *__restrict__ Xt, int64_t t, const int64_t *__restrict__ toff,
                    const int64_t *__restrict__ tidx, PredParams pp, int routed, double *__restrict__ out) {
    const int j = blockIdx.x;
    const PartDesc P = parts[j];
    const int64_t cnt = toff ? toff[j + 1] - toff[j] : t;
    const int64_t q0 = (int64_t)blockIdx.y * PT;
    if (q0 >= cnt) return;
    __shared__ double sY[PG][256];
    const int G = pp.nsig * pp.nlam;
    const int qc = threadIdx.x >> 2, part = threadIdx.x & 3;
    const bool live = q0 + qc < cnt;
    const int64_t pos = (toff ? toff[j] : 0) + q0 + qc;
    const int64_t row = live ? (tidx ? tidx[pos] : pos) : 0;
    for (int g = 0; g < G; ++g) sY[g][threadIdx.x] = 0.0;
    if (live) {
        for (int r = part; r < P.m; r += 4) {
            const double *xa = X64 + (P.prow0 + r) * d;
            const double *xb = Xt + row * d;
            double D = 0.0;
            if (pp.kind == KRR_KERNEL_LINEAR) {
                for (int f = 0; f < d; ++f) D = fma(xa[f], xb[f], D);  // x_a . x_b
            } else {
                for (int f = 0; f < d; ++f) {
                    const double df_ = xa[f] - xb[f];
                    D = fma(df_, df_, D);
                }
            }
            for (int is = 0; is < pp.nsig; ++is) {
                const double k = pp.kind == KRR_KERNEL_LINEAR ? D : exp(D * pp.c64[is]);
                for (int il = 0; il < pp.nlam; ++il) {
                    const int g = is * pp.nlam + il;
                    const SolveDesc S = solves[(int64_t)j * pp.Gtot + pp.sig0 * pp.nlam + g];
                    sY[g][threadIdx.x] = fma(alpha[S.vec0 + r], k, sY[g][threadIdx.x]);
                }
            }
        }
    }
    for (int g = 0; g < G; ++g) {
        double v = sY[g][threadIdx.x];
        const double o1 = __shfl_xor_sync(0xffffffffu, v, 1);
        v = (part & 1) ? o1 + v : v + o1;
        const double o2 = __shfl_xor_sync(0xffffffffu, v, 2);
        v = (part & 2) ? o2 + v : v + o2;
        if (part == 0 && live) {
            const int gm = pp.sig0 * pp.nlam + g;
            const int64_t orow = routed ? (int64_t)gm : (int64_t)j * pp.Gtot + gm;
            out[orow * t + row] = v;
        }
    }
}

// ---------------------------------------------------------------- selection
__device__ __forceinline__ double bsum256(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    return sh[0];
}

// mode 0/1: row = blockIdx.x of yhat; mode 2 average over p; mode 3 per-point best
__global__ void mse_kernel(const double *__restrict__ yhat, const double *__restrict__ yt, int64_t t, int p, int G,
                           int mode, double *__restrict__ mse) {
    __shared__ double sh[256];
    const int row = blockIdx.x;
    double acc = 0.0;
    for (int64_t q = threadIdx.x; q < t; q += 256) {
        double v;
        if (mode == KRR_SEL_AVERAGE) {
            double s = 0.0;
            for (int j = 0; j < p; ++j) s += yhat[((int64_t)j * G + row) * t + q];
            v = s / (double)p;
        } else if (mode == KRR_SEL_ORACLE) {
            double best = INFINITY;
            v = 0.0;
            for (int j = 0; j < p; ++j) {
                const double c = yhat[((int64_t)j * G + row) * t + q];
                const double e = (c - yt[q]) * (c - yt[q]);
                if (e < best) {
                    best = e;
                    v = c;
                }
            }
        } else {
            v = yhat[(int64_t)row * t + q];
        }
        const double e = v - yt[q];
        acc += e * e;
    }
    acc = bsum256(acc, sh);
    if (threadIdx.x == 0) mse[row] = t > 0 ? acc / (double)t : 0.0;
}

__global__ void argmin_kernel(const double *__restrict__ v, int n, int32_t *__restrict__ best) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int b = 0;
        for (int i = 1; i < n; ++i)
            if (v[i] < v[b]) b = i;
        *best = b;
    }
}

// ---------------------------------------------------------------- host
static size_t predict_df_smem() {
    return (size_t)KRR_TILE * PT * sizeof(float2) + PG * KRR_TILE * sizeof(float2) + 2 * PKC * PT * sizeof(float) +
           2 * PKC * KRR_TILE * sizeof(float) + PT * sizeof(float2) + PT * sizeof(int64_t) +
           (size_t)PG * 256 * sizeof(float2) + 256 * sizeof(float2) + (size_t)PG * 256 * (sizeof(float2) + sizeof(int));
}

void launch_predict(cudaStream_t st, const Model &M, const double *Xt, int64_t t, const int64_t *toff,
                    const int64_t *tidx, int64_t tmax, int routed, double *out) {
    if (tmax <= 0 || M.p == 0) return;
    const int per_pass = std::max(1, PG / std::max(1, M.nlam));
    for (int s0 = 0; s0 < M.nsig; s0 += per_pass) {
        PredParams pp;
        pp.kind = M.kind;
        pp.nsig = std::min(per_pass, M.nsig - s0);
        pp.nlam = M.nlam;
        pp.sig0 = s0;
        pp.Gtot = M.nsig * M.nlam;
        for (int i = 0; i < PG; ++i) {
            const double c = i < pp.nsig ? -1.0 / (2.0 * M.sigmas[s0 + i] * M.sigmas[s0 + i]) : 0.0;
            pp.c64[i] = c;
            pp.c_hi[i] = (float)c;
            pp.c_lo[i] = (float)(c - (double)(float)c);
        }
        dim3 grid((unsigned)M.p, (unsigned)((tmax + PT - 1) / PT));
        if (M.prec == KRR_PREC_FP64) {
            KRR_LAUNCHED(), predict_fp64_kernel<<<grid, 256, 0, st>>>(M.X64, M.d, M.d_parts, M.d_solves, M.alpha, Xt, t, toff,
                                                      tidx, pp, routed, out);
        } else {
            const size_t sm = predict_df_smem();
            allow_max_dyn_smem(predict_df_kernel);
            KRR_LAUNCHED(), predict_df_kernel<<<grid, 256, sm, st>>>(M.Xh, M.Xl, M.nrm, M.dp, M.d_parts, M.d_solves, M.alpha, Xt, t,
                                                     M.d, toff, tidx, pp, routed, out);
        }
    }
}

void launch_select(cudaStream_t st, const double *yhat, const double *yt, int64_t t, int p, int G, int mode,
                   double *mse, int32_t *best) {
    const int rows = (mode == KRR_SEL_PER_MODEL) ? p * G : G;
    KRR_LAUNCHED(), mse_kernel<<<rows, 256, 0, st>>>(yhat, yt, t, p, G, mode, mse);
    KRR_LAUNCHED(), argmin_kernel<<<1, 32, 0, st>>>(mse, rows, best);
}

}  // namespace krr
