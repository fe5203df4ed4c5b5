// Internal definitions shared by the libsic translation units (never installed).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sic.h"

// Device-side error word: the first kernel that records an error wins.
struct DevStatus {
    int code;
    int pad;
    long long unit;
};

// One tuned launch choice: op (what is tuned), a bucket key (a, b), the chosen value and its
// measured time.  The handle keeps a small table (sic_tune_* in tune.cpp).
struct TuneEntry {
    int32_t op, a, b, value;
    float ms;
};
constexpr int TUNE_MAX = 64;
constexpr int TUNE_FILL_SPLIT = 1;  // k_fill size classes: groups of <= value members in the first launch
constexpr int TUNE_FILL_BIGNT = 2;  // worker threads of the large-group k_fill launch (256 or 384)
// supernodal selection launch, keyed a = k + 256 * precision, b = 128 * max_cand + max_m:
// value = 2 * threads per CTA + 1 if the state lives in shared memory (generic kernel), or the
// threads per CTA of the register-resident kernel (128 or 256)
constexpr int TUNE_SELECT_AGG = 3;
inline int tune_select_key_a(int k, int prec) { return k + 256 * prec; }
inline int tune_select_key_b(int max_cand, int max_m) { return 128 * max_cand + max_m; }

struct sic_handle {
    int device;
    int num_sms;
    DevStatus* d_status;  // one word in device memory, owned by the handle
    long long last_unit;
    int n_tune;
    TuneEntry tune[TUNE_MAX];
};

// tuned value for (op, a, b), or `fallback` (tune.cpp)
int tune_get(const sic_handle* h, int op, int a, int b, int fallback);
void tune_put(sic_handle* h, int op, int a, int b, int value, float ms);

__device__ __forceinline__ void record_error(DevStatus* st, int code, long long unit) {
    if (atomicCAS(&st->code, 0, code) == 0) st->unit = unit;
}

// Matern parameters in the arithmetic of the selection kernel.
template <typename T>
struct KP {
    T s2;          // variance
    T nugget;      // added on the diagonal
    T c_over_ell;  // sqrt(2 nu) / length_scale
    int nu_x2;     // 1, 3, 5
};

template <typename T>
inline KP<T> make_kp(const sic_kernel& k) {
    double c = (k.nu_x2 == 1) ? 1.0 : (k.nu_x2 == 3 ? sqrt(3.0) : sqrt(5.0));
    KP<T> p;
    p.s2 = (T)k.variance;
    p.nugget = (T)k.nugget;
    p.c_over_ell = (T)(c / k.length_scale);
    p.nu_x2 = k.nu_x2;
    return p;
}

__device__ __forceinline__ double sic_exp(double x) { return exp(x); }
__device__ __forceinline__ float sic_exp(float x) { return __expf(x); }
__device__ __forceinline__ double sic_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float sic_sqrt(float x) { return sqrtf(x); }

// Matern covariance at distance r (Section 2; sqrt(2 nu) r / ell parameterisation), no nugget.
template <typename T>
__device__ __forceinline__ T matern(const KP<T>& k, T r) {
    T t = k.c_over_ell * r;
    T e = sic_exp(-t);
    if (k.nu_x2 == 1) return k.s2 * e;
    if (k.nu_x2 == 3) return k.s2 * ((T)1 + t) * e;
    return k.s2 * ((T)1 + t + t * t * (T)(1.0 / 3.0)) * e;
}

// ---- FP64 Matern with few FP64-pipe instructions (GB300 issues 2 DFMA / clk / SM) ----
//
// The routines below keep FP64 operations for the steps that need 53 bits (an exact
// reduction, one Newton step, the final fused rounding) and do the rest on the FP32 pipe in
// double-float arithmetic: a value hi + lo of two FP32 numbers, built from the error-free
// transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and the exact product a b = p + e,
// e = fma(a, b, -p); the explicit-rounding intrinsics keep the compiler from contracting
// or reassociating them.

// A float as the FP64 number of the same value, by its bit pattern (integer operations only;
// zero for zero and subnormal inputs, below 1.2e-38)
__device__ __forceinline__ double f32_as_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return e ? __hiloint2double((int)hi, (int)(u << 29)) : 0.0;
}

// x split by its bits into hi + lo (integer operations and one integer-to-float conversion):
// hi = x with the significand truncated to 24 bits, lo = the remaining 29 bits rounded to 24,
// so |x - hi - lo| <= 2^-48 |x|.  Valid for 2^-74 <= |x| < 2^128 and for x = 0; below 2^-74
// lo is 0 (|x - hi| < 2^-23 |x|) and below 2^-126 hi is 0 as well.
__device__ __forceinline__ void f64_split(double x, float& hi, float& lo) {
    const unsigned H = (unsigned)__double2hiint(x), L = (unsigned)__double2loint(x);
    const unsigned e = (H >> 20) & 0x7ffu, sg = H & 0x80000000u;
    hi = e > 896u ? __uint_as_float(sg | ((e - 896u) << 23) | ((H & 0xfffffu) << 3) | (L >> 29)) : 0.f;
    const float m = __uint2float_rn(L & 0x1fffffffu);  // the low 29 bits, times 2^(e - 1075)
    lo = e >= 949u ? __fmul_rn(m, __uint_as_float(sg | ((e - 948u) << 23))) : 0.f;
}

// exp(x), -700 <= x <= 700: table-driven reduction after Tang (ACM TOMS 15(2), 1989).  With
// k = round(256 x / ln 2) = 256 q + j (from an FP32 product: off by at most one from the
// nearest integer, which only widens |r| to ~1.6e-3), x = k ln2/256 + r and
// exp(x) = 2^q * 2^(j/256) * e^r.  ln2/256 = L1 + L2 with L1 rounded to 35 significant bits,
// so k L1 is exact for |k| < 2^18 and r1 = x - k L1 is an exact FP64 operation; r = r1 - k L2
// (|k L2| < 1.4e-8) and s = e^r - 1 = r + r^2/2 + r^3/6 + r^4/24 + r^5/120 (truncation below
// 3e-20) are formed in double-float (relative error about 2^-47 of s, |s| < 2e-3), s goes to
// FP64 in one addition, and the result is T_j + T_j s in one fused operation, scaled by adding
// q to the exponent field.  Error: the table's rounding plus one final rounding.  3 FP64
// operations.  Arguments below -700 return 0 (exp(-700) ~ 1e-304).  `tab` holds
// scale * 2^(j/256), j = 0..255 (exp_table_fill), so the routine returns scale * exp(x) (the
// Matern fill folds the variance in this way).
constexpr int EXP_TAB = 256;

__device__ __forceinline__ void exp_table_fill(double* tab, double scale = 1.0) {
    for (int j = threadIdx.x; j < EXP_TAB; j += blockDim.x) tab[j] = scale * exp2((double)j * (1.0 / EXP_TAB));
}

__device__ __forceinline__ double exp_neg_table(double x, const double* __restrict__ tab) {
    constexpr float INV_L = 369.329925537109375f;              // 256 / ln 2 (any rounding works)
    constexpr double L1 = 0.0027076061741126978;               // ln2/256 to 35 bits (0x1.62e42fefcp-9)
    constexpr float L2_HI = -5.0411406413196705e-14f;          // ln2/256 - L1, as a double-float
    constexpr float L2_LO = -8.917921829536205e-22f;
    constexpr float THIRD_HI = 0.3333333432674408f, THIRD_LO = -9.934107758624577e-09f;  // 1/3
    const unsigned xh = (unsigned)__double2hiint(x);
    // x < -700 <=> (x negative) high word above that of -700.0 (integer compare, no FP64 op)
    if (xh > 0xC085E000u) return 0.0;
    const unsigned ex = (xh >> 20) & 0x7ffu;
    const float xf = ex > 896u ? __uint_as_float((xh & 0x80000000u) | ((ex - 896u) << 23) | ((xh & 0xfffffu) << 3))
                               : 0.f;  // x to ~2^-20 (a float of the high word)
    const float kf = rintf(__fmul_rn(xf, INV_L));
    const int k = (int)kf;
    const double r1 = fma(-f32_as_f64(kf), L1, x);  // exact
    float ah, al;
    f64_split(r1, ah, al);
    // r = (ah + al) - k L2, k L2 = kl + kle
    const float kl = __fmul_rn(kf, L2_HI);
    const float kle = __fmaf_rn(kf, L2_LO, __fmaf_rn(kf, L2_HI, -kl));
    float rh = __fadd_rn(ah, -kl);
    float rl = __fadd_rn(__fsub_rn(ah, __fsub_rn(rh, __fsub_rn(rh, ah))), __fsub_rn(-kl, __fsub_rn(rh, ah)));  // TwoSum
    rl = __fadd_rn(rl, __fsub_rn(al, kle));
    {  // renormalise (Fast2Sum: |rh| >= |rl|)
        const float t = __fadd_rn(rh, rl);
        rl = __fsub_rn(rl, __fsub_rn(t, rh));
        rh = t;
    }
    // r^2 = p + pl (pl: the product's error and the cross term 2 rh rl)
    const float p = __fmul_rn(rh, rh);
    const float pl = __fmaf_rn(2.f * rh, rl, __fmaf_rn(rh, rh, -p));
    // r^3/6 = (r^2/2)(r/3): r/3 = t3 + t3l, then (p/2) t3 exactly as c3 + c3l
    const float t3 = __fmul_rn(rh, THIRD_HI);
    const float t3l = __fmaf_rn(rl, THIRD_HI, __fmaf_rn(rh, THIRD_LO, __fmaf_rn(rh, THIRD_HI, -t3)));
    const float ph = 0.5f * p;
    const float c3 = __fmul_rn(ph, t3);
    const float c3l = __fmaf_rn(0.5f * pl, t3, __fmaf_rn(ph, t3l, __fmaf_rn(ph, t3, -c3)));
    // r^4/24 + r^5/120 in FP32 (below 3e-13)
    const float c4 = __fmul_rn(__fmul_rn(p, p), __fmaf_rn(rh, 1.f / 120.f, 1.f / 24.f));
    // q = ph + c3 (TwoSum) + the small terms; s = rh + q.hi (TwoSum) + the rest
    const float qh = __fadd_rn(ph, c3);
    const float qb = __fsub_rn(qh, ph);
    const float ql = __fadd_rn(__fadd_rn(__fsub_rn(ph, __fsub_rn(qh, qb)), __fsub_rn(c3, qb)),
                               __fadd_rn(__fadd_rn(0.5f * pl, c3l), c4));
    const float sh = __fadd_rn(rh, qh);
    const float sb = __fsub_rn(sh, rh);
    const float sl = __fadd_rn(__fadd_rn(__fsub_rn(rh, __fsub_rn(sh, sb)), __fsub_rn(qh, sb)), __fadd_rn(rl, ql));
    const double s = f32_as_f64(sh) + f32_as_f64(sl);
    const double tj = tab[k & (EXP_TAB - 1)];
    const double e = fma(tj, s, tj);
    return __hiloint2double(__double2hiint(e) + ((k >> 8) << 20), __double2loint(e));
}

// sqrt(d2), d2 >= 0.  For 2^-74 <= d2 < 2^120: an FP32 root r0 = dh rsqrt(dh) of the high part
// (~2^-22), one Newton step on the exact residual dh + dl - r0^2 in double-float
// (r1 = r0 + c to ~2^-43), then one FP64 Newton step r = r1 + (d2 - r1^2) / (2 r0): under one
// rounding of the last fused operation.  3 FP64 operations.  Below 2^-74: the FP32 seed of the
// high word refined by two FP64 Newton steps (5 operations); below 2^-120 the result is 0 (the
// square root is below 1e-18); from 2^120 on, sqrt().
__device__ __forceinline__ double sqrt_newton(double d2) {
    const unsigned hi = (unsigned)__double2hiint(d2);
    if (hi >= 0x47700000u) return sqrt(d2);  // 2^120
    if (hi < 0x3B500000u) {                  // 2^-74
        if (hi < 0x38700000u) return 0.0;    // 2^-120 (and +0)
        const float f = __uint_as_float((hi << 3) - (896u << 23));  // exponent rebased 1023 -> 127
        const unsigned yb = __float_as_uint(rsqrtf(f));
        const unsigned yhi = (yb >> 3) + (896u << 20), ylo = yb << 29;
        const double y = __hiloint2double((int)yhi, (int)ylo);
        const double h = __hiloint2double((int)(yhi - (1u << 20)), (int)ylo);  // y / 2
        double r = d2 * y;
        r = fma(h, fma(-r, r, d2), r);
        return fma(h, fma(-r, r, d2), r);
    }
    float dh, dl;
    f64_split(d2, dh, dl);
    const float y = rsqrtf(dh);
    const float r0 = __fmul_rn(dh, y);
    const float h0 = 0.5f * y;  // 1 / (2 r0), ~2^-22
    const float p = __fmul_rn(r0, r0);
    const float pe = __fmaf_rn(r0, r0, -p);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(dh, p), pe), dl);  // dh - p exact (Sterbenz)
    const double r1 = f32_as_f64(r0) + f32_as_f64(__fmul_rn(res, h0));
    return fma(f32_as_f64(h0), fma(-r1, r1, d2), r1);
}

// 1/sqrt(x), x > 0, in FP64.  For 2^-74 <= x < 2^100: an FP32 reciprocal square root y of the
// high part (~2^-22), one Newton step on the residual 1 - (xh + xl) y^2 in double-float
// (y1 = y + c to ~2^-43), then one FP64 Newton step y1 + (y/2)(1 - (x y1) y1) (~2^-86 before
// two roundings: about 1 ulp).  4 FP64 operations.  Outside that range, 1 / sqrt(x).
__device__ __forceinline__ double rsqrt_newton(double x) {
    const unsigned hi = (unsigned)__double2hiint(x);
    if (hi < 0x3B500000u || hi >= 0x46300000u) return 1.0 / sqrt(x);
    float xh, xl;
    f64_split(x, xh, xl);
    const float y = rsqrtf(xh);
    const float y2 = __fmul_rn(y, y);
    const float y2e = __fmaf_rn(y, y, -y2);  // y^2 = y2 + y2e exactly
    const float p = __fmul_rn(xh, y2);
    const float pe = __fmaf_rn(xh, y2, -p);  // xh y2 = p + pe exactly
    // e0 = 1 - x y^2 = ((1 - p) - pe) - xh y2e - xl y2 (1 - p exact: p is within 2^-20 of 1)
    const float e0 = __fmaf_rn(-xl, y2, __fmaf_rn(-xh, y2e, __fsub_rn(__fsub_rn(1.f, p), pe)));
    const float h = 0.5f * y;
    const double y1 = f32_as_f64(y) + f32_as_f64(__fmul_rn(h, e0));
    return fma(f32_as_f64(h), fma(-(x * y1), y1, 1.0), y1);
}

// FP64 Matern from a squared distance with the two routines above (same parameterisation
// as matern<double>); `tab_s2` is the exp table filled with scale = the variance.
__device__ __forceinline__ double matern_d2_fast(const KP<double>& k, double d2, const double* __restrict__ tab_s2) {
    const double t = k.c_over_ell * sqrt_newton(d2);
    const double e = exp_neg_table(-t, tab_s2);  // s2 exp(-t)
    if (k.nu_x2 == 1) return e;
    if (k.nu_x2 == 3) return fma(t, e, e);
    return fma(fma(t, 1.0 / 3.0, 1.0), t * e, e);
}

#define SIC_CUDA_TRY(expr)                        \
    do {                                          \
        cudaError_t _e = (expr);                  \
        if (_e != cudaSuccess) return SIC_ERR_CUDA; \
    } while (0)

static inline int sic_valid_kernel(const sic_kernel* kp) {
    if (!kp) return 0;
    if (kp->dim < 1 || kp->dim > 3) return 0;
    if (kp->nu_x2 != 1 && kp->nu_x2 != 3 && kp->nu_x2 != 5) return 0;
    if (!(kp->length_scale > 0) || !(kp->variance > 0) || !(kp->nugget >= 0)) return 0;
    return 1;
}

static inline double sic_floor_of(const sic_kernel* kp) {
    return kp->nugget > 0 ? 0.5 * kp->nugget : 1e-14 * kp->variance;
}

// Persistent grid size: resident CTAs per SM times the SM count, capped by the work.
template <typename K>
static inline int persistent_grid(const sic_handle* h, K kernel, int threads, size_t smem, long long work) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    long long g = (long long)per_sm * h->num_sms;
    if (work < g) g = work;
    if (g < 1) g = 1;
    return (int)g;
}

// register-resident FP32 supernodal selection (select_agg_reg.cu): used by
// sic_select_aggregated when agg_reg_applies; its workspace holds the targets' factors
bool agg_reg_applies(sic_precision prec, int max_cand, int max_m, int k);
size_t agg_reg_workspace(long long n_grp, int max_m);
sic_status launch_agg_reg(sic_handle* h, const double* pts, long long n, const sic_kernel* kp,
                          const int64_t* grp_ptr, int64_t n_grp, const int64_t* cand_ptr, const int32_t* cand_idx,
                          int max_cand, int max_m, int k, int32_t* sel_idx, int32_t* sel_count, double* gain,
                          void* ws, size_t ws_bytes, cudaStream_t s);

// fixed-order sum of log v (fill.cu); ws holds sic_build_factor_workspace(n) bytes
sic_status launch_sum_logv(const double* logv, long long n, double* sum_logv, void* ws, cudaStream_t s);

// tcgen05 BF16 GEMM of the training (mlp_tc.cu): C (M x 128 FP32) [+ z * M * 128 per K-split]
// = A (M x K, strides sam / sak) * B (K x 128, strides sbk / sbn), operands rounded to BF16
sic_status gemm_tc(sic_handle* h, cudaStream_t s, int M, int K, const float* A, long long sam, long long sak,
                   const float* B, long long sbk, long long sbn, float* C, int nz);

// tcgen05 scoring kernel of the proposal network (mlp_tc.cu)
sic_status sic_proposal_score_tc(sic_handle* h, const float* params, const float* feat, int64_t rows, float* score,
                                 cudaStream_t s);
