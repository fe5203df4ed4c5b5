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
// exp(x), x <= 0: table-driven reduction after Tang (ACM TOMS 15(2), 1989).  With
// k = round(256 x / ln 2) = 256 q + j, x = k ln2/256 + r, |r| <= ln2/512, and
// exp(x) = 2^q * 2^(j/256) * e^r.  ln2/256 is split into its double rounding and the tail,
// so r carries ~1e-19 absolute error for |k| < 2^18; e^r - 1 = r + r^2 (1/2 + r/6 + r^2/24),
// truncation below 4e-17.  The result is formed as T_j + T_j p in one fused operation and
// scaled by adding q to the exponent field.  Error: the table's rounding plus one final
// rounding (about 1.5 ulp).  9 FP64 operations.  Arguments below -700 return 0
// (exp(-700) ~ 1e-304).  `tab` holds scale * 2^(j/256), j = 0..255 (exp_table_fill), so the
// routine returns scale * exp(x) (the Matern fill folds the variance in this way).
constexpr int EXP_TAB = 256;

__device__ __forceinline__ void exp_table_fill(double* tab, double scale = 1.0) {
    for (int j = threadIdx.x; j < EXP_TAB; j += blockDim.x) tab[j] = scale * exp2((double)j * (1.0 / EXP_TAB));
}

__device__ __forceinline__ double exp_neg_table(double x, const double* __restrict__ tab) {
    constexpr double SHIFT = 6755399441055744.0;                // 1.5 * 2^52
    constexpr double INV_L = 369.32993046757463228;             // 256 / ln 2
    constexpr double L1 = 0.6931471805599453094172321 / 256.0;  // ln2/256, rounded
    constexpr double L2 = 2.3190468138462996e-17 / 256.0;       // ln2/256 - L1
    // x < -700 <=> (x negative) high word above that of -700.0 (integer compare, no FP64 op)
    if ((unsigned)__double2hiint(x) > 0xC085E000u) return 0.0;
    double kd = fma(x, INV_L, SHIFT);  // k in the low word, two's complement
    const int k = __double2loint(kd);
    kd -= SHIFT;
    double r = fma(-kd, L1, x);
    r = fma(-kd, L2, r);
    double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    const double p = fma(r * r, q, r);  // e^r - 1
    const double tj = tab[k & (EXP_TAB - 1)];
    const double e = fma(tj, p, tj);
    return __hiloint2double(__double2hiint(e) + ((k >> 8) << 20), __double2loint(e));
}

// sqrt(d2), d2 >= 0: an FP32 reciprocal-square-root seed (from the high word, ~2^-20)
// refined by two Newton steps on the residual d2 - r^2 with the fixed half-reciprocal h:
// the relative error goes 2^-20 -> 1.5 * 2^-40 -> ~2^-59, under one rounding of the last
// fused step.  5 FP64 operations; the range tests are integer compares on the high word.
// d2 < 2^-120 returns 0 (the square root is below 1e-18); d2 > 2^120 uses sqrt().
__device__ __forceinline__ double sqrt_newton(double d2) {
    const unsigned hi = (unsigned)__double2hiint(d2);
    if (hi < 0x38700000u) return 0.0;  // 2^-120 (and +0)
    if (hi >= 0x47700000u) return sqrt(d2);  // 2^120
    const float f = __uint_as_float((hi << 3) - (896u << 23));  // exponent rebased 1023 -> 127
    const unsigned yb = __float_as_uint(rsqrtf(f));
    const unsigned yhi = (yb >> 3) + (896u << 20), ylo = yb << 29;
    const double y = __hiloint2double((int)yhi, (int)ylo);
    const double h = __hiloint2double((int)(yhi - (1u << 20)), (int)ylo);  // y / 2
    double r = d2 * y;
    r = fma(h, fma(-r, r, d2), r);
    r = fma(h, fma(-r, r, d2), r);
    return r;
}

// 1/sqrt(x), x > 0, in FP64: the FP32 seed of sqrt_newton refined by two Newton steps
// y <- y (3/2 - (x/2) y^2) (relative error 2^-20 -> ~2^-39 -> ~2^-77, then rounding:
// about 2 ulp).  7 FP64 operations; x outside [2^-120, 2^120) uses 1 / sqrt(x).
__device__ __forceinline__ double rsqrt_newton(double x) {
    const unsigned hi = (unsigned)__double2hiint(x);
    if (hi < 0x38700000u || hi >= 0x47700000u) return 1.0 / sqrt(x);
    const float f = __uint_as_float((hi << 3) - (896u << 23));
    const unsigned yb = __float_as_uint(rsqrtf(f));
    double y = __hiloint2double((int)((yb >> 3) + (896u << 20)), (int)(yb << 29));
    const double hx = 0.5 * x;
    y = y * fma(-hx * y, y, 1.5);
    y = y * fma(-hx * y, y, 1.5);
    return y;
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
