// Double-float arithmetic on the FP32 pipe, and the Matern covariance evaluated with it.
//
// GB300 retires about one FP64 warp instruction per 80 clocks per SM sub-partition against
// one FP32 warp instruction per clock, so the FP64 fill spends its FP64 instructions on the
// factorisation and evaluates the kernel entries here.  A double-float value is the
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2 (about 48 significant
// bits).  The operations are built from error-free transformations: TwoSum (Knuth, The Art
// of Computer Programming vol. 2, 4.2.2), Fast2Sum (Dekker 1971; needs |a| >= |b|) and the
// exact product a b = p + e with e = fma(a, b, -p).  Every operation uses the explicit-
// rounding intrinsics, which the compiler may not contract or reassociate.
#pragma once

#include "sic_internal.cuh"

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {  // |a| >= |b| (or a = 0)
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// x + y: TwoSum of the high parts, the low parts added to its error, renormalised.  Relative
// error about 2^-47 without cancellation; with cancellation of the high parts the absolute
// error stays about 2^-48 (|x| + |y|).
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
    const dfl s = df_two_sum(x.hi, y.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }

// x y: the exact product of the high parts plus the cross terms (relative error about 2^-46)
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
    const dfl p = df_two_prod(x.hi, y.hi);
    return df_fast_two_sum(p.hi, __fadd_rn(p.lo, __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi))));
}

// An FP64 number as a double-float (FP64 operations: for per-point or per-launch values)
__device__ __forceinline__ dfl df_from_double(double x) {
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
}

// hi + lo in FP64: exact (the two parts' 48 bits fit in 53), one FP64 addition
__device__ __forceinline__ double df_to_double(dfl x) { return f32_as_f64(x.hi) + f32_as_f64(x.lo); }

// sqrt(a), a >= 0: the correctly rounded FP32 root refined by one Newton step on the exact
// residual a - r^2 (relative error about 2^-47)
__device__ __forceinline__ dfl df_sqrt(dfl a) {
    if (!(a.hi > 0.f)) return {0.f, 0.f};
    const float r = __fsqrt_rn(a.hi);
    const dfl r2 = df_two_prod(r, r);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, r2.hi), r2.lo), a.lo);  // a.hi - r2.hi is exact
    return df_fast_two_sum(r, __fdiv_rn(res, __fadd_rn(r, r)));
}

// Per-launch constants of the double-float Matern: the exp table scale * 2^(j/256) as
// double-floats (j = 0..255), sqrt(2 nu) / ell, and the scale in FP32.
constexpr int DF_EXP_TAB = 256;

struct DfMatern {
    dfl c;         // sqrt(2 nu) / length_scale
    float scale;   // the variance (for the FP32 tail of the exponential)
    int nu_x2;
};

__device__ __forceinline__ DfMatern df_matern_params(const KP<double>& k) {
    return {df_from_double(k.c_over_ell), (float)k.s2, k.nu_x2};
}

// tab[j] = scale * 2^(j/256) (hi parts at tab_hi, low parts at tab_lo), by the threads of the block
__device__ __forceinline__ void df_exp_table_fill(float* tab_hi, float* tab_lo, double scale) {
    for (int j = threadIdx.x; j < DF_EXP_TAB; j += blockDim.x) {
        const dfl v = df_from_double(scale * exp2((double)j * (1.0 / DF_EXP_TAB)));
        tab_hi[j] = v.hi;
        tab_lo[j] = v.lo;
    }
}

// scale * exp(-t), t >= 0 double-float.  For t <= 36: Tang's table-driven reduction (ACM TOMS
// 15(2), 1989) carried out in double-float.  k = round(256 t / ln 2), r = k ln2/256 - t with
// |r| <= ln2/512 (about); ln2/256 is split into L_HI (9 significant bits, so k L_HI is exact
// for k < 2^15; here k <= 13296), L_MID and L_LO3, the product k L_MID taken exactly, so r is exact up to the
// rounding of terms below 1e-9.  e^r - 1 = r + r^2/2 + r^2 (r/6 + r^2/24) (the r^5 term is below
// 4e-17), r and r^2 in double-float; with -k = 256 q + j (0 <= j < 256) the result is
// 2^q (T_j + T_j (e^r - 1)), T_j = scale 2^(j/256) from the table, the power of two exact.
// Absolute error about 2^-48 (1 + t) scale exp(-t), below 4e-15 scale for every t.  For t > 36
// the value is below 2.4e-16 scale and the FP32 exponential (relative error about 1e-6, the
// rounding of its argument included) keeps the absolute error below 1e-18 scale even after the
// Matern polynomial (below 470 there); t above 80 returns 0.
__device__ __forceinline__ dfl df_exp_neg(dfl t, float scale, const float* __restrict__ tab_hi,
                                          const float* __restrict__ tab_lo) {
    if (t.hi > 36.f) return {t.hi > 80.f ? 0.f : __fmul_rn(scale, __expf(-t.hi)), 0.f};
    constexpr float INV_L = 369.329925537109375f;             // 256 / ln 2 (any rounding works)
    constexpr float L_HI = 0.00270843505859375f;              // ln2/256 to 9 bits
    constexpr float L_MID = -8.288845378956466e-07f;          // ln2/256 - L_HI, FP32
    constexpr float L_LO3 = 6.432011600578363e-15f;           // the rest (below 5e-23 remains)
    constexpr float MAGIC = 12582912.f;                       // 1.5 * 2^23: rounds to an integer
    const float kf = __fsub_rn(__fadd_rn(__fmul_rn(t.hi, INV_L), MAGIC), MAGIC);
    const int k = (int)kf;  // exact: 0 <= kf <= 13296
    const float a0 = __fsub_rn(__fmul_rn(kf, L_HI), t.hi);   // exact: k L_HI exact, Sterbenz
    const dfl m = df_two_prod(kf, L_MID);
    const float rest = __fadd_rn(__fsub_rn(m.lo, t.lo), __fmul_rn(kf, L_LO3));
    const dfl s = df_two_sum(a0, m.hi);
    const dfl r = df_two_sum(s.hi, __fadd_rn(s.lo, rest));  // r may be tinier than its correction
    // e^r - 1
    const dfl r2 = df_two_prod(r.hi, r.hi);
    const float w = __fmul_rn(r.hi, __fmaf_rn(r.hi, 1.f / 24.f, 1.f / 6.f));
    const float tail = __fadd_rn(__fadd_rn(__fmul_rn(0.5f, r2.lo), __fmul_rn(r.hi, r.lo)), __fmul_rn(r2.hi, w));
    dfl p = df_two_sum(r.hi, __fmul_rn(0.5f, r2.hi));
    p = df_fast_two_sum(p.hi, __fadd_rn(p.lo, __fadd_rn(r.lo, tail)));
    // exp(-t) = 2^(-k/256) e^r, -k = 256 q + j
    const int mk = -k;
    const int q = mk >> 8;  // floor(-k / 256), in [-52, 0]
    const int j = mk & (DF_EXP_TAB - 1);
    const dfl T = {tab_hi[j], tab_lo[j]};
    const dfl e = df_add(T, df_mul(T, p));
    const float sc = __int_as_float((127 + q) << 23);  // 2^q
    return {__fmul_rn(e.hi, sc), __fmul_rn(e.lo, sc)};
}

// The Matern covariance (no nugget) between points i and j given as double-float coordinates
// relative to a common nearby origin (xh / xl: [dim][ld] high and low parts), returned in
// FP64.  Same parameterisation as matern<double>: t = sqrt(2 nu) r / ell; nu = 1/2: s2 e^-t;
// 3/2: s2 (1 + t) e^-t; 5/2: s2 (1 + t + t^2/3) e^-t (s2 folded into the table).  Absolute
// error a few 1e-15 s2 (coordinates relative to the origin carry 2^-48 of their size).
__device__ __forceinline__ double matern_df(const DfMatern& k, const float* __restrict__ xh,
                                            const float* __restrict__ xl, int i, int j, int ld, int dim,
                                            const float* __restrict__ tab_hi, const float* __restrict__ tab_lo) {
    dfl d2 = {0.f, 0.f};
    for (int d = 0; d < dim; ++d) {
        const dfl a = {xh[d * ld + i], xl[d * ld + i]};
        const dfl b = {xh[d * ld + j], xl[d * ld + j]};
        const dfl dx = df_add(a, df_neg(b));
        d2 = df_add(d2, df_mul(dx, dx));
    }
    const dfl t = df_mul(k.c, df_sqrt(d2));
    const dfl e = df_exp_neg(t, k.scale, tab_hi, tab_lo);
    dfl v = e;
    if (k.nu_x2 == 3) {
        v = df_add(e, df_mul(e, t));
    } else if (k.nu_x2 == 5) {
        const dfl third = {0.3333333432674408f, -9.934107758624577e-09f};  // 1/3
        v = df_add(e, df_mul(e, df_add(t, df_mul(df_mul(t, t), third))));
    }
    return df_to_double(v);
}
