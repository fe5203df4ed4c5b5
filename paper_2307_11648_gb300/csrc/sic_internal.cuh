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

struct sic_handle {
    int device;
    int num_sms;
    DevStatus* d_status;  // one word in device memory, owned by the handle
    long long last_unit;
};

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

// tcgen05 scoring kernel of the proposal network (mlp_tc.cu)
sic_status sic_proposal_score_tc(sic_handle* h, const float* params, const float* feat, int64_t rows, float* score,
                                 cudaStream_t s);
