// Directed Gaussian-process selection for one target over n training points
// (Section 3; the selection step of the directed regression algorithm).
//
// One CTA of 1024 threads; the partial Cholesky factor of the candidates is kept in
// the caller's workspace, column-major [k][n] (thread r touches row r of every column).
// The conditional variances and covariances with the target, var[n] and cov[n], sit
// in the workspace too.  Per step: score cov^2/var (eq. obj_gp), block argmax (ties:
// lowest training index), the pivot's row staged in shared memory, then every thread
// appends u_j = (Theta_{jq} - F_j . F_q)/sqrt(var_q) and downdates var and cov
// (eq. cond_select).  out_var traces the target's conditional variance.
#include "sic_internal.cuh"

namespace {

constexpr int NT = 1024;
constexpr int NW = NT / 32;

template <typename T>
__device__ __forceinline__ bool better(T s, long long i, T bs, long long bi) {
    return s > bs || (s == bs && i < bi);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_select_single(const double* __restrict__ xtr, long long n, int dim,
                                                      const double* __restrict__ xt, KP<T> kp, T floor_, int k,
                                                      int32_t* __restrict__ out_idx, double* __restrict__ out_var,
                                                      int32_t* __restrict__ out_count, T* __restrict__ ws) {
    extern __shared__ unsigned char smem_raw[];
    T* piv = reinterpret_cast<T*>(smem_raw);  // k
    __shared__ T wsc[NW];
    __shared__ long long wix[NW];
    T* F = ws;
    T* var = F + (long long)k * n;
    T* cov = var + n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T NEG = -INFINITY;
    double org[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < dim; ++d) org[d] = xt[d];
    auto coord = [&](long long j, int d) -> T {
        if constexpr (sizeof(T) == 8) return (T)xtr[j * dim + d];
        return (T)(xtr[j * dim + d] - org[d]);
    };
    for (long long j = tid; j < n; j += NT) {
        T d2 = (T)0;
        for (int d = 0; d < dim; ++d) {
            T df = (T)(xtr[j * dim + d] - org[d]);
            d2 += df * df;
        }
        var[j] = kp.s2 + kp.nugget;
        cov[j] = matern<T>(kp, sic_sqrt(d2));
    }
    double vt = (double)(kp.s2 + kp.nugget);
    if (tid == 0) out_var[0] = vt;
    __syncthreads();
    int t = 0;
    for (; t < k; ++t) {
        T bs = NEG;
        long long bi = 0x7fffffffffffffffLL;
        for (long long j = tid; j < n; j += NT) {
            T v = var[j];
            if (v >= floor_) {
                T c = cov[j];
                T s = c * c / v;
                if (better(s, j, bs, bi)) { bs = s; bi = j; }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            T os = __shfl_xor_sync(0xffffffffu, bs, off);
            long long oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (better(os, oi, bs, bi)) { bs = os; bi = oi; }
        }
        if (lane == 0) {
            wsc[warp] = bs;
            wix[warp] = bi;
        }
        __syncthreads();
        T gs = wsc[0];
        long long q = wix[0];
        for (int w = 1; w < NW; ++w)
            if (better(wsc[w], wix[w], gs, q)) { gs = wsc[w]; q = wix[w]; }
        if (q == 0x7fffffffffffffffLL || !(gs > (T)0)) break;
        const T vq = var[q], cq = cov[q];
        T qx[3] = {(T)0, (T)0, (T)0};
        for (int d = 0; d < dim; ++d) qx[d] = coord(q, d);
        for (int tau = tid; tau < t; tau += NT) piv[tau] = F[(long long)tau * n + q];
        __syncthreads();
        const T rs = (T)1 / sic_sqrt(vq);
        const T ut = cq * rs;
        for (long long j = tid; j < n; j += NT) {
            if (var[j] == NEG) continue;
            T d2 = (T)0;
            for (int d = 0; d < dim; ++d) {
                T df = coord(j, d) - qx[d];
                d2 += df * df;
            }
            T num = matern<T>(kp, sic_sqrt(d2));
            if (j == q) num += kp.nugget;
            for (int tau = 0; tau < t; ++tau) num = fma(-F[(long long)tau * n + j], piv[tau], num);
            const T u = num * rs;
            F[(long long)t * n + j] = u;
            if (j == q) {
                var[j] = NEG;
            } else {
                var[j] = fma(-u, u, var[j]);
                cov[j] = fma(-u, ut, cov[j]);
            }
        }
        vt -= (double)ut * (double)ut;
        if (tid == 0) {
            out_idx[t] = (int32_t)q;
            out_var[t + 1] = vt;
        }
        __syncthreads();
    }
    if (tid == 0) *out_count = t;
    for (int q = t + tid; q < k; q += NT) out_idx[q] = -1;
}

}  // namespace

extern "C" sic_status sic_select_single_workspace(int64_t n, int32_t k, sic_precision prec, size_t* bytes) {
    if (!bytes || n < 1 || k < 1) return SIC_ERR_INVALID;
    size_t el = (prec == SIC_FP64) ? 8 : 4;
    *bytes = el * ((size_t)k * (size_t)n + 2 * (size_t)n);
    return SIC_OK;
}

extern "C" sic_status sic_select_single(sic_handle* h, const double* x_train, int64_t n, const double* x_target,
                                        const sic_kernel* kp, int32_t k, sic_precision prec, int32_t* out_idx,
                                        double* out_var, int32_t* out_count, void* ws, size_t ws_bytes,
                                        void* stream) {
    if (!h || !x_train || !x_target || !sic_valid_kernel(kp) || n < 1 || k < 1 || !out_idx || !out_var ||
        !out_count)
        return SIC_ERR_INVALID;
    if (n > 0x7fffffffLL) return SIC_ERR_UNSUPPORTED;
    size_t need = 0;
    sic_select_single_workspace(n, k, prec, &need);
    if (!ws || ws_bytes < need) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == SIC_FP64) {
        k_select_single<double><<<1, NT, sizeof(double) * k, s>>>(x_train, n, kp->dim, x_target,
                                                                   make_kp<double>(*kp), sic_floor_of(kp), k,
                                                                   out_idx, out_var, out_count, (double*)ws);
    } else if (prec == SIC_FP32_MIXED) {
        k_select_single<float><<<1, NT, sizeof(float) * k, s>>>(x_train, n, kp->dim, x_target, make_kp<float>(*kp),
                                                                 (float)sic_floor_of(kp), k, out_idx, out_var,
                                                                 out_count, (float*)ws);
    } else {
        return SIC_ERR_INVALID;
    }
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}
