// Directed GP regression (Section 3): the posterior of the latent process at each target
// from the training points its directed selection picked, in FP64.
//
//   G G^T = Theta_{I,I} (nugget on its diagonal),  z = G^-1 Theta_{I,t},  u = G^-1 y_I,
//   mean = z . u = Theta_{t,I} Theta_{I,I}^-1 y_I,  var = variance - z . z.
//
// One warp per target (several independent warps per CTA, no block barriers): the warp
// forms Theta_{I,I} in packed lower storage in shared memory (one entry per lane),
// factors it left-looking (lane = row; the pivot's square root taken once and broadcast
// by shuffle), and runs both forward substitutions together with the right-hand sides in
// registers.  Kernel entries use the FP64 Matern of the fill (matern_d2_fast).
#include "sic_internal.cuh"

namespace {

constexpr int GP_MAXK = 128;
constexpr int GP_SLOTS = GP_MAXK / 32;  // rows per lane

__device__ __forceinline__ int gpk(int i, int j) { return i * (i + 1) / 2 + j; }

__device__ __forceinline__ int gpk_row(int e) {
    int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (i * (i + 1) / 2 > e) --i;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    return i;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__global__ void k_gp_predict(const double* __restrict__ pts, long long n, int dim, KP<double> kp,
                             const int32_t* __restrict__ targets, long long n_targets,
                             const int32_t* __restrict__ sel_idx, const int32_t* __restrict__ sel_count, int k,
                             const double* __restrict__ y, double* __restrict__ mean, double* __restrict__ var,
                             DevStatus* st) {
    extern __shared__ double gsm[];
    double* tab = gsm;  // variance * 2^(j/256), shared by the warps
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per_warp = k * (k + 1) / 2 + 3 * k;
    double* G = gsm + EXP_TAB + (size_t)warp * per_warp;  // packed lower k x k
    double* xyz = G + k * (k + 1) / 2;                      // 3 x k coordinates of the picks
    exp_table_fill(tab, kp.s2);
    __syncthreads();
    const double NaN = __longlong_as_double(0x7ff8000000000000LL);

    for (long long t = (long long)blockIdx.x * nw + warp; t < n_targets; t += (long long)gridDim.x * nw) {
        const long long tp = targets ? (long long)targets[t] : t;
        const int cnt = sel_count[t];
        bool bad = tp < 0 || tp >= n || cnt < 0 || cnt > k;
        double tx = 0.0, ty = 0.0, tz = 0.0;
        if (!bad) {
            tx = pts[tp * dim];
            if (dim > 1) ty = pts[tp * dim + 1];
            if (dim > 2) tz = pts[tp * dim + 2];
        }
        // coordinates of the picks, Theta_{I,t} and y_I in the lanes' row slots
        double th[GP_SLOTS], yy[GP_SLOTS];
#pragma unroll
        for (int h = 0; h < GP_SLOTS; ++h) {
            const int i = lane + 32 * h;
            th[h] = 0.0;
            yy[h] = 0.0;
            if (!bad && i < cnt) {
                const long long p = sel_idx[t * k + i];
                if (p < 0 || p >= n || p == tp) {
                    bad = true;
                } else {
                    const double px = pts[p * dim], py = dim > 1 ? pts[p * dim + 1] : 0.0,
                                 pz = dim > 2 ? pts[p * dim + 2] : 0.0;
                    xyz[i] = px;
                    xyz[k + i] = py;
                    xyz[2 * k + i] = pz;
                    const double dx = px - tx, dy = py - ty, dz = pz - tz;
                    th[h] = matern_d2_fast(kp, fma(dz, dz, fma(dy, dy, dx * dx)), tab);
                    yy[h] = y[p];
                }
            }
        }
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) {
                record_error(st, SIC_ERR_INVALID, t);
                if (t >= 0) {
                    mean[t] = NaN;
                    var[t] = NaN;
                }
            }
            continue;
        }
        __syncwarp();
        // Theta_{I,I}, packed lower, one entry per lane
        const int tri = cnt * (cnt + 1) / 2;
        for (int e = lane; e < tri; e += 32) {
            const int i = gpk_row(e), j = e - i * (i + 1) / 2;
            const double dx = xyz[i] - xyz[j], dy = xyz[k + i] - xyz[k + j], dz = xyz[2 * k + i] - xyz[2 * k + j];
            double v = matern_d2_fast(kp, fma(dz, dz, fma(dy, dy, dx * dx)), tab);
            if (i == j) v += kp.nugget;
            G[e] = v;
        }
        __syncwarp();
        // left-looking Cholesky, lane = rows lane + 32 h
        bool pd = true;
        for (int j = 0; j < cnt; ++j) {
            double sv[GP_SLOTS];
#pragma unroll
            for (int h = 0; h < GP_SLOTS; ++h) {
                const int i = lane + 32 * h;
                sv[h] = 0.0;
                if (i >= j && i < cnt) {
                    const int ri = gpk(i, 0), rj = gpk(j, 0);
                    double s0 = G[ri + j], s1 = 0.0;
                    int l = 0;
                    for (; l + 2 <= j; l += 2) {
                        s0 = fma(-G[ri + l], G[rj + l], s0);
                        s1 = fma(-G[ri + l + 1], G[rj + l + 1], s1);
                    }
                    if (l < j) s0 = fma(-G[ri + l], G[rj + l], s0);
                    sv[h] = s0 + s1;
                }
            }
            double sjj = 0.0;
#pragma unroll
            for (int h = 0; h < GP_SLOTS; ++h) {
                const double o = __shfl_sync(0xffffffffu, sv[h], j & 31);
                if (h == (j >> 5)) sjj = o;
            }
            if (!(sjj > 0.0)) {
                pd = false;
                break;
            }
            const double rd = rsqrt_newton(sjj);
#pragma unroll
            for (int h = 0; h < GP_SLOTS; ++h) {
                const int i = lane + 32 * h;
                if (i > j && i < cnt) G[gpk(i, j)] = sv[h] * rd;
                if (i == j) G[gpk(j, j)] = sjj * rd;
            }
            __syncwarp();
        }
        if (!pd) {
            if (lane == 0) {
                record_error(st, SIC_ERR_NOT_PD, t);
                mean[t] = NaN;
                var[t] = NaN;
            }
            continue;
        }
        // forward substitutions G z = Theta_{I,t} and G u = y_I, column by column
        for (int j = 0; j < cnt; ++j) {
            double zj = 0.0, uj = 0.0;
#pragma unroll
            for (int h = 0; h < GP_SLOTS; ++h) {
                const double oz = __shfl_sync(0xffffffffu, th[h], j & 31);
                const double ou = __shfl_sync(0xffffffffu, yy[h], j & 31);
                if (h == (j >> 5)) {
                    zj = oz;
                    uj = ou;
                }
            }
            const double rjj = 1.0 / G[gpk(j, j)];
            zj *= rjj;
            uj *= rjj;
#pragma unroll
            for (int h = 0; h < GP_SLOTS; ++h) {
                const int i = lane + 32 * h;
                if (i == j) {
                    th[h] = zj;
                    yy[h] = uj;
                } else if (i > j && i < cnt) {
                    const double g = G[gpk(i, j)];
                    th[h] = fma(-g, zj, th[h]);
                    yy[h] = fma(-g, uj, yy[h]);
                }
            }
        }
        double zu = 0.0, zz = 0.0;
#pragma unroll
        for (int h = 0; h < GP_SLOTS; ++h)
            if (lane + 32 * h < cnt) {
                zu = fma(th[h], yy[h], zu);
                zz = fma(th[h], th[h], zz);
            }
        zu = warp_sum(zu);
        zz = warp_sum(zz);
        if (lane == 0) {
            mean[t] = zu;
            var[t] = kp.s2 - zz;
        }
        __syncwarp();
    }
}

}  // namespace

extern "C" sic_status sic_gp_predict(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                     const int32_t* targets, int64_t n_targets, const int32_t* sel_idx,
                                     const int32_t* sel_count, int32_t k, const double* y, double* mean,
                                     double* var, void* stream) {
    if (!h || !pts || !sic_valid_kernel(kp) || n < 1 || n_targets < 0 || !sel_idx || !sel_count || !y || !mean ||
        !var || k < 1)
        return SIC_ERR_INVALID;
    if (k > GP_MAXK) return SIC_ERR_UNSUPPORTED;
    if (n_targets == 0) return SIC_OK;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    const size_t per_warp = sizeof(double) * ((size_t)k * (k + 1) / 2 + 3 * (size_t)k);
    int warps = (int)((200 * 1024 - sizeof(double) * EXP_TAB) / per_warp);
    if (warps > 8) warps = 8;
    if (warps < 1) warps = 1;
    const size_t smem = sizeof(double) * EXP_TAB + per_warp * warps;
    SIC_CUDA_TRY(cudaFuncSetAttribute(k_gp_predict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    long long work = (n_targets + warps - 1) / warps;
    const int grid = persistent_grid(h, k_gp_predict, 32 * warps, smem, work);
    k_gp_predict<<<grid, 32 * warps, smem, (cudaStream_t)stream>>>(pts, n, kp->dim, make_kp<double>(*kp), targets,
                                                                   n_targets, sel_idx, sel_count, k, y, mean, var,
                                                                   h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}
