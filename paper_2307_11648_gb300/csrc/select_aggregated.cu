// Supernodal greedy selection (Section 5.2, multiple targets sharing one selection).
//
// One CTA (512 threads) owns one group at a time over a persistent grid.  The two
// partial Cholesky factors of the paper's Cholesky approach (Appendix C.2) live in a
// per-CTA slab of the caller's workspace, column-major with leading dimension
// ld = max_cand + max_m so that thread r touches row r of every column (coalesced):
//   F1 [k][ld]        columns of the picks, conditioned on earlier picks only;
//   F2 [max_m+k][ld]  first the m target columns (left-looking Cholesky of the
//                     targets), then the picks conditioned on targets and picks;
//   X  [3][ld]        staged coordinates (FP32 mode: relative to the first member);
//   V1, V2 [ld]       var_j = Theta_{jj|I} and var_j|P = Theta_{jj|I,P}.
// Rows 0..C-1 are the candidates, rows C..C+m-1 the targets.
// Per step the score is V1_j / V2_j (eq. greedy_mult: picking j changes
// logdet Theta_{PP|I} by log V2_j - log V1_j); the argmax (ties: lowest candidate
// index) is found by warp shuffles and one shared-memory pass; the pivot rows of F1
// and F2 are staged in shared memory and every thread appends its entries of the two
// new columns (left-looking) and downdates V1 and V2.  Picked rows are marked by
// V2 = -inf.
#include "sic_internal.cuh"

namespace {

constexpr int NT = 512;
constexpr int NW = NT / 32;

template <typename T>
__device__ __forceinline__ bool better(T s, int i, T bs, int bi) {
    return s > bs || (s == bs && i < bi);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_select_agg(
    const double* __restrict__ pts, long long n, int dim, KP<T> kp, T floor_, const long long* __restrict__ grp_ptr,
    long long n_grp, const long long* __restrict__ cand_ptr, const int32_t* __restrict__ cand_idx, int max_cand,
    int max_m, int k, int32_t* __restrict__ sel_idx, int32_t* __restrict__ sel_count, T* __restrict__ ws,
    long long ld, long long slab, DevStatus* st) {
    extern __shared__ unsigned char smem_raw[];
    T* p1 = reinterpret_cast<T*>(smem_raw);  // k
    T* p2 = p1 + k;                          // max_m + k
    __shared__ T wsc[NW];
    __shared__ int wix[NW];
    __shared__ int s_fail;

    T* F1 = ws + (long long)blockIdx.x * slab;
    T* F2 = F1 + (long long)k * ld;
    T* X = F2 + (long long)(max_m + k) * ld;
    T* V1 = X + 3 * ld;
    T* V2 = V1 + ld;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T NEG = -INFINITY;
    const T diag = kp.s2 + kp.nugget;

    for (long long g = blockIdx.x; g < n_grp; g += gridDim.x) {
        const long long g0 = grp_ptr[g];
        const int m = (int)(grp_ptr[g + 1] - g0);
        const long long b0 = cand_ptr[g];
        const int C = (int)(cand_ptr[g + 1] - b0);
        if (m < 1 || m > max_m || C < 0 || C > max_cand || g0 < 0 || g0 + m > n) {
            if (tid == 0) {
                record_error(st, SIC_ERR_INVALID, g);
                sel_count[g] = 0;
            }
            for (int q = tid; q < k; q += NT) sel_idx[g * k + q] = -1;
            continue;
        }
        const int R = C + m;
        double org[3] = {0.0, 0.0, 0.0};
        if constexpr (sizeof(T) == 4)
            for (int d = 0; d < dim; ++d) org[d] = pts[g0 * dim + d];
        for (int r = tid; r < R; r += NT) {
            long long p = (r < C) ? (long long)cand_idx[b0 + r] : g0 + (r - C);
            bool ok = true;
            if (r < C && (p < g0 + m || p >= n)) {  // candidates must lie after the group
                record_error(st, SIC_ERR_INVALID, g);
                p = g0;
                ok = false;
            }
            for (int d = 0; d < 3; ++d) X[d * ld + r] = (d < dim) ? (T)(pts[p * dim + d] - org[d]) : (T)0;
            if (r < C) {
                V1[r] = ok ? diag : NEG;
                V2[r] = ok ? diag : NEG;
            }
        }
        if (tid == 0) s_fail = 0;
        __syncthreads();

        // ---- the target columns of F2 (left-looking Cholesky of the targets) ----
        for (int a = 0; a < m; ++a) {
            const int pr = C + a;
            if (tid < a) p2[tid] = F2[(long long)tid * ld + pr];
            __syncthreads();
            T dv = diag;
            for (int b = 0; b < a; ++b) dv = fma(-p2[b], p2[b], dv);
            if (!(dv > (T)0)) {
                if (tid == 0) {
                    record_error(st, SIC_ERR_NOT_PD, g);
                    s_fail = 1;
                }
                break;
            }
            const T rs = (T)1 / sic_sqrt(dv);
            const T ax = X[pr], ay = X[ld + pr], az = X[2 * ld + pr];
            for (int r = tid; r < R; r += NT) {
                T u;
                if (r >= C && r < pr) {
                    u = (T)0;
                } else if (r == pr) {
                    u = sic_sqrt(dv);
                } else {
                    T dx = X[r] - ax, dy = X[ld + r] - ay, dz = X[2 * ld + r] - az;
                    T num = matern<T>(kp, sic_sqrt(dx * dx + dy * dy + dz * dz));
                    for (int b = 0; b < a; ++b) num = fma(-F2[(long long)b * ld + r], p2[b], num);
                    u = num * rs;
                    if (r < C) V2[r] = fma(-u, u, V2[r]);
                }
                F2[(long long)a * ld + r] = u;
            }
            __syncthreads();
        }
        __syncthreads();
        int t = 0;
        if (s_fail) {
            t = 0;
        } else {
            for (; t < k; ++t) {
                T bs = NEG;
                int bi = 0x7fffffff;
                for (int r = tid; r < C; r += NT) {
                    T v2 = V2[r];
                    if (v2 >= floor_) {
                        T s = V1[r] / v2;
                        if (better(s, r, bs, bi)) { bs = s; bi = r; }
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    T os = __shfl_xor_sync(0xffffffffu, bs, off);
                    int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                    if (better(os, oi, bs, bi)) { bs = os; bi = oi; }
                }
                if (lane == 0) {
                    wsc[warp] = bs;
                    wix[warp] = bi;
                }
                __syncthreads();
                T gs = wsc[0];
                int q = wix[0];
#pragma unroll
                for (int w = 1; w < NW; ++w)
                    if (better(wsc[w], wix[w], gs, q)) { gs = wsc[w]; q = wix[w]; }
                if (q == 0x7fffffff) break;
                const T v1q = V1[q], v2q = V2[q];
                const T qx = X[q], qy = X[ld + q], qz = X[2 * ld + q];
                for (int tau = tid; tau < t; tau += NT) p1[tau] = F1[(long long)tau * ld + q];
                for (int tau = tid; tau < m + t; tau += NT) p2[tau] = F2[(long long)tau * ld + q];
                __syncthreads();
                const T r1 = (T)1 / sic_sqrt(v1q);
                const T r2 = (T)1 / sic_sqrt(v2q);
                for (int r = tid; r < C; r += NT) {
                    if (V2[r] == NEG) continue;
                    T dx = X[r] - qx, dy = X[ld + r] - qy, dz = X[2 * ld + r] - qz;
                    T th = matern<T>(kp, sic_sqrt(dx * dx + dy * dy + dz * dz));
                    if (r == q) th += kp.nugget;
                    T n1 = th, n2 = th;
                    for (int tau = 0; tau < t; ++tau) n1 = fma(-F1[(long long)tau * ld + r], p1[tau], n1);
                    for (int tau = 0; tau < m + t; ++tau) n2 = fma(-F2[(long long)tau * ld + r], p2[tau], n2);
                    const T u1 = n1 * r1, u2 = n2 * r2;
                    F1[(long long)t * ld + r] = u1;
                    F2[(long long)(m + t) * ld + r] = u2;
                    if (r == q) {
                        V1[r] = NEG;
                        V2[r] = NEG;
                    } else {
                        V1[r] = fma(-u1, u1, V1[r]);
                        V2[r] = fma(-u2, u2, V2[r]);
                    }
                }
                if (tid == 0) sel_idx[g * k + t] = cand_idx[b0 + q];
            }
        }
        if (tid == 0) sel_count[g] = t;
        for (int q = t + tid; q < k; q += NT) sel_idx[g * k + q] = -1;
        __syncthreads();
    }
}

template <typename T>
long long slab_elems(int max_cand, int max_m, int k, long long* ld_out) {
    long long ld = max_cand + max_m;
    ld = (ld + 31) / 32 * 32;
    if (ld_out) *ld_out = ld;
    return ld * (long long)(k + max_m + k + 3 + 2);
}

template <typename T>
int agg_grid(sic_handle* h, int k, int max_m, long long n_grp) {
    size_t sm = sizeof(T) * (size_t)(k + max_m + k);
    int g = persistent_grid(h, k_select_agg<T>, NT, sm, n_grp);
    long long cap = 2LL * h->num_sms;
    if (g > cap) g = (int)cap;
    return g;
}

}  // namespace

extern "C" sic_status sic_select_aggregated_workspace(sic_handle* h, int64_t n_grp, int32_t max_cand,
                                                      int32_t max_m, int32_t k, sic_precision prec,
                                                      size_t* bytes) {
    if (!h || !bytes || n_grp < 0 || max_cand < 0 || max_m < 1 || k < 1) return SIC_ERR_INVALID;
    if (max_m > 64 || max_cand > 4096 || k > 128) return SIC_ERR_UNSUPPORTED;
    if (cudaSetDevice(h->device) != cudaSuccess) return SIC_ERR_CUDA;
    if (prec == SIC_FP64) {
        *bytes = sizeof(double) * (size_t)slab_elems<double>(max_cand, max_m, k, nullptr) *
                 (size_t)agg_grid<double>(h, k, max_m, n_grp > 0 ? n_grp : 1);
    } else if (prec == SIC_FP32_MIXED) {
        *bytes = sizeof(float) * (size_t)slab_elems<float>(max_cand, max_m, k, nullptr) *
                 (size_t)agg_grid<float>(h, k, max_m, n_grp > 0 ? n_grp : 1);
    } else {
        return SIC_ERR_INVALID;
    }
    return SIC_OK;
}

namespace {
template <typename T>
sic_status launch_agg(sic_handle* h, const double* pts, long long n, const sic_kernel* kp, const int64_t* grp_ptr, int64_t n_grp,
                      const int64_t* cand_ptr, const int32_t* cand_idx, int max_cand, int max_m, int k,
                      int32_t* sel_idx, int32_t* sel_count, void* ws, size_t ws_bytes, cudaStream_t s) {
    long long ld = 0;
    long long slab = slab_elems<T>(max_cand, max_m, k, &ld);
    int grid = agg_grid<T>(h, k, max_m, n_grp);
    if (ws_bytes < sizeof(T) * (size_t)slab * (size_t)grid || !ws) return SIC_ERR_INVALID;
    size_t sm = sizeof(T) * (size_t)(k + max_m + k);
    k_select_agg<T><<<grid, NT, sm, s>>>(pts, n, kp->dim, make_kp<T>(*kp), (T)sic_floor_of(kp),
                                         (const long long*)grp_ptr, n_grp, (const long long*)cand_ptr, cand_idx,
                                         max_cand, max_m, k, sel_idx, sel_count, (T*)ws, ld, slab, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}
}  // namespace

extern "C" sic_status sic_select_aggregated(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                            const int64_t* grp_ptr, int64_t n_grp, const int64_t* cand_ptr,
                                            const int32_t* cand_idx, int32_t max_cand, int32_t max_m, int32_t k,
                                            sic_precision prec, int32_t* sel_idx, int32_t* sel_count, void* ws,
                                            size_t ws_bytes, void* stream) {
    if (!h || !pts || !sic_valid_kernel(kp) || !grp_ptr || !cand_ptr || !sel_idx || !sel_count || n < 1 ||
        n_grp < 0 || max_cand < 0 || max_m < 1 || k < 1)
        return SIC_ERR_INVALID;
    if (max_m > 64 || max_cand > 4096 || k > 128) return SIC_ERR_UNSUPPORTED;
    if (n_grp == 0) return SIC_OK;
    if (max_cand > 0 && !cand_idx) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == SIC_FP64)
        return launch_agg<double>(h, pts, n, kp, grp_ptr, n_grp, cand_ptr, cand_idx, max_cand, max_m, k, sel_idx,
                                  sel_count, ws, ws_bytes, s);
    if (prec == SIC_FP32_MIXED)
        return launch_agg<float>(h, pts, n, kp, grp_ptr, n_grp, cand_ptr, cand_idx, max_cand, max_m, k, sel_idx,
                                 sel_count, ws, ws_bytes, s);
    return SIC_ERR_INVALID;
}
