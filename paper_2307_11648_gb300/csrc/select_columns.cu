// Per-column greedy conditional selection (Section 3.1 / Section 4), one persistent launch.
//
// Layout: one CTA of 256 threads owns one column at a time (columns are dealt
// round-robin over a persistent grid).  Thread tid owns candidate rows
// tid, tid + 256, ... (ROWS of them); the row's slice of the partial Cholesky
// factor F (KMAX entries), its conditional variance var_j = Theta_{jj|I} and
// covariance with the target cov_j = Theta_{tj|I} live in registers for the whole
// column.  Per step:
//   score_j = cov_j^2 / var_j (eq. obj_gp) over rows not yet picked and not exhausted;
//   argmax by warp shuffles, then across the 8 warps through shared memory
//   (ties: lowest candidate index); the winning lane publishes its F row, var, cov
//   and coordinates to a per-warp slot, so one __syncthreads per step suffices
//   (slots are double buffered by step parity);
//   every thread forms its entry of the new column
//   u_j = (Theta_{jq} - F_j . F_q) / sqrt(var_q) (left-looking, Appendix B.1),
//   then var_j -= u_j^2 and cov_j -= u_j u_t with u_t = cov_q / sqrt(var_q)
//   (eq. cond_select; the target's own row of the factor is never stored).
// FP32 mode works in coordinates relative to the target (formed in FP64) so that
// candidate-to-candidate differences keep their digits.
// With `gain` non-null, thread 0 also carries the target's variance v_t in FP64
// (v_{t+1} = v_t - u_t^2, kept at or above the exhaustion floor: the target's own nugget is
// never explained) and, after the column's last step, the threads write the picks'
// decreases of 2 KL, log(v_t / v_{t+1}) (Section 5.4.1: minus the log of one minus the
// squared conditional correlation) -- the logarithms stay off the step chain.
#include "sic_internal.cuh"

namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;

template <typename T, int KMAX>
struct Slot {
    T f[KMAX];
    T var, cov;
    T x[3];
};

template <typename T>
__device__ __forceinline__ bool better(T s, int i, T bs, int bi) {
    return s > bs || (s == bs && i < bi);
}

template <typename T, int KMAX, int ROWS>
__global__ void __launch_bounds__(NT) k_select_columns(
    const double* __restrict__ pts, long long n, int dim, KP<T> kp, T floor_, const int32_t* __restrict__ targets,
    long long n_cols, const long long* __restrict__ cand_ptr, const int32_t* __restrict__ cand_idx,
    int max_cand, int k, int32_t* __restrict__ sel_idx, int32_t* __restrict__ sel_count, double v0,
    double vfloor, double* __restrict__ gain, DevStatus* st) {
    __shared__ Slot<T, KMAX> slot[2][NW];
    __shared__ T wscore[2][NW];
    __shared__ int widx[2][NW];
    __shared__ double gv[KMAX + 1];  // target variance before each pick (gains only)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T NEG = -INFINITY;

    for (long long c = blockIdx.x; c < n_cols; c += gridDim.x) {
        const long long tgt = targets ? (long long)targets[c] : c;
        const long long b0 = cand_ptr[c];
        const int C = (int)(cand_ptr[c + 1] - b0);
        if (C < 0 || C > max_cand || C > ROWS * NT || tgt < 0 || tgt >= n) {
            if (tid == 0) {
                record_error(st, SIC_ERR_INVALID, c);
                sel_count[c] = 0;
            }
            for (int t = tid; t < k; t += NT) sel_idx[c * k + t] = -1;
            continue;
        }
        double tx[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) tx[d] = (d < dim) ? pts[tgt * dim + d] : 0.0;

        T F[ROWS][KMAX];
        T var[ROWS], cov[ROWS];
        T x[ROWS][3];
        bool live[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int row = tid + r * NT;
            live[r] = row < C;
#pragma unroll
            for (int q = 0; q < KMAX; ++q) F[r][q] = (T)0;
            x[r][0] = x[r][1] = x[r][2] = (T)0;
            var[r] = (T)0;
            cov[r] = (T)0;
            const long long p = live[r] ? (long long)cand_idx[b0 + row] : 0;
            if (live[r] && (p <= tgt || p >= n)) {
                record_error(st, SIC_ERR_INVALID, c);  // candidates must lie after the target
                live[r] = false;
            }
            if (live[r]) {
                T d2 = (T)0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (d >= dim) continue;
                    double v = pts[p * dim + d];
                    if constexpr (sizeof(T) == 8) {
                        x[r][d] = (T)v;
                        T df = (T)(v - tx[d]);
                        d2 += df * df;
                    } else {
                        x[r][d] = (T)(v - tx[d]);
                        d2 += x[r][d] * x[r][d];
                    }
                }
                var[r] = kp.s2 + kp.nugget;
                cov[r] = matern<T>(kp, sic_sqrt(d2));
            }
        }
        double vt = v0;  // target variance (thread 0, gains only)
        int t = 0;
        for (; t < k; ++t) {
            const int buf = t & 1;
            T bs = NEG;
            int bi = 0x7fffffff;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                if (live[r] && var[r] >= floor_) {
                    T s = cov[r] * cov[r] / var[r];
                    int row = tid + r * NT;
                    if (better(s, row, bs, bi)) { bs = s; bi = row; }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                T os = __shfl_xor_sync(0xffffffffu, bs, off);
                int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (better(os, oi, bs, bi)) { bs = os; bi = oi; }
            }
            if (bi != 0x7fffffff && (bi % NT) == tid) {
                // this lane owns the warp's best row: publish it (selects, not indexing,
                // so that the row arrays stay in registers)
                Slot<T, KMAX>& S = slot[buf][warp];
                const int rsel = bi / NT;
#pragma unroll
                for (int q0 = 0; q0 < KMAX; q0 += 8) {
                    if (q0 < t) {
#pragma unroll
                        for (int q = q0; q < q0 + 8; ++q) {
                            T v = F[0][q];
#pragma unroll
                            for (int r = 1; r < ROWS; ++r) v = (rsel == r) ? F[r][q] : v;
                            S.f[q] = v;
                        }
                    }
                }
                T sv = var[0], sc = cov[0], s0 = x[0][0], s1 = x[0][1], s2 = x[0][2];
#pragma unroll
                for (int r = 1; r < ROWS; ++r) {
                    const bool b = (rsel == r);
                    sv = b ? var[r] : sv;
                    sc = b ? cov[r] : sc;
                    s0 = b ? x[r][0] : s0;
                    s1 = b ? x[r][1] : s1;
                    s2 = b ? x[r][2] : s2;
                }
                S.var = sv;
                S.cov = sc;
                S.x[0] = s0;
                S.x[1] = s1;
                S.x[2] = s2;
            }
            if (lane == 0) {
                wscore[buf][warp] = bs;
                widx[buf][warp] = bi;
            }
            __syncthreads();
            T gs = wscore[buf][0];
            int gi = widx[buf][0], gw = 0;
#pragma unroll
            for (int w = 1; w < NW; ++w) {
                T s = wscore[buf][w];
                int i = widx[buf][w];
                if (better(s, i, gs, gi)) { gs = s; gi = i; gw = w; }
            }
            if (gi == 0x7fffffff || !(gs > (T)0)) break;
            const Slot<T, KMAX>& P = slot[buf][gw];
            const T d = sic_sqrt(P.var);
            const T rs = (T)1 / d;
            const T ut = P.cov * rs;
            const T px0 = P.x[0], px1 = P.x[1], px2 = P.x[2];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                if (live[r]) {
                const int row = tid + r * NT;
                T d0 = x[r][0] - px0, d1 = x[r][1] - px1, d2v = x[r][2] - px2;
                T rr = sic_sqrt(d0 * d0 + d1 * d1 + d2v * d2v);
                T num = matern<T>(kp, rr);
                if (row == gi) num += kp.nugget;
#pragma unroll
                for (int q0 = 0; q0 < KMAX; q0 += 8) {
                    if (q0 < t) {
#pragma unroll
                        for (int q = q0; q < q0 + 8; ++q) num = fma(-F[r][q], P.f[q], num);
                    }
                }
                const T u = num * rs;
#pragma unroll
                for (int q0 = 0; q0 < KMAX; q0 += 8) {
                    if (q0 <= t && t < q0 + 8) {
#pragma unroll
                        for (int q = q0; q < q0 + 8; ++q)
                            if (q == t) F[r][q] = u;
                    }
                }
                var[r] = fma(-u, u, var[r]);
                cov[r] = fma(-u, ut, cov[r]);
                if (row == gi) live[r] = false;
                }
            }
            if (tid == 0) {
                sel_idx[c * k + t] = cand_idx[b0 + gi];
                if (gain) {
                    gv[t] = vt;
                    vt = fmax(vt - (double)ut * (double)ut, vfloor);
                    gv[t + 1] = vt;
                }
            }
        }
        if (gain) {
            __syncthreads();
            for (int q = tid; q < t; q += NT) gain[c * k + q] = log(gv[q] / gv[q + 1]);
        }
        if (tid == 0) sel_count[c] = t;
        for (int q = t + tid; q < k; q += NT) sel_idx[c * k + q] = -1;
        __syncthreads();
    }
}

template <typename T, int KMAX, int ROWS>
sic_status launch_cols(sic_handle* h, const double* pts, long long n, int dim, const sic_kernel* kp, const int32_t* targets,
                       long long n_cols, const int64_t* cand_ptr, const int32_t* cand_idx, int max_cand, int k,
                       int32_t* sel_idx, int32_t* sel_count, double* gain, cudaStream_t s) {
    auto kern = k_select_columns<T, KMAX, ROWS>;
    int grid = persistent_grid(h, kern, NT, 0, n_cols);
    KP<T> p = make_kp<T>(*kp);
    kern<<<grid, NT, 0, s>>>(pts, n, dim, p, (T)sic_floor_of(kp), targets, n_cols, (const long long*)cand_ptr,
                             cand_idx, max_cand, k, sel_idx, sel_count, kp->variance + kp->nugget,
                             sic_floor_of(kp), gain, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

}  // namespace

extern "C" sic_status sic_select_columns_gain(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                              const int32_t* targets, int64_t n_cols, const int64_t* cand_ptr,
                                              const int32_t* cand_idx, int32_t max_cand, int32_t k,
                                              sic_precision prec, int32_t* sel_idx, int32_t* sel_count,
                                              double* gain, void* stream) {
    if (!h || !pts || !sic_valid_kernel(kp) || !cand_ptr || !sel_idx || !sel_count || n < 1 || n_cols < 0)
        return SIC_ERR_INVALID;
    if (k < 1 || max_cand < 0 || (n_cols > 0 && !cand_idx)) return SIC_ERR_INVALID;
    if (k > 64 || max_cand > 1024) return SIC_ERR_UNSUPPORTED;
    if (n_cols == 0) return SIC_OK;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int dim = kp->dim;
    const int kb = (k <= 16) ? 16 : (k <= 32 ? 32 : 64);
    const int rows = (max_cand <= 256) ? 1 : (max_cand <= 512 ? 2 : 4);
    if (prec == SIC_FP64) {
        if (kb == 16 && rows == 1) return launch_cols<double, 16, 1>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 16 && rows == 2) return launch_cols<double, 16, 2>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 16 && rows == 4) return launch_cols<double, 16, 4>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 32 && rows == 1) return launch_cols<double, 32, 1>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 32 && rows == 2) return launch_cols<double, 32, 2>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 64 && rows == 1) return launch_cols<double, 64, 1>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        return SIC_ERR_UNSUPPORTED;
    } else if (prec == SIC_FP32_MIXED) {
        if (kb == 16 && rows == 1) return launch_cols<float, 16, 1>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 16 && rows == 2) return launch_cols<float, 16, 2>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 16 && rows == 4) return launch_cols<float, 16, 4>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 32 && rows == 1) return launch_cols<float, 32, 1>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 32 && rows == 2) return launch_cols<float, 32, 2>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 32 && rows == 4) return launch_cols<float, 32, 4>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 64 && rows == 1) return launch_cols<float, 64, 1>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 64 && rows == 2) return launch_cols<float, 64, 2>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        return SIC_ERR_UNSUPPORTED;
    }
    return SIC_ERR_INVALID;
}

extern "C" sic_status sic_select_columns(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                         const int32_t* targets, int64_t n_cols, const int64_t* cand_ptr,
                                         const int32_t* cand_idx, int32_t max_cand, int32_t k,
                                         sic_precision prec, int32_t* sel_idx, int32_t* sel_count,
                                         void* stream) {
    return sic_select_columns_gain(h, pts, n, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, prec, sel_idx,
                                   sel_count, nullptr, stream);
}
