// Partial selection for nonadjacent groups (Section 5.1.1; Section 5.2 "Partial selection";
// Appendix C.3).
//
// A group's targets P (positions i_1 < ... < i_m, not consecutive) share one selection, but a
// candidate j conditions only the targets before it (i < j).  Objective: the log-determinant
// of the partially conditioned target covariance, sum_i log Theta_{ii | s_i \ i} (eq.
// partial_kl), greedily minimised.  The state is the Cholesky factor L of the joint
// covariance of the targets and picks, columns ordered from the latest position to the
// earliest (a column's pivot is then conditioned on exactly the later points), with a row for
// every candidate and target:
//   score    thread = candidate row j: walk the columns carrying v = Theta_{jj | columns so
//            far}; a target column e with e < j gets the factor (v - L_jc^2) / v -- its
//            variance ratio after conditioning on j (eq. obj_partial) -- and v -= L_jc^2 (eq.
//            partial_induct).  The product of the factors is the exponential of minus the
//            objective's decrease; it never falls below v_last / v_0, so it cannot underflow;
//            the least product wins (ties: the earliest candidate).  A candidate whose v after
//            the last column is below the floor is exhausted.
//   insert   the pick q goes to its place p (the number of columns of later points): the
//            columns before p stay; the new column is Theta_{:,q | first p} / sqrt(Theta_{qq |
//            first p}) by left-looking; the columns from p on are downdated in place by it
//            column by column (eq. chol_partial_update): one warp forms the rotations in order
//            from the pivot rows (the targets and picks), then every candidate row applies them
//            all, with one barrier in between.
// Columns live in physical slots in insertion order; `ordr/ords/opos` map the logical
// (latest-first) order to the pivot row, the slot and the target position (INT_MAX for a
// pick).  One CTA per group (persistent), L in shared memory, rows spread over the threads.
#include <limits.h>

#include "sic_internal.cuh"

namespace {

constexpr int PT_NT = 512;

__device__ __forceinline__ float pt_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double pt_div(double a, double b) { return a / b; }

// A column's rotation from its pivot entry lee and downdate value xe: the new pivot
// rr = sqrt(lee^2 - xe^2), cos = rr / lee, sin = xe / lee and 1 / cos.  FP32 takes one fast
// reciprocal and one reciprocal square root (it sits on the insertion's serial chain); FP64
// divides exactly.
__device__ __forceinline__ bool pt_rot(float lee, float xe, float& rr, float& cth, float& sth, float& icth) {
    const float rr2 = fmaf(-xe, xe, lee * lee);
    const float irr = rsqrtf(rr2), ilee = __fdividef(1.f, lee);
    rr = rr2 * irr;
    cth = rr * ilee;
    sth = xe * ilee;
    icth = lee * irr;
    return rr2 > 0.f && lee > 0.f;
}
__device__ __forceinline__ bool pt_rot(double lee, double xe, double& rr, double& cth, double& sth, double& icth) {
    const double rr2 = fma(-xe, xe, lee * lee);
    rr = sqrt(rr2 > 0.0 ? rr2 : 0.0);
    cth = rr / lee;
    sth = xe / lee;
    icth = lee / rr;
    return rr2 > 0.0 && lee > 0.0;
}

struct PtLayout {
    int R, W, P;  // rows (candidates + targets), columns (targets + picks), row pitch (odd)
    __host__ __device__ size_t bytes(size_t tsz) const {
        return tsz * ((size_t)R * P + 4 * (size_t)R + 3 * (size_t)W) + sizeof(int) * (2 * (size_t)R + 3 * (size_t)W);
    }
};

template <typename T>
__global__ void __launch_bounds__(PT_NT, 1) k_select_partial(
    const double* __restrict__ pts, long long n, int dim, KP<T> kp, T floor_, const long long* __restrict__ grp_ptr,
    const long long* __restrict__ members, long long n_grp, const long long* __restrict__ cand_ptr,
    const int32_t* __restrict__ cand_idx, int max_cand, int max_m, int k, int32_t* __restrict__ sel_idx,
    int32_t* __restrict__ sel_count, double* __restrict__ gain, PtLayout Lay, DevStatus* st) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Lm = reinterpret_cast<T*>(smraw);              // [R][P]
    T* X = Lm + (size_t)Lay.R * Lay.P;                // [3][R] coordinates
    T* xv = X + 3 * Lay.R;                            // [R] downdate vector
    T* rc = xv + Lay.R;                               // [W] rotation of logical column c: cos,
    T* rsn = rc + Lay.W;                              //     sin,
    T* ric = rsn + Lay.W;                             //     1 / cos
    int* pos = reinterpret_cast<int*>(ric + Lay.W);   // [R] positions
    int* rank = pos + Lay.R;                          // [R] logical column of an element row, -1 otherwise
    int* ordr = rank + Lay.R;                         // [W] pivot row of logical column c
    int* ords = ordr + Lay.W;                         // [W] physical slot of logical column c
    int* opos = ords + Lay.W;                         // [W] target position of column c (INT_MAX: a pick)
    __shared__ T s_rs, s_d;
    __shared__ int s_p, s_fail;
    __shared__ T wkey[PT_NT / 32];
    __shared__ int widx[PT_NT / 32];
    __shared__ double gprod[128];
    __shared__ int gcnd[128];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int PP = Lay.P, RR = Lay.R;
    const T diag = kp.s2 + kp.nugget;
    const T INF = (T)INFINITY;

    for (long long g = blockIdx.x; g < n_grp; g += gridDim.x) {
        const long long a0 = grp_ptr[g];
        const int m = (int)(grp_ptr[g + 1] - a0);
        const long long b0 = cand_ptr[g];
        const int C = (int)(cand_ptr[g + 1] - b0);
        if (m < 1 || m > max_m || C < 0 || C > max_cand) {
            if (tid == 0) {
                record_error(st, SIC_ERR_INVALID, g);
                sel_count[g] = 0;
            }
            for (int q = tid; q < k; q += PT_NT) sel_idx[g * k + q] = -1;
            continue;
        }
        const int R = C + m;
        const long long first = members[a0];
        if (tid == 0) s_fail = (first < 0 || first >= n) ? 1 : 0;
        double org[3] = {0.0, 0.0, 0.0};
        if constexpr (sizeof(T) == 4)
            if (first >= 0 && first < n)
                for (int d = 0; d < dim; ++d) org[d] = pts[first * dim + d];
        __syncthreads();
        for (int r = tid; r < R; r += PT_NT) {
            long long p = r < C ? (long long)cand_idx[b0 + r] : members[a0 + (r - C)];
            const bool bad = p < 0 || p >= n || (r < C && p <= first) ||
                             (r > C && p <= members[a0 + (r - C) - 1]);
            if (bad) {
                s_fail = 1;
                p = 0;
            }
            pos[r] = (int)p;
            rank[r] = -1;
#pragma unroll
            for (int d = 0; d < 3; ++d) X[d * RR + r] = (d < dim) ? (T)(pts[p * dim + d] - org[d]) : (T)0;
        }
        __syncthreads();
        if (s_fail) {
            if (tid == 0) {
                record_error(st, SIC_ERR_INVALID, g);
                sel_count[g] = 0;
            }
            for (int q = tid; q < k; q += PT_NT) sel_idx[g * k + q] = -1;
            __syncthreads();
            continue;
        }

        int ncol = 0;
        // inserts row q's point: place p, left-looking column into slot ncol, in-place
        // downdate of the columns from p on; false (uniformly) when a pivot is not positive
        auto insert = [&](int q) -> bool {
            if (warp == 0) {
                // its place: binary search of the columns (positions descending)
                int p = 0;
                if (lane == 0) {
                    int lo = 0, hi = ncol;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (pos[ordr[mid]] > pos[q]) lo = mid + 1; else hi = mid;
                    }
                    p = lo;
                }
                p = __shfl_sync(0xffffffffu, p, 0);
                T part = (T)0;
                for (int c = lane; c < p; c += 32) {
                    const T l = Lm[q * PP + ords[c]];
                    part = fma(l, l, part);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
                if (lane == 0) {
                    const T d = diag - part;  // Theta_{qq | first p}
                    s_p = p;
                    s_d = d;
                    if (!(d > (T)0)) s_fail = 2;
                    s_rs = (d > (T)0) ? (T)1 / sic_sqrt(d) : (T)0;
                }
            }
            __syncthreads();
            if (s_fail) return false;
            const int p = s_p;
            const T rs = s_rs;
            const T qx = X[q], qy = X[RR + q], qz = X[2 * RR + q];
            for (int r = tid; r < R; r += PT_NT) {
                const int rk = rank[r];
                T u = (T)0;
                if (r == q) {
                    u = s_d * rs;  // sqrt(d)
                } else if (rk < 0 || rk >= p) {
                    const T dx = X[r] - qx, dy = X[RR + r] - qy, dz = X[2 * RR + r] - qz;
                    T num = matern<T>(kp, sic_sqrt(dx * dx + dy * dy + dz * dz));
                    for (int c = 0; c < p; ++c) num = fma(-Lm[r * PP + ords[c]], Lm[q * PP + ords[c]], num);
                    u = num * rs;
                }
                Lm[r * PP + ncol] = u;
                xv[r] = (r == q) ? (T)0 : u;
            }
            __syncthreads();
            // the downdate of the columns from p on, in two phases.  (1) Warp 0 forms the
            // columns' rotations in order from the pivot rows alone -- the rows of the targets and
            // picks at earlier positions than q, which are the pivots of those same columns --
            // each lane carrying a few of those rows; the rotations go to shared memory.  (2)
            // Every other row below (the candidates) applies them in order, with no barrier
            // between columns.
            if (warp == 0) {
                bool bad = false;
                for (int c = p; c < ncol; ++c) {
                    const int e = ordr[c], s = ords[c];
                    T rr, cth, sth, icth;
                    bad = !pt_rot(Lm[e * PP + s], xv[e], rr, cth, sth, icth) || bad;
                    __syncwarp();  // every lane has read the pivot's entries
                    if (lane == 0) {
                        rc[c] = cth;
                        rsn[c] = sth;
                        ric[c] = icth;
                        Lm[e * PP + s] = rr;
                    }
                    for (int c2 = c + 1 + lane; c2 < ncol; c2 += 32) {
                        const int r = ordr[c2];
                        const T xr = xv[r];
                        const T nl = (Lm[r * PP + s] - sth * xr) * icth;
                        Lm[r * PP + s] = nl;
                        xv[r] = cth * xr - sth * nl;
                    }
                    __syncwarp();  // the next pivot row is final
                }
                if (bad && lane == 0) s_fail = 2;
            }
            __syncthreads();
            if (s_fail) return false;
            for (int r = tid; r < R; r += PT_NT) {
                if (rank[r] >= 0 || r == q) continue;
                T xr = xv[r];
                for (int c = p; c < ncol; ++c) {
                    const int s = ords[c];
                    const T nl = (Lm[r * PP + s] - rsn[c] * xr) * ric[c];
                    Lm[r * PP + s] = nl;
                    xr = rc[c] * xr - rsn[c] * nl;
                }
            }
            __syncthreads();
            // row q now holds a pivot: nothing in the columns after its own; the column maps
            // shift one place from p on (each thread carries one entry across the barrier)
            for (int c = p + tid; c < ncol; c += PT_NT) Lm[q * PP + ords[c]] = (T)0;
            const int cm = p + 1 + tid;  // the new index of the entry this thread moves
            int mr = 0, ms = 0, mp = 0;
            if (cm <= ncol) {
                mr = ordr[cm - 1];
                ms = ords[cm - 1];
                mp = opos[cm - 1];
            }
            __syncthreads();
            if (cm <= ncol) {
                ordr[cm] = mr;
                ords[cm] = ms;
                opos[cm] = mp;
            }
            if (tid == 0) {
                ordr[p] = q;
                ords[p] = ncol;
                opos[p] = (q >= C) ? pos[q] : INT_MAX;
            }
            for (int r = tid; r < R; r += PT_NT) {
                if (r == q) rank[r] = p;
                else if (rank[r] >= p) rank[r] += 1;
            }
            __syncthreads();
            ++ncol;
            return true;
        };

        bool ok = true;
        // the targets, latest first: each lands after every column so far (no downdate)
        for (int a = m - 1; a >= 0 && ok; --a) ok = insert(C + a);
        int t = 0;
        for (; t < k && ok; ++t) {
            T bk = INF;
            int bi = INT_MAX;
            for (int j = tid; j < C; j += PT_NT) {
                if (rank[j] >= 0) continue;
                const int pj = pos[j];
                T v = diag, pr = (T)1;
                for (int c = 0; c < ncol; ++c) {
                    const T l = Lm[j * PP + ords[c]];
                    const T vn = fma(-l, l, v);
                    if (opos[c] < pj) pr = pt_div(pr * vn, v);  // a target j conditions (eq. obj_partial)
                    v = vn;                              // eq. partial_induct
                }
                if (v >= floor_ && (pr < bk || (pr == bk && j < bi))) {
                    bk = pr;
                    bi = j;
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T ok_ = __shfl_xor_sync(0xffffffffu, bk, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ok_ < bk || (ok_ == bk && oi < bi)) {
                    bk = ok_;
                    bi = oi;
                }
            }
            if (lane == 0) {
                wkey[warp] = bk;
                widx[warp] = bi;
            }
            __syncthreads();
            T gk = wkey[0];
            int q = widx[0];
#pragma unroll
            for (int w = 1; w < PT_NT / 32; ++w)
                if (wkey[w] < gk || (wkey[w] == gk && widx[w] < q)) {
                    gk = wkey[w];
                    q = widx[w];
                }
            if (q == INT_MAX) break;
            // the targets the pick conditions (its nonzeros)
            const int nc = __syncthreads_count(tid < ncol && opos[tid] < pos[q]);
            if (tid == 0) {
                gprod[t] = (double)gk;
                gcnd[t] = nc;
                sel_idx[g * k + t] = pos[q];
            }
            ok = insert(q);
            if (!ok) break;
        }
        if (!ok && tid == 0) record_error(st, SIC_ERR_NOT_PD, g);
        if (tid == 0) sel_count[g] = t;
        for (int q = t + tid; q < k; q += PT_NT) sel_idx[g * k + q] = -1;
        if (gain) {
            __syncthreads();
            // decrease of the objective per nonzero (the targets the pick conditions)
            for (int q = tid; q < t; q += PT_NT) gain[g * k + q] = -log(gprod[q]) / (gcnd[q] > 0 ? gcnd[q] : 1);
        }
        __syncthreads();
    }
}

// Per-column selection lists of nonadjacent groups for the fill: member i's column holds the
// later members and the picks after i (Section 5.1.1); one warp per group.
__global__ void k_partial_columns(long long n, const long long* __restrict__ grp_ptr,
                                  const long long* __restrict__ members, long long n_grp,
                                  const int32_t* __restrict__ sel_idx, const int32_t* __restrict__ sel_count, int k,
                                  int kc, int32_t* __restrict__ col_sel, int32_t* __restrict__ col_count,
                                  DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_grp; g += nw) {
        const long long a0 = grp_ptr[g], a1 = grp_ptr[g + 1];
        int cnt = sel_count[g];
        if (cnt < 0 || cnt > k) {
            if (lane == 0) record_error(st, SIC_ERR_INVALID, g);
            cnt = 0;
        }
        for (long long a = a0 + lane; a < a1; a += 32) {
            const long long i = members[a];
            if (i < 0 || i >= n) {
                record_error(st, SIC_ERR_INVALID, g);
                continue;
            }
            if (!col_sel) {  // counts only
                int w = (int)(a1 - a - 1);
                for (int t = 0; t < cnt; ++t) w += sel_idx[g * k + t] > i;
                col_count[i] = w;
                continue;
            }
            int w = 0;
            int32_t* out = col_sel + i * kc;
            for (long long b = a + 1; b < a1 && w < kc; ++b) out[w++] = (int32_t)members[b];
            for (int t = 0; t < cnt && w < kc; ++t) {
                const int32_t q = sel_idx[g * k + t];
                if (q > i) out[w++] = q;
            }
            if ((a1 - a - 1) + cnt > kc && w == kc) record_error(st, SIC_ERR_INVALID, g);
            col_count[i] = w;
        }
    }
}

}  // namespace

extern "C" sic_status sic_select_partial(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                         const int64_t* grp_ptr, const int64_t* members, int64_t n_grp,
                                         const int64_t* cand_ptr, const int32_t* cand_idx, int32_t max_cand,
                                         int32_t max_m, int32_t k, sic_precision prec, int32_t* sel_idx,
                                         int32_t* sel_count, double* gain, void* stream) {
    if (!h || !pts || !sic_valid_kernel(kp) || !grp_ptr || !members || !cand_ptr || !sel_idx || !sel_count ||
        n < 1 || n_grp < 0 || max_cand < 0 || max_m < 1 || k < 1)
        return SIC_ERR_INVALID;
    if (k > 128 || max_m > 64 || n > INT_MAX) return SIC_ERR_UNSUPPORTED;
    if (n_grp == 0) return SIC_OK;
    if (max_cand > 0 && !cand_idx) return SIC_ERR_INVALID;
    PtLayout L;
    L.R = max_cand + max_m;
    L.W = max_m + k;
    L.P = L.W | 1;
    const size_t smem = L.bytes(prec == SIC_FP64 ? sizeof(double) : sizeof(float));
    if (smem > 227 * 1024 - 4096) return SIC_ERR_UNSUPPORTED;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const long long* gp = (const long long*)grp_ptr;
    const long long* mb = (const long long*)members;
    const long long* cp = (const long long*)cand_ptr;
    if (prec == SIC_FP64) {
        auto kern = k_select_partial<double>;
        SIC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int grid = persistent_grid(h, kern, PT_NT, smem, n_grp);
        kern<<<grid, PT_NT, smem, s>>>(pts, n, kp->dim, make_kp<double>(*kp), sic_floor_of(kp), gp, mb, n_grp, cp,
                                       cand_idx, max_cand, max_m, k, sel_idx, sel_count, gain, L, h->d_status);
    } else if (prec == SIC_FP32_MIXED) {
        auto kern = k_select_partial<float>;
        SIC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int grid = persistent_grid(h, kern, PT_NT, smem, n_grp);
        kern<<<grid, PT_NT, smem, s>>>(pts, n, kp->dim, make_kp<float>(*kp), (float)sic_floor_of(kp), gp, mb, n_grp,
                                       cp, cand_idx, max_cand, max_m, k, sel_idx, sel_count, gain, L, h->d_status);
    } else {
        return SIC_ERR_INVALID;
    }
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_partial_columns(sic_handle* h, int64_t n, const int64_t* grp_ptr, const int64_t* members,
                                          int64_t n_grp, const int32_t* sel_idx, const int32_t* sel_count, int32_t k,
                                          int32_t kc, int32_t* col_sel, int32_t* col_count, void* stream) {
    if (!h || n < 1 || n_grp < 0 || k < 1 || kc < 1 || !grp_ptr || !members || !sel_idx || !sel_count || !col_count)
        return SIC_ERR_INVALID;
    if (n_grp == 0) return SIC_OK;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    const int grid = persistent_grid(h, k_partial_columns, 256, 0, (n_grp + 7) / 8);
    k_partial_columns<<<grid, 256, 0, (cudaStream_t)stream>>>(n, (const long long*)grp_ptr,
                                                              (const long long*)members, n_grp, sel_idx, sel_count, k,
                                                              kc, col_sel, col_count, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}
