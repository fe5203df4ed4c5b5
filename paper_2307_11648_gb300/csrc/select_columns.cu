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
// k_select_columns serves FP64 (it evaluates Theta with the fill's table-driven exp and
// Newton square root, and 1/sqrt(var_q) by Newton steps); FP32 runs k_select_columns_f32
// below, which works in coordinates relative to the target (formed in FP64) so that
// candidate-to-candidate differences keep their digits, and reads the pivot's row from a
// shared-memory mirror instead of a published slot.
// With `gain` non-null, thread 0 also carries the target's variance v_t in FP64
// (v_{t+1} = v_t - u_t^2, kept at or above the exhaustion floor: the target's own nugget is
// never explained) and, after the column's last step, the threads write the picks'
// decreases of 2 KL, log(v_t / v_{t+1}) (Section 5.4.1: minus the log of one minus the
// squared conditional correlation) -- the logarithms stay off the step chain.
#include <type_traits>

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
    __shared__ int qs[KMAX];         // the picks' candidate rows, translated after the steps
    __shared__ double tab[sizeof(T) == 8 ? EXP_TAB : 1];  // s2 2^(j/256): the FP64 Matern's exp

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T NEG = -INFINITY;
    if constexpr (sizeof(T) == 8) {
        exp_table_fill(tab, kp.s2);
        __syncthreads();
    }
    // Theta at squared distance d2 (no nugget): in FP64 the table-driven exp and the Newton
    // square root (few FP64-pipe operations, about 2 ulp)
    auto theta = [&](T d2) -> T {
        if constexpr (sizeof(T) == 8)
            return matern_d2_fast(kp, d2, tab);
        else
            return matern<T>(kp, sic_sqrt(d2));
    };

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
                cov[r] = theta(d2);
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
            T rs;
            if constexpr (sizeof(T) == 8)
                rs = rsqrt_newton(P.var);
            else
                rs = (T)1 / sic_sqrt(P.var);
            const T ut = P.cov * rs;
            const T px0 = P.x[0], px1 = P.x[1], px2 = P.x[2];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                if (live[r]) {
                const int row = tid + r * NT;
                T d0 = x[r][0] - px0, d1 = x[r][1] - px1, d2v = x[r][2] - px2;
                T num = theta(fma(d2v, d2v, fma(d1, d1, d0 * d0)));
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
                qs[t] = gi;  // no global load on the step chain
                if (gain) {
                    gv[t] = vt;
                    vt = fmax(vt - (double)ut * (double)ut, vfloor);
                    gv[t + 1] = vt;
                }
            }
        }
        __syncthreads();
        for (int q = tid; q < t; q += NT) {
            sel_idx[c * k + q] = cand_idx[b0 + qs[q]];
            if (gain) gain[c * k + q] = log(gv[q] / gv[q + 1]);
        }
        if (tid == 0) sel_count[c] = t;
        for (int q = t + tid; q < k; q += NT) sel_idx[c * k + q] = -1;
        __syncthreads();
    }
}

// ---- FP32: the same selection with the factor rows mirrored in shared memory ----
//
// Thread rows and the per-step arithmetic are those of k_select_columns; what changes is how
// the pivot reaches the other threads and how a row's factor entries are kept.  Every thread
// writes its new factor entry of each step into a shared-memory mirror of all rows (row pitch
// KMAX + 4 floats, zeroed at the column's start), so after the step's barrier every thread
// reads the pivot's row straight from the mirror as broadcast 16-byte words: the winning lane
// no longer copies its row into a slot.  The steps run in blocks of 8 with the block index a
// compile-time constant: the dot products take the completed blocks from registers and the
// current block from the row's own mirror, and a completed block moves into registers, so no
// register is indexed by the step and no predicated select touches the whole row.  The
// pivot's coordinates sit beside the mirror (one float4 per row, written once per column).  The warp argmax is two redux operations on order-preserving
// score keys (the maximum, then the lowest candidate index among the lanes holding it), and
// the eight warp winners are reduced the same way by every warp (lane w reads warp w's).  Scores use the fast FP32 divide,
// the pivot's 1/sqrt(var) and the distances the hardware reciprocal square root (about 2 ulp,
// far inside the tolerance of FP32 selection).
template <int KMAX>
__host__ __device__ constexpr int mirror_pitch() { return KMAX + 4; }

template <int KMAX, int ROWS>
constexpr size_t mirror_bytes() {
    return sizeof(float) * (size_t)ROWS * NT * (size_t)(mirror_pitch<KMAX>() + 4);
}

// f(integral_constant<B>), B = B0 .. NB-1, in order
template <int B, int NB, typename Fn>
__device__ __forceinline__ void static_for(Fn& f) {
    if constexpr (B < NB) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, NB>(f);
    }
}

__device__ __forceinline__ unsigned col_score_key(float s) {
    return (s >= 0.f) ? (__float_as_uint(s) | 0x80000000u) : 0u;  // 0: not a candidate (or NaN)
}

__device__ __forceinline__ float matern_f32_d2(const KP<float>& k, float d2) {
    return matern<float>(k, d2 > 1e-30f ? d2 * rsqrtf(d2) : 0.f);
}

template <int KMAX, int ROWS>
__global__ void __launch_bounds__(NT) k_select_columns_f32(
    const double* __restrict__ pts, long long n, int dim, KP<float> kp, float floor_,
    const int32_t* __restrict__ targets, long long n_cols, const long long* __restrict__ cand_ptr,
    const int32_t* __restrict__ cand_idx, int max_cand, int k, int32_t* __restrict__ sel_idx,
    int32_t* __restrict__ sel_count, double v0, double vfloor, double* __restrict__ gain, DevStatus* st) {
    constexpr int P = mirror_pitch<KMAX>();
    extern __shared__ float4 sm4[];
    float* Fm = reinterpret_cast<float*>(sm4);  // [ROWS * NT][P]
    float4* Xm = sm4 + ROWS * NT * P / 4;       // [ROWS * NT] coordinates relative to the target
    __shared__ unsigned wkey[2][NW];
    __shared__ int widx[2][NW];
    __shared__ float wvar[2][NW], wcov[2][NW];
    __shared__ double gv[KMAX + 1];  // target variance before each pick (gains only)
    __shared__ int qs[KMAX];         // the picks' candidate rows, translated after the steps
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr unsigned FULL = 0xffffffffu;

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

        float F[ROWS][KMAX];
        float var[ROWS], cov[ROWS];
        float x[ROWS][3];
        bool live[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int row = tid + r * NT;
            live[r] = row < C;
#pragma unroll
            for (int q = 0; q < KMAX; ++q) F[r][q] = 0.f;
#pragma unroll
            for (int q = 0; q < P; q += 4)
                *reinterpret_cast<float4*>(Fm + row * P + q) = make_float4(0.f, 0.f, 0.f, 0.f);
            x[r][0] = x[r][1] = x[r][2] = 0.f;
            var[r] = 0.f;
            cov[r] = 0.f;
            const long long p = live[r] ? (long long)cand_idx[b0 + row] : 0;
            if (live[r] && (p <= tgt || p >= n)) {
                record_error(st, SIC_ERR_INVALID, c);  // candidates must lie after the target
                live[r] = false;
            }
            if (live[r]) {
                float d2 = 0.f;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (d >= dim) continue;
                    x[r][d] = (float)(pts[p * dim + d] - tx[d]);
                    d2 += x[r][d] * x[r][d];
                }
                var[r] = kp.s2 + kp.nugget;
                cov[r] = matern_f32_d2(kp, d2);
            }
            Xm[row] = make_float4(x[r][0], x[r][1], x[r][2], 0.f);
        }
        double vt = v0;  // target variance (thread 0, gains only)
        int t = 0;
        bool go = true;
        // the k steps in blocks of 8: within block TB, step t = 8 TB + tt appends entry t; the
        // dot products take the completed blocks 0..TB-1 from registers and block TB from the
        // row's own mirror (entries from t on are zero on both sides); after the block's steps
        // the block moves from the mirror into registers -- all register indices static
        auto block = [&](auto tbc) {
            constexpr int TB = decltype(tbc)::value;
            for (int tt = 0; tt < 8 && go; ++tt, ++t) {
                if (t >= k) {
                    go = false;
                    break;
                }
                const int buf = t & 1;
                unsigned bk = 0u;
                int bi = 0x7fffffff;
                float bv = 0.f, bc = 0.f;
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {  // rows ascend with r: strict > keeps the lowest on ties
                    const unsigned key =
                        (live[r] && var[r] >= floor_) ? col_score_key(__fdividef(cov[r] * cov[r], var[r])) : 0u;
                    if (key > bk) {
                        bk = key;
                        bi = tid + r * NT;
                        bv = var[r];
                        bc = cov[r];
                    }
                }
                const unsigned wmax = __reduce_max_sync(FULL, bk);
                const int wi = (int)__reduce_min_sync(FULL, (bk == wmax) ? (unsigned)bi : 0x7fffffffu);
                const unsigned hit = __ballot_sync(FULL, bi == wi && bk == wmax);
                if (lane == __ffs(hit) - 1) {  // the warp's best row (one lane)
                    wkey[buf][warp] = wmax;
                    widx[buf][warp] = wi;
                    wvar[buf][warp] = bv;
                    wcov[buf][warp] = bc;
                }
                __syncthreads();
                // the eight warp winners, reduced by every warp: lane w < 8 holds warp w's
                const unsigned kw = (lane < NW) ? wkey[buf][lane] : 0u;
                const int iw = (lane < NW) ? widx[buf][lane] : 0x7fffffff;
                const unsigned gk = __reduce_max_sync(FULL, kw);
                const int gi = (int)__reduce_min_sync(FULL, (kw == gk) ? (unsigned)iw : 0x7fffffffu);
                if (gk <= 0x80000000u) {  // no candidate left, or the best score is 0
                    go = false;
                    break;
                }
                const int gw = __ffs(__ballot_sync(FULL, lane < NW && kw == gk && iw == gi)) - 1;
                const float rs = rsqrtf(wvar[buf][gw]);
                const float ut = wcov[buf][gw] * rs;
                const float4 px = Xm[gi];
                const float* Fp = Fm + gi * P;
                const float4 c0 = *reinterpret_cast<const float4*>(Fp + 8 * TB);
                const float4 c1 = *reinterpret_cast<const float4*>(Fp + 8 * TB + 4);
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    if (live[r]) {
                        const int row = tid + r * NT;
                        const float d0 = x[r][0] - px.x, d1 = x[r][1] - px.y, d2v = x[r][2] - px.z;
                        float num = matern_f32_d2(kp, fmaf(d2v, d2v, fmaf(d1, d1, d0 * d0)));
                        if (row == gi) num += kp.nugget;
                        float a1 = 0.f;
#pragma unroll
                        for (int q = 0; q < 8 * TB; q += 4) {
                            const float4 p = *reinterpret_cast<const float4*>(Fp + q);
                            num = fmaf(-F[r][q], p.x, num);
                            a1 = fmaf(-F[r][q + 1], p.y, a1);
                            num = fmaf(-F[r][q + 2], p.z, num);
                            a1 = fmaf(-F[r][q + 3], p.w, a1);
                        }
                        const float* Fo = Fm + row * P + 8 * TB;
                        const float4 o0 = *reinterpret_cast<const float4*>(Fo);
                        const float4 o1 = *reinterpret_cast<const float4*>(Fo + 4);
                        num = fmaf(-o0.x, c0.x, num);
                        a1 = fmaf(-o0.y, c0.y, a1);
                        num = fmaf(-o0.z, c0.z, num);
                        a1 = fmaf(-o0.w, c0.w, a1);
                        num = fmaf(-o1.x, c1.x, num);
                        a1 = fmaf(-o1.y, c1.y, a1);
                        num = fmaf(-o1.z, c1.z, num);
                        a1 = fmaf(-o1.w, c1.w, a1);
                        const float u = (num + a1) * rs;
                        // the pivot's own row is never read again (and is being read this step)
                        if (row != gi) Fm[row * P + t] = u;
                        var[r] = fmaf(-u, u, var[r]);
                        cov[r] = fmaf(-u, ut, cov[r]);
                        if (row == gi) live[r] = false;
                    }
                }
                if (tid == 0) {
                    qs[t] = gi;  // no global load on the step chain
                    if (gain) {
                        gv[t] = vt;
                        vt = fmax(vt - (double)ut * (double)ut, vfloor);
                        gv[t + 1] = vt;
                    }
                }
            }
            if (go) {
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    const float* Fo = Fm + (tid + r * NT) * P + 8 * TB;
                    const float4 o0 = *reinterpret_cast<const float4*>(Fo);
                    const float4 o1 = *reinterpret_cast<const float4*>(Fo + 4);
                    F[r][8 * TB + 0] = o0.x;
                    F[r][8 * TB + 1] = o0.y;
                    F[r][8 * TB + 2] = o0.z;
                    F[r][8 * TB + 3] = o0.w;
                    F[r][8 * TB + 4] = o1.x;
                    F[r][8 * TB + 5] = o1.y;
                    F[r][8 * TB + 6] = o1.z;
                    F[r][8 * TB + 7] = o1.w;
                }
            }
        };
        static_for<0, KMAX / 8>(block);
        __syncthreads();
        for (int q = tid; q < t; q += NT) {
            sel_idx[c * k + q] = cand_idx[b0 + qs[q]];
            if (gain) gain[c * k + q] = log(gv[q] / gv[q + 1]);
        }
        if (tid == 0) sel_count[c] = t;
        for (int q = t + tid; q < k; q += NT) sel_idx[c * k + q] = -1;
        __syncthreads();
    }
}

template <int KMAX, int ROWS>
sic_status launch_cols_f32(sic_handle* h, const double* pts, long long n, int dim, const sic_kernel* kp,
                           const int32_t* targets, long long n_cols, const int64_t* cand_ptr, const int32_t* cand_idx,
                           int max_cand, int k, int32_t* sel_idx, int32_t* sel_count, double* gain, cudaStream_t s) {
    auto kern = k_select_columns_f32<KMAX, ROWS>;
    constexpr size_t smem = mirror_bytes<KMAX, ROWS>();
    // opt in at any size: the static arrays count against the 48 KB default as well
    SIC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = persistent_grid(h, kern, NT, smem, n_cols);
    kern<<<grid, NT, smem, s>>>(pts, n, dim, make_kp<float>(*kp), (float)sic_floor_of(kp), targets, n_cols,
                                (const long long*)cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count,
                                kp->variance + kp->nugget, sic_floor_of(kp), gain, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
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
        if (kb == 16 && rows == 1) return launch_cols_f32<16, 1>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 16 && rows == 2) return launch_cols_f32<16, 2>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 16 && rows == 4) return launch_cols_f32<16, 4>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 32 && rows == 1) return launch_cols_f32<32, 1>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 32 && rows == 2) return launch_cols_f32<32, 2>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 32 && rows == 4) return launch_cols_f32<32, 4>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 64 && rows == 1) return launch_cols_f32<64, 1>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
        if (kb == 64 && rows == 2) return launch_cols_f32<64, 2>(h, pts, n, dim, kp, targets, n_cols, cand_ptr, cand_idx, max_cand, k, sel_idx, sel_count, gain, s);
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
