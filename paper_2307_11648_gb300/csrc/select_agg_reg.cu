// Supernodal greedy selection with register-resident factor rows (Section 5.2, the
// Cholesky approach of Appendix C.2), FP32, for up to 256 candidates, m <= 64 targets and
// k <= 64 picks: the shape of the learned proposal's survivor lists.
//
// Thread r owns candidate row r for the whole group.  Its rows of the two partial factors
// live in registers: F2P[0..m) (targets' columns of F2, i.e. Theta_{r,P} chol(Theta_PP)^-T),
// F2S[0..t) (the picks' columns of F2) and F1[0..t) (the picks' columns of F1).  A step's
// left-looking dot products therefore read only the pivot's rows, which every thread
// reads as the same (broadcast) 16-byte words from a shared-memory mirror of all rows;
// the mirror is written one entry per row per step.  Register arrays are indexed
// statically: the k steps run as four blocks of 16 with the block index a compile-time
// constant; the dot products over F1 and F2S take the completed blocks from registers and
// the current block from the own row's mirror (entries beyond the current length are zero
// on both sides), and a completed block moves from the mirror into registers.
//
// Per group: the targets' factor chol(Theta_PP) comes from a separate launch over all
// groups (FP32, one warp per group) through the workspace; every thread evaluates its
// Theta_{r,P} and solves for F2P by forward substitution, in loops over its own row of
// the F2P mirror (compact code: the setup runs once per group), then loads the row into registers;
// then k steps, each with a single block barrier: the warp argmax is one redux over
// order-preserving score keys (ties: lowest lane = lowest candidate index), the warp
// winners go to double-buffered shared slots with their V1/V2, and every warp reduces the
// eight slots itself with one more redux.  Same scores, exhaustion rule and tie-break as k_select_agg.
#include <type_traits>

#include "sic_internal.cuh"

namespace {

constexpr int RNT = 256;       // largest thread count = max candidates
constexpr int RK = 64;         // max picks
constexpr int RM = 64;         // max targets
constexpr int RP = RK + 4;     // mirror pitch of F1 and F2S rows (floats)
constexpr int RPM = RM + 4;    // mirror pitch of F2P rows and of the target factor
constexpr unsigned FULL = 0xffffffffu;
// workspace slot of one group: chol(Theta_PP) packed by rows (RM (RM + 1) / 2), its reciprocal
// diagonal (RM) and a failure flag
constexpr int LP_PACKED = RM * (RM + 1) / 2;
constexpr int LP_SLOT = LP_PACKED + RM + 4;
constexpr int LP_WARPS = 2;  // groups per CTA in the targets' Cholesky kernel (36 KB static smem)

// Two FP32 FMAs in one instruction (sm_100+ packed f32x2): lane-wise exactly the two fmaf with
// round to nearest, so the dot products below give the same bits as their scalar form with half
// the FMA instructions.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ unsigned score_key(float s) {
    const unsigned b = __float_as_uint(s);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // monotone in s; 0 is below every key
}

// acc - r . piv over the 16-element blocks that start below len (r is zero from len on,
// piv is finite everywhere)
template <int N>
__device__ __forceinline__ float reg_dot(float acc, const float (&r)[N], const float* __restrict__ piv, int len) {
    float2 a01 = make_float2(acc, 0.f), a23 = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < N / 16; ++b) {
        if (16 * b < len) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int e = 16 * b + 4 * c;
                const float4 p = *reinterpret_cast<const float4*>(piv + e);
                a01 = fma2(make_float2(-r[e], -r[e + 1]), make_float2(p.x, p.y), a01);
                a23 = fma2(make_float2(-r[e + 2], -r[e + 3]), make_float2(p.z, p.w), a23);
            }
        }
    }
    return (a01.x + a01.y) + (a23.x + a23.y);
}

// acc - r . piv over the first NB 16-element blocks (static)
template <int NB, int N>
__device__ __forceinline__ float dot_blocks(float acc, const float (&r)[N], const float* __restrict__ piv) {
    float2 a01 = make_float2(acc, 0.f), a23 = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < 16 * NB; e += 4) {
        const float4 p = *reinterpret_cast<const float4*>(piv + e);
        a01 = fma2(make_float2(-r[e], -r[e + 1]), make_float2(p.x, p.y), a01);
        a23 = fma2(make_float2(-r[e + 2], -r[e + 3]), make_float2(p.z, p.w), a23);
    }
    return (a01.x + a01.y) + (a23.x + a23.y);
}

// acc - own . piv over one 16-element block, both read from shared memory
__device__ __forceinline__ float dot_mirror(float acc, const float* __restrict__ own, const float* __restrict__ piv) {
    float2 a01 = make_float2(acc, 0.f), a23 = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 r = *reinterpret_cast<const float4*>(own + 4 * c);
        const float4 p = *reinterpret_cast<const float4*>(piv + 4 * c);
        a01 = fma2(make_float2(-r.x, -r.y), make_float2(p.x, p.y), a01);
        a23 = fma2(make_float2(-r.z, -r.w), make_float2(p.z, p.w), a23);
    }
    return (a01.x + a01.y) + (a23.x + a23.y);
}

// Sums of a step's products of the own factor rows with the pivot's rows, a[0..3] += four
// independent partial sums.  They do not depend on the kernel entry Theta_{r,q}, so they start
// as soon as the pivot is known and run beside its evaluation; the new column's numerator is
// Theta_{r,q} - (a0 + a1) - (a2 + a3).
// over the 16-element blocks B0 .. NB-1 (static)
template <int B0, int NB, int N>
__device__ __forceinline__ void acc_blocks(float (&a)[4], const float (&r)[N], const float* __restrict__ piv) {
    float2 a01 = make_float2(a[0], a[1]), a23 = make_float2(a[2], a[3]);
#pragma unroll
    for (int e = 16 * B0; e < 16 * NB; e += 4) {
        const float4 p = *reinterpret_cast<const float4*>(piv + e);
        a01 = fma2(make_float2(r[e], r[e + 1]), make_float2(p.x, p.y), a01);
        a23 = fma2(make_float2(r[e + 2], r[e + 3]), make_float2(p.z, p.w), a23);
    }
    a[0] = a01.x;
    a[1] = a01.y;
    a[2] = a23.x;
    a[3] = a23.y;
}

// the current block: entries below `len` (< 16) of the own row and the pivot's, from shared
// memory, four at a time (entries from len on are zero on both sides)
__device__ __forceinline__ void acc_mirror(float (&a)[4], const float* __restrict__ own, const float* __restrict__ piv,
                                           int len) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (4 * c < len) {
            const float4 r = *reinterpret_cast<const float4*>(own + 4 * c);
            const float4 p = *reinterpret_cast<const float4*>(piv + 4 * c);
            const float2 a01 = fma2(make_float2(r.x, r.y), make_float2(p.x, p.y), make_float2(a[0], a[1]));
            const float2 a23 = fma2(make_float2(r.z, r.w), make_float2(p.z, p.w), make_float2(a[2], a[3]));
            a[0] = a01.x;
            a[1] = a01.y;
            a[2] = a23.x;
            a[3] = a23.y;
        }
    }
}

// The targets' Cholesky factor Lp = chol(Theta_PP) of every group, FP32, one warp per
// group (left-looking, lane owns rows lane and lane + 32), from the same FP32 coordinates
// relative to the first member that the selection kernel stages.  Runs as its own
// launch over all groups at once, ahead of the latency-bound selection.
__global__ void __launch_bounds__(32 * LP_WARPS) k_agg_target_chol(const double* __restrict__ pts, long long n,
                                                                    int dim, KP<float> kp,
                                                                    const long long* __restrict__ grp_ptr,
                                                                    long long n_grp, float* __restrict__ ws,
                                                                    unsigned long long* __restrict__ ctr) {
    __shared__ __align__(16) float lsm[LP_WARPS][RM * RPM + 3 * RM];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float* Lp = lsm[w];
    float* XP = Lp + RM * RPM;
    // each warp takes its next group from a work counter zeroed before the launch (the
    // groups' m^3 / 6 costs differ by a factor of up to 512)
    auto fetch = [&]() -> long long {
        unsigned long long v = 0ULL;
        if (lane == 0) v = atomicAdd(ctr, 1ULL);
        return (long long)__shfl_sync(0xffffffffu, v, 0);
    };
    for (long long g = fetch(); g < n_grp; g = fetch()) {
        const long long g0 = grp_ptr[g];
        const int m = (int)(grp_ptr[g + 1] - g0);
        float* out = ws + g * (long long)LP_SLOT;
        if (m < 1 || m > RM || g0 < 0 || g0 + m > n) {
            if (lane == 0) out[LP_PACKED + RM] = 1.f;  // reported by the selection kernel
            continue;
        }
        double org[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < dim; ++d) org[d] = pts[g0 * dim + d];
        for (int a = lane; a < m; a += 32)
            for (int d = 0; d < 3; ++d) XP[d * RM + a] = (d < dim) ? (float)(pts[(g0 + a) * dim + d] - org[d]) : 0.f;
        __syncwarp();
        bool ok = true;
        for (int j = 0; j < m; ++j) {
            const float xj = XP[j], yj = XP[RM + j], zj = XP[2 * RM + j];
            float sv[2] = {0.f, 0.f};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = lane + 32 * h;
                if (i >= j && i < m) {
                    const float dx = XP[i] - xj, dy = XP[RM + i] - yj, dz = XP[2 * RM + i] - zj;
                    float th = matern<float>(kp, sqrtf(dx * dx + dy * dy + dz * dz));
                    if (i == j) th += kp.nugget;
                    const float* ri = Lp + i * RPM;
                    const float* rj = Lp + j * RPM;
                    float s0 = th, s1 = 0.f, s2 = 0.f, s3 = 0.f;
                    int l = 0;
                    for (; l + 4 <= j; l += 4) {
                        const float4 a = *reinterpret_cast<const float4*>(ri + l);
                        const float4 b = *reinterpret_cast<const float4*>(rj + l);
                        s0 = fmaf(-a.x, b.x, s0);
                        s1 = fmaf(-a.y, b.y, s1);
                        s2 = fmaf(-a.z, b.z, s2);
                        s3 = fmaf(-a.w, b.w, s3);
                    }
                    for (; l < j; ++l) s0 = fmaf(-ri[l], rj[l], s0);
                    sv[h] = (s0 + s1) + (s2 + s3);
                }
            }
            const float sjj = __shfl_sync(FULL, j < 32 ? sv[0] : sv[1], j & 31);
            if (!(sjj > 0.f)) {
                ok = false;
                break;
            }
            const float d = sqrtf(sjj), rd = 1.f / d;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = lane + 32 * h;
                if (i > j && i < m) {
                    Lp[i * RPM + j] = sv[h] * rd;
                    out[i * (i + 1) / 2 + j] = sv[h] * rd;
                }
            }
            if (lane == 0) {
                Lp[j * RPM + j] = d;
                out[j * (j + 1) / 2 + j] = d;
                out[LP_PACKED + j] = rd;
            }
            __syncwarp();
        }
        if (lane == 0) out[LP_PACKED + RM] = ok ? 0.f : 2.f;
        __syncwarp();
    }
}

// The targets' columns F2P = Theta_{r,P} chol(Theta_PP)^-T of every candidate row r of every
// group, FP32, for k_select_agg_reg: one thread per row, one group per CTA and two CTAs per
// SM, so that the per-row chains (m kernel entries, then a forward substitution of m steps)
// of several groups are in flight together -- inside the selection kernel, with one group per SM,
// they left the SM waiting.  The kernel entries take the distance as d2 rsqrt(d2), as the
// selection kernel's own entries do; each substitution step's dot product runs in 4-entry
// chunks over two packed FP32x2 accumulators.  Output: group g's entry (a, r) at
// f2p[(g0 - G0 + a) * NT + r], g0 =
// grp_ptr[g], G0 = grp_ptr[0] (the groups are consecutive positions).  Rows of candidates that
// are not valid, and groups whose targets' factor failed, are skipped (the selection kernel
// reports them).
constexpr int TC_ROWS = RNT;  // one CTA per group: the targets' factor is staged once
constexpr size_t TC_SMEM = sizeof(float) * ((size_t)RM * RPM + RM + 3 * RM + (size_t)TC_ROWS * RPM);

template <int NT>
__global__ void __launch_bounds__(TC_ROWS) k_agg_target_cols(const double* __restrict__ pts, long long n, int dim,
                                                              KP<float> kp, const long long* __restrict__ grp_ptr,
                                                              long long n_grp, const long long* __restrict__ cand_ptr,
                                                              const int32_t* __restrict__ cand_idx,
                                                              const float* __restrict__ lp_ws, float* __restrict__ f2p,
                                                              int max_m, unsigned long long* __restrict__ ctr) {
    extern __shared__ __align__(16) float smc[];
    float* Lp = smc;                  // [RM][RPM]
    float* rLp = Lp + RM * RPM;       // [RM]
    float* XP = rLp + RM;             // [3][RM] the targets' coordinates
    float* rows = XP + 3 * RM;        // [TC_ROWS][RPM] the threads' rows
    constexpr int CH = NT >= TC_ROWS ? NT / TC_ROWS : 1;  // row chunks per group
    const int tid = threadIdx.x;
    const long long G0 = grp_ptr[0];
    // items (group, row chunk) from a work counter zeroed before the launch: the groups' costs
    // differ with their sizes (s_next double-buffered, one barrier per fetch)
    __shared__ long long s_next[2];
    int nb_ = 0;
    auto fetch = [&]() -> long long {
        nb_ ^= 1;
        if (tid == 0) s_next[nb_] = (long long)atomicAdd(ctr, 1ULL);
        __syncthreads();
        return s_next[nb_];
    };
    for (long long it = fetch(); it < n_grp * CH; it = fetch()) {
        const long long g = it / CH;
        const int ch = (int)(it % CH);
        const long long g0 = grp_ptr[g];
        const int m = (int)(grp_ptr[g + 1] - g0);
        const long long b0 = cand_ptr[g];
        const int C = (int)(cand_ptr[g + 1] - b0);
        const float* src = lp_ws + g * (long long)LP_SLOT;
        if (m < 1 || m > max_m || C < 0 || C > NT || g0 < 0 || g0 + m > n || src[LP_PACKED + RM] != 0.f ||
            ch * TC_ROWS >= C || g0 - G0 + m > n_grp * (long long)max_m)
            continue;  // uniform over the CTA; the selection kernel reports what is invalid
        double org[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) org[d] = pts[g0 * dim + d];
        // Lp negated below the diagonal and zero from the diagonal to the end of its 4-entry chunk,
        // so that the substitution's dot products run over whole chunks (fma(x, -l, s) = fma(-x, l, s))
        const int tri = m * (m + 1) / 2;
        for (int e = tid; e < tri; e += TC_ROWS) {
            int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
            while (i * (i + 1) / 2 > e) --i;
            while ((i + 1) * (i + 2) / 2 <= e) ++i;
            const int j = e - i * (i + 1) / 2;
            Lp[i * RPM + j] = j < i ? -src[e] : 0.f;
        }
        for (int e = tid; e < 4 * m; e += TC_ROWS) {
            const int i = e >> 2, j = (i & ~3) + (e & 3);
            if (j > i) Lp[i * RPM + j] = 0.f;
        }
        if (tid < m) {
            rLp[tid] = src[LP_PACKED + tid];
#pragma unroll
            for (int d = 0; d < 3; ++d) XP[d * RM + tid] = (d < dim) ? (float)(pts[(g0 + tid) * dim + d] - org[d]) : 0.f;
        }
        __syncthreads();
        const int r = ch * TC_ROWS + tid;
        if (r < C) {
            const long long p = cand_idx[b0 + r];
            if (p >= g0 + m && p < n) {
                const float xr = (float)(pts[p * dim] - org[0]);
                const float yr = dim > 1 ? (float)(pts[p * dim + 1] - org[1]) : 0.f;
                const float zr = dim > 2 ? (float)(pts[p * dim + 2] - org[2]) : 0.f;
                float* own = rows + tid * RPM;
                for (int a0 = 0; a0 < m; a0 += 4) {  // four independent entries in flight
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int a = min(a0 + u, m - 1);  // (past m: a finite value, multiplied by Lp's zeros)
                        const float dx = xr - XP[a], dy = yr - XP[RM + a], dz = zr - XP[2 * RM + a];
                        const float d2 = dx * dx + dy * dy + dz * dz;
                        v[u] = matern<float>(kp, d2 > 0.f ? d2 * rsqrtf(d2) : 0.f);
                    }
                    *reinterpret_cast<float4*>(own + a0) = make_float4(v[0], v[1], v[2], v[3]);
                }
                float* out = f2p + (g0 - G0) * NT + r;
                for (int a = 0; a < m; ++a) {
                    const float* la = Lp + a * RPM;
                    float2 s01 = make_float2(own[a], 0.f), s23 = make_float2(0.f, 0.f);
                    for (int c = 0; c < a; c += 4) {  // whole chunks: Lp is zero from the diagonal on
                        const float4 x4 = *reinterpret_cast<const float4*>(own + c);
                        const float4 l4 = *reinterpret_cast<const float4*>(la + c);
                        s01 = fma2(make_float2(x4.x, x4.y), make_float2(l4.x, l4.y), s01);
                        s23 = fma2(make_float2(x4.z, x4.w), make_float2(l4.z, l4.w), s23);
                    }
                    const float u = ((s01.x + s01.y) + (s23.x + s23.y)) * rLp[a];
                    own[a] = u;
                    out[(long long)a * NT] = u;
                }
            }
        }
        __syncthreads();
    }
}

// NT threads (candidate rows) per group: 256, one CTA per SM; or 128 for lists of at most 128
// candidates, two CTAs (groups) per SM with the same per-thread state
template <int NT>
__global__ void __launch_bounds__(NT, RNT / NT) k_select_agg_reg(
    const double* __restrict__ pts, long long n, int dim, KP<float> kp, float floor_,
    const long long* __restrict__ grp_ptr, long long n_grp, const long long* __restrict__ cand_ptr,
    const int32_t* __restrict__ cand_idx, int k, int max_m, int32_t* __restrict__ sel_idx,
    int32_t* __restrict__ sel_count, const float* __restrict__ lp_ws, const float* __restrict__ f2p,
    double* __restrict__ gain, unsigned long long* __restrict__ ctr, DevStatus* st) {
    constexpr int LDX = NT + RM;      // staged coordinates: candidates then targets
    constexpr int NW = NT / 32;       // warps
    extern __shared__ __align__(16) float smf[];
    float* F1m = smf;                 // [NT][RP]
    float* F2Sm = F1m + NT * RP;      // [NT][RP]
    float* F2Pm = F2Sm + NT * RP;     // [NT][RPM]
    float* X = F2Pm + NT * RPM;       // [3][LDX]
    __shared__ __align__(16) unsigned pkey[2][NW];
    __shared__ int pidx[2][NW];
    __shared__ float pv1[2][NW], pv2[2][NW];
    __shared__ float gv1[RK], gv2[RK];  // the picks' two conditional variances (gains only)
    __shared__ int qs[RK];              // the picks' candidate rows, translated after the steps
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float NEG = -INFINITY;
    const float diag = kp.s2 + kp.nugget;

    // groups from a work counter zeroed before the launch, so that the CTAs finish together
    // whatever the groups' sizes (s_next double-buffered, one barrier per fetch)
    __shared__ long long s_next[2];
    int nb_ = 0;
    auto fetch = [&]() -> long long {
        nb_ ^= 1;
        if (tid == 0) s_next[nb_] = (long long)atomicAdd(ctr, 1ULL);
        __syncthreads();
        return s_next[nb_];
    };
    for (long long g = fetch(); g < n_grp; g = fetch()) {
        const long long g0 = grp_ptr[g];
        const int m = (int)(grp_ptr[g + 1] - g0);
        const long long b0 = cand_ptr[g];
        const int C = (int)(cand_ptr[g + 1] - b0);
        if (m < 1 || m > RM || m > max_m || C < 0 || C > NT || g0 < 0 || g0 + m > n ||
            g0 - grp_ptr[0] + m > n_grp * (long long)max_m) {  // (the last: its targets' columns lie beyond the workspace)
            if (tid == 0) {
                record_error(st, SIC_ERR_INVALID, g);
                sel_count[g] = 0;
            }
            for (int q = tid; q < k; q += NT) sel_idx[g * k + q] = -1;
            continue;
        }
        // ---- stage coordinates relative to the first member (differences formed in FP64)
        double org[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) org[d] = pts[g0 * dim + d];
        bool live = false;
        if (tid < C) {
            long long p = cand_idx[b0 + tid];
            live = true;
            if (p < g0 + m || p >= n) {  // candidates must lie after the group
                record_error(st, SIC_ERR_INVALID, g);
                p = g0;
                live = false;
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) X[d * LDX + tid] = (d < dim) ? (float)(pts[p * dim + d] - org[d]) : 0.f;
        }
        // zero this thread's rows of the pick mirrors
#pragma unroll
        for (int c = 0; c < RP / 4; ++c) {
            *reinterpret_cast<float4*>(F1m + tid * RP + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(F2Sm + tid * RP + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // the targets' factor failed? (reported here; k_agg_target_cols skipped the group)
        if (tid == 0) {
            const float f = lp_ws[g * (long long)LP_SLOT + LP_PACKED + RM];
            s_fail = 0;
            if (f != 0.f) {
                record_error(st, f == 2.f ? SIC_ERR_NOT_PD : SIC_ERR_INVALID, g);
                s_fail = 1;
            }
        }
        __syncthreads();
        const float xr = live ? X[tid] : 0.f, yr = live ? X[LDX + tid] : 0.f, zr = live ? X[2 * LDX + tid] : 0.f;
        if (s_fail) {
            if (tid == 0) sel_count[g] = 0;
            for (int q = tid; q < k; q += NT) sel_idx[g * k + q] = -1;
            __syncthreads();
            continue;
        }
        // ---- the own row of F2P (k_agg_target_cols) into registers and the mirror, and
        // V2 = Theta_rr|P = Theta_rr - |F2P row|^2 (downdated in the same order as the solve)
        float F2P[RM];
        float V1 = live ? diag : NEG, V2 = live ? diag : NEG;
        {
            const float* src = f2p + (g0 - grp_ptr[0]) * NT + tid;
#pragma unroll
            for (int a = 0; a < RM; ++a) {
                F2P[a] = 0.f;
                if (live && a < m) F2P[a] = src[(long long)a * NT];
            }
#pragma unroll
            for (int a = 0; a < RM; ++a)
                if (live && a < m) V2 = fmaf(-F2P[a], F2P[a], V2);
#pragma unroll
            for (int c = 0; c < RM / 4; ++c)
                *reinterpret_cast<float4*>(F2Pm + tid * RPM + 4 * c) =
                    make_float4(F2P[4 * c], F2P[4 * c + 1], F2P[4 * c + 2], F2P[4 * c + 3]);
            *reinterpret_cast<float4*>(F2Pm + tid * RPM + RM) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float F1[RK], F2S[RK];
#pragma unroll
        for (int c = 0; c < RK; ++c) {
            F1[c] = 0.f;
            F2S[c] = 0.f;
        }
        __syncthreads();

        // ---- the greedy steps, in four blocks of 16: within block TB the step t = 16 TB + tt
        // appends entry t, so the dot products over F1 and F2S run over the blocks 0..TB
        // (entries from t on are zero) and the put touches block TB only -- all statically
        int t = 0;
        auto steps = [&](auto tbc) -> bool {  // false once the selection has ended
            constexpr int TB = decltype(tbc)::value;
            for (int tt = 0; tt < 16; ++tt, ++t) {
                if (t >= k) return false;
                const int buf = t & 1;
                const unsigned key = (V2 >= floor_) ? score_key(__fdividef(V1, V2)) : 0u;
                const unsigned wmax = __reduce_max_sync(FULL, key);
                const unsigned hit = __ballot_sync(FULL, key == wmax);
                if (lane == __ffs(hit) - 1) {  // the warp's best row (lowest lane among equal keys)
                    pkey[buf][warp] = wmax;
                    pidx[buf][warp] = tid;
                    pv1[buf][warp] = V1;
                    pv2[buf][warp] = V2;
                }
                __syncthreads();
                // the warp winners (ascending rows), reduced by every warp: lane w < NW
                // reads warp w's key; the lowest warp holding the maximum wins
                const unsigned kw = (lane < NW) ? pkey[buf][lane] : 0u;
                const unsigned bk = __reduce_max_sync(FULL, kw);
                if (bk == 0u) return false;
                const int bw = __ffs(__ballot_sync(FULL, lane < NW && kw == bk)) - 1;
                const int q = pidx[buf][bw];
                const float r1 = rsqrtf(pv1[buf][bw]);
                const float r2 = rsqrtf(pv2[buf][bw]);
                if (V2 != NEG) {
                    // the own rows' products with the pivot's rows: blocks 0..TB-1 from registers,
                    // the current block TB (tt entries so far) from the own row's mirror
                    // (the first segment of each sum -- F1's first block, F2's target columns, which
                    // usually carry most of the correlation -- is subtracted from the kernel entry
                    // term by term, as fused operations, so that its cancellation loses nothing;
                    // the other segments are summed first, while the entry is evaluated)
                    float s1[4] = {0.f, 0.f, 0.f, 0.f}, s2[4] = {0.f, 0.f, 0.f, 0.f};
                    if constexpr (TB >= 1) {
                        acc_blocks<1, TB>(s1, F1, F1m + q * RP);
                        acc_mirror(s1, F1m + tid * RP + 16 * TB, F1m + q * RP + 16 * TB, tt);
                    }
                    acc_blocks<0, TB>(s2, F2S, F2Sm + q * RP);
                    acc_mirror(s2, F2Sm + tid * RP + 16 * TB, F2Sm + q * RP + 16 * TB, tt);
                    const float dx = xr - X[q], dy = yr - X[LDX + q], dz = zr - X[2 * LDX + q];
                    const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    float th = matern<float>(kp, d2 > 0.f ? d2 * rsqrtf(d2) : 0.f);
                    if (tid == q) th += kp.nugget;
                    float n1;
                    if constexpr (TB >= 1) n1 = dot_blocks<1>(th, F1, F1m + q * RP);
                    else n1 = dot_mirror(th, F1m + tid * RP, F1m + q * RP);
                    n1 -= (s1[0] + s1[1]) + (s1[2] + s1[3]);
                    const float n2 = reg_dot(th, F2P, F2Pm + q * RPM, m) - ((s2[0] + s2[1]) + (s2[2] + s2[3]));
                    const float u1 = n1 * r1, u2 = n2 * r2;
                    F1m[tid * RP + t] = u1;
                    F2Sm[tid * RP + t] = u2;
                    if (tid == q) {
                        V1 = NEG;
                        V2 = NEG;
                    } else {
                        V1 = fmaf(-u1, u1, V1);
                        V2 = fmaf(-u2, u2, V2);
                    }
                }
                if (tid == 0) {
                    qs[t] = q;  // no global load on the step chain
                    if (gain) {
                        gv1[t] = pv1[buf][bw];
                        gv2[t] = pv2[buf][bw];
                    }
                }
            }
            // block TB is complete: move the own row's entries into registers
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float4 a = *reinterpret_cast<const float4*>(F1m + tid * RP + 16 * TB + 4 * c);
                const float4 b = *reinterpret_cast<const float4*>(F2Sm + tid * RP + 16 * TB + 4 * c);
                F1[16 * TB + 4 * c] = a.x;
                F1[16 * TB + 4 * c + 1] = a.y;
                F1[16 * TB + 4 * c + 2] = a.z;
                F1[16 * TB + 4 * c + 3] = a.w;
                F2S[16 * TB + 4 * c] = b.x;
                F2S[16 * TB + 4 * c + 1] = b.y;
                F2S[16 * TB + 4 * c + 2] = b.z;
                F2S[16 * TB + 4 * c + 3] = b.w;
            }
            return true;
        };
        if (steps(std::integral_constant<int, 0>{}) && steps(std::integral_constant<int, 1>{}) &&
            steps(std::integral_constant<int, 2>{}))
            steps(std::integral_constant<int, 3>{});
        // the picks' global indices and (with gain) the decreases of logdet Theta_{PP|I} per
        // nonzero (Section 5.4.2), off the step chain
        __syncthreads();
        for (int q = tid; q < t; q += NT) {
            sel_idx[g * k + q] = cand_idx[b0 + qs[q]];
            if (gain) gain[g * k + q] = log((double)gv1[q] / (double)gv2[q]) / m;
        }
        if (tid == 0) sel_count[g] = t;
        for (int q = t + tid; q < k; q += NT) sel_idx[g * k + q] = -1;
        __syncthreads();
    }
}

}  // namespace

bool agg_reg_applies(sic_precision prec, int max_cand, int max_m, int k) {
    return prec == SIC_FP32_MIXED && max_cand <= RNT && max_m <= RM && k <= RK;
}

// the targets' factors (LP_SLOT floats per group), then the targets' columns of every
// candidate row (at most n_grp * max_m positions of RNT rows)
static size_t agg_reg_floats_bytes(long long n_grp, int max_m) {
    const long long g = n_grp > 0 ? n_grp : 1;
    return (sizeof(float) * ((size_t)LP_SLOT * (size_t)g + (size_t)g * (size_t)max_m * RNT) + 15) & ~(size_t)15;
}

// ... and three work counters (the selection, the targets' columns, the targets' factors)
size_t agg_reg_workspace(long long n_grp, int max_m) {
    return agg_reg_floats_bytes(n_grp, max_m) + 3 * sizeof(unsigned long long);
}

sic_status launch_agg_reg(sic_handle* h, const double* pts, long long n, const sic_kernel* kp,
                          const int64_t* grp_ptr, int64_t n_grp, const int64_t* cand_ptr, const int32_t* cand_idx,
                          int max_cand, int max_m, int k, int32_t* sel_idx, int32_t* sel_count, double* gain, void* ws,
                          size_t ws_bytes, cudaStream_t s) {
    if (!ws || ws_bytes < agg_reg_workspace(n_grp, max_m)) return SIC_ERR_INVALID;
    const KP<float> kpf = make_kp<float>(*kp);
    float* lp = (float*)ws;
    float* f2p = lp + (size_t)LP_SLOT * (size_t)(n_grp > 0 ? n_grp : 1);
    unsigned long long* ctr =
        reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ws) + agg_reg_floats_bytes(n_grp, max_m));
    SIC_CUDA_TRY(cudaMemsetAsync(ctr, 0, 3 * sizeof(unsigned long long), s));
    const int lgrid = persistent_grid(h, k_agg_target_chol, 32 * LP_WARPS, 0, (n_grp + LP_WARPS - 1) / LP_WARPS);
    k_agg_target_chol<<<lgrid, 32 * LP_WARPS, 0, s>>>(pts, n, kp->dim, kpf, (const long long*)grp_ptr, n_grp, lp,
                                                      ctr + 2);
    // 128 threads (two groups per SM) when every list has at most 128 candidates, unless the
    // autotuner chose 256 for this bucket (each row's arithmetic is the same either way)
    int nt = max_cand <= 128 ? 128 : RNT;
    if (max_cand <= 128 &&
        tune_get(h, TUNE_SELECT_AGG, tune_select_key_a(k, SIC_FP32_MIXED), tune_select_key_b(max_cand, max_m), 0) ==
            RNT)
        nt = RNT;
    auto cols = nt == 128 ? k_agg_target_cols<128> : k_agg_target_cols<RNT>;
    SIC_CUDA_TRY(cudaFuncSetAttribute(cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    const int cgrid = persistent_grid(h, cols, TC_ROWS, TC_SMEM, n_grp * (nt >= TC_ROWS ? nt / TC_ROWS : 1));
    cols<<<cgrid, TC_ROWS, TC_SMEM, s>>>(pts, n, kp->dim, kpf, (const long long*)grp_ptr, n_grp,
                                          (const long long*)cand_ptr, cand_idx, lp, f2p, max_m, ctr + 1);
    auto kern = nt == 128 ? k_select_agg_reg<128> : k_select_agg_reg<RNT>;
    const size_t smem = sizeof(float) * ((size_t)nt * RP * 2 + (size_t)nt * RPM + 3 * (size_t)(nt + RM));
    SIC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = persistent_grid(h, kern, nt, smem, n_grp > 0 ? n_grp : 1);
    kern<<<grid, nt, smem, s>>>(pts, n, kp->dim, kpf, (float)sic_floor_of(kp), (const long long*)grp_ptr, n_grp,
                                (const long long*)cand_ptr, cand_idx, k, max_m, sel_idx, sel_count, lp, f2p, gain,
                                ctr, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}
