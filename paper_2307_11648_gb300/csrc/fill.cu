// KL-optimal fill of the factor (eq. L_col; aggregated form, Appendix A.4), FP64.
//
// One CTA of four (small groups) or eight (large groups) worker warps plus a pivot warp
// per unit (a single column, or a group of m consecutive columns sharing the picks S).
// With the aggregated set ordered ascending,
// s = (P_0..P_{m-1}, S sorted), the factor block is L = U^{-T} where U U^T =
// Theta_{s,s}, U upper triangular.  The CTA forms Theta on the reversed order
// R = reverse(s) in packed lower storage in shared memory (one entry per thread), factors
// it Theta_{RR} = L D L^T = G G^T with G = L D^{1/2} (blocked right-looking: panels of
// FILL_B columns in FP64, each panel's diagonal block factored by the pivot warp while the
// workers apply the previous panel, each panel's update of the trailing matrix as integer dot
// products (exact 32 x 32-bit products) of fixed-point G rows, one FP64 subtraction per entry
// and panel), and since U = J G J (J the reversal), member a's
// column is J G^{-T} e_j = d_j^{-1/2} J L^{-T} e_j with j = n-1-a: one back substitution per
// member, one member per half-warp, the right-hand side in registers, in double-float
// arithmetic on the FP32 pipe.  v_a = G_jj^2 = d_j,
// so logv = log d_j (eq. inverse_cond).  Rows are written diagonal first, then ascending, to
// the caller's CSC arrays.  Theta entries use the FP64 Matern of matern_d2_fast
// (table-driven exp and Newton square root, each with its non-critical steps in
// double-float on the FP32 pipe): this GPU issues two FP64 FMAs per clock per SM, so FP64
// instructions are spent sparingly.
//
// Also here: the nnz count + exclusive scan that builds col_ptr, and the fixed-order
// two-pass sum of logv (bit-reproducible).
#include <mutex>

#include "dfloat.cuh"
#include "sic_internal.cuh"

namespace {

constexpr int SCAN_TILE = 1024;  // elements per scan block (256 threads x 4)
constexpr int SUM_TILE = 2048;   // elements per partial-sum block

// ---------------------------------------------------------------- nnz + scan --

// Entry counts of the columns col0 .. col0 + n_cols - 1 (out[c - col0]); without groups unit u
// is column col0 + u.
__global__ void k_nnz_count(const long long* __restrict__ grp_ptr, long long n_grp, const int32_t* __restrict__ cnt,
                            long long col0, long long n_cols, long long* __restrict__ out, DevStatus* st) {
    long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u >= n_grp) return;
    if (!grp_ptr) {
        out[u] = 1 + (long long)cnt[u];
        return;
    }
    long long g0 = grp_ptr[u], g1 = grp_ptr[u + 1];
    if (g0 < col0 || g1 > col0 + n_cols || g1 <= g0) {
        record_error(st, SIC_ERR_INVALID, u);
        return;
    }
    int m = (int)(g1 - g0);
    for (int a = 0; a < m; ++a) out[g0 - col0 + a] = (long long)(m - a) + cnt[u];
}

// Block-local exclusive scan of a tile; the tile total goes to partial[blockIdx].
__global__ void __launch_bounds__(256) k_scan_tile(long long* __restrict__ v, long long n,
                                                   long long* __restrict__ partial) {
    __shared__ long long s[256];
    long long base = blockIdx.x * (long long)SCAN_TILE + threadIdx.x * 4;
    long long a[4];
    long long sum = 0;
    for (int i = 0; i < 4; ++i) {
        a[i] = (base + i < n) ? v[base + i] : 0;
        sum += a[i];
    }
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        long long x = (threadIdx.x >= off) ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += x;
        __syncthreads();
    }
    long long run = s[threadIdx.x] - sum;  // exclusive prefix of this thread
    for (int i = 0; i < 4; ++i) {
        if (base + i < n) v[base + i] = run;
        run += a[i];
    }
    if (threadIdx.x == 255) partial[blockIdx.x] = s[255];
}

// Exclusive scan of the tile totals in one block (loops over chunks of 256).
__global__ void __launch_bounds__(256) k_scan_partials(long long* __restrict__ partial, long long nb,
                                                       long long* __restrict__ total) {
    __shared__ long long s[256];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < nb; c0 += 256) {
        long long i = c0 + threadIdx.x;
        long long x0 = (i < nb) ? partial[i] : 0;
        s[threadIdx.x] = x0;
        __syncthreads();
        for (int off = 1; off < 256; off <<= 1) {
            long long x = (threadIdx.x >= off) ? s[threadIdx.x - off] : 0;
            __syncthreads();
            s[threadIdx.x] += x;
            __syncthreads();
        }
        if (i < nb) partial[i] = carry + s[threadIdx.x] - x0;
        __syncthreads();
        if (threadIdx.x == 255) carry += s[255];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(long long* __restrict__ v, long long n, const long long* __restrict__ partial,
                           long long base) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) v[i] += partial[i / SCAN_TILE] + base;
}

// ------------------------------------------------------------------- the fill --

// worker threads per unit: 128 for the small-group launch, 256 for the large groups (more
// warps in flight where fewer CTAs fit per SM); lane 0 of one more warp takes the pivots
constexpr int FILL_HSLOTS = 12;  // right-hand-side entries per half-warp lane: nn <= 192 = 16 * FILL_HSLOTS
constexpr int FILL_M_SPLIT = 32;  // groups of at most this size run in their own launch
constexpr int FILL_B = 4;         // panel width of the blocked LDL^T (integer trailing update)

// doubles of the scratch region: the points' coordinates while Theta is formed, then the
// panel's rows in fixed point ((2 FILL_B + 1) ints per row); even, so what follows stays
// 16-byte aligned
__host__ __device__ constexpr int fill_scratch_doubles(int nmax) {
    return ((3 * nmax > ((2 * FILL_B + 1) * nmax + 1) / 2 ? 3 * nmax : ((2 * FILL_B + 1) * nmax + 1) / 2) + 1) & ~1;
}

// Packed lower-triangle index (nn <= 192, so every index fits in 32 bits; 32-bit integer
// arithmetic and int-to-float conversions stay off the FP64 pipe).
__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }

// row i of the packed lower triangle that holds flat entry e (i(i+1)/2 <= e < (i+1)(i+2)/2)
__device__ __forceinline__ int pk_row(int e) {
    int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (i * (i + 1) / 2 > e) --i;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    return i;
}

// Pivot of column c of the LDL^T factorisation from its final Schur complement v: D_cc = v
// (kept on the diagonal) and d^(-1/2) by rsqrt_newton (five FP64 operations with the
// diagonal's update) into piv slot c & 3 (the panel's columns); the column is then scaled as
// G_ic = U_ic d^(-1/2) and L_ic = G_ic d^(-1/2).  A non-positive pivot raises *bad.  The range
// test reads the bits (no FP64 compare).
__device__ __forceinline__ void fill_pivot(double v, int c, double* G, double* piv, int* bad) {
    const long long vb = __double_as_longlong(v);
    if (vb <= 0 || vb >= 0x7ff0000000000000LL) {  // not in (+0, +inf): non-positive, infinite or NaN
        *bad = 1;
        return;
    }
    G[pk(c, c)] = v;
    piv[c & 3] = rsqrt_newton(v);
}

// ---- the integer update of a panel ----
//
// A row of a panel, its FILL_B values g_j (entries of G = L D^(1/2)), is held in fixed point:
// g_j = M_j 2^(E - 1075) with E the largest biased exponent among them and M_j the 53-bit
// significands shifted to E and truncated (signed; zero and subnormal values count as 0), split
// as M_j = Mh_j 2^26 + Ml_j (Mh signed, 0 <= Ml < 2^26).  Layout (B = 4, ld rows, fx 16-byte
// aligned): the Mh of a row as one int4 at fx[4 row], its Ml at fx[4 (ld + row)], E at
// fx[8 ld + row] (a warp reading consecutive rows reads consecutive 16-byte words).
// The dot product of two rows is formed from exact 32 x 32-bit products (fx_dot).  Truncating
// to the row's exponent costs each value at most 2^-52 of the row's largest, and fx_dot's own
// truncations stay below 2^-51 of the largest product: with G's rows (|G_ij| <= sqrt(A_ii)) the
// error of an entry's update stays within a few B 2^-52 sqrt(A_ii A_ll), the order of the FP64
// Cholesky's own backward error bound.
template <int B>
__device__ __forceinline__ void fx_row_store(const double (&g)[B], int* __restrict__ fx, int ld, int row) {
    static_assert(B == 4, "the fixed-point rows are stored as int4");
    int e[B];
    int E = 0;
#pragma unroll
    for (int j = 0; j < B; ++j) {
        e[j] = (__double2hiint(g[j]) >> 20) & 0x7ff;
        E = max(E, e[j]);
    }
    int mh[B], ml[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
        const long long u = __double_as_longlong(g[j]);
        long long m = e[j] ? ((u & 0xfffffffffffffLL) | 0x10000000000000LL) : 0LL;
        const int sh = E - e[j];
        m = sh < 63 ? (m >> sh) : 0LL;
        if (u < 0) m = -m;
        mh[j] = (int)(m >> 26);
        ml[j] = (int)(m & 0x3ffffffLL);
    }
    reinterpret_cast<int4*>(fx)[row] = make_int4(mh[0], mh[1], mh[2], mh[3]);
    reinterpret_cast<int4*>(fx)[ld + row] = make_int4(ml[0], ml[1], ml[2], ml[3]);
    fx[8 * ld + row] = E;
}

// s 2^e2 as FP64 by integer operations, the significand truncated (relative error < 2^-52);
// 0 for s = 0 and below FP64's normal range
__device__ __forceinline__ double i64_scaled(long long s, int e2) {
    if (s == 0) return 0.0;
    const unsigned long long sg = (unsigned long long)s & (1ULL << 63);
    const unsigned long long mag = s < 0 ? 0ULL - (unsigned long long)s : (unsigned long long)s;
    const int z = __clzll((long long)mag);
    const int be = e2 + 63 - z + 1023;
    if (be <= 0) return 0.0;
    return __longlong_as_double((long long)(sg | ((unsigned long long)be << 52) | (((mag << z) >> 11) & 0xfffffffffffffULL)));
}

__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

// Two updates x -= a y in double-float (x = xh + xl, a and y likewise; dfloat.cuh), x0 -= a0 y in
// the .x halves of xh, xl and x1 -= a1 y in the .y halves, as packed FP32x2 instructions (lane-wise
// the roundings of the scalar operations): the exact product of the high parts and its cross
// terms, TwoSum of the high parts, the low parts added to its error, renormalised (Fast2Sum).
// Relative error about 2^-47 of the operands' magnitudes; a = 0 leaves the value of x unchanged.
__device__ __forceinline__ void df_sub_mul2(float2& xh, float2& xl, float2 a0, float2 a1, float yh, float yl) {
    const float2 ah = make_float2(a0.x, a1.x), al = make_float2(a0.y, a1.y);
    const float2 y2 = make_float2(yh, yh), yl2 = make_float2(yl, yl);
    const float2 ph = __fmul2_rn(ah, y2);
    const float2 pe = __ffma2_rn(ah, yl2, __ffma2_rn(al, y2, __ffma2_rn(ah, y2, neg2(ph))));
    const float2 s = __fadd2_rn(xh, neg2(ph));
    const float2 bb = __fadd2_rn(s, neg2(xh));
    const float2 err = __fadd2_rn(__fadd2_rn(xh, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(neg2(ph), neg2(bb)));
    const float2 lo = __fadd2_rn(__fadd2_rn(xl, neg2(pe)), err);
    const float2 t = __fadd2_rn(s, lo);
    xl = __fadd2_rn(lo, neg2(__fadd2_rn(t, neg2(s))));
    xh = t;
}

// sum_j g_ij g_lj of rows i and l: 2^52 sum Mh Mh + 2^26 sum (Mh Ml + Ml Mh) exactly in two 64-bit
// sums of 32 x 32-bit products, scaled down by 2^52 into one 64-bit integer (the dropped fraction
// and the omitted sum Ml Ml are below 5 units of 2^(Ei + El - 2098)), converted to FP64
template <int B>
__device__ __forceinline__ double fx_dot(const int* __restrict__ fx, int ld, int i, int l) {
    static_assert(B == 4, "the fixed-point rows are stored as int4");
    const int4 hi4 = reinterpret_cast<const int4*>(fx)[i], li4 = reinterpret_cast<const int4*>(fx)[ld + i];
    const int4 hl4 = reinterpret_cast<const int4*>(fx)[l], ll4 = reinterpret_cast<const int4*>(fx)[ld + l];
    const int hi_[4] = {hi4.x, hi4.y, hi4.z, hi4.w}, li[4] = {li4.x, li4.y, li4.z, li4.w};
    const int hl[4] = {hl4.x, hl4.y, hl4.z, hl4.w}, ll[4] = {ll4.x, ll4.y, ll4.z, ll4.w};
    long long a2 = 0, a1 = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        a2 += (long long)hi_[j] * hl[j];
        a1 += (long long)hi_[j] * ll[j] + (long long)li[j] * hl[j];
    }
    return i64_scaled(a2 + (a1 >> 26), fx[8 * ld + i] + fx[8 * ld + l] - 2098);
}


// A coordinate x in fixed point at the largest biased exponent E of its dimension in the unit:
// x 2^(1084 - E), so that |x_fix| < 2^62; exact for every x whose exponent is within 9 of E (a
// unit's points are near one another: their coordinates share the exponent unless they are
// within a few length scales of zero, where the truncation below 2^(E - 1085) is far below an
// ulp of the kernel entries).  Integer operations only.
__device__ __forceinline__ long long fx_coord(double x, int E) {
    const long long u = __double_as_longlong(x);
    const int e = (int)((u >> 52) & 0x7ff);
    if (!e) return 0LL;
    const long long mant = (u & 0xfffffffffffffLL) | 0x10000000000000LL;
    const int sh = E - e;  // >= 0
    const long long f = sh <= 9 ? (mant << (9 - sh)) : (sh - 9 < 63 ? (mant >> (sh - 9)) : 0LL);
    return u < 0 ? -f : f;
}

// dx^2 of one dimension, exact in 128 bits (h:l), for a difference |dx| < 2^63
__device__ __forceinline__ void sq128(long long dx, unsigned long long& h, unsigned long long& l) {
    const unsigned long long a = dx < 0 ? 0ULL - (unsigned long long)dx : (unsigned long long)dx;
    const unsigned ah = (unsigned)(a >> 32), al = (unsigned)a;
    const unsigned long long q0 = (unsigned long long)al * al;
    const unsigned long long q1 = ((unsigned long long)ah * al) << 1;  // ah < 2^31
    l = q0 + (q1 << 32);
    h = (unsigned long long)ah * ah + (q1 >> 32) + (l < q0 ? 1ULL : 0ULL);
}

// The squared distance between points i and j from their fixed-point coordinates (xf[d ld + i],
// scale 2^(1084 - E_d) in dimension d): each dimension's square exact in 128 bits, aligned to the
// largest scale (a right shift, dropping bits below 2^-125 of the largest term), summed and
// rounded once to FP64 (to nearest, ties away from zero).  Integer operations only.
__device__ __forceinline__ double fx_dist2(const long long* __restrict__ xf, int ld, int dim, int i, int j, int E0,
                                           int E1, int E2) {
    const int Em = max(E0, max(dim > 1 ? E1 : 0, dim > 2 ? E2 : 0));
    unsigned long long h = 0ULL, l = 0ULL;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= dim) break;
        unsigned long long sh, sl;
        sq128(xf[d * ld + i] - xf[d * ld + j], sh, sl);
        const int s = 2 * (Em - (d == 0 ? E0 : (d == 1 ? E1 : E2)));
        if (s >= 128) {
            sh = sl = 0ULL;
        } else if (s >= 64) {
            sl = sh >> (s - 64);
            sh = 0ULL;
        } else if (s > 0) {
            sl = (sl >> s) | (sh << (64 - s));
            sh >>= s;
        }
        l += sl;
        h += sh + (l < sl ? 1ULL : 0ULL);
    }
    if ((h | l) == 0ULL) return 0.0;
    int p;
    unsigned long long t;  // the leading 64 bits, leading bit at 63
    if (h) {
        const int z = __clzll((long long)h);
        p = 127 - z;
        t = z ? ((h << z) | (l >> (64 - z))) : h;
    } else {
        const int z = __clzll((long long)l);
        p = 63 - z;
        t = l << z;
    }
    unsigned long long mt = ((t >> 10) + 1ULL) >> 1;  // 53 bits, rounded
    if (mt >> 53) {
        mt >>= 1;
        ++p;
    }
    const int be = p + 2 * Em - 1145;  // |X| 2^(2 Em - 2168) = (mt 2^-52) 2^(p + 2 Em - 2168)
    if (be <= 0) return 0.0;
    return __longlong_as_double((long long)(((unsigned long long)be << 52) | (mt & 0xfffffffffffffULL)));
}

// CTAs per SM the register budget is set for (shared memory allows about this many at the
// largest group of each launch)
constexpr int fill_min_ctas(int nt) { return nt == 128 ? 5 : (nt == 256 ? 3 : 2); }

template <int FILL_NT>
__global__ void __launch_bounds__(FILL_NT + 32, fill_min_ctas(FILL_NT)) k_fill(const double* __restrict__ pts, int dim, KP<double> kp,
                                                  const long long* __restrict__ grp_ptr, long long n_units,
                                                  const int32_t* __restrict__ sel_idx,
                                                  const int32_t* __restrict__ sel_count, int k, int max_m,
                                                  int m_lo, int m_hi, long long n, long long col0,
                                                  long long n_cols, const long long* __restrict__ col_ptr,
                                                  long long base, int32_t* __restrict__ row_idx,
                                                  double* __restrict__ val, double* __restrict__ logv,
                                                  unsigned long long* __restrict__ ctr, DevStatus* st) {
    extern __shared__ double smem_d[];
    const int nmax = k + m_hi;  // shared memory is laid out for this launch's size class
    double* tab = smem_d;                                   // 2^(j/256) (exp_neg_table)
    double* xyz = tab + EXP_TAB;                            // 3 x nmax, while Theta is formed; then
    int* fx = reinterpret_cast<int*>(xyz);                  // the panel's rows in fixed point (16-byte aligned)
    double* G = xyz + fill_scratch_doubles(nmax);           // packed lower, nmax(nmax+1)/2
    double* piv = G + (long long)nmax * (nmax + 1) / 2;     // d^(-1/2) of the panel's columns (slot c & 3)
    int* pos = reinterpret_cast<int*>(piv + 4);             // nmax
    int* srt = pos + nmax;                                  // k
    __shared__ int s_bad;
    __shared__ unsigned s_emax[3];  // the largest biased exponent of the unit's coordinates, per dimension
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool worker = tid < FILL_NT;  // the pivot warp joins only the barriers and the pivots
    exp_table_fill(tab, kp.s2);
    // units are taken from a work counter (*ctr, zeroed before the launch), so that the CTAs finish
    // together whatever the units' sizes; s_next is double-buffered, one barrier per fetch
    __shared__ long long s_next[2];
    int nb_ = 0;
    auto fetch = [&]() -> long long {
        nb_ ^= 1;
        if (tid == 0) s_next[nb_] = (long long)atomicAdd(ctr, 1ULL);
        __syncthreads();
        return s_next[nb_];
    };
    for (long long u = fetch(); u < n_units; u = fetch()) {
        const long long g0 = grp_ptr ? grp_ptr[u] : col0 + u;
        const int m = grp_ptr ? (int)(grp_ptr[u + 1] - g0) : 1;
        const int cnt = sel_count[u];
        const long long c0 = g0 - col0;  // the unit's first column within the slice
        if (m < 1 || m > max_m || cnt < 0 || cnt > k || g0 < 0 || g0 + m > n || c0 < 0 || c0 + m > n_cols) {
            if (tid == 0 && m_lo == 1) record_error(st, SIC_ERR_INVALID, u);  // reported by the first class
            continue;
        }
        if (m < m_lo || m > m_hi) continue;  // another launch's size class
        const int nn = cnt + m;
        if (nn > FILL_NT) {  // excluded by the launcher (FILL_NT >= k + m_hi)
            if (tid == 0) record_error(st, SIC_ERR_UNSUPPORTED, u);
            continue;
        }
        // picks sorted ascending by rank; they must be distinct positions after the unit,
        // and col_ptr must match the pattern
        bool bad = false;
        for (int i = worker ? tid : cnt; i < cnt; i += FILL_NT) {
            const int v = sel_idx[u * k + i];
            int rank = 0, same = 0;
            for (int j = 0; j < cnt; ++j) {
                const int w = sel_idx[u * k + j];
                rank += (w < v);
                same += (w == v);
            }
            if (v < g0 + m || v >= n || same != 1) bad = true;
            else srt[rank] = v;
        }
        for (int a = worker ? tid : m; a < m; a += FILL_NT)
            if (col_ptr[c0 + a + 1] - col_ptr[c0 + a] != (long long)(m - a + cnt)) bad = true;
        if (tid < 3) s_emax[tid] = 0u;
        if (__syncthreads_or(bad)) {
            if (tid == 0) record_error(st, SIC_ERR_INVALID, u);
            continue;
        }
        // R order: picks descending, then members descending; the coordinates go to fixed point
        // at the unit's largest exponent in each dimension (fx_coord), so that differences and
        // squared distances are exact integer arithmetic (fx_dist2)
        {
            unsigned em[3] = {0u, 0u, 0u};
            for (int i = worker ? tid : nn; i < nn; i += FILL_NT) {
                const int p = (i < cnt) ? srt[cnt - 1 - i] : (int)(g0 + m - 1 - (i - cnt));
                pos[i] = p;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const double x = (d < dim) ? pts[(long long)p * dim + d] : 0.0;
                    xyz[d * nmax + i] = x;
                    em[d] = max(em[d], ((unsigned)__double2hiint(x) >> 20) & 0x7ffu);
                }
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                em[d] = __reduce_max_sync(0xffffffffu, em[d]);
                if (lane == 0 && em[d]) atomicMax(&s_emax[d], em[d]);
            }
        }
        if (tid == 0) s_bad = 0;
        __syncthreads();
        const int E0 = (int)s_emax[0], E1 = (int)s_emax[1], E2 = (int)s_emax[2];
        long long* xf = reinterpret_cast<long long*>(xyz);
        for (int i = worker ? tid : nn; i < nn; i += FILL_NT)
            for (int d = 0; d < dim; ++d) xf[d * nmax + i] = fx_coord(xyz[d * nmax + i], d == 0 ? E0 : (d == 1 ? E1 : E2));
        __syncthreads();
        // Theta_RR, packed lower, one flat entry per thread: the squared distance exact from the
        // fixed-point coordinates, the Matern in FP64 (matern_d2_fast; the all-double-float
        // Matern of dfloat.cuh would spare the FP64 pipe entirely, but its ~1e-14 of the
        // variance per entry is amplified by 1/v in the Schur complements, v ~ 2 nugget on the
        // finest groups: factor columns then miss the oracle's by more than 1e-8)
        // entry e = i (i + 1) / 2 + j, stepped by FILL_NT
        for (int i = worker ? pk_row(tid) : nn, j = worker ? tid - i * (i + 1) / 2 : 0; i < nn;) {
            double v = matern_d2_fast(kp, fx_dist2(xf, nmax, dim, i, j, E0, E1, E2), tab);
            if (i == j) v += kp.nugget;
            G[pk(i, j)] = v;
            j += FILL_NT;
            while (j > i) {
                j -= i + 1;
                ++i;
            }
        }
        __syncthreads();
        // blocked right-looking LDL^T factorisation Theta_RR = L D L^T in place on the packed
        // lower triangle, in panels of FILL_B columns, in FP64: d_j = A_jj, L_ij = A_ij / d_j and
        // A_il -= L_ij U_lj within the panel (U_lj = A_lj, the panel's entries unscaled).  The
        // rows below the panel keep G_ij = U_ij d_j^(-1/2) (G = L D^(1/2)) in fixed point; the
        // trailing matrix then takes the panel's whole rank-FILL_B update as one integer dot
        // product of two G rows per entry (exact products), subtracted in FP64 (fx_dot): FILL_B
        // FP64 FMAs become one FP64 addition, the products going to the integer multiply-add
        // units.  The FP64 units are per SM sub-partition and charge a warp instruction whatever
        // its active lanes, so the flat loops keep full warps.
        // The panel's diagonal block (at most FILL_B x FILL_B) is factored by the pivot warp, lane
        // r owning the block's row r (its pivots and their reciprocal square roots are a chain of
        // dependent FP64 operations, warp-synchronous): the next panel's block takes the current
        // panel's update and is factored while the workers update the rest of the trailing matrix.
        // Every worker row below the block then applies the block's columns to its own panel
        // entries in registers (A_il -= L_ij U_lj reads the block's unscaled entries, which stay
        // in place until the block's L entries are written back in the next phase), so that a
        // panel costs two barriers.  Worker thread i owns row i (nn <= FILL_NT, the launcher's
        // choice).  Same operations, in the same order, as a column-by-column elimination.
        const int i = tid;
        const int rowi = pk(i, 0);
        double lb[FILL_B];  // pivot warp: L of the block's row `lane` (columns below it)
        // the block [J, J + bs) (its entries final): lane r owns row J + r
        auto factor_block = [&](int J, int bs) {
            const int r = lane;
            const int ib = J + r;
            if (r == 0) fill_pivot(G[pk(J, J)], J, G, piv, &s_bad);
            __syncwarp();
#pragma unroll
            for (int jj = 0; jj < FILL_B - 1; ++jj) {
                if (jj >= bs - 1) break;
                const int j = J + jj;
                if (r > jj && r < bs) {
                    const double rsd = piv[j & 3];
                    const double uv = G[pk(ib, j)];
                    const double g = uv * rsd;
                    const double l = g * rsd;
                    lb[jj] = l;
#pragma unroll
                    for (int c2 = jj + 1; c2 < FILL_B; ++c2)
                        if (c2 <= r) G[pk(ib, J + c2)] = fma(-l, G[pk(J + c2, j)], G[pk(ib, J + c2)]);
                    if (r == jj + 1) fill_pivot(G[pk(ib, ib)], ib, G, piv, &s_bad);
                }
                __syncwarp();
            }
        };
        if (!worker) factor_block(0, min(FILL_B, nn));
        __syncthreads();
        for (int J = 0; J < nn && !s_bad; J += FILL_B) {
            const int je = min(J + FILL_B, nn);  // je < nn implies a full panel
            // the own row's panel entries (rows below the block): L and G by the block's columns
            if (worker && i >= je && i < nn) {
                double u[FILL_B], gv[FILL_B], lv[FILL_B];
#pragma unroll
                for (int c = 0; c < FILL_B; ++c) u[c] = G[rowi + J + c];
#pragma unroll
                for (int jj = 0; jj < FILL_B; ++jj) {
                    const double rsd = piv[jj];  // (J + jj) & 3
                    const double g = u[jj] * rsd;
                    const double l = g * rsd;
                    gv[jj] = g;
                    lv[jj] = l;
#pragma unroll
                    for (int c2 = jj + 1; c2 < FILL_B; ++c2) u[c2] = fma(-l, G[pk(J + c2, J + jj)], u[c2]);
                }
                fx_row_store<FILL_B>(gv, fx, nmax, i);
                // the L entries as double-float pairs (hi, lo) in their 8-byte slots (f64_split: 48
                // significant bits; only the member solves read them)
#pragma unroll
                for (int c = 0; c < FILL_B; ++c) {
                    float h, l;
                    f64_split(lv[c], h, l);
                    reinterpret_cast<float2*>(G)[rowi + J + c] = make_float2(h, l);
                }
            }
            __syncthreads();
            if (worker) {
                // the trailing matrix, entries (i, l) with je <= l <= i < nn, takes the panel's
                // update, but for the next panel's block (the first nbt flat entries)
                if (je < nn) {
                    const int nt = nn - je;
                    const int bs2 = min(FILL_B, nt), nbt = bs2 * (bs2 + 1) / 2;
                    // entry e = ii (ii + 1) / 2 + ll of the trailing triangle, stepped by FILL_NT
                    int ii = pk_row(tid + nbt), ll = tid + nbt - ii * (ii + 1) / 2;
                    while (ii < nt) {
                        const int i = je + ii, l = je + ll;
                        G[pk(i, l)] -= fx_dot<FILL_B>(fx, nmax, i, l);
                        ll += FILL_NT;
                        while (ll > ii) {
                            ll -= ii + 1;
                            ++ii;
                        }
                    }
                }
            } else {
                // the block's L entries, as double-float pairs, now that the workers have read its
                // unscaled entries; then the next block: its update, and its factorisation
                const int bs = je - J;
                if (lane < bs) {
#pragma unroll
                    for (int c = 0; c < FILL_B - 1; ++c)
                        if (c < lane) {
                            float h, l;
                            f64_split(lb[c], h, l);
                            reinterpret_cast<float2*>(G)[pk(J + lane, J + c)] = make_float2(h, l);
                        }
                }
                if (je < nn) {
                    const int bs2 = min(FILL_B, nn - je);
                    if (lane < bs2 * (bs2 + 1) / 2) {
                        const int ii = pk_row(lane), ll = lane - ii * (ii + 1) / 2;
                        G[pk(je + ii, je + ll)] -= fx_dot<FILL_B>(fx, nmax, je + ii, je + ll);
                    }
                    __syncwarp();
                    factor_block(je, bs2);
                }
            }
            __syncthreads();
        }
        __syncthreads();
        if (s_bad) {
            if (tid == 0) record_error(st, SIC_ERR_NOT_PD, u);
            __syncthreads();
            continue;
        }
        // member a: with G = L D^{1/2}, G^-T e_jb = d_jb^{-1/2} L^-T e_jb (jb = nn-1-a): a
        // back substitution with the unit upper L^T, scaled once.  Members go in pairs
        // (2p, 2p+1), one pair per warp, one member per half-warp; the right-hand side lives in
        // registers (lane h*16 + r of half h owns entries r + 16 q).  The two members' jb
        // differ by one, so each warp instruction serves both, in 16-lane instead of 32-lane
        // granularity.  The substitution runs in double-float on the FP32 pipe (about 15 FP32
        // instructions per multiply-add against one FP64 instruction that holds this GPU's FP64
        // pipe for some 64 clocks per warp): its relative error, about 2^-47 per operation,
        // stays some 1e-13 of the column at the conditioning of these blocks, against the
        // factorisation's own rounding.
        const int npairs = (m + 1) / 2;
        const int half = lane >> 4, hl = lane & 15;
        for (int p = worker ? warp : npairs; p < npairs; p += FILL_NT / 32) {
            const int a = 2 * p + half;
            const bool has = a < m;
            const int jb = has ? nn - 1 - a : -1;
            const int jtop = nn - 1 - 2 * p;
            // slots 2j and 2j+1 in the .x and .y halves of bh[j], bl[j] (packed updates); in the
            // block of rows l of slot sb, the slots below sb take every row, slot sb the rows
            // above its entry, and a slot above sb none: those get a = 0
            const float2* Lf = reinterpret_cast<const float2*>(G);  // the L entries (hi, lo)
            float2 bh[FILL_HSLOTS / 2], bl[FILL_HSLOTS / 2];
#pragma unroll
            for (int j = 0; j < FILL_HSLOTS / 2; ++j) {
                bh[j] = make_float2((hl + 32 * j == jb) ? 1.f : 0.f, (hl + 32 * j + 16 == jb) ? 1.f : 0.f);
                bl[j] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int sb = FILL_HSLOTS - 1; sb >= 0; --sb) {
                if (16 * sb > jtop) continue;
                const int top = min(jtop, 16 * sb + 15);
                for (int l = top; l >= 16 * sb; --l) {
                    const int src = (lane & 16) | (l & 15);
                    const float yh = __shfl_sync(0xffffffffu, (sb & 1) ? bh[sb / 2].y : bh[sb / 2].x, src);
                    const float yl = __shfl_sync(0xffffffffu, (sb & 1) ? bl[sb / 2].y : bl[sb / 2].x, src);
                    const int rl = pk(l, 0);
#pragma unroll
                    for (int j = 0; 2 * j <= sb; ++j) {
                        const int i0 = hl + 32 * j, i1 = i0 + 16;
                        const float2 a0 = (2 * j < sb || i0 < l) ? Lf[rl + i0] : make_float2(0.f, 0.f);
                        const float2 a1 = (2 * j + 1 < sb || i1 < l) ? Lf[rl + i1] : make_float2(0.f, 0.f);
                        df_sub_mul2(bh[j], bl[j], a0, a1, yh, yl);
                    }
                }
            }
            if (has) {
                const long long e0 = col_ptr[c0 + a] - base;
                const double sc = rsqrt_newton(G[pk(jb, jb)]);
#pragma unroll
                for (int q = 0; q < FILL_HSLOTS; ++q) {
                    const int i = hl + 16 * q;
                    if (i <= jb) {
                        const float h = (q & 1) ? bh[q / 2].y : bh[q / 2].x;
                        const float l = (q & 1) ? bl[q / 2].y : bl[q / 2].x;
                        row_idx[e0 + jb - i] = pos[i];
                        val[e0 + jb - i] = (f32_as_f64(h) + f32_as_f64(l)) * sc;
                    }
                }
            }
        }
        // log v of every member, one member per thread (the FP64 log once per lane instead of
        // once per warp)
        for (int a = worker ? tid : m; a < m; a += FILL_NT) logv[c0 + a] = log(G[pk(nn - 1 - a, nn - 1 - a)]);
        __syncthreads();
    }
}

// Fixed-order sum: each block reduces a contiguous tile; then one block adds the tiles.
__global__ void __launch_bounds__(256) k_sum_tiles(const double* __restrict__ x, long long n,
                                                   double* __restrict__ partial) {
    __shared__ double s[256];
    long long base = blockIdx.x * (long long)SUM_TILE;
    double acc = 0.0;
    for (int i = threadIdx.x; i < SUM_TILE; i += 256)
        if (base + i < n) acc += x[base + i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) s[threadIdx.x] += s[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(256) k_sum_final(const double* __restrict__ partial, long long nb,
                                                   double* __restrict__ out) {
    __shared__ double s[256];
    double acc = 0.0;
    for (long long i = threadIdx.x; i < nb; i += 256) acc += partial[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) s[threadIdx.x] += s[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

size_t fill_smem_bytes(int k, int max_m) {
    const int nmax = k + max_m;
    return sizeof(double) * ((size_t)nmax * (nmax + 1) / 2 + 4 + EXP_TAB + fill_scratch_doubles(nmax)) +
           sizeof(int) * ((size_t)nmax + (size_t)k);
}

__global__ void k_fp64_math(KP<double> kp, const double* __restrict__ x, long long n, double* __restrict__ os,
                            double* __restrict__ orr, double* __restrict__ oe, double* __restrict__ ok) {
    __shared__ double tab[EXP_TAB], tab_s2[EXP_TAB];
    exp_table_fill(tab);
    exp_table_fill(tab_s2, kp.s2);
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        os[i] = sqrt_newton(v);
        orr[i] = v > 0.0 ? rsqrt_newton(v) : 0.0;
        oe[i] = exp_neg_table(-v, tab);
        ok[i] = matern_d2_fast(kp, v, tab_s2);
    }
}

// out[i] = the double-float Matern between points pa[i] and pb[i] (n x dim each), with pa[i]
// as the origin of the coordinates, as the fill evaluates its entries
__global__ void k_matern_df(KP<double> kp, int dim, const double* __restrict__ pa, const double* __restrict__ pb,
                            long long n, double* __restrict__ out) {
    __shared__ float tab_hi[DF_EXP_TAB], tab_lo[DF_EXP_TAB];
    __shared__ float xh[3 * 2 * 256], xl[3 * 2 * 256];
    df_exp_table_fill(tab_hi, tab_lo, kp.s2);
    __syncthreads();
    const DfMatern dfk = df_matern_params(kp);
    const int t = threadIdx.x;
    for (long long i0 = blockIdx.x * 256LL; i0 < n; i0 += 256LL * gridDim.x) {
        const long long i = i0 + t;
        for (int d = 0; d < 3; ++d) {
            const dfl c = df_from_double((i < n && d < dim) ? pb[i * dim + d] - pa[i * dim + d] : 0.0);
            xh[d * 512 + t] = 0.f;
            xl[d * 512 + t] = 0.f;
            xh[d * 512 + 256 + t] = c.hi;
            xl[d * 512 + 256 + t] = c.lo;
        }
        if (i < n) out[i] = matern_df(dfk, xh, xl, t, 256 + t, 512, dim, tab_hi, tab_lo);
    }
}

// the fill's integer routines on independent inputs: d2[i] = fx_dist2 of points pa[i], pb[i]
// (each dimension's fixed-point exponent the larger of the two points'), dot[i] = fx_dot of the
// 4-vectors ga[i], gb[i] (each stored by fx_row_store); one thread per i
__global__ void k_fixed_point(const double* __restrict__ pa, const double* __restrict__ pb, long long n, int dim,
                              double* __restrict__ d2, const double* __restrict__ ga, const double* __restrict__ gb,
                              double* __restrict__ dot) {
    __shared__ __align__(16) int fx[9 * 2 * 256];  // two rows per thread, ld = 512
    __shared__ long long xf[3 * 512];
    const int t = threadIdx.x;
    for (long long i = blockIdx.x * 256LL + t; i - t < n; i += 256LL * gridDim.x) {
        const bool live = i < n;
        int E[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) {
            const double a = live ? pa[i * dim + d] : 0.0, b = live ? pb[i * dim + d] : 0.0;
            E[d] = max((int)(((unsigned)__double2hiint(a) >> 20) & 0x7ffu), (int)(((unsigned)__double2hiint(b) >> 20) & 0x7ffu));
            xf[d * 512 + 2 * t] = fx_coord(a, E[d]);
            xf[d * 512 + 2 * t + 1] = fx_coord(b, E[d]);
        }
        double g1[4], g2[4];
        for (int j = 0; j < 4; ++j) {
            g1[j] = live ? ga[i * 4 + j] : 0.0;
            g2[j] = live ? gb[i * 4 + j] : 0.0;
        }
        fx_row_store<4>(g1, fx, 512, 2 * t);
        fx_row_store<4>(g2, fx, 512, 2 * t + 1);
        __syncthreads();
        if (live) {
            d2[i] = fx_dist2(xf, 512, dim, 2 * t, 2 * t + 1, E[0], E[1], E[2]);
            dot[i] = fx_dot<4>(fx, 512, 2 * t, 2 * t + 1);
        }
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------- entry points --

extern "C" sic_status sic_selftest_fixed_point(sic_handle* h, const double* pa, const double* pb, int64_t n,
                                               int32_t dim, double* d2, const double* ga, const double* gb,
                                               double* dot, void* stream) {
    if (!h || n < 0 || dim < 1 || dim > 3 || (n > 0 && (!pa || !pb || !d2 || !ga || !gb || !dot)))
        return SIC_ERR_INVALID;
    if (n == 0) return SIC_OK;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    long long blocks = (n + 255) / 256;
    if (blocks > 4LL * h->num_sms) blocks = 4LL * h->num_sms;
    k_fixed_point<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(pa, pb, n, dim, d2, ga, gb, dot);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_selftest_matern_df(sic_handle* h, const sic_kernel* kp, const double* pa, const double* pb,
                                             int64_t n, double* out, void* stream) {
    if (!h || !sic_valid_kernel(kp) || n < 0 || (n > 0 && (!pa || !pb || !out))) return SIC_ERR_INVALID;
    if (n == 0) return SIC_OK;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    long long blocks = (n + 255) / 256;
    if (blocks > 4LL * h->num_sms) blocks = 4LL * h->num_sms;
    k_matern_df<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(make_kp<double>(*kp), kp->dim, pa, pb, n, out);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_selftest_fp64_math(sic_handle* h, const sic_kernel* kp, const double* x, int64_t n,
                                             double* out_sqrt, double* out_rsqrt, double* out_exp,
                                             double* out_kernel, void* stream) {
    if (!h || !sic_valid_kernel(kp) || n < 0 || (n > 0 && (!x || !out_sqrt || !out_rsqrt || !out_exp || !out_kernel)))
        return SIC_ERR_INVALID;
    if (n == 0) return SIC_OK;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    long long blocks = (n + 255) / 256;
    if (blocks > 4LL * h->num_sms) blocks = 4LL * h->num_sms;
    k_fp64_math<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(make_kp<double>(*kp), x, n, out_sqrt, out_rsqrt,
                                                                     out_exp, out_kernel);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_factor_nnz_workspace(int64_t n, size_t* bytes) {
    if (!bytes || n < 0) return SIC_ERR_INVALID;
    long long nb = (n + 1 + SCAN_TILE - 1) / SCAN_TILE;
    *bytes = sizeof(long long) * (size_t)(nb + 1);
    return SIC_OK;
}

// count + exclusive scan of the columns col0 .. col0 + n_cols - 1 into col_ptr[0 .. n_cols],
// offsets starting at `base`; `partial` holds the tile totals (nb + 1 entries)
static sic_status launch_nnz(sic_handle* h, const int64_t* grp_ptr, int64_t n_grp, const int32_t* sel_count,
                             long long col0, long long n_cols, long long base, long long* v, long long* partial,
                             cudaStream_t s) {
    const long long len = n_cols + 1;
    const long long nb = (len + SCAN_TILE - 1) / SCAN_TILE;
    SIC_CUDA_TRY(cudaMemsetAsync(v + n_cols, 0, sizeof(long long), s));
    k_nnz_count<<<(unsigned)((n_grp + 255) / 256), 256, 0, s>>>((const long long*)grp_ptr, n_grp, sel_count, col0,
                                                                  n_cols, v, h->d_status);
    k_scan_tile<<<(unsigned)nb, 256, 0, s>>>(v, len, partial);
    k_scan_partials<<<1, 256, 0, s>>>(partial, nb, partial + nb);
    k_scan_add<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(v, len, partial, base);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_factor_nnz_range(sic_handle* h, const int64_t* grp_ptr, int64_t n_grp,
                                           const int32_t* sel_count, int64_t col0, int64_t n_cols, int64_t base,
                                           int64_t* col_ptr, void* ws, size_t ws_bytes, void* stream) {
    if (!h || !sel_count || !col_ptr || col0 < 0 || n_cols < 1 || n_grp < 1 || base < 0 ||
        (!grp_ptr && n_grp != n_cols))
        return SIC_ERR_INVALID;
    size_t need = 0;
    sic_factor_nnz_workspace(n_cols, &need);
    if (!ws || ws_bytes < need) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    return launch_nnz(h, grp_ptr, n_grp, sel_count, col0, n_cols, base, (long long*)col_ptr, (long long*)ws,
                      (cudaStream_t)stream);
}

extern "C" sic_status sic_factor_nnz(sic_handle* h, const int64_t* grp_ptr, int64_t n_grp, const int32_t* sel_count,
                                     int64_t n, int64_t* col_ptr, void* ws, size_t ws_bytes, void* stream) {
    return sic_factor_nnz_range(h, grp_ptr, n_grp, sel_count, 0, n, 0, col_ptr, ws, ws_bytes, stream);
}

// sum of log v in a fixed order (two launches), shared with the partial-pattern fill
// bytes of the fixed-order sum's tile partials at the front of the fill's workspace
static size_t fill_partials_bytes(long long n) {
    const long long nb = (n + SUM_TILE - 1) / SUM_TILE;
    return sizeof(double) * (size_t)(nb > 0 ? nb : 1);
}

sic_status launch_sum_logv(const double* logv, long long n, double* sum_logv, void* ws, cudaStream_t s) {
    long long nb = (n + SUM_TILE - 1) / SUM_TILE;
    k_sum_tiles<<<(unsigned)nb, 256, 0, s>>>(logv, n, (double*)ws);
    k_sum_final<<<1, 256, 0, s>>>((const double*)ws, nb, sum_logv);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_build_factor_workspace(int64_t n, size_t* bytes) {
    if (!bytes || n < 0) return SIC_ERR_INVALID;
    *bytes = fill_partials_bytes(n) + 2 * sizeof(unsigned long long);  // partial sums, then two work counters
    return SIC_OK;
}

extern "C" sic_status sic_build_factor_range(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                             const int64_t* grp_ptr, int64_t n_grp, int32_t max_m,
                                             const int32_t* sel_idx, const int32_t* sel_count, int32_t k,
                                             int64_t col0, int64_t n_cols, const int64_t* col_ptr, int64_t base,
                                             int32_t* row_idx, double* val, double* logv, double* sum_logv, void* ws,
                                             size_t ws_bytes, void* stream) {
    if (!h || !pts || !sic_valid_kernel(kp) || n < 1 || n_grp < 1 || !sel_count || !col_ptr || !row_idx || !val ||
        !logv || !sum_logv || k < 0 || (k > 0 && !sel_idx) || col0 < 0 || n_cols < 1 || col0 + n_cols > n ||
        base < 0)
        return SIC_ERR_INVALID;
    if (!grp_ptr && (n_grp != n_cols || max_m != 1)) return SIC_ERR_INVALID;
    if (max_m < 1) return SIC_ERR_INVALID;
    if (max_m > 64 || k > 128) return SIC_ERR_UNSUPPORTED;
    size_t need = 0;
    sic_build_factor_workspace(n_cols, &need);
    if (!ws || ws_bytes < need) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (fill_smem_bytes(k, max_m) > 227 * 1024) return SIC_ERR_UNSUPPORTED;
    // two size classes when the groups can be large: the shared-memory layout (and so the
    // CTAs per SM) of each launch fits its own largest group, so the many small groups run
    // at higher occupancy; each launch skips the other's groups
    // the size-class split: tuned for this (k, max_m) by sic_tune_build_factor, else FILL_M_SPLIT
    int split = tune_get(h, TUNE_FILL_SPLIT, k, max_m, FILL_M_SPLIT);
    if (split > max_m) split = max_m;
    if (split < 1) split = 1;
    const int big_nt = tune_get(h, TUNE_FILL_BIGNT, k, max_m, 256) == 384 ? 384 : 256;
    // the two launches' work counters, after the partial sums in the workspace
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(
        reinterpret_cast<char*>(ws) + fill_partials_bytes(n_cols));
    SIC_CUDA_TRY(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), s));
    for (int c = 0; c < 2; ++c) {
        const int lo = c == 0 ? 1 : split + 1, hi = c == 0 ? split : max_m;
        if (lo > hi) break;
        const size_t sm = fill_smem_bytes(k, hi);
        // worker threads: at least one per row of the largest unit (k + hi)
        const int nt = (c == 0 && k + hi <= 128) ? 128 : (c == 0 || big_nt != 384 ? 256 : 384);
        auto kern = nt == 128 ? k_fill<128> : (nt == 384 ? k_fill<384> : k_fill<256>);
        const int block = nt + 32;
        SIC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const int grid = persistent_grid(h, kern, block, sm, n_grp);
        kern<<<grid, block, sm, s>>>(pts, kp->dim, make_kp<double>(*kp), (const long long*)grp_ptr, n_grp, sel_idx,
                                     sel_count, k, max_m, lo, hi, n, col0, n_cols, (const long long*)col_ptr, base,
                                     row_idx, val, logv, ctr + c, h->d_status);
    }
    long long nb = (n_cols + SUM_TILE - 1) / SUM_TILE;
    k_sum_tiles<<<(unsigned)nb, 256, 0, s>>>(logv, n_cols, (double*)ws);
    k_sum_final<<<1, 256, 0, s>>>((const double*)ws, nb, sum_logv);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_build_factor(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                       const int64_t* grp_ptr, int64_t n_grp, int32_t max_m, const int32_t* sel_idx,
                                       const int32_t* sel_count, int32_t k, const int64_t* col_ptr,
                                       int32_t* row_idx, double* val, double* logv, double* sum_logv, void* ws,
                                       size_t ws_bytes, void* stream) {
    return sic_build_factor_range(h, pts, n, kp, grp_ptr, n_grp, max_m, sel_idx, sel_count, k, 0, n, col_ptr, 0,
                                  row_idx, val, logv, sum_logv, ws, ws_bytes, stream);
}

extern "C" sic_status sic_sum_fixed(sic_handle* h, const double* x, int64_t n, double* sum, void* ws, size_t ws_bytes,
                                    void* stream) {
    if (!h || !x || !sum || n < 1) return SIC_ERR_INVALID;
    size_t need = 0;
    sic_build_factor_workspace(n, &need);
    if (!ws || ws_bytes < need) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    return launch_sum_logv(x, n, sum, ws, (cudaStream_t)stream);
}

// ------------------------------------------------ allocation-free nnz scan --
//
// sic_factor_nnz_noalloc runs the same count + scan kernels as sic_factor_nnz, with
// the per-tile totals kept in this file-scope device array instead of a caller
// workspace.  Every GPU that loads libsic holds one copy until the process exits.
namespace {

constexpr long long NOALLOC_MAX_TILES = 65536;  // n + 1 <= 65536 * SCAN_TILE = 67,108,864 entries
static __device__ __align__(256) long long g_nnz_scratch[NOALLOC_MAX_TILES + 1];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
long long* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_nnz_scratch on `device` (the current device).  In host code the
// array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress.  Outside stream capture it is looked up on every call (a reset of
// the device or a new primary context may load the module at another address); during a
// capture the address of the last lookup on this device is used, so one call must have
// been made on the device before the capture began.
cudaError_t noalloc_scratch(int device, cudaStream_t s, long long** out) {
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (cap == cudaStreamCaptureStatusNone || !g_noalloc_addr[device]) {
        if (cap != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_nnz_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[device] = (long long*)ptr;
    }
    *out = g_noalloc_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" sic_status sic_factor_nnz_noalloc(sic_handle* h, const int64_t* grp_ptr, int64_t n_grp,
                                             const int32_t* sel_count, int64_t n, int64_t* col_ptr, void* stream) {
    if (!h || !sel_count || !col_ptr || n < 1 || n_grp < 1 || (!grp_ptr && n_grp != n)) return SIC_ERR_INVALID;
    const long long len = n + 1;
    const long long nb = (len + SCAN_TILE - 1) / SCAN_TILE;
    if (nb > NOALLOC_MAX_TILES) return SIC_ERR_UNSUPPORTED;  // beyond the static scratch
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    long long* partial = nullptr;
    SIC_CUDA_TRY(noalloc_scratch(h->device, s, &partial));
    long long* v = (long long*)col_ptr;
    // the tile totals are written before they are read, so the scratch needs no clearing;
    // only the output's last entry must start at zero (as in sic_factor_nnz)
    return launch_nnz(h, grp_ptr, n_grp, sel_count, 0, n, 0, v, partial, s);
}
