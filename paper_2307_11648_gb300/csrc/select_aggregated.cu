// Supernodal greedy selection (Section 5.2, multiple targets sharing one selection).
// (FP32 with at most 256 candidates, m <= 64 and k <= 64 goes to the register-resident
// kernel of select_agg_reg.cu.)
//
// One CTA owns one group at a time over a persistent grid.  The two partial Cholesky
// factors of the paper's Cholesky approach (Appendix C.2) live in shared memory when
// they fit (e.g. 256 candidates in FP32) and otherwise in a per-CTA slab of the
// caller's workspace.  Layout (elements of T), column-major so that thread r touches
// row r of every column:
//   F1  [k][Cm]       columns of the picks, conditioned on earlier picks only;
//   F2c [mm+k][Cm]    candidate rows of F2: first the m target columns (left-looking
//                     Cholesky of the targets), then the picks conditioned on targets
//                     and earlier picks;
//   F2t [mm][mm]      target rows of the m target columns (only they are non-zero);
//   X   [3][Cm+mm]    staged coordinates, candidates then targets (FP32 mode: relative
//                     to the first member, formed in FP64);
//   V1, V2 [Cm]       var_j = Theta_{jj|I} and var_j|P = Theta_{jj|I,P}.
// Cm = max_cand rounded up to 32, mm = max_m.
// Per step the score is V1_j / V2_j (eq. greedy_mult: picking j changes
// logdet Theta_{PP|I} by log V2_j - log V1_j); the argmax (ties: lowest candidate
// index) is found by warp shuffles and one shared-memory pass; the pivot rows of F1
// and F2 are staged in shared memory and every thread appends its entries of the two
// new columns (left-looking) and downdates V1 and V2.  Picked rows are marked by
// V2 = -inf.
#include "sic_internal.cuh"

namespace {

template <typename T>
__device__ __forceinline__ bool better(T s, int i, T bs, int bi) {
    return s > bs || (s == bs && i < bi);
}

// acc - sum_{tau < len} col[tau * ld] * piv[tau], with four independent partial sums so
// that the loads of consecutive terms are in flight together
template <typename T>
__device__ __forceinline__ T dot_down(T acc, const T* __restrict__ col, long long ld, const T* __restrict__ piv,
                                      int len) {
    T a1 = (T)0, a2 = (T)0, a3 = (T)0;
    int tau = 0;
    for (; tau + 4 <= len; tau += 4) {
        acc = fma(-col[(long long)tau * ld], piv[tau], acc);
        a1 = fma(-col[(long long)(tau + 1) * ld], piv[tau + 1], a1);
        a2 = fma(-col[(long long)(tau + 2) * ld], piv[tau + 2], a2);
        a3 = fma(-col[(long long)(tau + 3) * ld], piv[tau + 3], a3);
    }
    for (; tau < len; ++tau) acc = fma(-col[(long long)tau * ld], piv[tau], acc);
    return (acc + a1) + (a2 + a3);
}

// Shared-memory variant: factor rows are row-major with a pitch of 4 (mod 32) elements, so
// that a thread reads its own row, and every thread the broadcast pivot row, with 128-bit
// loads without bank conflicts.  Workspace variant: column-major [column][row], so that
// the threads of a warp touch consecutive addresses.
__host__ __device__ inline long long pitch4(long long x) { return ((x + 27) / 32) * 32 + 4; }

struct AggLayout {
    long long Cm, mm, k;
    bool rowmajor;
    __host__ __device__ long long p1() const { return pitch4(k); }
    __host__ __device__ long long p2() const { return pitch4(mm + k); }
    __host__ __device__ long long p2t() const { return pitch4(mm); }
    __host__ __device__ long long f1() const { return 0; }
    __host__ __device__ long long f2c() const { return rowmajor ? Cm * p1() : k * Cm; }
    __host__ __device__ long long f2t() const { return f2c() + (rowmajor ? Cm * p2() : (mm + k) * Cm); }
    __host__ __device__ long long x() const { return f2t() + (rowmajor ? mm * p2t() : mm * mm); }
    __host__ __device__ long long v1() const { return x() + 3 * (Cm + mm); }
    __host__ __device__ long long v2() const { return v1() + Cm; }
    __host__ __device__ long long size() const { return (v2() + Cm + 3) / 4 * 4; }
};

inline AggLayout agg_layout(int max_cand, int max_m, int k, bool rowmajor) {
    AggLayout L;
    L.Cm = ((long long)max_cand + 31) / 32 * 32;
    if (L.Cm < 32) L.Cm = 32;
    L.mm = max_m;
    L.k = k;
    L.rowmajor = rowmajor;
    return L;
}

// acc - sum_{tau < len} row[tau] * piv[tau] over a contiguous row (shared memory)
template <typename T>
__device__ __forceinline__ T dot_row(T acc, const T* __restrict__ row, const T* __restrict__ piv, int len) {
    T a1 = (T)0, a2 = (T)0, a3 = (T)0;
    int tau = 0;
    if constexpr (sizeof(T) == 4) {
        const float4* r4 = reinterpret_cast<const float4*>(row);
        const float4* p4 = reinterpret_cast<const float4*>(piv);
        for (; tau + 4 <= len; tau += 4) {
            const float4 a = r4[tau >> 2], b = p4[tau >> 2];
            acc = fmaf(-a.x, b.x, acc);
            a1 = fmaf(-a.y, b.y, a1);
            a2 = fmaf(-a.z, b.z, a2);
            a3 = fmaf(-a.w, b.w, a3);
        }
    } else {
        for (; tau + 4 <= len; tau += 4) {
            acc = fma(-row[tau], piv[tau], acc);
            a1 = fma(-row[tau + 1], piv[tau + 1], a1);
            a2 = fma(-row[tau + 2], piv[tau + 2], a2);
            a3 = fma(-row[tau + 3], piv[tau + 3], a3);
        }
    }
    for (; tau < len; ++tau) acc = fma(-row[tau], piv[tau], acc);
    return (acc + a1) + (a2 + a3);
}

template <typename T, int NT, bool SMEM>
__global__ void __launch_bounds__(NT, 1) k_select_agg(
    const double* __restrict__ pts, long long n, int dim, KP<T> kp, T floor_, const long long* __restrict__ grp_ptr,
    long long n_grp, const long long* __restrict__ cand_ptr, const int32_t* __restrict__ cand_idx, int max_cand,
    int max_m, int k, int32_t* __restrict__ sel_idx, int32_t* __restrict__ sel_count, T* __restrict__ ws,
    AggLayout L, double* __restrict__ gain, DevStatus* st) {
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* base = SMEM ? sm : ws + (long long)blockIdx.x * L.size();
    T* p1 = SMEM ? sm + L.size() : sm;       // k (16-byte aligned: L.size() is a multiple of 4)
    T* p2 = p1 + (k + 3) / 4 * 4;             // max_m + k
    __shared__ T wsc[NW];
    __shared__ int wix[NW];
    __shared__ int s_fail;
    __shared__ double gv1[128], gv2[128];  // the picks' two conditional variances (gains only)
    __shared__ int qs[128];                // the picks' candidate rows, translated after the steps

    const long long Cm = L.Cm, mm = L.mm, ldx = L.Cm + L.mm;
    const long long P1 = L.p1(), P2 = L.p2(), P2t = L.p2t();
    // element (row, column) of F1, F2c (candidate rows) and F2t (target rows)
#define E1(r, c) (SMEM ? F1[(long long)(r) * P1 + (c)] : F1[(long long)(c) * Cm + (r)])
#define E2(r, c) (SMEM ? F2c[(long long)(r) * P2 + (c)] : F2c[(long long)(c) * Cm + (r)])
#define E2T(a, c) (SMEM ? F2t[(long long)(a) * P2t + (c)] : F2t[(long long)(c) * mm + (a)])
    T* F1 = base + L.f1();
    T* F2c = base + L.f2c();
    T* F2t = base + L.f2t();
    T* X = base + L.x();
    T* V1 = base + L.v1();
    T* V2 = base + L.v2();

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T NEG = -INFINITY;
    const T diag = kp.s2 + kp.nugget;
    // FP64: Theta by the fill's table-driven exp and Newton square root (about 2 ulp); the
    // table s2 2^(j/256) follows the pivot rows
    double* tab = reinterpret_cast<double*>(p2 + (L.mm + k));
    if constexpr (sizeof(T) == 8) {
        exp_table_fill(tab, kp.s2);
        __syncthreads();
    }
    auto theta = [&](T d2) -> T {
        if constexpr (sizeof(T) == 8)
            return matern_d2_fast(kp, d2, tab);
        else
            return matern<T>(kp, sic_sqrt(d2));
    };
    auto rsqrt_t = [](T v) -> T {
        if constexpr (sizeof(T) == 8)
            return rsqrt_newton(v);
        else
            return (T)1 / sic_sqrt(v);
    };

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
        double org[3] = {0.0, 0.0, 0.0};
        if constexpr (sizeof(T) == 4)
            for (int d = 0; d < dim; ++d) org[d] = pts[g0 * dim + d];
        for (int i = tid; i < C + m; i += NT) {
            const bool cnd = i < C;
            long long p = cnd ? (long long)cand_idx[b0 + i] : g0 + (i - C);
            const long long xi = cnd ? i : Cm + (i - C);
            bool ok = true;
            if (cnd && (p < g0 + m || p >= n)) {  // candidates must lie after the group
                record_error(st, SIC_ERR_INVALID, g);
                p = g0;
                ok = false;
            }
            for (int d = 0; d < 3; ++d) X[d * ldx + xi] = (d < dim) ? (T)(pts[p * dim + d] - org[d]) : (T)0;
            if (cnd) {
                V1[i] = ok ? diag : NEG;
                V2[i] = ok ? diag : NEG;
            }
        }
        if (tid == 0) s_fail = 0;
        __syncthreads();

        // ---- the target columns of F2 (left-looking Cholesky of the targets) ----
        for (int a = 0; a < m; ++a) {
            if (tid < a) p2[tid] = E2T(a, tid);
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
            const T dsq = sic_sqrt(dv);
            const T rs = (T)1 / dsq;
            const long long xa = Cm + a;
            const T ax = X[xa], ay = X[ldx + xa], az = X[2 * ldx + xa];
            for (int i = tid; i < C + m; i += NT) {
                if (i < C) {
                    T dx = X[i] - ax, dy = X[ldx + i] - ay, dz = X[2 * ldx + i] - az;
                    T num = theta(fma(dz, dz, fma(dy, dy, dx * dx)));
                    num = SMEM ? dot_row(num, F2c + (long long)i * P2, p2, a) : dot_down(num, F2c + i, Cm, p2, a);
                    const T u = num * rs;
                    E2(i, a) = u;
                    V2[i] = fma(-u, u, V2[i]);
                } else {
                    const int ta = i - C;
                    T u;
                    if (ta < a) {
                        u = (T)0;
                    } else if (ta == a) {
                        u = dsq;
                    } else {
                        const long long xt = Cm + ta;
                        T dx = X[xt] - ax, dy = X[ldx + xt] - ay, dz = X[2 * ldx + xt] - az;
                        T num = theta(fma(dz, dz, fma(dy, dy, dx * dx)));
                        num = SMEM ? dot_row(num, F2t + (long long)ta * P2t, p2, a) : dot_down(num, F2t + ta, mm, p2, a);
                        u = num * rs;
                    }
                    E2T(ta, a) = u;
                }
            }
            __syncthreads();
        }
        __syncthreads();
        int t = 0;
        if (!s_fail) {
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
                const T qx = X[q], qy = X[ldx + q], qz = X[2 * ldx + q];
                for (int tau = tid; tau < t; tau += NT) p1[tau] = E1(q, tau);
                for (int tau = tid; tau < m + t; tau += NT) p2[tau] = E2(q, tau);
                __syncthreads();
                const T r1 = rsqrt_t(v1q);
                const T r2 = rsqrt_t(v2q);
                for (int r = tid; r < C; r += NT) {
                    if (V2[r] == NEG) continue;
                    T dx = X[r] - qx, dy = X[ldx + r] - qy, dz = X[2 * ldx + r] - qz;
                    T th = theta(fma(dz, dz, fma(dy, dy, dx * dx)));
                    if (r == q) th += kp.nugget;
                    const T n1 = SMEM ? dot_row(th, F1 + (long long)r * P1, p1, t) : dot_down(th, F1 + r, Cm, p1, t);
                    const T n2 = SMEM ? dot_row(th, F2c + (long long)r * P2, p2, m + t)
                                      : dot_down(th, F2c + r, Cm, p2, m + t);
                    const T u1 = n1 * r1, u2 = n2 * r2;
                    E1(r, t) = u1;
                    E2(r, m + t) = u2;
                    if (r == q) {
                        V1[r] = NEG;
                        V2[r] = NEG;
                    } else {
                        V1[r] = fma(-u1, u1, V1[r]);
                        V2[r] = fma(-u2, u2, V2[r]);
                    }
                }
                if (tid == 0) {
                    qs[t] = q;  // no global load on the step chain
                    if (gain) {
                        gv1[t] = (double)v1q;
                        gv2[t] = (double)v2q;
                    }
                }
            }
        }
        // the picks' global indices and (with gain) the decreases of logdet Theta_{PP|I} per
        // nonzero (Section 5.4.2), off the step chain
        __syncthreads();
        for (int q = tid; q < t; q += NT) {
            sel_idx[g * k + q] = cand_idx[b0 + qs[q]];
            if (gain) gain[g * k + q] = log(gv1[q] / gv2[q]) / m;
        }
        if (tid == 0) sel_count[g] = t;
        for (int q = t + tid; q < k; q += NT) sel_idx[g * k + q] = -1;
        __syncthreads();
    }
}

#undef E1
#undef E2
#undef E2T

constexpr size_t SMEM_LIMIT = 227 * 1024 - 4096;  // dynamic part; the static arrays take < 4 KB

template <typename T>
size_t agg_smem_bytes(const AggLayout& L, bool in_smem) {
    size_t piv = sizeof(T) * (size_t)((L.k + 3) / 4 * 4 + L.mm + L.k);
    const size_t tab = sizeof(T) == 8 ? sizeof(double) * EXP_TAB : 0;  // the FP64 Matern's exp table
    return (in_smem ? sizeof(T) * (size_t)L.size() + piv : piv) + tab;
}

// Plan of one launch: where the state lives, threads per CTA, grid, workspace.
struct AggPlan {
    AggLayout L;
    bool smem;
    int nt;
    int grid;
    size_t smem_bytes;
    size_t ws_bytes;
};

template <typename T, int NT, bool SMEM>
int agg_grid_for(sic_handle* h, size_t smem, long long n_grp) {
    auto kern = k_select_agg<T, NT, SMEM>;
    // opt in at any size: the static arrays count against the 48 KB default as well
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int g = persistent_grid(h, kern, NT, smem, n_grp);
    if (!SMEM) {
        long long cap = 2LL * h->num_sms;  // bound the workspace (and keep the slabs L2-friendly)
        if (g > cap) g = (int)cap;
    }
    return g;
}

// The launch plan: state in shared memory when it fits, 256 threads up to 256 candidates and 512
// beyond -- or, with `variant` (2 * threads + 1 if in shared memory, as the autotuner stores
// it), that plan when it is possible.  Every plan gives the same picks: each candidate row's
// arithmetic and the argmax's tie-break do not depend on the thread count, and the shared-
// memory and workspace dot products sum in the same order.
template <typename T>
AggPlan agg_plan(sic_handle* h, long long n_grp, int max_cand, int max_m, int k, int variant = 0) {
    AggPlan P;
    P.L = agg_layout(max_cand, max_m, k, true);
    P.smem = agg_smem_bytes<T>(P.L, true) <= SMEM_LIMIT;
    P.nt = (max_cand <= 256) ? 256 : 512;
    if (variant) {
        const int vnt = variant / 2;
        if (vnt == 256 || vnt == 512) P.nt = vnt;
        if (!(variant & 1)) P.smem = false;
    }
    if (!P.smem) P.L = agg_layout(max_cand, max_m, k, false);
    P.smem_bytes = agg_smem_bytes<T>(P.L, P.smem);
    long long work = n_grp > 0 ? n_grp : 1;
    if (P.nt == 256)
        P.grid = P.smem ? agg_grid_for<T, 256, true>(h, P.smem_bytes, work)
                        : agg_grid_for<T, 256, false>(h, P.smem_bytes, work);
    else
        P.grid = P.smem ? agg_grid_for<T, 512, true>(h, P.smem_bytes, work)
                        : agg_grid_for<T, 512, false>(h, P.smem_bytes, work);
    P.ws_bytes = P.smem ? 0 : sizeof(T) * (size_t)P.L.size() * (size_t)P.grid;
    return P;
}

}  // namespace

extern "C" sic_status sic_select_aggregated_workspace(sic_handle* h, int64_t n_grp, int32_t max_cand,
                                                      int32_t max_m, int32_t k, sic_precision prec,
                                                      size_t* bytes) {
    if (!h || !bytes || n_grp < 0 || max_cand < 0 || max_m < 1 || k < 1) return SIC_ERR_INVALID;
    if (max_m > 64 || max_cand > 4096 || k > 128) return SIC_ERR_UNSUPPORTED;
    if (cudaSetDevice(h->device) != cudaSuccess) return SIC_ERR_CUDA;
    if (agg_reg_applies(prec, max_cand, max_m, k))
        *bytes = agg_reg_workspace(n_grp, max_m);
    else if (prec == SIC_FP64)
        *bytes = agg_plan<double>(h, n_grp, max_cand, max_m, k).ws_bytes;
    else if (prec == SIC_FP32_MIXED)
        *bytes = agg_plan<float>(h, n_grp, max_cand, max_m, k).ws_bytes;
    else
        return SIC_ERR_INVALID;
    return SIC_OK;
}

namespace {
template <typename T>
sic_status launch_agg(sic_handle* h, const double* pts, long long n, const sic_kernel* kp, const int64_t* grp_ptr,
                      int64_t n_grp, const int64_t* cand_ptr, const int32_t* cand_idx, int max_cand, int max_m, int k,
                      int32_t* sel_idx, int32_t* sel_count, double* gain, void* ws, size_t ws_bytes,
                      cudaStream_t s) {
    const int prec = sizeof(T) == 8 ? SIC_FP64 : SIC_FP32_MIXED;
    const int variant = tune_get(h, TUNE_SELECT_AGG, tune_select_key_a(k, prec), tune_select_key_b(max_cand, max_m), 0);
    AggPlan P = agg_plan<T>(h, n_grp, max_cand, max_m, k, variant);
    if (variant && P.ws_bytes > 0 && (!ws || ws_bytes < P.ws_bytes))
        P = agg_plan<T>(h, n_grp, max_cand, max_m, k);  // the tuned plan needs more workspace than given
    if (P.ws_bytes > 0 && (!ws || ws_bytes < P.ws_bytes)) return SIC_ERR_INVALID;
    KP<T> kpt = make_kp<T>(*kp);
    T fl = (T)sic_floor_of(kp);
    const long long* gp = (const long long*)grp_ptr;
    const long long* cp = (const long long*)cand_ptr;
#define SIC_AGG_LAUNCH(NTV, SM)                                                                                   \
    k_select_agg<T, NTV, SM><<<P.grid, NTV, P.smem_bytes, s>>>(pts, n, kp->dim, kpt, fl, gp, n_grp, cp, cand_idx, \
                                                               max_cand, max_m, k, sel_idx, sel_count, (T*)ws,    \
                                                               P.L, gain, h->d_status)
    if (P.nt == 256) {
        if (P.smem) SIC_AGG_LAUNCH(256, true); else SIC_AGG_LAUNCH(256, false);
    } else {
        if (P.smem) SIC_AGG_LAUNCH(512, true); else SIC_AGG_LAUNCH(512, false);
    }
#undef SIC_AGG_LAUNCH
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}
}  // namespace

extern "C" sic_status sic_select_aggregated_gain(sic_handle* h, const double* pts, int64_t n,
                                                 const sic_kernel* kp, const int64_t* grp_ptr, int64_t n_grp,
                                                 const int64_t* cand_ptr, const int32_t* cand_idx, int32_t max_cand,
                                                 int32_t max_m, int32_t k, sic_precision prec, int32_t* sel_idx,
                                                 int32_t* sel_count, double* gain, void* ws, size_t ws_bytes,
                                                 void* stream) {
    if (!h || !pts || !sic_valid_kernel(kp) || !grp_ptr || !cand_ptr || !sel_idx || !sel_count || n < 1 ||
        n_grp < 0 || max_cand < 0 || max_m < 1 || k < 1)
        return SIC_ERR_INVALID;
    if (max_m > 64 || max_cand > 4096 || k > 128) return SIC_ERR_UNSUPPORTED;
    if (n_grp == 0) return SIC_OK;
    if (max_cand > 0 && !cand_idx) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (agg_reg_applies(prec, max_cand, max_m, k))
        return launch_agg_reg(h, pts, n, kp, grp_ptr, n_grp, cand_ptr, cand_idx, max_cand, max_m, k, sel_idx,
                              sel_count, gain, ws, ws_bytes, s);
    if (prec == SIC_FP64)
        return launch_agg<double>(h, pts, n, kp, grp_ptr, n_grp, cand_ptr, cand_idx, max_cand, max_m, k, sel_idx,
                                  sel_count, gain, ws, ws_bytes, s);
    if (prec == SIC_FP32_MIXED)
        return launch_agg<float>(h, pts, n, kp, grp_ptr, n_grp, cand_ptr, cand_idx, max_cand, max_m, k, sel_idx,
                                 sel_count, gain, ws, ws_bytes, s);
    return SIC_ERR_INVALID;
}

extern "C" sic_status sic_select_aggregated(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                            const int64_t* grp_ptr, int64_t n_grp, const int64_t* cand_ptr,
                                            const int32_t* cand_idx, int32_t max_cand, int32_t max_m, int32_t k,
                                            sic_precision prec, int32_t* sel_idx, int32_t* sel_count, void* ws,
                                            size_t ws_bytes, void* stream) {
    return sic_select_aggregated_gain(h, pts, n, kp, grp_ptr, n_grp, cand_ptr, cand_idx, max_cand, max_m, k, prec,
                                      sel_idx, sel_count, nullptr, ws, ws_bytes, stream);
}

// ------------------------------------------------------------------ autotuning --
//
// sic_tune_select_aggregated: every launch plan of this problem's kind that gives the same
// picks (threads per CTA; the generic kernel's state in shared memory or in the workspace,
// where the given workspace holds it) is run three times on the caller's stream and problem,
// the first run warming up; the fastest is kept in the handle for (k, precision, max_cand,
// max_m), later sic_select_aggregated calls launch it, and the outputs of a final run with it
// are left in sel_idx / sel_count.
namespace {
template <typename T>
int agg_variants(sic_handle* h, long long n_grp, int max_cand, int max_m, int k, size_t ws_bytes, int* out) {
    int nv = 0;
    for (int nt : {256, 512})
        for (int sm = 1; sm >= 0; --sm) {
            const int v = 2 * nt + sm;
            AggPlan P = agg_plan<T>(h, n_grp, max_cand, max_m, k, v);
            if (P.nt != nt || (int)P.smem != sm || P.ws_bytes > ws_bytes) continue;  // not possible here
            out[nv++] = v;
        }
    return nv;
}
}  // namespace

extern "C" sic_status sic_tune_select_aggregated(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                                 const int64_t* grp_ptr, int64_t n_grp, const int64_t* cand_ptr,
                                                 const int32_t* cand_idx, int32_t max_cand, int32_t max_m, int32_t k,
                                                 sic_precision prec, int32_t* sel_idx, int32_t* sel_count, void* ws,
                                                 size_t ws_bytes, void* stream, int32_t* choice) {
    if (!h || (prec != SIC_FP64 && prec != SIC_FP32_MIXED) || max_cand < 0 || max_m < 1 || k < 1)
        return SIC_ERR_INVALID;
    if (max_m > 64 || max_cand > 4096 || k > 128) return SIC_ERR_UNSUPPORTED;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    const int a = tune_select_key_a(k, prec), b = tune_select_key_b(max_cand, max_m);
    int vars[4], nv = 0;
    if (agg_reg_applies(prec, max_cand, max_m, k)) {
        vars[nv++] = 256;
        if (max_cand <= 128) vars[nv++] = 128;
    } else if (prec == SIC_FP64) {
        nv = agg_variants<double>(h, n_grp, max_cand, max_m, k, ws ? ws_bytes : 0, vars);
    } else {
        nv = agg_variants<float>(h, n_grp, max_cand, max_m, k, ws ? ws_bytes : 0, vars);
    }
    if (nv == 0) return SIC_ERR_INVALID;  // no plan fits the given workspace
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    SIC_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SIC_ERR_CUDA;
    }
    sic_status st = SIC_OK;
    int best = -1;
    float best_ms = 0.f;
    for (int vi = 0; vi < nv && st == SIC_OK; ++vi) {
        tune_put(h, TUNE_SELECT_AGG, a, b, vars[vi], 0.f);
        float ms = 0.f;
        for (int rep = 0; rep < 3 && st == SIC_OK; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess) st = SIC_ERR_CUDA;
            if (st == SIC_OK)
                st = sic_select_aggregated(h, pts, n, kp, grp_ptr, n_grp, cand_ptr, cand_idx, max_cand, max_m, k, prec,
                                           sel_idx, sel_count, ws, ws_bytes, stream);
            if (st == SIC_OK && cudaEventRecord(e1, s) != cudaSuccess) st = SIC_ERR_CUDA;
            if (st == SIC_OK && cudaEventSynchronize(e1) != cudaSuccess) st = SIC_ERR_CUDA;
            float t = 0.f;
            if (st == SIC_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) st = SIC_ERR_CUDA;
            if (rep == 1 || (rep > 1 && t < ms)) ms = t;
        }
        if (st == SIC_OK && (best < 0 || ms < best_ms)) {
            best = vars[vi];
            best_ms = ms;
        }
    }
    if (st == SIC_OK) {
        tune_put(h, TUNE_SELECT_AGG, a, b, best, best_ms);
        st = sic_select_aggregated(h, pts, n, kp, grp_ptr, n_grp, cand_ptr, cand_idx, max_cand, max_m, k, prec, sel_idx,
                                   sel_count, ws, ws_bytes, stream);
        if (choice) *choice = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}
