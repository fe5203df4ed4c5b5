// FP64 side state of a selection: the picks' conditional variances in FP64.
//
// For the picks q_0, q_1, ... (in pick order) of a unit with targets P (a supernode's m
// members, or one column's target),
//   var1_t = Theta_{q_t q_t | q_0..q_t-1}      the pivot's conditional variance given the
//                                              earlier picks,
//   var2_t = Theta_{q_t q_t | P, q_0..q_t-1}   the same given the targets as well,
// and the pick's decrease of logdet Theta_{PP|I} per nonzero, log(var1_t / var2_t) / m
// (eq. greedy_mult; for one target it is log(v_t / v_t+1), eq. global_obj).  The pivots
// of a left-to-right factorisation are the conditional variances given what precedes
// them (eq. cond_select), so var1 is the diagonal D of the LDL^T of Theta_SS (S in pick
// order) and var2 the diagonal of the LDL^T of Theta over [P; S] at the picks' rows.
//
// One CTA of 256 threads per unit (persistent): Theta over [P; S] is built once in packed
// lower storage (FP64 Matern from the table-driven exp of the fill), its trailing S
// block copied; both factorisations run right-looking, flat over the CTA so that every
// warp carries FP64 work, and share each pivot's two barriers: (1) the column of
// multipliers l_a = A_aj / d_j, (2) the trailing update A_ab -= l_a A_bj, where the
// thread that produces the next pivot also forms its reciprocal.
#include "sic_internal.cuh"

namespace {

constexpr int SIDE_NT = 256;

__device__ __forceinline__ int spk(int a, int b) { return a * (a + 1) / 2 + b; }

// row r of the packed lower-triangle element e: r (r + 1) / 2 <= e < (r + 1) (r + 2) / 2
__device__ __forceinline__ int tri_row(int e) {
    int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (r * (r + 1) / 2 > e) --r;
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    return r;
}

struct SideLayout {
    int nmax, k;
    int dec;  // 1: the packed-triangle decode table follows the doubles (when it fits)
    __host__ __device__ int tab() const { return 0; }
    __host__ __device__ int A() const { return EXP_TAB; }
    __host__ __device__ int B() const { return A() + nmax * (nmax + 1) / 2; }
    __host__ __device__ int xyz() const { return B() + k * (k + 1) / 2; }
    __host__ __device__ int clA() const { return xyz() + 3 * nmax; }
    __host__ __device__ int clB() const { return clA() + nmax; }
    __host__ __device__ int rdA() const { return clB() + k; }
    __host__ __device__ int rdB() const { return rdA() + nmax; }
    __host__ __device__ int size() const { return rdB() + k; }  // doubles
    // then the decode table of the packed triangle: entry e -> (row << 8) | column
    __host__ __device__ int tri() const { return nmax * (nmax + 1) / 2; }
    __host__ __device__ size_t bytes() const {
        return sizeof(double) * (size_t)size() + (dec ? sizeof(uint16_t) * (size_t)tri() : 0);
    }
};

__global__ void __launch_bounds__(SIDE_NT) k_side(const double* __restrict__ pts, long long n, int dim,
                                                  KP<double> kp, const long long* __restrict__ grp_ptr,
                                                  const int32_t* __restrict__ targets, long long n_units,
                                                  const int32_t* __restrict__ sel_idx,
                                                  const int32_t* __restrict__ sel_count, int k, int max_m,
                                                  SideLayout L, double* __restrict__ pvar,
                                                  double* __restrict__ pvar_p, double* __restrict__ gain,
                                                  DevStatus* st) {
    extern __shared__ double sm[];
    double* tab = sm + L.tab();
    double* A = sm + L.A();
    double* B = sm + L.B();
    double* xyz = sm + L.xyz();
    double* clA = sm + L.clA();
    double* clB = sm + L.clB();
    double* rdA = sm + L.rdA();
    double* rdB = sm + L.rdB();
    uint16_t* dec = reinterpret_cast<uint16_t*>(sm + L.size());  // packed-triangle decode table
    __shared__ int s_bad;  // 1: invalid unit or pick, 2: a pivot not positive
    const int tid = threadIdx.x, NMAX = L.nmax;
    const double diag = kp.s2 + kp.nugget;
    const double NaN = __longlong_as_double(0x7ff8000000000000LL);
    exp_table_fill(tab, kp.s2);
    if (L.dec)
        for (int e = threadIdx.x; e < L.tri(); e += blockDim.x) {
            const int r = tri_row(e);
            dec[e] = (uint16_t)((r << 8) | (e - r * (r + 1) / 2));
        }
    // row and column of packed-triangle element e: from the table, else by the square root
    auto decode = [&](int e, int& r, int& c) {
        if (L.dec) {
            const unsigned v = dec[e];
            r = (int)(v >> 8);
            c = (int)(v & 255u);
        } else {
            r = tri_row(e);
            c = e - r * (r + 1) / 2;
        }
    };

    for (long long u = blockIdx.x; u < n_units; u += gridDim.x) {
        long long p0;
        int m;
        if (grp_ptr) {
            p0 = grp_ptr[u];
            m = (int)(grp_ptr[u + 1] - p0);
        } else {
            p0 = targets ? (long long)targets[u] : u;
            m = 1;
        }
        const int cnt_raw = sel_count[u];
        const bool bad_unit = m < 1 || m > max_m || p0 < 0 || p0 + m > n || cnt_raw < 0 || cnt_raw > k;
        const int cnt = bad_unit ? 0 : cnt_raw;
        const int nn = m + cnt;
        if (tid == 0) s_bad = bad_unit ? 1 : 0;
        __syncthreads();
        for (int i = tid; i < (bad_unit ? 0 : nn); i += SIDE_NT) {
            long long p = i < m ? p0 + i : (long long)sel_idx[u * k + (i - m)];
            if (p < 0 || p >= n) {
                s_bad = 1;
                p = p0;
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) xyz[d * NMAX + i] = (d < dim) ? pts[p * dim + d] : 0.0;
        }
        __syncthreads();
        if (!s_bad && cnt > 0) {
            // Theta over [P; S] (packed lower) and a copy of its S block
            const int tri = nn * (nn + 1) / 2;
            for (int e = tid; e < tri; e += SIDE_NT) {
                int a, b;
                decode(e, a, b);
                double v = diag;
                if (a != b) {
                    const double dx = xyz[a] - xyz[b], dy = xyz[NMAX + a] - xyz[NMAX + b],
                                 dz = xyz[2 * NMAX + a] - xyz[2 * NMAX + b];
                    v = matern_d2_fast(kp, fma(dz, dz, fma(dy, dy, dx * dx)), tab);
                }
                A[e] = v;
                if (b >= m) B[spk(a - m, b - m)] = v;
            }
            if (tid == 0) {
                rdA[0] = 1.0 / diag;
                rdB[0] = 1.0 / diag;
            }
            __syncthreads();
            for (int j = 0; j < nn; ++j) {
                const bool jb = j < cnt;
                const double ra = rdA[j], rb = jb ? rdB[j] : 0.0;
                for (int a = j + 1 + tid; a < nn; a += SIDE_NT) clA[a] = A[spk(a, j)] * ra;
                if (jb)
                    for (int a = j + 1 + tid; a < cnt; a += SIDE_NT) clB[a] = B[spk(a, j)] * rb;
                __syncthreads();
                const int TA = nn - j - 1, TB = jb ? cnt - j - 1 : 0;
                const int eA = TA * (TA + 1) / 2, eB = TB * (TB + 1) / 2;
                for (int e = tid; e < eA + eB; e += SIDE_NT) {
                    const bool inA = e < eA;
                    const int f = inA ? e : e - eA;
                    int r, c;
                    decode(f, r, c);
                    const int a = j + 1 + r, b = j + 1 + c;
                    double* M = inA ? A : B;
                    const double* cl = inA ? clA : clB;
                    const double v = fma(-cl[a], M[spk(b, j)], M[spk(a, b)]);
                    M[spk(a, b)] = v;
                    if (r == 0) {  // the next pivot (a = b = j + 1)
                        if (!(v > 0.0)) s_bad = 2;
                        (inA ? rdA : rdB)[j + 1] = 1.0 / v;
                    }
                }
                __syncthreads();
            }
        }
        const int bad = s_bad;
        if (bad && tid == 0) record_error(st, bad == 2 ? SIC_ERR_NOT_PD : SIC_ERR_INVALID, u);
        const int nout = bad_unit ? ((cnt_raw > 0 && cnt_raw <= k) ? cnt_raw : 0) : cnt;
        for (int t = tid; t < nout; t += SIDE_NT) {
            double v1 = NaN, v2 = NaN, g = NaN;
            if (!bad) {
                v1 = B[spk(t, t)];
                v2 = A[spk(m + t, m + t)];
                g = log(v1 / v2) / m;
            }
            if (pvar) pvar[u * k + t] = v1;
            if (pvar_p) pvar_p[u * k + t] = v2;
            if (gain) gain[u * k + t] = g;
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" sic_status sic_side_state_fp64(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                          const int64_t* grp_ptr, const int32_t* targets, int64_t n_units,
                                          int32_t max_m, const int32_t* sel_idx, const int32_t* sel_count,
                                          int32_t k, double* pvar, double* pvar_p, double* gain, void* stream) {
    if (!h || !pts || !sic_valid_kernel(kp) || n < 1 || n_units < 0 || k < 1 || max_m < 1) return SIC_ERR_INVALID;
    if (!grp_ptr && max_m != 1) return SIC_ERR_INVALID;
    if (k > 128 || max_m > 64) return SIC_ERR_UNSUPPORTED;
    if (!pvar && !pvar_p && !gain) return SIC_ERR_INVALID;
    if (n_units == 0) return SIC_OK;
    if (!sel_idx || !sel_count) return SIC_ERR_INVALID;
    SideLayout L;
    L.nmax = max_m + k;
    L.k = k;
    L.dec = 1;
    if (L.bytes() > 227 * 1024 - 1024) L.dec = 0;
    const size_t smem = L.bytes();
    if (smem > 227 * 1024 - 1024) return SIC_ERR_UNSUPPORTED;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    // opt in at any size: the static arrays count against the 48 KB default as well
    SIC_CUDA_TRY(cudaFuncSetAttribute(k_side, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = persistent_grid(h, k_side, SIDE_NT, smem, n_units);
    k_side<<<grid, SIDE_NT, smem, (cudaStream_t)stream>>>(pts, n, kp->dim, make_kp<double>(*kp),
                                                          (const long long*)grp_ptr, targets, n_units, sel_idx,
                                                          sel_count, k, max_m, L, pvar, pvar_p, gain, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}
