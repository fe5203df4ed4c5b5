// Aggregated FP64 fill of a partial-selection pattern (nonadjacent groups; Section 5.1.1 and the
// aggregated computation of Appendix A.4).
//
// Member i of a group holds s_i = {i} + {later members} + {picks after i}.  Sort the group's
// union U = members + picks from the latest position to the earliest, u_0 > u_1 > ...; then
// s_{u_a} = {u_0, ..., u_a}, a leading block.  With Theta_UU = L D L^T (unit lower L, in this
// order), the leading block's factor is the leading block of L, and the KL-optimal column
// (eq. L_col) of u_a is x with  L_S^T x = e_a / sqrt(d_a)  (S = 0..a):  x_a = d_a^{-1/2},
// x_r = -sum_{c = r+1..a} L_cr x_c;  log Theta_{u_a u_a | s \ u_a} = log d_a.  One LDL^T per
// group serves every member, as in the consecutive-group fill, instead of one per column.
//
// One CTA of 256 threads per group (persistent): the union sorted by rank counting, Theta in
// packed lower storage (FP64 Matern from the table-driven exp), a right-looking LDL^T flat over
// the CTA (two barriers per pivot, the next pivot's reciprocal formed by the thread that
// produces it), then one warp per member for the back substitution (lanes own rows, the
// column-oriented recurrence in registers), written straight into the CSC column.
#include <limits.h>

#include "sic_internal.cuh"

namespace {

constexpr int FP_NT = 256;

__device__ __forceinline__ int fpk(int a, int b) { return a * (a + 1) / 2 + b; }

__device__ __forceinline__ int fp_tri_row(int e) {
    int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (r * (r + 1) / 2 > e) --r;
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    return r;
}

struct FpLayout {
    int nmax;
    int dec;  // 1: a packed-triangle decode table follows
    __host__ __device__ int A() const { return EXP_TAB; }
    __host__ __device__ int xyz() const { return A() + nmax * (nmax + 1) / 2; }
    __host__ __device__ int cl() const { return xyz() + 3 * nmax; }
    __host__ __device__ int cu() const { return cl() + nmax; }
    __host__ __device__ int rd() const { return cu() + nmax; }
    __host__ __device__ int doubles() const { return rd() + nmax; }
    __host__ __device__ size_t bytes() const {
        return sizeof(double) * (size_t)doubles() + sizeof(int) * 3 * (size_t)nmax +
               (dec ? sizeof(uint16_t) * (size_t)(nmax * (nmax + 1) / 2) : 0);
    }
};

__global__ void __launch_bounds__(FP_NT) k_fill_partial(const double* __restrict__ pts, long long n, int dim,
                                                        KP<double> kp, const long long* __restrict__ grp_ptr,
                                                        const long long* __restrict__ members, long long n_grp,
                                                        const int32_t* __restrict__ sel_idx,
                                                        const int32_t* __restrict__ sel_count, int k, int max_m,
                                                        FpLayout L, const long long* __restrict__ col_ptr,
                                                        int32_t* __restrict__ row_idx, double* __restrict__ val,
                                                        double* __restrict__ logv, DevStatus* st) {
    extern __shared__ double sm[];
    double* tab = sm;
    double* A = sm + L.A();
    double* xyz = sm + L.xyz();
    double* cl = sm + L.cl();
    double* cu = sm + L.cu();
    double* rd = sm + L.rd();
    int* upos = reinterpret_cast<int*>(sm + L.doubles());  // [nmax] position of order index a
    int* umem = upos + L.nmax;                              // [nmax] 1: a member
    int* raw = umem + L.nmax;                               // [nmax] positions, members then picks
    uint16_t* dec = reinterpret_cast<uint16_t*>(raw + L.nmax);
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NMAX = L.nmax;
    const double diag = kp.s2 + kp.nugget;
    exp_table_fill(tab, kp.s2);
    if (L.dec)
        for (int e = tid; e < NMAX * (NMAX + 1) / 2; e += FP_NT) {
            const int r = fp_tri_row(e);
            dec[e] = (uint16_t)((r << 8) | (e - r * (r + 1) / 2));
        }
    auto decode = [&](int e, int& r, int& c) {
        if (L.dec) {
            const unsigned v = dec[e];
            r = (int)(v >> 8);
            c = (int)(v & 255u);
        } else {
            r = fp_tri_row(e);
            c = e - r * (r + 1) / 2;
        }
    };

    for (long long g = blockIdx.x; g < n_grp; g += gridDim.x) {
        const long long a0 = grp_ptr[g];
        const int m = (int)(grp_ptr[g + 1] - a0);
        const int cnt = sel_count[g];
        const bool bad_grp = m < 1 || m > max_m || cnt < 0 || cnt > k;
        const int nn = bad_grp ? 0 : m + cnt;
        if (tid == 0) s_bad = bad_grp ? 1 : 0;
        for (int e = tid; e < nn; e += FP_NT) {
            const long long p = e < m ? members[a0 + e] : (long long)sel_idx[g * k + (e - m)];
            raw[e] = (p < 0 || p >= n) ? -1 : (int)p;
        }
        __syncthreads();
        // the union sorted by position, latest first: element e goes to index (number of
        // elements after it)
        for (int e = tid; e < nn; e += FP_NT) {
            const int p = raw[e];
            int later = 0, same = 0;
            if (p < 0) {
                s_bad = 1;
            } else {
                for (int f = 0; f < nn; ++f) {
                    later += raw[f] > p;
                    same += raw[f] == p;
                }
                if (same != 1 || (e >= m && p <= raw[0])) s_bad = 1;  // repeated, or before the group
            }
            if (later < nn) {
                upos[later] = (int)p;
                umem[later] = e < m;
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    xyz[d * NMAX + later] = (d < dim && p >= 0 && p < n) ? pts[p * dim + d] : 0.0;
            }
        }
        __syncthreads();
        if (!s_bad && nn > 0) {
            const int tri = nn * (nn + 1) / 2;
            for (int e = tid; e < tri; e += FP_NT) {
                int a, b;
                decode(e, a, b);
                double v = diag;
                if (a != b) {
                    const double dx = xyz[a] - xyz[b], dy = xyz[NMAX + a] - xyz[NMAX + b],
                                 dz = xyz[2 * NMAX + a] - xyz[2 * NMAX + b];
                    v = matern_d2_fast(kp, fma(dz, dz, fma(dy, dy, dx * dx)), tab);
                }
                A[e] = v;
            }
            if (tid == 0) rd[0] = 1.0 / diag;
            __syncthreads();
            // LDL^T, right-looking: multipliers stored below the diagonal, pivots on it
            for (int j = 0; j + 1 < nn; ++j) {
                const double r = rd[j];
                for (int a = j + 1 + tid; a < nn; a += FP_NT) {
                    const double u = A[fpk(a, j)];
                    cu[a] = u;
                    cl[a] = u * r;
                    A[fpk(a, j)] = u * r;
                }
                __syncthreads();
                const int T = nn - j - 1, eT = T * (T + 1) / 2;
                for (int e = tid; e < eT; e += FP_NT) {
                    int rr, cc;
                    decode(e, rr, cc);
                    const int a = j + 1 + rr, b = j + 1 + cc;
                    const double v = fma(-cl[a], cu[b], A[fpk(a, b)]);
                    A[fpk(a, b)] = v;
                    if (rr == 0) {  // the next pivot
                        if (!(v > 0.0)) s_bad = 2;
                        rd[j + 1] = 1.0 / v;
                    }
                }
                __syncthreads();
            }
        }
        const int bad = s_bad;
        if (bad) {
            if (tid == 0) record_error(st, bad == 2 ? SIC_ERR_NOT_PD : SIC_ERR_INVALID, g);
        } else {
            // one warp per member: x_a = d_a^-1/2, x_r = -sum_{c > r} L_cr x_c (lanes own rows r)
            for (int a = warp; a < nn; a += FP_NT / 32) {
                if (!umem[a]) continue;
                const long long P = upos[a];
                const long long c0 = col_ptr[P];
                if (col_ptr[P + 1] - c0 != a + 1) {
                    if (lane == 0) record_error(st, SIC_ERR_INVALID, g);
                    continue;
                }
                const double da = A[fpk(a, a)];
                double acc[6];  // rows r = lane + 32 h, nmax <= 192
#pragma unroll
                for (int h = 0; h < 6; ++h) acc[h] = 0.0;
                double xc = rsqrt_newton(da);
                for (int c = a; c >= 0; --c) {
                    if (c < a) {
                        double o = 0.0;
#pragma unroll
                        for (int h = 0; h < 6; ++h) {
                            const double w = __shfl_sync(0xffffffffu, acc[h], c & 31);
                            if (h == (c >> 5)) o = w;
                        }
                        xc = o;
                    }
                    if (lane == 0) {
                        row_idx[c0 + (a - c)] = upos[c];
                        val[c0 + (a - c)] = xc;
                    }
#pragma unroll
                    for (int h = 0; h < 6; ++h) {
                        const int r = lane + 32 * h;
                        if (r < c) acc[h] = fma(-A[fpk(c, r)], xc, acc[h]);
                    }
                }
                if (lane == 0) logv[P] = log(da);
            }
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" sic_status sic_build_factor_partial(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                               const int64_t* grp_ptr, const int64_t* members, int64_t n_grp,
                                               int32_t max_m, const int32_t* sel_idx, const int32_t* sel_count,
                                               int32_t k, const int64_t* col_ptr, int32_t* row_idx, double* val,
                                               double* logv, double* sum_logv, void* ws, size_t ws_bytes,
                                               void* stream) {
    if (!h || !pts || !sic_valid_kernel(kp) || n < 1 || n_grp < 0 || !grp_ptr || !members || !sel_idx ||
        !sel_count || !col_ptr || !row_idx || !val || !logv || !sum_logv || k < 1 || max_m < 1)
        return SIC_ERR_INVALID;
    if (max_m > 64 || k > 128 || n > INT_MAX) return SIC_ERR_UNSUPPORTED;
    size_t need = 0;
    sic_build_factor_workspace(n, &need);
    if (!ws || ws_bytes < need) return SIC_ERR_INVALID;
    FpLayout L;
    L.nmax = max_m + k;
    L.dec = 1;
    if (L.bytes() > 227 * 1024 - 1024) L.dec = 0;
    if (L.bytes() > 227 * 1024 - 1024) return SIC_ERR_UNSUPPORTED;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (n_grp > 0) {
        SIC_CUDA_TRY(cudaFuncSetAttribute(k_fill_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)L.bytes()));
        const int grid = persistent_grid(h, k_fill_partial, FP_NT, L.bytes(), n_grp);
        k_fill_partial<<<grid, FP_NT, L.bytes(), s>>>(pts, n, kp->dim, make_kp<double>(*kp),
                                                      (const long long*)grp_ptr, (const long long*)members, n_grp,
                                                      sel_idx, sel_count, k, max_m, L, (const long long*)col_ptr,
                                                      row_idx, val, logv, h->d_status);
        SIC_CUDA_TRY(cudaGetLastError());
    }
    return launch_sum_logv(logv, n, sum_logv, ws, s);
}
