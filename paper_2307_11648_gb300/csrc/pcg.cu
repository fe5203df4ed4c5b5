// Preconditioned conjugate gradients on (Theta + shift I) x = b with the sparse factor
// as preconditioner M^{-1} = L L^T (the use of the factor studied in Section 6.4).
//
// k_matvec<T>: y = (Theta + shift I) x for up to 8 right-hand sides without forming Theta:
// one thread per target row, source points staged in shared-memory tiles.  With T = float
// the kernel entries are FP32 (a fixed, symmetric rounding of Theta: K(|x_i - x_j|) is
// evaluated identically for (i, j) and (j, i)); x is carried as an unevaluated sum of two
// FP32 numbers (hi + lo) and each tile's sum of products is accumulated as a double-FP32
// pair with the error-free transformations TwoProduct (by fma) and TwoSum (Knuth), then
// added to an FP64 accumulator -- so the product is accurate to ~1e-14 of sum |K x| and
// CG can reach small residuals.  With T = double everything is FP64 (reference mode; the
// kernel entries by the fill's table-driven exp and Newton square root, about 2 ulp).
// The diagonal adds the nugget and the shift in FP64.
// The CG vector updates and dot products are fused kernels with fixed-order reductions
// (bit-reproducible); the scalars alpha and beta are formed on the device per RHS.
// The iteration loop runs on the host (C++), reading back the residual norms each step.
#include <math.h>

#include <vector>

#include "sic_internal.cuh"

namespace {

constexpr int MV_NT = 128;   // target rows per CTA
constexpr int MV_TILE = 256; // source points per shared-memory tile
constexpr int RED_TILE = 4096;

template <typename T, int NR>
__global__ void __launch_bounds__(MV_NT) k_matvec(const double* __restrict__ pts, long long n, int dim, KP<T> kp,
                                                  double diag_extra, const double* __restrict__ x,
                                                  double* __restrict__ y, int nrhs) {
    constexpr bool F32 = sizeof(T) == 4;
    __shared__ T sx[MV_TILE], sy[MV_TILE], sz[MV_TILE];
    __shared__ T sv[MV_TILE * NR];
    __shared__ float svl[F32 ? MV_TILE * NR : 1];  // low parts of x in FP32 mode
    __shared__ double tab[F32 ? 1 : EXP_TAB];      // FP64 mode: s2 2^(j/256) for the table-driven exp
    if constexpr (!F32) exp_table_fill(tab, kp.s2);  // ordered before use by the tile loop's barrier
    const long long i = blockIdx.x * (long long)MV_NT + threadIdx.x;
    const bool live = i < n;
    T xi = 0, yi = 0, zi = 0;
    if (live) {
        xi = (T)pts[i * dim];
        if (dim > 1) yi = (T)pts[i * dim + 1];
        if (dim > 2) zi = (T)pts[i * dim + 2];
    }
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0;
    for (long long j0 = 0; j0 < n; j0 += MV_TILE) {
        __syncthreads();
        for (int t = threadIdx.x; t < MV_TILE; t += MV_NT) {
            const long long j = j0 + t;
            const bool ok = j < n;
            sx[t] = ok ? (T)pts[j * dim] : (T)0;
            sy[t] = (ok && dim > 1) ? (T)pts[j * dim + 1] : (T)0;
            sz[t] = (ok && dim > 2) ? (T)pts[j * dim + 2] : (T)0;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const double v = (ok && r < nrhs) ? x[j * nrhs + r] : 0.0;
                sv[t * NR + r] = (T)v;
                if constexpr (F32) svl[t * NR + r] = (float)(v - (double)(float)v);
            }
        }
        __syncthreads();
        const int cnt = (int)min((long long)MV_TILE, n - j0);
        if constexpr (F32) {
            float hi[NR], lo[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) hi[r] = lo[r] = 0.f;
            for (int t = 0; t < cnt; ++t) {
                const float dx = xi - sx[t], dy = yi - sy[t], dz = zi - sz[t];
                const float kv = matern<float>(kp, sqrtf(dx * dx + dy * dy + dz * dz));
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    // explicit-rounding intrinsics keep the compiler from fusing the
                    // error-free transformations
                    const float xh = sv[t * NR + r];
                    const float p = __fmul_rn(kv, xh);
                    const float pe = fmaf(kv, svl[t * NR + r], fmaf(kv, xh, -p));  // TwoProduct error + low part
                    const float s = __fadd_rn(hi[r], p);                          // TwoSum(hi, p)
                    const float bp = __fsub_rn(s, hi[r]);
                    const float se = __fadd_rn(__fsub_rn(hi[r], __fsub_rn(s, bp)), __fsub_rn(p, bp));
                    hi[r] = s;
                    lo[r] += se + pe;
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] += (double)hi[r] + (double)lo[r];
        } else {
            T part[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) part[r] = (T)0;
            for (int t = 0; t < cnt; ++t) {
                const T dx = xi - sx[t], dy = yi - sy[t], dz = zi - sz[t];
                const T kv = matern_d2_fast(kp, fma(dz, dz, fma(dy, dy, dx * dx)), tab);
#pragma unroll
                for (int r = 0; r < NR; ++r) part[r] = fma(kv, sv[t * NR + r], part[r]);
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] += (double)part[r];
        }
    }
    if (live) {
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (r < nrhs) y[i * nrhs + r] = acc[r] + diag_extra * x[i * nrhs + r];
    }
}

// partial[b * nrhs + r] = sum over rows of tile b of a[row][r] * c[row][r]
__global__ void __launch_bounds__(256) k_dot_tiles(const double* __restrict__ a, const double* __restrict__ c,
                                                   long long n, int nrhs, double* __restrict__ partial) {
    __shared__ double s[256];
    const long long base = blockIdx.x * (long long)RED_TILE;
    for (int r = 0; r < nrhs; ++r) {
        double acc = 0.0;
        for (int t = threadIdx.x; t < RED_TILE; t += 256) {
            const long long i = base + t;
            if (i < n) acc = fma(a[i * nrhs + r], c[i * nrhs + r], acc);
        }
        s[threadIdx.x] = acc;
        __syncthreads();
        for (int off = 128; off > 0; off >>= 1) {
            if (threadIdx.x < off) s[threadIdx.x] += s[threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[blockIdx.x * nrhs + r] = s[0];
        __syncthreads();
    }
}

__global__ void k_dot_final(const double* __restrict__ partial, long long nb, int nrhs, double* __restrict__ out) {
    const int r = threadIdx.x;
    if (r >= nrhs) return;
    double s = 0.0;
    for (long long b = 0; b < nb; ++b) s += partial[b * nrhs + r];
    out[r] = s;
}

// x += alpha p, r -= alpha q with alpha = rz / pq (0 for converged right-hand sides)
__global__ void k_cg_xr(double* __restrict__ x, double* __restrict__ res, const double* __restrict__ p,
                        const double* __restrict__ q, const double* __restrict__ rz, const double* __restrict__ pq,
                        const int* __restrict__ active, long long n, int nrhs) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    const int r = (int)(e % nrhs);
    if (!active[r]) return;
    const double alpha = rz[r] / pq[r];
    x[e] = fma(alpha, p[e], x[e]);
    res[e] = fma(-alpha, q[e], res[e]);
}

// p = z + beta p with beta = rz_new / rz; then rz = rz_new
__global__ void k_cg_p(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ rz_new,
                       const double* __restrict__ rz, const int* __restrict__ active, long long n, int nrhs) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    const int r = (int)(e % nrhs);
    if (!active[r]) return;
    p[e] = fma(rz_new[r] / rz[r], p[e], z[e]);
}

__global__ void k_copy_rz(double* __restrict__ rz, const double* __restrict__ rz_new, int nrhs) {
    if (threadIdx.x < nrhs) rz[threadIdx.x] = rz_new[threadIdx.x];
}

template <typename T, int NR>
void matvec(cudaStream_t s, const double* pts, long long n, int dim, const sic_kernel* kp, double shift,
            const double* x, double* y, int nrhs) {
    unsigned blocks = (unsigned)((n + MV_NT - 1) / MV_NT);
    k_matvec<T, NR><<<blocks, MV_NT, 0, s>>>(pts, n, dim, make_kp<T>(*kp), kp->nugget + shift, x, y, nrhs);
}

template <typename T>
void matvec_t(cudaStream_t s, const double* pts, long long n, int dim, const sic_kernel* kp, double shift,
              const double* x, double* y, int nrhs) {
    if (nrhs == 1) matvec<T, 1>(s, pts, n, dim, kp, shift, x, y, nrhs);
    else if (nrhs <= 2) matvec<T, 2>(s, pts, n, dim, kp, shift, x, y, nrhs);
    else if (nrhs <= 4) matvec<T, 4>(s, pts, n, dim, kp, shift, x, y, nrhs);
    else matvec<T, 8>(s, pts, n, dim, kp, shift, x, y, nrhs);
}

void matvec_any(cudaStream_t s, const double* pts, long long n, int dim, const sic_kernel* kp, double shift,
                sic_precision prec, const double* x, double* y, int nrhs) {
    if (prec == SIC_FP64) matvec_t<double>(s, pts, n, dim, kp, shift, x, y, nrhs);
    else matvec_t<float>(s, pts, n, dim, kp, shift, x, y, nrhs);
}

void dots(cudaStream_t s, const double* a, const double* c, long long n, int nrhs, double* partial, double* out) {
    long long nb = (n + RED_TILE - 1) / RED_TILE;
    k_dot_tiles<<<(unsigned)nb, 256, 0, s>>>(a, c, n, nrhs, partial);
    k_dot_final<<<1, 32, 0, s>>>(partial, nb, nrhs, out);
}

// workspace layout (doubles): r, z, p, q (n x nrhs each), partial (nb x nrhs), scalars
struct PcgWs {
    long long n;
    int nrhs;
    long long nb() const { return (n + RED_TILE - 1) / RED_TILE; }
    long long vec() const { return n * nrhs; }
    long long size() const { return 4 * vec() + nb() * nrhs + 8 * 8 + n * nrhs /* LL^T intermediate */ + 8; }
};

}  // namespace

extern "C" sic_status sic_matern_matvec(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                        double shift, sic_precision prec, const double* x, double* y, int32_t nrhs,
                                        void* stream) {
    if (!h || !pts || n < 1 || !sic_valid_kernel(kp) || !x || !y || nrhs < 1) return SIC_ERR_INVALID;
    if (prec != SIC_FP64 && prec != SIC_FP32_MIXED) return SIC_ERR_INVALID;
    if (nrhs > 8) return SIC_ERR_UNSUPPORTED;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    matvec_any((cudaStream_t)stream, pts, n, kp->dim, kp, shift, prec, x, y, nrhs);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_pcg_workspace(int64_t n, int32_t nrhs, size_t* bytes) {
    if (!bytes || n < 1 || nrhs < 1) return SIC_ERR_INVALID;
    PcgWs W{n, nrhs};
    *bytes = sizeof(double) * (size_t)W.size() + 64;
    return SIC_OK;
}

extern "C" sic_status sic_apply_factor(sic_handle* h, int64_t n, const int64_t* col_ptr, const int32_t* row_idx,
                                       const double* val, sic_op op, const double* x, double* y, int32_t nrhs,
                                       void* ws, size_t ws_bytes, void* stream);

extern "C" sic_status sic_pcg_solve(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp, double shift,
                                    sic_precision prec, const int64_t* col_ptr, const int32_t* row_idx, const double* val,
                                    const double* b, double* x, int32_t nrhs, double tol, int32_t max_iter,
                                    int32_t* iters, double* relres, void* ws, size_t ws_bytes, void* stream) {
    if (!h || !pts || n < 1 || !sic_valid_kernel(kp) || !b || !x || nrhs < 1 || !(tol > 0) || max_iter < 0 ||
        !iters || !relres || !ws)
        return SIC_ERR_INVALID;
    if (prec != SIC_FP64 && prec != SIC_FP32_MIXED) return SIC_ERR_INVALID;
    if (nrhs > 8) return SIC_ERR_UNSUPPORTED;
    if ((col_ptr != nullptr) != (row_idx != nullptr) || (col_ptr != nullptr) != (val != nullptr))
        return SIC_ERR_INVALID;
    PcgWs W{n, nrhs};
    if (ws_bytes < sizeof(double) * (size_t)W.size()) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    double* base = (double*)ws;
    double* r = base;
    double* z = r + W.vec();
    double* p = z + W.vec();
    double* q = p + W.vec();
    double* partial = q + W.vec();
    double* sc = partial + W.nb() * nrhs;  // 8 x 8 scalars
    double* rz = sc, *pq = sc + 8, *rzn = sc + 16, *rr = sc + 24, *bb = sc + 32;
    int* active = (int*)(sc + 40);
    double* llt = sc + 64;  // n x nrhs intermediate of L L^T
    const size_t vb = sizeof(double) * (size_t)W.vec();
    const unsigned eb = (unsigned)((W.vec() + 255) / 256);
    auto precond = [&](const double* in, double* out) -> sic_status {
        if (!col_ptr) return cudaMemcpyAsync(out, in, vb, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? SIC_OK
                                                                                                  : SIC_ERR_CUDA;
        return sic_apply_factor(h, n, col_ptr, row_idx, val, SIC_OP_LLT, in, out, nrhs, llt, vb, stream);
    };
    // x = 0, r = b
    SIC_CUDA_TRY(cudaMemsetAsync(x, 0, vb, s));
    SIC_CUDA_TRY(cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, s));
    dots(s, b, b, n, nrhs, partial, bb);
    sic_status e = precond(r, z);
    if (e != SIC_OK) return e;
    SIC_CUDA_TRY(cudaMemcpyAsync(p, z, vb, cudaMemcpyDeviceToDevice, s));
    dots(s, r, z, n, nrhs, partial, rz);
    std::vector<int> act(nrhs, 1);
    std::vector<double> hbb(nrhs), hrr(nrhs);
    SIC_CUDA_TRY(cudaMemcpyAsync(hbb.data(), bb, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
    SIC_CUDA_TRY(cudaStreamSynchronize(s));
    for (int c = 0; c < nrhs; ++c) {
        iters[c] = 0;
        relres[c] = hbb[c] > 0 ? 1.0 : 0.0;
        if (!(hbb[c] > 0)) act[c] = 0;
    }
    for (int it = 1; it <= max_iter; ++it) {
        bool any = false;
        for (int c = 0; c < nrhs; ++c) any |= act[c] != 0;
        if (!any) break;
        SIC_CUDA_TRY(cudaMemcpyAsync(active, act.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
        matvec_any(s, pts, n, kp->dim, kp, shift, prec, p, q, nrhs);
        dots(s, p, q, n, nrhs, partial, pq);
        k_cg_xr<<<eb, 256, 0, s>>>(x, r, p, q, rz, pq, active, n, nrhs);
        dots(s, r, r, n, nrhs, partial, rr);
        SIC_CUDA_TRY(cudaMemcpyAsync(hrr.data(), rr, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
        SIC_CUDA_TRY(cudaStreamSynchronize(s));
        for (int c = 0; c < nrhs; ++c) {
            if (!act[c]) continue;
            iters[c] = it;
            relres[c] = sqrt(hrr[c] / hbb[c]);
            if (relres[c] < tol) act[c] = 0;
        }
        SIC_CUDA_TRY(cudaMemcpyAsync(active, act.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
        e = precond(r, z);
        if (e != SIC_OK) return e;
        dots(s, r, z, n, nrhs, partial, rzn);
        k_cg_p<<<eb, 256, 0, s>>>(p, z, rzn, rz, active, n, nrhs);
        k_copy_rz<<<1, 32, 0, s>>>(rz, rzn, nrhs);
    }
    SIC_CUDA_TRY(cudaGetLastError());
    SIC_CUDA_TRY(cudaStreamSynchronize(s));
    return SIC_OK;
}
