// y = op(L) x for the CSC factor (its use as a preconditioner, Section 6.4).
// L^T x is a gather (one warp per column, groups of lanes over the column's entries, a fixed
// shuffle tree across the groups); L x scatters with FP64 atomics (one warp per column).
// L L^T x chains the two through the caller's workspace.
#include "sic_internal.cuh"

namespace {

// NR lanes share one nonzero (NR = 1, 2, 4, 8: the right-hand sides rounded up to a power of
// two); lane r of such a group handles right-hand side r, so a nonzero's x row (or y row) is
// one coalesced access, and a warp walks 32 / NR nonzeros of its column at a time.
template <int NR>
__global__ void __launch_bounds__(256) k_apply_lt(long long n, const long long* __restrict__ cp,
                                                  const int32_t* __restrict__ ri, const double* __restrict__ v,
                                                  const double* __restrict__ x, double* __restrict__ y, int nrhs) {
    const long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, g = lane / NR, r = lane % NR;
    if (c >= n) return;
    double acc = 0.0;
    const long long e = cp[c + 1];
    for (long long p = cp[c] + g; p < e; p += 32 / NR) {
        const double a = v[p];
        const long long row = ri[p];
        if (row < 0 || row >= n || r >= nrhs) continue;  // malformed factor: skip the entry
        acc = fma(a, x[row * nrhs + r], acc);
    }
#pragma unroll
    for (int off = 16; off >= NR; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane < nrhs) y[c * nrhs + lane] = acc;
}

template <int NR>
__global__ void __launch_bounds__(256) k_apply_l(long long n, const long long* __restrict__ cp,
                                                 const int32_t* __restrict__ ri, const double* __restrict__ v,
                                                 const double* __restrict__ x, double* __restrict__ y, int nrhs) {
    const long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, g = lane / NR, r = lane % NR;
    if (c >= n || r >= nrhs) return;
    const double xc = x[c * nrhs + r];
    const long long e = cp[c + 1];
    for (long long p = cp[c] + g; p < e; p += 32 / NR) {
        const double a = v[p];
        const long long row = ri[p];
        if (row < 0 || row >= n) continue;  // malformed factor: skip the entry
        atomicAdd(&y[row * nrhs + r], a * xc);
    }
}

template <int NR>
void run(long long n, const int64_t* cp, const int32_t* ri, const double* v, sic_op op, const double* x, double* y,
         int nrhs, double* z, cudaStream_t s) {
    const unsigned blocks = (unsigned)((n * 32 + 255) / 256);
    const long long* c = (const long long*)cp;
    if (op == SIC_OP_LT) {
        k_apply_lt<NR><<<blocks, 256, 0, s>>>(n, c, ri, v, x, y, nrhs);
    } else if (op == SIC_OP_L) {
        cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n * nrhs, s);
        k_apply_l<NR><<<blocks, 256, 0, s>>>(n, c, ri, v, x, y, nrhs);
    } else {
        k_apply_lt<NR><<<blocks, 256, 0, s>>>(n, c, ri, v, x, z, nrhs);
        cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n * nrhs, s);
        k_apply_l<NR><<<blocks, 256, 0, s>>>(n, c, ri, v, z, y, nrhs);
    }
}

}  // namespace

extern "C" sic_status sic_apply_factor_workspace(int64_t n, int32_t nrhs, sic_op op, size_t* bytes) {
    if (!bytes || n < 0 || nrhs < 1) return SIC_ERR_INVALID;
    *bytes = (op == SIC_OP_LLT) ? sizeof(double) * (size_t)n * (size_t)nrhs : 0;
    return SIC_OK;
}

extern "C" sic_status sic_apply_factor(sic_handle* h, int64_t n, const int64_t* col_ptr, const int32_t* row_idx,
                                       const double* val, sic_op op, const double* x, double* y, int32_t nrhs,
                                       void* ws, size_t ws_bytes, void* stream) {
    if (!h || n < 1 || !col_ptr || !row_idx || !val || !x || !y || nrhs < 1) return SIC_ERR_INVALID;
    if (op != SIC_OP_L && op != SIC_OP_LT && op != SIC_OP_LLT) return SIC_ERR_INVALID;
    if (nrhs > 8) return SIC_ERR_UNSUPPORTED;
    if (op == SIC_OP_LLT && (!ws || ws_bytes < sizeof(double) * (size_t)n * (size_t)nrhs)) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    double* z = (double*)ws;
    if (nrhs == 1)
        run<1>(n, col_ptr, row_idx, val, op, x, y, nrhs, z, s);
    else if (nrhs <= 2)
        run<2>(n, col_ptr, row_idx, val, op, x, y, nrhs, z, s);
    else if (nrhs <= 4)
        run<4>(n, col_ptr, row_idx, val, op, x, y, nrhs, z, s);
    else
        run<8>(n, col_ptr, row_idx, val, op, x, y, nrhs, z, s);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}
