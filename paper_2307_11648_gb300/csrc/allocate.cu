// Global greedy allocation of nonzeros (Section 5.4) without a priority queue.
//
// The paper pops, from a queue of every unit's best candidate, the pick that lowers the
// KL divergence most per nonzero.  A unit's candidate values change only when the unit
// itself gains an entry, so the picks of a unit come in its local greedy order, and the
// queue pops pick t of unit u exactly when e(u, t) = min(gain(u, 0..t)), the running
// minimum of the unit's decreases, is the largest key left (equal keys: lower unit, then
// earlier pick).  The queue's result is therefore the longest prefix, in the order of
// (e descending, u, t), whose costs fit in the budget -- one global threshold, found here
// by a weighted radix selection:
//   k_alloc_keys   one warp per unit: running minimum by a warp scan, written as 64-bit
//                  order-preserving keys (0 marks an empty slot); clears the histograms;
//   k_alloc_hist   8 passes over the keys, 8 bits each from the top: every CTA first
//                  replays the earlier passes' histograms to learn the prefix of the
//                  threshold key T (the key of the first pick that does not fit) and the
//                  cost of the keys above that prefix, then adds the cost m_u of each key
//                  under the prefix to the bin of its next digit;
//   k_alloc_ties   units dealt in contiguous chunks, one per CTA: the number of keys above
//                  T and equal to T per unit (binary searches: a unit's keys never
//                  increase), and the chunk's total cost of picks with key T;
//   k_alloc_final  the picks with key T are taken in unit order while they fit: an
//                  exclusive scan of the tie costs (chunk offsets plus a CTA scan) gives
//                  each unit its share; out_count = (keys above T) + (ties taken).
// Every launch is sized by the SM count; the only global atomics are the 256 bins per
// pass; results do not depend on the launch shape.
#include "sic_internal.cuh"

namespace {

constexpr int AL_NT = 256;
constexpr int AL_PASSES = 8;
constexpr int AL_MAXB = 1024;  // CTAs of the tie kernels (chunks of units)
typedef unsigned long long u64;

// workspace: keys [n_units * k] | hist [AL_PASSES][256] | chunk tie costs [AL_MAXB] | cut [4]
struct AllocWs {
    u64* keys;
    u64* hist;
    u64* bsum;
    u64* cut;  // state (1: everything fits), T, cost above T
};

size_t alloc_keys_bytes(long long n_units, int k) { return ((size_t)n_units * (size_t)k * 8 + 255) / 256 * 256; }

size_t alloc_ws_bytes(long long n_units, int k) {
    return alloc_keys_bytes(n_units, k) + 8 * ((size_t)AL_PASSES * 256 + AL_MAXB + 4);
}

AllocWs alloc_ws(void* ws, long long n_units, int k) {
    AllocWs w;
    w.keys = (u64*)ws;
    w.hist = (u64*)((char*)ws + alloc_keys_bytes(n_units, k));
    w.bsum = w.hist + AL_PASSES * 256;
    w.cut = w.bsum + AL_MAXB;
    return w;
}

// order-preserving map of a non-NaN double to a nonzero 64-bit key
__device__ __forceinline__ u64 dkey(double x) {
    const u64 b = (u64)__double_as_longlong(x + 0.0);  // -0 -> +0
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ int unit_count(const int32_t* sel_count, long long u, int k) {
    const int c = sel_count[u];
    return (c < 0 || c > k) ? -1 : c;
}

__device__ __forceinline__ u64 unit_cost(const long long* grp_ptr, long long u) {
    return grp_ptr ? (u64)(grp_ptr[u + 1] - grp_ptr[u]) : 1ull;
}

__global__ void __launch_bounds__(AL_NT) k_alloc_keys(long long n_units, const long long* __restrict__ grp_ptr,
                                                      const double* __restrict__ gain,
                                                      const int32_t* __restrict__ sel_count, int k,
                                                      AllocWs w, DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const long long gtid = (long long)blockIdx.x * AL_NT + threadIdx.x;
    for (long long e = gtid; e < AL_PASSES * 256 + 4; e += (long long)gridDim.x * AL_NT) {
        if (e < AL_PASSES * 256) w.hist[e] = 0ull;
        else w.cut[e - AL_PASSES * 256] = 0ull;
    }
    const long long nwarps = (long long)gridDim.x * (AL_NT / 32);
    for (long long u = gtid >> 5; u < n_units; u += nwarps) {
        int cnt = unit_count(sel_count, u, k);
        if (cnt < 0) {
            if (lane == 0) record_error(st, SIC_ERR_INVALID, u);
            cnt = 0;
        }
        if (grp_ptr && lane == 0 && grp_ptr[u + 1] <= grp_ptr[u]) record_error(st, SIC_ERR_INVALID, u);
        double run = INFINITY;
        for (int t0 = 0; t0 < k; t0 += 32) {
            const int t = t0 + lane;
            double x = INFINITY;
            if (t < cnt) {
                x = gain[u * k + t];
                if (x != x) {
                    record_error(st, SIC_ERR_INVALID, u);
                    x = -INFINITY;
                }
            }
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const double y = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x = fmin(x, y);
            }
            x = fmin(x, run);
            run = __shfl_sync(0xffffffffu, x, 31);
            if (t < k) w.keys[u * k + t] = (t < cnt) ? dkey(x) : 0ull;
        }
    }
}

// Replays the histograms of passes 0 .. passes-1: the threshold's known digits (prefix,
// mask) and the cost of the keys above them.  Block-wide; result in shared memory.
struct Cut {
    u64 prefix, mask, above;
    int all;  // every pick fits
};

__device__ void replay(const u64* __restrict__ hist, int passes, long long budget, u64* bins, Cut* cut) {
    if (threadIdx.x == 0) {
        cut->prefix = 0ull;
        cut->mask = 0ull;
        cut->above = 0ull;
        cut->all = 0;
    }
    for (int p = 0; p < passes; ++p) {
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += blockDim.x) bins[d] = hist[p * 256 + d];
        __syncthreads();
        if (threadIdx.x == 0 && !cut->all) {
            u64 acc = cut->above;
            int dig = -1;
            for (int d = 255; d >= 0; --d) {
                if ((long long)(acc + bins[d]) > budget) {
                    dig = d;
                    break;
                }
                acc += bins[d];
            }
            if (dig < 0) {
                cut->all = 1;  // only possible at the first pass: the total fits
            } else {
                const int shift = 56 - 8 * p;
                cut->prefix |= (u64)dig << shift;
                cut->mask |= 0xFFull << shift;
                cut->above = acc;
            }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(AL_NT) k_alloc_hist(long long n_units, const long long* __restrict__ grp_ptr,
                                                      int k, long long budget, int pass, AllocWs w) {
    __shared__ u64 bins[256];
    __shared__ Cut cut;
    replay(w.hist, pass, budget, bins, &cut);
    if (cut.all) return;
    for (int d = threadIdx.x; d < 256; d += AL_NT) bins[d] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31, shift = 56 - 8 * pass;
    const u64 prefix = cut.prefix, mask = cut.mask;
    const long long nwarps = (long long)gridDim.x * (AL_NT / 32);
    for (long long u = ((long long)blockIdx.x * AL_NT + threadIdx.x) >> 5; u < n_units; u += nwarps) {
        const u64 c = unit_cost(grp_ptr, u);
        for (int t = lane; t < k; t += 32) {
            const u64 key = w.keys[u * k + t];
            if (key != 0ull && (key & mask) == prefix) atomicAdd(&bins[(key >> shift) & 255], c);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += AL_NT)
        if (bins[d]) atomicAdd(&w.hist[pass * 256 + d], bins[d]);
}

// keys above T (n_gt) and equal to T (n_eq) of unit u; a unit's keys never increase
__device__ __forceinline__ void unit_split(const u64* __restrict__ row, int cnt, u64 T, int& n_gt, int& n_eq) {
    int lo = 0, hi = cnt;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (row[mid] > T) lo = mid + 1; else hi = mid;
    }
    n_gt = lo;
    hi = cnt;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (row[mid] >= T) lo = mid + 1; else hi = mid;
    }
    n_eq = lo - n_gt;
}

__device__ __forceinline__ void chunk_of(long long n_units, long long& u0, long long& u1) {
    const long long per = (n_units + gridDim.x - 1) / gridDim.x;
    u0 = (long long)blockIdx.x * per;
    u1 = u0 + per < n_units ? u0 + per : n_units;
}

__device__ __forceinline__ u64 warp_incl_scan(u64 v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += y;
    }
    return v;
}

__global__ void __launch_bounds__(AL_NT) k_alloc_ties(long long n_units, const long long* __restrict__ grp_ptr,
                                                      const int32_t* __restrict__ sel_count, int k,
                                                      long long budget, AllocWs w) {
    __shared__ u64 bins[256];
    __shared__ Cut cut;
    __shared__ u64 wsum[AL_NT / 32];
    replay(w.hist, AL_PASSES, budget, bins, &cut);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        w.cut[0] = (u64)cut.all;
        w.cut[1] = cut.prefix;
        w.cut[2] = cut.above;
    }
    if (cut.all) return;
    const u64 T = cut.prefix;
    long long u0, u1;
    chunk_of(n_units, u0, u1);
    u64 s = 0ull;
    for (long long u = u0 + threadIdx.x; u < u1; u += AL_NT) {
        const int cnt = unit_count(sel_count, u, k);
        if (cnt <= 0) continue;
        int n_gt, n_eq;
        unit_split(w.keys + u * k, cnt, T, n_gt, n_eq);
        s += unit_cost(grp_ptr, u) * (u64)n_eq;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 b = 0ull;
        for (int i = 0; i < AL_NT / 32; ++i) b += wsum[i];
        w.bsum[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(AL_NT) k_alloc_final(long long n_units, const long long* __restrict__ grp_ptr,
                                                       const int32_t* __restrict__ sel_count, int k,
                                                       long long budget, AllocWs w, int32_t* __restrict__ out) {
    __shared__ u64 wtot[AL_NT / 32];
    __shared__ u64 s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long u0, u1;
    chunk_of(n_units, u0, u1);
    const bool all = w.cut[0] != 0ull;
    if (all) {
        for (long long u = u0 + threadIdx.x; u < u1; u += AL_NT) {
            const int cnt = unit_count(sel_count, u, k);
            out[u] = cnt < 0 ? 0 : cnt;
        }
        return;
    }
    const u64 T = w.cut[1];
    const long long rem = budget - (long long)w.cut[2];  // what is left for the picks with key T
    // tie costs of the chunks before this one
    u64 b = 0ull;
    for (int i = threadIdx.x; i < (int)blockIdx.x; i += AL_NT) b += w.bsum[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) b += __shfl_xor_sync(0xffffffffu, b, off);
    if (lane == 0) wtot[warp] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 t = 0ull;
        for (int i = 0; i < AL_NT / 32; ++i) t += wtot[i];
        s_base = t;
    }
    __syncthreads();
    u64 base = s_base;
    for (long long t0 = u0; t0 < u1; t0 += AL_NT) {
        const long long u = t0 + threadIdx.x;
        int cnt = 0, n_gt = 0, n_eq = 0;
        u64 m = 1ull;
        if (u < u1) {
            cnt = unit_count(sel_count, u, k);
            if (cnt > 0) {
                unit_split(w.keys + u * k, cnt, T, n_gt, n_eq);
                m = unit_cost(grp_ptr, u);
            }
        }
        const u64 c = m * (u64)n_eq;
        const u64 incl = warp_incl_scan(c);
        __syncthreads();  // wtot is reused
        if (lane == 31) wtot[warp] = incl;
        __syncthreads();
        u64 before = base + incl - c;
        u64 tile = 0ull;
        for (int i = 0; i < AL_NT / 32; ++i) {
            if (i < warp) before += wtot[i];
            tile += wtot[i];
        }
        if (u < u1) {
            long long take = 0;
            const long long avail = rem - (long long)before;
            if (n_eq > 0 && avail > 0) {
                take = avail / (long long)m;
                if (take > n_eq) take = n_eq;
            }
            out[u] = n_gt + (int)take;
        }
        base += tile;
    }
}

}  // namespace

extern "C" sic_status sic_allocate_global_workspace(int64_t n_units, int32_t k, size_t* bytes) {
    if (!bytes || n_units < 0 || k < 1) return SIC_ERR_INVALID;
    if (k > 128) return SIC_ERR_UNSUPPORTED;
    *bytes = alloc_ws_bytes(n_units, k);
    return SIC_OK;
}

extern "C" sic_status sic_allocate_global(sic_handle* h, int64_t n_units, const int64_t* grp_ptr, const double* gain,
                                          const int32_t* sel_count, int32_t k, int64_t budget, int32_t* out_count,
                                          void* ws, size_t ws_bytes, void* stream) {
    if (!h || n_units < 0 || k < 1 || budget < 0) return SIC_ERR_INVALID;
    if (k > 128) return SIC_ERR_UNSUPPORTED;
    if (n_units == 0) return SIC_OK;
    if (!gain || !sel_count || !out_count || !ws || ws_bytes < alloc_ws_bytes(n_units, k)) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const AllocWs w = alloc_ws(ws, n_units, k);
    const long long* gp = (const long long*)grp_ptr;
    const long long wblocks = (n_units + AL_NT / 32 - 1) / (AL_NT / 32);  // one warp per unit
    const int gk = persistent_grid(h, k_alloc_keys, AL_NT, 0, wblocks);
    k_alloc_keys<<<gk, AL_NT, 0, s>>>(n_units, gp, gain, sel_count, k, w, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    const int gh = persistent_grid(h, k_alloc_hist, AL_NT, 0, wblocks);
    for (int p = 0; p < AL_PASSES; ++p) k_alloc_hist<<<gh, AL_NT, 0, s>>>(n_units, gp, k, budget, p, w);
    SIC_CUDA_TRY(cudaGetLastError());
    long long nb = (n_units + AL_NT - 1) / AL_NT;
    if (nb > AL_MAXB) nb = AL_MAXB;
    k_alloc_ties<<<(unsigned)nb, AL_NT, 0, s>>>(n_units, gp, sel_count, k, budget, w);
    k_alloc_final<<<(unsigned)nb, AL_NT, 0, s>>>(n_units, gp, sel_count, k, budget, w, out_count);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}
