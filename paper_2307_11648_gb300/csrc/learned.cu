// Learned candidate proposal for supernodal selection (not part of the paper: a
// small MLP ranks each group's candidates so that the exact greedy selection of
// Section 5.2 runs only on the best `top` of them).
//
//   k_features      8 features per (group, candidate), FP32
//   (inference)     8 -> 128 -> 128 -> 1 on the tcgen05 tensor cores: mlp_tc.cu
//   k_topk_*        per group: keep the `top` best-scored candidates, in list order
//   training        FP32 forward/backward (strided tiled GEMM, split over K with a
//                   fixed-order reduction), weighted BCE with logits, AdamW
//
// Feature definitions (R = distance from the last, i.e. farthest, candidate of the list to
// its nearest member -- the group's candidate radius -- or 1 if zero; a* the nearest
// member, lowest index on ties; K the kernel without nugget):
//   f0, f1 = (x_j - x_a*)[0], [1] / R;  f2 = |x_j - x_a*| / R;
//   f3 = |x_j - centroid| / R;  f4 = rank / C;  f5 = K(|x_j - x_a*|) / sigma^2;
//   f6 = m / 64;  f7 = mean_a K(|x_j - x_a|) / sigma^2.
// All features are O(1), whatever the group's scale.
#include <cuda_bf16.h>

#include "sic_internal.cuh"

namespace {

constexpr int NF = 8;
constexpr int HID = 128;
constexpr int OFF_W1 = 0, OFF_B1 = NF * HID, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID, NPARAM = OFF_B3 + 1;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float dgelu_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ------------------------------------------------------------------ features --

// The Matern (no nugget) at two distances r in packed FP32 pairs: t = sqrt(2 nu) r / ell,
// e^-t = 2^(-t log2 e) by the hardware 2^x, s2 e^-t (nu = 1/2), s2 (1 + t) e^-t (3/2),
// s2 ((1 + t) + t^2 / 3) e^-t (5/2)
__device__ __forceinline__ float ex2_hw(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 matern_f2(const KP<float>& k, float2 r) {
    const float2 t = __fmul2_rn(make_float2(k.c_over_ell, k.c_over_ell), r);
    const float2 l = __fmul2_rn(t, make_float2(-1.4426950408889634f, -1.4426950408889634f));
    const float2 e = make_float2(ex2_hw(l.x), ex2_hw(l.y));
    const float2 s2 = make_float2(k.s2, k.s2);
    if (k.nu_x2 == 1) return __fmul2_rn(s2, e);
    float2 p = __fadd2_rn(make_float2(1.f, 1.f), t);
    if (k.nu_x2 != 3) p = __ffma2_rn(__fmul2_rn(t, t), make_float2(1.f / 3.f, 1.f / 3.f), p);
    return __fmul2_rn(__fmul2_rn(s2, p), e);
}

__global__ void __launch_bounds__(256) k_features(const double* __restrict__ pts, long long n, int dim, KP<float> kp,
                                                  const long long* __restrict__ grp_ptr, long long n_grp,
                                                  const long long* __restrict__ cand_ptr,
                                                  const int32_t* __restrict__ cand_idx, float* __restrict__ feat,
                                                  DevStatus* st) {
    // member coordinates relative to the first member (formed in FP64, kept in FP32),
    // so that candidate-member differences keep their digits in FP32
    __shared__ float mx[64 * 3];
    __shared__ float cen[3];
    __shared__ float s_ri;
    __shared__ double org[3];
    for (long long g = blockIdx.x; g < n_grp; g += gridDim.x) {
        const long long g0 = grp_ptr[g];
        const int m = (int)(grp_ptr[g + 1] - g0);
        const long long b0 = cand_ptr[g];
        const int C = (int)(cand_ptr[g + 1] - b0);
        if (m < 1 || m > 64 || g0 < 0 || g0 + m > n || C < 0) {
            if (threadIdx.x == 0) record_error(st, SIC_ERR_INVALID, g);
            continue;
        }
        if (threadIdx.x < 3) org[threadIdx.x] = ((int)threadIdx.x < dim) ? pts[g0 * dim + threadIdx.x] : 0.0;
        __syncthreads();
        for (int i = threadIdx.x; i < m * 3; i += blockDim.x) {
            int a = i / 3, d = i % 3;
            mx[i] = (d < dim) ? (float)(pts[(g0 + a) * dim + d] - org[d]) : 0.f;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            float s = 0.f;
            for (int a = 0; a < m; ++a) s += mx[a * 3 + threadIdx.x];
            cen[threadIdx.x] = s / (float)m;
        }
        if (threadIdx.x == 32) {
            // candidate radius: nearest-member distance of the last candidate
            float R = 0.f;
            if (C > 0) {
                const long long pl = cand_idx[b0 + C - 1];
                if (pl >= 0 && pl < n) {
                    float xl[3];
                    for (int d = 0; d < 3; ++d) xl[d] = (d < dim) ? (float)(pts[pl * dim + d] - org[d]) : 0.f;
                    float best = INFINITY;
                    for (int a = 0; a < m; ++a) {
                        float dx = xl[0] - mx[a * 3], dy = xl[1] - mx[a * 3 + 1], dz = xl[2] - mx[a * 3 + 2];
                        best = fminf(best, dx * dx + dy * dy + dz * dz);
                    }
                    R = sqrtf(best);
                }
            }
            s_ri = (R > 0.f) ? 1.f / R : 1.f;
        }
        __syncthreads();
        const float ri = s_ri;
        const float inv_s2 = 1.f / kp.s2, inv_m = 1.f / (float)m;
        for (int r = threadIdx.x; r < C; r += blockDim.x) {
            const long long p = cand_idx[b0 + r];
            float* f = feat + (b0 + r) * NF;
            if (p < 0 || p >= n) {
                record_error(st, SIC_ERR_INVALID, g);
                for (int q = 0; q < NF; ++q) f[q] = 0.f;
                continue;
            }
            float x[3];
            for (int d = 0; d < 3; ++d) x[d] = (d < dim) ? (float)(pts[p * dim + d] - org[d]) : 0.f;
            float best = INFINITY, ksum = 0.f;
            int ab = 0;
            // members two at a time in packed FP32 pairs (sm_100+ f32x2: half the instructions),
            // the same operations lane-wise as the scalar tail; K summed and the nearest member
            // taken in member order (lowest index on ties)
            const float2 nx = make_float2(-x[0], -x[0]), ny = make_float2(-x[1], -x[1]),
                         nz = make_float2(-x[2], -x[2]);
            int a = 0;
            for (; a + 1 < m; a += 2) {
                const float2 dx = __fadd2_rn(make_float2(mx[a * 3], mx[a * 3 + 3]), nx);
                const float2 dy = __fadd2_rn(make_float2(mx[a * 3 + 1], mx[a * 3 + 4]), ny);
                const float2 dz = __fadd2_rn(make_float2(mx[a * 3 + 2], mx[a * 3 + 5]), nz);
                const float2 d2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                const float2 v = matern_f2(kp, make_float2(d2.x > 1e-30f ? d2.x * rsqrtf(d2.x) : 0.f,
                                                           d2.y > 1e-30f ? d2.y * rsqrtf(d2.y) : 0.f));
                ksum += v.x;
                ksum += v.y;
                if (d2.x < best) { best = d2.x; ab = a; }
                if (d2.y < best) { best = d2.y; ab = a + 1; }
            }
            if (a < m) {
                const float dx = __fadd_rn(mx[a * 3], -x[0]), dy = __fadd_rn(mx[a * 3 + 1], -x[1]),
                            dz = __fadd_rn(mx[a * 3 + 2], -x[2]);
                const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                const float r = d2 > 1e-30f ? d2 * rsqrtf(d2) : 0.f;
                ksum += matern_f2(kp, make_float2(r, r)).x;
                if (d2 < best) { best = d2; ab = a; }
            }
            const float dmin = sqrtf(best);
            float cx = x[0] - cen[0], cy = x[1] - cen[1], cz = x[2] - cen[2];
            // two 16-byte stores per candidate (the row of 8 features is 32-byte aligned)
            reinterpret_cast<float4*>(f)[0] = make_float4((x[0] - mx[ab * 3]) * ri, (x[1] - mx[ab * 3 + 1]) * ri, dmin * ri,
                                                          sqrtf(cx * cx + cy * cy + cz * cz) * ri);
            reinterpret_cast<float4*>(f)[1] = make_float4((float)r / (float)C, matern<float>(kp, dmin) * inv_s2,
                                                          (float)m * (1.f / 64.f), ksum * inv_m * inv_s2);
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------------- top-k --

__global__ void k_topk_counts(const long long* __restrict__ cand_ptr, long long n_grp, int top,
                              long long* __restrict__ out_ptr) {
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= n_grp) return;
    long long c = cand_ptr[g + 1] - cand_ptr[g];
    out_ptr[g] = c < top ? c : top;
}

// single-CTA exclusive scan of out_ptr[0..n) in place; out_ptr[n] receives the total
__global__ void __launch_bounds__(1024) k_scan_one_block(long long* __restrict__ v, long long n) {
    __shared__ long long s[1024];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < n; c0 += 1024) {
        long long i = c0 + threadIdx.x;
        long long x0 = (i < n) ? v[i] : 0;
        s[threadIdx.x] = x0;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            long long x = (threadIdx.x >= off) ? s[threadIdx.x - off] : 0;
            __syncthreads();
            s[threadIdx.x] += x;
            __syncthreads();
        }
        if (i < n) v[i] = carry + s[threadIdx.x] - x0;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) v[n] = carry;
}

// Order key: larger score first, then lower list index.  Scores are finite floats
// (NaN is treated as -inf).
__device__ __forceinline__ unsigned long long topk_key(float s, int r) {
    if (!(s == s)) s = -INFINITY;
    unsigned int u = __float_as_uint(s);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);  // monotone in s
    return ((unsigned long long)u << 32) | (unsigned int)(0x7fffffff - r);
}

// Per-group top-k by radix selection: the threshold key T (the top-th largest 32-bit
// order-preserving score key) is found digit by digit (4 passes of 8 bits, each a shared
// histogram of the keys that match the digits chosen so far and a one-warp scan from the
// top bin); then the list is compacted in order, keeping keys > T and, among keys == T,
// the first `need` in list order -- the same set as sorting by (score desc, position asc).
// A group is a short chain of barrier-separated phases, so the CTAs are small (4 warps) and
// many per SM: the histograms are double-buffered (the scanning warp clears the buffer of the
// previous pass), two barriers per pass; the compaction counts every slot's keys == T and
// kept keys per warp in two barrier phases and writes in a third (eleven barriers a group).
constexpr int TOPK_NT = 128;
constexpr int TOPK_NW = TOPK_NT / 32;
constexpr int TOPK_KPT = 4096 / TOPK_NT;  // key slots per thread (key r = tid + q TOPK_NT in slot q)
constexpr int TOPK_RK = 8;                // slots held in registers (lists of up to 1024); later ones re-read

__global__ void __launch_bounds__(TOPK_NT, 12) k_topk_compact(const long long* __restrict__ cand_ptr,
                                                          const int32_t* __restrict__ cand_idx,
                                                          const float* __restrict__ score, long long n_grp, int top,
                                                          const long long* __restrict__ out_ptr,
                                                          int32_t* __restrict__ out_idx, DevStatus* st) {
    __shared__ unsigned hist[2][256];
    __shared__ unsigned s_digit[2], s_need[2];
    __shared__ int cnt_eq[TOPK_KPT][TOPK_NW], cnt_k[TOPK_KPT][TOPK_NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (long long g = blockIdx.x; g < n_grp; g += gridDim.x) {
        const long long b0 = cand_ptr[g];
        const int C = (int)(cand_ptr[g + 1] - b0);
        const long long o0 = out_ptr[g];
        if (C <= top) {
            for (int r = tid; r < C; r += TOPK_NT) out_idx[o0 + r] = cand_idx[b0 + r];
            continue;
        }
        if (C > 4096) {
            if (tid == 0) record_error(st, SIC_ERR_UNSUPPORTED, g);
            continue;
        }
        const int nq = (C + TOPK_NT - 1) / TOPK_NT;  // slots holding keys
        unsigned key[TOPK_RK];
#pragma unroll
        for (int q = 0; q < TOPK_RK; ++q) {
            const int r = tid + q * TOPK_NT;
            key[q] = (r < C) ? (unsigned)(topk_key(score[b0 + r], r) >> 32) : 0u;
        }
        // slot q's key (q a compile-time index after unrolling)
        auto kq = [&](int q) -> unsigned {
            if (q < TOPK_RK) return key[q];
            const int r = tid + q * TOPK_NT;
            return (r < C) ? (unsigned)(topk_key(score[b0 + r], r) >> 32) : 0u;
        };
        for (int b = tid; b < 512; b += TOPK_NT) (&hist[0][0])[b] = 0u;
        __syncthreads();
        unsigned prefix = 0, mask = 0, need = (unsigned)top;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int shift = 24 - 8 * p;
            unsigned* h = hist[p & 1];
#pragma unroll
            for (int q = 0; q < TOPK_KPT; ++q) {
                if (q >= nq) break;
                const int r = tid + q * TOPK_NT;
                const unsigned kv = kq(q);
                if (r < C && (kv & mask) == prefix) atomicAdd(&h[(kv >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (warp == 0) {  // bins from the top: lane l holds bins 255 - 8l - i, i < 8
                unsigned c[8], sum = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    c[i] = h[255 - 8 * lane - i];
                    sum += c[i];
                }
                unsigned incl = sum;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const unsigned o = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += o;
                }
                const unsigned excl = incl - sum;
                if (excl < need && need <= incl) {
                    unsigned run = excl;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (run + c[i] >= need) {
                            s_digit[p & 1] = 255u - 8u * lane - i;
                            s_need[p & 1] = need - run;
                            break;
                        }
                        run += c[i];
                    }
                }
                // the previous pass's buffer (scanned before the barrier above) for the next pass
#pragma unroll
                for (int i = 0; i < 8; ++i) hist[(p + 1) & 1][lane + 32 * i] = 0u;
            }
            __syncthreads();
            prefix |= s_digit[p & 1] << shift;
            mask |= 255u << shift;
            need = s_need[p & 1];
        }
        // compaction in list order (slot-major: r = tid + q TOPK_NT): keys > T, then the first
        // `need` keys == T
        const unsigned T = prefix;
#pragma unroll
        for (int q = 0; q < TOPK_KPT; ++q) {
            if (q >= nq) break;
            const unsigned beq = __ballot_sync(0xffffffffu, tid + q * TOPK_NT < C && kq(q) == T);
            if (lane == 0) cnt_eq[q][warp] = __popc(beq);
        }
        __syncthreads();
        unsigned keepm = 0u;  // bit q: key slot q is kept
        int eq_run = 0;
#pragma unroll
        for (int q = 0; q < TOPK_KPT; ++q) {
            if (q >= nq) break;
            int tot = 0, bef = 0;
#pragma unroll
            for (int w = 0; w < TOPK_NW; ++w) {
                const int c = cnt_eq[q][w];
                tot += c;
                if (w < warp) bef += c;
            }
            const bool in = tid + q * TOPK_NT < C;
            const unsigned kv = kq(q);
            const bool eq = in && kv == T;
            const unsigned beq = __ballot_sync(0xffffffffu, eq);
            const bool kp = in && (kv > T || (eq && eq_run + bef + __popc(beq & lt) < (int)need));
            if (kp) keepm |= 1u << q;
            const unsigned bk = __ballot_sync(0xffffffffu, kp);
            if (lane == 0) cnt_k[q][warp] = __popc(bk);
            eq_run += tot;
        }
        __syncthreads();
        int base = 0;
#pragma unroll
        for (int q = 0; q < TOPK_KPT; ++q) {
            if (q >= nq) break;
            int tot = 0, bef = 0;
#pragma unroll
            for (int w = 0; w < TOPK_NW; ++w) {
                const int c = cnt_k[q][w];
                tot += c;
                if (w < warp) bef += c;
            }
            const bool kp = (keepm >> q) & 1u;
            const unsigned bk = __ballot_sync(0xffffffffu, kp);
            if (kp) out_idx[o0 + base + bef + __popc(bk & lt)] = cand_idx[b0 + tid + q * TOPK_NT];
            base += tot;
        }
        // (the next group rewrites the counts only after its own barriers)
    }
}

// label[b0 + r] = 1 if candidate r of group g is among the group's picks
__global__ void __launch_bounds__(256) k_labels(const long long* __restrict__ cand_ptr,
                                                const int32_t* __restrict__ cand_idx,
                                                const int32_t* __restrict__ sel_idx,
                                                const int32_t* __restrict__ sel_count, int k, long long n_grp,
                                                float* __restrict__ label) {
    __shared__ int sel[256];
    for (long long g = blockIdx.x; g < n_grp; g += gridDim.x) {
        const int cnt = min(sel_count[g], min(k, 256));
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) sel[i] = sel_idx[g * k + i];
        __syncthreads();
        const long long b0 = cand_ptr[g];
        const int C = (int)(cand_ptr[g + 1] - b0);
        for (int r = threadIdx.x; r < C; r += blockDim.x) {
            const int p = cand_idx[b0 + r];
            float y = 0.f;
            for (int i = 0; i < cnt; ++i) y = (sel[i] == p) ? 1.f : y;
            label[b0 + r] = y;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- training --

// C[z] = A * B over the K-range of split z (C has M x N, row-major; z-th partial at
// C + z * M * N).  A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn].
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, int kchunk, const float* __restrict__ A,
                                              long long sam, long long sak, const float* __restrict__ B,
                                              long long sbk, long long sbn, float* __restrict__ C) {
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    float acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += 16) {
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            int kk = i / 64, mm = i % 64;
            int k = k0 + kk;
            As[kk][mm] = (k < ke && m0 + mm < M) ? A[(long long)(m0 + mm) * sam + (long long)k * sak] : 0.f;
            Bs[kk][mm] = (k < ke && n0 + mm < N) ? B[(long long)k * sbk + (long long)(n0 + mm) * sbn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                b[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* Cz = C + (long long)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) Cz[(long long)m * N + n] = acc[i][j];
        }
}

// out[i] = sum_z part[z * len + i] (fixed order)
__global__ void k_sum_splits(const float* __restrict__ part, int nz, long long len, float* __restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= len) return;
    float s = 0.f;
    for (int z = 0; z < nz; ++z) s += part[(long long)z * len + i];
    out[i] = s;
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// W_used = round_bf16(master) (or a copy when bf16 is off)
__global__ void k_round_params(const float* __restrict__ p, float* __restrict__ q, int n, int bf16) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = bf16 ? bf16_round(p[i]) : p[i];
}

__global__ void k_round_rows(const float* __restrict__ x, float* __restrict__ y, long long n, int bf16) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = bf16 ? bf16_round(x[i]) : x[i];
}

// Z += bias (row-broadcast); H = gelu(Z) (H optionally rounded to bf16)
__global__ void k_bias_gelu(float* __restrict__ Z, float* __restrict__ H, const float* __restrict__ bias,
                            long long rows, int bf16) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows * HID) return;
    float z = Z[i] + bias[i % HID];
    Z[i] = z;
    float h = gelu_f(z);
    H[i] = bf16 ? bf16_round(h) : h;
}

// s = H2 w3 + b3; per-row loss and dS = (pw y (sigma - 1) + (1 - y) sigma) / B
__global__ void __launch_bounds__(128) k_head(const float* __restrict__ H2, const float* __restrict__ w3,
                                              const float* __restrict__ b3, const float* __restrict__ y,
                                              long long rows, float pw, float* __restrict__ s_out,
                                              float* __restrict__ dS, float* __restrict__ lrow) {
    long long r = blockIdx.x * (long long)(blockDim.x / 32) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (r >= rows) return;
    float acc = 0.f;
    for (int j = lane; j < HID; j += 32) acc = fmaf(H2[r * HID + j], w3[j], acc);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
        float s = acc + b3[0];
        float yy = y[r];
        float sig = 1.f / (1.f + expf(-s));
        // softplus(x) = max(x, 0) + log1p(exp(-|x|))
        float spn = fmaxf(-s, 0.f) + log1pf(expf(-fabsf(s)));
        float spp = fmaxf(s, 0.f) + log1pf(expf(-fabsf(s)));
        lrow[r] = pw * yy * spn + (1.f - yy) * spp;
        dS[r] = (pw * yy * (sig - 1.f) + (1.f - yy) * sig) / (float)rows;
        if (s_out) s_out[r] = s;
    }
}

// dZ2 = (dS w3^T) .* gelu'(Z2)
__global__ void k_dz2(const float* __restrict__ dS, const float* __restrict__ w3, const float* __restrict__ Z2,
                      float* __restrict__ dZ, long long rows) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows * HID) return;
    dZ[i] = dS[i / HID] * w3[i % HID] * dgelu_f(Z2[i]);
}

__global__ void k_mul_dgelu(float* __restrict__ dH, const float* __restrict__ Z, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dH[i] *= dgelu_f(Z[i]);
}

// column sums of a rows x cols matrix in fixed order: one thread per column
__global__ void k_colsum(const float* __restrict__ M, long long rows, int cols, float* __restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (long long r = 0; r < rows; ++r) s += M[r * cols + c];
    out[c] = s;
}

__global__ void __launch_bounds__(256) k_sum_loss(const float* __restrict__ l, long long n, float* __restrict__ out) {
    __shared__ float s[256];
    float a = 0.f;
    for (long long i = threadIdx.x; i < n; i += 256) a += l[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) s[threadIdx.x] += s[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0] / (float)n;
}

__global__ void k_adamw(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                        const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float wd,
                        float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float mh = mi / c1, vh = vi / c2;
    p[i] = p[i] - lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
}

// scratch layout of one training step on B rows (floats)
struct TrainWs {
    long long B;
    int nz;  // K-splits of the weight-gradient GEMMs
    long long q() const { return 0; }                        // rounded params, NPARAM
    long long xr() const { return NPARAM + 15; }             // rounded features B x 8
    long long z1() const { return xr() + B * NF; }           // B x 128
    long long h1() const { return z1() + B * HID; }
    long long z2() const { return h1() + B * HID; }
    long long h2() const { return z2() + B * HID; }
    long long ds() const { return h2() + B * HID; }          // B
    long long lrow() const { return ds() + B; }              // B
    long long part() const { return lrow() + B; }            // nz x 128 x 128
    long long size() const { return part() + (long long)nz * HID * HID; }
};

TrainWs train_ws(long long B) {
    TrainWs w;
    w.B = B;
    w.nz = (int)((B + 4095) / 4096);
    if (w.nz > 64) w.nz = 64;
    return w;
}

// the training GEMMs: 128-wide products in BF16 on the tensor cores (gemm_tc) when `tc`, the
// rest (and everything in the FP32 mode) in the CUDA-core tiled GEMM; K-splits summed in a
// fixed order either way
void gemm(cudaStream_t s, int M, int N, int K, const float* A, long long sam, long long sak, const float* B,
          long long sbk, long long sbn, float* C, int nz, float* part, sic_handle* tc = nullptr) {
    if (tc && N == HID) {
        gemm_tc(tc, s, M, K, A, sam, sak, B, sbk, sbn, nz == 1 ? C : part, nz);
        if (nz > 1) {
            long long len = (long long)M * N;
            k_sum_splits<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(part, nz, len, C);
        }
        return;
    }
    int kchunk = (K + nz - 1) / nz;
    kchunk = (kchunk + 15) / 16 * 16;
    dim3 grid((N + 63) / 64, (M + 63) / 64, nz);
    if (nz == 1) {
        k_gemm<<<grid, 256, 0, s>>>(M, N, K, kchunk, A, sam, sak, B, sbk, sbn, C);
    } else {
        k_gemm<<<grid, 256, 0, s>>>(M, N, K, kchunk, A, sam, sak, B, sbk, sbn, part);
        long long len = (long long)M * N;
        k_sum_splits<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(part, nz, len, C);
    }
}

}  // namespace

// ---------------------------------------------------------------- entry points --

extern "C" sic_status sic_proposal_features(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp, const int64_t* grp_ptr, int64_t n_grp,
                                            const int64_t* cand_ptr, const int32_t* cand_idx, float* feat,
                                            void* stream) {
    if (!h || !pts || n < 1 || !sic_valid_kernel(kp) || !grp_ptr || n_grp < 1 || !cand_ptr || !cand_idx ||
        !feat || ((uintptr_t)feat & 15u))
        return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    int grid = persistent_grid(h, k_features, 256, 0, n_grp);
    k_features<<<grid, 256, 0, s>>>(pts, n, kp->dim, make_kp<float>(*kp), (const long long*)grp_ptr, n_grp,
                                    (const long long*)cand_ptr, cand_idx, feat, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_proposal_score(sic_handle* h, const float* params, const float* feat, int64_t rows,
                                         float* score, void* stream) {
    if (!h || !params || !feat || rows < 0 || !score) return SIC_ERR_INVALID;
    if (rows == 0) return SIC_OK;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    return sic_proposal_score_tc(h, params, feat, rows, score, (cudaStream_t)stream);
}

extern "C" sic_status sic_proposal_topk(sic_handle* h, const int64_t* cand_ptr, const int32_t* cand_idx,
                                        const float* score, int64_t n_grp, int32_t top, int64_t* out_ptr,
                                        int32_t* out_idx, void* stream) {
    if (!h || !cand_ptr || !cand_idx || !score || n_grp < 1 || top < 1 || !out_ptr || !out_idx)
        return SIC_ERR_INVALID;
    if (top > 4096) return SIC_ERR_UNSUPPORTED;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    k_topk_counts<<<(unsigned)((n_grp + 255) / 256), 256, 0, s>>>((const long long*)cand_ptr, n_grp, top,
                                                                    (long long*)out_ptr);
    k_scan_one_block<<<1, 1024, 0, s>>>((long long*)out_ptr, n_grp);
    int grid = persistent_grid(h, k_topk_compact, TOPK_NT, 0, n_grp);
    k_topk_compact<<<grid, TOPK_NT, 0, s>>>((const long long*)cand_ptr, cand_idx, score, n_grp, top,
                                        (const long long*)out_ptr, out_idx, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_proposal_labels(sic_handle* h, const int64_t* cand_ptr, const int32_t* cand_idx,
                                          int64_t n_grp, const int32_t* sel_idx, const int32_t* sel_count, int32_t k,
                                          float* label, void* stream) {
    if (!h || !cand_ptr || !cand_idx || n_grp < 1 || !sel_idx || !sel_count || k < 1 || !label)
        return SIC_ERR_INVALID;
    if (k > 256) return SIC_ERR_UNSUPPORTED;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    int grid = persistent_grid(h, k_labels, 256, 0, n_grp);
    k_labels<<<grid, 256, 0, (cudaStream_t)stream>>>((const long long*)cand_ptr, cand_idx, sel_idx, sel_count, k,
                                                      n_grp, label);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_mlp_train_workspace(int64_t batch, size_t* bytes) {
    if (!bytes || batch < 1) return SIC_ERR_INVALID;
    *bytes = sizeof(float) * (size_t)train_ws(batch).size();
    return SIC_OK;
}

extern "C" sic_status sic_mlp_grads(sic_handle* h, const float* params, const float* feat, const float* label,
                                    int64_t batch, float pos_weight, int32_t bf16, float* grads, float* loss,
                                    float* score, void* ws, size_t ws_bytes, void* stream) {
    if (!h || !params || !feat || !label || batch < 1 || !grads || !loss || !ws) return SIC_ERR_INVALID;
    TrainWs L = train_ws(batch);
    if (ws_bytes < sizeof(float) * (size_t)L.size()) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    float* W = (float*)ws;
    float* q = W + L.q();
    float* xr = W + L.xr();
    float* Z1 = W + L.z1();
    float* H1 = W + L.h1();
    float* Z2 = W + L.z2();
    float* H2 = W + L.h2();
    float* dS = W + L.ds();
    float* lrow = W + L.lrow();
    float* part = W + L.part();
    const long long B = batch;
    const unsigned ew = (unsigned)((B * HID + 255) / 256);
    k_round_params<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, q, NPARAM, bf16);
    k_round_rows<<<(unsigned)((B * NF + 255) / 256), 256, 0, s>>>(feat, xr, B * NF, bf16);
    // forward (with bf16: the 128-wide products on the tensor cores, operands in BF16)
    sic_handle* tc = bf16 ? h : nullptr;
    gemm(s, (int)B, HID, NF, xr, NF, 1, q + OFF_W1, HID, 1, Z1, 1, part, tc);
    k_bias_gelu<<<ew, 256, 0, s>>>(Z1, H1, q + OFF_B1, B, bf16);
    gemm(s, (int)B, HID, HID, H1, HID, 1, q + OFF_W2, HID, 1, Z2, 1, part, tc);
    k_bias_gelu<<<ew, 256, 0, s>>>(Z2, H2, q + OFF_B2, B, 0);
    k_head<<<(unsigned)((B + 3) / 4), 128, 0, s>>>(H2, q + OFF_W3, q + OFF_B3, label, B, pos_weight, score, dS,
                                                   lrow);
    k_sum_loss<<<1, 256, 0, s>>>(lrow, B, loss);
    // backward: w3, b3
    gemm(s, HID, 1, (int)B, H2, 1, HID, dS, 1, 1, grads + OFF_W3, L.nz, part);
    k_colsum<<<1, 32, 0, s>>>(dS, B, 1, grads + OFF_B3);
    // dZ2 into H2's storage (H2 is no longer needed)
    k_dz2<<<ew, 256, 0, s>>>(dS, q + OFF_W3, Z2, H2, B);
    float* dZ2 = H2;
    gemm(s, HID, HID, (int)B, H1, 1, HID, dZ2, HID, 1, grads + OFF_W2, L.nz, part, tc);
    k_colsum<<<1, 128, 0, s>>>(dZ2, B, HID, grads + OFF_B2);
    // dH1 = dZ2 W2^T  -> into Z2's storage, then dZ1 = dH1 .* gelu'(Z1)
    gemm(s, (int)B, HID, HID, dZ2, HID, 1, q + OFF_W2, 1, HID, Z2, 1, part, tc);
    float* dZ1 = Z2;
    k_mul_dgelu<<<ew, 256, 0, s>>>(dZ1, Z1, B * HID);
    gemm(s, NF, HID, (int)B, xr, 1, NF, dZ1, HID, 1, grads + OFF_W1, L.nz, part, tc);
    k_colsum<<<1, 128, 0, s>>>(dZ1, B, HID, grads + OFF_B1);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_adamw_step(sic_handle* h, float* params, float* m, float* v, const float* grads,
                                     int32_t n, int32_t step, float lr, float beta1, float beta2, float eps,
                                     float wd, void* stream) {
    if (!h || !params || !m || !v || !grads || n < 1 || step < 1) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adamw<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, m, v, grads, n, lr, beta1, beta2, eps, wd,
                                                               c1, c2);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" int32_t sic_mlp_param_count(void) { return NPARAM; }
