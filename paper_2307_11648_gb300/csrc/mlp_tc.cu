// Proposal-network inference on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// One CTA of 128 threads scores 128 candidate rows at a time (persistent over row tiles):
//   layer 1  D = X W1 + b1  M = 128 rows, N = 128 hidden, K = 16: 8 features, a constant
//            1 whose weight row is b1, 7 zeros (the bias comes out of the MMA)
//   GELU     read D from TMEM (tcgen05.ld, thread = row), 2 gelu(D) (tanh form, see
//            gelu2_f2), round to BF16 and store as the next A operand in shared memory
//   layer 2  D = (2 H1) (W2 / 2)   M = 128, N = 128, K = 128 (8 MMAs of K = 16)
//   head     read D (thread = row: the whole hidden row is in the thread's registers),
//            s = sum_j 2 gelu(D_j + b2_j) (w3_j / 2) + b3 -- no cross-thread reduction.
// The factors 2 and 1/2 are exact in BF16 and FP32, so folding the GELU's 1/2 into W2 and
// w3 changes no rounding; it saves one multiply per hidden value.
// Operands are BF16 in shared memory in the K-major layout without swizzle: 8 x 16-byte
// "core matrices" (8 rows x 8 elements, 128 contiguous bytes), core matrices adjacent
// along K at LBO = 128 bytes, 8-row groups at SBO = (K / 8) * 128 bytes.  The weights
// are packed once per CTA.  Accumulators are FP32 in TMEM (128 lanes x 128 columns).
// One elected thread issues tcgen05.mma and commits to an mbarrier; every wait on the
// mbarrier is bounded (the kernel records SIC_ERR_TIMEOUT, frees its TMEM and returns).
#include <cuda_bf16.h>

#include "sic_internal.cuh"

namespace {

constexpr int NF = 8, HID = 128;
constexpr int OFF_B1 = NF * HID, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID,
              OFF_B3 = OFF_W3 + HID;
constexpr int TC_NT = 128;
constexpr unsigned TMEM_COLS = 128;
constexpr long long WAIT_CAP = 1LL << 28;

// shared-memory byte offsets of the operands (dynamic smem, 1024-byte aligned base)
constexpr int SA1 = 0;                    // 128 x 16 bf16 = 4 KiB
constexpr int SB1 = SA1 + 128 * 16 * 2;   // 128 x 16 bf16 = 4 KiB
constexpr int SA2 = SB1 + 128 * 16 * 2;   // 128 x 128 bf16 = 32 KiB
constexpr int SB2 = SA2 + 128 * 128 * 2;  // 128 x 128 bf16 = 32 KiB
constexpr int SVEC = SB2 + 128 * 128 * 2; // b2, w3 / 2 (FP32)
constexpr int SBAR = SVEC + 3 * HID * 4;  // mbarrier (8 B) + TMEM address (4 B)
constexpr int SMEM_TC = SBAR + 16;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) in the K-major no-swizzle core-matrix layout with K columns
__device__ __forceinline__ int core_off(int row, int k, int K) {
    return (row >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, relative LBO, no swizzle
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, N = 128, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// bounded wait for the mbarrier phase `parity`; returns false on timeout
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < WAIT_CAP; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Inference GELU: the tanh form of Hendrycks and Gimpel (2016),
// 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))), with the hardware tanh.  It departs
// from the erf form by at most 4.7e-4 (at |z| ~ 2.7), plus the tanh approximation's
// ~5e-4 relative, i.e. by less than the BF16 rounding of the hidden activations that
// follows (2^-9 relative); one MUFU operation and four FP32 operations instead of erf.
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// twice the GELU of a pair: z (1 + tanh(u)), u = z (0.7978845608 + 0.0356774081 z^2), the 1/2
// being folded into the consumer's weights; packed FP32 operations (sm_100+ f32x2: lane-wise
// the same round-to-nearest operations as the scalar form, half the instructions)
__device__ __forceinline__ float2 gelu2_f2(float2 z) {
    const float2 w = __ffma2_rn(make_float2(0.0356774081f, 0.0356774081f), __fmul2_rn(z, z),
                                make_float2(0.7978845608f, 0.7978845608f));
    const float2 u = __fmul2_rn(z, w);
    return __ffma2_rn(z, make_float2(tanh_hw(u.x), tanh_hw(u.y)), z);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__global__ void __launch_bounds__(TC_NT) k_mlp_tc(const float* __restrict__ X, long long rows,
                                                  const float* __restrict__ params, float* __restrict__ out,
                                                  DevStatus* st) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    float* sb2 = reinterpret_cast<float*>(sm + SVEC);
    float* sw3 = sb2 + HID;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + SBAR);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + SBAR + 8);
    const uint32_t bar_a = smem_u32(bar);

    // weights (W^T as N x K, K-major; row K = NF of layer 1 is b1, W2 and w3 halved), b2
    for (int e = tid; e < HID * 16; e += TC_NT) {
        const int n = e / 16, k = e % 16;
        const float w = (k < NF) ? params[k * HID + n] : (k == NF ? params[OFF_B1 + n] : 0.f);
        *reinterpret_cast<__nv_bfloat16*>(sm + SB1 + core_off(n, k, 16)) = __float2bfloat16_rn(w);
    }
    for (int e = tid; e < HID * HID; e += TC_NT) {
        const int n = e / HID, k = e % HID;
        *reinterpret_cast<__nv_bfloat16*>(sm + SB2 + core_off(n, k, HID)) =
            __float2bfloat16_rn(0.5f * params[OFF_W2 + k * HID + n]);
    }
    for (int i = tid; i < HID; i += TC_NT) {
        sb2[i] = params[OFF_B2 + i];
        sw3[i] = 0.5f * params[OFF_W3 + i];
    }
    const float b3 = params[OFF_B3];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    const uint64_t dA1 = smem_desc(smem_u32(sm + SA1), 128, 2 * 128);
    const uint64_t dB1 = smem_desc(smem_u32(sm + SB1), 128, 2 * 128);
    uint32_t parity = 0;
    bool failed = false;

    const long long ntiles = (rows + 127) / 128;
    for (long long tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        const long long r = tile * 128 + tid;
        // A1 row: 8 features, then 1 (picks up b1) and 7 zeros (two core matrices along K)
        float f[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) f[q] = (r < rows) ? X[r * NF + q] : 0.f;
        *reinterpret_cast<uint4*>(sm + SA1 + core_off(tid, 0, 16)) =
            make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
        *reinterpret_cast<uint4*>(sm + SA1 + core_off(tid, 8, 16)) = make_uint4(pack2(1.f, 0.f), 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            mma_f16(tmem, dA1, dB1, 0u);
            mma_commit(bar_a);
        }
        if (!bar_wait(bar_a, parity)) failed = true;
        parity ^= 1u;
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // layer-1 epilogue: thread = row, 128 hidden values in 4 chunks of 32 columns
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float v[32];
            tmem_ld32(lane_addr + c * 32, v);
            uint32_t pk[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float2 g = gelu2_f2(make_float2(v[2 * j], v[2 * j + 1]));
                pk[j] = pack2(g.x, g.y);
            }
#pragma unroll
            for (int g = 0; g < 4; ++g)
                *reinterpret_cast<uint4*>(sm + SA2 + core_off(tid, c * 32 + g * 8, HID)) =
                    make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const uint64_t dA = smem_desc(smem_u32(sm + SA2 + kk * 256), 128, 16 * 128);
                const uint64_t dB = smem_desc(smem_u32(sm + SB2 + kk * 256), 128, 16 * 128);
                mma_f16(tmem, dA, dB, kk > 0 ? 1u : 0u);
            }
            mma_commit(bar_a);
        }
        if (!bar_wait(bar_a, parity)) failed = true;
        parity ^= 1u;
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float v[32];
            tmem_ld32(lane_addr + c * 32, v);
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
                const float2 g = gelu2_f2(__fadd2_rn(make_float2(v[j], v[j + 1]),
                                                     make_float2(sb2[c * 32 + j], sb2[c * 32 + j + 1])));
                s = fmaf(g.x, sw3[c * 32 + j], s);
                s = fmaf(g.y, sw3[c * 32 + j + 1], s);
            }
        }
        if (r < rows) out[r] = s + b3;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (failed && tid == 0) record_error(st, SIC_ERR_TIMEOUT, blockIdx.x);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Self-test of the bounded wait: waits on an mbarrier that nothing arrives at, with the
// given iteration cap, and records SIC_ERR_TIMEOUT when the cap runs out.
__global__ void k_wait_selftest(long long cap, int* out, DevStatus* st) {
    __shared__ uint64_t bar;
    const uint32_t a = smem_u32(&bar);
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    __syncthreads();
    bool ok = false;
    for (long long it = 0; it < cap && !ok; ++it) {
        uint32_t r;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(r)
            : "r"(a), "r"(0u)
            : "memory");
        ok = r != 0;
    }
    if (threadIdx.x == 0) {
        out[0] = ok ? 1 : 0;
        if (!ok) record_error(st, SIC_ERR_TIMEOUT, -2);
    }
}

// ---- training GEMMs on the tensor cores ----
//
// C (M x 128, FP32, row-major) = A (M x K) * B (K x 128): A(m, k) = A[m * sam + k * sak],
// B(k, n) = B[k * sbk + n * sbn], so the same kernel serves X W, H^T dZ and dZ W^T.  Each CTA
// owns a 128-row tile of C and one K-range (split z, partial written at C + z * M * 128);
// per chunk of 64 along K, the 128 threads stage A and B rounded to BF16 into the K-major
// core-matrix layout (rows beyond M and entries beyond the K-range are zero), one thread
// issues four K = 16 MMAs accumulating in TMEM, and a bounded mbarrier wait ends the chunk.
// The epilogue reads the accumulator row by row (thread = row).
constexpr int GT_K = 64;                  // K per staged chunk
constexpr int GSA = 0;                    // 128 x 64 bf16 = 16 KiB
constexpr int GSB = GSA + 128 * GT_K * 2; // 128 x 64 bf16 = 16 KiB
constexpr int GSBAR = GSB + 128 * GT_K * 2;
// the dynamic shared memory requested is padded to 64 KiB so that at most three CTAs share an
// SM: 3 x 128 of the 512 TMEM columns, no CTA waits in tcgen05.alloc
constexpr int SMEM_GT = 64 * 1024;
static_assert(GSBAR + 16 <= SMEM_GT, "training GEMM shared memory");

__global__ void __launch_bounds__(TC_NT) k_gemm_tc(int M, int K, int kchunk, const float* __restrict__ A,
                                                   long long sam, long long sak, const float* __restrict__ B,
                                                   long long sbk, long long sbn, float* __restrict__ C,
                                                   DevStatus* st) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + GSBAR);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + GSBAR + 8);
    const uint32_t bar_a = smem_u32(bar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int m0 = blockIdx.x * 128;
    const int kb = blockIdx.y * kchunk, ke = min(K, kb + kchunk);
    uint32_t parity = 0;
    bool failed = false, any = false;
    for (int k0 = kb; k0 < ke && !failed; k0 += GT_K) {
        // stage: consecutive threads walk the operand's contiguous direction
        for (int e = tid; e < 128 * GT_K; e += TC_NT) {
            int m, kk;
            if (sak == 1) { m = e / GT_K; kk = e % GT_K; } else { kk = e / 128; m = e % 128; }
            const int k = k0 + kk;
            const float v = (m0 + m < M && k < ke) ? A[(long long)(m0 + m) * sam + (long long)k * sak] : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(sm + GSA + core_off(m, kk, GT_K)) = __float2bfloat16_rn(v);
        }
        for (int e = tid; e < 128 * GT_K; e += TC_NT) {
            int n, kk;
            if (sbk == 1) { n = e / GT_K; kk = e % GT_K; } else { kk = e / 128; n = e % 128; }
            const int k = k0 + kk;
            const float v = (k < ke) ? B[(long long)k * sbk + (long long)n * sbn] : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(sm + GSB + core_off(n, kk, GT_K)) = __float2bfloat16_rn(v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int q = 0; q < GT_K / 16; ++q) {
                const uint64_t dA = smem_desc(smem_u32(sm + GSA + q * 256), 128, (GT_K / 8) * 128);
                const uint64_t dB = smem_desc(smem_u32(sm + GSB + q * 256), 128, (GT_K / 8) * 128);
                mma_f16(tmem, dA, dB, (any || q > 0) ? 1u : 0u);
            }
            mma_commit(bar_a);
        }
        any = true;
        if (!bar_wait(bar_a, parity)) failed = true;
        parity ^= 1u;
        if (__syncthreads_or(failed)) failed = true;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!failed) {
        float* Cz = C + (long long)blockIdx.y * M * 128;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        const int m = m0 + tid;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float v[32];
            if (any) {
                tmem_ld32(lane_addr + c * 32, v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0.f;  // an empty K-range
            }
            if (m < M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) Cz[(long long)m * 128 + c * 32 + j] = v[j];
            }
        }
    } else if (tid == 0) {
        record_error(st, SIC_ERR_TIMEOUT, blockIdx.x);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace

sic_status gemm_tc(sic_handle* h, cudaStream_t s, int M, int K, const float* A, long long sam, long long sak,
                   const float* B, long long sbk, long long sbn, float* C, int nz) {
    (void)h;
    int kchunk = (K + nz - 1) / nz;
    kchunk = (kchunk + GT_K - 1) / GT_K * GT_K;
    SIC_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_GT));
    dim3 grid((unsigned)((M + 127) / 128), (unsigned)nz);
    k_gemm_tc<<<grid, TC_NT, SMEM_GT, s>>>(M, K, kchunk, A, sam, sak, B, sbk, sbn, C, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

extern "C" sic_status sic_selftest_wait_timeout(sic_handle* h, int64_t cap, int32_t* out, void* stream) {
    if (!h || !out || cap < 1) return SIC_ERR_INVALID;
    if (cap > (1LL << 24)) return SIC_ERR_INVALID;  // keep the self-test short
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(cap, out, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}

// Scores with the tcgen05 kernel (same contract as sic_proposal_score).
sic_status sic_proposal_score_tc(sic_handle* h, const float* params, const float* feat, int64_t rows, float* score,
                                 cudaStream_t s) {
    SIC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TC));
    // three CTAs per SM: 3 x (73 KiB + 1 KiB reserved) of shared memory and 3 x 128 of the
    // 512 TMEM columns; the epilogues of one CTA overlap the MMAs of the others
    long long tiles = (rows + 127) / 128;
    long long g = 3LL * h->num_sms;
    if (tiles < g) g = tiles;
    k_mlp_tc<<<(unsigned)g, TC_NT, SMEM_TC, s>>>(feat, rows, params, score, h->d_status);
    SIC_CUDA_TRY(cudaGetLastError());
    return SIC_OK;
}
