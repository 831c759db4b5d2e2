// The GEMMs of the correction network (the learned smoothing sweep) on the fifth-generation
// tensor cores: C[M][N] = sum_k A(m, k) B(k, n) with FP32 accumulation in tensor memory and
// FP32-accurate products from TF32 MMAs: every FP32 operand is split into a TF32 head and a
// TF32 tail (v = hi + lo to about 2^-22 |v|) and the products hi*hi + lo*hi + hi*lo are
// accumulated (the tail*tail term is below FP32 rounding).  A is FP32 (activations, residuals,
// output gradients), B FP32 or BF16 (the weights' BF16 copies are exact in TF32, so they need no
// tail and two MMAs suffice); either operand may be read transposed:
//     A(m, k) = TA ? A[k lda + m] : A[m lda + k],   B(k, n) = TB ? B[n ldb + k] : B[k ldb + n].
// A CTA computes a 128 x 128 tile of C over a K range (blockIdx.z splits K for the weight
// gradients, whose K is the batch), 32 K per step: its 128 threads load the A and B tiles from
// global memory (coalesced along whichever index is contiguous), round them to TF32 and store
// them in the canonical no-swizzle K-major core-matrix layout into one of two shared-memory
// stages; one thread issues four tcgen05.mma per step and commits them to the stage's mbarrier,
// so the loads of the next step overlap the MMAs of this one.  Epilogues as in mlp.cu: store,
// + bias, + bias with ReLU (the pre-activation kept), or atomic accumulation (split K).  Every
// wait is bounded (1 s); a wait that runs out sets the error flag and the kernel returns with
// its tensor memory freed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mlp.hpp"

namespace sem {

namespace {

constexpr int kGBM = 128, kGBN = 128, kGBK = 32;
constexpr uint32_t kGTile = kGBM * kGBK * 4;                 // one operand tile (16 KB)
constexpr uint32_t kGStage = 4 * kGTile;                      // A head, A tail, B head, B tail
constexpr uint32_t kGSmem = 2 * kGStage;                      // two stages
constexpr unsigned long long kGWaitNs = 1000000000ULL;

__host__ __device__ constexpr uint32_t gopoff(int r, int k) {
    return (uint32_t)((r >> 3) * (kGBK * 32) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__host__ __device__ constexpr uint32_t gidesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t g_smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t g_sdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)(((kGBK * 32) >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ float g_tf32(float f) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
    return __uint_as_float(r);
}

__device__ __forceinline__ float g_to_f(float v) { return v; }
__device__ __forceinline__ float g_to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ bool g_wait(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = [] {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        return t;
    }();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > kGWaitNs) return false;
    }
}

// head and tail of a value in TF32: v = hi + lo to about 2^-22 |v|
__device__ __forceinline__ float4 g_head(const float (&v)[4]) {
    return make_float4(g_tf32(v[0]), g_tf32(v[1]), g_tf32(v[2]), g_tf32(v[3]));
}
__device__ __forceinline__ float4 g_tail(const float (&v)[4], float4 h) {
    return make_float4(g_tf32(v[0] - h.x), g_tf32(v[1] - h.y), g_tf32(v[2] - h.z), g_tf32(v[3] - h.w));
}

// tile (rows r of the operand, K columns k) of an operand X(r, k) = T ? X[k ld + r] : X[r ld + k]
// into shared memory as TF32 head (dst) and tail (dst + kGTile, when TAIL) in the K-major
// core-matrix layout; rows >= R or columns >= kend are zero
template <bool T, typename TX, bool TAIL>
__device__ __forceinline__ void g_load_tile(unsigned char* dst, const TX* __restrict__ X, int ld, int r0, int R,
                                            int k0, int kend) {
    const int t = threadIdx.x;
    if (!T) {
        // row r = t, eight consecutive k per load group: two 16-byte shared stores
        const int r = r0 + t;
#pragma unroll
        for (int j = 0; j < kGBK / 8; ++j) {
            float v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int k = k0 + 8 * j + c;
                v[c] = (r < R && k < kend) ? g_to_f(X[(size_t)r * ld + k]) : 0.f;
            }
            const float va[4] = {v[0], v[1], v[2], v[3]}, vb[4] = {v[4], v[5], v[6], v[7]};
            const float4 ha = g_head(va), hb = g_head(vb);
            *reinterpret_cast<float4*>(dst + gopoff(t, 8 * j)) = ha;
            *reinterpret_cast<float4*>(dst + gopoff(t, 8 * j + 4)) = hb;
            if (TAIL) {
                *reinterpret_cast<float4*>(dst + kGTile + gopoff(t, 8 * j)) = g_tail(va, ha);
                *reinterpret_cast<float4*>(dst + kGTile + gopoff(t, 8 * j + 4)) = g_tail(vb, hb);
            }
        }
    } else {
        // row r = t is the contiguous index: consecutive threads read consecutive addresses
        const int r = r0 + t;
#pragma unroll 2
        for (int kq = 0; kq < kGBK / 4; ++kq) {
            float v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int k = k0 + 4 * kq + c;
                v[c] = (r < R && k < kend) ? g_to_f(X[(size_t)k * ld + r]) : 0.f;
            }
            const float4 h = g_head(v);
            *reinterpret_cast<float4*>(dst + gopoff(t, 4 * kq)) = h;
            if (TAIL) *reinterpret_cast<float4*>(dst + kGTile + gopoff(t, 4 * kq)) = g_tail(v, h);
        }
    }
}

template <bool TA, bool TB, typename TBt, int EPI>
__global__ void __launch_bounds__(128, 1)
    k_gemm_t5(int M, int N, int K, const float* __restrict__ A, int lda, const TBt* __restrict__ B, int ldb,
              float* __restrict__ C, int ldc, const float* __restrict__ bias, float* __restrict__ Cpre, int kchunk,
              int* err) {
    constexpr bool BTAIL = sizeof(TBt) == sizeof(float);     // FP32 B operands carry a tail
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t s_tmem;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int m0 = blockIdx.y * kGBM, n0 = blockIdx.x * kGBN;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    const uint32_t sbase = g_smem_u32(gsm);
    const uint32_t bar0 = g_smem_u32(&mbar[0]);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(g_smem_u32(&s_tmem)),
                     "r"(kGBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t id = gidesc(kGBM, kGBN);
    const int steps = (kend - kbeg + kGBK - 1) / kGBK;
    bool ok = true;
    for (int i = 0; i < steps; ++i) {
        const int st = i & 1;
        // the MMAs of step i - 2 read this stage: wait for them before overwriting it
        if (i >= 2 && !__syncthreads_and(g_wait(bar0 + 8u * st, (uint32_t)(((i - 2) >> 1) & 1)))) {
            ok = false;      // uniform: every thread leaves the loop here
            break;
        }
        unsigned char* sa = gsm + st * kGStage;
        unsigned char* sb = sa + 2 * kGTile;
        const int k0 = kbeg + i * kGBK;
        g_load_tile<TA, float, true>(sa, A, lda, m0, M, k0, kend);
        // B's operand rows are n: B(k, n) = X(n, k); BF16 weights are exact in TF32 (no tail)
        g_load_tile<!TB, TBt, BTAIL>(sb, B, ldb, n0, N, k0, kend);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = sbase + st * kGStage, b0 = a0 + 2 * kGTile;
            auto mma = [&](uint64_t ad, uint64_t bd, uint32_t acc) {
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
                        tmem),
                    "l"(ad), "l"(bd), "r"(id), "r"(acc)
                    : "memory");
            };
#pragma unroll
            for (int ks = 0; ks < kGBK / 8; ++ks) {
                const uint64_t ah = g_sdesc(a0 + ks * 256), al = g_sdesc(a0 + kGTile + ks * 256);
                const uint64_t bh = g_sdesc(b0 + ks * 256), bl = g_sdesc(b0 + kGTile + ks * 256);
                mma(ah, bh, (i > 0 || ks > 0) ? 1u : 0u);
                mma(al, bh, 1u);
                if (BTAIL) mma(ah, bl, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             bar0 + 8u * st)
                         : "memory");
        }
    }
    // the last step's MMAs (and the one before, whose completion nobody waited for)
    if (ok && steps >= 2 && !g_wait(bar0 + 8u * ((steps - 2) & 1), (uint32_t)(((steps - 2) >> 1) & 1))) ok = false;
    if (ok && steps >= 1 && !g_wait(bar0 + 8u * ((steps - 1) & 1), (uint32_t)(((steps - 1) >> 1) & 1))) ok = false;
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (t == 0) atomicExch(err, 1);
    } else if (steps > 0) {
        const int m = m0 + 32 * warp + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < kGBN; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(trow + c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m >= M) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = n0 + c0 + j;
                if (n >= N) continue;
                float x = __uint_as_float(v[j]);
                const size_t o = (size_t)m * ldc + n;
                if (EPI == EPI_ATOMIC) {
                    atomicAdd(&C[o], x);
                } else {
                    if (EPI == EPI_BIAS || EPI == EPI_BIAS_RELU) x += bias[n];
                    if (EPI == EPI_BIAS_RELU) {
                        Cpre[o] = x;
                        x = fmaxf(x, 0.f);
                    }
                    C[o] = x;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGBN) : "memory");
    }
}

}  // namespace

template <bool TA, bool TB, typename TBt, int EPI>
cudaError_t gemm_t5(int M, int N, int K, const float* A, int lda, const TBt* B, int ldb, float* C, int ldc,
                    const float* bias, float* Cpre, int splitk, int* err, cudaStream_t s) {
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        e = cudaFuncSetAttribute(k_gemm_t5<TA, TB, TBt, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kGSmem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    if (M < 1 || N < 1 || K < 1) return cudaSuccess;
    splitk = std::max(1, splitk);
    const int kchunk = ((K + splitk - 1) / splitk + kGBK - 1) / kGBK * kGBK;
    const int nz = (K + kchunk - 1) / kchunk;
    dim3 grid((N + kGBN - 1) / kGBN, (M + kGBM - 1) / kGBM, nz);
    k_gemm_t5<TA, TB, TBt, EPI><<<grid, 128, kGSmem, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, Cpre, kchunk, err);
    return cudaGetLastError();
}

// the shapes of the network's forward and backward passes
template cudaError_t gemm_t5<false, true, __nv_bfloat16, EPI_BIAS_RELU>(int, int, int, const float*, int,
                                                                        const __nv_bfloat16*, int, float*, int,
                                                                        const float*, float*, int, int*, cudaStream_t);
template cudaError_t gemm_t5<false, true, __nv_bfloat16, EPI_BIAS>(int, int, int, const float*, int,
                                                                   const __nv_bfloat16*, int, float*, int, const float*,
                                                                   float*, int, int*, cudaStream_t);
template cudaError_t gemm_t5<true, false, float, EPI_ATOMIC>(int, int, int, const float*, int, const float*, int,
                                                             float*, int, const float*, float*, int, int*,
                                                             cudaStream_t);
template cudaError_t gemm_t5<false, false, __nv_bfloat16, EPI_STORE>(int, int, int, const float*, int,
                                                                     const __nv_bfloat16*, int, float*, int,
                                                                     const float*, float*, int, int*, cudaStream_t);

}  // namespace sem
