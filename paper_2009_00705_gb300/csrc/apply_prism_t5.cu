// Prism apply of order 6 on the fifth-generation tensor cores (tcgen05) for the
// smoothing sweeps of the mixed-precision V-cycle (Eq. laplaceproblemdiscrete; the
// same contraction as apply_prism.cu and apply_prism_tc.cu).  Per CTA pass of 16
// elements the two triangle contractions are TF32 tcgen05.mma with M = 128 rows
// (16 elements x 8 vertical points, the eighth zero) and FP32 accumulators in
// tensor memory:
//
//   forward   [Ur | Us](e,qz; qt) = U(e,qz; n) [Dr | Ds](n; qt),  Ut = W(e,qz; n) Bt(n; qt)
//             (K = n: 28 -> 32, N = qt: 49 -> 64, three accumulators of 64 columns)
//   backward  Xr(e,qz; n) = Vr(e,qz; qt) Dr(qt; n) + Vs Ds,  Xt = Vt Bt
//             (K = qt: 49 -> 56, N = n: 28 -> 32, two accumulators of 32 columns)
//
// The forward operands come from shared memory through matrix descriptors (K-major, no
// swizzle: 8-row x 16-byte core matrices, K-adjacent ones 128 B apart, row groups K * 32 B
// apart), so the contractions put no load on the LSU pipe that bounds the warp-MMA form.
// Between the two, each thread owns one accumulator row (tcgen05.ld from its warp's lane
// quarter), applies the BF16 geometric factors and writes V over the accumulators it read
// (tcgen05.st): the backward MMAs take V as their A operand straight from tensor memory,
// so no shared memory holds it.  The vertical stages, the gather and the direct-stiffness
// summation stay on the SIMT pipes.  One thread issues the MMAs and commits them to an
// mbarrier; every wait is bounded (1 s), after which the kernel sets an error flag and
// returns with its tensor memory freed.  Two CTAs per SM (102 KB of shared memory and 256
// of the SM's 512 TMEM columns each), so one computes while the other waits.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sem_internal.hpp"

namespace sem {

namespace {

constexpr int kT5SMs = 152;
constexpr int kT5Threads = 256;
constexpr unsigned long long kT5WaitNs = 1000000000ULL;

constexpr int NT = 28, NZ = 7, QT = 49, QZ = 7, Np = NT * NZ, QTP = 50, GE = 6 * QZ * QTP;
constexpr int EB = 16;                 // elements per pass: 16 x 8 rows = M = 128
constexpr int KF = 32, NF = 64;        // forward K (n) and N (qt), padded
constexpr int KB = 56, NB = 32;        // backward K (qt) and N (n), padded

// byte offset of entry (r, k) of a K-major operand with K columns
__host__ __device__ constexpr uint32_t opoff(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K * 32) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

constexpr uint32_t SZ_BF = NF * KF * 4;          // one forward reference operand
constexpr uint32_t SZ_BB = NB * KB * 4;          // one backward reference operand
constexpr uint32_t SZ_AF = 128 * KF * 4;         // U, W
constexpr uint32_t SZ_MAP = EB * Np * 4;
constexpr uint32_t OFF_BF = 0;                   // Dr, Ds, Bt as (qt, n)
constexpr uint32_t OFF_BB = OFF_BF + 3 * SZ_BF;  // Dr, Ds, Bt as (n, qt)
constexpr uint32_t OFF_U = OFF_BB + 3 * SZ_BB;  // U, W; after the forward MMAs: Xr, Xt staging
constexpr uint32_t OFF_W = OFF_U + SZ_AF;
constexpr uint32_t OFF_X = OFF_U;
constexpr uint32_t OFF_MAP = OFF_W + SZ_AF;      // two map buffers
constexpr uint32_t OFF_Z = OFF_MAP + 2 * SZ_MAP; // Bz, Dz as [QZ][NZ] floats
constexpr uint32_t SMEM = OFF_Z + 2 * QZ * NZ * 4 + 8;   // multiple of 16
constexpr uint32_t SZ_X = EB * NT * 8 * 4;       // Xr or Xt staging, [EB][NT][8]
static_assert(SMEM % 16 == 0 && 2 * (SMEM + 2048) <= 233472, "two CTAs per SM");
static_assert(2 * SZ_X <= 2 * SZ_AF, "X staging fits in the U, W region");
static_assert(OFF_MAP % 16 == 0 && SZ_MAP % 16 == 0, "bulk copies of the map land on 16-byte boundaries");
static_assert((EB * Np * 4) % 16 == 0, "every pass's map block starts on a 16-byte boundary");

constexpr uint32_t TM_DR = 0, TM_DS = 64, TM_DT = 128, TM_XR = 192, TM_XT = 224, TM_COLS = 256;

// instruction descriptor of kind::tf32: F32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading (K-direction) byte offset 128, stride
// (row-group) byte offset sbo, no swizzle, descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t to_tf32(float f) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
    return r;
}

__device__ __forceinline__ unsigned long long t5_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool t5_wait(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = t5_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (t5_ns() - t0 > kT5WaitNs) return false;
    }
}

// one thread: bulk-copy `bytes` (a multiple of 16) from global to shared, completing on `bar`
__device__ void t5_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    const char* s = reinterpret_cast<const char*>(src);
    for (uint32_t off = 0; off < bytes; off += 16384u) {
        const uint32_t n = (bytes - off < 16384u) ? (bytes - off) : 16384u;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         dst + off),
                     "l"(s + off), "r"(n), "r"(bar)
                     : "memory");
    }
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

// D (tensor memory) = A (tensor memory) B^T (shared memory)
__device__ __forceinline__ void mma_tf32_ta(uint32_t tmem, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem),
        "r"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__global__ void __launch_bounds__(kT5Threads, 2)
    k_apply_prism_t5(int E, int N, const int* __restrict__ map, const __nv_bfloat16* __restrict__ G16,
                     const float* __restrict__ refm, const float* __restrict__ x, float* __restrict__ y,
                     const int* __restrict__ skip, int* err) {
    if (skip != nullptr && *skip) return;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) unsigned long long mbar[2];   // [0] MMA completion, [1] element-map copies
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t sbase = smem_u32(sm);
    const uint32_t bara = smem_u32(&mbar[0]), barm = smem_u32(&mbar[1]);

    // every pad entry of every operand must be zero
    for (uint32_t i = tid; i < SMEM / 16; i += kT5Threads) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int i = tid; i < QT * NT; i += kT5Threads) {
        const int qt = i / NT, n = i - qt * NT;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            // reference blocks in refm: Bt, Dr, Ds as [QT][NT]; operands m = Dr, Ds, Bt
            const float v = __uint_as_float(to_tf32(refm[((m + 1) % 3) * QT * NT + i]));
            *reinterpret_cast<float*>(sm + OFF_BF + m * SZ_BF + opoff(qt, n, KF)) = v;
            *reinterpret_cast<float*>(sm + OFF_BB + m * SZ_BB + opoff(n, qt, KB)) = v;
        }
    }
    float* sZ = reinterpret_cast<float*>(sm + OFF_Z);
    for (int i = tid; i < 2 * QZ * NZ; i += kT5Threads) sZ[i] = refm[6 * QT * NT + i];   // Bz, Dz as [QZ][NZ]
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bara) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barm) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t idF = idesc(128, NF), idB = idesc(128, NB);
    const int stride = gridDim.x * EB;
    uint32_t pa = 0, pm = 0;
    int buf = 0;
    if (tid == 0 && blockIdx.x * EB < E) {
        fence_async_smem();
        const int e = blockIdx.x * EB;
        t5_copy(sbase + OFF_MAP, map + (size_t)e * Np, (uint32_t)min(EB, E - e) * Np * 4u, barm);
    }
    // this thread's accumulator row in the epilogues: lane quarter of its warp
    const int q4 = warp & 3, half = warp >> 2;
    const int row = 32 * q4 + lane, rb = row >> 3, rqz = row & 7;
    const uint32_t trow = tmem + ((uint32_t)(32 * q4) << 16);

    for (int e0 = blockIdx.x * EB; e0 < E; e0 += stride) {
        const int nb = min(EB, E - e0);
        const int* sMap = reinterpret_cast<const int*>(sm + OFF_MAP + buf * SZ_MAP);
        if (!t5_wait(barm, pm)) s_fail = 1; else pm ^= 1u;
        __syncthreads();
        if (s_fail) break;
        // the next pass's map into the other buffer (its last reader finished last pass)
        if (tid == 0 && e0 + stride < E) {
            fence_async_smem();
            const int en = e0 + stride;
            t5_copy(sbase + OFF_MAP + (buf ^ 1) * SZ_MAP, map + (size_t)en * Np, (uint32_t)min(EB, E - en) * Np * 4u,
                    barm);
        }
        {   // the next pass's factors into L2 while this one computes
            const int en = e0 + stride;
            if (en < E) {
                const char* g0 = reinterpret_cast<const char*>(G16 + (size_t)en * GE);
                const size_t gb = (size_t)min(EB, E - en) * GE * 2;
                for (size_t off = (size_t)tid * 128; off < gb; off += (size_t)kT5Threads * 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(g0 + off));
            }
        }
        // pads of U and W (the last pass's X staging overwrote them): columns n = 28..31 of every
        // row (one core-matrix row each) and the eighth vertical row of every element
        for (int i = tid; i < 2 * 128 + 2 * EB * (NT / 4); i += kT5Threads) {
            uint32_t o;
            if (i < 256) {
                o = (i < 128 ? OFF_U : OFF_W) + opoff(i & 127, NT, KF);
            } else {
                const int j = i - 256, mtx = j / (EB * (NT / 4)), jj = j - mtx * (EB * (NT / 4));
                o = (mtx ? OFF_W : OFF_U) + opoff(8 * (jj / (NT / 4)) + 7, 4 * (jj % (NT / 4)), KF);
            }
            *reinterpret_cast<uint4*>(sm + o) = make_uint4(0, 0, 0, 0);
        }
        // gather and vertical stage: U(e,qz; n) = Bz(qz; k) x(k; n), W = Dz x
        for (int i = tid; i < EB * NT; i += kT5Threads) {
            const int b = i / NT, n = i - b * NT;
            float xk[NZ];
#pragma unroll
            for (int k = 0; k < NZ; ++k) {
                float v = 0.f;
                if (b < nb) {
                    const int m = sMap[b * Np + k * NT + n];
                    if (m >= 0 && m < N) v = x[m];
                }
                xk[k] = v;
            }
#pragma unroll
            for (int qz = 0; qz < QZ; ++qz) {
                float u = 0.f, w = 0.f;
#pragma unroll
                for (int k = 0; k < NZ; ++k) {
                    u += sZ[qz * NZ + k] * xk[k];
                    w += sZ[QZ * NZ + qz * NZ + k] * xk[k];
                }
                *reinterpret_cast<float*>(sm + OFF_U + opoff(8 * b + qz, n, KF)) = __uint_as_float(to_tf32(u));
                *reinterpret_cast<float*>(sm + OFF_W + opoff(8 * b + qz, n, KF)) = __uint_as_float(to_tf32(w));
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < KF / 8; ++ks) {
                const uint64_t au = sdesc(sbase + OFF_U + ks * 256, KF * 32);
                const uint64_t aw = sdesc(sbase + OFF_W + ks * 256, KF * 32);
                mma_tf32(tmem + TM_DR, au, sdesc(sbase + OFF_BF + ks * 256, KF * 32), idF, ks);
                mma_tf32(tmem + TM_DS, au, sdesc(sbase + OFF_BF + SZ_BF + ks * 256, KF * 32), idF, ks);
                mma_tf32(tmem + TM_DT, aw, sdesc(sbase + OFF_BF + 2 * SZ_BF + ks * 256, KF * 32), idF, ks);
            }
            mma_commit(bara);
        }
        if (!t5_wait(bara, pa)) s_fail = 1; else pa ^= 1u;
        fence_after();
        __syncthreads();
        if (s_fail) break;
        // geometric factors: thread (row, half) takes the 8-column chunks c = half, half + 2, half + 4,
        // half + 6 (qt in [8c, 8c + 8), c < 7 = K of the backward MMAs) and writes V over them
        {
            const bool valid = rb < nb && rqz < QZ;
            const __nv_bfloat16* Ge = G16 + (size_t)(e0 + (valid ? rb : 0)) * GE + rqz * QTP;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int c = half + 2 * cc;
                if (c >= KB / 8) continue;
                const int c0 = 8 * c;
                float g[4][6][2];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int qt = c0 + 2 * j;
#pragma unroll
                    for (int m = 0; m < 6; ++m) {
                        float2 f = make_float2(0.f, 0.f);
                        if (valid && qt < QT)
                            f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(Ge + m * QZ * QTP + qt));
                        g[j][m][0] = f.x;
                        g[j][m][1] = f.y;
                    }
                }
                uint32_t ur[8], us[8], ut[8];
                tmem_ld8(trow + TM_DR + c0, ur);
                tmem_ld8(trow + TM_DS + c0, us);
                tmem_ld8(trow + TM_DT + c0, ut);
                tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float* gg[6] = {g[k >> 1][0], g[k >> 1][1], g[k >> 1][2], g[k >> 1][3], g[k >> 1][4], g[k >> 1][5]};
                    const int hh = k & 1;
                    const float a = __uint_as_float(ur[k]), b = __uint_as_float(us[k]), t = __uint_as_float(ut[k]);
                    const float vr = gg[0][hh] * a + gg[1][hh] * b + gg[2][hh] * t;
                    const float vs = gg[1][hh] * a + gg[3][hh] * b + gg[4][hh] * t;
                    const float vt = gg[2][hh] * a + gg[4][hh] * b + gg[5][hh] * t;
                    ur[k] = to_tf32(vr);
                    us[k] = to_tf32(vs);
                    ut[k] = to_tf32(vt);
                }
                tmem_st8(trow + TM_DR + c0, ur);
                tmem_st8(trow + TM_DS + c0, us);
                tmem_st8(trow + TM_DT + c0, ut);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < KB / 8; ++ks) {
                const uint32_t o = ks * 256;
                mma_tf32_ta(tmem + TM_XR, tmem + TM_DR + 8 * ks, sdesc(sbase + OFF_BB + o, KB * 32), idB, ks);
                mma_tf32_ta(tmem + TM_XR, tmem + TM_DS + 8 * ks, sdesc(sbase + OFF_BB + SZ_BB + o, KB * 32), idB, 1);
                mma_tf32_ta(tmem + TM_XT, tmem + TM_DT + 8 * ks, sdesc(sbase + OFF_BB + 2 * SZ_BB + o, KB * 32), idB, ks);
            }
            mma_commit(bara);
        }
        if (!t5_wait(bara, pa)) s_fail = 1; else pa ^= 1u;
        fence_after();
        __syncthreads();
        if (s_fail) break;
        {   // Xr (warps 0-3) or Xt (warps 4-7) of this row into the staging area [e][n][qz]
            uint32_t xa[16], xb[16];
            const uint32_t col = half ? TM_XT : TM_XR;
            tmem_ld16(trow + col, xa);
            tmem_ld16(trow + col + 16, xb);
            tmem_wait_ld();
            float* X = reinterpret_cast<float*>(sm + OFF_X + half * SZ_X) + rb * NT * 8 + rqz;
#pragma unroll
            for (int n = 0; n < 16; ++n) X[n * 8] = __uint_as_float(xa[n]);
#pragma unroll
            for (int n = 16; n < NT; ++n) X[n * 8] = __uint_as_float(xb[n - 16]);
        }
        fence_before();
        __syncthreads();
        // transposed vertical stage and direct-stiffness summation:
        // y(k; n) = Bz(qz; k) Xr(qz; n) + Dz(qz; k) Xt(qz; n)
        for (int i = tid; i < nb * NT; i += kT5Threads) {
            const int b = i / NT, n = i - b * NT;
            const float4* pr = reinterpret_cast<const float4*>(sm + OFF_X + (b * NT + n) * 32);
            const float4* pt = reinterpret_cast<const float4*>(sm + OFF_X + SZ_X + (b * NT + n) * 32);
            const float4 r0 = pr[0], r1 = pr[1], t0 = pt[0], t1 = pt[1];
            const float xr[QZ] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z};
            const float xt[QZ] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z};
#pragma unroll
            for (int k = 0; k < NZ; ++k) {
                float s = 0.f;
#pragma unroll
                for (int qz = 0; qz < QZ; ++qz) s += sZ[qz * NZ + k] * xr[qz] + sZ[QZ * NZ + qz * NZ + k] * xt[qz];
                const int m = sMap[b * Np + k * NT + n];
                if (m >= 0 && m < N) atomicAdd(&y[m], s);
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    if (s_fail && tid == 0) {
        // a wait ran out: report it and give the copy or MMAs it waited for a second bounded wait
        // (the parity of a wait that ran out was not advanced)
        atomicExch(err, 1);
        t5_wait(barm, pm);
        t5_wait(bara, pa);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM_COLS) : "memory");
    }
}

}  // namespace

bool prism_t5_supported(int p) { return p == 6; }

cudaError_t launch_apply_prism_t5(const Level& L, const float* x, float* y, const int* skip, int* err, cudaStream_t s) {
    if (L.p != 6 || L.pz != 6 || L.dim != 3) return cudaErrorInvalidValue;
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        e = cudaFuncSetAttribute(k_apply_prism_t5, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    if (L.G16 == nullptr) return cudaErrorInvalidValue;
    const int passes = (L.E + EB - 1) / EB;
    const int grid = passes < 2 * kT5SMs ? passes : 2 * kT5SMs;
    if (grid < 1) return cudaSuccess;
    k_apply_prism_t5<<<grid, kT5Threads, SMEM, s>>>(L.E, (int)L.N, L.map,
                                                    reinterpret_cast<const __nv_bfloat16*>(L.G16), L.ref32.m, x, y,
                                                    skip, err);
    return cudaGetLastError();
}

}  // namespace sem
