// Prism apply of order 6 on the fifth-generation tensor cores (tcgen05) for the
// smoothing sweeps of the mixed-precision V-cycle (Eq. laplaceproblemdiscrete; the
// same contraction as apply_prism.cu and apply_prism_tc.cu).  A CTA pass takes 16
// elements; the two triangle contractions are TF32 tcgen05.mma with M = 128 rows,
// row r = 16 qz + b (vertical point qz = 0..7, the eighth zero, element b = 0..15),
// and FP32 accumulators in tensor memory:
//
//   forward   [Ur | Us](r; qt) = U(r; n) [Dr | Ds](n; qt),  Ut = W(r; n) Bt(n; qt)
//             (K = n: 28 -> 32, N = qt: 49 -> 64, three accumulators of 64 columns)
//   backward  Xr(r; n) = Vr(r; qt) Dr(qt; n) + Vs Ds,  Xt = Vt Bt
//             (K = qt: 49 -> 56, N = n: 28 -> 32, two accumulators of 32 columns)
//
// The kernel is warp-specialised and pipelined over passes, one CTA per SM:
//   * warps 0-3 and 4-7 are two compute groups that take alternate passes, each with
//     its own 256 TMEM columns and operand buffers, so one group's memory waits
//     overlap the other's arithmetic.  A group gathers x through the element map
//     and forms U = Bz x, W = Dz x (SIMT, written as K-major TF32 operands), one of
//     its threads issues the forward MMAs, the group applies the geometric factors
//     between tcgen05.ld and tcgen05.st (V overwrites the accumulators and is the A
//     operand of the backward MMAs straight from tensor memory), then stages Xr, Xt
//     through shared memory for the transposed vertical stage and the atomic
//     direct-stiffness summation;
//   * warp 8 streams each pass's element map (bulk copy, two buffers per group);
//   * warp 9 streams the BF16 geometric factors through a ring of six slots, one
//     8-column chunk of quadrature points per slot: the factors are stored per pass
//     of 16 elements chunk by chunk ([chunk][factor][qz][element][8 qt]), so the
//     next pass's chunk streams in as soon as this pass's has been used, and every
//     read of a slot is a conflict-free 16-byte load.  Consecutive uses of a slot belong
//     to different groups, so the producer publishes the use it issued to each slot and
//     a consumer begins its parity wait only once its use is issued (the use before has
//     then landed: a parity wait cannot tell it apart from the one two uses earlier).
// The operands sit in shared memory in the canonical no-swizzle K-major layout
// (8-row x 16-byte core matrices, K-adjacent ones 128 B apart, row groups K * 32 B
// apart); the row order r = 16 qz + b makes the gather's operand stores conflict-free.
// Every mbarrier wait is bounded (1 s); a wait that runs out sets the error flag, the
// other roles stop at their next wait or group barrier, every role gives the copies and
// MMAs it started a second bounded wait, and the tensor memory is freed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sem_internal.hpp"

namespace sem {

namespace {

constexpr int kT6Threads = 320;                   // 8 compute warps + 2 producer warps
constexpr unsigned long long kT6WaitNs = 1000000000ULL;

constexpr int NT = 28, NZ = 7, QT = 49, QZ = 7, Np = NT * NZ;
constexpr int EB = 16;                 // elements per pass
constexpr int KF = 32, NF = 64;        // forward K (n) and N (qt), padded
constexpr int KB = 56, NB = 32;        // backward K (qt) and N (n), padded
constexpr int NCH = 7;                 // factor chunks per pass: 6 x 8 quadrature points + 1
constexpr int NSLOT = 6;               // factor ring slots
constexpr uint32_t CH_BYTES = 6 * QZ * EB * 8 * 2;             // 10752
constexpr uint32_t CH_LAST = 6 * QZ * EB * 1 * 2;              // 1344
constexpr uint32_t PASS_G = 6 * CH_BYTES + CH_LAST;            // 65856 bytes of factors per pass
static_assert(PASS_G == (uint32_t)EB * 6 * QZ * QT * 2, "factor chunks cover the pass");
constexpr uint32_t MAP_BYTES = EB * Np * 4;                    // 12544
constexpr int XS = 8 * 16 + 16;        // X staging: floats per node n ([n][qz][b], padded)

// byte offset of entry (r, k) of a K-major operand with K columns
__host__ __device__ constexpr uint32_t opoff(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K * 32) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

constexpr uint32_t SZ_BF = NF * KF * 4;           // one forward reference operand (8192)
constexpr uint32_t SZ_BB = NB * KB * 4;           // one backward reference operand (7168)
constexpr uint32_t SZ_A = 128 * KF * 4;           // U or W (16384)
constexpr uint32_t OFF_BF = 0;                    // Dr, Ds, Bt as (qt, n)
constexpr uint32_t OFF_BB = OFF_BF + 3 * SZ_BF;   // Dr, Ds, Bt as (n, qt)
constexpr uint32_t OFF_UW = OFF_BB + 3 * SZ_BB;   // per group: U, W; after the forward MMAs Xr, Xt staging
constexpr uint32_t OFF_MAP = OFF_UW + 4 * SZ_A;   // [group][buffer] element maps
constexpr uint32_t OFF_G = OFF_MAP + 4 * MAP_BYTES;   // factor ring
constexpr uint32_t SMEM = OFF_G + NSLOT * CH_BYTES;
static_assert(SMEM <= 232448 - 512, "within one CTA's shared memory");
static_assert(OFF_UW % 1024 == 0 && OFF_MAP % 16 == 0 && OFF_G % 16 == 0 && CH_BYTES % 16 == 0, "alignment");
static_assert((NT * XS) * 4 <= SZ_A, "Xr / Xt staging fits in U / W");

// tensor memory columns of a group (base 0 or 256)
constexpr uint32_t TM_UR = 0, TM_US = 64, TM_UT = 128, TM_XR = 192, TM_XT = 224, TM_GROUP = 256;

// the vertical factors Bz, Dz ([QZ][NZ]) as a kernel argument: every FMA of the vertical
// stages reads its coefficient from the constant bank
struct Vert {
    float bz[QZ * NZ];
    float dz[QZ * NZ];
};

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

__device__ __forceinline__ unsigned long long t6_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for phase `parity` of mbarrier `bar`.  Returns false when another role has failed
// (honour_fail) or after kT6WaitNs, in which case the failure is recorded.
__device__ bool t6_wait(uint32_t bar, uint32_t parity, volatile int* fail, int* err, bool honour_fail = true) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = t6_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (honour_fail && *fail) return false;
        if (t6_ns() - t0 > kT6WaitNs) {
            *fail = 1;
            atomicExch(err, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void st_release_shared(int* p, int v) {
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire_shared(const int* p) {
    int v;
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}

// Wait until the producer has issued use `use` of a factor slot.  The slot's uses go to both
// groups, so a consumer has not seen the previous use complete; a parity wait begun before that
// use landed would take the completion of the use before it (same parity) for its own.  Once
// use `use` is issued, the previous use was consumed, hence landed, and the parity names `use`.
// Same bounds and failure recording as t6_wait.
__device__ bool t6_wait_issued(const int* issued, int use, volatile int* fail, int* err) {
    if (ld_acquire_shared(issued) >= use) return true;
    const unsigned long long t0 = t6_ns();
    for (;;) {
        if (ld_acquire_shared(issued) >= use) return true;
        if (*fail) return false;
        if (t6_ns() - t0 > kT6WaitNs) {
            *fail = 1;
            atomicExch(err, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// one thread: bulk-copy `bytes` (a multiple of 16) from global to shared, completing on `bar`
__device__ void t6_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

// D (tensor memory) = A (tensor memory) B^T (shared memory)
__device__ __forceinline__ void mma_tf32_ta(uint32_t tmem, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem),
        "r"(a), "l"(b), "r"(id), "r"(acc)
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

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// barrier of one compute group (128 threads; ids 1 and 2)
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }
// the same barrier returning whether any thread of the group passed v = true (uniform result)
__device__ __forceinline__ bool group_sync_any(int g, bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, 128, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + g)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

__global__ void __launch_bounds__(kT6Threads, 1)
    k_apply_prism_t6(int E, int N, int npass, const int* __restrict__ map, const __nv_bfloat16* __restrict__ G6,
                     const float* __restrict__ refm, const __grid_constant__ Vert vc, const float* __restrict__ x,
                     float* __restrict__ y, const int* __restrict__ skip, int* err) {
    if (skip != nullptr && *skip) return;
    extern __shared__ __align__(1024) unsigned char sm[];
    // [0..3] map full [g][buf], [4..7] map empty, [8..13] factor slot full, [14..19] slot empty,
    // [20, 21] MMA completion of group 0 / 1
    __shared__ __align__(8) unsigned long long mbar[22];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ int s_issued[NSLOT];    // use of each factor slot last issued by the producer
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t sbase = smem_u32(sm);
    const uint32_t mb0 = smem_u32(&mbar[0]);
    auto bar_mapf = [&](int g, int b) { return mb0 + 8u * (uint32_t)(2 * g + b); };
    auto bar_mape = [&](int g, int b) { return mb0 + 8u * (uint32_t)(4 + 2 * g + b); };
    auto bar_slotf = [&](int s) { return mb0 + 8u * (uint32_t)(8 + s); };
    auto bar_slote = [&](int s) { return mb0 + 8u * (uint32_t)(14 + s); };
    auto bar_mma = [&](int g) { return mb0 + 8u * (uint32_t)(20 + g); };
    volatile int* fail = &s_fail;

    // every pad entry of every operand must be zero
    for (uint32_t i = tid; i < OFF_MAP / 16; i += kT6Threads) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int i = tid; i < QT * NT; i += kT6Threads) {
        const int qt = i / NT, n = i - qt * NT;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            // reference blocks in refm: Bt, Dr, Ds as [QT][NT]; operands m = Dr, Ds, Bt
            const float v = __uint_as_float(to_tf32(refm[((m + 1) % 3) * QT * NT + i]));
            *reinterpret_cast<float*>(sm + OFF_BF + m * SZ_BF + opoff(qt, n, KF)) = v;
            *reinterpret_cast<float*>(sm + OFF_BB + m * SZ_BB + opoff(n, qt, KB)) = v;
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(2 * TM_GROUP)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        s_fail = 0;
        for (int i = 0; i < NSLOT; ++i) s_issued[i] = -1;
        for (int i = 0; i < 22; ++i) {
            const uint32_t cnt = (i >= 14 && i < 20) ? 4u : 1u;      // slot empty: one arrival per consumer warp
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb0 + 8u * i), "r"(cnt) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    const int first = blockIdx.x, step = gridDim.x;

    if (warp == 8) {
        // ------------------------------------------------------------ element-map producer
        if (lane == 0) {
            int issued[4] = {-1, -1, -1, -1};       // last use issued per (group, buffer)
            for (int k = 0, p = first; p < npass; ++k, p += step) {
                const int g = k & 1, b = (k >> 1) & 1, use = k >> 2;
                if (use > 0 && !t6_wait(bar_mape(g, b), (uint32_t)((use - 1) & 1), fail, err)) break;
                if (*fail) break;
                const int e0 = p * EB, nb = min(EB, E - e0);
                t6_copy(sbase + OFF_MAP + (uint32_t)(2 * g + b) * MAP_BYTES, map + (size_t)e0 * Np,
                        (uint32_t)nb * Np * 4u, bar_mapf(g, b));
                issued[2 * g + b] = use;
            }
            // every copy this warp started has landed before the CTA exits
            for (int i = 0; i < 4; ++i)
                if (issued[i] >= 0) t6_wait(bar_mapf(i >> 1, i & 1), (uint32_t)(issued[i] & 1), fail, err, false);
        }
    } else if (warp == 9) {
        // ------------------------------------------------------------ geometric-factor producer
        if (lane == 0) {
            int issued[NSLOT];
            for (int s = 0; s < NSLOT; ++s) issued[s] = -1;
            int j = 0;
            bool stop = false;
            for (int p = first; p < npass && !stop; p += step) {
                const char* src = reinterpret_cast<const char*>(G6) + (size_t)p * PASS_G;
                for (int c = 0; c < NCH; ++c, ++j) {
                    const int s = j % NSLOT, use = j / NSLOT;
                    if (use > 0 && !t6_wait(bar_slote(s), (uint32_t)((use - 1) & 1), fail, err)) { stop = true; break; }
                    if (*fail) { stop = true; break; }
                    st_release_shared(&s_issued[s], use);
                    t6_copy(sbase + OFF_G + (uint32_t)s * CH_BYTES, src + (size_t)c * CH_BYTES,
                            c < NCH - 1 ? CH_BYTES : CH_LAST, bar_slotf(s));
                    issued[s] = use;
                }
            }
            for (int s = 0; s < NSLOT; ++s)
                if (issued[s] >= 0) t6_wait(bar_slotf(s), (uint32_t)(issued[s] & 1), fail, err, false);
        }
    } else {
        // ------------------------------------------------------------ compute groups
        const int g = warp >> 2, q4 = warp & 3, gt = tid & 127;
        const uint32_t tg = tmem + (uint32_t)g * TM_GROUP;
        const uint32_t trow = tg + ((uint32_t)(32 * q4) << 16);
        unsigned char* U = sm + OFF_UW + (uint32_t)g * 2 * SZ_A;
        unsigned char* Wm = U + SZ_A;
        const uint32_t uaddr = sbase + OFF_UW + (uint32_t)g * 2 * SZ_A, waddr = uaddr + SZ_A;
        float* Xr = reinterpret_cast<float*>(U);
        float* Xt = reinterpret_cast<float*>(Wm);
        // this thread's accumulator row: r = 32 q4 + lane = 16 qz + b
        const int row = 32 * q4 + lane, rqz = row >> 4, rb = row & 15;
        const uint32_t idF = idesc(128, NF), idB = idesc(128, NB);
        int pend = -1;              // thread 0 of the group: parity of a commit not yet seen complete
        for (int k = g, p = first + g * step; p < npass; k += 2, p += 2 * step) {
            const int b = (k >> 1) & 1, use = k >> 2;
            const int e0 = p * EB, nb = min(EB, E - e0);
            const int* sMap = reinterpret_cast<const int*>(sm + OFF_MAP + (uint32_t)(2 * g + b) * MAP_BYTES);
            // pads of U and W (the last pass's X staging overwrote them): columns n = 28..31 of
            // every row and the rows of the eighth vertical point
            for (int i = gt; i < 2 * 128 + 2 * 16 * (NT / 4); i += 128) {
                uint32_t o;
                if (i < 256) {
                    o = (i < 128 ? 0u : SZ_A) + opoff(i & 127, NT, KF);
                } else {
                    const int jj = i - 256, mtx = jj / (16 * (NT / 4)), t = jj - mtx * (16 * (NT / 4));
                    o = (mtx ? SZ_A : 0u) + opoff(112 + t / (NT / 4), 4 * (t % (NT / 4)), KF);
                }
                *reinterpret_cast<uint4*>(U + o) = make_uint4(0, 0, 0, 0);
            }
            t6_wait(bar_mapf(g, b), (uint32_t)(use & 1), fail, err);
            // gather and vertical stage: U(qz, b; n) = Bz(qz; k) x(k; n), W = Dz x.  Warp task
            // wt = (bh, nh): lane -> element 8 bh + lane / 4, node 4 nh + lane % 4, so the 32 lanes
            // of every operand store fall on 32 distinct banks
            if (!*fail) {
                float xv[4][NZ];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int wt = q4 + 4 * t;
                    const int eb = (lane >> 2) + 8 * (wt / 7), n = 4 * (wt % 7) + (lane & 3);
#pragma unroll
                    for (int kk = 0; kk < NZ; ++kk) {
                        float v = 0.f;
                        if (wt < 14 && eb < nb) {
                            const int m = sMap[eb * Np + kk * NT + n];
                            if (m >= 0 && m < N) v = __ldg(x + m);   // Dirichlet ids (m < 0) act as zero
                        }
                        xv[t][kk] = v;
                    }
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int wt = q4 + 4 * t;
                    if (wt >= 14) continue;
                    const int eb = (lane >> 2) + 8 * (wt / 7), n = 4 * (wt % 7) + (lane & 3);
#pragma unroll
                    for (int qz = 0; qz < QZ; ++qz) {
                        float u = 0.f, w = 0.f;
#pragma unroll
                        for (int kk = 0; kk < NZ; ++kk) {
                            u = fmaf(vc.bz[qz * NZ + kk], xv[t][kk], u);
                            w = fmaf(vc.dz[qz * NZ + kk], xv[t][kk], w);
                        }
                        const uint32_t o = opoff(16 * qz + eb, n, KF);
                        *reinterpret_cast<uint32_t*>(U + o) = to_tf32(u);
                        *reinterpret_cast<uint32_t*>(Wm + o) = to_tf32(w);
                    }
                }
            }
            fence_async_smem();
            fence_before();
            if (group_sync_any(g, *fail)) break;
            if (gt == 0) {
                fence_after();
#pragma unroll
                for (int ks = 0; ks < KF / 8; ++ks) {
                    const uint64_t au = sdesc(uaddr + ks * 256, KF * 32);
                    const uint64_t aw = sdesc(waddr + ks * 256, KF * 32);
                    mma_tf32(tg + TM_UR, au, sdesc(sbase + OFF_BF + ks * 256, KF * 32), idF, ks);
                    mma_tf32(tg + TM_US, au, sdesc(sbase + OFF_BF + SZ_BF + ks * 256, KF * 32), idF, ks);
                    mma_tf32(tg + TM_UT, aw, sdesc(sbase + OFF_BF + 2 * SZ_BF + ks * 256, KF * 32), idF, ks);
                }
                mma_commit(bar_mma(g));
                pend = 0;
            }
            if (t6_wait(bar_mma(g), 0u, fail, err) && gt == 0) pend = -1;
            fence_after();
            // geometric factors, chunk by chunk: V over the accumulators
            const bool valid = rqz < QZ && rb < nb;
            for (int c = 0; c < NCH; ++c) {
                const int j = k * NCH + c, s = j % NSLOT;      // the producer's chunk sequence
                const int c0 = 8 * c;
                uint32_t ur[8], us[8], ut[8];
                tmem_ld8(trow + TM_UR + c0, ur);
                tmem_ld8(trow + TM_US + c0, us);
                tmem_ld8(trow + TM_UT + c0, ut);
                const bool ok = t6_wait_issued(&s_issued[s], j / NSLOT, fail, err) &&
                                t6_wait(bar_slotf(s), (uint32_t)((j / NSLOT) & 1), fail, err);
                const unsigned char* slot = sm + OFF_G + (uint32_t)s * CH_BYTES;
                float gf[6][8];
                if (c < NCH - 1) {
#pragma unroll
                    for (int f = 0; f < 6; ++f) {
                        uint4 v = make_uint4(0, 0, 0, 0);
                        if (ok && valid) v = *reinterpret_cast<const uint4*>(slot + ((f * QZ + rqz) * EB + rb) * 16);
                        gf[f][0] = bf16_lo(v.x); gf[f][1] = bf16_hi(v.x);
                        gf[f][2] = bf16_lo(v.y); gf[f][3] = bf16_hi(v.y);
                        gf[f][4] = bf16_lo(v.z); gf[f][5] = bf16_hi(v.z);
                        gf[f][6] = bf16_lo(v.w); gf[f][7] = bf16_hi(v.w);
                    }
                } else {
#pragma unroll
                    for (int f = 0; f < 6; ++f) {
                        uint32_t v = 0;
                        if (ok && valid) v = *reinterpret_cast<const unsigned short*>(slot + ((f * QZ + rqz) * EB + rb) * 2);
                        gf[f][0] = bf16_lo(v);
#pragma unroll
                        for (int h = 1; h < 8; ++h) gf[f][h] = 0.f;     // quadrature columns 49..55 are padding
                    }
                }
                // the slot may be refilled once every lane has read it (not after a failed wait: its
                // copy may still be in flight)
                if (__all_sync(0xffffffffu, ok) && lane == 0) mbar_arrive(bar_slote(s));
                tmem_wait_ld();
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    const float a = __uint_as_float(ur[h]), bb = __uint_as_float(us[h]), t = __uint_as_float(ut[h]);
                    const float vr = gf[0][h] * a + gf[1][h] * bb + gf[2][h] * t;
                    const float vs = gf[1][h] * a + gf[3][h] * bb + gf[4][h] * t;
                    const float vt = gf[2][h] * a + gf[4][h] * bb + gf[5][h] * t;
                    ur[h] = to_tf32(vr);
                    us[h] = to_tf32(vs);
                    ut[h] = to_tf32(vt);
                }
                tmem_st8(trow + TM_UR + c0, ur);
                tmem_st8(trow + TM_US + c0, us);
                tmem_st8(trow + TM_UT + c0, ut);
            }
            tmem_wait_st();
            fence_before();
            if (group_sync_any(g, *fail)) break;
            if (gt == 0) {
                fence_after();
#pragma unroll
                for (int ks = 0; ks < KB / 8; ++ks) {
                    const uint32_t o = ks * 256;
                    mma_tf32_ta(tg + TM_XR, tg + TM_UR + 8 * ks, sdesc(sbase + OFF_BB + o, KB * 32), idB, ks);
                    mma_tf32_ta(tg + TM_XR, tg + TM_US + 8 * ks, sdesc(sbase + OFF_BB + SZ_BB + o, KB * 32), idB, 1);
                    mma_tf32_ta(tg + TM_XT, tg + TM_UT + 8 * ks, sdesc(sbase + OFF_BB + 2 * SZ_BB + o, KB * 32), idB, ks);
                }
                mma_commit(bar_mma(g));
                pend = 1;
            }
            if (t6_wait(bar_mma(g), 1u, fail, err) && gt == 0) pend = -1;
            fence_after();
            {   // Xr, Xt of this row into the staging areas [n][qz][b] (row stride XS per node)
                uint32_t xa[16], xb[16], ta[16], tb[16];
                tmem_ld16(trow + TM_XR, xa);
                tmem_ld16(trow + TM_XR + 16, xb);
                tmem_ld16(trow + TM_XT, ta);
                tmem_ld16(trow + TM_XT + 16, tb);
                tmem_wait_ld();
                if (rqz < QZ) {
                    float* pr = Xr + rqz * 16 + rb;
                    float* pt = Xt + rqz * 16 + rb;
#pragma unroll
                    for (int n = 0; n < 16; ++n) {
                        pr[n * XS] = __uint_as_float(xa[n]);
                        pt[n * XS] = __uint_as_float(ta[n]);
                    }
#pragma unroll
                    for (int n = 16; n < NT; ++n) {
                        pr[n * XS] = __uint_as_float(xb[n - 16]);
                        pt[n * XS] = __uint_as_float(tb[n - 16]);
                    }
                }
            }
            fence_before();
            group_sync(g);
            // transposed vertical stage and direct-stiffness summation:
            // y(k; n) = Bz(qz; k) Xr(qz; n) + Dz(qz; k) Xt(qz; n).  Warp task nt: lane -> element
            // lane % 16, node 2 nt + lane / 16
            if (!*fail) {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int nt = q4 + 4 * t;
                    if (nt >= 14) continue;
                    const int eb = lane & 15, n = 2 * nt + (lane >> 4);
                    float xr[QZ], xt[QZ];
#pragma unroll
                    for (int qz = 0; qz < QZ; ++qz) {
                        xr[qz] = Xr[n * XS + qz * 16 + eb];
                        xt[qz] = Xt[n * XS + qz * 16 + eb];
                    }
                    if (eb < nb) {
#pragma unroll
                        for (int kk = 0; kk < NZ; ++kk) {
                            float s = 0.f;
#pragma unroll
                            for (int qz = 0; qz < QZ; ++qz) {
                                s = fmaf(vc.bz[qz * NZ + kk], xr[qz], s);
                                s = fmaf(vc.dz[qz * NZ + kk], xt[qz], s);
                            }
                            const int m = sMap[eb * Np + kk * NT + n];
                            if (m >= 0 && m < N) atomicAdd(&y[m], s);
                        }
                    }
                }
            }
            if (group_sync_any(g, *fail)) break;
            // this pass's map buffer may be refilled
            if (gt == 0) mbar_arrive(bar_mape(g, b));
        }
        // MMAs this group started and did not see complete get a second bounded wait
        if (gt == 0 && pend >= 0) t6_wait(bar_mma(g), (uint32_t)pend, fail, err, false);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TM_GROUP) : "memory");
    }
}

// The order-6 factors in the kernel's layout: per pass of 16 elements, chunk c of 8
// quadrature points (the seventh chunk holds the 49th point) as [factor][qz][element][8 qt]
// (BF16; elements past E are zero).
__global__ void k_factors_t6(int E, int npass, const float* __restrict__ G32, __nv_bfloat16* __restrict__ out) {
    constexpr int PER = (int)(PASS_G / 2);            // BF16 entries per pass
    constexpr int CH = (int)(CH_BYTES / 2);
    const long long n = (long long)npass * PER;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i / PER);
        const int r = (int)(i - (long long)p * PER);
        int c, rr, wc;
        if (r < 6 * CH) { c = r / CH; rr = r - c * CH; wc = 8; }
        else { c = 6; rr = r - 6 * CH; wc = 1; }
        const int w = rr % wc;
        int t = rr / wc;
        const int e = t % EB;
        t /= EB;
        const int qz = t % QZ, f = t / QZ;
        const int ea = p * EB + e, qt = 8 * c + w;
        float v = 0.f;
        if (ea < E) v = G32[((size_t)ea * 6 + f) * (QZ * QT) + qz * QT + qt];
        out[i] = __float2bfloat16_rn(v);
    }
}

}  // namespace

bool prism_t5_supported(int p) { return p == 6; }

cudaError_t build_g16_t6(Level& L, cudaStream_t s) {
    if (!(L.dim == 3 && L.p == 6 && L.pz == 6) || L.G32 == nullptr) return cudaSuccess;
    const int npass = (L.E + EB - 1) / EB;
    cudaError_t e = cudaSuccess;
    if (L.G16T == nullptr) {
        void* p = nullptr;
        e = cudaMalloc(&p, (size_t)npass * PASS_G);
        if (e != cudaSuccess) return e;
        L.G16T = static_cast<unsigned short*>(p);
    }
    const long long n = (long long)npass * (PASS_G / 2);
    const long long blocks = (n + 255) / 256;
    k_factors_t6<<<(int)(blocks < 8192 ? (blocks > 0 ? blocks : 1) : 8192), 256, 0, s>>>(
        L.E, npass, L.G32, static_cast<__nv_bfloat16*>(static_cast<void*>(L.G16T)));
    return cudaGetLastError();
}

cudaError_t launch_apply_prism_t5(const Level& L, const float* x, float* y, const int* skip, int* err, cudaStream_t s) {
    if (L.p != 6 || L.pz != 6 || L.dim != 3 || L.G16T == nullptr) return cudaErrorInvalidValue;
    static bool configured[64] = {};
    static int sms[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        e = cudaFuncSetAttribute(k_apply_prism_t6, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    Vert vc;
    for (int i = 0; i < QZ * NZ; ++i) {
        vc.bz[i] = (float)L.ref.Bz[i];
        vc.dz[i] = (float)L.ref.Dz[i];
    }
    const int npass = (L.E + EB - 1) / EB;
    const int grid = npass < sms[dev] ? npass : sms[dev];
    if (grid < 1) return cudaSuccess;
    k_apply_prism_t6<<<grid, kT6Threads, SMEM, s>>>(L.E, (int)L.N, npass, L.map,
                                                   reinterpret_cast<const __nv_bfloat16*>(L.G16T), L.ref32.m, vc, x,
                                                   y, skip, err);
    return cudaGetLastError();
}

}  // namespace sem
