// Tensor-core prism apply for the smoothing sweeps of the mixed-precision V-cycle
// (Eq. laplaceproblemdiscrete, same contraction as apply_prism.cu).  Both triangle
// contractions run as TF32 warp MMAs (m16n8k8) with FP32 accumulation, with the
// element data as the A operand -- 16 rows = two elements x 8 vertical points -- and
// the reference matrices as the B operand:
//
//   forward   [Ur Us Ut](e,qz; qt) = U(e,qz; n) [Dr Ds](n; qt),  W(e,qz; n) Bt(n; qt)
//   backward  Xr(e,qz; n) = Vr(e,qz; qt) Dr(qt; n) + Vs Ds,  Xt = Vt Bt
//
// The geometric factors come from a BF16 copy of G (half the bytes of the FP32
// factors), staged per CTA pass into shared memory by bulk asynchronous copies on an
// mbarrier; the pass's element map arrives the same way into a double buffer.  The
// vertical stages, the gather and the direct-stiffness summation stay on the SIMT
// pipes.  Shared memory stays below half an SM so that two CTAs share each SM and one
// computes while the other waits.  Rounding the operands to TF32 and the factors to
// BF16 makes the result differ from the FP32 apply by a few 1e-3 relative: the kernel
// serves the Chebyshev sweeps only, where the operator need not be exact.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sem_internal.hpp"

namespace sem {

namespace {

constexpr int kTcSMs = 152;
constexpr int kTcWarps = 8;
constexpr int kTcThreads = 32 * kTcWarps;
constexpr unsigned long long kTcWaitNs = 1000000000ULL;   // 1 s bound on a copy wait

// elements per CTA pass by order: even, and every pass's map and factor block starts
// on a 16-byte boundary (checked below)
__host__ __device__ constexpr int tc_pass_elems(int P) {
    return P == 6 ? 4 : (P == 5 ? 8 : (P == 4 ? 12 : 16));
}

template <int P>
struct TcTile {
    static constexpr int NT = (P + 1) * (P + 2) / 2, NZ = P + 1, QT = (P + 1) * (P + 1), QZ = P + 1;
    static constexpr int Np = NT * NZ, Nq = QT * QZ;
    static_assert(QZ <= 8 && NZ <= 8, "an element's vertical points / nodes fill 8 MMA rows");
    static constexpr int NTF = (QT + 7) / 8;       // forward n-tiles (qt)
    static constexpr int KSF = (NT + 7) / 8;       // forward k-steps (n)
    static constexpr int NTB = KSF;                // backward n-tiles (n)
    static constexpr int KSB = NTF;                // backward k-steps (qt)
    // row strides (words) of ldmatrix operands: stride/4 odd puts the 8 rows of a
    // fragment on distinct bank quads
    static constexpr int LDF = KSF * 8 + 4;        // reference matrices as (qt, n)
    static constexpr int LDB = KSB * 8 + 4;        // reference matrices as (n, qt)
    static constexpr int LDU = KSF * 8 + 4;        // U, W as (qz, n)
    static constexpr int LDV = KSB * 8 + 4;        // Vr, Vs, Vt as (qz, qt)
    static constexpr int LDX = 20;                 // [Xr | Xt] as (n, 16): scalar fragment loads, 20/4 odd
    static constexpr int EB = tc_pass_elems(P);
    static constexpr int NPAIR = EB / 2;
    static constexpr int NGF = (NTF + 1) / 2;      // forward warp tasks per pair (2 qt tiles each)
    static constexpr int NGB = (NTB + 1) / 2;      // backward warp tasks per pair (2 node tiles each)
    // forward tasks fill the warps exactly: every warp keeps one task, so the B fragments of
    // its two qt tiles stay in registers for the whole launch (P = 2, 3, 6)
    static constexpr bool FSTAT = NPAIR * NGF == kTcWarps;
    // BF16 factors as [6][QZ][QTP], rows padded to even length so a lane's two points
    // (qt, qt + 1), qt even, are one aligned 32-bit word
    static constexpr int QTP = (QT + 1) / 2 * 2;
    static constexpr int GE = 6 * QZ * QTP;        // BF16 entries per element
    static_assert(EB % 2 == 0, "elements pair up into MMA rows");
    static_assert((EB * Np * 4) % 16 == 0, "map blocks of a pass start on 16-byte boundaries");
    static_assert((EB * GE * 2) % 16 == 0, "factor blocks of a pass start on 16-byte boundaries");
    __host__ __device__ static constexpr int r4(int v) { return (v + 3) / 4 * 4; }
    // shared-memory regions in 4-byte words, each a multiple of 4 words (16 bytes)
    static constexpr int GSZ = r4((EB * GE + 1) / 2);         // BF16 factors of a pass
    static constexpr int BF = 3 * NTF * 8 * LDF;              // Dr, Ds, Bt as [qt][n]
    static constexpr int BB = 3 * NTB * 8 * LDB;              // Dr, Ds, Bt as [n][qt]
    static constexpr int MAP = r4(EB * Np);                    // one map buffer (ints)
    // vertical-stage MMA tasks (element, node tile) of a pass per warp: each lane keeps the
    // x values of its B fragments for the next pass in registers
    static constexpr int TPW = (EB * NTB + kTcWarps - 1) / kTcWarps;
    // per element: region R1 holds U, W [qz][n] until the forward contraction, then
    // [Xr | Xt] [n][LDX]; V holds Vr, Vs, Vt [qz][qt]
    static constexpr int UW = 8 * LDU;
    static constexpr int XX = NTB * 8 * LDX;
    static constexpr int R1 = (2 * UW > XX) ? 2 * UW : XX;
    static constexpr int VS = 8 * LDV;
    static constexpr int WORK = R1 + 3 * VS;
    static constexpr int TOTAL = GSZ + BF + BB + 2 * MAP + EB * WORK;
    static constexpr size_t SMEM = 4 * (size_t)TOTAL;
    static_assert(SMEM + 1024 + 256 <= 233472 / 2, "two CTAs per SM");
};

__device__ __forceinline__ uint32_t to_tf32(float f) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
    return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&a)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& b0, uint32_t& b1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(b0), "=r"(b1) : "r"(addr));
}

__device__ __forceinline__ unsigned long long tc_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase `parity` to complete; false after kTcWaitNs.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = tc_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (tc_ns() - t0 > kTcWaitNs) return false;
    }
}

// One thread: bulk-copy `bytes` (rounded up to 16; the source allocations carry 64
// bytes of padding) from global `src` to shared `dst`, in pieces of at most 16 KB,
// completing on mbarrier `bar`.
__device__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
    bytes = (bytes + 15u) & ~15u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    const uint32_t d = smem_u32(dst);
    const char* s = reinterpret_cast<const char*>(src);
    for (uint32_t off = 0; off < bytes; off += 16384u) {
        const uint32_t n = (bytes - off < 16384u) ? (bytes - off) : 16384u;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d + off),
            "l"(s + off), "r"(n), "r"(bar)
            : "memory");
    }
}

template <int P>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_apply_prism_tc(int E, int N, const int* __restrict__ map, const __nv_bfloat16* __restrict__ G16,
                     const float* __restrict__ refm, const float* __restrict__ x, float* __restrict__ y,
                     const int* __restrict__ skip, int* err) {
    using D = TcTile<P>;
    constexpr int NT = D::NT, NZ = D::NZ, QT = D::QT, QZ = D::QZ, Np = D::Np, EB = D::EB;
    if (skip != nullptr && *skip) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long mbar[2];   // [0] geometric factors, [1] element map
    __shared__ int s_fail;
    float* sm = reinterpret_cast<float*>(smem_raw);
    __nv_bfloat16* sG = reinterpret_cast<__nv_bfloat16*>(sm);
    float* sBF = sm + D::GSZ;                  // [3][NTF*8][LDF]: Dr, Ds, Bt as (qt, n), TF32 bits
    float* sBB = sBF + D::BF;                  // [3][NTB*8][LDB]: Dr, Ds, Bt as (n, qt)
    int* sMap0 = reinterpret_cast<int*>(sBB + D::BB);   // two map buffers of D::MAP ints
    float* work = sBB + D::BB + 2 * D::MAP;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    // ldmatrix lane addressing: A (16 x 8 tile of two elements' 8 rows): row lane&7 of
    // element (lane>>3)&1 at column offset (lane>>4)*4; B (8 x 8 tile): row lane&7 at
    // column offset ((lane>>3)&1)*4
    const int lrow = lane & 7, lsel = (lane >> 3) & 1, lcolA = (lane >> 4) * 4, lcolB = lsel * 4;

    // every pad entry must be finite (and zero where it meets a non-zero operand)
    for (int i = tid; i < D::TOTAL; i += kTcThreads) sm[i] = 0.f;
    __syncthreads();
    for (int i = tid; i < QT * NT; i += kTcThreads) {
        const int qt = i / NT, n = i - qt * NT;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            // reference blocks in refm: Bt, Dr, Ds as [QT][NT]; here Dr, Ds, Bt
            const float v = refm[((m + 1) % 3) * QT * NT + i];
            sBF[(m * D::NTF * 8 + qt) * D::LDF + n] = __uint_as_float(to_tf32(v));
            sBB[(m * D::NTB * 8 + n) * D::LDB + qt] = __uint_as_float(to_tf32(v));
        }
    }
    // constant A operands of the vertical stages, in registers.  Forward: rows 0-7 Bz(qz, k),
    // rows 8-15 Dz(qz, k).  Transposed: k-step 0 Bz(qz, k) as (k, qz), k-step 1 Dz(qz, k) as
    // (k, qz), rows 8-15 zero.  refm ends with [Bz | Dz] as [QZ][NZ].
    const float* rBz = refm + 6 * QT * NT;
    const float* rDz = rBz + QZ * NZ;
    auto zq = [&](const float* M, int qz, int k) -> uint32_t {
        return (qz < QZ && k < NZ) ? to_tf32(M[qz * NZ + k]) : 0u;
    };
    const uint32_t av[4] = {zq(rBz, g, t), zq(rDz, g, t), zq(rBz, g, t + 4), zq(rDz, g, t + 4)};
    const uint32_t at0[4] = {zq(rBz, t, g), 0u, zq(rBz, t + 4, g), 0u};
    const uint32_t at1[4] = {zq(rDz, t, g), 0u, zq(rDz, t + 4, g), 0u};
    const uint32_t barg = smem_u32(&mbar[0]), barm = smem_u32(&mbar[1]);
    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barg) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barm) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // register-resident B fragments of the forward contraction (FSTAT): [tile][k-step][Dr, Ds, Bt pairs]
    uint32_t bst[2][D::KSF][6];
    if constexpr (D::FSTAT) {
        const int j0 = 2 * (warp % D::NGF);
#pragma unroll
        for (int jj = 0; jj < 2; ++jj)
#pragma unroll
            for (int ks = 0; ks < D::KSF; ++ks) {
                if (j0 + jj < D::NTF) {
                    const float* Bb = sBF + ((j0 + jj) * 8 + lrow) * D::LDF + lcolB + ks * 8;
                    ldsm_x2(smem_u32(Bb), bst[jj][ks][0], bst[jj][ks][1]);
                    ldsm_x2(smem_u32(Bb + D::NTF * 8 * D::LDF), bst[jj][ks][2], bst[jj][ks][3]);
                    ldsm_x2(smem_u32(Bb + 2 * D::NTF * 8 * D::LDF), bst[jj][ks][4], bst[jj][ks][5]);
                } else {
#pragma unroll
                    for (int r = 0; r < 6; ++r) bst[jj][ks][r] = 0u;
                }
            }
    }
    uint32_t pg = 0, pm = 0;
    int buf = 0;
    const int stride = gridDim.x * EB;
    // B fragments of the vertical-stage MMA for a pass: lane (g, t) of a warp's task
    // (element b, node tile jj) holds x(k = t, n) and x(k = t + 4, n), n = 8 jj + g
    uint32_t xf[D::TPW][2];
    auto prefetch_x = [&](const int* mp, int nbx) {
#pragma unroll
        for (int q = 0; q < D::TPW; ++q) {
            const int task = warp + q * kTcWarps;
            const int b = task / D::NTB, n = (task - b * D::NTB) * 8 + g;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = t + 4 * h;
                float v = 0.f;
                if (b < nbx && n < NT && k < NZ) {
                    const int m = mp[b * Np + k * NT + n];
                    if (m >= 0 && m < N) v = x[m];      // every node id of a valid map is < N
                }
                xf[q][h] = __float_as_uint(v);        // raw bits: nothing waits on the load here
            }
        }
    };
    // Each mbarrier carries one copy at a time, and it is re-armed only after a barrier that
    // every thread reaches after its wait: a phase never completes twice before all threads
    // have observed the first completion (parity waits would then misread it).
    if (tid == 0 && blockIdx.x * EB < E) {
        const int e = blockIdx.x * EB, nb0 = min(EB, E - e);
        bulk_copy(sMap0, map + (size_t)e * Np, (uint32_t)nb0 * Np * 4u, barm);
        bulk_copy(sG, G16 + (size_t)e * D::GE, (uint32_t)nb0 * D::GE * 2u, barg);
    }
    if (blockIdx.x * EB < E) {
        // a map that did not arrive is never read: its indices would be arbitrary
        const bool ok = mbar_wait(barm, pm);
        if (!ok) s_fail = 1;
        pm ^= 1u;
        prefetch_x(sMap0, ok ? min(EB, E - blockIdx.x * EB) : 0);
    }
    __syncthreads();
    if (tid == 0 && !s_fail) {
        const int e1 = blockIdx.x * EB + stride;
        if (e1 < E) bulk_copy(sMap0 + D::MAP, map + (size_t)e1 * Np, (uint32_t)min(EB, E - e1) * Np * 4u, barm);
    }

    for (int e0 = blockIdx.x * EB; e0 < E; e0 += stride) {
        const int nb = min(EB, E - e0);
        const int en = e0 + stride;
        const int* sMap = sMap0 + buf * D::MAP;
        // vertical stage on the tensor cores from the prefetched x: [U; W](qz; n) =
        // [Bz; Dz](qz; k) X(k; n)
#pragma unroll
        for (int q = 0; q < D::TPW; ++q) {
            const int task = warp + q * kTcWarps;
            const int b = task / D::NTB, j = task - b * D::NTB;
            if (b >= nb) continue;
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma_tf32(c, av, to_tf32(__uint_as_float(xf[q][0])), to_tf32(__uint_as_float(xf[q][1])));
            float* U = work + b * D::WORK + g * D::LDU + j * 8 + 2 * t;
            float* W = U + D::UW;
            U[0] = __uint_as_float(to_tf32(c[0]));
            U[1] = __uint_as_float(to_tf32(c[1]));
            W[0] = __uint_as_float(to_tf32(c[2]));
            W[1] = __uint_as_float(to_tf32(c[3]));
        }
        // this pass's geometric factors
        if (!mbar_wait(barg, pg)) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        pg ^= 1u;
        // forward contractions and the geometric factors: warp task = (element pair, two qt
        // tiles); each A fragment serves both tiles
        for (int task = warp; task < D::NPAIR * D::NGF; task += kTcWarps) {
            const int pr = task / D::NGF, j0 = 2 * (task - pr * D::NGF);
            const bool two = j0 + 1 < D::NTF;
            const float* Ua = work + (2 * pr + lsel) * D::WORK + lrow * D::LDU + lcolA;
            float cr[2][4], cs[2][4], ct[2][4];
#pragma unroll
            for (int jj = 0; jj < 2; ++jj)
#pragma unroll
                for (int r = 0; r < 4; ++r) cr[jj][r] = cs[jj][r] = ct[jj][r] = 0.f;
#pragma unroll
            for (int ks = 0; ks < D::KSF; ++ks) {
                uint32_t au[4], aw[4];
                ldsm_x4(smem_u32(Ua + ks * 8), au);
                ldsm_x4(smem_u32(Ua + D::UW + ks * 8), aw);
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    if (jj == 1 && !two) break;
                    uint32_t br0, br1, bs0, bs1, bt0, bt1;
                    if constexpr (D::FSTAT) {
                        br0 = bst[jj][ks][0]; br1 = bst[jj][ks][1];
                        bs0 = bst[jj][ks][2]; bs1 = bst[jj][ks][3];
                        bt0 = bst[jj][ks][4]; bt1 = bst[jj][ks][5];
                    } else {
                        const float* Bb = sBF + ((j0 + jj) * 8 + lrow) * D::LDF + lcolB + ks * 8;
                        ldsm_x2(smem_u32(Bb), br0, br1);
                        ldsm_x2(smem_u32(Bb + D::NTF * 8 * D::LDF), bs0, bs1);
                        ldsm_x2(smem_u32(Bb + 2 * D::NTF * 8 * D::LDF), bt0, bt1);
                    }
                    mma_tf32(cr[jj], au, br0, br1);
                    mma_tf32(cs[jj], au, bs0, bs1);
                    mma_tf32(ct[jj], aw, bt0, bt1);
                }
            }
            // lane (g, t) holds points (qz = g, qt0 + h), qt0 = 8 (j0 + jj) + 2 t, of both
            // elements of the pair: fragment entries 2 e + h
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                if (jj == 1 && !two) break;
                const int qz = g, qt0 = (j0 + jj) * 8 + 2 * t;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int b = 2 * pr + e;
                    if (b >= nb) continue;
                    float vr[2] = {0.f, 0.f}, vs[2] = {0.f, 0.f}, vt[2] = {0.f, 0.f};
                    if (qz < QZ && qt0 < QT) {
                        const __nv_bfloat162* Gp = reinterpret_cast<const __nv_bfloat162*>(
                            sG + (size_t)b * D::GE + qz * D::QTP + qt0);
                        constexpr int FS = QZ * D::QTP / 2;      // factor stride in BF16 pairs
                        const float2 g0 = __bfloat1622float2(Gp[0]), g1 = __bfloat1622float2(Gp[FS]);
                        const float2 g2 = __bfloat1622float2(Gp[2 * FS]), g3 = __bfloat1622float2(Gp[3 * FS]);
                        const float2 g4 = __bfloat1622float2(Gp[4 * FS]), g5 = __bfloat1622float2(Gp[5 * FS]);
                        const float gg[6][2] = {{g0.x, g0.y}, {g1.x, g1.y}, {g2.x, g2.y},
                                                {g3.x, g3.y}, {g4.x, g4.y}, {g5.x, g5.y}};
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (qt0 + h >= QT) continue;
                            const float ur = cr[jj][2 * e + h], us = cs[jj][2 * e + h], ut = ct[jj][2 * e + h];
                            vr[h] = gg[0][h] * ur + gg[1][h] * us + gg[2][h] * ut;
                            vs[h] = gg[1][h] * ur + gg[3][h] * us + gg[4][h] * ut;
                            vt[h] = gg[2][h] * ur + gg[4][h] * us + gg[5][h] * ut;
                        }
                    }
                    float* V = work + b * D::WORK + D::R1 + qz * D::LDV + qt0;
                    *reinterpret_cast<float2*>(V) =
                        make_float2(__uint_as_float(to_tf32(vr[0])), __uint_as_float(to_tf32(vr[1])));
                    *reinterpret_cast<float2*>(V + D::VS) =
                        make_float2(__uint_as_float(to_tf32(vs[0])), __uint_as_float(to_tf32(vs[1])));
                    *reinterpret_cast<float2*>(V + 2 * D::VS) =
                        make_float2(__uint_as_float(to_tf32(vt[0])), __uint_as_float(to_tf32(vt[1])));
                }
            }
        }
        __syncthreads();
        // the factors are consumed: stream in the next pass's while this one finishes, and
        // start the next pass's gather (its map arrived during this pass)
        if (tid == 0 && en < E)
            bulk_copy(sG, G16 + (size_t)en * D::GE, (uint32_t)min(EB, E - en) * D::GE * 2u, barg);
        if (en < E) {
            const bool ok = mbar_wait(barm, pm);
            if (!ok) s_fail = 1;
            pm ^= 1u;
            prefetch_x(sMap0 + (buf ^ 1) * D::MAP, ok ? min(EB, E - en) : 0);
        }
        // backward contractions: warp task = (element pair, two node tiles); [Xr | Xt] over R1
        for (int task = warp; task < D::NPAIR * D::NGB; task += kTcWarps) {
            const int pr = task / D::NGB, j0 = 2 * (task - pr * D::NGB);
            const bool two = j0 + 1 < D::NTB;
            const float* Va = work + (2 * pr + lsel) * D::WORK + D::R1 + lrow * D::LDV + lcolA;
            float xr[2][4], xt[2][4];
#pragma unroll
            for (int jj = 0; jj < 2; ++jj)
#pragma unroll
                for (int r = 0; r < 4; ++r) xr[jj][r] = xt[jj][r] = 0.f;
#pragma unroll
            for (int ks = 0; ks < D::KSB; ++ks) {
                uint32_t a0[4], a1[4], a2[4];
                ldsm_x4(smem_u32(Va + ks * 8), a0);
                ldsm_x4(smem_u32(Va + D::VS + ks * 8), a1);
                ldsm_x4(smem_u32(Va + 2 * D::VS + ks * 8), a2);
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    if (jj == 1 && !two) break;
                    const float* Bb = sBB + ((j0 + jj) * 8 + lrow) * D::LDB + lcolB + ks * 8;
                    uint32_t b00, b01, b10, b11, b20, b21;
                    ldsm_x2(smem_u32(Bb), b00, b01);
                    ldsm_x2(smem_u32(Bb + D::NTB * 8 * D::LDB), b10, b11);
                    ldsm_x2(smem_u32(Bb + 2 * D::NTB * 8 * D::LDB), b20, b21);
                    mma_tf32(xr[jj], a0, b00, b01);
                    mma_tf32(xr[jj], a1, b10, b11);
                    mma_tf32(xt[jj], a2, b20, b21);
                }
            }
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                if (jj == 1 && !two) break;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int b = 2 * pr + (r >> 1);
                    if (b >= nb) continue;
                    const int n = (j0 + jj) * 8 + 2 * t + (r & 1);
                    float* X = work + b * D::WORK + n * D::LDX + g;
                    X[0] = __uint_as_float(to_tf32(xr[jj][r]));
                    X[8] = __uint_as_float(to_tf32(xt[jj][r]));
                }
            }
        }
        __syncthreads();
        // transposed vertical stage on the tensor cores and direct-stiffness summation:
        // y(k; n) = Bz^T(k; qz) Xr(qz; n) + Dz^T(k; qz) Xt(qz; n), rows k < NZ of the tile
        for (int task = warp; task < nb * D::NTB; task += kTcWarps) {
            const int b = task / D::NTB, j = task - b * D::NTB;
            const float* X = work + b * D::WORK + (j * 8 + g) * D::LDX + t;
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma_tf32(c, at0, __float_as_uint(X[0]), __float_as_uint(X[4]));
            mma_tf32(c, at1, __float_as_uint(X[8]), __float_as_uint(X[12]));
            const int k = g, n = j * 8 + 2 * t;
            if (k < NZ) {
                const int* mp = sMap + b * Np + k * NT;
                if (n < NT && mp[n] >= 0 && mp[n] < N) atomicAdd(&y[mp[n]], c[0]);
                if (n + 1 < NT && mp[n + 1] >= 0 && mp[n + 1] < N) atomicAdd(&y[mp[n + 1]], c[1]);
            }
        }
        __syncthreads();
        if (s_fail) break;          // a map wait ran out (uniform after the barrier)
        // the map two passes ahead into the buffer this pass has finished with
        if (tid == 0 && en + stride < E)
            bulk_copy(sMap0 + buf * D::MAP, map + (size_t)(en + stride) * Np,
                      (uint32_t)min(EB, E - en - stride) * Np * 4u, barm);
        buf ^= 1;
    }
    if (s_fail) {
        // a copy did not complete in time: report it, give the copies in flight a second
        // bounded wait, return
        if (tid == 0) {
            atomicExch(err, 1);
            mbar_wait(barm, pm);
            mbar_wait(barg, pg);
        }
        __syncthreads();
    }
}

template <int P>
cudaError_t apply_tc_impl(const Level& L, const float* x, float* y, const int* skip, int* err, cudaStream_t s) {
    using D = TcTile<P>;
    static bool configured[64] = {};          // the attribute is per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        e = cudaFuncSetAttribute(k_apply_prism_tc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D::SMEM);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    if (L.G16 == nullptr) return cudaErrorInvalidValue;
    const int passes = (L.E + D::EB - 1) / D::EB;
    const int grid = passes < 2 * kTcSMs ? passes : 2 * kTcSMs;
    if (grid < 1) return cudaSuccess;
    k_apply_prism_tc<P><<<grid, kTcThreads, D::SMEM, s>>>(
        L.E, (int)L.N, L.map, reinterpret_cast<const __nv_bfloat16*>(L.G16), L.ref32.m, x, y, skip, err);
    return cudaGetLastError();
}


}  // namespace

cudaError_t launch_apply_prism_tc(const Level& L, const float* x, float* y, const int* skip, int* err,
                                  cudaStream_t s) {
    switch (L.p) {
        case 2: return apply_tc_impl<2>(L, x, y, skip, err, s);
        case 3: return apply_tc_impl<3>(L, x, y, skip, err, s);
        case 4: return apply_tc_impl<4>(L, x, y, skip, err, s);
        case 5: return apply_tc_impl<5>(L, x, y, skip, err, s);
        case 6: return apply_tc_impl<6>(L, x, y, skip, err, s);
        default: return cudaErrorInvalidValue;
    }
}

bool prism_tc_supported(int p) { return p >= 2 && p <= 6; }

// BF16 copy of a prism level's FP32 geometric factors for the tensor-core apply, as
// [E][6][QZ][QTP] with QTP = QT rounded up to even (pads zero), plus 64 bytes of padding
// for its 16-byte-rounded bulk copies.
__global__ void k_to_bf16_padded(long long E, int QT, int QZ, int QTP, const float* __restrict__ a,
                                 __nv_bfloat16* __restrict__ b) {
    const long long per = 6LL * QZ * QTP, n = E * per;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long e = i / per;
        const int r = (int)(i - e * per);
        const int row = r / QTP, qt = r - row * QTP;       // row = f * QZ + qz
        b[i] = qt < QT ? __float2bfloat16_rn(a[e * 6 * QZ * QT + (long long)row * QT + qt]) : __float2bfloat16_rn(0.f);
    }
}

cudaError_t build_g16(Level& L, cudaStream_t s) {
    if (!level_tc(L) || L.G32 == nullptr) return cudaSuccess;
    const int QTP = (L.QT + 1) / 2 * 2;
    const long long n = (long long)L.E * 6 * L.QZ * QTP;
    void* p = L.G16;
    cudaError_t e = cudaSuccess;
    if (p == nullptr) {          // first build; later ones (a new surface elevation) reuse it
        e = cudaMalloc(&p, sizeof(__nv_bfloat16) * (size_t)(n + 32));
        if (e != cudaSuccess) return e;
        L.G16 = static_cast<unsigned short*>(p);
    }
    e = cudaMemsetAsync(p, 0, sizeof(__nv_bfloat16) * (size_t)(n + 32), s);
    if (e != cudaSuccess) return e;
    const long long blocks = (n + 255) / 256;
    k_to_bf16_padded<<<(int)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096), 256, 0, s>>>(
        L.E, L.QT, L.QZ, QTP, L.G32, static_cast<__nv_bfloat16*>(p));
    return cudaGetLastError();
}

}  // namespace sem
