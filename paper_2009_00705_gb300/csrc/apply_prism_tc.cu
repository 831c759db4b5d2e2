// Tensor-core prism apply for the smoothing sweeps of the mixed-precision V-cycle
// (Eq. laplaceproblemdiscrete, same contraction as apply_prism.cu): the two triangle
// contractions per element run as TF32 warp MMAs (m16n8k8) with FP32 accumulation.
//
//   forward   [Ur; Us] = [Dr; Ds] U,  Ut = Bt W      rows qt, columns qz (one 8-wide tile)
//   backward  Xr = Dr^T Vr + Ds^T Vs,  Xt = Bt^T Vt  rows n,  columns qz
//
// The reference matrices are the A operands (constant, TF32-rounded once into shared
// memory with a padded row stride so ldmatrix is conflict-free); an element's nodal
// data is the B operand with its vertical points as the 8 MMA columns, so every
// element is one n-tile and a warp reuses each A fragment across several elements.
// The geometric factors of a whole CTA pass (one contiguous range of G) arrive in
// shared memory by one bulk asynchronous copy signalled on an mbarrier, issued as
// soon as the previous pass has consumed its factors; the vertical stages and the
// direct-stiffness summation stay on the SIMT pipes.  Operand rounding to TF32 makes
// the result differ from the FP32 apply by a few 1e-4 relative: the kernel serves the
// Chebyshev sweeps only, where the operator need not be exact.
#include <cuda_runtime.h>

#include <cstdint>

#include "sem_internal.hpp"

namespace sem {

namespace {

constexpr int kTcSMs = 152;
constexpr int kTcWarps = 8;
constexpr int kTcThreads = 32 * kTcWarps;
constexpr unsigned long long kTcWaitNs = 1000000000ULL;   // 1 s bound on the copy wait

template <int P>
struct TcTile {
    static constexpr int NT = (P + 1) * (P + 2) / 2, NZ = P + 1, QT = (P + 1) * (P + 1), QZ = P + 1;
    static constexpr int Np = NT * NZ, Nq = QT * QZ;
    static_assert(QZ <= 8, "an element's vertical points fill one 8-wide MMA column tile");
    static constexpr int MTF = (QT + 15) / 16;     // forward m-tiles (rows qt)
    static constexpr int KSF = (NT + 7) / 8;       // forward k-steps (columns n)
    static constexpr int MTB = (NT + 15) / 16;     // backward m-tiles (rows n)
    static constexpr int KSB = (QT + 7) / 8;       // backward k-steps (columns qt)
    static_assert(MTF * 16 >= KSB * 8, "forward rows cover the backward K extent");
    static constexpr int LDF = KSF * 8 + 4;        // row stride of the forward A matrices (floats)
    static constexpr int LDB = KSB * 8 + 4;        // row stride of the backward A matrices
    static constexpr int GE = 4;                   // elements per forward warp task
    static constexpr int GB = 2;                   // elements per backward warp task
    static constexpr int EB = GE * ((kTcWarps + MTF - 1) / MTF);   // elements per CTA pass (even)
    static_assert(EB % 2 == 0 && EB % GB == 0, "pass size");
    __host__ __device__ static constexpr int r4(int v) { return (v + 3) / 4 * 4; }
    // shared-memory regions, in floats (every offset a multiple of 4 floats = 16 bytes)
    static constexpr int GSZ = r4(EB * 6 * Nq);
    static constexpr int AF = 3 * MTF * 16 * LDF;
    static constexpr int AB = 3 * MTB * 16 * LDB;
    static constexpr int ZZ = r4(2 * QZ * NZ);
    static constexpr int MAP = r4(EB * Np);
    static constexpr int XS = r4(Np);              // gathered nodal values [NZ][NT]
    static constexpr int US = KSF * 8 * 8;         // U or W: [KSF*8][8]
    static constexpr int VS = KSB * 8 * 8;         // Vr, Vs or Vt: [KSB*8][8]
    static constexpr int RS = MTB * 16 * 8;        // Xr or Xt: [MTB*16][8]
    static constexpr int WORK = XS + 2 * US + 3 * VS + 2 * RS;
    static constexpr int TOTAL = GSZ + AF + AB + ZZ + MAP + EB * WORK;
    static constexpr size_t SMEM = sizeof(float) * (size_t)TOTAL;
};

__device__ __forceinline__ uint32_t to_tf32(float f) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
    return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&a)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
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

// One thread: bulk-copy the geometric factors of elements [e, e + nb) into sG.  The
// byte count is rounded up to 16 (the G allocation carries 64 bytes of padding) and
// split into 16 KB pieces on the same mbarrier.
template <int P>
__device__ void issue_g(const float* G, int e, int nb, float* sG, uint32_t bar) {
    using D = TcTile<P>;
    const char* src = reinterpret_cast<const char*>(G + (size_t)e * 6 * D::Nq);
    const uint32_t bytes = ((uint32_t)nb * 6u * D::Nq * 4u + 15u) & ~15u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    const uint32_t dst = smem_u32(sG);
    for (uint32_t off = 0; off < bytes; off += 16384u) {
        const uint32_t n = (bytes - off < 16384u) ? (bytes - off) : 16384u;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst + off),
            "l"(src + off), "r"(n), "r"(bar)
            : "memory");
    }
}

template <int P>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_apply_prism_tc(int E, const int* __restrict__ map, const float* __restrict__ G, const float* __restrict__ refm,
                     const float* __restrict__ x, float* __restrict__ y, const int* __restrict__ skip, int* err) {
    using D = TcTile<P>;
    constexpr int NT = D::NT, NZ = D::NZ, QT = D::QT, QZ = D::QZ, Np = D::Np, Nq = D::Nq, EB = D::EB;
    if (skip != nullptr && *skip) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ int s_fail;
    float* sm = reinterpret_cast<float*>(smem_raw);
    float* sG = sm;
    float* sAF = sG + D::GSZ;                 // [3][MTF*16][LDF]: Dr, Ds, Bt (TF32 bits)
    float* sAB = sAF + D::AF;                 // [3][MTB*16][LDB]: Dr^T, Ds^T, Bt^T
    float* sZ = sAB + D::AB;                  // [Bz | Dz] as [QZ][NZ]
    int* sMap = reinterpret_cast<int*>(sZ + D::ZZ);
    float* work = sZ + D::ZZ + D::MAP;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;

    // every pad entry must be finite (and zero where it meets a non-zero operand)
    for (int i = tid; i < D::TOTAL; i += kTcThreads) sm[i] = 0.f;
    __syncthreads();
    const float* rBt = refm;
    const float* rDr = refm + QT * NT;
    const float* rDs = refm + 2 * QT * NT;
    for (int i = tid; i < QT * NT; i += kTcThreads) {
        const int qt = i / NT, n = i - qt * NT;
        sAF[(0 * D::MTF * 16 + qt) * D::LDF + n] = __uint_as_float(to_tf32(rDr[i]));
        sAF[(1 * D::MTF * 16 + qt) * D::LDF + n] = __uint_as_float(to_tf32(rDs[i]));
        sAF[(2 * D::MTF * 16 + qt) * D::LDF + n] = __uint_as_float(to_tf32(rBt[i]));
        sAB[(0 * D::MTB * 16 + n) * D::LDB + qt] = __uint_as_float(to_tf32(rDr[i]));
        sAB[(1 * D::MTB * 16 + n) * D::LDB + qt] = __uint_as_float(to_tf32(rDs[i]));
        sAB[(2 * D::MTB * 16 + n) * D::LDB + qt] = __uint_as_float(to_tf32(rBt[i]));
    }
    for (int i = tid; i < 2 * QZ * NZ; i += kTcThreads) sZ[i] = refm[6 * QT * NT + i];
    const float* sBz = sZ;
    const float* sDz = sZ + QZ * NZ;
    const uint32_t bar = smem_u32(&mbar);
    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t parity = 0;
    if (tid == 0 && blockIdx.x * EB < E) issue_g<P>(G, blockIdx.x * EB, min(EB, E - blockIdx.x * EB), sG, bar);

    for (int e0 = blockIdx.x * EB; e0 < E; e0 += gridDim.x * EB) {
        const int nb = min(EB, E - e0);
        // gather: element-local nodal values and the map of the pass
        for (int i = tid; i < nb * Np; i += kTcThreads) {
            const int b = i / Np, l = i - b * Np;
            const int m = map[(size_t)(e0 + b) * Np + l];
            sMap[b * Np + l] = m;
            work[b * D::WORK + l] = (m >= 0) ? x[m] : 0.f;
        }
        __syncthreads();
        // vertical stage: U[n][qz] = sum_k Bz[qz][k] X[k][n], W likewise with Dz (TF32-rounded)
        for (int i = tid; i < nb * NT; i += kTcThreads) {
            const int b = i / NT, n = i - b * NT;
            float* wb = work + b * D::WORK;
            float xk[NZ];
#pragma unroll
            for (int k = 0; k < NZ; ++k) xk[k] = wb[k * NT + n];
            float* U = wb + D::XS + n * 8;
            float* W = wb + D::XS + D::US + n * 8;
#pragma unroll
            for (int qz = 0; qz < QZ; ++qz) {
                float u = 0.f, w = 0.f;
#pragma unroll
                for (int k = 0; k < NZ; ++k) {
                    u += sBz[qz * NZ + k] * xk[k];
                    w += sDz[qz * NZ + k] * xk[k];
                }
                U[qz] = __uint_as_float(to_tf32(u));
                W[qz] = __uint_as_float(to_tf32(w));
            }
        }
        // this pass's geometric factors
        if (!mbar_wait(bar, parity)) s_fail = 1;
        __syncthreads();
        if (s_fail) break;          // uniform: every thread read s_fail after the barrier
        parity ^= 1u;
        // forward contractions and the geometric factors: warp task = (m-tile, GE elements)
        for (int task = warp; task < D::MTF * (EB / D::GE); task += kTcWarps) {
            const int mt = task % D::MTF, grp = task / D::MTF;
            float c[3][D::GE][4];
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int j = 0; j < D::GE; ++j)
#pragma unroll
                    for (int r = 0; r < 4; ++r) c[m][j][r] = 0.f;
            const int arow = mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
            const int acol = (lane >> 4) * 4;
#pragma unroll
            for (int ks = 0; ks < D::KSF; ++ks) {
                uint32_t ar[4], as[4], at[4];
                ldsm_x4(smem_u32(sAF + (0 * D::MTF * 16 + arow) * D::LDF + ks * 8 + acol), ar);
                ldsm_x4(smem_u32(sAF + (1 * D::MTF * 16 + arow) * D::LDF + ks * 8 + acol), as);
                ldsm_x4(smem_u32(sAF + (2 * D::MTF * 16 + arow) * D::LDF + ks * 8 + acol), at);
#pragma unroll
                for (int j = 0; j < D::GE; ++j) {
                    const float* wb = work + (grp * D::GE + j) * D::WORK;
                    const float* U = wb + D::XS;
                    const float* W = wb + D::XS + D::US;
                    const uint32_t u0 = __float_as_uint(U[(ks * 8 + t) * 8 + g]);
                    const uint32_t u1 = __float_as_uint(U[(ks * 8 + t + 4) * 8 + g]);
                    const uint32_t w0 = __float_as_uint(W[(ks * 8 + t) * 8 + g]);
                    const uint32_t w1 = __float_as_uint(W[(ks * 8 + t + 4) * 8 + g]);
                    mma_tf32(c[0][j], ar, u0, u1);
                    mma_tf32(c[1][j], as, u0, u1);
                    mma_tf32(c[2][j], at, w0, w1);
                }
            }
#pragma unroll
            for (int j = 0; j < D::GE; ++j) {
                const int b = grp * D::GE + j;
                if (b >= nb) continue;
                float* wb = work + b * D::WORK;
                float* Vr = wb + D::XS + 2 * D::US;
                float* Vs = Vr + D::VS;
                float* Vt = Vs + D::VS;
                const float* Gb = sG + (size_t)b * 6 * Nq;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int qt = mt * 16 + g + ((r >> 1) << 3);
                    const int qz = 2 * t + (r & 1);
                    float vr = 0.f, vs = 0.f, vt = 0.f;
                    if (qt < QT && qz < QZ) {
                        const int q = qz * QT + qt;
                        const float g0 = Gb[q], g1 = Gb[Nq + q], g2 = Gb[2 * Nq + q];
                        const float g3 = Gb[3 * Nq + q], g4 = Gb[4 * Nq + q], g5 = Gb[5 * Nq + q];
                        const float ur = c[0][j][r], us = c[1][j][r], ut = c[2][j][r];
                        vr = g0 * ur + g1 * us + g2 * ut;
                        vs = g1 * ur + g3 * us + g4 * ut;
                        vt = g2 * ur + g4 * us + g5 * ut;
                    }
                    if (qt < D::KSB * 8) {
                        Vr[qt * 8 + qz] = __uint_as_float(to_tf32(vr));
                        Vs[qt * 8 + qz] = __uint_as_float(to_tf32(vs));
                        Vt[qt * 8 + qz] = __uint_as_float(to_tf32(vt));
                    }
                }
            }
        }
        __syncthreads();
        // the factors are consumed: stream in the next pass's while this one finishes
        if (tid == 0) {
            const int en = e0 + gridDim.x * EB;
            if (en < E) issue_g<P>(G, en, min(EB, E - en), sG, bar);
        }
        // backward contractions: warp task = (m-tile, GB elements)
        for (int task = warp; task < D::MTB * (EB / D::GB); task += kTcWarps) {
            const int mt = task % D::MTB, grp = task / D::MTB;
            float xr[D::GB][4], xt[D::GB][4];
#pragma unroll
            for (int j = 0; j < D::GB; ++j)
#pragma unroll
                for (int r = 0; r < 4; ++r) xr[j][r] = xt[j][r] = 0.f;
            const int arow = mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
            const int acol = (lane >> 4) * 4;
#pragma unroll 1
            for (int ks = 0; ks < D::KSB; ++ks) {
                uint32_t ar[4], as[4], at[4];
                ldsm_x4(smem_u32(sAB + (0 * D::MTB * 16 + arow) * D::LDB + ks * 8 + acol), ar);
                ldsm_x4(smem_u32(sAB + (1 * D::MTB * 16 + arow) * D::LDB + ks * 8 + acol), as);
                ldsm_x4(smem_u32(sAB + (2 * D::MTB * 16 + arow) * D::LDB + ks * 8 + acol), at);
#pragma unroll
                for (int j = 0; j < D::GB; ++j) {
                    const float* Vr = work + (grp * D::GB + j) * D::WORK + D::XS + 2 * D::US;
                    const float* Vs = Vr + D::VS;
                    const float* Vt = Vs + D::VS;
                    const int o0 = (ks * 8 + t) * 8 + g, o1 = (ks * 8 + t + 4) * 8 + g;
                    mma_tf32(xr[j], ar, __float_as_uint(Vr[o0]), __float_as_uint(Vr[o1]));
                    mma_tf32(xr[j], as, __float_as_uint(Vs[o0]), __float_as_uint(Vs[o1]));
                    mma_tf32(xt[j], at, __float_as_uint(Vt[o0]), __float_as_uint(Vt[o1]));
                }
            }
#pragma unroll
            for (int j = 0; j < D::GB; ++j) {
                const int b = grp * D::GB + j;
                if (b >= nb) continue;
                float* Xr = work + b * D::WORK + D::XS + 2 * D::US + 3 * D::VS;
                float* Xt = Xr + D::RS;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int n = mt * 16 + g + ((r >> 1) << 3);
                    const int qz = 2 * t + (r & 1);
                    Xr[n * 8 + qz] = xr[j][r];
                    Xt[n * 8 + qz] = xt[j][r];
                }
            }
        }
        __syncthreads();
        // transposed vertical stage and direct-stiffness summation
        for (int i = tid; i < nb * NT; i += kTcThreads) {
            const int b = i / NT, n = i - b * NT;
            const float* Xr = work + b * D::WORK + D::XS + 2 * D::US + 3 * D::VS + n * 8;
            const float* Xt = Xr + D::RS;
            float xr[QZ], xt[QZ];
#pragma unroll
            for (int qz = 0; qz < QZ; ++qz) {
                xr[qz] = Xr[qz];
                xt[qz] = Xt[qz];
            }
#pragma unroll
            for (int k = 0; k < NZ; ++k) {
                float s = 0.f;
#pragma unroll
                for (int qz = 0; qz < QZ; ++qz) s += sBz[qz * NZ + k] * xr[qz] + sDz[qz * NZ + k] * xt[qz];
                const int m = sMap[b * Np + k * NT + n];
                if (m >= 0) atomicAdd(&y[m], s);
            }
        }
        __syncthreads();
    }
    if (s_fail) {
        // a copy did not complete in time: report it, give it a second bounded wait, return
        if (tid == 0) {
            atomicExch(err, 1);
            mbar_wait(bar, parity);
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
    const int passes = (L.E + D::EB - 1) / D::EB;
    const int grid = passes < kTcSMs ? passes : kTcSMs;
    if (grid < 1) return cudaSuccess;
    k_apply_prism_tc<P><<<grid, kTcThreads, D::SMEM, s>>>(L.E, L.map, L.G32, L.ref32.m, x, y, skip, err);
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

}  // namespace sem
