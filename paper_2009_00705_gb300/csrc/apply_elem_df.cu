// FP64-accurate stiffness apply y = sum_e Q_e^T A_e Q_e x (Eq. laplaceproblemdiscrete) from
// precomputed element matrices held in double-FP32 form, on the FP32 pipe.
//
// Every entry a of A_e is stored as a pair of floats (a_hi, a_lo) with a_hi = fl32(a) and
// a_lo = fl32(a - a_hi), and x as the same kind of pair, so a x = a_hi x_hi + a_hi x_lo +
// a_lo x_hi up to 2^-48 |a x|.  The head product a_hi x_hi is split exactly into p + e with
// one FMA (the TwoProduct of Ogita, Rump and Oishi, "Accurate sum and dot product", 2005),
// p is added to a running FP32 sum with Knuth's TwoSum (exact), and the rounding errors, e
// and the two cross terms go to three FP32 compensation sums.  After every tile (28 or so
// terms) the compensation sums are renormalised into the head by another TwoSum, so they
// never gather more than one tile's rounding errors; the partial sums of a node meet as
// (head, tail) pairs and become one FP64 value at the end.  A row's error stays within
// about 3e-12 of sum_j |A_ij x_j| in the worst case and near 1e-14 in practice: FP64-class
// results at the FP32 pipe's rate, which on GB300 is dozens of times the FP64 pipe's.
//
// A_e is symmetric, so only its upper block triangle is stored: the Np rows are cut into NB
// blocks of T (T <= 32, one warp lane per row or column), and the NB (NB + 1) / 2 tiles
// A_IJ, J >= I in cyclic order, each T x S pairs with an odd row stride S so that a lane
// reading its row and a lane reading its column both hit distinct shared-memory banks.  An
// off-diagonal tile serves twice: y_I += A_IJ x_J (lane r takes row r) and y_J += A_IJ^T x_I
// (lane c takes column c).  At order 6 (Np = 196, NB = 7, T = 28) an element streams 182 KB
// against 307 KB for the full FP64 matrix.
//
// A CTA of NB warps takes one element at a time; warp w owns the tiles (w, w + d mod NB),
// d = 0 .. NB/2 (for even NB the last difference only for w < NB/2: every unordered block
// pair once).  Each warp streams its tiles through a two-slot shared-memory ring with bulk
// copies (cp.async.bulk, completion on an mbarrier, every wait bounded), so the next tile
// is in flight while the current one is multiplied.  Per element: gather x (prefetched one
// element ahead), the warps' tile products into per-block partial sums, and, two elements
// later, the per-node sums of the partials and the direct-stiffness summation (FP64
// atomics, or element results for the fixed-order sums of deterministic handles).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sem_internal.hpp"

namespace sem {

namespace {

constexpr int kSMs = 152;
constexpr unsigned long long kDfWaitNs = 1000000000ull;   // bound on every mbarrier wait (1 s)

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long df_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool df_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for phase `parity` of `bar`, at most kDfWaitNs; false (and the error flag set) after that.
__device__ bool df_wait(uint32_t bar, uint32_t parity, int* err) {
    if (df_try(bar, parity)) return true;
    const unsigned long long t0 = df_ns();
    for (;;) {
        if (df_try(bar, parity)) return true;
        if (df_ns() - t0 > kDfWaitNs) {
            if (err != nullptr) atomicExch(err, 1);
            return false;
        }
    }
}

// one thread: bulk-copy `bytes` (a multiple of 16, both addresses 16-byte aligned) from global
// to shared memory, completing on `bar`
__device__ __forceinline__ void df_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// (s, l) += (a, b): the heads by Knuth's TwoSum (s + a = t + d exactly), d and b into l.
// Rounded intrinsics keep the compiler from contracting or reassociating.
__device__ __forceinline__ void df_add(float& s, float& l, float a, float b) {
    const float t = __fadd_rn(s, a);
    const float bp = __fsub_rn(t, s);
    const float d = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(a, bp));
    s = t;
    l = __fadd_rn(l, __fadd_rn(d, b));
}

// (s, l, c1, c2) += a x in double-FP32 arithmetic: s the running head sum, l its TwoSum and
// TwoProduct errors, c1 and c2 the cross terms a_hi x_lo and a_lo x_hi.
__device__ __forceinline__ void df_mac(float& s, float& l, float& c1, float& c2, const float2 a, const float2 x) {
    const float p = __fmul_rn(a.x, x.x);
    const float e = __fmaf_rn(a.x, x.x, -p);          // a_hi x_hi = p + e exactly
    c1 = __fmaf_rn(a.x, x.y, c1);
    c2 = __fmaf_rn(a.y, x.x, c2);
    df_add(s, l, p, e);
}

// one block row (lane r: row r of the tile) and, off the diagonal, one block column (lane c)
template <int TT, bool OFF>
__device__ __forceinline__ void df_tile(const float2* __restrict__ A, int T, int S, int lane, const float2* xJ,
                                        const float2* xI, float& zs, float& zl, float& z1, float& z2, float& ws,
                                        float& wl, float& w1, float& w2) {
    if constexpr (TT > 0) {
        // even T: the x blocks start on 16-byte boundaries, two pairs per shared-memory load
        static_assert(TT % 2 == 0, "even block size");
        constexpr int SS = TT | 1;
#pragma unroll
        for (int c = 0; c < TT; c += 2) {
            const float4 xj = *reinterpret_cast<const float4*>(xJ + c);
            df_mac(zs, zl, z1, z2, A[lane * SS + c], make_float2(xj.x, xj.y));
            df_mac(zs, zl, z1, z2, A[lane * SS + c + 1], make_float2(xj.z, xj.w));
            if constexpr (OFF) {
                const float4 xi = *reinterpret_cast<const float4*>(xI + c);
                df_mac(ws, wl, w1, w2, A[c * SS + lane], make_float2(xi.x, xi.y));
                df_mac(ws, wl, w1, w2, A[(c + 1) * SS + lane], make_float2(xi.z, xi.w));
            }
        }
    } else {
#pragma unroll 4
        for (int c = 0; c < T; ++c) {
            df_mac(zs, zl, z1, z2, A[lane * S + c], xJ[c]);
            if constexpr (OFF) df_mac(ws, wl, w1, w2, A[c * S + lane], xI[c]);
        }
    }
}

__device__ __forceinline__ float2 df_split(double v) {
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}

template <int TT, bool LIFT>
__global__ void __launch_bounds__(256) k_apply_elem_df(int E, int Np, int Tr, int NB, int S, int TS,
                                                       const int* __restrict__ map, const float2* __restrict__ Adf,
                                                       const double* __restrict__ x, double* __restrict__ y,
                                                       const int* __restrict__ skip, const int* __restrict__ elist,
                                                       double* __restrict__ ye, int* err) {
    if (skip != nullptr && *skip) return;
    const int T = TT > 0 ? TT : Tr;
    const int H = NB / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int nd = df_tiles_of(warp, NB);
    int off = 0;
    for (int w = 0; w < warp; ++w) off += df_tiles_of(w, NB);
    const int ntiles = NB * (NB + 1) / 2;
    const int NT = NB * T;                          // padded rows

    extern __shared__ __align__(16) unsigned char df_smem[];
    float2* ring = reinterpret_cast<float2*>(df_smem);              // [NB][2][TS]
    float2* xs = ring + (size_t)NB * 2 * TS;                         // [2][NT]
    float2* part = xs + 2 * NT;                                      // [2][H + 1][NB][T] (head, tail)
    uint64_t* bars = reinterpret_cast<uint64_t*>(part + (size_t)2 * (H + 1) * NB * T);   // [NB][2]
    float2* myring = ring + (size_t)warp * 2 * TS;
    const uint32_t bar0 = saddr(bars + 2 * warp), bar1 = bar0 + 8;

    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const long long count = E > (int)blockIdx.x ? (long long)(E - 1 - (int)blockIdx.x) / gridDim.x + 1 : 0;
    auto elem = [&](long long it) -> long long {
        const long long eb = (long long)blockIdx.x + it * gridDim.x;
        return elist != nullptr ? (long long)elist[eb] : eb;
    };
    const long long njobs = count * nd;
    const uint32_t tile_bytes = (uint32_t)TS * 8u;
    // lane 0: job j = it * nd + k, tile k of this warp for element `it`, into slot j & 1
    auto issue = [&](long long j, long long it, int k) {
        const float2* src = Adf + ((size_t)elem(it) * ntiles + off + k) * TS;
        df_copy(saddr(myring + (size_t)(j & 1) * TS), src, tile_bytes, (j & 1) ? bar1 : bar0);
    };
    bool failed = false;
    long long pend0 = -1, pend1 = -1;          // job in flight in slot 0 / 1 (lane 0's view)
    if (lane == 0 && njobs > 0) {
        issue(0, 0, 0);
        pend0 = 0;
    }

    // x of the next element, prefetched into registers one element ahead
    int m_next = -1, m_cur = -1, m_prev = -1, m_prev2 = -1;
    double x_next = 0.0;
    auto prefetch = [&](long long it) {
        if (tid < Np) {
            m_next = map[(size_t)elem(it) * Np + tid];
            x_next = m_next >= 0 ? x[m_next] : (LIFT ? x[-m_next - 1] : 0.0);
        }
    };
    if (count > 0) prefetch(0);

    for (long long it = 0; it < count + 2; ++it) {
        const int slot = (int)(it & 1);
        // ---- phase A: stage x of element `it`, prefetch the next, finish element it - 2
        m_prev2 = m_prev;
        m_prev = m_cur;
        if (it < count) {
            if (tid < NT) xs[slot * NT + tid] = tid < Np ? df_split(x_next) : make_float2(0.f, 0.f);
            m_cur = m_next;
            if (it + 1 < count) prefetch(it + 1);
        }
        if (it >= 2 && tid < Np) {
            const int b = tid / T, r = tid - b * T;
            const float2* pp = part + (size_t)slot * (H + 1) * NB * T;
            float2 q = pp[(size_t)b * T + r];
            float hs = q.x, hl = q.y;
            for (int d = 1; d <= H; ++d) {
                const int w = b - d < 0 ? b - d + NB : b - d;
                if (d < df_tiles_of(w, NB)) {
                    q = pp[((size_t)d * NB + b) * T + r];
                    df_add(hs, hl, q.x, q.y);
                }
            }
            const double v = (double)hs + (double)hl;
            if (ye != nullptr) ye[(size_t)elem(it - 2) * Np + tid] = v;
            else if (m_prev2 >= 0) atomicAdd(&y[m_prev2], v);
        }
        __syncthreads();
        if (it >= count) continue;

        // ---- phase B: this warp's tiles of element `it`
        const float2* xv = xs + slot * NT;
        float2* pp = part + (size_t)slot * (H + 1) * NB * T;
        float zs = 0.f, zl = 0.f;            // this warp's block row, all its tiles
        for (int k = 0; k < nd; ++k) {
            const long long j = it * nd + k;
            if (lane == 0 && !failed && j + 1 < njobs) {
                // the slot was last read by job j - 1 (generic proxy); order that before the copy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (k + 1 < nd) issue(j + 1, it, k + 1);
                else issue(j + 1, it + 1, 0);
                if ((j + 1) & 1) pend1 = j + 1;
                else pend0 = j + 1;
            }
            bool ok = true;
            if (!failed) ok = df_wait((j & 1) ? bar1 : bar0, (uint32_t)((j >> 1) & 1), err);
            failed = failed || !__all_sync(0xffffffffu, ok);
            if (!failed && lane == 0) {
                if (j & 1) pend1 = -1;
                else pend0 = -1;
            }
            const int J = warp + k < NB ? warp + k : warp + k - NB;
            if (!failed && lane < T) {
                const float2* A = myring + (size_t)(j & 1) * TS;
                float z1 = 0.f, z2 = 0.f, ws = 0.f, wl = 0.f, w1 = 0.f, w2 = 0.f;
                if (k == 0)
                    df_tile<TT, false>(A, T, S, lane, xv + J * T, nullptr, zs, zl, z1, z2, ws, wl, w1, w2);
                else
                    df_tile<TT, true>(A, T, S, lane, xv + J * T, xv + warp * T, zs, zl, z1, z2, ws, wl, w1, w2);
                // renormalise the row sum once per tile (s + l exact, |l| <= ulp(s) / 2), so that
                // the compensation sums never gather more than one tile's rounding errors
                const float c = __fadd_rn(__fadd_rn(zl, z1), z2);
                zl = 0.f;
                df_add(zs, zl, c, 0.f);
                if (k > 0) pp[((size_t)k * NB + J) * T + lane] = make_float2(ws, __fadd_rn(__fadd_rn(wl, w1), w2));
            }
            __syncwarp();
        }
        if (lane < T) pp[(size_t)warp * T + lane] = failed ? make_float2(0.f, 0.f) : make_float2(zs, zl);
    }
    // copies still in flight after a failed wait: let them land before the CTA exits
    if (lane == 0) {
        if (pend0 >= 0) df_wait(bar0, (uint32_t)((pend0 >> 1) & 1), nullptr);
        if (pend1 >= 0) df_wait(bar1, (uint32_t)((pend1 >> 1) & 1), nullptr);
    }
    __syncwarp();
}

template <int TT, bool LIFT>
cudaError_t launch_df(const Level& L, int E, const int* elist, const double* x, double* y, const int* skip, double* ye,
                      cudaStream_t s) {
    const int NB = L.df_NB, T = L.df_T, H = NB / 2;
    const size_t smem = sizeof(float2) * ((size_t)NB * 2 * L.df_TS + 2 * (size_t)NB * T) +
                        sizeof(double) * (size_t)2 * (H + 1) * NB * T + sizeof(uint64_t) * 2 * NB;
    auto kern = k_apply_elem_df<TT, LIFT>;
    static size_t smem_set = 0;                             // largest size allowed so far
    static int per_sm[8] = {0, 0, 0, 0, 0, 0, 0, 0};       // by NB
    if (smem > smem_set) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set = smem;
    }
    if (per_sm[NB] == 0) {
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[NB], kern, NB * 32, smem);
        if (e != cudaSuccess) return e;
        if (per_sm[NB] < 1) per_sm[NB] = 1;
    }
    const int grid = (int)std::min<long long>((long long)E, (long long)kSMs * per_sm[NB]);
    if (grid < 1) return cudaSuccess;
    kern<<<grid, NB * 32, smem, s>>>(E, L.Np, T, NB, L.df_S, L.df_TS, L.map, L.Adf, x, y, skip, elist, ye, L.df_err);
    return cudaGetLastError();
}

}  // namespace

// Block layout of the double-FP32 element matrices: NB = ceil(Np / 32) row blocks of
// T = ceil(Np / NB) rows, odd row stride S, tiles of TS pairs (an even count: 16-byte copies).
void df_layout(int Np, int* T, int* NB, int* S, int* TS) {
    const int nb = (Np + 31) / 32;
    const int t = (Np + nb - 1) / nb;
    const int st = (t & 1) ? t : t + 1;
    *NB = nb;
    *T = t;
    *S = st;
    *TS = (t * st + 1) / 2 * 2;
}

cudaError_t apply_elem_df(const Level& L, const double* x, double* y, bool lift, const int* skip, cudaStream_t s) {
    if (L.df_NB < 1 || L.df_NB > 7 || L.df_T > 32 || L.df_S != (L.df_T | 1)) return cudaErrorInvalidValue;
    double* ye = L.ye64;
    const bool sub = lift && L.lift_elems != nullptr && ye == nullptr;
    const int E = sub ? L.nlift : L.E;
    const int* elist = sub ? L.lift_elems : nullptr;
    cudaError_t e;
    if (L.df_T == 28)
        e = lift ? launch_df<28, true>(L, E, elist, x, y, skip, ye, s) : launch_df<28, false>(L, E, elist, x, y, skip, ye, s);
    else if (L.df_T == 32)
        e = lift ? launch_df<32, true>(L, E, elist, x, y, skip, ye, s) : launch_df<32, false>(L, E, elist, x, y, skip, ye, s);
    else
        e = lift ? launch_df<0, true>(L, E, elist, x, y, skip, ye, s) : launch_df<0, false>(L, E, elist, x, y, skip, ye, s);
    if (e != cudaSuccess || ye == nullptr) return e;
    return dss_gather64(L, ye, y, skip, s, true);
}

}  // namespace sem
