// The whole Laplace solve of a small problem in one launch of one thread-block cluster: lifting of the
// Dirichlet data (Eq. laplaceproblem), the outer FGMRES(m) or PCG iteration, and its
// preconditioner, the p-multigrid V-cycle of Algorithm 1 with Chebyshev-Jacobi sweeps and
// the direct coarse solve that the algorithm names (a dense inverse of the order-1
// free-node matrix, formed at setup).  FP64 throughout.
//
// Launch latency, not bandwidth, bounds such problems: the 2D slice of 128 triangles at
// P = 4 (1,040 free nodes) takes a few hundred kernels per FGMRES iteration on the
// multi-kernel path.  Here every level's operator is a set of precomputed FP64 element
// matrices (y = sum_e Q_e^T A_e Q_e x), the transfers use the reference interpolation matrix
// of each level pair, and every vector stays in global memory that only this launch touches
// (L2-resident).  One CTA would leave the solve bound by the FP64 pipe of a single SM (GB300
// executes about two FP64 FMAs per clock per SM), so a cluster of up to eight CTAs shares the
// work: each CTA takes a range of elements (its element sums in its own shared memory, summed
// across the cluster through distributed shared memory) and a range of nodes for the vector
// operations; the phases are separated by the cluster's hardware barrier, which its CTAs,
// scheduled together, cannot wait on from outside.  The host reads the result once.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sem_internal.hpp"

namespace sem {

struct SmallLevel {
    int N, E, Np, Npc;                 // nodes, elements, nodes per element (this and the next coarser level)
    const int* map;                    // [E][Np], negative for Dirichlet nodes (-id - 1)
    const int* mapc;                   // [E][Npc] of the next coarser level (null on the coarsest)
    const double* Ae;                  // [E][Np][Np] symmetric FP64 element matrices
    const double* dinv;                // [N] inverse assembled diagonal, 0 at Dirichlet nodes
    const double* wmult;               // [N] inverse multiplicities (restriction weights)
    const unsigned char* owner;        // [E][Np] the element that writes a prolonged node
    const double* I;                   // [Np][Npc] interpolation from the next coarser level
    double c0, c1[16], c2[16];         // Chebyshev coefficients of the level
    double *u, *f, *y, *d;             // work vectors [N]
};

struct SmallPlan {
    int nl, k_cheb, nu1, nu2, outer, m, imax, nd, Nc;
    const long long* dir;              // Dirichlet node ids of the finest level
    const double* Cinv;                // [Nc][Nc] inverse of the coarse free-node matrix (zero at Dirichlet)
    double *V, *Z, *r, *q, *fr, *x, *p, *z;
    double* out;                       // iterations, fnorm, final residual, status, V-cycles, finest applies
    SmallLevel lv[SEM_MAX_LEVELS];
};

struct SmallHost {
    SmallPlan plan{};                  // host copy (device pointers)
    SmallPlan* dplan = nullptr;        // device copy
    std::vector<void*> owned;          // device buffers of the plan
    size_t smem = 0;
    int N0 = 0;
    int cluster = 1;                   // CTAs of the launch's one cluster
};

namespace {

namespace cg = cooperative_groups;

constexpr int kSmallThreads = 256;
constexpr int kSmallMaxN = 8192;                 // finest nodes (the shared-memory sums)
constexpr long long kSmallMaxWork = 1LL << 20;   // E Np^2 of the finest level
constexpr int kSmallCluster = 8;                 // CTAs of the cluster at most (portable size; 16 was no faster)
constexpr int kSlot = 72;                        // partial sums exchanged per reduction

// Per-CTA state: the cluster, this CTA's shared-memory buffers.  The CTAs of the cluster
// split every element loop by elements and every vector loop by node ranges; data written by
// one CTA and read by another crosses a cluster barrier (global memory read through L2).
struct Ctx {
    int rank, size;
    double* acc;        // [N0] this CTA's element sums
    double* xs;         // [N0] staged input vector
    double* slot;       // [2][kSlot] this CTA's partial sums (read by the others)
    double* tot;        // [kSlot] totals
    int parity;
};

__device__ __forceinline__ void csync() { cg::this_cluster().sync(); }
__device__ __forceinline__ int lo_of(int n, const Ctx& c) { return (int)((long long)n * c.rank / c.size); }
__device__ __forceinline__ int hi_of(int n, const Ctx& c) { return (int)((long long)n * (c.rank + 1) / c.size); }

__device__ __forceinline__ double sw_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// the cluster totals of nv values, entry i of this CTA's partials already in slot[parity][i]
// (written by its threads before the call); every CTA sums the ranks in order, so all hold
// the same totals, in tot[0 .. nv)
__device__ void c_totals(Ctx& c, int nv) {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        double v[kSmallCluster];
#pragma unroll
        for (int r = 0; r < kSmallCluster; ++r)          // all remote loads first, then the sum in rank order
            v[r] = r < c.size ? cl.map_shared_rank(c.slot, r)[c.parity * kSlot + i] : 0.0;
        double t = 0.0;
#pragma unroll
        for (int r = 0; r < kSmallCluster; ++r) t += v[r];
        c.tot[i] = t;
    }
    __syncthreads();
    c.parity ^= 1;      // the other half is next; this one is rewritten only after another barrier
}

// cluster sum of one value per thread
__device__ double c_sum(Ctx& c, double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = sw_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double w = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        w = sw_sum(w);
        if (lane == 0) c.slot[c.parity * kSlot] = w;
    }
    c_totals(c, 1);
    return c.tot[0];
}

// (a, b) over the cluster (each CTA its node range)
__device__ double c_dot(Ctx& c, const double* a, const double* b, int n, double* red) {
    double v = 0.0;
    for (int i = lo_of(n, c) + threadIdx.x; i < hi_of(n, c); i += blockDim.x) v += __ldcg(a + i) * __ldcg(b + i);
    return c_sum(c, v, red);
}

// the element rows of this CTA's elements: acc[map_i] += sum_j A_e[i][j] xs[map_j]
template <int NP>
__device__ void s_rows(const SmallLevel& L, const double* xs, bool lift, double* acc, int e0, int e1) {
    const int Np = NP > 0 ? NP : L.Np;
    const int rows = (e1 - e0) * Np;
    for (int t = threadIdx.x; t < rows; t += blockDim.x) {
        const int row = e0 * Np + t;
        const int mi = L.map[row];
        if (mi < 0) continue;
        const int e = row / Np, i = row - e * Np;
        const int* me = L.map + (size_t)e * Np;
        const double* A = L.Ae + (size_t)e * Np * Np + i;          // column i = row i (symmetric)
        double v0 = 0.0, v1 = 0.0;
#pragma unroll
        for (int j = 0; j < (NP > 0 ? NP : 1); ++j) {
            if (NP == 0) break;
            const int mj = me[j];
            const double xj = mj >= 0 ? xs[mj] : (lift ? xs[-mj - 1] : 0.0);
            if (j & 1) v1 = fma(A[(size_t)j * Np], xj, v1);
            else v0 = fma(A[(size_t)j * Np], xj, v0);
        }
        if (NP == 0)
            for (int j = 0; j < Np; ++j) {
                const int mj = me[j];
                const double xj = mj >= 0 ? xs[mj] : (lift ? xs[-mj - 1] : 0.0);
                v0 = fma(A[(size_t)j * Np], xj, v0);
            }
        atomicAdd(&acc[mi], v0 + v1);
    }
}

// y_i = sum over the cluster's CTAs of acc[i] for this CTA's node range of n nodes, handed to
// epi(i, y_i), which writes what the next phase reads
template <typename Epi>
__device__ void c_gather_sums(Ctx& c, int n, Epi epi) {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();                                        // every CTA's sums are complete
    for (int i = lo_of(n, c) + threadIdx.x; i < hi_of(n, c); i += blockDim.x) {
        double v[kSmallCluster];
#pragma unroll
        for (int r = 0; r < kSmallCluster; ++r) v[r] = r < c.size ? cl.map_shared_rank(c.acc, r)[i] : 0.0;
        double t = 0.0;
#pragma unroll
        for (int r = 0; r < kSmallCluster; ++r) t += v[r];
        epi(i, t);
    }
    cl.sync();                                        // results complete; acc free for reuse
}

// The element sums acc of y = A x on a level (free rows; y = 0 at Dirichlet nodes); lift: x
// also at the Dirichlet nodes (the lifting product A_FD x_D), else x there counts as zero
__device__ void c_rows(Ctx& c, const SmallLevel& L, const double* x, bool lift) {
    for (int i = threadIdx.x; i < L.N; i += blockDim.x) {
        c.acc[i] = 0.0;
        c.xs[i] = __ldcg(x + i);
    }
    __syncthreads();
    const int e0 = lo_of(L.E, c), e1 = hi_of(L.E, c);
    switch (L.Np) {
        case 3: s_rows<3>(L, c.xs, lift, c.acc, e0, e1); break;
        case 6: s_rows<6>(L, c.xs, lift, c.acc, e0, e1); break;
        case 10: s_rows<10>(L, c.xs, lift, c.acc, e0, e1); break;
        case 15: s_rows<15>(L, c.xs, lift, c.acc, e0, e1); break;
        case 18: s_rows<18>(L, c.xs, lift, c.acc, e0, e1); break;
        case 21: s_rows<21>(L, c.xs, lift, c.acc, e0, e1); break;
        case 28: s_rows<28>(L, c.xs, lift, c.acc, e0, e1); break;
        case 40: s_rows<40>(L, c.xs, lift, c.acc, e0, e1); break;
        default: s_rows<0>(L, c.xs, lift, c.acc, e0, e1); break;
    }
}

// y = A x.  Ends with a cluster barrier, as does every phase below that writes a vector another
// CTA reads.
__device__ void c_apply(Ctx& c, const SmallLevel& L, const double* x, double* y, bool lift) {
    c_rows(c, L, x, lift);
    c_gather_sums(c, L.N, [&](int i, double v) { y[i] = v; });
}

// one Chebyshev-Jacobi sweep of k steps (u = 0 on entry when zero_init), node ranges
__device__ void c_sweep(Ctx& c, const SmallLevel& L, int k, const double* f, double* u, bool zero_init) {
    const int n0 = lo_of(L.N, c), n1 = hi_of(L.N, c);
    if (zero_init) {
        for (int i = n0 + threadIdx.x; i < n1; i += blockDim.x) {
            const double v = L.c0 * L.dinv[i] * __ldcg(f + i);
            L.d[i] = v;
            u[i] = v;
        }
        csync();
    } else {
        c_rows(c, L, u, false);
        c_gather_sums(c, L.N, [&](int i, double y) {          // the step on the fly from (A u)_i
            const double v = L.c0 * L.dinv[i] * (__ldcg(f + i) - y);
            L.d[i] = v;
            u[i] = __ldcg(u + i) + v;
        });
    }
    for (int j = 1; j < k; ++j) {
        c_rows(c, L, u, false);
        const double c1 = L.c1[j], c2 = L.c2[j];
        c_gather_sums(c, L.N, [&](int i, double y) {
            const double v = c1 * L.d[i] + c2 * L.dinv[i] * (__ldcg(f + i) - y);
            L.d[i] = v;
            u[i] = __ldcg(u + i) + v;
        });
    }
}

// fc = R (f - y) onto the next coarser level C (R = P^T, fine values weighted by 1/multiplicity)
__device__ void c_restrict(Ctx& c, const SmallLevel& F, const SmallLevel& C, const double* f, const double* y,
                           double* fc) {
    for (int i = threadIdx.x; i < C.N; i += blockDim.x) c.acc[i] = 0.0;
    __syncthreads();
    const int e0 = lo_of(F.E, c), e1 = hi_of(F.E, c);
    const int rows = (e1 - e0) * F.Npc;
    for (int t = threadIdx.x; t < rows; t += blockDim.x) {
        const int row = e0 * F.Npc + t;
        const int mc = F.mapc[row];
        if (mc < 0) continue;
        const int e = row / F.Npc, nc = row - e * F.Npc;
        const int* mf = F.map + (size_t)e * F.Np;
        double v = 0.0;
        for (int nf = 0; nf < F.Np; ++nf) {
            const int m = mf[nf];
            if (m >= 0) v = fma(F.I[(size_t)nf * F.Npc + nc], F.wmult[m] * (__ldcg(f + m) - __ldcg(y + m)), v);
        }
        atomicAdd(&c.acc[mc], v);
    }
    c_gather_sums(c, C.N, [&](int i, double v) { fc[i] = v; });
}

// uf += P uc from the next coarser level (each fine node written by its owner element)
__device__ void c_prolong(Ctx& c, const SmallLevel& F, const double* uc, double* uf) {
    const int e0 = lo_of(F.E, c), e1 = hi_of(F.E, c);
    const int rows = (e1 - e0) * F.Np;
    for (int t = threadIdx.x; t < rows; t += blockDim.x) {
        const int row = e0 * F.Np + t;
        const int m = F.map[row];
        if (m < 0 || !F.owner[row]) continue;
        const int e = row / F.Np, nf = row - e * F.Np;
        const int* mc = F.mapc + (size_t)e * F.Npc;
        double v = 0.0;
        for (int nc = 0; nc < F.Npc; ++nc) {
            const int cc = mc[nc];
            if (cc >= 0) v = fma(F.I[(size_t)nf * F.Npc + nc], __ldcg(uc + cc), v);
        }
        uf[m] = __ldcg(uf + m) + v;
    }
    csync();
}

// u = A_c^{-1} f on the coarsest level (the dense inverse is symmetric: column i read as row i)
__device__ void c_coarse(Ctx& c, const SmallPlan& P, const double* f, double* u) {
    for (int i = lo_of(P.Nc, c) + threadIdx.x; i < hi_of(P.Nc, c); i += blockDim.x) {
        double v = 0.0;
        for (int j = 0; j < P.Nc; ++j) v = fma(P.Cinv[(size_t)j * P.Nc + i], __ldcg(f + j), v);
        u[i] = v;
    }
    csync();
}

// z = M^{-1} f: Algorithm 1 with u = 0 on entry at every level
__device__ void c_vcycle(Ctx& c, const SmallPlan& P, const double* f0, double* u0) {
    const int nl = P.nl;
    if (nl == 1) {
        c_coarse(c, P, f0, u0);
        return;
    }
    for (int li = 0; li + 1 < nl; ++li) {
        const SmallLevel& L = P.lv[li];
        const double* f = li == 0 ? f0 : L.f;
        double* u = li == 0 ? u0 : L.u;
        for (int m = 0; m < P.nu1; ++m) c_sweep(c, L, P.k_cheb, f, u, m == 0);
        if (P.nu1 == 0) {
            for (int i = lo_of(L.N, c) + threadIdx.x; i < hi_of(L.N, c); i += blockDim.x) u[i] = 0.0;
            csync();
        }
        c_apply(c, L, u, L.y, false);
        c_restrict(c, L, P.lv[li + 1], f, L.y, P.lv[li + 1].f);
    }
    c_coarse(c, P, P.lv[nl - 1].f, P.lv[nl - 1].u);
    for (int li = nl - 2; li >= 0; --li) {
        const SmallLevel& L = P.lv[li];
        const double* f = li == 0 ? f0 : L.f;
        double* u = li == 0 ? u0 : L.u;
        c_prolong(c, L, P.lv[li + 1].u, u);
        for (int m = 0; m < P.nu2; ++m) c_sweep(c, L, P.k_cheb, f, u, false);
    }
}

// The solve: lifting, then FGMRES(m) (classical Gram-Schmidt twice, Givens rotations,
// restarts) or PCG, each preconditioned by one V-cycle, to ||f - A u|| <= rtol ||f|| + atol.
// Every CTA of the cluster runs the same control flow: the loop tests read totals that all
// CTAs compute alike, and the small dense work (rotations, the triangular solve) is repeated
// by thread 0 of every CTA on identical data.
__global__ void __launch_bounds__(kSmallThreads) k_small_solve(const SmallPlan* __restrict__ plan,
                                                              const double* __restrict__ rhs,
                                                              const double* __restrict__ eta, double* phi,
                                                              double rtol, double atol) {
    __shared__ SmallPlan P;
    __shared__ double sc[4];
    __shared__ double red[33];
    __shared__ double slot[2 * kSlot];
    __shared__ double tot[kSlot];
    {
        const int* src = reinterpret_cast<const int*>(plan);
        int* dst = reinterpret_cast<int*>(&P);
        for (int i = threadIdx.x; i < (int)(sizeof(SmallPlan) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const SmallLevel& L0 = P.lv[0];
    const int N = L0.N, m = P.m;
    extern __shared__ __align__(16) double ssm[];
    Ctx c;
    c.rank = (int)cg::this_cluster().block_rank();
    c.size = (int)cg::this_cluster().num_blocks();
    c.acc = ssm;                                // [N0]
    c.xs = ssm + N;                             // [N0]
    c.slot = slot;
    c.tot = tot;
    c.parity = 0;
    double* H = ssm + 2 * N;                    // [(m + 1) m]
    double* cs = H + (size_t)(m + 1) * m;      // [m]
    double* sn = cs + m;                       // [m]
    double* g = sn + m;                        // [m + 1]
    double* yv = g + m + 1;                    // [m]
    double* hk = yv + m;                       // [2 (m + 1)] the two Gram-Schmidt passes
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    const int n0 = lo_of(N, c), n1 = hi_of(N, c);
    const int d0 = lo_of(P.nd, c), d1 = hi_of(P.nd, c);
    int vcycles = 0, applies = 0;

    // lifting: f = rhs - A_FD phi_D on the free nodes
    for (int i = n0 + t; i < n1; i += blockDim.x) P.x[i] = 0.0;
    csync();
    for (int k = d0 + t; k < d1; k += blockDim.x) P.x[P.dir[k]] = eta[k];
    csync();
    c_apply(c, L0, P.x, P.q, true);
    for (int i = n0 + t; i < n1; i += blockDim.x) P.fr[i] = (rhs != nullptr ? rhs[i] : 0.0) - __ldcg(P.q + i);
    csync();
    for (int k = d0 + t; k < d1; k += blockDim.x) P.fr[P.dir[k]] = 0.0;
    csync();
    const double fnorm = sqrt(c_dot(c, P.fr, P.fr, N, red));
    const double thr = rtol * fnorm + atol;
    for (int i = n0 + t; i < n1; i += blockDim.x) phi[i] = 0.0;
    csync();
    int status = isfinite(fnorm) ? (int)SEM_OK : (int)SEM_NAN;
    int it = 0;
    double res = fnorm;
    if (status == SEM_OK && P.outer == SEM_OUTER_FGMRES) {
        for (int i = n0 + t; i < n1; i += blockDim.x) P.r[i] = __ldcg(P.fr + i);
        csync();
        double beta = fnorm;
        while (beta > thr) {
            if (it >= P.imax) { status = SEM_NOT_CONVERGED; break; }
            for (int i = n0 + t; i < n1; i += blockDim.x) P.V[i] = __ldcg(P.r + i) / beta;
            for (int i = t; i < (m + 1) * m; i += blockDim.x) H[i] = 0.0;
            for (int i = t; i <= m; i += blockDim.x) g[i] = 0.0;
            csync();
            if (t == 0) g[0] = beta;
            int j = 0;
            while (j < m && it < P.imax) {
                const double* vj = P.V + (size_t)j * N;
                double* zj = P.Z + (size_t)j * N;
                double* w = P.V + (size_t)(j + 1) * N;
                c_vcycle(c, P, vj, zj);
                ++vcycles;
                c_apply(c, L0, zj, w, false);
                ++applies;
                for (int pass = 0; pass < 2; ++pass) {           // classical Gram-Schmidt, twice
                    for (int k = wid; k <= j; k += nw) {
                        const double* vk = P.V + (size_t)k * N;
                        double v = 0.0;
                        for (int i = n0 + lane; i < n1; i += 32) v += __ldcg(vk + i) * __ldcg(w + i);
                        v = sw_sum(v);
                        if (lane == 0) c.slot[c.parity * kSlot + k] = v;
                    }
                    __syncthreads();
                    c_totals(c, j + 1);
                    for (int k = t; k <= j; k += blockDim.x) hk[pass * (m + 1) + k] = c.tot[k];
                    __syncthreads();
                    for (int i = n0 + t; i < n1; i += blockDim.x) {
                        double wi = __ldcg(w + i);
                        for (int k = 0; k <= j; ++k) wi -= hk[pass * (m + 1) + k] * __ldcg(P.V + (size_t)k * N + i);
                        w[i] = wi;
                    }
                    csync();
                }
                const double hn = sqrt(c_dot(c, w, w, N, red));
                if (t == 0) {
                    for (int k = 0; k <= j; ++k) H[(size_t)k * m + j] = hk[k] + hk[m + 1 + k];
                    H[(size_t)(j + 1) * m + j] = hn;
                    for (int k = 0; k < j; ++k) {
                        const double a = cs[k] * H[(size_t)k * m + j] + sn[k] * H[(size_t)(k + 1) * m + j];
                        H[(size_t)(k + 1) * m + j] = -sn[k] * H[(size_t)k * m + j] + cs[k] * H[(size_t)(k + 1) * m + j];
                        H[(size_t)k * m + j] = a;
                    }
                    const double den = hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
                    cs[j] = H[(size_t)j * m + j] / den;
                    sn[j] = H[(size_t)(j + 1) * m + j] / den;
                    H[(size_t)j * m + j] = den;
                    H[(size_t)(j + 1) * m + j] = 0.0;
                    g[j + 1] = -sn[j] * g[j];
                    g[j] = cs[j] * g[j];
                    sc[0] = fabs(g[j + 1]);
                }
                if (hn > 0.0)
                    for (int i = n0 + t; i < n1; i += blockDim.x) w[i] = __ldcg(w + i) / hn;
                csync();
                ++j;
                ++it;
                res = sc[0];
                if (!isfinite(hn)) { status = SEM_NAN; break; }
                if (res <= thr || hn == 0.0) break;
            }
            if (status != SEM_OK) break;
            if (t == 0)
                for (int k = j - 1; k >= 0; --k) {
                    double v = g[k];
                    for (int l = k + 1; l < j; ++l) v -= H[(size_t)k * m + l] * yv[l];
                    yv[k] = v / H[(size_t)k * m + k];
                }
            __syncthreads();
            for (int i = n0 + t; i < n1; i += blockDim.x) {
                double u = __ldcg(phi + i);
                for (int k = 0; k < j; ++k) u += yv[k] * __ldcg(P.Z + (size_t)k * N + i);
                phi[i] = u;
            }
            csync();
            c_apply(c, L0, phi, P.q, false);
            ++applies;
            for (int i = n0 + t; i < n1; i += blockDim.x) P.r[i] = __ldcg(P.fr + i) - __ldcg(P.q + i);
            csync();
            beta = sqrt(c_dot(c, P.r, P.r, N, red));
            res = beta;
            if (!isfinite(beta)) { status = SEM_NAN; break; }
        }
    } else if (status == SEM_OK) {                          // PCG
        for (int i = n0 + t; i < n1; i += blockDim.x) P.r[i] = __ldcg(P.fr + i);
        csync();
        if (res > thr) {
            c_vcycle(c, P, P.r, P.z);
            ++vcycles;
            for (int i = n0 + t; i < n1; i += blockDim.x) P.p[i] = __ldcg(P.z + i);
            csync();
            double rz = c_dot(c, P.z, P.r, N, red);
            for (;;) {
                if (it >= P.imax) { status = SEM_NOT_CONVERGED; break; }
                c_apply(c, L0, P.p, P.q, false);
                ++applies;
                const double pq = c_dot(c, P.p, P.q, N, red);
                const double alpha = rz / pq;
                for (int i = n0 + t; i < n1; i += blockDim.x) {
                    phi[i] = __ldcg(phi + i) + alpha * __ldcg(P.p + i);
                    P.r[i] = __ldcg(P.r + i) - alpha * __ldcg(P.q + i);
                }
                csync();
                ++it;
                res = sqrt(c_dot(c, P.r, P.r, N, red));
                if (!isfinite(res)) { status = SEM_NAN; break; }
                if (!(pq > 0.0)) { status = SEM_BREAKDOWN; break; }
                if (res <= thr) break;
                c_vcycle(c, P, P.r, P.z);
                ++vcycles;
                const double rzn = c_dot(c, P.z, P.r, N, red);
                const double beta = rzn / rz;
                rz = rzn;
                for (int i = n0 + t; i < n1; i += blockDim.x) P.p[i] = __ldcg(P.z + i) + beta * __ldcg(P.p + i);
                csync();
            }
        }
    }
    for (int k = d0 + t; k < d1; k += blockDim.x) phi[P.dir[k]] = eta[k];
    if (c.rank == 0 && t == 0) {
        P.out[0] = it;
        P.out[1] = fnorm;
        P.out[2] = res;
        P.out[3] = status;
        P.out[4] = vcycles;
        P.out[5] = applies;
    }
    csync();            // no CTA leaves while another may still read its shared memory
}

}  // namespace

namespace {

template <typename T>
cudaError_t small_alloc(SmallHost& S, T** p, size_t count) {
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1));
    if (e != cudaSuccess) return e;
    S.owned.push_back(q);
    *p = static_cast<T*>(q);
    return cudaSuccess;
}

template <typename T>
cudaError_t small_upload(SmallHost& S, T** p, const std::vector<T>& h) {
    cudaError_t e = small_alloc(S, p, h.size());
    if (e == cudaSuccess && !h.empty()) e = cudaMemcpy(*p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
    return e;
}

void small_release(SmallHost* S) {
    if (S == nullptr) return;
    for (void* q : S->owned) cudaFree(q);
    delete S;
}

}  // namespace

void free_small_plan(sem_handle* h) {
    small_release(static_cast<SmallHost*>(h->small));
    h->small = nullptr;
}

// The one-launch plan of a small problem (sem_options.fused_small): FP64 handles with the
// Chebyshev smoother, FGMRES or PCG outside, not batched, whose finest level has at most
// kSmallMaxN nodes and E Np^2 <= kSmallMaxWork, and whose coarse level is assembled (at most
// 2,048 nodes).  Anything else keeps the multi-kernel path.  Rebuilt when the geometry changes.
sem_status build_small_plan(sem_handle* h) {
    free_small_plan(h);
    const sem_options& o = h->opts;
    // (debug_barrier_extra targets the coarse CG kernel of the multi-kernel path)
    if (!o.fused_small || o.precision != SEM_PREC_FP64 || o.smoother != SEM_SMOOTH_CHEBYSHEV || o.batch != 0 ||
        (o.outer != SEM_OUTER_FGMRES && o.outer != SEM_OUTER_PCG) || o.k_cheb > 16 || o.debug_barrier_extra != 0)
        return SEM_OK;
    const int nl = (int)h->lv.size();
    const Level& L0 = h->lv[0];
    const Level& Cl = h->lv[nl - 1];
    if (L0.N > kSmallMaxN || (long long)L0.E * L0.Np * L0.Np > kSmallMaxWork || Cl.csr_val == nullptr || Cl.N > 2048)
        return SEM_OK;
    SmallHost* S = new SmallHost();
    SmallPlan& P = S->plan;
    P.nl = nl;
    P.k_cheb = o.k_cheb;
    P.nu1 = o.nu1;
    P.nu2 = o.nu2;
    P.outer = o.outer;
    P.m = o.outer == SEM_OUTER_FGMRES ? o.gmres_m : 1;
    P.imax = o.imax;
    P.nd = (int)L0.hdir.size();
    P.dir = L0.dir;
    P.Nc = (int)Cl.N;
    cudaError_t e = cudaSuccess;
    for (int li = 0; li < nl && e == cudaSuccess; ++li) {
        const Level& L = h->lv[li];
        SmallLevel& D = P.lv[li];
        D.N = (int)L.N;
        D.E = L.E;
        D.Np = L.Np;
        D.map = L.map;
        D.dinv = L.dinv;
        D.wmult = L.wmult;
        D.owner = L.owner;
        for (double** v : {&D.u, &D.f, &D.y, &D.d})
            if (e == cudaSuccess) e = small_alloc(*S, v, L.N);
        if (li + 1 == nl) break;
        const Level& C = h->lv[li + 1];
        D.Npc = C.Np;
        D.mapc = C.map;
        double* Ae = nullptr;
        if (e == cudaSuccess) e = small_alloc(*S, &Ae, (size_t)L.E * L.Np * L.Np);
        if (e == cudaSuccess) e = element_matrices64(L, Ae, 0);
        D.Ae = Ae;
        // interpolation from C: I[nf][nc] = Bt[n_f][n_c] Bz[k_f][k_c], node l = k NT + n
        std::vector<double> Bt, Bz, I((size_t)L.Np * C.Np);
        interp_factors(L.dim, L.p, C.p, L.pz, C.pz, Bt, Bz);
        for (int kf = 0; kf < L.NZ; ++kf)
            for (int nf = 0; nf < L.NT; ++nf)
                for (int kc = 0; kc < C.NZ; ++kc)
                    for (int nc = 0; nc < C.NT; ++nc)
                        I[(size_t)(kf * L.NT + nf) * C.Np + kc * C.NT + nc] = Bt[(size_t)nf * C.NT + nc] * Bz[(size_t)kf * C.NZ + kc];
        double* dI = nullptr;
        if (e == cudaSuccess) e = small_upload(*S, &dI, I);
        D.I = dI;
        const Cheb c = cheb_coeffs(L.lam, o);
        D.c0 = c.c0;
        for (int j = 0; j < 16; ++j) {
            D.c1[j] = c.c1[j];
            D.c2[j] = c.c2[j];
        }
    }
    // the coarsest level's operator for the lifting of a single-level handle, and its inverse
    if (e == cudaSuccess && nl == 1) {
        double* Ae = nullptr;
        e = small_alloc(*S, &Ae, (size_t)Cl.E * Cl.Np * Cl.Np);
        if (e == cudaSuccess) e = element_matrices64(Cl, Ae, 0);
        P.lv[0].Ae = Ae;
    }
    if (e == cudaSuccess) {
        const long long Nc = Cl.N;
        std::vector<int> rowptr(Nc + 1), col((size_t)Cl.csr_nnz);
        std::vector<double> val((size_t)Cl.csr_nnz);
        e = cudaMemcpy(rowptr.data(), Cl.csr_rowptr, sizeof(int) * (Nc + 1), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(col.data(), Cl.csr_col, sizeof(int) * col.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(val.data(), Cl.csr_val, sizeof(double) * val.size(), cudaMemcpyDeviceToHost);
        std::vector<int> fr;
        for (long long i = 0; i < Nc; ++i)
            if (rowptr[i + 1] > rowptr[i]) fr.push_back((int)i);
        const int nf = (int)fr.size();
        std::vector<int> pos(Nc, -1);
        for (int k = 0; k < nf; ++k) pos[fr[k]] = k;
        std::vector<double> a((size_t)nf * nf, 0.0);
        for (int k = 0; k < nf; ++k)
            for (int t = rowptr[fr[k]]; t < rowptr[fr[k] + 1]; ++t)
                if (pos[col[t]] >= 0) a[(size_t)k * nf + pos[col[t]]] = val[t];
        for (int i = 0; i < nf; ++i)
            for (int j = 0; j < i; ++j)
                a[(size_t)i * nf + j] = a[(size_t)j * nf + i] = 0.5 * (a[(size_t)i * nf + j] + a[(size_t)j * nf + i]);
        if (e == cudaSuccess && !spd_inverse(a, nf)) {
            small_release(S);
            set_error("fused small solve: the coarse matrix is not positive definite");
            return SEM_BREAKDOWN;
        }
        std::vector<double> cinv((size_t)Nc * Nc, 0.0);
        for (int i = 0; i < nf; ++i)
            for (int j = 0; j < nf; ++j) cinv[(size_t)fr[i] * Nc + fr[j]] = a[(size_t)i * nf + j];
        double* dC = nullptr;
        if (e == cudaSuccess) e = small_upload(*S, &dC, cinv);
        P.Cinv = dC;
    }
    const size_t N0 = L0.N;
    const int m = P.m;
    if (e == cudaSuccess) e = small_alloc(*S, &P.V, (size_t)(m + 1) * N0);
    if (e == cudaSuccess) e = small_alloc(*S, &P.Z, (size_t)m * N0);
    for (double** v : {&P.r, &P.q, &P.fr, &P.x, &P.p, &P.z})
        if (e == cudaSuccess) e = small_alloc(*S, v, N0);
    if (e == cudaSuccess) e = small_alloc(*S, &P.out, 8);
    if (e == cudaSuccess) e = small_alloc(*S, &S->dplan, 1);
    if (e == cudaSuccess) e = cudaMemcpy(S->dplan, &P, sizeof(SmallPlan), cudaMemcpyHostToDevice);
    S->N0 = (int)N0;
    S->smem = sizeof(double) * (2 * N0 + 40 + (size_t)(m + 1) * m + 2 * (size_t)m + (m + 1) + m + 2 * (size_t)(m + 1));
    S->cluster = std::max(1, std::min(kSmallCluster, L0.E / 16));     // at least 16 elements per CTA
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_small_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S->smem);
    if (e != cudaSuccess) {
        small_release(S);
        set_error(std::string("fused small solve: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SEM_ENOMEM : SEM_ECUDA;
    }
    h->small = S;
    return SEM_OK;
}

// One launch of the fused solve; fills the statistics and returns its status.
sem_status small_solve(sem_handle* h, const double* rhs, const double* eta, double rtol, double* phi, sem_stats* st,
                       cudaStream_t s) {
    SmallHost* S = static_cast<SmallHost*>(h->small);
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)S->cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)S->cluster);
        cfg.blockDim = dim3(kSmallThreads);
        cfg.dynamicSmemBytes = S->smem;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const SmallPlan* dp = S->dplan;
        const double at_ = h->opts.atol;
        e = cudaLaunchKernelEx(&cfg, k_small_solve, dp, rhs, eta, phi, rtol, at_);
    }
    double out[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->sc.hpinned + 110, S->plan.out, 6 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error(std::string("fused small solve: ") + cudaGetErrorString(e));
        return SEM_ECUDA;
    }
    std::memcpy(out, h->sc.hpinned + 110, 6 * sizeof(double));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    sem_stats r{};
    r.iters = (int)out[0];
    r.fnorm = out[1];
    r.res0 = out[1];
    r.res_final = out[2];
    r.status = (int)out[3];
    r.vcycles = (long long)out[4];
    r.fine_applies = (long long)out[5];
    r.ms = ms;
    r.kernel_launches = 1;
    if (st) *st = r;
    if (r.status == SEM_NOT_CONVERGED) set_error("the outer iteration reached imax");
    else if (r.status == SEM_NAN) set_error("non-finite residual");
    else if (r.status == SEM_BREAKDOWN) set_error("PCG breakdown: p^T A p <= 0");
    return (sem_status)r.status;
}

}  // namespace sem
