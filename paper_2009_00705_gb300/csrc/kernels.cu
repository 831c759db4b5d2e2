// CUDA kernels of the p-multigrid SEM Laplace solver (sm_103a).
//
//  * matrix-free stiffness apply (Eq. laplaceproblemdiscrete), sum-factorised in
//    the vertical direction of the prisms: gather -> reference derivatives at
//    the quadrature points -> geometric factors -> transposed contraction ->
//    direct-stiffness summation into the global vector;
//  * geometric factors G = w |det J| J^{-1} J^{-T} of the sigma-layer prism map
//    (Section 3.1, Eq. jacobian / K) and of straight triangles;
//  * the assembled diagonal (Jacobi smoother), p-restriction R = P^T and
//    prolongation P (Section 4.1, Eq. rest), Chebyshev smoothing updates and
//    the FP64 reductions of the Krylov iterations (Algorithms 2, 3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "sem_internal.hpp"

namespace sem {

namespace {

constexpr int kVecThreads = 256;
constexpr int kRedThreads = 256;
constexpr int kSMs = 152;

inline int vec_grid(long long n) {
    long long g = (n + kVecThreads - 1) / kVecThreads;
    if (g > kSMs * 16) g = kSMs * 16;
    if (g < 1) g = 1;
    return (int)g;
}

template <int P, bool PRISM>
struct Dims {
    static constexpr int NT = (P + 1) * (P + 2) / 2;
    static constexpr int NZ = PRISM ? P + 1 : 1;
    static constexpr int QT = (P + 1) * (P + 1);
    static constexpr int QZ = PRISM ? P + 1 : 1;
    static constexpr int Np = NT * NZ;
    static constexpr int Nq = QT * QZ;
    static constexpr int NC = PRISM ? 6 : 3;
    static constexpr int NREF = 6 * QT * NT + 2 * QZ * NZ;
    static constexpr int NWORK = Np + 2 * NT * QZ + 3 * Nq;
};

__device__ __forceinline__ int decode(int m) { return m >= 0 ? m : -m - 1; }

// ------------------------------------------------------------------ apply
// One CTA processes elements e = blockIdx.x, blockIdx.x + gridDim.x, ...
// Shared memory: the level's reference matrices, then per-element work arrays.
template <int P, bool PRISM, typename T, bool LIFT>
__global__ void __launch_bounds__(128) k_apply(int E, const int* __restrict__ map, const T* __restrict__ G,
                                               const T* __restrict__ refm, const T* __restrict__ x,
                                               T* __restrict__ y, const int* __restrict__ skip) {
    using D = Dims<P, PRISM>;
    if (skip != nullptr && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const T* sBt = sm;                       // [QT][NT]
    const T* sDr = sBt + D::QT * D::NT;
    const T* sDs = sDr + D::QT * D::NT;
    const T* sBtT = sDs + D::QT * D::NT;     // [NT][QT]
    const T* sDrT = sBtT + D::QT * D::NT;
    const T* sDsT = sDrT + D::QT * D::NT;
    const T* sBz = sDsT + D::QT * D::NT;     // [QZ][NZ]
    const T* sDz = sBz + D::QZ * D::NZ;
    T* xe = sm + D::NREF;                    // [Np]
    T* U = xe + D::Np;                       // [NT][QZ]  (z-interpolated values; later X_r)
    T* W = U + D::NT * D::QZ;                // [NT][QZ]  (z-derivatives; later X_t)
    T* vr = W + D::NT * D::QZ;               // [Nq]
    T* vs = vr + D::Nq;
    T* vt = vs + D::Nq;
    for (int i = threadIdx.x; i < D::NREF; i += blockDim.x) sm[i] = refm[i];
    __syncthreads();
    for (int e = blockIdx.x; e < E; e += gridDim.x) {
        const int* me = map + (size_t)e * D::Np;
        for (int i = threadIdx.x; i < D::Np; i += blockDim.x) {
            const int m = me[i];
            xe[i] = (m >= 0) ? x[m] : (LIFT ? x[-m - 1] : T(0));
        }
        __syncthreads();
        if (PRISM) {
            // vertical stage: values and t-derivatives at the vertical Gauss points
            for (int i = threadIdx.x; i < D::NT * D::QZ; i += blockDim.x) {
                const int n = i / D::QZ, qz = i - n * D::QZ;
                T u = 0, w = 0;
#pragma unroll
                for (int k = 0; k < D::NZ; ++k) {
                    const T xv = xe[k * D::NT + n];
                    u += sBz[qz * D::NZ + k] * xv;
                    w += sDz[qz * D::NZ + k] * xv;
                }
                U[i] = u;
                W[i] = w;
            }
        } else {
            for (int i = threadIdx.x; i < D::NT; i += blockDim.x) U[i] = xe[i];
        }
        __syncthreads();
        // triangle stage and geometric factors at every quadrature point
        const T* Ge = G + (size_t)e * D::NC * D::Nq;
        for (int q = threadIdx.x; q < D::Nq; q += blockDim.x) {
            const int qz = q / D::QT, qt = q - qz * D::QT;
            T ur = 0, us = 0, ut = 0;
#pragma unroll 4
            for (int n = 0; n < D::NT; ++n) {
                const T uv = U[n * D::QZ + qz];
                ur += sDrT[n * D::QT + qt] * uv;
                us += sDsT[n * D::QT + qt] * uv;
                if (PRISM) ut += sBtT[n * D::QT + qt] * W[n * D::QZ + qz];
            }
            if (PRISM) {
                const T g0 = Ge[q], g1 = Ge[D::Nq + q], g2 = Ge[2 * D::Nq + q];
                const T g3 = Ge[3 * D::Nq + q], g4 = Ge[4 * D::Nq + q], g5 = Ge[5 * D::Nq + q];
                vr[q] = g0 * ur + g1 * us + g2 * ut;
                vs[q] = g1 * ur + g3 * us + g4 * ut;
                vt[q] = g2 * ur + g4 * us + g5 * ut;
            } else {
                const T g0 = Ge[q], g1 = Ge[D::Nq + q], g2 = Ge[2 * D::Nq + q];
                vr[q] = g0 * ur + g1 * us;
                vs[q] = g1 * ur + g2 * us;
            }
        }
        __syncthreads();
        // transposed triangle stage
        for (int i = threadIdx.x; i < D::NT * D::QZ; i += blockDim.x) {
            const int qz = i / D::NT, n = i - qz * D::NT;
            T a = 0, b = 0;
#pragma unroll 4
            for (int qt = 0; qt < D::QT; ++qt) {
                const int q = qz * D::QT + qt;
                a += sDr[qt * D::NT + n] * vr[q] + sDs[qt * D::NT + n] * vs[q];
                if (PRISM) b += sBt[qt * D::NT + n] * vt[q];
            }
            U[n * D::QZ + qz] = a;
            W[n * D::QZ + qz] = b;
        }
        __syncthreads();
        // transposed vertical stage and direct-stiffness summation (free rows only)
        for (int i = threadIdx.x; i < D::Np; i += blockDim.x) {
            T s;
            if (PRISM) {
                const int k = i / D::NT, n = i - k * D::NT;
                s = 0;
#pragma unroll
                for (int qz = 0; qz < D::QZ; ++qz)
                    s += sBz[qz * D::NZ + k] * U[n * D::QZ + qz] + sDz[qz * D::NZ + k] * W[n * D::QZ + qz];
            } else {
                s = U[i];
            }
            const int m = me[i];
            if (m >= 0) atomicAdd(&y[m], s);
        }
        __syncthreads();
    }
}

template <int P, bool PRISM, typename T, bool LIFT>
cudaError_t apply_impl(const Level& L, const T* refm, const T* G, const T* x, T* y, const int* skip,
                       cudaStream_t s) {
    using D = Dims<P, PRISM>;
    const size_t smem = sizeof(T) * (D::NREF + D::NWORK);
    static bool configured = false;   // per template instance; attribute is per-function
    if (!configured) {
        cudaError_t err = cudaFuncSetAttribute(k_apply<P, PRISM, T, LIFT>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        configured = true;
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply<P, PRISM, T, LIFT>, 128, smem);
    if (per_sm < 1) per_sm = 1;
    int grid = kSMs * per_sm;
    if (grid > L.E) grid = L.E;
    if (grid < 1) return cudaSuccess;
    k_apply<P, PRISM, T, LIFT><<<grid, 128, smem, s>>>(L.E, L.map, G, refm, x, y, skip);
    return cudaGetLastError();
}

// triangles (2D vertical slices); prisms are in apply_prism.cu
template <typename T, bool LIFT>
cudaError_t apply_dispatch(const Level& L, const T* refm, const T* G, const T* x, T* y, const int* skip,
                           cudaStream_t s) {
#define SEM_CASE(PP)                                                                     \
    case PP:                                                                             \
        return apply_impl<PP, false, T, LIFT>(L, refm, G, x, y, skip, s);
    switch (L.p) {
        SEM_CASE(1)
        SEM_CASE(2)
        SEM_CASE(3)
        SEM_CASE(4)
        SEM_CASE(5)
        SEM_CASE(6)
        default:
            return cudaErrorInvalidValue;
    }
#undef SEM_CASE
}

// ------------------------------------------------------------------ geometry
// Sigma-layer prism: x, y affine over the base triangle, z = -h + sigma (h + eta_P(r, s)),
// sigma = (l + (t + 1)/2) / nlayers.  J = [[M, 0], [z_r z_s, z_t]] (block lower triangular),
// so J^{-1} has rows grad r = (M^{-1})_0, grad s = (M^{-1})_1 and
// grad t = (-(z_r, z_s) M^{-1} / z_t, 1 / z_t).
__global__ void k_geom_prism(int E, int nlayers, int QT, int QZ, int NTP, double depth,
                             const double* __restrict__ vtri, const double* __restrict__ etaP,
                             const double* __restrict__ BP, const double* __restrict__ DrP,
                             const double* __restrict__ DsP, const double* __restrict__ qinfo,
                             double* __restrict__ G, float* __restrict__ G32) {
    const int Nq = QT * QZ;
    const long long total = (long long)E * Nq;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(t / Nq), q = (int)(t - (long long)e * Nq);
        const int qz = q / QT, qt = q - qz * QT;
        const int b = e / nlayers, l = e - b * nlayers;
        const double* v = vtri + 6 * (size_t)b;
        const double m00 = 0.5 * (v[2] - v[0]), m01 = 0.5 * (v[4] - v[0]);
        const double m10 = 0.5 * (v[3] - v[1]), m11 = 0.5 * (v[5] - v[1]);
        const double* et = etaP + (size_t)b * NTP;
        double eta = 0, er = 0, es = 0;
        for (int n = 0; n < NTP; ++n) {
            eta += BP[qt * NTP + n] * et[n];
            er += DrP[qt * NTP + n] * et[n];
            es += DsP[qt * NTP + n] * et[n];
        }
        const double tw = qinfo[qt], zq = qinfo[QT + qz], zw = qinfo[QT + QZ + qz];
        const double sigma = (l + 0.5 * (zq + 1.0)) / nlayers;
        const double zr = sigma * er, zs = sigma * es, zt = (depth + eta) / (2.0 * nlayers);
        const double a2 = m00 * m11 - m01 * m10;
        const double i00 = m11 / a2, i01 = -m01 / a2, i10 = -m10 / a2, i11 = m00 / a2;
        const double gr[3] = {i00, i01, 0.0};
        const double gs[3] = {i10, i11, 0.0};
        const double gt[3] = {-(zr * i00 + zs * i10) / zt, -(zr * i01 + zs * i11) / zt, 1.0 / zt};
        const double wdet = tw * zw * fabs(zt * a2);
        const double c[6] = {
            wdet * (gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]),
            wdet * (gr[0] * gs[0] + gr[1] * gs[1] + gr[2] * gs[2]),
            wdet * (gr[0] * gt[0] + gr[1] * gt[1] + gr[2] * gt[2]),
            wdet * (gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2]),
            wdet * (gs[0] * gt[0] + gs[1] * gt[1] + gs[2] * gt[2]),
            wdet * (gt[0] * gt[0] + gt[1] * gt[1] + gt[2] * gt[2])};
        double* Ge = G + (size_t)e * 6 * Nq;
        float* Ge32 = G32 + (size_t)e * 6 * Nq;
        for (int k = 0; k < 6; ++k) {
            Ge[k * Nq + q] = c[k];
            Ge32[k * Nq + q] = (float)c[k];
        }
    }
}

// Prisms of a general mesh (curved base triangles, partial columns, given layer interfaces):
// x, y = the order-P interpolant of the base triangle's node xy; in layer l
// z = (1 - tau) z_l + tau z_{l+1}, tau = (t + 1)/2, z_k = a_k + b_k eta_P.  The Jacobian keeps
// the block form [[M, 0], [z_r z_s, z_t]] with M = d(x, y)/d(r, s) now varying over the element.
__global__ void k_geom_prism_general(int E, const int* __restrict__ eb, const int* __restrict__ el, int QT, int QZ,
                                     int NTP, const double* __restrict__ xyP, const double* __restrict__ etaP,
                                     const double* __restrict__ zif, const double* __restrict__ BP,
                                     const double* __restrict__ DrP, const double* __restrict__ DsP,
                                     const double* __restrict__ qinfo, double* __restrict__ G,
                                     float* __restrict__ G32) {
    const int Nq = QT * QZ;
    const long long total = (long long)E * Nq;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(t / Nq), q = (int)(t - (long long)e * Nq);
        const int qz = q / QT, qt = q - qz * QT;
        const int b = eb[e], l = el[e];
        const double* xy = xyP + 2 * (size_t)b * NTP;
        const double* et = etaP + (size_t)b * NTP;
        double m00 = 0, m01 = 0, m10 = 0, m11 = 0, eta = 0, er = 0, es = 0;
        for (int n = 0; n < NTP; ++n) {
            const double dr = DrP[qt * NTP + n], ds = DsP[qt * NTP + n], bb = BP[qt * NTP + n];
            m00 += dr * xy[2 * n];
            m01 += ds * xy[2 * n];
            m10 += dr * xy[2 * n + 1];
            m11 += ds * xy[2 * n + 1];
            eta += bb * et[n];
            er += dr * et[n];
            es += ds * et[n];
        }
        const double tw = qinfo[qt], zq = qinfo[QT + qz], zw = qinfo[QT + QZ + qz];
        const double tau = 0.5 * (zq + 1.0);
        const double a0 = zif[2 * l], b0 = zif[2 * l + 1], a1 = zif[2 * l + 2], b1 = zif[2 * l + 3];
        const double bl = (1.0 - tau) * b0 + tau * b1;
        const double zr = bl * er, zs = bl * es, zt = 0.5 * ((a1 - a0) + (b1 - b0) * eta);
        const double a2 = m00 * m11 - m01 * m10;
        const double i00 = m11 / a2, i01 = -m01 / a2, i10 = -m10 / a2, i11 = m00 / a2;
        const double gr[3] = {i00, i01, 0.0};
        const double gs[3] = {i10, i11, 0.0};
        const double gt[3] = {-(zr * i00 + zs * i10) / zt, -(zr * i01 + zs * i11) / zt, 1.0 / zt};
        const double wdet = tw * zw * fabs(zt * a2);
        const double c[6] = {
            wdet * (gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]),
            wdet * (gr[0] * gs[0] + gr[1] * gs[1] + gr[2] * gs[2]),
            wdet * (gr[0] * gt[0] + gr[1] * gt[1] + gr[2] * gt[2]),
            wdet * (gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2]),
            wdet * (gs[0] * gt[0] + gs[1] * gt[1] + gs[2] * gt[2]),
            wdet * (gt[0] * gt[0] + gt[1] * gt[1] + gt[2] * gt[2])};
        double* Ge = G + (size_t)e * 6 * Nq;
        float* Ge32 = G32 + (size_t)e * 6 * Nq;
        for (int k = 0; k < 6; ++k) {
            Ge[k * Nq + q] = c[k];
            Ge32[k * Nq + q] = (float)c[k];
        }
    }
}

// Straight triangle in the (x, z) plane: constant Jacobian M, G = w |det M| M^{-1} M^{-T}.
__global__ void k_geom_tri(int E, int QT, const double* __restrict__ vtri, const double* __restrict__ qinfo,
                           double* __restrict__ G, float* __restrict__ G32) {
    const long long total = (long long)E * QT;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(t / QT), q = (int)(t - (long long)e * QT);
        const double* v = vtri + 6 * (size_t)e;
        const double m00 = 0.5 * (v[2] - v[0]), m01 = 0.5 * (v[4] - v[0]);
        const double m10 = 0.5 * (v[3] - v[1]), m11 = 0.5 * (v[5] - v[1]);
        const double a2 = m00 * m11 - m01 * m10;
        const double i00 = m11 / a2, i01 = -m01 / a2, i10 = -m10 / a2, i11 = m00 / a2;
        const double w = qinfo[q] * fabs(a2);
        const double c[3] = {w * (i00 * i00 + i01 * i01), w * (i00 * i10 + i01 * i11), w * (i10 * i10 + i11 * i11)};
        double* Ge = G + (size_t)e * 3 * QT;
        float* Ge32 = G32 + (size_t)e * 3 * QT;
        for (int k = 0; k < 3; ++k) {
            Ge[k * QT + q] = c[k];
            Ge32[k * QT + q] = (float)c[k];
        }
    }
}

// ------------------------------------------------------------------ diagonal
// diag(A)_i = sum over elements of sum_q grad N_l^T G_q grad N_l, sum-factorised
// over the vertical direction for prisms.
__global__ void k_diag(int E, int dim, int NT, int NZ, int QT, int QZ, const int* __restrict__ map,
                       const double* __restrict__ G, const double* __restrict__ refm, double* __restrict__ diag,
                       double* __restrict__ ye) {
    extern __shared__ double sdiag[];       // [6][NT][QZ]
    const int Nq = QT * QZ, Np = NT * NZ;
    const int nc = (dim == 3) ? 6 : 3;
    const double* Bt = refm;
    const double* Dr = Bt + QT * NT;
    const double* Ds = Dr + QT * NT;
    const double* Bz = refm + 6 * QT * NT;
    const double* Dz = Bz + QZ * NZ;
    for (int e = blockIdx.x; e < E; e += gridDim.x) {
        const double* Ge = G + (size_t)e * nc * Nq;
        for (int i = threadIdx.x; i < NT * QZ; i += blockDim.x) {
            const int n = i / QZ, qz = i - n * QZ;
            double s[6] = {0, 0, 0, 0, 0, 0};
            for (int qt = 0; qt < QT; ++qt) {
                const int q = qz * QT + qt;
                const double dr = Dr[qt * NT + n], ds = Ds[qt * NT + n], bt = Bt[qt * NT + n];
                if (dim == 3) {
                    s[0] += dr * dr * Ge[q];
                    s[1] += dr * ds * Ge[Nq + q];
                    s[2] += dr * bt * Ge[2 * Nq + q];
                    s[3] += ds * ds * Ge[3 * Nq + q];
                    s[4] += ds * bt * Ge[4 * Nq + q];
                    s[5] += bt * bt * Ge[5 * Nq + q];
                } else {
                    s[0] += dr * dr * Ge[q];
                    s[1] += dr * ds * Ge[Nq + q];
                    s[3] += ds * ds * Ge[2 * Nq + q];
                }
            }
            for (int c = 0; c < 6; ++c) sdiag[c * NT * QZ + i] = s[c];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < Np; i += blockDim.x) {
            const int k = i / NT, n = i - k * NT;
            double v = 0;
            for (int qz = 0; qz < QZ; ++qz) {
                const int j = n * QZ + qz;
                const double bz = Bz[qz * NZ + k], dz = Dz[qz * NZ + k];
                v += bz * bz * (sdiag[j] + 2.0 * sdiag[NT * QZ + j] + sdiag[3 * NT * QZ + j]) +
                     2.0 * bz * dz * (sdiag[2 * NT * QZ + j] + sdiag[4 * NT * QZ + j]) +
                     dz * dz * sdiag[5 * NT * QZ + j];
            }
            if (ye != nullptr) ye[(size_t)e * Np + i] = v;      // summed by node afterwards
            else atomicAdd(&diag[decode(map[(size_t)e * Np + i])], v);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ transfers
// The element prolongation is a tensor product, I = Bt (x) Bz with Bt [NTf][NTc]
// the coarse triangle basis at the fine triangle nodes and Bz [NZf][NZc] the
// coarse 1D basis at the fine GLL nodes (Bz = [1] for triangles), so both
// transfers are applied in two sum-factorised stages.  A CTA handles kTrEB
// elements per pass.
// Direct-stiffness summation without atomics (deterministic handles): node g sums the
// element results of its slots ye[e Np + l] in the fixed order of the node's segment
// [ptr[g], ptr[g+1]) of the precomputed node -> slot map (ascending element, then local
// index).  masked: Dirichlet nodes (negative map entries) get 0, as in the masked operator;
// nodes in no element get 0.
__global__ void k_dss_gather(long long N, const int* __restrict__ ptr, const int* __restrict__ slot,
                             const int* __restrict__ map, int masked, const double* __restrict__ ye,
                             double* __restrict__ y, const int* __restrict__ skip) {
    if (skip != nullptr && *skip) return;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
        const int a = ptr[g], b = ptr[g + 1];
        double v = 0.0;
        if (!(masked && b > a && map[slot[a]] < 0))
            for (int i = a; i < b; ++i) v += ye[slot[i]];
        y[g] = v;
    }
}

}  // namespace

cudaError_t dss_gather64(const Level& L, const double* ye, double* y, const int* skip, cudaStream_t s, bool masked) {
    if (L.dss_ptr == nullptr || L.dss_slot == nullptr) return cudaErrorInvalidValue;
    k_dss_gather<<<vec_grid(L.N), kVecThreads, 0, s>>>(L.N, L.dss_ptr, L.dss_slot, L.map, masked ? 1 : 0, ye, y,
                                                        skip);
    return cudaGetLastError();
}

namespace {

constexpr int kTrEB = 8;

// Restriction (R = P^T): fine residual r = f - y weighted by 1/multiplicity,
// T[kf][nc] = sum_nf Bt[nf][nc] r[kf][nf], coarse[kc][nc] = sum_kf Bz[kf][kc] T[kf][nc],
// summed into the coarse right-hand side (free coarse rows).
template <typename T>
__global__ void k_restrict(int E, int NTf, int NZf, int NTc, int NZc, const int* __restrict__ mapf,
                           const int* __restrict__ mapc, const T* __restrict__ wmult, const T* __restrict__ Bt,
                           const T* __restrict__ Bz, const T* __restrict__ f, const T* __restrict__ y,
                           T* __restrict__ fc, T* __restrict__ yec) {
    extern __shared__ __align__(16) unsigned char smr[];
    const int Npf = NTf * NZf, Npc = NTc * NZc;
    T* sBt = reinterpret_cast<T*>(smr);
    T* sBz = sBt + NTf * NTc;
    T* re = sBz + NZf * NZc;                    // [EB][Npf]
    T* tt = re + kTrEB * Npf;                   // [EB][NZf][NTc]
    for (int i = threadIdx.x; i < NTf * NTc; i += blockDim.x) sBt[i] = Bt[i];
    for (int i = threadIdx.x; i < NZf * NZc; i += blockDim.x) sBz[i] = Bz[i];
    for (int e0 = blockIdx.x * kTrEB; e0 < E; e0 += gridDim.x * kTrEB) {
        const int nb = min(kTrEB, E - e0);
        __syncthreads();
        for (int i = threadIdx.x; i < nb * Npf; i += blockDim.x) {
            const int b = i / Npf, l = i - b * Npf;
            const int m = mapf[(size_t)(e0 + b) * Npf + l];
            re[b * Npf + l] = (m >= 0) ? wmult[m] * (f[m] - y[m]) : T(0);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb * NZf * NTc; i += blockDim.x) {
            const int b = i / (NZf * NTc), rem = i - b * NZf * NTc, kf = rem / NTc, nc = rem - kf * NTc;
            const T* rr = re + b * Npf + kf * NTf;
            T v = 0;
            for (int nf = 0; nf < NTf; ++nf) v += sBt[nf * NTc + nc] * rr[nf];
            tt[b * NZf * NTc + kf * NTc + nc] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb * Npc; i += blockDim.x) {
            const int b = i / Npc, c = i - b * Npc, kc = c / NTc, nc = c - kc * NTc;
            const int m = mapc[(size_t)(e0 + b) * Npc + c];
            if (m < 0) continue;
            T v = 0;
            for (int kf = 0; kf < NZf; ++kf) v += sBz[kf * NZc + kc] * tt[b * NZf * NTc + kf * NTc + nc];
            if (yec != nullptr) yec[(size_t)(e0 + b) * Npc + c] = v;    // summed by node afterwards
            else atomicAdd(&fc[m], v);
        }
    }
}

// Prolongation and correction: uf += P uc, each fine node written by its owner element.
// T[kc][nf] = sum_nc Bt[nf][nc] uc[kc][nc], fine[kf][nf] = sum_kc Bz[kf][kc] T[kc][nf].
template <typename T>
__global__ void k_prolong(int E, int NTf, int NZf, int NTc, int NZc, const int* __restrict__ mapf,
                          const int* __restrict__ mapc, const unsigned char* __restrict__ owner,
                          const T* __restrict__ Bt, const T* __restrict__ Bz, const T* __restrict__ uc,
                          T* __restrict__ uf) {
    extern __shared__ __align__(16) unsigned char smp[];
    const int Npf = NTf * NZf, Npc = NTc * NZc;
    T* sBt = reinterpret_cast<T*>(smp);
    T* sBz = sBt + NTf * NTc;
    T* ce = sBz + NZf * NZc;                    // [EB][Npc]
    T* tt = ce + kTrEB * Npc;                   // [EB][NZc][NTf]
    for (int i = threadIdx.x; i < NTf * NTc; i += blockDim.x) sBt[i] = Bt[i];
    for (int i = threadIdx.x; i < NZf * NZc; i += blockDim.x) sBz[i] = Bz[i];
    for (int e0 = blockIdx.x * kTrEB; e0 < E; e0 += gridDim.x * kTrEB) {
        const int nb = min(kTrEB, E - e0);
        __syncthreads();
        for (int i = threadIdx.x; i < nb * Npc; i += blockDim.x) {
            const int b = i / Npc, c = i - b * Npc;
            const int m = mapc[(size_t)(e0 + b) * Npc + c];
            ce[b * Npc + c] = (m >= 0) ? uc[m] : T(0);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb * NZc * NTf; i += blockDim.x) {
            const int b = i / (NZc * NTf), rem = i - b * NZc * NTf, kc = rem / NTf, nf = rem - kc * NTf;
            const T* cc = ce + b * Npc + kc * NTc;
            T v = 0;
            for (int nc = 0; nc < NTc; ++nc) v += sBt[nf * NTc + nc] * cc[nc];
            tt[b * NZc * NTf + kc * NTf + nf] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb * Npf; i += blockDim.x) {
            const int b = i / Npf, l = i - b * Npf, kf = l / NTf, nf = l - kf * NTf;
            if (!owner[(size_t)(e0 + b) * Npf + l]) continue;
            T v = 0;
            for (int kc = 0; kc < NZc; ++kc) v += sBz[kf * NZc + kc] * tt[b * NZc * NTf + kc * NTf + nf];
            uf[mapf[(size_t)(e0 + b) * Npf + l]] += v;
        }
    }
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed tree) of one value per thread; result in thread 0.
__device__ double block_sum(double v) {
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum(v);
    return v;
}

// Writes this block's NS partial sums; returns true in the block that finishes
// last, after which part[] holds every block's partials (read them in order).
template <int NS>
__device__ bool partials_done(const double* s, double* part, unsigned* counter) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        for (int k = 0; k < NS; ++k) part[(size_t)k * gridDim.x + blockIdx.x] = s[k];
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

template <int NS>
__device__ void final_sums(const double* part, double* out) {
    for (int k = 0; k < NS; ++k) {
        double v = 0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            v += ((volatile const double*)part)[(size_t)k * gridDim.x + b];
        v = block_sum(v);
        if (threadIdx.x == 0) out[k] = v;
        __syncthreads();
    }
}

// num / den computed once per block (FP64 division is a multi-instruction sequence on
// the FP64 pipe) and broadcast through shared memory.
__device__ __forceinline__ double block_ratio(const double* num, const double* den) {
    __shared__ double ratio;
    if (threadIdx.x == 0) ratio = (*num) / (*den);
    __syncthreads();
    return ratio;
}

__global__ void k_dot(long long n, const double* __restrict__ a, const double* __restrict__ b,
                      double* part, unsigned* counter, double* out) {
    double s = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += a[i] * b[i];
    double v[1] = {block_sum(s)};
    if (partials_done<1>(v, part, counter)) {
        double r[1];
        final_sums<1>(part, r);
        if (threadIdx.x == 0) { out[0] = r[0]; *counter = 0; }
    }
}

__global__ void k_residual(long long n, const double* __restrict__ f, const double* __restrict__ y,
                           double* __restrict__ r, double* part, unsigned* counter, double* out) {
    double s = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = f[i] - y[i];
        r[i] = v;
        s += v * v;
    }
    double v[1] = {block_sum(s)};
    if (partials_done<1>(v, part, counter)) {
        double rr[1];
        final_sums<1>(part, rr);
        if (threadIdx.x == 0) { out[0] = rr[0]; *counter = 0; }
    }
}

// PCG (Algorithm 3): alpha = delta / (p^T q); u += alpha p; r -= alpha q; rr = r^T r.
__global__ void k_pcg_update(long long n, const double* num, const double* den, const double* __restrict__ p,
                             const double* __restrict__ q, double* __restrict__ u, double* __restrict__ r,
                             double* part, unsigned* counter, double* out) {
    const double alpha = block_ratio(num, den);
    double s = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        u[i] += alpha * p[i];
        const double v = r[i] - alpha * q[i];
        r[i] = v;
        s += v * v;
    }
    double v[1] = {block_sum(s)};
    if (partials_done<1>(v, part, counter)) {
        double rr[1];
        final_sums<1>(part, rr);
        if (threadIdx.x == 0) { out[0] = rr[0]; *counter = 0; }
    }
}

__global__ void k_pcg_dir(long long n, const double* num, const double* den, const double* __restrict__ z,
                          double* __restrict__ p) {
    const double beta = block_ratio(num, den);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

// FP32 data, FP64 accumulation (inner PCG of the mixed-precision path)
// A thread's share of an FP32 dot product, summed without FP64 arithmetic per element (the FP64
// pipe of GB300 is a small fraction of the FP32 one): each product a b = p + e exactly (one FMA),
// p added to the running sum by Knuth's TwoSum, the errors into a compensation term; one
// conversion to FP64 per thread.  The result carries about the FP64 sum's accuracy.
struct Dot32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float d = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(d, e));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__global__ void k_dot32(long long n, const float* __restrict__ a, const float* __restrict__ b, double* part,
                        unsigned* counter, double* out) {
    Dot32 acc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc.add(a[i], b[i]);
    double v[1] = {block_sum(acc.value())};
    if (partials_done<1>(v, part, counter)) {
        double r[1];
        final_sums<1>(part, r);
        if (threadIdx.x == 0) { out[0] = r[0]; *counter = 0; }
    }
}

__global__ void k_pcg_update32(long long n, const double* num, const double* den, const float* __restrict__ p,
                               const float* __restrict__ q, float* __restrict__ u, float* __restrict__ r,
                               double* part, unsigned* counter, double* out) {
    const float alpha = (float)block_ratio(num, den);
    Dot32 acc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        u[i] += alpha * p[i];
        const float v = r[i] - alpha * q[i];
        r[i] = v;
        acc.add(v, v);
    }
    double v[1] = {block_sum(acc.value())};
    if (partials_done<1>(v, part, counter)) {
        double rr[1];
        final_sums<1>(part, rr);
        if (threadIdx.x == 0) { out[0] = rr[0]; *counter = 0; }
    }
}

__global__ void k_pcg_dir32(long long n, const double* num, const double* den, const float* __restrict__ z,
                            float* __restrict__ p) {
    const float beta = (float)block_ratio(num, den);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

// ------------------------------------------------------------------ coarse CG (FP64)
// Jacobi-preconditioned CG with every scalar on the device; all kernels are
// predicated on flags[F_CG_DONE] so that the host may launch several iterations
// ahead of the convergence test.
__global__ void k_cg_init(long long n, const double* __restrict__ b, const double* __restrict__ dinv,
                          double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                          double* __restrict__ p, double* part, unsigned* counter, double* scal, int* flags,
                          double rtol2) {
    double s[2] = {0, 0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double bi = b[i];
        const double zi = dinv[i] * bi;
        x[i] = 0;
        r[i] = bi;
        z[i] = zi;
        p[i] = zi;
        s[0] += bi * zi;
        s[1] += bi * bi;
    }
    double v[2] = {block_sum(s[0]), block_sum(s[1])};
    if (partials_done<2>(v, part, counter)) {
        double t[2];
        final_sums<2>(part, t);
        if (threadIdx.x == 0) {
            scal[S_CG_RHO] = t[0];
            scal[S_CG_RR] = t[1];
            scal[S_CG_TOL2] = rtol2 * t[1];
            flags[F_CG_DONE] = (t[1] <= rtol2 * t[1]) || (t[1] == 0.0);
            flags[F_CG_ITERS] = 0;
            *counter = 0;
        }
    }
}

__global__ void k_cg_pq(long long n, const double* __restrict__ p, const double* __restrict__ q, double* part,
                        unsigned* counter, double* scal, const int* flags) {
    if (flags[F_CG_DONE]) return;
    double s = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += p[i] * q[i];
    double v[1] = {block_sum(s)};
    if (partials_done<1>(v, part, counter)) {
        double t[1];
        final_sums<1>(part, t);
        if (threadIdx.x == 0) { scal[S_CG_PQ] = t[0]; *counter = 0; }
    }
}

__global__ void k_cg_update(long long n, const double* __restrict__ dinv, double* __restrict__ x,
                            double* __restrict__ r, double* __restrict__ z, const double* __restrict__ p,
                            const double* __restrict__ q, double* part, unsigned* counter, double* scal, int* flags) {
    if (flags[F_CG_DONE]) return;
    const double alpha = block_ratio(scal + S_CG_RHO, scal + S_CG_PQ);
    double s[2] = {0, 0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        const double zi = dinv[i] * ri;
        z[i] = zi;
        s[0] += ri * zi;
        s[1] += ri * ri;
    }
    double v[2] = {block_sum(s[0]), block_sum(s[1])};
    if (partials_done<2>(v, part, counter)) {
        double t[2];
        final_sums<2>(part, t);
        if (threadIdx.x == 0) {
            scal[S_CG_BETA] = t[0] / scal[S_CG_RHO];
            scal[S_CG_RHO] = t[0];
            scal[S_CG_RR] = t[1];
            flags[F_CG_ITERS] += 1;
            if (t[1] <= scal[S_CG_TOL2] || !(t[1] == t[1])) flags[F_CG_DONE] = 1;
            *counter = 0;
        }
    }
}

__global__ void k_cg_dir(long long n, const double* __restrict__ z, double* __restrict__ p, const double* scal,
                         const int* flags) {
    if (flags[F_CG_DONE]) return;
    const double beta = scal[S_CG_BETA];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

// ------------------------------------------------------------------ persistent coarse CG
// The whole Jacobi-preconditioned CG of the order-1 coarse level in one
// cooperative launch (all CTAs co-resident).  Phases are separated by a grid
// barrier whose waits are bounded: a CTA that waits longer than kBarrierSpins
// polls sets bar[2] (timeout) and every CTA leaves at the next check, so the
// host reads SEM_TIMEOUT instead of a hung GPU.  Reductions are deterministic:
// block partial sums, then every CTA sums the partials in the same order.
constexpr unsigned long long kBarrierTimeoutNs = 1000000000ULL;   // 1 s per barrier wait

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier for co-resident CTAs.  bar[0] counts the arrivals of the whole launch (it is
// zeroed before the launch), bar[2] is the timeout flag.  Each CTA counts its barriers
// (epoch); the k-th releases when bar[0] reaches k * expected (`expected` arrivals per
// barrier, gridDim.x in normal use), so an arrival is one fenced atomic and the release needs
// no reset and no generation word: the last arrival's own atomic is what the others see.
// A wait that runs out sets the flag and returns false; every other CTA then runs out on its
// own wait.
__device__ bool grid_barrier(unsigned* bar, unsigned expected, unsigned& epoch) {
    __shared__ int ok;
    __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        const unsigned target = epoch * expected;
        int good = 1;
        __threadfence();
        const unsigned old = atomicAdd(bar, 1u);
        if (old + 1 < target) {
            volatile unsigned* vcount = bar;
            const unsigned long long t0 = global_ns();
            while (*vcount < target) {
                if (global_ns() - t0 > kBarrierTimeoutNs) {
                    atomicExch(bar + 2, 1u);
                    good = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// sum of part[0..gridDim) in a fixed order; every CTA gets the same value
__device__ double grid_total(const double* part) {
    __shared__ double tot;
    if (threadIdx.x < 32) {
        double v = 0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) v += ((volatile const double*)part)[b];
        v = warp_sum(v);
        if (threadIdx.x == 0) tot = v;
    }
    __syncthreads();
    const double t = tot;
    __syncthreads();
    return t;
}

// Deterministic coarse assembly: CSR entry k sums its element entries ev[eidx[i]],
// i in [eptr[k], eptr[k+1]), in that fixed order.
__global__ void k_entry_sums(long long nnz, const int* __restrict__ eptr, const int* __restrict__ eidx,
                             const double* __restrict__ ev, double* __restrict__ vals) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int i = eptr[k]; i < eptr[k + 1]; ++i) v += ev[eidx[i]];
        vals[k] = v;
    }
}

// Element matrices of the coarsest level summed into its CSR matrix (free rows and
// columns only): A_e[i][j] = sum_q sum_ab gref[a][q][i] G_ab(q) gref[b][q][j];
// slot[e][i][j] is the CSR position of (map_i, map_j) or -1.  One thread per (e, i).
__global__ void k_coarse_assemble(int E, int dim, int Np, int Nq, const double* __restrict__ G,
                                  const double* __restrict__ gref, const int* __restrict__ slot,
                                  double* __restrict__ vals, double* __restrict__ ev) {
    const int nc = dim == 3 ? 6 : 3;
    const long long total = (long long)E * Np;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(t / Np), i = (int)(t - (long long)e * Np);
        const double* Ge = G + (size_t)e * nc * Nq;
        for (int j = 0; j < Np; ++j) {
            const int sl = slot[((size_t)e * Np + i) * Np + j];
            if (sl < 0) continue;
            double v = 0;
            for (int q = 0; q < Nq; ++q) {
                double gi[3], gj[3];
                for (int a = 0; a < dim; ++a) {
                    gi[a] = gref[(a * Nq + q) * Np + i];
                    gj[a] = gref[(a * Nq + q) * Np + j];
                }
                double g[3][3];
                if (dim == 3) {
                    g[0][0] = Ge[q]; g[0][1] = g[1][0] = Ge[Nq + q]; g[0][2] = g[2][0] = Ge[2 * Nq + q];
                    g[1][1] = Ge[3 * Nq + q]; g[1][2] = g[2][1] = Ge[4 * Nq + q]; g[2][2] = Ge[5 * Nq + q];
                } else {
                    g[0][0] = Ge[q]; g[0][1] = g[1][0] = Ge[Nq + q]; g[1][1] = Ge[2 * Nq + q];
                }
                for (int a = 0; a < dim; ++a)
                    for (int c = 0; c < dim; ++c) v += gi[a] * g[a][c] * gj[c];
            }
            if (ev != nullptr) ev[((size_t)e * Np + i) * Np + j] = v;    // summed per entry afterwards
            else atomicAdd(&vals[sl], v);
        }
    }
}

// Whole CG on the assembled coarse matrix; two grid barriers per iteration.  The search
// direction lives in two buffers that alternate: while forming q = A p the lane group that
// owns a row writes p_new(row) = z(row) + beta p_old(row), and every gathered entry of p
// is formed on the fly from z(c) = dinv(c) r(c) and p_old(c), so no barrier is needed
// between the direction update and the product.  The caller's z buffer is the second
// direction buffer (z itself is never stored).  Values written by other CTAs (r, p) are
// read through L2 (__ldcg).
__global__ void __launch_bounds__(512) k_coarse_cg(long long n, const int* __restrict__ rowptr,
                                                   const int* __restrict__ col, const double* __restrict__ vals,
                                                   const double* __restrict__ dinv, const double* __restrict__ b,
                                                   double* x, double* r, double* z, double* p, double* q,
                                                   double* part, unsigned* bar, double* scal, int* flags,
                                                   double rtol2, int imax, unsigned extra_arrivals) {
    const unsigned nb = gridDim.x;
    const unsigned expected = nb + extra_arrivals;   // extra_arrivals > 0 only in the timeout test
    unsigned epoch = 0;                               // grid barriers passed
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    double* p_old = p;        // direction of the previous iteration (zero before the first)
    double* p_new = z;
    double s0 = 0, s1 = 0;
    for (long long i = tid; i < n; i += stride) {
        const double bi = b[i];
        x[i] = 0;
        r[i] = bi;
        p_old[i] = 0;
        s0 += bi * dinv[i] * bi;
        s1 += bi * bi;
    }
    s0 = block_sum(s0);
    s1 = block_sum(s1);
    if (threadIdx.x == 0) { part[blockIdx.x] = s0; part[nb + blockIdx.x] = s1; }
    if (!grid_barrier(bar, expected, epoch)) return;
    double rho = grid_total(part);
    const double bb = grid_total(part + nb);
    const double tol2 = rtol2 * bb;
    int it = 0;
    double rr = bb;
    double beta = 0.0;
    __shared__ double s_alpha, s_beta;
    while (rr > tol2 && rr > 0.0 && it < imax) {
        // q = A p with 4 lanes per row; lane 0 of the group owns q[row], p_new[row] and the
        // row's share of p^T q.  The loop runs over warp-uniform groups of 8 rows (all 32
        // lanes reach the shuffles); lanes past the last row contribute zero.
        double pq = 0;
        const int l4 = threadIdx.x & 3;
        const long long rstride = stride >> 2;                  // multiple of 8 (blockDim % 32 == 0)
        for (long long rb = (tid >> 2) & ~7LL; rb < n; rb += rstride) {
            const long long row = rb + ((tid >> 2) & 7);
            const bool active = row < n;
            double v = 0;
            if (active) {
                const int k0 = rowptr[row], k1 = rowptr[row + 1];
                for (int k = k0 + l4; k < k1; k += 32) {    // up to 8 independent gathers per lane
                    int c[8];
                    double a[8], pv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int kk = k + 4 * u;
                        c[u] = (kk < k1) ? col[kk] : -1;
                        a[u] = (kk < k1) ? vals[kk] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        pv[u] = c[u] >= 0 ? dinv[c[u]] * __ldcg(r + c[u]) + beta * __ldcg(p_old + c[u]) : 0.0;
#pragma unroll
                    for (int u = 0; u < 8; ++u) v += a[u] * pv[u];
                }
            }
            v += __shfl_down_sync(0xffffffffu, v, 2, 4);
            v += __shfl_down_sync(0xffffffffu, v, 1, 4);
            if (active && l4 == 0) {
                const double pn = dinv[row] * __ldcg(r + row) + beta * __ldcg(p_old + row);
                p_new[row] = pn;
                q[row] = v;
                pq += pn * v;
            }
        }
        pq = block_sum(pq);
        if (threadIdx.x == 0) part[2 * nb + blockIdx.x] = pq;
        if (!grid_barrier(bar, expected, epoch)) return;
        {
            const double pq_all = grid_total(part + 2 * nb);
            if (threadIdx.x == 0) s_alpha = rho / pq_all;
            __syncthreads();
        }
        const double alpha = s_alpha;
        double t0 = 0, t1 = 0;
        for (long long i = tid; i < n; i += stride) {
            x[i] += alpha * __ldcg(p_new + i);                // p_new[i], q[i] written by another lane group
            const double ri = r[i] - alpha * __ldcg(q + i);
            r[i] = ri;
            t0 += ri * dinv[i] * ri;
            t1 += ri * ri;
        }
        t0 = block_sum(t0);
        t1 = block_sum(t1);
        if (threadIdx.x == 0) { part[blockIdx.x] = t0; part[nb + blockIdx.x] = t1; }
        if (!grid_barrier(bar, expected, epoch)) return;
        const double rho_new = grid_total(part);
        rr = grid_total(part + nb);
        if (threadIdx.x == 0) s_beta = rho_new / rho;
        __syncthreads();
        beta = s_beta;
        rho = rho_new;
        ++it;
        double* t = p_old;
        p_old = p_new;
        p_new = t;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        flags[F_CG_ITERS] = it;
        flags[F_CG_DONE] = (rr <= tol2 || rr == 0.0) ? 1 : 0;
        scal[S_CG_RR] = rr;
    }
}

// Block-Jacobi preconditioned CG on the assembled coarse matrix.  CTA b owns the free rows
// brows[bptr[b] .. bptr[b+1]) (a compact patch of the mesh, at most kBjMax rows) and holds in
// shared memory their rows of the matrix (a local CSR copy, at most nnzmax entries) and the
// inverse of their diagonal block in FP32 (symmetrised before rounding, so the
// preconditioner is an exactly symmetric positive definite matrix).  z = M r is then local
// to the CTA: r, q and the previous z of its rows stay in shared memory, and only z and the
// direction, which neighbouring rows read in the product, go through global memory (read
// through L2).  The direction is formed on the fly inside the product from two alternating
// buffers, as in k_coarse_cg, so an iteration has two grid barriers; the partial sums of a
// phase are reduced together.  beta takes the Polak-Ribiere form (r_new, z_new - z_old) /
// (r_old, z_old), which absorbs the FP32 rounding of the block products (Golub and Ye,
// "Inexact preconditioned conjugate gradient method with inner-outer iteration", 1999).
// Partial sums: part[b] (r, z), part[nb + b] (r, r), part[2 nb + b] (p, q), part[3 nb + b]
// (r, z_old).
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// z_k = sum_j inv[k][j] rf[j] for the CTA's nk rows, one warp per row; written to out[k]
__device__ void bj_block_product(const float* inv, const float* rf, int nk, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = wid; k < nk; k += nw) {
        float v = 0.f;
        for (int j = lane; j < nk; j += 32) v = fmaf(inv[k * kBjMax + j], rf[j], v);
        v = warp_sumf(v);
        if (lane == 0) out[k] = (double)v;
    }
}

// Block sums (fixed tree) of NV values per thread, of which only threads below nact hold any,
// written by thread 0 to part[o[i] * nb + b].  The warps past nact skip their shuffle sums:
// FP64 adds run on GB300's narrow FP64 pipe.
template <int NV>
__device__ void bj_partials(const double (&v)[NV], const int (&o)[NV], double* part, int nact) {
    __shared__ double ws[NV][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (nact + 31) >> 5;
    if (wid < nw) {
        double w[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) w[i] = warp_sum(v[i]);
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < NV; ++i) ws[i][wid] = w[i];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double u = lane < nw ? ws[i][lane] : 0.0;
            if (nw > 1) u = warp_sum(u);
            if (lane == 0) part[(size_t)o[i] * gridDim.x + blockIdx.x] = u;
        }
    }
}

// Totals of NV partial arrays part[o[i] * nb ...], summed in a fixed order; every CTA gets the
// same values
template <int NV>
__device__ void bj_totals(const double* part, const int (&o)[NV], double (&t)[NV]) {
    __shared__ double tot[NV];
    if (threadIdx.x < 32) {
        double v[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32)
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] += ((volatile const double*)part)[(size_t)o[i] * gridDim.x + b];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            v[i] = warp_sum(v[i]);
            if (threadIdx.x == 0) tot[i] = v[i];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) t[i] = tot[i];
    __syncthreads();
}

__global__ void __launch_bounds__(512) k_coarse_bjcg(long long n, const int* __restrict__ rowptr,
                                                     const int* __restrict__ col, const double* __restrict__ vals,
                                                     const int* __restrict__ bptr, const int* __restrict__ brows,
                                                     const float* __restrict__ binv, const int* __restrict__ blptr, const int* __restrict__ blidx,
                                                     int nnzmax, const double* __restrict__ b, double* x, double* zg,
                                                     double* pa,
                                                     double* pb, double* part, unsigned* bar, double* scal, int* flags,
                                                     double rtol2, int imax, unsigned extra_arrivals) {
    extern __shared__ __align__(16) unsigned char bj_smem[];
    float* inv = reinterpret_cast<float*>(bj_smem);                  // [kBjMax][kBjMax]
    double* rs = reinterpret_cast<double*>(inv + kBjMax * kBjMax);   // r of the CTA's rows
    double* zo = rs + kBjMax;                                        // z of the previous iteration
    double* qs = zo + kBjMax;                                        // q, then the new z
    double* pn = qs + kBjMax;                                        // the new direction
    double* lval = pn + kBjMax;                                      // [nnzmax] the rows' entries
    float* rf = reinterpret_cast<float*>(lval + nnzmax);             // r rounded to FP32
    int* rw = reinterpret_cast<int*>(rf + kBjMax);                   // global row ids
    int* lptr = rw + kBjMax;                                         // [kBjMax + 1] local row offsets
    int* lcol = lptr + kBjMax + 1;                                   // [nnzmax] global column ids
    const unsigned nb = gridDim.x;
    const unsigned expected = nb + extra_arrivals;   // extra_arrivals > 0 only in the timeout test
    unsigned epoch = 0;                               // grid barriers passed
    const int t = threadIdx.x;
    const int k0 = bptr[blockIdx.x], nk = bptr[blockIdx.x + 1] - k0;
    {
        const float4* src = reinterpret_cast<const float4*>(binv + (size_t)blockIdx.x * kBjMax * kBjMax);
        float4* dst = reinterpret_cast<float4*>(inv);
        for (int i = t; i < kBjMax * kBjMax / 4; i += blockDim.x) dst[i] = src[i];
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + t; i < n; i += (long long)gridDim.x * blockDim.x) x[i] = 0.0;
    double* p_old = pa;       // direction of the previous iteration (zero before the first)
    double* p_new = pb;
    if (t < nk) {
        const int row = brows[k0 + t];
        rw[t] = row;
        rs[t] = b[row];
        rf[t] = (float)rs[t];
        p_old[row] = 0.0;
    }
    if (t <= nk) lptr[t] = blptr[(size_t)blockIdx.x * (kBjMax + 1) + t];   // local row offsets
    __syncthreads();
    for (int e = t; e < lptr[nk]; e += blockDim.x) {      // the rows' entries, by their CSR positions
        const int g = blidx[(size_t)blockIdx.x * nnzmax + e];
        lcol[e] = col[g];
        lval[e] = vals[g];
    }
    bj_block_product(inv, rf, nk, zo);
    __syncthreads();
    {
        double v[2] = {0.0, 0.0};
        if (t < nk) {
            zg[rw[t]] = zo[t];
            v[0] = rs[t] * zo[t];
            v[1] = rs[t] * rs[t];
        }
        bj_partials<2>(v, {0, 1}, part, nk);
    }
    if (!grid_barrier(bar, expected, epoch)) return;
    double tt[2];
    bj_totals<2>(part, {0, 1}, tt);
    double rho = tt[0];
    const double bb = tt[1];
    const double tol2 = rtol2 * bb;
    int it = 0;
    double rr = bb;
    double beta = 0.0;
    while (rr > tol2 && rr > 0.0 && it < imax) {
        // q = A p for the CTA's rows, 4 lanes per row (blockDim = 4 kBjMax: one pass); p formed
        // on the fly from z and the previous direction
        double pq = 0;
        {
            const int k = t >> 2, l4 = t & 3;
            double v = 0;
            if (k < nk) {
                const int a1 = lptr[k + 1];
#pragma unroll 4
                for (int a = lptr[k] + l4; a < a1; a += 4) {
                    const int c = lcol[a];
                    v += lval[a] * (__ldcg(zg + c) + beta * __ldcg(p_old + c));
                }
            }
            v += __shfl_down_sync(0xffffffffu, v, 2, 4);
            v += __shfl_down_sync(0xffffffffu, v, 1, 4);
            if (k < nk && l4 == 0) {
                const int row = rw[k];
                const double pv = __ldcg(zg + row) + beta * __ldcg(p_old + row);
                p_new[row] = pv;
                pn[k] = pv;
                qs[k] = v;
                pq = pv * v;
            }
        }
        {
            const double v[1] = {pq};
            bj_partials<1>(v, {2}, part, 4 * nk);     // held by the lane groups of the rows
        }
        if (!grid_barrier(bar, expected, epoch)) return;
        double ta[1];
        bj_totals<1>(part, {2}, ta);
        const double alpha = rho / ta[0];
        if (t < nk) {
            x[rw[t]] += alpha * pn[t];
            rs[t] -= alpha * qs[t];
            rf[t] = (float)rs[t];
        }
        __syncthreads();
        bj_block_product(inv, rf, nk, qs);       // the new z, over q (no longer needed)
        __syncthreads();
        {
            double v[3] = {0.0, 0.0, 0.0};
            if (t < nk) {
                const double zn = qs[t];
                v[0] = rs[t] * zn;
                v[1] = rs[t] * rs[t];
                v[2] = rs[t] * zo[t];
                zg[rw[t]] = zn;
                zo[t] = zn;
            }
            bj_partials<3>(v, {0, 1, 3}, part, nk);
        }
        if (!grid_barrier(bar, expected, epoch)) return;
        double tb[3];
        bj_totals<3>(part, {0, 1, 3}, tb);
        rr = tb[1];
        beta = (tb[0] - tb[2]) / rho;
        rho = tb[0];
        ++it;
        double* tmp = p_old;
        p_old = p_new;
        p_new = tmp;
    }
    if (blockIdx.x == 0 && t == 0) {
        flags[F_CG_ITERS] = it;
        flags[F_CG_DONE] = (rr <= tol2 || rr == 0.0) ? 1 : 0;
        scal[S_CG_RR] = rr;
    }
}

// The same block-Jacobi CG in its pipelined form (Ghysels and Vanroose, "Hiding global
// synchronization latency in the preconditioned Conjugate Gradient algorithm", 2014): the
// recurrences for w = A u, m = M w, n = A m, z, q and s let the dot products of an iteration
// be reduced while the next product is formed, so an iteration has ONE grid barrier: read the
// totals, n = A m (m of the neighbouring rows from the other CTAs), update the CTA's rows,
// m = M w in shared memory, write m and the partial sums, barrier.  Only m goes through
// global memory (two alternating buffers ma / mb); every other vector of the CTA's rows
// stays in shared memory.  Its recurrences drift from the true residual by more rounding
// than the plain form's, so it serves loose coarse tolerances (coarse_rtol >= 1e-6).
// Partial sums of gamma = (r, u), (r, r) and delta = (w, u) in part[(o + i) nb + b], o = 0 and
// 3 alternating: a CTA writes a set again only after every CTA has passed the barrier that
// follows its reading of that set.
__global__ void __launch_bounds__(512) k_coarse_bjpcg(long long n, const int* __restrict__ rowptr,
                                                      const int* __restrict__ col, const double* __restrict__ vals,
                                                      const int* __restrict__ bptr, const int* __restrict__ brows,
                                                      const float* __restrict__ binv, const int* __restrict__ blptr, const int* __restrict__ blidx,
                                                      int nnzmax, const double* __restrict__ b, double* x, double* ma,
                                                      double* mb,
                                                      double* part, unsigned* bar, double* scal, int* flags,
                                                      double rtol2, int imax, unsigned extra_arrivals) {
    extern __shared__ __align__(16) unsigned char bj_smem[];
    float* inv = reinterpret_cast<float*>(bj_smem);                  // [kBjMax][kBjMax]
    double* vr = reinterpret_cast<double*>(inv + kBjMax * kBjMax);   // r, u, w, m, z, q, s, p of the rows
    double* vu = vr + kBjMax;
    double* vw = vu + kBjMax;
    double* vm = vw + kBjMax;
    double* vz = vm + kBjMax;
    double* vq = vz + kBjMax;
    double* vs = vq + kBjMax;
    double* vp = vs + kBjMax;
    double* sn = vp + kBjMax;                                        // n = A m
    double* lval = sn + kBjMax;                                      // [nnzmax] the rows' entries
    float* rf = reinterpret_cast<float*>(lval + nnzmax);             // block-product input in FP32
    int* rw = reinterpret_cast<int*>(rf + kBjMax);                   // global row ids
    int* lptr = rw + kBjMax;                                         // [kBjMax + 1] local row offsets
    int* lcol = lptr + kBjMax + 1;                                   // [nnzmax] global column ids
    const unsigned nb = gridDim.x;
    const unsigned expected = nb + extra_arrivals;   // extra_arrivals > 0 only in the timeout test
    unsigned epoch = 0;                               // grid barriers passed
    const int t = threadIdx.x;
    const int k0 = bptr[blockIdx.x], nk = bptr[blockIdx.x + 1] - k0;
    {
        const float4* src = reinterpret_cast<const float4*>(binv + (size_t)blockIdx.x * kBjMax * kBjMax);
        float4* dst = reinterpret_cast<float4*>(inv);
        for (int i = t; i < kBjMax * kBjMax / 4; i += blockDim.x) dst[i] = src[i];
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + t; i < n; i += (long long)gridDim.x * blockDim.x) x[i] = 0.0;
    if (t < nk) {
        const int row = brows[k0 + t];
        rw[t] = row;
        vr[t] = b[row];
        rf[t] = (float)vr[t];
        vz[t] = vq[t] = vs[t] = vp[t] = 0.0;
    }
    if (t <= nk) lptr[t] = blptr[(size_t)blockIdx.x * (kBjMax + 1) + t];   // local row offsets
    __syncthreads();
    for (int e = t; e < lptr[nk]; e += blockDim.x) {      // the rows' entries, by their CSR positions
        const int g = blidx[(size_t)blockIdx.x * nnzmax + e];
        lcol[e] = col[g];
        lval[e] = vals[g];
    }
    bj_block_product(inv, rf, nk, vu);           // u = M r
    __syncthreads();
    if (t < nk) ma[rw[t]] = vu[t];
    // out[k] = (A v)(row k) for the CTA's rows, v read from global memory, 4 lanes per row
    auto product = [&](const double* v, double* out) {
        const int k = t >> 2, l4 = t & 3;
        double a = 0;
        if (k < nk) {
            const int a1 = lptr[k + 1];
#pragma unroll 4
            for (int e = lptr[k] + l4; e < a1; e += 4) a += lval[e] * __ldcg(v + lcol[e]);
        }
        a += __shfl_down_sync(0xffffffffu, a, 2, 4);
        a += __shfl_down_sync(0xffffffffu, a, 1, 4);
        if (k < nk && l4 == 0) out[k] = a;
    };
    if (!grid_barrier(bar, expected, epoch)) return;
    product(ma, vw);                             // w = A u
    __syncthreads();
    if (t < nk) rf[t] = (float)vw[t];
    __syncthreads();
    bj_block_product(inv, rf, nk, vm);           // m = M w
    __syncthreads();
    double* mcur = mb;
    double* mnext = ma;
    {
        double v[3] = {0.0, 0.0, 0.0};
        if (t < nk) {
            mcur[rw[t]] = vm[t];
            v[0] = vr[t] * vu[t];
            v[1] = vr[t] * vr[t];
            v[2] = vw[t] * vu[t];
        }
        bj_partials<3>(v, {0, 1, 2}, part, nk);
    }
    if (!grid_barrier(bar, expected, epoch)) return;
    double tot[3];
    bj_totals<3>(part, {0, 1, 2}, tot);
    const double bb = tot[1];
    const double tol2 = rtol2 * bb;
    double rr = bb, gamma_old = 0.0, alpha_old = 1.0;
    int it = 0;
    while (rr > tol2 && rr > 0.0 && it < imax) {
        const double gamma = tot[0], delta = tot[2];
        const double beta = it > 0 ? gamma / gamma_old : 0.0;
        const double alpha = it > 0 ? gamma / (delta - beta * gamma / alpha_old) : gamma / delta;
        product(mcur, sn);                       // n = A m
        __syncthreads();
        if (t < nk) {
            vz[t] = sn[t] + beta * vz[t];
            vq[t] = vm[t] + beta * vq[t];
            vs[t] = vw[t] + beta * vs[t];
            vp[t] = vu[t] + beta * vp[t];
            x[rw[t]] += alpha * vp[t];
            vr[t] -= alpha * vs[t];
            vu[t] -= alpha * vq[t];
            vw[t] -= alpha * vz[t];
            rf[t] = (float)vw[t];
        }
        __syncthreads();
        bj_block_product(inv, rf, nk, vm);       // m = M w
        __syncthreads();
        {
            double v[3] = {0.0, 0.0, 0.0};
            if (t < nk) {
                mnext[rw[t]] = vm[t];
                v[0] = vr[t] * vu[t];
                v[1] = vr[t] * vr[t];
                v[2] = vw[t] * vu[t];
            }
            if (it & 1) bj_partials<3>(v, {0, 1, 2}, part, nk);
            else bj_partials<3>(v, {3, 4, 5}, part, nk);
        }
        if (!grid_barrier(bar, expected, epoch)) return;
        if (it & 1) bj_totals<3>(part, {0, 1, 2}, tot);
        else bj_totals<3>(part, {3, 4, 5}, tot);
        rr = tot[1];
        gamma_old = gamma;
        alpha_old = alpha;
        ++it;
        double* tmp = mcur;
        mcur = mnext;
        mnext = tmp;
    }
    if (blockIdx.x == 0 && t == 0) {
        flags[F_CG_ITERS] = it;
        flags[F_CG_DONE] = (rr <= tol2 || rr == 0.0) ? 1 : 0;
        scal[S_CG_RR] = rr;
    }
}

// Whole coarse CG in one CTA (no grid barrier, so any number of these may run
// concurrently and inside captured graphs): used for batched tanks and small
// coarse problems.  Global-memory writes of the CTA's threads are ordered by
// __syncthreads.
__device__ double block_allsum(double v) {
    __shared__ double bc;
    v = block_sum(v);
    if (threadIdx.x == 0) bc = v;
    __syncthreads();
    v = bc;
    __syncthreads();
    return v;
}

__global__ void __launch_bounds__(1024) k_coarse_cg_block(long long n, const int* __restrict__ rowptr,
                                                          const int* __restrict__ col,
                                                          const double* __restrict__ vals,
                                                          const double* __restrict__ dinv,
                                                          const double* __restrict__ b, double* x, double* r,
                                                          double* z, double* p, double* q, double* scal, int* flags,
                                                          double rtol2, int imax) {
    double s0 = 0, s1 = 0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const double bi = b[i], zi = dinv[i] * bi;
        x[i] = 0;
        r[i] = bi;
        z[i] = zi;
        p[i] = zi;
        s0 += bi * zi;
        s1 += bi * bi;
    }
    double rho = block_allsum(s0);
    const double bb = block_allsum(s1);
    const double tol2 = rtol2 * bb;
    double rr = bb;
    int it = 0;
    __shared__ double s_ratio;
    while (rr > tol2 && rr > 0.0 && it < imax) {
        double pq = 0;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            double v = 0;
            for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) v += vals[k] * p[col[k]];
            q[i] = v;
            pq += p[i] * v;
        }
        pq = block_allsum(pq);
        if (threadIdx.x == 0) s_ratio = rho / pq;
        __syncthreads();
        const double alpha = s_ratio;
        double t0 = 0, t1 = 0;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            x[i] += alpha * p[i];
            const double ri = r[i] - alpha * q[i];
            r[i] = ri;
            const double zi = dinv[i] * ri;
            z[i] = zi;
            t0 += ri * zi;
            t1 += ri * ri;
        }
        const double rho_new = block_allsum(t0);
        rr = block_allsum(t1);
        ++it;
        if (rr <= tol2) break;
        if (threadIdx.x == 0) s_ratio = rho_new / rho;
        __syncthreads();
        const double beta = s_ratio;
        rho = rho_new;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) p[i] = z[i] + beta * p[i];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        flags[F_CG_ITERS] = it;
        flags[F_CG_DONE] = (rr <= tol2 || rr == 0.0) ? 1 : 0;
        scal[S_CG_RR] = rr;
    }
}

// ------------------------------------------------------------------ FGMRES helpers
constexpr int kMaxMulti = 65;

__global__ void k_multidot(long long n, int k, const double* __restrict__ V, const double* __restrict__ w,
                           double* part, unsigned* counter, double* out) {
    __shared__ bool last;
    for (int j = 0; j < k; ++j) {
        double s = 0;
        const double* vj = V + (size_t)j * n;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
            s += vj[i] * w[i];
        s = block_sum(s);
        if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = s;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int j = 0; j < k; ++j) {
        double v = 0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            v += ((volatile const double*)part)[(size_t)j * gridDim.x + b];
        v = block_sum(v);
        if (threadIdx.x == 0) out[j] = v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *counter = 0;
}

__global__ void k_multiaxpy(long long n, int k, const double* __restrict__ V, const double* __restrict__ c,
                            double sign, double* __restrict__ w) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = 0;
        for (int j = 0; j < k; ++j) s += c[j] * V[(size_t)j * n + i];
        w[i] += sign * s;
    }
}

__global__ void k_scale(long long n, const double* __restrict__ w, const double* nrm2, double* __restrict__ v) {
    __shared__ double sinv;
    if (threadIdx.x == 0) sinv = 1.0 / sqrt(*nrm2);
    __syncthreads();
    const double inv = sinv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = w[i] * inv;
}

// ------------------------------------------------------------------ element-wise vector kernels
template <typename T>
__global__ void k_cheb_first(long long n, T c, const T* __restrict__ dinv, const T* __restrict__ f,
                             T* __restrict__ u, T* __restrict__ d, const int* __restrict__ skip) {
    if (skip != nullptr && *skip) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T v = c * dinv[i] * f[i];
        d[i] = v;
        u[i] = v;
    }
}

template <typename T>
__global__ void k_cheb_restart(long long n, T c, const T* __restrict__ dinv, const T* __restrict__ f,
                               const T* __restrict__ y, T* __restrict__ u, T* __restrict__ d,
                               const int* __restrict__ skip) {
    if (skip != nullptr && *skip) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T v = c * dinv[i] * (f[i] - y[i]);
        d[i] = v;
        u[i] += v;
    }
}

template <typename T>
__global__ void k_cheb_step(long long n, T c1, T c2, const T* __restrict__ dinv, const T* __restrict__ f,
                            const T* __restrict__ y, T* __restrict__ u, T* __restrict__ d,
                            const int* __restrict__ skip) {
    if (skip != nullptr && *skip) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T v = c1 * d[i] + c2 * dinv[i] * (f[i] - y[i]);
        d[i] = v;
        u[i] += v;
    }
}

__global__ void k_axpy(long long n, double a, const double* __restrict__ x, double* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

template <typename T>
__global__ void k_copy_idx(long long nd, const long long* __restrict__ idx, const T* __restrict__ src,
                           T* __restrict__ dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nd; i += (long long)gridDim.x * blockDim.x)
        dst[idx[i]] = src[idx[i]];
}

__global__ void k_scatter_idx(long long nd, const long long* __restrict__ idx, const double* __restrict__ vals,
                              double* __restrict__ dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nd; i += (long long)gridDim.x * blockDim.x)
        dst[idx[i]] = vals[i];
}

__global__ void k_zero_idx(long long nd, const long long* __restrict__ idx, double* __restrict__ v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nd; i += (long long)gridDim.x * blockDim.x)
        v[idx[i]] = 0.0;
}

__global__ void k_to_f32(long long n, const double* __restrict__ a, float* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

__global__ void k_to_f64(long long n, const float* __restrict__ a, double* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

}  // namespace

// ====================================================================== launchers
// Largest grid of the reduction kernels (their partial-sum arrays are sized for it); a launch
// takes about four elements per thread, so that a stream of several vectors keeps enough loads
// in flight for HBM.
int reduce_blocks() { return 8 * kSMs; }
static int red_grid(long long n) {
    const long long g = (n + 4LL * kRedThreads - 1) / (4LL * kRedThreads);
    return (int)std::max<long long>(1, std::min<long long>(g, reduce_blocks()));
}

cudaError_t launch_apply64(const Level& L, const double* x, double* y, bool lift, const int* skip, cudaStream_t s) {
    if (L.dim == 3) return launch_apply_prism64(L, x, y, lift, skip, L.tile64, s);
    return lift ? apply_dispatch<double, true>(L, L.ref64.m, L.G, x, y, skip, s)
                : apply_dispatch<double, false>(L, L.ref64.m, L.G, x, y, skip, s);
}

cudaError_t launch_apply32(const Level& L, const float* x, float* y, cudaStream_t s, const int* skip) {
    if (L.dim == 3) return launch_apply_prism32(L, x, y, skip, L.tile32, s);
    return apply_dispatch<float, false>(L, L.ref32.m, L.G32, x, y, skip, s);
}

cudaError_t launch_geometry(Level& L, const double* vtri, const double* etaP, const double* BP, const double* DrP,
                            const double* DsP, int NTP, int nlayers, double depth, cudaStream_t s) {
    // quadrature info: [tw (QT) | zq (QZ) | zw (QZ)]
    std::vector<double> qi(L.ref.tw);
    qi.insert(qi.end(), L.ref.zq.begin(), L.ref.zq.end());
    qi.insert(qi.end(), L.ref.zw.begin(), L.ref.zw.end());
    double* dq = nullptr;
    cudaError_t err = cudaMalloc(&dq, qi.size() * sizeof(double));
    if (err != cudaSuccess) return err;
    err = cudaMemcpyAsync(dq, qi.data(), qi.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) {
        const long long total = (long long)L.E * L.Nq;
        const int grid = (int)std::min<long long>((total + 255) / 256, kSMs * 32);
        if (L.dim == 3)
            k_geom_prism<<<grid, 256, 0, s>>>(L.E, nlayers, L.QT, L.QZ, NTP, depth, vtri, etaP, BP, DrP, DsP, dq, L.G,
                                              L.G32);
        else
            k_geom_tri<<<grid, 256, 0, s>>>(L.E, L.QT, vtri, dq, L.G, L.G32);
        err = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(dq);
    return err != cudaSuccess ? err : e2;
}

cudaError_t launch_geometry_general(Level& L, const int* eb, const int* el, const double* xyP, const double* etaP,
                                    const double* zif, const double* BP, const double* DrP, const double* DsP,
                                    int NTP, cudaStream_t s) {
    std::vector<double> qi(L.ref.tw);
    qi.insert(qi.end(), L.ref.zq.begin(), L.ref.zq.end());
    qi.insert(qi.end(), L.ref.zw.begin(), L.ref.zw.end());
    double* dq = nullptr;
    cudaError_t err = cudaMalloc(&dq, qi.size() * sizeof(double));
    if (err != cudaSuccess) return err;
    err = cudaMemcpyAsync(dq, qi.data(), qi.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) {
        const long long total = (long long)L.E * L.Nq;
        const int grid = (int)std::min<long long>((total + 255) / 256, kSMs * 32);
        k_geom_prism_general<<<grid, 256, 0, s>>>(L.E, eb, el, L.QT, L.QZ, NTP, xyP, etaP, zif, BP, DrP, DsP, dq,
                                                  L.G, L.G32);
        err = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(dq);
    return err != cudaSuccess ? err : e2;
}

cudaError_t launch_diag(const Level& L, double* diag, cudaStream_t s) {
    const size_t smem = sizeof(double) * 6 * L.NT * L.QZ;
    const int grid = std::min(L.E, kSMs * 8);
    k_diag<<<grid, 128, smem, s>>>(L.E, L.dim, L.NT, L.NZ, L.QT, L.QZ, L.map, L.G, L.ref64.m, diag, L.ye64);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || L.ye64 == nullptr) return e;
    return dss_gather64(L, L.ye64, diag, nullptr, s, false);
}

template <typename T>
static cudaError_t restrict_t(const Level& F, const Level& C, const T* wm, const T* Bt, const T* Bz, const T* f,
                              const T* y, T* fc, cudaStream_t s) {
    const int grid = std::min((F.E + kTrEB - 1) / kTrEB, kSMs * 8);
    const size_t smem = sizeof(T) * (F.NT * C.NT + F.NZ * C.NZ + kTrEB * (F.Np + F.NZ * C.NT));
    T* yec = nullptr;
    if constexpr (sizeof(T) == sizeof(double)) yec = C.ye64;
    k_restrict<T><<<grid, 256, smem, s>>>(F.E, F.NT, F.NZ, C.NT, C.NZ, F.map, C.map, wm, Bt, Bz, f, y, fc, yec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || yec == nullptr) return e;
    if constexpr (sizeof(T) == sizeof(double)) return dss_gather64(C, C.ye64, fc, nullptr, s, true);
    return e;
}

template <typename T>
static cudaError_t prolong_t(const Level& F, const Level& C, const T* Bt, const T* Bz, const T* uc, T* uf,
                             cudaStream_t s) {
    const int grid = std::min((F.E + kTrEB - 1) / kTrEB, kSMs * 8);
    const size_t smem = sizeof(T) * (F.NT * C.NT + F.NZ * C.NZ + kTrEB * (C.Np + C.NZ * F.NT));
    k_prolong<T><<<grid, 256, smem, s>>>(F.E, F.NT, F.NZ, C.NT, C.NZ, F.map, C.map, F.owner, Bt, Bz, uc, uf);
    return cudaGetLastError();
}

cudaError_t launch_restrict64(const Level& F, const Level& C, const double* f, const double* y, double* fc,
                              cudaStream_t s) {
    return restrict_t<double>(F, C, F.wmult, F.It64, F.Iz64, f, y, fc, s);
}
cudaError_t launch_restrict32(const Level& F, const Level& C, const float* f, const float* y, float* fc,
                              cudaStream_t s) {
    return restrict_t<float>(F, C, F.wmult32, F.It32, F.Iz32, f, y, fc, s);
}
cudaError_t launch_prolong64(const Level& F, const Level& C, const double* uc, double* uf, cudaStream_t s) {
    return prolong_t<double>(F, C, F.It64, F.Iz64, uc, uf, s);
}
cudaError_t launch_prolong32(const Level& F, const Level& C, const float* uc, float* uf, cudaStream_t s) {
    return prolong_t<float>(F, C, F.It32, F.Iz32, uc, uf, s);
}

template <typename T>
cudaError_t cheb_first(long long n, T c, const T* dinv, const T* f, T* u, T* d, cudaStream_t s, const int* skip) {
    k_cheb_first<T><<<vec_grid(n), kVecThreads, 0, s>>>(n, c, dinv, f, u, d, skip);
    return cudaGetLastError();
}
template <typename T>
cudaError_t cheb_restart(long long n, T c, const T* dinv, const T* f, const T* y, T* u, T* d, cudaStream_t s,
                         const int* skip) {
    k_cheb_restart<T><<<vec_grid(n), kVecThreads, 0, s>>>(n, c, dinv, f, y, u, d, skip);
    return cudaGetLastError();
}
template <typename T>
cudaError_t cheb_step(long long n, T c1, T c2, const T* dinv, const T* f, const T* y, T* u, T* d, cudaStream_t s,
                      const int* skip) {
    k_cheb_step<T><<<vec_grid(n), kVecThreads, 0, s>>>(n, c1, c2, dinv, f, y, u, d, skip);
    return cudaGetLastError();
}
template cudaError_t cheb_first<double>(long long, double, const double*, const double*, double*, double*, cudaStream_t,
                                        const int*);
template cudaError_t cheb_first<float>(long long, float, const float*, const float*, float*, float*, cudaStream_t,
                                       const int*);
template cudaError_t cheb_restart<double>(long long, double, const double*, const double*, const double*, double*,
                                          double*, cudaStream_t, const int*);
template cudaError_t cheb_restart<float>(long long, float, const float*, const float*, const float*, float*, float*,
                                         cudaStream_t, const int*);
template cudaError_t cheb_step<double>(long long, double, double, const double*, const double*, const double*,
                                       double*, double*, cudaStream_t, const int*);
template cudaError_t cheb_step<float>(long long, float, float, const float*, const float*, const float*, float*,
                                      float*, cudaStream_t, const int*);

cudaError_t dot64(long long n, const double* a, const double* b, Scratch& sc, double* out, cudaStream_t s) {
    k_dot<<<red_grid(n), kRedThreads, 0, s>>>(n, a, b, sc.part, sc.counter, out);
    return cudaGetLastError();
}
__global__ void k_batch_loop(double* scal, int* flags, double rtol, double atol, int imax,
                             cudaGraphConditionalHandle cond, int init) {
    const double ff = scal[S_FF];
    const double thr = rtol * sqrt(ff) + atol;
    int it = flags[F_BATCH_ITERS];
    double rr = ff;
    if (init) {
        it = 0;
    } else {
        rr = scal[S_RR];
        it += 1;
    }
    flags[F_BATCH_ITERS] = it;
    const bool finite = isfinite(rr);
    const bool met = finite && rr <= thr * thr;
    const bool more = finite && !met && it < imax;
    flags[F_BATCH_STATUS] = !finite ? -4 : (met ? 0 : 1);
    cudaGraphSetConditional(cond, more ? 1u : 0u);
}

cudaError_t batch_loop_init(double* scal, int* flags, double rtol, double atol, int imax,
                            cudaGraphConditionalHandle cond, cudaStream_t s) {
    k_batch_loop<<<1, 1, 0, s>>>(scal, flags, rtol, atol, imax, cond, 1);
    return cudaGetLastError();
}
cudaError_t batch_loop_check(double* scal, int* flags, double rtol, double atol, int imax,
                             cudaGraphConditionalHandle cond, cudaStream_t s) {
    k_batch_loop<<<1, 1, 0, s>>>(scal, flags, rtol, atol, imax, cond, 0);
    return cudaGetLastError();
}

cudaError_t residual64(long long n, const double* f, const double* y, double* r, Scratch& sc, double* rr,
                       cudaStream_t s) {
    k_residual<<<red_grid(n), kRedThreads, 0, s>>>(n, f, y, r, sc.part, sc.counter, rr);
    return cudaGetLastError();
}
cudaError_t pcg_update(long long n, const double* num, const double* den, const double* p, const double* q, double* u,
                       double* r, Scratch& sc, double* rr, cudaStream_t s) {
    k_pcg_update<<<red_grid(n), kRedThreads, 0, s>>>(n, num, den, p, q, u, r, sc.part, sc.counter, rr);
    return cudaGetLastError();
}
cudaError_t pcg_direction(long long n, const double* num, const double* den, const double* z, double* p,
                          cudaStream_t s) {
    k_pcg_dir<<<vec_grid(n), kVecThreads, 0, s>>>(n, num, den, z, p);
    return cudaGetLastError();
}
cudaError_t dot32(long long n, const float* a, const float* b, Scratch& sc, double* out, cudaStream_t s) {
    k_dot32<<<red_grid(n), kRedThreads, 0, s>>>(n, a, b, sc.part, sc.counter, out);
    return cudaGetLastError();
}
cudaError_t pcg_update32(long long n, const double* num, const double* den, const float* p, const float* q, float* u,
                         float* r, Scratch& sc, double* rr, cudaStream_t s) {
    k_pcg_update32<<<red_grid(n), kRedThreads, 0, s>>>(n, num, den, p, q, u, r, sc.part, sc.counter, rr);
    return cudaGetLastError();
}
cudaError_t pcg_direction32(long long n, const double* num, const double* den, const float* z, float* p,
                            cudaStream_t s) {
    k_pcg_dir32<<<vec_grid(n), kVecThreads, 0, s>>>(n, num, den, z, p);
    return cudaGetLastError();
}
cudaError_t axpy64(long long n, double a, const double* x, double* y, cudaStream_t s) {
    k_axpy<<<vec_grid(n), kVecThreads, 0, s>>>(n, a, x, y);
    return cudaGetLastError();
}
cudaError_t copy_dirichlet(long long nd, const long long* idx, const double* src, double* dst, cudaStream_t s) {
    if (nd <= 0) return cudaSuccess;
    k_copy_idx<double><<<vec_grid(nd), kVecThreads, 0, s>>>(nd, idx, src, dst);
    return cudaGetLastError();
}
cudaError_t copy_dirichlet32(long long nd, const long long* idx, const float* src, float* dst, cudaStream_t s) {
    if (nd <= 0) return cudaSuccess;
    k_copy_idx<float><<<vec_grid(nd), kVecThreads, 0, s>>>(nd, idx, src, dst);
    return cudaGetLastError();
}
cudaError_t scatter_dirichlet(long long nd, const long long* idx, const double* vals, double* dst, cudaStream_t s) {
    if (nd <= 0) return cudaSuccess;
    k_scatter_idx<<<vec_grid(nd), kVecThreads, 0, s>>>(nd, idx, vals, dst);
    return cudaGetLastError();
}
cudaError_t zero_dirichlet(long long nd, const long long* idx, double* v, cudaStream_t s) {
    if (nd <= 0) return cudaSuccess;
    k_zero_idx<<<vec_grid(nd), kVecThreads, 0, s>>>(nd, idx, v);
    return cudaGetLastError();
}
cudaError_t to_f32(long long n, const double* a, float* b, cudaStream_t s) {
    k_to_f32<<<vec_grid(n), kVecThreads, 0, s>>>(n, a, b);
    return cudaGetLastError();
}
cudaError_t to_f64(long long n, const float* a, double* b, cudaStream_t s) {
    k_to_f64<<<vec_grid(n), kVecThreads, 0, s>>>(n, a, b);
    return cudaGetLastError();
}
cudaError_t multidot64(long long n, int k, const double* V, const double* w, Scratch& sc, double* out, cudaStream_t s) {
    if (k > kMaxMulti) return cudaErrorInvalidValue;
    k_multidot<<<red_grid(n), kRedThreads, 0, s>>>(n, k, V, w, sc.part, sc.counter, out);
    return cudaGetLastError();
}
cudaError_t multiaxpy64(long long n, int k, const double* V, const double* c, double sign, double* w, cudaStream_t s) {
    k_multiaxpy<<<vec_grid(n), kVecThreads, 0, s>>>(n, k, V, c, sign, w);
    return cudaGetLastError();
}
cudaError_t scale64(long long n, const double* w, const double* nrm2, double* v, cudaStream_t s) {
    k_scale<<<vec_grid(n), kVecThreads, 0, s>>>(n, w, nrm2, v);
    return cudaGetLastError();
}
cudaError_t coarse_assemble(const Level& C, const double* gref, const int* slot, double* vals, cudaStream_t s) {
    const long long total = (long long)C.E * C.Np;
    const int grid = (int)std::min<long long>((total + 255) / 256, kSMs * 16);
    k_coarse_assemble<<<grid, 256, 0, s>>>(C.E, C.dim, C.Np, C.Nq, C.G, gref, slot, vals, C.csr_ev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || C.csr_ev == nullptr) return e;
    k_entry_sums<<<vec_grid(C.csr_nnz), kVecThreads, 0, s>>>(C.csr_nnz, C.csr_eptr, C.csr_eidx, C.csr_ev, vals);
    return cudaGetLastError();
}

cudaError_t coarse_cg_persistent(const Level& C, const int* rowptr, const int* col, const double* vals,
                                 const double* b, double* x, double* r, double* z, double* p, double* q, Scratch& sc,
                                 double rtol2, int imax, unsigned extra_arrivals, cudaStream_t s) {
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_cg, 512, 0);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    int dev = 0, sms = kSMs;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one CTA per SM at most (fewer participants make the grid barrier cheaper);
    // the SpMV uses 4 lanes per row, so 128 rows per CTA
    int grid = (int)std::min<long long>((C.N + 127) / 128, (long long)sms);
    if (grid < 1) grid = 1;
    err = cudaMemsetAsync(sc.counter + 1, 0, 3 * sizeof(unsigned), s);
    if (err != cudaSuccess) return err;
    long long n = C.N;
    const double* dinv = C.dinv;
    double* part = sc.part;
    unsigned* bar = sc.counter + 1;
    double* scal = sc.scal;
    int* flags = sc.flags;
    void* args[] = {&n,    &rowptr, &col,  &vals,  &dinv,  &b,     &x,    &r,   &z,
                    &p,    &q,      &part, &bar,   &scal,  &flags, &rtol2, &imax, &extra_arrivals};
    err = cudaLaunchCooperativeKernel((void*)k_coarse_cg, grid, 512, args, 0, s);
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

// shared memory of the block-Jacobi CG kernels (the pipelined one keeps 9 vectors of its rows,
// the plain one 4)
size_t coarse_bj_smem(int nnzmax, bool pipelined = true) {
    return sizeof(float) * kBjMax * kBjMax + sizeof(double) * ((pipelined ? 9 : 4) * kBjMax + nnzmax) +
           sizeof(float) * kBjMax + sizeof(int) * (2 * kBjMax + 1 + nnzmax);
}

// Largest number of blocks the block-Jacobi CG can take (all CTAs co-resident) when no block
// holds more than nnzmax matrix entries, 0 if none.
int coarse_bj_capacity(int nnzmax) {
    const size_t smem = coarse_bj_smem(nnzmax);
    if (smem > 200 * 1024) return 0;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_coarse_bjcg, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess ||
            cudaFuncSetAttribute(k_coarse_bjpcg, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
            return 0;
        attr = true;
    }
    int per_sm = 0, per_sm2 = 0, dev = 0, sms = kSMs;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_bjcg, 4 * kBjMax, coarse_bj_smem(nnzmax, false)) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_coarse_bjpcg, 4 * kBjMax, smem) != cudaSuccess)
        return 0;
    per_sm = std::min(per_sm, per_sm2);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * sms;
}

cudaError_t coarse_cg_bj(const Level& C, const double* b, double* x, double* z, double* pa, double* pb, Scratch& sc,
                         double rtol2, int imax, unsigned extra_arrivals, cudaStream_t s) {
    const int grid = C.bj_nb;
    int nnzmax = C.bj_nnzmax;
    if (grid < 1 || grid > coarse_bj_capacity(nnzmax)) return cudaErrorCooperativeLaunchTooLarge;
    cudaError_t err = cudaMemsetAsync(sc.counter + 1, 0, 3 * sizeof(unsigned), s);
    if (err != cudaSuccess) return err;
    long long n = C.N;
    const int* rowptr = C.csr_rowptr;
    const int* col = C.csr_col;
    const double* vals = C.csr_val;
    const int* bptr = C.bj_ptr;
    const int* brows = C.bj_rows;
    const float* binv = C.bj_inv;
    const int* blptr = C.bj_lptr;
    const int* blidx = C.bj_lidx;
    double* part = sc.part;
    unsigned* bar = sc.counter + 1;
    double* scal = sc.scal;
    int* flags = sc.flags;
    // loose tolerances (>= 1e-6): the pipelined form, one grid barrier per iteration
    const bool pipelined = rtol2 >= 1e-12;
    if (pipelined) {
        void* args[] = {&n,  &rowptr, &col,  &vals, &bptr, &brows, &binv,  &blptr, &blidx, &nnzmax, &b,
                        &x,  &pa,     &pb,   &part, &bar,  &scal,  &flags, &rtol2, &imax,   &extra_arrivals};
        err = cudaLaunchCooperativeKernel((void*)k_coarse_bjpcg, grid, 4 * kBjMax, args, coarse_bj_smem(nnzmax, true), s);
        if (err != cudaSuccess) return err;
        return cudaGetLastError();
    }
    void* args[] = {&n, &rowptr, &col, &vals, &bptr,  &brows, &binv,  &blptr, &blidx, &nnzmax, &b,  &x,
                    &z, &pa,     &pb,  &part, &bar,   &scal,  &flags, &rtol2, &imax,   &extra_arrivals};
    err = cudaLaunchCooperativeKernel((void*)k_coarse_bjcg, grid, 4 * kBjMax, args, coarse_bj_smem(nnzmax, false), s);
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

cudaError_t coarse_cg_single(const Level& C, const int* rowptr, const int* col, const double* vals, const double* b,
                             double* x, double* r, double* z, double* p, double* q, Scratch& sc, double rtol2, int imax,
                             cudaStream_t s) {
    k_coarse_cg_block<<<1, 1024, 0, s>>>(C.N, rowptr, col, vals, C.dinv, b, x, r, z, p, q, sc.scal, sc.flags, rtol2,
                                         imax);
    return cudaGetLastError();
}

cudaError_t cg_init(long long n, const double* b, const double* dinv, double* x, double* r, double* z, double* p,
                    Scratch& sc, double rtol2, cudaStream_t s) {
    k_cg_init<<<red_grid(n), kRedThreads, 0, s>>>(n, b, dinv, x, r, z, p, sc.part, sc.counter, sc.scal, sc.flags,
                                                       rtol2);
    return cudaGetLastError();
}
cudaError_t cg_pq(long long n, const double* p, const double* q, Scratch& sc, cudaStream_t s) {
    k_cg_pq<<<red_grid(n), kRedThreads, 0, s>>>(n, p, q, sc.part, sc.counter, sc.scal, sc.flags);
    return cudaGetLastError();
}
cudaError_t cg_update(long long n, const double* dinv, double* x, double* r, double* z, const double* p,
                      const double* q, Scratch& sc, cudaStream_t s) {
    k_cg_update<<<red_grid(n), kRedThreads, 0, s>>>(n, dinv, x, r, z, p, q, sc.part, sc.counter, sc.scal,
                                                         sc.flags);
    return cudaGetLastError();
}
cudaError_t cg_direction(long long n, const double* z, double* p, Scratch& sc, cudaStream_t s) {
    k_cg_dir<<<vec_grid(n), kVecThreads, 0, s>>>(n, z, p, sc.scal, sc.flags);
    return cudaGetLastError();
}


// ====================================================================== FP64 pipe rate
// Sixteen independent fused multiply-add chains per thread on every SM: the FP64 rate the
// device reaches on plain dependent-free arithmetic, the denominator of the FP64 apply's
// roofline.
template <int kFmaChains>
__global__ void k_fp64_fma_chains(int iters, double seed, double* sink) {
    double a[kFmaChains];
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) a[j] = seed + 1e-3 * (threadIdx.x + j);
    const double m = 0.9999999, c = 1e-9;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kFmaChains; ++j) a[j] = fma(a[j], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) s += a[j];
    if (s == 12345.678) sink[0] = s;          // never true: keeps the chains alive
}

}  // namespace sem

namespace {
// one timed launch of the chain kernel with `chains` independent FMA chains per thread
template <int chains>
cudaError_t fp64_rate_run(int blocks, int threads, int iters, double* tflops) {
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    float ms = 0.f;
    if (err == cudaSuccess) {
        sem::k_fp64_fma_chains<chains><<<blocks, threads>>>(iters / 8, 1.0, nullptr);      // warm-up
        err = cudaEventRecord(e0, 0);
    }
    if (err == cudaSuccess) {
        sem::k_fp64_fma_chains<chains><<<blocks, threads>>>(iters, 1.0, nullptr);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err == cudaSuccess && !(ms > 0.f)) err = cudaErrorUnknown;
    if (err == cudaSuccess) *tflops = 2.0 * chains * iters * (double)threads * blocks / (ms * 1e-3) / 1e12;
    return err;
}
}  // namespace

// The best of three shapes (8, 16 and 24 independent chains per thread, as many threads as fit):
// the FP64 pipe's rate on this device as a roofline denominator beside the nominal one.
extern "C" sem_status sem_fp64_rate(double* tflops_host) {
    using namespace sem;
    if (!tflops_host) {
        set_error("sem_fp64_rate: NULL result");
        return SEM_EINVAL;
    }
    int dev = 0, sms = kSMs;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256, blocks = 8 * sms, iters = 1 << 13;
    double r8 = 0, r16 = 0, r24 = 0;
    cudaError_t err = fp64_rate_run<8>(blocks, threads, 2 * iters, &r8);
    if (err == cudaSuccess) err = fp64_rate_run<16>(blocks, threads, iters, &r16);
    if (err == cudaSuccess) err = fp64_rate_run<24>(blocks, threads, iters, &r24);
    if (err != cudaSuccess) {
        set_error(std::string("sem_fp64_rate: ") + cudaGetErrorString(err));
        return SEM_ECUDA;
    }
    *tflops_host = std::max(r8, std::max(r16, r24));
    return SEM_OK;
}

namespace sem {

// ====================================================================== no-allocation CG
// A variant of the coarse CG launch for callers that cannot allocate device
// memory: the CG vectors r, z, p, q, the reduction partials, the barrier state
// and the result flags live in one file-scope device array instead of
// handle-owned workspaces.  Every GPU that loads the library holds the array
// until the process exits.  All calls share it and it keeps the last call's
// contents, so calls that overlap on the GPU race; the barrier state and the
// flags are cleared at the start of every call.
namespace {

constexpr long long kNoAllocMaxRows = 1LL << 17;          // 131,072 rows
constexpr long long kNoAllocPart = 1024;                  // >= 3 x (CTAs of one launch)
constexpr size_t kNoAllocBytes = sizeof(double) * (4 * kNoAllocMaxRows + kNoAllocPart + 32) + 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
unsigned char* g_noalloc_ptr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mutex;

// Device address of the scratch array on the current device (looked up once per device,
// with that device current).
cudaError_t noalloc_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_ptr[dev] == nullptr) {
        void* ptr = nullptr;
        err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (err != cudaSuccess) return err;
        g_noalloc_ptr[dev] = static_cast<unsigned char*>(ptr);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace sem

extern "C" sem_status sem_cg_csr_noalloc(long long n, const int* rowptr, const int* col, const double* vals,
                                         const double* dinv, const double* b, double* x, double rtol, int imax,
                                         int* iters_host, void* stream) {
    using namespace sem;
    if (n < 1 || n > kNoAllocMaxRows) {
        set_error("sem_cg_csr_noalloc: n must be in 1.." + std::to_string(kNoAllocMaxRows) +
                  " (the size of the library's static scratch)");
        return SEM_EINVAL;
    }
    if (!rowptr || !col || !vals || !dinv || !b || !x || !(rtol > 0.0) || imax < 0) {
        set_error("sem_cg_csr_noalloc: bad arguments");
        return SEM_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    cudaError_t err = noalloc_scratch(&base);
    if (err != cudaSuccess) {
        set_error(std::string("sem_cg_csr_noalloc: ") + cudaGetErrorString(err));
        return SEM_ECUDA;
    }
    double* r = reinterpret_cast<double*>(base);
    double* z = r + kNoAllocMaxRows;
    double* p = z + kNoAllocMaxRows;
    double* q = p + kNoAllocMaxRows;
    double* part = q + kNoAllocMaxRows;
    double* scal = part + kNoAllocPart;
    int* flags = reinterpret_cast<int*>(scal + 32);
    unsigned* bar = reinterpret_cast<unsigned*>(flags + 8);
    int per_sm = 0, dev = 0, sms = kSMs;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_cg, 512, 0);
    if (err == cudaSuccess && per_sm < 1) err = cudaErrorCooperativeLaunchTooLarge;
    // one CTA per SM at most, and never more CTAs than the partial-sum slots hold (three per CTA)
    const long long cap = std::min<long long>((long long)sms, kNoAllocPart / 3);
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + 127) / 128, cap));
    if (err == cudaSuccess) err = cudaMemsetAsync(flags, 0, 8 * sizeof(int) + 4 * sizeof(unsigned), s);
    double rtol2 = rtol * rtol;
    unsigned extra = 0;
    if (err == cudaSuccess) {
        void* args[] = {&n, &rowptr, &col, &vals, &dinv, &b, &x, &r, &z, &p, &q, &part, &bar, &scal, &flags,
                        &rtol2, &imax, &extra};
        err = cudaLaunchCooperativeKernel((void*)k_coarse_cg, grid, 512, args, 0, s);
    }
    int hf[2] = {0, 0};
    unsigned timeout = 0;
    double rr = 0.0;
    if (err == cudaSuccess) err = cudaMemcpyAsync(hf, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(&timeout, bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(&rr, scal + S_CG_RR, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) {
        set_error(std::string("sem_cg_csr_noalloc: ") + cudaGetErrorString(err));
        return SEM_ECUDA;
    }
    if (iters_host) *iters_host = hf[F_CG_ITERS];
    if (timeout) {
        set_error("sem_cg_csr_noalloc: a grid barrier wait ran out (device timeout)");
        return SEM_TIMEOUT;
    }
    if (!std::isfinite(rr)) {
        set_error("sem_cg_csr_noalloc: non-finite residual (a non-finite value in b, vals or dinv)");
        return SEM_NAN;
    }
    if (!hf[F_CG_DONE]) {
        set_error("sem_cg_csr_noalloc: rtol not reached within imax iterations");
        return SEM_NOT_CONVERGED;
    }
    return SEM_OK;
}
