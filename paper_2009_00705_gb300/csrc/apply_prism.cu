// Matrix-free stiffness apply on sigma-layer prisms (Eq. laplaceproblemdiscrete),
// sum-factorised in the vertical: gather -> reference derivatives at the
// quadrature points -> geometric factors -> transposed contraction ->
// direct-stiffness summation.  Two tile shapes (elements per CTA pass) are
// compiled per order and precision; the autotuner in setup.cpp picks one per level.
#include <cuda_runtime.h>

#include "sem_internal.hpp"

namespace sem {

namespace {

constexpr int kSMs = 152;

// ------------------------------------------------------------------ prism apply, register-tiled
// Same contraction as k_apply for prisms, organised for throughput: a CTA takes
// EB elements at a time; in the triangle stage one thread owns a quadrature
// point qt of one element and keeps the values at all QZ vertical points in
// registers, and in the transposed stage one thread owns a triangle node n and
// keeps all QZ partial sums, so the transposed vertical stage and the
// direct-stiffness summation follow without another pass through shared memory.
template <int P, int PZ, typename T, int V>
struct PrismTile {
    // triangle order P, vertical order PZ (= P unless the level is anisotropic)
    static constexpr int NT = (P + 1) * (P + 2) / 2, NZ = PZ + 1, QT = (P + 1) * (P + 1), QZ = PZ + 1;
    static constexpr int Np = NT * NZ, Nq = QT * QZ;
    static constexpr int VEC = 16 / sizeof(T);                  // elements per 16-byte load
    static constexpr int QZP = (QZ + VEC - 1) / VEC * VEC;      // padded row length
    // elements per CTA pass (the tile shape; variant V = 0 or 1 is picked by the
    // autotuner): 8 at P = 6 fills whole warps in both heavy stages (8 * 49
    // quadrature columns, 8 * 28 triangle nodes), half of that for V = 1; more at low order
    static constexpr int EB = (V == 0 ? 8 : 4) * (P <= 2 ? 4 : (P == 3 ? 2 : 1));
    static constexpr int THR_RAW = ((EB * NT + 31) / 32) * 32;
    static constexpr int NTHR = THR_RAW < 64 ? 64 : (THR_RAW > 256 ? 256 : THR_RAW);
    static constexpr bool TRANSPOSED = (sizeof(T) == 4);       // conflict-free copies for FP32 only
    __host__ __device__ static constexpr int round4(int v) { return (v + 3) / 4 * 4; }
    static constexpr int REF = round4(3 * QT * NT) + (TRANSPOSED ? round4(3 * QT * NT) : 0) + round4(2 * QZ * NZ);
    static constexpr int WORK = round4(Np) + 2 * round4(NT * QZP) + 3 * round4(QT * QZP);
    static constexpr size_t SMEM = sizeof(T) * (REF + (size_t)EB * WORK);
};

template <typename T, int N, int NP>
__device__ __forceinline__ void load_row(const T* __restrict__ src, T (&out)[N]) {
    static_assert(NP >= N, "row padding");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int c = 0; c < NP / 4; ++c) {
            const float4 v = reinterpret_cast<const float4*>(src)[c];
            if (4 * c + 0 < N) out[4 * c + 0] = v.x;
            if (4 * c + 1 < N) out[4 * c + 1] = v.y;
            if (4 * c + 2 < N) out[4 * c + 2] = v.z;
            if (4 * c + 3 < N) out[4 * c + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int c = 0; c < NP / 2; ++c) {
            const double2 v = reinterpret_cast<const double2*>(src)[c];
            if (2 * c + 0 < N) out[2 * c + 0] = v.x;
            if (2 * c + 1 < N) out[2 * c + 1] = v.y;
        }
    }
}

template <int P, int PZ, typename T, bool LIFT, int V>
__global__ void __launch_bounds__(PrismTile<P, PZ, T, V>::NTHR)
    k_apply_prism(int E, const int* __restrict__ map, const T* __restrict__ G, const T* __restrict__ refm,
                  const T* __restrict__ x, T* __restrict__ y, const int* __restrict__ skip,
                  const int* __restrict__ elist, T* __restrict__ ye) {
    using D = PrismTile<P, PZ, T, V>;
    constexpr int NT = D::NT, NZ = D::NZ, QT = D::QT, QZ = D::QZ, Np = D::Np, Nq = D::Nq, QZP = D::QZP, EB = D::EB;
    if (skip != nullptr && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    // reference matrices: [Bt | Dr | Ds] as [QT][NT]; (FP32) [BtT | DrT | DsT] as [NT][QT]; [Bz | Dz] as [QZ][NZ]
    T* sB = sm;
    T* sBT = sm + D::round4(3 * QT * NT);
    T* sZ = sBT + (D::TRANSPOSED ? D::round4(3 * QT * NT) : 0);
    for (int i = threadIdx.x; i < 3 * QT * NT; i += blockDim.x) sB[i] = refm[i];
    if (D::TRANSPOSED)
        for (int i = threadIdx.x; i < 3 * QT * NT; i += blockDim.x) sBT[i] = refm[3 * QT * NT + i];
    for (int i = threadIdx.x; i < 2 * QZ * NZ; i += blockDim.x) sZ[i] = refm[6 * QT * NT + i];
    T* work = sm + D::REF;
    const T* sBt = sB;
    const T* sDr = sB + QT * NT;
    const T* sDs = sB + 2 * QT * NT;
    const T* sBz = sZ;
    const T* sDz = sZ + QZ * NZ;
    __syncthreads();
    for (int e0 = blockIdx.x * EB; e0 < E; e0 += gridDim.x * EB) {
        const int nb = min(EB, E - e0);
        {   // pull the next pass's geometric factors and map into L2 while this pass computes
            const int en = e0 + gridDim.x * EB;
            if (en < E && elist == nullptr) {
                const int nn = min(EB, E - en);
                const char* g0 = reinterpret_cast<const char*>(G + (size_t)en * 6 * Nq);
                const size_t gbytes = (size_t)nn * 6 * Nq * sizeof(T);
                for (size_t off = (size_t)threadIdx.x * 128; off < gbytes; off += (size_t)blockDim.x * 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(g0 + off));
                const char* m0 = reinterpret_cast<const char*>(map + (size_t)en * Np);
                for (size_t off = (size_t)threadIdx.x * 128; off < (size_t)nn * Np * 4; off += (size_t)blockDim.x * 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(m0 + off));
            }
        }
        // gather
        for (int i = threadIdx.x; i < nb * Np; i += blockDim.x) {
            const int b = i / Np, l = i - b * Np;
            const int e = elist ? elist[e0 + b] : e0 + b;
            const int m = map[(size_t)e * Np + l];
            work[b * D::WORK + l] = (m >= 0) ? x[m] : (LIFT ? x[-m - 1] : T(0));
        }
        __syncthreads();
        // vertical stage: U[n][qz], W[n][qz] (values / t-derivatives at the vertical Gauss points)
        for (int i = threadIdx.x; i < nb * NT; i += blockDim.x) {
            const int b = i / NT, n = i - b * NT;
            T* wb = work + b * D::WORK;
            T xk[NZ];
#pragma unroll
            for (int k = 0; k < NZ; ++k) xk[k] = wb[k * NT + n];
            T* U = wb + D::round4(Np) + n * QZP;
            T* W = wb + D::round4(Np) + D::round4(NT * QZP) + n * QZP;
#pragma unroll
            for (int qz = 0; qz < QZ; ++qz) {
                T u = 0, w = 0;
#pragma unroll
                for (int k = 0; k < NZ; ++k) {
                    u += sBz[qz * NZ + k] * xk[k];
                    w += sDz[qz * NZ + k] * xk[k];
                }
                U[qz] = u;
                W[qz] = w;
            }
        }
        __syncthreads();
        // triangle stage + geometric factors: thread (b, qt), all qz in registers
        for (int i = threadIdx.x; i < nb * QT; i += blockDim.x) {
            const int b = i / QT, qt = i - b * QT;
            T* wb = work + b * D::WORK;
            const T* U = wb + D::round4(Np);
            const T* W = U + D::round4(NT * QZP);
            T ur[QZ], us[QZ], ut[QZ];
#pragma unroll
            for (int qz = 0; qz < QZ; ++qz) ur[qz] = us[qz] = ut[qz] = T(0);
#pragma unroll 2
            for (int n = 0; n < NT; ++n) {
                T dr, ds, bt;
                if (D::TRANSPOSED) {
                    dr = sBT[QT * NT + n * QT + qt];
                    ds = sBT[2 * QT * NT + n * QT + qt];
                    bt = sBT[n * QT + qt];
                } else {
                    dr = sDr[qt * NT + n];
                    ds = sDs[qt * NT + n];
                    bt = sBt[qt * NT + n];
                }
                T uv[QZ], wv[QZ];
                load_row<T, QZ, QZP>(U + n * QZP, uv);
                load_row<T, QZ, QZP>(W + n * QZP, wv);
#pragma unroll
                for (int qz = 0; qz < QZ; ++qz) {
                    ur[qz] += dr * uv[qz];
                    us[qz] += ds * uv[qz];
                    ut[qz] += bt * wv[qz];
                }
            }
            const T* Ge = G + (size_t)(elist ? elist[e0 + b] : e0 + b) * 6 * Nq;
            T* vr = wb + D::round4(Np) + 2 * D::round4(NT * QZP) + qt * QZP;
            T* vs = vr + D::round4(QT * QZP);
            T* vt = vs + D::round4(QT * QZP);
#pragma unroll
            for (int qz = 0; qz < QZ; ++qz) {
                const int q = qz * QT + qt;
                const T g0 = Ge[q], g1 = Ge[Nq + q], g2 = Ge[2 * Nq + q];
                const T g3 = Ge[3 * Nq + q], g4 = Ge[4 * Nq + q], g5 = Ge[5 * Nq + q];
                vr[qz] = g0 * ur[qz] + g1 * us[qz] + g2 * ut[qz];
                vs[qz] = g1 * ur[qz] + g3 * us[qz] + g4 * ut[qz];
                vt[qz] = g2 * ur[qz] + g4 * us[qz] + g5 * ut[qz];
            }
        }
        __syncthreads();
        // transposed triangle stage (thread (b, n), all qz), transposed vertical stage, summation
        for (int i = threadIdx.x; i < nb * NT; i += blockDim.x) {
            const int b = i / NT, n = i - b * NT;
            const T* wb = work + b * D::WORK;
            const T* vr = wb + D::round4(Np) + 2 * D::round4(NT * QZP);
            const T* vs = vr + D::round4(QT * QZP);
            const T* vt = vs + D::round4(QT * QZP);
            T xr[QZ], xt[QZ];
#pragma unroll
            for (int qz = 0; qz < QZ; ++qz) xr[qz] = xt[qz] = T(0);
#pragma unroll 2
            for (int qt = 0; qt < QT; ++qt) {
                const T dr = sDr[qt * NT + n], ds = sDs[qt * NT + n], bt = sBt[qt * NT + n];
                T a[QZ], c[QZ], d[QZ];
                load_row<T, QZ, QZP>(vr + qt * QZP, a);
                load_row<T, QZ, QZP>(vs + qt * QZP, c);
                load_row<T, QZ, QZP>(vt + qt * QZP, d);
#pragma unroll
                for (int qz = 0; qz < QZ; ++qz) {
                    xr[qz] += dr * a[qz] + ds * c[qz];
                    xt[qz] += bt * d[qz];
                }
            }
            const size_t eid = (size_t)(elist ? elist[e0 + b] : e0 + b);
            const int* me = map + eid * Np;
#pragma unroll
            for (int k = 0; k < NZ; ++k) {
                T s = 0;
#pragma unroll
                for (int qz = 0; qz < QZ; ++qz) s += sBz[qz * NZ + k] * xr[qz] + sDz[qz * NZ + k] * xt[qz];
                // element results (deterministic summation afterwards by node) or atomic summation
                if (ye != nullptr) {
                    ye[eid * Np + k * NT + n] = s;
                } else {
                    const int m = me[k * NT + n];
                    if (m >= 0) atomicAdd(&y[m], s);
                }
            }
        }
        __syncthreads();
    }
}

// FP64 apply from precomputed element matrices: y_e = A_e x_e with A_e = sum_q sum_ab
// D_a^T G_ab D_b (Eq. laplaceproblemdiscrete at the same quadrature), 2 Np^2 flops per element
// against 132 k for the sum-factorised contraction at P = 6; A_e streamed once per apply.
// The rows of all elements form one flat index space, kElemRows consecutive rows per CTA
// pass, so every lane of every warp holds a row (no lanes idle at element boundaries: the FP64
// pipe bounds this kernel).  A pass stages x of the elements its rows touch in shared memory
// (an element at either end may be shared with the neighbouring pass); thread t forms row
// i = r mod Np of element e = r / Np from column i of the symmetric A_e (coalesced across the
// warp), with four partial sums.  Gather masking, lifting, element lists and the element-result
// output as in k_apply_prism.
constexpr int kElemRows = 512;

template <bool LIFT>
__global__ void __launch_bounds__(kElemRows) k_apply_elem64(int E, int Np, const int* __restrict__ map,
                                                         const double* __restrict__ Ae, const double* __restrict__ x,
                                                         double* __restrict__ y, const int* __restrict__ skip,
                                                         const int* __restrict__ elist, double* __restrict__ ye) {
    if (skip != nullptr && *skip) return;
    extern __shared__ __align__(16) double xs[];      // [elements of the pass][Np]
    const long long R = (long long)E * Np;
    for (long long r0 = (long long)blockIdx.x * kElemRows; r0 < R; r0 += (long long)gridDim.x * kElemRows) {
        const long long r1 = r0 + kElemRows < R ? r0 + kElemRows : R;
        const long long ea = r0 / Np, eb = (r1 - 1) / Np;        // first and last element of the pass
        const int nx = (int)(eb - ea + 1) * Np;
        for (int k = threadIdx.x; k < nx; k += blockDim.x) {
            const long long el = ea + k / Np;
            const size_t e = (size_t)(elist ? elist[el] : el);
            const int m = map[e * Np + (k % Np)];
            xs[k] = (m >= 0) ? x[m] : (LIFT ? x[-m - 1] : 0.0);
        }
        __syncthreads();
        const long long r = r0 + threadIdx.x;
        if (r < r1) {
            const long long el = r / Np;
            const int i = (int)(r - el * Np);
            const size_t e = (size_t)(elist ? elist[el] : el);
            const double* A = Ae + e * (size_t)Np * Np + i;
            const double* xv = xs + (el - ea) * Np;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int j = 0;
            for (; j + 3 < Np; j += 4) {
                s0 = fma(__ldcs(A + (size_t)j * Np), xv[j], s0);
                s1 = fma(__ldcs(A + (size_t)(j + 1) * Np), xv[j + 1], s1);
                s2 = fma(__ldcs(A + (size_t)(j + 2) * Np), xv[j + 2], s2);
                s3 = fma(__ldcs(A + (size_t)(j + 3) * Np), xv[j + 3], s3);
            }
            for (; j < Np; ++j) s0 = fma(__ldcs(A + (size_t)j * Np), xv[j], s0);
            const double v = (s0 + s1) + (s2 + s3);
            if (ye != nullptr) ye[e * Np + i] = v;
            else {
                const int m = map[e * Np + i];
                if (m >= 0) atomicAdd(&y[m], v);
            }
        }
        __syncthreads();
    }
}

cudaError_t apply_elem64(const Level& L, const double* x, double* y, bool lift, const int* skip, cudaStream_t s) {
    double* ye = L.ye64;
    const bool sub = lift && L.lift_elems != nullptr && ye == nullptr;
    const int E = sub ? L.nlift : L.E;
    const long long passes = ((long long)E * L.Np + kElemRows - 1) / kElemRows;
    const int grid = (int)std::min<long long>(passes, (long long)kSMs * 4);
    if (grid < 1) return cudaSuccess;
    // a pass touches at most kElemRows / Np + 2 elements
    const size_t smem = sizeof(double) * (size_t)(kElemRows / L.Np + 2) * L.Np;
    if (lift)
        k_apply_elem64<true><<<grid, kElemRows, smem, s>>>(E, L.Np, L.map, L.Ae64, x, y, skip,
                                                           sub ? L.lift_elems : nullptr, ye);
    else
        k_apply_elem64<false><<<grid, kElemRows, smem, s>>>(E, L.Np, L.map, L.Ae64, x, y, skip, nullptr, ye);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || ye == nullptr) return e;
    return dss_gather64(L, ye, y, skip, s, true);
}

template <int P, int PZ, typename T, bool LIFT, int V>
cudaError_t apply_prism_impl(const Level& L, const T* refm, const T* G, const T* x, T* y, const int* skip, T* ye,
                             cudaStream_t s) {
    using D = PrismTile<P, PZ, T, V>;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t err = cudaFuncSetAttribute(k_apply_prism<P, PZ, T, LIFT, V>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D::SMEM);
        if (err != cudaSuccess) return err;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_prism<P, PZ, T, LIFT, V>, D::NTHR, D::SMEM);
        if (err != cudaSuccess) return err;
        if (per_sm < 1) per_sm = 1;
    }
    // the lifting apply (x zero on the free nodes) only needs the elements that touch a
    // Dirichlet node: every other element gathers zeros
    const bool sub = LIFT && L.lift_elems != nullptr && ye == nullptr;   // element results need every element
    const int E = sub ? L.nlift : L.E;
    const int batches = (E + D::EB - 1) / D::EB;
    int grid = kSMs * per_sm;
    if (grid > batches) grid = batches;
    if (grid < 1) return cudaSuccess;
    k_apply_prism<P, PZ, T, LIFT, V><<<grid, D::NTHR, D::SMEM, s>>>(E, L.map, G, refm, x, y, skip,
                                                                    sub ? L.lift_elems : nullptr, ye);
    return cudaGetLastError();
}

}  // namespace

template <typename T, bool LIFT, int V>
static cudaError_t prism_dispatch(const Level& L, const T* refm, const T* G, const T* x, T* y, const int* skip,
                                  T* ye, cudaStream_t s) {
#define SEM_PRISM_PAIR(a, b) \
    case (a) * 8 + (b): return apply_prism_impl<a, b, T, LIFT, V>(L, refm, G, x, y, skip, ye, s);
    switch (L.p * 8 + L.pz) {
        // isotropic orders
        SEM_PRISM_PAIR(1, 1) SEM_PRISM_PAIR(2, 2) SEM_PRISM_PAIR(3, 3)
        SEM_PRISM_PAIR(4, 4) SEM_PRISM_PAIR(5, 5) SEM_PRISM_PAIR(6, 6)
        // anisotropic orders (vertical order one or two below the triangle order)
        SEM_PRISM_PAIR(2, 1) SEM_PRISM_PAIR(3, 2) SEM_PRISM_PAIR(3, 1)
        SEM_PRISM_PAIR(4, 3) SEM_PRISM_PAIR(4, 2) SEM_PRISM_PAIR(5, 4)
        SEM_PRISM_PAIR(5, 3) SEM_PRISM_PAIR(6, 5) SEM_PRISM_PAIR(6, 4)
        default: return cudaErrorInvalidValue;
    }
#undef SEM_PRISM_PAIR
}

bool prism_pair_supported(int p, int pz) {
    return p >= 1 && p <= 6 && (pz == p || (p >= 2 && (pz == p - 1 || (p >= 3 && pz == p - 2))));
}

cudaError_t launch_apply_prism64(const Level& L, const double* x, double* y, bool lift, const int* skip, int variant,
                                 cudaStream_t s) {
    if (L.Adf != nullptr) return apply_elem_df(L, x, y, lift, skip, s);
    if (L.Ae64 != nullptr) return apply_elem64(L, x, y, lift, skip, s);
    // deterministic handles: element results, then the per-node sums in a fixed order
    double* ye = L.ye64;
    cudaError_t e;
    if (lift) e = variant ? prism_dispatch<double, true, 1>(L, L.ref64.m, L.G, x, y, skip, ye, s)
                          : prism_dispatch<double, true, 0>(L, L.ref64.m, L.G, x, y, skip, ye, s);
    else e = variant ? prism_dispatch<double, false, 1>(L, L.ref64.m, L.G, x, y, skip, ye, s)
                     : prism_dispatch<double, false, 0>(L, L.ref64.m, L.G, x, y, skip, ye, s);
    if (e != cudaSuccess || ye == nullptr) return e;
    return dss_gather64(L, ye, y, skip, s, true);
}

cudaError_t launch_apply_prism32(const Level& L, const float* x, float* y, const int* skip, int variant,
                                 cudaStream_t s) {
    return variant ? prism_dispatch<float, false, 1>(L, L.ref32.m, L.G32, x, y, skip, nullptr, s)
                   : prism_dispatch<float, false, 0>(L, L.ref32.m, L.G32, x, y, skip, nullptr, s);
}

int prism_tile_elements(int P, int variant) { return (variant == 0 ? 8 : 4) * (P <= 2 ? 4 : (P == 3 ? 2 : 1)); }

}  // namespace sem
