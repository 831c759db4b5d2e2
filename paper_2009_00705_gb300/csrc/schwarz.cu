// Overlapping additive Schwarz smoother (Section 4.3, Eqs. sec_form, Mass, weights).
//
// One smoothing step is u <- u + S^{-1} (f - A u) with
//   S^{-1} = W sum_k R_k^T (R_k A R_k^T)^{-1} R_k,   W = (sum_k R_k R_k^T)^{-1},
// one subdomain per element k: the element's nodes and every node within `overlap`
// lattice steps of them (a step joins two nodes of one element whose lattice indices
// (i, j) of the triangle and k of the vertical line differ by at most one in i, j,
// i + j and k), of which the free nodes form the block.  Post-smoothing applies the
// adjoint S^{-T} = sum_k R_k^T (R_k A R_k^T)^{-1} R_k W, which keeps the V-cycle
// symmetric for the conjugate gradient outer iteration.
//
// Setup: the subdomains are built on the host (breadth-first search over lattice
// steps); the element matrices, the blocks R_k A R_k^T (principal submatrices of the
// free-node matrix, summed from the element matrices of every element touching the
// subdomain) and their inverses (blocked Gauss-Jordan, in place) are computed on the
// device.  Block k is stored densely, row-major with a row stride ld = n_k rounded up
// to a multiple of 4, in the V-cycle's precision (FP64 or FP32).
//
// Smoothing: one CTA per subdomain gathers x = R_k (f - A u) (times W for the
// adjoint), forms y = B_k x with one warp per row streaming the block from HBM (the
// bound of the step: n_k * ld_k words per subdomain), and adds W y (or y) into u with
// atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "sem_internal.hpp"

namespace sem {

namespace {

constexpr int kAsmThreads = 256;

__host__ __device__ inline int asm_ld(int n) { return (n + 3) & ~3; }

// ------------------------------------------------------------ element matrices
// A_e[a][b] = sum_q sum_{c,d} G_cd(q) g_c(q, a) g_d(q, b) (the Galerkin stiffness of
// Eq. laplaceproblemdiscrete with the quadrature of the apply): one CTA per 64 x 64 tile
// of one element, a 4 x 4 register tile per thread (rows ty + 16 i, columns tx + 16 j),
// quadrature points staged in chunks of 8.  gref: [dim][Nq][Np] full reference gradients;
// G: [E][ncomp][Nq] (rr, rs, rt, ss, st, tt in 3D; rr, rs, ss in 2D).
template <typename T>
__global__ void __launch_bounds__(kAsmThreads) k_elem_matrix(int E, int dim, int Np, int Nq, const T* __restrict__ G,
                                                             const T* __restrict__ gref, T* __restrict__ Ae) {
    constexpr int TILE = 64, QC = 8;
    __shared__ T sa[3][QC][TILE];
    __shared__ T sb[3][QC][TILE];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int nc = dim == 3 ? 6 : 3;
    const int ntile = (Np + TILE - 1) / TILE;
    const long long work = (long long)E * ntile * ntile;
    for (long long w = blockIdx.x; w < work; w += gridDim.x) {
        const int e = (int)(w / (ntile * ntile));
        const int rem = (int)(w - (long long)e * ntile * ntile);
        const int ta = rem / ntile, tb = rem - ta * ntile;
        const T* Ge = G + (size_t)e * nc * Nq;
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        for (int q0 = 0; q0 < Nq; q0 += QC) {
            for (int idx = threadIdx.x; idx < QC * TILE; idx += kAsmThreads) {
                const int qq = idx / TILE, col = idx - qq * TILE, q = q0 + qq;
                const int a = ta * TILE + col, b = tb * TILE + col;
                T ga[3] = {T(0), T(0), T(0)}, gb[3] = {T(0), T(0), T(0)}, psi[3] = {T(0), T(0), T(0)};
                if (q < Nq) {
                    for (int c = 0; c < dim; ++c) {
                        if (a < Np) ga[c] = gref[((size_t)c * Nq + q) * Np + a];
                        if (b < Np) gb[c] = gref[((size_t)c * Nq + q) * Np + b];
                    }
                    T g[3][3];
                    if (dim == 3) {
                        g[0][0] = Ge[q]; g[0][1] = g[1][0] = Ge[Nq + q]; g[0][2] = g[2][0] = Ge[2 * Nq + q];
                        g[1][1] = Ge[3 * Nq + q]; g[1][2] = g[2][1] = Ge[4 * Nq + q]; g[2][2] = Ge[5 * Nq + q];
                    } else {
                        g[0][0] = Ge[q]; g[0][1] = g[1][0] = Ge[Nq + q]; g[1][1] = Ge[2 * Nq + q];
                    }
                    for (int c = 0; c < dim; ++c) {
                        T s = T(0);
                        for (int d = 0; d < dim; ++d) s += g[c][d] * gb[d];
                        psi[c] = s;
                    }
                }
                for (int c = 0; c < 3; ++c) {
                    sa[c][qq][col] = ga[c];
                    sb[c][qq][col] = psi[c];
                }
            }
            __syncthreads();
            for (int qq = 0; qq < QC; ++qq)
                for (int c = 0; c < dim; ++c) {
                    T av[4], bv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        av[i] = sa[c][qq][ty + 16 * i];
                        bv[i] = sb[c][qq][tx + 16 * i];
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
                }
            __syncthreads();
        }
        T* out = Ae + (size_t)e * Np * Np;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int a = ta * TILE + ty + 16 * i;
            if (a >= Np) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int b = tb * TILE + tx + 16 * j;
                if (b < Np) out[(size_t)a * Np + b] = acc[i][j];
            }
        }
    }
}

// ------------------------------------------------------------ block assembly
// B_k = R_k A R_k^T: for every element touching subdomain k, the entries of its element
// matrix whose two nodes are both in the subdomain.  One CTA per subdomain; the nodes of
// one element map to distinct block positions, so one element's entries never collide
// and the elements are added in the order of the touch list (deterministic sums).
template <typename T>
__global__ void __launch_bounds__(kAsmThreads) k_asm_assemble(int nsub, int Np, const int* __restrict__ map,
                                                              const int* __restrict__ sptr,
                                                              const int* __restrict__ snodes,
                                                              const long long* __restrict__ off,
                                                              const int* __restrict__ tptr,
                                                              const int* __restrict__ telems,
                                                              const T* __restrict__ Ae, T* __restrict__ blocks) {
    extern __shared__ int asm_sm[];
    int* la = asm_sm;          // [Np] local node of the element
    int* pa = asm_sm + Np;     // [Np] its position in the subdomain
    __shared__ int cnt;
    for (int k = blockIdx.x; k < nsub; k += gridDim.x) {
        const int n = sptr[k + 1] - sptr[k], ld = asm_ld(n);
        const int* nodes = snodes + sptr[k];
        T* B = blocks + off[k];
        for (long long i = threadIdx.x; i < (long long)n * ld; i += kAsmThreads) B[i] = T(0);
        __syncthreads();
        for (int t = tptr[k]; t < tptr[k + 1]; ++t) {
            const int e = telems[t];
            if (threadIdx.x == 0) cnt = 0;
            __syncthreads();
            for (int a = threadIdx.x; a < Np; a += kAsmThreads) {
                const int g = map[(size_t)e * Np + a];
                if (g < 0) continue;                       // Dirichlet node
                int lo = 0, hi = n;                        // nodes[] ascending
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (nodes[mid] < g) lo = mid + 1;
                    else hi = mid;
                }
                if (lo < n && nodes[lo] == g) {
                    const int slot = atomicAdd(&cnt, 1);
                    la[slot] = a;
                    pa[slot] = lo;
                }
            }
            __syncthreads();
            const int m = cnt;
            const T* Ael = Ae + (size_t)e * Np * Np;
            for (int ij = threadIdx.x; ij < m * m; ij += kAsmThreads) {
                const int i = ij / m, j = ij - i * m;
                B[(size_t)pa[i] * ld + pa[j]] += Ael[(size_t)la[i] * Np + la[j]];
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------ block inversion
// In-place inverse of every SPD block by blocked Gauss-Jordan elimination (no pivoting:
// the pivot blocks are leading blocks of Schur complements of an SPD matrix).  For the
// panel J of PB columns, with I the other indices and D = M_JJ:
//   M_JJ <- D^{-1},  M_JI <- D^{-1} M_JI,  M_IJ <- -M_IJ D^{-1},  M_II <- M_II - M_IJ D^{-1} M_JI
// (the right-hand sides use the values before the panel step).  The column panel
// (nmax x PB) and the row panel (PB x nmax) are staged in shared memory; M_II is updated
// in register-tiled 64 x 64 tiles.
// A pivot that is not positive (or not finite) sets *bad.
template <typename T, int PB>
__global__ void __launch_bounds__(kAsmThreads) k_asm_invert(int nsub, int nmax, const int* __restrict__ sptr,
                                                            const long long* __restrict__ off,
                                                            T* __restrict__ blocks, int* bad) {
    extern __shared__ __align__(16) unsigned char inv_sm[];
    T* Cp = reinterpret_cast<T*>(inv_sm);    // [nmax][PB]
    T* Rp = Cp + (size_t)nmax * PB;          // [PB][nmax]
    __shared__ T D[PB][PB + 1];
    for (int k = blockIdx.x; k < nsub; k += gridDim.x) {
        const int n = sptr[k + 1] - sptr[k], ld = asm_ld(n);
        T* M = blocks + off[k];
        for (int J0 = 0; J0 < n; J0 += PB) {
            const int pb = min(PB, n - J0);
            for (int idx = threadIdx.x; idx < n * PB; idx += kAsmThreads) {
                const int i = idx / PB, m = idx - i * PB;
                Cp[idx] = m < pb ? M[(size_t)i * ld + J0 + m] : T(0);
            }
            for (int idx = threadIdx.x; idx < PB * n; idx += kAsmThreads) {
                const int m = idx / n, c = idx - m * n;
                Rp[(size_t)m * nmax + c] = m < pb ? M[(size_t)(J0 + m) * ld + c] : T(0);
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < PB * PB; idx += kAsmThreads) {
                const int r = idx / PB, c = idx - r * PB;
                D[r][c] = (r < pb && c < pb) ? Cp[(size_t)(J0 + r) * PB + c] : (r == c ? T(1) : T(0));
            }
            __syncthreads();
            for (int t = 0; t < pb; ++t) {                 // D <- D^{-1} (unblocked, in place)
                const T piv = D[t][t];
                if (threadIdx.x == 0 && !(piv > T(0))) atomicExch(bad, 1);
                const T ip = T(1) / piv;
                T v = T(0);
                const int r = threadIdx.x / PB, c = threadIdx.x - r * PB;
                if (r < PB) {
                    if (r == t && c == t) v = ip;
                    else if (r == t) v = D[t][c] * ip;
                    else if (c == t) v = -D[r][t] * ip;
                    else v = D[r][c] - D[r][t] * D[t][c] * ip;
                }
                __syncthreads();
                if (r < PB) D[r][c] = v;
                __syncthreads();
            }
            // (D is read through a volatile pointer: kept in registers across the column loop it
            // would take PB * PB of them)
            const volatile T* Dv = &D[0][0];
            for (int c = threadIdx.x; c < n; c += kAsmThreads) {   // row panel R' = D^{-1} R
                if (c >= J0 && c < J0 + pb) continue;
                T col[PB], o[PB];
#pragma unroll
                for (int m = 0; m < PB; ++m) col[m] = Rp[(size_t)m * nmax + c];
#pragma unroll
                for (int m = 0; m < PB; ++m) {
                    T s = T(0);
#pragma unroll
                    for (int l = 0; l < PB; ++l) s += Dv[m * (PB + 1) + l] * col[l];
                    o[m] = m < pb ? s : T(0);
                }
#pragma unroll
                for (int m = 0; m < PB; ++m) Rp[(size_t)m * nmax + c] = o[m];
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < n * PB; idx += kAsmThreads) {   // column panel -C D^{-1}
                const int i = idx / PB, m = idx - i * PB;
                if (m >= pb || (i >= J0 && i < J0 + pb)) continue;
                T s = T(0);
                for (int l = 0; l < pb; ++l) s += Cp[(size_t)i * PB + l] * D[l][m];
                M[(size_t)i * ld + J0 + m] = -s;
            }
            for (int idx = threadIdx.x; idx < PB * n; idx += kAsmThreads) {   // row panel
                const int m = idx / n, c = idx - m * n;
                if (m >= pb || (c >= J0 && c < J0 + pb)) continue;
                M[(size_t)(J0 + m) * ld + c] = Rp[(size_t)m * nmax + c];
            }
            for (int idx = threadIdx.x; idx < pb * pb; idx += kAsmThreads) {
                const int r = idx / pb, c = idx - r * pb;
                M[(size_t)(J0 + r) * ld + J0 + c] = D[r][c];
            }
            // M_II -= C R' in 64 x 64 tiles, a 4 x 4 register tile per thread (rows ty + 16 i,
            // columns tx + 16 j): sixteen independent loads per thread in flight, C and R'
            // read from shared memory (broadcast along the tile's rows and columns)
            const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
            const int nt = (n + 63) >> 6;
            for (int t = 0; t < nt * nt; ++t) {
                const int r0 = (t / nt) * 64 + ty, c0 = (t % nt) * 64 + tx;
                T acc[4][4];
                bool ok[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int r = r0 + 16 * a, c = c0 + 16 * b;
                        ok[a][b] = r < n && c < n && !(r >= J0 && r < J0 + pb) && !(c >= J0 && c < J0 + pb);
                        acc[a][b] = ok[a][b] ? M[(size_t)r * ld + c] : T(0);
                    }
                for (int m = 0; m < pb; ++m) {
                    T cv[4], rv[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int r = r0 + 16 * a, c = c0 + 16 * a;
                        cv[a] = r < n ? Cp[(size_t)r * PB + m] : T(0);
                        rv[a] = c < n ? Rp[(size_t)m * nmax + c] : T(0);
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] -= cv[a] * rv[b];
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (ok[a][b]) M[(size_t)(r0 + 16 * a) * ld + c0 + 16 * b] = acc[a][b];
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------ smoothing
template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = double2;
};

__device__ inline float dot_vec(const float4& b, const float4& x) { return b.x * x.x + b.y * x.y + b.z * x.z + b.w * x.w; }
__device__ inline double dot_vec(const double2& b, const double2& x) { return b.x * x.x + b.y * x.y; }

// u += W sum_k R_k^T B_k R_k r (adjoint = 0) or u += sum_k R_k^T B_k R_k W r (adjoint = 1)
// with r = f - y (y = A u, or null for r = f).  One CTA per subdomain (grid-stride);
// the gathered r_k sits in shared memory, one warp per block row reads it with 16-byte
// loads (rows are padded to ld = n rounded up to 4, padding columns are zero).
template <typename T>
__global__ void __launch_bounds__(kAsmThreads, 6) k_asm_apply(int nsub, const int* __restrict__ sptr,
                                                           const int* __restrict__ snodes,
                                                           const long long* __restrict__ off,
                                                           const T* __restrict__ blocks, const T* __restrict__ w,
                                                           const T* __restrict__ f, const T* __restrict__ y,
                                                           int adjoint, T* u) {
    using V = typename Vec4<T>::type;
    constexpr int kv = sizeof(V) / sizeof(T);
    extern __shared__ __align__(16) unsigned char app_sm[];
    T* xs = reinterpret_cast<T*>(app_sm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kAsmThreads / 32;
    for (int k = blockIdx.x; k < nsub; k += gridDim.x) {
        const int n = sptr[k + 1] - sptr[k], ld = asm_ld(n);
        const int* nodes = snodes + sptr[k];
        const T* B = blocks + off[k];
        for (int i = threadIdx.x; i < ld; i += kAsmThreads) {
            T v = T(0);
            if (i < n) {
                const int g = nodes[i];
                v = f[g] - (y ? y[g] : T(0));
                if (adjoint) v *= w[g];
            }
            xs[i] = v;
        }
        __syncthreads();
        const V* xv = reinterpret_cast<const V*>(xs);
        const int nv = ld / kv;
        // two rows per warp at a time, unrolled twice: four 16-byte loads per lane in flight
        // (with 6 CTAs per SM this streams the blocks at the device's copy bandwidth)
        for (int i = warp; i < n; i += 2 * kWarps) {
            const int i2 = i + kWarps;
            const V* row = reinterpret_cast<const V*>(B + (size_t)i * ld);
            const V* row2 = reinterpret_cast<const V*>(B + (size_t)(i2 < n ? i2 : i) * ld);
            T s = T(0), s2 = T(0);
#pragma unroll 2
            for (int j = lane; j < nv; j += 32) {
                const V b1 = __ldcs(row + j), b2 = __ldcs(row2 + j), x = xv[j];
                s += dot_vec(b1, x);
                s2 += dot_vec(b2, x);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s += __shfl_xor_sync(0xffffffffu, s, o);
                s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            }
            if (lane == 0) {
                const int g = nodes[i];
                atomicAdd(u + g, adjoint ? s : s * w[g]);
                if (i2 < n) {
                    const int g2 = nodes[i2];
                    atomicAdd(u + g2, adjoint ? s2 : s2 * w[g2]);
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ host side
// Lattice steps of the level's reference element (triangle order p, vertical order pz):
// for every local node, the local nodes whose lattice indices differ by at most one in
// i, j, i + j and k.
std::vector<std::vector<int>> lattice_steps(int dim, int p, int pz) {
    std::vector<int> li, lj, lk;
    const int nz = dim == 3 ? pz + 1 : 1;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= p; ++j)
            for (int i = 0; i + j <= p; ++i) {
                li.push_back(i);
                lj.push_back(j);
                lk.push_back(k);
            }
    const int np = (int)li.size();
    std::vector<std::vector<int>> out(np);
    for (int a = 0; a < np; ++a)
        for (int b = 0; b < np; ++b) {
            if (a == b) continue;
            const int di = li[b] - li[a], dj = lj[b] - lj[a], dk = lk[b] - lk[a];
            if (std::abs(di) <= 1 && std::abs(dj) <= 1 && std::abs(di + dj) <= 1 && std::abs(dk) <= 1)
                out[a].push_back(b);
        }
    return out;
}

int level_overlap(int p, int overlap) { return overlap < 0 ? (p + 2) / 2 : overlap; }   // ceil((p+1)/2)

template <typename T>
std::vector<T> full_gradients(const Level& L) {
    const RefLevel& r = L.ref;
    std::vector<T> g((size_t)L.dim * L.Nq * L.Np);
    for (int qz = 0; qz < L.QZ; ++qz)
        for (int qt = 0; qt < L.QT; ++qt)
            for (int k = 0; k < L.NZ; ++k)
                for (int n = 0; n < L.NT; ++n) {
                    const int q = qz * L.QT + qt, l = k * L.NT + n;
                    const double bz = r.Bz[qz * L.NZ + k], dz = r.Dz[qz * L.NZ + k];
                    g[(size_t)(0 * L.Nq + q) * L.Np + l] = (T)(r.Drt[qt * L.NT + n] * bz);
                    g[(size_t)(1 * L.Nq + q) * L.Np + l] = (T)(r.Dst[qt * L.NT + n] * bz);
                    if (L.dim == 3) g[(size_t)(2 * L.Nq + q) * L.Np + l] = (T)(r.Bt[qt * L.NT + n] * dz);
                }
    return g;
}

template <typename T>
cudaError_t to_device(T** p, const std::vector<T>& h) {
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(h.size(), 1) * sizeof(T));
    if (e == cudaSuccess && !h.empty()) e = cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

int device_sms() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Element matrices of level L in T (temporary [E][Np][Np]), the blocks assembled from
// them and inverted in place.
template <typename T>
sem_status asm_blocks(Level& L, const T* G, int* dflag) {
    const std::vector<T> g = full_gradients<T>(L);
    T* dg = nullptr;
    T* Ae = nullptr;
    cudaError_t e = to_device(&dg, g);
    if (e == cudaSuccess) e = cudaMalloc((void**)&Ae, (size_t)L.E * L.Np * L.Np * sizeof(T));
    const int sms = device_sms();
    if (e == cudaSuccess) {
        const int ntile = (L.Np + 63) / 64;
        const long long work = (long long)L.E * ntile * ntile;
        const int grid = (int)std::min<long long>(work, (long long)sms * 8);
        k_elem_matrix<T><<<grid, kAsmThreads>>>(L.E, L.dim, L.Np, L.Nq, G, dg, Ae);
        e = cudaGetLastError();
    }
    T* blk = static_cast<T*>(L.asm_blk);
    if (e == cudaSuccess) {
        const int grid = std::min(L.E, sms * 8);
        k_asm_assemble<T><<<grid, kAsmThreads, 2 * L.Np * sizeof(int)>>>(L.E, L.Np, L.map, L.asm_ptr, L.asm_nodes,
                                                                         L.asm_off, L.asm_tptr, L.asm_telems, Ae, blk);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemset(dflag, 0, sizeof(int));
    if (e == cudaSuccess) {
        const int grid = L.E;                 // one CTA per block (balanced by the scheduler)
        const size_t PB16 = 2 * (size_t)L.asm_nmax * 16 * sizeof(T);
        if (PB16 <= 200 * 1024) {
            auto kern = k_asm_invert<T, 16>;
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PB16);
            if (e == cudaSuccess) kern<<<grid, kAsmThreads, PB16>>>(L.E, L.asm_nmax, L.asm_ptr, L.asm_off, blk, dflag);
        } else {
            const size_t PB8 = PB16 / 2;
            auto kern = k_asm_invert<T, 8>;
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PB8);
            if (e == cudaSuccess) kern<<<grid, kAsmThreads, PB8>>>(L.E, L.asm_nmax, L.asm_ptr, L.asm_off, blk, dflag);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&bad, dflag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(dg);
    cudaFree(Ae);
    if (e != cudaSuccess) {
        set_error(std::string("Schwarz blocks: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SEM_ENOMEM : SEM_ECUDA;
    }
    if (bad) {
        set_error("Schwarz blocks: a block R_k A R_k^T is not positive definite");
        return SEM_BREAKDOWN;
    }
    return SEM_OK;
}


// The double-FP32 block layout of a chunk of element matrices Ae [n][Np][Np]: tile t of
// element e (row block I, column block J, in the order of df_tiles_of) holds rows I T + r,
// columns J T + c as (hi, lo) = (fl32(a), fl32(a - hi)), zero in the padding.
__global__ void k_pack_df(long long n, int Np, int T, int NB, int S, int TS, const double* __restrict__ Ae,
                          float2* __restrict__ out) {
    const int ntiles = NB * (NB + 1) / 2;
    const long long total = n * ntiles * TS;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long e = idx / ((long long)ntiles * TS);
        const int rem = (int)(idx - e * ntiles * TS);
        const int t = rem / TS, q = rem - t * TS;
        int I = 0, k = t;
        while (k >= df_tiles_of(I, NB)) k -= df_tiles_of(I++, NB);
        const int J = (I + k) % NB;
        const int r = q / S, c = q - r * S;
        const int row = I * T + r, col = J * T + c;
        double v = 0.0;
        if (r < T && c < T && row < Np && col < Np) v = Ae[((size_t)e * Np + row) * Np + col];
        const float hi = __double2float_rn(v);
        out[idx] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

}  // namespace

// FP64 element matrices of a 3D level, [E][Np][Np] (symmetric), for the element-matrix apply.
cudaError_t element_matrices64(const Level& L, double* Ae, cudaStream_t s) {
    const std::vector<double> g = full_gradients<double>(L);
    double* dg = nullptr;
    cudaError_t e = to_device(&dg, g);
    if (e == cudaSuccess) {
        const int ntile = (L.Np + 63) / 64;
        const long long work = (long long)L.E * ntile * ntile;
        const int grid = (int)std::min<long long>(work, (long long)device_sms() * 8);
        k_elem_matrix<double><<<grid, kAsmThreads, 0, s>>>(L.E, L.dim, L.Np, L.Nq, L.G, dg, Ae);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dg);
    return e;
}

cudaError_t element_matrices_df(const Level& L, float2* Adf, cudaStream_t s) {
    const std::vector<double> g = full_gradients<double>(L);
    const int Np = L.Np, Nq = L.Nq, nc = L.dim == 3 ? 6 : 3;
    const int ntiles = L.df_NB * (L.df_NB + 1) / 2;
    // FP64 matrices of up to 4096 elements at a time (1.2 GB at order 6), then packed
    const long long chunk = std::min<long long>(L.E, 4096);
    double *dg = nullptr, *Ae = nullptr;
    cudaError_t e = to_device(&dg, g);
    if (e == cudaSuccess) e = cudaMalloc(&Ae, sizeof(double) * (size_t)chunk * Np * Np);
    const int ntile = (Np + 63) / 64;
    for (long long e0 = 0; e == cudaSuccess && e0 < L.E; e0 += chunk) {
        const long long n = std::min<long long>(chunk, L.E - e0);
        const int grid = (int)std::min<long long>(n * ntile * ntile, (long long)device_sms() * 8);
        k_elem_matrix<double><<<grid, kAsmThreads, 0, s>>>((int)n, L.dim, Np, Nq, L.G + (size_t)e0 * nc * Nq, dg, Ae);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            const long long total = n * ntiles * L.df_TS;
            const int pg = (int)std::min<long long>((total + 255) / 256, (long long)device_sms() * 16);
            k_pack_df<<<pg, 256, 0, s>>>(n, Np, L.df_T, L.df_NB, L.df_S, L.df_TS, Ae,
                                         Adf + (size_t)e0 * ntiles * L.df_TS);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(Ae);
    cudaFree(dg);
    return e;
}

// Largest subdomain (nodes) the inversion kernel stages in shared memory.
int asm_max_block(bool fp64) { return fp64 ? (200 * 1024) / (2 * 8 * 8) : (200 * 1024) / (2 * 8 * 4); }

sem_status build_asm_level(sem_handle* h, int li) {
    Level& L = h->lv[li];
    const bool fp64 = h->opts.precision == SEM_PREC_FP64;
    const int ell = level_overlap(L.p, h->opts.asm_overlap);
    const std::vector<std::vector<int>> steps = lattice_steps(L.dim, L.p, L.pz);
    const int Np = L.Np, E = L.E;
    const long long N = L.N;
    // node -> (element, local index) incidence
    std::vector<long long> iptr(N + 1, 0);
    for (size_t t = 0; t < L.hmap.size(); ++t) {
        const int v = L.hmap[t];
        iptr[(v >= 0 ? v : -v - 1) + 1] += 1;
    }
    for (long long i = 0; i < N; ++i) iptr[i + 1] += iptr[i];
    std::vector<int> inc((size_t)iptr[N]);
    {
        std::vector<long long> fill(iptr.begin(), iptr.end() - 1);
        for (size_t t = 0; t < L.hmap.size(); ++t) {
            const int v = L.hmap[t];
            inc[(size_t)fill[v >= 0 ? v : -v - 1]++] = (int)t;   // t = e * Np + a
        }
    }
    auto gid = [&](size_t t) { const int v = L.hmap[t]; return v >= 0 ? v : -v - 1; };
    std::vector<int> stamp(N, -1), estamp(E, -1);
    std::vector<int> sptr(1, 0), snodes, tptr(1, 0), telems;
    std::vector<long long> off;
    std::vector<int> frontier, next, sub;
    long long words = 0;
    int nmax = 0;
    for (int e = 0; e < E; ++e) {
        frontier.clear();
        sub.clear();
        for (int a = 0; a < Np; ++a) {
            const int g = gid((size_t)e * Np + a);
            if (stamp[g] != e) {
                stamp[g] = e;
                frontier.push_back(g);
                sub.push_back(g);
            }
        }
        for (int d = 0; d < ell && !frontier.empty(); ++d) {
            next.clear();
            for (int g : frontier)
                for (long long t = iptr[g]; t < iptr[g + 1]; ++t) {
                    const int e2 = inc[(size_t)t] / Np, a = inc[(size_t)t] - e2 * Np;
                    for (int b : steps[a]) {
                        const int g2 = gid((size_t)e2 * Np + b);
                        if (stamp[g2] != e) {
                            stamp[g2] = e;
                            next.push_back(g2);
                            sub.push_back(g2);
                        }
                    }
                }
            frontier.swap(next);
        }
        std::sort(sub.begin(), sub.end());
        int n = 0;
        for (int g : sub) {
            // free nodes only (a Dirichlet node appears as -(g+1) in the element map)
            const long long t0 = iptr[g];
            if (L.hmap[(size_t)inc[(size_t)t0]] < 0) continue;
            snodes.push_back(g);
            ++n;
            for (long long t = iptr[g]; t < iptr[g + 1]; ++t) {
                const int e2 = inc[(size_t)t] / Np;
                if (estamp[e2] != e) {
                    estamp[e2] = e;
                    telems.push_back(e2);
                }
            }
        }
        if (n == 0) {
            set_error("Schwarz subdomain without a free node");
            return SEM_EINVAL;
        }
        sptr.push_back((int)snodes.size());
        tptr.push_back((int)telems.size());
        off.push_back(words);
        words += (long long)n * asm_ld(n);
        nmax = std::max(nmax, n);
        if (snodes.size() > (size_t)(1LL << 31) - 1 || telems.size() > (size_t)(1LL << 31) - 1) {
            set_error("Schwarz subdomains too large for 32-bit offsets");
            return SEM_EINVAL;
        }
    }
    if (nmax > asm_max_block(fp64)) {
        set_error("Schwarz subdomain of " + std::to_string(nmax) + " nodes exceeds the inversion kernel's limit of " +
                  std::to_string(asm_max_block(fp64)) + " (lower the overlap)");
        return SEM_EINVAL;
    }
    const size_t word = fp64 ? sizeof(double) : sizeof(float);
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) return SEM_ECUDA;
    const double need = (double)words * word + (double)E * Np * Np * word;
    if (need > 0.9 * (double)freeb) {
        set_error("Schwarz blocks need " + std::to_string(need / 1e9) + " GB, more than the free device memory");
        return SEM_ENOMEM;
    }
    std::vector<double> w(N, 0.0);
    for (int g : snodes) w[g] += 1.0;
    for (long long i = 0; i < N; ++i) w[i] = w[i] > 0.0 ? 1.0 / w[i] : 0.0;
    std::vector<float> w32(w.begin(), w.end());
    L.asm_nmax = nmax;
    L.asm_words = words;
    L.hasm_ptr = sptr;
    L.hasm_nodes = snodes;
    cudaError_t e = to_device(&L.asm_ptr, sptr);
    if (e == cudaSuccess) e = to_device(&L.asm_nodes, snodes);
    if (e == cudaSuccess) e = to_device(&L.asm_off, off);
    if (e == cudaSuccess) e = to_device(&L.asm_tptr, tptr);
    if (e == cudaSuccess) e = to_device(&L.asm_telems, telems);
    if (e == cudaSuccess) e = to_device(&L.asm_w, w);
    if (e == cudaSuccess) e = to_device(&L.asm_w32, w32);
    if (e == cudaSuccess) e = cudaMalloc(&L.asm_blk, std::max<size_t>((size_t)words * word, 16));
    if (e != cudaSuccess) {
        set_error(std::string("Schwarz setup: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SEM_ENOMEM : SEM_ECUDA;
    }
    return refresh_asm_level(h, li);
}

sem_status refresh_asm_level(sem_handle* h, int li) {
    Level& L = h->lv[li];
    int* dflag = h->sc.flags + F_ASM_BAD;
    if (h->opts.precision == SEM_PREC_FP64) return asm_blocks<double>(L, L.G, dflag);
    return asm_blocks<float>(L, L.G32, dflag);
}

void free_asm_level(Level& L) {
    for (void* p : {(void*)L.asm_ptr, (void*)L.asm_nodes, (void*)L.asm_off, (void*)L.asm_tptr, (void*)L.asm_telems,
                    (void*)L.asm_w, (void*)L.asm_w32, L.asm_blk})
        if (p) cudaFree(p);
    L.asm_ptr = L.asm_nodes = L.asm_tptr = L.asm_telems = nullptr;
    L.asm_off = nullptr;
    L.asm_w = nullptr;
    L.asm_w32 = nullptr;
    L.asm_blk = nullptr;
}

template <typename T>
cudaError_t asm_apply(const Level& L, const T* w, const T* f, const T* y, int adjoint, T* u, cudaStream_t s) {
    // one CTA per subdomain: the hardware scheduler balances the waves (a grid-stride grid
    // larger than the resident CTAs would leave a tail of lone CTAs per SM)
    const int grid = L.E;
    const size_t smem = (size_t)asm_ld(L.asm_nmax) * sizeof(T);
    k_asm_apply<T><<<grid, kAsmThreads, smem, s>>>(L.E, L.asm_ptr, L.asm_nodes, L.asm_off,
                                                    static_cast<const T*>(L.asm_blk), w, f, y, adjoint, u);
    return cudaGetLastError();
}

cudaError_t asm_apply64(const Level& L, const double* f, const double* y, int adjoint, double* u, cudaStream_t s) {
    return asm_apply<double>(L, L.asm_w, f, y, adjoint, u, s);
}

cudaError_t asm_apply32(const Level& L, const float* f, const float* y, int adjoint, float* u, cudaStream_t s) {
    return asm_apply<float>(L, L.asm_w32, f, y, adjoint, u, s);
}

}  // namespace sem
