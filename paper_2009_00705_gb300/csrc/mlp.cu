// Per-element correction network (the learned smoothing sweep): a two-layer MLP
// y = W2 relu(W1 x + b1) + b2 on element-local residuals, with BF16 weights,
// FP32 activations and FP32 accumulation; forward, backward and Adam kernels,
// and the gather/scatter that turn a global residual into network inputs and
// network outputs into a global correction.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "mlp.hpp"

namespace sem {

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// C[M][N] = sum_k A(m,k) B(k,n) with A(m,k) = TA ? A[k*lda+m] : A[m*lda+k] and
// B(k,n) = TB ? B[n*ldb+k] : B[k*ldb+n]; blockIdx.z splits K into chunks of kchunk.
// Epilogues: EPI_STORE, EPI_BIAS (C = acc + bias[n]), EPI_BIAS_RELU (Cpre = acc + bias,
// C = relu(Cpre)), EPI_ATOMIC (C += acc, for split-K weight gradients).
template <bool TA, bool TB, typename TBt, int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                              const TBt* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                              const float* __restrict__ bias, float* __restrict__ Cpre, int kchunk) {
    __shared__ float As[kBK][kBM + 4];
    __shared__ float Bs[kBK][kBN + 4];
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += kBK) {
        for (int i = threadIdx.x; i < kBM * kBK; i += 256) {
            int mm, kk;
            if (TA) { mm = i % kBM; kk = i / kBM; } else { kk = i % kBK; mm = i / kBK; }
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.f;
            if (m < M && k < kend) v = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
            As[kk][mm] = v;
        }
        for (int i = threadIdx.x; i < kBN * kBK; i += 256) {
            int nn, kk;
            if (TB) { kk = i % kBK; nn = i / kBK; } else { nn = i % kBN; kk = i / kBN; }
            const int n = n0 + nn, k = k0 + kk;
            float v = 0.f;
            if (n < N && k < kend) v = TB ? to_f(B[(size_t)n * ldb + k]) : to_f(B[(size_t)k * ldb + n]);
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float v = acc[i][j];
            const size_t o = (size_t)m * ldc + n;
            if (EPI == EPI_ATOMIC) {
                atomicAdd(&C[o], v);
            } else {
                if (EPI == EPI_BIAS || EPI == EPI_BIAS_RELU) v += bias[n];
                if (EPI == EPI_BIAS_RELU) {
                    Cpre[o] = v;
                    v = fmaxf(v, 0.f);
                }
                C[o] = v;
            }
        }
    }
}

template <bool TA, bool TB, typename TBt, int EPI>
cudaError_t gemm(int M, int N, int K, const float* A, int lda, const TBt* B, int ldb, float* C, int ldc,
                 const float* bias, float* Cpre, int splitk, cudaStream_t s) {
    const int kchunk = ((K + splitk - 1) / splitk + kBK - 1) / kBK * kBK;
    const int nz = (K + kchunk - 1) / kchunk;
    dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, nz);
    k_gemm<TA, TB, TBt, EPI><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, Cpre, kchunk);
    return cudaGetLastError();
}

// dY = 2 (Y - T) / B and the loss sum((Y - T)^2) / B (FP64 accumulation, one atomic per block).
__global__ void k_mse(long long n, float inv_b, const float* __restrict__ Y, const float* __restrict__ T,
                      float* __restrict__ dY, double* loss) {
    __shared__ double ws[8];
    double s = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        dY[i] = 2.f * d * inv_b;
        s += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        atomicAdd(loss, t * inv_b);
    }
}

// dA1 = dH1 where the pre-activation is positive (ReLU derivative), in place.
__global__ void k_relu_back(long long n, const float* __restrict__ A1, float* __restrict__ dH) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(A1[i] > 0.f)) dH[i] = 0.f;
}

// db[n] = sum over rows of D[rows][N] (atomic per block and column).
__global__ void k_colsum(int rows, int N, const float* __restrict__ D, float* __restrict__ db) {
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        float s = 0.f;
        for (int r = blockIdx.x; r < rows; r += gridDim.x) s += D[(size_t)r * N + n];
        atomicAdd(&db[n], s);
    }
}

// Adam with bias correction; writes the FP32 master and its BF16 copy.
__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ pb, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (pb) pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(long long n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

// Network inputs of element e: X[e][l] = r[g(e,l)] / s_e (0 at Dirichlet nodes),
// s_e = ||r_e||_2 (1 if zero); optionally the target T[e][l] = t[g] / s_e.  One warp per element.
template <typename V>
__global__ void k_gather_scaled(int E, int Np, const int* __restrict__ map, const V* __restrict__ r,
                                const V* __restrict__ t, float* __restrict__ X, float* __restrict__ T,
                                float* __restrict__ scale) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int e = warp; e < E; e += nwarps) {
        const int* me = map + (size_t)e * Np;
        float ss = 0.f;
        for (int l = lane; l < Np; l += 32) {
            const int m = me[l];
            const float v = m >= 0 ? (float)r[m] : 0.f;
            ss += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float se = ss > 0.f ? sqrtf(ss) : 1.f;
        const float inv = 1.f / se;
        for (int l = lane; l < Np; l += 32) {
            const int m = me[l];
            X[(size_t)e * Np + l] = m >= 0 ? (float)r[m] * inv : 0.f;
            if (T) T[(size_t)e * Np + l] = m >= 0 ? (float)t[m] * inv : 0.f;
        }
        if (lane == 0) scale[e] = se;
    }
}

// Global correction: d[g] += w_g * s_e * Y[e][l] over the free nodes of every element
// (w_g = 1 / number of elements sharing the node, so shared nodes get the average).
__global__ void k_scatter_corr(int E, int Np, const int* __restrict__ map, const float* __restrict__ w,
                               const float* __restrict__ Y, const float* __restrict__ scale, float* __restrict__ d) {
    const long long total = (long long)E * Np;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(i / Np);
        const int m = map[i];
        if (m >= 0) atomicAdd(&d[m], w[m] * scale[e] * Y[i]);
    }
}

inline int vgrid(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 16)); }

// out = a + sign * b
__global__ void k_axpby32(long long n, const float* __restrict__ a, const float* __restrict__ b, float sign,
                          float* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] + sign * b[i];
}

// out = a * b (element-wise)
__global__ void k_mul32(long long n, const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] * b[i];
}

// accept = (rr_new < rr_old) for the learned sweep; counts accepts and fallbacks.
__global__ void k_judge_mr(const double* rr, const double* rq, const double* qq, double* alpha, int* flags,
                           int accept_idx, int count_idx, double tau2) {
    const double a = (*qq > 0.0) ? *rq / *qq : 0.0;
    const double after = *rr - a * *rq;            // ||r - a q||^2 at the minimising a
    const int acc = (a > 0.0 && isfinite(a) && after < tau2 * *rr) ? 1 : 0;
    *alpha = acc ? a : 0.0;
    flags[accept_idx] = acc;
    flags[count_idx + (acc ? 0 : 1)] += 1;
}

__global__ void k_axpy_accepted32(long long n, const int* flags, int idx, const double* alpha,
                                  const float* __restrict__ delta, float* __restrict__ u) {
    if (!flags[idx]) return;
    const float a = (float)*alpha;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        u[i] += a * delta[i];
}

// SplitMix64 (Steele, Lea & Flood 2014) of (seed, counter) mapped to a uniform in [-1, 1)
__device__ __forceinline__ float splitmix_uniform(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}

// v[i] = uniform(-1, 1) on free nodes (dinv != 0), 0 on Dirichlet nodes
__global__ void k_random_free(long long n, unsigned long long seed, const float* __restrict__ dinv,
                              float* __restrict__ v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = dinv[i] != 0.f ? splitmix_uniform(seed, (unsigned long long)i) : 0.f;
}

}  // namespace

cudaError_t axpby32(long long n, const float* a, const float* b, float sign, float* out, cudaStream_t s) {
    k_axpby32<<<vgrid(n), 256, 0, s>>>(n, a, b, sign, out);
    return cudaGetLastError();
}
cudaError_t mul32(long long n, const float* a, const float* b, float* out, cudaStream_t s) {
    k_mul32<<<vgrid(n), 256, 0, s>>>(n, a, b, out);
    return cudaGetLastError();
}
cudaError_t judge_min_residual(const double* rr, const double* rq, const double* qq, double* alpha, int* flags,
                               int accept_idx, int count_idx, double tau2, cudaStream_t s) {
    k_judge_mr<<<1, 1, 0, s>>>(rr, rq, qq, alpha, flags, accept_idx, count_idx, tau2);
    return cudaGetLastError();
}
cudaError_t axpy_accepted32(long long n, const int* flags, int idx, const double* alpha, const float* delta, float* u,
                            cudaStream_t s) {
    k_axpy_accepted32<<<vgrid(n), 256, 0, s>>>(n, flags, idx, alpha, delta, u);
    return cudaGetLastError();
}
cudaError_t random_free(long long n, unsigned long long seed, const float* dinv, float* v, cudaStream_t s) {
    k_random_free<<<vgrid(n), 256, 0, s>>>(n, seed, dinv, v);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const MlpNet& net, int B, const float* X, float* A1, float* H1, float* Y, cudaStream_t s) {
    // H1 = relu(X W1^T + b1) (A1 the pre-activation), Y = H1 W2^T + b2 on the tensor cores
    cudaError_t e = gemm_t5<false, true, __nv_bfloat16, EPI_BIAS_RELU>(B, net.H, net.nin, X, net.nin, net.W1b, net.nin,
                                                                        H1, net.H, net.b1, A1, 1, net.err, s);
    if (e != cudaSuccess) return e;
    return gemm_t5<false, true, __nv_bfloat16, EPI_BIAS>(B, net.nout, net.H, H1, net.H, net.W2b, net.H, Y, net.nout,
                                                          net.b2, nullptr, 1, net.err, s);
}

cudaError_t mlp_backward(const MlpNet& net, int B, const float* X, const float* T, float* A1, float* H1, float* Y,
                         float* dY, float* dH, MlpGrads& g, double* loss, cudaStream_t s) {
    cudaError_t e;
    const long long ny = (long long)B * net.nout, nh = (long long)B * net.H;
    if ((e = cudaMemsetAsync(loss, 0, sizeof(double), s)) != cudaSuccess) return e;
    k_mse<<<vgrid(ny), 256, 0, s>>>(ny, 1.f / B, Y, T, dY, loss);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(g.dW1, 0, sizeof(float) * net.H * net.nin, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(g.dW2, 0, sizeof(float) * net.nout * net.H, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(g.db1, 0, sizeof(float) * net.H, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(g.db2, 0, sizeof(float) * net.nout, s)) != cudaSuccess) return e;
    const int split = std::max(1, std::min(128, B / 256));
    // dW2 [nout][H] = dY^T H1
    if ((e = gemm_t5<true, false, float, EPI_ATOMIC>(net.nout, net.H, B, dY, net.nout, H1, net.H, g.dW2, net.H,
                                                     nullptr, nullptr, split, net.err, s)) != cudaSuccess)
        return e;
    k_colsum<<<std::min(B, 1024), 256, 0, s>>>(B, net.nout, dY, g.db2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // dH [B][H] = dY W2, then the ReLU derivative
    if ((e = gemm_t5<false, false, __nv_bfloat16, EPI_STORE>(B, net.H, net.nout, dY, net.nout, net.W2b, net.H, dH,
                                                             net.H, nullptr, nullptr, 1, net.err, s)) != cudaSuccess)
        return e;
    k_relu_back<<<vgrid(nh), 256, 0, s>>>(nh, A1, dH);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // dW1 [H][nin] = dA1^T X
    if ((e = gemm_t5<true, false, float, EPI_ATOMIC>(net.H, net.nin, B, dH, net.H, X, net.nin, g.dW1, net.nin,
                                                     nullptr, nullptr, split, net.err, s)) != cudaSuccess)
        return e;
    k_colsum<<<std::min(B, 1024), 256, 0, s>>>(B, net.H, dH, g.db1);
    return cudaGetLastError();
}

cudaError_t mlp_adam(MlpNet& net, const MlpGrads& g, MlpAdam& st, float lr, cudaStream_t s) {
    st.t += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)st.t), c2 = 1.f - powf(b2, (float)st.t);
    struct P { float* p; const float* g; float* m; float* v; __nv_bfloat16* pb; long long n; };
    const P ps[4] = {{net.W1, g.dW1, st.m[0], st.v[0], net.W1b, (long long)net.H * net.nin},
                     {net.b1, g.db1, st.m[1], st.v[1], nullptr, net.H},
                     {net.W2, g.dW2, st.m[2], st.v[2], net.W2b, (long long)net.nout * net.H},
                     {net.b2, g.db2, st.m[3], st.v[3], nullptr, net.nout}};
    for (const P& p : ps) {
        k_adam<<<vgrid(p.n), 256, 0, s>>>(p.n, p.p, p.g, p.m, p.v, p.pb, lr, b1, b2, eps, c1, c2);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t mlp_sync_bf16(MlpNet& net, cudaStream_t s) {
    const long long n1 = (long long)net.H * net.nin, n2 = (long long)net.nout * net.H;
    k_to_bf16<<<vgrid(n1), 256, 0, s>>>(n1, net.W1, net.W1b);
    k_to_bf16<<<vgrid(n2), 256, 0, s>>>(n2, net.W2, net.W2b);
    return cudaGetLastError();
}

template <typename V>
cudaError_t gather_scaled(int E, int Np, const int* map, const V* r, const V* t, float* X, float* T, float* scale,
                          cudaStream_t s) {
    const int grid = std::max(1, std::min((E * 32 + 255) / 256, 152 * 16));
    k_gather_scaled<V><<<grid, 256, 0, s>>>(E, Np, map, r, t, X, T, scale);
    return cudaGetLastError();
}
template cudaError_t gather_scaled<float>(int, int, const int*, const float*, const float*, float*, float*, float*,
                                          cudaStream_t);
template cudaError_t gather_scaled<double>(int, int, const int*, const double*, const double*, float*, float*, float*,
                                           cudaStream_t);

cudaError_t scatter_correction(int E, int Np, const int* map, const float* w, const float* Y, const float* scale,
                               float* d, cudaStream_t s) {
    k_scatter_corr<<<vgrid((long long)E * Np), 256, 0, s>>>(E, Np, map, w, Y, scale, d);
    return cudaGetLastError();
}

}  // namespace sem
