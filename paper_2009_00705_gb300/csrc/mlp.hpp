// Per-element correction network (learned smoothing sweep): device buffers and launchers.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sem {

enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_RELU = 2, EPI_ATOMIC = 3 };

// y = W2 relu(W1 x + b1) + b2; W1 [H][nin], W2 [nout][H] (FP32 masters + BF16 copies used by the GEMMs)
struct MlpNet {
    int nin = 0, H = 0, nout = 0;
    float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr;
    int* err = nullptr;         // device flag set when a bounded wait of the tensor-core GEMMs ran out
};

// mlp_gemm_t5.cu: C[M][N] = A(m, k) B(k, n) on the tensor cores (TF32, FP32 accumulation),
// A(m, k) = TA ? A[k lda + m] : A[m lda + k], B(k, n) = TB ? B[n ldb + k] : B[k ldb + n];
// epilogues EPI_*; splitk chunks of K for EPI_ATOMIC
template <bool TA, bool TB, typename TBt, int EPI>
cudaError_t gemm_t5(int M, int N, int K, const float* A, int lda, const TBt* B, int ldb, float* C, int ldc,
                    const float* bias, float* Cpre, int splitk, int* err, cudaStream_t s);

struct MlpGrads {
    float *dW1 = nullptr, *db1 = nullptr, *dW2 = nullptr, *db2 = nullptr;
};

struct MlpAdam {
    float* m[4] = {};
    float* v[4] = {};
    long long t = 0;
};

// A1, H1: [B][H]; Y: [B][nout]
cudaError_t mlp_forward(const MlpNet& net, int B, const float* X, float* A1, float* H1, float* Y, cudaStream_t s);
// loss = sum ||Y - T||^2 / B (device double); gradients into g.  dY [B][nout], dH [B][H] are work buffers.
cudaError_t mlp_backward(const MlpNet& net, int B, const float* X, const float* T, float* A1, float* H1, float* Y,
                         float* dY, float* dH, MlpGrads& g, double* loss, cudaStream_t s);
cudaError_t mlp_adam(MlpNet& net, const MlpGrads& g, MlpAdam& st, float lr, cudaStream_t s);
cudaError_t mlp_sync_bf16(MlpNet& net, cudaStream_t s);
template <typename V>
cudaError_t gather_scaled(int E, int Np, const int* map, const V* r, const V* t, float* X, float* T, float* scale,
                          cudaStream_t s);
cudaError_t scatter_correction(int E, int Np, const int* map, const float* w, const float* Y, const float* scale,
                               float* d, cudaStream_t s);
cudaError_t mul32(long long n, const float* a, const float* b, float* out, cudaStream_t s);
cudaError_t axpby32(long long n, const float* a, const float* b, float sign, float* out, cudaStream_t s);
// Minimal-residual verdict on a correction delta with q = A delta: alpha = (r, q) / (q, q);
// accepted (flags[accept_idx] = 1, *alpha kept) when alpha > 0 and the residual after the
// step, rr - alpha (r, q), is below tau2 * rr; counts accepts / fallbacks at count_idx.
cudaError_t judge_min_residual(const double* rr, const double* rq, const double* qq, double* alpha, int* flags,
                               int accept_idx, int count_idx, double tau2, cudaStream_t s);
// u += alpha * delta when flags[idx] is set
cudaError_t axpy_accepted32(long long n, const int* flags, int idx, const double* alpha, const float* delta, float* u,
                            cudaStream_t s);
cudaError_t random_free(long long n, unsigned long long seed, const float* dinv, float* v, cudaStream_t s);

}  // namespace sem
