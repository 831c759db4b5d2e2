// Free-surface fields of the time stepping around the Laplace solve (Section 2,
// Eqs. FSeta and FSphi): horizontal gradients of surface fields, the vertical
// velocity w~ = dphi/dz at the surface, the right-hand sides of the kinematic and
// dynamic conditions, and the stage combinations of the classical four-stage
// Runge-Kutta method.  Surface fields live at the order-P 2D nodes (N2 values).
#include <cuda_runtime.h>

#include "sem_internal.hpp"

namespace sem {

namespace {

constexpr int kFsThreads = 256;

inline int fs_grid(long long n) {
    const long long b = (n + kFsThreads - 1) / kFsThreads;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// Gradient of the order-P interpolant of f2 on base triangle b at its node n, summed
// into (gx, gy) at the node's global id (the caller divides by the multiplicity).
// Drn, Dsn: [NT][NT] reference derivatives of the nodal basis at the nodes; vtri:
// [ntri][3][2] vertex coordinates (affine map x = -(r+s)/2 v0 + (1+r)/2 v1 + (1+s)/2 v2).
__global__ void k_surface_grad(int ntri, int NT, const int* __restrict__ map2, const double* __restrict__ vtri,
                               const double* __restrict__ Drn, const double* __restrict__ Dsn,
                               const double* __restrict__ f2, double* __restrict__ gx, double* __restrict__ gy) {
    const long long total = (long long)ntri * NT;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / NT), n = (int)(t - (long long)b * NT);
        const int* mb = map2 + (size_t)b * NT;
        double fr = 0.0, fs = 0.0;
        for (int m = 0; m < NT; ++m) {
            const double v = f2[mb[m]];
            fr += Drn[n * NT + m] * v;
            fs += Dsn[n * NT + m] * v;
        }
        const double* v = vtri + (size_t)b * 6;
        const double xr = 0.5 * (v[2] - v[0]), xs = 0.5 * (v[4] - v[0]);
        const double yr = 0.5 * (v[3] - v[1]), ys = 0.5 * (v[5] - v[1]);
        const double det = xr * ys - xs * yr;
        const double rx = ys / det, ry = -xs / det, sx = -yr / det, sy = xr / det;
        atomicAdd(&gx[mb[n]], rx * fr + sx * fs);
        atomicAdd(&gy[mb[n]], ry * fr + sy * fs);
    }
}

__global__ void k_scale2(long long n, const double* __restrict__ w, double* __restrict__ a, double* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        a[i] *= w[i];
        b[i] *= w[i];
    }
}

// w~[g] = (sum_k Dtop[k] phi[(k0 + k) N2 + g]) / ((depth + eta[g]) / (2 nlayers)): the
// vertical derivative along node g's line in the top sigma layer, k0 = (nl - 1) p.
__global__ void k_surface_w(long long N2, int NZ, long long k0, const double* __restrict__ Dtop, double depth,
                            int nlayers, const double* __restrict__ phi, const double* __restrict__ eta,
                            double* __restrict__ w) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N2; g += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < NZ; ++k) s += Dtop[k] * phi[(k0 + k) * N2 + g];
        w[g] = s * (2.0 * nlayers) / (depth + eta[g]);
    }
}

// Right-hand sides of Eqs. FSeta and FSphi (linear = 1: d eta/dt = w~, d phi~/dt = -g eta).
__global__ void k_fnpf_rhs(long long N2, int linear, double grav, const double* __restrict__ eta,
                           const double* __restrict__ w, const double* __restrict__ ex,
                           const double* __restrict__ ey, const double* __restrict__ px,
                           const double* __restrict__ py, double* __restrict__ deta, double* __restrict__ dphi) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N2; i += (long long)gridDim.x * blockDim.x) {
        if (linear) {
            deta[i] = w[i];
            dphi[i] = -grav * eta[i];
        } else {
            const double gg = 1.0 + ex[i] * ex[i] + ey[i] * ey[i];
            deta[i] = -(ex[i] * px[i] + ey[i] * py[i]) + w[i] * gg;
            dphi[i] = -grav * eta[i] - 0.5 * (px[i] * px[i] + py[i] * py[i] - w[i] * w[i] * gg);
        }
    }
}

// out = x + c * k for the two surface fields
__global__ void k_stage(long long n, double c, const double* __restrict__ x0, const double* __restrict__ k0,
                        const double* __restrict__ x1, const double* __restrict__ k1, double* __restrict__ o0,
                        double* __restrict__ o1) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        o0[i] = x0[i] + c * k0[i];
        o1[i] = x1[i] + c * k1[i];
    }
}

// x += dt/6 (k1 + 2 k2 + 2 k3 + k4) for one field, k = [4][n]
__global__ void k_rk4_combine(long long n, double dt, const double* __restrict__ k, double* __restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += dt / 6.0 * (k[i] + 2.0 * k[n + i] + 2.0 * k[2 * n + i] + k[3 * n + i]);
}

}  // namespace

cudaError_t surface_gradient(int ntri, int NT, long long N2, const int* map2, const double* vtri, const double* Drn,
                             const double* Dsn, const double* inv_mult, const double* f2, double* gx, double* gy,
                             cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(gx, 0, sizeof(double) * N2, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(gy, 0, sizeof(double) * N2, s);
    if (e != cudaSuccess) return e;
    k_surface_grad<<<fs_grid((long long)ntri * NT), kFsThreads, 0, s>>>(ntri, NT, map2, vtri, Drn, Dsn, f2, gx, gy);
    k_scale2<<<fs_grid(N2), kFsThreads, 0, s>>>(N2, inv_mult, gx, gy);
    return cudaGetLastError();
}

cudaError_t surface_w(long long N2, int NZ, long long k0, const double* Dtop, double depth, int nlayers,
                      const double* phi, const double* eta, double* w, cudaStream_t s) {
    k_surface_w<<<fs_grid(N2), kFsThreads, 0, s>>>(N2, NZ, k0, Dtop, depth, nlayers, phi, eta, w);
    return cudaGetLastError();
}

cudaError_t fnpf_rhs(long long N2, int linear, double grav, const double* eta, const double* w, const double* ex,
                     const double* ey, const double* px, const double* py, double* deta, double* dphi,
                     cudaStream_t s) {
    k_fnpf_rhs<<<fs_grid(N2), kFsThreads, 0, s>>>(N2, linear, grav, eta, w, ex, ey, px, py, deta, dphi);
    return cudaGetLastError();
}

cudaError_t rk_stage(long long n, double c, const double* x0, const double* k0, const double* x1, const double* k1,
                     double* o0, double* o1, cudaStream_t s) {
    k_stage<<<fs_grid(n), kFsThreads, 0, s>>>(n, c, x0, k0, x1, k1, o0, o1);
    return cudaGetLastError();
}

cudaError_t rk4_combine(long long n, double dt, const double* k, double* x, cudaStream_t s) {
    k_rk4_combine<<<fs_grid(n), kFsThreads, 0, s>>>(n, dt, k, x);
    return cudaGetLastError();
}

}  // namespace sem
