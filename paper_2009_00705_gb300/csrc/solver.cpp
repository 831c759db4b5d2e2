// Solver driver and C ABI: Chebyshev-Jacobi smoothing, the p-multigrid V-cycle
// (Algorithm 1), the FP64 coarse solve, PCG (Algorithm 3), preconditioned
// defect correction (Algorithm 2) and flexible GMRES, plus the entry points
// declared in include/sem.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sem_internal.hpp"

namespace sem {
const char* last_error();
void tri_numbering(int nvert, int ntri, const int* tri, int p, std::vector<int>& map2, long long& N2);
void tri_coords(int ntri, const int* tri, const double* vxy, int p, const std::vector<int>& map2, long long N2,
                std::vector<double>& xy);
void blended_nodes(int ntri, const int* tri, const double* vxy, const double* arc, int p, std::vector<double>& out);
void tri_coords_mapped(int ntri, int P, const std::vector<double>& xyP, int p, const std::vector<int>& map2,
                       long long N2, std::vector<double>& xy);
sem_status check_layers(const sem_handle* h, const std::vector<double>& eta);
sem_status build_level(sem_handle* h, const sem_mesh* m, int li, int p, int pz);
sem_status build_geometry(sem_handle* h, const sem_mesh* m);
sem_status build_diagonals(sem_handle* h);
sem_status build_transfers(sem_handle* h);
sem_status build_coarse_gradients(sem_handle* h);
sem_status geometry_levels(sem_handle* h, int first, int last, bool flat);
sem_status diagonal_level(sem_handle* h, int li);
sem_status reassemble_coarse(sem_handle* h);
sem_status build_mlp(sem_handle* h);
sem_status build_workspace(sem_handle* h);
}  // namespace sem

using namespace sem;

#define CKS(expr)                                                                        \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess) {                                                         \
            set_error(std::string("CUDA error: ") + cudaGetErrorString(_e) + " (" #expr ")"); \
            return SEM_ECUDA;                                                            \
        }                                                                                \
    } while (0)

// K(): one kernel launch of this library (counted in sem_stats.kernel_launches).
#define K(expr)              \
    do {                     \
        CKS(expr);           \
        h->launches += 1;    \
    } while (0)

#define CKST(expr)                      \
    do {                                \
        sem_status _s = (expr);         \
        if (_s != SEM_OK) return _s;    \
    } while (0)

namespace {

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Event timing of finest-level applies (profile = 1, outside graph capture): the pair of
// events brackets the apply kernel alone, on the stream it is launched on.
static bool timed_begin(sem_handle* h, int li, cudaStream_t s) {
    const bool timed = (li == 0) && h->opts.profile && !h->capturing && (h->ev_used + 2 <= (int)h->ev.size());
    if (timed) cudaEventRecord(h->ev[h->ev_used], s);
    return timed;
}
static void timed_end(sem_handle* h, int kind, cudaStream_t s) {
    cudaEventRecord(h->ev[h->ev_used + 1], s);
    h->ev_kind[h->ev_used / 2] = kind;
    h->ev_used += 2;
    if (kind == 0) h->apply_launches += 1;
    else if (kind == 1) h->apply32_launches += 1;
    else if (kind == 2) h->apply_tc_launches += 1;
    else if (kind == 3) h->asm_launches += 1;
    else h->lift_launches += 1;
}

// Finest-level apply with optional event timing (profile = 1).
sem_status apply_level64(sem_handle* h, int li, const double* x, double* y, bool lift, cudaStream_t s) {
    const Level& L = h->lv[li];
    CKS(cudaMemsetAsync(y, 0, sizeof(double) * L.N, s));
    const bool timed = timed_begin(h, li, s);
    K(launch_apply64(L, x, y, lift, nullptr, s));
    if (timed) timed_end(h, lift ? 4 : 0, s);     // the lifting apply covers only the elements at the surface
    if (li == 0) h->fine_applies += 1;
    return SEM_OK;
}

sem_status apply_level32(sem_handle* h, int li, const float* x, float* y, cudaStream_t s,
                         const int* skip = nullptr) {
    const Level& L = h->lv[li];
    CKS(cudaMemsetAsync(y, 0, sizeof(float) * L.N, s));
    const bool timed = timed_begin(h, li, s);
    K(launch_apply32(L, x, y, s, skip));
    if (timed) timed_end(h, 1, s);
    if (li == 0) h->fine_applies += 1;
    return SEM_OK;
}

// Sum the elapsed times of recorded apply events (the stream has been synchronised).
void flush_events(sem_handle* h) {
    for (int i = 0; i + 1 < h->ev_used; i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) != cudaSuccess) continue;
        const int kind = h->ev_kind[i / 2];
        (kind == 0 ? h->apply_ms : kind == 1 ? h->apply32_ms : kind == 2 ? h->apply_tc_ms : kind == 3 ? h->asm_ms
                                                                                                : h->lift_ms) += ms;
    }
    h->ev_used = 0;
}

// FP64 block-Jacobi or Jacobi CG on the coarsest level: x = A_c^{-1} b to coarse_rtol.  The coarse
// matrix is assembled in CSR at setup and the whole CG runs in one persistent
// cooperative launch; coarse levels too large to assemble (high-order single-level
// configurations) launch one kernel per CG step, predicated on a device-side done
// flag, and test convergence every 8 iterations.
sem_status coarse_solve(sem_handle* h, const double* b, double* x, cudaStream_t s) {
    const Level& C = h->lv.back();
    Scratch& sc = h->sc;
    const double rt = h->opts.coarse_rtol;
    if (C.csr_val != nullptr) {
        // one CTA for batched tanks (tanks run concurrently; no inter-CTA waits), the
        // cooperative multi-CTA kernel otherwise
        const bool single = h->opts.batch != 0;
        if (!single && C.bj_nb > 0)
            K(coarse_cg_bj(C, b, x, h->cz, h->cp, h->cq, sc, rt * rt, h->opts.coarse_imax,
                           (unsigned)h->opts.debug_barrier_extra, s));
        else if (single)
            K(coarse_cg_single(C, C.csr_rowptr, C.csr_col, C.csr_val, b, x, h->cr, h->cz, h->cp, h->cq, sc, rt * rt,
                               h->opts.coarse_imax, s));
        else
            K(coarse_cg_persistent(C, C.csr_rowptr, C.csr_col, C.csr_val, b, x, h->cr, h->cz, h->cp, h->cq, sc,
                                   rt * rt, h->opts.coarse_imax, (unsigned)h->opts.debug_barrier_extra, s));
        if (h->capturing) return SEM_OK;     // checked after the batched solve
        CKS(cudaMemcpyAsync(sc.hflags, sc.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CKS(cudaMemcpyAsync(sc.hpinned + S_CG_RR, sc.scal + S_CG_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
        sc.hflags[4] = 0;
        if (!single) CKS(cudaMemcpyAsync(sc.hflags + 4, sc.counter + 3, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CKS(cudaStreamSynchronize(s));
        if (sc.hflags[4] != 0) {
            set_error("coarse CG: a grid barrier wait ran out (device timeout)");
            return SEM_TIMEOUT;
        }
        if (!std::isfinite(sc.hpinned[S_CG_RR])) {
            set_error("coarse CG: non-finite residual (non-finite right-hand side)");
            return SEM_NAN;
        }
    } else {
        K(cg_init(C.N, b, C.dinv, x, h->cr, h->cz, h->cp, sc, rt * rt, s));
        int it = 0;
        const int chunk = 8;
        while (it < h->opts.coarse_imax) {
            for (int k = 0; k < chunk; ++k) {
                CKS(cudaMemsetAsync(h->cq, 0, sizeof(double) * C.N, s));
                K(launch_apply64(C, h->cp, h->cq, false, sc.flags + F_CG_DONE, s));
                K(cg_pq(C.N, h->cp, h->cq, sc, s));
                K(cg_update(C.N, C.dinv, x, h->cr, h->cz, h->cp, h->cq, sc, s));
                K(cg_direction(C.N, h->cz, h->cp, sc, s));
            }
            it += chunk;
            CKS(cudaMemcpyAsync(sc.hflags, sc.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
            CKS(cudaStreamSynchronize(s));
            if (sc.hflags[F_CG_DONE]) break;
        }
    }
    const int used = sc.hflags[F_CG_ITERS];
    h->coarse_iters_max = std::max(h->coarse_iters_max, used);
    if (!sc.hflags[F_CG_DONE]) {
        set_error("coarse CG did not reach coarse_rtol within coarse_imax iterations");
        return SEM_NOT_CONVERGED;
    }
    return SEM_OK;
}

// One smoothing sweep of level li (u = 0 on entry when zero_init; post: after the
// coarse-grid correction): Chebyshev-Jacobi, or the additive Schwarz step
// u <- u + S^{-1}(f - A u) (Eq. sec_form) with the adjoint of S^{-1} after the correction.
template <typename T>
sem_status smooth(sem_handle* h, int li, const T* f, T* u, bool zero_init, bool post, cudaStream_t s,
                  const int* skip = nullptr);

static sem_status asm_sweep64(sem_handle* h, int li, const double* f, double* u, bool zero_init, bool post,
                              cudaStream_t s) {
    Level& L = h->lv[li];
    if (zero_init) CKS(cudaMemsetAsync(u, 0, sizeof(double) * L.N, s));
    else CKST(apply_level64(h, li, u, L.y, false, s));
    const bool timed = timed_begin(h, li, s);
    K(asm_apply64(L, f, zero_init ? nullptr : L.y, post ? 1 : 0, u, s));
    if (timed) timed_end(h, 3, s);
    return SEM_OK;
}

template <>
sem_status smooth<double>(sem_handle* h, int li, const double* f, double* u, bool zero_init, bool post,
                          cudaStream_t s, const int*) {
    if (h->opts.smoother == SEM_SMOOTH_ASM) return asm_sweep64(h, li, f, u, zero_init, post, s);
    const Level& L = h->lv[li];
    const Cheb c = cheb_coeffs(L.lam, h->opts);
    if (zero_init) {
        K(cheb_first<double>(L.N, c.c0, L.dinv, f, u, L.d, s));
    } else {
        CKST(apply_level64(h, li, u, L.y, false, s));
        K(cheb_restart<double>(L.N, c.c0, L.dinv, f, L.y, u, L.d, s));
    }
    for (int j = 1; j < h->opts.k_cheb; ++j) {
        CKST(apply_level64(h, li, u, L.y, false, s));
        K(cheb_step<double>(L.N, c.c1[j], c.c2[j], L.dinv, f, L.y, u, L.d, s));
    }
    return SEM_OK;
}

// The operator inside the single-precision V-cycle (Chebyshev sweeps and the residual
// before restriction): the TF32 tensor-core prism apply in MIXED_TF32 (orders 2..6), the
// FP32 apply otherwise.  The inner PCG's own products keep the FP32 apply.
static sem_status apply_vcycle32(sem_handle* h, int li, const float* x, float* y, cudaStream_t s, const int* skip) {
    const Level& L = h->lv[li];
    if (h->opts.precision != SEM_PREC_MIXED_TF32 || !level_tc(L))
        return apply_level32(h, li, x, y, s, skip);
    CKS(cudaMemsetAsync(y, 0, sizeof(float) * L.N, s));
    const bool timed = timed_begin(h, li, s);
    K(launch_apply_tensor(L, x, y, skip, h->sc.flags + F_TC_ERR, s, L.tc_kind == 1 && L.G16T != nullptr));
    if (timed) timed_end(h, 2, s);
    if (li == 0) h->fine_applies += 1;
    return SEM_OK;
}

static sem_status asm_sweep32(sem_handle* h, int li, const float* f, float* u, bool zero_init, bool post,
                              cudaStream_t s) {
    Level& L = h->lv[li];
    if (zero_init) CKS(cudaMemsetAsync(u, 0, sizeof(float) * L.N, s));
    else CKST(apply_vcycle32(h, li, u, L.y32, s, nullptr));
    const bool timed = timed_begin(h, li, s);
    K(asm_apply32(L, f, zero_init ? nullptr : L.y32, post ? 1 : 0, u, s));
    if (timed) timed_end(h, 3, s);
    return SEM_OK;
}

template <>
sem_status smooth<float>(sem_handle* h, int li, const float* f, float* u, bool zero_init, bool post,
                         cudaStream_t s, const int* skip) {
    if (h->opts.smoother == SEM_SMOOTH_ASM) return asm_sweep32(h, li, f, u, zero_init, post, s);
    const Level& L = h->lv[li];
    const Cheb c = cheb_coeffs(L.lam, h->opts);
    if (zero_init) {
        K(cheb_first<float>(L.N, (float)c.c0, L.dinv32, f, u, L.d32, s, skip));
    } else {
        CKST(apply_vcycle32(h, li, u, L.y32, s, skip));
        K(cheb_restart<float>(L.N, (float)c.c0, L.dinv32, f, L.y32, u, L.d32, s, skip));
    }
    for (int j = 1; j < h->opts.k_cheb; ++j) {
        CKST(apply_vcycle32(h, li, u, L.y32, s, skip));
        K(cheb_step<float>(L.N, (float)c.c1[j], (float)c.c2[j], L.dinv32, f, L.y32, u, L.d32, s, skip));
    }
    return SEM_OK;
}

// The learned sweep that stands in for the first finest-level post-smoothing sweep: the
// network's correction delta = W sum_e Q_e^T s_e MLP(z_e / s_e), z = D^{-1}(f - A u),
// s_e = ||z_e||, taken with the minimal-residual step alpha = (r, A delta) / ||A delta||^2
// (the alpha minimising ||r - alpha A delta||, one apply as before).  It is kept only if it
// lowers the residual norm below learned_tau times its value; otherwise the Chebyshev sweep
// it replaces runs instead (its kernels are predicated on the device-side verdict).
sem_status learned_sweep(sem_handle* h, const float* f, float* u, cudaStream_t s) {
    Level& L = h->lv[0];
    const long long N = L.N;
    Scratch& sc = h->sc;
    CKST(apply_level32(h, 0, u, L.y32, s));
    K(axpby32(N, f, L.y32, -1.f, h->lr32, s));                     // r = f - A u
    K(dot32(N, h->lr32, h->lr32, sc, sc.scal + S_L0, s));
    K(mul32(N, L.dinv32, h->lr32, h->ld32, s));
    K(gather_scaled<float>(L.E, L.Np, L.map, h->ld32, (const float*)nullptr, h->mX, nullptr, h->mscale, s));
    CKS(mlp_forward(h->net, L.E, h->mX, h->mA1, h->mH1, h->mY, s));
    h->launches += 2;
    CKS(cudaMemsetAsync(h->ld32, 0, sizeof(float) * N, s));
    K(scatter_correction(L.E, L.Np, L.map, L.wmult32, h->mY, h->mscale, h->ld32, s));   // delta
    CKST(apply_level32(h, 0, h->ld32, L.y32, s));                  // q = A delta
    K(dot32(N, h->lr32, L.y32, sc, sc.scal + S_RQ, s));
    K(dot32(N, L.y32, L.y32, sc, sc.scal + S_QQ, s));
    const double tau = h->opts.learned_tau;
    K(judge_min_residual(sc.scal + S_L0, sc.scal + S_RQ, sc.scal + S_QQ, sc.scal + S_ALPHA, sc.flags, F_LEARN_ACCEPT,
                         F_LEARN_COUNT, tau * tau, s));
    K(axpy_accepted32(N, sc.flags, F_LEARN_ACCEPT, sc.scal + S_ALPHA, h->ld32, u, s));
    return smooth<float>(h, 0, f, u, false, true, s, sc.flags + F_LEARN_ACCEPT);
}

// Algorithm 1 with zero initial guess on every level, FP64 throughout.
sem_status vcycle64(sem_handle* h, const double* f0, double* u0, cudaStream_t s) {
    const int nl = (int)h->lv.size();
    h->vcycles += 1;
    if (nl == 1) return coarse_solve(h, f0, u0, s);
    for (int li = 0; li + 1 < nl; ++li) {
        Level& L = h->lv[li];
        Level& C = h->lv[li + 1];
        const double* f = (li == 0) ? f0 : L.f;
        double* u = (li == 0) ? u0 : L.u;
        for (int m = 0; m < h->opts.nu1; ++m) CKST(smooth<double>(h, li, f, u, m == 0, false, s));
        if (h->opts.nu1 == 0) CKS(cudaMemsetAsync(u, 0, sizeof(double) * L.N, s));
        CKST(apply_level64(h, li, u, L.y, false, s));
        CKS(cudaMemsetAsync(C.f, 0, sizeof(double) * C.N, s));
        K(launch_restrict64(L, C, f, L.y, C.f, s));
    }
    const sem_status cs = coarse_solve(h, h->lv[nl - 1].f, h->lv[nl - 1].u, s);
    if (cs != SEM_OK) return cs;
    for (int li = nl - 2; li >= 0; --li) {
        Level& L = h->lv[li];
        const Level& C = h->lv[li + 1];
        const double* f = (li == 0) ? f0 : L.f;
        double* u = (li == 0) ? u0 : L.u;
        K(launch_prolong64(L, C, C.u, u, s));
        for (int m = 0; m < h->opts.nu2; ++m) CKST(smooth<double>(h, li, f, u, false, true, s));
    }
    return SEM_OK;
}

// Algorithm 1 in FP32 on every level but the coarsest, which is solved in FP64.
sem_status vcycle32(sem_handle* h, const float* f0, float* u0, cudaStream_t s) {
    const int nl = (int)h->lv.size();
    h->vcycles += 1;
    Level& Cc = h->lv[nl - 1];
    if (nl == 1) {
        K(to_f64(Cc.N, f0, h->cb, s));
        CKST(coarse_solve(h, h->cb, Cc.u, s));
        K(to_f32(Cc.N, Cc.u, u0, s));
        return SEM_OK;
    }
    for (int li = 0; li + 1 < nl; ++li) {
        Level& L = h->lv[li];
        Level& C = h->lv[li + 1];
        const float* f = (li == 0) ? f0 : L.f32;
        float* u = (li == 0) ? u0 : L.u32;
        const bool skip_fine = (li == 0) && h->cgc_only;
        if (!skip_fine)
            for (int m = 0; m < h->opts.nu1; ++m) CKST(smooth<float>(h, li, f, u, m == 0, false, s));
        if (h->opts.nu1 == 0 || skip_fine) CKS(cudaMemsetAsync(u, 0, sizeof(float) * L.N, s));
        if (skip_fine) CKS(cudaMemsetAsync(L.y32, 0, sizeof(float) * L.N, s));
        else CKST(apply_vcycle32(h, li, u, L.y32, s, nullptr));
        CKS(cudaMemsetAsync(C.f32, 0, sizeof(float) * C.N, s));
        K(launch_restrict32(L, C, f, L.y32, C.f32, s));
    }
    K(to_f64(Cc.N, Cc.f32, h->cb, s));
    const sem_status cs = coarse_solve(h, h->cb, Cc.u, s);
    if (cs != SEM_OK) return cs;
    K(to_f32(Cc.N, Cc.u, Cc.u32, s));
    for (int li = nl - 2; li >= 0; --li) {
        Level& L = h->lv[li];
        const Level& C = h->lv[li + 1];
        const float* f = (li == 0) ? f0 : L.f32;
        float* u = (li == 0) ? u0 : L.u32;
        K(launch_prolong32(L, C, C.u32, u, s));
        const bool learned = (li == 0) && h->opts.smoother == SEM_SMOOTH_LEARNED && h->mlp_trained && h->learned_active;
        if ((li == 0) && h->cgc_only) continue;
        for (int m = 0; m < h->opts.nu2; ++m) {
            if (learned && m == 0) CKST(learned_sweep(h, f, u, s));
            else CKST(smooth<float>(h, li, f, u, false, true, s));
        }
    }
    return SEM_OK;
}

sem_status read_scalars(sem_handle* h, int first, int count, cudaStream_t s);

// Inner FP32 PCG on A e = r (FP32 V-cycle preconditioner, FP64-accumulated dots) to
// inner_rtol; e is returned in FP64.  r has zero Dirichlet entries.
sem_status inner_pcg32(sem_handle* h, const double* r, double* e, cudaStream_t s) {
    const Level& L = h->lv[0];
    const long long N = L.N;
    Scratch& sc = h->sc;
    K(to_f32(N, r, h->ir, s));
    CKS(cudaMemsetAsync(h->ie, 0, sizeof(float) * N, s));
    K(dot32(N, h->ir, h->ir, sc, sc.scal + S_IRR, s));
    CKST(read_scalars(h, S_IRR, 1, s));
    const double tol2 = h->opts.inner_rtol * h->opts.inner_rtol * sc.hpinned[S_IRR];
    if (sc.hpinned[S_IRR] > 0.0) {
        CKST(vcycle32(h, h->ir, h->iz, s));
        CKS(cudaMemcpyAsync(h->ip, h->iz, sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
        int cur = S_IDELTA0, nxt = S_IDELTA1;
        K(dot32(N, h->iz, h->ir, sc, sc.scal + cur, s));
        for (int it = 0; it < h->opts.inner_imax; ++it) {
            CKST(apply_level32(h, 0, h->ip, h->iq, s));
            K(dot32(N, h->ip, h->iq, sc, sc.scal + S_IPQ, s));
            K(pcg_update32(N, sc.scal + cur, sc.scal + S_IPQ, h->ip, h->iq, h->ie, h->ir, sc, sc.scal + S_IRR, s));
            h->inner_iters += 1;
            CKST(read_scalars(h, S_IRR, 2, s));
            if (!(sc.hpinned[S_IPQ] > 0.0) || !std::isfinite(sc.hpinned[S_IRR])) break;
            if (sc.hpinned[S_IRR] <= tol2) break;
            CKST(vcycle32(h, h->ir, h->iz, s));
            K(dot32(N, h->iz, h->ir, sc, sc.scal + nxt, s));
            K(pcg_direction32(N, sc.scal + nxt, sc.scal + cur, h->iz, h->ip, s));
            std::swap(cur, nxt);
        }
    }
    K(to_f64(N, h->ie, e, s));
    return SEM_OK;
}

// z = M^{-1} r on the finest level in the configured precision (r has zero Dirichlet entries).
sem_status precondition(sem_handle* h, const double* r, double* z, cudaStream_t s) {
    if (h->opts.precision != SEM_PREC_FP64) {
        if (h->opts.inner_imax > 0) return inner_pcg32(h, r, z, s);
        Level& L = h->lv[0];
        K(to_f32(L.N, r, L.f32, s));
        CKST(vcycle32(h, L.f32, L.u32, s));
        K(to_f64(L.N, L.u32, z, s));
        return SEM_OK;
    }
    return vcycle64(h, r, z, s);
}

sem_status read_scalars(sem_handle* h, int first, int count, cudaStream_t s) {
    CKS(cudaMemcpyAsync(h->sc.hpinned + first, h->sc.scal + first, count * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKS(cudaStreamSynchronize(s));
    if (h->opts.profile) flush_events(h);
    return SEM_OK;
}

// Largest eigenvalue of the symmetric tridiagonal matrix with diagonal a[0..k) and
// off-diagonal b[0..k-1), by bisection on the Sturm count (the number of
// eigenvalues below x equals the number of negative pivots of T - x I).
static double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
    const int k = (int)a.size();
    double lo = a[0], hi = a[0];
    for (int j = 0; j < k; ++j) {
        const double r = (j > 0 ? std::fabs(b[j - 1]) : 0.0) + (j + 1 < k ? std::fabs(b[j]) : 0.0);
        lo = std::min(lo, a[j] - r);
        hi = std::max(hi, a[j] + r);
    }
    auto below = [&](double x) {
        int cnt = 0;
        double d = 1.0;
        for (int j = 0; j < k; ++j) {
            const double bb = j > 0 ? b[j - 1] * b[j - 1] : 0.0;
            d = (a[j] - x) - (j > 0 ? bb / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0.0) ++cnt;
        }
        return cnt;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (below(mid) < k) lo = mid;     // some eigenvalue lies at or above mid
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// lambda_hat of D^{-1} A on level li: the largest Ritz value of lanczos_steps Lanczos
// steps, taken from Jacobi-preconditioned CG on A x = x0 (x0_i = sin(i + 1) on the
// free nodes) through the CG-Lanczos relation T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
// T_j,j+1 = sqrt(beta_j)/alpha_j (e.g. Saad, Iterative Methods for Sparse Linear
// Systems, Sec. 6.7.3).  The estimate is a lower bound of lambda_max; power
// iteration converges too slowly on some sigma-prism meshes for the Chebyshev
// interval to cover the top of the spectrum.
sem_status estimate_lambda(sem_handle* h, int li, bool fp32_apply) {
    Level& L = h->lv[li];
    std::vector<double> x0(L.N, 0.0);
    std::vector<char> dm(L.N, 0);
    for (long long i : L.hdir) dm[i] = 1;
    for (long long i = 0; i < L.N; ++i)
        if (!dm[i]) x0[i] = std::sin((double)i + 1.0);
    CKS(cudaMemcpy(L.f, x0.data(), sizeof(double) * L.N, cudaMemcpyHostToDevice));
    cudaStream_t s = 0;
    Scratch& sc = h->sc;
    K(cg_init(L.N, L.f, L.dinv, L.u, h->r, h->z, h->p, sc, 0.0, s));
    std::vector<double> alpha, beta;
    for (int it = 0; it < h->opts.lanczos_steps; ++it) {
        if (fp32_apply) {
            // the single-precision operator the mixed V-cycle smooths with (FP64 Lanczos recurrence)
            K(to_f32(L.N, h->p, L.u32, s));
            CKS(cudaMemsetAsync(L.y32, 0, sizeof(float) * L.N, s));
            K(launch_apply32(L, L.u32, L.y32, s));
            K(to_f64(L.N, L.y32, h->q, s));
        } else {
            CKS(cudaMemsetAsync(h->q, 0, sizeof(double) * L.N, s));
            K(launch_apply64(L, h->p, h->q, false, nullptr, s));
        }
        K(cg_pq(L.N, h->p, h->q, sc, s));
        double rp[2];                                          // rho_j, p_j^T A p_j
        CKS(cudaMemcpy(rp, sc.scal + S_CG_RHO, 2 * sizeof(double), cudaMemcpyDeviceToHost));
        if (!(rp[0] > 0.0) || !(rp[1] > 0.0) || !std::isfinite(rp[0] / rp[1])) break;
        alpha.push_back(rp[0] / rp[1]);
        K(cg_update(L.N, L.dinv, L.u, h->r, h->z, h->p, h->q, sc, s));
        double bt = 0.0;
        CKS(cudaMemcpy(&bt, sc.scal + S_CG_BETA, sizeof(double), cudaMemcpyDeviceToHost));
        if (!(bt > 0.0) || !std::isfinite(bt)) break;          // Krylov space exhausted: T is exact
        beta.push_back(bt);
        K(cg_direction(L.N, h->z, h->p, sc, s));
    }
    if (alpha.empty()) { set_error("eigenvalue estimate: no Lanczos step (zero or indefinite level)"); return SEM_BREAKDOWN; }
    const int k = (int)alpha.size();
    std::vector<double> a(k), b(k > 1 ? k - 1 : 0);
    for (int j = 0; j < k; ++j) {
        a[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
        if (j + 1 < k) b[j] = std::sqrt(beta[j]) / alpha[j];
    }
    L.lam = tridiag_max_eig(a, b);
    if (!std::isfinite(L.lam) || !(L.lam > 0.0)) { set_error("eigenvalue estimate not finite"); return SEM_NAN; }
    return SEM_OK;
}

// Tile-shape autotuner of the prism apply: times both compiled variants (elements per
// CTA pass) on this level's own mesh and keeps the faster; the choice is cached per
// (order, precision, element-count bucket) for the rest of the process, so the tanks
// of a batch are tuned once per kind.
std::map<std::tuple<int, int, int>, int> g_tile_cache;
std::mutex g_tile_mutex;

cudaError_t tune_prism(Level& L, bool fp32) {
    int bucket = 0;
    while ((1 << (bucket + 1)) <= L.E) ++bucket;
    const auto key = std::make_tuple(L.p * 8 + L.pz, fp32 ? 4 : 8, bucket);
    {
        std::lock_guard<std::mutex> lock(g_tile_mutex);
        auto it = g_tile_cache.find(key);
        if (it != g_tile_cache.end()) {
            (fp32 ? L.tile32 : L.tile64) = it->second;
            return cudaSuccess;
        }
    }
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    float best = 1e30f;
    int choice = 0;
    for (int v = 0; v < 2 && err == cudaSuccess; ++v) {
        for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
            if (rep == 1) err = cudaEventRecord(e0, 0);
            if (fp32) {
                cudaMemsetAsync(L.y32, 0, sizeof(float) * L.N, 0);
                err = launch_apply_prism32(L, L.u32, L.y32, nullptr, v, 0);
            } else {
                cudaMemsetAsync(L.y, 0, sizeof(double) * L.N, 0);
                err = launch_apply_prism64(L, L.u, L.y, false, nullptr, v, 0);
            }
        }
        if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && ms < best) { best = ms; choice = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return err;
    (fp32 ? L.tile32 : L.tile64) = choice;
    std::lock_guard<std::mutex> lock(g_tile_mutex);
    g_tile_cache[key] = choice;
    return cudaSuccess;
}

// The tensor-core smoothing operator of an order-6 level: times the warp-level MMA kernel and
// the tcgen05 kernel on the level's own mesh and keeps the faster (cached like the tile shapes).
std::map<std::pair<int, int>, int> g_tc_cache;

cudaError_t tune_tc(Level& L) {
    L.tc_kind = 0;
    if (!level_tc(L) || L.G16T == nullptr || !prism_t5_supported(L.p)) return cudaSuccess;
    int bucket = 0;
    while ((1 << (bucket + 1)) <= L.E) ++bucket;
    const auto key = std::make_pair(L.p, bucket);
    {
        std::lock_guard<std::mutex> lock(g_tile_mutex);
        auto it = g_tc_cache.find(key);
        if (it != g_tc_cache.end()) {
            L.tc_kind = it->second;
            return cudaSuccess;
        }
    }
    // the kernels' error flag: a kernel whose bounded copy or MMA wait ran out sets it, and such
    // a kernel is not a candidate; none completing is an error of the setup
    int* err = nullptr;
    cudaError_t e = cudaMalloc(&err, sizeof(int));
    if (e != cudaSuccess) return e;
    e = cudaMemset(err, 0, sizeof(int));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    int choice = 0;
    bool any = false;
    for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
            if (rep == 1) e = cudaEventRecord(e0, 0);
            cudaMemsetAsync(L.y32, 0, sizeof(float) * L.N, 0);
            if (e == cudaSuccess) e = launch_apply_tensor(L, L.u32, L.y32, nullptr, err, 0, v == 1);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        int timed_out = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&timed_out, err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && timed_out) {
            e = cudaMemset(err, 0, sizeof(int));
            continue;
        }
        if (e == cudaSuccess && ms < best) { best = ms; choice = v; }
        if (e == cudaSuccess) any = true;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(err);
    if (e == cudaSuccess && !any) e = cudaErrorLaunchTimeout;
    if (e != cudaSuccess) return e;
    L.tc_kind = choice;
    std::lock_guard<std::mutex> lock(g_tile_mutex);
    g_tc_cache[key] = choice;
    return cudaSuccess;
}

// The node -> element-slot map of a level for the atomic-free direct-stiffness summation:
// for every node g, the slots e * Np + l whose map entry names g (free or Dirichlet) in
// ascending (e, l) order (a counting sort over the element map), and the FP64
// element-result buffer.
sem_status build_dss(Level& L) {
    const long long slots = (long long)L.E * L.Np;
    if (slots >= (1LL << 31) || L.N >= (1LL << 31)) {
        set_error("deterministic: the level has too many element slots for 32-bit indices");
        return SEM_EINVAL;
    }
    auto node = [&](long long i) -> long long { const int m = L.hmap[i]; return m >= 0 ? m : -(long long)m - 1; };
    std::vector<int> ptr((size_t)L.N + 1, 0);
    for (long long i = 0; i < slots; ++i) ++ptr[(size_t)node(i) + 1];
    for (long long g = 0; g < L.N; ++g) ptr[(size_t)g + 1] += ptr[(size_t)g];
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    std::vector<int> slot((size_t)slots);
    for (long long i = 0; i < slots; ++i) slot[(size_t)fill[(size_t)node(i)]++] = (int)i;
    void* p = nullptr;
    CKS(cudaMalloc(&p, sizeof(int) * ptr.size()));
    L.dss_ptr = static_cast<int*>(p);
    CKS(cudaMemcpy(L.dss_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice));
    CKS(cudaMalloc(&p, sizeof(int) * (slot.empty() ? 1 : slot.size())));
    L.dss_slot = static_cast<int*>(p);
    if (!slot.empty()) CKS(cudaMemcpy(L.dss_slot, slot.data(), sizeof(int) * slot.size(), cudaMemcpyHostToDevice));
    CKS(cudaMalloc(&p, sizeof(double) * (size_t)slots));
    L.ye64 = static_cast<double*>(p);
    CKS(cudaMemset(L.ye64, 0, sizeof(double) * (size_t)slots));
    return SEM_OK;
}

// Element matrices held by all live handles that took them by the auto rule.
std::atomic<size_t> g_auto_elem_bytes{0};
constexpr size_t kAutoElemBudget = (size_t)48 << 30;

// Device storage of the element matrices of the FP64 applies (sem_options.elem_matrices): every
// level of an FP64 handle but the coarsest, the finest of a mixed-precision one; FP64 matrices or
// the double-FP32 block triangle; in auto mode only when they take at most a quarter of the free
// device memory and, with those of the other live handles (many batched tanks), 48 GB.
sem_status alloc_element_matrices(sem_handle* h) {
    const int nl = (int)h->lv.size();
    const int last = h->opts.precision == SEM_PREC_FP64 ? nl - 1 : std::min(1, nl - 1);
    int kind = h->opts.elem_matrices;
    if (kind < 0) kind = h->opts.precision == SEM_PREC_FP64 ? SEM_ELEM_FP64 : SEM_ELEM_DF32;
    auto level_bytes = [&](Level& L) -> size_t {
        if (kind == SEM_ELEM_FP64) return sizeof(double) * (size_t)L.E * L.Np * L.Np;
        df_layout(L.Np, &L.df_T, &L.df_NB, &L.df_S, &L.df_TS);
        return sizeof(float2) * (size_t)L.E * (L.df_NB * (L.df_NB + 1) / 2) * L.df_TS;
    };
    size_t bytes = 0;
    for (int li = 0; li < last; ++li) bytes += level_bytes(h->lv[li]);
    if (bytes == 0) return SEM_OK;
    if (h->opts.elem_matrices < 0) {
        if (h->opts.batch != 0) return SEM_OK;          // many small tanks: setup time would dominate
        size_t fr = 0, tot = 0;
        CKS(cudaMemGetInfo(&fr, &tot));
        if (bytes > fr / 4) return SEM_OK;                                   // sum factorisation
        size_t cur = g_auto_elem_bytes.load();
        do {
            if (cur + bytes > kAutoElemBudget) return SEM_OK;
        } while (!g_auto_elem_bytes.compare_exchange_weak(cur, cur + bytes));
        h->auto_elem_bytes = bytes;
    }
    for (int li = 0; li < last; ++li) {
        Level& L = h->lv[li];
        void* p = nullptr;
        const cudaError_t e = cudaMalloc(&p, level_bytes(L));
        if (e != cudaSuccess) {
            set_error("element matrices: " + std::string(cudaGetErrorString(e)));
            return SEM_ENOMEM;
        }
        if (kind == SEM_ELEM_FP64) L.Ae64 = static_cast<double*>(p);
        else L.Adf = static_cast<float2*>(p);
    }
    return SEM_OK;
}

void free_level(Level& L) {
    void* ptrs[] = {L.map, L.G, L.G32, L.G16, L.G16T, L.lift_elems, L.dinv, L.dinv32, L.dir, L.ref64.m, L.ref32.m, L.It64, L.Iz64, L.It32, L.Iz32, L.gref,
                    L.csr_rowptr, L.csr_col, L.csr_val, L.csr_slot, L.dss_ptr, L.dss_slot, L.ye64, L.csr_eptr, L.csr_eidx, L.csr_ev, L.Ae64, L.Adf, L.bj_ptr, L.bj_rows, L.bj_inv, L.bj_lptr, L.bj_lidx,
                    L.owner, L.wmult, L.wmult32, L.u, L.f, L.y, L.d, L.u32, L.f32, L.y32, L.d32};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    free_asm_level(L);
}

sem_status check_mesh(const sem_mesh* m, int P) {
    if (!m || (m->dim != 2 && m->dim != 3)) { set_error("mesh->dim must be 2 or 3"); return SEM_EINVAL; }
    if (P < 1 || P > 6) { set_error("P must be in 1..6"); return SEM_EINVAL; }
    if (m->nvert < 3 || m->ntri < 1 || !m->vxy || !m->tri || !m->face_bc) {
        set_error("mesh arrays missing or empty");
        return SEM_EINVAL;
    }
    for (long long i = 0; i < 3LL * m->ntri; ++i)
        if (m->tri[i] < 0 || m->tri[i] >= m->nvert) { set_error("triangle vertex id out of range"); return SEM_EINVAL; }
    for (int b = 0; b < m->ntri; ++b) {
        const double* a = m->vxy + 2 * m->tri[3 * b];
        const double* c1 = m->vxy + 2 * m->tri[3 * b + 1];
        const double* c2 = m->vxy + 2 * m->tri[3 * b + 2];
        const double area2 = (c1[0] - a[0]) * (c2[1] - a[1]) - (c2[0] - a[0]) * (c1[1] - a[1]);
        if (!(area2 > 0.0)) { set_error("triangle not counter-clockwise or degenerate"); return SEM_EINVAL; }
    }
    if (m->dim == 3 && (m->nlayers < 1 || !(m->depth > 0.0))) {
        set_error("dim 3 needs nlayers >= 1 and depth > 0");
        return SEM_EINVAL;
    }
    if (m->dim == 2 && (m->col_layers || m->z_iface || m->edge_arc)) {
        set_error("col_layers, z_iface and edge_arc describe prism meshes only");
        return SEM_EINVAL;
    }
    if (m->col_layers)
        for (int b = 0; b < m->ntri; ++b)
            if (m->col_layers[b] < 1 || m->col_layers[b] > m->nlayers) {
                set_error("col_layers entries must lie in 1..nlayers");
                return SEM_EINVAL;
            }
    if (m->z_iface)
        for (int k = 0; k <= 2 * m->nlayers + 1; ++k)
            if (!std::isfinite(m->z_iface[k])) { set_error("z_iface entries must be finite"); return SEM_EINVAL; }
    if (m->edge_arc)
        for (int b = 0; b < m->ntri; ++b)
            for (int f = 0; f < 3; ++f) {
                const double* c = m->edge_arc + 9 * (size_t)b + 3 * f;
                if (!(c[2] >= 0.0) || !std::isfinite(c[0]) || !std::isfinite(c[1]) || !std::isfinite(c[2])) {
                    set_error("edge_arc: radius must be >= 0 and finite");
                    return SEM_EINVAL;
                }
                if (c[2] == 0.0) continue;
                const double* va = m->vxy + 2 * m->tri[3 * b + f];
                const double* vb = m->vxy + 2 * m->tri[3 * b + (f + 1) % 3];
                const double ra = std::hypot(va[0] - c[0], va[1] - c[1]), rb = std::hypot(vb[0] - c[0], vb[1] - c[1]);
                const double dth = std::remainder(std::atan2(vb[1] - c[1], vb[0] - c[0]) -
                                                      std::atan2(va[1] - c[1], va[0] - c[0]), 2.0 * M_PI);
                if (std::fabs(ra - c[2]) > 1e-9 * c[2] || std::fabs(rb - c[2]) > 1e-9 * c[2] ||
                    !(std::fabs(dth) < 0.5 * M_PI + 1e-12)) {
                    set_error("edge_arc: a curved edge's vertices must lie on its circle, at most a quarter turn apart");
                    return SEM_EINVAL;
                }
            }
    return SEM_OK;
}

// Vertical order of level li: level_pz[li] when set (prisms), else the triangle order.
int level_pz(const sem_options& o, int li, int dim) {
    return (dim == 3 && o.level_pz[li] > 0) ? o.level_pz[li] : o.level_p[li];
}

// Orders per level: neither order grows from one level to the next and at least one
// falls (semi-coarsening lowers one direction only); the coarsest level is (1, 1);
// anisotropic prism levels must be pairs the prism apply is compiled for.
sem_status check_orders(const sem_options& o, int dim) {
    for (int i = 0; i < o.nlevels; ++i) {
        const int p = o.level_p[i], pz = level_pz(o, i, dim);
        if (dim == 2 && o.level_pz[i] != 0 && o.level_pz[i] != p) {
            set_error("level_pz: a separate vertical order needs a prism mesh");
            return SEM_EINVAL;
        }
        if (p < 1 || p > 6 || pz < 1 || pz > 6) { set_error("orders in 1..6"); return SEM_EINVAL; }
        if (dim == 3 && !prism_pair_supported(p, pz)) {
            set_error("prism orders (" + std::to_string(p) + ", " + std::to_string(pz) +
                      ") not compiled: the vertical order must equal the triangle order or lie one or two below it");
            return SEM_EINVAL;
        }
        if (i > 0) {
            const int pp = o.level_p[i - 1], ppz = level_pz(o, i - 1, dim);
            if (p > pp || pz > ppz || (p == pp && pz == ppz)) {
                set_error("level orders: neither may grow and one must fall from one level to the next");
                return SEM_EINVAL;
            }
        }
    }
    if (level_pz(o, o.nlevels - 1, dim) != 1) { set_error("the coarsest level must be of order (1, 1)"); return SEM_EINVAL; }
    return SEM_OK;
}

sem_status check_options(const sem_options& o, int P) {
    if (o.nlevels < 1 || o.nlevels > SEM_MAX_LEVELS || o.level_p[0] != P || o.level_p[o.nlevels - 1] != 1) {
        set_error("levels must run from P down to 1");
        return SEM_EINVAL;
    }
    if (o.k_cheb < 1 || o.k_cheb > 15 || o.nu1 < 0 || o.nu2 < 0 || o.lanczos_steps < 1) {
        set_error("smoother parameters out of range");
        return SEM_EINVAL;
    }
    if (!(o.cheb_hi > 0) || !(o.cheb_lo > 0) || !(o.cheb_lo < 1)) { set_error("Chebyshev bounds"); return SEM_EINVAL; }
    if (o.outer < 0 || o.outer > 2 || o.precision < 0 || o.precision > 2) { set_error("outer/precision"); return SEM_EINVAL; }
    if (o.outer == SEM_OUTER_FGMRES && (o.gmres_m < 1 || o.gmres_m > 64)) { set_error("gmres_m in 1..64"); return SEM_EINVAL; }
    if (o.imax < 0 || o.coarse_imax < 1 || !(o.coarse_rtol > 0)) { set_error("iteration limits"); return SEM_EINVAL; }
    if (o.batch_mode < 0 || o.batch_mode > 1) { set_error("batch_mode 0 or 1"); return SEM_EINVAL; }
    if (!(o.learned_tau > 0.0 && o.learned_tau <= 1.0)) { set_error("0 < learned_tau <= 1"); return SEM_EINVAL; }
    if (o.smoother < SEM_SMOOTH_CHEBYSHEV || o.smoother > SEM_SMOOTH_ASM) { set_error("smoother"); return SEM_EINVAL; }
    if (o.smoother == SEM_SMOOTH_ASM && (o.asm_overlap < -1 || o.asm_overlap > 16)) {
        set_error("asm_overlap in -1..16");
        return SEM_EINVAL;
    }
    if (o.smoother == SEM_SMOOTH_LEARNED && (o.precision == SEM_PREC_FP64 || o.mlp_hidden < 1 || o.mlp_hidden > 4096)) {
        set_error("the learned smoother needs a mixed precision and 1 <= mlp_hidden <= 4096");
        return SEM_EINVAL;
    }
    if (o.inner_imax < 0 || (o.inner_imax > 0 && !(o.inner_rtol > 0 && o.inner_rtol < 1))) {
        set_error("inner_imax >= 0 and 0 < inner_rtol < 1");
        return SEM_EINVAL;
    }
    if (o.coarse_bj < 0 || o.coarse_bj > 1) { set_error("coarse_bj must be 0 or 1"); return SEM_EINVAL; }
    if (o.fused_small < 0 || o.fused_small > 1) { set_error("fused_small must be 0 or 1"); return SEM_EINVAL; }
    if (o.elem_matrices < -1 || o.elem_matrices > SEM_ELEM_DF32) {
        set_error("elem_matrices must be -1, SEM_ELEM_OFF, SEM_ELEM_FP64 or SEM_ELEM_DF32");
        return SEM_EINVAL;
    }
    return SEM_OK;
}

// A timed-out copy inside the tensor-core apply, the network's GEMMs or the double-FP32 apply
// (flag set on the device): turns *ret into SEM_TIMEOUT and clears the flag.  Synchronous;
// reads the flag of MIXED_TF32 handles and of handles with double-FP32 element matrices, or
// of any handle when `always`.
sem_status check_tc_flag(sem_handle* h, sem_status* ret, bool always = false) {
    bool df = false;
    for (const Level& L : h->lv) df = df || L.Adf != nullptr;
    if (!always && !df && h->opts.precision != SEM_PREC_MIXED_TF32) return SEM_OK;
    int terr = 0;
    CKS(cudaMemcpy(&terr, h->sc.flags + F_TC_ERR, sizeof(int), cudaMemcpyDeviceToHost));
    if (terr) {
        CKS(cudaMemset(h->sc.flags + F_TC_ERR, 0, sizeof(int)));
        set_error("a bulk copy of the tensor-core or double-FP32 apply did not complete within its wait bound");
        *ret = SEM_TIMEOUT;
    }
    return SEM_OK;
}

sem_status fail_nan(double v) {
    if (!std::isfinite(v)) { set_error("non-finite residual"); return SEM_NAN; }
    return SEM_OK;
}

// ---------------------------------------------------------------- outer iterations
// Each works on the free-node system in place: f = h->fr, u = phi (zero Dirichlet entries).
sem_status outer_pcg(sem_handle* h, double* u, double tol, sem_stats* st, cudaStream_t s) {
    const long long N = h->lv[0].N;
    Scratch& sc = h->sc;
    CKS(cudaMemcpyAsync(h->r, h->fr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    double rn = st->fnorm;
    st->res0 = rn;
    int i = 0;
    sem_status ret = SEM_OK;
    if (rn > tol) {
        CKST(precondition(h, h->r, h->z, s));
        CKS(cudaMemcpyAsync(h->p, h->z, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        int cur = S_DELTA0, nxt = S_DELTA1;
        K(dot64(N, h->z, h->r, sc, sc.scal + cur, s));
        while (true) {
            if (i >= h->opts.imax) { set_error("the outer iteration reached imax"); ret = SEM_NOT_CONVERGED; break; }
            CKST(apply_level64(h, 0, h->p, h->q, false, s));
            K(dot64(N, h->p, h->q, sc, sc.scal + S_PQ, s));
            K(pcg_update(N, sc.scal + cur, sc.scal + S_PQ, h->p, h->q, u, h->r, sc, sc.scal + S_RR, s));
            ++i;
            CKST(read_scalars(h, 0, 4, s));
            const double pq = sc.hpinned[S_PQ];
            rn = std::sqrt(sc.hpinned[S_RR]);
            CKST(fail_nan(rn));
            if (!(pq > 0.0)) { set_error("PCG breakdown: p^T A p <= 0"); ret = SEM_BREAKDOWN; break; }
            if (rn <= tol) break;
            CKST(precondition(h, h->r, h->z, s));
            K(dot64(N, h->z, h->r, sc, sc.scal + nxt, s));
            K(pcg_direction(N, sc.scal + nxt, sc.scal + cur, h->z, h->p, s));
            std::swap(cur, nxt);
        }
    }
    st->iters = i;
    st->res_final = rn;
    return ret;
}

// The learned sweep's verdict counts travel with the outer iteration's scalar read: once a
// solve has rejected the network three times without accepting it once, the rest of the
// solve runs the plain V-cycle (the sweep would only add its cost).
static void learned_queue_counts(sem_handle* h, cudaStream_t s) {
    if (h->opts.smoother == SEM_SMOOTH_LEARNED && h->learned_active)
        cudaMemcpyAsync(h->sc.hflags + 5, h->sc.flags + F_LEARN_COUNT, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
}
static void learned_review(sem_handle* h) {
    if (h->opts.smoother == SEM_SMOOTH_LEARNED && h->learned_active && h->sc.hflags[5] == 0 && h->sc.hflags[6] >= 3)
        h->learned_active = false;
}

sem_status outer_pdc(sem_handle* h, double* u, double tol, sem_stats* st, cudaStream_t s) {
    const long long N = h->lv[0].N;
    Scratch& sc = h->sc;
    CKS(cudaMemcpyAsync(h->r, h->fr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    double rn = st->fnorm;
    st->res0 = rn;
    int i = 0;
    sem_status ret = SEM_OK;
    while (rn > tol) {
        if (i >= h->opts.imax) { set_error("the outer iteration reached imax"); ret = SEM_NOT_CONVERGED; break; }
        CKST(precondition(h, h->r, h->z, s));
        K(axpy64(N, 1.0, h->z, u, s));
        CKST(apply_level64(h, 0, u, h->q, false, s));
        K(residual64(N, h->fr, h->q, h->r, sc, sc.scal + S_RR, s));
        ++i;
        learned_queue_counts(h, s);
        CKST(read_scalars(h, S_RR, 1, s));
        learned_review(h);
        rn = std::sqrt(sc.hpinned[S_RR]);
        CKST(fail_nan(rn));
    }
    st->iters = i;
    st->res_final = rn;
    return ret;
}

sem_status outer_fgmres(sem_handle* h, double* u, double tol, sem_stats* st, cudaStream_t s) {
    const long long N = h->lv[0].N;
    const int m = h->opts.gmres_m;
    Scratch& sc = h->sc;
    double* hm = sc.scal + S_MULTI;
    CKS(cudaMemcpyAsync(h->r, h->fr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    double beta = st->fnorm;
    st->res0 = beta;
    int it = 0;
    sem_status ret = SEM_OK;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    double* dy = h->gm_y;
    while (beta > tol) {
        if (it >= h->opts.imax) { set_error("the outer iteration reached imax"); ret = SEM_NOT_CONVERGED; break; }
        // v0 = r / beta
        h->sc.hpinned[S_TMP] = beta * beta;
        CKS(cudaMemcpyAsync(sc.scal + S_TMP, h->sc.hpinned + S_TMP, sizeof(double), cudaMemcpyHostToDevice, s));
        K(scale64(N, h->r, sc.scal + S_TMP, h->V, s));
        std::fill(H.begin(), H.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        double resid = beta;
        while (j < m && it < h->opts.imax) {
            double* vj = h->V + (size_t)j * N;
            double* zj = h->Zb + (size_t)j * N;
            double* w = h->V + (size_t)(j + 1) * N;
            CKST(precondition(h, vj, zj, s));
            CKST(apply_level64(h, 0, zj, w, false, s));
            // classical Gram-Schmidt, twice
            K(multidot64(N, j + 1, h->V, w, sc, hm, s));
            K(multiaxpy64(N, j + 1, h->V, hm, -1.0, w, s));
            CKST(read_scalars(h, S_MULTI, j + 1, s));
            std::vector<double> h1(sc.hpinned + S_MULTI, sc.hpinned + S_MULTI + j + 1);
            K(multidot64(N, j + 1, h->V, w, sc, hm, s));
            K(multiaxpy64(N, j + 1, h->V, hm, -1.0, w, s));
            K(dot64(N, w, w, sc, sc.scal + S_TMP, s));
            CKST(read_scalars(h, S_MULTI, j + 1, s));
            CKST(read_scalars(h, S_TMP, 1, s));
            for (int i2 = 0; i2 <= j; ++i2) H[(size_t)i2 * m + j] = h1[i2] + sc.hpinned[S_MULTI + i2];
            const double hn = std::sqrt(sc.hpinned[S_TMP]);
            CKST(fail_nan(hn));
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0) K(scale64(N, w, sc.scal + S_TMP, w, s));
            for (int i2 = 0; i2 < j; ++i2) {
                const double t = cs[i2] * H[(size_t)i2 * m + j] + sn[i2] * H[(size_t)(i2 + 1) * m + j];
                H[(size_t)(i2 + 1) * m + j] = -sn[i2] * H[(size_t)i2 * m + j] + cs[i2] * H[(size_t)(i2 + 1) * m + j];
                H[(size_t)i2 * m + j] = t;
            }
            const double den = std::hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
            cs[j] = H[(size_t)j * m + j] / den;
            sn[j] = H[(size_t)(j + 1) * m + j] / den;
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++j;
            ++it;
            resid = std::fabs(g[j]);
            if (resid <= tol || hn == 0.0) break;
        }
        for (int i2 = j - 1; i2 >= 0; --i2) {
            double v = g[i2];
            for (int k = i2 + 1; k < j; ++k) v -= H[(size_t)i2 * m + k] * y[k];
            y[i2] = v / H[(size_t)i2 * m + i2];
        }
        CKS(cudaMemcpyAsync(dy, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
        K(multiaxpy64(N, j, h->Zb, dy, 1.0, u, s));
        CKST(apply_level64(h, 0, u, h->q, false, s));
        K(residual64(N, h->fr, h->q, h->r, sc, sc.scal + S_RR, s));
        CKST(read_scalars(h, S_RR, 1, s));
        beta = std::sqrt(sc.hpinned[S_RR]);
        CKST(fail_nan(beta));
    }
    st->iters = it;
    st->res_final = beta;
    return ret;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* sem_last_error(void) { return sem::last_error(); }

void sem_default_options(sem_options* o, int P) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->outer = SEM_OUTER_PCG;
    o->precision = SEM_PREC_FP64;
    o->nu1 = 1;
    o->nu2 = 1;
    o->k_cheb = 5;
    o->cheb_lo = 0.01;
    o->cheb_hi = 1.05;
    o->lanczos_steps = 30;
    static const int table[7][3] = {{1, 0, 0}, {1, 0, 0}, {2, 1, 0}, {3, 2, 1}, {4, 2, 1}, {5, 3, 1}, {6, 3, 1}};
    if (P < 1 || P > 6) P = 1;
    int n = 0;
    for (int k = 0; k < 3; ++k)
        if (table[P][k] > 0) o->level_p[n++] = table[P][k];
    o->nlevels = n;
    o->rtol = 1e-8;
    o->atol = 0.0;
    o->imax = 200;
    o->gmres_m = 30;
    o->coarse_rtol = 1e-2;
    o->coarse_imax = 5000;
    o->profile = 0;
    o->inner_imax = 0;
    o->inner_rtol = 1e-4;
    o->debug_barrier_extra = 0;
    o->smoother = SEM_SMOOTH_CHEBYSHEV;
    o->mlp_hidden = 256;
    o->mlp_seed = 20090705ULL;
    o->batch = 0;
    o->autotune = 1;
    o->batch_mode = 0;
    o->learned_tau = 0.5;
    o->surface_ops = 0;
    o->asm_overlap = 1;
    o->deterministic = 0;
    o->elem_matrices = -1;
    o->coarse_bj = 1;
    o->fused_small = 1;
}

sem_status sem_mesh_nodes2d(const sem_mesh* m, int p, long long* n2, double* xy) {
    if (!m || !n2 || p < 1 || p > 6 || !m->tri || !m->vxy || m->ntri < 1) {
        set_error("sem_mesh_nodes2d: bad arguments");
        return SEM_EINVAL;
    }
    for (long long i = 0; i < 3LL * m->ntri; ++i)
        if (m->tri[i] < 0 || m->tri[i] >= m->nvert) { set_error("triangle vertex id out of range"); return SEM_EINVAL; }
    std::vector<int> map2;
    long long N2 = 0;
    tri_numbering(m->nvert, m->ntri, m->tri, p, map2, N2);
    *n2 = N2;
    if (xy) {
        std::vector<double> c;
        if (m->dim == 3 && m->edge_arc) {
            // the blended map at the order-p nodes, first appearance wins
            std::vector<double> nodes;
            blended_nodes(m->ntri, m->tri, m->vxy, m->edge_arc, p, nodes);
            const int NT = (p + 1) * (p + 2) / 2;
            c.assign(2 * N2, 0.0);
            std::vector<char> seen(N2, 0);
            for (size_t i = 0; i < (size_t)m->ntri * NT; ++i) {
                const int g = map2[i];
                if (seen[g]) continue;
                seen[g] = 1;
                c[2 * g] = nodes[2 * i];
                c[2 * g + 1] = nodes[2 * i + 1];
            }
        } else {
            tri_coords(m->ntri, m->tri, m->vxy, p, map2, N2, c);
        }
        std::memcpy(xy, c.data(), sizeof(double) * c.size());
    }
    return SEM_OK;
}

sem_status sem_setup(const sem_mesh* m, int P, const sem_options* opts, sem_handle** out) {
    if (!out) { set_error("out is NULL"); return SEM_EINVAL; }
    *out = nullptr;
    CKST(check_mesh(m, P));
    sem_options o;
    if (opts) o = *opts; else sem_default_options(&o, P);
    CKST(check_options(o, P));
    CKST(check_orders(o, m->dim));
    sem_handle* h = new (std::nothrow) sem_handle();
    if (!h) { set_error("host allocation failed"); return SEM_ENOMEM; }
    h->dim = m->dim;
    h->P = P;
    h->opts = o;
    h->nlayers = (m->dim == 3) ? m->nlayers : 1;
    h->depth = (m->dim == 3) ? m->depth : 0.0;
    cudaGetDevice(&h->device);
    h->vxy.assign(m->vxy, m->vxy + 2 * (size_t)m->nvert);
    h->tri.assign(m->tri, m->tri + 3 * (size_t)m->ntri);
    if (m->dim == 3) {
        const int nl = m->nlayers;
        for (int b = 0; b < m->ntri; ++b)
            for (int l = 0; l < (m->col_layers ? m->col_layers[b] : nl); ++l) {
                h->elem_b.push_back(b);
                h->elem_l.push_back(l);
            }
        h->general = m->col_layers || m->z_iface || m->edge_arc;
        h->zif.resize(2 * (size_t)(nl + 1));
        for (int k = 0; k <= nl; ++k) {
            h->zif[2 * k] = m->z_iface ? m->z_iface[2 * k] : -m->depth * (1.0 - (double)k / nl);
            h->zif[2 * k + 1] = m->z_iface ? m->z_iface[2 * k + 1] : (double)k / nl;
        }
        if (m->edge_arc) h->arc.assign(m->edge_arc, m->edge_arc + 9 * (size_t)m->ntri);
        if (h->general)
            blended_nodes(m->ntri, m->tri, m->vxy, m->edge_arc, P, h->xyP);
    }
    h->lv.resize(o.nlevels);
    h->map2.resize(o.nlevels);
    sem_status st = SEM_OK;
    for (int li = 0; li < o.nlevels && st == SEM_OK; ++li)
        st = build_level(h, m, li, o.level_p[li], level_pz(o, li, m->dim));
    if (st == SEM_OK && o.deterministic && m->dim == 3)
        for (Level& L : h->lv) {
            if (st != SEM_OK) break;
            st = build_dss(L);
        }
    if (st == SEM_OK && o.elem_matrices != 0 && m->dim == 3) st = alloc_element_matrices(h);
    if (st == SEM_OK) st = build_geometry(h, m);       // fills the element matrices too
    if (st == SEM_OK) st = build_diagonals(h);
    if (st == SEM_OK) st = build_transfers(h);
    if (st == SEM_OK) st = build_coarse_gradients(h);
    if (st == SEM_OK) st = build_mlp(h);
    if (st == SEM_OK) st = build_workspace(h);
    if (o.smoother == SEM_SMOOTH_ASM)
        for (int li = 0; li + 1 < o.nlevels && st == SEM_OK; ++li) st = build_asm_level(h, li);
    // lambda_hat sets the Chebyshev interval; the Schwarz smoother has none (reported as 0)
    if (o.smoother != SEM_SMOOTH_ASM)
        for (int li = 0; li + 1 < o.nlevels && st == SEM_OK; ++li) st = estimate_lambda(h, li, false);
    if (st == SEM_OK && o.autotune && m->dim == 3) {
        // u holds the Lanczos iterate on the smoothed levels; zero it on the coarsest (and
        // everywhere when no Lanczos estimate ran)
        for (Level& L : h->lv) {
            if (st != SEM_OK) break;
            const bool zero = &L == &h->lv.back() || o.smoother == SEM_SMOOTH_ASM;
            cudaError_t e = zero ? cudaMemset(L.u, 0, sizeof(double) * L.N) : cudaSuccess;
            if (e == cudaSuccess) e = to_f32(L.N, L.u, L.u32, 0);
            if (e == cudaSuccess) e = tune_prism(L, false);
            if (e == cudaSuccess) e = tune_prism(L, true);
            if (e == cudaSuccess && o.precision == SEM_PREC_MIXED_TF32) e = tune_tc(L);
            if (e != cudaSuccess) { set_error(std::string("autotune: ") + cudaGetErrorString(e)); st = SEM_ECUDA; }
        }
    }
    if (st == SEM_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { set_error(std::string("setup: ") + cudaGetErrorString(e)); st = SEM_ECUDA; }
    }
    if (st == SEM_OK) st = build_small_plan(h);
    if (st != SEM_OK) {
        sem_teardown(h);
        return st;
    }
    h->fine_applies = 0;
    static std::atomic<unsigned long long> next_uid{1};
    h->uid = next_uid.fetch_add(1);
    *out = h;
    return SEM_OK;
}

void sem_teardown(sem_handle* h) {
    if (!h) return;
    // no kernel or copy of this handle may still be in flight when its memory goes away
    if (h->bstream) cudaStreamSynchronize(h->bstream);
    cudaDeviceSynchronize();
    free_small_plan(h);
    for (Level& L : h->lv) free_level(L);
    if (h->auto_elem_bytes) g_auto_elem_bytes.fetch_sub(h->auto_elem_bytes);
    void* ptrs[] = {h->sc.part, h->sc.counter, h->sc.scal, h->sc.flags, h->r, h->z, h->p, h->q, h->x, h->fr,
                    h->V, h->Zb, h->cx, h->cr, h->cz, h->cp, h->cq, h->cb, h->st_eta, h->st_rhs, h->st_phi,
                    h->ir, h->iz, h->ip, h->iq, h->ie, h->gm_y, h->net.W1, h->net.b1, h->net.W2, h->net.b2,
                    h->net.W1b, h->net.W2b, h->grads.dW1, h->grads.db1, h->grads.dW2, h->grads.db2,
                    h->adam.m[0], h->adam.m[1], h->adam.m[2], h->adam.m[3], h->adam.v[0], h->adam.v[1],
                    h->adam.v[2], h->adam.v[3], h->mX, h->mT, h->mA1, h->mH1, h->mY, h->mdY, h->mdH, h->mscale,
                    h->lr32, h->ld32, h->lu32, h->te0, h->tf, h->tu, h->tz, h->bu, h->fs_map2, h->fs_vtri,
                    h->fs_Drn, h->fs_Dsn, h->fs_Dtop, h->fs_invm, h->fs_eta, h->fs_phi, h->fs_w, h->fs_ex,
                    h->fs_ey, h->fs_px, h->fs_py, h->fs_k, h->fs_se, h->fs_sp};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->sc.hpinned) cudaFreeHost(h->sc.hpinned);
    if (h->sc.hflags) cudaFreeHost(h->sc.hflags);
    if (h->fs_hpin) cudaFreeHost(h->fs_hpin);
    for (auto& e : h->ev) cudaEventDestroy(e);
    if (h->bgraph) cudaGraphExecDestroy(h->bgraph);
    if (h->bplan) {
        if (h->bplan->exec) cudaGraphExecDestroy(h->bplan->exec);
        delete h->bplan;
    }
    if (h->bstream) cudaStreamDestroy(h->bstream);
    delete h;
}

static sem_status check_level(const sem_handle* h, int level) {
    if (!h) { set_error("handle is NULL"); return SEM_EINVAL; }
    if (level < 0 || level >= (int)h->lv.size()) { set_error("level out of range"); return SEM_EINVAL; }
    return SEM_OK;
}

sem_status sem_query(const sem_handle* h, int level, long long* ndof, long long* ndir, long long* nelem, int* np) {
    CKST(check_level(h, level));
    const Level& L = h->lv[level];
    if (ndof) *ndof = L.N;
    if (ndir) *ndir = (long long)L.hdir.size();
    if (nelem) *nelem = L.E;
    if (np) *np = L.Np;
    return SEM_OK;
}

sem_status sem_dirichlet_nodes(const sem_handle* h, int level, long long* idx) {
    CKST(check_level(h, level));
    if (!idx) { set_error("idx is NULL"); return SEM_EINVAL; }
    std::memcpy(idx, h->lv[level].hdir.data(), sizeof(long long) * h->lv[level].hdir.size());
    return SEM_OK;
}

sem_status sem_element_map(const sem_handle* h, int level, int* map) {
    CKST(check_level(h, level));
    if (!map) { set_error("map is NULL"); return SEM_EINVAL; }
    const Level& L = h->lv[level];
    for (size_t i = 0; i < L.hmap.size(); ++i) map[i] = L.hmap[i] >= 0 ? L.hmap[i] : -L.hmap[i] - 1;
    return SEM_OK;
}

sem_status sem_lambda_max(const sem_handle* h, double* lam) {
    if (!h || !lam) { set_error("bad arguments"); return SEM_EINVAL; }
    for (size_t i = 0; i < h->lv.size(); ++i) lam[i] = h->lv[i].lam;
    return SEM_OK;
}

sem_status sem_tile_shapes(const sem_handle* h, int level, int* elems_fp64, int* elems_fp32) {
    CKST(check_level(h, level));
    const Level& L = h->lv[level];
    if (elems_fp64) *elems_fp64 = L.dim == 3 ? prism_tile_elements(L.p, L.tile64) : 1;
    if (elems_fp32) *elems_fp32 = L.dim == 3 ? prism_tile_elements(L.p, L.tile32) : 1;
    return SEM_OK;
}

sem_status sem_elem_matrices(const sem_handle* h, int level, int* kind) {
    CKST(check_level(h, level));
    if (!kind) { set_error("kind is NULL"); return SEM_EINVAL; }
    const Level& L = h->lv[level];
    *kind = L.Adf != nullptr ? SEM_ELEM_DF32 : (L.Ae64 != nullptr ? SEM_ELEM_FP64 : SEM_ELEM_OFF);
    return SEM_OK;
}

sem_status sem_tc_kernel(const sem_handle* h, int level, int* kind) {
    CKST(check_level(h, level));
    if (!kind) { set_error("kind is NULL"); return SEM_EINVAL; }
    const Level& L = h->lv[level];
    *kind = (h->opts.precision != SEM_PREC_MIXED_TF32 || !level_tc(L)) ? 0 : (L.tc_kind == 1 && L.G16T ? 2 : 1);
    return SEM_OK;
}

sem_status sem_diagonal(const sem_handle* h, int level, double* diag) {
    CKST(check_level(h, level));
    if (!diag) { set_error("diag is NULL"); return SEM_EINVAL; }
    std::memcpy(diag, h->lv[level].hdiag.data(), sizeof(double) * h->lv[level].hdiag.size());
    return SEM_OK;
}

sem_status sem_node_coords(const sem_handle* h, int level, double* xyz) {
    CKST(check_level(h, level));
    if (!xyz) { set_error("xyz is NULL"); return SEM_EINVAL; }
    const Level& L = h->lv[level];
    std::vector<double> xy;
    if (h->general)
        tri_coords_mapped((int)(h->tri.size() / 3), h->P, h->xyP, L.p, h->map2[level], L.N2, xy);
    else
        tri_coords((int)(h->tri.size() / 3), h->tri.data(), h->vxy.data(), L.p, h->map2[level], L.N2, xy);
    if (h->dim == 2) {
        std::memcpy(xyz, xy.data(), sizeof(double) * xy.size());
        return SEM_OK;
    }
    // eta_P at this level's 2D nodes: the order-P surface interpolated per base triangle
    const Level& L0 = h->lv[0];
    std::vector<double> eta(L.N2, 0.0);
    std::vector<double> B, Dr, Ds;
    tri_lagrange(h->P, L.ref.tnodes.data(), L.NT, B, Dr, Ds);
    const int ntri = (int)(h->tri.size() / 3);
    for (int b = 0; b < ntri; ++b)
        for (int n = 0; n < L.NT; ++n) {
            double v = 0;
            for (int k = 0; k < L0.NT; ++k) v += B[(size_t)n * L0.NT + k] * h->eta2[h->map2[0][(size_t)b * L0.NT + k]];
            eta[h->map2[level][(size_t)b * L.NT + n]] = v;
        }
    const int nl = h->nlayers, p = L.pz;             // vertical order
    for (int kz = 0; kz <= nl * p; ++kz) {
        int l = kz / p, k = kz - l * p;
        if (l == nl) { l = nl - 1; k = p; }
        const double sigma = (l + 0.5 * (L.ref.znodes[k] + 1.0)) / nl;
        const double tau = 0.5 * (L.ref.znodes[k] + 1.0);
        const double* zi = h->zif.data() + 2 * l;   // interfaces l and l + 1
        for (long long g = 0; g < L.N2; ++g) {
            const long long id = (long long)kz * L.N2 + g;
            xyz[3 * id] = xy[2 * g];
            xyz[3 * id + 1] = xy[2 * g + 1];
            xyz[3 * id + 2] = h->general ? (1.0 - tau) * (zi[0] + zi[1] * eta[g]) + tau * (zi[2] + zi[3] * eta[g])
                                         : -h->depth + sigma * (h->depth + eta[g]);
        }
    }
    return SEM_OK;
}

sem_status sem_apply(sem_handle* h, int level, const double* x, double* y, void* stream) {
    CKST(check_level(h, level));
    if (!x || !y || x == y) { set_error("sem_apply: x and y must be distinct device buffers"); return SEM_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const Level& L = h->lv[level];
    CKST(apply_level64(h, level, x, y, false, s));
    K(copy_dirichlet((long long)L.hdir.size(), L.dir, x, y, s));
    return SEM_OK;
}

sem_status sem_apply32(sem_handle* h, int level, const float* x, float* y, int tensor_cores, void* stream) {
    CKST(check_level(h, level));
    if (!x || !y || x == y) { set_error("sem_apply32: x and y must be distinct device buffers"); return SEM_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const Level& L = h->lv[level];
    if (tensor_cores < 0 || tensor_cores > 2) { set_error("sem_apply32: tensor_cores 0, 1 or 2"); return SEM_EINVAL; }
    if (tensor_cores) {
        if (!level_tc(L)) {
            set_error("sem_apply32: the tensor-core apply needs an isotropic prism level of order 2..6");
            return SEM_EINVAL;
        }
        if (tensor_cores == 2 && !prism_t5_supported(L.p)) {
            set_error("sem_apply32: the tcgen05 apply is compiled for order 6 only");
            return SEM_EINVAL;
        }
        CKS(cudaMemsetAsync(y, 0, sizeof(float) * L.N, s));
        K(launch_apply_tensor(L, x, y, nullptr, h->sc.flags + F_TC_ERR, s, tensor_cores == 2));
        CKS(cudaStreamSynchronize(s));
        sem_status ret = SEM_OK;
        CKST(check_tc_flag(h, &ret, true));
        if (ret != SEM_OK) return ret;
    } else {
        CKST(apply_level32(h, level, x, y, s));
    }
    K(copy_dirichlet32((long long)L.hdir.size(), L.dir, x, y, s));
    return SEM_OK;
}

static sem_status check_asm(const sem_handle* h, int level) {
    CKST(check_level(h, level));
    if (h->lv[level].asm_blk == nullptr) {
        set_error("no Schwarz blocks on this level (smoother = ASM, every level but the coarsest)");
        return SEM_EINVAL;
    }
    return SEM_OK;
}

sem_status sem_asm_subdomains(const sem_handle* h, int level, long long* ptr, int* nodes) {
    CKST(check_asm(h, level));
    const Level& L = h->lv[level];
    if (ptr)
        for (size_t i = 0; i < L.hasm_ptr.size(); ++i) ptr[i] = L.hasm_ptr[i];
    if (nodes) std::memcpy(nodes, L.hasm_nodes.data(), sizeof(int) * L.hasm_nodes.size());
    return SEM_OK;
}

sem_status sem_asm_apply(sem_handle* h, int level, const double* r, double* z, int adjoint, void* stream) {
    CKST(check_asm(h, level));
    if (h->opts.precision != SEM_PREC_FP64) { set_error("sem_asm_apply: FP64 handles (sem_asm_apply32 otherwise)"); return SEM_EINVAL; }
    if (!r || !z || r == z) { set_error("sem_asm_apply: distinct r and z"); return SEM_EINVAL; }
    const Level& L = h->lv[level];
    cudaStream_t s = as_stream(stream);
    CKS(cudaMemsetAsync(z, 0, sizeof(double) * L.N, s));
    K(asm_apply64(L, r, nullptr, adjoint ? 1 : 0, z, s));
    return SEM_OK;
}

sem_status sem_asm_apply32(sem_handle* h, int level, const float* r, float* z, int adjoint, void* stream) {
    CKST(check_asm(h, level));
    if (h->opts.precision == SEM_PREC_FP64) { set_error("sem_asm_apply32: mixed-precision handles (sem_asm_apply otherwise)"); return SEM_EINVAL; }
    if (!r || !z || r == z) { set_error("sem_asm_apply32: distinct r and z"); return SEM_EINVAL; }
    const Level& L = h->lv[level];
    cudaStream_t s = as_stream(stream);
    CKS(cudaMemsetAsync(z, 0, sizeof(float) * L.N, s));
    K(asm_apply32(L, r, nullptr, adjoint ? 1 : 0, z, s));
    return SEM_OK;
}

sem_status sem_update_eta(sem_handle* h, const double* eta_nodal_host, int strategy) {
    if (!h || !eta_nodal_host) { set_error("sem_update_eta: bad arguments"); return SEM_EINVAL; }
    if (h->dim != 3) { set_error("sem_update_eta: the surface elevation moves only in 3D handles"); return SEM_EINVAL; }
    if (strategy < SEM_ETA_FINEST || strategy > SEM_ETA_ALL) { set_error("sem_update_eta: strategy 0, 1 or 2"); return SEM_EINVAL; }
    CKS(cudaDeviceSynchronize());
    const Level& L0 = h->lv[0];
    CKST(check_layers(h, std::vector<double>(eta_nodal_host, eta_nodal_host + L0.N2)));
    h->eta2.assign(eta_nodal_host, eta_nodal_host + L0.N2);
    if (h->fs_eta) CKS(cudaMemcpy(h->fs_eta, h->eta2.data(), sizeof(double) * L0.N2, cudaMemcpyHostToDevice));
    const int nl = (int)h->lv.size();
    // element matrices taken by the auto rule serve a fixed geometry: recomputing them costs
    // seconds at the benchmark size (Np^2 entries, each a quadrature sum), far more than the
    // sum-factorised applies lose, so a moving surface returns the handle to sum factorisation
    if (h->auto_elem_bytes) {
        for (Level& L : h->lv) {
            if (L.Ae64) cudaFree(L.Ae64);
            if (L.Adf) cudaFree(L.Adf);
            L.Ae64 = nullptr;
            L.Adf = nullptr;
        }
        g_auto_elem_bytes.fetch_sub(h->auto_elem_bytes);
        h->auto_elem_bytes = 0;
    }
    // a mixed-precision handle smooths with the single-precision operator: its lambda_hat is
    // re-estimated with that operator (the estimate at setup uses the FP64 one)
    const bool fp32 = h->opts.precision != SEM_PREC_FP64;
    const bool asm_on = h->opts.smoother == SEM_SMOOTH_ASM;
    auto lambda = [&](int li) { return asm_on ? SEM_OK : estimate_lambda(h, li, fp32); };
    if (strategy == SEM_ETA_FINEST) {
        // the finest operator; the diagonal and the coarse operators of t = 0.  The Chebyshev
        // interval must still cover the spectrum of D_0^{-1} A(eta), or the sweep amplifies its
        // top: lambda_hat of the finest level is re-estimated against the new operator.
        CKST(geometry_levels(h, 0, 1, false));
        if (nl > 1) CKST(lambda(0));
        // the Schwarz blocks of t = 0 stay (they are the smoother the strategy keeps)
    } else if (strategy == SEM_ETA_LINEAR_COARSE) {
        // the finest operator and its smoother follow eta; the coarse levels use the linear
        // (flat-surface) operators, built once and then fixed
        CKST(geometry_levels(h, 0, 1, false));
        CKST(diagonal_level(h, 0));
        if (nl > 1) CKST(lambda(0));
        if (asm_on && nl > 1) CKST(refresh_asm_level(h, 0));
        if (!h->coarse_flat && nl > 1) {
            CKST(geometry_levels(h, 1, nl, true));
            for (int li = 1; li < nl; ++li) CKST(diagonal_level(h, li));
            CKST(reassemble_coarse(h));
            for (int li = 1; li + 1 < nl; ++li) CKST(lambda(li));
            if (asm_on)
                for (int li = 1; li + 1 < nl; ++li) CKST(refresh_asm_level(h, li));
            h->coarse_flat = true;
        }
    } else {
        // every operator of every level from the new eta
        CKST(geometry_levels(h, 0, nl, false));
        for (int li = 0; li < nl; ++li) CKST(diagonal_level(h, li));
        CKST(reassemble_coarse(h));
        for (int li = 0; li + 1 < nl; ++li) CKST(lambda(li));
        if (asm_on)
            for (int li = 0; li + 1 < nl; ++li) CKST(refresh_asm_level(h, li));
        h->coarse_flat = false;
    }
    CKS(cudaDeviceSynchronize());
    if (h->small != nullptr) CKST(build_small_plan(h));     // element matrices, lambda_hat, coarse inverse
    return SEM_OK;
}

// Right-hand sides of Eqs. FSeta / FSphi at the order-P surface nodes for the fields
// (eta, phis); the nonlinear form first moves the geometry to eta with `strategy`.  The
// solve's iterations and time are added to *acc.
static sem_status fnpf_rhs_impl(sem_handle* h, const double* eta, const double* phis, double g, int linear,
                                int strategy, double tol, double* deta, double* dphi, sem_stats* acc, cudaStream_t s) {
    const Level& L0 = h->lv[0];
    const long long N2 = L0.N2;
    const int ntri = (int)(h->tri.size() / 3);
    if (!linear) {
        CKS(cudaMemcpyAsync(h->fs_hpin, eta, sizeof(double) * N2, cudaMemcpyDeviceToHost, s));
        CKS(cudaStreamSynchronize(s));
        CKST(sem_update_eta(h, h->fs_hpin, strategy));
    }
    sem_stats st{};
    const sem_status rs = laplace_solve(h, nullptr, phis, tol, h->fs_phi, &st, s);
    if (acc) {
        acc->iters += st.iters;
        acc->ms += st.ms;
        acc->fine_applies += st.fine_applies;
        acc->res_final = st.res_final;
        acc->fnorm = st.fnorm;
    }
    if (rs != SEM_OK) return rs;
    K(surface_w(N2, L0.NZ, (long long)(h->nlayers - 1) * L0.pz, h->fs_Dtop, h->depth, h->nlayers, h->fs_phi,
                h->fs_eta, h->fs_w, s));
    if (!linear) {
        K(surface_gradient(ntri, L0.NT, N2, h->fs_map2, h->fs_vtri, h->fs_Drn, h->fs_Dsn, h->fs_invm, eta, h->fs_ex,
                           h->fs_ey, s));
        K(surface_gradient(ntri, L0.NT, N2, h->fs_map2, h->fs_vtri, h->fs_Drn, h->fs_Dsn, h->fs_invm, phis, h->fs_px,
                           h->fs_py, s));
    }
    K(fnpf_rhs(N2, linear, g, eta, h->fs_w, h->fs_ex, h->fs_ey, h->fs_px, h->fs_py, deta, dphi, s));
    return SEM_OK;
}

static sem_status fnpf_check(const sem_handle* h, const void* eta, const void* phis, int strategy, const char* who) {
    if (!h || !eta || !phis) { set_error(std::string(who) + ": bad arguments"); return SEM_EINVAL; }
    if (!h->fs_k) { set_error(std::string(who) + ": the handle was set up without surface_ops"); return SEM_EINVAL; }
    if (strategy < SEM_ETA_FINEST || strategy > SEM_ETA_ALL) {
        set_error(std::string(who) + ": strategy 0, 1 or 2");
        return SEM_EINVAL;
    }
    return SEM_OK;
}

sem_status sem_fnpf_rhs(sem_handle* h, const double* eta, const double* phis, double g, int linear, int strategy,
                        double tol, double* deta, double* dphis, void* stream) {
    CKST(fnpf_check(h, eta, phis, strategy, "sem_fnpf_rhs"));
    if (!deta || !dphis) { set_error("sem_fnpf_rhs: bad arguments"); return SEM_EINVAL; }
    cudaStream_t s = as_stream(stream);
    CKST(fnpf_rhs_impl(h, eta, phis, g, linear, strategy, tol, deta, dphis, nullptr, s));
    CKS(cudaStreamSynchronize(s));
    return SEM_OK;
}

sem_status sem_fnpf_step(sem_handle* h, double* eta, double* phis, double dt, double g, int linear, int strategy,
                         double tol, sem_stats* stats, void* stream) {
    CKST(fnpf_check(h, eta, phis, strategy, "sem_fnpf_step"));
    if (!std::isfinite(dt)) { set_error("sem_fnpf_step: dt must be finite"); return SEM_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const long long N2 = h->lv[0].N2;
    double* ke = h->fs_k;            // slopes of eta, [4][N2]
    double* kp = h->fs_k + 4 * N2;   // slopes of phi~
    sem_stats acc{};
    const double c[4] = {0.0, 0.5 * dt, 0.5 * dt, dt};
    for (int j = 0; j < 4; ++j) {
        const double* ej = eta;
        const double* pj = phis;
        if (j > 0) {
            K(rk_stage(N2, c[j], eta, ke + (j - 1) * N2, phis, kp + (j - 1) * N2, h->fs_se, h->fs_sp, s));
            ej = h->fs_se;
            pj = h->fs_sp;
        }
        const sem_status r = fnpf_rhs_impl(h, ej, pj, g, linear, strategy, tol, ke + j * N2, kp + j * N2, &acc, s);
        if (r != SEM_OK) {
            acc.status = r;
            if (stats) *stats = acc;
            return r;
        }
    }
    K(rk4_combine(N2, dt, ke, eta, s));
    K(rk4_combine(N2, dt, kp, phis, s));
    CKS(cudaStreamSynchronize(s));
    acc.status = SEM_OK;
    if (stats) *stats = acc;
    return SEM_OK;
}

sem_status pmg_vcycle(sem_handle* h, const double* r, double* z, void* stream) {
    if (!h || !r || !z || r == z) { set_error("pmg_vcycle: bad arguments"); return SEM_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const Level& L = h->lv[0];
    CKS(cudaMemcpyAsync(h->r, r, sizeof(double) * L.N, cudaMemcpyDeviceToDevice, s));
    K(zero_dirichlet((long long)L.hdir.size(), L.dir, h->r, s));
    return precondition(h, h->r, z, s);
}

sem_status laplace_solve(sem_handle* h, const double* rhs, const double* eta, double tol, double* phi,
                         sem_stats* stats, void* stream) {
    if (!h || !eta || !phi) { set_error("laplace_solve: bad arguments"); return SEM_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const Level& L = h->lv[0];
    const long long N = L.N, nd = (long long)L.hdir.size();
    if (h->small != nullptr && !h->capturing) {
        // small problems: the whole solve in one launch
        sem_stats sst{};
        const sem_status r = small_solve(h, rhs, eta, (tol > 0) ? tol : h->opts.rtol, phi, &sst, s);
        if (stats) *stats = sst;
        return r;
    }
    sem_stats st{};
    h->fine_applies = 0;
    h->vcycles = 0;
    h->coarse_iters_max = 0;
    h->apply_ms = h->apply32_ms = h->apply_tc_ms = h->asm_ms = h->lift_ms = 0;
    h->apply_launches = h->apply32_launches = h->apply_tc_launches = h->asm_launches = h->lift_launches = 0;
    h->launches = 0;
    h->inner_iters = 0;
    CKS(cudaMemsetAsync(h->sc.flags + F_LEARN_COUNT, 0, 2 * sizeof(int), s));
    h->sc.hflags[5] = h->sc.hflags[6] = 0;
    h->learned_active = true;
    h->ev_used = 0;
    cudaEvent_t e0, e1;
    CKS(cudaEventCreate(&e0));
    CKS(cudaEventCreate(&e1));
    CKS(cudaEventRecord(e0, s));
    // lifting: f = rhs_F - A_FD phi~
    CKS(cudaMemsetAsync(h->x, 0, sizeof(double) * N, s));
    K(scatter_dirichlet(nd, L.dir, eta, h->x, s));
    CKST(apply_level64(h, 0, h->x, h->q, true, s));
    h->fine_applies -= 1;   // lifting is not an iteration apply
    if (rhs) {
        CKS(cudaMemcpyAsync(h->fr, rhs, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        K(axpy64(N, -1.0, h->q, h->fr, s));
        K(zero_dirichlet(nd, L.dir, h->fr, s));
    } else {
        CKS(cudaMemsetAsync(h->fr, 0, sizeof(double) * N, s));
        K(axpy64(N, -1.0, h->q, h->fr, s));
    }
    K(dot64(N, h->fr, h->fr, h->sc, h->sc.scal + S_FF, s));
    CKST(read_scalars(h, S_FF, 1, s));
    st.fnorm = std::sqrt(h->sc.hpinned[S_FF]);
    CKST(fail_nan(st.fnorm));
    const double rtol = (tol > 0) ? tol : h->opts.rtol;
    const double thr = rtol * st.fnorm + h->opts.atol;
    CKS(cudaMemsetAsync(phi, 0, sizeof(double) * N, s));
    sem_status ret;
    switch (h->opts.outer) {
        case SEM_OUTER_PDC: ret = outer_pdc(h, phi, thr, &st, s); break;
        case SEM_OUTER_FGMRES: ret = outer_fgmres(h, phi, thr, &st, s); break;
        default: ret = outer_pcg(h, phi, thr, &st, s); break;
    }
    K(scatter_dirichlet(nd, L.dir, eta, phi, s));
    CKS(cudaEventRecord(e1, s));
    CKS(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (h->opts.profile) flush_events(h);
    st.ms = ms;
    CKST(check_tc_flag(h, &ret));
    st.status = ret;
    st.fine_applies = h->fine_applies;
    st.vcycles = h->vcycles;
    st.coarse_iters_max = h->coarse_iters_max;
    st.apply_ms = h->apply_ms;
    st.apply_launches = h->apply_launches;
    st.apply32_ms = h->apply32_ms;
    st.apply32_launches = h->apply32_launches;
    st.apply_tc_ms = h->apply_tc_ms;
    st.apply_tc_launches = h->apply_tc_launches;
    st.asm_ms = h->asm_ms;
    st.asm_launches = h->asm_launches;
    st.lift_ms = h->lift_ms;
    st.lift_launches = h->lift_launches;
    st.kernel_launches = h->launches;
    st.inner_iters = h->inner_iters;
    if (h->opts.smoother == SEM_SMOOTH_LEARNED) {
        int cnt[2] = {0, 0};
        CKS(cudaMemcpy(cnt, h->sc.flags + F_LEARN_COUNT, 2 * sizeof(int), cudaMemcpyDeviceToHost));
        st.learned_accepts = cnt[0];
        st.learned_fallbacks = cnt[1];
    }
    st.q_mean = (st.iters > 0 && st.res0 > 0) ? std::pow(st.res_final / st.res0, 1.0 / st.iters) : 0.0;
    if (stats) *stats = st;
    return ret;
}

sem_status laplace_solve_host(sem_handle* h, const double* rhs_host, const double* eta_host, double tol,
                              double* phi_host, sem_stats* stats, void* stream) {
    if (!h || !eta_host || !phi_host) { set_error("laplace_solve_host: bad arguments"); return SEM_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const Level& L = h->lv[0];
    const long long N = L.N, nd = (long long)L.hdir.size();
    CKS(cudaMemcpyAsync(h->st_eta, eta_host, sizeof(double) * nd, cudaMemcpyHostToDevice, s));
    if (rhs_host) CKS(cudaMemcpyAsync(h->st_rhs, rhs_host, sizeof(double) * N, cudaMemcpyHostToDevice, s));
    const sem_status ret = laplace_solve(h, rhs_host ? h->st_rhs : nullptr, h->st_eta, tol, h->st_phi, stats, stream);
    CKS(cudaMemcpyAsync(phi_host, h->st_phi, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    CKS(cudaStreamSynchronize(s));
    return ret;
}

static sem_status check_mlp(const sem_handle* h) {
    if (!h) { set_error("handle is NULL"); return SEM_EINVAL; }
    if (h->opts.smoother != SEM_SMOOTH_LEARNED || !h->net.W1) {
        set_error("the handle has no correction network (smoother != SEM_SMOOTH_LEARNED)");
        return SEM_EINVAL;
    }
    return SEM_OK;
}

sem_status sem_mlp_get_weights(const sem_handle* h, float* W1, float* b1, float* W2, float* b2) {
    CKST(check_mlp(h));
    const MlpNet& n = h->net;
    if (W1) CKS(cudaMemcpy(W1, n.W1, sizeof(float) * n.H * n.nin, cudaMemcpyDeviceToHost));
    if (b1) CKS(cudaMemcpy(b1, n.b1, sizeof(float) * n.H, cudaMemcpyDeviceToHost));
    if (W2) CKS(cudaMemcpy(W2, n.W2, sizeof(float) * n.nout * n.H, cudaMemcpyDeviceToHost));
    if (b2) CKS(cudaMemcpy(b2, n.b2, sizeof(float) * n.nout, cudaMemcpyDeviceToHost));
    return SEM_OK;
}

sem_status sem_mlp_set_weights(sem_handle* h, const float* W1, const float* b1, const float* W2, const float* b2) {
    CKST(check_mlp(h));
    MlpNet& n = h->net;
    if (!W1 || !b1 || !W2 || !b2) { set_error("sem_mlp_set_weights: NULL array"); return SEM_EINVAL; }
    CKS(cudaMemcpy(n.W1, W1, sizeof(float) * n.H * n.nin, cudaMemcpyHostToDevice));
    CKS(cudaMemcpy(n.b1, b1, sizeof(float) * n.H, cudaMemcpyHostToDevice));
    CKS(cudaMemcpy(n.W2, W2, sizeof(float) * n.nout * n.H, cudaMemcpyHostToDevice));
    CKS(cudaMemcpy(n.b2, b2, sizeof(float) * n.nout, cudaMemcpyHostToDevice));
    CKS(mlp_sync_bf16(n, 0));
    CKS(cudaDeviceSynchronize());
    h->mlp_trained = true;        // weights supplied by the caller (e.g. a checkpoint)
    return SEM_OK;
}

sem_status sem_mlp_forward(sem_handle* h, int B, const float* X, float* Y, void* stream) {
    CKST(check_mlp(h));
    if (B < 1 || B > h->lv[0].E || !X || !Y) { set_error("sem_mlp_forward: need 1 <= B <= elements"); return SEM_EINVAL; }
    CKS(mlp_forward(h->net, B, X, h->mA1, h->mH1, Y, as_stream(stream)));
    return SEM_OK;
}

sem_status sem_mlp_adam(sem_handle* h, const float* dW1, const float* db1, const float* dW2, const float* db2,
                        double lr, int reset, void* stream) {
    CKST(check_mlp(h));
    if (!dW1 || !db1 || !dW2 || !db2 || !(lr > 0.0)) { set_error("sem_mlp_adam: NULL gradient or lr <= 0"); return SEM_EINVAL; }
    cudaStream_t s = as_stream(stream);
    MlpNet& n = h->net;
    const long long cnt[4] = {(long long)n.H * n.nin, n.H, (long long)n.nout * n.H, n.nout};
    if (reset) {
        for (int k = 0; k < 4; ++k) {
            CKS(cudaMemsetAsync(h->adam.m[k], 0, sizeof(float) * cnt[k], s));
            CKS(cudaMemsetAsync(h->adam.v[k], 0, sizeof(float) * cnt[k], s));
        }
        h->adam.t = 0;
    }
    CKS(cudaMemcpyAsync(h->grads.dW1, dW1, sizeof(float) * cnt[0], cudaMemcpyHostToDevice, s));
    CKS(cudaMemcpyAsync(h->grads.db1, db1, sizeof(float) * cnt[1], cudaMemcpyHostToDevice, s));
    CKS(cudaMemcpyAsync(h->grads.dW2, dW2, sizeof(float) * cnt[2], cudaMemcpyHostToDevice, s));
    CKS(cudaMemcpyAsync(h->grads.db2, db2, sizeof(float) * cnt[3], cudaMemcpyHostToDevice, s));
    CKS(mlp_adam(n, h->grads, h->adam, (float)lr, s));
    CKS(cudaStreamSynchronize(s));
    h->mlp_trained = true;
    return SEM_OK;
}

sem_status sem_learned_sweep(sem_handle* h, const float* f, float* u, int* accepted, double* alpha, void* stream) {
    CKST(check_mlp(h));
    if (!f || !u) { set_error("sem_learned_sweep: NULL vector"); return SEM_EINVAL; }
    cudaStream_t s = as_stream(stream);
    CKS(cudaMemsetAsync(h->sc.flags + F_LEARN_ACCEPT, 0, sizeof(int), s));
    CKST(learned_sweep(h, f, u, s));
    int acc = 0;
    double a = 0.0;
    CKS(cudaMemcpyAsync(&acc, h->sc.flags + F_LEARN_ACCEPT, sizeof(int), cudaMemcpyDeviceToHost, s));
    CKS(cudaMemcpyAsync(&a, h->sc.scal + S_ALPHA, sizeof(double), cudaMemcpyDeviceToHost, s));
    CKS(cudaStreamSynchronize(s));
    if (accepted) *accepted = acc;
    if (alpha) *alpha = a;
    return SEM_OK;
}

sem_status sem_mlp_gradient(sem_handle* h, int B, const float* X, const float* T, double* loss, float* dW1,
                            float* db1, float* dW2, float* db2, void* stream) {
    CKST(check_mlp(h));
    if (B < 1 || B > h->lv[0].E || !X || !T) { set_error("sem_mlp_gradient: need 1 <= B <= elements"); return SEM_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const MlpNet& n = h->net;
    CKS(mlp_forward(n, B, X, h->mA1, h->mH1, h->mY, s));
    CKS(mlp_backward(n, B, X, T, h->mA1, h->mH1, h->mY, h->mdY, h->mdH, h->grads, h->sc.scal + S_LOSS, s));
    CKS(cudaStreamSynchronize(s));
    if (loss) CKS(cudaMemcpy(loss, h->sc.scal + S_LOSS, sizeof(double), cudaMemcpyDeviceToHost));
    if (dW1) CKS(cudaMemcpy(dW1, h->grads.dW1, sizeof(float) * n.H * n.nin, cudaMemcpyDeviceToHost));
    if (db1) CKS(cudaMemcpy(db1, h->grads.db1, sizeof(float) * n.H, cudaMemcpyDeviceToHost));
    if (dW2) CKS(cudaMemcpy(dW2, h->grads.dW2, sizeof(float) * n.nout * n.H, cudaMemcpyDeviceToHost));
    if (db2) CKS(cudaMemcpy(db2, h->grads.db2, sizeof(float) * n.nout, cudaMemcpyDeviceToHost));
    return SEM_OK;
}

// One training pair at the point where the replaced sweep acts: the error e
// (FP32; read before lr32 / tz / lu32 / ld32 are written) after the coarse-grid correction of the plain
// V-cycle, e_post = e - P A_c^{-1} R A e, and its residual r_post = A e_post; the
// network sees z = D^{-1} r_post per element (scaled to unit norm) and must
// return e_post in the same scale.  Fills mX / mT / mscale.
static sem_status make_pair(sem_handle* h, const float* e, cudaStream_t s) {
    Level& L = h->lv[0];
    const long long N = L.N;
    CKST(apply_level32(h, 0, e, h->lr32, s));                  // r = A e
    h->cgc_only = true;
    const sem_status st = vcycle32(h, h->lr32, h->tz, s);      // coarse-grid correction of e
    h->cgc_only = false;
    CKST(st);
    K(axpby32(N, e, h->tz, -1.f, h->lu32, s));                 // e_post
    CKST(apply_level32(h, 0, h->lu32, h->lr32, s));            // r_post
    K(mul32(N, L.dinv32, h->lr32, h->ld32, s));                // z = D^{-1} r_post
    K(gather_scaled<float>(L.E, L.Np, L.map, h->ld32, h->lu32, h->mX, h->mT, h->mscale, s));
    return SEM_OK;
}

static sem_status pair_loss(sem_handle* h, double* loss, cudaStream_t s) {
    Level& L = h->lv[0];
    CKS(mlp_forward(h->net, L.E, h->mX, h->mA1, h->mH1, h->mY, s));
    CKS(mlp_backward(h->net, L.E, h->mX, h->mT, h->mA1, h->mH1, h->mY, h->mdY, h->mdH, h->grads,
                     h->sc.scal + S_LOSS, s));
    CKST(read_scalars(h, S_LOSS, 1, s));
    *loss = h->sc.hpinned[S_LOSS];
    return SEM_OK;
}

sem_status sem_learned_train(sem_handle* h, int snapshots, int steps, double lr, unsigned long long seed,
                             double* loss_first, double* loss_last, void* stream) {
    CKST(check_mlp(h));
    if (snapshots < 1 || steps < 1 || !(lr > 0)) { set_error("sem_learned_train: bad arguments"); return SEM_EINVAL; }
    cudaStream_t s = as_stream(stream);
    Level& L = h->lv[0];
    const long long N = L.N;
    h->learned_active = false;          // the plain V-cycle generates the data
    // fixed validation pair (a held-out error of the plain iteration, after 3 V-cycles):
    // the loss on it before and after training
    const unsigned long long vseed = seed * 0x9E3779B97F4A7C15ULL + 0x5851F42D4C957F2DULL;
    double l0 = 0, l1 = 0;
    auto validation_pair = [&]() -> sem_status {
        K(random_free(N, vseed, L.dinv32, h->te0, s));
        CKST(apply_level32(h, 0, h->te0, h->tf, s));
        CKS(cudaMemsetAsync(h->tu, 0, sizeof(float) * N, s));
        for (int k = 0; k < 3; ++k) {
            CKST(apply_level32(h, 0, h->tu, L.y32, s));
            K(axpby32(N, h->tf, L.y32, -1.f, h->lr32, s));
            CKST(vcycle32(h, h->lr32, h->tz, s));
            K(axpby32(N, h->tu, h->tz, 1.f, h->tu, s));
        }
        K(axpby32(N, h->te0, h->tu, -1.f, h->ld32, s));
        return make_pair(h, h->ld32, s);
    };
    sem_status ret = validation_pair();
    if (ret == SEM_OK) ret = pair_loss(h, &l0, s);
    for (int sn = 0; sn < snapshots && ret == SEM_OK; ++sn) {
        const unsigned long long sseed = seed * 0x9E3779B97F4A7C15ULL + (unsigned long long)(sn + 1) * 0xD1B54A32D192ED03ULL;
        K(random_free(N, sseed, L.dinv32, h->te0, s));           // e0; the plain iteration solves A u = A e0
        ret = apply_level32(h, 0, h->te0, h->tf, s);
        if (ret != SEM_OK) break;
        CKS(cudaMemsetAsync(h->tu, 0, sizeof(float) * N, s));
        for (int k = 0; k < steps && ret == SEM_OK; ++k) {
            K(axpby32(N, h->te0, h->tu, -1.f, h->ld32, s));      // the plain solver's error e = e0 - u
            ret = make_pair(h, h->ld32, s);
            if (ret != SEM_OK) break;
            CKS(mlp_forward(h->net, L.E, h->mX, h->mA1, h->mH1, h->mY, s));
            CKS(mlp_backward(h->net, L.E, h->mX, h->mT, h->mA1, h->mH1, h->mY, h->mdY, h->mdH, h->grads,
                             h->sc.scal + S_LOSS, s));
            CKS(mlp_adam(h->net, h->grads, h->adam, (float)lr, s));
            h->launches += 2;
            // advance the plain iteration: u <- u + M (f - A u)
            CKST(apply_level32(h, 0, h->tu, L.y32, s));
            K(axpby32(N, h->tf, L.y32, -1.f, h->lr32, s));
            ret = vcycle32(h, h->lr32, h->tz, s);
            if (ret != SEM_OK) break;
            K(axpby32(N, h->tu, h->tz, 1.f, h->tu, s));
        }
    }
    if (ret == SEM_OK) ret = validation_pair();
    if (ret == SEM_OK) ret = pair_loss(h, &l1, s);
    if (ret == SEM_OK) h->mlp_trained = true;
    h->learned_active = true;
    if (loss_first) *loss_first = l0;
    if (loss_last) *loss_last = l1;
    return ret;
}

// One defect-correction iteration of a batched tank (no host synchronisation,
// capturable): z = M^{-1} r; u += z; r = f - A u; ||r||^2 -> scal[S_RR] (and its pinned
// host mirror when host_copy).
static sem_status batch_iteration(sem_handle* h, cudaStream_t s, bool host_copy = true) {
    const long long N = h->lv[0].N;
    CKST(precondition(h, h->r, h->z, s));
    K(axpy64(N, 1.0, h->z, h->bu, s));
    CKST(apply_level64(h, 0, h->bu, h->q, false, s));
    K(residual64(N, h->fr, h->q, h->r, h->sc, h->sc.scal + S_RR, s));
    if (host_copy)
        CKS(cudaMemcpyAsync(h->sc.hpinned + S_RR, h->sc.scal + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
    return SEM_OK;
}

// Capture batch_iteration into the handle's graph (once); on any capture failure the
// tank keeps running its iterations as direct launches.
static void batch_capture(sem_handle* h) {
    if (h->bgraph || h->bgraph_failed) return;
    cudaStream_t s = h->bstream;
    const long long l0 = h->launches, a0 = h->fine_applies, v0 = h->vcycles;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        h->bgraph_failed = true;
        return;
    }
    h->capturing = true;
    const sem_status st = batch_iteration(h, s);
    h->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &g);
    if (st != SEM_OK || ee != cudaSuccess || g == nullptr ||
        cudaGraphInstantiate(&h->bgraph, g, 0) != cudaSuccess) {
        cudaGetLastError();
        h->bgraph = nullptr;
        h->bgraph_failed = true;
    }
    if (g) cudaGraphDestroy(g);
    h->bgraph_launches = h->launches - l0;
    h->bgraph_applies = h->fine_applies - a0;
    h->bgraph_vcycles = h->vcycles - v0;
    h->launches = l0;
    h->fine_applies = a0;
    h->vcycles = v0;
}

// Lifting of a batched tank from its staged Dirichlet data (h->st_eta): f = -A_FD phi~,
// ||f||^2 -> scal[S_FF], r = f, u = 0.  Capturable.
static sem_status batch_lift(sem_handle* h, cudaStream_t s) {
    const Level& L = h->lv[0];
    const long long N = L.N, nd = (long long)L.hdir.size();
    CKS(cudaMemsetAsync(h->x, 0, sizeof(double) * N, s));
    K(scatter_dirichlet(nd, L.dir, h->st_eta, h->x, s));
    CKST(apply_level64(h, 0, h->x, h->q, true, s));
    CKS(cudaMemsetAsync(h->fr, 0, sizeof(double) * N, s));
    K(axpy64(N, -1.0, h->q, h->fr, s));
    K(dot64(N, h->fr, h->fr, h->sc, h->sc.scal + S_FF, s));
    CKS(cudaMemcpyAsync(h->r, h->fr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    CKS(cudaMemsetAsync(h->bu, 0, sizeof(double) * N, s));
    return SEM_OK;
}

// End every capture still open on the listed streams (after a failed graph build).
static void end_captures(const std::vector<cudaStream_t>& streams) {
    for (cudaStream_t s : streams) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
        }
    }
    cudaGetLastError();
}

// Build the graph-resident batched solve (see BatchPlan).  The capture starts on a private
// origin stream (the caller's may be the legacy default stream, which cannot capture);
// every tank's branch runs on its own stream and the WHILE bodies are captured on a
// second private stream.  Returns nullptr when any step fails (all captures ended,
// errors cleared).
static BatchPlan* build_batch_plan(sem_handle* const* hs, int n, const std::vector<double>& rtol) {
    BatchPlan* plan = new (std::nothrow) BatchPlan();
    if (!plan) return nullptr;
    plan->rtol = rtol;
    plan->pro_launches.assign(n, 0);
    plan->body_launches.assign(n, 0);
    plan->body_applies.assign(n, 0);
    plan->body_vcycles.assign(n, 0);
    cudaStream_t cs = nullptr, body = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join(n, nullptr);
    std::vector<cudaStream_t> streams;
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    for (int t = 0; t < n && ok; ++t) ok = cudaEventCreateWithFlags(&join[t], cudaEventDisableTiming) == cudaSuccess;
    if (cs) streams.push_back(cs);
    if (body) streams.push_back(body);
    for (int t = 0; t < n; ++t) {
        streams.push_back(hs[t]->bstream);
        plan->uids.push_back(hs[t]->uid);
    }
    ok = ok && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    ok = ok && cudaEventRecord(fork, cs) == cudaSuccess;
    for (int t = 0; t < n && ok; ++t) {
        sem_handle* h = hs[t];
        cudaStream_t s = h->bstream;
        const long long l0 = h->launches, a0 = h->fine_applies, v0 = h->vcycles;
        h->capturing = true;
        ok = cudaStreamWaitEvent(s, fork, 0) == cudaSuccess && batch_lift(h, s) == SEM_OK;
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        cudaGraphConditionalHandle cond{};
        ok = ok && cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &ndeps) == cudaSuccess &&
             cst == cudaStreamCaptureStatusActive;
        ok = ok && cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault) == cudaSuccess;
        ok = ok && batch_loop_init(h->sc.scal, h->sc.flags, rtol[t], h->opts.atol, h->opts.imax, cond, s) == cudaSuccess;
        if (ok) h->launches += 1;
        plan->pro_launches[t] = h->launches - l0;
        ok = ok && cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &ndeps) == cudaSuccess;
        cudaGraphNodeParams p{};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = cond;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        ok = ok && cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &p) == cudaSuccess;
        ok = ok && cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                       cudaSuccess;
        if (ok) {
            const long long l1 = h->launches, a1 = h->fine_applies, v1 = h->vcycles;
            ok = cudaStreamBeginCaptureToGraph(body, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                ok = batch_iteration(h, body, false) == SEM_OK &&
                     batch_loop_check(h->sc.scal, h->sc.flags, rtol[t], h->opts.atol, h->opts.imax, cond, body) ==
                         cudaSuccess;
                h->launches += 1;
                cudaGraph_t bg = nullptr;
                ok = (cudaStreamEndCapture(body, &bg) == cudaSuccess) && ok;
            }
            plan->body_launches[t] = h->launches - l1;
            plan->body_applies[t] = h->fine_applies - a1;
            plan->body_vcycles[t] = h->vcycles - v1;
        }
        h->capturing = false;
        h->launches = l0;
        h->fine_applies = a0;
        h->vcycles = v0;
        ok = ok && cudaEventRecord(join[t], s) == cudaSuccess && cudaStreamWaitEvent(cs, join[t], 0) == cudaSuccess;
    }
    cudaGraph_t top = nullptr;
    const cudaError_t ee = cs ? cudaStreamEndCapture(cs, &top) : cudaErrorInvalidValue;
    ok = ok && ee == cudaSuccess && top != nullptr;
    ok = ok && cudaGraphInstantiate(&plan->exec, top, 0) == cudaSuccess;
    if (top) cudaGraphDestroy(top);
    end_captures(streams);
    if (body) cudaStreamDestroy(body);
    if (cs) cudaStreamDestroy(cs);
    if (fork) cudaEventDestroy(fork);
    for (cudaEvent_t e : join)
        if (e) cudaEventDestroy(e);
    if (!ok) {
        if (plan->exec) cudaGraphExecDestroy(plan->exec);
        delete plan;
        cudaGetLastError();
        return nullptr;
    }
    return plan;
}

// One launch of a graph-resident batched solve: stage every tank's Dirichlet data, launch
// the graph, write phi, then read each tank's iteration count and status from the device.
static sem_status batch_run_plan(BatchPlan* plan, sem_handle* const* hs, int n, const double* const* eta,
                                 double* const* phi, sem_stats* stats, cudaStream_t cs) {
    for (int t = 0; t < n; ++t) {
        sem_handle* h = hs[t];
        const long long nd = (long long)h->lv[0].hdir.size();
        if (nd > 0) CKS(cudaMemcpyAsync(h->st_eta, eta[t], sizeof(double) * nd, cudaMemcpyDeviceToDevice, cs));
    }
    CKS(cudaGraphLaunch(plan->exec, cs));
    for (int t = 0; t < n; ++t) {
        sem_handle* h = hs[t];
        const Level& L = h->lv[0];
        CKS(cudaMemcpyAsync(phi[t], h->bu, sizeof(double) * L.N, cudaMemcpyDeviceToDevice, cs));
        K(scatter_dirichlet((long long)L.hdir.size(), L.dir, eta[t], phi[t], cs));
    }
    CKS(cudaStreamSynchronize(cs));
    sem_status worst = SEM_OK;
    for (int t = 0; t < n; ++t) {
        sem_handle* h = hs[t];
        int fl[2] = {0, 0};
        double sc2[2] = {0, 0};
        CKS(cudaMemcpy(fl, h->sc.flags + F_BATCH_ITERS, 2 * sizeof(int), cudaMemcpyDeviceToHost));
        CKS(cudaMemcpy(&sc2[0], h->sc.scal + S_RR, sizeof(double), cudaMemcpyDeviceToHost));
        CKS(cudaMemcpy(&sc2[1], h->sc.scal + S_FF, sizeof(double), cudaMemcpyDeviceToHost));
        const int iters = fl[0];
        sem_status st_t = fl[1] == 0 ? SEM_OK : (fl[1] == 1 ? SEM_NOT_CONVERGED : SEM_NAN);
        CKST(check_tc_flag(h, &st_t));
        const double fnorm = std::sqrt(sc2[1]);
        const double rn = iters > 0 ? std::sqrt(sc2[0]) : fnorm;
        h->graph_iters = iters;
        h->fine_applies = iters * plan->body_applies[t];
        h->vcycles = iters * plan->body_vcycles[t];
        h->launches = plan->pro_launches[t] + iters * plan->body_launches[t];
        if (stats) {
            sem_stats st{};
            st.status = st_t;
            st.iters = iters;
            st.fnorm = fnorm;
            st.res0 = fnorm;
            st.res_final = rn;
            st.q_mean = (iters > 0 && fnorm > 0) ? std::pow(rn / fnorm, 1.0 / iters) : 0.0;
            st.fine_applies = h->fine_applies;
            st.vcycles = h->vcycles;
            st.kernel_launches = h->launches;
            st.graph_iterations = iters;
            stats[t] = st;
        }
        if (st_t != SEM_OK && (worst == SEM_OK || st_t < 0)) worst = st_t;
    }
    if (worst == SEM_NAN) set_error("laplace_solve_batch: non-finite residual");
    else if (worst == SEM_NOT_CONVERGED) set_error("laplace_solve_batch: a tank reached imax");
    else if (worst == SEM_TIMEOUT) set_error("laplace_solve_batch: a tensor-core copy wait ran out");
    return worst;
}

static sem_status batch_impl(sem_handle* const* hs, int n, const double* const* eta, double tol, double* const* phi,
                             sem_stats* stats, void* stream) {
    for (int t = 0; t < n; ++t) {
        if (!hs[t] || !eta[t] || !phi[t]) { set_error("laplace_solve_batch: NULL tank entry"); return SEM_EINVAL; }
        if (!hs[t]->opts.batch || hs[t]->opts.inner_imax != 0) {
            set_error("laplace_solve_batch: every handle needs batch = 1 and inner_imax = 0");
            return SEM_EINVAL;
        }
    }
    cudaStream_t cs = as_stream(stream);
    // graph-resident form first: the whole batch as one graph launch, loops decided on the device
    sem_handle* h0 = hs[0];
    if (!h0->bplan_failed && (h0->opts.batch_mode == 0)) {
        std::vector<double> rtolv(n);
        for (int t = 0; t < n; ++t) rtolv[t] = (tol > 0) ? tol : hs[t]->opts.rtol;
        bool valid = h0->bplan != nullptr && (int)h0->bplan->uids.size() == n && h0->bplan->rtol == rtolv;
        for (int t = 0; t < n && valid; ++t) valid = h0->bplan->uids[t] == hs[t]->uid;
        if (!valid) {
            if (h0->bplan) {
                if (h0->bplan->exec) cudaGraphExecDestroy(h0->bplan->exec);
                delete h0->bplan;
                h0->bplan = nullptr;
            }
            CKS(cudaStreamSynchronize(cs));
            h0->bplan = build_batch_plan(hs, n, rtolv);
            if (!h0->bplan) h0->bplan_failed = true;
        }
        if (h0->bplan) return batch_run_plan(h0->bplan, hs, n, eta, phi, stats, cs);
    }
    cudaEvent_t start, done;
    CKS(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    CKS(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    CKS(cudaEventRecord(start, cs));
    std::vector<double> thr(n), fnorm(n);
    std::vector<int> active(n, 1), iters(n, 0);
    std::vector<sem_status> status(n, SEM_OK);
    std::vector<double> rn(n);
    // lifting of every tank on its own stream, then one synchronisation for all
    for (int t = 0; t < n; ++t) {
        sem_handle* h = hs[t];
        cudaStream_t s = h->bstream;
        const Level& L = h->lv[0];
        const long long N = L.N, nd = (long long)L.hdir.size();
        h->fine_applies = h->vcycles = h->launches = 0;
        h->graph_iters = 0;
        h->coarse_iters_max = 0;
        CKS(cudaStreamWaitEvent(s, start, 0));
        CKS(cudaMemsetAsync(h->sc.flags + F_LEARN_COUNT, 0, 2 * sizeof(int), s));
        CKS(cudaMemsetAsync(h->x, 0, sizeof(double) * N, s));
        K(scatter_dirichlet(nd, L.dir, eta[t], h->x, s));
        CKST(apply_level64(h, 0, h->x, h->q, true, s));
        h->fine_applies -= 1;
        CKS(cudaMemsetAsync(h->fr, 0, sizeof(double) * N, s));
        K(axpy64(N, -1.0, h->q, h->fr, s));
        K(dot64(N, h->fr, h->fr, h->sc, h->sc.scal + S_FF, s));
        CKS(cudaMemcpyAsync(h->sc.hpinned + S_FF, h->sc.scal + S_FF, sizeof(double), cudaMemcpyDeviceToHost, s));
        CKS(cudaMemcpyAsync(h->r, h->fr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        CKS(cudaMemsetAsync(h->bu, 0, sizeof(double) * N, s));
    }
    for (int t = 0; t < n; ++t) {
        sem_handle* h = hs[t];
        CKS(cudaStreamSynchronize(h->bstream));
        fnorm[t] = std::sqrt(h->sc.hpinned[S_FF]);
        rn[t] = fnorm[t];
        const double rtol = (tol > 0) ? tol : h->opts.rtol;
        thr[t] = rtol * fnorm[t] + h->opts.atol;
        if (!std::isfinite(fnorm[t])) { status[t] = SEM_NAN; active[t] = 0; }
        else if (fnorm[t] <= thr[t]) active[t] = 0;
    }
    // lockstep iterations
    for (bool any = true; any;) {
        any = false;
        for (int t = 0; t < n; ++t) {
            if (!active[t]) continue;
            sem_handle* h = hs[t];
            if (iters[t] >= h->opts.imax) { active[t] = 0; status[t] = SEM_NOT_CONVERGED; continue; }
            batch_capture(h);
            if (h->bgraph) {
                CKS(cudaGraphLaunch(h->bgraph, h->bstream));
                h->graph_iters += 1;
                h->launches += h->bgraph_launches;
                h->fine_applies += h->bgraph_applies;
                h->vcycles += h->bgraph_vcycles;
            } else {
                CKST(batch_iteration(h, h->bstream));
            }
            any = true;
        }
        for (int t = 0; t < n; ++t) {
            if (!active[t]) continue;
            sem_handle* h = hs[t];
            CKS(cudaStreamSynchronize(h->bstream));
            iters[t] += 1;
            rn[t] = std::sqrt(h->sc.hpinned[S_RR]);
            if (!std::isfinite(rn[t])) { status[t] = SEM_NAN; active[t] = 0; }
            else if (rn[t] <= thr[t]) active[t] = 0;
        }
    }
    // results and join
    sem_status worst = SEM_OK;
    for (int t = 0; t < n; ++t) {
        sem_handle* h = hs[t];
        cudaStream_t s = h->bstream;
        const Level& L = h->lv[0];
        CKS(cudaMemcpyAsync(phi[t], h->bu, sizeof(double) * L.N, cudaMemcpyDeviceToDevice, s));
        K(scatter_dirichlet((long long)L.hdir.size(), L.dir, eta[t], phi[t], s));
        unsigned timeout = 0;
        CKS(cudaMemcpyAsync(&timeout, h->sc.counter + 3, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CKS(cudaStreamSynchronize(s));
        if (timeout && status[t] == SEM_OK) status[t] = SEM_TIMEOUT;
        CKST(check_tc_flag(h, &status[t]));
        CKS(cudaEventRecord(done, s));
        CKS(cudaStreamWaitEvent(cs, done, 0));
        if (stats) {
            sem_stats st{};
            st.status = status[t];
            st.iters = iters[t];
            st.fnorm = fnorm[t];
            st.res0 = fnorm[t];
            st.res_final = rn[t];
            st.q_mean = (iters[t] > 0 && fnorm[t] > 0) ? std::pow(rn[t] / fnorm[t], 1.0 / iters[t]) : 0.0;
            st.fine_applies = h->fine_applies;
            st.vcycles = h->vcycles;
            st.kernel_launches = h->launches;
            st.graph_iterations = h->graph_iters;
            stats[t] = st;
        }
        if (status[t] != SEM_OK && (worst == SEM_OK || status[t] < 0)) worst = status[t];
    }
    cudaEventDestroy(start);
    cudaEventDestroy(done);
    if (worst == SEM_TIMEOUT) set_error("laplace_solve_batch: a coarse-CG barrier wait ran out");
    else if (worst == SEM_NAN) set_error("laplace_solve_batch: non-finite residual");
    else if (worst == SEM_NOT_CONVERGED) set_error("laplace_solve_batch: a tank reached imax");
    return worst;
}

sem_status laplace_solve_batch(sem_handle* const* hs, int n, const double* const* eta, double tol, double* const* phi,
                               sem_stats* stats, void* stream) {
    if (!hs || n < 1 || !eta || !phi) { set_error("laplace_solve_batch: bad arguments"); return SEM_EINVAL; }
    for (int t = 0; t < n; ++t) {
        if (!hs[t] || !eta[t] || !phi[t]) { set_error("laplace_solve_batch: NULL tank entry"); return SEM_EINVAL; }
        if (!hs[t]->opts.batch || hs[t]->opts.inner_imax != 0 || !hs[t]->bstream) {
            set_error("laplace_solve_batch: every handle needs batch = 1 and inner_imax = 0");
            return SEM_EINVAL;
        }
        for (int u = 0; u < t; ++u)
            if (hs[u] == hs[t]) { set_error("laplace_solve_batch: a handle appears twice"); return SEM_EINVAL; }
    }
    const sem_status st = batch_impl(hs, n, eta, tol, phi, stats, stream);
    if (st != SEM_OK && st != SEM_NOT_CONVERGED && st != SEM_NAN && st != SEM_TIMEOUT) {
        // an error left the loop early: wait for every tank's work before returning
        for (int t = 0; t < n; ++t) cudaStreamSynchronize(hs[t]->bstream);
        cudaStreamSynchronize(as_stream(stream));
    }
    return st;
}

}  // extern "C"
