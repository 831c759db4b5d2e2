// Internal state of a sem_handle and the kernel launchers shared by the
// translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/sem.h"
#include "mlp.hpp"
#include "refelem.hpp"

namespace sem {

void set_error(const std::string& msg);

// Device copies of one level's reference matrices (Section 3.1):
// [Bt | DrT | DsT | Drt | Dst | Bz | Dz] where Bt/Drt/Dst are [QT][NT] and
// BtT/DrT/DsT the transposes [NT][QT].
template <typename T>
struct RefDev {
    T* m = nullptr;      // device block
    size_t count = 0;
};

struct Level {
    int dim = 3, p = 1, pz = 1;            // triangle order, vertical order (prisms; = p in 2D)
    int NT = 0, NZ = 1, QT = 0, QZ = 1, Np = 0, Nq = 0, ncomp = 6;
    int E = 0;           // elements
    long long N = 0;     // global nodes
    long long N2 = 0;    // 2D nodes (per vertical level in 3D)
    RefLevel ref;
    std::vector<int> hmap;                 // [E][Np]: g >= 0 free, -(g+1) Dirichlet
    std::vector<long long> hdir;           // Dirichlet node ids, ascending
    std::vector<double> hdiag;             // assembled diagonal (all nodes)
    double lam = 0.0;                      // lambda_hat of D^{-1}A
    // device
    int* map = nullptr;
    double* G = nullptr;                   // [E][ncomp][Nq]
    float* G32 = nullptr;
    unsigned short* G16 = nullptr;         // BF16 copy of G32 for the tensor-core apply (prisms, p >= 2)
    unsigned short* G16T = nullptr;        // order-6 prisms: BF16 factors in the tcgen05 apply's chunked layout
    int* lift_elems = nullptr;             // finest prism level: elements with a Dirichlet node (lifting apply)
    int nlift = 0;
    double* dinv = nullptr;                // 1/diag on free nodes, 0 on Dirichlet
    float* dinv32 = nullptr;
    long long* dir = nullptr;              // Dirichlet node ids
    RefDev<double> ref64;
    RefDev<float> ref32;
    // transfer to the next coarser level (valid for all but the coarsest)
    double* It64 = nullptr;                // [NT][NT_c]: coarse triangle basis at the fine triangle nodes
    double* Iz64 = nullptr;                // [NZ][NZ_c]: coarse 1D basis at the fine GLL nodes ([1] in 2D)
    float* It32 = nullptr;
    float* Iz32 = nullptr;
    unsigned char* owner = nullptr;        // [E][Np]: this element writes the prolonged value
    double* wmult = nullptr;               // 1 / (elements sharing the node)
    float* wmult32 = nullptr;
    // workspaces (length N)
    double *u = nullptr, *f = nullptr, *y = nullptr, *d = nullptr;
    float *u32 = nullptr, *f32 = nullptr, *y32 = nullptr, *d32 = nullptr;
    double* gref = nullptr;                // [dim][Nq][Np] full reference gradients (coarse level)
    int tile64 = 0, tile32 = 0;            // prism apply tile-shape variant (autotuned)
    int tc_kind = 1;                       // tensor-core smoothing operator (MIXED_TF32): 0 warp-level MMA,
                                           // 1 tcgen05 where compiled (order 6); autotuned at setup
    int* csr_rowptr = nullptr;             // coarse level: assembled matrix, free rows/cols
    int* csr_col = nullptr;
    double* csr_val = nullptr;
    int* csr_slot = nullptr;               // [E][Np][Np] CSR position of each element entry (or -1)
    // deterministic handles (prisms): node -> element-slot map and the FP64 element results
    int* dss_ptr = nullptr;                // [N + 1] segment of each node in dss_slot
    int* dss_slot = nullptr;               // slots e * Np + l of the free nodes, ascending (e, l) per node
    double* ye64 = nullptr;                // [E][Np] element results of the FP64 apply / restriction / diagonal
    double* Ae64 = nullptr;                // [E][Np][Np] FP64 element matrices (element-matrix apply) or null
    float2* Adf = nullptr;                 // [E][tiles][TS] upper block triangle of the element matrices as
                                           // (hi, lo) float pairs (double-FP32 apply) or null
    int df_T = 0, df_NB = 0, df_S = 0, df_TS = 0;   // its block layout (df_layout)
    int* df_err = nullptr;                 // set when a tile copy of that apply misses its wait bound
    int* csr_eptr = nullptr;               // coarse level: CSR entry -> element entries (e Np + i) Np + j, ascending
    int* csr_eidx = nullptr;
    double* csr_ev = nullptr;              // [E][Np][Np] element-matrix entries before their fixed-order sums
    long long csr_nnz = 0;
    // coarse level, block-Jacobi CG: blocks of free rows (compact patches), their FP32 inverses
    int bj_nb = 0;                         // number of blocks (0: point-Jacobi CG)
    int bj_nnzmax = 0;                     // most matrix entries in the rows of one block
    int* bj_ptr = nullptr;                 // [bj_nb + 1] offsets into bj_rows
    int* bj_rows = nullptr;                // free row ids, block by block
    float* bj_inv = nullptr;               // [bj_nb][kBjMax][kBjMax] symmetric inverse of each diagonal block
    int* bj_lptr = nullptr;                // [bj_nb][kBjMax + 1] offsets of the block's rows in its local CSR copy
    int* bj_lidx = nullptr;                // [bj_nb][bj_nnzmax] global CSR position of each local entry
    std::vector<int> hbj_ptr, hbj_rows;
    // additive Schwarz smoother (smoother = ASM; every level but the coarsest)
    int asm_nmax = 0;                      // largest subdomain (free nodes)
    long long asm_words = 0;               // block storage (elements of the V-cycle's type)
    int* asm_ptr = nullptr;                // [E+1] subdomain node-list offsets
    int* asm_nodes = nullptr;              // free global ids, ascending per subdomain
    long long* asm_off = nullptr;          // [E] offset of block k (row stride ld = n rounded up to 4)
    int* asm_tptr = nullptr;               // [E+1] offsets of the elements touching each subdomain
    int* asm_telems = nullptr;
    double* asm_w = nullptr;               // diagonal of W (0 at Dirichlet nodes)
    float* asm_w32 = nullptr;
    void* asm_blk = nullptr;               // inverted blocks, double (FP64 handles) or float
    std::vector<int> hasm_ptr, hasm_nodes;
};

// The whole batched solve of a list of tanks as one instantiated CUDA graph: per tank a
// branch with the lifting, a loop-control kernel and a WHILE conditional node whose body
// is one defect-correction iteration (the device decides when the tank has converged).
// Owned by the first handle of the list; valid while the list (by handle uid) and rtol
// are unchanged.
struct BatchPlan {
    std::vector<unsigned long long> uids;
    std::vector<double> rtol;
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> pro_launches, body_launches, body_applies, body_vcycles;
};

struct Scratch {
    double* part = nullptr;        // block partial sums
    unsigned* counter = nullptr;   // last-block counters
    double* scal = nullptr;        // device scalars
    int* flags = nullptr;          // device flags / counters
    double* hpinned = nullptr;     // pinned host mirror of scal (D2H of scalars)
    int* hflags = nullptr;
};

}  // namespace sem

struct sem_handle {
    int dim = 3, P = 1, nlayers = 0;
    double depth = 1.0;
    sem_options opts{};
    std::vector<sem::Level> lv;
    sem::Scratch sc;
    // outer-iteration vectors on the finest level (FP64)
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *x = nullptr, *fr = nullptr;
    // FGMRES basis
    double* V = nullptr;           // [(m+1)][N]
    double* Zb = nullptr;          // [m][N]
    double* gm_y = nullptr;        // [m] least-squares coefficients
    // coarse CG (FP64) on the coarsest level
    double *cx = nullptr, *cr = nullptr, *cz = nullptr, *cp = nullptr, *cq = nullptr, *cb = nullptr;
    // inner FP32 PCG of the mixed-precision path (finest level)
    float *ir = nullptr, *iz = nullptr, *ip = nullptr, *iq = nullptr, *ie = nullptr;
    long long inner_iters = 0;
    // learned smoothing sweep (per-element correction network) on the finest level
    sem::MlpNet net;
    sem::MlpGrads grads;
    sem::MlpAdam adam;
    float *mX = nullptr, *mT = nullptr, *mA1 = nullptr, *mH1 = nullptr, *mY = nullptr, *mdY = nullptr, *mdH = nullptr;
    float* mscale = nullptr;
    float *lr32 = nullptr, *ld32 = nullptr, *lu32 = nullptr;        // sweep work vectors
    float *te0 = nullptr, *tf = nullptr, *tu = nullptr, *tz = nullptr; // training data generation
    bool mlp_trained = false;
    bool learned_active = true;
    bool cgc_only = false;          // FP32 V-cycle without finest-level smoothing (coarse-grid correction)
    // batched lockstep solves (laplace_solve_batch): own stream, iterate, captured iteration graph
    bool capturing = false;         // launches are being captured: no host synchronisation
    cudaStream_t bstream = nullptr;
    double* bu = nullptr;
    cudaGraphExec_t bgraph = nullptr;
    bool bgraph_failed = false;
    unsigned long long uid = 0;     // unique per sem_setup in this process
    sem::BatchPlan* bplan = nullptr;   // graph-resident batched solve (this handle first in the list)
    bool coarse_flat = false;       // coarse levels built for a flat surface (sem_update_eta strategy 1)
    // free-surface time stepping (opts.surface_ops): surface operators and work fields
    int* fs_map2 = nullptr;         // [ntri][NT] order-P 2D node ids
    double *fs_vtri = nullptr, *fs_Drn = nullptr, *fs_Dsn = nullptr, *fs_Dtop = nullptr, *fs_invm = nullptr;
    double* fs_eta = nullptr;       // the surface elevation the finest geometry was built with [N2]
    double* fs_phi = nullptr;       // Laplace solution on the finest level [N]
    double *fs_w = nullptr, *fs_ex = nullptr, *fs_ey = nullptr, *fs_px = nullptr, *fs_py = nullptr;   // [N2]
    double* fs_k = nullptr;         // stage slopes: [4][N2] for eta, then [4][N2] for phi~
    double *fs_se = nullptr, *fs_sp = nullptr;   // stage values [N2]
    double* fs_hpin = nullptr;      // pinned host copy of a stage elevation [N2]
    bool bplan_failed = false;
    long long bgraph_launches = 0, bgraph_applies = 0, bgraph_vcycles = 0;
    long long graph_iters = 0;
    // staging buffers of laplace_solve_host
    double *st_eta = nullptr, *st_rhs = nullptr, *st_phi = nullptr;
    // host geometry copies for coordinate queries
    std::vector<double> vxy;
    std::vector<int> tri;
    std::vector<double> eta2;      // eta at order-P 2D nodes
    std::vector<std::vector<int>> map2;   // per level: [ntri][NT] 2D ids
    // prisms: base triangle and layer of every element (column by column, bottom up)
    std::vector<int> elem_b, elem_l;
    // optional geometry of a tank with a body (sem_mesh.col_layers / z_iface / edge_arc)
    bool general = false;          // any of them given: the general geometry kernel
    std::vector<double> zif;       // [nlayers+1][2] interfaces z = a + b eta (always filled in 3D)
    std::vector<double> arc;       // [ntri][3][3] or empty
    std::vector<double> xyP;       // [ntri][NT_P][2] order-P node xy (general meshes)
    // profiling events
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;      // per event pair: 0 FP64, 1 FP32, 2 TF32 tensor-core apply, 3 Schwarz blocks
    int ev_used = 0;
    double apply_ms = 0.0;         // FP64 finest-level applies
    long long apply_launches = 0;
    double apply32_ms = 0.0, apply_tc_ms = 0.0;
    long long apply32_launches = 0, apply_tc_launches = 0;
    double asm_ms = 0.0;
    long long asm_launches = 0;
    double lift_ms = 0.0;
    size_t auto_elem_bytes = 0;     // element matrices allocated by the auto rule (process-wide budget)
    void* small = nullptr;          // plan of the one-launch solve of small problems (small_solve.cu)
    long long lift_launches = 0;
    long long fine_applies = 0;
    long long launches = 0;        // kernels launched since the counter was reset
    long long vcycles = 0;
    int coarse_iters_max = 0;
    int device = 0;
};

namespace sem {

// Chebyshev coefficients of one sweep (three-term recurrence on [a, b]).
struct Cheb {
    double c0;               // first step: d = c0 D^{-1} r
    double c1[16], c2[16];   // step j >= 1: d = c1 d + c2 D^{-1} r
};

inline Cheb cheb_coeffs(double lam, const sem_options& o) {
    Cheb c{};
    const double b = o.cheb_hi * lam, a = o.cheb_lo * b;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
    c.c0 = 1.0 / theta;
    double rho = 1.0 / sigma;
    for (int j = 1; j < o.k_cheb && j < 16; ++j) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        c.c1[j] = rn * rho;
        c.c2[j] = 2.0 * rn / delta;
        rho = rn;
    }
    return c;
}

// small_solve.cu: the whole solve of a small FP64 problem in one launch (sem_options.fused_small)
sem_status build_small_plan(sem_handle* h);
void free_small_plan(sem_handle* h);
sem_status small_solve(sem_handle* h, const double* rhs, const double* eta, double rtol, double* phi, sem_stats* st,
                       cudaStream_t s);
// setup.cpp: inverse of an SPD matrix (n x n, row major) in place by Cholesky; false if not SPD
bool spd_inverse(std::vector<double>& a, int n);

// ---------------------------------------------------------------- kernels.cu
int reduce_blocks();
cudaError_t launch_apply64(const Level& L, const double* x, double* y, bool lift, const int* skip,
                           cudaStream_t s);
cudaError_t launch_apply32(const Level& L, const float* x, float* y, cudaStream_t s, const int* skip = nullptr);
// apply_prism.cu: prism apply with tile-shape variant 0 or 1 (elements per CTA pass)
cudaError_t launch_apply_prism64(const Level& L, const double* x, double* y, bool lift, const int* skip, int variant,
                                 cudaStream_t s);
cudaError_t launch_apply_prism32(const Level& L, const float* x, float* y, const int* skip, int variant,
                                 cudaStream_t s);
int prism_tile_elements(int P, int variant);
// apply_prism_tc.cu: TF32 tensor-core prism apply (FP32 in/out) for the mixed V-cycle's
// Chebyshev sweeps, orders 2..6; *err is set when its bounded copy wait runs out
cudaError_t launch_apply_prism_tc(const Level& L, const float* x, float* y, const int* skip, int* err,
                                  cudaStream_t s);
bool prism_tc_supported(int p);
// apply_prism_t5.cu: the order-6 prism apply on tcgen05 (TMEM accumulators, operands read from
// shared memory by descriptor); same arguments and error flag as launch_apply_prism_tc
cudaError_t launch_apply_prism_t5(const Level& L, const float* x, float* y, const int* skip, int* err,
                                  cudaStream_t s);
bool prism_t5_supported(int p);
// the tensor-core apply of a level: the warp-MMA kernel (the V-cycle's), or the tcgen05 kernel
// where it is compiled (order 6) when tcgen05 is set
inline cudaError_t launch_apply_tensor(const Level& L, const float* x, float* y, const int* skip, int* err,
                                       cudaStream_t s, bool tcgen05 = false) {
    return tcgen05 ? launch_apply_prism_t5(L, x, y, skip, err, s) : launch_apply_prism_tc(L, x, y, skip, err, s);
}
// the tensor-core apply serves isotropic prism levels of order 2..6
inline bool level_tc(const Level& L) { return L.dim == 3 && L.pz == L.p && prism_tc_supported(L.p); }
// apply_prism.cu: (triangle order, vertical order) pairs the prism apply is compiled for
bool prism_pair_supported(int p, int pz);
cudaError_t build_g16(Level& L, cudaStream_t s);
// schwarz.cu: FP64 element matrices [E][Np][Np] of a 3D level (synchronous)
cudaError_t element_matrices64(const Level& L, double* Ae, cudaStream_t s);
// apply_elem_df.cu: the FP64-accurate apply from the double-FP32 element matrices (L.Adf), and
// their block layout for Np nodes per element
cudaError_t apply_elem_df(const Level& L, const double* x, double* y, bool lift, const int* skip, cudaStream_t s);
void df_layout(int Np, int* T, int* NB, int* S, int* TS);
// tiles (w, w + d mod NB) of row block w in that layout: d = 0 .. NB/2, the last difference of an
// even NB only for w < NB/2, so every unordered block pair appears once
#if defined(__CUDACC__)
__host__ __device__
#endif
inline int df_tiles_of(int w, int NB) { return (NB & 1) || w < NB / 2 ? NB / 2 + 1 : NB / 2; }
// schwarz.cu: the double-FP32 element matrices of a 3D level in that layout (synchronous)
cudaError_t element_matrices_df(const Level& L, float2* Adf, cudaStream_t s);
// kernels.cu: y[g] = sum of the element results ye over node g's slots (fixed order); masked:
// 0 at the Dirichlet nodes
cudaError_t dss_gather64(const Level& L, const double* ye, double* y, const int* skip, cudaStream_t s,
                         bool masked);
// apply_prism_t5.cu: the factors of an order-6 prism level in the tcgen05 kernel's layout
cudaError_t build_g16_t6(Level& L, cudaStream_t s);
// fnpf.cu: surface fields of the free-surface time stepping
cudaError_t surface_gradient(int ntri, int NT, long long N2, const int* map2, const double* vtri, const double* Drn,
                             const double* Dsn, const double* inv_mult, const double* f2, double* gx, double* gy,
                             cudaStream_t s);
cudaError_t surface_w(long long N2, int NZ, long long k0, const double* Dtop, double depth, int nlayers,
                      const double* phi, const double* eta, double* w, cudaStream_t s);
cudaError_t fnpf_rhs(long long N2, int linear, double grav, const double* eta, const double* w, const double* ex,
                     const double* ey, const double* px, const double* py, double* deta, double* dphi,
                     cudaStream_t s);
cudaError_t rk_stage(long long n, double c, const double* x0, const double* k0, const double* x1, const double* k1,
                     double* o0, double* o1, cudaStream_t s);
cudaError_t rk4_combine(long long n, double dt, const double* k, double* x, cudaStream_t s);
// schwarz.cu: additive Schwarz smoother (subdomains, W, inverted blocks per level)
sem_status build_asm_level(sem_handle* h, int li);
sem_status refresh_asm_level(sem_handle* h, int li);   // new geometry: blocks recomputed in place
void free_asm_level(Level& L);
int asm_max_block(bool fp64);
// u += W sum_k R_k^T B_k R_k (f - y) (adjoint 0) or u += sum_k R_k^T B_k R_k W (f - y); y may be null
cudaError_t asm_apply64(const Level& L, const double* f, const double* y, int adjoint, double* u, cudaStream_t s);
cudaError_t asm_apply32(const Level& L, const float* f, const float* y, int adjoint, float* u, cudaStream_t s);
cudaError_t launch_geometry(Level& L, const double* vtri, const double* etaP, const double* BP,
                            const double* DrP, const double* DsP, int NTP, int nlayers, double depth,
                            cudaStream_t s);
// prisms of a general mesh: per-element (base triangle, layer), order-P node xy per base
// triangle, layer interfaces z = a + b eta
cudaError_t launch_geometry_general(Level& L, const int* eb, const int* el, const double* xyP, const double* etaP,
                                    const double* zif, const double* BP, const double* DrP, const double* DsP,
                                    int NTP, cudaStream_t s);
cudaError_t launch_diag(const Level& L, double* diag, cudaStream_t s);
cudaError_t launch_restrict64(const Level& F, const Level& C, const double* f, const double* y,
                              double* fc, cudaStream_t s);
cudaError_t launch_restrict32(const Level& F, const Level& C, const float* f, const float* y,
                              float* fc, cudaStream_t s);
cudaError_t launch_prolong64(const Level& F, const Level& C, const double* uc, double* uf, cudaStream_t s);
cudaError_t launch_prolong32(const Level& F, const Level& C, const float* uc, float* uf, cudaStream_t s);

// vector kernels (n = vector length)
// skip (optional): a device flag; when it is set the kernel does nothing
template <typename T>
cudaError_t cheb_first(long long n, T c, const T* dinv, const T* f, T* u, T* d, cudaStream_t s,
                       const int* skip = nullptr);
template <typename T>
cudaError_t cheb_restart(long long n, T c, const T* dinv, const T* f, const T* y, T* u, T* d, cudaStream_t s,
                         const int* skip = nullptr);
template <typename T>
cudaError_t cheb_step(long long n, T c1, T c2, const T* dinv, const T* f, const T* y, T* u, T* d,
                      cudaStream_t s, const int* skip = nullptr);
cudaError_t dot64(long long n, const double* a, const double* b, Scratch& sc, double* out, cudaStream_t s);
cudaError_t residual64(long long n, const double* f, const double* y, double* r, Scratch& sc, double* rr,
                       cudaStream_t s);
cudaError_t pcg_update(long long n, const double* num, const double* den, const double* p, const double* q,
                       double* u, double* r, Scratch& sc, double* rr, cudaStream_t s);
cudaError_t pcg_direction(long long n, const double* num, const double* den, const double* z, double* p,
                          cudaStream_t s);
cudaError_t axpy64(long long n, double a, const double* x, double* y, cudaStream_t s);
// Device-side loop control of the graph-resident batched solve: `init` (before the
// loop) and `check` (end of every iteration) set the WHILE node's condition from
// ||r||^2 = scal[S_RR] (or ||f||^2 = scal[S_FF] at init) against (rtol ||f|| + atol)^2
// and count iterations in flags[F_BATCH_ITERS]; flags[F_BATCH_STATUS] ends as 0 (met),
// 1 (imax reached) or -4 (non-finite).
cudaError_t batch_loop_init(double* scal, int* flags, double rtol, double atol, int imax,
                            cudaGraphConditionalHandle cond, cudaStream_t s);
cudaError_t batch_loop_check(double* scal, int* flags, double rtol, double atol, int imax,
                             cudaGraphConditionalHandle cond, cudaStream_t s);
cudaError_t dot32(long long n, const float* a, const float* b, Scratch& sc, double* out, cudaStream_t s);
cudaError_t pcg_update32(long long n, const double* num, const double* den, const float* p, const float* q, float* u,
                         float* r, Scratch& sc, double* rr, cudaStream_t s);
cudaError_t pcg_direction32(long long n, const double* num, const double* den, const float* z, float* p,
                            cudaStream_t s);
cudaError_t copy_dirichlet(long long nd, const long long* idx, const double* src, double* dst, cudaStream_t s);
cudaError_t copy_dirichlet32(long long nd, const long long* idx, const float* src, float* dst, cudaStream_t s);
cudaError_t scatter_dirichlet(long long nd, const long long* idx, const double* vals, double* dst, cudaStream_t s);
cudaError_t zero_dirichlet(long long nd, const long long* idx, double* v, cudaStream_t s);
cudaError_t to_f32(long long n, const double* a, float* b, cudaStream_t s);
cudaError_t to_f64(long long n, const float* a, double* b, cudaStream_t s);
cudaError_t multidot64(long long n, int k, const double* V, const double* w, Scratch& sc, double* out,
                       cudaStream_t s);
cudaError_t multiaxpy64(long long n, int k, const double* V, const double* c, double sign, double* w,
                        cudaStream_t s);
cudaError_t scale64(long long n, const double* w, const double* nrm2, double* v, cudaStream_t s);
// coarse CG: device-resident scalars, predicated on a done flag
cudaError_t cg_init(long long n, const double* b, const double* dinv, double* x, double* r, double* z,
                    double* p, Scratch& sc, double rtol2, cudaStream_t s);
cudaError_t cg_pq(long long n, const double* p, const double* q, Scratch& sc, cudaStream_t s);
cudaError_t cg_update(long long n, const double* dinv, double* x, double* r, double* z, const double* p,
                      const double* q, Scratch& sc, cudaStream_t s);
cudaError_t cg_direction(long long n, const double* z, double* p, Scratch& sc, cudaStream_t s);
// coarse level: assembled CSR matrix (free rows/cols) and the whole CG in one
// cooperative launch; the barrier timeout flag is counter[3]
cudaError_t coarse_assemble(const Level& C, const double* gref, const int* slot, double* vals, cudaStream_t s);
// the same CG in a single CTA (no inter-CTA waits): batched tanks and small coarse levels
cudaError_t coarse_cg_single(const Level& C, const int* rowptr, const int* col, const double* vals, const double* b,
                             double* x, double* r, double* z, double* p, double* q, Scratch& sc, double rtol2, int imax,
                             cudaStream_t s);
cudaError_t coarse_cg_persistent(const Level& C, const int* rowptr, const int* col, const double* vals,
                                 const double* b, double* x, double* r, double* z, double* p, double* q, Scratch& sc,
                                 double rtol2, int imax, unsigned extra_arrivals, cudaStream_t s);
// block-Jacobi preconditioned CG (one CTA per block of C.bj_ptr / C.bj_rows, the FP32 block
// inverses C.bj_inv in shared memory), one cooperative launch; same flags as the above
constexpr int kBjMax = 128;                 // rows per block at most
int coarse_bj_capacity(int nnzmax);         // blocks that can be co-resident with nnzmax entries each
cudaError_t coarse_cg_bj(const Level& C, const double* b, double* x, double* z, double* pa, double* pb, Scratch& sc,
                         double rtol2, int imax, unsigned extra_arrivals, cudaStream_t s);

// scalar slots in Scratch::scal
enum {
    S_RR = 0, S_PQ = 1, S_DELTA0 = 2, S_DELTA1 = 3, S_FF = 4, S_TMP = 5,
    S_CG_RHO = 8, S_CG_PQ = 9, S_CG_RR = 10, S_CG_TOL2 = 11, S_CG_RHONEW = 12, S_CG_BETA = 13,
    S_IRR = 6, S_IPQ = 7, S_IDELTA0 = 14, S_IDELTA1 = 15, S_L0 = 100, S_L1 = 101, S_LOSS = 102, S_RQ = 103, S_QQ = 104, S_ALPHA = 105,
    S_MULTI = 16                    // FGMRES dots start here (up to 64 + 1)
};
enum { F_CG_DONE = 0, F_CG_ITERS = 1, F_LEARN_ACCEPT = 2, F_LEARN_COUNT = 3 /* +0 accepts, +1 fallbacks */,
       F_TC_ERR = 5, F_BATCH_ITERS = 6, F_BATCH_STATUS = 7, F_ASM_BAD = 8 };
constexpr int kFlagCount = 16;

}  // namespace sem
