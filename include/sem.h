/*
 * sem.h - C ABI of the GB300 p-multigrid spectral element Laplace solver.
 *
 * The library solves the Laplace problem for the velocity potential of the
 * fully nonlinear potential-flow model (Section 2, Eq. laplaceproblem):
 *     phi = phi~ on the free surface z = eta,  laplace(phi) = 0 in the fluid,
 *     n . grad(phi) = 0 on the bottom and the walls,
 * discretised by a Galerkin spectral element method with a continuous nodal
 * basis of order P on straight triangles (2D vertical slices) or sigma-layer
 * prisms with a curvilinear free surface (3D) (Section 3.1, Eq.
 * laplaceproblemdiscrete), and solved by PCG (Algorithm 3), preconditioned
 * defect correction (Algorithm 2) or flexible GMRES, each preconditioned by
 * one geometric p-multigrid V-cycle (Algorithm 1) with Chebyshev-Jacobi
 * smoothing, p-transfers P and R = P^T (Section 4.1, Eq. rest) and an FP64
 * coarse solve at order 1.
 *
 * Conventions shared by every entry point
 *  - The stiffness matrix is A = -L^p (L^p of Eq. laplaceproblemdiscrete), so
 *    that A restricted to the free (non-Dirichlet) nodes is symmetric
 *    positive definite.
 *  - Vectors are FP64, one entry per global node of a level, in the library's
 *    canonical numbering (first appearance over elements for triangle meshes;
 *    id = kz * N2 + g2 for prism meshes, g2 the 2D id, kz the vertical index).
 *  - "_dev" pointers are CUDA device pointers owned by the caller; "_host"
 *    pointers are host memory owned by the caller.  The handle owns all other
 *    device memory (geometry, maps, workspaces); no entry point allocates after
 *    sem_setup.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *    asynchronous with respect to the host except where stated.
 *  - Errors are returned as sem_status; nothing exits, aborts or traps.  The
 *    message of the last error of the calling thread is sem_last_error().
 */
#ifndef SEM_GB300_H
#define SEM_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

#define SEM_MAX_LEVELS 8

typedef enum {
    SEM_OK = 0,
    SEM_NOT_CONVERGED = 1,  /* i_max reached; the last iterate and stats are written */
    SEM_EINVAL = -1,        /* invalid argument (message in sem_last_error) */
    SEM_ECUDA = -2,         /* CUDA runtime error */
    SEM_ENOMEM = -3,        /* device or host allocation failed (sem_setup only) */
    SEM_NAN = -4,           /* non-finite residual */
    SEM_BREAKDOWN = -5,     /* p^T A p <= 0 in PCG, or a zero Krylov vector */
    SEM_TIMEOUT = -6        /* a bounded device-side wait ran out */
} sem_status;

typedef enum { SEM_OUTER_PCG = 0, SEM_OUTER_FGMRES = 1, SEM_OUTER_PDC = 2 } sem_outer;
/* MIXED_FP32: FP32 V-cycle (and optional FP32 inner PCG) inside an FP64 outer iteration with
 * FP64 residual and FP64 coarse solve.  MIXED_TF32: the same, with the V-cycle's operator on
 * prism levels of order 2..6 (Chebyshev sweeps and the residual before restriction) on the
 * tensor cores (TF32 operands, BF16 geometric factors, FP32 accumulation); the inner PCG's
 * products stay FP32. */
typedef enum { SEM_PREC_FP64 = 0, SEM_PREC_MIXED_FP32 = 1, SEM_PREC_MIXED_TF32 = 2 } sem_precision;
/* Smoothers: Chebyshev-Jacobi (default); LEARNED (see sem_options.smoother); ASM, the
 * paper's overlapping additive Schwarz smoother (Section 4.3, Eqs. sec_form, Mass, weights):
 * u <- u + S^{-1}(f - A u), S^{-1} = W sum_k R_k^T (R_k A R_k^T)^{-1} R_k with one subdomain
 * per element (its nodes and those within asm_overlap lattice steps; a step joins two nodes
 * of one element whose lattice indices (i, j) of the triangle and k of the vertical line
 * differ by at most one in i, j, i + j and k), W = (sum_k R_k R_k^T)^{-1}.  Pre-smoothing
 * applies S^{-1}, post-smoothing its adjoint sum_k R_k^T (R_k A R_k^T)^{-1} R_k W (a
 * symmetric V-cycle).  The blocks are inverted at setup and held densely in the V-cycle's
 * precision (FP64, or FP32 in the mixed precisions). */
typedef enum { SEM_SMOOTH_CHEBYSHEV = 0, SEM_SMOOTH_LEARNED = 1, SEM_SMOOTH_ASM = 2 } sem_smoother;
/* Forms of the FP64 operator apply (sem_options.elem_matrices): sum-factorised contraction,
 * FP64 element matrices, or double-FP32 element matrices (upper block triangle). */
typedef enum { SEM_ELEM_OFF = 0, SEM_ELEM_FP64 = 1, SEM_ELEM_DF32 = 2 } sem_elem_form;

/* Mesh description (host memory, read during sem_setup only).
 * dim 2: ntri straight triangles in the (x, z) plane; vxy holds (x, z).
 * dim 3: ntri base triangles in the (x, y) plane extruded into nlayers sigma
 *        layers between the flat bottom z = -depth and the free surface
 *        z = eta(x, y): the node at sigma in [0, 1] sits at
 *        z = -depth + sigma * (depth + eta).  Prism e lies over base triangle
 *        e / nlayers in layer e % nlayers (layer 0 at the bottom).
 * Triangles are counter-clockwise; vertex ids index vxy.
 * eta: free-surface elevation at the order-P 2D nodes of the base mesh in
 *      canonical order (see sem_mesh_nodes2d), or NULL for a flat surface.
 * face_bc: [nelem][nfaces] flags, 1 = Dirichlet (phi = phi~), 0 = homogeneous
 *      Neumann or interior.  Triangle faces: f0=(v0,v1), f1=(v1,v2), f2=(v2,v0).
 *      Prism faces: f0..f2 lateral quads over those edges, f3 bottom, f4 top.
 *
 * Optional dim-3 fields for a tank with a surface-piercing body (all NULL for the
 * plain sigma-layer mesh above; NULL fields keep its rule):
 * col_layers: [ntri], 1..nlayers: the prisms over base triangle b are its layers
 *      0 .. col_layers[b]-1; prisms are numbered column by column, bottom up, so
 *      nelem = sum col_layers.  Node ids keep the layout kz * N2 + g2; ids that lie
 *      in no prism (above a body) are identity rows of every operator and are listed
 *      with the Dirichlet nodes (their phi~ is copied through unchanged).
 * z_iface: [nlayers+1][2] (a_k, b_k): layer interface k lies at z = a_k + b_k eta(x, y)
 *      and the node at local t in [-1, 1] of layer l at
 *      z = (1 - tau) z_l + tau z_{l+1}, tau = (t + 1)/2 (NULL: the sigma layers,
 *      a_k = -depth (1 - k/nlayers), b_k = k/nlayers).  Two zones around a hull: flat
 *      interfaces (b = 0) below its draft, sigma interfaces above.  Every layer must
 *      keep a positive thickness at every surface node.
 * edge_arc: [ntri][3][3]: for base edge f of triangle b (faces as above) the circle
 *      (cx, cy, R) the edge follows between its two vertices (both on the circle,
 *      at most a quarter turn apart), R = 0 for a straight edge.  The base triangle's
 *      map is the affine map plus, per curved edge (a, b), the edge's displacement
 *      from its chord times 4 l_a l_b / (1 - xi^2), xi = l_b - l_a (l barycentric),
 *      the arc point taken at angle theta_a + (1 + xi)/2 (theta_b - theta_a) (the
 *      triangle blending map of Szabo and Babuska, Finite Element Analysis, Ch. 6);
 *      the element geometry is its order-P interpolant (isoparametric).
 * sem_update_eta works on such meshes; the free-surface operators (surface_ops)
 * need the plain sigma-layer mesh. */
typedef struct {
    int dim;
    int nvert;
    const double* vxy;          /* [nvert][2] */
    int ntri;
    const int* tri;             /* [ntri][3] */
    int nlayers;                /* dim 3 only (>= 1) */
    double depth;               /* dim 3 only (> 0) */
    const double* eta;          /* dim 3 only, [N2 at order P] or NULL */
    const signed char* face_bc; /* [nelem][nfaces] */
    const int* col_layers;      /* dim 3 only, [ntri] or NULL */
    const double* z_iface;      /* dim 3 only, [nlayers+1][2] or NULL */
    const double* edge_arc;     /* dim 3 only, [ntri][3][3] or NULL */
} sem_mesh;

/* Solver options; fill with sem_default_options and adjust.
 * level_p[0] = P >= level_p[1] >= ... >= level_p[nlevels-1] = 1 (triangle order per level;
 * prisms may give a separate vertical order per level in level_pz).
 * Smoother: k_cheb-step Chebyshev iteration on D^{-1}A over [cheb_lo*b, b],
 * b = cheb_hi * lambda_hat, lambda_hat = the largest Ritz value of lanczos_steps
 * Lanczos steps on D^{-1}A started from x_i = sin(i+1) on free nodes (a lower
 * bound of lambda_max); nu1 pre- and nu2 post-sweeps (Algorithm 1).
 * Stop test ||r||_2 <= rtol*||f||_2 + atol on the FP64 free-node residual.
 * The coarse order-1 system is solved by FP64 block-Jacobi or Jacobi CG (coarse_bj) to coarse_rtol
 * relative residual (at most coarse_imax iterations). */
typedef struct {
    int outer;                  /* sem_outer */
    int precision;              /* sem_precision: FP64, or FP32 V-cycle inside an FP64 outer */
    int nu1, nu2, k_cheb;
    double cheb_lo, cheb_hi;
    int lanczos_steps;
    int nlevels;
    int level_p[SEM_MAX_LEVELS];
    double rtol, atol;
    int imax;
    int gmres_m;                /* FGMRES restart length */
    double coarse_rtol;
    int coarse_imax;
    int profile;                /* 1: time every operator apply with CUDA events (sem_stats.apply_ms) */
    int inner_imax;             /* MIXED_FP32 only: 0 = one FP32 V-cycle per outer iteration; > 0 = FP32 PCG
                                   (FP32 V-cycle preconditioner) to inner_rtol, at most inner_imax iterations */
    double inner_rtol;
    int debug_barrier_extra;    /* testing only (default 0): > 0 makes every grid barrier of the persistent
                                   coarse CG wait for arrivals that never come, so each wait runs into its
                                   1 s limit and the call returns SEM_TIMEOUT with the context intact */
    int smoother;               /* sem_smoother.  LEARNED (MIXED_FP32 only): once sem_learned_train has
                                   run, the first finest-level post-smoothing sweep of the FP32 V-cycle is
                                   the correction network's, kept only if it lowers the residual norm
                                   (otherwise the Chebyshev sweep runs).  The V-cycle is then nonlinear:
                                   use the PDC or FGMRES outer iteration. */
    int mlp_hidden;             /* hidden width of the correction network (default 256) */
    unsigned long long mlp_seed; /* seed of the network's initial weights */
    int batch;                  /* 1: prepare the handle for laplace_solve_batch (own stream and iterate) */
    int autotune;               /* 1 (default): time the prism apply's tile shapes (elements per CTA pass)
                                   on every level at setup and keep the faster (cached per order,
                                   precision and element-count bucket for the process) */
    double learned_tau;         /* the learned sweep's correction (minimal-residual step) is kept when it
                                   brings ||r|| below learned_tau * ||r|| (default 0.5); after three
                                   rejections and no acceptance a solve continues without it */
    int surface_ops;            /* 1: prepare the free-surface operators of sem_fnpf_rhs / sem_fnpf_step
                                   (3D meshes whose Dirichlet nodes are exactly the surface nodes) */
    int batch_mode;             /* laplace_solve_batch with this handle first in the list: 0 (default)
                                   the whole batch as one CUDA graph launch with the convergence test
                                   on the device, 1 host-stepped lockstep */
    int asm_overlap;            /* smoother = ASM: overlap in nodes (default 1; 0 = block Jacobi over the
                                   element node sets; -1 = "refined Schwarz", ceil((p+1)/2) on the
                                   order-p level).  Subdomains of more than 1600 (FP64) or 3200 (FP32)
                                   nodes are refused with SEM_EINVAL */
    int level_pz[SEM_MAX_LEVELS]; /* prisms: vertical order of each level (0 = level_p, the default).  With
                                   level_pz[0] < P the finest prisms are anisotropic (P_xy = P, P_z =
                                   level_pz[0]; Section 6); semi-coarsening lowers one order at a time,
                                   e.g. (5,3) -> (3,3) -> (1,1).  Per level neither order may grow and one
                                   must fall; the coarsest level is (1,1); the vertical order equals the
                                   triangle order or lies one or two below it */
    int deterministic;          /* 3D meshes: 1 = the FP64 operator applies and restrictions write element
                                   results that each node then sums over a precomputed node -> element-slot
                                   map in a fixed order (no atomics), so FP64 solves are bit-reproducible run
                                   to run; 0 (default) = atomic summation.  The single-precision applies
                                   keep atomic summation */
    int elem_matrices;          /* 3D meshes: the FP64 operator applies multiply by precomputed element
                                   matrices A_e (2 Np^2 flops per element, 42 % fewer than the
                                   sum-factorised contraction at P = 6; held on the device and recomputed
                                   when eta changes) on every level of an FP64 handle but the coarsest,
                                   and on the finest level (the residual) of a mixed-precision one.
                                   SEM_ELEM_FP64 (1): FP64 matrices, FP64 arithmetic (Np^2 doubles per
                                   element).  SEM_ELEM_DF32 (2): the upper block triangle as double-FP32
                                   pairs, multiplied in compensated FP32 arithmetic (TwoProduct/TwoSum)
                                   with FP64 sums per block: a row's error stays within a few 1e-13 of
                                   sum_j |A_ij x_j| (FP64: about 1e-15), on the FP32 pipe (182 KB per
                                   element at P = 6 against 307 KB).  SEM_ELEM_OFF (0): sum
                                   factorisation.  -1 (default): SEM_ELEM_FP64 for FP64 handles and
                                   SEM_ELEM_DF32 for mixed-precision ones, when they take at most a
                                   quarter of the free device memory and 48 GB (across all live handles)
                                   and the handle is not batched, else off; matrices taken by this rule
                                   are dropped at the first sem_update_eta (a moving surface would
                                   recompute them at every update, seconds at the benchmark size), while
                                   explicitly requested ones are recomputed */
    int coarse_bj;              /* 1 (default) = the coarse CG is preconditioned by block Jacobi: the free
                                   order-1 nodes are cut into compact patches of at most 128 (recursive
                                   coordinate bisection in the horizontal), each patch's diagonal block is
                                   inverted at setup (and whenever the coarse matrix is reassembled) and
                                   applied from shared memory, one CTA per patch (about half the CG
                                   iterations of point Jacobi); used when every patch fits one co-resident
                                   CTA and the handle is not batched.  0 = point-Jacobi CG */
    int fused_small;            /* 1 (default) = small FP64 problems (finest level at most 8,192 nodes
                                   and E Np^2 <= 2^18, FGMRES or PCG outside, Chebyshev smoother, an
                                   assembled coarse level of at most 2,048 nodes, not batched) are solved
                                   in one kernel launch by one CTA: lifting, outer iteration and V-cycle
                                   with every level's operator as FP64 element matrices and the coarse
                                   level solved directly by a dense inverse formed at setup (coarse_rtol
                                   does not apply).  0 = the multi-kernel path */
} sem_options;

typedef struct {
    int status;                 /* sem_status of the solve */
    int iters;                  /* outer iterations (preconditioner applications after the first) */
    double fnorm;               /* ||f||_2 of the lifted right-hand side */
    double res0, res_final;     /* ||r||_2 at start and end (FP64 residual) */
    double q_mean;              /* geometric mean residual contraction per iteration (Eq. convrate) */
    long long fine_applies;     /* operator applies on the finest level (work units, Section 4.4) */
    long long vcycles;
    int coarse_iters_max;       /* largest coarse CG iteration count seen */
    double ms;                  /* wall time of the call on the stream (CUDA events) */
    double apply_ms;            /* summed time of finest-level FP64 apply kernels (profile = 1) */
    long long apply_launches;   /* finest-level FP64 apply kernel launches (profile = 1) */
    long long kernel_launches;  /* kernels of this library launched by the call */
    long long inner_iters;      /* FP32 inner PCG iterations (MIXED_FP32 with inner_imax > 0) */
    long long learned_accepts;  /* learned sweeps kept (smoother = LEARNED) */
    long long learned_fallbacks; /* learned sweeps rejected by the residual test (Chebyshev ran instead) */
    long long graph_iterations; /* laplace_solve_batch: iterations replayed from the captured CUDA graph */
    double apply32_ms;          /* profile = 1: summed event time of the finest-level FP32 applies */
    long long apply32_launches;
    double apply_tc_ms;         /* profile = 1: same for the TF32 tensor-core applies (MIXED_TF32) */
    long long apply_tc_launches;
    double asm_ms;              /* profile = 1: summed event time of the finest-level Schwarz block kernels */
    long long asm_launches;
    double lift_ms;             /* profile = 1: event time of the lifting apply (f = -A_FD phi~, only the
                                   finest elements that touch a Dirichlet node); not in apply_ms */
    long long lift_launches;
} sem_stats;

typedef struct sem_handle sem_handle;

/* Defaults for finest order P: PCG, FP64, nu1 = nu2 = 1, k_cheb = 5,
 * cheb_lo = 0.01, cheb_hi = 1.05, lanczos_steps = 30, levels P -> ... -> 1 from the
 * table {6:6,3,1; 5:5,3,1; 4:4,2,1; 3:3,2,1; 2:2,1; 1:1}, rtol 1e-8, atol 0,
 * imax 200, gmres_m 30, coarse_rtol 1e-2, coarse_imax 5000, inner_imax 0,
 * inner_rtol 1e-4.  The smoother and coarse-tolerance defaults minimise the
 * time to a 1e-8 residual on the 64x64x4-prism P = 6 box; a coarse_rtol of
 * 1e-14 makes the V-cycle the exact-coarse-solve Algorithm 1 to rounding. */
void sem_default_options(sem_options* opts, int P);

/* Canonical order-p 2D node coordinates of the triangle mesh in `mesh`
 * (x, z for dim 2; x, y of the base mesh for dim 3; with edge_arc, the blended map
 * at the order-p reference nodes).  Pass xy = NULL to get the count in *n2 only;
 * otherwise xy must hold 2 * (*n2) doubles.  Host only, synchronous.  This is where
 * the caller samples eta before sem_setup. */
sem_status sem_mesh_nodes2d(const sem_mesh* mesh, int p, long long* n2, double* xy);

/* Build every level (numbering, geometric factors, Jacobi diagonals, Chebyshev
 * bounds, transfers, coarse workspace) and allocate all device memory on the
 * current CUDA device.  Synchronous.  P in 1..6; opts NULL = defaults. */
sem_status sem_setup(const sem_mesh* mesh, int P, const sem_options* opts, sem_handle** out);
/* Free a handle (synchronises the device first).  Not named sem_destroy: that is the POSIX
 * semaphore call, which the statically linked CUDA runtime inside the library uses. */
void sem_teardown(sem_handle* h);

/* Sizes of a level: global nodes, Dirichlet nodes, elements, nodes per element. */
sem_status sem_query(const sem_handle* h, int level, long long* ndof, long long* ndirichlet,
                     long long* nelem, int* np);
/* Host copies: Dirichlet node ids (ascending; the order of dirichlet_eta),
 * node coordinates [N][dim] (x, y of a level of order p < P on curved base
 * triangles: the order-P geometry interpolated at the level's nodes), the element
 * map [E][Np] (global ids), the lambda_hat estimate of every level (coarsest entry 0). */
sem_status sem_dirichlet_nodes(const sem_handle* h, int level, long long* idx_host);
sem_status sem_node_coords(const sem_handle* h, int level, double* xyz_host);
sem_status sem_element_map(const sem_handle* h, int level, int* map_host);
sem_status sem_lambda_max(const sem_handle* h, double* lam_host);
/* Elements per CTA pass of the prism apply chosen for a level (FP64 and FP32 kernels). */
sem_status sem_tile_shapes(const sem_handle* h, int level, int* elems_fp64, int* elems_fp32);
/* The operator of a level's Chebyshev sweeps under MIXED_TF32: 0 the FP32 apply (not a
 * tensor-core level), 1 the warp-level MMA kernel, 2 the tcgen05 kernel (order 6; chosen at
 * setup by timing both when autotune is set, else the tcgen05 kernel). */
sem_status sem_tc_kernel(const sem_handle* h, int level, int* kind);
/* The form of a level's FP64 applies (sem_options.elem_matrices): SEM_ELEM_FP64 or SEM_ELEM_DF32
 * when they multiply by precomputed element matrices, SEM_ELEM_OFF for the sum-factorised
 * contraction. */
sem_status sem_elem_matrices(const sem_handle* h, int level, int* kind);
/* The assembled diagonal of A at a level (all nodes), host copy. */
sem_status sem_diagonal(const sem_handle* h, int level, double* diag_host);

/* Matrix-free operator (Eq. laplaceproblemdiscrete, a2 of the hot path):
 * y_F = A_FF x_F on the free nodes and y_D = x_D on the Dirichlet nodes of
 * `level` (0 = finest).  x_dev, y_dev: N doubles, distinct buffers. */
sem_status sem_apply(sem_handle* h, int level, const double* x_dev, double* y_dev, void* stream);

/* The same operator in single precision, as the mixed V-cycle applies it: the FP32
 * kernel (tensor_cores = 0) or the TF32 tensor-core kernel of the MIXED_TF32
 * Chebyshev sweeps (tensor_cores = 1: warp-level MMA; prism levels of order 2..6, else
 * SEM_EINVAL; operands rounded to TF32, FP32 accumulation).  tensor_cores = 2 runs the
 * same operator on tcgen05 (TMEM accumulators, operands read by descriptor; order 6
 * only, else SEM_EINVAL), a second kernel that the V-cycle does not use.  x_dev, y_dev:
 * N floats, distinct; y_D = x_D.  The tensor-core forms synchronise the stream and
 * return SEM_TIMEOUT if a copy or an MMA inside the kernel did not complete within 1 s. */
sem_status sem_apply32(sem_handle* h, int level, const float* x_dev, float* y_dev, int tensor_cores,
                       void* stream);

/* Subdomains of the additive Schwarz smoother on `level` (smoother = ASM; every level but
 * the coarsest): ptr_host [nelem + 1] offsets (int64, may be NULL), nodes_host [ptr[nelem]]
 * the free global node ids of element k's subdomain, ascending, at ptr[k] .. ptr[k+1]-1
 * (int32, may be NULL).  SEM_EINVAL if the level has no Schwarz blocks. */
sem_status sem_asm_subdomains(const sem_handle* h, int level, long long* ptr_host, int* nodes_host);

/* z = S^{-1} r (adjoint = 0) or S^{-T} r (adjoint = 1) on `level`, Eq. Mass, with the
 * handle's blocks: sem_asm_apply for FP64 handles (N device doubles), sem_asm_apply32
 * for mixed-precision handles (N device floats); the Dirichlet entries of z are zero.
 * SEM_EINVAL for the other precision or a level without blocks. */
sem_status sem_asm_apply(sem_handle* h, int level, const double* r_dev, double* z_dev, int adjoint, void* stream);
sem_status sem_asm_apply32(sem_handle* h, int level, const float* r_dev, float* z_dev, int adjoint, void* stream);

/* Strategies for a new surface elevation (the paper's operator-reuse strategies I-III,
 * Section 5): SEM_ETA_FINEST updates the finest operator and keeps the diagonals and coarse
 * operators of t = 0 (the finest lambda_hat is re-estimated against the new operator: the
 * Chebyshev interval has to cover its spectrum); SEM_ETA_LINEAR_COARSE also updates the
 * finest smoother
 * (diagonal, lambda_hat) and uses linear (flat-surface) operators on the coarse levels;
 * SEM_ETA_ALL rebuilds every operator of every level from the new elevation. */
typedef enum { SEM_ETA_FINEST = 0, SEM_ETA_LINEAR_COARSE = 1, SEM_ETA_ALL = 2 } sem_eta_strategy;

/* New free-surface elevation for a 3D handle (time stepping): eta_nodal_host holds eta at
 * the order-P 2D nodes (the order of sem_mesh_nodes2d, as sem_mesh.eta).  Recomputes the
 * geometric factors and, per `strategy`, the diagonals, lambda_hat estimates and the
 * assembled coarse matrix, in place (no allocation after the first call, except the
 * temporary element matrices from which a Schwarz handle rebuilds its blocks; captured
 * batch graphs stay valid).  With smoother = ASM the blocks follow the strategy: FINEST
 * keeps those of t = 0, LINEAR_COARSE rebuilds the finest level's (coarse levels flat),
 * ALL rebuilds every level's.  A mixed-precision handle re-estimates lambda_hat with the FP32
 * operator its V-cycle smooths with (the FP64 Lanczos recurrence is kept); sem_setup
 * estimates with the FP64 operator in every precision.  Synchronous.  SEM_EINVAL for a 2D
 * handle or an unknown strategy. */
sem_status sem_update_eta(sem_handle* h, const double* eta_nodal_host, int strategy);

/* Free-surface time stepping around the Laplace solve (Section 2, Eqs. FSeta, FSphi), for
 * handles set up with surface_ops = 1.  Surface fields live at the order-P 2D nodes (N2
 * device doubles, the order of sem_mesh_nodes2d): eta (elevation) and phis (potential phi~).
 * The right-hand sides
 *   d eta/dt  = -grad eta . grad phi~ + w~ (1 + |grad eta|^2)
 *   d phi~/dt = -g eta - (|grad phi~|^2 - w~^2 (1 + |grad eta|^2)) / 2
 * take w~ = dphi/dz at the surface from laplace_solve with phi = phi~ on z = eta (to rtol
 * tol), the geometry first moved to eta by sem_update_eta(strategy); grad is the horizontal
 * gradient of the order-P interpolant on each surface triangle, averaged over the triangles
 * sharing a node.  linear = 1: the small-amplitude form d eta/dt = w~, d phi~/dt = -g eta on
 * the handle's fixed geometry (set it up with a flat surface).  Synchronous. */
sem_status sem_fnpf_rhs(sem_handle* h, const double* eta_dev, const double* phis_dev, double g, int linear,
                        int strategy, double tol, double* deta_dev, double* dphis_dev, void* stream);
/* One step of the classical four-stage Runge-Kutta method (ERK4) on (eta, phis) in place: four
 * right-hand sides, four Laplace solves.  stats (nullable): status, the solves' summed
 * iterations (iters), fine-level applies and time (ms).  A failed solve stops the step and
 * returns its status with eta and phis unchanged. */
sem_status sem_fnpf_step(sem_handle* h, double* eta_dev, double* phis_dev, double dt, double g, int linear,
                         int strategy, double tol, sem_stats* stats, void* stream);

/* One V-cycle (Algorithm 1, zero initial guess on every level): z = M^{-1} r on
 * the finest level.  Dirichlet entries of r are ignored; those of z are 0. */
sem_status pmg_vcycle(sem_handle* h, const double* r_dev, double* z_dev, void* stream);

/* Solve for phi on the finest level.  dirichlet_eta_dev: phi~ at the Dirichlet
 * nodes (order of sem_dirichlet_nodes); rhs_dev: optional load vector added to
 * the free rows (NULL = 0, the Laplace problem); tol: rtol (atol from options;
 * tol <= 0 uses the options' rtol).  phi_dev receives phi on all nodes
 * (phi = phi~ on Dirichlet nodes).  Synchronises the stream once per outer
 * iteration to read the residual norm.  Returns SEM_NOT_CONVERGED with the last
 * iterate when imax is reached.  stats may be NULL. */
sem_status laplace_solve(sem_handle* h, const double* rhs_dev, const double* dirichlet_eta_dev,
                         double tol, double* phi_dev, sem_stats* stats, void* stream);

/* As laplace_solve, with host buffers: copies dirichlet_eta (and rhs) to the
 * device, solves, copies phi back; the copies are inside the timed call.
 * Synchronous. */
sem_status laplace_solve_host(sem_handle* h, const double* rhs_host, const double* dirichlet_eta_host,
                              double tol, double* phi_host, sem_stats* stats, void* stream);

/* Per-element correction network of the learned smoothing sweep (needs a handle set up
 * with smoother = SEM_SMOOTH_LEARNED).  y = W2 relu(W1 x + b1) + b2 with x, y of
 * length Np (nodes of a finest-level element) and hidden width H = mlp_hidden;
 * W1 [H][Np], b1 [H], W2 [Np][H], b2 [Np] row-major FP32 host arrays.  The
 * GEMMs use BF16 copies of W1 and W2 with FP32 activations and accumulation.
 * Network inputs are element residuals scaled to unit norm (Jacobi-scaled:
 * x_e = z_e / ||z_e||, z = D^{-1} r); outputs are the element correction in the
 * same scale.  There is no counterpart in the paper, whose smoother is the
 * element-block Schwarz method (Eq. Mass); the network learns such a local map. */
sem_status sem_mlp_get_weights(const sem_handle* h, float* W1, float* b1, float* W2, float* b2);
sem_status sem_mlp_set_weights(sem_handle* h, const float* W1, const float* b1, const float* W2, const float* b2);
/* Y [B][Np] = network(X [B][Np]) for B <= number of finest elements (device buffers). */
sem_status sem_mlp_forward(sem_handle* h, int B, const float* X_dev, float* Y_dev, void* stream);
/* Mean squared error L = sum_b ||y_b - t_b||^2 / B and its gradients (host arrays shaped
 * like the weights), for B <= number of finest elements; synchronous. */
sem_status sem_mlp_gradient(sem_handle* h, int B, const float* X_dev, const float* T_dev, double* loss_host,
                            float* dW1, float* db1, float* dW2, float* db2, void* stream);
/* One Adam step (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) of the
 * network's FP32 master weights with caller-supplied gradients (host arrays shaped like
 * the weights), the kernel sem_learned_train uses after each gradient; the BF16 copies
 * are refreshed.  reset = 1 zeroes the moments and the step count first.  Synchronous. */
sem_status sem_mlp_adam(sem_handle* h, const float* dW1, const float* db1, const float* dW2, const float* db2,
                        double lr, int reset, void* stream);
/* One learned sweep on the finest level, as it runs inside the FP32 V-cycle (the
 * analogue of the weighted Schwarz correction of Section 4.3, Eqs. Mass and weights):
 * r = f - A u, z = D^{-1} r, per element s_e = ||z_e||, delta = W sum_e Q_e^T s_e
 * MLP(z_e / s_e) (W: inverse node multiplicity), alpha = (r, A delta) / ||A delta||^2;
 * u <- u + alpha delta when alpha > 0 and ||r - alpha A delta|| < learned_tau ||r||,
 * otherwise the Chebyshev sweep it replaces.  f, u: FP32 device vectors of the finest
 * level with zero Dirichlet entries; u is updated in place.  *accepted and *alpha
 * (host, may be NULL) receive the verdict and the step (0 when rejected).  Synchronous. */
sem_status sem_learned_sweep(sem_handle* h, const float* f_dev, float* u_dev, int* accepted_host,
                             double* alpha_host, void* stream);
/* Train the network with Adam (learning rate lr) on residual/error pairs that the plain
 * solver generates: for each of `snapshots` seeded random errors e0 (SplitMix64 of
 * (seed, snapshot, node)), the plain FP32 V-cycle iteration for A u = A e0 from u = 0
 * runs `steps` times; at every iterate its error e = e0 - u is taken to the point where
 * the replaced sweep acts, after the V-cycle's coarse-grid correction
 * (e_post = e - P A_c^{-1} R A e), and (A e_post, e_post) is one pair, every finest
 * element of which is a training sample.  Nothing is stored: each pair is one Adam
 * step.  loss_first / loss_last (host, may be NULL) receive the loss on one held-out
 * pair (a separately seeded error after 3 plain V-cycles) before and after training.
 * Synchronous. */
sem_status sem_learned_train(sem_handle* h, int snapshots, int steps, double lr, unsigned long long seed,
                             double* loss_first, double* loss_last, void* stream);

/* Jacobi-preconditioned FP64 CG on a caller-supplied CSR matrix that allocates no
 * memory at all.  The paper has no counterpart: this is a variant of the
 * library's coarse-level CG for callers that cannot call cudaMalloc - code whose
 * device memory is owned by another framework's pool allocator, code running in
 * a time-critical loop that cannot absorb the device-wide synchronisation of an
 * allocation, or plug-ins given only fixed buffers - and that have no sem_setup
 * handle.  The caller passes every input and output (device pointers): rowptr
 * [n+1], col and vals [nnz] of an SPD matrix (rows with no entries are treated
 * as excluded: give them dinv = 0 and b = 0), dinv [n] (inverse diagonal), b [n];
 * x [n] receives the solution.  The CG's work vectors, reduction partials and
 * barrier state live in one static device array of the library sized for
 * n <= 131072 rows (about 4.2 MB, held on every GPU that loads the library until
 * the process exits); larger n returns SEM_EINVAL.  The first call on a device
 * looks up that array's device address (with the device current), so make one
 * call before capturing any stream.  All calls share the array: calls that
 * overlap on the GPU race.  Synchronous (it copies its status words to the host
 * and waits for `stream`): stops at ||r|| <= rtol ||b|| (SEM_OK) or after imax
 * iterations (SEM_NOT_CONVERGED, x holds the last iterate); *iters_host (may be
 * NULL) receives the iteration count; SEM_NAN if the residual is not finite (a
 * non-finite value in b, vals or dinv); SEM_TIMEOUT if a grid-barrier wait ran out. */
sem_status sem_cg_csr_noalloc(long long n, const int* rowptr, const int* col, const double* vals,
                              const double* dinv, const double* b, double* x, double rtol, int imax,
                              int* iters_host, void* stream);

/* Measured FP64 rate of the current device in TFLOP/s: sixteen independent FMA chains per
 * thread on every SM, timed with CUDA events.  The paper has no counterpart: it is the
 * denominator of the FP64 operator apply's roofline (the FP64 pipe, not HBM, bounds that
 * kernel on this device).  Synchronous; about 10 ms. */
sem_status sem_fp64_rate(double* tflops_host);

/* Solve n independent problems (tanks), each set up by its own sem_setup with
 * batch = 1 and inner_imax = 0 (Section 4.1-4.4 per tank, Algorithm 2 outer iteration:
 * u <- u + M^{-1} r with the handle's V-cycle in its precision, FP64 residual).
 * batch_mode 0 of hs[0] (default): the whole batch is one instantiated CUDA graph, one
 * branch per tank, each a WHILE conditional node around one iteration whose last kernel
 * tests ||r|| <= rtol ||f|| + atol and the iteration limit on the device; one graph
 * launch and one host synchronisation per call.  The graph is built on the first call
 * and reused while the list of handles and the tolerances are the same (it is owned by
 * hs[0]).  If it cannot be built, or with batch_mode 1: host-stepped lockstep, every
 * tank's iteration captured into its own graph, one graph launch per active tank and
 * one host synchronisation per iteration.  dirichlet_eta[t] / phi[t]: device arrays of
 * tank t as in laplace_solve; a handle may appear once.  stats: n entries or NULL.
 * Ordered after prior work on `stream`; synchronous.  Returns the worst tank status. */
sem_status laplace_solve_batch(sem_handle* const* hs, int n, const double* const* dirichlet_eta_dev, double tol,
                               double* const* phi_dev, sem_stats* stats, void* stream);

/* Thread-local message of the last error ("" if none). */
const char* sem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SEM_GB300_H */
