/*
 * mstopo -- two-level spectral-MsFEM preconditioned CG for SIMP Q4 plane elasticity on one
 * NVIDIA GB300 (sm_103a).  C ABI.
 *
 * Method: Alexandersen & Lazarov, "Robust topology optimisation of microstructural details
 * without length scale separation -- using a spectral coarse basis preconditioner"
 * (arXiv:1411.3923).  Section numbers below refer to that paper.
 *
 * Conventions shared by every entry point
 *  - Mesh: nelx x nely unit-square bilinear (Q4) elements, plane stress, unit thickness.
 *    Node (i, j), i in [0, nelx] along x, j in [0, nely] along y (upwards).
 *  - Nodal vectors (displacements, forces, residuals): double[nely+1][nelx+1][2],
 *    row-major, component 0 = x, 1 = y  ("nodal layout").
 *  - Element fields: double[nely][nelx], row-major, row 0 = bottom row ("element layout").
 *  - Design fields: element layout of the whole mesh, or double[cell_y][cell_x] for a
 *    periodic unit cell that is tiled over the mesh (Sec. 4.1).
 *  - Pointers marked DEVICE must be CUDA device (or managed) memory on the handle's device;
 *    pointers marked HOST are ordinary host memory.  The caller owns every array it passes;
 *    the library never keeps a caller pointer beyond the call.  Inputs are read on the
 *    handle's stream, outputs are complete when the call returns (every call synchronises
 *    the handle's stream before returning, except where stated).
 *  - Every call returns an mstopo_status.  No call aborts, traps or throws; on failure
 *    mstopo_last_error(h) describes the cause.  A handle is not thread-safe.
 *  - Dirichlet DOFs: every displacement and residual the library returns is zero there;
 *    input vectors are read as if their Dirichlet entries were zero.
 */
#ifndef MSTOPO_H
#define MSTOPO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MSTOPO_OK = 0,
  MSTOPO_INVALID_ARG = 1,     /* a size, pointer or parameter is out of range            */
  MSTOPO_OUT_OF_MEMORY = 2,   /* a device allocation failed                               */
  MSTOPO_CUDA_ERROR = 3,      /* a CUDA runtime call or kernel launch failed              */
  MSTOPO_NOT_SPD = 4,         /* a Cholesky pivot or a CG curvature p^T K p was <= 0      */
  MSTOPO_MAX_ITER = 5,        /* the solve stopped at max_iter before reaching tol        */
  MSTOPO_NONFINITE = 6,       /* a NaN or Inf appeared in an input or an iterate          */
  MSTOPO_TIMEOUT = 7,         /* a bounded device-side wait gave up                        */
  MSTOPO_NOT_READY = 8        /* a prerequisite call (set_design / build) has not run      */
} mstopo_status;

typedef enum {
  MSTOPO_FP64 = 0,   /* everything in FP64: matvec, preconditioner, Krylov vectors        */
  MSTOPO_MIXED = 1   /* FP64 flexible CG (x, r, dot products, residual replacement, coarse
                        solve); FP32 matvec, patch solves, restriction and prolongation   */
} mstopo_precision;

typedef enum {
  MSTOPO_COARSE_AUTO = 0,      /* explicit inverse up to 4096 coarse unknowns, sweeps above  */
  MSTOPO_COARSE_DENSE = 1,     /* explicit FP64 inverse of K_c: one GEMV per application     */
  MSTOPO_COARSE_BLOCKTRI = 2   /* FP64 block Cholesky of K_c over lines of coarse nodes, two
                                  block sweeps per application (one cooperative launch); lines
                                  of at most 640 unknowns (coarse nodes per line x n_eig)     */
} mstopo_coarse_solver;

typedef enum {
  MSTOPO_PREC_ADDITIVE = 0,       /* two-level additive Schwarz: spectral coarse solve plus the
                                     overlapping exact patch solves on every agglomerate     */
  MSTOPO_PREC_MULTIPLICATIVE_SGS = 1  /* the paper's own preconditioner (Sec. 2.4.2): one
                                     symmetric Gauss-Seidel sweep, the spectral coarse
                                     correction, a second sweep, applied multiplicatively.
                                     The sweeps visit the nodes in 4 colours, (i mod 2) +
                                     2 (j mod 2), solving each node's 2x2 block; the operator
                                     is symmetric positive definite, so the flexible CG runs
                                     it unchanged. No patch factors are built. */
} mstopo_preconditioner;

/* Kernel of the FP32 patch solves (MIXED).  The tensor-core kernel (H = 8, 16, 32 only) takes
 * up to 128 patches of one type as the rows of each MMA (TF32 high and low parts of both
 * operands); it wins when a launch holds many patches per type.  AUTO compares the two by a
 * measured cost per wave; TENSOR_CORES with another H makes the build fail with INVALID_ARG. */
typedef enum {
  MSTOPO_PATCH_AUTO = 0,           /* the cheaper by the cost model, per build                  */
  MSTOPO_PATCH_CUDA_CORES = 1,     /* FP32 and FP64 patch solves on the CUDA cores              */
  MSTOPO_PATCH_TENSOR_CORES = 2    /* MIXED: FP32 patch solves on the tensor cores              */
} mstopo_patch_kernel;

typedef enum {
  MSTOPO_KRYLOV_FCG = 0,           /* flexible conjugate gradients FCG(1) with reliable updates */
  MSTOPO_KRYLOV_GMRES = 1          /* restarted GMRES(m), right preconditioned and flexible (the
                                      preconditioned directions z_j are kept): the outer method
                                      the paper uses with its multiplicative preconditioner
                                      (Sec. 2.4.2); each restart starts from the true FP64
                                      residual and the solve stops on it, as with FCG */
} mstopo_krylov;

/* mstopo_problem.exec_flags (bits; 0 = defaults) */
#define MSTOPO_EXEC_NO_GRAPHS 1       /* run every flexible-CG iteration as direct launches      */
#define MSTOPO_EXEC_NO_SIDE_STREAM 2  /* run the preconditioner's coarse chain on the main stream
                                         instead of a side stream beside the patch solves        */
#define MSTOPO_EXEC_AUTOTUNE 4        /* with MSTOPO_PATCH_AUTO: the first build of a problem shape
                                         times every FP32 patch-solve configuration (CUDA cores
                                         with 4, 8 and 16 columns per group; the tensor cores
                                         where compiled) and the process keeps the fastest for
                                         that shape; without it a measured cost model chooses.
                                         The chosen kernel fixes the FP32 rounding, so two
                                         processes may differ in the last bits.                */

typedef enum {
  MSTOPO_FIELD_RHO_TILDE = 0,  /* filtered design (design layout)                         */
  MSTOPO_FIELD_RHO_BAR = 1,    /* projected density of one realisation (design layout)    */
  MSTOPO_FIELD_YOUNG = 2       /* SIMP Young's modulus of one realisation (element layout) */
} mstopo_field;

typedef struct mstopo_handle mstopo_handle;

/* Problem description (Sec. 2.1-2.2 and 2.4). */
typedef struct {
  int32_t nelx, nely;        /* elements along x and y; both multiples of H               */
  double nu;                 /* Poisson's ratio, 0 <= nu < 0.5                             */
  double E0, Emin, penal;    /* modified SIMP: E = Emin + (E0 - Emin) rho_bar^penal (Sec. 2.2) */
  const uint8_t* fixed;      /* HOST, nodal layout of uint8: nonzero = Dirichlet DOF (u = 0) */
  int32_t H;                 /* coarse cell edge in elements, 2..32 (Sec. 2.4); agglomerates are 2H x 2H */
  int32_t n_eig;             /* eigenvectors kept per agglomerate (cap when lambda_thresh > 0), 1..16 */
  double lambda_thresh;      /* > 0: keep only eigenvalues below it (Sec. 2.4, lambda_Omega) */
  int32_t precision;         /* mstopo_precision                                           */
  double tol;                /* stop when ||f - K u||_2 / ||f||_2 <= tol (true FP64 residual) */
  int32_t max_iter;          /* flexible-CG iteration cap                                   */
  double local_shift;        /* MIXED only: patch matrices are factorised as K_i + s diag(K_i)
                                (s >= 0, 0 = exact local solves)                            */
  void* stream;              /* cudaStream_t for all work of this handle, NULL = default   */
  int32_t coarse_solver;     /* mstopo_coarse_solver for the coarse problem K_c u_c = r_c  */
  int32_t reuse_preconditioner; /* nonzero: mstopo_set_design keeps the preconditioner last
                                built (on an earlier design, with the same number of
                                realisations) instead of requiring a new build -- the basis
                                re-use of Sec. 5.1-5.2; solves still stop on the true residual */
  double rebuild_ratio;      /* with reuse_preconditioner, > 0: the update rule of Sec. 5.2 --
                                when an all-realisation solve needs more than rebuild_ratio x
                                the iterations of the first solve after the last build, the
                                next all-realisation solve first rebuilds the preconditioner on
                                the design set then (0 = never rebuild automatically) */
  int32_t preconditioner;    /* mstopo_preconditioner                                       */
  int32_t patch_kernel;      /* mstopo_patch_kernel: FP32 patch solves of the additive level */
  int32_t exec_flags;        /* MSTOPO_EXEC_* bits                                           */
  int32_t krylov;            /* mstopo_krylov: the outer Krylov method                       */
  int32_t gmres_restart;     /* GMRES(m) restart length m, 1..200 (0 = 50); GMRES keeps m + 1
                                FP64 basis vectors and m FP64 preconditioned ones per handle */
} mstopo_problem;

typedef struct {
  int32_t n_agglomerates;     /* coarse nodes N_c                                          */
  int32_t n_types;            /* distinct agglomerates after de-duplication (Sec. 2.4.1)    */
  int32_t n_coarse;           /* coarse unknowns N_t                                        */
  int32_t eig_sweeps;         /* largest number of subspace-iteration sweeps over all types */
  double eig_residual;        /* largest ||K psi - lambda D psi||_{D^-1} over kept pairs    */
  float ms_hash, ms_eigen, ms_patch_factor, ms_coarse, ms_total;   /* phase times (events)  */
  int32_t coarse_solver;      /* MSTOPO_COARSE_DENSE or MSTOPO_COARSE_BLOCKTRI, as built   */
  int32_t coarse_line;        /* unknowns per coarse line (block size of K_c)               */
  int32_t coarse_lines;       /* number of coarse lines (blocks of K_c)                     */
  int32_t patch_kernel;       /* FP32 patch solves as built: MSTOPO_PATCH_CUDA_CORES or
                                 MSTOPO_PATCH_TENSOR_CORES (0: no patch solves, SGS)        */
  int32_t patch_groups;       /* their work groups over all realisations (patches of one
                                 type and realisation each; 128 per tensor-core group)      */
  int32_t patch_cols;         /* patches per group: 4, 8, 16 (CUDA cores) or 128            */
  int32_t patch_tuned;        /* 0: cost model, 1: timed in this build (MSTOPO_EXEC_AUTOTUNE),
                                 2: the choice kept from an earlier build of the same shape */
} mstopo_build_info;

typedef struct {
  int32_t status;             /* mstopo_status of this system                              */
  int32_t iterations;         /* flexible-CG iterations                                    */
  int32_t replacements;       /* FP64 residual recomputations                              */
  double rel_residual;        /* final true ||f - K u||_2 / ||f||_2 (FP64)                  */
  double compliance;          /* f^T u (Sec. 2.2)                                           */
  float ms;                   /* device time of the solve (events on the handle's stream)  */
} mstopo_solve_info;

/* Create a handle for one mesh and boundary-condition set; allocates its device workspace.
 * Errors: INVALID_ARG (sizes not multiples of H, H outside 2..32, nelx/H < 2 or nely/H < 2, n_eig
 * outside 1..16, nu outside [0, 0.5), Emin <= 0 or Emin > E0, fixed == NULL, an unknown
 * preconditioner, coarse solver or patch kernel, unknown exec_flags bits),
 * OUT_OF_MEMORY, CUDA_ERROR.  *out is NULL on failure. */
mstopo_status mstopo_create(const mstopo_problem* desc, mstopo_handle** out);
void mstopo_destroy(mstopo_handle* h);
const char* mstopo_last_error(const mstopo_handle* h);
/* Degrees of freedom 2 (nelx+1)(nely+1), and the number of realisations last set. */
int64_t mstopo_num_dofs(const mstopo_handle* h);
int32_t mstopo_num_realisations(const mstopo_handle* h);

/* Design chain (Sec. 4.3, 2.2): density filter of radius rmin (weights max(0, rmin - d),
 * centroid distances in element units, normalised by the in-domain weight sum; periodic
 * wrap-around on the unit cell when cell_x > 0), then one Heaviside projection per
 * threshold eta[k] with sharpness beta, then modified SIMP moduli on the whole mesh.
 * rho: DEVICE, n_design doubles in design layout (n_design = nelx*nely, or cell_x*cell_y
 * with nelx % cell_x == 0 and nely % cell_y == 0).  eta: HOST, n_eta in 1..4 values in (0,1).
 * Errors: INVALID_ARG, NONFINITE (rho has a NaN/Inf), CUDA_ERROR. */
mstopo_status mstopo_set_design(mstopo_handle* h, const double* rho, int64_t n_design,
                                double rmin, double beta, const double* eta, int32_t n_eta,
                                int32_t cell_x, int32_t cell_y);
/* Copy a design-chain field to out (DEVICE; design or element layout, see mstopo_field). */
mstopo_status mstopo_get_field(mstopo_handle* h, int32_t field, int32_t realisation, double* out);

/* Build the two-level preconditioner (Sec. 2.4, 3.2, 5.3) on the moduli of realisation
 * ref (-1 = the dilated one, i.e. the smallest eta): agglomerate de-duplication, local
 * generalised eigenproblems K_w psi = lambda diag(K_w) psi, coarse basis chi_i psi_j,
 * K_c = R_c K R_c^T and its FP64 factor, and the factors of the overlapping patch matrices.
 * info: HOST, may be NULL.  Errors: NOT_READY (no design), NOT_SPD, CUDA_ERROR. */
mstopo_status mstopo_build_preconditioner(mstopo_handle* h, int32_t ref, mstopo_build_info* info);

/* Solve K(E_k) u_k = f for realisation k (or for all realisations when realisation == -1,
 * as one batch sharing the preconditioner, Sec. 5.3) by flexible CG from u0 (or zero).
 * f: DEVICE nodal layout (NULL = the zero load is rejected: INVALID_ARG);
 * u: DEVICE, n_sys nodal vectors back to back (n_sys = 1 or the number of realisations);
 * u0: DEVICE like u, or NULL.  infos: HOST array of n_sys, may be NULL.
 * The solution also stays in the handle for mstopo_compliance_and_sensitivity.
 * Returns the worst status over the systems (MAX_ITER, NOT_SPD, NONFINITE, ...). */
mstopo_status mstopo_solve(mstopo_handle* h, int32_t realisation, const double* f, double* u,
                           const double* u0, mstopo_solve_info* infos);
/* As mstopo_solve, with f, u (and u0) in HOST memory: the copies to and from the device
 * are part of the call. */
mstopo_status mstopo_solve_host(mstopo_handle* h, int32_t realisation, const double* f,
                                double* u, const double* u0, mstopo_solve_info* infos);

/* Batches of independent instances (for example meshes of uneven sizes), each on its own
 * handle and stream, so their kernels overlap on the GPU.  Handles must be distinct and
 * should not share a stream (a shared stream serialises them).  The builds run from up to
 * 16 host threads (a build waits for the GPU between its steps).  The solves run from the
 * calling thread alone, as one CUDA graph launch for the whole batch: every instance's whole
 * solve (its start, its flexible-CG loop as WHILE/IF conditional nodes with device-side
 * convergence tests, its outputs) is captured into one graph as an independent branch, the
 * graph runs once, and the instances are finished in turn (mstopo_stats.batch_graph_solves
 * counts these).  When an instance cannot take part (graphs off, per-kernel profiling on,
 * GMRES, a rebuild pending from the update rule, another device) or a capture step is
 * refused, every instance's solve is enqueued on its own stream instead, then finished in
 * turn.
 * mstopo_batch_build_preconditioner: as mstopo_build_preconditioner(hs[b], ref, infos + b)
 *   for every b; infos: HOST array of n, may be NULL.
 * mstopo_batch_solve: as mstopo_solve(hs[b], -1, f[b], u[b], NULL, infos + 4 b) for every
 *   b (all realisations of every instance); f, u: HOST arrays of n DEVICE pointers;
 *   infos: HOST array of 4 n (instance b's realisations at 4 b), may be NULL.
 * Both return OK, or the status of the first instance (in batch order) that failed; the
 * other instances still complete.  Errors: INVALID_ARG (NULL or repeated handle, n < 1). */
mstopo_status mstopo_batch_build_preconditioner(mstopo_handle* const* hs, int32_t n, int32_t ref,
                                                mstopo_build_info* infos);
mstopo_status mstopo_batch_solve(mstopo_handle* const* hs, int32_t n, const double* const* f,
                                 double* const* u, mstopo_solve_info* infos);

/* Compliances c_k = f^T u_k of the last all-realisation solve, the robust objective
 * mean(c) + kappa std(c) (population std, Sec. 4.4), and its gradient with respect to the
 * design: the self-adjoint element sensitivity -p (E0-Emin) rho_bar^(p-1) u_e^T K0 u_e
 * (Sec. 4.2) chained through the projection, the periodic tiling (sum over copies,
 * Sec. 4.1) and the filter transpose.  c: HOST [n_eta] or NULL; f_robust: HOST or NULL;
 * dfdrho: DEVICE design layout, or NULL.  Errors: NOT_READY (no all-realisation solve). */
mstopo_status mstopo_compliance_and_sensitivity(mstopo_handle* h, double kappa, double* c,
                                                double* f_robust, double* dfdrho);

/* ---- failure injection (tests of the bounded device waits) --------------------------- */
/* MSTOPO_INJECT_SWEEP_STALL: the next preconditioner application that runs the block-
 * tridiagonal coarse sweeps makes their first grid barrier wait for one arrival too many.
 * The barrier's bounded wait gives up (about half a second), the call returns
 * MSTOPO_TIMEOUT, nothing faults or hangs, and the handle stays usable.  Errors:
 * INVALID_ARG (unknown injection). */
#define MSTOPO_INJECT_NONE 0
#define MSTOPO_INJECT_SWEEP_STALL 1
mstopo_status mstopo_inject(mstopo_handle* h, int32_t what);

/* ---- kernel-level entry points (verification and measurement) --------------------- */

/* y = K(E_k) u on the free DOFs, matrix-free element by element (Sec. 2.1), in the given
 * precision (MSTOPO_MIXED = FP32 arithmetic and FP32 vectors).  u, y: DEVICE nodal layout. */
mstopo_status mstopo_apply_K(mstopo_handle* h, int32_t realisation, int32_t precision,
                             const double* u, double* y);
/* Same, on vectors already stored in FP32 (DEVICE, nodal layout, float, 8-byte aligned).
 * No conversions: this is the kernel the MIXED flexible CG runs.  Errors: INVALID_ARG (NULL
 * or misaligned pointer, realisation out of range), NOT_READY. */
mstopo_status mstopo_apply_K_f32(mstopo_handle* h, int32_t realisation, const float* u, float* y);
/* As mstopo_apply_K_f32, and realisation -1 applies every realisation's K to its own vector
 * (n_sys vectors back to back in u and y, one launch, as in the batched solve).
 * flags: MSTOPO_INPUT_MASKED = the caller guarantees u is zero at the Dirichlet DOFs (as the
 * flexible-CG directions are), so the input mask is not read. */
#define MSTOPO_INPUT_MASKED 1
mstopo_status mstopo_apply_K_f32_ex(mstopo_handle* h, int32_t realisation, const float* u, float* y,
                                    int32_t flags);
/* z = M^-1 r with the built two-level preconditioner, in the given precision.
 * Additive (MSTOPO_PREC_ADDITIVE): part 0 = both levels, 1 = coarse only
 * R_c^T K_c^-1 R_c r, 2 = patches only.
 * Multiplicative (MSTOPO_PREC_MULTIPLICATIVE_SGS, Sec. 2.4.2): part 0 = the operator (SGS,
 * coarse correction of the residual, SGS), 1 = coarse only, 2 = one symmetric Gauss-Seidel
 * sweep from zero (the smoother alone).
 * r, z: DEVICE nodal layout, one realisation (realisation 0).  Errors: INVALID_ARG, NOT_READY
 * (no preconditioner built), CUDA_ERROR. */
mstopo_status mstopo_apply_precond(mstopo_handle* h, int32_t precision, int32_t part,
                                   const double* r, double* z);
/* Eigenpairs kept for the agglomerate of coarse node (I, J) (Sec. 2.4):
 * lambda: HOST [n_eig]; psi: HOST [2H+1][2H+1][2][n_eig] on the agglomerate's node box
 * whose lower-left node is ((I-1)H, (J-1)H) (entries outside the mesh are zero);
 * *n_kept: HOST.  The vectors are normalised psi^T diag(K_w) psi = 1. */
mstopo_status mstopo_get_eigenpairs(mstopo_handle* h, int32_t I, int32_t J, double* lambda,
                                    double* psi, int32_t* n_kept);

/* ---- an entry point that allocates nothing (no counterpart in the paper) ------------- */

/* y = K(E) u on the free DOFs with the FP32 matrix-free matvec, exactly the arithmetic of
 * mstopo_apply_K(h, k, MSTOPO_MIXED, u, y), but without a handle and without allocating
 * any device memory.  For callers that cannot call cudaMalloc: code whose device memory is
 * owned by another allocator or a fixed arena, or that must not trigger the device-wide
 * synchronisation cudaMalloc can cause.
 *   u, y:  DEVICE, nodal layout, double;  E: DEVICE, element layout, float (Young's moduli);
 *   fixed: DEVICE, nodal layout of uint8 (nonzero = Dirichlet DOF);  nu: Poisson's ratio;
 *   stream: cudaStream_t or NULL.  The call returns after the stream has been synchronised.
 * Work space: one static device array of about 36 MB that every GPU loading this library
 * holds until the process exits; at most 4,194,304 DOFs (2 (nelx+1)(nely+1) <= 2^22),
 * larger meshes return MSTOPO_INVALID_ARG before any GPU work.  The first call on a device
 * looks the array's address up on that device (make that first call before any stream
 * capture).  All calls share the array: calls that overlap on the GPU race.
 * Errors: INVALID_ARG (null pointer, non-positive size, nu outside [0, 0.5), too many DOFs),
 * CUDA_ERROR. */
mstopo_status mstopo_apply_K_f32_noalloc(const double* u, double* y, const float* E,
                                        const uint8_t* fixed, int32_t nelx, int32_t nely,
                                        double nu, void* stream);

/* ---- PDE (Helmholtz) density filter with collapsed degrees of freedom (Sec. 4.3, 4.5) --- */

/* The filter of designs made of several microstructure blocks: on the filter mesh (unit Q4
 * elements, cells of nx x ny[c] elements stacked along y, each cell with its own nodes)
 *   -r^2 lap(phi) + phi = rho,  r = rmin / (2 sqrt(3)),  natural boundary conditions,
 *   rho_tilde_e = mean of phi over the element's four nodes,
 * where identified nodes share one unknown (periodicity and connectivity).  The operator
 * rho -> rho_tilde is symmetric: the sensitivity chain applies it unchanged.  Solved by
 * Jacobi-preconditioned CG in FP64 on the collapsed unknowns, matrix-free. */
typedef enum {
  MSTOPO_PDE_PLAIN = 0,           /* one cell, no identification (Neumann on the whole boundary) */
  MSTOPO_PDE_PERIODIC_CELL = 1,   /* one cell, left = right and bottom = top edges (a torus)     */
  MSTOPO_PDE_STACKED_BLOCKS = 2   /* n_cells cells of width nx stacked along y: each cell's left
                                     and right edges identified, and the bottom and top edges of
                                     all cells one set (periodic within each block, connected
                                     across the interfaces) */
} mstopo_pde_domain;

typedef struct {
  int32_t domain;            /* mstopo_pde_domain                                           */
  int32_t nx;                /* elements along x of every cell, >= 1                        */
  int32_t n_cells;           /* cells (1 unless MSTOPO_PDE_STACKED_BLOCKS)                  */
  const int32_t* ny;         /* HOST [n_cells]: elements along y of each cell, >= 1         */
  double rmin;               /* filter radius in elements, > 0                               */
  double tol;                /* CG stop: ||b - K phi|| <= tol ||b|| (0 = 1e-12)             */
  int32_t max_iter;          /* CG iteration cap (0 = 1000)                                  */
  void* stream;              /* cudaStream_t for all work of the filter, NULL = default      */
} mstopo_pde_desc;

typedef struct mstopo_pde_filter mstopo_pde_filter;

/* Builds the collapse map and the CG workspace (device memory owned by the filter).
 * Errors: INVALID_ARG (bad description; the message is mstopo_pde_filter_last_error(NULL)),
 * OUT_OF_MEMORY, CUDA_ERROR. */
mstopo_status mstopo_pde_filter_create(const mstopo_pde_desc* d, mstopo_pde_filter** out);
/* rho_tilde = filter(rho).  rho, rho_tilde: DEVICE [n_elements] FP64, elements cell by cell,
 * row by row (x fastest).  iterations, rel_residual: HOST, may be NULL.  Synchronises the
 * filter's stream.  Errors: INVALID_ARG (null pointer), MAX_ITER, NONFINITE, CUDA_ERROR. */
mstopo_status mstopo_pde_filter_apply(mstopo_pde_filter* f, const double* rho, double* rho_tilde,
                                      int32_t* iterations, double* rel_residual);
int64_t mstopo_pde_filter_num_elements(const mstopo_pde_filter* f);
int64_t mstopo_pde_filter_num_unknowns(const mstopo_pde_filter* f);   /* after collapsing */
const char* mstopo_pde_filter_last_error(const mstopo_pde_filter* f);
void mstopo_pde_filter_destroy(mstopo_pde_filter* f);

/* ---- the design loop (Sec. 4.4, 4.5) ------------------------------------------------- */

/* The expected-volume constraint of the robust problem (Sec. 4.4) at the current design:
 * g = E[vol(rho_bar)] / volfrac - 1 (the mean of rho_bar over the realisations and the
 * design elements; a periodic cell stands for each of its tiles equally) and its gradient
 * with respect to the design, through the projection and the filter transpose.
 * g: HOST, may be NULL; dgdrho: DEVICE [n_design], may be NULL.  Synchronises the stream.
 * Errors: NOT_READY (no design), INVALID_ARG (volfrac outside (0, 1]), CUDA_ERROR. */
mstopo_status mstopo_volume(mstopo_handle* h, double volfrac, double* g, double* dgdrho);

/* The method of moving asymptotes (Svanberg 1987) for one inequality constraint
 * g(x) <= 0 on xmin <= x <= xmax: asymptotes at x -/+ s0 (xmax - xmin) in the first two
 * steps, then moved by 0.7 / 1.2 where x oscillates / moves monotonically, and the convex
 * separable subproblem solved through its one-dimensional dual.  The object keeps the
 * asymptotes and the last two iterates (device memory it owns). */
typedef struct mstopo_mma mstopo_mma;
mstopo_status mstopo_mma_create(int64_t n, double xmin, double xmax, double s0, void* stream,
                                mstopo_mma** out);
/* One step from x with the objective f0, its gradient df0, the constraint value g and its
 * gradient dg: xnew.  x, df0, dg, xnew: DEVICE [n] FP64 (xnew must not alias x).  lam: HOST,
 * the constraint's multiplier, may be NULL.  Synchronises the stream.  Errors: INVALID_ARG,
 * NONFINITE (f0 or g), CUDA_ERROR. */
mstopo_status mstopo_mma_step(mstopo_mma* m, const double* x, double f0, const double* df0,
                              double g, const double* dg, double* xnew, double* lam);
const char* mstopo_mma_last_error(const mstopo_mma* m);
void mstopo_mma_destroy(mstopo_mma* m);

typedef struct {
  double penal;              /* SIMP exponent of this stage, >= 1                            */
  double beta;               /* projection sharpness of this stage, > 0                      */
  int32_t max_iter;          /* design iterations of this stage, >= 1                        */
} mstopo_opt_stage;

typedef struct {
  int32_t stage, iteration;
  double penal, beta;
  double f;                  /* robust objective E[c] + kappa std(c)                         */
  double g;                  /* volume constraint value                                     */
  double c[4];               /* compliance of every realisation                             */
  int32_t solve_iterations;  /* the largest Krylov iteration count of the state solves      */
} mstopo_opt_record;

/* Robust compliance minimisation (Sec. 4.4) with the continuation schedule of Sec. 4.5.
 * Every stage starts new asymptotes (s0 = 0.5 / (1 + beta)); each iteration sets the design
 * (the filter radius, thresholds and cell of the last mstopo_set_design, the stage's beta and
 * penal), builds the preconditioner unless it is reused, solves all realisations for the load
 * f (DEVICE [n_dof]), forms the objective, its gradient and the volume constraint, and takes
 * one MMA step; a stage ends after max_iter iterations or when the objective changes by at
 * most rel_change (relative) between two iterations.  rho: DEVICE [n_design], the start design
 * in, the final one out.  records: HOST [capacity] history (one per iteration), may be NULL
 * with capacity 0; n_records: HOST, the iterations made.  The handle keeps the last stage's
 * penal.  Errors: INVALID_ARG, NOT_READY (no design set before), and those of the steps. */
mstopo_status mstopo_optimise(mstopo_handle* h, double* rho, const double* f,
                              const mstopo_opt_stage* stages, int32_t n_stages, double volfrac,
                              double kappa, double rel_change, mstopo_opt_record* records,
                              int32_t capacity, int32_t* n_records);

/* Robust verification (Sec. 4.4): the compliance of one design under n thresholds (for
 * example uniformly spaced in [0.3, 0.7]), each an independent realisation.  The thresholds
 * run in batches of up to 4 realisations (one set_design, build and solve each) with the
 * filter radius, beta and cell of the last mstopo_set_design.  rho: DEVICE [n_design];
 * f: DEVICE [n_dof]; etas: HOST [n], each in (0, 1); c: HOST [n].  The handle is left with
 * the last batch as its design.  Errors: INVALID_ARG, NOT_READY, and those of the steps. */
mstopo_status mstopo_robust_verification(mstopo_handle* h, const double* rho, const double* f,
                                         const double* etas, int32_t n, double* c);

/* ---- measurement (not part of the paper's method) ----------------------------------- */

typedef struct {
  int64_t launches;            /* kernels launched by this library in this process so far    */
  int64_t kernel_launches[4];  /* profiled launches: [0] patch solves, [1] FP32 matvec,         */
  double kernel_ms[4];         /* [2] FP64 matvec, [3] coarse solve; device ms summed (events) */
  int64_t builds;              /* preconditioner builds of this handle (explicit + automatic) */
  int32_t base_iterations;     /* iterations of the first solve after the last build, or -1  */
  int32_t rebuild_pending;     /* 1: the next all-realisation solve rebuilds first            */
  int64_t device_loop_solves;  /* solves of this handle whose iteration loop ran as one CUDA
                                  graph with device-side convergence tests (the others ran a
                                  host-driven loop: graphs off or per-kernel profiling on) */
  int64_t batch_graph_solves;  /* mstopo_batch_solve calls in which this handle's whole solve
                                  ran inside the batch's single graph launch                  */
} mstopo_stats;

/* Turn per-kernel event timing on (1) or off (0) for this handle; resets its counters.
 * While on, every profiled launch is bracketed by two CUDA events on the handle's stream. */
mstopo_status mstopo_set_profiling(mstopo_handle* h, int32_t on);
/* Counters: out is HOST.  Synchronises the handle's stream. */
mstopo_status mstopo_get_stats(mstopo_handle* h, mstopo_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* MSTOPO_H */
