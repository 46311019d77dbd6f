// Internal declarations shared by the translation units of the mstopo library.
// Layouts: nodal vectors [nely+1][nelx+1][2] (x fastest, components interleaved), element
// fields [nely][nelx].  Everything runs on the handle's stream.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/mstopo.h"

#define MSTOPO_MAX_SYS 4      // realisations solved together with one preconditioner
#define MSTOPO_MAX_EIG 16     // eigenvectors kept per agglomerate
#define MSTOPO_RED_BLOCKS 304 // CTAs of the fused reduction kernels (2 per SM of a GB300)

// Every kernel launch of the library is counted (process-wide), see mstopo_get_stats.
extern std::atomic<long long> g_launch_count;
inline void note_launch() { g_launch_count.fetch_add(1, std::memory_order_relaxed); }

// Optional per-kernel device timing with CUDA events on the launching stream.
enum { PROF_PATCH = 0, PROF_MATVEC32 = 1, PROF_MATVEC64 = 2, PROF_COARSE = 3, PROF_N = 4 };
struct Prof {
  int on = 0;
  struct Pend { int which; cudaEvent_t a, b; };
  std::vector<cudaEvent_t> pool;
  std::vector<Pend> pend;
  double ms[PROF_N] = {0, 0, 0, 0};
  long long n[PROF_N] = {0, 0, 0, 0};
};
cudaEvent_t prof_begin(Prof& p, cudaStream_t s);
void prof_end(Prof& p, int which, cudaEvent_t a, cudaStream_t s);
void prof_collect(Prof& p);   // after a stream synchronisation
void prof_free(Prof& p);

// ---------------------------------------------------------------------------------------
// Element stiffness of a unit square, unit E, plane stress, derived in closed form
// (host, FP64).  Local node order (0,0),(1,0),(1,1),(0,1); DOF 2a = x, 2a+1 = y.
void element_stiffness_closed_form(double nu, double K0[64]);

// Coefficients of the node-centred matvec: for each of the four elements around a node
// (LL, LR, UL, UR) the 2x2 blocks coupling the node to the element's three other nodes.
template <typename T>
struct StencilCoef {
  T c[4][3][4];   // [element][other node][row-major 2x2 block]
};
void make_stencil(const double K0[64], StencilCoef<double>& cd, StencilCoef<float>& cf);

// ---------------------------------------------------------------------------------------
// Kernel launchers (each returns the launch status).
// mask_input: read Dirichlet entries of u as zero (false when u is known to be zero there)
cudaError_t launch_matvec_f32(const float* u, float* y, const float* E, const uint8_t* nmask,
                              int nelx, int nely, const StencilCoef<float>& c, int nsys,
                              long long vec_stride, long long e_stride, cudaStream_t s,
                              bool mask_input = true);
cudaError_t launch_matvec_f64(const double* u, double* y, const double* E, const uint8_t* nmask,
                              int nelx, int nely, const StencilCoef<double>& c, int nsys,
                              long long vec_stride, long long e_stride, cudaStream_t s,
                              bool mask_input = true);

// design chain
cudaError_t launch_filter(const double* rho, double* rho_tilde, double* wsum, int dx, int dy,
                          double rmin, int periodic, cudaStream_t s);
cudaError_t launch_project(const double* rho_tilde, double* rbar, double* drbar, int n,
                           const double* etas, int n_eta, double beta, cudaStream_t s);
cudaError_t launch_simp(const double* rbar, double* E64, float* E32, int nelx, int nely,
                        int dx, int dy, int periodic, int n_eta, int n_design,
                        double E0, double Emin, double penal, cudaStream_t s);
cudaError_t launch_sensitivity(const double* u, long long u_stride, const double* rbar,
                               const double* drbar, int n_eta, const double* w, int nelx,
                               int nely, int dx, int dy, int periodic, int n_design,
                               double dE, double penal, const double* K0, double* g_fine,
                               cudaStream_t s);
cudaError_t launch_tile_sum(const double* g_fine, double* g_design, int nelx, int nely,
                            int dx, int dy, cudaStream_t s);
cudaError_t launch_filter_T(const double* g, const double* wsum, double* out, int dx, int dy,
                            double rmin, int periodic, cudaStream_t s);
cudaError_t launch_check_finite(const double* x, long long n, int* flag, cudaStream_t s);

// Krylov / vector kernels (deterministic two-stage reductions)
cudaError_t launch_dot_partials(const double* a, const double* b, long long n, int nsys,
                                long long stride, double* partials, cudaStream_t s);
cudaError_t launch_dot_partials_f32(const float* a, const float* b, long long n, int nsys,
                                    long long stride, double* partials, cudaStream_t s);
cudaError_t launch_dot_partials_mix(const float* a, const double* b, long long n, int nsys,
                                    long long stride, double* partials, cudaStream_t s);
cudaError_t launch_finish_sum(const double* partials, int nsys, double* out, cudaStream_t s);

// generic precision helpers
cudaError_t launch_convert_d2f(const double* a, float* b, long long n, cudaStream_t s);
cudaError_t launch_convert_f2d(const float* a, double* b, long long n, cudaStream_t s);
cudaError_t launch_mask_copy(const double* a, double* b, const uint8_t* nmask, long long n_nodes,
                             int nsys, long long stride, cudaStream_t s);

// ---------------------------------------------------------------------------------------
// Flexible CG driver state (krylov.cu)
struct FcgScalars {            // per system, on the device
  double rr;                   // ||r||^2
  double ff;                   // ||f||^2
  double pq, pr, zq;           // p^T q, p^T r, z^T q_prev
  double pq_prev;              // previous p^T q
  double alpha, beta;
  int active;                  // 1 while iterating
  int status;                  // mstopo_status
  int iters;
  int restart;                 // 1: the next direction is p = z (first step)
  double rr_last;              // ||r||^2 at the last true-residual recomputation
  int done;                    // 1: converged or stopped (device-side loop)
  int repl;                    // true-residual recomputations
};

struct FcgGraph {              // one captured chunk of flexible-CG iterations
  cudaGraphExec_t exec = nullptr;
  int sys0 = -1, nsys = 0;
  long long generation = -1;
  long long launches = 0;
  // the whole iteration loop as one graph (conditional nodes: while not converged, if a true
  // residual is due); launches per loop pass and per true-residual pass
  cudaGraphExec_t loop = nullptr;
  int loop_sys0 = -1, loop_nsys = 0;
  long long loop_generation = -1;
  long long loop_launches = 0, true_launches = 0;
};

// ---------------------------------------------------------------------------------------
// Preconditioner (precond.cu)
// Patch-solve work groups: per realisation k and type t, up to P agglomerates (one
// right-hand-side column each); groups of realisation k are [h_begin[k], h_begin[k+1]).
struct PatchGroups {
  int* d_perm = nullptr;            // [nsv * Nc] agglomerates in group order
  int* d_type = nullptr;            // [n] realisation * T + type
  int* d_first = nullptr;           // [n] first entry of the group in d_perm
  int* d_count = nullptr;           // [n] agglomerates in the group
  int* d_sys = nullptr;             // [n] realisation
  int* d_agg = nullptr;             // [2][nsv][Nc] group and column of each agglomerate
  std::vector<int> h_begin;         // [nsv + 1]
  int n = 0, P = 1;
};

struct Precond {
  int H = 0, NA = 0, NP = 0, nbA = 0, nbP = 0, ncx = 0, ncy = 0, Nc = 0, kmax = 0;
  int n_types = 0, Nt = 0;
  int built = 0;
  double local_shift = 0.0;
  std::vector<int> h_type_of_agg, h_rep_agg, h_kept, h_coff;   // host copies
  int* d_type_of_agg = nullptr;     // [Nc]
  int* d_kept = nullptr;            // [n_types]
  int* d_coff = nullptr;            // [Nc+1] coarse-unknown offsets
  // patch-solve work groups: [0] FP32 on the CUDA cores, [1] FP32 on the tensor cores
  // (TW_M patches per group), [2] FP64 (at most 4 patches per group)
  PatchGroups pg[3];
  int nsv = 0;                      // realisations with their own operators
  // per-system patch matrices: block tridiagonal by node rows of the (2H+1)^2 agglomerate
  // box, artificial-boundary nodes Dirichlet
  uint8_t* d_pfree = nullptr;       // [T][NP*nbP] free DOFs of the patch box
  // patch solves on the CUDA cores (csrc/patch_tri.cu): per patch system the packed blocks of
  // the two-sided elimination (top chain, bottom chain, middle line), FP64 and FP32
  // [T*nsv][patch_tri_system_elems]
  double* d_tri64 = nullptr;
  float* d_tri32 = nullptr;
  // tensor-core FP32 patch solves on the two-sided elimination (csrc/patch_twtc.cu): packed
  // blocks [T*nsv][TwGeom::SS bytes] and the middle-line exchange [groups][2][TW_M][nbP]
  unsigned char* d_ptw = nullptr;
  float* d_twu = nullptr;
  int patch_tc = 0;                 // FP32 patch solves on the tensor cores
  int kind = 0;                     // mstopo_preconditioner
  void* d_sgs = nullptr;            // multiplicative SGS: [2][MSTOPO_MAX_SYS][n_dof] doubles of work space
  // per-type eigenpairs: lambda [T][kmax], Psi [T][NA*NA][2][kmax]
  double* d_lambda = nullptr; double* d_psi64 = nullptr; float* d_psi32 = nullptr;
  double* d_eigres = nullptr;       // [T] residual norms
  int* d_eigsweeps = nullptr;       // [T]
  // coarse problem: dense FP64 inverse of K_c [Nt][Nt] (MSTOPO_COARSE_DENSE), or the block
  // factor over coarse lines (MSTOPO_COARSE_BLOCKTRI): Linv, LinvT, W, V [NLc][nbc][nbc]
  int coarse_mode = 0, nbc = 0, NLc = 0, sweep_grid = 0;
  double* d_Kc = nullptr;
  double* d_Kcinv = nullptr;
  double *d_cLinv = nullptr, *d_cLinvT = nullptr, *d_cW = nullptr, *d_cV = nullptr;
  double *d_cy = nullptr, *d_cx = nullptr;   // [NLc][nbc][4] sweep work vectors
  int* d_s2o = nullptr;                      // [NLc*nbc] coarse unknown of each line slot
  unsigned int* d_cbar = nullptr;            // grid-barrier counter of the sweep
  // apply buffers
  double* d_rc = nullptr;           // [MAX_SYS][Nt]
  double* d_uc = nullptr;           // [MAX_SYS][Nt]
  float* d_zp32 = nullptr;          // [MAX_SYS][Nc][NP*NP*2]
  double* d_zp64 = nullptr;
  // workspaces for the build
  double* d_work = nullptr; size_t work_bytes = 0;
  int* d_flag = nullptr;
};

struct Solver {
  long long n = 0;                  // DOFs
  double *x = nullptr, *r = nullptr, *f = nullptr, *tmp = nullptr;    // [MAX_SYS][n] FP64
  double *p64 = nullptr, *q64 = nullptr, *z64 = nullptr;              // FP64 mode
  float *p32 = nullptr, *q32 = nullptr, *z32 = nullptr, *r32 = nullptr; // MIXED mode
  double* partials = nullptr;       // [MAX_SYS][4][RED_BLOCKS]
  FcgScalars* sc = nullptr;         // [MAX_SYS]
  FcgScalars* h_sc = nullptr;       // pinned host mirror
  int* loopstat = nullptr;          // [2] device-side loop passes, true-residual passes
  // a solve in flight (fcg_start .. fcg_finish): its outputs land in pinned host memory
  double* h_comp = nullptr;         // pinned [MAX_SYS] compliances, then [3] ints: loop passes, werr
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int run_sys0 = 0, run_nsys = 0, run_looped = 0, run_pending = 0;
  int run_repl[MSTOPO_MAX_SYS] = {0};
};

// GMRES(m) workspace (gmres.cu), allocated at the first GMRES solve of a handle
struct GmresWork {
  int m = 0;
  long long n = 0;
  double* V = nullptr;              // [m + 1][n] orthonormal basis
  double* Z = nullptr;              // [m][n] preconditioned directions
  double* w = nullptr;              // [n]
  double* small = nullptr;          // H, rotations, g, y, Gram-Schmidt columns, status
  double* partials = nullptr;       // [m + 1][RED_BLOCKS]
  double* h_st = nullptr;           // pinned [4]
};
void gmres_free(GmresWork& g);

struct mstopo_handle {
  mstopo_problem p{};
  int device = 0;                   // CUDA device current at creation
  cudaStream_t s = nullptr;
  int nelx = 0, nely = 0;
  long long n_nodes = 0, n_dof = 0, n_el = 0;
  std::string err;
  double K0[64];
  StencilCoef<double> st64;
  StencilCoef<float> st32;
  double* d_K0 = nullptr;
  uint8_t* d_nmask = nullptr;       // per node: bit0 = x fixed, bit1 = y fixed
  // design
  int design_ready = 0, n_eta = 0, periodic = 0, dx = 0, dy = 0;
  long long n_design = 0;
  double etas[MSTOPO_MAX_SYS] = {0}, beta = 0, rmin = 0;
  double *d_rho = nullptr, *d_rho_tilde = nullptr, *d_wsum = nullptr;
  double *d_rbar = nullptr, *d_drbar = nullptr;
  double* d_E64 = nullptr; float* d_E32 = nullptr;
  double *d_gfine = nullptr, *d_gdesign = nullptr, *d_w = nullptr;
  int* d_flag = nullptr;
  // preconditioner, solver
  Precond pc;
  Solver sv;
  GmresWork gm;
  int pc_ref = -1;
  int u_all_ready = 0;
  double* d_u_all = nullptr;        // [MAX_SYS][n_dof] last all-realisation solution
  double* d_f_all = nullptr;        // load used for it
  double* d_host_stage = nullptr;   // device staging for the host-pointer entry point
  Prof prof;
  cudaStream_t own_stream = nullptr;  // created when the caller passes no stream
  cudaStream_t s_side = nullptr;      // side stream of the preconditioner's coarse chain
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int graphs_enabled = 1;
  int loop_graph_failed = 0;          // the device-side solve loop could not be built: host loop
  long long device_loop_solves = 0;   // solves that ran the device-side loop
  int patch_tc = -1;                  // FP32 patch solves on the tensor cores: -1 by problem size, 0 off, 1 on
  int autotune = 0;                   // MSTOPO_EXEC_AUTOTUNE: time the patch-solve configurations
  // set while mstopo_batch_solve captures this handle's whole solve into one batch graph:
  // fcg_start then builds its device-side loop as nodes of that graph instead of launching
  // its own loop graph
  cudaGraph_t batch_graph = nullptr;
  long long batch_graph_solves = 0;   // batch solves that ran inside one graph launch
  int inject = 0;                     // test injection (mstopo_inject), consumed by its target
  long long builds = 0;               // preconditioner builds (explicit and automatic)
  int base_iters = -1;                // iterations of the first solve after the last build
  int rebuild_pending = 0;            // the update rule asked for a rebuild
  long long pc_generation = 0;        // bumped by every preconditioner build
  FcgGraph fcg_graph;
};

// coarse.cu
cudaError_t coarse_bt_factor(const double* A, const double* B, int nb, int NL, double* Linv,
                             double* LinvT, double* W, double* V, double* S, double* Cw,
                             double* Ld, int* status, cudaStream_t s);
cudaError_t coarse_bt_apply(const double* Linv, const double* LinvT, const double* W,
                            const double* V, const int* s2o, int nb, int NL, int Nt,
                            const double* rc, double* uc, int nsys, double* ywork,
                            double* xwork, unsigned int* bar, int* err, int grid,
                            int stall, cudaStream_t s);
int coarse_sweep_grid();
int coarse_sweep_max_nb(int grid, int nsys);

// precond.cu
mstopo_status precond_build(mstopo_handle* h, int ref, mstopo_build_info* info);
void precond_free(Precond& pc);
// Apply z = M_k^-1 r for realisations k = sys0 .. sys0+nsys-1 (vectors with stride n_dof,
// the first one of realisation sys0).  part: 0 both, 1 coarse, 2 patches.  FP32 variant
// reads/writes float vectors.
cudaError_t precond_apply_f64(mstopo_handle* h, const double* r, double* z, int sys0, int nsys,
                              int part);
cudaError_t precond_apply_f32(mstopo_handle* h, const float* r, float* z, int sys0, int nsys,
                              int part);

// krylov.cu
mstopo_status fcg_solve(mstopo_handle* h, int sys0, int nsys, const double* f, double* u,
                        const double* u0, mstopo_solve_info* infos);
// The same solve in two halves: fcg_start enqueues it on the handle's stream (with the
// device-side loop it returns before the solve ends; the host-driven loop runs to its end),
// fcg_finish waits for the stream and reports.  Every fcg_start is followed by fcg_finish.
mstopo_status fcg_start(mstopo_handle* h, int sys0, int nsys, const double* f, double* u,
                        const double* u0);
mstopo_status fcg_finish(mstopo_handle* h, mstopo_solve_info* infos);
// GMRES(m) of systems sys0 .. sys0 + nsys - 1 from the masked f and x0 in the solver's
// vectors; fills the solver's host scalars (status, iters, rr, ff, repl = cycles) (gmres.cu)
mstopo_status gmres_run(mstopo_handle* h, int sys0, int nsys);
mstopo_status solver_alloc(mstopo_handle* h);
void solver_free(Solver& sv);

// helpers
inline unsigned int cdiv(long long a, long long b) { return (unsigned int)((a + b - 1) / b); }

// Raise a kernel's dynamic shared-memory limit to the most the device allows beside its
// static shared memory, once per kernel (thread-safe).  Launches then pass their own size;
// a per-call limit set by concurrent builds of different sizes would race.
template <auto kernel>
cudaError_t smem_limit_max() {
  static const cudaError_t once = []() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
      return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
  }();
  return once;
}

// patch solves on the CUDA cores from the two-sided block elimination (csrc/patch_tri.cu)
bool patch_tri_assignment_ok(int nb);
// right-hand-side columns of a CUDA-core patch-solve CTA for groups of up to P patches
inline int patch_tri_cols(int P) { return P <= 4 ? 4 : (P <= 8 ? 8 : 16); }
// packed elements per patch system (all blocks of both chains and the middle line)
long long patch_tri_system_elems(int nb, int NL);
// CTAs of the FP32 kernel that fit on one SM for R columns (shared memory)
int patch_tri_ctas_per_sm(int nb, int R);
// Lt: top-down factor [nsys][NL] (Linv_k), Bt: [nsys][NL-1] (A_{k+1,k}); Lr, Br: the same for
// the first NLr lines of the line-reversed system; Lm: [nsys] inverse factor of the middle
// line's two-sided Schur complement.  out64 / out32 may be null.
cudaError_t patch_tri_pack(const double* Lt, const double* Bt, const double* Lr, const double* Br,
                           const double* Lm, int nsys, int nb, int NL, int NLr, double* out64,
                           float* out32, cudaStream_t s);
cudaError_t patch_tri_solve_f32(mstopo_handle* h, const PatchGroups& G, const float* r, int sys0,
                                int nsys, float* Xg);
cudaError_t patch_tri_solve_f64(mstopo_handle* h, const PatchGroups& G, const double* r, int sys0,
                                int nsys, double* Xg);

// tensor-core FP32 patch solves on the two-sided elimination (csrc/patch_twtc.cu): 128
// patches of one type and realisation per cluster of two CTAs.  Per packed block: KS K-steps of
// [TF32 hi tile | lo tile] of the symmetric inverse (npad rows x 8 columns each, core matrices
// of 8 rows x 16 B), then the FP32 couplings: a chain block [C][C^T], the middle block
// [C_0][C_1][C_0^T][C_1^T], each [4 KS nodes][2][6] (zero beyond nb).
struct TwGeom {
  int nb, npad, ks;          // DOFs per line, MMA N (a multiple of 16, >= nb), K-steps of 8
  int tile;                  // bytes of one tile (npad x 8 TF32)
  int cpl;                   // byte offset of the couplings in a block
  int cset;                  // bytes of one coupling set (6 x 8 KS FP32)
  long long LB, LBM, SS;     // bytes of a chain block, of the middle block, of a patch system
};
constexpr int TW_M = 128;    // patches per group of the tensor-core kernel
TwGeom patch_twtc_geometry(int nb, int NL);
// supported line sizes (the kernel is compiled for a few K-step counts) and shared memory
bool patch_twtc_ok(int nb);
// the tensor-core pack from the FP64 CUDA-core pack of the same systems
cudaError_t patch_twtc_pack(const double* tri64, int nsys, int nb, int NL, unsigned char* out,
                            cudaStream_t s);
// X: [group][NL][TW_M][nb] results; U: [group][2][TW_M][nb] exchange of the middle line
cudaError_t patch_twtc_solve(mstopo_handle* h, const PatchGroups& G, const float* r, int sys0,
                             int nsys, float* Xg, float* U);

// the paper's multiplicative SGS two-level preconditioner (csrc/smoother.cu); part 0 = the
// operator, 2 = one symmetric sweep from zero
cudaError_t sgs_apply_f64(mstopo_handle* h, const double* r, double* z, int sys0, int nsys, int part);
cudaError_t sgs_apply_f32(mstopo_handle* h, const float* r, float* z, int sys0, int nsys, int part);
