// C-ABI entry points of the mstopo library (declared in include/mstopo.h).
// Host orchestration only: argument checks, workspace ownership, kernel sequencing on the
// handle's stream.  Every step of the numerical path runs in the kernels of this library.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>

#include "internal.cuh"

#define CKA(x)                                                                  \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      h->err = std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x;      \
      return e_ == cudaErrorMemoryAllocation ? MSTOPO_OUT_OF_MEMORY : MSTOPO_CUDA_ERROR; \
    }                                                                           \
  } while (0)

#define CHECK_ARG(cond, msg)          \
  do {                                \
    if (!(cond)) {                    \
      h->err = msg;                   \
      return MSTOPO_INVALID_ARG;      \
    }                                 \
  } while (0)

static thread_local std::string g_create_error;
std::atomic<long long> g_launch_count{0};

cudaEvent_t prof_begin(Prof& p, cudaStream_t s) {
  cudaEvent_t e = nullptr;
  if (!p.on) return e;
  if (!p.pool.empty()) { e = p.pool.back(); p.pool.pop_back(); }
  else if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  cudaEventRecord(e, s);
  return e;
}

void prof_end(Prof& p, int which, cudaEvent_t a, cudaStream_t s) {
  if (!p.on || !a) return;
  cudaEvent_t b = nullptr;
  if (!p.pool.empty()) { b = p.pool.back(); p.pool.pop_back(); }
  else if (cudaEventCreate(&b) != cudaSuccess) return;
  cudaEventRecord(b, s);
  p.pend.push_back({which, a, b});
}

void prof_collect(Prof& p) {
  for (auto& q : p.pend) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      p.ms[q.which] += ms;
      p.n[q.which] += 1;
    }
    p.pool.push_back(q.a);
    p.pool.push_back(q.b);
  }
  p.pend.clear();
}

void prof_free(Prof& p) {
  for (auto& q : p.pend) { cudaEventDestroy(q.a); cudaEventDestroy(q.b); }
  for (auto e : p.pool) cudaEventDestroy(e);
  p.pend.clear();
  p.pool.clear();
}

extern "C" {

mstopo_status mstopo_create(const mstopo_problem* d, mstopo_handle** out) {
  if (!out) return MSTOPO_INVALID_ARG;
  *out = nullptr;
  if (!d) return MSTOPO_INVALID_ARG;
  mstopo_handle* h = new (std::nothrow) mstopo_handle();
  if (!h) return MSTOPO_OUT_OF_MEMORY;
  auto fail = [&](mstopo_status st) {
    g_create_error = h->err;
    mstopo_destroy(h);
    return st;
  };
  h->p = *d;
  h->p.fixed = nullptr;
  if (cudaGetDevice(&h->device) != cudaSuccess) h->device = 0;
  bool ok = d->nelx > 0 && d->nely > 0 && d->H >= 2 && d->nelx % d->H == 0 && d->nely % d->H == 0 &&
            d->nelx / d->H >= 2 && d->nely / d->H >= 2 && d->n_eig >= 1 && d->n_eig <= MSTOPO_MAX_EIG &&
            d->nu >= 0.0 && d->nu < 0.5 && d->Emin > 0.0 && d->Emin <= d->E0 && d->fixed != nullptr &&
            d->tol > 0.0 && d->max_iter > 0 && d->local_shift >= 0.0 && d->rebuild_ratio >= 0.0 &&
            (d->precision == MSTOPO_FP64 || d->precision == MSTOPO_MIXED) && d->H <= 32 &&
            d->coarse_solver >= MSTOPO_COARSE_AUTO && d->coarse_solver <= MSTOPO_COARSE_BLOCKTRI &&
            (d->preconditioner == MSTOPO_PREC_ADDITIVE ||
             d->preconditioner == MSTOPO_PREC_MULTIPLICATIVE_SGS) &&
            d->patch_kernel >= MSTOPO_PATCH_AUTO && d->patch_kernel <= MSTOPO_PATCH_TENSOR_CORES &&
            (d->exec_flags & ~(MSTOPO_EXEC_NO_GRAPHS | MSTOPO_EXEC_NO_SIDE_STREAM | MSTOPO_EXEC_AUTOTUNE)) == 0 &&
            (d->krylov == MSTOPO_KRYLOV_FCG || d->krylov == MSTOPO_KRYLOV_GMRES) &&
            d->gmres_restart >= 0 && d->gmres_restart <= 200;
  if (!ok) {
    h->err = "invalid problem description";
    return fail(MSTOPO_INVALID_ARG);
  }
  h->s = (cudaStream_t)d->stream;
  if (!h->s) {
    // a blocking stream of our own (it orders with the legacy default stream) so that the
    // flexible-CG chunks can be captured into CUDA graphs
    if (cudaStreamCreate(&h->own_stream) != cudaSuccess) {
      h->err = "could not create a stream";
      return fail(MSTOPO_CUDA_ERROR);
    }
    h->s = h->own_stream;
  }
  // side stream and events of the preconditioner's fork (coarse chain beside the patch solve)
  if (cudaStreamCreateWithFlags(&h->s_side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    h->err = "could not create the side stream";
    return fail(MSTOPO_CUDA_ERROR);
  }
  if (d->exec_flags & MSTOPO_EXEC_NO_GRAPHS) h->graphs_enabled = 0;
  if (d->exec_flags & MSTOPO_EXEC_AUTOTUNE) h->autotune = 1;
  h->patch_tc = d->patch_kernel == MSTOPO_PATCH_AUTO ? -1 : (d->patch_kernel == MSTOPO_PATCH_TENSOR_CORES ? 1 : 0);
  if (d->exec_flags & MSTOPO_EXEC_NO_SIDE_STREAM) {
    cudaStreamDestroy(h->s_side);
    h->s_side = nullptr;
  }
  h->nelx = d->nelx;
  h->nely = d->nely;
  h->n_nodes = ((long long)d->nelx + 1) * ((long long)d->nely + 1);
  if (h->n_nodes > (1LL << 30)) {   // index arithmetic of the kernels stays in range
    h->err = "mesh too large (more than 2^30 nodes)";
    return fail(MSTOPO_INVALID_ARG);
  }
  h->n_dof = 2 * h->n_nodes;
  h->n_el = (long long)d->nelx * d->nely;
  element_stiffness_closed_form(d->nu, h->K0);
  make_stencil(h->K0, h->st64, h->st32);
  std::vector<uint8_t> nm((size_t)h->n_nodes);
  for (long long i = 0; i < h->n_nodes; ++i)
    nm[i] = (uint8_t)((d->fixed[2 * i] ? 1 : 0) | (d->fixed[2 * i + 1] ? 2 : 0));
  cudaError_t e;
#define CKC(x)                                                       \
  do {                                                               \
    e = (x);                                                         \
    if (e != cudaSuccess) {                                          \
      h->err = std::string("CUDA: ") + cudaGetErrorString(e);        \
      return fail(e == cudaErrorMemoryAllocation ? MSTOPO_OUT_OF_MEMORY : MSTOPO_CUDA_ERROR); \
    }                                                                \
  } while (0)
  CKC(cudaMalloc(&h->d_nmask, h->n_nodes));
  CKC(cudaMemcpy(h->d_nmask, nm.data(), h->n_nodes, cudaMemcpyHostToDevice));
  CKC(cudaMalloc(&h->d_K0, 64 * 8));
  CKC(cudaMemcpy(h->d_K0, h->K0, 64 * 8, cudaMemcpyHostToDevice));
  CKC(cudaMalloc(&h->d_E64, (size_t)MSTOPO_MAX_SYS * h->n_el * 8));
  CKC(cudaMalloc(&h->d_E32, (size_t)MSTOPO_MAX_SYS * h->n_el * 4));
  CKC(cudaMalloc(&h->d_gfine, (size_t)h->n_el * 8));
  CKC(cudaMalloc(&h->d_flag, 16));
  CKC(cudaMalloc(&h->d_u_all, (size_t)MSTOPO_MAX_SYS * h->n_dof * 8));
  CKC(cudaMalloc(&h->d_f_all, (size_t)h->n_dof * 8));
#undef CKC
  *out = h;
  return MSTOPO_OK;
}

void mstopo_destroy(mstopo_handle* h) {
  if (!h) return;
  if (h->s) cudaStreamSynchronize(h->s);
  else cudaDeviceSynchronize();
  precond_free(h->pc);
  solver_free(h->sv);
  gmres_free(h->gm);
  prof_free(h->prof);
  if (h->fcg_graph.exec) cudaGraphExecDestroy(h->fcg_graph.exec);
  if (h->fcg_graph.loop) cudaGraphExecDestroy(h->fcg_graph.loop);
  void* ptrs[] = {h->d_K0, h->d_nmask, h->d_rho, h->d_rho_tilde, h->d_wsum, h->d_rbar, h->d_drbar,
                  h->d_E64, h->d_E32, h->d_gfine, h->d_gdesign, h->d_w, h->d_flag, h->d_u_all,
                  h->d_f_all, h->d_host_stage};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->s_side) cudaStreamDestroy(h->s_side);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
}

const char* mstopo_last_error(const mstopo_handle* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

int64_t mstopo_num_dofs(const mstopo_handle* h) { return h ? h->n_dof : 0; }
int32_t mstopo_num_realisations(const mstopo_handle* h) { return h ? h->n_eta : 0; }

mstopo_status mstopo_set_design(mstopo_handle* h, const double* rho, int64_t n_design, double rmin,
                                double beta, const double* eta, int32_t n_eta, int32_t cell_x,
                                int32_t cell_y) {
  if (!h) return MSTOPO_INVALID_ARG;
  CHECK_ARG(rho && eta, "null pointer");
  CHECK_ARG(n_eta >= 1 && n_eta <= MSTOPO_MAX_SYS, "n_eta must be 1..4");
  CHECK_ARG(rmin > 0.0 && rmin < 64.0 && beta > 0.0, "rmin must be in (0, 64) and beta > 0");
  const int periodic = cell_x > 0 ? 1 : 0;
  int dx = h->nelx, dy = h->nely;
  if (periodic) {
    CHECK_ARG(cell_y > 0 && h->nelx % cell_x == 0 && h->nely % cell_y == 0,
              "the unit cell must tile the mesh");
    dx = cell_x;
    dy = cell_y;
  }
  CHECK_ARG(n_design == (int64_t)dx * dy, "n_design does not match the design domain");
  for (int k = 0; k < n_eta; ++k) CHECK_ARG(eta[k] > 0.0 && eta[k] < 1.0, "eta must be in (0,1)");
  if (h->n_design != n_design || !h->d_rho) {
    cudaFree(h->d_rho); cudaFree(h->d_rho_tilde); cudaFree(h->d_wsum); cudaFree(h->d_rbar);
    cudaFree(h->d_drbar); cudaFree(h->d_gdesign);
    CKA(cudaMalloc(&h->d_rho, n_design * 8));
    CKA(cudaMalloc(&h->d_rho_tilde, n_design * 8));
    CKA(cudaMalloc(&h->d_wsum, n_design * 8));
    CKA(cudaMalloc(&h->d_rbar, (size_t)MSTOPO_MAX_SYS * n_design * 8));
    CKA(cudaMalloc(&h->d_drbar, (size_t)MSTOPO_MAX_SYS * n_design * 8));
    CKA(cudaMalloc(&h->d_gdesign, n_design * 8));
  }
  h->n_design = n_design;
  h->periodic = periodic;
  h->dx = dx;
  h->dy = dy;
  h->n_eta = n_eta;
  h->beta = beta;
  h->rmin = rmin;
  for (int k = 0; k < n_eta; ++k) h->etas[k] = eta[k];
  CKA(cudaMemcpyAsync(h->d_rho, rho, n_design * 8, cudaMemcpyDeviceToDevice, h->s));
  CKA(cudaMemsetAsync(h->d_flag, 0, 4, h->s));
  CKA(launch_check_finite(h->d_rho, n_design, h->d_flag, h->s));
  CKA(launch_filter(h->d_rho, h->d_rho_tilde, h->d_wsum, dx, dy, rmin, periodic, h->s));
  CKA(launch_project(h->d_rho_tilde, h->d_rbar, h->d_drbar, (int)n_design, eta, n_eta, beta, h->s));
  CKA(launch_simp(h->d_rbar, h->d_E64, h->d_E32, h->nelx, h->nely, dx, dy, periodic, n_eta,
                  (int)n_design, h->p.E0, h->p.Emin, h->p.penal, h->s));
  int flag = 0;
  CKA(cudaMemcpyAsync(&flag, h->d_flag, 4, cudaMemcpyDeviceToHost, h->s));
  CKA(cudaStreamSynchronize(h->s));
  h->design_ready = flag ? 0 : 1;
  h->u_all_ready = 0;
  if (!(h->p.reuse_preconditioner && h->pc.built && h->pc.nsv == n_eta && !flag)) h->pc.built = 0;
  if (flag) {
    h->err = "design contains NaN or Inf";
    return MSTOPO_NONFINITE;
  }
  return MSTOPO_OK;
}

mstopo_status mstopo_get_field(mstopo_handle* h, int32_t field, int32_t realisation, double* out) {
  if (!h) return MSTOPO_INVALID_ARG;
  if (!h->design_ready) { h->err = "no design set"; return MSTOPO_NOT_READY; }
  CHECK_ARG(out, "null pointer");
  CHECK_ARG(realisation >= 0 && realisation < h->n_eta, "realisation out of range");
  const double* src = nullptr;
  size_t n = 0;
  if (field == MSTOPO_FIELD_RHO_TILDE) { src = h->d_rho_tilde; n = h->n_design; }
  else if (field == MSTOPO_FIELD_RHO_BAR) { src = h->d_rbar + realisation * h->n_design; n = h->n_design; }
  else if (field == MSTOPO_FIELD_YOUNG) { src = h->d_E64 + realisation * h->n_el; n = h->n_el; }
  else CHECK_ARG(false, "unknown field");
  CKA(cudaMemcpyAsync(out, src, n * 8, cudaMemcpyDeviceToDevice, h->s));
  CKA(cudaStreamSynchronize(h->s));
  return MSTOPO_OK;
}

mstopo_status mstopo_build_preconditioner(mstopo_handle* h, int32_t ref, mstopo_build_info* info) {
  if (!h) return MSTOPO_INVALID_ARG;
  if (!h->design_ready) { h->err = "no design set"; return MSTOPO_NOT_READY; }
  if (ref < 0) {
    ref = 0;
    for (int k = 1; k < h->n_eta; ++k) if (h->etas[k] < h->etas[ref]) ref = k;
  }
  CHECK_ARG(ref < h->n_eta, "reference realisation out of range");
  h->pc_ref = ref;
  h->pc_generation++;
  h->builds++;
  h->base_iters = -1;
  h->rebuild_pending = 0;
  mstopo_status st = precond_build(h, ref, info);
  if (st != MSTOPO_OK) h->pc.built = 0;
  return st;
}

}  // extern "C"

// mstopo_solve in two halves (see fcg_start / fcg_finish): the start validates, applies the
// basis update rule, enqueues the solve and the copies for mstopo_compliance_and_sensitivity;
// the finish waits and reports.
static mstopo_status solve_start(mstopo_handle* h, int32_t realisation, const double* f, double* u,
                                 const double* u0) {
  if (!h) return MSTOPO_INVALID_ARG;
  if (!h->design_ready || !h->pc.built) { h->err = "design or preconditioner missing"; return MSTOPO_NOT_READY; }
  CHECK_ARG(f && u, "null pointer");
  CHECK_ARG(realisation >= -1 && realisation < h->n_eta, "realisation out of range");
  const int sys0 = realisation < 0 ? 0 : realisation;
  const int nsys = realisation < 0 ? h->n_eta : 1;
  const bool policy = realisation < 0 && h->p.reuse_preconditioner && h->p.rebuild_ratio > 0.0;
  if (policy && h->rebuild_pending) {   // the update rule of Sec. 5.2: new basis for this design
    mstopo_status sb = mstopo_build_preconditioner(h, -1, nullptr);
    if (sb != MSTOPO_OK) return sb;
  }
  if (realisation < 0) h->u_all_ready = 0;
  mstopo_status st = fcg_start(h, sys0, nsys, f, u, u0);
  if (st != MSTOPO_OK) return st;
  if (realisation < 0) {
    CKA(cudaMemcpyAsync(h->d_u_all, u, (size_t)nsys * h->n_dof * 8, cudaMemcpyDeviceToDevice, h->s));
    CKA(cudaMemcpyAsync(h->d_f_all, f, (size_t)h->n_dof * 8, cudaMemcpyDeviceToDevice, h->s));
  }
  return MSTOPO_OK;
}

static mstopo_status solve_finish(mstopo_handle* h, int32_t realisation, mstopo_solve_info* infos) {
  const int nsys = realisation < 0 ? h->n_eta : 1;
  const bool policy = realisation < 0 && h->p.reuse_preconditioner && h->p.rebuild_ratio > 0.0;
  mstopo_solve_info local[MSTOPO_MAX_SYS];
  mstopo_solve_info* inf = infos ? infos : local;
  mstopo_status st = fcg_finish(h, inf);
  if (policy && st == MSTOPO_OK) {
    int it = 0;
    for (int k = 0; k < nsys; ++k) it = std::max(it, (int)inf[k].iterations);
    if (h->base_iters < 0) h->base_iters = it;
    else if (it > h->p.rebuild_ratio * h->base_iters) h->rebuild_pending = 1;
  }
  if (realisation < 0) h->u_all_ready = (st == MSTOPO_OK) ? 1 : 0;
  return st;
}

extern "C" {

mstopo_status mstopo_solve(mstopo_handle* h, int32_t realisation, const double* f, double* u,
                           const double* u0, mstopo_solve_info* infos) {
  mstopo_status st = solve_start(h, realisation, f, u, u0);
  if (st != MSTOPO_OK) return st;
  return solve_finish(h, realisation, infos);
}

mstopo_status mstopo_solve_host(mstopo_handle* h, int32_t realisation, const double* f, double* u,
                                const double* u0, mstopo_solve_info* infos) {
  if (!h) return MSTOPO_INVALID_ARG;
  CHECK_ARG(f && u, "null pointer");
  CHECK_ARG(realisation >= -1 && realisation < h->n_eta, "realisation out of range");
  const int nsys = realisation < 0 ? h->n_eta : 1;
  const size_t nb = (size_t)h->n_dof * 8;
  if (!h->d_host_stage) CKA(cudaMalloc(&h->d_host_stage, (1 + 2 * MSTOPO_MAX_SYS) * nb));
  double* df = h->d_host_stage;
  double* du = df + h->n_dof;
  double* du0 = du + (size_t)MSTOPO_MAX_SYS * h->n_dof;
  CKA(cudaMemcpyAsync(df, f, nb, cudaMemcpyHostToDevice, h->s));
  if (u0) CKA(cudaMemcpyAsync(du0, u0, nsys * nb, cudaMemcpyHostToDevice, h->s));
  mstopo_status st = mstopo_solve(h, realisation, df, du, u0 ? du0 : nullptr, infos);
  CKA(cudaMemcpyAsync(u, du, nsys * nb, cudaMemcpyDeviceToHost, h->s));
  CKA(cudaStreamSynchronize(h->s));
  return st;
}

mstopo_status mstopo_compliance_and_sensitivity(mstopo_handle* h, double kappa, double* c,
                                                double* f_robust, double* dfdrho) {
  if (!h) return MSTOPO_INVALID_ARG;
  if (!h->u_all_ready) { h->err = "no all-realisation solve"; return MSTOPO_NOT_READY; }
  const int n = h->n_eta;
  // c_k = f^T u_k
  double* part = h->sv.partials;
  double* vtmp = part + (size_t)MSTOPO_MAX_SYS * 3 * MSTOPO_RED_BLOCKS;
  for (int k = 0; k < n; ++k) {
    CKA(launch_dot_partials(h->d_f_all, h->d_u_all + (size_t)k * h->n_dof, h->n_dof, 1, 0,
                            part + (size_t)k * MSTOPO_RED_BLOCKS, h->s));
  }
  CKA(launch_finish_sum(part, n, vtmp, h->s));
  double ck[MSTOPO_MAX_SYS];
  CKA(cudaMemcpyAsync(ck, vtmp, n * 8, cudaMemcpyDeviceToHost, h->s));
  CKA(cudaStreamSynchronize(h->s));
  // robust objective mean + kappa * std (population) and weights df/dc_k (Sec. 4.4)
  double mu = 0.0;
  for (int k = 0; k < n; ++k) mu += ck[k];
  mu /= n;
  double var = 0.0;
  for (int k = 0; k < n; ++k) var += (ck[k] - mu) * (ck[k] - mu);
  var /= n;
  const double sigma = std::sqrt(var);
  double w[MSTOPO_MAX_SYS];
  for (int k = 0; k < n; ++k)
    w[k] = 1.0 / n + ((n > 1 && sigma > 1e-300 * std::fmax(std::fabs(mu), 1e-300))
                          ? kappa * (ck[k] - mu) / (n * sigma) : 0.0);
  if (c) for (int k = 0; k < n; ++k) c[k] = ck[k];
  if (f_robust) *f_robust = mu + kappa * sigma;
  if (dfdrho) {
    CKA(launch_sensitivity(h->d_u_all, h->n_dof, h->d_rbar, h->d_drbar, n, w, h->nelx, h->nely,
                           h->dx, h->dy, h->periodic, (int)h->n_design, h->p.E0 - h->p.Emin,
                           h->p.penal, h->K0, h->d_gfine, h->s));
    const double* g = h->d_gfine;
    if (h->periodic) {
      CKA(launch_tile_sum(h->d_gfine, h->d_gdesign, h->nelx, h->nely, h->dx, h->dy, h->s));
      g = h->d_gdesign;
    }
    CKA(launch_filter_T(g, h->d_wsum, dfdrho, h->dx, h->dy, h->rmin, h->periodic, h->s));
    CKA(cudaStreamSynchronize(h->s));
  }
  return MSTOPO_OK;
}

mstopo_status mstopo_apply_K(mstopo_handle* h, int32_t realisation, int32_t precision,
                             const double* u, double* y) {
  if (!h) return MSTOPO_INVALID_ARG;
  if (!h->design_ready) { h->err = "no design set"; return MSTOPO_NOT_READY; }
  CHECK_ARG(u && y, "null pointer");
  CHECK_ARG(realisation >= 0 && realisation < h->n_eta, "realisation out of range");
  const long long n = h->n_dof;
  if (precision == MSTOPO_FP64) {
    CKA(launch_matvec_f64(u, y, h->d_E64 + realisation * h->n_el, h->d_nmask, h->nelx, h->nely,
                          h->st64, 1, n, h->n_el, h->s));
  } else {
    float *a, *b;
    CKA(cudaMallocAsync(&a, n * 4, h->s));
    CKA(cudaMallocAsync(&b, n * 4, h->s));
    CKA(launch_convert_d2f(u, a, n, h->s));
    CKA(launch_matvec_f32(a, b, h->d_E32 + realisation * h->n_el, h->d_nmask, h->nelx, h->nely,
                          h->st32, 1, n, h->n_el, h->s));
    CKA(launch_convert_f2d(b, y, n, h->s));
    CKA(cudaFreeAsync(a, h->s));
    CKA(cudaFreeAsync(b, h->s));
  }
  CKA(cudaStreamSynchronize(h->s));
  return MSTOPO_OK;
}

mstopo_status mstopo_apply_K_f32(mstopo_handle* h, int32_t realisation, const float* u, float* y) {
  return mstopo_apply_K_f32_ex(h, realisation, u, y, 0);
}

mstopo_status mstopo_apply_K_f32_ex(mstopo_handle* h, int32_t realisation, const float* u, float* y,
                                    int32_t flags) {
  if (!h) return MSTOPO_INVALID_ARG;
  if (!h->design_ready) { h->err = "no design set"; return MSTOPO_NOT_READY; }
  CHECK_ARG(u && y, "null pointer");
  CHECK_ARG(realisation >= -1 && realisation < h->n_eta, "realisation out of range");
  CHECK_ARG((flags & ~MSTOPO_INPUT_MASKED) == 0, "unknown flag");
  CHECK_ARG((reinterpret_cast<uintptr_t>(u) & 7) == 0 && (reinterpret_cast<uintptr_t>(y) & 7) == 0,
            "u and y must be 8-byte aligned (float2 nodes)");
  const int sys0 = realisation < 0 ? 0 : realisation;
  const int nsys = realisation < 0 ? h->n_eta : 1;
  cudaEvent_t pa = prof_begin(h->prof, h->s);
  CKA(launch_matvec_f32(u, y, h->d_E32 + sys0 * h->n_el, h->d_nmask, h->nelx, h->nely, h->st32,
                        nsys, h->n_dof, h->n_el, h->s, !(flags & MSTOPO_INPUT_MASKED)));
  prof_end(h->prof, PROF_MATVEC32, pa, h->s);
  CKA(cudaStreamSynchronize(h->s));
  return MSTOPO_OK;
}

mstopo_status mstopo_apply_precond(mstopo_handle* h, int32_t precision, int32_t part,
                                   const double* r, double* z) {
  if (!h) return MSTOPO_INVALID_ARG;
  if (!h->pc.built) { h->err = "preconditioner not built"; return MSTOPO_NOT_READY; }
  CHECK_ARG(r && z, "null pointer");
  CHECK_ARG(part >= 0 && part <= 2, "part must be 0, 1 or 2");
  const long long n = h->n_dof;
  CKA(cudaMemsetAsync(h->d_flag + 1, 0, sizeof(int), h->s));
  double* rm;
  CKA(cudaMallocAsync(&rm, n * 8, h->s));
  CKA(launch_mask_copy(r, rm, h->d_nmask, h->n_nodes, 1, n, h->s));
  if (precision == MSTOPO_FP64) {
    CKA(precond_apply_f64(h, rm, z, 0, 1, part));
  } else {
    float *a, *b;
    CKA(cudaMallocAsync(&a, n * 4, h->s));
    CKA(cudaMallocAsync(&b, n * 4, h->s));
    CKA(launch_convert_d2f(rm, a, n, h->s));
    CKA(precond_apply_f32(h, a, b, 0, 1, part));
    CKA(launch_convert_f2d(b, z, n, h->s));
    CKA(cudaFreeAsync(a, h->s));
    CKA(cudaFreeAsync(b, h->s));
  }
  CKA(cudaFreeAsync(rm, h->s));
  int werr = 0;
  CKA(cudaMemcpyAsync(&werr, h->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CKA(cudaStreamSynchronize(h->s));
  if (werr) { h->err = "bounded device wait gave up"; return MSTOPO_TIMEOUT; }
  return MSTOPO_OK;
}

mstopo_status mstopo_get_eigenpairs(mstopo_handle* h, int32_t I, int32_t J, double* lambda,
                                    double* psi, int32_t* n_kept) {
  if (!h) return MSTOPO_INVALID_ARG;
  if (!h->pc.built) { h->err = "preconditioner not built"; return MSTOPO_NOT_READY; }
  Precond& pc = h->pc;
  CHECK_ARG(I >= 0 && I <= pc.ncx && J >= 0 && J <= pc.ncy, "coarse node out of range");
  const int i = J * (pc.ncx + 1) + I;
  const int t = pc.h_type_of_agg[i];
  const size_t nA = (size_t)pc.NA * pc.NA * 2;
  if (n_kept) *n_kept = pc.h_kept[t];
  if (lambda) CKA(cudaMemcpyAsync(lambda, pc.d_lambda + (size_t)t * MSTOPO_MAX_EIG, pc.kmax * 8,
                                  cudaMemcpyDeviceToHost, h->s));
  if (psi) CKA(cudaMemcpyAsync(psi, pc.d_psi64 + (size_t)t * nA * pc.kmax, nA * pc.kmax * 8,
                               cudaMemcpyDeviceToHost, h->s));
  CKA(cudaStreamSynchronize(h->s));
  return MSTOPO_OK;
}

mstopo_status mstopo_set_profiling(mstopo_handle* h, int32_t on) {
  if (!h) return MSTOPO_INVALID_ARG;
  CKA(cudaStreamSynchronize(h->s));
  prof_collect(h->prof);
  h->prof.on = on ? 1 : 0;
  for (int k = 0; k < PROF_N; ++k) { h->prof.ms[k] = 0.0; h->prof.n[k] = 0; }
  return MSTOPO_OK;
}

mstopo_status mstopo_get_stats(mstopo_handle* h, mstopo_stats* out) {
  if (!h || !out) return MSTOPO_INVALID_ARG;
  CKA(cudaStreamSynchronize(h->s));
  prof_collect(h->prof);
  out->launches = g_launch_count.load();
  out->builds = h->builds;
  out->base_iterations = h->base_iters;
  out->rebuild_pending = h->rebuild_pending;
  out->device_loop_solves = h->device_loop_solves;
  out->batch_graph_solves = h->batch_graph_solves;
  for (int k = 0; k < 4; ++k) {
    out->kernel_launches[k] = h->prof.n[k];
    out->kernel_ms[k] = h->prof.ms[k];
  }
  return MSTOPO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------- batches
// Runs job(b) for b in [0, n) on up to 16 host threads (each bound to the handle's device);
// every handle's work stays on its own stream, so kernels of different instances overlap
// on the GPU.  Falls back to one thread if threads cannot be started.
template <typename Job>
static void run_batch(mstopo_handle* const* hs, int n, Job job) {
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int b; (b = next.fetch_add(1)) < n;) {
      cudaSetDevice(hs[b]->device);
      job(b);
    }
  };
  std::vector<std::thread> pool;
  const int nt = std::min(n, 16);
  try {
    for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  } catch (...) {
  }
  work();
  for (auto& th : pool) th.join();
}

static mstopo_status check_batch(mstopo_handle* const* hs, int32_t n) {
  if (!hs || n < 1) return MSTOPO_INVALID_ARG;
  for (int b = 0; b < n; ++b) {
    if (!hs[b]) return MSTOPO_INVALID_ARG;
    for (int c = 0; c < b; ++c)
      if (hs[c] == hs[b]) {
        hs[b]->err = "a handle appears twice in the batch";
        return MSTOPO_INVALID_ARG;
      }
  }
  return MSTOPO_OK;
}

mstopo_status mstopo_batch_build_preconditioner(mstopo_handle* const* hs, int32_t n, int32_t ref,
                                                mstopo_build_info* infos) {
  mstopo_status st0 = check_batch(hs, n);
  if (st0 != MSTOPO_OK) return st0;
  std::vector<mstopo_status> st(n, MSTOPO_OK);
  run_batch(hs, n, [&](int b) {
    st[b] = mstopo_build_preconditioner(hs[b], ref, infos ? infos + b : nullptr);
  });
  for (int b = 0; b < n; ++b)
    if (st[b] != MSTOPO_OK) return st[b];
  return MSTOPO_OK;
}

mstopo_status mstopo_batch_solve(mstopo_handle* const* hs, int32_t n, const double* const* f,
                                 double* const* u, mstopo_solve_info* infos) {
  mstopo_status st0 = check_batch(hs, n);
  if (st0 != MSTOPO_OK) return st0;
  if (!f || !u) return MSTOPO_INVALID_ARG;
  std::vector<mstopo_status> st(n, MSTOPO_OK);
  // One graph launch for the whole batch: every instance's solve (its start, its device-side
  // flexible-CG loop with WHILE/IF nodes, its outputs) is captured into one graph as an
  // independent branch, and the graph runs once.  It needs every instance on the device-side
  // loop (graphs on, no per-kernel profiling, flexible CG) on one device with its solver
  // workspace allocated; otherwise, or if any capture step is refused, the instances are
  // enqueued one after another below.
  bool one_graph = n > 0;
  for (int b = 0; b < n && one_graph; ++b) {
    mstopo_handle* h = hs[b];
    one_graph = h->graphs_enabled && !h->prof.on && !h->loop_graph_failed &&
                h->p.krylov == MSTOPO_KRYLOV_FCG && h->device == hs[0]->device &&
                h->design_ready && h->pc.built &&
                !(h->p.reuse_preconditioner && h->p.rebuild_ratio > 0.0 && h->rebuild_pending);
  }
  if (one_graph) {
    cudaSetDevice(hs[0]->device);
    for (int b = 0; b < n && one_graph; ++b) one_graph = solver_alloc(hs[b]) == MSTOPO_OK;
  }
  if (one_graph) {
    cudaGraph_t g = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    int captured = 0;
    std::vector<long long> dls(n);
    for (int b = 0; b < n; ++b) dls[b] = hs[b]->device_loop_solves;
    for (int b = 0; b < n && ok; ++b) {
      mstopo_handle* h = hs[b];
      if (cudaStreamBeginCaptureToGraph(h->s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        ok = false;
        break;
      }
      h->batch_graph = g;
      st[b] = solve_start(h, -1, f[b], u[b], nullptr);
      h->batch_graph = nullptr;
      cudaGraph_t out = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(h->s, &out);
      if (st[b] != MSTOPO_OK || ee != cudaSuccess) ok = false;
      ++captured;
    }
    cudaGraphExec_t ex = nullptr;
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    cudaEvent_t done = nullptr;
    if (ok) ok = cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = cudaGraphLaunch(ex, hs[0]->s) == cudaSuccess && cudaEventRecord(done, hs[0]->s) == cudaSuccess;
    // every instance's stream waits for the graph, so that its finish sees the results
    for (int b = 0; b < n && ok; ++b) ok = cudaStreamWaitEvent(hs[b]->s, done, 0) == cudaSuccess;
    if (ok) {
      for (int b = 0; b < n; ++b) {
        mstopo_status sb = solve_finish(hs[b], -1, infos ? infos + (size_t)b * MSTOPO_MAX_SYS : nullptr);
        if (st[b] == MSTOPO_OK) st[b] = sb;
      }
      for (int b = 0; b < n; ++b) hs[b]->batch_graph_solves++;
    }
    if (done) cudaEventDestroy(done);
    if (ex) cudaGraphExecDestroy(ex);
    if (g) cudaGraphDestroy(g);
    if (ok) {
      for (int b = 0; b < n; ++b)
        if (st[b] != MSTOPO_OK) return st[b];
      return MSTOPO_OK;
    }
    // refused: forget the captured starts and take the per-instance path
    cudaGetLastError();
    for (int b = 0; b < captured; ++b) {
      hs[b]->sv.run_pending = 0;
      hs[b]->device_loop_solves = dls[b];
      st[b] = MSTOPO_OK;
    }
  }
  // One host thread: every instance's solve is enqueued on its own stream first (with the
  // device-side loop each is a few launches and one graph launch, none waiting for the GPU),
  // then each is finished in turn; the GPU runs the instances concurrently meanwhile.
  for (int b = 0; b < n; ++b) {
    cudaSetDevice(hs[b]->device);
    st[b] = solve_start(hs[b], -1, f[b], u[b], nullptr);
  }
  for (int b = 0; b < n; ++b) {
    if (st[b] != MSTOPO_OK) continue;
    cudaSetDevice(hs[b]->device);
    st[b] = solve_finish(hs[b], -1, infos ? infos + (size_t)b * MSTOPO_MAX_SYS : nullptr);
  }
  for (int b = 0; b < n; ++b)
    if (st[b] != MSTOPO_OK) return st[b];
  return MSTOPO_OK;
}

mstopo_status mstopo_inject(mstopo_handle* h, int32_t what) {
  if (!h) return MSTOPO_INVALID_ARG;
  CHECK_ARG(what == MSTOPO_INJECT_NONE || what == MSTOPO_INJECT_SWEEP_STALL, "unknown injection");
  h->inject = what;
  return MSTOPO_OK;
}
