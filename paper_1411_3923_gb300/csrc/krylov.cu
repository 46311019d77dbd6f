// Flexible conjugate gradients in FP64 with the two-level preconditioner (paper Sec. 2.4.2:
// K and the preconditioner are SPD, so CG applies; the paper itself uses GMRES).
//
// FCG(1) (Notay): with z_k = B(r_k),
//   p_k = z_k - (z_k^T q_{k-1} / p_{k-1}^T q_{k-1}) p_{k-1},  q_k = K p_k,
//   alpha_k = p_k^T r_k / p_k^T q_k,  x += alpha p,  r -= alpha q.
// The explicit K-orthogonalisation against the previous direction keeps the recurrence
// valid when B varies slightly from one application to the next (FP32 preconditioner).
//
// Precision modes
//   FP64   p, q, z and every kernel in FP64.
//   MIXED  x, r and all dot products in FP64; p, q, z stored in FP32; q = K p with the FP32
//          difference-form matvec; the preconditioner in FP32 except the FP64 coarse solve.
//          The recursive residual drifts from the true one by the FP32 matvec error, so the
//          true residual f - K x is recomputed in FP64 whenever the recursive one has
//          dropped by 1e-2 since the last recomputation, and always before declaring
//          convergence ("reliable updates").
// Iteration loop: with CUDA graphs on, the whole loop is one graph launch -- a WHILE
// conditional node around one iteration and a check kernel, an IF node around the FP64
// true-residual recomputation the check asks for; the check and a continue kernel set the
// two conditions on the device (converged systems, the iteration cap, a bounded device wait
// that gave up), so no host round trip happens inside a solve.  Without graphs (and while
// per-kernel profiling is on) the host takes the same decisions after every iteration, so
// both loops give the same iterates bit for bit.
// Every reduction is two-stage (fixed per-CTA partials, then one CTA in fixed order), so
// results are bitwise repeatable run to run.
#include <cmath>
#include <cstring>

#include "internal.cuh"

#define RB MSTOPO_RED_BLOCKS
#define RT 256
#define FCG_CHUNK 8   // iterations per replayed graph when conditional nodes are unavailable

// --------------------------------------------------------------------------- reductions
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  v = 0.0;
  if (wid == 0) {
    v = lane < (blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;   // valid in thread 0
}

// The total of one system's RB block partials in every thread of the block: the same loop and
// reduction as k_finish_sum, so every block of a kernel that needs a scalar forms it bitwise
// alike (and alike to a separate finishing kernel).  sh holds 33 values.
__device__ __forceinline__ double partials_total(const double* __restrict__ part, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < RB; i += blockDim.x) s += part[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) sh[32] = s;
  __syncthreads();
  const double t = sh[32];
  __syncthreads();
  return t;
}

template <typename A, typename B>
__global__ void __launch_bounds__(RT) k_dot(const A* __restrict__ a, const B* __restrict__ b,
                                            long long n, long long stride,
                                            double* __restrict__ partials) {
  __shared__ double sh[32];
  a += blockIdx.y * stride;
  b += blockIdx.y * stride;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)RB * RT)
    s = fma((double)a[i], (double)b[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.y * RB + blockIdx.x] = s;
}

__global__ void k_finish_sum(const double* __restrict__ partials, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < RB; i += blockDim.x) s += partials[blockIdx.x * RB + i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

cudaError_t launch_dot_partials(const double* a, const double* b, long long n, int nsys,
                                long long stride, double* partials, cudaStream_t s) {
  note_launch(), k_dot<double, double><<<dim3(RB, nsys), RT, 0, s>>>(a, b, n, stride, partials);
  return cudaGetLastError();
}
cudaError_t launch_dot_partials_f32(const float* a, const float* b, long long n, int nsys,
                                    long long stride, double* partials, cudaStream_t s) {
  note_launch(), k_dot<float, float><<<dim3(RB, nsys), RT, 0, s>>>(a, b, n, stride, partials);
  return cudaGetLastError();
}
cudaError_t launch_dot_partials_mix(const float* a, const double* b, long long n, int nsys,
                                    long long stride, double* partials, cudaStream_t s) {
  note_launch(), k_dot<float, double><<<dim3(RB, nsys), RT, 0, s>>>(a, b, n, stride, partials);
  return cudaGetLastError();
}
cudaError_t launch_finish_sum(const double* partials, int nsys, double* out, cudaStream_t s) {
  note_launch(), k_finish_sum<<<nsys, RT, 0, s>>>(partials, out);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------- conversions
__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
// b = a with Dirichlet DOFs zeroed (a == NULL: b = 0)
__global__ void k_mask_copy(const double* __restrict__ a, double* __restrict__ b,
                            const uint8_t* __restrict__ m, long long n_nodes, long long stride) {
  a = a ? a + blockIdx.y * stride : nullptr;
  b += blockIdx.y * stride;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_nodes;
       i += (long long)gridDim.x * blockDim.x) {
    uint8_t f = m[i];
    double2 v = a ? reinterpret_cast<const double2*>(a)[i] : make_double2(0.0, 0.0);
    if (f & 1) v.x = 0.0;
    if (f & 2) v.y = 0.0;
    reinterpret_cast<double2*>(b)[i] = v;
  }
}

cudaError_t launch_convert_d2f(const double* a, float* b, long long n, cudaStream_t s) {
  note_launch(), k_d2f<<<608, 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}
cudaError_t launch_convert_f2d(const float* a, double* b, long long n, cudaStream_t s) {
  note_launch(), k_f2d<<<608, 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}
cudaError_t launch_mask_copy(const double* a, double* b, const uint8_t* nmask, long long n_nodes,
                             int nsys, long long stride, cudaStream_t s) {
  note_launch(), k_mask_copy<<<dim3(304, nsys), 256, 0, s>>>(a, b, nmask, n_nodes, stride);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------- FCG steps
// partial sums of p^T q and p^T r in one pass
template <typename PT>
__global__ void __launch_bounds__(RT) k_pq_pr(const PT* __restrict__ p, const PT* __restrict__ q,
                                              const double* __restrict__ r, long long n,
                                              long long stride, double* __restrict__ partials,
                                              const FcgScalars* __restrict__ sc) {
  __shared__ double sh[32];
  if (!sc[blockIdx.y].active) return;
  p += blockIdx.y * stride;
  q += blockIdx.y * stride;
  r += blockIdx.y * stride;
  double s1 = 0.0, s2 = 0.0;
  for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)RB * RT) {
    double pv = (double)p[i];
    s1 = fma(pv, (double)q[i], s1);
    s2 = fma(pv, r[i], s2);
  }
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    partials[(blockIdx.y * 2 + 0) * RB + blockIdx.x] = s1;
    partials[(blockIdx.y * 2 + 1) * RB + blockIdx.x] = s2;
  }
}

// p = z + beta p with beta = -(z^T q_prev) / (p_prev^T q_prev) formed in every block from the
// partials of z^T q (zero on the first step): the finishing sum and the scalar step of the
// recurrence fused into the update.  Block 0 records z^T q and beta.
template <typename PT>
__global__ void __launch_bounds__(RT) k_pupdate_beta(const PT* __restrict__ z, PT* __restrict__ p,
                                                     long long n, long long stride,
                                                     const double* __restrict__ zq_part,
                                                     FcgScalars* __restrict__ sc) {
  __shared__ double sh[33];
  FcgScalars& c = sc[blockIdx.y];
  if (!c.active) return;
  const double zq = partials_total(zq_part + (long long)blockIdx.y * RB, sh);
  const double beta = c.restart ? 0.0 : -zq / c.pq_prev;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c.zq = zq;
    c.beta = beta;
  }
  z += blockIdx.y * stride;
  p += blockIdx.y * stride;
  if (beta == 0.0) {   // (re)start: p = z (p may hold stale or uninitialised data)
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)RB * RT)
      p[i] = z[i];
    return;
  }
  for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)RB * RT)
    p[i] = (PT)((double)z[i] + beta * (double)p[i]);
}

// alpha = p^T r / p^T q formed in every block from the partials (a breakdown p^T q <= 0 or a
// non-finite value stops the system in every block alike), then x += alpha p, r -= alpha q,
// (MIXED: r32 = float(r)) and the partials of ||r||^2 into rr_part.  Block 0 records the
// scalars and ends the first-step state.
template <typename PT>
__global__ void __launch_bounds__(RT) k_xr_alpha(double* __restrict__ x, double* __restrict__ r,
                                                 float* __restrict__ r32, const PT* __restrict__ p,
                                                 const PT* __restrict__ q, long long n,
                                                 long long stride,
                                                 const double* __restrict__ pqr_part,
                                                 double* __restrict__ rr_part,
                                                 FcgScalars* __restrict__ sc) {
  __shared__ double sh[33];
  FcgScalars& c = sc[blockIdx.y];
  if (!c.active) return;
  const double pq = partials_total(pqr_part + (long long)(blockIdx.y * 2 + 0) * RB, sh);
  const double pr = partials_total(pqr_part + (long long)(blockIdx.y * 2 + 1) * RB, sh);
  const bool bad = !(pq > 0.0) || !isfinite(pq) || !isfinite(pr);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c.pq = pq;
    c.pr = pr;
    c.restart = 0;
    if (bad) {
      c.status = isfinite(pq) && isfinite(pr) ? MSTOPO_NOT_SPD : MSTOPO_NONFINITE;
      c.active = 0;
      c.alpha = 0.0;
    } else {
      c.alpha = pr / pq;
      c.pq_prev = pq;
    }
  }
  if (bad) return;
  const double alpha = pr / pq;
  x += blockIdx.y * stride;
  r += blockIdx.y * stride;
  p += blockIdx.y * stride;
  q += blockIdx.y * stride;
  if (r32) r32 += blockIdx.y * stride;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)RB * RT) {
    x[i] = fma(alpha, (double)p[i], x[i]);
    double rv = fma(-alpha, (double)q[i], r[i]);
    r[i] = rv;
    if (r32) r32[i] = (float)rv;
    s = fma(rv, rv, s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) rr_part[blockIdx.y * RB + blockIdx.x] = s;
}

__global__ void k_scalar_rr(FcgScalars* sc, const double* __restrict__ partials, double tol2) {
  __shared__ double sh[32];
  FcgScalars& c = sc[blockIdx.x];
  if (!c.active) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < RB; i += blockDim.x) s += partials[blockIdx.x * RB + i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    c.rr = s;
    c.iters += 1;
    if (!isfinite(s)) {
      c.status = MSTOPO_NONFINITE;
      c.active = 0;
    } else if (s <= tol2 * c.ff) {
      c.active = 0;   // candidate: the host confirms with the true residual
    }
  }
}

// r = f - t (t = K x), r32 = float(r), partial ||r||^2
__global__ void __launch_bounds__(RT) k_residual(const double* __restrict__ f,
                                                 const double* __restrict__ t,
                                                 double* __restrict__ r, float* __restrict__ r32,
                                                 long long n, long long stride,
                                                 double* __restrict__ partials) {
  __shared__ double sh[32];
  f += blockIdx.y * stride;
  t += blockIdx.y * stride;
  r += blockIdx.y * stride;
  if (r32) r32 += blockIdx.y * stride;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)RB * RT) {
    double v = f[i] - t[i];
    r[i] = v;
    if (r32) r32[i] = (float)v;
    s = fma(v, v, s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.y * RB + blockIdx.x] = s;
}

// ----------------------------------------------------------------- device-side loop control
// After an iteration: the decisions the host loop takes between chunks.  A system whose
// recursive residual passed the tolerance (k_scalar_rr made it inactive) or, in MIXED, dropped
// by 1e-4 (squared) since the last recomputation needs the FP64 true residual; a system at the
// iteration cap stops with MAX_ITER; a failed system stops.  The IF condition is set when any
// system needs the true residual.
__global__ void k_fcg_check(FcgScalars* sc, int nsys, int mixed, int max_iter,
                            cudaGraphConditionalHandle if_true, int* loopstat) {
  if (threadIdx.x != 0) return;
  int need = 0;
  for (int s = 0; s < nsys; ++s) {
    FcgScalars& c = sc[s];
    if (c.done) continue;
    if (c.status != MSTOPO_OK) { c.done = 1; c.active = 0; continue; }
    if (!c.active) need = 1;
    else if (mixed && c.rr < 1e-4 * c.rr_last) need = 1;
    if (c.iters >= max_iter) { c.status = MSTOPO_MAX_ITER; c.done = 1; c.active = 0; }
  }
  loopstat[0] += 1;
  cudaGraphSetConditional(if_true, need ? 1u : 0u);
}

// After a true-residual recomputation (rr_true[s] = ||f - K x||^2): it replaces the recursive
// residual of every system; a system within the tolerance is done, the others continue.
__global__ void k_fcg_after_true(FcgScalars* sc, const double* __restrict__ rr_true, int nsys,
                                 double tol2, int* loopstat) {
  if (threadIdx.x != 0) return;
  for (int s = 0; s < nsys; ++s) {
    FcgScalars& c = sc[s];
    c.repl += 1;
    c.rr = rr_true[s];
    c.rr_last = rr_true[s];
    if (c.done) { c.active = 0; continue; }
    if (rr_true[s] <= tol2 * c.ff) { c.active = 0; c.done = 1; }
    else c.active = 1;
  }
  loopstat[1] += 1;
}

// Start of the device-side loop: reference residual for the reliable updates, done flags
// (systems already within the tolerance; a zero load is reported as INVALID_ARG), and the
// WHILE condition (no pass at all when every system is done).
__global__ void k_fcg_loop_init(FcgScalars* sc, int nsys, cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0) return;
  int more = 0;
  for (int s = 0; s < nsys; ++s) {
    FcgScalars& c = sc[s];
    c.rr_last = c.rr;
    c.repl = 0;
    c.done = c.active ? 0 : 1;
    if (c.ff == 0.0) {
      c.status = MSTOPO_INVALID_ARG;
      c.done = 1;
      c.active = 0;
    }
    if (!c.done) more = 1;
  }
  cudaGraphSetConditional(loop, more ? 1u : 0u);
}

// WHILE condition: some system still iterating and no bounded device wait gave up (which
// stops every system with that status).
__global__ void k_fcg_continue(FcgScalars* sc, int nsys, const int* __restrict__ werr,
                               cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0) return;
  const int e = *werr;
  int more = 0;
  for (int s = 0; s < nsys; ++s) {
    FcgScalars& c = sc[s];
    if (e && !c.done) { c.status = e; c.done = 1; c.active = 0; }
    if (!c.done) more = 1;
  }
  cudaGraphSetConditional(loop, more ? 1u : 0u);
}

// --------------------------------------------------------------------------- host driver
#define CK(x)                                                                   \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      h->err = std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x;      \
      return e_ == cudaErrorMemoryAllocation ? MSTOPO_OUT_OF_MEMORY : MSTOPO_CUDA_ERROR; \
    }                                                                           \
  } while (0)

mstopo_status solver_alloc(mstopo_handle* h) {
  Solver& sv = h->sv;
  if (sv.x) return MSTOPO_OK;
  sv.n = h->n_dof;
  size_t nd = (size_t)MSTOPO_MAX_SYS * sv.n;
  CK(cudaMalloc(&sv.x, nd * 8));
  CK(cudaMalloc(&sv.r, nd * 8));
  CK(cudaMalloc(&sv.f, nd * 8));
  CK(cudaMalloc(&sv.tmp, nd * 8));
  if (h->p.precision == MSTOPO_FP64) {
    CK(cudaMalloc(&sv.p64, nd * 8));
    CK(cudaMalloc(&sv.q64, nd * 8));
    CK(cudaMalloc(&sv.z64, nd * 8));
  } else {
    CK(cudaMalloc(&sv.p32, nd * 4));
    CK(cudaMalloc(&sv.q32, nd * 4));
    CK(cudaMalloc(&sv.z32, nd * 4));
    CK(cudaMalloc(&sv.r32, nd * 4));
  }
  CK(cudaMalloc(&sv.partials, (size_t)MSTOPO_MAX_SYS * 4 * RB * 8));
  CK(cudaMalloc(&sv.sc, MSTOPO_MAX_SYS * sizeof(FcgScalars)));
  CK(cudaMallocHost(&sv.h_sc, MSTOPO_MAX_SYS * sizeof(FcgScalars)));
  CK(cudaMalloc(&sv.loopstat, 2 * sizeof(int)));
  CK(cudaMallocHost(&sv.h_comp, MSTOPO_MAX_SYS * 8 + 4 * sizeof(int)));
  CK(cudaEventCreate(&sv.ev0));
  CK(cudaEventCreate(&sv.ev1));
  return MSTOPO_OK;
}

void solver_free(Solver& sv) {
  cudaFree(sv.x); cudaFree(sv.r); cudaFree(sv.f); cudaFree(sv.tmp);
  cudaFree(sv.p64); cudaFree(sv.q64); cudaFree(sv.z64);
  cudaFree(sv.p32); cudaFree(sv.q32); cudaFree(sv.z32); cudaFree(sv.r32);
  cudaFree(sv.partials); cudaFree(sv.sc); cudaFree(sv.loopstat);
  if (sv.h_sc) cudaFreeHost(sv.h_sc);
  if (sv.h_comp) cudaFreeHost(sv.h_comp);
  if (sv.ev0) cudaEventDestroy(sv.ev0);
  if (sv.ev1) cudaEventDestroy(sv.ev1);
  sv = Solver();
}

// FP64 true residual for all systems: r = f - K64(E_k) x ; rr_out[s] = ||r||^2
static mstopo_status true_residual(mstopo_handle* h, int sys0, int nsys, double* rr_dev) {
  Solver& sv = h->sv;
  const long long n = sv.n;
  cudaEvent_t pa = prof_begin(h->prof, h->s);
  CK(launch_matvec_f64(sv.x, sv.tmp, h->d_E64 + (long long)sys0 * h->n_el, h->d_nmask, h->nelx,
                       h->nely, h->st64, nsys, n, h->n_el, h->s));
  prof_end(h->prof, PROF_MATVEC64, pa, h->s);
  note_launch(), k_residual<<<dim3(RB, nsys), RT, 0, h->s>>>(sv.f, sv.tmp, sv.r, sv.r32, n, n, sv.partials);
  CK(cudaGetLastError());
  CK(launch_finish_sum(sv.partials, nsys, rr_dev, h->s));
  return MSTOPO_OK;
}

__global__ void k_set_rr(FcgScalars* sc, const double* __restrict__ v, int which, double tol2) {
  FcgScalars& c = sc[threadIdx.x];
  if (which == 0) c.ff = v[threadIdx.x];
  else c.rr = v[threadIdx.x];
  if (which == 1) c.active = (c.rr > tol2 * c.ff) ? 1 : 0;
}

static mstopo_status precond(mstopo_handle* h, int sys0, int nsys) {
  Solver& sv = h->sv;
  cudaError_t e;
  if (h->p.precision == MSTOPO_FP64) e = precond_apply_f64(h, sv.r, sv.z64, sys0, nsys, 0);
  else e = precond_apply_f32(h, sv.r32, sv.z32, sys0, nsys, 0);
  CK(e);
  return MSTOPO_OK;
}

mstopo_status fcg_start(mstopo_handle* h, int sys0, int nsys, const double* f, double* u,
                        const double* u0) {
  Solver& sv = h->sv;
  mstopo_status st = solver_alloc(h);
  if (st != MSTOPO_OK) return st;
  const long long n = sv.n;
  const bool mixed = h->p.precision != MSTOPO_FP64;
  const double tol2 = h->p.tol * h->p.tol;
  sv.run_pending = 0;
  // inside a batch capture the timing events become event-record nodes of the batch graph
  const bool in_batch = h->batch_graph != nullptr;
  const unsigned ev_flags = in_batch ? cudaEventRecordExternal : cudaEventRecordDefault;
  CK(cudaEventRecordWithFlags(sv.ev0, h->s, ev_flags));
  CK(cudaMemsetAsync(h->d_flag + 1, 0, sizeof(int), h->s));   // device-wait timeout word
  // f (same load for every system), masked; x0
  for (int s = 0; s < nsys; ++s) CK(launch_mask_copy(f, sv.f + s * n, h->d_nmask, h->n_nodes, 1, n, h->s));
  CK(launch_mask_copy(u0, sv.x, h->d_nmask, h->n_nodes, nsys, n, h->s));
  FcgScalars init;
  memset(&init, 0, sizeof(init));
  init.active = 1;
  init.status = MSTOPO_OK;
  init.restart = 1;
  for (int s = 0; s < nsys; ++s) sv.h_sc[s] = init;
  CK(cudaMemcpyAsync(sv.sc, sv.h_sc, nsys * sizeof(FcgScalars), cudaMemcpyHostToDevice, h->s));
  double* vtmp = sv.partials + (size_t)MSTOPO_MAX_SYS * 3 * RB;   // small scratch [nsys]
  if (h->p.krylov == MSTOPO_KRYLOV_GMRES) {
    // GMRES(m) fills the host scalars itself; the outputs below are the same
    st = gmres_run(h, sys0, nsys);
    if (st != MSTOPO_OK) return st;
    CK(cudaEventRecord(sv.ev1, h->s));
    CK(cudaMemcpyAsync(u, sv.x, (size_t)nsys * n * 8, cudaMemcpyDeviceToDevice, h->s));
    CK(launch_dot_partials(sv.f, sv.x, n, nsys, n, sv.partials, h->s));
    CK(launch_finish_sum(sv.partials, nsys, vtmp, h->s));
    CK(cudaMemcpyAsync(sv.h_comp, vtmp, nsys * 8, cudaMemcpyDeviceToHost, h->s));
    sv.run_sys0 = sys0;
    sv.run_nsys = nsys;
    sv.run_looped = 0;
    for (int s = 0; s < nsys; ++s) sv.run_repl[s] = sv.h_sc[s].repl;
    sv.run_pending = 1;
    return MSTOPO_OK;
  }
  CK(launch_dot_partials(sv.f, sv.f, n, nsys, n, sv.partials, h->s));
  CK(launch_finish_sum(sv.partials, nsys, vtmp, h->s));
  note_launch(), k_set_rr<<<1, nsys, 0, h->s>>>(sv.sc, vtmp, 0, tol2);
  CK(cudaGetLastError());
  st = true_residual(h, sys0, nsys, vtmp);
  if (st != MSTOPO_OK) return st;
  note_launch(), k_set_rr<<<1, nsys, 0, h->s>>>(sv.sc, vtmp, 1, tol2);
  CK(cudaGetLastError());
  double rr_last[MSTOPO_MAX_SYS] = {0};
  int done[MSTOPO_MAX_SYS] = {0}, repl[MSTOPO_MAX_SYS] = {0};
  const float* E32 = h->d_E32 + (long long)sys0 * h->n_el;
  const double* E64 = h->d_E64 + (long long)sys0 * h->n_el;
  // one flexible-CG iteration for all systems (kernels skip finished systems)
  auto iteration = [&]() -> mstopo_status {
    mstopo_status s2 = precond(h, sys0, nsys);
    if (s2 != MSTOPO_OK) return s2;
    if (mixed) CK(launch_dot_partials_f32(sv.z32, sv.q32, n, nsys, n, sv.partials, h->s));
    else CK(launch_dot_partials(sv.z64, sv.q64, n, nsys, n, sv.partials, h->s));
    if (mixed) {
      note_launch(), k_pupdate_beta<float><<<dim3(RB, nsys), RT, 0, h->s>>>(sv.z32, sv.p32, n, n, sv.partials, sv.sc);
      CK(cudaGetLastError());
      cudaEvent_t pa = prof_begin(h->prof, h->s);
      CK(launch_matvec_f32(sv.p32, sv.q32, E32, h->d_nmask, h->nelx, h->nely, h->st32, nsys, n,
                           h->n_el, h->s, false));
      prof_end(h->prof, PROF_MATVEC32, pa, h->s);
      note_launch(), k_pq_pr<float><<<dim3(RB, nsys), RT, 0, h->s>>>(sv.p32, sv.q32, sv.r, n, n, sv.partials, sv.sc);
    } else {
      note_launch(), k_pupdate_beta<double><<<dim3(RB, nsys), RT, 0, h->s>>>(sv.z64, sv.p64, n, n, sv.partials, sv.sc);
      CK(cudaGetLastError());
      cudaEvent_t pa = prof_begin(h->prof, h->s);
      CK(launch_matvec_f64(sv.p64, sv.q64, E64, h->d_nmask, h->nelx, h->nely, h->st64, nsys, n,
                           h->n_el, h->s, false));
      prof_end(h->prof, PROF_MATVEC64, pa, h->s);
      note_launch(), k_pq_pr<double><<<dim3(RB, nsys), RT, 0, h->s>>>(sv.p64, sv.q64, sv.r, n, n, sv.partials, sv.sc);
    }
    CK(cudaGetLastError());
    // ||r||^2 partials after the p^T q, p^T r ones (the fused update still reads those)
    double* rr_part = sv.partials + (size_t)MSTOPO_MAX_SYS * 2 * RB;
    if (mixed)
      note_launch(), k_xr_alpha<float><<<dim3(RB, nsys), RT, 0, h->s>>>(sv.x, sv.r, sv.r32, sv.p32, sv.q32, n, n,
                                                         sv.partials, rr_part, sv.sc);
    else
      note_launch(), k_xr_alpha<double><<<dim3(RB, nsys), RT, 0, h->s>>>(sv.x, sv.r, nullptr, sv.p64, sv.q64, n,
                                                          n, sv.partials, rr_part, sv.sc);
    CK(cudaGetLastError());
    note_launch(), k_scalar_rr<<<nsys, RT, 0, h->s>>>(sv.sc, rr_part, tol2);
    CK(cudaGetLastError());
    return MSTOPO_OK;
  };
  // ---- the whole loop as one graph (no host round trip inside the solve) ----
  bool looped = false;
  FcgGraph& gr = h->fcg_graph;
  // The loop as a graph: into == nullptr builds and instantiates the handle's own loop graph;
  // otherwise h->s is capturing into `into` (a batch graph) and the loop becomes nodes of it:
  // the capture pauses at the WHILE node while the bodies are captured, then resumes after it.
  auto build_loop = [&](cudaGraph_t into) -> cudaError_t {
      cudaGraph_t top = into;
      cudaError_t e = cudaSuccess;
      if (!into && (e = cudaGraphCreate(&top, 0)) != cudaSuccess) return e;
      struct GraphGuard { cudaGraph_t g; ~GraphGuard() { if (g) cudaGraphDestroy(g); } } guard{into ? nullptr : top};
      cudaGraphConditionalHandle wh, ih;
      if ((e = cudaGraphConditionalHandleCreate(&wh, top, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
      if ((e = cudaGraphConditionalHandleCreate(&ih, top, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
      // (the params struct holds a union without a default constructor: zeroed storage)
      alignas(cudaGraphNodeParams) unsigned char wbuf[sizeof(cudaGraphNodeParams)] = {};
      cudaGraphNodeParams& wp = *reinterpret_cast<cudaGraphNodeParams*>(wbuf);
      wp.type = cudaGraphNodeTypeConditional;
      wp.conditional.handle = wh;
      wp.conditional.type = cudaGraphCondTypeWhile;
      wp.conditional.size = 1;
      // the loop's start (done flags, reference residuals, the WHILE condition), then the node
      if (!into && (e = cudaStreamBeginCaptureToGraph(h->s, top, nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return e;
      k_fcg_loop_init<<<1, 32, 0, h->s>>>(sv.sc, nsys, wh);
      cudaGraphNode_t wnode = nullptr;
      {
        cudaError_t ce0 = cudaGetLastError();
        cudaStreamCaptureStatus cst;
        cudaGraph_t cgraph;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        if (ce0 == cudaSuccess) ce0 = cudaStreamGetCaptureInfo(h->s, &cst, nullptr, &cgraph, &deps, nullptr, &nd);
        if (ce0 == cudaSuccess) ce0 = cudaGraphAddNode(&wnode, cgraph, deps, nullptr, nd, &wp);
        if (ce0 == cudaSuccess)
          ce0 = cudaStreamUpdateCaptureDependencies(h->s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
        cudaGraph_t captured0 = nullptr;
        cudaError_t ee0 = cudaStreamEndCapture(h->s, &captured0);
        if (ce0 != cudaSuccess) return ce0;
        if (ee0 != cudaSuccess) return ee0;
      }
      cudaGraph_t body = wp.conditional.phGraph_out[0];
      const long long l0 = g_launch_count.load();
      // loop body: one iteration, the check, the IF node, the continue kernel
      if ((e = cudaStreamBeginCaptureToGraph(h->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return e;
      mstopo_status cs = iteration();
      note_launch(), k_fcg_check<<<1, 32, 0, h->s>>>(sv.sc, nsys, mixed ? 1 : 0, h->p.max_iter, ih, sv.loopstat);
      cudaError_t ce = cudaGetLastError();
      cudaGraphNode_t inode = nullptr;
      alignas(cudaGraphNodeParams) unsigned char ibuf[sizeof(cudaGraphNodeParams)] = {};
      cudaGraphNodeParams& ip = *reinterpret_cast<cudaGraphNodeParams*>(ibuf);
      if (cs == MSTOPO_OK && ce == cudaSuccess) {
        cudaStreamCaptureStatus cst;
        cudaGraph_t cgraph;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        ce = cudaStreamGetCaptureInfo(h->s, &cst, nullptr, &cgraph, &deps, nullptr, &nd);
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = ih;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        if (ce == cudaSuccess) ce = cudaGraphAddNode(&inode, cgraph, deps, nullptr, nd, &ip);
        if (ce == cudaSuccess)
          ce = cudaStreamUpdateCaptureDependencies(h->s, &inode, nullptr, 1, cudaStreamSetCaptureDependencies);
      }
      if (ce == cudaSuccess) {
        note_launch(), k_fcg_continue<<<1, 32, 0, h->s>>>(sv.sc, nsys, h->d_flag + 1, wh);
        ce = cudaGetLastError();
      }
      cudaGraph_t captured = nullptr;
      cudaError_t ee = cudaStreamEndCapture(h->s, &captured);
      if (cs != MSTOPO_OK) return cudaErrorUnknown;
      if (ce != cudaSuccess) return ce;
      if (ee != cudaSuccess) return ee;
      const long long l1 = g_launch_count.load();
      // IF body: the FP64 true residual of every system and its bookkeeping
      if ((e = cudaStreamBeginCaptureToGraph(h->s, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return e;
      cs = true_residual(h, sys0, nsys, vtmp);
      if (cs == MSTOPO_OK) {
        note_launch(), k_fcg_after_true<<<1, 32, 0, h->s>>>(sv.sc, vtmp, nsys, tol2, sv.loopstat);
        ce = cudaGetLastError();
      }
      ee = cudaStreamEndCapture(h->s, &captured);
      if (cs != MSTOPO_OK) return cudaErrorUnknown;
      if (ce != cudaSuccess) return ce;
      if (ee != cudaSuccess) return ee;
      const long long l2 = g_launch_count.load();
      g_launch_count.fetch_sub(l2 - l0);   // counted per executed pass below
      gr.loop_launches = l1 - l0;
      gr.true_launches = l2 - l1;
      if (into) {   // resume the batch capture after the WHILE node
        return cudaStreamBeginCaptureToGraph(h->s, into, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal);
      }
      if ((e = cudaGraphInstantiate(&gr.loop, top, 0)) != cudaSuccess) { gr.loop = nullptr; return e; }
      gr.loop_sys0 = sys0;
      gr.loop_nsys = nsys;
      gr.loop_generation = h->pc_generation;
      return cudaSuccess;
  };
  if (!in_batch && h->graphs_enabled && !h->prof.on && !h->loop_graph_failed) {
    if (!gr.loop || gr.loop_sys0 != sys0 || gr.loop_nsys != nsys || gr.loop_generation != h->pc_generation) {
      if (gr.loop) { cudaGraphExecDestroy(gr.loop); gr.loop = nullptr; }
      if (build_loop(nullptr) != cudaSuccess) {
        // conditional graph nodes unavailable: the host-driven loop below takes over
        cudaGetLastError();
        h->loop_graph_failed = 1;
      }
    }
  }
  int* h_ints = reinterpret_cast<int*>(sv.h_comp + MSTOPO_MAX_SYS);   // loop passes [2], werr
  if (in_batch) {
    // the loop as nodes of the batch graph being captured
    looped = true;
    h->device_loop_solves++;
    CK(cudaMemsetAsync(sv.loopstat, 0, 2 * sizeof(int), h->s));
    if (build_loop(h->batch_graph) != cudaSuccess) {
      h->err = "batch graph: the flexible-CG loop could not be captured";
      return MSTOPO_CUDA_ERROR;
    }
    CK(cudaMemcpyAsync(sv.h_sc, sv.sc, nsys * sizeof(FcgScalars), cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(h_ints, sv.loopstat, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(h_ints + 2, h->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  } else if (h->graphs_enabled && !h->prof.on && !h->loop_graph_failed && h->fcg_graph.loop) {
    // one graph launch; nothing returns to the host before fcg_finish
    looped = true;
    h->device_loop_solves++;
    CK(cudaMemsetAsync(sv.loopstat, 0, 2 * sizeof(int), h->s));
    CK(cudaGraphLaunch(h->fcg_graph.loop, h->s));
    CK(cudaMemcpyAsync(sv.h_sc, sv.sc, nsys * sizeof(FcgScalars), cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(h_ints, sv.loopstat, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(h_ints + 2, h->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  } else {
    // host-driven loop: the starting state comes back first
    CK(cudaMemcpyAsync(sv.h_sc, sv.sc, nsys * sizeof(FcgScalars), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    for (int s = 0; s < nsys; ++s) {
      rr_last[s] = sv.h_sc[s].rr;
      if (sv.h_sc[s].ff == 0.0) {
        h->err = "zero load vector";
        return MSTOPO_INVALID_ARG;
      }
      if (!sv.h_sc[s].active) done[s] = 1;
    }
  }
  // Without graphs (or with per-kernel profiling) the host decides after every iteration,
  // exactly as the device-side loop does, so both take the same path bit for bit.  Only the
  // fallback for a missing conditional-node runtime replays chunks of iterations.
  const int chunk = (h->graphs_enabled && !h->prof.on) ? FCG_CHUNK : 1;
  int total_iters = 0;
  bool first_chunk = true;
  while (!looped) {
    int n_active = 0;
    for (int s = 0; s < nsys; ++s) n_active += !done[s];
    if (n_active == 0) break;
    // the first chunk runs directly (it also sets kernel attributes); later chunks replay
    // one captured graph of `chunk` iterations, unless per-kernel profiling is on
    const bool use_graph = !first_chunk && !h->prof.on && h->graphs_enabled;
    if (use_graph) {
      FcgGraph& gr = h->fcg_graph;
      if (!gr.exec || gr.sys0 != sys0 || gr.nsys != nsys || gr.generation != h->pc_generation) {
        if (gr.exec) { cudaGraphExecDestroy(gr.exec); gr.exec = nullptr; }
        cudaGraph_t graph;
        const long long l0 = g_launch_count.load();
        CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
        mstopo_status cs = MSTOPO_OK;
        for (int it = 0; it < chunk && cs == MSTOPO_OK; ++it) cs = iteration();
        cudaError_t ce = cudaStreamEndCapture(h->s, &graph);
        if (cs != MSTOPO_OK) return cs;
        CK(ce);
        CK(cudaGraphInstantiate(&gr.exec, graph, 0));
        cudaGraphDestroy(graph);
        gr.launches = g_launch_count.load() - l0;
        g_launch_count.fetch_sub(gr.launches);   // counted per replay below
        gr.sys0 = sys0;
        gr.nsys = nsys;
        gr.generation = h->pc_generation;
      }
      CK(cudaGraphLaunch(gr.exec, h->s));
      g_launch_count.fetch_add(gr.launches);
    } else {
      for (int it = 0; it < chunk; ++it) {
        st = iteration();
        if (st != MSTOPO_OK) return st;
      }
    }
    first_chunk = false;
    total_iters += chunk;
    int werr = 0;
    CK(cudaMemcpyAsync(sv.h_sc, sv.sc, nsys * sizeof(FcgScalars), cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(&werr, h->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    prof_collect(h->prof);
    if (werr) {
      for (int s = 0; s < nsys; ++s) { sv.h_sc[s].status = werr; sv.h_sc[s].active = 0; done[s] = 1; }
      break;
    }
    // host decisions: convergence candidates and reliable updates need the true residual
    bool need_true = false;
    for (int s = 0; s < nsys; ++s) {
      if (done[s]) continue;
      FcgScalars& c = sv.h_sc[s];
      if (c.status != MSTOPO_OK) { done[s] = 1; continue; }
      if (!c.active) need_true = true;
      else if (mixed && c.rr < 1e-4 * rr_last[s]) need_true = true;
      if (c.iters >= h->p.max_iter) { c.status = MSTOPO_MAX_ITER; done[s] = 1; }
    }
    if (need_true) {
      st = true_residual(h, sys0, nsys, vtmp);
      if (st != MSTOPO_OK) return st;
      double rr_true[MSTOPO_MAX_SYS];
      CK(cudaMemcpyAsync(rr_true, vtmp, nsys * 8, cudaMemcpyDeviceToHost, h->s));
      CK(cudaStreamSynchronize(h->s));
      for (int s = 0; s < nsys; ++s) {
        FcgScalars& c = sv.h_sc[s];
        repl[s]++;
        c.rr = rr_true[s];
        rr_last[s] = rr_true[s];
        if (done[s]) { c.active = 0; continue; }
        if (rr_true[s] <= tol2 * c.ff) { c.active = 0; done[s] = 1; }
        else c.active = 1;
      }
      // the true residual replaced r for every system (finished ones are unchanged in x)
      CK(cudaMemcpyAsync(sv.sc, sv.h_sc, nsys * sizeof(FcgScalars), cudaMemcpyHostToDevice, h->s));
    } else {
      for (int s = 0; s < nsys; ++s) if (done[s] && sv.h_sc[s].active) sv.h_sc[s].active = 0;
      CK(cudaMemcpyAsync(sv.sc, sv.h_sc, nsys * sizeof(FcgScalars), cudaMemcpyHostToDevice, h->s));
    }
    if (total_iters > h->p.max_iter + chunk) break;
  }
  CK(cudaEventRecordWithFlags(sv.ev1, h->s, ev_flags));
  // outputs
  CK(cudaMemcpyAsync(u, sv.x, (size_t)nsys * n * 8, cudaMemcpyDeviceToDevice, h->s));
  // compliance f^T u
  CK(launch_dot_partials(sv.f, sv.x, n, nsys, n, sv.partials, h->s));
  CK(launch_finish_sum(sv.partials, nsys, vtmp, h->s));
  CK(cudaMemcpyAsync(sv.h_comp, vtmp, nsys * 8, cudaMemcpyDeviceToHost, h->s));
  sv.run_sys0 = sys0;
  sv.run_nsys = nsys;
  sv.run_looped = looped ? 1 : 0;
  for (int s = 0; s < nsys; ++s) sv.run_repl[s] = repl[s];
  sv.run_pending = 1;
  return MSTOPO_OK;
}

mstopo_status fcg_finish(mstopo_handle* h, mstopo_solve_info* infos) {
  Solver& sv = h->sv;
  if (!sv.run_pending) {
    h->err = "no solve in flight";
    return MSTOPO_INVALID_ARG;
  }
  sv.run_pending = 0;
  CK(cudaStreamSynchronize(h->s));
  const int nsys = sv.run_nsys;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, sv.ev0, sv.ev1);
  const int* h_ints = reinterpret_cast<const int*>(sv.h_comp + MSTOPO_MAX_SYS);
  if (sv.run_looped) {
    const FcgGraph& gr = h->fcg_graph;
    // passes of the loop body and of the true-residual body, and the loop's start kernel
    g_launch_count.fetch_add((long long)h_ints[0] * gr.loop_launches + (long long)h_ints[1] * gr.true_launches + 1);
    const int werr = h_ints[2];
    for (int s = 0; s < nsys; ++s) {
      FcgScalars& c = sv.h_sc[s];
      sv.run_repl[s] = c.repl;
      if (werr && c.status == MSTOPO_OK && c.active) c.status = werr;
      if (c.ff == 0.0) {
        h->err = "zero load vector";
        return MSTOPO_INVALID_ARG;
      }
    }
  }
  for (int s = 0; s < nsys; ++s)
    if (sv.h_sc[s].status == MSTOPO_INVALID_ARG && sv.h_sc[s].ff == 0.0) {
      h->err = "zero load vector";
      return MSTOPO_INVALID_ARG;
    }
  mstopo_status worst = MSTOPO_OK;
  for (int s = 0; s < nsys; ++s) {
    const FcgScalars& c = sv.h_sc[s];
    if (c.status != MSTOPO_OK && worst == MSTOPO_OK) worst = (mstopo_status)c.status;
    if (infos) {
      infos[s].status = c.status;
      infos[s].iterations = c.iters;
      infos[s].replacements = sv.run_repl[s];
      infos[s].rel_residual = std::sqrt(c.rr / c.ff);
      infos[s].compliance = sv.h_comp[s];
      infos[s].ms = ms;
    }
  }
  if (worst != MSTOPO_OK) h->err = "flexible CG did not converge (see per-system status)";
  return worst;
}

mstopo_status fcg_solve(mstopo_handle* h, int sys0, int nsys, const double* f, double* u,
                        const double* u0, mstopo_solve_info* infos) {
  mstopo_status st = fcg_start(h, sys0, nsys, f, u, u0);
  if (st != MSTOPO_OK) return st;
  return fcg_finish(h, infos);
}
