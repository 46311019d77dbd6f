// The design loop around the solve (Sec. 4.4, 4.5): the expected-volume constraint and its
// gradient, the method of moving asymptotes (MMA, Svanberg 1987) for one constraint, and the
// continuation schedule on the SIMP exponent and beta.
//
// Problem (Sec. 4.4):  minimise f(rho) = E[c] + kappa sqrt(Var[c]) over the realisations,
// subject to g(rho) = E[vol(rho_bar)] / v_f - 1 <= 0 and 0 <= rho <= 1.  With every element of
// unit volume, E[vol] is the mean of rho_bar over the realisations and the design elements (a
// periodic cell stands for each of its tiles equally), and dg/drho = filter^T (mean over the
// realisations of d rho_bar / d rho_tilde) / (n_design v_f).
//
// MMA, one constraint, from the published method: asymptotes L_j < x_j < U_j, at
// x -/+ s0 (x_max - x_min) in the first two iterations, then moved by 0.7 where x_j
// oscillates and 1.2 where it moves monotonically (kept within [0.01, 10] (x_max - x_min) of
// x_j); convex separable approximations f~_i = f_i + sum_j p_ij (1/(U_j - x_j) - 1/(U_j - x^k_j))
// + q_ij (1/(x_j - L_j) - 1/(x^k_j - L_j)) with p = (U - x^k)^2 max(df, 0), q = (x^k - L)^2
// max(-df, 0); the subproblem on alpha <= x <= beta (alpha = max(x_min, 0.9 L + 0.1 x^k),
// beta = min(x_max, 0.9 U + 0.1 x^k)) through its dual: for lam >= 0,
// x_j(lam) = (L_j sqrt(P_j) + U_j sqrt(Q_j)) / (sqrt(P_j) + sqrt(Q_j)) clipped (P = p_0 + lam p_1,
// Q = q_0 + lam q_1), and lam is the root of the decreasing f~_1(x(lam)), by bracketing (x10)
// and bisection, or 0 when f~_1(x(0)) <= 0.  The element-wise parts run one thread per
// design variable; the dual runs in one CTA (block sums in a fixed order, every thread taking
// the same decisions), so the step is bitwise repeatable.
#include <cmath>
#include <string>
#include <vector>

#include "internal.cuh"

#define OT 1024

struct mstopo_mma {
  std::string err;
  cudaStream_t s = nullptr;
  long long n = 0;
  double xmin = 0.0, xmax = 1.0, s0 = 0.5, asydecr = 0.7, asyincr = 1.2;
  int k = 0;
  double *xold1 = nullptr, *xold2 = nullptr, *low = nullptr, *upp = nullptr;
  double *alpha = nullptr, *beta = nullptr, *p0 = nullptr, *q0 = nullptr, *p1 = nullptr, *q1 = nullptr;
  double* d_lam = nullptr;
};

namespace {

__device__ __forceinline__ double opt_block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();   // sh may still be read from the previous sum
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) sh[32] = v;
  }
  __syncthreads();
  return sh[32];
}

// asymptotes, bounds and approximation coefficients (one thread per variable)
__global__ void k_mma_prepare(long long n, int k, double s0, double decr, double incr, double xmin,
                              double xmax, const double* __restrict__ x,
                              const double* __restrict__ xold1, const double* __restrict__ xold2,
                              double* __restrict__ low, double* __restrict__ upp,
                              const double* __restrict__ df0, const double* __restrict__ dg,
                              double* __restrict__ alpha, double* __restrict__ beta,
                              double* __restrict__ p0, double* __restrict__ q0,
                              double* __restrict__ p1, double* __restrict__ q1) {
  const double span = xmax - xmin;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const double xj = x[j];
    double L, U;
    if (k < 2) {
      L = xj - s0 * span;
      U = xj + s0 * span;
    } else {
      const double s = (xj - xold1[j]) * (xold1[j] - xold2[j]);
      const double gam = s < 0.0 ? decr : (s > 0.0 ? incr : 1.0);
      L = xj - gam * (xold1[j] - low[j]);
      U = xj + gam * (upp[j] - xold1[j]);
      L = fmin(fmax(L, xj - 10.0 * span), xj - 0.01 * span);
      U = fmin(fmax(U, xj + 0.01 * span), xj + 10.0 * span);
    }
    low[j] = L;
    upp[j] = U;
    alpha[j] = fmax(xmin, 0.9 * L + 0.1 * xj);
    beta[j] = fmin(xmax, 0.9 * U + 0.1 * xj);
    const double ux = (U - xj) * (U - xj), xl = (xj - L) * (xj - L);
    p0[j] = ux * fmax(df0[j], 0.0);
    q0[j] = xl * fmax(-df0[j], 0.0);
    p1[j] = ux * fmax(dg[j], 0.0);
    q1[j] = xl * fmax(-dg[j], 0.0);
  }
}

__device__ __forceinline__ double mma_x_of(double lam, double x, double L, double U, double a,
                                           double b, double p0, double q0, double p1, double q1) {
  const double P = sqrt(p0 + lam * p1), Q = sqrt(q0 + lam * q1);
  const double xs = (P + Q > 0.0) ? (L * P + U * Q) / (P + Q) : x;
  return fmin(fmax(xs, a), b);
}

// The dual in one CTA: lam, then xnew = x(lam) and the state (xold2 = xold1, xold1 = x).
__global__ void __launch_bounds__(OT) k_mma_dual(long long n, double g0, const double* __restrict__ x,
                                                 const double* __restrict__ low, const double* __restrict__ upp,
                                                 const double* __restrict__ alpha, const double* __restrict__ beta,
                                                 const double* __restrict__ p0, const double* __restrict__ q0,
                                                 const double* __restrict__ p1, const double* __restrict__ q1,
                                                 double* __restrict__ xnew, double* __restrict__ xold1,
                                                 double* __restrict__ xold2, double* __restrict__ lam_out) {
  __shared__ double sh[33];
  auto g_of = [&](double lam) -> double {
    double s = 0.0;
    for (long long j = threadIdx.x; j < n; j += blockDim.x) {
      const double xj = x[j], L = low[j], U = upp[j];
      const double xt = mma_x_of(lam, xj, L, U, alpha[j], beta[j], p0[j], q0[j], p1[j], q1[j]);
      s += p1[j] * (1.0 / (U - xt) - 1.0 / (U - xj)) + q1[j] * (1.0 / (xt - L) - 1.0 / (xj - L));
    }
    return g0 + opt_block_sum(s, sh);
  };
  double lam = 0.0;
  if (g_of(0.0) > 0.0) {
    double hi = 1.0;
    while (g_of(hi) > 0.0 && hi < 1e40) hi *= 10.0;
    double lo = 0.0;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (g_of(mid) > 0.0) lo = mid;
      else hi = mid;
      if (hi - lo <= 1e-14 * fmax(hi, 1e-300)) break;
    }
    lam = hi;
  }
  for (long long j = threadIdx.x; j < n; j += blockDim.x) {
    const double xj = x[j];
    xnew[j] = mma_x_of(lam, xj, low[j], upp[j], alpha[j], beta[j], p0[j], q0[j], p1[j], q1[j]);
    xold2[j] = xold1[j];
    xold1[j] = xj;
  }
  if (threadIdx.x == 0) *lam_out = lam;
}

// volume: mean of rho_bar over realisations and elements (one CTA, fixed order); gradient
// scale * sum_k drbar_k (before the filter transpose)
__global__ void __launch_bounds__(OT) k_volume(const double* __restrict__ rbar, int n_eta,
                                               long long n_design, double* __restrict__ vol) {
  __shared__ double sh[33];
  double s = 0.0;
  for (long long j = threadIdx.x; j < (long long)n_eta * n_design; j += blockDim.x) s += rbar[j];
  s = opt_block_sum(s, sh);
  if (threadIdx.x == 0) *vol = s / ((double)n_eta * (double)n_design);
}

__global__ void k_volume_grad(const double* __restrict__ drbar, int n_eta, long long n_design,
                              double scale, double* __restrict__ out) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n_design;
       j += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < n_eta; ++k) s += drbar[(long long)k * n_design + j];
    out[j] = scale * s;
  }
}

int opt_grid(long long n) {
  const long long b = (n + 255) / 256;
  return (int)(b < 1024 ? (b > 0 ? b : 1) : 1024);
}

}  // namespace

#define OCK(x)                                                                  \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      H->err = std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x;      \
      return e_ == cudaErrorMemoryAllocation ? MSTOPO_OUT_OF_MEMORY : MSTOPO_CUDA_ERROR; \
    }                                                                           \
  } while (0)

static std::string g_mma_create_error;

static void mma_free(mstopo_mma* m) {
  double* ptrs[] = {m->xold1, m->xold2, m->low, m->upp, m->alpha, m->beta, m->p0, m->q0, m->p1, m->q1, m->d_lam};
  for (double* p : ptrs)
    if (p) cudaFree(p);
}

extern "C" {

mstopo_status mstopo_volume(mstopo_handle* H, double volfrac, double* g, double* dgdrho) {
  if (!H) return MSTOPO_INVALID_ARG;
  if (!H->design_ready) {
    H->err = "no design set";
    return MSTOPO_NOT_READY;
  }
  if (!(volfrac > 0.0 && volfrac <= 1.0)) {
    H->err = "volfrac must be in (0, 1]";
    return MSTOPO_INVALID_ARG;
  }
  const long long nd = H->n_design;
  double* vol_dev = H->d_gdesign;   // scratch until the gradient is formed
  // E[vol] / v_f - 1
  note_launch(), k_volume<<<1, OT, 0, H->s>>>(H->d_rbar, H->n_eta, nd, vol_dev);
  OCK(cudaGetLastError());
  double vol = 0.0;
  OCK(cudaMemcpyAsync(&vol, vol_dev, 8, cudaMemcpyDeviceToHost, H->s));
  OCK(cudaStreamSynchronize(H->s));
  if (g) *g = vol / volfrac - 1.0;
  if (dgdrho) {
    note_launch(), k_volume_grad<<<opt_grid(nd), 256, 0, H->s>>>(
        H->d_drbar, H->n_eta, nd, 1.0 / ((double)nd * volfrac * H->n_eta), H->d_gdesign);
    OCK(cudaGetLastError());
    OCK(launch_filter_T(H->d_gdesign, H->d_wsum, dgdrho, H->dx, H->dy, H->rmin, H->periodic, H->s));
    OCK(cudaStreamSynchronize(H->s));
  }
  return MSTOPO_OK;
}

mstopo_status mstopo_mma_create(int64_t n, double xmin, double xmax, double s0, void* stream,
                                mstopo_mma** out) {
  if (!out) return MSTOPO_INVALID_ARG;
  *out = nullptr;
  g_mma_create_error.clear();
  if (n < 1 || !(xmax > xmin) || !(s0 > 0.0)) {
    g_mma_create_error = "invalid MMA description";
    return MSTOPO_INVALID_ARG;
  }
  mstopo_mma* m = new mstopo_mma();
  m->n = n;
  m->xmin = xmin;
  m->xmax = xmax;
  m->s0 = s0;
  m->s = (cudaStream_t)stream;
  double** ptrs[] = {&m->xold1, &m->xold2, &m->low, &m->upp, &m->alpha, &m->beta, &m->p0, &m->q0, &m->p1, &m->q1};
  for (double** p : ptrs) {
    cudaError_t e = cudaMalloc(p, (size_t)n * 8);
    if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, (size_t)n * 8, m->s);
    if (e != cudaSuccess) {
      g_mma_create_error = std::string("CUDA: ") + cudaGetErrorString(e);
      mma_free(m);
      delete m;
      return e == cudaErrorMemoryAllocation ? MSTOPO_OUT_OF_MEMORY : MSTOPO_CUDA_ERROR;
    }
  }
  if (cudaMalloc(&m->d_lam, 8) != cudaSuccess) {
    g_mma_create_error = "CUDA: allocation failed";
    mma_free(m);
    delete m;
    return MSTOPO_OUT_OF_MEMORY;
  }
  *out = m;
  return MSTOPO_OK;
}

mstopo_status mstopo_mma_step(mstopo_mma* m, const double* x, double f0, const double* df0,
                              double g, const double* dg, double* xnew, double* lam) {
  if (!m) return MSTOPO_INVALID_ARG;
  if (!x || !df0 || !dg || !xnew) {
    m->err = "null pointer";
    return MSTOPO_INVALID_ARG;
  }
  if (!std::isfinite(f0) || !std::isfinite(g)) {
    m->err = "non-finite objective or constraint";
    return MSTOPO_NONFINITE;
  }
  (void)f0;   // the approximation of f_0 needs only its gradient (its value is a constant)
  note_launch(), k_mma_prepare<<<opt_grid(m->n), 256, 0, m->s>>>(
      m->n, m->k, m->s0, m->asydecr, m->asyincr, m->xmin, m->xmax, x, m->xold1, m->xold2, m->low,
      m->upp, df0, dg, m->alpha, m->beta, m->p0, m->q0, m->p1, m->q1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    note_launch(), k_mma_dual<<<1, OT, 0, m->s>>>(m->n, g, x, m->low, m->upp, m->alpha, m->beta,
                                                  m->p0, m->q0, m->p1, m->q1, xnew, m->xold1,
                                                  m->xold2, m->d_lam);
    e = cudaGetLastError();
  }
  double l = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&l, m->d_lam, 8, cudaMemcpyDeviceToHost, m->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->s);
  if (e != cudaSuccess) {
    m->err = std::string("CUDA: ") + cudaGetErrorString(e);
    return MSTOPO_CUDA_ERROR;
  }
  if (lam) *lam = l;
  m->k += 1;
  return MSTOPO_OK;
}

const char* mstopo_mma_last_error(const mstopo_mma* m) {
  return m ? m->err.c_str() : g_mma_create_error.c_str();
}

void mstopo_mma_destroy(mstopo_mma* m) {
  if (!m) return;
  mma_free(m);
  delete m;
}

mstopo_status mstopo_optimise(mstopo_handle* H, double* rho, const double* f,
                              const mstopo_opt_stage* stages, int32_t n_stages, double volfrac,
                              double kappa, double rel_change, mstopo_opt_record* records,
                              int32_t capacity, int32_t* n_records) {
  if (!H) return MSTOPO_INVALID_ARG;
  if (!rho || !f || !stages || n_stages < 1 || !(volfrac > 0.0 && volfrac <= 1.0) ||
      kappa < 0.0 || rel_change < 0.0 || capacity < 0 || (capacity > 0 && !records)) {
    H->err = "invalid optimisation arguments";
    return MSTOPO_INVALID_ARG;
  }
  for (int s = 0; s < n_stages; ++s)
    if (!(stages[s].penal >= 1.0) || !(stages[s].beta > 0.0) || stages[s].max_iter < 1) {
      H->err = "invalid optimisation stage";
      return MSTOPO_INVALID_ARG;
    }
  if (H->n_design < 1 || H->n_eta < 1) {
    H->err = "set a design first (its filter radius, thresholds and cell are kept)";
    return MSTOPO_NOT_READY;
  }
  const long long nd = H->n_design;
  const int n_eta = H->n_eta;
  const double rmin = H->rmin;
  const int cx = H->periodic ? H->dx : 0, cy = H->periodic ? H->dy : 0;
  double etas[MSTOPO_MAX_SYS];
  for (int k = 0; k < n_eta; ++k) etas[k] = H->etas[k];
  double *u = nullptr, *df = nullptr, *dg = nullptr, *xn = nullptr;
  OCK(cudaMalloc(&u, (size_t)n_eta * H->n_dof * 8));
  struct Free {
    std::vector<void*> p;
    ~Free() { for (void* q : p) cudaFree(q); }
  } guard;
  guard.p.push_back(u);
  OCK(cudaMalloc(&df, (size_t)nd * 8));
  guard.p.push_back(df);
  OCK(cudaMalloc(&dg, (size_t)nd * 8));
  guard.p.push_back(dg);
  OCK(cudaMalloc(&xn, (size_t)nd * 8));
  guard.p.push_back(xn);
  int nrec = 0;
  mstopo_status st = MSTOPO_OK;
  for (int s = 0; s < n_stages && st == MSTOPO_OK; ++s) {
    H->p.penal = stages[s].penal;
    mstopo_mma* mma = nullptr;
    st = mstopo_mma_create(nd, 0.0, 1.0, 0.5 / (1.0 + stages[s].beta), H->s, &mma);
    if (st != MSTOPO_OK) {
      H->err = g_mma_create_error;
      break;
    }
    double f_prev = 0.0;
    bool have_prev = false;
    for (int it = 0; it < stages[s].max_iter; ++it) {
      st = mstopo_set_design(H, rho, nd, rmin, stages[s].beta, etas, n_eta, cx, cy);
      if (st == MSTOPO_OK && !H->pc.built) st = mstopo_build_preconditioner(H, -1, nullptr);
      mstopo_solve_info infos[MSTOPO_MAX_SYS];
      if (st == MSTOPO_OK) st = mstopo_solve(H, -1, f, u, nullptr, infos);
      double c[MSTOPO_MAX_SYS] = {0}, fr = 0.0, g = 0.0;
      if (st == MSTOPO_OK) st = mstopo_compliance_and_sensitivity(H, kappa, c, &fr, df);
      if (st == MSTOPO_OK) st = mstopo_volume(H, volfrac, &g, dg);
      if (st != MSTOPO_OK) break;
      if (nrec < capacity) {
        mstopo_opt_record& r = records[nrec];
        r.stage = s;
        r.iteration = it;
        r.penal = stages[s].penal;
        r.beta = stages[s].beta;
        r.f = fr;
        r.g = g;
        int mx = 0;
        for (int k = 0; k < MSTOPO_MAX_SYS; ++k) r.c[k] = k < n_eta ? c[k] : 0.0;
        for (int k = 0; k < n_eta; ++k) mx = std::max(mx, (int)infos[k].iterations);
        r.solve_iterations = mx;
      }
      ++nrec;
      if (have_prev && std::fabs(fr - f_prev) <= rel_change * std::fabs(f_prev)) break;
      f_prev = fr;
      have_prev = true;
      st = mstopo_mma_step(mma, rho, fr, df, g, dg, xn, nullptr);
      if (st != MSTOPO_OK) {
        H->err = mma->err;
        break;
      }
      cudaError_t e = cudaMemcpyAsync(rho, xn, (size_t)nd * 8, cudaMemcpyDeviceToDevice, H->s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(H->s);
      if (e != cudaSuccess) {
        H->err = std::string("CUDA: ") + cudaGetErrorString(e);
        st = MSTOPO_CUDA_ERROR;
        break;
      }
    }
    mstopo_mma_destroy(mma);
  }
  if (n_records) *n_records = nrec;
  return st;
}

mstopo_status mstopo_robust_verification(mstopo_handle* H, const double* rho, const double* f,
                                         const double* etas, int32_t n, double* c) {
  if (!H) return MSTOPO_INVALID_ARG;
  if (!rho || !f || !etas || !c || n < 1) {
    H->err = "invalid verification arguments";
    return MSTOPO_INVALID_ARG;
  }
  if (H->n_design < 1) {
    H->err = "set a design first (its filter radius, beta and cell are kept)";
    return MSTOPO_NOT_READY;
  }
  const long long nd = H->n_design;
  const double rmin = H->rmin, beta = H->beta;
  const int cx = H->periodic ? H->dx : 0, cy = H->periodic ? H->dy : 0;
  double* u = nullptr;
  OCK(cudaMalloc(&u, (size_t)MSTOPO_MAX_SYS * H->n_dof * 8));
  mstopo_status st = MSTOPO_OK;
  for (int b = 0; b < n && st == MSTOPO_OK; b += MSTOPO_MAX_SYS) {
    const int m = std::min(MSTOPO_MAX_SYS, n - b);
    // each batch of thresholds is one set of realisations: its own coarse basis and factors
    st = mstopo_set_design(H, rho, nd, rmin, beta, etas + b, m, cx, cy);
    if (st == MSTOPO_OK && !H->pc.built) st = mstopo_build_preconditioner(H, -1, nullptr);
    if (st == MSTOPO_OK) st = mstopo_solve(H, -1, f, u, nullptr, nullptr);
    if (st == MSTOPO_OK) st = mstopo_compliance_and_sensitivity(H, 0.0, c + b, nullptr, nullptr);
  }
  cudaFree(u);
  return st;
}

}  // extern "C"
