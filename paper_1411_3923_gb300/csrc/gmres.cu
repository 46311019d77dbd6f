// Restarted GMRES(m), the outer method the paper pairs with its multiplicative preconditioner
// (Sec. 2.4.2: symmetric Gauss-Seidel, coarse correction, symmetric Gauss-Seidel), right
// preconditioned and flexible: z_j = M^-1 v_j is stored, x = x0 + Z y, so the MIXED
// preconditioner (FP32 sweeps) may vary slightly between applications.
//
// One cycle from x: r = f - K x (FP64), v_0 = r / ||r||, and for j = 0, 1, ..:
//   z_j = M^-1 v_j,  w = K z_j,
//   Gram-Schmidt of w against v_0..v_j, applied twice (h = V^T w, w -= V h, twice; the
//     column of H is the sum of both passes), H[j+1][j] = ||w||, v_{j+1} = w / H[j+1][j],
//   the earlier Givens rotations on column j, a new one that zeroes H[j+1][j], and the
//     same rotation on the right-hand side g (g_0 = ||r|| e_1); |g[j+1]| is the norm of the
//     residual of the least-squares iterate.
// The cycle ends at m steps, or when |g[j+1]| <= tol ||f||, or on a breakdown (the rotated
// diagonal is zero); then y solves the triangular system H y = g and x += Z y.  Each cycle
// starts from the true FP64 residual, so the solve stops on ||f - K x|| / ||f|| <= tol as the
// flexible CG does.  The Gram-Schmidt pair replaces the modified Gram-Schmidt of the textbook
// algorithm: both orthogonalise against the same basis, and the pair needs two reductions per
// pass instead of j + 1.  Realisations are solved one after the other.  Every reduction is
// two-stage in a fixed order: results are bitwise repeatable.
#include <cmath>

#include "internal.cuh"

#define GB MSTOPO_RED_BLOCKS
#define GT 256

namespace {

__device__ __forceinline__ double gm_block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// partials[i][b]: block b's share of V_i . w for i < gridDim.y
__global__ void k_gm_dots(const double* __restrict__ V, const double* __restrict__ w, long long n,
                          double* __restrict__ partials) {
  __shared__ double sh[32];
  const double* v = V + (long long)blockIdx.y * n;
  double s = 0.0;
  for (long long k = blockIdx.x * (long long)GT + threadIdx.x; k < n; k += (long long)GB * GT)
    s = fma(v[k], w[k], s);
  s = gm_block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.y * GB + blockIdx.x] = s;
}

// out[i] = sum of the GB partials of row i (fixed order)
__global__ void k_gm_finish(const double* __restrict__ partials, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < GB; b += blockDim.x) s += partials[blockIdx.x * GB + b];
  s = gm_block_sum(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// w -= sum_{i < nv} h[i] V_i
__global__ void k_gm_sub(const double* __restrict__ V, double* __restrict__ w, long long n,
                         const double* __restrict__ h, int nv) {
  __shared__ double hs[256];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    double a = w[k];
    for (int i = 0; i < nv; ++i) a = fma(-hs[i], V[(long long)i * n + k], a);
    w[k] = a;
  }
}

// r = f - t and block partials of ||r||^2
__global__ void k_gm_residual(const double* __restrict__ f, const double* __restrict__ t,
                              double* __restrict__ r, long long n, double* __restrict__ partials) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long k = blockIdx.x * (long long)GT + threadIdx.x; k < n; k += (long long)GB * GT) {
    const double v = f[k] - t[k];
    r[k] = v;
    s = fma(v, v, s);
  }
  s = gm_block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out = a / *d (or zero when *d is not positive)
__global__ void k_gm_scale(const double* __restrict__ a, double* __restrict__ out, long long n,
                           const double* __restrict__ d) {
  const double s = *d;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    out[k] = s > 0.0 ? a[k] / s : 0.0;
}

// Column j of H (column-major, leading dimension ld = m + 1) from the two Gram-Schmidt passes
// and ||w||^2, then the rotations.  st[0] = ||w|| (the unrotated H[j+1][j]), st[1] = |g[j+1]|,
// st[2] = the rotated diagonal.
__global__ void k_gm_column(double* __restrict__ H, int ld, int j, const double* __restrict__ h1,
                            const double* __restrict__ h2, const double* __restrict__ ww,
                            double* __restrict__ cs, double* __restrict__ sn,
                            double* __restrict__ g, double* __restrict__ st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* c = H + (long long)j * ld;
  for (int i = 0; i <= j; ++i) c[i] = h1[i] + h2[i];
  const double hn = sqrt(fmax(*ww, 0.0));
  c[j + 1] = hn;
  st[0] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = c[i], b = c[i + 1];
    c[i] = cs[i] * a + sn[i] * b;
    c[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double d = hypot(c[j], c[j + 1]);
  if (d > 0.0) {
    cs[j] = c[j] / d;
    sn[j] = c[j + 1] / d;
  } else {
    cs[j] = 1.0;
    sn[j] = 0.0;
  }
  c[j] = d;
  c[j + 1] = 0.0;
  const double gj = g[j];
  g[j] = cs[j] * gj;
  g[j + 1] = -sn[j] * gj;
  st[1] = fabs(g[j + 1]);
  st[2] = d;
}

// start of a cycle: g = ||r|| e_1 (g has ld entries), beta = ||r|| from rr = ||r||^2
__global__ void k_gm_start(const double* __restrict__ rr, double* __restrict__ g, int ld,
                           double* __restrict__ beta) {
  const double b = sqrt(fmax(*rr, 0.0));
  for (int i = threadIdx.x; i < ld; i += blockDim.x) g[i] = i == 0 ? b : 0.0;
  if (threadIdx.x == 0) *beta = b;
}

// y = triu(H[:k, :k])^-1 g[:k] by back substitution
__global__ void k_gm_solve_y(const double* __restrict__ H, int ld, const double* __restrict__ g,
                             int k, double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[(long long)c * ld + i] * y[c];
    const double d = H[(long long)i * ld + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

// x += sum_{i < k} y[i] Z_i
__global__ void k_gm_xupdate(double* __restrict__ x, const double* __restrict__ Z, long long n,
                             const double* __restrict__ y, int k) {
  __shared__ double ys[256];
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    double a = x[q];
    for (int i = 0; i < k; ++i) a = fma(ys[i], Z[(long long)i * n + q], a);
    x[q] = a;
  }
}

int gm_grid(long long n) {
  const long long b = (n + GT - 1) / GT;
  return (int)(b < 4 * GB ? (b > 0 ? b : 1) : 4 * GB);
}

}  // namespace

#define GCK(x)                                                                  \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      h->err = std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x;      \
      return e_ == cudaErrorMemoryAllocation ? MSTOPO_OUT_OF_MEMORY : MSTOPO_CUDA_ERROR; \
    }                                                                           \
  } while (0)

void gmres_free(GmresWork& g) {
  cudaFree(g.V); cudaFree(g.Z); cudaFree(g.w); cudaFree(g.small); cudaFree(g.partials);
  if (g.h_st) cudaFreeHost(g.h_st);
  g = GmresWork();
}

static mstopo_status gmres_alloc(mstopo_handle* h, int m) {
  GmresWork& g = h->gm;
  if (g.V && g.m == m && g.n == h->n_dof) return MSTOPO_OK;
  gmres_free(g);
  g.m = m;
  g.n = h->n_dof;
  GCK(cudaMalloc(&g.V, (size_t)(m + 1) * g.n * 8));
  GCK(cudaMalloc(&g.Z, (size_t)m * g.n * 8));
  GCK(cudaMalloc(&g.w, (size_t)g.n * 8));
  // H [m][m+1], cs, sn [m], g [m+1], y [m], two Gram-Schmidt columns [m+1] each, ||w||^2,
  // status [3]
  GCK(cudaMalloc(&g.small, (size_t)((m + 1) * m + 2 * m + (m + 1) + m + 2 * (m + 1) + 1 + 3) * 8));
  GCK(cudaMalloc(&g.partials, (size_t)(m + 1) * GB * 8));
  GCK(cudaMallocHost(&g.h_st, 4 * 8));
  return MSTOPO_OK;
}

// Solves systems sys0 .. sys0 + nsys - 1 from x = sv.x (masked f in sv.f) and fills
// sv.h_sc[s] (status, iters, rr = ||f - K x||^2, ff = ||f||^2, repl = cycles).
mstopo_status gmres_run(mstopo_handle* h, int sys0, int nsys) {
  Solver& sv = h->sv;
  const int m = h->p.gmres_restart > 0 ? h->p.gmres_restart : 50;
  mstopo_status st = gmres_alloc(h, m);
  if (st != MSTOPO_OK) return st;
  GmresWork& G = h->gm;
  const long long n = sv.n;
  const int ld = m + 1;
  double* Hm = G.small;
  double* cs = Hm + (size_t)ld * m;
  double* sn = cs + m;
  double* gv = sn + m;
  double* y = gv + ld;
  double* h1 = y + m;
  double* h2 = h1 + ld;
  double* ww = h2 + ld;
  double* dst = ww + 1;   // [3] column status
  const bool mixed = h->p.precision != MSTOPO_FP64;
  const double tol = h->p.tol;
  const int grid = gm_grid(n);
  for (int sl = 0; sl < nsys; ++sl) {
    const int sys = sys0 + sl;
    double* x = sv.x + (size_t)sl * n;
    const double* f = sv.f + (size_t)sl * n;
    const double* E64 = h->d_E64 + (long long)sys * h->n_el;
    FcgScalars& out = sv.h_sc[sl];
    // ||f||^2
    note_launch(), k_gm_dots<<<dim3(GB, 1), GT, 0, h->s>>>(f, f, n, G.partials);
    GCK(cudaGetLastError());
    note_launch(), k_gm_finish<<<1, GT, 0, h->s>>>(G.partials, dst);
    GCK(cudaGetLastError());
    GCK(cudaMemcpyAsync(G.h_st, dst, 8, cudaMemcpyDeviceToHost, h->s));
    GCK(cudaStreamSynchronize(h->s));
    const double ff = G.h_st[0];
    out.ff = ff;
    out.iters = 0;
    out.repl = 0;
    out.active = 0;
    if (!(ff > 0.0) || !std::isfinite(ff)) {
      out.status = ff == 0.0 ? MSTOPO_INVALID_ARG : MSTOPO_NONFINITE;
      out.rr = 0.0;
      if (ff == 0.0) out.ff = 0.0;
      continue;
    }
    const double nf = std::sqrt(ff);
    int it = 0;
    out.status = MSTOPO_MAX_ITER;
    while (true) {
      // true residual r = f - K x into V_0 (unscaled), beta = ||r||
      double* V0 = G.V;
      GCK(launch_matvec_f64(x, G.w, E64, h->d_nmask, h->nelx, h->nely, h->st64, 1, n, h->n_el, h->s));
      note_launch(), k_gm_residual<<<GB, GT, 0, h->s>>>(f, G.w, V0, n, G.partials);
      GCK(cudaGetLastError());
      note_launch(), k_gm_finish<<<1, GT, 0, h->s>>>(G.partials, dst);
      GCK(cudaGetLastError());
      GCK(cudaMemcpyAsync(G.h_st, dst, 8, cudaMemcpyDeviceToHost, h->s));
      GCK(cudaStreamSynchronize(h->s));
      const double rr = G.h_st[0];
      out.rr = rr;
      if (!std::isfinite(rr)) { out.status = MSTOPO_NONFINITE; break; }
      const double beta = std::sqrt(rr);
      if (beta <= tol * nf) { out.status = MSTOPO_OK; break; }
      if (it >= h->p.max_iter) break;
      const int mc = std::min(m, h->p.max_iter - it);
      // g = beta e_1, v_0 = r / beta
      note_launch(), k_gm_start<<<1, 32, 0, h->s>>>(dst, gv, ld, dst + 1);
      GCK(cudaGetLastError());
      note_launch(), k_gm_scale<<<grid, GT, 0, h->s>>>(V0, V0, n, dst + 1);
      GCK(cudaGetLastError());
      int jd = 0;
      for (int j = 0; j < mc; ++j) {
        double* Vj = G.V + (size_t)j * n;
        double* Zj = G.Z + (size_t)j * n;
        // z_j = M^-1 v_j
        if (mixed) {
          GCK(launch_convert_d2f(Vj, sv.r32, n, h->s));
          GCK(precond_apply_f32(h, sv.r32, sv.z32, sys, 1, 0));
          GCK(launch_convert_f2d(sv.z32, Zj, n, h->s));
        } else {
          GCK(precond_apply_f64(h, Vj, Zj, sys, 1, 0));
        }
        // w = K z_j
        GCK(launch_matvec_f64(Zj, G.w, E64, h->d_nmask, h->nelx, h->nely, h->st64, 1, n, h->n_el,
                              h->s, false));
        // two Gram-Schmidt passes against v_0..v_j
        for (int pass = 0; pass < 2; ++pass) {
          double* hc = pass ? h2 : h1;
          note_launch(), k_gm_dots<<<dim3(GB, j + 1), GT, 0, h->s>>>(G.V, G.w, n, G.partials);
          GCK(cudaGetLastError());
          note_launch(), k_gm_finish<<<j + 1, GT, 0, h->s>>>(G.partials, hc);
          GCK(cudaGetLastError());
          note_launch(), k_gm_sub<<<grid, GT, 0, h->s>>>(G.V, G.w, n, hc, j + 1);
          GCK(cudaGetLastError());
        }
        // ||w||^2, column j of H and the rotations, v_{j+1}
        note_launch(), k_gm_dots<<<dim3(GB, 1), GT, 0, h->s>>>(G.w, G.w, n, G.partials);
        GCK(cudaGetLastError());
        note_launch(), k_gm_finish<<<1, GT, 0, h->s>>>(G.partials, ww);
        GCK(cudaGetLastError());
        note_launch(), k_gm_column<<<1, 1, 0, h->s>>>(Hm, ld, j, h1, h2, ww, cs, sn, gv, dst);
        GCK(cudaGetLastError());
        note_launch(), k_gm_scale<<<grid, GT, 0, h->s>>>(G.w, G.V + (size_t)(j + 1) * n, n, dst);
        GCK(cudaGetLastError());
        GCK(cudaMemcpyAsync(G.h_st, dst, 3 * 8, cudaMemcpyDeviceToHost, h->s));
        GCK(cudaStreamSynchronize(h->s));
        ++it;
        jd = j + 1;
        if (!std::isfinite(G.h_st[1])) break;
        if (G.h_st[1] <= tol * nf || G.h_st[2] == 0.0) break;
      }
      // y = H^-1 g, x += Z y
      note_launch(), k_gm_solve_y<<<1, 1, 0, h->s>>>(Hm, ld, gv, jd, y);
      GCK(cudaGetLastError());
      note_launch(), k_gm_xupdate<<<grid, GT, 0, h->s>>>(x, G.Z, n, y, jd);
      GCK(cudaGetLastError());
      out.repl += 1;
    }
    out.iters = it;
  }
  return MSTOPO_OK;
}
