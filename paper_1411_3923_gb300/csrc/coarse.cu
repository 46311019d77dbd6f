// Coarse problem K_c u_c = r_c of the two-level preconditioner (paper Sec. 2.4, coarse
// projection R_c K R_c^T) for coarse spaces too large for an explicit inverse.
//
// K_c is block tridiagonal over lines of coarse nodes (a basis function chi_i psi_j only
// overlaps the agglomerates of the 3x3 coarse neighbours of node i): diagonal blocks A_k and
// sub-diagonal blocks B_k = K_c(line k+1, line k), nb x nb, nb = nodes per line x k_max.
//
// Build (block Cholesky over the lines, FP64, every dense block operation spread over the
// whole GPU; the lines themselves are sequential):
//   S_0 = A_0,  L_k = chol(S_k),  Linv_k = L_k^-1,  C_k = B_k Linv_k^T,
//   S_{k+1} = A_{k+1} - C_k C_k^T,
//   W_k = Linv_k C_{k-1}  (k >= 1),   V_k = Linv_k^T C_k^T  (k <= NL-2).
// Apply (one cooperative launch, FP64):
//   t_k = Linv_k b_k                       all lines at once
//   y_0 = t_0,  y_k = t_k - W_k y_{k-1}       sequential over lines
//   s_k = Linv_k^T y_k                     all lines at once
//   x_{NL-1} = s_{NL-1},  x_k = s_k - V_k x_{k+1}
// which is the forward sweep L y = b and the backward sweep L^T x = y of the block factor
// with the triangular solves inside a line replaced by products with the stored inverses.
// Lines are separated by a grid barrier whose waits are bounded (a timeout is recorded in
// the handle's wait-error word and the host reports MSTOPO_TIMEOUT).
#include "internal.cuh"

#define CB_TILE 32
#define SWEEP_THREADS 256
#define SWEEP_WAIT_LIMIT (1u << 22)

// ------------------------------------------------------------------ dense FP64 products
// C[M][N] = beta C0 + alpha op(A) op(B); row-major operands with leading dimensions.
// op(A) is M x K (TA: A stored K x M), op(B) is K x N (TB: B stored N x K).
// lower != 0: only 32 x 32 output tiles on or below the diagonal are computed.
// C may alias C0 (each element is read and written by one thread); A and B must not
// overlap the written tiles.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha,
                                               const double* __restrict__ A, int lda,
                                               const double* __restrict__ B, int ldb,
                                               double beta, const double* C0, int ldc0,
                                               double* C, int ldc, int lower) {
  const int tm = blockIdx.y, tn = blockIdx.x;
  if (lower && tn > tm) return;
  __shared__ double As[CB_TILE][CB_TILE + 1];   // As[m][k]
  __shared__ double Bs[CB_TILE][CB_TILE + 1];   // Bs[k][n]
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = tm * CB_TILE, n0 = tn * CB_TILE;
  double acc00 = 0.0, acc01 = 0.0, acc10 = 0.0, acc11 = 0.0;
  for (int k0 = 0; k0 < K; k0 += CB_TILE) {
    for (int t = threadIdx.x; t < CB_TILE * CB_TILE; t += blockDim.x) {
      const int a = t / CB_TILE, b = t % CB_TILE;   // b runs along contiguous memory
      if (!TA) {
        const int m = m0 + a, k = k0 + b;
        As[a][b] = (m < M && k < K) ? A[(long long)m * lda + k] : 0.0;
      } else {
        const int k = k0 + a, m = m0 + b;
        As[b][a] = (m < M && k < K) ? A[(long long)k * lda + m] : 0.0;
      }
      if (!TB) {
        const int k = k0 + a, n = n0 + b;
        Bs[a][b] = (k < K && n < N) ? B[(long long)k * ldb + n] : 0.0;
      } else {
        const int n = n0 + a, k = k0 + b;
        Bs[b][a] = (k < K && n < N) ? B[(long long)n * ldb + k] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < CB_TILE; ++k) {
      const double a0 = As[2 * ty][k], a1 = As[2 * ty + 1][k];
      const double b0 = Bs[k][2 * tx], b1 = Bs[k][2 * tx + 1];
      acc00 = fma(a0, b0, acc00);
      acc01 = fma(a0, b1, acc01);
      acc10 = fma(a1, b0, acc10);
      acc11 = fma(a1, b1, acc11);
    }
    __syncthreads();
  }
  auto put = [&](int i, int j, double a) {
    const int m = m0 + 2 * ty + i, n = n0 + 2 * tx + j;
    if (m < M && n < N) {
      double v = alpha * a;
      if (beta != 0.0) v = fma(beta, C0[(long long)m * ldc0 + n], v);
      C[(long long)m * ldc + n] = v;
    }
  };
  put(0, 0, acc00);
  put(0, 1, acc01);
  put(1, 0, acc10);
  put(1, 1, acc11);
}

template <bool TA, bool TB>
static cudaError_t dgemm(int M, int N, int K, double alpha, const double* A, int lda,
                         const double* B, int ldb, double beta, const double* C0, int ldc0,
                         double* C, int ldc, int lower, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid(cdiv(N, CB_TILE), cdiv(M, CB_TILE));
  note_launch(), k_dgemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta,
                                                      C0, ldc0, C, ldc, lower);
  return cudaGetLastError();
}

// ------------------------------------------------------------- blocked Cholesky panel
// Panel p of the lower Cholesky factor of S (nb x nb, row-major, lower triangle used):
// every CTA factors the 32 x 32 diagonal block in shared memory (the block in S stays
// unfactored, so CTAs that start late still read the original); CTA 0 stores the factored
// block in Ld[p] and CTA b > 0 overwrites row block p + b of the panel with S_ip L_pp^-T.
// A non-positive or non-finite pivot records 1 + (row_base + its row) in *status (first
// failure kept) and is replaced by 1 so that the factorisation still ends.
__global__ void __launch_bounds__(256) k_chol_panel(double* __restrict__ S, int nb, int p,
                                                    double* __restrict__ Ld, int row_base,
                                                    int* __restrict__ status) {
  __shared__ double D[CB_TILE][CB_TILE + 1];
  __shared__ double dinv[CB_TILE];   // 1 / L_jj, one FP64 division per pivot
  __shared__ int fail;
  const int c0 = p * CB_TILE, bs = min(CB_TILE, nb - c0);
  for (int t = threadIdx.x; t < CB_TILE * CB_TILE; t += blockDim.x) {
    const int i = t / CB_TILE, j = t % CB_TILE;
    D[i][j] = (i < bs && j <= i) ? S[(long long)(c0 + i) * nb + c0 + j] : 0.0;
  }
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < bs; ++j) {
    if (threadIdx.x == 0) {
      double d = D[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        if (!fail) fail = 1 + j;
        d = 1.0;
      }
      const double l = sqrt(d);
      D[j][j] = l;
      dinv[j] = 1.0 / l;
    }
    __syncthreads();
    const double inv = dinv[j];
    if ((int)threadIdx.x > j && (int)threadIdx.x < bs) D[threadIdx.x][j] *= inv;
    __syncthreads();
    for (int t = threadIdx.x; t < CB_TILE * CB_TILE; t += blockDim.x) {
      const int i = t / CB_TILE, l = t % CB_TILE;
      if (l > j && l <= i && i < bs) D[i][l] = fma(-D[i][j], D[l][j], D[i][l]);
    }
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    double* Lp = Ld + (long long)p * CB_TILE * CB_TILE;
    for (int t = threadIdx.x; t < CB_TILE * CB_TILE; t += blockDim.x) {
      const int i = t / CB_TILE, j = t % CB_TILE;
      Lp[t] = (i < bs && j <= i) ? D[i][j] : 0.0;
    }
    if (threadIdx.x == 0 && fail) atomicCAS(status, 0, row_base + c0 + fail);
    return;
  }
  const int r0 = (p + (int)blockIdx.x) * CB_TILE;
  const int rb = min(CB_TILE, nb - r0);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int rr = w; rr < rb; rr += blockDim.x / 32) {
    double* row = S + (long long)(r0 + rr) * nb + c0;
    double sv = lane < bs ? row[lane] : 0.0;
    double x = 0.0;
    for (int j = 0; j < bs; ++j) {     // x L_pp^T = s, column by column
      const double xj = __shfl_sync(0xffffffffu, sv * dinv[j], j);
      if (lane == j) x = xj;
      if (lane > j) sv = fma(-xj, D[lane][j], sv);
    }
    if (lane < bs) row[lane] = x;
  }
}

// ---------------------------------------------------------- inverse of a lower factor
// Linv = L^-1 and its transpose LinvT, TI_W columns per CTA.  L is held as the off-diagonal
// 32 x 32 blocks of S and the factored diagonal blocks Ld[q].  Rows are processed in the
// 32-row blocks of the factor, from the block holding the slab's first column down; the slab
// (rows from that block on, TI_W columns) lives in shared memory.
#define TI_W 4
__global__ void __launch_bounds__(128) k_tri_inv(const double* __restrict__ S,
                                                 const double* __restrict__ Ld, int nb,
                                                 double* __restrict__ Linv,
                                                 double* __restrict__ LinvT) {
  extern __shared__ double X[];                 // [nb - rbase][TI_W]
  __shared__ double Lb[CB_TILE][CB_TILE + 1];
  __shared__ double Lbi[CB_TILE];   // 1 / Lb[i][i]
  __shared__ double Rs[CB_TILE][TI_W];
  const int c0 = blockIdx.x * TI_W;
  const int cw = min(TI_W, nb - c0);
  const int rbase = (c0 / CB_TILE) * CB_TILE;
  for (int r0 = rbase; r0 < nb; r0 += CB_TILE) {
    const int rb = min(CB_TILE, nb - r0);
    {
      // Rs = e - L(r0 block, [rbase, r0)) X  (off-diagonal blocks of L)
      const int r = threadIdx.x / TI_W, j = threadIdx.x % TI_W;
      double acc = (r0 + r == c0 + j) ? 1.0 : 0.0;
      if (r < rb && j < cw) {
        const double* Lr = S + (long long)(r0 + r) * nb;
        for (int m = rbase; m < r0; ++m) acc = fma(-Lr[m], X[(m - rbase) * TI_W + j], acc);
      }
      Rs[r][j] = acc;
    }
    const double* Dq = Ld + (long long)(r0 / CB_TILE) * CB_TILE * CB_TILE;
    for (int t = threadIdx.x; t < CB_TILE * CB_TILE; t += blockDim.x) {
      const int i = t / CB_TILE, l = t % CB_TILE;
      Lb[i][l] = (i < rb && l < rb) ? Dq[t] : (i == l ? 1.0 : 0.0);
    }
    if (threadIdx.x < CB_TILE) {
      const int i = threadIdx.x;
      Lbi[i] = 1.0 / ((i < rb) ? Dq[i * CB_TILE + i] : 1.0);
    }
    __syncthreads();
    {
      const int lane = threadIdx.x & 31, j = threadIdx.x >> 5;   // warp j solves column j
      double sv = Rs[lane][j], x = 0.0;
      for (int m = 0; m < rb; ++m) {
        const double xm = __shfl_sync(0xffffffffu, sv * Lbi[m], m);
        if (lane == m) x = xm;
        if (lane > m) sv = fma(-xm, Lb[lane][m], sv);
      }
      if (lane < rb) X[(r0 - rbase + lane) * TI_W + j] = x;
    }
    __syncthreads();
  }
  for (long long t = threadIdx.x; t < (long long)nb * cw; t += blockDim.x) {
    const int r = (int)(t / cw), j = (int)(t % cw);
    const double v = r >= c0 ? X[(r - rbase) * TI_W + j] : 0.0;
    Linv[(long long)r * nb + c0 + j] = v;
    LinvT[(long long)(c0 + j) * nb + r] = v;
  }
}

// Factor the block-tridiagonal coarse matrix (A: [NL][nb][nb], B: [NL-1][nb][nb]) into
// Linv, LinvT, W, V ([NL][nb][nb] each; W_0 and V_{NL-1} are left untouched).
// Workspace: S (nb x nb), Cw (2 x nb x nb), Ld (ceil(nb/32) x 32 x 32).
// status: device int, 0 or 1 + the first failing row (line * nb + row in the line).
cudaError_t coarse_bt_factor(const double* A, const double* B, int nb, int NL, double* Linv,
                             double* LinvT, double* W, double* V, double* S, double* Cw,
                             double* Ld, int* status, cudaStream_t s) {
  const long long nn = (long long)nb * nb;
  const int np = (nb + CB_TILE - 1) / CB_TILE;
  const size_t ti_smem = (size_t)nb * TI_W * sizeof(double);
  if (ti_smem > 48 * 1024) {
    cudaError_t e = smem_limit_max<k_tri_inv>();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e;
  for (int k = 0; k < NL; ++k) {
    const double* Ak = A + k * nn;
    double* Ccur = Cw + (k & 1) * nn;          // C_k
    double* Cprev = Cw + ((k + 1) & 1) * nn;   // C_{k-1}
    // S = A_k - C_{k-1} C_{k-1}^T  (lower tiles)
    if (k == 0) {
      e = cudaMemcpyAsync(S, Ak, nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    } else {
      e = dgemm<false, true>(nb, nb, nb, -1.0, Cprev, nb, Cprev, nb, 1.0, Ak, nb, S, nb, 1, s);
    }
    if (e != cudaSuccess) return e;
    // S := chol(S), blocked by 32-column panels
    for (int p = 0; p < np; ++p) {
      note_launch(), k_chol_panel<<<np - p, 256, 0, s>>>(S, nb, p, Ld, k * nb, status);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      const int t0 = (p + 1) * CB_TILE;
      if (t0 < nb) {
        double* P = S + (long long)t0 * nb + p * CB_TILE;
        e = dgemm<false, true>(nb - t0, nb - t0, CB_TILE, -1.0, P, nb, P, nb, 1.0,
                               S + (long long)t0 * nb + t0, nb, S + (long long)t0 * nb + t0, nb,
                               1, s);
        if (e != cudaSuccess) return e;
      }
    }
    double* Li = Linv + k * nn;
    double* LiT = LinvT + k * nn;
    note_launch(), k_tri_inv<<<cdiv(nb, TI_W), 128, ti_smem, s>>>(S, Ld, nb, Li, LiT);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (k > 0) {   // W_k = Linv_k C_{k-1}
      e = dgemm<false, false>(nb, nb, nb, 1.0, Li, nb, Cprev, nb, 0.0, nullptr, 0, W + k * nn, nb, 0, s);
      if (e != cudaSuccess) return e;
    }
    if (k + 1 < NL) {
      // C_k = B_k Linv_k^T,  V_k = Linv_k^T C_k^T
      e = dgemm<false, true>(nb, nb, nb, 1.0, B + k * nn, nb, Li, nb, 0.0, nullptr, 0, Ccur, nb, 0, s);
      if (e != cudaSuccess) return e;
      e = dgemm<true, true>(nb, nb, nb, 1.0, Li, nb, Ccur, nb, 0.0, nullptr, 0, V + k * nn, nb, 0, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------ cooperative sweeps
// Grid barrier on a monotone arrival counter (reset to 0 before the launch): barrier number
// g completes when the counter reaches g * gridDim.x.  The wait is bounded; after a timeout
// (or once any wait has timed out) every later barrier returns at once.
__device__ __forceinline__ void sweep_sync(unsigned int* bar, unsigned int& target, int* err) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    unsigned int it = 0;
    while (true) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (*(volatile int*)err != 0) break;
      if (++it > SWEEP_WAIT_LIMIT) {
        atomicExch(err, (int)MSTOPO_TIMEOUT);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
}

struct SweepArgs {
  const double *Linv, *LinvT, *W, *V;   // [nsys][NL][nb][nb], system s at s * NL * nb * nb
  const int* s2o;                       // [NL*nb] coarse unknown of each line slot, -1 = none
  const double* rc;                     // [nsys][Nt]
  double* uc;                           // [nsys][Nt]
  double *y, *x;                        // [nsys][NL][nb]
  unsigned int* bar;
  int* err;
  int nb, NL, Nt, nsys;
  int stall;                            // test injection: the first barrier cannot complete
};

// Sum over the 32 lanes of a warp, all lanes receive it.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp index with consecutive indices on different CTAs (spreads a line over the SMs).
__device__ __forceinline__ int sweep_warp() { return (threadIdx.x >> 5) * gridDim.x + blockIdx.x; }

// Dense-row phase: out[s][line][i] = sum_{c in range} M_s,line[i][c] v[s][line][c] for
// every (system, line, row), one warp each.  LOWER: c <= i (Linv), else c >= i (LinvT).
template <bool LOWER>
__device__ __forceinline__ void sweep_diag(const double* __restrict__ M, const double* v,
                                           double* out, int nb, int NL, int nsys) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nn = (long long)nb * nb;
  const long long rows = (long long)NL * nb;
  for (long long R = sweep_warp(); R < (long long)nsys * rows; R += nwarps) {
    const long long sl = R / nb;                 // system * NL + line
    const int i = (int)(R % nb);
    const double* row = M + sl * nn + (long long)i * nb;
    const double* vl = v + sl * nb;
    const int c_lo = LOWER ? 0 : i, c_hi = LOWER ? i + 1 : nb;
    double acc = 0.0;
#pragma unroll 4
    for (int c = c_lo + lane; c < c_hi; c += 32) acc = fma(row[c], __ldcg(vl + c), acc);
    acc = warp_sum(acc);
    if (lane == 0) out[R] = acc;
  }
}

// One line of a sequential sweep: z_k[i] -= M_k[i] . z_prev for every (system, row) pair,
// one warp per pair (at most one pair per warp); the warp's matrix row is loaded into
// registers before the barrier that publishes z_prev.
#define SWEEP_PF 20   // register-held row entries per lane (nb <= 640)
__device__ __forceinline__ void sweep_load_row(const double* __restrict__ M, long long sys_stride,
                                               long long k_off, int nb, int pair, int npairs,
                                               double (&mr)[SWEEP_PF]) {
  const int lane = threadIdx.x & 31;
  const int sys = pair / nb, row = pair % nb;
  const double* Mr = M + (long long)sys * sys_stride + k_off + (long long)row * nb;
#pragma unroll
  for (int q = 0; q < SWEEP_PF; ++q) {
    const int c = lane + 32 * q;
    mr[q] = (pair < npairs && c < nb) ? Mr[c] : 0.0;
  }
}

__device__ __forceinline__ void sweep_row(const double (&mr)[SWEEP_PF], const double* zprev,
                                          double* zk, int nb) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < SWEEP_PF; ++q) {
    const int c = lane + 32 * q;
    if (c < nb) acc = fma(mr[q], __ldcg(zprev + c), acc);
  }
  acc = warp_sum(acc);
  if (lane == 0) *zk = __ldcg(zk) - acc;
}

__global__ void __launch_bounds__(SWEEP_THREADS, 2) k_coarse_sweep(SweepArgs a) {
  const int nb = a.nb, NL = a.NL, ns = a.nsys;
  const long long nn = (long long)nb * nb, lines = (long long)NL * nb;
  const long long sys_stride = (long long)NL * nn;
  unsigned int target = a.stall ? 1u : 0u;   // an injected stall waits for one arrival too many
  // 0. gather r_c into line order (padding slots 0)
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ns * lines;
       t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / lines);
    const int o = a.s2o[t % lines];
    a.x[t] = o >= 0 ? a.rc[(long long)s * a.Nt + o] : 0.0;
  }
  sweep_sync(a.bar, target, a.err);
  // 1. t_k = Linv_k b_k
  sweep_diag<true>(a.Linv, a.x, a.y, nb, NL, ns);
  // 2. forward: y_k = t_k - W_k y_{k-1}
  const int pair = sweep_warp(), npairs = ns * nb;
  const int psys = pair / nb, prow = pair % nb;
  for (int k = 1; k < NL; ++k) {
    double mr[SWEEP_PF];
    sweep_load_row(a.W, sys_stride, k * nn, nb, pair, npairs, mr);
    sweep_sync(a.bar, target, a.err);
    if (pair < npairs)
      sweep_row(mr, a.y + psys * lines + (long long)(k - 1) * nb,
                a.y + psys * lines + (long long)k * nb + prow, nb);
  }
  sweep_sync(a.bar, target, a.err);
  // 3. s_k = Linv_k^T y_k
  sweep_diag<false>(a.LinvT, a.y, a.x, nb, NL, ns);
  // 4. backward: x_k = s_k - V_k x_{k+1}
  for (int k = NL - 2; k >= 0; --k) {
    double mr[SWEEP_PF];
    sweep_load_row(a.V, sys_stride, k * nn, nb, pair, npairs, mr);
    sweep_sync(a.bar, target, a.err);
    if (pair < npairs)
      sweep_row(mr, a.x + psys * lines + (long long)(k + 1) * nb,
                a.x + psys * lines + (long long)k * nb + prow, nb);
  }
  sweep_sync(a.bar, target, a.err);
  // 5. scatter back to the agglomerate order
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ns * lines;
       t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / lines);
    const int o = a.s2o[t % lines];
    if (o >= 0) a.uc[(long long)s * a.Nt + o] = __ldcg(a.x + t);
  }
}

// Largest line width the sweep kernel handles for nsys systems (one register-held row of
// one system per warp).
int coarse_sweep_max_nb(int grid, int nsys) {
  const int nwarps = grid * SWEEP_THREADS / 32;
  return std::min(32 * SWEEP_PF, nwarps / std::max(nsys, 1));
}

// Grid of the cooperative sweep: every CTA co-resident, at most 2 per SM.
int coarse_sweep_grid() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_sweep, SWEEP_THREADS, 0) !=
      cudaSuccess)
    return 0;
  return sms * std::min(per_sm, 2);
}

// uc[s] = K_c,s^-1 rc[s] for nsys systems through their block factors (matrices of system s
// at offset s * NL * nb * nb).  err: the handle's wait-error word; bar: a device counter
// owned by the caller (reset here).  One cooperative launch.
cudaError_t coarse_bt_apply(const double* Linv, const double* LinvT, const double* W,
                            const double* V, const int* s2o, int nb, int NL, int Nt,
                            const double* rc, double* uc, int nsys, double* ywork,
                            double* xwork, unsigned int* bar, int* err, int grid,
                            int stall, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  SweepArgs a;
  a.stall = stall;
  a.Linv = Linv; a.LinvT = LinvT; a.W = W; a.V = V; a.s2o = s2o; a.rc = rc; a.uc = uc;
  a.y = ywork; a.x = xwork; a.bar = bar; a.err = err; a.nb = nb; a.NL = NL; a.Nt = Nt;
  a.nsys = nsys;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(SWEEP_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&cfg, k_coarse_sweep, a);
}
