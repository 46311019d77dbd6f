// Two-level preconditioner with a spectral MsFEM coarse space (paper Sec. 2.4, 2.4.1,
// 2.4.2, 3.2, 5.3).
//
// Build (once per design):
//   1. agglomerate de-duplication (Sec. 2.4.1): every agglomerate omega_i (the 2H x 2H
//      elements around coarse node y_i, clipped by the mesh) is hashed over its moduli, its
//      Dirichlet mask and which of its four box sides lie inside the mesh (those form the
//      artificial boundary of its patch); agglomerates with equal hashes whose boxes then
//      compare equal entry by entry share one "type" and therefore one eigenbasis and one
//      patch factor.  The paper observes three unique agglomerates for a periodic
//      double-clamped beam; the key generalises that to any design.
//   2. per type, the agglomerate's Neumann matrix K_w (its own elements only, physical
//      Dirichlet DOFs kept) is assembled block-tridiagonally by node rows; K_w + s diag(K_w)
//      is factorised (FP64) and block subspace iteration with Rayleigh-Ritz finds the
//      smallest eigenpairs of K_w psi = lambda diag(K_w) psi (Sec. 2.4 and the diagonal
//      weighting of Sec. 3.2), psi^T diag(K_w) psi = 1.  Either n_eig pairs or those below
//      lambda_Omega (capped) are kept.
//   3. the coarse basis phi_ij = chi_i psi_j with chi_i the bilinear hat of y_i (a partition
//      of unity with |grad chi| <= 1/H); K_c = R_c K R_c^T (Eq. coarse_projection) is
//      assembled element by element for each pair of overlapping agglomerates (3x3 coarse
//      neighbours), factorised block-tridiagonally by coarse-node lines in FP64, and
//      inverted explicitly (dense FP64) for a one-GEMV coarse solve.
//   4. per type, the overlapping patch matrix K_i = K restricted to the nodes of omega_i off
//      its artificial boundary (zero Dirichlet there, physical conditions kept) is factorised
//      block-tridiagonally (FP64, plus an FP32 copy for the MIXED solver).
// Apply (every Krylov iteration): z = R_c^T K_c^-1 R_c r + sum_i R_i^T K_i^-1 R_i r
// (two-level additive Schwarz, cited in Sec. 2.4.2), with deterministic gathers (no atomics).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include <cooperative_groups.h>

#include "blocktri.cuh"

namespace cg = cooperative_groups;

#define PC_THREADS 256
#define SOLVE_THREADS 320   // 160 rows x 2 threads per pass covers nb = 2(2H+1) up to H = 39
#define EIG_CL 4            // CTAs per agglomerate type in the eigen-solve (subspace columns split)
#define PATCH_COLS 16       // right-hand-side columns per CTA (patches x systems), at most
#define PATCH_COLS_F64 4    // the same for the FP64 patch solves
#define EIG_MAX_SWEEPS 80
#define EIG_TOL 1e-7
#define EIG_SHIFT 1e-5

struct K0P { double k[64]; };

// ------------------------------------------------------------------------------ hashing
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Artificial sides of agglomerate (I, J)'s box: bit 0 left, 1 right, 2 bottom, 3 top, set
// when that side lies strictly inside the mesh (a side on or beyond the mesh edge keeps the
// physical conditions).  Two boxes with equal moduli and masks but different sides have
// different patch matrices.
__host__ __device__ __forceinline__ int agg_sides(int I, int J, int H, int nelx, int nely) {
  const int ox = (I - 1) * H, oy = (J - 1) * H;
  return (ox > 0 ? 1 : 0) | (ox + 2 * H < nelx ? 2 : 0) | (oy > 0 ? 4 : 0) | (oy + 2 * H < nely ? 8 : 0);
}

// Hash of the moduli of realisation `salt` over the agglomerate (XOR-accumulated over the
// realisations, so equal hashes mean equal boxes in every realisation) and, once
// (with_mask), of its Dirichlet mask and its artificial sides.
__global__ void k_hash_agg(const double* __restrict__ E, const uint8_t* __restrict__ nmask,
                           int nelx, int nely, int H, int ncx, int salt, int with_mask,
                           unsigned long long* __restrict__ hash) {
  const int i = blockIdx.x;
  const int I = i % (ncx + 1), J = i / (ncx + 1);
  const int ox = (I - 1) * H, oy = (J - 1) * H;
  const int ne = 2 * H, nn = 2 * H + 1;
  const unsigned long long sk = mix64(0x5BD1E995ull + (unsigned long long)salt);
  unsigned long long h1 = 0, h2 = 0;
  if (with_mask && threadIdx.x == 0) {
    const unsigned long long sd = (unsigned long long)agg_sides(I, J, H, nelx, nely);
    h1 ^= mix64((sd + 0x3C6EF372ull) ^ 0xA54FF53A5F1D36F1ull);
    h2 ^= mix64(sd * 0x510E527FADE682D1ull + 0x9B05688C2B3E6C1Full);
  }
  for (int t = threadIdx.x; t < ne * ne; t += blockDim.x) {
    int ex = ox + t % ne, ey = oy + t / ne;
    unsigned long long v = 0xFFFFFFFFFFFFFFFFull;
    if (ex >= 0 && ex < nelx && ey >= 0 && ey < nely)
      v = (unsigned long long)__double_as_longlong(E[(long long)ey * nelx + ex]);
    h1 ^= mix64(v ^ mix64(((unsigned long long)t * 2 + 1) ^ sk));
    h2 ^= mix64(v * 0xD6E8FEB86659FD93ull + mix64((unsigned long long)t + 0x1234567ull + sk));
  }
  for (int t = threadIdx.x; with_mask && t < nn * nn; t += blockDim.x) {
    int x = ox + t % nn, y = oy + t / nn;
    unsigned long long v = 7;
    if (x >= 0 && x <= nelx && y >= 0 && y <= nely) v = nmask[(long long)y * (nelx + 1) + x];
    h1 ^= mix64((v + 11) ^ mix64(((unsigned long long)t << 20) + 3));
    h2 ^= mix64((v + 101) * 0x9E3779B97F4A7C15ull ^ ((unsigned long long)t << 7));
  }
  atomicXor(&hash[2 * i], h1);
  atomicXor(&hash[2 * i + 1], h2);
}

// Entry-by-entry check of a hash match: agglomerate i against the representative rep of its
// type, over the moduli of every realisation (bit patterns, and which elements lie inside
// the mesh), the Dirichlet mask of the box nodes and the artificial sides.  bad[i] = 1 on
// any difference (a hash collision); the host then gives i a type of its own.
__global__ void k_verify_agg(const double* __restrict__ E, long long e_stride, int nsys,
                             const uint8_t* __restrict__ nmask, int nelx, int nely, int H,
                             int ncx, const int* __restrict__ type_of,
                             const int* __restrict__ rep_of_type, int* __restrict__ bad) {
  const int i = blockIdx.x;
  const int ia = rep_of_type[type_of[i]];
  if (ia == i) {
    if (threadIdx.x == 0) bad[i] = 0;
    return;
  }
  const int I = i % (ncx + 1), J = i / (ncx + 1);
  const int Ia = ia % (ncx + 1), Ja = ia / (ncx + 1);
  const int ox = (I - 1) * H, oy = (J - 1) * H, oxa = (Ia - 1) * H, oya = (Ja - 1) * H;
  const int ne = 2 * H, nn = 2 * H + 1;
  int diff = agg_sides(I, J, H, nelx, nely) != agg_sides(Ia, Ja, H, nelx, nely);
  for (int t = threadIdx.x; !diff && t < ne * ne; t += blockDim.x) {
    const int ex = ox + t % ne, ey = oy + t / ne, fx = oxa + t % ne, fy = oya + t / ne;
    const bool in1 = ex >= 0 && ex < nelx && ey >= 0 && ey < nely;
    const bool in2 = fx >= 0 && fx < nelx && fy >= 0 && fy < nely;
    if (in1 != in2) { diff = 1; break; }
    if (!in1) continue;
    for (int k = 0; k < nsys; ++k)
      if (__double_as_longlong(E[k * e_stride + (long long)ey * nelx + ex]) !=
          __double_as_longlong(E[k * e_stride + (long long)fy * nelx + fx])) { diff = 1; break; }
  }
  for (int t = threadIdx.x; !diff && t < nn * nn; t += blockDim.x) {
    const int x = ox + t % nn, y = oy + t / nn, xa = oxa + t % nn, ya = oya + t / nn;
    const bool in1 = x >= 0 && x <= nelx && y >= 0 && y <= nely;
    const bool in2 = xa >= 0 && xa <= nelx && ya >= 0 && ya <= nely;
    if (in1 != in2) { diff = 1; break; }
    if (in1 && nmask[(long long)y * (nelx + 1) + x] != nmask[(long long)ya * (nelx + 1) + xa]) diff = 1;
  }
  diff = __syncthreads_or(diff);
  if (threadIdx.x == 0) bad[i] = diff ? 1 : 0;
}

// ----------------------------------------------------------------------------- assembly
// Block-tridiagonal assembly of a box operator.  Box node (a, b), a, b in [0, N), is global
// node (ox + a, oy + b); line = b, DOF in line = 2a + c.  Only elements with
// ex in [ex0, ex1), ey in [ey0, ey1) and inside the mesh contribute.  A DOF is free when its
// node is in the mesh and not Dirichlet; other rows/columns are identity.
struct BoxSpec { int ox, oy, N, ex0, ex1, ey0, ey1; };

// The box is the agglomerate's (2H+1)^2 node box with lower-left node ((I-1)H, (J-1)H);
// elements of the agglomerate only ([(I-1)H, (I+1)H) in each direction).  artificial = 1
// (patch matrices): box-edge nodes strictly inside the mesh form the artificial boundary and
// are Dirichlet; box-edge nodes on the mesh boundary keep the physical conditions.
__global__ void k_assemble_box(const double* __restrict__ E, const uint8_t* __restrict__ nmask,
                               int nelx, int nely, const int* __restrict__ rep, int H, int ncx,
                               int artificial, K0P K0, double* __restrict__ A,
                               double* __restrict__ B, uint8_t* __restrict__ freeo) {
  // blockIdx.x = type, blockIdx.y = line
  const int type = blockIdx.x, line = blockIdx.y;
  const int ia = rep[type];
  const int I = ia % (ncx + 1), J = ia / (ncx + 1);
  const int N = 2 * H + 1;
  const int ox = (I - 1) * H, oy = (J - 1) * H;
  const int ex0 = ox, ex1 = ox + 2 * H, ey0 = oy, ey1 = oy + 2 * H;
  const int nb = 2 * N;
  const long long nn = (long long)nb * nb;
  double* Ak = A + ((long long)type * N + line) * nn;
  double* Bk = line > 0 ? B + ((long long)type * (N - 1) + line - 1) * nn : nullptr;
  auto dof_free = [&](int a, int b, int c) -> bool {
    int x = ox + a, y = oy + b;
    if (a < 0 || a >= N || b < 0 || b >= N) return false;
    if (x < 0 || x > nelx || y < 0 || y > nely) return false;
    if (artificial && ((a == 0 && x > 0) || (a == N - 1 && x < nelx) || (b == 0 && y > 0) ||
                       (b == N - 1 && y < nely)))
      return false;
    return !((nmask[(long long)y * (nelx + 1) + x] >> c) & 1);
  };
  for (int r = threadIdx.x; r < nb; r += blockDim.x) {
    for (int c = 0; c < nb; ++c) {
      Ak[(long long)r * nb + c] = 0.0;
      if (Bk) Bk[(long long)r * nb + c] = 0.0;
    }
    const int a = r >> 1, cr = r & 1;
    const bool rf = dof_free(a, line, cr);
    freeo[((long long)type * N + line) * nb + r] = rf ? 1 : 0;
    if (!rf) {
      Ak[(long long)r * nb + r] = 1.0;
      continue;
    }
    const int gx = ox + a, gy = oy + line;
    // the four elements around the node; local node order (0,0),(1,0),(1,1),(0,1)
    for (int q = 0; q < 4; ++q) {
      const int ex = gx - 1 + (q & 1), ey = gy - 1 + (q >> 1);
      if (ex < ex0 || ex >= ex1 || ey < ey0 || ey >= ey1) continue;
      if (ex < 0 || ex >= nelx || ey < 0 || ey >= nely) continue;
      const double Ee = E[(long long)ey * nelx + ex];
      const int lx = gx - ex, ly = gy - ey;   // node position inside the element
      const int la = ly == 0 ? (lx == 0 ? 0 : 1) : (lx == 1 ? 2 : 3);
      for (int lb = 0; lb < 4; ++lb) {
        const int mx = ex + ((lb == 1 || lb == 2) ? 1 : 0), my = ey + (lb >= 2 ? 1 : 0);
        const int ma = mx - ox, mb = my - oy;
        for (int cc = 0; cc < 2; ++cc) {
          if (!dof_free(ma, mb, cc)) continue;
          const double v = Ee * K0.k[(2 * la + cr) * 8 + 2 * lb + cc];
          const int col = 2 * ma + cc;
          if (mb == line) Ak[(long long)r * nb + col] += v;
          else if (mb == line - 1) Bk[(long long)r * nb + col] += v;
          // mb == line + 1 belongs to A(line, line+1) = B_line^T, written by the next line
        }
      }
    }
  }
}

// ------------------------------------------------------------------------ factorisation
// systems [0, split) are factorised with diagonal shift s_lo, the others with s_hi
#define BT_MAX_NB 1024   // largest block the one-CTA factor handles (inverse diagonal in shared memory)
__global__ void k_bt_factor(const double* __restrict__ A, const double* __restrict__ B,
                            const uint8_t* __restrict__ freem, double s_lo, double s_hi,
                            int split, int nb, int NL, double* __restrict__ Linv,
                            double* __restrict__ C, double* __restrict__ Swork,
                            int* __restrict__ status) {
  __shared__ int sh_fail;
  __shared__ double dinv[BT_MAX_NB];
  const long long nn = (long long)nb * nb;
  const int sys = blockIdx.x;
  const double shift = sys < split ? s_lo : s_hi;
  int f = bt_factor(A + sys * NL * nn, B + sys * (NL - 1) * nn,
                    freem ? freem + (long long)sys * NL * nb : nullptr, shift, nb, NL,
                    Linv + sys * NL * nn, C + sys * (NL - 1) * nn, Swork + sys * nn, &sh_fail, dinv);
  if (threadIdx.x == 0) status[sys] = f;
}

// Two-sided elimination of the patch matrices (the middle line m = H meets both halves):
// lines 0..NLr-1 of the line-reversed systems, A'_j = A_{NL-1-j},
// B'_j = A'_{j+1,j} = (A_{NL-1-j,NL-2-j})^T = B_{NL-2-j}^T, free'_j = free_{NL-1-j}.
__global__ void k_reverse_lines(const double* __restrict__ A, const double* __restrict__ B,
                                const uint8_t* __restrict__ freem, int NL, int NLr, int nb,
                                double* __restrict__ Ar, double* __restrict__ Br,
                                uint8_t* __restrict__ fr) {
  const int sys = blockIdx.x, j = blockIdx.y, l = NL - 1 - j;
  const long long nn = (long long)nb * nb;
  const double* As = A + ((long long)sys * NL + l) * nn;
  double* Ad = Ar + ((long long)sys * NLr + j) * nn;
  for (long long t = threadIdx.x; t < nn; t += blockDim.x) Ad[t] = As[t];
  if (j + 1 < NLr) {
    const double* Bs = B + ((long long)sys * (NL - 1) + NL - 2 - j) * nn;
    double* Bd = Br + ((long long)sys * (NLr - 1) + j) * nn;
    for (long long t = threadIdx.x; t < nn; t += blockDim.x) {
      const long long i = t / nb, c = t % nb;
      Bd[t] = Bs[c * nb + i];
    }
  }
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    fr[((long long)sys * NLr + j) * nb + i] = freem[((long long)sys * NL + l) * nb + i];
}

// The middle line's Schur complement M = A_m (+ shift) - C_{m-1} C_{m-1}^T - C'_{m-1} C'_{m-1}^T
// (C = B L^-T of the top-down factor and of the line-reversed one, m = (NL - 1) / 2), its
// Cholesky factor in place and Lm = L_M^-1.  status[sys] = 0 or 1 + the failing pivot.
__global__ void k_twist_middle(const double* __restrict__ A, const double* __restrict__ Ct,
                               const double* __restrict__ Cr, const uint8_t* __restrict__ freem,
                               double shift, int NL, int NLr, int nb, double* __restrict__ S,
                               double* __restrict__ Lm, int* __restrict__ status) {
  __shared__ int sh_fail;
  __shared__ double dinv[BT_MAX_NB];
  const int sys = blockIdx.x, m = (NL - 1) / 2;
  const long long nn = (long long)nb * nb;
  const double* Am = A + ((long long)sys * NL + m) * nn;
  const double* C0 = Ct + ((long long)sys * (NL - 1) + m - 1) * nn;
  const double* C1 = Cr + ((long long)sys * (NLr - 1) + m - 1) * nn;
  const uint8_t* fm = freem + ((long long)sys * NL + m) * nb;
  double* Sm = S + sys * nn;
  for (long long t = threadIdx.x; t < nn; t += blockDim.x) {
    const int i = (int)(t / nb), l = (int)(t % nb);
    double v = Am[t];
    if (i == l && fm[i]) v *= (1.0 + shift);
    if (l <= i) {
      double s0 = 0.0, s1 = 0.0;
      for (int q = 0; q < nb; ++q) {
        s0 = fma(C0[(long long)i * nb + q], C0[(long long)l * nb + q], s0);
        s1 = fma(C1[(long long)i * nb + q], C1[(long long)l * nb + q], s1);
      }
      v -= s0;
      v -= s1;
    }
    Sm[t] = v;
  }
  __syncthreads();
  const int f = bt_chol_inplace(Sm, nb, &sh_fail, dinv);
  bt_tri_inverse(Sm, dinv, Lm + sys * nn, nb);
  if (threadIdx.x == 0) status[sys] = f;
}

// ------------------------------------------------------------------------------ eigen
// Small dense helpers (thread 0 only).  Cyclic Jacobi for a symmetric q x q matrix:
// on exit A is (numerically) diagonal and V holds the eigenvectors as columns.
__device__ void jacobi_eig(double* A, double* V, int q) {
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) V[i * q + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) {
        double v = A[i * q + j] * A[i * q + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < q - 1; ++p)
      for (int r = p + 1; r < q; ++r) {
        double apr = A[p * q + r];
        if (fabs(apr) < 1e-300) continue;
        double app = A[p * q + p], arr = A[r * q + r];
        double theta = (arr - app) / (2.0 * apr);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < q; ++k) {   // columns p, r
          double akp = A[k * q + p], akr = A[k * q + r];
          A[k * q + p] = c * akp - s * akr;
          A[k * q + r] = s * akp + c * akr;
        }
        for (int k = 0; k < q; ++k) {   // rows p, r
          double apk = A[p * q + k], ark = A[r * q + k];
          A[p * q + k] = c * apk - s * ark;
          A[r * q + k] = s * apk + c * ark;
        }
        for (int k = 0; k < q; ++k) {
          double vkp = V[k * q + p], vkr = V[k * q + r];
          V[k * q + p] = c * vkp - s * vkr;
          V[k * q + r] = s * vkp + c * vkr;
        }
      }
  }
}

// Rayleigh-Ritz on (G, M) (q x q, symmetric, M SPD): theta ascending, W (q x q) with
// W^T M W = I and W^T G W = diag(theta).  Uses scratch of 3 q^2 doubles.  Thread 0 only.
__device__ int rayleigh_ritz(double* G, double* M, int q, double* theta, double* W, double* s) {
  double* L = s;             // chol(M)
  double* T = s + q * q;     // L^-1 G L^-T
  double* V = s + 2 * q * q;
  for (int i = 0; i < q * q; ++i) L[i] = 0.0;
  for (int j = 0; j < q; ++j) {
    double d = M[j * q + j];
    for (int k = 0; k < j; ++k) d -= L[j * q + k] * L[j * q + k];
    if (!(d > 0.0)) return 1;
    d = sqrt(d);
    L[j * q + j] = d;
    for (int i = j + 1; i < q; ++i) {
      double v = M[i * q + j];
      for (int k = 0; k < j; ++k) v -= L[i * q + k] * L[j * q + k];
      L[i * q + j] = v / d;
    }
  }
  // Linv in V (temporarily)
  for (int c = 0; c < q; ++c)
    for (int i = 0; i < q; ++i) {
      if (i < c) { V[i * q + c] = 0.0; continue; }
      double v = (i == c) ? 1.0 : 0.0;
      for (int l = c; l < i; ++l) v -= L[i * q + l] * V[l * q + c];
      V[i * q + c] = v / L[i * q + i];
    }
  // T = Linv G Linv^T, as two products (W holds Linv G)
  for (int i = 0; i < q; ++i)
    for (int b = 0; b < q; ++b) {
      double v = 0.0;
      for (int a = 0; a <= i; ++a) v += V[i * q + a] * G[a * q + b];
      W[i * q + b] = v;
    }
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      double v = 0.0;
      for (int b = 0; b <= j; ++b) v += W[i * q + b] * V[j * q + b];
      T[i * q + j] = v;
    }
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < i; ++j) {
      double v = 0.5 * (T[i * q + j] + T[j * q + i]);
      T[i * q + j] = T[j * q + i] = v;
    }
  // keep Linv: copy into L's storage
  for (int i = 0; i < q * q; ++i) L[i] = V[i];
  jacobi_eig(T, V, q);
  // sort ascending
  int idx[MSTOPO_MAX_EIG * 2];
  for (int i = 0; i < q; ++i) idx[i] = i;
  for (int i = 1; i < q; ++i) {
    int v = idx[i], j = i - 1;
    while (j >= 0 && T[idx[j] * q + idx[j]] > T[v * q + v]) { idx[j + 1] = idx[j]; --j; }
    idx[j + 1] = v;
  }
  // W = Linv^T V(:, idx)
  for (int j = 0; j < q; ++j) {
    theta[j] = T[idx[j] * q + idx[j]];
    for (int i = 0; i < q; ++i) {
      double v = 0.0;
      for (int a = i; a < q; ++a) v += L[a * q + i] * V[a * q + idx[j]];
      W[i * q + j] = v;
    }
  }
  return 0;
}

struct EigArgs {
  const double* E; const uint8_t* nmask; int nelx, nely, H, ncx;
  const int* rep; const double* A; const uint8_t* freem;
  const double* Linv; const double* C;     // factor of K_w + shift diag(K_w)
  double* X; double* Y; double* KY; double* KX;   // [T][NL][nb][q]
  double* Ysc;                             // [T][EIG_CL][NL*nb][q/EIG_CL]
  double* GM; double* resg;                // [T][2][q][q], [T][q]
  int q, kmax; double lam_thresh;
  double* lambda; int* kept; double* res; int* sweeps;
  int* err;
  K0P K0;
};

// y = K_w x on the agglomerate box (elements of the agglomerate only) for the columns
// [j0, j0 + nc) of [N][nb][R]-laid-out vectors; zero on non-free DOFs.
__device__ void box_apply_cols(const EigArgs& a, int I, int J, const uint8_t* freem,
                               const double* x, double* y, int R, int j0, int nc) {
  const int H = a.H, N = 2 * H + 1, nb = 2 * N;
  const int ox = (I - 1) * H, oy = (J - 1) * H;
  for (int t = threadIdx.x; t < N * nb * nc; t += blockDim.x) {
    const int r = j0 + t % nc, dof = t / nc;
    const int line = dof / nb, rr = dof % nb, na = rr >> 1, cr = rr & 1;
    double s = 0.0;
    if (freem[dof]) {
      const int gx = ox + na, gy = oy + line;
      for (int q = 0; q < 4; ++q) {
        const int ex = gx - 1 + (q & 1), ey = gy - 1 + (q >> 1);
        if (ex < ox || ex >= ox + 2 * H || ey < oy || ey >= oy + 2 * H) continue;
        if (ex < 0 || ex >= a.nelx || ey < 0 || ey >= a.nely) continue;
        const double Ee = a.E[(long long)ey * a.nelx + ex];
        const int lx = gx - ex, ly = gy - ey;
        const int la = ly == 0 ? (lx == 0 ? 0 : 1) : (lx == 1 ? 2 : 3);
        double es = 0.0;
        for (int lb = 0; lb < 4; ++lb) {
          const int mx = ex + ((lb == 1 || lb == 2) ? 1 : 0) - ox, my = ey + (lb >= 2 ? 1 : 0) - oy;
          const long long md = (long long)my * nb + 2 * mx;
          es = fma(a.K0.k[(2 * la + cr) * 8 + 2 * lb], x[md * R + r], es);
          es = fma(a.K0.k[(2 * la + cr) * 8 + 2 * lb + 1], x[(md + 1) * R + r], es);
        }
        s = fma(Ee, es, s);
      }
    }
    y[(long long)dof * R + r] = s;
  }
}

// One EIG_CL-CTA cluster per agglomerate type.  CTA rank r owns the subspace columns
// [r*QC, (r+1)*QC): it applies the shifted inverse and K_w to them; the q x q projections
// G = Y^T K Y, M = Y^T D Y are assembled from all columns (global memory, cluster barriers)
// and every CTA performs the same small Rayleigh-Ritz step.
template <int Q>
__global__ void __cluster_dims__(EIG_CL, 1, 1) __launch_bounds__(SOLVE_THREADS) k_eigen(EigArgs a) {
  constexpr int QC = Q / EIG_CL;
  constexpr int q = Q;
  extern __shared__ double smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int type = blockIdx.x / EIG_CL;
  const int H = a.H, N = 2 * H + 1, nb = 2 * N;
  const long long n = (long long)N * nb, nn = (long long)nb * nb;
  const int ia = a.rep[type];
  const int I = ia % (a.ncx + 1), J = ia / (a.ncx + 1);
  const double* Ak = a.A + (long long)type * N * nn;
  const uint8_t* fr = a.freem + (long long)type * n;
  const double* Linv = a.Linv + (long long)type * N * nn;
  const double* C = a.C + (long long)type * (N - 1) * nn;
  double* X = a.X + (long long)type * n * q;
  double* Y = a.Y + (long long)type * n * q;
  double* KY = a.KY + (long long)type * n * q;
  double* KX = a.KX + (long long)type * n * q;
  double* Yc = a.Ysc + ((long long)type * EIG_CL + rank) * n * QC;   // my columns, contiguous
  double* GMg = a.GM + (long long)type * 2 * q * q;                    // G then M (global)
  double* resg = a.resg + (long long)type * q;
  double* stage = smem;                    // nn
  double* t0 = stage + nn;                 // nb*QC
  double* t1 = t0 + nb * QC;               // nb*QC
  double* G = t1 + nb * QC;                // q*q
  double* M = G + q * q;                   // q*q
  double* W = M + q * q;                   // q*q
  double* scr = W + q * q;                 // 3 q*q
  double* theta = scr + 3 * q * q;         // q
  __shared__ int s_done, s_fail;
  __shared__ __align__(8) uint64_t s_bars[2];
  const int j0 = rank * QC;
  auto Dof = [&](long long dof) -> double {
    long long line = dof / nb, r = dof % nb;
    return Ak[line * nn + r * nb + r];
  };
  // deterministic start block, zero on non-free DOFs (same values as a single-CTA start)
  for (long long t = threadIdx.x; t < n * QC; t += blockDim.x) {
    const long long dof = t / QC;
    const int j = j0 + (int)(t % QC);
    const long long g = dof * q + j;
    unsigned long long z = mix64((unsigned long long)g * 0x9E3779B97F4A7C15ull + 12345u);
    X[g] = fr[dof] ? ((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5) : 0.0;
  }
  if (threadIdx.x == 0) { s_done = 0; s_fail = 0; }
  cluster.sync();
  int sweep = 0;
  for (; sweep < EIG_MAX_SWEEPS && !s_done; ++sweep) {
    // my columns: Y = (K + s D)^-1 D X
    for (long long t = threadIdx.x; t < n * QC; t += blockDim.x) {
      const long long dof = t / QC;
      Yc[t] = Dof(dof) * X[dof * q + j0 + t % QC] * fr[dof];
    }
    __syncthreads();
    bt_solve_bulk<double, 1, QC, false>(Linv, C, nb, N, Yc, stage, t0, t1, s_bars, a.err);
    for (long long t = threadIdx.x; t < n * QC; t += blockDim.x) {
      const long long dof = t / QC;
      Y[dof * q + j0 + t % QC] = fr[dof] ? Yc[t] : 0.0;
    }
    __syncthreads();
    // my columns: KY = K_w Y
    box_apply_cols(a, I, J, fr, Y, KY, q, j0, QC);
    cluster.sync();
    // rows of G and M for my columns
    for (int t = threadIdx.x; t < QC * q; t += blockDim.x) {
      const int i = j0 + t / q, j = t % q;
      double g = 0.0, m = 0.0;
      for (long long d = 0; d < n; ++d) {
        const double yi = Y[d * q + i];
        g = fma(yi, KY[d * q + j], g);
        m = fma(yi * Dof(d), Y[d * q + j], m);
      }
      GMg[i * q + j] = g;
      GMg[q * q + i * q + j] = m;
    }
    cluster.sync();
    if (threadIdx.x == 0) {
      for (int t = 0; t < q * q; ++t) { G[t] = GMg[t]; M[t] = GMg[q * q + t]; }
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < i; ++j) {
          double g = 0.5 * (G[i * q + j] + G[j * q + i]), m = 0.5 * (M[i * q + j] + M[j * q + i]);
          G[i * q + j] = G[j * q + i] = g;
          M[i * q + j] = M[j * q + i] = m;
        }
      if (rayleigh_ritz(G, M, q, theta, W, scr)) s_fail = 1;
    }
    __syncthreads();
    // my columns: X = Y W, KX = KY W
    for (long long d = threadIdx.x; d < n; d += blockDim.x) {
      double yr[Q], kr[Q];
#pragma unroll
      for (int i = 0; i < q; ++i) { yr[i] = Y[d * q + i]; kr[i] = KY[d * q + i]; }
#pragma unroll
      for (int jj = 0; jj < QC; ++jj) {
        const int j = j0 + jj;
        double xs = 0.0, ks = 0.0;
#pragma unroll
        for (int i = 0; i < q; ++i) { xs = fma(yr[i], W[i * q + j], xs); ks = fma(kr[i], W[i * q + j], ks); }
        X[d * q + j] = xs;
        KX[d * q + j] = ks;
      }
    }
    __syncthreads();
    // residual norms of the wanted pairs among my columns: ||K x - theta D x||_{D^-1}
    for (int jj = 0; jj < QC; ++jj) {
      const int j = j0 + jj;
      if (j >= a.kmax) break;
      double sacc = 0.0;
      for (long long d = threadIdx.x; d < n; d += blockDim.x) {
        if (!fr[d]) continue;
        const double Dd = Dof(d);
        const double v = KX[d * q + j] - theta[j] * Dd * X[d * q + j];
        sacc = fma(v, v / Dd, sacc);
      }
      // block reduction into resg[j]
      for (int o = 16; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o);
      __shared__ double red[SOLVE_THREADS / 32];
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sacc;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        resg[j] = sqrt(tot);
      }
      __syncthreads();
    }
    cluster.sync();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int j = 0; j < a.kmax; ++j) m = fmax(m, resg[j]);
      if (m <= EIG_TOL || s_fail) s_done = 1;
    }
    __syncthreads();
  }
  if (rank == 0 && threadIdx.x == 0) {
    int kept = a.kmax;
    if (a.lam_thresh > 0.0) {
      kept = 0;
      while (kept < a.kmax && theta[kept] < a.lam_thresh) ++kept;
      if (kept < 1) kept = 1;
    }
    double m = 0.0;
    for (int j = 0; j < a.kmax; ++j) {
      a.lambda[type * MSTOPO_MAX_EIG + j] = theta[j];
      if (j < kept) m = fmax(m, resg[j]);
    }
    a.kept[type] = s_fail ? -1 : kept;
    a.res[type] = m;
    a.sweeps[type] = sweep;
  }
}

template <int Q>
static cudaError_t launch_eigen_q(int T, size_t esm, cudaStream_t s, const EigArgs& ea) {
  cudaError_t e = smem_limit_max<k_eigen<Q>>();
  if (e != cudaSuccess) return e;
  note_launch(), k_eigen<Q><<<T * EIG_CL, SOLVE_THREADS, esm, s>>>(ea);
  return cudaGetLastError();
}

static cudaError_t launch_eigen(int q, int T, size_t esm, cudaStream_t s, const EigArgs& ea) {
  switch (q) {
    case 8: return launch_eigen_q<8>(T, esm, s, ea);
    case 12: return launch_eigen_q<12>(T, esm, s, ea);
    case 16: return launch_eigen_q<16>(T, esm, s, ea);
    case 20: return launch_eigen_q<20>(T, esm, s, ea);
    case 24: return launch_eigen_q<24>(T, esm, s, ea);
    case 28: return launch_eigen_q<28>(T, esm, s, ea);
    default: return launch_eigen_q<32>(T, esm, s, ea);
  }
}

// Psi[type][node][c][j] from X[type][dof][q] (dof = node*2 + c), zero for j >= kept
__global__ void k_store_psi(const double* __restrict__ X, const int* __restrict__ kept, int n,
                            int q, int kmax, double* __restrict__ psi64, float* __restrict__ psi32) {
  const int type = blockIdx.y;
  const int k = kept[type];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * kmax;
       t += (long long)gridDim.x * blockDim.x) {
    long long dof = t / kmax;
    int j = t % kmax;
    double v = j < k ? X[((long long)type * n + dof) * q + j] : 0.0;
    psi64[(long long)type * n * kmax + t] = v;
    psi32[(long long)type * n * kmax + t] = (float)v;
  }
}

// ------------------------------------------------------------------- coarse assembly
// Coarse unknowns are ordered agglomerate by agglomerate (i = J*(ncx+1) + I), offsets coff.
// For the block-tridiagonal factorisation they are grouped in lines of coarse nodes along
// the shorter coarse dimension: line L, position p in the line, slot p*kmax + a.
struct CoarseMap { int by_columns; int ncx, ncy, kmax; };

__device__ __forceinline__ void coarse_line_pos(const CoarseMap& m, int I, int J, int& line, int& pos) {
  if (m.by_columns) { line = I; pos = J; } else { line = J; pos = I; }
}

// K_c = R_c K R_c^T element by element, organised by coarse cells: every element of cell
// (cx, cy) lies in the boxes of exactly four agglomerates a = (cx + (a&1), cy + (a>>1)), so
// per cell the ten blocks sum_e E_e phi_a,e^T K0 phi_b,e (a <= b) are formed from the four
// phi_a,e = chi_a psi_a once per element (k_coarse_cell), and each block of K_c is then the
// sum of the partials of the 1, 2 or 4 cells its two agglomerates share, in a fixed order
// (k_coarse_gather).  chi_a = (H - |x - IH|)(H - |y - JH|) / H^2 (integer numerators).
#define CC_CHUNK 16                   // elements of a cell staged together
#define CC_OUT 10                     // pair-block outputs per thread (10 x 16^2 / 256)
__device__ __forceinline__ int cc_pair(int a, int b) {   // a <= b in 0..3 -> 0..9
  return a * 4 - a * (a - 1) / 2 + (b - a);
}

__global__ void __launch_bounds__(PC_THREADS) k_coarse_cell(
    const double* __restrict__ E, int nelx, int nely, int H, int ncx,
    const int* __restrict__ type_of, const int* __restrict__ kept,
    const double* __restrict__ psi, int kmax, K0P K0, double* __restrict__ part) {
  // part: [cell][10][kmax][kmax], block (a, b) row index over agglomerate a's basis
  extern __shared__ double ccs[];
  double* phi = ccs;                                   // [CHUNK][4][8][kmax]
  double* G = phi + CC_CHUNK * 4 * 8 * kmax;           // [CHUNK][4][8][kmax] = E K0 phi
  const int cell = blockIdx.x;
  const int cx = cell % ncx, cy = cell / ncx;
  const int N = 2 * H + 1;
  const long long nbox = (long long)N * N * 2;
  int Ia[4], Ja[4], ka[4];
  const double* Pa[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    Ia[a] = cx + (a & 1);
    Ja[a] = cy + (a >> 1);
    const int i = Ja[a] * (ncx + 1) + Ia[a];
    const int t = type_of[i];
    ka[a] = kept[t];
    Pa[a] = psi + (long long)t * nbox * kmax;
  }
  const double invH2 = 1.0 / (double)(H * H);
  const int kk = kmax * kmax;
  // output slots: 10 pairs x kmax x kmax, several per thread
  const int nout = 10 * kk;
  double acc[CC_OUT];
  for (int q = 0; q < CC_OUT; ++q) acc[q] = 0.0;
  for (int e0 = 0; e0 < H * H; e0 += CC_CHUNK) {
    __syncthreads();
    // phi of the chunk: (element, agglomerate, dof, column)
    for (int t = threadIdx.x; t < CC_CHUNK * 4 * 8 * kmax; t += blockDim.x) {
      const int col = t % kmax, dof = (t / kmax) % 8, a = (t / (8 * kmax)) % 4, le = t / (32 * kmax);
      const int el = e0 + le;
      const int ex = cx * H + el % H, ey = cy * H + el / H;
      const int ln = dof >> 1, comp = dof & 1;
      const int nx = ex + ((ln == 1 || ln == 2) ? 1 : 0), ny = ey + (ln >= 2 ? 1 : 0);
      const int hx = max(H - abs(nx - Ia[a] * H), 0), hy = max(H - abs(ny - Ja[a] * H), 0);
      const long long l = (long long)(ny - (Ja[a] - 1) * H) * N + (nx - (Ia[a] - 1) * H);
      double v = 0.0;
      if (el < H * H && col < ka[a] && hx > 0 && hy > 0)
        v = (double)(hx * hy) * invH2 * Pa[a][(l * 2 + comp) * kmax + col];
      phi[t] = v;
    }
    __syncthreads();
    // G = E_e K0 phi  (per element, agglomerate and column: 8 outputs)
    for (int t = threadIdx.x; t < CC_CHUNK * 4 * kmax; t += blockDim.x) {
      const int col = t % kmax, a = (t / kmax) % 4, le = t / (4 * kmax);
      const int el = e0 + le;
      const int ex = cx * H + el % H, ey = cy * H + el / H;
      const double Ee = el < H * H ? E[(long long)ey * nelx + ex] : 0.0;
      const double* f = phi + ((le * 4 + a) * 8) * kmax + col;
      double fv[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) fv[c] = f[c * kmax];
      double* g = G + ((le * 4 + a) * 8) * kmax + col;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        double sdot = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) sdot = fma(K0.k[r * 8 + c], fv[c], sdot);
        g[r * kmax] = Ee * sdot;
      }
    }
    __syncthreads();
    // pair blocks: out(p, i, j) += sum_e sum_r phi[e][a][r][i] G[e][b][r][j]
    for (int q = 0; q < CC_OUT; ++q) {
      const int o = threadIdx.x + q * blockDim.x;
      if (o >= nout) break;
      const int pr = o / kk, ij = o % kk, i = ij / kmax, j = ij % kmax;
      int a = 0, b = 0;
      for (int aa = 0, cnt = 0; aa < 4; ++aa)
        for (int bb = aa; bb < 4; ++bb, ++cnt)
          if (cnt == pr) { a = aa; b = bb; }
      double sum = acc[q];
      for (int le = 0; le < CC_CHUNK; ++le) {
        const double* pa = phi + ((le * 4 + a) * 8) * kmax + i;
        const double* gb = G + ((le * 4 + b) * 8) * kmax + j;
#pragma unroll
        for (int r = 0; r < 8; ++r) sum = fma(pa[r * kmax], gb[r * kmax], sum);
      }
      acc[q] = sum;
    }
  }
  for (int q = 0; q < CC_OUT; ++q) {
    const int o = threadIdx.x + q * blockDim.x;
    if (o < nout) part[(long long)cell * nout + o] = acc[q];
  }
}

// Block (i, i2) of K_c from the cell partials (grid: agglomerate i x 9 neighbours); the
// storage and the padding rules are those of the line-blocked factor.
__global__ void __launch_bounds__(PC_THREADS) k_coarse_gather(
    const double* __restrict__ part, int ncx, int ncy, const int* __restrict__ type_of,
    const int* __restrict__ kept, int kmax, CoarseMap cm, double* __restrict__ Ac,
    double* __restrict__ Bc, int nbc) {
  const int i = blockIdx.x;
  const int I = i % (ncx + 1), J = i / (ncx + 1);
  const int I2 = I + (int)blockIdx.y % 3 - 1, J2 = J + (int)blockIdx.y / 3 - 1;
  if (I2 < 0 || I2 > ncx || J2 < 0 || J2 > ncy) return;
  int L1, P1, L2, P2;
  coarse_line_pos(cm, I, J, L1, P1);
  coarse_line_pos(cm, I2, J2, L2, P2);
  if (L2 == L1 - 1) return;   // stored through the transpose (block of line L2)
  const int i2 = J2 * (ncx + 1) + I2;
  const int k1 = kept[type_of[i]], k2 = kept[type_of[i2]];
  const int kk = kmax * kmax;
  for (int t = threadIdx.x; t < kk; t += blockDim.x) {
    const int aa = t / kmax, bb = t % kmax;   // row basis index (agglomerate i), column (i2)
    double s = 0.0;
    // cells shared by the two boxes: cx in {I-1, I} and {I2-1, I2}, inside the mesh
    for (int cy = max(J, J2) - 1; cy <= min(J, J2); ++cy) {
      if (cy < 0 || cy >= ncy) continue;
      for (int cx = max(I, I2) - 1; cx <= min(I, I2); ++cx) {
        if (cx < 0 || cx >= ncx) continue;
        const int a = (I - cx) + 2 * (J - cy), b = (I2 - cx) + 2 * (J2 - cy);
        const double* pc = part + ((long long)(cy * ncx + cx) * 10) * kk;
        s += (a <= b) ? pc[cc_pair(a, b) * kk + aa * kmax + bb] : pc[cc_pair(b, a) * kk + bb * kmax + aa];
      }
    }
    const int row_slot = P1 * kmax + aa, col_slot = P2 * kmax + bb;
    double v;
    if (aa < k1 && bb < k2) v = s;
    else v = (i == i2 && aa == bb) ? 1.0 : 0.0;   // padding slots: identity
    if (L2 == L1) Ac[((long long)L1 * nbc + row_slot) * nbc + col_slot] = v;
    else Bc[((long long)L1 * nbc + col_slot) * nbc + row_slot] = v;   // B_L1 = A(L1+1, L1)
  }
}

// dense inverse of the coarse matrix: solve with identity right-hand sides, RC columns
// (in line order) per CTA, scatter into Kcinv in the agglomerate order
#define RC 16
__global__ void __launch_bounds__(PC_THREADS) k_coarse_inverse(
    const double* __restrict__ Linv, const double* __restrict__ C, int nbc, int NLc,
    const int* __restrict__ slot2orig, int Nt, double* __restrict__ Xw, double* __restrict__ Kcinv) {
  extern __shared__ double smem[];
  double* t0 = smem;
  double* t1 = t0 + nbc * RC;
  const long long ntot = (long long)nbc * NLc;
  const long long j0 = (long long)blockIdx.x * RC;
  double* X = Xw + (long long)blockIdx.x * ntot * RC;
  for (long long t = threadIdx.x; t < ntot * RC; t += blockDim.x) {
    long long row = t / RC, r = t % RC;
    X[t] = (row == j0 + r) ? 1.0 : 0.0;
  }
  __syncthreads();
  bt_solve<double, false>(Linv, C, nbc, NLc, X, RC, nullptr, t0, t1);
  for (long long t = threadIdx.x; t < ntot * RC; t += blockDim.x) {
    long long row = t / RC, r = t % RC;
    long long col = j0 + r;
    if (col >= ntot) continue;
    int orow = slot2orig[row], ocol = slot2orig[col];
    if (orow < 0 || ocol < 0) continue;
    Kcinv[(long long)orow * Nt + ocol] = X[t];
  }
}

// ------------------------------------------------------------------------------ apply
// rc[s][coff[i] + a] = sum over the agglomerate box nodes of chi_i psi_a . r
// chi_i = (H - |x - IH|)(H - |y - JH|) / H^2 (the bilinear hat, integer numerator).
template <typename T>
__global__ void __launch_bounds__(PC_THREADS) k_restrict(
    const T* __restrict__ r, long long stride, int nelx, int nely, int H, int ncx,
    const int* __restrict__ type_of, const int* __restrict__ kept, const int* __restrict__ coff,
    const T* __restrict__ psi, int kmax, double* __restrict__ rc, int Nt) {
  __shared__ double sh[PC_THREADS / 32][MSTOPO_MAX_EIG];
  const int i = blockIdx.x, s = blockIdx.y;
  const int I = i % (ncx + 1), J = i / (ncx + 1);
  const int t = type_of[i], k = kept[t];
  const int N = 2 * H + 1;
  const T invH2 = T(1) / (T)(H * H);
  const T* P = psi + (long long)t * N * N * 2 * kmax;
  r += s * stride;
  T acc[MSTOPO_MAX_EIG];
#pragma unroll
  for (int a = 0; a < MSTOPO_MAX_EIG; ++a) acc[a] = T(0);
  // nodes with chi > 0: strictly inside the box
  const int M = N - 2;
  for (int u = threadIdx.x; u < M * M; u += blockDim.x) {
    const int la = 1 + u % M, lb = 1 + u / M;
    const int x = (I - 1) * H + la, y = (J - 1) * H + lb;
    if (x < 0 || x > nelx || y < 0 || y > nely) continue;
    const T chi = (T)((H - abs(la - H)) * (H - abs(lb - H))) * invH2;
    const long long node = (long long)y * (nelx + 1) + x;
    const T rx = chi * r[2 * node], ry = chi * r[2 * node + 1];
    const T* pp = P + ((long long)lb * N + la) * 2 * kmax;
#pragma unroll
    for (int a = 0; a < MSTOPO_MAX_EIG; ++a)
      if (a < k) acc[a] = fma(rx, pp[a], fma(ry, pp[kmax + a], acc[a]));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < MSTOPO_MAX_EIG; ++a) {
    if (a < k) {
      double v = (double)acc[a];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sh[w][a] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double v = 0.0;
    for (int q = 0; q < PC_THREADS / 32; ++q) v += sh[q][threadIdx.x];
    rc[(long long)s * Nt + coff[i] + threadIdx.x] = v;
  }
}

// uc[s] = Kcinv[sys0 + s] rc[s]   (one warp per row; blockIdx.y = system)
__global__ void k_coarse_gemv(const double* __restrict__ Kinv, const double* __restrict__ rc,
                              double* __restrict__ uc, int Nt, int sys0) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y;
  if (warp >= Nt) return;
  const double* row = Kinv + ((long long)(sys0 + s) * Nt + warp) * Nt;
  const double* v = rc + (long long)s * Nt;
  double acc = 0.0;
  for (int c = lane; c < Nt; c += 32) acc = fma(row[c], v[c], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) uc[(long long)s * Nt + warp] = acc;
}

// z(node) = sum over the agglomerates whose box contains the node of
//           chi_i psi_i uc_i  (coarse part)  +  patch solution of omega_i at the node.
// One thread per node (2D grid: x fastest), arithmetic in T.
template <typename T>
__global__ void __launch_bounds__(256) k_combine(
    T* __restrict__ z, long long stride, int sys0, int Nc, int nelx, int nely, int H, int ncx, int ncy,
    const int* __restrict__ type_of, const int* __restrict__ kept, const int* __restrict__ coff,
    const T* __restrict__ psi, int kmax, const double* __restrict__ uc, int Nt,
    const int* __restrict__ agg_group, const int* __restrict__ agg_slot, const T* __restrict__ Xg,
    int R, int pfast, const uint8_t* __restrict__ nmask, int part) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int s = blockIdx.z;
  if (x > nelx) return;
  const int N = 2 * H + 1, nbP = 2 * N;
  const T invH2 = T(1) / (T)(H * H);
  T zx = T(0), zy = T(0);
  const int Ib = x / H, Jb = y / H;
  for (int J = max(Jb - 1, 0); J <= min(Jb + 1, ncy); ++J) {
    const int dyj = abs(y - J * H);
    if (dyj > H) continue;
    for (int I = max(Ib - 1, 0); I <= min(Ib + 1, ncx); ++I) {
      const int dxi = abs(x - I * H);
      if (dxi > H) continue;
      const int i = J * (ncx + 1) + I;
      const int lb = y - (J - 1) * H, la = x - (I - 1) * H;
      const long long l = (long long)lb * N + la;
      if (part != 2 && dxi < H && dyj < H) {
        const int t = type_of[i], k = kept[t];
        const T chi = (T)((H - dxi) * (H - dyj)) * invH2;
        const T* pp = psi + ((long long)t * N * N + l) * 2 * kmax;
        const double* u = uc + (long long)s * Nt + coff[i];
        T ax = T(0), ay = T(0);
        for (int a = 0; a < k; ++a) {
          const T ua = (T)u[a];
          ax = fma(pp[a], ua, ax);
          ay = fma(pp[kmax + a], ua, ay);
        }
        zx = fma(chi, ax, zx);
        zy = fma(chi, ay, zy);
      }
      if (part != 1) {
        const long long gi = (long long)(sys0 + s) * Nc + i;
        const int col = agg_slot[gi];
        // work-buffer layout [group][line][column][DOF], or [group][line][node][column][2]
        // (pfast: the tensor-core kernel's, consecutive columns = consecutive patches)
        const long long gl = (long long)agg_group[gi] * N + lb;
        const long long base = pfast ? ((gl * (nbP / 2) + la) * R + col) * 2 : (gl * R + col) * nbP + 2 * la;
        zx += Xg[base];
        zy += Xg[base + 1];
      }
    }
  }
  const long long node = (long long)y * (nelx + 1) + x;
  const uint8_t f = nmask[node];
  z[s * stride + 2 * node] = (f & 1) ? T(0) : zx;
  z[s * stride + 2 * node + 1] = (f & 2) ? T(0) : zy;
}

// ------------------------------------------------------------------------------ host side
// Patch-solve configurations chosen by timing (MSTOPO_EXEC_AUTOTUNE), kept per problem shape
// for the process: (DOFs per patch line, lines, agglomerates, types, realisations) ->
// (tensor cores, patches per group).
namespace {
struct TuneKey {
  int nb, nl, nc, nt, ns;
  bool operator<(const TuneKey& o) const {
    return std::tie(nb, nl, nc, nt, ns) < std::tie(o.nb, o.nl, o.nc, o.nt, o.ns);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;
}  // namespace

#define CKB(x)                                                                  \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      h->err = std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x;      \
      return e_ == cudaErrorMemoryAllocation ? MSTOPO_OUT_OF_MEMORY : MSTOPO_CUDA_ERROR; \
    }                                                                           \
  } while (0)

static void dfree(void* p) { if (p) cudaFree(p); }

void precond_free(Precond& pc) {
  dfree(pc.d_type_of_agg); dfree(pc.d_kept); dfree(pc.d_coff);
  for (PatchGroups& G : pc.pg) {
    dfree(G.d_perm); dfree(G.d_type); dfree(G.d_first); dfree(G.d_count); dfree(G.d_sys); dfree(G.d_agg);
  }
  dfree(pc.d_pfree);
  dfree(pc.d_tri64); dfree(pc.d_tri32); dfree(pc.d_ptw); dfree(pc.d_twu);
  dfree(pc.d_lambda); dfree(pc.d_psi64); dfree(pc.d_psi32); dfree(pc.d_eigres); dfree(pc.d_eigsweeps);
  dfree(pc.d_Kc); dfree(pc.d_Kcinv);
  dfree(pc.d_cLinv); dfree(pc.d_cLinvT); dfree(pc.d_cW); dfree(pc.d_cV);
  dfree(pc.d_cy); dfree(pc.d_cx); dfree(pc.d_s2o); dfree(pc.d_cbar); dfree(pc.d_rc); dfree(pc.d_uc);
  dfree(pc.d_zp32); dfree(pc.d_zp64); dfree(pc.d_work); dfree(pc.d_flag); dfree(pc.d_sgs);
  pc = Precond();
}


mstopo_status precond_build(mstopo_handle* h, int ref, mstopo_build_info* info) {
  Precond old = h->pc;
  precond_free(old);
  h->pc = Precond();
  Precond& pc = h->pc;
  cudaStream_t s = h->s;
  const int H = h->p.H;
  pc.H = H; pc.NA = 2 * H + 1; pc.NP = 2 * H + 1; pc.nbA = 2 * pc.NA; pc.nbP = 2 * pc.NP;
  pc.ncx = h->nelx / H; pc.ncy = h->nely / H; pc.Nc = (pc.ncx + 1) * (pc.ncy + 1);
  pc.kmax = h->p.n_eig;
  pc.local_shift = h->p.precision == MSTOPO_MIXED ? h->p.local_shift : 0.0;
  // operators per realisation: the coarse basis comes from realisation ref (Sec. 5.3: the
  // dilated design embeds the others), K_c and the patch matrices from each realisation's
  // own moduli
  const int nsv = pc.nsv = h->n_eta;
  pc.kind = h->p.preconditioner;
  const bool sgs = pc.kind == MSTOPO_PREC_MULTIPLICATIVE_SGS;   // no patch solves to build
  if (sgs)
    CKB(cudaMalloc(&pc.d_sgs, (size_t)2 * MSTOPO_MAX_SYS * h->n_dof * sizeof(double)));
  const double* E = h->d_E64 + (long long)ref * h->n_el;
  K0P K0;
  for (int q = 0; q < 64; ++q) K0.k[q] = h->K0[q];
  cudaEvent_t ev[6];
  for (int q = 0; q < 6; ++q) CKB(cudaEventCreate(&ev[q]));
  CKB(cudaEventRecord(ev[0], s));
  // 1. hashes -> types
  unsigned long long* d_hash;
  CKB(cudaMalloc(&d_hash, (size_t)pc.Nc * 16));
  CKB(cudaMemsetAsync(d_hash, 0, (size_t)pc.Nc * 16, s));
  for (int k = 0; k < nsv; ++k) {
    note_launch(), k_hash_agg<<<pc.Nc, PC_THREADS, 0, s>>>(h->d_E64 + (long long)k * h->n_el, h->d_nmask,
                                                          h->nelx, h->nely, H, pc.ncx, k, k == 0, d_hash);
    CKB(cudaGetLastError());
  }
  std::vector<unsigned long long> hh((size_t)pc.Nc * 2);
  CKB(cudaMemcpyAsync(hh.data(), d_hash, (size_t)pc.Nc * 16, cudaMemcpyDeviceToHost, s));
  CKB(cudaStreamSynchronize(s));
  cudaFree(d_hash);
  std::map<std::pair<unsigned long long, unsigned long long>, int> tmap;
  pc.h_type_of_agg.resize(pc.Nc);
  for (int i = 0; i < pc.Nc; ++i) {
    auto key = std::make_pair(hh[2 * i], hh[2 * i + 1]);
    auto it = tmap.find(key);
    if (it == tmap.end()) {
      int t = (int)pc.h_rep_agg.size();
      tmap[key] = t;
      pc.h_rep_agg.push_back(i);
      pc.h_type_of_agg[i] = t;
    } else {
      pc.h_type_of_agg[i] = it->second;
    }
  }
  int* d_rep;
  CKB(cudaMalloc(&d_rep, pc.Nc * sizeof(int)));
  CKB(cudaMemcpyAsync(d_rep, pc.h_rep_agg.data(), pc.h_rep_agg.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  CKB(cudaMalloc(&pc.d_type_of_agg, pc.Nc * sizeof(int)));
  CKB(cudaMemcpyAsync(pc.d_type_of_agg, pc.h_type_of_agg.data(), pc.Nc * sizeof(int), cudaMemcpyHostToDevice, s));
  {
    // a hash match is trusted only after the boxes compare equal entry by entry
    int* d_bad;
    CKB(cudaMalloc(&d_bad, pc.Nc * sizeof(int)));
    note_launch(), k_verify_agg<<<pc.Nc, PC_THREADS, 0, s>>>(h->d_E64, h->n_el, nsv, h->d_nmask, h->nelx,
                                                             h->nely, H, pc.ncx, pc.d_type_of_agg, d_rep, d_bad);
    CKB(cudaGetLastError());
    std::vector<int> bad(pc.Nc);
    CKB(cudaMemcpyAsync(bad.data(), d_bad, pc.Nc * sizeof(int), cudaMemcpyDeviceToHost, s));
    CKB(cudaStreamSynchronize(s));
    cudaFree(d_bad);
    bool split = false;
    for (int i = 0; i < pc.Nc; ++i)
      if (bad[i]) {
        pc.h_type_of_agg[i] = (int)pc.h_rep_agg.size();
        pc.h_rep_agg.push_back(i);
        split = true;
      }
    if (split) {
      CKB(cudaMemcpyAsync(d_rep, pc.h_rep_agg.data(), pc.h_rep_agg.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      CKB(cudaMemcpyAsync(pc.d_type_of_agg, pc.h_type_of_agg.data(), pc.Nc * sizeof(int), cudaMemcpyHostToDevice, s));
    }
  }
  const int T = pc.n_types = (int)pc.h_rep_agg.size();
  CKB(cudaEventRecord(ev[1], s));

  // 2. agglomerate (Neumann, for the eigenproblem) and patch (artificial boundary Dirichlet)
  //    matrices of every type, all factorised in one launch: systems [0,T) are the shifted
  //    agglomerate matrices K_w + s diag(K_w) of realisation ref, systems T + k T + t the
  //    patch matrices of type t in realisation k
  const int NA = pc.NA, nbA = pc.nbA, NP = pc.NP, nbP = pc.nbP;
  const long long nnA = (long long)nbA * nbA, nA = (long long)NA * nbA;
  const long long nnP = nnA, nP = nA;
  const int TP = sgs ? 0 : T * nsv;   // patch operators
  const int NS = T + TP;              // factorised systems
  // subspace dimension: 2k + 4 rounded up to a multiple of the cluster size (compile-time variants)
  const int q = std::min(((2 * pc.kmax + 4) + EIG_CL - 1) / EIG_CL * EIG_CL, 2 * MSTOPO_MAX_EIG);
  double *dA, *dB, *dLi, *dC, *dS, *dX, *dY, *dKY, *dKX, *dYsc, *dGM, *dres;
  uint8_t* dfree_;
  int* d_st;
  CKB(cudaMalloc(&dA, (size_t)NS * NA * nnA * 8));
  CKB(cudaMalloc(&dB, (size_t)NS * (NA - 1) * nnA * 8));
  CKB(cudaMalloc(&dLi, (size_t)NS * NA * nnA * 8));
  CKB(cudaMalloc(&dC, (size_t)NS * (NA - 1) * nnA * 8));
  CKB(cudaMalloc(&dS, (size_t)NS * nnA * 8));
  CKB(cudaMalloc(&dfree_, (size_t)T * nA));
  if (TP) CKB(cudaMalloc(&pc.d_pfree, (size_t)TP * nP));
  CKB(cudaMalloc(&d_st, (size_t)std::max(NS, 2) * sizeof(int)));
  note_launch(), k_assemble_box<<<dim3(T, NA), PC_THREADS, 0, s>>>(E, h->d_nmask, h->nelx, h->nely, d_rep, H,
                                                    pc.ncx, 0, K0, dA, dB, dfree_);
  CKB(cudaGetLastError());
  for (int k = 0; k < nsv && !sgs; ++k) {
    const size_t o = (size_t)T + (size_t)k * T;
    note_launch(), k_assemble_box<<<dim3(T, NP), PC_THREADS, 0, s>>>(h->d_E64 + (long long)k * h->n_el, h->d_nmask,
                                                      h->nelx, h->nely, d_rep, H, pc.ncx, 1, K0,
                                                      dA + o * NA * nnA, dB + o * (NA - 1) * nnA,
                                                      pc.d_pfree + (size_t)k * T * nP);
    CKB(cudaGetLastError());
  }
  // the shift flags need a per-system free mask: agglomerate masks, then patch masks
  uint8_t* dfree2;
  CKB(cudaMalloc(&dfree2, (size_t)NS * nA));
  CKB(cudaMemcpyAsync(dfree2, dfree_, (size_t)T * nA, cudaMemcpyDeviceToDevice, s));
  if (TP) CKB(cudaMemcpyAsync(dfree2 + (size_t)T * nA, pc.d_pfree, (size_t)TP * nP, cudaMemcpyDeviceToDevice, s));
  note_launch(), k_bt_factor<<<NS, PC_THREADS, 0, s>>>(dA, dB, dfree2, EIG_SHIFT, pc.local_shift, T, nbA, NA,
                                                       dLi, dC, dS, d_st);
  CKB(cudaGetLastError());
  CKB(cudaMalloc(&dX, (size_t)T * nA * q * 8));
  CKB(cudaMalloc(&dY, (size_t)T * nA * q * 8));
  CKB(cudaMalloc(&dKY, (size_t)T * nA * q * 8));
  CKB(cudaMalloc(&dKX, (size_t)T * nA * q * 8));
  CKB(cudaMalloc(&dYsc, (size_t)T * nA * q * 8));
  CKB(cudaMalloc(&dGM, (size_t)T * 2 * q * q * 8));
  CKB(cudaMalloc(&dres, (size_t)T * q * 8));
  CKB(cudaMalloc(&pc.d_lambda, (size_t)T * MSTOPO_MAX_EIG * 8));
  CKB(cudaMemsetAsync(pc.d_lambda, 0, (size_t)T * MSTOPO_MAX_EIG * 8, s));
  CKB(cudaMalloc(&pc.d_kept, T * sizeof(int)));
  CKB(cudaMalloc(&pc.d_eigres, T * 8));
  CKB(cudaMalloc(&pc.d_eigsweeps, T * sizeof(int)));
  EigArgs ea;
  ea.E = E; ea.nmask = h->d_nmask; ea.nelx = h->nelx; ea.nely = h->nely; ea.H = H; ea.ncx = pc.ncx;
  ea.rep = d_rep; ea.A = dA; ea.freem = dfree_; ea.Linv = dLi; ea.C = dC;
  ea.X = dX; ea.Y = dY; ea.KY = dKY; ea.KX = dKX; ea.Ysc = dYsc; ea.GM = dGM; ea.resg = dres;
  ea.q = q; ea.kmax = pc.kmax; ea.lam_thresh = h->p.lambda_thresh;
  ea.lambda = pc.d_lambda; ea.kept = pc.d_kept; ea.res = pc.d_eigres; ea.sweeps = pc.d_eigsweeps;
  ea.K0 = K0;
  ea.err = h->d_flag + 1;
  const int qc = q / EIG_CL;
  size_t esm = (size_t)(nnA + 2 * nbA * qc + 6 * q * q + 2 * q) * 8;
  if (esm > 225 * 1024) {
    h->err = "n_eig too large for this H: the eigen-solve workspace exceeds shared memory";
    return MSTOPO_INVALID_ARG;
  }
  CKB(cudaMemsetAsync(h->d_flag + 1, 0, sizeof(int), s));
  {
    cudaError_t le = launch_eigen(q, T, esm, s, ea);
    CKB(le);
  }
  CKB(cudaGetLastError());
  std::vector<int> fst(NS);
  CKB(cudaMemcpyAsync(fst.data(), d_st, NS * sizeof(int), cudaMemcpyDeviceToHost, s));
  pc.h_kept.resize(T);
  CKB(cudaMemcpyAsync(pc.h_kept.data(), pc.d_kept, T * sizeof(int), cudaMemcpyDeviceToHost, s));
  int werr = 0;
  CKB(cudaMemcpyAsync(&werr, h->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKB(cudaStreamSynchronize(s));
  if (werr) {
    h->err = "bounded device wait gave up in the eigen-solve";
    return MSTOPO_TIMEOUT;
  }
  for (int t = 0; t < T; ++t) {
    if (fst[t] || pc.h_kept[t] < 1) {
      h->err = "agglomerate eigenproblem failed (non-positive pivot or Rayleigh-Ritz breakdown)";
      return MSTOPO_NOT_SPD;
    }
  }
  for (int t = 0; t < TP; ++t) {
    if (fst[T + t]) {
      h->err = "patch matrix not positive definite";
      return MSTOPO_NOT_SPD;
    }
  }
  CKB(cudaMalloc(&pc.d_psi64, (size_t)T * nA * pc.kmax * 8));
  CKB(cudaMalloc(&pc.d_psi32, (size_t)T * nA * pc.kmax * 4));
  note_launch(), k_store_psi<<<dim3(64, T), 256, 0, s>>>(dX, pc.d_kept, (int)nA, q, pc.kmax, pc.d_psi64, pc.d_psi32);
  CKB(cudaGetLastError());
  CKB(cudaEventRecord(ev[2], s));

  // 3. patch factors: W_k, V_k and the packed stage blocks (FP64 and FP32)
  // patches per work group (see step 5): it fixes the patch kernel's thread mapping
  int sms = 152;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  // Columns per FP32 group (4, 8 or 16 patches of one type and realisation): each group is a
  // cluster of two CTAs and patch_tri_ctas_per_sm(R) CTAs fit on an SM (3 at R = 4, 1 above),
  // so a choice costs ceil(2 groups / (CTAs per SM x SMs)) waves of its time per wave.
  // Measured on the 1024x512 workload (time per wave relative to a full R = 4 wave, three CTAs
  // per SM): R = 8 0.77, R = 16 1.44.  Fewer columns win ties.
  int P = 4;
  double tri_waves = 0.0;   // the chosen CUDA-core configuration in R = 4 wave units
  long long tw_groups = 0;  // groups of the tensor-core kernel (TW_M patches of one type)
  {
    std::vector<long long> per_type(T, 0);
    for (int i = 0; i < pc.Nc; ++i) per_type[pc.h_type_of_agg[i]]++;
    const int cols[3] = {4, 8, 16};
    const double cost[3] = {1.0, 0.77, 1.44};
    double best = 0.0;
    for (int c = 0; c < 3; ++c) {
      long long groups = 0;
      for (int t = 0; t < T; ++t) groups += (per_type[t] + cols[c] - 1) / cols[c];
      groups *= nsv;
      const long long slots = (long long)patch_tri_ctas_per_sm(nbP, cols[c]) * std::max(sms, 1);
      const double t = (double)((2 * groups + slots - 1) / slots) * cost[c];
      if (c == 0 || t < best - 1e-9) {
        best = t;
        P = cols[c];
      }
    }
    tri_waves = best;
    for (int t = 0; t < T; ++t) tw_groups += (per_type[t] + TW_M - 1) / TW_M;
    tw_groups *= nsv;
  }
  // autotuning: a shape timed before keeps its choice; otherwise every candidate is built and
  // timed after the work groups (step 5)
  const bool tune = !sgs && h->autotune && h->patch_tc < 0;
  const TuneKey tkey{nbP, NP, pc.Nc, T, nsv};
  int tuned = 0;              // 0 cost model, 1 timed now, 2 kept
  int tuned_tc = -1;
  if (tune) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tkey);
    if (it != g_tune.end()) {
      tuned = 2;
      tuned_tc = it->second.first;
      P = it->second.second == TW_M ? P : it->second.second;
    } else {
      tuned = 1;
    }
  }
  if (!patch_tri_assignment_ok(nbP)) {
    h->err = "H > 32 is not supported by the patch solve";
    return MSTOPO_INVALID_ARG;
  }
  if (!sgs) {
    const double* pLi = dLi + (size_t)T * NA * nnA;
    const double* pB = dB + (size_t)T * (NA - 1) * nnA;
    const double* pA = dA + (size_t)T * NA * nnA;
    const double* pCt = dC + (size_t)T * (NA - 1) * nnA;
    // two-sided elimination for the CUDA-core patch solves: the first H + 1 lines of the
    // line-reversed patch matrices, factorised top-down, are the bottom half; the middle line
    // H takes the Schur complements of both halves
    const int NLr = H + 1;
    double *dAr, *dBr, *dLr, *dCr, *dSr, *dLm;
    uint8_t* dfr;
    int* d_st2;
    CKB(cudaMalloc(&dAr, (size_t)TP * NLr * nnP * 8));
    CKB(cudaMalloc(&dBr, (size_t)TP * (NLr - 1) * nnP * 8));
    CKB(cudaMalloc(&dLr, (size_t)TP * NLr * nnP * 8));
    CKB(cudaMalloc(&dCr, (size_t)TP * (NLr - 1) * nnP * 8));
    CKB(cudaMalloc(&dSr, (size_t)TP * nnP * 8));
    CKB(cudaMalloc(&dLm, (size_t)TP * nnP * 8));
    CKB(cudaMalloc(&dfr, (size_t)TP * NLr * nbP));
    CKB(cudaMalloc(&d_st2, (size_t)2 * TP * sizeof(int)));
    note_launch(), k_reverse_lines<<<dim3(TP, NLr), PC_THREADS, 0, s>>>(pA, pB, pc.d_pfree, NP, NLr, nbP,
                                                                        dAr, dBr, dfr);
    CKB(cudaGetLastError());
    note_launch(), k_bt_factor<<<TP, PC_THREADS, 0, s>>>(dAr, dBr, dfr, pc.local_shift, pc.local_shift, 0,
                                                         nbP, NLr, dLr, dCr, dSr, d_st2);
    CKB(cudaGetLastError());
    note_launch(), k_twist_middle<<<TP, PC_THREADS, 0, s>>>(pA, pCt, dCr, pc.d_pfree, pc.local_shift, NP,
                                                            NLr, nbP, dSr, dLm, d_st2 + TP);
    CKB(cudaGetLastError());
    std::vector<int> st2(2 * (size_t)TP);
    CKB(cudaMemcpyAsync(st2.data(), d_st2, 2 * (size_t)TP * sizeof(int), cudaMemcpyDeviceToHost, s));
    CKB(cudaStreamSynchronize(s));
    for (int t = 0; t < 2 * TP; ++t)
      if (st2[t]) {
        h->err = "patch matrix not positive definite";
        return MSTOPO_NOT_SPD;
      }
    // The patch solves stream the packed blocks: FP64 always; FP32 on the CUDA cores or, for
    // H = 8, 16, 32, on the tensor cores (csrc/patch_twtc.cu: 128 patches of a type per MMA,
    // its own pack made from the FP64 one).  The tensor-core kernel runs one cluster of two
    // CTAs per group and one CTA per SM, and a line step is a fixed MMA chain whatever the
    // number of patches, so it pays off with many patches per type.  Measured (FP32 patch
    // solves of realisation 0, one launch):
    //   1024x512 (561 patches, 25 types): CUDA cores 0.26 ms, tensor cores 0.59 ms;
    //   2048x1024 (2,145 patches, 165 types): 0.77 ms, 1.72 ms;
    //   3200x4096 (13,029 patches, 25 types): 3.51 ms, 1.24 ms.
    // Cost model from these: a tensor-core wave (up to one CTA per SM) takes 2.3 times an
    // R = 4 CUDA-core wave; the automatic choice takes the cheaper.
    const bool tw_ok = patch_twtc_ok(nbP);
    if (h->patch_tc > 0 && !tw_ok) {
      h->err = "tensor-core patch solves need H = 8, 16 or 32";
      return MSTOPO_INVALID_ARG;
    }
    const double tw_waves = 2.3 * (double)((2 * tw_groups + std::max(sms, 1) - 1) / std::max(sms, 1));
    pc.patch_tc = tw_ok && (h->patch_tc > 0 || (h->patch_tc < 0 && tw_waves < tri_waves));
    if (tuned == 2) pc.patch_tc = tuned_tc;
    const size_t tl = (size_t)TP * patch_tri_system_elems(nbP, NP);
    CKB(cudaMalloc(&pc.d_tri64, tl * 8));
    // timing needs every candidate's pack: the FP32 CUDA-core one and, where compiled, the
    // tensor-core one
    if (!pc.patch_tc || tuned == 1) CKB(cudaMalloc(&pc.d_tri32, tl * 4));
    CKB(patch_tri_pack(pLi, pB, dLr, dBr, dLm, TP, nbP, NP, NLr, pc.d_tri64, pc.d_tri32, s));
    CKB(cudaStreamSynchronize(s));
    cudaFree(dAr); cudaFree(dBr); cudaFree(dLr); cudaFree(dCr); cudaFree(dSr); cudaFree(dLm);
    cudaFree(dfr); cudaFree(d_st2);
    if (pc.patch_tc || (tuned == 1 && tw_ok)) {
      const TwGeom tw = patch_twtc_geometry(nbP, NP);
      CKB(cudaMalloc(&pc.d_ptw, (size_t)TP * tw.SS));
      CKB(patch_twtc_pack(pc.d_tri64, TP, nbP, NP, pc.d_ptw, s));
    }
    CKB(cudaStreamSynchronize(s));
  }
  cudaFree(dLi); cudaFree(dC); cudaFree(dS); cudaFree(dX); cudaFree(dY); cudaFree(dKY);
  cudaFree(dKX); cudaFree(dYsc); cudaFree(dGM); cudaFree(dres);
  cudaFree(dA); cudaFree(dB); cudaFree(dfree_); cudaFree(dfree2); cudaFree(d_rep);
  CKB(cudaEventRecord(ev[3], s));

  // 4. coarse space: offsets, line mapping, assembly, factor, dense inverse
  pc.h_coff.resize(pc.Nc + 1);
  pc.h_coff[0] = 0;
  for (int i = 0; i < pc.Nc; ++i) pc.h_coff[i + 1] = pc.h_coff[i] + pc.h_kept[pc.h_type_of_agg[i]];
  const int Nt = pc.Nt = pc.h_coff[pc.Nc];
  CKB(cudaMalloc(&pc.d_coff, (pc.Nc + 1) * sizeof(int)));
  CKB(cudaMemcpyAsync(pc.d_coff, pc.h_coff.data(), (pc.Nc + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  CoarseMap cm;
  cm.by_columns = (pc.ncy + 1) <= (pc.ncx + 1);
  cm.ncx = pc.ncx; cm.ncy = pc.ncy; cm.kmax = pc.kmax;
  const int NLc = cm.by_columns ? pc.ncx + 1 : pc.ncy + 1;
  const int per_line = cm.by_columns ? pc.ncy + 1 : pc.ncx + 1;
  const int nbc = per_line * pc.kmax;
  const long long nnc = (long long)nbc * nbc;
  std::vector<int> slot2orig((size_t)NLc * nbc, -1);
  for (int J = 0; J <= pc.ncy; ++J)
    for (int I = 0; I <= pc.ncx; ++I) {
      int i = J * (pc.ncx + 1) + I;
      int L = cm.by_columns ? I : J, P = cm.by_columns ? J : I;
      int k = pc.h_kept[pc.h_type_of_agg[i]];
      for (int a = 0; a < k; ++a) slot2orig[(size_t)L * nbc + P * pc.kmax + a] = pc.h_coff[i] + a;
    }
  int* d_s2o;
  double *cA, *cB, *cLi, *cC, *cS, *cX = nullptr;
  const size_t nlA = (size_t)NLc * nnc, nlB = (size_t)std::max(NLc - 1, 1) * nnc;
  CKB(cudaMalloc(&d_s2o, slot2orig.size() * sizeof(int)));
  CKB(cudaMemcpyAsync(d_s2o, slot2orig.data(), slot2orig.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  CKB(cudaMalloc(&cA, nsv * nlA * 8));
  CKB(cudaMalloc(&cB, nsv * nlB * 8));
  CKB(cudaMemsetAsync(cA, 0, nsv * nlA * 8, s));
  CKB(cudaMemsetAsync(cB, 0, nsv * nlB * 8, s));
  {
    // K_c of every realisation on the shared basis: cell partials, then the blocks
    const int ncell = pc.ncx * pc.ncy;
    double* cpart;
    CKB(cudaMalloc(&cpart, (size_t)ncell * 10 * pc.kmax * pc.kmax * 8));
    const size_t ccs = (size_t)2 * CC_CHUNK * 4 * 8 * pc.kmax * 8;
    if (10 * pc.kmax * pc.kmax > CC_OUT * PC_THREADS || ccs > 200 * 1024) {
      cudaFree(cpart);
      h->err = "n_eig too large for the coarse assembly";
      return MSTOPO_INVALID_ARG;
    }
    CKB(smem_limit_max<k_coarse_cell>());
    for (int k = 0; k < nsv; ++k) {
      note_launch(), k_coarse_cell<<<ncell, PC_THREADS, ccs, s>>>(h->d_E64 + (long long)k * h->n_el,
                                                                 h->nelx, h->nely, H, pc.ncx,
                                                                 pc.d_type_of_agg, pc.d_kept,
                                                                 pc.d_psi64, pc.kmax, K0, cpart);
      CKB(cudaGetLastError());
      note_launch(), k_coarse_gather<<<dim3(pc.Nc, 9), PC_THREADS, 0, s>>>(cpart, pc.ncx, pc.ncy,
                                                              pc.d_type_of_agg, pc.d_kept, pc.kmax,
                                                              cm, cA + k * nlA, cB + k * nlB, nbc);
      CKB(cudaGetLastError());
    }
    CKB(cudaStreamSynchronize(s));
    cudaFree(cpart);
  }
  // slots beyond the mesh's coarse nodes do not exist (per_line covers them all)
  int mode = h->p.coarse_solver;
  if (mode == MSTOPO_COARSE_AUTO) mode = Nt <= 4096 ? MSTOPO_COARSE_DENSE : MSTOPO_COARSE_BLOCKTRI;
  pc.coarse_mode = mode;
  pc.nbc = nbc;
  pc.NLc = NLc;
  std::vector<int> cst(nsv, 0);
  CKB(cudaMemsetAsync(d_st, 0, nsv * sizeof(int), s));
  if (mode == MSTOPO_COARSE_DENSE && nbc > 640) {
    cudaFree(cA); cudaFree(cB); cudaFree(d_s2o);
    h->err = "coarse line too long for the dense coarse solver (coarse nodes per line x n_eig > 640)";
    return MSTOPO_INVALID_ARG;
  }
  if (mode == MSTOPO_COARSE_DENSE) {
    // one-CTA block factor per realisation, then the explicit inverses by identity columns
    CKB(cudaMalloc(&cLi, nsv * nlA * 8));
    CKB(cudaMalloc(&cC, nsv * nlB * 8));
    CKB(cudaMalloc(&cS, nsv * nnc * 8));
    note_launch(), k_bt_factor<<<nsv, PC_THREADS, 0, s>>>(cA, cB, nullptr, 0.0, 0.0, nsv, nbc, NLc, cLi, cC, cS, d_st);
    CKB(cudaGetLastError());
    CKB(cudaMalloc(&pc.d_Kcinv, (size_t)nsv * Nt * Nt * 8));
    const int nblk = cdiv((long long)NLc * nbc, RC);
    CKB(cudaMalloc(&cX, (size_t)nblk * NLc * nbc * RC * 8));
    CKB(smem_limit_max<k_coarse_inverse>());
    for (int k = 0; k < nsv; ++k) {
      note_launch(), k_coarse_inverse<<<nblk, PC_THREADS, 2 * nbc * RC * 8, s>>>(cLi + k * nlA, cC + k * nlB, nbc, NLc, d_s2o, Nt, cX,
                                                                                 pc.d_Kcinv + (size_t)k * Nt * Nt);
      CKB(cudaGetLastError());
    }
    CKB(cudaStreamSynchronize(s));
    cudaFree(cX); cudaFree(cLi); cudaFree(cC); cudaFree(cS);
    cudaFree(d_s2o);
  } else {
    // block factor with whole-GPU dense kernels per realisation, applied by cooperative sweeps
    pc.sweep_grid = coarse_sweep_grid();
    if (pc.sweep_grid <= 0 || nbc > coarse_sweep_max_nb(pc.sweep_grid, nsv)) {
      cudaFree(cA); cudaFree(cB); cudaFree(d_s2o);
      h->err = "coarse line too long for the block-tridiagonal coarse solver (coarse nodes per line x n_eig "
               "x realisations > 2432, or coarse nodes per line x n_eig > 640)";
      return MSTOPO_INVALID_ARG;
    }
    double* cLd;
    CKB(cudaMalloc(&pc.d_cLinv, nsv * nlA * 8));
    CKB(cudaMalloc(&pc.d_cLinvT, nsv * nlA * 8));
    CKB(cudaMalloc(&pc.d_cW, nsv * nlA * 8));
    CKB(cudaMalloc(&pc.d_cV, nsv * nlA * 8));
    CKB(cudaMalloc(&cLd, (size_t)cdiv(nbc, 32) * 32 * 32 * 8));
    CKB(cudaMalloc(&cC, (size_t)2 * nnc * 8));
    CKB(cudaMalloc(&cS, (size_t)nnc * 8));
    for (int k = 0; k < nsv; ++k)
      CKB(coarse_bt_factor(cA + k * nlA, cB + k * nlB, nbc, NLc, pc.d_cLinv + k * nlA,
                           pc.d_cLinvT + k * nlA, pc.d_cW + k * nlA, pc.d_cV + k * nlA, cS, cC, cLd,
                           d_st + k, s));
    CKB(cudaStreamSynchronize(s));
    cudaFree(cLd); cudaFree(cC); cudaFree(cS);
    pc.d_s2o = d_s2o;
    CKB(cudaMalloc(&pc.d_cy, (size_t)MSTOPO_MAX_SYS * NLc * nbc * 8));
    CKB(cudaMalloc(&pc.d_cx, (size_t)MSTOPO_MAX_SYS * NLc * nbc * 8));
    CKB(cudaMalloc(&pc.d_cbar, sizeof(unsigned int)));
  }
  CKB(cudaMemcpy(cst.data(), d_st, nsv * sizeof(int), cudaMemcpyDeviceToHost));
  cudaFree(cA); cudaFree(cB);
  for (int k = 0; k < nsv; ++k)
    if (cst[k]) {
      h->err = "coarse matrix K_c not positive definite";
      return MSTOPO_NOT_SPD;
    }
  CKB(cudaEventRecord(ev[4], s));

  // 5. patch-solve work groups: per realisation k and type t, P agglomerates each (one
  //    right-hand-side column per agglomerate); groups of realisation k are
  //    [grp_begin[k], grp_begin[k+1]).  P grows with the work so that about one CTA per SM
  //    runs on small meshes and the block streaming is shared by up to PATCH_COLS columns
  //    on large ones.
  std::vector<std::vector<int>> by_type(T);
  for (int i = 0; i < pc.Nc; ++i) by_type[pc.h_type_of_agg[i]].push_back(i);
  auto build_groups = [&](PatchGroups& G, int Pg) -> cudaError_t {
    std::vector<int> perm, gt, gf, gc, gs, agg((size_t)2 * nsv * pc.Nc);
    G.P = Pg;
    G.h_begin.assign(nsv + 1, 0);
    for (int k = 0; k < nsv; ++k) {
      G.h_begin[k] = (int)gt.size();
      for (int t = 0; t < T; ++t)
        for (size_t b = 0; b < by_type[t].size(); b += Pg) {
          const int g = (int)gt.size();
          gt.push_back(k * T + t);
          gs.push_back(k);
          gf.push_back((int)perm.size());
          const int c = (int)std::min<size_t>(Pg, by_type[t].size() - b);
          gc.push_back(c);
          for (int p = 0; p < c; ++p) {
            const int i = by_type[t][b + p];
            agg[(size_t)k * pc.Nc + i] = g;
            agg[((size_t)nsv + k) * pc.Nc + i] = p;
            perm.push_back(i);
          }
        }
    }
    G.h_begin[nsv] = (int)gt.size();
    G.n = (int)gt.size();
    cudaError_t e = cudaSuccess;
    auto up = [&](int*& d, const std::vector<int>& v) {
      if (e == cudaSuccess) e = cudaMalloc(&d, v.size() * sizeof(int));
      if (e == cudaSuccess) e = cudaMemcpy(d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice);
    };
    up(G.d_perm, perm); up(G.d_type, gt); up(G.d_first, gf); up(G.d_count, gc); up(G.d_sys, gs);
    up(G.d_agg, agg);
    return e;
  };
  CKB(cudaStreamSynchronize(s));
  if (!sgs) CKB(build_groups(pc.pg[0], P));
  if (!sgs && (pc.patch_tc || pc.d_ptw)) CKB(build_groups(pc.pg[1], TW_M));
  if (!sgs) CKB(build_groups(pc.pg[2], std::min(P, PATCH_COLS_F64)));
  if (pc.d_ptw) CKB(cudaMalloc(&pc.d_twu, (size_t)pc.pg[1].n * 2 * TW_M * nbP * 4));
  CKB(cudaMalloc(&pc.d_rc, (size_t)MSTOPO_MAX_SYS * Nt * 8));
  CKB(cudaMalloc(&pc.d_uc, (size_t)MSTOPO_MAX_SYS * Nt * 8));
  // work buffer of the patch results: [group][NL][columns][nbP] for the largest group set
  const size_t xg = std::max({(size_t)pc.pg[0].n * PATCH_COLS, (size_t)pc.pg[2].n * PATCH_COLS,
                              (size_t)pc.pg[1].n * TW_M}) * nP;
  if (xg) {
    CKB(cudaMalloc(&pc.d_zp32, xg * 4));
    CKB(cudaMalloc(&pc.d_zp64, xg * 8));
  }
  if (tuned == 1) {
    // time one launch of every candidate (after one untimed launch) on a zero input: the
    // kernels' time does not depend on the values; every exit frees what the timing holds
    float* r0 = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    PatchGroups Gt;
    auto free_groups = [&](PatchGroups& G) {
      dfree(G.d_perm); dfree(G.d_type); dfree(G.d_first); dfree(G.d_count); dfree(G.d_sys); dfree(G.d_agg);
      G = PatchGroups();
    };
    float best_ms = 0.f;
    int best_tc = 0, best_p = P;
    cudaError_t e = cudaMalloc(&r0, (size_t)nsv * h->n_dof * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(r0, 0, (size_t)nsv * h->n_dof * sizeof(float), s);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int cand[4] = {4, 8, 16, TW_M};
    bool first = true;
    for (int ci = 0; ci < 4 && e == cudaSuccess; ++ci) {
      const bool tc = cand[ci] == TW_M;
      if (tc && !pc.d_ptw) continue;
      const PatchGroups* G = &pc.pg[tc ? 1 : 0];
      if (!tc && cand[ci] != P) {
        e = build_groups(Gt, cand[ci]);
        G = &Gt;
      }
      float ms = 0.f;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(t0, s);
        if (e == cudaSuccess)
          e = tc ? patch_twtc_solve(h, *G, r0, 0, nsv, pc.d_zp32, pc.d_twu)
                 : patch_tri_solve_f32(h, *G, r0, 0, nsv, pc.d_zp32);
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
      }
      if (G == &Gt) free_groups(Gt);
      if (e == cudaSuccess && (first || ms < best_ms)) {
        best_ms = ms;
        best_tc = tc ? 1 : 0;
        best_p = cand[ci];
        first = false;
      }
    }
    free_groups(Gt);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    dfree(r0);
    CKB(e);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[tkey] = {best_tc, best_p};
    }
    // keep the winner's pack and groups only
    pc.patch_tc = best_tc;
    if (best_tc) {
      dfree(pc.d_tri32);
      pc.d_tri32 = nullptr;
    } else {
      PatchGroups& G1 = pc.pg[1];
      dfree(G1.d_perm); dfree(G1.d_type); dfree(G1.d_first); dfree(G1.d_count); dfree(G1.d_sys); dfree(G1.d_agg);
      G1 = PatchGroups();
      dfree(pc.d_ptw); dfree(pc.d_twu);
      pc.d_ptw = nullptr;
      pc.d_twu = nullptr;
      if (best_p != P) {
        PatchGroups& G0 = pc.pg[0];
        dfree(G0.d_perm); dfree(G0.d_type); dfree(G0.d_first); dfree(G0.d_count); dfree(G0.d_sys); dfree(G0.d_agg);
        G0 = PatchGroups();
        P = best_p;
        CKB(build_groups(G0, P));
      }
    }
  }
  CKB(cudaEventRecord(ev[5], s));
  // build report
  std::vector<double> eres(T);
  std::vector<int> esw(T);
  CKB(cudaMemcpyAsync(eres.data(), pc.d_eigres, T * 8, cudaMemcpyDeviceToHost, s));
  CKB(cudaMemcpyAsync(esw.data(), pc.d_eigsweeps, T * sizeof(int), cudaMemcpyDeviceToHost, s));
  CKB(cudaStreamSynchronize(s));
  if (info) {
    info->n_agglomerates = pc.Nc;
    info->n_types = T;
    info->n_coarse = Nt;
    info->coarse_solver = pc.coarse_mode;
    info->coarse_line = pc.nbc;
    info->coarse_lines = pc.NLc;
    info->patch_kernel = sgs ? 0 : (pc.patch_tc ? MSTOPO_PATCH_TENSOR_CORES : MSTOPO_PATCH_CUDA_CORES);
    info->patch_groups = sgs ? 0 : pc.pg[pc.patch_tc ? 1 : 0].n;
    info->patch_cols = sgs ? 0 : (pc.patch_tc ? TW_M : pc.pg[0].P);
    info->patch_tuned = tuned;
    info->eig_sweeps = *std::max_element(esw.begin(), esw.end());
    info->eig_residual = *std::max_element(eres.begin(), eres.end());
    cudaEventElapsedTime(&info->ms_hash, ev[0], ev[1]);
    cudaEventElapsedTime(&info->ms_eigen, ev[1], ev[2]);
    cudaEventElapsedTime(&info->ms_patch_factor, ev[2], ev[3]);
    cudaEventElapsedTime(&info->ms_coarse, ev[3], ev[4]);
    cudaEventElapsedTime(&info->ms_total, ev[0], ev[5]);
  }
  for (int q2 = 0; q2 < 6; ++q2) cudaEventDestroy(ev[q2]);
  pc.built = 1;
  return MSTOPO_OK;
}

template <typename T>
static cudaError_t apply_impl(mstopo_handle* h, const T* r, T* z, int sys0, int nsys, int part,
                              const T* psi, T* Xg) {
  Precond& pc = h->pc;
  cudaStream_t s = h->s;
  const long long n = h->n_dof;
  // With both levels, the restriction (and the dense coarse solve) run on the side stream
  // beside the patch solve, which leaves registers and threads free on every SM; the
  // cooperative block sweeps need the whole GPU and follow the join on the main stream.
  const bool fork = part == 0 && h->s_side != nullptr;
  const bool dense = pc.coarse_mode != MSTOPO_COARSE_BLOCKTRI;
  cudaStream_t sc = fork ? h->s_side : s;
  if (fork) {
    cudaError_t e = cudaEventRecord(h->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sc, h->ev_fork, 0);
    if (e != cudaSuccess) return e;
  }
  auto coarse_solve = [&](cudaStream_t st) -> cudaError_t {
    cudaEvent_t pa = prof_begin(h->prof, st);
    if (!dense) {
      const long long so = (long long)sys0 * pc.NLc * pc.nbc * pc.nbc;
      cudaError_t e = coarse_bt_apply(pc.d_cLinv + so, pc.d_cLinvT + so, pc.d_cW + so, pc.d_cV + so,
                                      pc.d_s2o, pc.nbc, pc.NLc, pc.Nt, pc.d_rc, pc.d_uc, nsys,
                                      pc.d_cy, pc.d_cx, pc.d_cbar, h->d_flag + 1, pc.sweep_grid,
                                      h->inject == MSTOPO_INJECT_SWEEP_STALL, st);
      if (h->inject == MSTOPO_INJECT_SWEEP_STALL) h->inject = 0;
      if (e != cudaSuccess) return e;
    } else {
      note_launch(), k_coarse_gemv<<<dim3(cdiv((long long)pc.Nt * 32, 256), nsys), 256, 0, st>>>(pc.d_Kcinv, pc.d_rc, pc.d_uc, pc.Nt, sys0);
    }
    prof_end(h->prof, PROF_COARSE, pa, st);
    return cudaGetLastError();
  };
  if (part != 2) {
    note_launch(), k_restrict<T><<<dim3(pc.Nc, nsys), PC_THREADS, 0, sc>>>(r, n, h->nelx, h->nely, pc.H, pc.ncx,
                                                          pc.d_type_of_agg, pc.d_kept, pc.d_coff,
                                                          psi, pc.kmax, pc.d_rc, pc.Nt);
    if (!fork || dense) {
      cudaError_t e = coarse_solve(sc);
      if (e != cudaSuccess) return e;
    }
  }
  if (fork) {
    cudaError_t e = cudaEventRecord(h->ev_join, sc);
    if (e != cudaSuccess) return e;
  }
  bool use_tc = false;
  if constexpr (sizeof(T) == 4) use_tc = pc.patch_tc != 0;
  const PatchGroups& G = pc.pg[sizeof(T) == 8 ? 2 : (use_tc ? 1 : 0)];
  int Rcols = 4;
  if (part != 1) {
    Rcols = use_tc ? TW_M : patch_tri_cols(G.P);
    cudaEvent_t pa = prof_begin(h->prof, s);
    cudaError_t e;
    if constexpr (sizeof(T) == 4) {
      e = use_tc ? patch_twtc_solve(h, G, r, sys0, nsys, Xg, pc.d_twu)
                 : patch_tri_solve_f32(h, G, r, sys0, nsys, Xg);
    } else {
      e = patch_tri_solve_f64(h, G, r, sys0, nsys, Xg);
    }
    if (e != cudaSuccess) return e;
    prof_end(h->prof, PROF_PATCH, pa, s);
  }
  if (fork) {
    cudaError_t e = cudaStreamWaitEvent(s, h->ev_join, 0);
    if (e != cudaSuccess) return e;
    if (!dense) {
      e = coarse_solve(s);
      if (e != cudaSuccess) return e;
    }
  }
  note_launch(), k_combine<T><<<dim3(cdiv(h->nelx + 1, 128), h->nely + 1, nsys), 128, 0, s>>>(z, n, sys0, pc.Nc, h->nelx, h->nely, pc.H, pc.ncx, pc.ncy,
                                               pc.d_type_of_agg, pc.d_kept, pc.d_coff, psi, pc.kmax,
                                               pc.d_uc, pc.Nt, G.d_agg, G.d_agg + (size_t)pc.nsv * pc.Nc, Xg,
                                               Rcols, use_tc ? 1 : 0, h->d_nmask, part);
  return cudaGetLastError();
}

cudaError_t precond_apply_f64(mstopo_handle* h, const double* r, double* z, int sys0, int nsys,
                              int part) {
  Precond& pc = h->pc;
  if (pc.kind == MSTOPO_PREC_MULTIPLICATIVE_SGS && part != 1)
    return sgs_apply_f64(h, r, z, sys0, nsys, part);
  return apply_impl<double>(h, r, z, sys0, nsys, part, pc.d_psi64, pc.d_zp64);
}

cudaError_t precond_apply_f32(mstopo_handle* h, const float* r, float* z, int sys0, int nsys,
                              int part) {
  Precond& pc = h->pc;
  if (pc.kind == MSTOPO_PREC_MULTIPLICATIVE_SGS && part != 1)
    return sgs_apply_f32(h, r, z, sys0, nsys, part);
  return apply_impl<float>(h, r, z, sys0, nsys, part, pc.d_psi32, pc.d_zp32);
}
