// Block-tridiagonal SPD factorisation and solves, one CTA per system.
//
// The structured sub-grid operators of the two-level preconditioner -- agglomerate and
// patch matrices (node rows of a (2H+-1)^2 box) and the coarse matrix (coarse-node lines,
// whose basis functions only overlap their 3x3 coarse neighbours) -- are block
// tridiagonal: diagonal blocks A_k and sub-diagonal blocks B_k = A_{k+1,k}, nb x nb each.
// Block Cholesky:  S_0 = A_0,  L_k = chol(S_k),  C_k = B_k L_k^-T,  S_{k+1} = A_{k+1} - C_k C_k^T.
// Stored per line: Linv_k = L_k^-1 (dense, lower) and C_k, so that both solve sweeps are
// dense block products with no sequential triangular substitution inside a line:
//   forward   y_k = Linv_k (b_k - C_{k-1} y_{k-1})
//   backward  x_k = Linv_k^T (y_k - C_k^T x_{k+1}).
// Matrices are row-major nb x nb.  Vectors of R right-hand sides are [NL][nb][R].
#pragma once
#include "internal.cuh"

// ------------------------------------------------------------------- factorisation (FP64)
// S (nb x nb, global or shared) := lower Cholesky factor of S, in place.  Returns 0 on
// success, or 1 + the failing pivot index.  Whole CTA participates.
__device__ inline int bt_chol_inplace(double* S, int nb, int* sh_fail, double* dinv) {
  __shared__ double sh_inv;
  if (threadIdx.x == 0) *sh_fail = 0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      double d = S[j * nb + j];
      if (!(d > 0.0) || !isfinite(d)) {
        if (*sh_fail == 0) *sh_fail = 1 + j;
        d = 1.0;
      }
      const double l = sqrt(d);
      S[j * nb + j] = l;
      sh_inv = 1.0 / l;             // one FP64 division per pivot, not one per thread
      dinv[j] = sh_inv;
    }
    __syncthreads();
    const double inv = sh_inv;
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) S[i * nb + j] *= inv;
    __syncthreads();
    // trailing update of the lower triangle: S[i][l] -= S[i][j] S[l][j], j < l <= i
    const int m = nb - j - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      int i = j + 1 + t / m, l = j + 1 + t % m;
      if (l <= i) S[i * nb + l] = fma(-S[i * nb + j], S[l * nb + j], S[i * nb + l]);
    }
    __syncthreads();
  }
  return *sh_fail;
}

// Linv := L^-1 for lower-triangular L (upper part of Linv set to 0), dinv[i] = 1 / L[i][i].
// One thread per column.
__device__ inline void bt_tri_inverse(const double* L, const double* dinv, double* Linv, int nb) {
  for (int c = threadIdx.x; c < nb; c += blockDim.x) {
    for (int i = 0; i < c; ++i) Linv[i * nb + c] = 0.0;
    for (int i = c; i < nb; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int l = c; l < i; ++l) s = fma(-L[i * nb + l], Linv[l * nb + c], s);
      Linv[i * nb + c] = s * dinv[i];
    }
  }
  __syncthreads();
}

// Factor one block-tridiagonal system.  A: [NL][nb][nb], B: [NL-1][nb][nb] (read only);
// shift: diagonal entries of A are multiplied by (1 + shift) on free DOFs (free[k*nb+i]).
// Outputs Linv [NL][nb][nb], C [NL-1][nb][nb]; S is an nb x nb workspace.
// Returns 0 or 1 + (global row index) of the first non-positive pivot.
__device__ inline int bt_factor(const double* A, const double* B, const uint8_t* free,
                                double shift, int nb, int NL, double* Linv, double* C,
                                double* S, int* sh_fail, double* dinv) {
  const int nn = nb * nb;
  int fail = 0;
  for (int k = 0; k < NL; ++k) {
    const double* Ak = A + (long long)k * nn;
    // S = A_k (+ shift) - C_{k-1} C_{k-1}^T   (C_{k-1} = L_{k,k-1})
    const double* Cp = k > 0 ? C + (long long)(k - 1) * nn : nullptr;
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
      int i = t / nb, l = t % nb;
      double v = Ak[t];
      if (i == l && free && free[k * nb + i]) v *= (1.0 + shift);
      if (Cp && l <= i) {
        double s = 0.0;
        for (int q = 0; q < nb; ++q) s = fma(Cp[i * nb + q], Cp[l * nb + q], s);
        v -= s;
      }
      S[t] = v;
    }
    __syncthreads();
    int f = bt_chol_inplace(S, nb, sh_fail, dinv);
    if (f && !fail) fail = k * nb + f;
    double* Li = Linv + (long long)k * nn;
    bt_tri_inverse(S, dinv, Li, nb);
    if (k + 1 < NL) {
      // C_k = B_k L_k^-T :  C[i][j] = sum_{l <= j} B[i][l] Linv[j][l]
      const double* Bk = B + (long long)k * nn;
      double* Ck = C + (long long)k * nn;
      for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        int i = t / nb, j = t % nb;
        double s = 0.0;
        for (int l = 0; l <= j; ++l) s = fma(Bk[i * nb + l], Li[j * nb + l], s);
        Ck[t] = s;
      }
      __syncthreads();
    }
  }
  return fail;
}

// ------------------------------------------------------------------------- solves
// out[i][r] (+)= sign * sum_c M[i][c] v[c][r]  (TRANS: M[c][i]).  LOWER: M is lower
// triangular (skip the zero half).  M may live in shared or global memory.
template <typename T, bool TRANS, bool LOWER>
__device__ __forceinline__ void bt_gemm(const T* M, const T* v, T* out, int nb, int R,
                                        bool accumulate, T sign) {
  for (int t = threadIdx.x; t < nb * R; t += blockDim.x) {
    int i = t / R, r = t % R;
    int c0 = 0, c1 = nb;
    if (LOWER) {
      if (TRANS) c0 = i;      // (M^T)[i][c] = M[c][i] nonzero for c >= i
      else c1 = i + 1;        // M[i][c] nonzero for c <= i
    }
    T s = T(0);
    for (int c = c0; c < c1; ++c) {
      T m = TRANS ? M[c * nb + i] : M[i * nb + c];
      s = fma(m, v[c * R + r], s);
    }
    out[t] = accumulate ? fma(sign, s, out[t]) : sign * s;
  }
}

// In-place solve with the stored factor.  X: [NL][nb][R] (global).  Shared scratch:
// stage (nb*nb, used when STAGE), t0, t1 (nb*R each).  Whole CTA participates.
template <typename T, bool STAGE>
__device__ void bt_solve(const T* __restrict__ Linv, const T* __restrict__ C, int nb, int NL,
                         T* X, int R, T* stage, T* t0, T* t1) {
  const int nn = nb * nb, nv = nb * R;
  auto mat = [&](const T* M) -> const T* {
    if (!STAGE) return M;
    __syncthreads();
    for (int q = threadIdx.x; q < nn; q += blockDim.x) stage[q] = M[q];
    __syncthreads();
    return stage;
  };
  // forward: t1 holds y_{k-1}
  for (int k = 0; k < NL; ++k) {
    T* Xk = X + (long long)k * nv;
    for (int q = threadIdx.x; q < nv; q += blockDim.x) t0[q] = Xk[q];
    __syncthreads();
    if (k > 0) {
      const T* M = mat(C + (long long)(k - 1) * nn);
      bt_gemm<T, false, false>(M, t1, t0, nb, R, true, T(-1));
    }
    const T* M = mat(Linv + (long long)k * nn);
    __syncthreads();
    bt_gemm<T, false, true>(M, t0, t1, nb, R, false, T(1));
    __syncthreads();
    for (int q = threadIdx.x; q < nv; q += blockDim.x) Xk[q] = t1[q];
  }
  // backward: t1 holds x_{k+1}
  for (int k = NL - 1; k >= 0; --k) {
    T* Xk = X + (long long)k * nv;
    __syncthreads();
    for (int q = threadIdx.x; q < nv; q += blockDim.x) t0[q] = Xk[q];
    __syncthreads();
    if (k + 1 < NL) {
      const T* M = mat(C + (long long)k * nn);
      bt_gemm<T, true, false>(M, t1, t0, nb, R, true, T(-1));
    }
    const T* M = mat(Linv + (long long)k * nn);
    __syncthreads();
    bt_gemm<T, true, true>(M, t0, t1, nb, R, false, T(1));
    __syncthreads();
    for (int q = threadIdx.x; q < nv; q += blockDim.x) Xk[q] = t1[q];
  }
  __syncthreads();
}

// ------------------------------------------------------------- bulk-copy (TMA) staging
// The factor blocks are streamed into shared memory with one cp.async.bulk per block,
// completion tracked by an mbarrier (transaction bytes).  Waits are bounded: after
// BT_WAIT_LIMIT polls the wait gives up, records MSTOPO_TIMEOUT in *err and the solve
// stops issuing work (the host reports the status).
#define BT_WAIT_LIMIT (1u << 24)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < BT_WAIT_LIMIT; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Register-blocked variant for a compile-time number of right-hand sides R: two threads per
// output row split the reduction range and combine with one shuffle; each thread keeps R
// independent accumulators (R-way ILP) and reads each matrix entry once.
template <typename T, bool TRANS, bool LOWER, int R>
__device__ __forceinline__ void bt_gemm_rb(const T* M, const T* v, T* out, int nb,
                                           bool accumulate, T sign) {
  const int rows_per_pass = blockDim.x >> 1;
  for (int base = 0; base < nb; base += rows_per_pass) {
    const int i = base + (threadIdx.x >> 1), half = threadIdx.x & 1;
    T acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = T(0);
    if (i < nb) {
      int c0 = 0, c1 = nb;
      if (LOWER) {
        if (TRANS) c0 = i;
        else c1 = i + 1;
      }
      const int mid = (c0 + c1) >> 1;
      const int cb = half ? mid : c0, ce = half ? c1 : mid;
#pragma unroll 4
      for (int c = cb; c < ce; ++c) {
        const T m = TRANS ? M[c * nb + i] : M[i * nb + c];
        const T* vc = v + c * R;
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = fma(m, vc[r], acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], 1);
    if (i < nb && !half) {
#pragma unroll
      for (int r = 0; r < R; ++r)
        out[i * R + r] = accumulate ? fma(sign, acc[r], out[i * R + r]) : sign * acc[r];
    }
  }
}

// Matrix m of the solve sequence: forward L0, C0, L1, C1, ..., L_{NL-1};
// backward L_{NL-1}, C_{NL-2}, L_{NL-2}, ..., C0, L0.
template <typename T>
__device__ __forceinline__ const T* bt_seq(const T* Linv, const T* C, long long nn, int NL, int m) {
  const int nf = 2 * NL - 1;
  if (m < nf) return (m & 1) ? C + (long long)(m >> 1) * nn : Linv + (long long)(m >> 1) * nn;
  const int b = m - nf;
  return (b & 1) ? C + (long long)(NL - 2 - (b >> 1)) * nn : Linv + (long long)(NL - 1 - (b >> 1)) * nn;
}

// In-place solve like bt_solve, with the factor blocks streamed by bulk copies into NBUF
// shared buffers (NBUF = 2: the next block loads while the current one is used).
// bars: NBUF mbarriers in shared memory; err: global status word.
// X layout: DOF_FAST = false -> [NL][nb][R] (right-hand sides fastest);
//           DOF_FAST = true  -> [NL][R][nb] (DOFs fastest, coalesced gathers and scatters).
template <typename T, int NBUF, int R, bool DOF_FAST>
__device__ void bt_solve_bulk(const T* __restrict__ Linv, const T* __restrict__ C, int nb, int NL,
                              T* X, T* stage, T* t0, T* t1, uint64_t* bars, int* err) {
  const long long nn = (long long)nb * nb;
  const int nv = nb * R;
  const uint32_t bytes = (uint32_t)(nn * sizeof(T));
  const int nseq = 2 * (2 * NL - 1);
  __shared__ int s_abort;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int b = 0; b < NBUF; ++b) mbar_init(&bars[b], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int b = 0; b < NBUF && b < nseq; ++b) {
      mbar_expect_tx(&bars[b], bytes);
      bulk_g2s(stage + b * nn, bt_seq(Linv, C, nn, NL, b), bytes, &bars[b]);
    }
  uint32_t phase[NBUF];
  for (int b = 0; b < NBUF; ++b) phase[b] = 0;
  int m = 0;   // position in the sequence
  auto acquire = [&]() -> const T* {
    const int b = m % NBUF;
    if (threadIdx.x == 0 && !s_abort && !mbar_wait(&bars[b], phase[b])) {
      s_abort = 1;
      atomicExch(err, (int)MSTOPO_TIMEOUT);
    }
    phase[b] ^= 1u;
    __syncthreads();
    return stage + b * nn;
  };
  auto release = [&]() {   // every thread is done with block m: refill its buffer
    __syncthreads();
    const int b = m % NBUF;
    if (threadIdx.x == 0 && !s_abort && m + NBUF < nseq) {
      mbar_expect_tx(&bars[b], bytes);
      bulk_g2s(stage + b * nn, bt_seq(Linv, C, nn, NL, m + NBUF), bytes, &bars[b]);
    }
    ++m;
  };
  auto load = [&](const T* Xk) {
    for (int q = threadIdx.x; q < nv; q += blockDim.x) {
      if (DOF_FAST) t0[(q % nb) * R + q / nb] = Xk[q];
      else t0[q] = Xk[q];
    }
  };
  auto store = [&](T* Xk) {
    for (int q = threadIdx.x; q < nv; q += blockDim.x) {
      if (DOF_FAST) Xk[q] = t1[(q % nb) * R + q / nb];
      else Xk[q] = t1[q];
    }
  };
  for (int k = 0; k < NL; ++k) {
    T* Xk = X + (long long)k * nv;
    load(Xk);
    __syncthreads();
    if (k > 0) {
      const T* M = acquire();
      bt_gemm_rb<T, false, false, R>(M, t1, t0, nb, true, T(-1));
      release();
    }
    const T* M = acquire();
    bt_gemm_rb<T, false, true, R>(M, t0, t1, nb, false, T(1));
    release();
    store(Xk);
  }
  for (int k = NL - 1; k >= 0; --k) {
    T* Xk = X + (long long)k * nv;
    __syncthreads();
    load(Xk);
    __syncthreads();
    if (k + 1 < NL) {
      const T* M = acquire();
      bt_gemm_rb<T, true, false, R>(M, t1, t0, nb, true, T(-1));
      release();
    }
    const T* M = acquire();
    bt_gemm_rb<T, true, true, R>(M, t0, t1, nb, false, T(1));
    release();
    store(Xk);
  }
  __syncthreads();
}
