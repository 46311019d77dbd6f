// Overlapping patch solves of the additive two-level preconditioner (Sec. 2.4.2: the exact
// local solves z_i = K_i^-1 R_i r on every agglomerate patch), one CTA per group of patches
// of one type and realisation (R right-hand sides), streaming one symmetric block per line.
//
// The patch matrix is block tridiagonal over the NL node rows ("lines") of its box, with
// diagonal blocks A_k and couplings B_k = A_{k,k-1} (each DOF couples with the 6 DOFs of the
// three neighbouring nodes of the previous line).  Block elimination gives the Schur
// complements S_0 = A_0, S_k = A_k - B_k S_{k-1}^-1 B_k^T (S_k = L_k L_k^T in the block
// Cholesky factor), and with w_k = S_k^-1 (b_k - B_k w_{k-1}) the two sweeps are
//   forward   w_k = S_k^-1 (b_k - B_k w_{k-1})                       (w_{-1} = 0)
//   backward  x_k = w_k - S_k^-1 t_k,   t_{k-1} = B_k^T x_k          (t_{NL-1} = 0)
// i.e. one product with the symmetric S_k^-1 per line and sweep, and two sparse products
// with B_k.  Per line and right-hand side that is nb^2 multiply-adds on a factor of about
// nb^2/2 stored entries: the work of a banded triangular solve pair, 4 n b flops per patch
// and application.  S_k^-1 = L_k^-T L_k^-1 is formed in FP64 and rounded once, so the FP32
// solve carries one rounding of each factor entry (no product of two inverse factors).
//
// Packed line block (one cp.async.bulk per line, ring of NBUF stages in shared memory):
//   rows of S_k^-1 in row blocks of 32: block I < nfull holds 32 rows of width 32(I+1) (the
//   lower triangle by 32 x 32 chunks, the diagonal chunk complete) at row stride 32(I+1) + 2;
//   the last, partial block (nb % 32 rows) holds its rows complete, width and stride
//   32 ceil(nb/32) (+ 2).  A stride of 2 mod 32 words puts the rows a warp reads along a row
//   on distinct banks; reads along a column take 32 consecutive words.  Entries beyond nb are
//   zero.  Then B_k as [6][nb] (entry q of row 2a+c is column 2a-2+q, zero outside the line;
//   zero for k = 0): consecutive rows on consecutive banks.
//
// Product y = S_k^-1 t: each warp owns 16 rows of a full row block I (lane = row, two lanes
// per row splitting the reduction) and forms them completely: the chunks (I, J <= I) along
// the rows (float2 loads, conflict-free at a stride of 2 mod 32 words), the chunks (J' > I, I)
// below them down their columns, and the rank-rem contribution of the partial block's rows;
// every row block costs the same nfull chunks, so the warps are balanced and no partial sums
// cross warps.  One more warp forms the partial block's complete rows (lanes over columns,
// warp reduction in a fixed order): the result is bitwise repeatable.  Every wait is bounded;
// on a timeout the CTA records MSTOPO_TIMEOUT, stops, waits (bounded) for the copies it issued
// and exits.
#include "blocktri.cuh"
#include "internal.cuh"

namespace {

constexpr int TMAXW = 9;              // warps per CTA: 2 per full row block (nb = 130: 8) + the edge warp

// bounded wait for a copy this CTA issued (the drain on exit ignores other aborts)
__device__ __forceinline__ bool tri_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < BT_WAIT_LIMIT; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// R consecutive T values -> registers (16-byte accesses; R a multiple of 16 / sizeof(T))
template <typename T, int R>
__device__ __forceinline__ void ld_row(const T* p, T (&v)[R]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int j = 0; j < R; j += 4) {
      const float4 q = *reinterpret_cast<const float4*>(p + j);
      v[j] = q.x; v[j + 1] = q.y; v[j + 2] = q.z; v[j + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < R; j += 2) {
      const double2 q = *reinterpret_cast<const double2*>(p + j);
      v[j] = q.x; v[j + 1] = q.y;
    }
  }
}

}  // namespace

// Geometry of one packed line block (host and device).
struct TriGeom {
  int nb, nfull, rem, nrb;   // DOFs per line, full 32-row blocks, rows of the last block, row blocks
  int S[6], off[6];          // row stride and offset of every row block
  int TB, LB;                // offset of the coupling block; elements per line block (16-byte multiple)
  int NV;                    // rows of the shared-memory vectors (32 nrb, zero beyond nb)
};

TriGeom tri_geometry(int nb) {
  TriGeom g{};
  g.nb = nb;
  g.nfull = nb / 32;
  g.rem = nb % 32;
  g.nrb = (nb + 31) / 32;
  int o = 0;
  for (int I = 0; I < g.nrb; ++I) {
    const bool full = I < g.nfull;
    g.S[I] = (full ? 32 * (I + 1) : 32 * g.nrb) + 2;
    g.off[I] = o;
    o += (full ? 32 : g.rem) * g.S[I];
  }
  g.TB = (o + 3) / 4 * 4;
  g.LB = (g.TB + 6 * nb + 3) / 4 * 4;
  g.NV = 32 * g.nrb;
  return g;
}

__device__ __forceinline__ int tri_rowoff(const TriGeom& g, int r) {
  const int I = r >> 5;
  return g.off[I] + (r & 31) * g.S[I];
}

// Pack per (system, line): S_k^-1 = Linv_k^T Linv_k (FP64 sums) in the row-block layout, then
// B_k = A_{k,k-1} as [6][nb].  Linv: [sys][NL][nb][nb] FP64 (lower triangular); B:
// [sys][NL-1][nb][nb] FP64.  out64 / out32 may be null.
__global__ void k_patch_tri_pack(const double* __restrict__ Linv, const double* __restrict__ B,
                                 int NL, TriGeom g, double* __restrict__ out64,
                                 float* __restrict__ out32) {
  const int sys = blockIdx.x, k = blockIdx.y;
  const int nb = g.nb;
  const long long nn = (long long)nb * nb;
  const double* Lk = Linv + ((long long)sys * NL + k) * nn;
  const double* Bk = k > 0 ? B + ((long long)sys * (NL - 1) + k - 1) * nn : nullptr;
  const long long o = ((long long)sys * NL + k) * g.LB;
  for (int t = threadIdx.x; t < g.LB; t += blockDim.x) {
    double v = 0.0;
    if (t < g.TB) {
      int I = g.nrb - 1;
      while (I > 0 && t < g.off[I]) --I;
      const int u = t - g.off[I];
      const int r = 32 * I + u / g.S[I], c = u % g.S[I];
      const int width = I < g.nfull ? 32 * (I + 1) : nb;
      if (r < nb && c < nb && c < width) {
        // (Linv^T Linv)[r][c] = sum over l >= max(r, c) of Linv[l][r] Linv[l][c]
        for (int l = r > c ? r : c; l < nb; ++l) v = fma(Lk[(long long)l * nb + r], Lk[(long long)l * nb + c], v);
      }
    } else if (t < g.TB + 6 * nb) {
      const int u = t - g.TB, q = u / nb, r = u % nb;
      const int c = 2 * (r >> 1) - 2 + q;
      if (Bk && c >= 0 && c < nb) v = Bk[(long long)r * nb + c];
    }
    if (out64) out64[o + t] = v;
    if (out32) out32[o + t] = (float)v;
  }
}

// Groups g0 + blockIdx.x (see PatchGroups): R columns = up to R patches of one type and
// realisation; right-hand sides gathered from system grp_sys[g] - sys0 of r.  Work buffer
// Xg: [group][NL][nb][R] holds w_k after the forward sweep, then [group][NL][R][nb] holds x_k.
// Launched with 32 (2 nfull + (rem > 0)) threads; TPF (row, 16-byte chunk) pairs per thread
// cover the vector phases (nb R / (16 / sizeof(T)) <= TPF x threads).
template <typename T, int R, int NBUF, int MINB, int TPF>
__global__ void __launch_bounds__(32 * TMAXW, MINB) k_patch_tri(
    const T* __restrict__ r, long long stride, int sys0, int g0, int nelx, int nely, int H,
    int ncx, const int* __restrict__ grp_type, const int* __restrict__ grp_sys,
    const int* __restrict__ grp_first, const int* __restrict__ grp_count,
    const int* __restrict__ perm, const uint8_t* __restrict__ pfree, const T* __restrict__ pack,
    TriGeom geo, T* __restrict__ Xg, int* __restrict__ err) {
  constexpr int VW = 16 / sizeof(T);          // elements per 16-byte chunk
  constexpr int RC = R / VW;                  // chunks per vector row
  static_assert(R % VW == 0, "R must fill 16-byte chunks");
  __shared__ __align__(8) uint64_t bars[NBUF];
  __shared__ int s_abort;
  __shared__ int s_node[16];
  __shared__ int s_rowoff[160];               // offset of every factor row in a line block
  extern __shared__ __align__(16) unsigned char smraw[];

  const int nb = geo.nb, NV = geo.NV, nfull = geo.nfull, rem = geo.rem;
  const int nrw = 2 * nfull;                  // row warps (16 rows each); warp nrw is the edge warp
  const int NTH = blockDim.x;
  const int N = 2 * H + 1, NL = N;
  const int grp = g0 + blockIdx.x;
  const int type = grp_type[grp], first = grp_first[grp], cnt = grp_count[grp];
  const T* rs = r + (long long)(grp_sys[grp] - sys0) * stride;
  const uint8_t* fr = pfree + (long long)type * N * nb;
  const T* src = pack + (long long)type * NL * geo.LB;
  T* X = Xg + (long long)grp * NL * R * nb;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool edge_warp = warp == nrw;

  T* ring = reinterpret_cast<T*>(smraw);                  // [NBUF][LB]
  T* vt = ring + (long long)NBUF * geo.LB;                // [NV][R] input t of the product
  T* vy = vt + NV * R;                                    // [NV][R] its result S^-1 t
  T* vw = vy + NV * R;                                    // [NV][R] w_k or x_k
  T* vp = vw + NV * R;                                    // [NV][R] w_{k-1} (forward)

  if (tid < 16) s_node[tid] = tid < cnt ? perm[first + tid] : -1;
  for (int q = tid; q < nb; q += NTH) s_rowoff[q] = tri_rowoff(geo, q);
  if (tid == 0) {
    s_abort = 0;
    for (int b = 0; b < NBUF; ++b) mbar_init(&bars[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // zero the vectors (rows nb..NV-1 stay zero for the whole solve)
  for (int q = tid; q < 4 * NV * R; q += NTH) vt[q] = T(0);
  __syncthreads();

  // ---- line-block stream: sequence m = 0 .. 2NL-1, line(m) = m (forward), 2NL-1-m (backward)
  const int nseq = 2 * NL;
  const uint32_t bytes = (uint32_t)((long long)geo.LB * sizeof(T));
  auto line_of = [&](int m) { return m < NL ? m : 2 * NL - 1 - m; };
  int issued = 0;   // copies issued (thread 0's count)
  if (tid == 0)
    for (; issued < NBUF && issued < nseq; ++issued) {
      mbar_expect_tx(&bars[issued], bytes);
      bulk_g2s(ring + (long long)issued * geo.LB, src + (long long)line_of(issued) * geo.LB, bytes,
               &bars[issued]);
    }
  uint32_t phase = 0u;   // bit b: parity of the next wait on stage b

  // vector phases: (row, 16-byte chunk) pairs q = tid + s NTH, s < TPF (nb RC <= TPF NTH)
  T pf[TPF][VW];                                   // next line's input chunks
  auto gather = [&](int k, T (&dst)[TPF][VW]) {    // forward input b_k: r at the patch's DOFs
#pragma unroll
    for (int s = 0; s < TPF; ++s) {
      const int q = tid + s * NTH;
#pragma unroll
      for (int e = 0; e < VW; ++e) dst[s][e] = T(0);
      if (q >= nb * RC) continue;
      const int row = q / RC, ch = q % RC;
      if (!fr[(long long)k * nb + row]) continue;
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const int p = ch * VW + e;
        if (p < cnt) {
          const int ia = s_node[p];
          const int I = ia % (ncx + 1), J = ia / (ncx + 1);
          const int x = (I - 1) * H + (row >> 1), y = (J - 1) * H + k;
          if (x >= 0 && x <= nelx && y >= 0 && y <= nely)
            dst[s][e] = rs[2 * ((long long)y * (nelx + 1) + x) + (row & 1)];
        }
      }
    }
  };
  auto load_w = [&](int k, T (&dst)[TPF][VW]) {   // w_k from the work buffer ([nb][R])
#pragma unroll
    for (int s = 0; s < TPF; ++s) {
      const int q = tid + s * NTH;
      if (q >= nb * RC) continue;
      const int row = q / RC, ch = q % RC;
      const T* p = X + ((long long)k * nb + row) * R + ch * VW;
      if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        dst[s][0] = v.x; dst[s][1] = v.y; dst[s][2] = v.z; dst[s][3] = v.w;
      } else {
        const double2 v = *reinterpret_cast<const double2*>(p);
        dst[s][0] = v.x; dst[s][1] = v.y;
      }
    }
  };

  // vy = S^-1 vt.  Row warp w owns rows 16 w .. 16 w + 15 (row block I = w / 2); lane
  // i + 16 h takes row 16 w + i and half h of every reduction.
  auto product = [&](const T* L) {
    if (warp < nrw) {
      const int I = warp >> 1, i = lane & 15, h = lane >> 4;
      const int row = 16 * warp + i;
      const int col = row - 32 * I;              // the row's column inside chunks (J' > I, I)
      T acc[R], acc1[R];          // even and odd columns: two independent FMA chains
#pragma unroll
      for (int j = 0; j < R; ++j) { acc[j] = T(0); acc1[j] = T(0); }
      // chunks (I, J <= I) along the row: columns 32 J + 16 h .. + 15, in pairs
      const T* Lr = L + s_rowoff[row] + 16 * h;
      for (int J = 0; J <= I; ++J) {
        const T* Lc = Lr + 32 * J;
        const T* tv = vt + (long long)(32 * J + 16 * h) * R;
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
          T a0, a1;
          if constexpr (sizeof(T) == 4) {
            const float2 a = *reinterpret_cast<const float2*>(Lc + c);
            a0 = a.x; a1 = a.y;
          } else {
            a0 = Lc[c]; a1 = Lc[c + 1];
          }
          T v0[R], v1[R];
          ld_row<T, R>(tv + c * R, v0);
          ld_row<T, R>(tv + (c + 1) * R, v1);
#pragma unroll
          for (int j = 0; j < R; ++j) { acc[j] = fma(a0, v0[j], acc[j]); acc1[j] = fma(a1, v1[j], acc1[j]); }
        }
      }
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] += acc1[j];
      // chunks (J' > I, I) down column `col`: half h takes the rows 32 J' + {0..7, 16..23} + 8 h
      // (8 rows apart, the two halves read disjoint banks)
      for (int J2 = I + 1; J2 < nfull; ++J2) {
        const int S2 = 32 * (J2 + 1) + 2;                       // row stride of block J2
        const T* La = L + s_rowoff[32 * J2 + 8 * h] + 32 * I + col;
        const T* ta = vt + (long long)(32 * J2 + 8 * h) * R;
        T acc2[R];
#pragma unroll
        for (int j = 0; j < R; ++j) acc2[j] = T(0);
#pragma unroll
        for (int s2 = 0; s2 < 16; ++s2) {
          const int dr = (s2 & 7) + ((s2 >> 3) << 4);           // 0..7, 16..23
          const T a = La[dr * S2];
          T v[R];
          ld_row<T, R>(ta + dr * R, v);
          if (s2 & 1) {
#pragma unroll
            for (int j = 0; j < R; ++j) acc2[j] = fma(a, v[j], acc2[j]);
          } else {
#pragma unroll
            for (int j = 0; j < R; ++j) acc[j] = fma(a, v[j], acc[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] += acc2[j];
      }
      // the partial block's rows (complete rows stored): column `row` of each
      for (int e = h; e < rem; e += 2) {
        const int rw = 32 * nfull + e;
        const T a = L[s_rowoff[rw] + row];
        T v[R];
        ld_row<T, R>(vt + (long long)rw * R, v);
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] = fma(a, v[j], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], 16);
      if (h == 0) {
#pragma unroll
        for (int j = 0; j < R; ++j) vy[(long long)row * R + j] = acc[j];
      }
    } else if (edge_warp) {
      // complete rows of the partial block
      for (int e0 = 0; e0 < rem; e0 += 2) {
        const int r0 = 32 * nfull + e0, r1 = r0 + 1 < nb ? r0 + 1 : r0;
        const T* L0 = L + s_rowoff[r0];
        const T* L1 = L + s_rowoff[r1];
        T a0[R], a1[R];
#pragma unroll
        for (int j = 0; j < R; ++j) { a0[j] = T(0); a1[j] = T(0); }
        for (int c = lane; c < NV; c += 32) {
          T v[R];
          ld_row<T, R>(vt + (long long)c * R, v);
          const T l0 = L0[c], l1 = L1[c];
#pragma unroll
          for (int j = 0; j < R; ++j) { a0[j] = fma(l0, v[j], a0[j]); a1[j] = fma(l1, v[j], a1[j]); }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int j = 0; j < R; ++j) {
            a0[j] += __shfl_xor_sync(0xffffffffu, a0[j], o);
            a1[j] += __shfl_xor_sync(0xffffffffu, a1[j], o);
          }
        if (lane == 0) {
#pragma unroll
          for (int j = 0; j < R; ++j) vy[(long long)r0 * R + j] = a0[j];
          if (r1 != r0) {
#pragma unroll
            for (int j = 0; j < R; ++j) vy[(long long)r1 * R + j] = a1[j];
          }
        }
      }
    }
  };
  auto result = [&](int q) -> T { return vy[q]; };

  T wk[TPF][VW];                 // backward: w_k of the current line (registers)
  gather(0, pf);
  bool abort = false;
  // thread 0 waits for the block of step m before a barrier that precedes its first use
  auto wait_stage = [&](int m) {
    const int b = m % NBUF;
    if (tid == 0 && !s_abort && !mbar_wait(&bars[b], (phase >> b) & 1u)) {
      s_abort = 1;
      atomicExch(err, (int)MSTOPO_TIMEOUT);
    }
    phase ^= 1u << b;
  };
  wait_stage(0);
  __syncthreads();
  for (int m = 0; m < nseq; ++m) {
    if constexpr (NBUF == 1) {   // one stage: block m was issued at the end of step m - 1
      if (m > 0) {
        wait_stage(m);
        __syncthreads();
      }
    }
    if (s_abort) { abort = true; break; }
    const bool fw = m < NL;
    const int k = line_of(m);
    const int b = m % NBUF;
    const T* L = ring + (long long)b * geo.LB;
    const T* Bq = L + geo.TB;
    if (fw) {
      // t = b_k - B_k w_{k-1}
#pragma unroll
      for (int s = 0; s < TPF; ++s) {
        const int q = tid + s * NTH;
        if (q >= nb * RC) continue;
        const int row = q / RC, ch = q % RC;
        T v[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) v[e] = pf[s][e];
        if (k > 0) {
          const int cb = 2 * (row >> 1) - 2;
#pragma unroll
          for (int qq = 0; qq < 6; ++qq) {
            const int c = cb + qq;
            if (c < 0 || c >= nb) continue;
            const T bq = Bq[qq * nb + row];
#pragma unroll
            for (int e = 0; e < VW; ++e) v[e] = fma(-bq, vp[c * R + ch * VW + e], v[e]);
          }
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) vt[row * R + ch * VW + e] = v[e];
      }
      if (k + 1 < NL) gather(k + 1, pf);   // next line's input, in flight during the product
      __syncthreads();
      product(L);
      if (NBUF > 1 && m + 1 < nseq) wait_stage(m + 1);
      __syncthreads();
      // w_k = S_k^-1 t (in vy): to the work buffer for the backward sweep (w_{NL-1} stays in
      // shared memory: the first backward line rewrites that slice with no barrier between);
      // it becomes w_{k-1} of the next line
      if (k + 1 < NL) {
        T* Xk = X + (long long)k * nb * R;
        for (int q = tid; q < nb * R; q += NTH) Xk[q] = vy[q];
      }
      T* tmp = vp; vp = vy; vy = tmp;
    } else {
      // backward line k: x_k = w_k - S_k^-1 t_k, t_k = B_{k+1}^T x_{k+1} already in vt.
      // w_k was loaded from the work buffer in the previous step (before its barrier, so no
      // load can see this step's x_k stores into the same slice); w_{NL-1} is still in vp.
      const bool first = m == NL;           // t_{NL-1} = 0: x = w
      if (first) {
#pragma unroll
        for (int s = 0; s < TPF; ++s) {
          const int q = tid + s * NTH;
          if (q >= nb * RC) continue;
          const int row = q / RC, ch = q % RC;
#pragma unroll
          for (int e = 0; e < VW; ++e) wk[s][e] = vp[row * R + ch * VW + e];
        }
      } else {
        product(L);
        __syncthreads();
      }
      T* Xk = X + (long long)k * nb * R;
#pragma unroll
      for (int s = 0; s < TPF; ++s) {
        const int q = tid + s * NTH;
        if (q >= nb * RC) continue;
        const int row = q / RC, ch = q % RC;
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          const int j = ch * VW + e;
          const T x = first ? wk[s][e] : wk[s][e] - result(row * R + j);
          vw[row * R + j] = x;
          Xk[(long long)j * nb + row] = x;   // [R][nb] for the combine step
        }
      }
      if (k > 0) load_w(k - 1, wk);
      __syncthreads();
      // t_{k-1} = B_k^T x_k  (column c of line k-1 gathers rows of nodes (c>>1) - 1 .. + 1)
      if (k > 0) {
        for (int q = tid; q < nb * RC; q += NTH) {
          const int c = q / RC, ch = q % RC;
          T v[VW];
#pragma unroll
          for (int e = 0; e < VW; ++e) v[e] = T(0);
          const int a = c >> 1;
          for (int an = a - 1; an <= a + 1; ++an) {
            if (an < 0 || 2 * an >= nb) continue;
#pragma unroll
            for (int cr = 0; cr < 2; ++cr) {
              const int row = 2 * an + cr;
              const int qq = c - (2 * an - 2);
              const T bq = Bq[qq * nb + row];
#pragma unroll
              for (int e = 0; e < VW; ++e) v[e] = fma(bq, vw[row * R + ch * VW + e], v[e]);
            }
          }
#pragma unroll
          for (int e = 0; e < VW; ++e) vt[c * R + ch * VW + e] = v[e];
        }
      }
      if (NBUF > 1 && m + 1 < nseq) wait_stage(m + 1);
      __syncthreads();
    }
    // every read of stage b is behind a barrier: refill it with block m + NBUF
    if (tid == 0 && issued < nseq && !s_abort) {
      const int st = issued % NBUF;   // == b
      mbar_expect_tx(&bars[st], bytes);
      bulk_g2s(ring + (long long)st * geo.LB, src + (long long)line_of(issued) * geo.LB, bytes,
               &bars[st]);
      ++issued;
    }
  }
  if (abort && tid == 0) {
    // every copy issued and not yet waited for lands before the CTA exits
    for (int m2 = 0; m2 < NBUF; ++m2) {
      const int last = issued - 1 - m2;    // copy `last` went to stage last % NBUF
      if (last < 0) break;
      const int st = last % NBUF;
      const uint32_t par = (uint32_t)((last / NBUF) & 1);
      if (!tri_wait(&bars[st], par)) atomicExch(err, (int)MSTOPO_TIMEOUT);
    }
  }
}

// ------------------------------------------------------------------------------ host side
static int tri_threads(int nb) { return 32 * (2 * (nb / 32) + (nb % 32 ? 1 : 0)); }

size_t patch_tri_smem(int nb, int R, int nbuf, size_t elem) {
  const TriGeom g = tri_geometry(nb);
  return ((size_t)nbuf * g.LB + 4 * (size_t)g.NV * R) * elem;
}

long long patch_tri_line_elems(int nb) { return tri_geometry(nb).LB; }

// the kernel's thread layout covers this line size: at most 9 warps, rows addressed through
// a 160-entry table, every vector phase within 4 pairs per thread (16 patches per CTA)
bool patch_tri_assignment_ok(int nb) {
  const int nt = tri_threads(nb);
  return nb >= 2 && nb <= 160 && nt <= 32 * TMAXW && nb * 4 <= 4 * nt;
}

cudaError_t patch_tri_pack(const double* Linv, const double* B, int nsys, int nb, int NL,
                           double* out64, float* out32, cudaStream_t s) {
  const TriGeom g = tri_geometry(nb);
  note_launch(), k_patch_tri_pack<<<dim3(nsys, NL), 256, 0, s>>>(Linv, B, NL, g, out64, out32);
  return cudaGetLastError();
}

template <typename T, int R, int NBUF, int TPF>
static cudaError_t launch_tri_kt(mstopo_handle* h, const PatchGroups& G, const T* r, int sys0,
                                 int nsys, const T* pack, T* Xg) {
  constexpr int MINB = (sizeof(T) == 4 && R <= 4) ? 2 : 1;   // two CTAs per SM at four columns
  Precond& pc = h->pc;
  const TriGeom geo = tri_geometry(pc.nbP);
  const size_t sm = patch_tri_smem(pc.nbP, R, NBUF, sizeof(T));
  {
    cudaError_t e = smem_limit_max<k_patch_tri<T, R, NBUF, MINB, TPF>>();
    if (e != cudaSuccess) return e;
  }
  if (sm > 225 * 1024 || !patch_tri_assignment_ok(pc.nbP)) return cudaErrorInvalidConfiguration;
  const int g0 = G.h_begin[sys0], ng = G.h_begin[sys0 + nsys] - g0;
  if (ng <= 0) return cudaSuccess;
  note_launch(), k_patch_tri<T, R, NBUF, MINB, TPF><<<ng, tri_threads(pc.nbP), sm, h->s>>>(
      r, h->n_dof, sys0, g0, h->nelx, h->nely, pc.H, pc.ncx, G.d_type, G.d_sys, G.d_first,
      G.d_count, G.d_perm, pc.d_pfree, pack, geo, Xg, h->d_flag + 1);
  return cudaGetLastError();
}

// one (row, 16-byte chunk) pair per thread when the threads cover the vector phases, else four
template <typename T, int R, int NBUF>
static cudaError_t launch_tri_k(mstopo_handle* h, const PatchGroups& G, const T* r, int sys0,
                                int nsys, const T* pack, T* Xg) {
  const int nb = h->pc.nbP;
  if (nb * (R * (int)sizeof(T) / 16) <= tri_threads(nb))
    return launch_tri_kt<T, R, NBUF, 1>(h, G, r, sys0, nsys, pack, Xg);
  return launch_tri_kt<T, R, NBUF, 4>(h, G, r, sys0, nsys, pack, Xg);
}

cudaError_t patch_tri_solve_f32(mstopo_handle* h, const PatchGroups& G, const float* r, int sys0,
                                int nsys, float* Xg) {
  const float* pack = h->pc.d_tri32;
  switch (patch_tri_cols(G.P)) {
    case 4: return launch_tri_k<float, 4, 2>(h, G, r, sys0, nsys, pack, Xg);
    case 8: return launch_tri_k<float, 8, 2>(h, G, r, sys0, nsys, pack, Xg);
    default: return launch_tri_k<float, 16, 2>(h, G, r, sys0, nsys, pack, Xg);
  }
}

cudaError_t patch_tri_solve_f64(mstopo_handle* h, const PatchGroups& G, const double* r, int sys0,
                                int nsys, double* Xg) {
  const double* pack = h->pc.d_tri64;
  switch (patch_tri_cols(G.P)) {
    case 4: return launch_tri_k<double, 4, 1>(h, G, r, sys0, nsys, pack, Xg);
    default: return cudaErrorInvalidConfiguration;   // FP64 groups hold at most 4 patches
  }
}
