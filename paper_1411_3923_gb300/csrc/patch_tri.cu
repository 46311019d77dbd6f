// Overlapping patch solves of the additive two-level preconditioner (Sec. 2.4.2: the exact
// local solves z_i = K_i^-1 R_i r on every agglomerate patch) by a two-sided block
// elimination: one cluster of two CTAs per group of patches of one type and realisation
// (R right-hand sides), each CTA streaming one symmetric block per line of its half.
//
// The patch matrix is block tridiagonal over the NL = 2H + 1 node rows ("lines") of its box,
// with diagonal blocks A_k and couplings A_{k,k-1} (each DOF couples with the 6 DOFs of the
// three neighbouring nodes of the previous line).  The elimination runs from both ends toward
// the middle line m = H at once ("twisted" order), so the dependent chain is H + 1 lines long
// instead of NL:
//   top     S_0 = A_0,        S_k = A_k - A_{k,k-1} S_{k-1}^-1 A_{k-1,k}            k < m
//   bottom  U_{NL-1} = A_{NL-1}, U_k = A_k - A_{k,k+1} U_{k+1}^-1 A_{k+1,k}         k > m
//   middle  M = A_m - A_{m,m-1} S_{m-1}^-1 A_{m-1,m} - A_{m,m+1} U_{m+1}^-1 A_{m+1,m}
// and with the forward sweeps of both halves
//   w_k = S_k^-1 (b_k - A_{k,k-1} w_{k-1})  (k < m),   v_k = U_k^-1 (b_k - A_{k,k+1} v_{k+1})  (k > m)
// the solution is
//   x_m = M^-1 (b_m - A_{m,m-1} w_{m-1} - A_{m,m+1} v_{m+1})
//   x_k = w_k - S_k^-1 A_{k,k+1} x_{k+1}  (k < m),   x_k = v_k - U_k^-1 A_{k,k-1} x_{k-1}  (k > m).
// The bottom half is the top half of the line-reversed matrix, so both CTAs run the same
// "chain": line j of CTA rank 1 is patch line NL-1-j, and its coupling block is A_{l,l+1}.
// Per line and right-hand side that is one product with a symmetric inverse (nb^2
// multiply-adds on about nb^2/2 stored entries) and two sparse products with the coupling:
// the work of a banded triangular solve pair, 4 n b flops per patch and application.  The
// inverses are formed in FP64 (S^-1 = L^-T L^-1) and rounded once.
//
// Packed block (one cp.async.bulk each, ring of NBUF stages in shared memory):
//   rows of the symmetric inverse in row blocks of 32: block I < nfull holds 32 rows of width
//   32(I+1) (the lower triangle by 32 x 32 chunks, the diagonal chunk complete) at row stride
//   32(I+1) + 2; the last, partial block (nb % 32 rows) holds its rows complete, width and
//   stride 32 ceil(nb/32) (+ 2).  A stride of 2 mod 32 words puts the rows a warp reads along
//   a row on distinct banks; reads along a column take 32 consecutive words.  Entries beyond
//   nb are zero.  Then the coupling as [6][nb] (entry q of row 2a+c is column 2a-2+q of the
//   neighbouring line, zero outside it; zero for the first line of a chain).  The middle
//   block carries two couplings, A_{m,m-1} (rank 0's) then A_{m,m+1} (rank 1's).
// Per patch system: chain blocks of rank 0 (lines 0..H-1), of rank 1 (lines NL-1..H+1), then
// the middle block.
//
// Product y = S^-1 t: two warps own the 32 rows of a full row block I (each lane two rows,
// 16 apart, two lanes per row pair splitting the reduction, so every vector load feeds two
// rows) and form them completely: the chunks (I, J <= I) along the rows (pairs of columns),
// the chunks (J' > I, I) below them down their columns (pairs of rows), and the partial
// block's rows, split between the two warps, which add their sums behind a barrier of the
// pair.  The partial sums of even and odd columns are carried as pairs (one paired FP32 FMA
// per matrix pair and right-hand side).  Every row block costs the same nfull chunks, so the
// warp pairs are balanced.  One more warp forms the partial block's complete rows (lanes over
// column pairs, warp reduction in a fixed order).  Vectors are [R][NV] in shared memory; the
// vector phases map one thread to a (node, right-hand side) pair.  The results are bitwise
// repeatable.
//
// The two CTAs meet once, at the middle line: each publishes its coupling contribution in its
// own shared memory, both cross a cluster barrier, and both form x_m from the two
// contributions in the same order (identical bits), so nothing else is exchanged.  Every
// mbarrier wait is bounded; on a timeout the CTA records MSTOPO_TIMEOUT, stops computing, still
// crosses both cluster barriers (the partner never waits forever), waits (bounded) for the
// copies it issued and exits.
#include <cooperative_groups.h>

#include <algorithm>

#include "blocktri.cuh"
#include "internal.cuh"
#include "tcgen05.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int TMAXW = 9;        // warps per CTA: 2 per full row block (nb = 130: 8) + the edge warp
constexpr int TMINTH = 128;     // at least this many threads (small boxes: the vector phases)

// bounded wait for a copy this CTA issued (the drain on exit ignores other aborts)
__device__ __forceinline__ bool tri_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < BT_WAIT_LIMIT; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// c + a * b elementwise on a pair: one paired FP32 FMA, two FP64 FMAs
__device__ __forceinline__ float2 fma_pair(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 fma_pair(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}

// barrier of the two warps that share row block I (ids 1..5; id 0 is __syncthreads), with
// constant ids so that the CTA reserves six barriers only
__device__ __forceinline__ void pair_barrier(int I) {
  switch (I) {
    case 0: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
    case 1: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
    case 2: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
    case 3: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
    default: asm volatile("bar.sync 5, 64;" ::: "memory"); break;
  }
}

// four consecutive T as two pairs (16-byte aligned)
template <typename T, typename V2>
__device__ __forceinline__ void ld_quad(const T* p, V2& lo, V2& hi) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    lo = make_float2(q.x, q.y);
    hi = make_float2(q.z, q.w);
  } else {
    lo = *reinterpret_cast<const double2*>(p);
    hi = *reinterpret_cast<const double2*>(p + 2);
  }
}

}  // namespace

// Geometry of one packed block (host and device).
struct TriGeom {
  int nb, nfull, rem, nrb;   // DOFs per line, full 32-row blocks, rows of the last block, row blocks
  int S[6], off[6];          // row stride and offset of every row block
  int TB;                    // offset of the coupling block(s)
  int LB, LBM;               // elements of a chain block / of the middle block (16-byte multiples)
  int NV;                    // rows of the shared-memory vectors (32 nrb, zero beyond nb)
  long long SS;              // elements per patch system
};

static TriGeom tri_geometry(int nb, int NL) {
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
  g.LB = g.TB + 6 * nb;    // nb even: 6 nb is a multiple of 4
  g.LBM = g.TB + 12 * nb;
  g.NV = 32 * g.nrb;
  g.SS = (long long)(NL - 1) * g.LB + g.LBM;
  return g;
}

// offset of factor row r in a block, in closed form (no dynamic indexing of the geometry):
// full row block I starts at sum_{i<I} 32 (32 (i + 1) + 2) = 512 I (I + 1) + 64 I
__device__ __forceinline__ int tri_rowoff(const TriGeom& g, int r) {
  const int I = r >> 5;
  const int S = (I < g.nfull ? 32 * (I + 1) : 32 * g.nrb) + 2;
  return 512 * I * (I + 1) + 64 * I + (r & 31) * S;
}

// Pack per (system, block b): b < H the top chain (line b: Linv_b of the top-down factor,
// coupling A_{b,b-1} = Bt[b-1]); H <= b < 2H the bottom chain (reversed line j = b - H: Linv
// of the reversed factor, coupling A'_{j,j-1} = Br[j-1]); b = 2H the middle line (M^-1 from
// Lm, couplings A_{m,m-1} = Bt[m-1] and A_{m,m+1} = Br[m-1]).  The symmetric inverse is
// (Linv^T Linv)[r][c] = sum over l >= max(r, c) of Linv[l][r] Linv[l][c], in FP64.
__global__ void k_patch_tri_pack(const double* __restrict__ Lt, const double* __restrict__ Bt,
                                 const double* __restrict__ Lr, const double* __restrict__ Br,
                                 const double* __restrict__ Lm, int NL, int NLr, TriGeom g,
                                 double* __restrict__ out64, float* __restrict__ out32) {
  const int sys = blockIdx.x, b = blockIdx.y;
  const int nb = g.nb, H = (NL - 1) / 2;
  const long long nn = (long long)nb * nb;
  const double* Li;
  const double* C0 = nullptr;
  const double* C1 = nullptr;
  int size = g.LB;
  if (b < H) {
    Li = Lt + ((long long)sys * NL + b) * nn;
    if (b > 0) C0 = Bt + ((long long)sys * (NL - 1) + b - 1) * nn;
  } else if (b < 2 * H) {
    const int j = b - H;
    Li = Lr + ((long long)sys * NLr + j) * nn;
    if (j > 0) C0 = Br + ((long long)sys * (NLr - 1) + j - 1) * nn;
  } else {
    Li = Lm + (long long)sys * nn;
    C0 = Bt + ((long long)sys * (NL - 1) + H - 1) * nn;
    C1 = Br + ((long long)sys * (NLr - 1) + H - 1) * nn;
    size = g.LBM;
  }
  const long long o = (long long)sys * g.SS + (long long)b * g.LB;
  for (int t = threadIdx.x; t < size; t += blockDim.x) {
    double v = 0.0;
    if (t < g.TB) {
      int I = g.nrb - 1;
      while (I > 0 && t < g.off[I]) --I;
      const int u = t - g.off[I];
      const int r = 32 * I + u / g.S[I], c = u % g.S[I];
      const int width = I < g.nfull ? 32 * (I + 1) : nb;
      if (r < nb && c < nb && c < width) {
        for (int l = r > c ? r : c; l < nb; ++l) v = fma(Li[(long long)l * nb + r], Li[(long long)l * nb + c], v);
      }
    } else {
      const int u = t - g.TB, rho = u / (6 * nb), u2 = u % (6 * nb);
      const int q = u2 / nb, r = u2 % nb;
      const int c = 2 * (r >> 1) - 2 + q;
      const double* Bk = rho == 0 ? C0 : C1;
      if (Bk && c >= 0 && c < nb) v = Bk[(long long)r * nb + c];
    }
    if (out64) out64[o + t] = v;
    if (out32) out32[o + t] = (float)v;
  }
}

// The tensor-core kernel's blocks (csrc/patch_twtc.cu) from the FP64 pack of the same system:
// the symmetric inverse as TF32 hi/lo tiles (B[n][k] = S^-1[n][k], zero beyond nb; the lower
// triangle of the pack read across the diagonal where a row stores fewer columns), and every
// coupling C with its transpose CT, K[q][c] = the coefficient of neighbour DOF 2(c/2) - 2 + q in
// row c: CT[2 dn + 2 + f][2a + e] = C[2 - 2 dn + e][2 (a + dn) + f] (zero outside the line), so
// that both sweeps apply a coupling with the same six-term stencil; stored per node a as
// [e][q] (12 floats), the pairs (q, q + 1) of one row adjacent.
__global__ void k_patch_twtc_pack(const double* __restrict__ tri64, TriGeom g, TwGeom w, int NL,
                                  unsigned char* __restrict__ out) {
  const int sys = blockIdx.x, b = blockIdx.y;
  const int H = (NL - 1) / 2, nb = g.nb, NN = nb / 2;
  const bool mid = b == 2 * H;
  const double* blk = tri64 + (long long)sys * g.SS + (long long)b * g.LB;
  unsigned char* ob = out + (long long)sys * w.SS + (long long)b * w.LB;
  auto S = [&](int r, int c) -> double {
    const int I = r >> 5;
    const int width = I < g.nfull ? 32 * (I + 1) : nb;
    if (c >= width) {
      const int t = r; r = c; c = t;
    }
    return blk[tri_rowoff(g, r) + c];
  };
  const int te = w.npad * 8;
  for (int t = threadIdx.x; t < w.ks * te; t += blockDim.x) {
    const int k = t / te, e = t % te;
    const int n = e >> 3, kk = e & 7, c = 8 * k + kk;
    const double v = (n < nb && c < nb) ? S(n, c) : 0.0;
    const uint32_t hi = tf32_rna((float)v);
    const uint32_t lo = tf32_rna((float)(v - (double)__uint_as_float(hi)));
    const int o = k * 2 * w.tile + (n >> 3) * 256 + (kk >> 2) * 128 + (n & 7) * 16 + (kk & 3) * 4;
    *reinterpret_cast<uint32_t*>(ob + o) = hi;
    *reinterpret_cast<uint32_t*>(ob + o + w.tile) = lo;
  }
  const int nsets = mid ? 2 : 1, KP = 8 * w.ks;
  float* cp = reinterpret_cast<float*>(ob + w.cpl);
  for (int t = threadIdx.x; t < 2 * nsets * 6 * KP; t += blockDim.x) {
    // set element (node a, DOF e of the node, term q) = K[q][2a + e], 12 floats per node
    const int set = t / (6 * KP), u = t % (6 * KP), q = u % 6, c = u / 6;
    const bool tr = set >= nsets;
    const double* C = blk + g.TB + (long long)(tr ? set - nsets : set) * 6 * nb;
    double v = 0.0;
    if (c < nb) {
      if (!tr) {
        v = C[q * nb + c];
      } else {
        const int a = c >> 1, e = c & 1, dn = (q >> 1) - 1, f = q & 1, n = a + dn;
        v = (n >= 0 && n < NN) ? C[(2 - 2 * dn + e) * nb + 2 * n + f] : 0.0;
      }
    }
    cp[t] = (float)v;
  }
}

// Groups g0 + blockIdx.x / 2 (see PatchGroups): R columns = up to R patches of one type and
// realisation; right-hand sides gathered from system grp_sys[g] - sys0 of r.  Work buffer
// Xg: [group][NL][R][nb] holds w_k after the forward sweeps, then x_k.  Launched as clusters
// of two CTAs (rank 0 the top half, rank 1 the bottom half) of max(32 (2 nfull + (rem > 0)),
// 128) threads; TPF (node, right-hand side) pairs per thread cover the vector phases
// (nb / 2 R <= TPF x threads).
template <typename T, int R, int NBUF, int MINB, int TPF>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(32 * TMAXW, MINB) k_patch_tri(
    const T* __restrict__ r, long long stride, int sys0, int g0, int nelx, int nely, int H,
    int ncx, const int* __restrict__ grp_type, const int* __restrict__ grp_sys,
    const int* __restrict__ grp_first, const int* __restrict__ grp_count,
    const int* __restrict__ perm, const uint8_t* __restrict__ pfree, const T* __restrict__ pack,
    TriGeom geo, T* __restrict__ Xg, int* __restrict__ err) {
  using V2 = typename Pair<T>::type;
  // one stage (NBUF = 1): the block is split into its symmetric inverse (one buffer, refilled
  // as soon as the product that reads it is done) and its coupling (two buffers, filled a
  // step ahead), so that neither copy waits at the top of a step; bars[0] the inverse,
  // bars[1], bars[2] the couplings.  Two stages: a ring of whole blocks.
  constexpr bool SPLIT = NBUF == 1;
  __shared__ __align__(8) uint64_t bars[NBUF + 2];
  __shared__ int s_abort;
  __shared__ int s_ox[16], s_oy[16];          // lower-left node of each patch's box
  __shared__ int s_rowoff[160];               // offset of every factor row in a block
  extern __shared__ __align__(16) unsigned char smraw[];

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int nb = geo.nb, NV = geo.NV, nfull = geo.nfull, rem = geo.rem, NN = nb >> 1;
  const int nrw = 2 * nfull;                  // row warps (16 rows each); warp nrw is the edge warp
  const int NTH = blockDim.x;
  const int N = 2 * H + 1, NL = N, Lc = H;    // lines of the box; chain length; middle line Lc
  const int grp = g0 + (blockIdx.x >> 1);
  const int type = grp_type[grp], first = grp_first[grp], cnt = grp_count[grp];
  const T* rs = r + (long long)(grp_sys[grp] - sys0) * stride;
  const uint8_t* fr = pfree + (long long)type * N * nb;
  const T* src = pack + (long long)type * geo.SS;
  T* X = Xg + (long long)grp * NL * R * nb;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  T* ring = reinterpret_cast<T*>(smraw);                  // [NBUF][LBM], or [TB] when split
  T* cbuf = ring + geo.TB;                                // split: [2][12 nb] couplings
  T* vt = ring + (SPLIT ? (long long)geo.TB + 24LL * nb : (long long)NBUF * geo.LBM);   // [R][NV] input t
  T* vy = vt + NV * R;                                    // [R][NV] its result S^-1 t
  T* vw = vy + NV * R;                                    // [R][NV] x of the current line
  T* vp = vw + NV * R;                                    // [R][NV] w of the previous line
  T* vu = vp + NV * R;                                    // [R][NV] this CTA's middle contribution
  T* vq = vu + NV * R;                                    // [R][NV] partial sums of the product

  if (tid < 16) {
    int ox = 0, oy = 0;
    if (tid < cnt) {
      const int ia = perm[first + tid];
      ox = (ia % (ncx + 1) - 1) * H;
      oy = (ia / (ncx + 1) - 1) * H;
    }
    s_ox[tid] = ox;
    s_oy[tid] = oy;
  }
  for (int q = tid; q < nb; q += NTH) s_rowoff[q] = tri_rowoff(geo, q);
  if (tid == 0) {
    s_abort = 0;
    for (int b = 0; b < NBUF + 2; ++b) mbar_init(&bars[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // zero the vectors (rows nb..NV-1 stay zero for the whole solve)
  for (int q = tid; q < 6 * NV * R; q += NTH) vt[q] = T(0);
  __syncthreads();

  // ---- block stream: s = 0 .. 2 Lc; s < Lc forward chain line s, s = Lc the middle line,
  //      s > Lc backward chain line 2 Lc - s.  Chain line j is patch line j (rank 0) or
  //      NL - 1 - j (rank 1).
  const int nseq = 2 * Lc + 1;
  auto line_of = [&](int j) { return rank ? NL - 1 - j : j; };
  auto block_off = [&](int s) -> long long {
    if (s == Lc) return (long long)(NL - 1) * geo.LB;
    const int j = s < Lc ? s : 2 * Lc - s;
    return (long long)(rank * Lc + j) * geo.LB;
  };
  auto block_bytes = [&](int s) -> uint32_t {
    return (uint32_t)((long long)(s == Lc ? geo.LBM : geo.LB) * sizeof(T));
  };
  int issued = 0;   // copies issued (thread 0's count; split: inverses)
  int cissued = 0;  // split: couplings issued
  auto issue_S = [&](int s) {   // split: the symmetric inverse of step s's block
    const uint32_t bytes = (uint32_t)((long long)geo.TB * sizeof(T));
    mbar_expect_tx(&bars[0], bytes);
    bulk_g2s(ring, src + block_off(s), bytes, &bars[0]);
    ++issued;
  };
  auto issue_C = [&](int s) {   // split: the coupling(s) of step s's block
    const uint32_t bytes = (uint32_t)((s == Lc ? 12LL : 6LL) * nb * sizeof(T));
    mbar_expect_tx(&bars[1 + (s & 1)], bytes);
    bulk_g2s(cbuf + (long long)(s & 1) * 12 * nb, src + block_off(s) + geo.TB, bytes, &bars[1 + (s & 1)]);
    ++cissued;
  };
  if (tid == 0) {
    if constexpr (SPLIT) {
      issue_S(0);
      issue_C(0);
      if (nseq > 1) issue_C(1);
    } else {
      for (; issued < NBUF && issued < nseq; ++issued) {
        mbar_expect_tx(&bars[issued], block_bytes(issued));
        bulk_g2s(ring + (long long)issued * geo.LBM, src + block_off(issued), block_bytes(issued),
                 &bars[issued]);
      }
    }
  }
  uint32_t phase = 0u;   // bit b: parity of the next wait on stage b

  // vector phases: (node a, right-hand side jj) pairs q = tid + s NTH, s < TPF
  int qa[TPF], qj[TPF];
  bool qv[TPF];
#pragma unroll
  for (int s = 0; s < TPF; ++s) {
    const int q = tid + s * NTH;
    qv[s] = q < NN * R;
    qa[s] = q % NN;
    qj[s] = q / NN;
  }
  V2 pf[TPF];   // the next line's input pairs
  auto gather = [&](int l, V2 (&dst)[TPF]) {   // b_l: r at the patch's DOFs of line l
#pragma unroll
    for (int s = 0; s < TPF; ++s) {
      V2 v;
      v.x = T(0);
      v.y = T(0);
      const int a = qa[s], jj = qj[s];
      if (qv[s] && jj < cnt) {
        const int x = s_ox[jj] + a, y = s_oy[jj] + l;
        if (x >= 0 && x <= nelx && y >= 0 && y <= nely) {
          const V2 g = *reinterpret_cast<const V2*>(rs + 2 * ((long long)y * (nelx + 1) + x));
          const uint8_t* f = fr + (long long)l * nb + 2 * a;
          if (f[0]) v.x = g.x;
          if (f[1]) v.y = g.y;
        }
      }
      dst[s] = v;
    }
  };
  auto load_w = [&](int l, V2 (&dst)[TPF]) {   // w of patch line l from the work buffer
#pragma unroll
    for (int s = 0; s < TPF; ++s)
      if (qv[s]) dst[s] = *reinterpret_cast<const V2*>(X + ((long long)l * R + qj[s]) * nb + 2 * qa[s]);
  };
  auto store_line = [&](int l, const T* v) {   // v ([R][NV]) to the work buffer slot of line l
#pragma unroll
    for (int s = 0; s < TPF; ++s)
      if (qv[s])
        *reinterpret_cast<V2*>(X + ((long long)l * R + qj[s]) * nb + 2 * qa[s]) =
            *reinterpret_cast<const V2*>(v + qj[s] * NV + 2 * qa[s]);
  };
  // out = base + sign C w: rows of this line, C = [6][nb] coupling, w = the neighbour line
  // (base: the prefetched input b, or zero)
  auto couple = [&](const T* C, const T* w, T sign, bool with_base, T* out) {
#pragma unroll
    for (int s = 0; s < TPF; ++s) {
      if (!qv[s]) continue;
      const int a = qa[s], jj = qj[s];
      V2 t;
      t.x = with_base ? pf[s].x : T(0);
      t.y = with_base ? pf[s].y : T(0);
      const T* wj = w + jj * NV;
#pragma unroll
      for (int dn = -1; dn <= 1; ++dn) {
        // node n = a + dn: its columns 2n, 2n + 1 are entries q0, q0 + 1 of rows 2a, 2a + 1
        const int n = a + dn;
        if (n < 0 || n >= NN) continue;
        const int q0 = 2 + 2 * dn;
        const V2 wv = *reinterpret_cast<const V2*>(wj + 2 * n);
        const V2 c0 = *reinterpret_cast<const V2*>(C + q0 * nb + 2 * a);
        const V2 c1 = *reinterpret_cast<const V2*>(C + (q0 + 1) * nb + 2 * a);
        const T w0 = sign * wv.x, w1 = sign * wv.y;
        t.x = fma(c0.x, w0, t.x);
        t.y = fma(c0.y, w0, t.y);
        t.x = fma(c1.x, w1, t.x);
        t.y = fma(c1.y, w1, t.y);
      }
      *reinterpret_cast<V2*>(out + jj * NV + 2 * a) = t;
    }
  };
  // out = C^T x: column c = 2a + e of the neighbour line gathers the rows of nodes a-1..a+1
  auto couple_t = [&](const T* C, const T* x, T* out) {
#pragma unroll
    for (int s = 0; s < TPF; ++s) {
      if (!qv[s]) continue;
      const int a = qa[s], jj = qj[s];
      const T* xj = x + jj * NV;
      T t0 = T(0), t1 = T(0);
#pragma unroll
      for (int dn = -1; dn <= 1; ++dn) {
        const int n = a + dn;
        if (n < 0 || n >= NN) continue;
        const int q0 = 2 - 2 * dn;               // column 2a is entry q0 of rows 2n, 2n + 1
        const V2 xv = *reinterpret_cast<const V2*>(xj + 2 * n);
        const V2 cA = *reinterpret_cast<const V2*>(C + q0 * nb + 2 * n);
        const V2 cB = *reinterpret_cast<const V2*>(C + (q0 + 1) * nb + 2 * n);
        t0 = fma(cA.x, xv.x, t0);
        t0 = fma(cA.y, xv.y, t0);
        t1 = fma(cB.x, xv.x, t1);
        t1 = fma(cB.y, xv.y, t1);
      }
      V2 t;
      t.x = t0;
      t.y = t1;
      *reinterpret_cast<V2*>(out + jj * NV + 2 * a) = t;
    }
  };

  // vy = S^-1 vt.  Warps 2I and 2I + 1 share the 32 rows of row block I: lane i + 16 h takes
  // rows 32 I + i and 32 I + i + 16 and half h of every reduction (each vector load feeds both
  // rows); the block's nfull chunks are split between the two warps (the first half of the
  // list (I, 0), .., (I, I), (I + 1, I), .., (nfull - 1, I) to warp 2I, the rest and the
  // partial block's rows to warp 2I + 1), which add their sums through vq behind a barrier of
  // the pair.
  auto product = [&](const T* L) {
    if (warp < nrw) {
      const int I = warp >> 1, side = warp & 1, i = lane & 15, h = lane >> 4;
      const int r0 = 32 * I + i;                 // rows r0 and r0 + 16 (columns i, i + 16 of chunks (J', I))
      const int half = (nfull + 1) >> 1;
      V2 acc0[R], acc1[R];                       // (even, odd) columns of every right-hand side
#pragma unroll
      for (int j = 0; j < R; ++j) {
        acc0[j].x = T(0); acc0[j].y = T(0);
        acc1[j].x = T(0); acc1[j].y = T(0);
      }
      const int k1 = side ? nfull : half;
      for (int k = side ? half : 0; k < k1; ++k) {
        if (k <= I) {
          // chunk (I, k) along rows r0, r0 + 16: columns 32 k + 16 h .. + 15, by pairs
          const T* L0 = L + s_rowoff[r0] + 32 * k + 16 * h;
          const T* L1 = L + s_rowoff[r0 + 16] + 32 * k + 16 * h;
          const T* tv = vt + 32 * k + 16 * h;
#pragma unroll
          for (int c = 0; c < 16; c += 4) {
            const V2 a01 = *reinterpret_cast<const V2*>(L0 + c);
            const V2 a23 = *reinterpret_cast<const V2*>(L0 + c + 2);
            const V2 b01 = *reinterpret_cast<const V2*>(L1 + c);
            const V2 b23 = *reinterpret_cast<const V2*>(L1 + c + 2);
#pragma unroll
            for (int j = 0; j < R; ++j) {
              V2 v01, v23;
              ld_quad<T, V2>(tv + j * NV + c, v01, v23);
              acc0[j] = fma_pair(a01, v01, acc0[j]);
              acc1[j] = fma_pair(b01, v01, acc1[j]);
              acc0[j] = fma_pair(a23, v23, acc0[j]);
              acc1[j] = fma_pair(b23, v23, acc1[j]);
            }
          }
        } else {
          // chunk (k, I) down columns i and i + 16: half h takes the rows 32 k + {0..7, 16..23}
          // + 8 h (8 rows apart, the two halves read disjoint banks), by pairs of rows
          const int S2 = 32 * (k + 1) + 2;                      // row stride of block k
          const T* La = L + s_rowoff[32 * k + 8 * h] + 32 * I + i;
          const T* ta = vt + 32 * k + 8 * h;
#pragma unroll
          for (int g4 = 0; g4 < 4; ++g4) {
            const int dr = (g4 & 1) * 4 + (g4 >> 1) * 16;       // 0, 4, 16, 20
            V2 a01, a23, b01, b23;
            a01.x = La[dr * S2];            a01.y = La[(dr + 1) * S2];
            a23.x = La[(dr + 2) * S2];      a23.y = La[(dr + 3) * S2];
            b01.x = La[dr * S2 + 16];       b01.y = La[(dr + 1) * S2 + 16];
            b23.x = La[(dr + 2) * S2 + 16]; b23.y = La[(dr + 3) * S2 + 16];
#pragma unroll
            for (int j = 0; j < R; ++j) {
              V2 v01, v23;
              ld_quad<T, V2>(ta + j * NV + dr, v01, v23);
              acc0[j] = fma_pair(a01, v01, acc0[j]);
              acc1[j] = fma_pair(b01, v01, acc1[j]);
              acc0[j] = fma_pair(a23, v23, acc0[j]);
              acc1[j] = fma_pair(b23, v23, acc1[j]);
            }
          }
        }
      }
      if (side) {
        // the partial block's rows (complete rows stored): columns r0, r0 + 16 of each
        for (int e = h; e < rem; e += 2) {
          const int rw = 32 * nfull + e;
          const T a0 = L[s_rowoff[rw] + r0], a1 = L[s_rowoff[rw] + r0 + 16];
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const T v = vt[j * NV + rw];
            acc0[j].x = fma(a0, v, acc0[j].x);
            acc1[j].x = fma(a1, v, acc1[j].x);
          }
        }
      }
      T s0[R], s1[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        s0[j] = acc0[j].x + acc0[j].y;
        s1[j] = acc1[j].x + acc1[j].y;
        s0[j] += __shfl_xor_sync(0xffffffffu, s0[j], 16);
        s1[j] += __shfl_xor_sync(0xffffffffu, s1[j], 16);
      }
      if (side && h == 0) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          vq[j * NV + r0] = s0[j];
          vq[j * NV + r0 + 16] = s1[j];
        }
      }
      pair_barrier(I);   // warp 2I + 1's sums are in vq
      if (!side && h == 0) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          vy[j * NV + r0] = s0[j] + vq[j * NV + r0];
          vy[j * NV + r0 + 16] = s1[j] + vq[j * NV + r0 + 16];
        }
      }
    } else if (warp == nrw && rem > 0) {
      // complete rows of the partial block: lanes over column pairs
      for (int e0 = 0; e0 < rem; e0 += 2) {
        const int r0 = 32 * nfull + e0, r1 = r0 + 1 < nb ? r0 + 1 : r0;
        const T* L0 = L + s_rowoff[r0];
        const T* L1 = L + s_rowoff[r1];
        V2 a0[R], a1[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
          a0[j].x = T(0); a0[j].y = T(0);
          a1[j].x = T(0); a1[j].y = T(0);
        }
        for (int c = 2 * lane; c < NV; c += 64) {
          const V2 l0 = *reinterpret_cast<const V2*>(L0 + c);
          const V2 l1 = *reinterpret_cast<const V2*>(L1 + c);
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const V2 v = *reinterpret_cast<const V2*>(vt + j * NV + c);
            a0[j] = fma_pair(l0, v, a0[j]);
            a1[j] = fma_pair(l1, v, a1[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
          T s0 = a0[j].x + a0[j].y, s1 = a1[j].x + a1[j].y;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
          }
          if (lane == 0) {
            vy[j * NV + r0] = s0;
            if (r1 != r0) vy[j * NV + r1] = s1;
          }
        }
      }
    }
  };

  V2 wk[TPF];                    // backward: w of the current line (registers)
  gather(line_of(0), pf);
  bool abort = false, met = false;
  // thread 0 waits for the block of step s before a barrier that precedes its first use
  auto wait_stage = [&](int s) {
    const int b = s % NBUF;
    if (tid == 0 && !s_abort && !mbar_wait(&bars[b], (phase >> b) & 1u)) {
      s_abort = 1;
      atomicExch(err, (int)MSTOPO_TIMEOUT);
    }
    phase ^= 1u << b;
  };
  auto wait_bar = [&](int b, uint32_t parity) {   // split: thread 0, before a barrier
    if (tid == 0 && !s_abort && !mbar_wait(&bars[b], parity)) {
      s_abort = 1;
      atomicExch(err, (int)MSTOPO_TIMEOUT);
    }
  };
  auto wait_S = [&](int s) { wait_bar(0, (uint32_t)(s & 1)); };
  auto wait_C = [&](int s) { wait_bar(1 + (s & 1), (uint32_t)((s >> 1) & 1)); };
  // split: the next step's inverse, once every read of this one is behind a barrier
  auto refill_S = [&](int s) {
    if constexpr (SPLIT)
      if (tid == 0 && s + 1 < nseq && !s_abort) issue_S(s + 1);
  };
  if constexpr (!SPLIT) wait_stage(0);
  __syncthreads();
  for (int s = 0; s < nseq; ++s) {
    if constexpr (SPLIT) {
      // the coupling (issued a step ahead) and, for a backward line (product first), the inverse
      wait_C(s);
      if (s > Lc) wait_S(s);
      __syncthreads();
    }
    if (s_abort) { abort = true; break; }
    const T* L = ring + (long long)(s % NBUF) * geo.LBM;
    const T* Cs = SPLIT ? cbuf + (long long)(s & 1) * 12 * nb : L + geo.TB;   // coupling(s) of the block
    if (s < Lc) {
      // forward chain line j: t = b - C_j w_{j-1}, w_j = S_j^-1 t
      const int j = s, l = line_of(j);
      if (j > 0) {
        couple(Cs, vp, T(-1), true, vt);
      } else {
#pragma unroll
        for (int q = 0; q < TPF; ++q)
          if (qv[q]) *reinterpret_cast<V2*>(vt + qj[q] * NV + 2 * qa[q]) = pf[q];
      }
      gather(j + 1 < Lc ? line_of(j + 1) : Lc, pf);   // next line's input (the middle line last)
      if constexpr (SPLIT) wait_S(s);
      __syncthreads();
      product(L);
      if (NBUF > 1 && s + 1 < nseq) wait_stage(s + 1);
      __syncthreads();
      refill_S(s);
      // w_j (in vy) to the work buffer for the backward sweep (the last one stays in shared
      // memory: the first backward line rewrites that slot); it becomes w_{j-1} of the next line
      if (j + 1 < Lc) store_line(l, vy);
      T* tmp = vp; vp = vy; vy = tmp;
    } else if (s == Lc) {
      // middle line: u = C_mid w_{Lc-1} published, then x_m = M^-1 (b_m - u_0 - u_1) in both CTAs
      const T* Cown = Cs + rank * 6 * nb;
      couple(Cown, vp, T(1), false, vu);
      cluster.sync();   // both contributions are in shared memory
      met = true;
      const T* vu0 = rank == 0 ? vu : cluster.map_shared_rank(vu, 0);
      const T* vu1 = rank == 1 ? vu : cluster.map_shared_rank(vu, 1);
#pragma unroll
      for (int q = 0; q < TPF; ++q) {
        if (!qv[q]) continue;
        const int o = qj[q] * NV + 2 * qa[q];
        const V2 u0 = *reinterpret_cast<const V2*>(vu0 + o);
        const V2 u1 = *reinterpret_cast<const V2*>(vu1 + o);
        V2 t;
        t.x = (pf[q].x - u0.x) - u1.x;
        t.y = (pf[q].y - u0.y) - u1.y;
        *reinterpret_cast<V2*>(vt + o) = t;
        wk[q] = *reinterpret_cast<const V2*>(vp + o);   // w_{Lc-1} for the first backward line
      }
      if constexpr (SPLIT) wait_S(s);
      __syncthreads();
      product(L);
      __syncthreads();
      refill_S(s);
      if (rank == 0) store_line(Lc, vy);
      couple_t(Cown, vy, vt);   // t of chain line Lc - 1
      if (NBUF > 1 && s + 1 < nseq) wait_stage(s + 1);
      __syncthreads();
    } else {
      // backward chain line j: x_j = w_j - S_j^-1 t_j, then t_{j-1} = C_j^T x_j
      const int j = 2 * Lc - s, l = line_of(j);
      product(L);
      __syncthreads();
      refill_S(s);
#pragma unroll
      for (int q = 0; q < TPF; ++q) {
        if (!qv[q]) continue;
        const int o = qj[q] * NV + 2 * qa[q];
        const V2 y = *reinterpret_cast<const V2*>(vy + o);
        V2 x;
        x.x = wk[q].x - y.x;
        x.y = wk[q].y - y.y;
        *reinterpret_cast<V2*>(vw + o) = x;
        *reinterpret_cast<V2*>(X + ((long long)l * R + qj[q]) * nb + 2 * qa[q]) = x;
      }
      if (j > 0) load_w(line_of(j - 1), wk);
      __syncthreads();
      if (j > 0) couple_t(Cs, vw, vt);
      if (NBUF > 1 && s + 1 < nseq) wait_stage(s + 1);
      __syncthreads();
    }
    if constexpr (SPLIT) {
      // every read of this step's coupling buffer is behind a barrier: the coupling two steps on
      if (tid == 0 && s + 2 < nseq && !s_abort) issue_C(s + 2);
    } else {
      // every read of stage s % NBUF is behind a barrier: refill it with block s + NBUF
      if (tid == 0 && issued < nseq && !s_abort) {
        const int st = issued % NBUF;
        mbar_expect_tx(&bars[st], block_bytes(issued));
        bulk_g2s(ring + (long long)st * geo.LBM, src + block_off(issued), block_bytes(issued),
                 &bars[st]);
        ++issued;
      }
    }
  }
  if (!met) cluster.sync();   // the partner meets this CTA at the middle line in any case
  if (SPLIT && abort && tid == 0) {
    // every copy issued lands before the CTA exits (waits on completed phases return at once)
    if (issued > 0 && !tri_wait(&bars[0], (uint32_t)((issued - 1) & 1))) atomicExch(err, (int)MSTOPO_TIMEOUT);
    for (int c = cissued - 1; c >= 0 && c >= cissued - 2; --c)
      if (!tri_wait(&bars[1 + (c & 1)], (uint32_t)((c >> 1) & 1))) atomicExch(err, (int)MSTOPO_TIMEOUT);
  }
  if (!SPLIT && abort && tid == 0) {
    // every copy issued and not yet waited for lands before the CTA exits
    for (int m2 = 0; m2 < NBUF; ++m2) {
      const int last = issued - 1 - m2;    // copy `last` went to stage last % NBUF
      if (last < 0) break;
      const int st = last % NBUF;
      const uint32_t par = (uint32_t)((last / NBUF) & 1);
      if (!tri_wait(&bars[st], par)) atomicExch(err, (int)MSTOPO_TIMEOUT);
    }
  }
  cluster.sync();   // the partner has read this CTA's contribution
}

// ------------------------------------------------------------------------------ host side
// Stages of the block ring and CTAs per SM of a launch: FP32 at four columns streams one stage
// and runs three CTAs per SM (about 66 KB of shared memory and 72 registers each: the 318 CTAs
// of the 1024x512 workload in one wave, each CTA's copy wait covered by the other two); more
// columns stream two stages at one CTA per SM; FP64 one stage at one CTA per SM.
template <typename T, int R> struct TriCfg {
  static constexpr int NBUF = (sizeof(T) == 4 && R > 4) ? 2 : 1;
  static constexpr int MINB = (sizeof(T) == 4 && R <= 4) ? 3 : 1;
};

static int tri_threads(int nb) {
  const int t = 32 * (2 * (nb / 32) + (nb % 32 ? 1 : 0));
  return t < TMINTH ? TMINTH : t;
}

static size_t patch_tri_smem(int nb, int R, int nbuf, size_t elem) {
  const TriGeom g = tri_geometry(nb, 3);
  // one stage: the inverse part [TB] and two coupling buffers [2][12 nb]
  const size_t blocks = nbuf == 1 ? (size_t)g.TB + 24 * (size_t)nb : (size_t)nbuf * g.LBM;
  return (blocks + 6 * (size_t)g.NV * R) * elem;
}

long long patch_tri_system_elems(int nb, int NL) { return tri_geometry(nb, NL).SS; }

int patch_tri_ctas_per_sm(int nb, int R) {
  // 228 KB of shared memory per SM, 1 KB reserved per CTA, the static arrays below 2 KB;
  // registers allow the launch bound's CTAs per SM
  const int nbuf = R <= 4 ? TriCfg<float, 4>::NBUF : TriCfg<float, 8>::NBUF;
  const int minb = R <= 4 ? TriCfg<float, 4>::MINB : TriCfg<float, 8>::MINB;
  const size_t per = patch_tri_smem(nb, R, nbuf, 4) + 3 * 1024;
  return std::max(1, std::min(minb, (int)((228 * 1024) / per)));
}

// the kernel's thread layout covers this line size: at most 9 warps, rows addressed through
// a 160-entry table, every vector phase within 4 pairs per thread (16 patches per CTA)
bool patch_tri_assignment_ok(int nb) {
  const int nt = tri_threads(nb);
  return nb >= 2 && nb % 2 == 0 && nb <= 160 && nt <= 32 * TMAXW && (nb / 2) * 16 <= 4 * nt;
}

cudaError_t patch_tri_pack(const double* Lt, const double* Bt, const double* Lr, const double* Br,
                           const double* Lm, int nsys, int nb, int NL, int NLr, double* out64,
                           float* out32, cudaStream_t s) {
  const TriGeom g = tri_geometry(nb, NL);
  note_launch(), k_patch_tri_pack<<<dim3(nsys, NL), 256, 0, s>>>(Lt, Bt, Lr, Br, Lm, NL, NLr, g,
                                                                 out64, out32);
  return cudaGetLastError();
}

TwGeom patch_twtc_geometry(int nb, int NL) {
  TwGeom w{};
  w.nb = nb;
  w.npad = (nb + 15) / 16 * 16;
  w.ks = (nb + 7) / 8;
  w.tile = w.npad * 32;
  w.cpl = w.ks * 2 * w.tile;
  w.cset = 6 * 8 * w.ks * 4;
  w.LB = (long long)w.cpl + 2LL * w.cset;
  w.LBM = (long long)w.cpl + 4LL * w.cset;
  w.SS = (long long)(NL - 1) * w.LB + w.LBM;
  return w;
}

cudaError_t patch_twtc_pack(const double* tri64, int nsys, int nb, int NL, unsigned char* out,
                            cudaStream_t s) {
  const TriGeom g = tri_geometry(nb, NL);
  const TwGeom w = patch_twtc_geometry(nb, NL);
  note_launch(), k_patch_twtc_pack<<<dim3(nsys, NL), 256, 0, s>>>(tri64, g, w, NL, out);
  return cudaGetLastError();
}

template <typename T, int R, int TPF>
static cudaError_t launch_tri_kt(mstopo_handle* h, const PatchGroups& G, const T* r, int sys0,
                                 int nsys, const T* pack, T* Xg) {
  constexpr int NBUF = TriCfg<T, R>::NBUF, MINB = TriCfg<T, R>::MINB;
  Precond& pc = h->pc;
  const TriGeom geo = tri_geometry(pc.nbP, pc.NP);
  const size_t sm = patch_tri_smem(pc.nbP, R, NBUF, sizeof(T));
  {
    cudaError_t e = smem_limit_max<k_patch_tri<T, R, NBUF, MINB, TPF>>();
    if (e != cudaSuccess) return e;
  }
  if (sm > 225 * 1024 || !patch_tri_assignment_ok(pc.nbP) || pc.NP % 2 == 0)
    return cudaErrorInvalidConfiguration;
  const int g0 = G.h_begin[sys0], ng = G.h_begin[sys0 + nsys] - g0;
  if (ng <= 0) return cudaSuccess;
  note_launch(), k_patch_tri<T, R, NBUF, MINB, TPF><<<2 * ng, tri_threads(pc.nbP), sm, h->s>>>(
      r, h->n_dof, sys0, g0, h->nelx, h->nely, pc.H, pc.ncx, G.d_type, G.d_sys, G.d_first,
      G.d_count, G.d_perm, pc.d_pfree, pack, geo, Xg, h->d_flag + 1);
  return cudaGetLastError();
}

// the fewest (node, right-hand side) pairs per thread that cover the vector phases
template <typename T, int R>
static cudaError_t launch_tri_k(mstopo_handle* h, const PatchGroups& G, const T* r, int sys0,
                                int nsys, const T* pack, T* Xg) {
  const int pairs = (h->pc.nbP / 2) * R, nt = tri_threads(h->pc.nbP);
  if (pairs <= nt) return launch_tri_kt<T, R, 1>(h, G, r, sys0, nsys, pack, Xg);
  if (pairs <= 2 * nt) return launch_tri_kt<T, R, 2>(h, G, r, sys0, nsys, pack, Xg);
  return launch_tri_kt<T, R, 4>(h, G, r, sys0, nsys, pack, Xg);
}

cudaError_t patch_tri_solve_f32(mstopo_handle* h, const PatchGroups& G, const float* r, int sys0,
                                int nsys, float* Xg) {
  const float* pack = h->pc.d_tri32;
  switch (patch_tri_cols(G.P)) {
    case 4: return launch_tri_k<float, 4>(h, G, r, sys0, nsys, pack, Xg);
    case 8: return launch_tri_k<float, 8>(h, G, r, sys0, nsys, pack, Xg);
    default: return launch_tri_k<float, 16>(h, G, r, sys0, nsys, pack, Xg);
  }
}

cudaError_t patch_tri_solve_f64(mstopo_handle* h, const PatchGroups& G, const double* r, int sys0,
                                int nsys, double* Xg) {
  const double* pack = h->pc.d_tri64;
  switch (patch_tri_cols(G.P)) {
    case 4: return launch_tri_k<double, 4>(h, G, r, sys0, nsys, pack, Xg);
    default: return cudaErrorInvalidConfiguration;   // FP64 groups hold at most 4 patches
  }
}
