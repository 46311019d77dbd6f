// Tensor-core FP32 patch solves of the additive two-level preconditioner (Sec. 2.4.2: the exact
// local solves z_i = K_i^-1 R_i r on every agglomerate patch), on the two-sided block
// elimination of csrc/patch_tri.cu with the patches as the MMA's M dimension.
//
// A patch matrix is block tridiagonal over the NL = 2H + 1 node rows ("lines") of its box.  All
// patches of one type and realisation share its factors, so the line step of the elimination
// is, for up to 128 such patches at once, one product of the right-hand sides T (patches x
// DOFs) with the line's symmetric inverse: Y = T S^-1 (S^-1 symmetric).  On tcgen05 that is
// M = 128 patches (TMEM lanes), N = the line's nb DOFs padded to a multiple of 16, K = nb in
// steps of 8; FP32 accuracy from TF32 splits of both operands, T = Th + Tl and S^-1 = Sh + Sl,
// as three MMAs per K-step (Th Sh + Th Sl + Tl Sh) into one FP32 accumulator.  The sparse
// couplings between lines (six neighbour DOFs per row) stay on the CUDA cores: the epilogue
// thread of patch m reads row m of the accumulator (its whole line) and forms the next line's
// right-hand side with no data from other threads:
//   forward  (chain line j < H)  w_j = S_j^-1 t_j,   t_{j+1} = b_{j+1} - C_{j+1} w_j
//   middle   (both chains met)   t_m = b_m - C_0 w^0_{H-1} - C_1 w^1_{H-1},  x_m = M^-1 t_m
//   backward (j = H-1 .. 0)      x_j = w_j - S_j^-1 t_j,  t_{j-1} = C_j^T x_j
// with C the stored coupling of a block and C^T its transpose, both as six-term stencils.
// CTA rank 0 of a cluster of two runs the top chain, rank 1 the bottom chain (the top chain
// of the line-reversed matrix); they exchange their middle-line contributions C_r w^r through
// global memory behind one cluster barrier and both form x_m with the same operations.
//
// Roles (320 threads): warps 0-7 epilogue (warps w and w + 4 read TMEM lane quarter w: patch
// m = 32 w + lane, the first and the second half of the line's K-steps), warp 8 streams the
// packed blocks in units of up to four K-steps and the couplings (cp.async.bulk into rings,
// mbarrier transaction counts, L2 prefetch two blocks ahead), warp 9 issues the MMAs (one
// lane): one readiness wait, one stage wait and one commit per unit.  Two accumulators in
// TMEM alternate by line, so the epilogue of line s (reading accumulator s mod 2, writing the
// next A unit by unit) overlaps the MMAs of line s + 1, which start on each unit of A as soon
// as it is written.  Every accumulator column sums every K-step, so a line's epilogue starts
// only after all of its MMAs: a line step is one MMA chain plus the epilogue's lead-in to its
// first unit.
// Every mbarrier wait is bounded; on a timeout the CTA records MSTOPO_TIMEOUT, the roles stop,
// the copies and MMAs in flight are drained, every thread still arrives at the cluster barrier
// once, and TMEM is released before the CTA exits.
#include <algorithm>
#include <type_traits>

#include "blocktri.cuh"
#include "internal.cuh"
#include "tcgen05.cuh"

namespace {

constexpr int TW_EPI = 256;                  // epilogue threads (8 warps, two per TMEM lane quarter)
constexpr int TW_THREADS = TW_EPI + 64;      // + producer warp + MMA warp
constexpr int TW_PROD = TW_EPI / 32, TW_MMA = TW_PROD + 1;   // their warp indices
constexpr int TW_ATILE = TW_M * 32;          // bytes of one K-step of A (128 rows x 8 TF32)
constexpr int TW_D1 = 256;                   // TMEM column of the second accumulator
constexpr int TW_TMEM_COLS = 512;
constexpr int TW_MAX_NST = 16;               // stages of the block ring
constexpr int TW_SMEM = 227 * 1024 - 1024;   // dynamic shared memory budget of one CTA

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait;" ::: "memory"); }
// the epilogue threads (named barrier 1) OR a flag over them
__device__ __forceinline__ bool epi_any(bool flag) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 256, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)flag)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

}  // namespace

// Groups g0 + blockIdx.x / 2 of G (up to TW_M patches of one type and realisation each), NB
// DOFs per line.  X: [group][NL][NB / 2 nodes][TW_M][2] holds w_j after the forward chain, x_j
// at the end; U: [group][2][NB / 2][TW_M][2] the middle-line contributions of both ranks
// (consecutive patches adjacent: the epilogue's stores and loads coalesce).
template <int NB>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TW_THREADS, 1) k_patch_twtc(
    const float* __restrict__ r, long long stride, int sys0, int g0, int nelx, int nely, int H,
    int ncx, const int* __restrict__ grp_type, const int* __restrict__ grp_sys,
    const int* __restrict__ grp_first, const int* __restrict__ grp_count,
    const int* __restrict__ perm, const uint8_t* __restrict__ pfree,
    const unsigned char* __restrict__ pack, TwGeom w, int nst, float* __restrict__ Xg,
    float* __restrict__ U, int* __restrict__ err) {
  constexpr int KS = (NB + 7) / 8;           // K-steps (chunks of 8 DOFs = 4 nodes)
  constexpr int NN = NB / 2;                 // nodes of a line
  constexpr int KP = 8 * KS;                 // padded DOFs of a line
  constexpr int CS = (KS + 1) / 2;           // chunks of the first half
  // units of up to four chunks (K-steps) within each half: one bulk copy, one readiness
  // barrier and one commit each
  constexpr int G0 = (CS + 3) / 4, NG = G0 + (KS - CS + 3) / 4;
  auto glo = [](int g) { return g < G0 ? 4 * g : CS + 4 * (g - G0); };
  auto ghi = [](int g) { return g < G0 ? (4 * g + 4 < CS ? 4 * g + 4 : CS) : (CS + 4 * (g - G0) + 4 < KS ? CS + 4 * (g - G0) + 4 : KS); };
  auto gof = [](int c) { return c < CS ? c / 4 : G0 + (c - CS) / 4; };
  __shared__ __align__(8) uint64_t full[TW_MAX_NST], empty[TW_MAX_NST], dfull[2], dempty[2],
      cfull[2], cempty[2], aready[NG], fin;
  __shared__ volatile int s_abort;
  __shared__ uint32_t s_tmem;
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* Ahi = smraw;                                  // [KS][TW_ATILE]
  unsigned char* Alo = smraw + KS * TW_ATILE;                  // [KS][TW_ATILE]
  float* cs = reinterpret_cast<float*>(smraw + 2 * KS * TW_ATILE);   // [2][4 KS][2][6] couplings
  unsigned char* ring = smraw + 2 * KS * TW_ATILE + 2 * w.cset;      // [nst][4][hi tile | lo tile]
  const uint32_t kb = 2u * (uint32_t)w.tile;                   // bytes of one K-step of a block
  const uint32_t sb = 4u * kb;                                  // bytes of one ring stage

  const int rank = (int)cluster_rank();
  const int N = 2 * H + 1, NL = N, Lc = H, nseq = 2 * Lc + 1;
  const int grp = g0 + (blockIdx.x >> 1);
  const int type = grp_type[grp], first = grp_first[grp], cnt = grp_count[grp];
  const float* rs = r + (long long)(grp_sys[grp] - sys0) * stride;
  const uint8_t* fr = pfree + (long long)type * N * NB;
  const unsigned char* src = pack + (long long)type * w.SS;
  float2* X = reinterpret_cast<float2*>(Xg) + (long long)grp * NL * NN * TW_M;
  float2* Ug = reinterpret_cast<float2*>(U) + (long long)grp * 2 * NN * TW_M;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto line_of = [&](int j) { return rank ? NL - 1 - j : j; };
  // bytes: the packed block of step s (s < Lc forward chain line s, s = Lc the middle line,
  // s > Lc backward chain line 2 Lc - s)
  auto block_off = [&](int s) -> long long {
    if (s == Lc) return (long long)(NL - 1) * w.LB;
    const int j = s < Lc ? s : 2 * Lc - s;
    return (long long)(rank * Lc + j) * w.LB;
  };
  // bytes: the coupling of step s (forward the next chain block's C, the last forward step
  // this rank's C_r of the middle block, the middle line its C_r^T, backward the block's C^T;
  // none for the last backward line)
  auto cpl_off = [&](int s) -> long long {
    if (s < Lc - 1) return (long long)(rank * Lc + s + 1) * w.LB + w.cpl;
    if (s <= Lc) return (long long)(NL - 1) * w.LB + w.cpl + (long long)(s == Lc ? 2 + rank : rank) * w.cset;
    return (long long)(rank * Lc + 2 * Lc - s) * w.LB + w.cpl + w.cset;
  };

  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < nst; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&dfull[i], 1);
      mbar_init(&dempty[i], TW_EPI);
      mbar_init(&cfull[i], 1);
      mbar_init(&cempty[i], TW_EPI);
    }
    for (int i = 0; i < NG; ++i) mbar_init(&aready[i], TW_M);   // one half writes a unit
    mbar_init(&fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(TW_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = s_tmem;

  if (warp == TW_PROD) {
    // ------------------------------------------------------------------ producer
    cluster_arrive();   // this thread has no part in the middle-line exchange
    if (lane == 0) {
      int u = 0, nc = 0, st = 0;
      uint32_t eph = 0;   // parity of the next wait on a stage's empty barrier (rounds >= 1)
      bool ok = true;
      // the factor stream comes from DRAM when the packs exceed L2: blocks are prefetched into
      // L2 two steps ahead of their copies into the ring
      auto l2_prefetch = [&](int s2) {
        if (s2 >= nseq) return;
        const unsigned char* b = src + block_off(s2);
        for (int k = 0; k < KS; ++k)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b + (size_t)k * kb), "r"(kb) : "memory");
        if (s2 + 1 < nseq)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src + cpl_off(s2)), "r"((uint32_t)w.cset)
                       : "memory");
      };
      l2_prefetch(0);
      l2_prefetch(1);
      for (int s = 0; s < nseq && ok; ++s) {
        l2_prefetch(s + 2);
        // the coupling of step s, once the epilogue has finished step s - 2 (same buffer)
        if (s + 1 < nseq) {
          if (s >= 2 && !tc_wait(&cempty[s & 1], ((s >> 1) - 1) & 1, &s_abort, err)) break;
          mbar_expect_tx(&cfull[s & 1], (uint32_t)w.cset);
          bulk_g2s(cs + (s & 1) * 6 * KP, src + cpl_off(s), (uint32_t)w.cset, &cfull[s & 1]);
          ++nc;
        }
        const unsigned char* blk = src + block_off(s);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          if (u >= nst && !tc_wait(&empty[st], eph, &s_abort, err)) {
            ok = false;
            break;
          }
          const uint32_t bytes = (uint32_t)(ghi(g) - glo(g)) * kb;
          mbar_expect_tx(&full[st], bytes);
          bulk_g2s(ring + (size_t)st * sb, blk + (size_t)glo(g) * kb, bytes, &full[st]);
          ++u;
          if (++st == nst) {
            st = 0;
            if (u > nst) eph ^= 1u;
          }
        }
      }
      // drain: the last fill of every stage and coupling buffer has landed before the exit
      for (int st = 0; st < nst && st < u; ++st) tc_drain(&full[st], ((u - 1 - st) / nst) & 1, err);
      for (int b = 0; b < 2 && b < nc; ++b) tc_drain(&cfull[(nc - 1 - b) & 1], ((nc - 1 - b) >> 1) & 1, err);
    }
    cluster_wait();
  } else if (warp == TW_MMA) {
    // ------------------------------------------------------------------ MMA issue
    cluster_arrive();
    if (lane == 0) {
      const uint32_t idesc = tc_idesc(TW_M, w.npad);
      const uint64_t dAh = tc_sdesc(smem_u32(Ahi), 128, 256);
      const uint64_t dAl = tc_sdesc(smem_u32(Alo), 128, 256);
      const uint64_t dR = tc_sdesc(smem_u32(ring), 128, 256);
      int st = 0;
      uint32_t fph = 0;   // parity of the next wait on a stage's full barrier
      bool issued = false, ok = true;
      for (int s = 0; s < nseq && ok; ++s) {
        const uint32_t d = tm + (uint32_t)((s & 1) * TW_D1);
        // the epilogue has read this accumulator's previous line (s - 2)
        if (s >= 2 && !tc_wait(&dempty[s & 1], ((s >> 1) - 1) & 1, &s_abort, err)) break;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          if (!tc_wait(&aready[g], s & 1, &s_abort, err) || !tc_wait(&full[st], fph, &s_abort, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t bs = dR + (uint64_t)((st * sb) >> 4);
#pragma unroll
          for (int k = glo(g); k < ghi(g); ++k) {
            const uint64_t ah = dAh + (uint64_t)((k * TW_ATILE) >> 4);
            const uint64_t al = dAl + (uint64_t)((k * TW_ATILE) >> 4);
            const uint64_t bh = bs + (uint64_t)(((k - glo(g)) * kb) >> 4);
            const uint64_t bl = bh + (uint64_t)(w.tile >> 4);
            tc_mma(d, ah, bh, idesc, k > 0 ? 1u : 0u);   // Th Sh
            tc_mma(d, ah, bl, idesc, 1u);                // Th Sl
            tc_mma(d, al, bh, idesc, 1u);                // Tl Sh
          }
          tc_commit(&empty[st]);
          issued = true;
          if (++st == nst) {
            st = 0;
            fph ^= 1u;
          }
        }
        if (!ok) break;
        tc_commit(&dfull[s & 1]);
      }
      if (issued) {   // drain: every MMA this thread issued has completed
        tc_commit(&fin);
        tc_drain(&fin, 0, err);
      }
    }
    cluster_wait();
  } else {
    // ------------------------------------------------------------------ epilogue
    const int q4 = warp & 3;
    const int m = 32 * q4 + lane;                // patch of this thread = TMEM lane
    const bool live = m < cnt;
    int ox, oy;
    {
      // rows beyond the group's patches repeat its last one (finite data, results unused)
      const int ia = perm[first + (live ? m : cnt - 1)];
      ox = (ia % (ncx + 1) - 1) * H;
      oy = (ia / (ncx + 1) - 1) * H;
    }
    const uint32_t tl = tm + ((uint32_t)(32 * q4) << 16);
    const float2 neg1 = f2(-1.f, -1.f);
    // chunk c (K-step c: DOFs 8c .. 8c + 7, nodes 4c .. 4c + 3) of the next line's A as TF32
    // hi and lo parts; release() hands chunks [c0, c1) to the MMA warp after one proxy fence
    auto put_a = [&](int c, const float2 (&t)[4]) {
      uint32_t h[8], l[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        h[2 * i] = tf32_rna(t[i].x);
        h[2 * i + 1] = tf32_rna(t[i].y);
        const float2 lo = __ffma2_rn(neg1, f2(__uint_as_float(h[2 * i]), __uint_as_float(h[2 * i + 1])), t[i]);
        l[2 * i] = tf32_rna(lo.x);
        l[2 * i + 1] = tf32_rna(lo.y);
      }
      const int o = c * TW_ATILE + (m >> 3) * 256 + (m & 7) * 16;
      *reinterpret_cast<uint4*>(Ahi + o) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(Ahi + o + 128) = make_uint4(h[4], h[5], h[6], h[7]);
      *reinterpret_cast<uint4*>(Alo + o) = make_uint4(l[0], l[1], l[2], l[3]);
      *reinterpret_cast<uint4*>(Alo + o + 128) = make_uint4(l[4], l[5], l[6], l[7]);
    };
    auto release = [&](int g) {   // unit g's chunks are written
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&aready[g]);
    };

    // The two halves of the line: chunks [CL, CH), with the node window [A0, A0 + NW) of
    // inputs (one node beyond each end for the stencils).
    auto half_body = [&](auto half_c) {
      constexpr int HALF = decltype(half_c)::value;
      constexpr int CL = HALF ? CS : 0, CH = HALF ? KS : CS;
      constexpr int A0 = 4 * CL - 1, NW = 4 * (CH - CL) + 2;
      float2 nx[NW];   // the next input per window node: b of a line, or w_j
      auto gather = [&](int l) {
        const int y = oy + l;
        const bool yin = y >= 0 && y <= nely;
        const float* row = rs + 2LL * y * (nelx + 1);
        const uint8_t* f = fr + (long long)l * NB;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
          const int a = A0 + i;
          float2 v = f2(0.f, 0.f);
          if (a >= 0 && a < NN) {
            const int x = ox + a;
            if (yin && x >= 0 && x <= nelx) {
              const float2 g = *reinterpret_cast<const float2*>(row + 2 * x);
              const uint16_t fm = *reinterpret_cast<const uint16_t*>(f + 2 * a);   // DOFs 2a, 2a + 1
              v.x = (fm & 0xFFu) ? g.x : 0.f;
              v.y = (fm >> 8) ? g.y : 0.f;
            }
          }
          nx[i] = v;
        }
      };
      auto load_w = [&](int l) {
        const float2* row = X + (long long)l * NN * TW_M + m;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
          const int a = A0 + i;
          nx[i] = (a >= 0 && a < NN) ? row[a * TW_M] : f2(0.f, 0.f);
        }
      };
      // the next step's input (step s + 1 of the sequence)
      auto prefetch = [&](int s1) {
        if (s1 < Lc - 1) gather(line_of(s1 + 1));
        else if (s1 == Lc - 1) gather(Lc);
        else if (s1 > Lc && s1 < nseq) load_w(line_of(2 * Lc - s1));
      };

      // line 0: A = b of the first chain line
      gather(line_of(0));
#pragma unroll
      for (int c = CL; c < CH; ++c) {
        float2 t[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) t[i] = nx[4 * c + i - A0];
        put_a(c, t);
        if (c + 1 == ghi(gof(c))) release(gof(c));
      }
      prefetch(0);

      // one step of the sequence with its mode fixed: 0 forward, 1 last forward line (middle
      // contribution), 2 middle line, 3 backward, 4 the last backward line (no next line)
      auto step = [&](auto mode_c, int s) {
        constexpr int MODE = decltype(mode_c)::value;
        const int j = s <= Lc ? s : 2 * Lc - s;
        const float* K = cs + (s & 1) * 6 * KP;
        const uint32_t dc = tl + (uint32_t)((s & 1) * TW_D1);
        // stored line of this step's result (w_j forward, x_m by rank 0, x_j backward)
        float2* xrow = nullptr;
        if (MODE != 2 || rank == 0) xrow = X + (long long)(MODE == 2 ? Lc : line_of(j)) * NN * TW_M + m;
        // v at node a from accumulator words (d0, d1): the accumulator, or w_j minus it
        auto to_v = [&](int a, uint32_t d0, uint32_t d1) -> float2 {
          const float2 d = f2(__uint_as_float(d0), __uint_as_float(d1));
          if constexpr (MODE >= 3) return __ffma2_rn(neg1, d, nx[a - A0]);
          else return d;
        };
        // chunks c and c + 1 (two = true) or c alone, with one TMEM wait
        auto load_pair = [&](int c, bool two, float2 (&v)[8]) {
          uint32_t u[16];
          if (two) {
            tc_ld<16>(dc + 8 * c, u);
          } else {
            uint32_t u8[8];
            tc_ld<8>(dc + 8 * c, u8);
#pragma unroll
            for (int i = 0; i < 8; ++i) u[i] = u8[i];
          }
          tc_wait_ld();
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (i >= 4 && !two) break;
            const int a = 4 * c + i;
            v[i] = to_v(a, u[2 * i], u[2 * i + 1]);
            if (xrow && a < NN) xrow[a * TW_M] = v[i];
          }
        };
        auto load_node = [&](int a) -> float2 {   // one halo node of the neighbouring half
          uint32_t u[2];
          tc_ld<2>(dc + 2 * a, u);
          tc_wait_ld();
          return to_v(a, u[0], u[1]);
        };
        // output of chunk c from nodes 4c - 1 .. 4c + 4: sum_q K[2a + e][q] v[2a - 2 + q]
        auto emit = [&](int c, float2 vl, const float2 (&vc)[4], float2 vr) {
          float2 t[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int a = 4 * c + i;
            const float4* Kn = reinterpret_cast<const float4*>(K + 12 * a);
            const float4 k0 = Kn[0], k1 = Kn[1], k2 = Kn[2];
            const float2 va = i == 0 ? vl : vc[i - 1], vb = vc[i], vd = i == 3 ? vr : vc[i + 1];
            float2 s0 = __ffma2_rn(f2(k0.x, k0.y), va, f2(0.f, 0.f));
            s0 = __ffma2_rn(f2(k0.z, k0.w), vb, s0);
            s0 = __ffma2_rn(f2(k1.x, k1.y), vd, s0);
            float2 s1 = __ffma2_rn(f2(k1.z, k1.w), va, f2(0.f, 0.f));
            s1 = __ffma2_rn(f2(k2.x, k2.y), vb, s1);
            s1 = __ffma2_rn(f2(k2.z, k2.w), vd, s1);
            const float2 o = f2(s0.x + s0.y, s1.x + s1.y);
            if constexpr (MODE == 0) t[i] = __ffma2_rn(neg1, o, nx[a - A0]);   // b - C w
            else t[i] = o;
          }
          if constexpr (MODE == 1) {
            // this rank's middle-line contribution C_r w_{H-1}
            float2* uo = Ug + (long long)rank * NN * TW_M + m;
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (4 * c + i < NN) uo[(4 * c + i) * TW_M] = t[i];
          } else {
            put_a(c, t);
          }
        };

        float2 vl = f2(0.f, 0.f), vc[4], P[8];
        if (CL > 0) vl = load_node(4 * CL - 1);
        load_pair(CL, CL + 1 < CH, P);
#pragma unroll
        for (int i = 0; i < 4; ++i) vc[i] = P[i];
#pragma unroll
        for (int c = CL; c < CH; ++c) {
          float2 vn[4];
          float2 vr = f2(0.f, 0.f);
          if (c + 1 < CH) {
            if (((c - CL) & 1) == 0) {   // chunk c + 1 came with chunk c
#pragma unroll
              for (int i = 0; i < 4; ++i) vn[i] = P[4 + i];
            } else {                     // chunks c + 1, c + 2 in one load
              load_pair(c + 1, c + 2 < CH, P);
#pragma unroll
              for (int i = 0; i < 4; ++i) vn[i] = P[i];
            }
            vr = vn[0];
          } else if (CH < KS) {
            vr = load_node(4 * CH);
          }
          if (c + 1 == CH) {   // this half has read every accumulator column it needs
            tc_fence_before();
            mbar_arrive(&dempty[s & 1]);
          }
          if constexpr (MODE != 4) {
            emit(c, vl, vc, vr);
            if constexpr (MODE != 1)
              if (c + 1 == ghi(gof(c))) release(gof(c));
          }
          vl = vc[3];
#pragma unroll
          for (int i = 0; i < 4; ++i) vc[i] = vn[i];
        }
        if constexpr (MODE != 4) mbar_arrive(&cempty[s & 1]);   // this step's coupling is read
        if constexpr (MODE == 1) {
          // both ranks' contributions are in global memory: t_m = (b_m - u_0) - u_1
          cluster_arrive();
          cluster_wait();
          const float2* u0 = Ug + m;
          const float2* u1 = Ug + (long long)NN * TW_M + m;
#pragma unroll
          for (int c = CL; c < CH; ++c) {
            float2 t[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int a = 4 * c + i;
              float2 a0 = f2(0.f, 0.f), a1 = f2(0.f, 0.f);
              if (a < NN) {
                a0 = __ldcg(u0 + a * TW_M);
                a1 = __ldcg(u1 + a * TW_M);
              }
              const float2 p = nx[a - A0];
              t[i] = f2((p.x - a0.x) - a1.x, (p.y - a0.y) - a1.y);
            }
            put_a(c, t);
            if (c + 1 == ghi(gof(c))) release(gof(c));
          }
        }
        prefetch(s + 1);
      };

      bool met = false;
      for (int s = 0; s < nseq; ++s) {
        {
          bool ok = tc_wait_warp(&dfull[s & 1], (s >> 1) & 1, &s_abort, err);
          if (ok && s + 1 < nseq) ok = tc_wait_warp(&cfull[s & 1], (s >> 1) & 1, &s_abort, err);
          if (epi_any(!ok)) break;
        }
        tc_fence_after();
        if (s < Lc - 1) step(std::integral_constant<int, 0>{}, s);
        else if (s == Lc - 1) { step(std::integral_constant<int, 1>{}, s); met = true; }
        else if (s == Lc) step(std::integral_constant<int, 2>{}, s);
        else if (s + 1 < nseq) step(std::integral_constant<int, 3>{}, s);
        else step(std::integral_constant<int, 4>{}, s);
      }
      if (!met) {   // the partner meets this CTA at the middle line in any case
        cluster_arrive();
        cluster_wait();
      }
    };
    if (warp < 4) half_body(std::integral_constant<int, 0>{});
    else half_body(std::integral_constant<int, 1>{});
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(TW_TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------------------------ host side
static size_t twtc_fixed_smem(int ks) { return (size_t)2 * ks * TW_ATILE + (size_t)2 * 6 * 8 * ks * 4; }  // A + couplings

static int twtc_stages(const TwGeom& w) {
  const size_t kb = 8 * (size_t)w.tile;   // a stage holds four K-steps
  const size_t fx = twtc_fixed_smem(w.ks);
  if (fx + 2 * kb > (size_t)TW_SMEM) return 0;
  return (int)std::min<size_t>(TW_MAX_NST, ((size_t)TW_SMEM - fx) / kb);
}

bool patch_twtc_ok(int nb) {
  if (nb != 34 && nb != 66 && nb != 130) return false;   // H = 8, 16, 32
  const TwGeom w = patch_twtc_geometry(nb, 3);
  return twtc_stages(w) >= 2;
}

template <int NB>
static cudaError_t launch_twtc(mstopo_handle* h, const PatchGroups& G, const float* r, int sys0,
                               int nsys, float* Xg, float* U) {
  Precond& pc = h->pc;
  const TwGeom w = patch_twtc_geometry(pc.nbP, pc.NP);
  const int nst = twtc_stages(w);
  if (nst < 2 || w.nb != NB || pc.NP % 2 == 0 || pc.NP < 5) return cudaErrorInvalidConfiguration;
  const size_t sm = twtc_fixed_smem(w.ks) + (size_t)nst * 8 * w.tile;
  {
    cudaError_t e = smem_limit_max<k_patch_twtc<NB>>();
    if (e != cudaSuccess) return e;
  }
  const int g0 = G.h_begin[sys0], ng = G.h_begin[sys0 + nsys] - g0;
  if (ng <= 0) return cudaSuccess;
  note_launch(), k_patch_twtc<NB><<<2 * ng, TW_THREADS, sm, h->s>>>(
      r, h->n_dof, sys0, g0, h->nelx, h->nely, pc.H, pc.ncx, G.d_type, G.d_sys, G.d_first,
      G.d_count, G.d_perm, pc.d_pfree, pc.d_ptw, w, nst, Xg, U, h->d_flag + 1);
  return cudaGetLastError();
}

cudaError_t patch_twtc_solve(mstopo_handle* h, const PatchGroups& G, const float* r, int sys0,
                             int nsys, float* Xg, float* U) {
  switch (h->pc.nbP) {
    case 34: return launch_twtc<34>(h, G, r, sys0, nsys, Xg, U);
    case 66: return launch_twtc<66>(h, G, r, sys0, nsys, Xg, U);
    case 130: return launch_twtc<130>(h, G, r, sys0, nsys, Xg, U);
    default: return cudaErrorInvalidConfiguration;
  }
}
