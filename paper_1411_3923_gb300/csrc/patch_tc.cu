// Tensor-core FP32 patch solve: the overlapping local solves of the additive Schwarz level
// (Sec. 3.2, Eq. 3.4: z_i = A_i^{-1} R_i r on every patch omega_i) as block-tridiagonal line
// sweeps on tcgen05.mma (kind::tf32, accumulators in TMEM).
//
// Per patch type, direction and line k the work is one product
//   forward   y_k = [Linv_k | -W_k] [b_k ; y_{k-1}]
//   backward  x_k = [Linv_k^T | -V_k] [y_k ; x_{k+1}]
// of an nb x 2nb factor with nb x R right-hand sides (R patches of one type and realisation).
// The factor is the MMA's A operand (rows 0..127 of a line; nb = 4H + 2 <= 130, rows 128 and
// 129 of H = 32 run on the CUDA cores), the vectors are B.  FP32 accuracy comes from a TF32
// split A = Ahi + Alo (from the FP64 factor when the pack is written) and B = Bhi + Blo (in the
// epilogue): two MMAs per K-step, Ahi [Bhi | Blo] and Alo [Bhi | Blo], into separate TMEM
// columns, and the K-steps spread over TC_P accumulators (K-step s into s mod TC_P) that the
// epilogue sums with round-to-nearest FP32 adds.  The tensor core's FP32 accumulation rounds
// less accurately than an FMA chain; with few K-steps per accumulator the result is as
// accurate as the sequential FP32 dot product (measured: 1.9e-7 against 2.4e-7 relative).
//
// Roles (192 threads): warps 0-3 epilogue (thread i owns TMEM lane = factor row i: reads the
// accumulator, publishes the line, writes the next line's B, gathers the next input), warp 4
// streams the packed factor (cp.async.bulk into a ring of NST stages, mbarrier transaction
// counts), warp 5 issues the MMAs (one elected lane).  Every wait is bounded; a timeout
// records MSTOPO_TIMEOUT, the roles stop, in-flight copies and MMAs are drained and TMEM is
// released before the CTA exits.
#include "internal.cuh"
#include "blocktri.cuh"

namespace {

constexpr int TC_M = 128;                 // factor rows per line on the tensor cores
constexpr int TC_NB = 16;                 // B rows per split half (right-hand sides, padded)
constexpr int TC_TILE = 4096;             // bytes of one 128 x 8 TF32 tile
constexpr int TC_STEP = 2 * TC_TILE;      // hi and lo tiles of one K-step (8 factor columns)
constexpr int TC_KCM = 144;               // byte stride of K-adjacent 8 x 16 B core matrices of B
constexpr int TC_EPI = 128;               // epilogue threads
constexpr int TC_THREADS = TC_EPI + 64;   // + producer warp + MMA warp
constexpr int TC_P = 4;                   // K-partitioned accumulators
constexpr int TC_TMEM_COLS = 64 * TC_P;   // per accumulator: Ahi Bhi | Ahi Blo | Alo Bhi | Alo Blo
constexpr uint32_t TC_WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance of K-adjacent core
// matrices, sbo = of M/N-adjacent ones
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor: D f32, A and B tf32, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 32 lanes x NC columns of 32 bits from TMEM (this warp's lane quarter); the caller waits
template <int NC>
__device__ __forceinline__ void tc_ld(uint32_t taddr, uint32_t (&u)[NC]);
template <>
__device__ __forceinline__ void tc_ld<4>(uint32_t taddr, uint32_t (&u)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3])
               : "r"(taddr));
}
template <>
__device__ __forceinline__ void tc_ld<8>(uint32_t taddr, uint32_t (&u)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]),
                 "=r"(u[6]), "=r"(u[7])
               : "r"(taddr));
}
template <>
__device__ __forceinline__ void tc_ld<16>(uint32_t taddr, uint32_t (&u)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
        "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
        "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// epilogue-only barrier (named barrier 1, 128 threads) that also ORs a flag over them
__device__ __forceinline__ bool epi_sync_or(bool flag) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)flag)
      : "memory");
  return r != 0;
}

// bounded mbarrier wait that also gives up when another role has aborted
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                        int* err) {
  for (uint32_t it = 0; it < TC_WAIT_LIMIT; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && *abort) return false;
  }
  *abort = 1;
  atomicExch(err, (int)MSTOPO_TIMEOUT);
  return false;
}

// wait for work this CTA issued itself (bulk copies, MMAs) before it frees TMEM and exits: an
// abort of another role does not cut it short, only the iteration limit does
__device__ __forceinline__ void tc_drain(uint64_t* bar, uint32_t parity, int* err) {
  for (uint32_t it = 0; it < TC_WAIT_LIMIT; ++it)
    if (mbar_try_wait(bar, parity)) return;
  atomicExch(err, (int)MSTOPO_TIMEOUT);
}

// the same wait for a whole warp: lane 0 polls, the warp takes its result (and its ordering)
__device__ __forceinline__ bool tc_wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort,
                                             int* err) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = tc_wait(bar, parity, abort, err) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

// byte offset of element (n, c) of the B operand: n = right-hand side (hi rows 0..15, lo rows
// 16..31), c = factor column (0..KT); core matrices of 8 rows x 4 columns, K-adjacent ones
// TC_KCM apart, N-adjacent ones sbo apart
__device__ __forceinline__ int b_off(int n, int c, int sbo) {
  return (c >> 2) * TC_KCM + (n >> 3) * sbo + (n & 7) * 16 + (c & 3) * 4;
}

}  // namespace


// Bytes of one packed line: KS K-steps of [hi tile | lo tile] (128 rows x 8 columns, core
// matrices of 8 rows x 16 B: row groups 256 B apart, column halves 128 B apart) followed by
// the factor rows 128..129 in plain FP32 ([2][KT]).
long long patch_tc_line_bytes(int nb) {
  const int KL = (nb + 7) / 8 * 8, KT = 2 * KL, KS = KT / 8;
  return (long long)KS * TC_STEP + 2LL * KT * 4;
}

// Pack per (type, line, direction): forward [Linv_k | -W_k], backward [Linv_k^T | -V_k]
// (the coupling block is zero on the first line of each sweep), split into TF32 hi and lo.
__global__ void k_patch_pack_tc(const double* __restrict__ Linv, const double* __restrict__ W,
                                const double* __restrict__ V, int nb, int NL,
                                long long line_bytes, unsigned char* __restrict__ out) {
  const int type = blockIdx.x, k = blockIdx.y, bw = blockIdx.z;
  const int KL = (nb + 7) / 8 * 8, KT = 2 * KL, KS = KT / 8;
  const long long nn = (long long)nb * nb;
  const double* Lk = Linv + ((long long)type * NL + k) * nn;
  const bool has_c = bw ? (k < NL - 1) : (k > 0);
  const double* Mk = (bw ? V : W) + ((long long)type * NL + k) * nn;
  unsigned char* line = out + (((long long)type * 2 + bw) * NL + k) * line_bytes;
  auto value = [&](int r, int c) -> double {
    if (r >= nb) return 0.0;
    if (c < KL) {
      if (c >= nb) return 0.0;
      return bw ? Lk[(long long)c * nb + r] : Lk[(long long)r * nb + c];
    }
    const int cc = c - KL;
    if (cc >= nb || !has_c) return 0.0;
    return -Mk[(long long)r * nb + cc];
  };
  for (long long t = threadIdx.x; t < (long long)KS * TC_M * 8; t += blockDim.x) {
    const int s = (int)(t / (TC_M * 8)), e = (int)(t % (TC_M * 8));
    const int r = e >> 3, kk = e & 7;
    const double v = value(r, 8 * s + kk);
    const uint32_t hi = tf32_rna((float)v);
    const uint32_t lo = tf32_rna((float)(v - (double)__uint_as_float(hi)));
    const long long o = (long long)s * TC_STEP + (r >> 3) * 256 + (kk >> 2) * 128 + (r & 7) * 16 + (kk & 3) * 4;
    *reinterpret_cast<uint32_t*>(line + o) = hi;
    *reinterpret_cast<uint32_t*>(line + o + TC_TILE) = lo;
  }
  float* tail = reinterpret_cast<float*>(line + (long long)KS * TC_STEP);
  for (int t = threadIdx.x; t < 2 * KT; t += blockDim.x)
    tail[t] = (float)value(TC_M + t / KT, t % KT);
}

template <int Q, int NST, int SU>
__global__ void __launch_bounds__(TC_THREADS) k_patch_solve_tc(
    const float* __restrict__ r, long long stride, int sys0, int g0, int nelx, int nely, int H,
    int ncx, const int* __restrict__ grp_type, const int* __restrict__ grp_sys,
    const int* __restrict__ grp_first, const int* __restrict__ grp_count,
    const int* __restrict__ perm, const uint8_t* __restrict__ pfree,
    const unsigned char* __restrict__ pack, long long line_bytes, float* __restrict__ Xg,
    int* __restrict__ err) {
  constexpr int R = 4 * Q;
  constexpr int RC = R <= 4 ? 4 : R <= 8 ? 8 : 16;   // accumulator columns read per block
  static_assert(R <= TC_NB, "right-hand sides per CTA");
  __shared__ __align__(8) uint64_t full[NST], empty[NST], tfull[2], tempty[2], bready, ldone, fin;
  __shared__ volatile int s_abort;
  __shared__ uint32_t s_tmem;
  __shared__ int s_node[TC_NB];
  extern __shared__ __align__(16) unsigned char smraw[];

  const int N = 2 * H + 1, nb = 2 * N, NL = N;
  const int KL = (nb + 7) / 8 * 8, KT = 2 * KL, KS = KT / 8;
  const int nunits = (KS + SU - 1) / SU;
  const int ntail = nb > TC_M ? nb - TC_M : 0;   // 0 or 2 (H = 32)
  const int sbo = (KT / 4) * TC_KCM;              // N-group stride of B
  unsigned char* ring = smraw;                                  // [NST][SU][TC_STEP]
  unsigned char* bmat = ring + NST * SU * TC_STEP;              // [4 N-groups][sbo]
  float* tailbuf = reinterpret_cast<float*>(bmat + 4 * sbo);    // [2][2][KT]
  const uint32_t tail_bytes = (uint32_t)(2 * KT * 4);

  const int g = g0 + blockIdx.x;
  const int type = grp_type[g], first = grp_first[g], cnt = grp_count[g];
  const float* rs = r + (long long)(grp_sys[g] - sys0) * stride;
  const uint8_t* fr = pfree + (long long)type * N * nb;
  float* X = Xg + (long long)g * NL * R * nb;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid < TC_NB) s_node[tid] = tid < cnt ? perm[first + tid] : -1;
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < NST; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
    for (int i = 0; i < 2; ++i) { mbar_init(&tfull[i], 1); mbar_init(&tempty[i], TC_EPI); }
    mbar_init(&bready, TC_EPI);
    mbar_init(&ldone, 1);
    mbar_init(&fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // B starts at zero: its padding columns and the coupling part of the first line stay zero
  for (int q = tid; q < sbo / 4; q += TC_THREADS)   // 4 N-groups x sbo bytes, 16 B per store
    reinterpret_cast<uint4*>(bmat)[q] = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = s_tmem;

  if (warp == 4) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int ug = 0, tfills = 0;
      bool ok = true;
      for (int ls = 0; ls < 2 * NL && ok; ++ls) {
        const bool fw = ls < NL;
        const int k = fw ? ls : 2 * NL - 1 - ls;
        const unsigned char* lb = pack + (((long long)type * 2 + (fw ? 0 : 1)) * NL + k) * line_bytes;
        if (ntail) {
          const int b = ls & 1;
          if (ls >= 2 && !tc_wait(&tempty[b], ((ls >> 1) + 1) & 1, &s_abort, err)) { ok = false; break; }
          mbar_expect_tx(&tfull[b], tail_bytes);
          bulk_g2s(tailbuf + b * 2 * KT, lb + (long long)KS * TC_STEP, tail_bytes, &tfull[b]);
          ++tfills;
        }
        for (int u = 0; u < nunits; ++u, ++ug) {
          const int st = ug % NST;
          if (ug >= NST && !tc_wait(&empty[st], ((ug / NST) + 1) & 1, &s_abort, err)) { ok = false; break; }
          const int s0 = u * SU, ns = min(SU, KS - s0);
          mbar_expect_tx(&full[st], (uint32_t)(ns * TC_STEP));
          bulk_g2s(ring + st * SU * TC_STEP, lb + (long long)s0 * TC_STEP, (uint32_t)(ns * TC_STEP), &full[st]);
        }
      }
      // drain: the last fill of every stage (and tail buffer) has landed before the CTA exits
      for (int st = 0; st < NST && st < ug; ++st) {
        const int last = (ug - 1 - st) / NST;   // index of the last fill of stage st
        tc_drain(&full[st], last & 1, err);
      }
      for (int b = 0; b < 2 && b < tfills; ++b) tc_drain(&tfull[b], ((tfills - 1 - b) / 2) & 1, err);
    }
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      // descriptors advance by address only: stage/K-step offsets added to the start field
      const uint64_t da0 = tc_sdesc(smem_u32(ring), 128, 256);
      const uint64_t db0 = tc_sdesc(smem_u32(bmat), TC_KCM, (uint32_t)sbo);
      constexpr uint32_t id2 = tc_idesc(TC_M, 2 * TC_NB);
      int ug = 0;
      bool issued = false;
      for (int ls = 0; ls < 2 * NL; ++ls) {
        if (!tc_wait(&bready, ls & 1, &s_abort, err)) break;
        tc_fence_after();
        bool ok = true;
        for (int u = 0; u < nunits; ++u, ++ug) {
          const int st = ug % NST;
          if (!tc_wait(&full[st], (ug / NST) & 1, &s_abort, err)) { ok = false; break; }
          const int s0 = u * SU, ns = min(SU, KS - s0);
          uint64_t da = da0 + (uint64_t)((st * SU * TC_STEP) >> 4);
          uint64_t db = db0 + (uint64_t)((2 * s0 * TC_KCM) >> 4);
          for (int q = 0; q < ns; ++q) {
            const int s = s0 + q;
            const uint32_t d = tm + (uint32_t)((s % TC_P) * 64);
            const uint32_t acc = s >= TC_P ? 1u : 0u;
            tc_mma(d, da, db, id2, acc);                                 // Ahi [Bhi | Blo]
            tc_mma(d + 32, da + (uint64_t)(TC_TILE >> 4), db, id2, acc);  // Alo [Bhi | Blo]
            da += (uint64_t)(TC_STEP >> 4);
            db += (uint64_t)((2 * TC_KCM) >> 4);
          }
          tc_commit(&empty[st]);
          issued = true;
        }
        if (!ok) break;
        tc_commit(&ldone);
      }
      if (issued) {   // drain: every MMA this thread issued has completed
        tc_commit(&fin);
        tc_drain(&fin, 0, err);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int i = tid;   // factor row = TMEM lane
    float pf[R], pft[R], y[R];
    // input of line ls for factor row c (forward: gather of r; backward: y_k of the forward sweep)
    auto load_input = [&](int ls, int c, float (&v)[R]) {
      const bool fw = ls < NL;
      const int k = fw ? ls : 2 * NL - 1 - ls;
#pragma unroll
      for (int p = 0; p < R; ++p) v[p] = 0.f;
      if (c >= nb) return;
      if (fw) {
        if (!fr[(long long)k * nb + c]) return;
#pragma unroll
        for (int p = 0; p < R; ++p) {
          if (p < cnt) {
            const int ia = s_node[p];
            const int I = ia % (ncx + 1), J = ia / (ncx + 1);
            const int x = (I - 1) * H + (c >> 1), yy = (J - 1) * H + k;
            if (x >= 0 && x <= nelx && yy >= 0 && yy <= nely)
              v[p] = rs[2 * ((long long)yy * (nelx + 1) + x) + (c & 1)];
          }
        }
      } else {
        const float4* src = reinterpret_cast<const float4*>(X + (long long)k * nb * R + (long long)c * R);
#pragma unroll
        for (int p = 0; p < R; p += 4) {
          const float4 q = src[p / 4];
          v[p] = q.x; v[p + 1] = q.y; v[p + 2] = q.z; v[p + 3] = q.w;
        }
      }
    };
    // B rows of factor column c <- v (hi and lo parts)
    auto put_b = [&](int c, const float (&v)[R]) {
#pragma unroll
      for (int p = 0; p < R; ++p) {
        const uint32_t hi = tf32_rna(v[p]);
        const uint32_t lo = tf32_rna(v[p] - __uint_as_float(hi));
        *reinterpret_cast<uint32_t*>(bmat + b_off(p, c, sbo)) = hi;
        *reinterpret_cast<uint32_t*>(bmat + b_off(TC_NB + p, c, sbo)) = lo;
      }
    };
    auto put_b1 = [&](int p, int c, float v) {
      const uint32_t hi = tf32_rna(v);
      const uint32_t lo = tf32_rna(v - __uint_as_float(hi));
      *reinterpret_cast<uint32_t*>(bmat + b_off(p, c, sbo)) = hi;
      *reinterpret_cast<uint32_t*>(bmat + b_off(TC_NB + p, c, sbo)) = lo;
    };
    // tail-row work split: (row t, column j, quarter part) per thread; part 0 owns the result
    const int tq = KT / 4;   // columns per quarter (KT is a multiple of 16)
    const int t_row = i / (4 * R), t_j = (i % (4 * R)) >> 2, t_part = i & 3;
    const bool t_active = t_row < ntail;
    float yt = 0.f;

    // line 0: input gathered, coupling part zero
    load_input(0, i, pf);
    if (i < nb) put_b(i, pf);
    if (i < ntail) { load_input(0, TC_M + i, pft); put_b(TC_M + i, pft); }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive(&bready);

    bool abort = false;
    for (int ls = 0; ls < 2 * NL && !abort; ++ls) {
      const bool fw = ls < NL;
      const int k = fw ? ls : 2 * NL - 1 - ls;
      const int nxt = ls + 1;
      // (a) factor rows 128.. on the CUDA cores, beside the MMA chain
      if (ntail) {
        const int b = ls & 1;
        const bool ok = tc_wait_warp(&tfull[b], (ls >> 1) & 1, &s_abort, err);
        if (epi_sync_or(!ok)) { abort = true; break; }
        float acc = 0.f;
        if (t_active) {
          const float* trow = tailbuf + (b * 2 + t_row) * KT;
          for (int c = t_part * tq; c < (t_part + 1) * tq; c += 4) {
            const float4 f = *reinterpret_cast<const float4*>(trow + c);
            const float4 h = *reinterpret_cast<const float4*>(bmat + b_off(t_j, c, sbo));
            const float4 l = *reinterpret_cast<const float4*>(bmat + b_off(TC_NB + t_j, c, sbo));
            acc = fmaf(f.x, h.x + l.x, acc);
            acc = fmaf(f.y, h.y + l.y, acc);
            acc = fmaf(f.z, h.z + l.z, acc);
            acc = fmaf(f.w, h.w + l.w, acc);
          }
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        yt = acc;
        mbar_arrive(&tempty[b]);
      }
      // (b) next line's input (not for the first backward line: that is this line's result)
      if (nxt < 2 * NL && nxt != NL) {
        load_input(nxt, i, pf);
        if (i < ntail) load_input(nxt, TC_M + i, pft);
      }
      // (c) accumulator of this line
      {
        const bool ok = tc_wait_warp(&ldone, ls & 1, &s_abort, err);
        if (epi_sync_or(!ok)) { abort = true; break; }
      }
      tc_fence_after();
      {
        // y = sum over the accumulators of Ahi Bhi, plus the sum of the three correction products
        float big[R], small[R];
#pragma unroll
        for (int p = 0; p < R; ++p) { big[p] = 0.f; small[p] = 0.f; }
        const uint32_t tl = tm + ((uint32_t)(warp * 32) << 16);
        for (int a = 0; a < TC_P && a < KS; ++a) {
          uint32_t u[4][RC];
#pragma unroll
          for (int q = 0; q < 4; ++q) tc_ld<RC>(tl + (uint32_t)(a * 64 + q * TC_NB), u[q]);
          tc_wait_ld();
#pragma unroll
          for (int p = 0; p < R; ++p) {
            big[p] += __uint_as_float(u[0][p]);
            small[p] += __uint_as_float(u[1][p]) + __uint_as_float(u[2][p]) + __uint_as_float(u[3][p]);
          }
        }
#pragma unroll
        for (int p = 0; p < R; ++p) y[p] = big[p] + small[p];
      }
      // (d) every read of this line's B and accumulator is done
      tc_fence_before();
      epi_sync_or(false);
      // (e) publish: forward y_k -> [nb][R], backward x_k -> [R][nb]
      float* Xk = X + (long long)k * nb * R;
      if (i < nb) {
        if (fw) {
          float4* dst = reinterpret_cast<float4*>(Xk + (long long)i * R);   // 16-byte aligned: R = 4Q
#pragma unroll
          for (int p = 0; p < R; p += 4) dst[p / 4] = make_float4(y[p], y[p + 1], y[p + 2], y[p + 3]);
        } else {
#pragma unroll
          for (int p = 0; p < R; ++p) Xk[(long long)p * nb + i] = y[p];
        }
      }
      const bool t_owner = t_active && t_part == 0 && t_j < R;
      if (t_owner) {
        const int row = TC_M + t_row;
        if (fw) Xk[(long long)row * R + t_j] = yt;
        else Xk[(long long)t_j * nb + row] = yt;
      }
      // (f) B of the next line: input part (columns 0..nb) and coupling part (KL..KL+nb)
      if (nxt < 2 * NL) {
        const bool first_bwd = nxt == NL;
        if (i < nb) {
          if (first_bwd) {
            put_b(i, y);
            float z[R];
#pragma unroll
            for (int p = 0; p < R; ++p) z[p] = 0.f;
            put_b(KL + i, z);
          } else {
            put_b(i, pf);
            put_b(KL + i, y);
          }
        }
        if (i < ntail && !first_bwd) put_b(TC_M + i, pft);
        if (t_owner) {
          const int row = TC_M + t_row;
          if (first_bwd) { put_b1(t_j, row, yt); put_b1(t_j, KL + row, 0.f); }
          else put_b1(t_j, KL + row, yt);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&bready);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(TC_TMEM_COLS)
                 : "memory");
  }
}

cudaError_t patch_tc_pack(const double* Linv, const double* W, const double* V, int T, int nb,
                          int NL, unsigned char* out, cudaStream_t s) {
  note_launch(), k_patch_pack_tc<<<dim3(T, NL, 2), 256, 0, s>>>(Linv, W, V, nb, NL,
                                                                patch_tc_line_bytes(nb), out);
  return cudaGetLastError();
}

// Factor ring: stages of TC_SU K-steps (16 KB).  The stream is latency-bound (bytes in flight
// per SM / copy latency), so with at most one CTA per SM the ring is deep (TC_NST_DEEP stages,
// ~160 KB); with more CTAs than SMs two shallower CTAs share each SM and overlap one
// CTA's epilogue with the other's MMA chain.
#define TC_SU 2
#define TC_NST 4
#define TC_NST_DEEP 10

size_t patch_tc_smem(int nb, int nst) {
  const int KL = (nb + 7) / 8 * 8, KT = 2 * KL;
  return (size_t)nst * TC_SU * TC_STEP + 4 * (size_t)(KT / 4) * TC_KCM + 2 * 2 * (size_t)KT * 4;
}

template <int Q, int NST>
static cudaError_t launch_tc_k(mstopo_handle* h, const float* r, int sys0, int g0, int ng, float* Xg) {
  Precond& pc = h->pc;
  const size_t sm = patch_tc_smem(pc.nbP, NST);
  {
    cudaError_t e = smem_limit_max<k_patch_solve_tc<Q, NST, TC_SU>>();
    if (e != cudaSuccess) return e;
  }
  if (sm > 225 * 1024) return cudaErrorInvalidConfiguration;
  note_launch(), k_patch_solve_tc<Q, NST, TC_SU><<<ng, TC_THREADS, sm, h->s>>>(
      r, h->n_dof, sys0, g0, h->nelx, h->nely, pc.H, pc.ncx, pc.pg[1].d_type, pc.pg[1].d_sys,
      pc.pg[1].d_first, pc.pg[1].d_count, pc.pg[1].d_perm, pc.d_pfree, pc.d_ptc, pc.tc_line_bytes, Xg,
      h->d_flag + 1);
  return cudaGetLastError();
}

template <int Q>
static cudaError_t launch_tc(mstopo_handle* h, const float* r, int sys0, int nsys, float* Xg) {
  Precond& pc = h->pc;
  const int g0 = pc.pg[1].h_begin[sys0], ng = pc.pg[1].h_begin[sys0 + nsys] - g0;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, n = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    sms = n;
  }
  const bool deep = ng <= sms;
  return deep ? launch_tc_k<Q, TC_NST_DEEP>(h, r, sys0, g0, ng, Xg)
              : launch_tc_k<Q, TC_NST>(h, r, sys0, g0, ng, Xg);
}

cudaError_t patch_tc_solve(mstopo_handle* h, int Q, const float* r, int sys0, int nsys, float* Xg) {
  switch (Q) {
    case 1: return launch_tc<1>(h, r, sys0, nsys, Xg);
    case 2: return launch_tc<2>(h, r, sys0, nsys, Xg);
    case 3: return launch_tc<3>(h, r, sys0, nsys, Xg);
    default: return launch_tc<4>(h, r, sys0, nsys, Xg);
  }
}
