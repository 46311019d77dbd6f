// Matrix-free Q4 stiffness matvec with SIMP moduli (paper Sec. 2.1, Eq. for K_e in Sec. 2.2).
//
// y_n = sum over the four elements e around node n of E_e * (K0 u_e)_n, evaluated node by
// node.  Because K0 annihilates rigid translations, (K0 u_e)_n = sum over the other three
// nodes m of K0_nm (u_m - u_n): the kernel forms the eight neighbour differences first, so
// FP32 rounding is relative to the (small) differences of a smooth field rather than to
// the field itself.  Dirichlet DOFs of u are read as zero, Dirichlet DOFs of y are zero.
//
// Work split: one thread per node column i, a strip of MV_TY node rows per thread; the 3x3
// neighbourhood and the 2x2 surrounding moduli slide up the strip in registers, so each
// node row of u and each element row of E is loaded once (the neighbour columns come from
// the adjacent lanes).  Grid: ceil((nelx+1)/MV_TX) x ceil((nely+1)/MV_TY) x systems.
#include "internal.cuh"

#define MV_TX 128
#define MV_TY 18   // node rows per thread (a multiple of the 3-row chunk)

void element_stiffness_closed_form(double nu, double K0[64]) {
  // Bilinear shape functions on [0,1]^2: N0=(1-x)(1-y), N1=x(1-y), N2=xy, N3=(1-x)y.
  // dNa/dx = sx[a] * (y-factor), dNa/dy = sy[a] * (x-factor); the integrals of products of
  // the linear factors are 1/3 (same factor) or 1/6 (complementary), of one factor 1/2.
  const int sx[4] = {-1, 1, 1, -1}, sy[4] = {-1, -1, 1, 1};
  const int fy[4] = {0, 0, 1, 1};   // y-factor of dN/dx: 0 -> (1-y), 1 -> y
  const int fx[4] = {0, 1, 1, 0};   // x-factor of dN/dy: 0 -> (1-x), 1 -> x
  const double s = 1.0 / (1.0 - nu * nu);
  const double C11 = s, C12 = nu * s, C33 = 0.5 * (1.0 - nu) * s;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      double Ixx = sx[a] * sx[b] * (fy[a] == fy[b] ? 1.0 / 3.0 : 1.0 / 6.0);
      double Iyy = sy[a] * sy[b] * (fx[a] == fx[b] ? 1.0 / 3.0 : 1.0 / 6.0);
      double Ixy = sx[a] * sy[b] * 0.25;   // int dNa/dx dNb/dy
      double Iyx = sy[a] * sx[b] * 0.25;   // int dNa/dy dNb/dx
      K0[(2 * a) * 8 + 2 * b] = C11 * Ixx + C33 * Iyy;
      K0[(2 * a) * 8 + 2 * b + 1] = C12 * Ixy + C33 * Iyx;
      K0[(2 * a + 1) * 8 + 2 * b] = C12 * Iyx + C33 * Ixy;
      K0[(2 * a + 1) * 8 + 2 * b + 1] = C11 * Iyy + C33 * Ixx;
    }
}

// Node n is local node SELF[e] of surrounding element e (LL, LR, UL, UR); the other three
// local nodes of e are OTHER[e][m].
static const int SELF[4] = {2, 3, 1, 0};
static const int OTHER[4][3] = {{0, 1, 3}, {0, 1, 2}, {0, 2, 3}, {1, 2, 3}};

void make_stencil(const double K0[64], StencilCoef<double>& cd, StencilCoef<float>& cf) {
  for (int e = 0; e < 4; ++e)
    for (int m = 0; m < 3; ++m) {
      int a = SELF[e], b = OTHER[e][m];
      double blk[4] = {K0[(2 * a) * 8 + 2 * b], K0[(2 * a) * 8 + 2 * b + 1],
                       K0[(2 * a + 1) * 8 + 2 * b], K0[(2 * a + 1) * 8 + 2 * b + 1]};
      for (int q = 0; q < 4; ++q) {
        cd.c[e][m][q] = blk[q];
        cf.c[e][m][q] = (float)blk[q];
      }
    }
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

template <typename T>
__device__ __forceinline__ T load_E(const T* __restrict__ E, int ex, int ey, int nelx, int nely) {
  return (ex >= 0 && ex < nelx && ey >= 0 && ey < nely) ? E[(long long)ey * nelx + ex] : T(0);
}

// acc += B * (d) for a row-major 2x2 block B
template <typename T>
__device__ __forceinline__ void blk(T& ax, T& ay, const T* b, T dx, T dy) {
  ax = fma(b[0], dx, ax); ax = fma(b[1], dy, ax);
  ay = fma(b[2], dx, ay); ay = fma(b[3], dy, ay);
}

template <typename T>
__device__ __forceinline__ typename Vec2<T>::type shfl_up2(typename Vec2<T>::type v) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_up_sync(0xffffffffu, v.y, 1);
  return v;
}
template <typename T>
__device__ __forceinline__ typename Vec2<T>::type shfl_down2(typename Vec2<T>::type v) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_down_sync(0xffffffffu, v.y, 1);
  return v;
}

// Rows come in chunks of three: the node row entering the window, its element row and the
// output mask are loaded one chunk ahead (software pipelining), and the three window rows
// rotate through the unrolled chunk by renaming, so no register moves are needed.  A warp
// covers 32 consecutive node columns; left/right neighbours come from the adjacent lanes by
// shuffles (the edge lanes load their own).  MASK_IN: read Dirichlet entries of u as zero
// (the flexible-CG vectors are already zero there, so its instance skips this).
template <typename T>
struct RowV {
  typename Vec2<T>::type l, c, r;
};

template <typename T, bool MASK_IN>
__device__ __forceinline__ typename Vec2<T>::type ld_node(const T* __restrict__ u,
                                                          const uint8_t* __restrict__ m, int i,
                                                          int j, int nx1, int ny1) {
  typedef typename Vec2<T>::type V;
  V v;
  v.x = T(0); v.y = T(0);
  if (i >= 0 && i < nx1 && j >= 0 && j < ny1) {
    const long long n = (long long)j * nx1 + i;
    v = reinterpret_cast<const V*>(u)[n];
    if (MASK_IN) {
      const uint8_t f = m[n];
      if (f & 1) v.x = T(0);
      if (f & 2) v.y = T(0);
    }
  }
  return v;
}

// pending loads of one row: centre node, edge-lane neighbour, element moduli (centre, left)
// and the output mask of the row below
template <typename T>
struct Pend {
  typename Vec2<T>::type c, e;
  T ec, el;
  uint8_t m;
};

template <typename T, bool MASK_IN>
__device__ __forceinline__ void issue_row(Pend<T>& p, const T* __restrict__ u,
                                          const T* __restrict__ E, const uint8_t* __restrict__ nm,
                                          int i, int lane, int jn, int nelx, int nely, int nx1,
                                          int ny1, bool in) {
  p.c = ld_node<T, MASK_IN>(u, nm, i, jn, nx1, ny1);
  p.e = ld_node<T, MASK_IN>(u, nm, lane == 0 ? i - 1 : i + 1, jn, nx1, ny1);
  p.ec = load_E(E, i, jn - 1, nelx, nely);
  p.el = load_E(E, i - 1, jn - 1, nelx, nely);
  p.m = (in && jn - 1 >= 0 && jn - 1 < ny1) ? nm[(long long)(jn - 1) * nx1 + i] : (uint8_t)3;
}

// Interior blocks (every touched node and element inside the mesh): no bounds checks; the
// caller passes the row pointers of node row jn and element row jn-1 at column i.
template <typename T, bool MASK_IN>
__device__ __forceinline__ void issue_row_fast(Pend<T>& p, const T* __restrict__ urow,
                                               const T* __restrict__ erow,
                                               const uint8_t* __restrict__ mrow,
                                               const uint8_t* __restrict__ mrow_below, int lane) {
  typedef typename Vec2<T>::type V;
  const V* ur = reinterpret_cast<const V*>(urow);
  p.c = ur[0];
  const int off = lane == 0 ? -1 : 1;
  p.e = ur[off];
  if (MASK_IN) {
    const uint8_t fc = mrow[0], fe = mrow[off];
    if (fc & 1) p.c.x = T(0);
    if (fc & 2) p.c.y = T(0);
    if (fe & 1) p.e.x = T(0);
    if (fe & 2) p.e.y = T(0);
  }
  p.ec = erow[0];
  p.el = erow[-1];
  p.m = mrow_below[0];
}

template <typename T>
__device__ __forceinline__ RowV<T> make_row(const Pend<T>& p, int lane) {
  RowV<T> w;
  w.c = p.c;
  w.l = shfl_up2<T>(p.c);
  w.r = shfl_down2<T>(p.c);
  if (lane == 0) w.l = p.e;
  if (lane == 31) w.r = p.e;
  return w;
}

// y(i, j) from the window rows (b: j-1, m: j, t: j+1) and the moduli of the four elements
template <typename T>
__device__ __forceinline__ void node_force(const RowV<T>& b, const RowV<T>& m, const RowV<T>& t,
                                           T eLL, T eLR, T eUL, T eUR, const StencilCoef<T>& c,
                                           T& yx, T& yy) {
  const T cx = m.c.x, cy = m.c.y;
  const T d00x = b.l.x - cx, d00y = b.l.y - cy, d01x = b.c.x - cx, d01y = b.c.y - cy;
  const T d02x = b.r.x - cx, d02y = b.r.y - cy, d10x = m.l.x - cx, d10y = m.l.y - cy;
  const T d12x = m.r.x - cx, d12y = m.r.y - cy, d20x = t.l.x - cx, d20y = t.l.y - cy;
  const T d21x = t.c.x - cx, d21y = t.c.y - cy, d22x = t.r.x - cx, d22y = t.r.y - cy;
  T ax, ay;
  yx = T(0); yy = T(0);
  ax = T(0); ay = T(0);   // LL element (i-1, j-1): others (i-1,j-1), (i,j-1), (i-1,j)
  blk(ax, ay, c.c[0][0], d00x, d00y); blk(ax, ay, c.c[0][1], d01x, d01y); blk(ax, ay, c.c[0][2], d10x, d10y);
  yx = fma(eLL, ax, yx); yy = fma(eLL, ay, yy);
  ax = T(0); ay = T(0);   // LR element (i, j-1): others (i,j-1), (i+1,j-1), (i+1,j)
  blk(ax, ay, c.c[1][0], d01x, d01y); blk(ax, ay, c.c[1][1], d02x, d02y); blk(ax, ay, c.c[1][2], d12x, d12y);
  yx = fma(eLR, ax, yx); yy = fma(eLR, ay, yy);
  ax = T(0); ay = T(0);   // UL element (i-1, j): others (i-1,j), (i,j+1), (i-1,j+1)
  blk(ax, ay, c.c[2][0], d10x, d10y); blk(ax, ay, c.c[2][1], d21x, d21y); blk(ax, ay, c.c[2][2], d20x, d20y);
  yx = fma(eUL, ax, yx); yy = fma(eUL, ay, yy);
  ax = T(0); ay = T(0);   // UR element (i, j): others (i+1,j), (i+1,j+1), (i,j+1)
  blk(ax, ay, c.c[3][0], d12x, d12y); blk(ax, ay, c.c[3][1], d22x, d22y); blk(ax, ay, c.c[3][2], d21x, d21y);
  yx = fma(eUR, ax, yx); yy = fma(eUR, ay, yy);
}

template <typename T, bool MASK_IN, bool FAST>
__device__ __forceinline__ void matvec_strip(const T* __restrict__ u, T* __restrict__ y,
                                             const T* __restrict__ E,
                                             const uint8_t* __restrict__ nmask, int nelx, int nely,
                                             const StencilCoef<T>& c, int i, int j0, int lane,
                                             bool in) {
  typedef typename Vec2<T>::type V;
  const int nx1 = nelx + 1, ny1 = nely + 1;
  // row pointers for the fast path: node row j at column i, element row j-1 at column i
  const T* up = u + 2 * ((long long)(j0 - 1) * nx1 + i);
  const T* ep = E + ((long long)(j0 - 2) * nelx + i);
  const uint8_t* mp = nmask + ((long long)(j0 - 1) * nx1 + i);
  auto issue = [&](Pend<T>& p, int jn) {
    if (FAST) {
      const long long dr = jn - (j0 - 1);
      issue_row_fast<T, MASK_IN>(p, up + 2 * dr * nx1, ep + dr * nelx, mp + dr * nx1,
                                 mp + (dr - 1) * nx1, lane);
    } else {
      issue_row<T, MASK_IN>(p, u, E, nmask, i, lane, jn, nelx, nely, nx1, ny1, in);
    }
  };
  Pend<T> p0, p1, p2;
  issue(p0, j0 - 1);
  issue(p1, j0);
  RowV<T> w0 = make_row<T>(p0, lane), w1 = make_row<T>(p1, lane), w2;
  T eL0 = __shfl_up_sync(0xffffffffu, p1.ec, 1), eC0 = p1.ec;   // element row j0-1
  if (lane == 0) eL0 = p1.el;
  T eL1, eC1, eL2, eC2;
  const int jend = min(j0 + MV_TY, ny1);
  issue(p0, j0 + 1);
  issue(p1, j0 + 2);
  issue(p2, j0 + 3);
  auto emit = [&](int j, uint8_t f, T yx, T yy) {
    if (in && j < jend) {
      V out;
      out.x = (f & 1) ? T(0) : yx;
      out.y = (f & 2) ? T(0) : yy;
      reinterpret_cast<V*>(y)[(long long)j * nx1 + i] = out;
    }
  };
  for (int jb = j0; jb < jend; jb += 3) {
    T yx, yy;
    // row jb: window (w0, w1, w2 <- p0), element rows jb-1 (eL0, eC0) and jb
    w2 = make_row<T>(p0, lane);
    eC1 = p0.ec; eL1 = __shfl_up_sync(0xffffffffu, p0.ec, 1); if (lane == 0) eL1 = p0.el;
    const uint8_t f0 = p0.m;
    if (jb + 4 <= jend + 1) issue(p0, jb + 4);
    node_force<T>(w0, w1, w2, eL0, eC0, eL1, eC1, c, yx, yy);
    emit(jb, f0, yx, yy);
    // row jb+1: window (w1, w2, w0 <- p1), element rows jb (eL1, eC1) and jb+1
    w0 = make_row<T>(p1, lane);
    eC2 = p1.ec; eL2 = __shfl_up_sync(0xffffffffu, p1.ec, 1); if (lane == 0) eL2 = p1.el;
    const uint8_t f1 = p1.m;
    if (jb + 5 <= jend + 1) issue(p1, jb + 5);
    node_force<T>(w1, w2, w0, eL1, eC1, eL2, eC2, c, yx, yy);
    emit(jb + 1, f1, yx, yy);
    // row jb+2: window (w2, w0, w1 <- p2), element rows jb+1 (eL2, eC2) and jb+2
    w1 = make_row<T>(p2, lane);
    eC0 = p2.ec; eL0 = __shfl_up_sync(0xffffffffu, p2.ec, 1); if (lane == 0) eL0 = p2.el;
    const uint8_t f2 = p2.m;
    if (jb + 6 <= jend + 1) issue(p2, jb + 6);
    node_force<T>(w2, w0, w1, eL2, eC2, eL0, eC0, c, yx, yy);
    emit(jb + 2, f2, yx, yy);
    // now w0 = row jb+2, w1 = row jb+3 and (eL0, eC0) = element row jb+2: the state the
    // next chunk starts from
  }
}

template <typename T, bool MASK_IN>
__global__ void __launch_bounds__(MV_TX) k_matvec(const T* __restrict__ u, T* __restrict__ y,
                                                  const T* __restrict__ E,
                                                  const uint8_t* __restrict__ nmask, int nelx,
                                                  int nely, StencilCoef<T> c,
                                                  long long vec_stride, long long e_stride) {
  const int lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * MV_TX;
  const int i = i0 + threadIdx.x;
  const int j0 = blockIdx.y * MV_TY;
  const bool in = i < nelx + 1;
  u += blockIdx.z * vec_stride;
  y += blockIdx.z * vec_stride;
  E += blockIdx.z * e_stride;
  // a block is interior when all nodes it reads (columns i0-1 .. i0+MV_TX, rows j0-1 ..
  // j0+MV_TY+1) and all elements it reads (columns i0-1 .. i0+MV_TX-1, rows j0-2 .. j0+MV_TY)
  // lie inside the mesh
  const bool fast = i0 >= 1 && i0 + MV_TX < nelx && j0 >= 2 && j0 + MV_TY + 1 <= nely;
  if (fast)
    matvec_strip<T, MASK_IN, true>(u, y, E, nmask, nelx, nely, c, i, j0, lane, in);
  else
    matvec_strip<T, MASK_IN, false>(u, y, E, nmask, nelx, nely, c, i, j0, lane, in);
}


// ---------------------------------------------------------------------------------------
// FP32 variant with two adjacent node columns (i0 = 2t, i0 + 1) per thread: the neighbour
// columns and the element moduli between the two nodes are shared inside the thread, so
// loads, shuffles and index arithmetic per node are halved.  A warp covers 64 columns.
struct Row4 { float2 L, A, B, R; };            // node columns i0-1, i0, i0+1, i0+2
struct ERow { float l, a, b; };                 // element columns i0-1, i0, i0+1

struct Pend2 {
  float2 A, B, e;    // centre nodes and the edge-lane neighbour (lane 0: i0-1, lane 31: i0+2)
  float ea, eb, el;  // element moduli (i0, i0+1) of the row below, and lane 0's (i0-1)
  uint8_t ma, mb;    // output masks of the row below
};

template <bool MASK_IN, bool FAST>
__device__ __forceinline__ void issue2(Pend2& p, const float* __restrict__ u,
                                       const float* __restrict__ E,
                                       const uint8_t* __restrict__ nm, int i0, int lane, int jn,
                                       int nelx, int nely) {
  const int nx1 = nelx + 1, ny1 = nely + 1;
  const int ie = lane == 0 ? i0 - 1 : i0 + 2;
  if (FAST) {
    const float2* ur = reinterpret_cast<const float2*>(u) + (long long)jn * nx1;
    p.A = ur[i0];
    p.B = ur[i0 + 1];
    p.e = ur[ie];
    if (MASK_IN) {
      const uint8_t* mr = nm + (long long)jn * nx1;
      const uint8_t fa = mr[i0], fb = mr[i0 + 1], fe = mr[ie];
      if (fa & 1) p.A.x = 0.f;
      if (fa & 2) p.A.y = 0.f;
      if (fb & 1) p.B.x = 0.f;
      if (fb & 2) p.B.y = 0.f;
      if (fe & 1) p.e.x = 0.f;
      if (fe & 2) p.e.y = 0.f;
    }
    const float* er = E + (long long)(jn - 1) * nelx;
    p.ea = er[i0];
    p.eb = er[i0 + 1];
    p.el = er[i0 - 1];
    const uint8_t* mb = nm + (long long)(jn - 1) * nx1;
    p.ma = mb[i0];
    p.mb = mb[i0 + 1];
  } else {
    p.A = ld_node<float, MASK_IN>(u, nm, i0, jn, nx1, ny1);
    p.B = ld_node<float, MASK_IN>(u, nm, i0 + 1, jn, nx1, ny1);
    p.e = ld_node<float, MASK_IN>(u, nm, ie, jn, nx1, ny1);
    p.ea = load_E(E, i0, jn - 1, nelx, nely);
    p.eb = load_E(E, i0 + 1, jn - 1, nelx, nely);
    p.el = load_E(E, i0 - 1, jn - 1, nelx, nely);
    const bool rv = jn - 1 >= 0 && jn - 1 < ny1;
    p.ma = (rv && i0 < nx1) ? nm[(long long)(jn - 1) * nx1 + i0] : (uint8_t)3;
    p.mb = (rv && i0 + 1 < nx1) ? nm[(long long)(jn - 1) * nx1 + i0 + 1] : (uint8_t)3;
  }
}

__device__ __forceinline__ void make_row2(const Pend2& p, int lane, Row4& w, ERow& er) {
  w.A = p.A;
  w.B = p.B;
  w.L = shfl_up2<float>(p.B);
  w.R = shfl_down2<float>(p.A);
  if (lane == 0) w.L = p.e;
  if (lane == 31) w.R = p.e;
  er.a = p.ea;
  er.b = p.eb;
  er.l = __shfl_up_sync(0xffffffffu, p.eb, 1);
  if (lane == 0) er.l = p.el;
}


// forces at nodes i0 (columns L,A,B) and i0+1 (columns A,B,R); element rows below (eb) and
// at the node row (et)
__device__ __forceinline__ void pair_force(const Row4& b, const Row4& m, const Row4& t,
                                           const ERow& eb, const ERow& et,
                                           const StencilCoef<float>& c, float& ax0, float& ay0,
                                           float& ax1, float& ay1) {
  RowV<float> b0{b.L, b.A, b.B}, m0{m.L, m.A, m.B}, t0{t.L, t.A, t.B};
  RowV<float> b1{b.A, b.B, b.R}, m1{m.A, m.B, m.R}, t1{t.A, t.B, t.R};
  node_force<float>(b0, m0, t0, eb.l, eb.a, et.l, et.a, c, ax0, ay0);
  node_force<float>(b1, m1, t1, eb.a, eb.b, et.a, et.b, c, ax1, ay1);
}

template <bool MASK_IN, bool FAST>
__device__ __forceinline__ void matvec2_strip(const float* __restrict__ u, float* __restrict__ y,
                                              const float* __restrict__ E,
                                              const uint8_t* __restrict__ nmask, int nelx,
                                              int nely, const StencilCoef<float>& c, int i0,
                                              int j0, int lane) {
  const int nx1 = nelx + 1, ny1 = nely + 1;
  Pend2 p0, p1, p2;
  issue2<MASK_IN, FAST>(p0, u, E, nmask, i0, lane, j0 - 1, nelx, nely);
  issue2<MASK_IN, FAST>(p1, u, E, nmask, i0, lane, j0, nelx, nely);
  Row4 w0, w1, w2;
  ERow e0, e1, e2, dummy;
  make_row2(p0, lane, w0, dummy);
  make_row2(p1, lane, w1, e0);     // e0 = element row j0-1
  const int jend = min(j0 + MV_TY, ny1);
  issue2<MASK_IN, FAST>(p0, u, E, nmask, i0, lane, j0 + 1, nelx, nely);
  issue2<MASK_IN, FAST>(p1, u, E, nmask, i0, lane, j0 + 2, nelx, nely);
  issue2<MASK_IN, FAST>(p2, u, E, nmask, i0, lane, j0 + 3, nelx, nely);
  auto emit = [&](int j, uint8_t fa, uint8_t fb, float x0, float y0, float x1, float y1) {
    if (j < jend) {
      float2* yr = reinterpret_cast<float2*>(y) + (long long)j * nx1;
      if (i0 < nx1) yr[i0] = make_float2((fa & 1) ? 0.f : x0, (fa & 2) ? 0.f : y0);
      if (i0 + 1 < nx1) yr[i0 + 1] = make_float2((fb & 1) ? 0.f : x1, (fb & 2) ? 0.f : y1);
    }
  };
  for (int jb = j0; jb < jend; jb += 3) {
    float x0, y0, x1, y1;
    make_row2(p0, lane, w2, e1);
    uint8_t fa = p0.ma, fb = p0.mb;
    if (jb + 4 <= jend + 1) issue2<MASK_IN, FAST>(p0, u, E, nmask, i0, lane, jb + 4, nelx, nely);
    pair_force(w0, w1, w2, e0, e1, c, x0, y0, x1, y1);
    emit(jb, fa, fb, x0, y0, x1, y1);
    make_row2(p1, lane, w0, e2);
    fa = p1.ma; fb = p1.mb;
    if (jb + 5 <= jend + 1) issue2<MASK_IN, FAST>(p1, u, E, nmask, i0, lane, jb + 5, nelx, nely);
    pair_force(w1, w2, w0, e1, e2, c, x0, y0, x1, y1);
    emit(jb + 1, fa, fb, x0, y0, x1, y1);
    make_row2(p2, lane, w1, e0);
    fa = p2.ma; fb = p2.mb;
    if (jb + 6 <= jend + 1) issue2<MASK_IN, FAST>(p2, u, E, nmask, i0, lane, jb + 6, nelx, nely);
    pair_force(w2, w0, w1, e2, e0, c, x0, y0, x1, y1);
    emit(jb + 2, fa, fb, x0, y0, x1, y1);
  }
}

template <bool MASK_IN>
__global__ void __launch_bounds__(MV_TX) k_matvec2(const float* __restrict__ u,
                                                   float* __restrict__ y,
                                                   const float* __restrict__ E,
                                                   const uint8_t* __restrict__ nmask, int nelx,
                                                   int nely, StencilCoef<float> c,
                                                   long long vec_stride, long long e_stride) {
  const int lane = threadIdx.x & 31;
  const int c0 = blockIdx.x * MV_TX * 2;           // first node column of the block
  const int i0 = c0 + 2 * threadIdx.x;
  const int j0 = blockIdx.y * MV_TY;
  u += blockIdx.z * vec_stride;
  y += blockIdx.z * vec_stride;
  E += blockIdx.z * e_stride;
  // interior: node columns c0-1 .. c0+2*MV_TX, rows j0-1 .. j0+MV_TY+1, element columns
  // c0-1 .. c0+2*MV_TX-1 and rows j0-2 .. j0+MV_TY all inside the mesh
  const bool fast = c0 >= 1 && c0 + 2 * MV_TX < nelx && j0 >= 2 && j0 + MV_TY + 1 <= nely;
  if (fast)
    matvec2_strip<MASK_IN, true>(u, y, E, nmask, nelx, nely, c, i0, j0, lane);
  else
    matvec2_strip<MASK_IN, false>(u, y, E, nmask, nelx, nely, c, i0, j0, lane);
}

cudaError_t launch_matvec_f32(const float* u, float* y, const float* E, const uint8_t* nmask,
                              int nelx, int nely, const StencilCoef<float>& c, int nsys,
                              long long vec_stride, long long e_stride, cudaStream_t s,
                              bool mask_input) {
  dim3 grid(cdiv(nelx + 1, 2 * MV_TX), cdiv(nely + 1, MV_TY), nsys);
  if (mask_input)
    note_launch(), k_matvec2<true><<<grid, MV_TX, 0, s>>>(u, y, E, nmask, nelx, nely, c, vec_stride, e_stride);
  else
    note_launch(), k_matvec2<false><<<grid, MV_TX, 0, s>>>(u, y, E, nmask, nelx, nely, c, vec_stride, e_stride);
  return cudaGetLastError();
}

cudaError_t launch_matvec_f64(const double* u, double* y, const double* E, const uint8_t* nmask,
                              int nelx, int nely, const StencilCoef<double>& c, int nsys,
                              long long vec_stride, long long e_stride, cudaStream_t s,
                              bool mask_input) {
  dim3 grid(cdiv(nelx + 1, MV_TX), cdiv(nely + 1, MV_TY), nsys);
  if (mask_input)
    note_launch(), k_matvec<double, true><<<grid, MV_TX, 0, s>>>(u, y, E, nmask, nelx, nely, c, vec_stride, e_stride);
  else
    note_launch(), k_matvec<double, false><<<grid, MV_TX, 0, s>>>(u, y, E, nmask, nelx, nely, c, vec_stride, e_stride);
  return cudaGetLastError();
}
