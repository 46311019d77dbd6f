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
#define MV_TY 16

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
__device__ __forceinline__ typename Vec2<T>::type load_node(const T* __restrict__ u,
                                                            const uint8_t* __restrict__ m,
                                                            int i, int j, int nx1, int ny1) {
  typedef typename Vec2<T>::type V;
  V v;
  v.x = T(0); v.y = T(0);
  if (i >= 0 && i < nx1 && j >= 0 && j < ny1) {
    long long n = (long long)j * nx1 + i;
    v = reinterpret_cast<const V*>(u)[n];
    uint8_t f = m[n];
    if (f & 1) v.x = T(0);
    if (f & 2) v.y = T(0);
  }
  return v;
}

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

// Rows are processed in chunks of MV_U: the loads of the next MV_U node rows and element rows
// are all issued before any of them is used, so each thread keeps MV_U rows of loads in
// flight.  A warp covers 32 consecutive node columns; the left/right neighbours come from
// the adjacent lanes by shuffles (edge lanes load their own).
#define MV_U 4
template <typename T>
__global__ void __launch_bounds__(MV_TX) k_matvec(const T* __restrict__ u, T* __restrict__ y,
                                                  const T* __restrict__ E,
                                                  const uint8_t* __restrict__ nmask, int nelx,
                                                  int nely, StencilCoef<T> c,
                                                  long long vec_stride, long long e_stride) {
  typedef typename Vec2<T>::type V;
  const int nx1 = nelx + 1, ny1 = nely + 1;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * MV_TX + threadIdx.x;
  const int j0 = blockIdx.y * MV_TY;
  const bool in = i < nx1;
  u += blockIdx.z * vec_stride;
  y += blockIdx.z * vec_stride;
  E += blockIdx.z * e_stride;
  // window rows: 0 -> j-1, 1 -> j, 2 -> j+1 ; columns: left (i-1), centre (i), right (i+1)
  V wl[3], wc[3], wr[3];
  T el[2], ec[2];   // moduli of elements (i-1, row) and (i, row) for rows j-1 (0) and j (1)
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int jj = j0 - 1 + r;
    V cv = load_node(u, nmask, i, jj, nx1, ny1);
    V lv = shfl_up2<T>(cv), rv = shfl_down2<T>(cv);
    if (lane == 0) lv = load_node(u, nmask, i - 1, jj, nx1, ny1);
    if (lane == 31) rv = load_node(u, nmask, i + 1, jj, nx1, ny1);
    wl[r] = lv; wc[r] = cv; wr[r] = rv;
  }
  {
    T ce = load_E(E, i, j0 - 1, nelx, nely);
    T le = __shfl_up_sync(0xffffffffu, ce, 1);
    if (lane == 0) le = load_E(E, i - 1, j0 - 1, nelx, nely);
    el[1] = le; ec[1] = ce;
  }
  const int jend = min(j0 + MV_TY, ny1);
  for (int jb = j0; jb < jend; jb += MV_U) {
    V pc[MV_U], pe2[MV_U];
    T pe[MV_U], ple[MV_U];
    uint8_t pm[MV_U];
#pragma unroll
    for (int r = 0; r < MV_U; ++r) {
      const int jn = jb + 1 + r;
      pc[r] = load_node(u, nmask, i, jn, nx1, ny1);
      pe2[r] = load_node(u, nmask, lane == 0 ? i - 1 : i + 1, jn, nx1, ny1);
      pe[r] = load_E(E, i, jb + r, nelx, nely);
      ple[r] = load_E(E, i - 1, jb + r, nelx, nely);
      pm[r] = (in && jb + r < ny1) ? nmask[(long long)(jb + r) * nx1 + i] : (uint8_t)3;
    }
#pragma unroll
    for (int r = 0; r < MV_U; ++r) {
      const int j = jb + r;
      {
        V cv = pc[r];
        V lv = shfl_up2<T>(cv), rv = shfl_down2<T>(cv);
        if (lane == 0) lv = pe2[r];
        if (lane == 31) rv = pe2[r];
        wl[2] = lv; wc[2] = cv; wr[2] = rv;
        T ce = pe[r];
        T le = __shfl_up_sync(0xffffffffu, ce, 1);
        if (lane == 0) le = ple[r];
        el[0] = el[1]; ec[0] = ec[1];
        el[1] = le; ec[1] = ce;
      }
      const T cx = wc[1].x, cy = wc[1].y;
      // neighbour differences u(i-1+q, j-1+r) - u(i, j)
      T dxv[3][3], dyv[3][3];
#pragma unroll
      for (int rr = 0; rr < 3; ++rr) {
        dxv[rr][0] = wl[rr].x - cx; dyv[rr][0] = wl[rr].y - cy;
        dxv[rr][1] = wc[rr].x - cx; dyv[rr][1] = wc[rr].y - cy;
        dxv[rr][2] = wr[rr].x - cx; dyv[rr][2] = wr[rr].y - cy;
      }
      T yx = T(0), yy = T(0);
      {  // LL element (i-1, j-1): others (i-1,j-1), (i,j-1), (i-1,j)
        T ax = T(0), ay = T(0);
        blk(ax, ay, c.c[0][0], dxv[0][0], dyv[0][0]);
        blk(ax, ay, c.c[0][1], dxv[0][1], dyv[0][1]);
        blk(ax, ay, c.c[0][2], dxv[1][0], dyv[1][0]);
        yx = fma(el[0], ax, yx); yy = fma(el[0], ay, yy);
      }
      {  // LR element (i, j-1): others (i,j-1), (i+1,j-1), (i+1,j)
        T ax = T(0), ay = T(0);
        blk(ax, ay, c.c[1][0], dxv[0][1], dyv[0][1]);
        blk(ax, ay, c.c[1][1], dxv[0][2], dyv[0][2]);
        blk(ax, ay, c.c[1][2], dxv[1][2], dyv[1][2]);
        yx = fma(ec[0], ax, yx); yy = fma(ec[0], ay, yy);
      }
      {  // UL element (i-1, j): others (i-1,j), (i,j+1), (i-1,j+1)
        T ax = T(0), ay = T(0);
        blk(ax, ay, c.c[2][0], dxv[1][0], dyv[1][0]);
        blk(ax, ay, c.c[2][1], dxv[2][1], dyv[2][1]);
        blk(ax, ay, c.c[2][2], dxv[2][0], dyv[2][0]);
        yx = fma(el[1], ax, yx); yy = fma(el[1], ay, yy);
      }
      {  // UR element (i, j): others (i+1,j), (i+1,j+1), (i,j+1)
        T ax = T(0), ay = T(0);
        blk(ax, ay, c.c[3][0], dxv[1][2], dyv[1][2]);
        blk(ax, ay, c.c[3][1], dxv[2][2], dyv[2][2]);
        blk(ax, ay, c.c[3][2], dxv[2][1], dyv[2][1]);
        yx = fma(ec[1], ax, yx); yy = fma(ec[1], ay, yy);
      }
      if (in && j < jend) {
        const uint8_t f = pm[r];
        V out;
        out.x = (f & 1) ? T(0) : yx;
        out.y = (f & 2) ? T(0) : yy;
        reinterpret_cast<V*>(y)[(long long)j * nx1 + i] = out;
      }
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) { wl[rr] = wl[rr + 1]; wc[rr] = wc[rr + 1]; wr[rr] = wr[rr + 1]; }
    }
  }
}

cudaError_t launch_matvec_f32(const float* u, float* y, const float* E, const uint8_t* nmask,
                              int nelx, int nely, const StencilCoef<float>& c, int nsys,
                              long long vec_stride, long long e_stride, cudaStream_t s) {
  dim3 grid(cdiv(nelx + 1, MV_TX), cdiv(nely + 1, MV_TY), nsys);
  note_launch(), k_matvec<float><<<grid, MV_TX, 0, s>>>(u, y, E, nmask, nelx, nely, c, vec_stride, e_stride);
  return cudaGetLastError();
}

cudaError_t launch_matvec_f64(const double* u, double* y, const double* E, const uint8_t* nmask,
                              int nelx, int nely, const StencilCoef<double>& c, int nsys,
                              long long vec_stride, long long e_stride, cudaStream_t s) {
  dim3 grid(cdiv(nelx + 1, MV_TX), cdiv(nely + 1, MV_TY), nsys);
  note_launch(), k_matvec<double><<<grid, MV_TX, 0, s>>>(u, y, E, nmask, nelx, nely, c, vec_stride, e_stride);
  return cudaGetLastError();
}
