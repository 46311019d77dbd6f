// Design chain and its adjoint (paper Sec. 4.1-4.4, Sec. 2.2).
//
//  filter      rho~_e = sum_j w_ej rho_j / W_e, w_ej = max(0, rmin - |x_e - x_j|), W_e = sum_j w_ej
//              over the neighbours inside the design domain (or wrapping around the periodic
//              unit cell, which equals filtering a 3x3 block of cells, Sec. 4.3)
//  projection  rho_bar = (tanh(beta eta) + tanh(beta (rho~ - eta))) / (tanh(beta eta) + tanh(beta (1 - eta)))
//  SIMP        E = Emin + (E0 - Emin) rho_bar^p on the fine mesh (periodic designs are tiled)
//  adjoint     dc_k/drho_bar_e = -p (E0 - Emin) rho_bar^(p-1) u_e^T K0 u_e (Sec. 4.2), times
//              the robust weight w_k and drho_bar/drho~, summed over the copies of a periodic
//              cell (Sec. 4.1), then the transpose of the normalised filter.
// All FP64: these passes are a few percent of a design iteration.
#include "internal.cuh"

__device__ __forceinline__ int wrap(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

__global__ void k_filter(const double* __restrict__ rho, double* __restrict__ rt,
                         double* __restrict__ wsum, int dx, int dy, double rmin, int R,
                         int periodic) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y;
  if (x >= dx) return;
  double s = 0.0, ws = 0.0;
  for (int oy = -R; oy <= R; ++oy)
    for (int ox = -R; ox <= R; ++ox) {
      double w = rmin - sqrt((double)(ox * ox + oy * oy));
      if (w <= 0.0) continue;
      int jx = x + ox, jy = y + oy;
      if (periodic) {
        jx = wrap(jx, dx);
        jy = wrap(jy, dy);
      } else if (jx < 0 || jx >= dx || jy < 0 || jy >= dy) {
        continue;
      }
      s = fma(w, rho[(long long)jy * dx + jx], s);
      ws += w;
    }
  long long e = (long long)y * dx + x;
  rt[e] = s / ws;
  wsum[e] = ws;
}

// out_j = sum_e w_ej g_e / W_e (transpose of the normalised filter; w is symmetric)
__global__ void k_filter_T(const double* __restrict__ g, const double* __restrict__ wsum,
                           double* __restrict__ out, int dx, int dy, double rmin, int R,
                           int periodic) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y;
  if (x >= dx) return;
  double s = 0.0;
  for (int oy = -R; oy <= R; ++oy)
    for (int ox = -R; ox <= R; ++ox) {
      double w = rmin - sqrt((double)(ox * ox + oy * oy));
      if (w <= 0.0) continue;
      int ex = x + ox, ey = y + oy;
      if (periodic) {
        ex = wrap(ex, dx);
        ey = wrap(ey, dy);
      } else if (ex < 0 || ex >= dx || ey < 0 || ey >= dy) {
        continue;
      }
      long long e = (long long)ey * dx + ex;
      s = fma(w, g[e] / wsum[e], s);
    }
  out[(long long)y * dx + x] = s;
}

struct Etas { double eta[MSTOPO_MAX_SYS]; };

__global__ void k_project(const double* __restrict__ rt, double* __restrict__ rbar,
                          double* __restrict__ drbar, int n, Etas et, int n_eta, double beta) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double x = rt[e];
  for (int k = 0; k < n_eta; ++k) {
    double eta = et.eta[k];
    double a = tanh(beta * eta);
    double den = a + tanh(beta * (1.0 - eta));
    double t = tanh(beta * (x - eta));
    rbar[(long long)k * n + e] = (a + t) / den;
    drbar[(long long)k * n + e] = beta * (1.0 - t * t) / den;
  }
}

__global__ void k_simp(const double* __restrict__ rbar, double* __restrict__ E64,
                       float* __restrict__ E32, int nelx, int nely, int dx, int dy,
                       int periodic, int n_design, double E0, double Emin, double penal) {
  int ex = blockIdx.x * blockDim.x + threadIdx.x;
  int ey = blockIdx.y;
  int k = blockIdx.z;
  if (ex >= nelx) return;
  long long d = periodic ? (long long)(ey % dy) * dx + (ex % dx) : (long long)ey * nelx + ex;
  double rb = rbar[(long long)k * n_design + d];
  double E = Emin + (E0 - Emin) * pow(rb, penal);
  long long e = (long long)k * nelx * nely + (long long)ey * nelx + ex;
  E64[e] = E;
  E32[e] = (float)E;
}

struct K0Mat { double k[64]; };
struct Weights { double w[MSTOPO_MAX_SYS]; };

__global__ void k_sensitivity(const double* __restrict__ u, long long u_stride,
                              const double* __restrict__ rbar, const double* __restrict__ drbar,
                              int n_eta, Weights wk, int nelx, int nely, int dx, int dy,
                              int periodic, int n_design, double dE, double penal, K0Mat K0,
                              double* __restrict__ g_fine) {
  int ex = blockIdx.x * blockDim.x + threadIdx.x;
  int ey = blockIdx.y;
  if (ex >= nelx) return;
  const int nx1 = nelx + 1;
  long long d = periodic ? (long long)(ey % dy) * dx + (ex % dx) : (long long)ey * nelx + ex;
  // local nodes (ex,ey), (ex+1,ey), (ex+1,ey+1), (ex,ey+1)
  long long n0 = (long long)ey * nx1 + ex, n3 = n0 + nx1;
  double g = 0.0;
  for (int k = 0; k < n_eta; ++k) {
    const double2* uk = reinterpret_cast<const double2*>(u + k * u_stride);
    double2 a = uk[n0], b = uk[n0 + 1], c = uk[n3 + 1], dd = uk[n3];
    double ue[8] = {a.x, a.y, b.x, b.y, c.x, c.y, dd.x, dd.y};
    double en = 0.0;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) t = fma(K0.k[r * 8 + q], ue[q], t);
      en = fma(ue[r], t, en);
    }
    double rb = rbar[(long long)k * n_design + d];
    double dc = -penal * dE * pow(rb, penal - 1.0) * en;
    g = fma(wk.w[k] * dc, drbar[(long long)k * n_design + d], g);
  }
  g_fine[(long long)ey * nelx + ex] = g;
}

// sum of the fine-mesh field over all copies of the unit cell, fixed order
__global__ void k_tile_sum(const double* __restrict__ gf, double* __restrict__ gd, int nelx,
                           int nely, int dx, int dy) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y;
  if (x >= dx) return;
  double s = 0.0;
  for (int ty = 0; ty < nely / dy; ++ty)
    for (int tx = 0; tx < nelx / dx; ++tx)
      s += gf[(long long)(ty * dy + y) * nelx + tx * dx + x];
  gd[(long long)y * dx + x] = s;
}

__global__ void k_check_finite(const double* __restrict__ x, long long n, int* flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicOr(flag, 1);
}

cudaError_t launch_filter(const double* rho, double* rho_tilde, double* wsum, int dx, int dy,
                          double rmin, int periodic, cudaStream_t s) {
  int R = (int)ceil(rmin);
  note_launch(), k_filter<<<dim3(cdiv(dx, 128), dy), 128, 0, s>>>(rho, rho_tilde, wsum, dx, dy, rmin, R, periodic);
  return cudaGetLastError();
}

cudaError_t launch_filter_T(const double* g, const double* wsum, double* out, int dx, int dy,
                            double rmin, int periodic, cudaStream_t s) {
  int R = (int)ceil(rmin);
  note_launch(), k_filter_T<<<dim3(cdiv(dx, 128), dy), 128, 0, s>>>(g, wsum, out, dx, dy, rmin, R, periodic);
  return cudaGetLastError();
}

cudaError_t launch_project(const double* rho_tilde, double* rbar, double* drbar, int n,
                           const double* etas, int n_eta, double beta, cudaStream_t s) {
  Etas et;
  for (int k = 0; k < MSTOPO_MAX_SYS; ++k) et.eta[k] = k < n_eta ? etas[k] : 0.0;
  note_launch(), k_project<<<cdiv(n, 256), 256, 0, s>>>(rho_tilde, rbar, drbar, n, et, n_eta, beta);
  return cudaGetLastError();
}

cudaError_t launch_simp(const double* rbar, double* E64, float* E32, int nelx, int nely,
                        int dx, int dy, int periodic, int n_eta, int n_design,
                        double E0, double Emin, double penal, cudaStream_t s) {
  note_launch(), k_simp<<<dim3(cdiv(nelx, 128), nely, n_eta), 128, 0, s>>>(rbar, E64, E32, nelx, nely, dx, dy,
                                                             periodic, n_design, E0, Emin, penal);
  return cudaGetLastError();
}

cudaError_t launch_sensitivity(const double* u, long long u_stride, const double* rbar,
                               const double* drbar, int n_eta, const double* w, int nelx,
                               int nely, int dx, int dy, int periodic, int n_design,
                               double dE, double penal, const double* K0, double* g_fine,
                               cudaStream_t s) {
  Weights wk;
  for (int k = 0; k < MSTOPO_MAX_SYS; ++k) wk.w[k] = k < n_eta ? w[k] : 0.0;
  K0Mat km;
  for (int q = 0; q < 64; ++q) km.k[q] = K0[q];
  note_launch(), k_sensitivity<<<dim3(cdiv(nelx, 128), nely), 128, 0, s>>>(u, u_stride, rbar, drbar, n_eta, wk,
                                                            nelx, nely, dx, dy, periodic,
                                                            n_design, dE, penal, km, g_fine);
  return cudaGetLastError();
}

cudaError_t launch_tile_sum(const double* g_fine, double* g_design, int nelx, int nely,
                            int dx, int dy, cudaStream_t s) {
  note_launch(), k_tile_sum<<<dim3(cdiv(dx, 128), dy), 128, 0, s>>>(g_fine, g_design, nelx, nely, dx, dy);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* x, long long n, int* flag, cudaStream_t s) {
  note_launch(), k_check_finite<<<304, 256, 0, s>>>(x, n, flag);
  return cudaGetLastError();
}
