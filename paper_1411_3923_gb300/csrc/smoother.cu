// The paper's own two-level preconditioner (Sec. 2.4.2): one symmetric Gauss-Seidel sweep,
// the spectral coarse correction, a second symmetric sweep, applied multiplicatively:
//   z = SGS(0; r);   z += R_c^T K_c^-1 R_c (r - K z);   z = SGS(z; r)
// SGS(z; r) is a forward sweep (node colours 0, 1, 2, 3) followed by a backward sweep
// (3, 2, 1, 0).  Colour = (i mod 2) + 2 (j mod 2): two nodes of one colour share no Q4
// element, so every node of a colour is updated at once, each solving its own 2x2 block
// (1x1 when one DOF is fixed) against the current values of its neighbours:
//   z_n <- z_n + K_nn^-1 (r_n - (K z)_n)
// With the same symmetric sweep before and after the coarse correction the operator is
// symmetric positive definite, so the flexible CG applies it unchanged.
#include <algorithm>

#include "internal.cuh"

namespace {

template <typename T>
struct K0Arg { T k[64]; };   // unit element stiffness, local DOF 2a + d (a: (0,0) (1,0) (1,1) (0,1))

constexpr int GS_TX = 128;

// local index of the element corner (ox, oy) in {0,1}^2
__device__ __forceinline__ int corner(int ox, int oy) { return oy ? (ox ? 2 : 3) : (ox ? 1 : 0); }

// One colour pass on nsys systems: block z (x), r, E advance by blockIdx.z strides.
template <typename T>
__global__ void __launch_bounds__(GS_TX) k_gs_colour(T* __restrict__ z, const T* __restrict__ r,
                                                    const T* __restrict__ E,
                                                    const uint8_t* __restrict__ nmask, int nelx,
                                                    int nely, int colour, K0Arg<T> K0,
                                                    long long vec_stride, long long e_stride) {
  const int i = 2 * (blockIdx.x * GS_TX + threadIdx.x) + (colour & 1);
  const int j = 2 * blockIdx.y + (colour >> 1);
  if (i > nelx || j > nely) return;
  z += blockIdx.z * vec_stride;
  r += blockIdx.z * vec_stride;
  E += blockIdx.z * e_stride;
  const int nx1 = nelx + 1;
  const long long n = (long long)j * nx1 + i;
  const uint8_t m = nmask[n];
  if ((m & 3) == 3) return;
  T kx = T(0), ky = T(0), bxx = T(0), bxy = T(0), byy = T(0);
  for (int dy = -1; dy <= 0; ++dy) {
    const int ey = j + dy;
    if (ey < 0 || ey >= nely) continue;
    for (int dx = -1; dx <= 0; ++dx) {
      const int ex = i + dx;
      if (ex < 0 || ex >= nelx) continue;
      const T Ee = E[(long long)ey * nelx + ex];
      const int a = corner(-dx, -dy);
      const T* ka = K0.k + 2 * a * 8;   // rows 2a (x) and 2a + 1 (y)
      T sx = T(0), sy = T(0);
#pragma unroll
      for (int oy = 0; oy < 2; ++oy)
#pragma unroll
        for (int ox = 0; ox < 2; ++ox) {
          const int b = corner(ox, oy);
          const long long nb = (long long)(ey + oy) * nx1 + (ex + ox);
          const T ux = z[2 * nb], uy = z[2 * nb + 1];
          sx += ka[2 * b] * ux + ka[2 * b + 1] * uy;
          sy += ka[8 + 2 * b] * ux + ka[8 + 2 * b + 1] * uy;
        }
      kx += Ee * sx;
      ky += Ee * sy;
      bxx += Ee * ka[2 * a];
      bxy += Ee * ka[2 * a + 1];
      byy += Ee * ka[8 + 2 * a + 1];
    }
  }
  const T rx = r[2 * n] - kx, ry = r[2 * n + 1] - ky;
  T dxv, dyv;
  if (m & 1) {            // x fixed: the y DOF alone
    dxv = T(0);
    dyv = ry / byy;
  } else if (m & 2) {     // y fixed
    dxv = rx / bxx;
    dyv = T(0);
  } else {
    const T det = bxx * byy - bxy * bxy;
    dxv = (byy * rx - bxy * ry) / det;
    dyv = (bxx * ry - bxy * rx) / det;
  }
  z[2 * n] += dxv;
  z[2 * n + 1] += dyv;
}

// res = r - y on free DOFs, 0 on fixed ones (nsys systems back to back)
template <typename T>
__global__ void k_sgs_residual(T* res, const T* __restrict__ r, const T* y,   // res may be y
                               const uint8_t* __restrict__ nmask, long long n_dof, long long total) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long d = q % n_dof;
    const bool fixed = (nmask[d >> 1] >> (d & 1)) & 1;
    res[q] = fixed ? T(0) : r[q] - y[q];
  }
}

template <typename T>
__global__ void k_sgs_add(T* __restrict__ z, const T* __restrict__ w, long long total) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x)
    z[q] += w[q];
}

}  // namespace

// ------------------------------------------------------------------------------ host side
template <typename T> static const T* moduli(mstopo_handle* h);
template <> const double* moduli<double>(mstopo_handle* h) { return h->d_E64; }
template <> const float* moduli<float>(mstopo_handle* h) { return h->d_E32; }

static cudaError_t matvec_t(mstopo_handle* h, const double* u, double* y, const double* E, int nsys) {
  return launch_matvec_f64(u, y, E, h->d_nmask, h->nelx, h->nely, h->st64, nsys, h->n_dof,
                           h->n_el, h->s, true);
}
static cudaError_t matvec_t(mstopo_handle* h, const float* u, float* y, const float* E, int nsys) {
  return launch_matvec_f32(u, y, E, h->d_nmask, h->nelx, h->nely, h->st32, nsys, h->n_dof,
                           h->n_el, h->s, true);
}
static cudaError_t coarse_t(mstopo_handle* h, const double* r, double* z, int sys0, int nsys) {
  return precond_apply_f64(h, r, z, sys0, nsys, 1);
}
static cudaError_t coarse_t(mstopo_handle* h, const float* r, float* z, int sys0, int nsys) {
  return precond_apply_f32(h, r, z, sys0, nsys, 1);
}

// SGS(z; r): colours 0, 1, 2, 3 then 3, 2, 1, 0
template <typename T>
static cudaError_t sgs_sweep(mstopo_handle* h, T* z, const T* r, const T* E, int nsys,
                             const K0Arg<T>& k0) {
  const dim3 grid((unsigned)cdiv((h->nelx + 2) / 2, GS_TX), (unsigned)((h->nely + 2) / 2), (unsigned)nsys);
  static const int order[8] = {0, 1, 2, 3, 3, 2, 1, 0};
  for (int q = 0; q < 8; ++q)
    note_launch(), k_gs_colour<T><<<grid, GS_TX, 0, h->s>>>(z, r, E, h->d_nmask, h->nelx, h->nely,
                                                            order[q], k0, h->n_dof, h->n_el);
  return cudaGetLastError();
}

// part 0: the multiplicative operator; part 2: one symmetric sweep from zero (the smoother
// alone).  r and z hold nsys systems from realisation sys0 on, n_dof apart.
template <typename T>
static cudaError_t sgs_apply(mstopo_handle* h, const T* r, T* z, int sys0, int nsys, int part) {
  Precond& pc = h->pc;
  const long long n = h->n_dof, total = n * nsys;
  const T* E = moduli<T>(h) + (long long)sys0 * h->n_el;
  K0Arg<T> k0;
  for (int q = 0; q < 64; ++q) k0.k[q] = (T)h->K0[q];
  cudaError_t e = cudaMemsetAsync(z, 0, (size_t)total * sizeof(T), h->s);
  if (e == cudaSuccess) e = sgs_sweep<T>(h, z, r, E, nsys, k0);
  if (e != cudaSuccess || part == 2) return e;
  T* y = reinterpret_cast<T*>(pc.d_sgs);           // [MSTOPO_MAX_SYS][n]: K z, then r - K z
  T* w = y + (size_t)MSTOPO_MAX_SYS * n;           // coarse correction
  const int blocks = (int)std::min<long long>(cdiv(total, 256), 4LL * 1024);
  e = matvec_t(h, z, y, E, nsys);
  if (e != cudaSuccess) return e;
  note_launch(), k_sgs_residual<T><<<blocks, 256, 0, h->s>>>(y, r, y, h->d_nmask, n, total);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = coarse_t(h, y, w, sys0, nsys);
  if (e != cudaSuccess) return e;
  note_launch(), k_sgs_add<T><<<blocks, 256, 0, h->s>>>(z, w, total);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = sgs_sweep<T>(h, z, r, E, nsys, k0);
  return e;
}

cudaError_t sgs_apply_f64(mstopo_handle* h, const double* r, double* z, int sys0, int nsys, int part) {
  return sgs_apply<double>(h, r, z, sys0, nsys, part);
}
cudaError_t sgs_apply_f32(mstopo_handle* h, const float* r, float* z, int sys0, int nsys, int part) {
  return sgs_apply<float>(h, r, z, sys0, nsys, part);
}
