// PDE (Helmholtz) density filter with periodicity and connectivity imposed by collapsed
// degrees of freedom (Sec. 4.3 and 4.5: the filter used for designs of several microstructure
// blocks).  On the filter mesh (the design elements, unit Q4 elements, cells of nx x ny_c
// elements stacked along y, each with its own nodes):
//   K_F = sum_e (r^2 K_e^lap + M_e),  r = r_min / (2 sqrt(3)),  b = T_F rho (rho_e / 4 to each
//   node of e),  rho_tilde = T_F^T P (P^T K_F P)^-1 P^T T_F rho,
// with P the collapse map (identified nodes share one unknown).  The operator is symmetric, so
// the sensitivity chain applies it unchanged.  The collapsed system P^T K_F P is solved by
// Jacobi-preconditioned CG in FP64, matrix-free: one thread per collapsed unknown sums, over
// its member nodes in ascending order, each node's 9-point element stencil (a fixed order:
// results are bitwise repeatable).  The collapse map comes from a union-find of the
// identified node pairs on the host (integer bookkeeping), as index tables on the device.
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "internal.cuh"

#define PB MSTOPO_RED_BLOCKS
#define PT 256

// Q4 Laplacian stiffness and consistent mass of the unit square, local nodes (0,0), (1,0),
// (1,1), (0,1): the integrals of grad N_a . grad N_b and N_a N_b in closed form
__constant__ double c_pde_kl[16] = {4.0 / 6, -1.0 / 6, -2.0 / 6, -1.0 / 6,  -1.0 / 6, 4.0 / 6, -1.0 / 6, -2.0 / 6,
                                    -2.0 / 6, -1.0 / 6, 4.0 / 6, -1.0 / 6,  -1.0 / 6, -2.0 / 6, -1.0 / 6, 4.0 / 6};
__constant__ double c_pde_me[16] = {4.0 / 36, 2.0 / 36, 1.0 / 36, 2.0 / 36,  2.0 / 36, 4.0 / 36, 2.0 / 36, 1.0 / 36,
                                    1.0 / 36, 2.0 / 36, 4.0 / 36, 2.0 / 36,  2.0 / 36, 1.0 / 36, 2.0 / 36, 4.0 / 36};

struct PdeGeom {
  int nx;                          // elements along x of every cell
  long long n_nodes, n_el;
  int ncol;                        // collapsed unknowns
  double r2;                       // r^2
  const int* ny;                   // [cells]
  const long long* node_off;       // [cells]
  const long long* el_off;         // [cells]
  const int* node_cell;            // [n_nodes]
  const int* col;                  // [n_nodes] collapsed unknown of each node
  const int* mem_off;              // [ncol + 1] members of each unknown (ascending node ids)
  const int* mem;                  // [n_nodes]
};

struct mstopo_pde_filter {
  std::string err;
  cudaStream_t s = nullptr;
  PdeGeom g{};
  double tol = 1e-12;
  int max_iter = 1000;
  int n_cells = 0;
  int *d_ny = nullptr, *d_node_cell = nullptr, *d_col = nullptr, *d_mem_off = nullptr, *d_mem = nullptr;
  long long *d_node_off = nullptr, *d_el_off = nullptr;
  double *d_diag = nullptr, *d_x = nullptr, *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_q = nullptr;
  double *d_partials = nullptr, *d_scal = nullptr, *h_scal = nullptr;
};

namespace {

__device__ __forceinline__ double pde_block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// node n -> (cell, i, j)
__device__ __forceinline__ void pde_node(const PdeGeom& g, long long n, int& c, int& i, int& j) {
  c = g.node_cell[n];
  const long long loc = n - g.node_off[c];
  j = (int)(loc / (g.nx + 1));
  i = (int)(loc % (g.nx + 1));
}

// The contribution of node n's row of K_F (element stencils in the order (i-1,j-1), (i,j-1),
// (i-1,j), (i,j)) applied to the collapsed vector x; with diag_of >= 0, only the entries whose
// column node collapses to diag_of (the diagonal of P^T K_F P).
__device__ double pde_row(const PdeGeom& g, long long n, const double* __restrict__ x, int diag_of) {
  int c, i, j;
  pde_node(g, n, c, i, j);
  const int ny = g.ny[c];
  const long long o = g.node_off[c];
  double y = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int ex = i - 1 + (q & 1), ey = j - 1 + (q >> 1);
    if (ex < 0 || ex >= g.nx || ey < 0 || ey >= ny) continue;
    const int li = i - ex, lj = j - ey;
    const int a = lj == 0 ? (li == 0 ? 0 : 1) : (li == 1 ? 2 : 3);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int bi = ex + ((b == 1 || b == 2) ? 1 : 0), bj = ey + (b >= 2 ? 1 : 0);
      const long long m = o + (long long)bj * (g.nx + 1) + bi;
      const double k = g.r2 * c_pde_kl[a * 4 + b] + c_pde_me[a * 4 + b];
      const int cm = g.col[m];
      if (diag_of >= 0) {
        if (cm == diag_of) y += k;
      } else {
        y = fma(k, x[cm], y);
      }
    }
  }
  return y;
}

// y = P^T K_F P x (or, with x null, the diagonal of P^T K_F P)
__global__ void k_pde_apply(PdeGeom g, const double* __restrict__ x, double* __restrict__ y) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncol; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = g.mem_off[c]; t < g.mem_off[c + 1]; ++t) s += pde_row(g, g.mem[t], x, x ? -1 : c);
    y[c] = s;
  }
}

// b = P^T T_F rho: every node gathers rho_e / 4 of its elements
__global__ void k_pde_rhs(PdeGeom g, const double* __restrict__ rho, double* __restrict__ b) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncol; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = g.mem_off[c]; t < g.mem_off[c + 1]; ++t) {
      int cc, i, j;
      pde_node(g, g.mem[t], cc, i, j);
      const int ny = g.ny[cc];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int ex = i - 1 + (q & 1), ey = j - 1 + (q >> 1);
        if (ex < 0 || ex >= g.nx || ey < 0 || ey >= ny) continue;
        s += 0.25 * rho[g.el_off[cc] + (long long)ey * g.nx + ex];
      }
    }
    b[c] = s;
  }
}

// rho_tilde_e = (1/4) sum of phi over the element's nodes (T_F^T P phi); one thread per element
__global__ void k_pde_out(PdeGeom g, int n_cells, const double* __restrict__ phi,
                          double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.n_el;
       e += (long long)gridDim.x * blockDim.x) {
    int c = 0;
    while (c + 1 < n_cells && e >= g.el_off[c + 1]) ++c;
    const long long loc = e - g.el_off[c];
    const int ey = (int)(loc / g.nx), ex = (int)(loc % g.nx);
    const long long o = g.node_off[c] + (long long)ey * (g.nx + 1) + ex;
    const double s = phi[g.col[o]] + phi[g.col[o + 1]] + phi[g.col[o + g.nx + 2]] + phi[g.col[o + g.nx + 1]];
    out[e] = 0.25 * s;
  }
}

// CG vector steps (one thread per unknown, block partials of the dot products)
__global__ void k_pde_dot(const double* __restrict__ a, const double* __restrict__ b, int n,
                          double* __restrict__ partials) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int k = blockIdx.x * PT + threadIdx.x; k < n; k += PB * PT) s = fma(a[k], b[k], s);
  s = pde_block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}
__global__ void k_pde_finish(const double* __restrict__ partials, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < PB; b += blockDim.x) s += partials[b];
  s = pde_block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}
// z = r / diag
__global__ void k_pde_jacobi(const double* __restrict__ r, const double* __restrict__ d,
                             double* __restrict__ z, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) z[k] = r[k] / d[k];
}
// p = z + beta p (beta = sc[0] / sc[1], 0 when sc[1] = 0)
__global__ void k_pde_pupdate(const double* __restrict__ z, double* __restrict__ p, int n,
                              const double* __restrict__ sc) {
  const double beta = sc[1] != 0.0 ? sc[0] / sc[1] : 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    p[k] = fma(beta, p[k], z[k]);
}
// x += alpha p, r -= alpha q (alpha = sc[0] / sc[2])
__global__ void k_pde_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                         const double* __restrict__ q, int n, const double* __restrict__ sc) {
  const double alpha = sc[2] != 0.0 ? sc[0] / sc[2] : 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    x[k] = fma(alpha, p[k], x[k]);
    r[k] = fma(-alpha, q[k], r[k]);
  }
}

int pde_grid(long long n) {
  const long long b = (n + PT - 1) / PT;
  return (int)(b < 4 * PB ? (b > 0 ? b : 1) : 4 * PB);
}

}  // namespace

#define PCK(x)                                                                  \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      f->err = std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x;      \
      return e_ == cudaErrorMemoryAllocation ? MSTOPO_OUT_OF_MEMORY : MSTOPO_CUDA_ERROR; \
    }                                                                           \
  } while (0)

static std::string g_pde_create_error;

static void pde_free(mstopo_pde_filter* f) {
  void* ptrs[] = {f->d_ny, f->d_node_cell, f->d_col, f->d_mem_off, f->d_mem, f->d_node_off,
                  f->d_el_off, f->d_diag, f->d_x, f->d_r, f->d_z, f->d_p, f->d_q, f->d_partials,
                  f->d_scal};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (f->h_scal) cudaFreeHost(f->h_scal);
}

static mstopo_status pde_setup(mstopo_pde_filter* f, const mstopo_pde_desc* d) {
  const int nx = d->nx, nc = d->n_cells;
  std::vector<int> ny(d->ny, d->ny + nc);
  std::vector<long long> node_off(nc), el_off(nc);
  long long nn = 0, ne = 0;
  for (int c = 0; c < nc; ++c) {
    node_off[c] = nn;
    el_off[c] = ne;
    nn += (long long)(nx + 1) * (ny[c] + 1);
    ne += (long long)nx * ny[c];
  }
  if (nn >= (1LL << 31)) {
    f->err = "PDE filter mesh too large";
    return MSTOPO_INVALID_ARG;
  }
  std::vector<int> node_cell(nn);
  for (int c = 0; c < nc; ++c)
    for (long long t = 0; t < (long long)(nx + 1) * (ny[c] + 1); ++t) node_cell[node_off[c] + t] = c;
  // identified node pairs of the domain (Sec. 4.5), then a union-find to collapsed unknowns
  std::vector<int> parent(nn);
  std::iota(parent.begin(), parent.end(), 0);
  auto find = [&](int a) {
    while (parent[a] != a) {
      parent[a] = parent[parent[a]];
      a = parent[a];
    }
    return a;
  };
  auto unite = [&](long long a, long long b) {
    const int ra = find((int)a), rb = find((int)b);
    if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
  };
  auto node = [&](int c, int i, int j) { return node_off[c] + (long long)j * (nx + 1) + i; };
  if (d->domain == MSTOPO_PDE_PERIODIC_CELL) {
    for (int j = 0; j <= ny[0]; ++j) unite(node(0, 0, j), node(0, nx, j));
    for (int i = 0; i <= nx; ++i) unite(node(0, i, 0), node(0, i, ny[0]));
  } else if (d->domain == MSTOPO_PDE_STACKED_BLOCKS) {
    for (int c = 0; c < nc; ++c) {
      for (int j = 0; j <= ny[c]; ++j) unite(node(c, 0, j), node(c, nx, j));   // left = right
      for (int i = 0; i <= nx; ++i) {
        unite(node(c, i, 0), node(0, i, 0));                                    // all bottoms
        unite(node(c, i, ny[c]), node(0, i, 0));                                // all tops
      }
    }
  }
  std::vector<int> root(nn), col(nn), first(nn, -1);
  int ncol = 0;
  for (long long n = 0; n < nn; ++n) root[n] = find((int)n);
  for (long long n = 0; n < nn; ++n)   // unknowns numbered by their smallest node
    if (first[root[n]] < 0) first[root[n]] = ncol++;
  for (long long n = 0; n < nn; ++n) col[n] = first[root[n]];
  std::vector<int> mem_off(ncol + 1, 0), mem(nn);
  for (long long n = 0; n < nn; ++n) mem_off[col[n] + 1]++;
  for (int c = 0; c < ncol; ++c) mem_off[c + 1] += mem_off[c];
  std::vector<int> fill(mem_off.begin(), mem_off.end() - 1);
  for (long long n = 0; n < nn; ++n) mem[fill[col[n]]++] = (int)n;   // ascending node ids
  f->n_cells = nc;
  auto up = [&](auto*& dst, const auto& v) -> cudaError_t {
    cudaError_t e = cudaMalloc(&dst, v.size() * sizeof(v[0]));
    if (e == cudaSuccess) e = cudaMemcpy(dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice);
    return e;
  };
  PCK(up(f->d_ny, ny));
  PCK(up(f->d_node_off, node_off));
  PCK(up(f->d_el_off, el_off));
  PCK(up(f->d_node_cell, node_cell));
  PCK(up(f->d_col, col));
  PCK(up(f->d_mem_off, mem_off));
  PCK(up(f->d_mem, mem));
  PdeGeom& g = f->g;
  g.nx = nx;
  g.n_nodes = nn;
  g.n_el = ne;
  g.ncol = ncol;
  const double r = d->rmin / (2.0 * std::sqrt(3.0));
  g.r2 = r * r;
  g.ny = f->d_ny;
  g.node_off = f->d_node_off;
  g.el_off = f->d_el_off;
  g.node_cell = f->d_node_cell;
  g.col = f->d_col;
  g.mem_off = f->d_mem_off;
  g.mem = f->d_mem;
  const size_t vb = (size_t)ncol * 8;
  PCK(cudaMalloc(&f->d_diag, vb));
  PCK(cudaMalloc(&f->d_x, vb));
  PCK(cudaMalloc(&f->d_r, vb));
  PCK(cudaMalloc(&f->d_z, vb));
  PCK(cudaMalloc(&f->d_p, vb));
  PCK(cudaMalloc(&f->d_q, vb));
  PCK(cudaMalloc(&f->d_partials, PB * 8));
  PCK(cudaMalloc(&f->d_scal, 8 * 8));
  PCK(cudaMallocHost(&f->h_scal, 8 * 8));
  note_launch(), k_pde_apply<<<pde_grid(ncol), PT, 0, f->s>>>(g, nullptr, f->d_diag);
  PCK(cudaGetLastError());
  PCK(cudaStreamSynchronize(f->s));
  return MSTOPO_OK;
}

extern "C" {

mstopo_status mstopo_pde_filter_create(const mstopo_pde_desc* d, mstopo_pde_filter** out) {
  if (!out) return MSTOPO_INVALID_ARG;
  *out = nullptr;
  g_pde_create_error.clear();
  if (!d || d->nx < 1 || d->n_cells < 1 || !d->ny || !(d->rmin > 0.0) || d->tol < 0.0 ||
      d->max_iter < 0 ||
      (d->domain != MSTOPO_PDE_PLAIN && d->domain != MSTOPO_PDE_PERIODIC_CELL &&
       d->domain != MSTOPO_PDE_STACKED_BLOCKS) ||
      (d->domain != MSTOPO_PDE_STACKED_BLOCKS && d->n_cells != 1)) {
    g_pde_create_error = "invalid PDE filter description";
    return MSTOPO_INVALID_ARG;
  }
  for (int c = 0; c < d->n_cells; ++c)
    if (d->ny[c] < 1) {
      g_pde_create_error = "invalid PDE filter description";
      return MSTOPO_INVALID_ARG;
    }
  mstopo_pde_filter* f = new mstopo_pde_filter();
  f->s = (cudaStream_t)d->stream;
  f->tol = d->tol > 0.0 ? d->tol : 1e-12;
  f->max_iter = d->max_iter > 0 ? d->max_iter : 1000;
  mstopo_status st = pde_setup(f, d);
  if (st != MSTOPO_OK) {
    g_pde_create_error = f->err;
    pde_free(f);
    delete f;
    return st;
  }
  *out = f;
  return MSTOPO_OK;
}

mstopo_status mstopo_pde_filter_apply(mstopo_pde_filter* f, const double* rho, double* rho_tilde,
                                      int32_t* iterations, double* rel_residual) {
  if (!f) return MSTOPO_INVALID_ARG;
  if (!rho || !rho_tilde) {
    f->err = "null pointer";
    return MSTOPO_INVALID_ARG;
  }
  const PdeGeom& g = f->g;
  const int n = g.ncol, grid = pde_grid(n);
  cudaStream_t s = f->s;
  double* sc = f->d_scal;   // [0] rz, [1] rz_old, [2] pq, [3] rr, [4] bb
  // b = P^T T_F rho into r; x = 0
  note_launch(), k_pde_rhs<<<grid, PT, 0, s>>>(g, rho, f->d_r);
  PCK(cudaGetLastError());
  PCK(cudaMemsetAsync(f->d_x, 0, (size_t)n * 8, s));
  PCK(cudaMemsetAsync(f->d_p, 0, (size_t)n * 8, s));
  PCK(cudaMemsetAsync(sc, 0, 8 * 8, s));
  note_launch(), k_pde_dot<<<PB, PT, 0, s>>>(f->d_r, f->d_r, n, f->d_partials);
  note_launch(), k_pde_finish<<<1, PT, 0, s>>>(f->d_partials, sc + 4);
  PCK(cudaGetLastError());
  PCK(cudaMemcpyAsync(f->h_scal, sc, 8 * 8, cudaMemcpyDeviceToHost, s));
  PCK(cudaStreamSynchronize(s));
  const double bb = f->h_scal[4];
  double rr = bb;
  int it = 0;
  while (rr > f->tol * f->tol * bb && it < f->max_iter) {
    // z = D^-1 r; rz_old = rz; rz = r.z; p = z + (rz / rz_old) p
    note_launch(), k_pde_jacobi<<<grid, PT, 0, s>>>(f->d_r, f->d_diag, f->d_z, n);
    PCK(cudaMemcpyAsync(sc + 1, sc, 8, cudaMemcpyDeviceToDevice, s));
    note_launch(), k_pde_dot<<<PB, PT, 0, s>>>(f->d_r, f->d_z, n, f->d_partials);
    note_launch(), k_pde_finish<<<1, PT, 0, s>>>(f->d_partials, sc);
    note_launch(), k_pde_pupdate<<<grid, PT, 0, s>>>(f->d_z, f->d_p, n, sc);
    // q = K p; alpha = rz / p.q; x += alpha p; r -= alpha q; rr = r.r
    note_launch(), k_pde_apply<<<grid, PT, 0, s>>>(g, f->d_p, f->d_q);
    note_launch(), k_pde_dot<<<PB, PT, 0, s>>>(f->d_p, f->d_q, n, f->d_partials);
    note_launch(), k_pde_finish<<<1, PT, 0, s>>>(f->d_partials, sc + 2);
    note_launch(), k_pde_xr<<<grid, PT, 0, s>>>(f->d_x, f->d_r, f->d_p, f->d_q, n, sc);
    note_launch(), k_pde_dot<<<PB, PT, 0, s>>>(f->d_r, f->d_r, n, f->d_partials);
    note_launch(), k_pde_finish<<<1, PT, 0, s>>>(f->d_partials, sc + 3);
    PCK(cudaGetLastError());
    PCK(cudaMemcpyAsync(f->h_scal, sc, 8 * 8, cudaMemcpyDeviceToHost, s));
    PCK(cudaStreamSynchronize(s));
    rr = f->h_scal[3];
    ++it;
    if (!std::isfinite(rr)) {
      f->err = "non-finite value in the PDE filter solve";
      return MSTOPO_NONFINITE;
    }
  }
  note_launch(), k_pde_out<<<pde_grid(g.n_el), PT, 0, s>>>(g, f->n_cells, f->d_x, rho_tilde);
  PCK(cudaGetLastError());
  PCK(cudaStreamSynchronize(s));
  if (iterations) *iterations = it;
  if (rel_residual) *rel_residual = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
  if (rr > f->tol * f->tol * bb) {
    f->err = "PDE filter solve reached max_iter";
    return MSTOPO_MAX_ITER;
  }
  return MSTOPO_OK;
}

int64_t mstopo_pde_filter_num_elements(const mstopo_pde_filter* f) { return f ? f->g.n_el : 0; }
int64_t mstopo_pde_filter_num_unknowns(const mstopo_pde_filter* f) { return f ? f->g.ncol : 0; }

const char* mstopo_pde_filter_last_error(const mstopo_pde_filter* f) {
  return f ? f->err.c_str() : g_pde_create_error.c_str();
}

void mstopo_pde_filter_destroy(mstopo_pde_filter* f) {
  if (!f) return;
  pde_free(f);
  delete f;
}

}  // extern "C"
