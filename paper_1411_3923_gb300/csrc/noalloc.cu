// An entry point that allocates no device memory: the FP32 matrix-free stiffness matvec
// of mstopo_apply_K (MIXED precision) for callers that own no handle and may not call
// cudaMalloc.  Its FP32 work vectors and node mask live in one file-scope __device__
// array of fixed size, which every GPU that loads this library holds until the process
// exits.  Calls share that array, so calls that overlap on the GPU race; the array keeps
// the last call's contents (every call overwrites all of the part it uses).
#include <mutex>

#include "internal.cuh"

#define NOALLOC_MAX_DOFS (1LL << 22)          // 4,194,304 DOFs = 2,097,152 nodes
#define NOALLOC_MAX_DEVICES 64
// [u32: MAX_DOFS floats][y32: MAX_DOFS floats][node mask: MAX_DOFS/2 bytes]
#define NOALLOC_BYTES (NOALLOC_MAX_DOFS * 4 * 2 + NOALLOC_MAX_DOFS / 2)

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device (looked up once per device).
static cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

__global__ void k_noalloc_node_mask(const uint8_t* __restrict__ fixed, uint8_t* __restrict__ nmask,
                                    long long n_nodes) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_nodes;
       i += (long long)gridDim.x * blockDim.x)
    nmask[i] = (uint8_t)((fixed[2 * i] ? 1 : 0) | (fixed[2 * i + 1] ? 2 : 0));
}

extern "C" mstopo_status mstopo_apply_K_f32_noalloc(const double* u, double* y, const float* E,
                                                   const uint8_t* fixed, int32_t nelx,
                                                   int32_t nely, double nu, void* stream) {
  if (!u || !y || !E || !fixed || nelx <= 0 || nely <= 0 || !(nu >= 0.0 && nu < 0.5))
    return MSTOPO_INVALID_ARG;
  // sizes in 64 bits before any addition (nelx = INT32_MAX must not wrap to a small count)
  const long long n_nodes = ((long long)nelx + 1) * ((long long)nely + 1);
  const long long n_dof = 2 * n_nodes;
  if (n_dof <= 0 || n_dof > NOALLOC_MAX_DOFS) return MSTOPO_INVALID_ARG;
  void* base = nullptr;
  if (noalloc_scratch(&base) != cudaSuccess) return MSTOPO_CUDA_ERROR;
  float* u32 = reinterpret_cast<float*>(base);
  float* y32 = u32 + NOALLOC_MAX_DOFS;
  uint8_t* nmask = reinterpret_cast<uint8_t*>(y32 + NOALLOC_MAX_DOFS);
  cudaStream_t s = (cudaStream_t)stream;
  double K0[64];
  element_stiffness_closed_form(nu, K0);
  StencilCoef<double> c64;
  StencilCoef<float> c32;
  make_stencil(K0, c64, c32);
  note_launch(), k_noalloc_node_mask<<<304, 256, 0, s>>>(fixed, nmask, n_nodes);
  if (cudaGetLastError() != cudaSuccess) return MSTOPO_CUDA_ERROR;
  if (launch_convert_d2f(u, u32, n_dof, s) != cudaSuccess) return MSTOPO_CUDA_ERROR;
  if (launch_matvec_f32(u32, y32, E, nmask, nelx, nely, c32, 1, n_dof, 0, s) != cudaSuccess)
    return MSTOPO_CUDA_ERROR;
  if (launch_convert_f2d(y32, y, n_dof, s) != cudaSuccess) return MSTOPO_CUDA_ERROR;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MSTOPO_CUDA_ERROR;
  return MSTOPO_OK;
}
