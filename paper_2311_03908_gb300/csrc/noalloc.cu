// noalloc.cu -- overall reduction degree of caller-owned parcel arrays, allocating nothing.
//
// This is the allocation-free twin of the reduction-degree kernels behind
// dem_reduction_degree. Those keep their per-parcel and per-block scratch in the context's
// arena; here the per-block partial sums live in a file-scope __device__ array instead, so
// a caller that owns its parcel arrays and may not call cudaMalloc (for example code whose
// device memory is all handed out by another framework's allocator, or a latency-critical
// loop that cannot afford cudaMalloc's implicit device-wide synchronisation) can still get
// the bed's reduction degree. The paper has no counterpart of this entry point.
#include <cuda_runtime.h>

#include <atomic>

#include "../../include/dem.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;                              // parcels per thread in pass 1
constexpr int kMaxBlocks = 4096;                       // rows of the scratch array
constexpr int kPerBlock = kThreads * kItems;           // 2048 parcels per block
static_assert((long long)kMaxBlocks * kPerBlock == DEM_NOALLOC_MAX_PARCELS, "stated maximum");

// Scratch: three partial sums (f_ov, lattice oxygen, oxygen of the ore's basis) per block
// of pass 1. 96 KiB; every GPU that loads this library holds it until the process exits.
static __device__ __align__(256) double g_partials[kMaxBlocks * 3];

// Molar masses (kg/mol) of Fe2O3, Fe3O4, FeO, Fe.
__device__ __constant__ static const double cM[4] = {159.69e-3, 231.533e-3, 71.844e-3, 55.845e-3};

// Pass 1: per-block sums in a fixed order (per-thread strided sums, then a shared tree).
__global__ void __launch_bounds__(kThreads) k_fov_partials(const double *m0, const double *m1,
                                                           const double *m2, const double *m3,
                                                           const int32_t *ore, int n,
                                                           double *partials) {
  __shared__ double sh[3][kThreads];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  const int base = blockIdx.x * kPerBlock;
  for (int it = 0; it < kItems; ++it) {
    const int i = base + it * kThreads + threadIdx.x;
    if (i >= n) break;
    const double n0 = m0[i] / cM[0], n1 = m1[i] / cM[1], n2 = m2[i] / cM[2], n3 = m3[i] / cM[3];
    const double nfe = 2.0 * n0 + 3.0 * n1 + n2 + n3;   // iron moles, eqs (2-15)..(2-17)
    double f = 0.0;
    if (nfe > 0.0) {
      const double fh = (3.0 * n1 + n2 + n3) / nfe, fm = (n2 + n3) / nfe, fw = n3 / nfe;
      f = ore[i] == 0 ? fh / 9.0 + 2.0 * fm / 9.0 + 6.0 * fw / 9.0 : 0.25 * fm + 0.75 * fw;
    }
    a0 += f;
    a1 += 3.0 * n0 + 4.0 * n1 + n2;
    a2 += (ore[i] == 0 ? 1.5 : 4.0 / 3.0) * nfe;
  }
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  sh[2][threadIdx.x] = a2;
  __syncthreads();
  for (int off = kThreads / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x < 3) partials[blockIdx.x * 3 + threadIdx.x] = sh[threadIdx.x][0];
}

// Pass 2: one block adds the partials of pass 1 in a fixed order.
__global__ void __launch_bounds__(kThreads) k_fov_final(const double *partials, int nblocks, int n,
                                                        double *out) {
  __shared__ double sh[3][kThreads];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) {
    a0 += partials[b * 3 + 0];
    a1 += partials[b * 3 + 1];
    a2 += partials[b * 3 + 2];
  }
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  sh[2][threadIdx.x] = a2;
  __syncthreads();
  for (int off = kThreads / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sh[0][0] / (double)n;
    out[1] = sh[2][0] > 0.0 ? 1.0 - sh[1][0] / sh[2][0] : 0.0;
  }
}

// Device address of g_partials per device. In host code the name g_partials is only a
// host-side stand-in, so kernels must be given this address. It is looked up again on every
// call made outside a stream capture (the lookup is cheap, and a context that was torn down
// and created again may have loaded the module at another address); a call made inside a
// capture uses the address of the last uncaptured call on that device. Atomic, because host
// threads may make their first calls on one device at the same time.
constexpr int kMaxDevices = 64;
std::atomic<double *> s_scratch[kMaxDevices];

}  // namespace

extern "C" int dem_reduction_degree_noalloc(const double *m_fe2o3, const double *m_fe3o4,
                                            const double *m_feo, const double *m_fe,
                                            const int32_t *ore_type, int32_t n, double *out,
                                            void *cuda_stream) {
  if (!m_fe2o3 || !m_fe3o4 || !m_feo || !m_fe || !ore_type || !out || n <= 0) return DEM_EINVAL;
  if (n > DEM_NOALLOC_MAX_PARCELS) return DEM_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return DEM_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return DEM_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return DEM_ECUDA;
  double *scratch = nullptr;
  if (cap == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return DEM_ECUDA;
    scratch = (double *)p;
    s_scratch[dev].store(scratch, std::memory_order_release);
  } else {
    // inside a capture no lookup is made: an uncaptured call on this device must come first
    scratch = s_scratch[dev].load(std::memory_order_acquire);
    if (!scratch) return DEM_ESTATE;
  }
  const int nblocks = (n + kPerBlock - 1) / kPerBlock;
  // pass 1 writes every row that pass 2 reads, so nothing has to be cleared first. Each
  // launch's own status is checked (an error left pending by other code is not reported).
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kThreads);
  cfg.stream = st;
  cfg.gridDim = dim3(nblocks);
  if (cudaLaunchKernelEx(&cfg, k_fov_partials, m_fe2o3, m_fe3o4, m_feo, m_fe, ore_type, n, scratch) !=
      cudaSuccess)
    return DEM_ECUDA;
  cfg.gridDim = dim3(1);
  if (cudaLaunchKernelEx(&cfg, k_fov_final, (const double *)scratch, nblocks, n, out) != cudaSuccess)
    return DEM_ECUDA;
  return DEM_OK;
}
