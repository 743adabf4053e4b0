// radix.cu -- least-significant-digit radix sort of (key, value) pairs of 32-bit words:
// the binning step of the particle path (parcels sorted on their DEM-cell key).
//
// Each pass sorts on one 8-bit digit, stably, in three kernels: per-tile digit histograms,
// an exclusive scan of each digit's row over the tiles (one block per digit), and a scatter in which every tile ranks its keys
// with warp-level match masks (__match_any_sync) and per-warp digit counts in shared
// memory, so equal digits keep their input order.
#include <cuda_runtime.h>

#include "radix.cuh"

namespace dem {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void __launch_bounds__(RS_THREADS) rs_hist(const unsigned *keys, int n, int shift,
                                                     unsigned *hist, int ntiles) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int it = 0; it < RS_ITEMS; ++it) {
    const int idx = base + it * RS_THREADS + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of each digit's row hist[d][0..ntiles) (one block per digit, in place);
// the row totals go to tot[d]. The scatter adds the digits' exclusive offsets itself.
constexpr int RS_SCAN_THREADS = 512;
__global__ void __launch_bounds__(RS_SCAN_THREADS) rs_scan_rows(unsigned *hist, int ntiles, unsigned *tot) {
  __shared__ unsigned part[RS_SCAN_THREADS];
  unsigned *row = hist + (size_t)blockIdx.x * ntiles;
  const int per = (ntiles + RS_SCAN_THREADS - 1) / RS_SCAN_THREADS;
  const int b = threadIdx.x * per;
  const int e = min(b + per, ntiles);
  unsigned s = 0;
  for (int t = b; t < e; ++t) s += row[t];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < RS_SCAN_THREADS; off <<= 1) {
    const unsigned v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int t = b; t < e; ++t) {
    const unsigned v = row[t];
    row[t] = run;
    run += v;
  }
  if (threadIdx.x == RS_SCAN_THREADS - 1) tot[blockIdx.x] = part[RS_SCAN_THREADS - 1];
}

__global__ void __launch_bounds__(RS_THREADS) rs_scatter(const unsigned *kin, const unsigned *vin,
                                                        unsigned *kout, unsigned *vout, int n,
                                                        int shift, const unsigned *hist, int ntiles,
                                                        const unsigned *tot) {
  __shared__ unsigned run[256];
  __shared__ unsigned gbase[256];
  __shared__ unsigned wc[RS_WARPS][257];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // exclusive offset of this digit: scan of the 256 digit totals (Hillis-Steele in run[])
  run[tid] = tot[tid];
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    const unsigned v = tid >= off ? run[tid - off] : 0u;
    __syncthreads();
    run[tid] += v;
    __syncthreads();
  }
  gbase[tid] = hist[tid * ntiles + blockIdx.x] + (run[tid] - tot[tid]);
  __syncthreads();
  run[tid] = 0;
  const unsigned lt = (1u << lane) - 1u;
  const int base = blockIdx.x * RS_TILE;
  for (int it = 0; it < RS_ITEMS; ++it) {
    const int idx = base + it * RS_THREADS + tid;
    const bool valid = idx < n;
    const unsigned key = valid ? kin[idx] : 0u;
    const unsigned val = valid ? vin[idx] : 0u;
    const unsigned dig = valid ? ((key >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, dig);
    const unsigned rank = __popc(peers & lt);
    for (int t = tid; t < RS_WARPS * 257; t += RS_THREADS) (&wc[0][0])[t] = 0u;
    __syncthreads();
    if (rank == 0) wc[warp][dig] = __popc(peers);
    __syncthreads();
    {
      unsigned acc = run[tid];
#pragma unroll
      for (int w = 0; w < RS_WARPS; ++w) {
        const unsigned t = wc[w][tid];
        wc[w][tid] = acc;
        acc += t;
      }
      run[tid] = acc;
    }
    __syncthreads();
    if (valid) {
      const unsigned pos = gbase[dig] + wc[warp][dig] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
  }
}

size_t radix_hist_words(int n) { return (size_t)256 * (size_t)((n + RS_TILE - 1) / RS_TILE) + 256; }

int radix_sort_pairs(unsigned *k, unsigned *v, unsigned *k2, unsigned *v2, unsigned *hist, int n,
                     int bits, cudaStream_t st, unsigned **kres, unsigned **vres, long long *launches) {
  const int ntiles = (n + RS_TILE - 1) / RS_TILE;
  const int passes = (bits + 7) / 8;
  unsigned *ka = k, *va = v, *kb = k2, *vb = v2;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    unsigned *tot = hist + (size_t)256 * ntiles;
    rs_hist<<<ntiles, RS_THREADS, 0, st>>>(ka, n, shift, hist, ntiles);
    rs_scan_rows<<<256, RS_SCAN_THREADS, 0, st>>>(hist, ntiles, tot);
    rs_scatter<<<ntiles, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, hist, ntiles, tot);
    if (launches) *launches += 3;
    unsigned *t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
  }
  *kres = ka;
  *vres = va;
  return (int)cudaPeekAtLastError();
}

}  // namespace dem
