// resort.cu -- re-sorting parcels whose cell keys changed little since the last sort.
//
// Input: kold, the previous sorted keys (position = previous index), and knew[i], the new key
// of the parcel at previous index i. Output: (kout, vout) = the stable sort of (knew, i), i.e.
// keys ascending and equal keys in previous-index order -- the same permutation the LSD radix
// sort gives, bit for bit. Parcels whose key did not change ("stayers") are already in
// order; the few that changed ("movers") are compacted in previous-index order (a
// deterministic block scan), ranked on (key, index) by counting (every mover against every
// other, in shared memory, up to 4096 movers; one block's bitonic sort in global memory
// beyond), and every parcel's output position follows from two counts (a merge of two sorted
// sequences):
//   stayer i:  (stayers before i) + (movers with (key, index) < (knew[i], i));
//   mover t:   t + (stayers before it) = t + P(clamp(idx, lb, ub)), where [lb, ub) is the run
//              of kold equal to its new key and P(x) the number of stayers in positions < x
//              (stayers keep their key, so kold orders them).
// Three kernels: compaction (each block sums the counts of the blocks before it: no separate
// scan pass), ranking (with one extra block that takes the large case), merge.
#include <cuda_runtime.h>

#include "radix.cuh"
#include "pdl.cuh"

namespace dem {
namespace {

constexpr int RZ_BLOCK = 1024;
constexpr int RZ_SMEM_SORT = 4096;

// movers before each position (pre[0..n], pre[n] = total) and the compacted movers; a block
// of RZ_COMPACT threads covers RZ_BLOCK positions, four consecutive ones per thread (vector
// loads and stores). blk holds the movers of every block of RZ_BLOCK positions; a block adds
// up those of the blocks before it itself (at most a few thousand counts, from L2), in a
// fixed order, so no scan pass runs between the key kernel and this one.
constexpr int RZ_COMPACT = RZ_BLOCK / 4;
__global__ void __launch_bounds__(RZ_COMPACT) rz_compact(const unsigned *kold, const unsigned *knew, int n,
                                                         const int *blk, int *pre, unsigned long long *comp) {
  pdl_wait();
  __shared__ int wsum[RZ_COMPACT / 32];
  __shared__ int wbase[RZ_COMPACT / 32];
  const int i0 = blockIdx.x * RZ_BLOCK + 4 * threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int base = 0;   // this thread's share of the counts of the blocks before this one
  for (int t = threadIdx.x; t < (int)blockIdx.x; t += RZ_COMPACT) base += blk[t];
  unsigned kn[4] = {0u, 0u, 0u, 0u};
  bool mv[4] = {false, false, false, false};
  if (i0 + 4 <= n) {
    const uint4 a = *reinterpret_cast<const uint4 *>(knew + i0);
    const uint4 b = *reinterpret_cast<const uint4 *>(kold + i0);
    kn[0] = a.x; kn[1] = a.y; kn[2] = a.z; kn[3] = a.w;
    mv[0] = a.x != b.x; mv[1] = a.y != b.y; mv[2] = a.z != b.z; mv[3] = a.w != b.w;
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u < n) { kn[u] = knew[i0 + u]; mv[u] = kn[u] != kold[i0 + u]; }
  }
  const int c = (int)mv[0] + (int)mv[1] + (int)mv[2] + (int)mv[3];
  int incl = c;   // inclusive scan of the counts over the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) base += __shfl_xor_sync(0xffffffffu, base, o);
  if (lane == 31) wsum[warp] = incl;
  if (lane == 0) wbase[warp] = base;
  __syncthreads();
  if (warp == 0) {
    const int v = lane < RZ_COMPACT / 32 ? wsum[lane] : 0;
    int wi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    int bb = lane < RZ_COMPACT / 32 ? wbase[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bb += __shfl_xor_sync(0xffffffffu, bb, o);
    if (lane < RZ_COMPACT / 32) wsum[lane] = bb + wi - v;   // movers before the warp
  }
  __syncthreads();
  int rank = wsum[warp] + incl - c;
  int r[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    r[u] = rank;
    if (mv[u]) {
      comp[rank] = ((unsigned long long)kn[u] << 32) | (unsigned)(i0 + u);
      ++rank;
    }
  }
  if (i0 + 4 <= n) {
    *reinterpret_cast<int4 *>(pre + i0) = make_int4(r[0], r[1], r[2], r[3]);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u < n) pre[i0 + u] = r[u];
  }
  if (i0 <= n - 1 && n - 1 < i0 + 4) pre[n] = rank;   // the last position's thread: all movers
}

__device__ __forceinline__ void cmpswap(unsigned long long &a, unsigned long long &b, bool asc) {
  if ((a > b) == asc) { const unsigned long long t = a; a = b; b = t; }
}

// more movers than fit in shared memory: one block sorts them in global memory (bitonic;
// padded with the largest value up to a power of two)
__device__ __noinline__ void rz_sort_big(int m, const unsigned long long *comp, unsigned long long *a, int cap) {
  int P = 1;
  while (P < m) P <<= 1;
  if (P > cap) return;   // cannot happen: cap is the next power of two of n
  for (int t = threadIdx.x; t < P; t += blockDim.x) a[t] = t < m ? comp[t] : ~0ull;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < P; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          unsigned long long x = a[t], y = a[u];
          cmpswap(x, y, (t & k) == 0);
          a[t] = x;
          a[u] = y;
        }
      }
      __syncthreads();
    }
  }
}

// rank of every mover by counting the movers below it (composites are unique), written to
// sorted[rank]; RZ_RANK_SPLIT consecutive lanes share a mover and count a share of the others
// each. More than RZ_SMEM_SORT movers: the grid's last block sorts them (rz_sort_big) and the
// others return.
constexpr int RZ_RANK_SPLIT = 8;
constexpr int RZ_RANK_BLOCKS = RZ_SMEM_SORT * RZ_RANK_SPLIT / 256;
__global__ void __launch_bounds__(256) rz_rank(const int *pre, int n, const unsigned long long *comp,
                                               unsigned long long *sorted, int cap) {
  pdl_wait();
  __shared__ unsigned long long s[RZ_SMEM_SORT];
  const int m = pre[n];
  if (m > RZ_SMEM_SORT) {
    if (blockIdx.x == gridDim.x - 1) rz_sort_big(m, comp, sorted, cap);
    return;
  }
  if (blockIdx.x * blockDim.x >= m * RZ_RANK_SPLIT) return;   // whole block beyond the movers
  for (int q = threadIdx.x; q < m; q += blockDim.x) s[q] = comp[q];
  __syncthreads();
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) / RZ_RANK_SPLIT;
  const int part = threadIdx.x % RZ_RANK_SPLIT;
  const unsigned long long v = t < m ? s[t] : 0ull;
  int r = 0;
  if (t < m)
    for (int q = part; q < m; q += RZ_RANK_SPLIT) r += s[q] < v ? 1 : 0;
#pragma unroll
  for (int o = RZ_RANK_SPLIT / 2; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o, RZ_RANK_SPLIT);
  if (t < m && part == 0) sorted[r] = v;
}

// Entries of the sorted c[lo, hi) below v (before(e, v) = e < v), or not above it
// (before(e, v) = e <= v), by the whole warp: each round every lane tests one of 32 evenly
// spaced entries and the ballot narrows the range 32-fold (three dependent loads for a few
// thousand entries, five for millions, instead of 11-21). All 32 lanes must call it together.
template <class T, bool Strict>
__device__ __forceinline__ int warp_bound(const T *c, int lo, int hi, T v, int lane) {
  auto before = [v](T e) { return Strict ? e <= v : e < v; };
  while (hi > lo) {
    const int len = hi - lo;
    if (len <= 32) return lo + __popc(__ballot_sync(0xffffffffu, lane < len && before(c[lo + lane])));
    const int s = (len + 31) / 32;
    const int p = lo + lane * s;
    const int k = __popc(__ballot_sync(0xffffffffu, p < hi && before(c[p])));   // samples before v
    const int nlo = k > 0 ? lo + (k - 1) * s + 1 : lo;
    hi = min(lo + k * s, hi);
    lo = nlo;
  }
  return lo;
}

// output positions. A warp of stayers sees only the movers between the composites of its
// first and last position (kold is sorted, so (kold[g], g) increases with g): two searches
// per warp, then a short scan per thread. The per-position loads are issued before the
// searches, so that their latency overlaps.
constexpr int RZ_MERGE = 256;
__global__ void __launch_bounds__(RZ_MERGE) rz_merge(const unsigned *kold, const unsigned *knew, int n,
                                                     const int *pre, const unsigned long long *sorted,
                                                     const unsigned *vmap, unsigned *kout, unsigned *vout) {
  pdl_wait();
  const int m = pre[n];
  const int g = blockIdx.x * RZ_MERGE + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int w0 = g - lane;
  unsigned key = 0u, ko = 0u, vg = 0u;
  int pg = 0;
  if (g < n) {
    key = knew[g];
    ko = kold[g];
    pg = pre[g];
    vg = vmap ? vmap[g] : (unsigned)g;
  }
  int lo = 0, hi = 0;
  if (w0 < n) {   // warp-uniform
    const int g1 = min(w0 + 32, n) - 1;
    const unsigned k0 = __shfl_sync(0xffffffffu, ko, 0);
    const unsigned k1 = __shfl_sync(0xffffffffu, ko, g1 - w0);
    const unsigned long long c0 = ((unsigned long long)k0 << 32) | (unsigned)w0;
    const unsigned long long c1 = ((unsigned long long)k1 << 32) | (unsigned)g1;
    lo = warp_bound<unsigned long long, false>(sorted, 0, m, c0, lane);
    hi = warp_bound<unsigned long long, false>(sorted, lo, m, c1 + 1, lane);
  }
  if (g < n && key == ko) {   // stayer
    const unsigned long long c = ((unsigned long long)key << 32) | (unsigned)g;
    int below = lo;
    for (int t = lo; t < hi; ++t) below += sorted[t] < c ? 1 : 0;
    const int pos = g - pg + below;
    kout[pos] = key;
    vout[pos] = vg;
  }
  // movers: one warp each (warp-uniform loop), bounds of the new key in kold
  const int wid = g >> 5, nw = (gridDim.x * RZ_MERGE) >> 5;
  for (int t = wid; t < m; t += nw) {
    const unsigned long long c = sorted[t];
    const unsigned mk = (unsigned)(c >> 32);
    const int idx = (int)(c & 0xffffffffu);
    const int lb = warp_bound<unsigned, false>(kold, 0, n, mk, lane);
    const int ub = warp_bound<unsigned, true>(kold, lb, n, mk, lane);
    if (lane == 0) {
      const int x = idx < lb ? lb : (idx > ub ? ub : idx);
      const int pos = t + (x - pre[x]);
      kout[pos] = mk;
      vout[pos] = vmap ? vmap[idx] : (unsigned)idx;
    }
  }
}

}  // namespace

size_t resort_words(int n, int *pow2) {
  int P = 1;
  while (P < n) P <<= 1;
  *pow2 = P;
  const size_t nb = (size_t)(n + RZ_BLOCK - 1) / RZ_BLOCK;
  // comp and sorted (2 words per entry each), pre (n + 1), blk (nb + 1)
  return 4 * (size_t)P + (size_t)n + 1 + nb + 1 + 2;
}

int *resort_counts(unsigned *scratch, int pow2, int n) {
  return reinterpret_cast<int *>(scratch + 4 * (size_t)pow2) + n + 1;
}

int resort_pairs(const unsigned *kold, const unsigned *knew, const unsigned *vmap, unsigned *kout, unsigned *vout,
                 unsigned *scratch, int pow2, int n, cudaStream_t st, long long *launches, bool pdl) {
  const int nb = (n + RZ_BLOCK - 1) / RZ_BLOCK;
  unsigned long long *comp = reinterpret_cast<unsigned long long *>(scratch);
  unsigned long long *sorted = comp + pow2;
  int *pre = reinterpret_cast<int *>(scratch + 4 * (size_t)pow2);
  int *blk = pre + n + 1;
  launch_k(pdl, rz_compact, nb, RZ_COMPACT, st, kold, knew, n, (const int *)blk, pre, comp);
  launch_k(pdl, rz_rank, RZ_RANK_BLOCKS + 1, 256, st, (const int *)pre, n, (const unsigned long long *)comp, sorted,
           pow2);
  launch_k(pdl, rz_merge, (n + RZ_MERGE - 1) / RZ_MERGE, RZ_MERGE, st, kold, knew, n, (const int *)pre,
           (const unsigned long long *)sorted, vmap, kout, vout);
  if (launches) *launches += 3;
  return (int)cudaPeekAtLastError();
}

}  // namespace dem
