// radix.cuh -- LSD radix sort of 32-bit (key, value) pairs (see radix.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace dem {
// words of scratch the histogram needs for n keys
size_t radix_hist_words(int n);
// Sort (k, v) on the low `bits` bits of k, ping-ponging with (k2, v2). *kres / *vres receive
// the buffers that hold the result. Returns a cudaError_t code (0 on success).
int radix_sort_pairs(unsigned *k, unsigned *v, unsigned *k2, unsigned *v2, unsigned *hist, int n,
                     int bits, cudaStream_t st, unsigned **kres, unsigned **vres, long long *launches);
// Incremental re-sort (resort.cu): kold = previous sorted keys, knew[i] = new key of the
// parcel at previous index i; writes the stable sort of (knew, i) to (kout, vout), the
// values being vmap[i] (or i when vmap is null). Scratch:
// resort_words(n, &pow2) 32-bit words, 8-byte aligned. Before the call, the counts
// resort_counts(...)[i >> 10] must hold the number of changed keys (knew[i] != kold[i]) in
// each block of 1024 positions (the key kernel adds them while it computes the keys).
// Returns a cudaError_t code.
size_t resort_words(int n, int *pow2);
int *resort_counts(unsigned *scratch, int pow2, int n);
int resort_pairs(const unsigned *kold, const unsigned *knew, const unsigned *vmap, unsigned *kout, unsigned *vout,
                 unsigned *scratch, int pow2, int n, cudaStream_t st, long long *launches, bool pdl = false);
}  // namespace dem
