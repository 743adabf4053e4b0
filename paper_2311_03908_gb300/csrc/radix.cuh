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
}  // namespace dem
