// inst_kahan.cu -- the split-Kahan form: as the split form, with layer masses and cell sums
// kept as Kahan-compensated FP32 pairs instead of FP64.
#include "launch.cuh"
namespace dem {
DEM_INSTANTIATE(PrecKahan)
}
