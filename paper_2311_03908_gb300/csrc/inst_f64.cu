// inst_f64.cu -- the all-FP64 form of the per-step kernels.
#include "launch.cuh"
namespace dem {
DEM_INSTANTIATE(PrecF64)
}
