// inst_f32.cu -- the split form: FP32 forces, drag, heat and kinetics; FP64 positions,
// layer masses and cell sums.
#include "launch.cuh"
namespace dem {
DEM_INSTANTIATE(PrecSplit)
}
