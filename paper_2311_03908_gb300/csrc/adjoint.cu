// adjoint.cu -- placeholder translation unit for the adjoint kernels.
#include "ctx.cuh"
