// Fused-step kernels with __half population storage, for D2Q9 and D2Q21.
#include "step_impl.cuh"

LBM_INSTANTIATE_STEP(9, __half)
LBM_INSTANTIATE_STEP(21, __half)
