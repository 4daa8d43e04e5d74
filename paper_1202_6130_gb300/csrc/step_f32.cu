// Fused-step kernels with float population storage, for D2Q9 and D2Q21.
#include "step_impl.cuh"

LBM_INSTANTIATE_STEP(9, float)
LBM_INSTANTIATE_STEP(21, float)
