// Fused-step kernels with double population storage, for D2Q9 and D2Q21.
#include "step_impl.cuh"

LBM_INSTANTIATE_STEP(9, double)
LBM_INSTANTIATE_STEP(21, double)
