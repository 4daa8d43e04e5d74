// Fused-step kernels with __nv_bfloat16 population storage, for D2Q9 and D2Q21.
#include "step_impl.cuh"

LBM_INSTANTIATE_STEP(9, __nv_bfloat16)
LBM_INSTANTIATE_STEP(21, __nv_bfloat16)
