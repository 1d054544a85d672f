// Instantiation of the D3 kernels for __nv_bfloat16 storage (one translation unit per variant so that
// they compile in parallel).
#include "cm_kernels.cuh"

CM_INSTANTIATE(3, __nv_bfloat16)
