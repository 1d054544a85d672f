// Instantiation of the D3 kernels for double storage (one translation unit per variant so that
// they compile in parallel).
#include "cm_kernels.cuh"

CM_INSTANTIATE(3, double)
