// Host helpers of the TMA-staged step (the kernels are in step_tma.cuh, instantiated per
// storage type in step_tma_{f32,bf16,f16}.cu so that they compile in parallel).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "cm_launch.h"

namespace cm {

int tma_row_width(const Params& p, int esize) {
    const int align = 16 / esize;
    if (p.nx % align) return 0;
    if (p.nx % 256 == 0) return 256;
    if (p.nx % 128 == 0) return 128;
    return 0;
}

// Tensor maps of one state buffer: the buffer viewed as [Q][nz][ny][nx], boxes of (TX, 1, 1, 1)
// (main) and (16 bytes, 1, 1, 1) (halo). Returns false when the driver entry point is missing or
// the encoding is rejected (the caller then uses the direct-load kernel).
bool encode_tma_maps(const void* base, const Params& p, int storage, void* map_main, void* map_halo) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    CUtensorMapDataType dt;
    int esize;
    switch (storage) {
        case 1: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; esize = 4; break;
        case 2: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; esize = 2; break;
        case 3: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; esize = 2; break;
        default: return false;
    }
    const int tx = tma_row_width(p, esize);
    if (tx == 0) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)p.nz, 27};
    const cuuint64_t strides[3] = {(cuuint64_t)p.nx * esize, (cuuint64_t)p.nx * p.ny * esize,
                                   (cuuint64_t)p.nx * p.ny * p.nz * esize};
    const cuuint32_t box_main[4] = {(cuuint32_t)tx, 1, 1, 1};
    const cuuint32_t box_halo[4] = {(cuuint32_t)(16 / esize), 1, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r1 = encode((CUtensorMap*)map_main, dt, 4, const_cast<void*>(base), dims, strides, box_main, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = encode((CUtensorMap*)map_halo, dt, 4, const_cast<void*>(base), dims, strides, box_halo, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS;
}

}  // namespace cm
