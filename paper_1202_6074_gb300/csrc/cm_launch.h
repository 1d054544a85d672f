// Declarations of the host launchers defined in cm_kernels.cuh and instantiated in inst_*.cu.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cm_core.cuh"

namespace cm {
template <int D, class S>
cudaError_t launch_step(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st);
// moments and the initial state of the z-planes z0 .. z0 + nzc - 1
template <int D, class S>
cudaError_t launch_moments(const void* src, const void* Ff, const Params& p, double* rho, double* u, cudaStream_t st,
                           int z0, int nzc);
template <int D, class S>
cudaError_t launch_init(void* dst, const void* Ff, const Params& p, const double* rho, const double* u, cudaStream_t st,
                        int z0, int nzc);
template <int D, class S>
cudaError_t launch_reduce(const void* src, const void* Ff, const Params& p, double* part, double* out, cudaStream_t st);
cudaError_t launch_convert_force(const double* in, void* out, long long n, bool fp64, cudaStream_t st);

template <int D, class R>
cudaError_t launch_adjoint_terminal(const void* state, const void* Ff, const Params& p, const double* dLdu,
                                    const double* dLdrho, void* lambda, double* dLdF, cudaStream_t st);
// acc: 0 = add into the FP64 dLdF, 1 = add into the segment accumulator seg (arithmetic type),
// 2 = add into seg, then fold seg into dLdF and reset it (see adjoint.cu)
template <int D, class R>
cudaError_t launch_adjoint_step(const void* state, const void* Ff, const Params& p, const void* lam_in, void* lam_out,
                                double* dLdF, void* seg, int acc, cudaStream_t st);

constexpr int kReduceMaxBlocks = 1216;

// The two-cells-per-thread step (k_step_pair) covers D3Q27 with FP32 arithmetic, periodic x,
// and nx a multiple of 64 (each warp's 32 lanes read 32 consecutive cells, or both halves of
// the row), in every collision form.
inline bool pair_eligible(const Params& p, int D, bool fp32_arith) {
    return D == 3 && fp32_arith && p.bc[0] == 0 && p.nx % 64 == 0;
}

// Two steps per pass for FP32 storage (launch_pair_two_steps, inst_pair_tb_f32.cu): planes in
// groups of kTwoStepGroup, the intermediate state in a ring of kTwoStepRing + 2 planes.
constexpr int kTwoStepGroup = 8;
constexpr int kTwoStepRing = kTwoStepGroup + 2;     // the planes a group's second step reads
inline bool two_steps_eligible(const Params& p, int D, int storage_f32, bool slab) {
    return storage_f32 && !slab && pair_eligible(p, D, true) && p.nz >= 2 * kTwoStepGroup && p.attractor == 0 &&
           !p.reduced;
}
// enqueue one pass (steps t -> t+2) from A into C; returns the number of kernel launches or -1
int launch_two_steps_f32(const void* A, void* C, void* ring, const void* Ff, const Params& p, cudaStream_t st);

// turbulence as forcing (turbulence.cu): scratch holds 10 N arithmetic values
template <int D, class S>
cudaError_t launch_turbulence_force(const void* state, void* force, const Params& p, double cs, void* scratch,
                                    cudaStream_t st);

// TMA-staged D3Q27 step (step_tma.cu)
int tma_row_width(const Params& p, int esize);
bool encode_tma_maps(const void* base, const Params& p, int storage, void* map_main, void* map_halo);
template <class S>
cudaError_t launch_step_tma(const void* map_main, const void* map_halo, const void* src, void* dst, const void* Ff,
                            const Params& p, int* err, int nsm, cudaStream_t st);
}  // namespace cm
