// ir_strip.h -- the float64 refinement residual of the mixed-precision solve for 2D cell-centred
// levels with a constant diffusivity (ir_strip.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace fasmg {

// True if the strip kernel handles the level (2D, cell-centred, constant kappa, nx a multiple of 128).
bool ir_strip_supported(const LevelDesc<double>& L);

// r32 = (float)(b - A u) and per-block partials of sum (s r32)^2 (s = *nsp, or 1) into
// partials[0 .. *nblocks). At most max_blocks blocks are launched.
cudaError_t launch_ir_strip(float* r32, const double* u, const double* b, const LevelDesc<double>& L,
                            const float* nsp, double* partials, int sm_count, int max_blocks, int* nblocks,
                            cudaStream_t stream);

}  // namespace fasmg
