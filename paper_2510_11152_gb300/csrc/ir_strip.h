// ir_strip.h -- the float64 refinement residual of the mixed-precision solve with a constant
// diffusivity (ir_strip.cu): 2D cell-centred levels and 3D levels (cells or faces).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace fasmg {

// True if the strip kernels handle the level: constant kappa, nx a multiple of 128; 2D cell-centred,
// or 3D (cells or faces) with ny a multiple of 8.
bool ir_strip_supported(const LevelDesc<double>& L);

// r32 = (float)(b - A u) and per-block partials of sum (s r32)^2 (s = *nsp, or 1) into
// partials[0 .. *nblocks). At most max_blocks blocks are launched. ticket: two zeroed counters the 2D
// kernel hands out its work with (it leaves them zero again); launches sharing them must not overlap.
cudaError_t launch_ir_strip(float* r32, const double* u, const double* b, const LevelDesc<double>& L,
                            const float* nsp, double* partials, unsigned* ticket, int sm_count, int max_blocks,
                            int* nblocks, cudaStream_t stream);

}  // namespace fasmg
