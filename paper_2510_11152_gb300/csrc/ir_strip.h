// ir_strip.h -- the float64 refinement residual of the mixed-precision solve with a constant
// diffusivity (ir_strip.cu): 2D cell-centred levels and 3D levels (cells or faces).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace fasmg {

// True if the strip kernels handle the level: constant kappa, nx a multiple of 128; 2D cell-centred,
// or 3D (cells or faces) with ny a multiple of 8.
bool ir_strip_supported(const LevelDesc<double>& L);

// Bounded waits of the 3D kernel's tile loads: the deadline per wait, and a test hook that withholds
// one copy (block 0's first) so that its waits must run out.
struct Ir3Wait {
  unsigned long long limit_ns;
  int withhold;
};

// Kernel attributes (dynamic shared memory of the 3D kernel); call once before any launch or capture.
cudaError_t ir_strip_prepare();

// r32 = (float)(b - A u) and per-block partials of sum (s r32)^2 (s = *nsp, or 1) into
// partials[0 .. *nblocks). At most max_blocks blocks are launched. ticket: three zeroed counters; the
// kernels hand out their work with the first two (and leave them zero again); the 3D kernel sets the
// third when a bounded wait ran out (the caller reports FAS_ETIMEOUT and clears it). Launches sharing
// them must not overlap.
cudaError_t launch_ir_strip(float* r32, const double* u, const double* b, const LevelDesc<double>& L,
                            const float* nsp, double* partials, unsigned* ticket, int sm_count, int max_blocks,
                            int* nblocks, cudaStream_t stream, Ir3Wait wt);

}  // namespace fasmg
