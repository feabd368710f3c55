// stream3d.h -- launch API of the sweep-fused float32 X-MCGS sweep for 3D levels (stream3d.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace fasmg {

// True if the fused sweep handles the level: 3D, cell-centred, constant kappa, no periodic axis,
// nx a multiple of 128.
bool sweep3d_supported(const LevelDesc<float>& L);

// Kernel attributes (dynamic shared memory); call once before any launch or capture.
cudaError_t sweep3d_prepare();

// One X-MCGS sweep: uout = S(uin) for right-hand side f, the cells of colour c1 first (first_colour),
// then the others. uout and uin must be different 16-byte aligned buffers of the level's size. A tile
// wait that runs out after wait_ns sets *err (the caller reports FAS_ETIMEOUT); withhold != 0 (a test
// hook) withholds the first copy of block 0 so that its waits run out.
cudaError_t launch_sweep3d(float* uout, const float* uin, const float* f, const LevelDesc<float>& L, int c1,
                           int sm_count, unsigned* err, unsigned long long wait_ns, int withhold, cudaStream_t stream);

}  // namespace fasmg
