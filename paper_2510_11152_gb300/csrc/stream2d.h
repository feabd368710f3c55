// stream2d.h -- launch API of the sweep-fused float32 kernels for 2D levels (stream2d.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace fasmg {

constexpr int kStripHalo = 8;                       // recomputed columns on each side of a strip
constexpr int kStripOut = 32 * 4 - 2 * kStripHalo;  // columns a strip writes (112)

// Set the kernels' shared-memory attributes (once per process; call before launching or capturing).
cudaError_t stream2d_prepare();

// True if the fused kernels handle a level of nx x ny cells with nu sweeps per smoothing step.
bool stream2d_supported(int nx, int ny, int nu);

// Pre-smoothing: uout = S^nu(uin) (uin = 0 when zero_init) for right-hand side fin, or, when tau,
// for f = fin + A uin (fin holding R(r) of the finer level; f is also written to fout). When uc is
// not null, also the residual r = f - A uout and its restriction: uc = R(uout), rc = R(r).
cudaError_t launch_stream2d_pre(const float* uin, const float* fin, float* fout, float* uout, float* uc, float* rc,
                                const LevelDesc<float>& L, int nu, bool zero_init, bool tau, int seg,
                                cudaStream_t stream);

// Post-smoothing: e = S^nu(uin + P(uc - R(uin))); uout = e, or, when u64 is not null, u64 += e in
// float64 (the update of a mixed-precision refinement step) and uout is not written.
cudaError_t launch_stream2d_post(const float* uin, const float* f, const float* uc, float* uout, double* u64,
                                 const LevelDesc<float>& L, int nu, int seg, cudaStream_t stream);

}  // namespace fasmg
