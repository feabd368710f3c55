// context.h -- host-side state of a solver context (shared between the C-ABI translation units).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/fas.h"
#include "common.cuh"

namespace fasmg {

// Level hierarchy of one value type: descriptors (host and device copies) and device buffers.
//   u[l], f[l], u0[l] : solution, right-hand side and restricted start of level l >= 1
//                       (for the float hierarchy of mixed precision also level 0: e and r32)
//   r[l]              : residual scratch of level l
template <typename T>
struct Hier {
  int nlev = 0;
  int switch_level = 0;  // levels >= switch_level run inside the single-CTA kernel
  std::vector<LevelDesc<T>> desc;
  LevelDesc<T>* d_desc = nullptr;
  std::vector<T*> u, f, u0;
  std::vector<T*> u2, rc;  // fused path: second u buffer (ping-pong) and R(r) from the finer level
  int nfast = 0;           // levels 0..nfast-1 use the fused kernels
  SmemLayout smem;         // shared-memory layout of the single-CTA kernel (levels >= switch_level)
  size_t smem_bytes = 0;
  T** d_u = nullptr;
  T** d_f = nullptr;
  T** d_u0 = nullptr;
  T* cinv = nullptr;
  std::vector<void*> owned;  // every device allocation above
  bool allocated = false;
};

// Record the message fas_last_error() returns on this thread.
void set_last_error(const std::string& msg);

struct LevelShape {
  int nx, ny, nz;
  double h;
  int64_t cells() const { return (int64_t)nx * ny * nz; }
};

}  // namespace fasmg

// A captured solve: prologue, then a while node whose body is one cycle (see fas_api.cu).
struct SolveGraph {
  double* u = nullptr;
  const double* f = nullptr;
  const double* fsrc = nullptr;
  double dt = 0.0;
  int kind = 0;  // 0 solve, 1 heat step (forms b = u + dt fsrc first)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long n_pro = 0, n_body = 0;  // kernel launches of the prologue and of one body pass
};

struct ProfSpan {
  cudaEvent_t beg, end;
  int family, level;
  double units;
};

struct fas_ctx {
  fas_params p;
  cudaStream_t stream = nullptr;
  int sm_count = 148;
  int nlev = 0;
  std::vector<fasmg::LevelShape> shape;
  fasmg::Hier<double> h64;
  fasmg::Hier<float> h32;
  bool singular = false;
  double* partials = nullptr;  // per-block partial sums
  int max_blocks = 0;
  double* d_scalar = nullptr;  // small device scalars
  unsigned* ir_ticket = nullptr;  // refinement residual: work counter, finished blocks, timeout word
  double* h_scalar = nullptr;  // pinned host mirror
  unsigned* h_flag = nullptr;  // pinned: the timeout word of ir_ticket read back after a solve
  double* b = nullptr;         // heat-step right-hand side (fine, float64)
  double* fproj = nullptr;     // mean-free copy of f for singular problems
  std::vector<double*> adj;     // adjoint buffers: checkpoints, segment states, lambda, mu, work
  double* host_u = nullptr;    // device buffers of fas_heat_run_host
  double* host_f = nullptr;
  long long launches = 0;
  fasmg::SolveState* S = nullptr;   // device state of the current solve
  fasmg::SolveState* Sh = nullptr;  // pinned host mirror
  cudaStream_t side = nullptr;      // captures a solve graph's prologue
  cudaStream_t side2 = nullptr;     // captures the while node's body
  std::vector<SolveGraph> graphs;
  bool capturing = false;
  // kernel timing
  bool prof = false;
  std::vector<ProfSpan> spans;
  std::vector<cudaEvent_t> event_pool;
  size_t pool_next = 0;
};
