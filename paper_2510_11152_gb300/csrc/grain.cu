// grain.cu -- the grain-growth step of Sec. 3.3.1 (multi-order-parameter Allen-Cahn, Fan and Chen)
// on the GPU: one kernel forms the q right-hand sides of the linearly implicit step from the old
// order parameters, then the q periodic solves run as batches of concurrent graph branches through
// fas_solve_batched. The step and its reading are stated in include/grain.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/grain.h"

namespace fasmg {
void set_last_error(const std::string& msg);  // fas_api.cu
namespace {

constexpr int kGgBlock = 256;

// rhs_i = eta_i - dt L ( -alpha eta_i + beta eta_i^3 + 2 gamma eta_i (phi - eta_i^2) ) for every order
// parameter i at each cell, phi = sum_j eta_j^2 summed in the order j = 0..q-1. One thread per cell
// walks the q fields twice (phi, then the right-hand sides); consecutive threads read consecutive
// cells of a field, so every pass is coalesced. The products and sums are rounded one by one (no
// contraction into FMAs), the cube as (eta eta) eta.
__global__ void __launch_bounds__(kGgBlock) k_gg_rhs(double* __restrict__ rhs, const double* __restrict__ eta,
                                                     int q, int64_t cells, gg_model m, double dt) {
  const double na = -m.alpha, b = m.beta, g2 = 2.0 * m.gamma, dtl = dt * m.L;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (int64_t)gridDim.x * blockDim.x) {
    double phi = 0.0;
    for (int i = 0; i < q; ++i) {
      const double e = eta[(int64_t)i * cells + c];
      phi = __dadd_rn(phi, __dmul_rn(e, e));
    }
    for (int i = 0; i < q; ++i) {
      const double e = eta[(int64_t)i * cells + c];
      const double e2 = __dmul_rn(e, e);
      double local = __dadd_rn(__dmul_rn(na, e), __dmul_rn(b, __dmul_rn(e2, e)));
      local = __dadd_rn(local, __dmul_rn(__dmul_rn(g2, e), __dsub_rn(phi, e2)));
      rhs[(int64_t)i * cells + c] = __dsub_rn(e, __dmul_rn(dtl, local));
    }
  }
}

fas_status gg_fail(fas_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

}  // namespace
}  // namespace fasmg

struct gg_ctx {
  int dim = 2;
  int64_t cells = 0;
  int q = 0;
  double dt = 0.0;
  gg_model model{};
  cudaStream_t stream = nullptr;
  int sm_count = 148;
  std::vector<fas_ctx*> solvers;  // one per problem of a batch
  double* rhs = nullptr;          // q right-hand sides
};

using namespace fasmg;

extern "C" {

fas_status gg_destroy(gg_ctx* c) {
  if (!c) return FAS_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (fas_ctx* s : c->solvers) fas_destroy(s);
  if (c->rhs) cudaFree(c->rhs);
  delete c;
  return FAS_OK;
}

fas_status gg_create(int dim, const int n[3], double h, double dt, int q, const gg_model* model,
                     const fas_params* solver, int batch, void* stream, gg_ctx** out) {
  if (!out || !n) return gg_fail(FAS_EINVAL, "gg_create: null argument");
  *out = nullptr;
  if (dim != 2 && dim != 3) return gg_fail(FAS_EINVAL, "gg_create: dim must be 2 or 3");
  for (int a = 0; a < dim; ++a)
    if (n[a] < 4 || (n[a] & (n[a] - 1))) return gg_fail(FAS_EINVAL, "gg_create: every n must be a power of two >= 4");
  if (!(h > 0.0) || !(dt > 0.0) || q < 1) return gg_fail(FAS_EINVAL, "gg_create: h, dt must be positive and q >= 1");
  gg_model m = model ? *model : gg_model{1.0, 1.0, 1.0, 1.0, 2.0};
  if (!(m.L > 0.0) || !(m.kappa > 0.0)) return gg_fail(FAS_EINVAL, "gg_create: L and kappa must be positive");
  gg_ctx* c = new gg_ctx();
  c->dim = dim;
  c->q = q;
  c->dt = dt;
  c->model = m;
  c->stream = (cudaStream_t)stream;
  c->cells = (int64_t)n[0] * n[1] * (dim == 3 ? n[2] : 1);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMalloc(&c->rhs, (size_t)q * c->cells * sizeof(double)) != cudaSuccess) {
    gg_destroy(c);
    return gg_fail(FAS_ENOMEM, "gg_create: right-hand sides");
  }
  fas_params p;
  fas_default_params(&p);
  if (solver) {
    p.nu1 = solver->nu1;
    p.nu2 = solver->nu2;
    p.nu_coarse = solver->nu_coarse;
    p.kmax = solver->kmax;
    p.coarsest = solver->coarsest;
    p.tol = solver->tol;
    p.tol_relative = solver->tol_relative;
    p.precision = solver->precision;
    p.inner_cycles = solver->inner_cycles;
    p.use_graph = solver->use_graph;
  }
  p.dim = dim;
  for (int a = 0; a < 3; ++a) p.n[a] = a < dim ? n[a] : 1;
  p.h = h;
  p.alpha = 1.0;
  p.beta = dt * m.L * m.kappa;
  p.kappa = nullptr;
  p.kappa_const = 1.0;
  for (int k = 0; k < 6; ++k) p.bc[k] = FAS_BC_PERIODIC;
  p.location = FAS_CELL;
  p.coarse_exact = 0;
  const int nb = std::max(1, std::min(q, batch > 0 ? batch : 128));
  for (int k = 0; k < nb; ++k) {
    fas_ctx* s = nullptr;
    const fas_status st = fas_create(&p, stream, &s);
    if (st != FAS_OK) {
      gg_destroy(c);
      return st;
    }
    c->solvers.push_back(s);
  }
  *out = c;
  return FAS_OK;
}

fas_status gg_rhs(gg_ctx* c, const double* eta, double* rhs) {
  if (!c || !eta || !rhs) return gg_fail(FAS_EINVAL, "gg_rhs: null argument");
  if (((uintptr_t)eta | (uintptr_t)rhs) & 15) return gg_fail(FAS_EINVAL, "gg_rhs: fields must be 16-byte aligned");
  const int64_t want = (c->cells + kGgBlock - 1) / kGgBlock;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c->sm_count * 8));
  k_gg_rhs<<<grid, kGgBlock, 0, c->stream>>>(rhs, eta, c->q, c->cells, c->model, c->dt);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gg_fail(FAS_ECUDA, std::string("gg_rhs: ") + cudaGetErrorString(e));
  return FAS_OK;
}

fas_status gg_step(gg_ctx* c, double* eta, fas_info* infos) {
  if (!c || !eta) return gg_fail(FAS_EINVAL, "gg_step: null argument");
  fas_status st = gg_rhs(c, eta, c->rhs);
  if (st != FAS_OK) return st;
  const int nb = (int)c->solvers.size();
  std::vector<double*> u(nb);
  std::vector<const double*> f(nb);
  std::vector<fas_info> inf(nb);
  fas_status worst = FAS_OK;
  for (int k0 = 0; k0 < c->q; k0 += nb) {
    const int m = std::min(nb, c->q - k0);
    for (int i = 0; i < m; ++i) {
      u[i] = eta + (int64_t)(k0 + i) * c->cells;
      f[i] = c->rhs + (int64_t)(k0 + i) * c->cells;
    }
    st = fas_solve_batched(c->solvers.data(), m, u.data(), f.data(), inf.data(), c->stream);
    if (st != FAS_OK && st != FAS_ENOTCONV && st != FAS_ENONFINITE) return st;
    if (st == FAS_ENONFINITE || (st != FAS_OK && worst == FAS_OK)) worst = st;
    if (infos)
      for (int i = 0; i < m; ++i) infos[k0 + i] = inf[i];
  }
  if (worst != FAS_OK)
    return gg_fail(worst, worst == FAS_ENOTCONV ? "gg_step: a solve missed its tolerance within kmax"
                                                : "gg_step: a residual is not finite");
  return FAS_OK;
}

}  // extern "C"
