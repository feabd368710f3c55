// small_static.cu -- V-cycles on a small grid without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a solve:
//   - programs whose memory allocator reserved all device memory up front and hands it out itself
//     (a cudaMalloc from this library would fail or fragment that pool);
//   - applications that give a solver plugin a fixed memory budget and only device pointers to work in;
//   - real-time loops that cannot afford an allocation's latency, or the chance of its failure, in
//     steady state.
// fas_vcycle_small_static serves them for grids small enough that the whole level hierarchy fits in
// one CTA's shared memory: it runs the same single-CTA V-cycle kernel as the library's small levels,
// with the only global scratch that kernel needs -- the level-descriptor table and one slot for the
// residual norm -- held in a file-scope static device array instead of memory from fas_create.
//
// The array lives on every GPU that loads the library until the process exits. All calls share it:
// a call overwrites the descriptors and the norm slot of the previous one, so calls that overlap on
// the GPU (for example on two streams) race and must be serialised by the caller (one stream, or
// events). Its device address is looked up once per device, on the first call made with that device
// current; make that first call before any stream capture begins, and do not use the entry point on a
// device after cudaDeviceReset in the same process (the address looked up before the reset is stale).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/fas.h"
#include "basic_kernels.cuh"
#include "context.h"

namespace fasmg {

// Maximum sizes of the static path: at most kStaticLevels levels, and u, f of every level plus the
// restricted start of the coarser ones within kStaticSmem bytes of shared memory (in float64: up to
// 64 x 64 cells in 2D, 16 x 16 x 16 in 3D, or any grid of at most 8000 cells whose hierarchy fits).
constexpr int kStaticLevels = 16;
constexpr size_t kStaticSmem = 200 * 1024;

struct StaticScratch {
  LevelDesc<double> desc[kStaticLevels];
  double norm[2];
};

// The scratch: about 27 KB.
static __device__ __align__(256) StaticScratch g_static_scratch;

namespace {

// Address of the scratch on each device, looked up once per device with that device current.
std::mutex g_addr_mutex;
void* g_addr[128] = {nullptr};

cudaError_t scratch_address(StaticScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = reinterpret_cast<StaticScratch*>(g_addr[dev]);
  return cudaSuccess;
}

// One level descriptor, passed by value as the kernel argument, stored into the static table (the
// descriptors reach the device without a host-memory copy).
__global__ void k_static_store_desc(LevelDesc<double> d, StaticScratch* S, int level) {
  const int words = (int)(sizeof(LevelDesc<double>) / sizeof(int));
  const int* src = reinterpret_cast<const int*>(&d);
  int* dst = reinterpret_cast<int*>(&S->desc[level]);
  for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
}

// ||f - A u||_2 of level 0 by one CTA (the grid is small), into norm[0].
template <int DIM>
__global__ void __launch_bounds__(1024) k_static_norm(const double* u, const double* f, StaticScratch* S) {
  const LevelDesc<double>& L = S->desc[0];
  double acc = 0.0;
  const int64_t n = (int64_t)L.nx * L.ny * L.nz;
  for (int64_t idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int i = (int)(idx & (L.nx - 1));
    const int j = (int)((idx >> L.lx) & (L.ny - 1));
    const int l = (int)(idx >> (L.lx + L.ly));
    const double r = residual_point<double, DIM>(u, f, L, idx, i, j, l);
    acc = fma(r, r, acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) S->norm[0] = sqrt(acc);
}

fas_status fail_static(fas_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

int log2i(int v) {
  int k = 0;
  while ((1 << k) < v) ++k;
  return k;
}

}  // namespace
}  // namespace fasmg

using namespace fasmg;

extern "C" fas_status fas_vcycle_small_static(const fas_params* p, double* u, const double* f, int ncycles,
                                              double* res_host, void* stream) {
  if (!p || !u || !f) return fail_static(FAS_EINVAL, "fas_vcycle_small_static: null argument");
  if (p->dim != 2 && p->dim != 3) return fail_static(FAS_EINVAL, "fas_vcycle_small_static: dim must be 2 or 3");
  if (ncycles < 1) return fail_static(FAS_EINVAL, "fas_vcycle_small_static: ncycles must be >= 1");
  if (p->ordering != FAS_ORDER_FORWARD && p->ordering != FAS_ORDER_SYMMETRIC)
    return fail_static(FAS_EINVAL, "fas_vcycle_small_static: unknown ordering");
  for (int k = 0; k < 2 * p->dim; ++k)
    if (p->bc[k] != FAS_BC_NEUMANN && p->bc[k] != FAS_BC_DIRICHLET)
      return fail_static(FAS_EUNSUPPORTED, "fas_vcycle_small_static: Neumann and Dirichlet faces only");
  if (p->kappa || p->coarse_exact || p->precision != FAS_FP64 || p->location != FAS_CELL)
    return fail_static(FAS_EUNSUPPORTED,
                       "fas_vcycle_small_static: cell-centred unknowns, constant kappa, smoothed coarsest level "
                       "and float64 only");
  for (int a = 0; a < p->dim; ++a)
    if (p->n[a] < 2 || (p->n[a] & (p->n[a] - 1)))
      return fail_static(FAS_EINVAL, "fas_vcycle_small_static: every n must be a power of two >= 2");
  if (!(p->h > 0.0) || !(p->beta > 0.0) || p->alpha < 0.0 || !(p->kappa_const > 0.0) || p->nu1 < 0 ||
      p->nu2 < 0 || p->nu1 + p->nu2 < 1 || p->coarsest < 2)
    return fail_static(FAS_EINVAL, "fas_vcycle_small_static: invalid operator or smoothing parameters");
  const int dim = p->dim;
  int nx = p->n[0], ny = p->n[1], nz = dim == 3 ? p->n[2] : 1;
  double h = p->h;
  // level shapes and descriptors (same definitions as fas_create)
  LevelDesc<double> desc[kStaticLevels];
  int64_t cells[kStaticLevels];
  int nlev = 0;
  const int nfaces = 2 * dim;
  const double bk = p->beta * p->kappa_const;
  while (true) {
    if (nlev == kStaticLevels)
      return fail_static(FAS_EINVAL, "fas_vcycle_small_static: more than 16 levels; grid too large");
    LevelDesc<double>& L = desc[nlev];
    std::memset(&L, 0, sizeof(L));
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.lx = log2i(nx);
    L.ly = log2i(ny);
    L.lz = log2i(nz);
    L.fax = -1;
    const double h2 = h * h;
    L.h2 = h2;
    L.ih2 = 1.0 / h2;
    L.c = bk / h2;
    L.alpha = p->alpha;
    for (int cls = 0; cls < kClasses; ++cls) {
      double m = 0.0;
      for (int face = 0; face < nfaces; ++face)
        m += ((cls >> face) & 1) ? (p->bc[face] == FAS_BC_DIRICHLET ? 2.0 : 0.0) : 1.0;
      const double D = p->alpha * h2 + bk * m;
      L.mt[cls] = (unsigned char)m;
      L.a[cls] = D != 0.0 ? bk / D : 0.0;
      L.b[cls] = D != 0.0 ? h2 / D : 0.0;
      L.d[cls] = D / h2;
    }
    cells[nlev] = (int64_t)nx * ny * nz;
    ++nlev;
    const int shortest = dim == 3 ? std::min(nx, std::min(ny, nz)) : std::min(nx, ny);
    if (shortest <= p->coarsest) break;
    nx /= 2;
    ny /= 2;
    if (dim == 3) nz /= 2;
    h *= 2.0;
  }
  // shared-memory layout of the single-CTA kernel (u, f per level, u0 below the top)
  SmemLayout S;
  std::memset(&S, 0, sizeof(S));
  int64_t off = 0;
  for (int l = 0; l < nlev; ++l) {
    const int64_t n = (cells[l] + 1) / 2 * 2;  // 16-byte alignment of every array
    S.off_u[l] = off;
    off += n;
    S.off_f[l] = off;
    off += n;
    if (l > 0) {
      S.off_u0[l] = off;
      off += n;
    }
  }
  S.total = off;
  const size_t smem = (size_t)off * sizeof(double) + (size_t)nlev * sizeof(LevelDesc<double>);
  if (smem > kStaticSmem)
    return fail_static(FAS_EINVAL, "fas_vcycle_small_static: grid too large (its levels need " +
                                       std::to_string(smem) + " bytes of shared memory, at most " +
                                       std::to_string(kStaticSmem) + ")");

  cudaStream_t st = (cudaStream_t)stream;
  StaticScratch* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return fail_static(FAS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  // the descriptors are rewritten on every call (by value, one small kernel per level); the norm slot
  // is written by the norm kernel
  static_assert(sizeof(LevelDesc<double>) % sizeof(int) == 0, "descriptor copied as 32-bit words");
  for (int l = 0; l < nlev; ++l) k_static_store_desc<<<1, 128, 0, st>>>(desc[l], scratch, l);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_static(FAS_ECUDA, std::string("descriptor store: ") + cudaGetErrorString(e));

  CoarseArgs<double> A;
  std::memset(&A, 0, sizeof(A));
  A.desc = scratch->desc;
  A.l0 = 0;
  A.nlev = nlev;
  A.nu1 = p->nu1;
  A.nu2 = p->nu2;
  A.nuc = p->nu_coarse > 0 ? p->nu_coarse : p->nu1;
  A.ordering = p->ordering;
  for (int k = 0; k < ncycles; ++k) {
    if (dim == 2) {
      cudaFuncSetAttribute(k_coarse_smem<double, 2, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStaticSmem);
      k_coarse_smem<double, 2, -1><<<1, 1024, smem, st>>>(A, S, u, f);
    } else {
      cudaFuncSetAttribute(k_coarse_smem<double, 3, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStaticSmem);
      k_coarse_smem<double, 3, -1><<<1, 1024, smem, st>>>(A, S, u, f);
    }
  }
  if (dim == 2)
    k_static_norm<2><<<1, 1024, 0, st>>>(u, f, scratch);
  else
    k_static_norm<3><<<1, 1024, 0, st>>>(u, f, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_static(FAS_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  if (res_host) {
    e = cudaMemcpyAsync(res_host, scratch->norm, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_static(FAS_ECUDA, std::string("norm copy: ") + cudaGetErrorString(e));
  }
  return FAS_OK;
}
