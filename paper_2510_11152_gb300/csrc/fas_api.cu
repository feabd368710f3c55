// fas_api.cu -- C-ABI entry points, level hierarchy set-up and the host-side FAS driver.
//
// The V-cycle follows Algorithm 1 with the recursion of the remark after it: on every level
// nu1 X-MCGS sweeps, the residual r = f - A u, u_c = R(u) and f_c = R(r) + A_c u_c (the tau
// correction; f_c overwrites R(r) in place as in the paper's reuse of r0), the coarse problem,
// u += P(u_c - R(u)_start), nu2 sweeps. Levels too small to fill the GPU run inside one CTA.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "basic_kernels.cuh"
#include "context.h"
#include "ir_strip.h"
#include "stream2d.h"
#include "stream3d.h"
#include "tma.cuh"

using namespace fasmg;

namespace {

thread_local std::string g_last_error;

// Bounded waits of the tile copies (the 3D refinement residual): the deadline of one wait, and the
// test hook that withholds one copy of the next launch (fas_debug_bounded_wait).
std::atomic<unsigned long long> g_wait_limit_ns{kTmaWaitNs};
std::atomic<int> g_withhold_copy{0};  // 0 none, 1 the next refinement residual, 2 the next fused sweep

// 1 (and the request cleared) when the test hook asks to withhold a copy of the next launch of kernel
// `which` (1 refinement residual, 2 fused 3D sweep).
int take_withhold(int which) {
  int expect = which;
  return g_withhold_copy.compare_exchange_strong(expect, 0) ? 1 : 0;
}

fas_status fail(fas_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define CUDA_TRY(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(FAS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));               \
  } while (0)

#define STATUS_TRY(call)            \
  do {                              \
    fas_status s_ = (call);         \
    if (s_ != FAS_OK) return s_;    \
  } while (0)

bool is_pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

constexpr int kBlock = 256;
constexpr int kCoarseThreads = 1024;
constexpr int64_t kSwitchCells2D = 16384;  // levels at or below this size run in one CTA
constexpr int64_t kSwitchCells2DLarge = 4096;  // the same on 2D grids of at least kLargeGrid2D cells
constexpr int64_t kLargeGrid2D = (int64_t)1 << 24;
constexpr int64_t kSwitchCells3D = 4096;
constexpr size_t kCoarseSmemMax = 200 * 1024;    // field arrays of the single-CTA kernel
constexpr size_t kCoarseSmemLimit = 227 * 1024;  // with its level descriptors (per-CTA maximum)
constexpr int64_t kSweep3dMinCells = (int64_t)1 << 26;  // smallest 3D level smoothed by the fused sweep
constexpr int64_t kFusedMinCells2D = (int64_t)1 << 20;  // smallest 2D level below the finest run fused

int grid_for(const fas_ctx* c, int64_t work) {
  int64_t g = (work + kBlock - 1) / kBlock;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, c->max_blocks));
}

// ---------------------------------------------------------------------------------------------
// kernel timing: an event pair around each launch while recording is on
// ---------------------------------------------------------------------------------------------

cudaEvent_t pool_event(fas_ctx* c) {
  if (c->pool_next == c->event_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->event_pool.push_back(e);
  }
  return c->event_pool[c->pool_next++];
}

struct Prof {
  fas_ctx* c;
  ProfSpan span;
  bool on;
  Prof(fas_ctx* ctx, int family, int level, double units) : c(ctx), on(ctx->prof && !ctx->capturing) {
    c->launches += 1;
    if (!on) return;
    span.beg = pool_event(c);
    span.end = pool_event(c);
    span.family = family;
    span.level = level;
    span.units = units;
    on = span.beg && span.end;
    if (on) cudaEventRecord(span.beg, c->stream);
  }
  ~Prof() {
    if (!on) return;
    cudaEventRecord(span.end, c->stream);
    c->spans.push_back(span);
  }
};

// ---------------------------------------------------------------------------------------------
// level descriptors
// ---------------------------------------------------------------------------------------------

// boundary multiplicity of a face: 0 Neumann (ghost = cell), 2 Dirichlet (ghost = -cell), 1 periodic
// (the face is an interior face whose neighbour is the wrapped cell)
int bc_mult(int kind) { return kind == FAS_BC_DIRICHLET ? 2 : (kind == FAS_BC_PERIODIC ? 1 : 0); }

// periodic axes as a bit mask (bit 0 x, 1 y, 2 z)
int periodic_mask(const fas_params& p) {
  int m = 0;
  for (int a = 0; a < p.dim; ++a)
    if (p.bc[2 * a] == FAS_BC_PERIODIC) m |= 1 << a;
  return m;
}

template <typename T>
LevelDesc<T> make_desc(const fas_params& p, const LevelShape& s) {
  LevelDesc<T> L;
  std::memset(&L, 0, sizeof(L));
  L.nx = s.nx;
  L.ny = s.ny;
  L.nz = s.nz;
  auto lg = [](int v) {
    int k = 0;
    while ((1 << k) < v) ++k;
    return k;
  };
  L.lx = lg(s.nx);
  L.ly = lg(s.ny);
  L.lz = lg(s.nz);
  L.varkappa = p.kappa != nullptr;
  L.fax = p.location - 1;  // FAS_CELL -> -1, FAS_FACE_X/Y/Z -> 0/1/2
  L.per = periodic_mask(p);
  const double h2 = s.h * s.h;
  L.h2 = (T)h2;
  L.ih2 = (T)(1.0 / h2);
  const double bk = p.beta * p.kappa_const;
  L.c = (T)(bk / h2);
  L.alpha = (T)p.alpha;
  const int nfaces = 2 * p.dim;
  for (int cls = 0; cls < kClasses; ++cls) {
    double m = 0.0;
    for (int face = 0; face < nfaces; ++face) {
      const bool boundary = (cls >> face) & 1;
      // face grid, own axis: the near wall face is a neighbour of value 0 (weight 1); the far one is
      // stored (the frozen slot), so only the near side is ever a boundary of an unknown
      const double mb = face / 2 == L.fax ? 1.0 : bc_mult(p.bc[face]);
      m += boundary ? mb : 1.0;
    }
    const double D = p.alpha * h2 + bk * m;
    L.mt[cls] = (unsigned char)m;
    L.a[cls] = (T)(D != 0.0 ? bk / D : 0.0);
    L.b[cls] = (T)(D != 0.0 ? h2 / D : 0.0);
    L.d[cls] = (T)(D / h2);
  }
  return L;
}

template <typename T, typename U>
fas_status dev_alloc(Hier<T>& H, U** ptr, int64_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, (size_t)std::max<int64_t>(count, 1) * sizeof(U));
  if (e != cudaSuccess) return fail(FAS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  H.owned.push_back(q);
  *ptr = (U*)q;
  return FAS_OK;
}

template <typename T>
void free_hier(Hier<T>& H) {
  for (void* q : H.owned) cudaFree(q);
  H.owned.clear();
  H.u.clear();
  H.f.clear();
  H.u0.clear();
  H.u2.clear();
  H.rc.clear();
  H.nfast = 0;
  H.d_desc = nullptr;
  H.cinv = nullptr;
  H.allocated = false;
}

// Dense matrix of the coarsest operator (h^-2 scaled like A), assembled from the descriptor, then
// inverted (pseudo-inverse through A + J/n when the problem is singular).
fas_status coarse_inverse(const fas_ctx* c, const LevelShape& s, const std::vector<double>& wx,
                          const std::vector<double>& wy, const std::vector<double>& wz,
                          const std::vector<double>& Dh, std::vector<double>& inv) {
  const int n = (int)s.cells();
  if (n > 1024) return fail(FAS_EUNSUPPORTED, "coarse_exact: coarsest level above 1024 cells");
  const fas_params& p = c->p;
  const LevelDesc<double> L = make_desc<double>(p, s);
  std::vector<double> M((size_t)n * n, 0.0);
  const int dim = p.dim;
  for (int l = 0; l < s.nz; ++l)
    for (int j = 0; j < s.ny; ++j)
      for (int i = 0; i < s.nx; ++i) {
        const int q = (l * s.ny + j) * s.nx + i;
        const int cls = (i == 0) | ((i == s.nx - 1) << 1) | ((j == 0) << 2) | ((j == s.ny - 1) << 3) |
                        (dim == 3 ? (((l == 0) << 4) | ((l == s.nz - 1) << 5)) : 0);
        const bool var = p.kappa != nullptr;
        M[(size_t)q * n + q] = var ? Dh[q] : L.d[cls];
        auto off = [&](int nb, double w) { M[(size_t)q * n + nb] -= w / (s.h * s.h); };
        const double bk = p.beta * p.kappa_const;
        if (i > 0) off(q - 1, var ? wx[q - 1] : bk);
        if (i < s.nx - 1) off(q + 1, var ? wx[q] : bk);
        if (j > 0) off(q - s.nx, var ? wy[q - s.nx] : bk);
        if (j < s.ny - 1) off(q + s.nx, var ? wy[q] : bk);
        if (dim == 3) {
          if (l > 0) off(q - s.nx * s.ny, var ? wz[q - s.nx * s.ny] : bk);
          if (l < s.nz - 1) off(q + s.nx * s.ny, var ? wz[q] : bk);
        }
        // periodic axes (constant kappa): the wrapped neighbours across the boundary
        if ((L.per & 1) && i == 0) off(q + s.nx - 1, bk);
        if ((L.per & 1) && i == s.nx - 1) off(q - (s.nx - 1), bk);
        if ((L.per & 2) && j == 0) off(q + (s.ny - 1) * s.nx, bk);
        if ((L.per & 2) && j == s.ny - 1) off(q - (s.ny - 1) * s.nx, bk);
        if ((L.per & 4) && l == 0) off(q + (s.nz - 1) * s.nx * s.ny, bk);
        if ((L.per & 4) && l == s.nz - 1) off(q - (s.nz - 1) * s.nx * s.ny, bk);
      }
  if (c->singular)
    for (auto& v : M) v += 1.0 / n;
  // Gauss-Jordan with partial pivoting on [M | I]
  inv.assign((size_t)n * n, 0.0);
  for (int q = 0; q < n; ++q) inv[(size_t)q * n + q] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(M[(size_t)r * n + col]) > std::fabs(M[(size_t)piv * n + col])) piv = r;
    if (M[(size_t)piv * n + col] == 0.0) return fail(FAS_EINVAL, "coarse_exact: singular coarsest matrix");
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(M[(size_t)piv * n + k], M[(size_t)col * n + k]);
        std::swap(inv[(size_t)piv * n + k], inv[(size_t)col * n + k]);
      }
    const double d = M[(size_t)col * n + col];
    for (int k = 0; k < n; ++k) {
      M[(size_t)col * n + k] /= d;
      inv[(size_t)col * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double fct = M[(size_t)r * n + col];
      if (fct == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        M[(size_t)r * n + k] -= fct * M[(size_t)col * n + k];
        inv[(size_t)r * n + k] -= fct * inv[(size_t)col * n + k];
      }
    }
  }
  if (c->singular)
    for (auto& v : inv) v -= 1.0 / n;
  return FAS_OK;
}

// Build one hierarchy: descriptors for every level, buffers when `buffers`, variable-kappa arrays.
template <typename T>
fas_status build_hier(fas_ctx* c, Hier<T>& H, bool buffers, bool level0_buffers) {
  const fas_params& p = c->p;
  H.nlev = c->nlev;
  H.desc.clear();
  for (int l = 0; l < c->nlev; ++l) H.desc.push_back(make_desc<T>(p, c->shape[l]));
  // single-CTA switch level: the first level small enough that the GPU cannot be filled and whose
  // whole sub-hierarchy (u, f on every level, u0 below it) fits in the CTA's shared memory. On a
  // large 2D grid nothing else runs beside the small levels, and one CTA smoothing 128^2 is slower than
  // per-operation launches across the GPU (8192^2: 118.1 -> 116.1 ms per 20-step run with the switch
  // at 64^2); smaller grids, often solved side by side in a batch, keep the switch at 128^2 (the
  // 96-problem batch was 2 % slower with 64^2).
  const int64_t sw_cells =
      p.dim == 2 ? (c->shape[0].cells() >= kLargeGrid2D ? kSwitchCells2DLarge : kSwitchCells2D) : kSwitchCells3D;
  H.switch_level = c->nlev - 1;
  for (int l = 0; l < c->nlev; ++l) {
    if (c->shape[l].cells() > sw_cells) continue;
    int64_t elems = 2 * c->shape[l].cells();
    for (int k = l + 1; k < c->nlev; ++k) elems += 3 * c->shape[k].cells();
    if ((size_t)elems * sizeof(T) <= kCoarseSmemMax) {
      H.switch_level = l;
      break;
    }
  }
  {
    int64_t off = 0;
    for (int l = H.switch_level; l < c->nlev; ++l) {
      const int64_t n = c->shape[l].cells();
      const int64_t pad = (16 / sizeof(T));  // keep every array 16-byte aligned
      H.smem.off_u[l] = off;
      off += (n + pad - 1) / pad * pad;
      H.smem.off_f[l] = off;
      off += (n + pad - 1) / pad * pad;
      if (l > H.switch_level) {
        H.smem.off_u0[l] = off;
        off += (n + pad - 1) / pad * pad;
      }
    }
    H.smem.total = off;
    H.smem_bytes = (size_t)off * sizeof(T) + (size_t)(c->nlev - H.switch_level) * sizeof(LevelDesc<T>);
    if (H.smem_bytes > kCoarseSmemLimit)
      return fail(FAS_EUNSUPPORTED, "coarsest levels do not fit in shared memory");
  }
  // per-cell diffusivity: kappa on every level (cell averages), then weights per level
  std::vector<double> cwx, cwy, cwz, cDh;  // coarsest level, for the dense inverse
  if (p.kappa) {
    double* kap = nullptr;
    const double* kprev = p.kappa;
    for (int l = 0; l < c->nlev; ++l) {
      const LevelShape& s = c->shape[l];
      const int64_t n = s.cells();
      if (l > 0) {
        void* q = nullptr;
        CUDA_TRY(cudaMalloc(&q, n * sizeof(double)));
        H.owned.push_back(q);
        kap = (double*)q;
        const LevelShape& sf = c->shape[l - 1];
        if (p.dim == 2)
          k_restrict<double, 2><<<grid_for(c, n), kBlock, 0, c->stream>>>(kap, nullptr, nullptr, kprev, nullptr,
                                                                          sf.nx, sf.ny, sf.nz);
        else
          k_restrict<double, 3><<<grid_for(c, n), kBlock, 0, c->stream>>>(kap, nullptr, nullptr, kprev, nullptr,
                                                                          sf.nx, sf.ny, sf.nz);
        kprev = kap;
      }
      T *wx, *wy, *wz, *rD, *Dh;
      STATUS_TRY(dev_alloc(H, &wx, n));
      STATUS_TRY(dev_alloc(H, &wy, n));
      STATUS_TRY(dev_alloc(H, &wz, p.dim == 3 ? n : 1));
      STATUS_TRY(dev_alloc(H, &rD, n));
      STATUS_TRY(dev_alloc(H, &Dh, n));
      const int4 lo = make_int4(bc_mult(p.bc[0]), bc_mult(p.bc[2]), p.dim == 3 ? bc_mult(p.bc[4]) : 0, 0);
      const int4 hi = make_int4(bc_mult(p.bc[1]), bc_mult(p.bc[3]), p.dim == 3 ? bc_mult(p.bc[5]) : 0, 0);
      if (p.dim == 2)
        k_kappa_weights<T, 2><<<grid_for(c, n), kBlock, 0, c->stream>>>(wx, wy, wz, rD, Dh, kprev, s.nx, s.ny,
                                                                         s.nz, p.alpha, p.beta, s.h, lo, hi);
      else
        k_kappa_weights<T, 3><<<grid_for(c, n), kBlock, 0, c->stream>>>(wx, wy, wz, rD, Dh, kprev, s.nx, s.ny,
                                                                         s.nz, p.alpha, p.beta, s.h, lo, hi);
      CUDA_TRY(cudaGetLastError());
      H.desc[l].wx = wx;
      H.desc[l].wy = wy;
      H.desc[l].wz = wz;
      H.desc[l].rD = rD;
      H.desc[l].Dh = Dh;
      if (l == c->nlev - 1 && p.coarse_exact) {
        // weights of the coarsest level in float64 for the dense inverse
        std::vector<double> kh(n);
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        CUDA_TRY(cudaMemcpy(kh.data(), kprev, n * sizeof(double), cudaMemcpyDeviceToHost));
        cwx.assign(n, 0.0);
        cwy.assign(n, 0.0);
        cwz.assign(n, 0.0);
        cDh.assign(n, 0.0);
        const double h2 = s.h * s.h;
        for (int l2 = 0; l2 < s.nz; ++l2)
          for (int j = 0; j < s.ny; ++j)
            for (int i = 0; i < s.nx; ++i) {
              const int q = (l2 * s.ny + j) * s.nx + i;
              double D = p.alpha * h2;
              const double kc = kh[q];
              auto face = [&](bool inside, int nb, int mult) {
                return inside ? p.beta * (0.5 * (kc + kh[nb])) : mult * p.beta * kc;
              };
              D += face(i > 0, q - 1, bc_mult(p.bc[0])) + face(i < s.nx - 1, q + 1, bc_mult(p.bc[1]));
              D += face(j > 0, q - s.nx, bc_mult(p.bc[2])) + face(j < s.ny - 1, q + s.nx, bc_mult(p.bc[3]));
              if (p.dim == 3)
                D += face(l2 > 0, q - s.nx * s.ny, bc_mult(p.bc[4])) +
                     face(l2 < s.nz - 1, q + s.nx * s.ny, bc_mult(p.bc[5]));
              if (i < s.nx - 1) cwx[q] = p.beta * (0.5 * (kc + kh[q + 1]));
              if (j < s.ny - 1) cwy[q] = p.beta * (0.5 * (kc + kh[q + s.nx]));
              if (p.dim == 3 && l2 < s.nz - 1) cwz[q] = p.beta * (0.5 * (kc + kh[q + s.nx * s.ny]));
              cDh[q] = D / h2;
            }
      }
    }
  }
  if (buffers) {
    H.u.assign(c->nlev, nullptr);
    H.f.assign(c->nlev, nullptr);
    H.u0.assign(c->nlev, nullptr);
    for (int l = 0; l < c->nlev; ++l) {
      const int64_t n = c->shape[l].cells();
      if (l > 0 || level0_buffers) {
        STATUS_TRY(dev_alloc(H, &H.u[l], n));
        STATUS_TRY(dev_alloc(H, &H.f[l], n));
      }
      if (l > 0) STATUS_TRY(dev_alloc(H, &H.u0[l], n));
    }
    // sweep-fused 2D path (float32 only): consecutive levels from the finest that the fused kernels
    // handle and that are larger than the single-CTA switch level
    H.nfast = 0;
    if (sizeof(T) == 4 && p.dim == 2 && p.path != 1 && !p.kappa && p.location == FAS_CELL &&
        p.ordering == FAS_ORDER_FORWARD && p.nu1 >= 1 && p.nu2 >= 1 && periodic_mask(p) == 0) {
      // below 2^20 cells a level's fused kernels are latency-bound (one warp streams a long segment of
      // rows) and the per-operation kernels measured faster (8192^2 run: 127.8 -> 125.8 ms); the finest
      // level stays fused for its float64 update
      while (H.nfast < H.switch_level &&
             stream2d_supported(c->shape[H.nfast].nx, c->shape[H.nfast].ny, std::max(p.nu1, p.nu2)) &&
             (H.nfast == 0 || c->shape[H.nfast].cells() >= kFusedMinCells2D || p.path == 2))
        H.nfast++;
    }
    H.u2.assign(c->nlev, nullptr);
    H.rc.assign(c->nlev, nullptr);
    for (int l = 0; l < H.nfast; ++l) {
      STATUS_TRY(dev_alloc(H, &H.u2[l], c->shape[l].cells()));
      if (l + 1 < H.nfast) STATUS_TRY(dev_alloc(H, &H.rc[l + 1], c->shape[l + 1].cells()));
    }
    // sweep-fused 3D smoothing (float32): a second buffer on every level that the fused sweep handles
    // (its sweeps ping-pong between the two) and that is large enough for it to pay: measured at
    // 512^3 it beats two colour launches (0.58 against 0.67 ms), at 256^3 it does not
    if constexpr (std::is_same<T, float>::value) {
      if (p.dim == 3 && p.path != 1 && p.ordering == FAS_ORDER_FORWARD && p.nu1 + p.nu2 >= 2)
        for (int l = 0; l < H.switch_level; ++l)
          if (sweep3d_supported(H.desc[l]) && (c->shape[l].cells() >= kSweep3dMinCells || p.path == 2))
            STATUS_TRY(dev_alloc(H, &H.u2[l], c->shape[l].cells()));
    }
    T** arrs[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k) STATUS_TRY(dev_alloc(H, &arrs[k], kMaxLevels));
    H.d_u = arrs[0];
    H.d_f = arrs[1];
    H.d_u0 = arrs[2];
    CUDA_TRY(cudaMemcpy(H.d_u, H.u.data(), c->nlev * sizeof(T*), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(H.d_f, H.f.data(), c->nlev * sizeof(T*), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(H.d_u0, H.u0.data(), c->nlev * sizeof(T*), cudaMemcpyHostToDevice));
    if (p.coarse_exact) {
      std::vector<double> inv;
      STATUS_TRY(coarse_inverse(c, c->shape[c->nlev - 1], cwx, cwy, cwz, cDh, inv));
      std::vector<T> invT(inv.begin(), inv.end());
      STATUS_TRY(dev_alloc(H, &H.cinv, (int64_t)invT.size()));
      CUDA_TRY(cudaMemcpy(H.cinv, invT.data(), invT.size() * sizeof(T), cudaMemcpyHostToDevice));
    }
    H.allocated = true;
  }
  STATUS_TRY(dev_alloc(H, &H.d_desc, c->nlev));
  CUDA_TRY(cudaMemcpy(H.d_desc, H.desc.data(), c->nlev * sizeof(LevelDesc<T>), cudaMemcpyHostToDevice));
  return FAS_OK;
}

// ---------------------------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------------------------

// Calls fn(std::integral_constant<int, FAX>) for the context's unknown location (FAX = -1 cells,
// 0..2 faces normal to x, y, z).
template <typename F>
void with_fax(const fas_ctx* c, F&& fn) {
  switch (c->p.location) {
    case FAS_FACE_X: fn(std::integral_constant<int, 0>()); break;
    case FAS_FACE_Y: fn(std::integral_constant<int, 1>()); break;
    case FAS_FACE_Z: fn(std::integral_constant<int, 2>()); break;
    default: fn(std::integral_constant<int, -1>()); break;
  }
}

// u (and u0) at level+1 from u, f at level+1 from r: Appendix C on cells, Appendix D on faces.
template <typename T, int DIM>
void launch_restrict(fas_ctx* c, int64_t nc, T* uc, T* uc0, T* fc, const T* u, const T* r, int nx, int ny, int nz) {
  with_fax(c, [&](auto tag) {
    constexpr int FAX = decltype(tag)::value;
    if constexpr (FAX < 0)
      k_restrict<T, DIM><<<grid_for(c, nc), kBlock, 0, c->stream>>>(uc, uc0, fc, u, r, nx, ny, nz);
    else
      k_restrict_face<T, DIM, FAX><<<grid_for(c, nc), kBlock, 0, c->stream>>>(uc, uc0, fc, u, r, nx, ny, nz);
  });
}

// u += P(uc - uc0) (uc0 may be null), u of a level with n cells.
template <typename T, int DIM>
void launch_prolong(fas_ctx* c, int64_t n, T* u, const T* uc, const T* uc0, int nx, int ny, int nz) {
  with_fax(c, [&](auto tag) {
    constexpr int FAX = decltype(tag)::value;
    if constexpr (FAX < 0)
      k_prolong<T, DIM><<<grid_for(c, n >> DIM), kBlock, 0, c->stream>>>(u, uc, uc0, nx, ny, nz);
    else
      k_prolong_face<T, DIM, FAX><<<grid_for(c, n), kBlock, 0, c->stream>>>(u, uc, uc0, nx, ny, nz);
  });
}

// `sweeps` X-MCGS sweeps in place on u. With a scratch buffer of the level's size (3D float32 levels
// the fused sweep handles), sweeps run in pairs through the sweep-fused kernel, u -> scratch -> u; an
// odd last sweep, and every other level, runs one launch per colour phase.
template <typename T, int DIM>
void launch_smooth(fas_ctx* c, const LevelDesc<T>& L, int level, T* u, const T* f, int sweeps, T* scratch = nullptr) {
  const int64_t half = (int64_t)(L.nx / 2) * L.ny * L.nz;
  const bool g4ok = !L.varkappa && L.nx % 4 == 0;  // 16-byte groups of 4 cells
  const int g = grid_for(c, g4ok ? half / 2 : half);
  int s0 = 0;
  if constexpr (std::is_same<T, float>::value && DIM == 3) {
    if (scratch && c->p.ordering == FAS_ORDER_FORWARD)
      for (; s0 + 2 <= sweeps; s0 += 2) {
        cudaError_t e;
        {
          Prof pr(c, FAS_K_SMOOTH, level, (double)(2 * half));
          e = launch_sweep3d(scratch, u, f, L, first_colour(c->p.ordering, s0), c->sm_count, c->ir_ticket + 2,
                             g_wait_limit_ns.load(), take_withhold(2), c->stream);
        }
        if (e != cudaSuccess) break;  // nothing was launched: the colour launches below do the sweeps
        {
          Prof pr(c, FAS_K_SMOOTH, level, (double)(2 * half));
          e = launch_sweep3d(u, scratch, f, L, first_colour(c->p.ordering, s0 + 1), c->sm_count, c->ir_ticket + 2,
                             g_wait_limit_ns.load(), take_withhold(2), c->stream);
        }
        if (e != cudaSuccess) {  // one sweep done, into scratch: bring it back
          cudaMemcpyAsync(u, scratch, (size_t)(2 * half) * sizeof(T), cudaMemcpyDeviceToDevice, c->stream);
          s0 += 1;
          break;
        }
      }
  }
  for (int s = s0; s < sweeps; ++s) {
    const int c0 = first_colour(c->p.ordering, s);
    for (const int colour : {c0, 1 - c0}) {
      Prof pr(c, FAS_K_SMOOTH, level, (double)half);
      if (g4ok)
        k_smooth_colour4<T, DIM><<<g, kBlock, 0, c->stream>>>(u, f, L, colour);
      else
        k_smooth_colour<T, DIM><<<g, kBlock, 0, c->stream>>>(u, f, L, colour);
    }
  }
}

// ||f - A u||_2 into *out (device); r (nullable) receives the residual; nsp: device norm scale or null.
template <typename T, int DIM>
void launch_residual(fas_ctx* c, const LevelDesc<T>& L, int level, T* r, const T* u, const T* f, const float* nsp,
                     double* out) {
  const int64_t n = (int64_t)L.nx * L.ny * L.nz;
  const int g = grid_for(c, n);
  {
    Prof pr(c, FAS_K_RESIDUAL, level, (double)n);
    k_residual<T, DIM><<<g, kBlock, 0, c->stream>>>(r, u, f, L, nsp, c->partials);
  }
  Prof pr(c, FAS_K_NORM, level, 0.0);
  k_finish_norm<<<1, kBlock, 0, c->stream>>>(c->partials, g, out, nsp);
}

template <typename T, int DIM>
fas_status launch_coarse(fas_ctx* c, Hier<T>& H, int l0, T* utop, const T* ftop) {
  const fas_params& p = c->p;
  if (l0 != H.switch_level) return fail(FAS_ECUDA, "single-CTA kernel launched above its shared-memory level");
  CoarseArgs<T> A;
  A.desc = H.d_desc;
  A.u = H.d_u;
  A.f = H.d_f;
  A.u0 = H.d_u0;
  A.cinv = H.cinv;
  A.l0 = l0;
  A.nlev = H.nlev;
  A.nu1 = p.nu1;
  A.nu2 = p.nu2;
  A.nuc = p.nu_coarse > 0 ? p.nu_coarse : p.nu1;
  A.ordering = p.ordering;
  Prof pr(c, FAS_K_COARSE, l0, (double)c->shape[l0].cells());
  with_fax(c, [&](auto tag) {
    k_coarse_smem<T, DIM, decltype(tag)::value><<<1, kCoarseThreads, H.smem_bytes, c->stream>>>(A, H.smem, utop, ftop);
  });
  return FAS_OK;
}

// Levels lfrom..switch-1 through the per-operation kernels around the single-CTA kernel (any value
// type, 2D or 3D). Level lfrom works on (utop, ftop); deeper levels on the hierarchy's buffers.
template <typename T, int DIM>
fas_status vcycle_basic_from(fas_ctx* c, Hier<T>& H, int lfrom, T* utop, const T* ftop) {
  const fas_params& p = c->p;
  const int sw = H.switch_level;
  for (int l = lfrom; l < sw; ++l) {
    const LevelDesc<T>& L = H.desc[l];
    T* u = l == lfrom ? utop : H.u[l];
    const T* f = l == lfrom ? ftop : H.f[l];
    T* scratch = (DIM == 3 && l < (int)H.u2.size()) ? H.u2[l] : nullptr;  // fused 3D sweeps
    launch_smooth<T, DIM>(c, L, l, u, f, p.nu1, scratch);
    const int64_t n = (int64_t)L.nx * L.ny * L.nz;
    const int64_t nc = n >> DIM;
    {  // residual and its restriction in one pass (the residual is not stored)
      Prof pr(c, FAS_K_RESTRICT, l, (double)n);
      bool blocks = false;  // 3D float32 cell levels: 4 x 2 x 2 fine cells per thread (path 1: one per cell)
      if constexpr (std::is_same<T, float>::value && DIM == 3) {
        if (c->p.path != 1 && L.fax < 0 && !L.per && !L.varkappa && (L.nx & 3) == 0) {
          k_restrict_resid4_3d<<<grid_for(c, nc / 2), kBlock, 0, c->stream>>>(H.u[l + 1], H.u0[l + 1], H.f[l + 1],
                                                                             u, f, L);
          blocks = true;
        }
      }
      if (!blocks) with_fax(c, [&](auto tag) {
        constexpr int FAX = decltype(tag)::value;
        k_restrict_resid<T, DIM, FAX><<<grid_for(c, nc), kBlock, 0, c->stream>>>(H.u[l + 1], H.u0[l + 1],
                                                                                 H.f[l + 1], u, f, L);
      });
    }
    {
      Prof pr(c, FAS_K_TAU, l + 1, (double)nc);
      const LevelDesc<T>& Lc = H.desc[l + 1];
      bool groups = false;  // 3D float32 cell levels: 4 cells per thread (path 1: one per cell)
      if constexpr (std::is_same<T, float>::value && DIM == 3) {
        if (c->p.path != 1 && Lc.fax < 0 && !Lc.per && !Lc.varkappa && (Lc.nx & 3) == 0) {
          k_tau4_3d<<<grid_for(c, nc / 4), kBlock, 0, c->stream>>>(H.f[l + 1], H.u[l + 1], Lc);
          groups = true;
        }
      }
      if (!groups) k_tau<T, DIM><<<grid_for(c, nc), kBlock, 0, c->stream>>>(H.f[l + 1], H.u[l + 1], Lc);
    }
  }
  STATUS_TRY((launch_coarse<T, DIM>(c, H, sw, sw == lfrom ? utop : H.u[sw], sw == lfrom ? ftop : H.f[sw])));
  for (int l = sw - 1; l >= lfrom; --l) {
    const LevelDesc<T>& L = H.desc[l];
    T* u = l == lfrom ? utop : H.u[l];
    const T* f = l == lfrom ? ftop : H.f[l];
    const int64_t n = (int64_t)L.nx * L.ny * L.nz;
    {
      Prof pr(c, FAS_K_PROLONG, l, (double)n);
      launch_prolong<T, DIM>(c, n, u, H.u[l + 1], H.u0[l + 1], L.nx, L.ny, L.nz);
    }
    launch_smooth<T, DIM>(c, L, l, u, f, p.nu2, (DIM == 3 && l < (int)H.u2.size()) ? H.u2[l] : nullptr);
  }
  return FAS_OK;
}

// Rows per warp segment of the fused kernels on a level: a multiple of 8 (row pairs stay aligned),
// chosen so that the level's strips x segments fill about one wave of 16 warps per SM (shorter
// segments recompute more halo rows, longer ones leave SMs idle), at most 128; seg_rows overrides.
int seg_for_level(const fas_ctx* c, int nx, int ny) {
  if (c->p.seg_rows > 0) return std::max(8, (c->p.seg_rows + 7) / 8 * 8);
  const int64_t nstrips = (nx + kStripOut - 1) / kStripOut;
  const int64_t target = (int64_t)c->sm_count * 16;
  const int64_t seg = ((int64_t)ny * nstrips + target - 1) / target;  // rounded up: at most one wave
  return (int)std::max<int64_t>(8, std::min<int64_t>(128, (seg + 7) / 8 * 8));
}

// One float32 V-cycle through the sweep-fused 2D kernels on levels 0..nfast-1 (ping-pong buffers u/u2,
// R(r) in rc), the per-operation tau kernel and the single-CTA kernel below. Result in H.u[0].
// zero_init: the level-0 initial guess is 0 (H.u[0] is not read).
// u64 (nullable): add the result to this float64 field instead of storing it in H.u[0].
fas_status vcycle_fast(fas_ctx* c, Hier<float>& H, bool zero_init, double* u64) {
  const fas_params& p = c->p;
  const int nf = H.nfast;
  for (int l = 0; l < nf; ++l) {
    const LevelDesc<float>& L = H.desc[l];
    const int seg = seg_for_level(c, L.nx, L.ny);
    const bool tau = l > 0;
    float* rc_next = (l + 1 == nf) ? H.f[l + 1] : H.rc[l + 1];
    Prof pr(c, FAS_K_SMOOTH, l, (double)c->shape[l].cells());
    cudaError_t e = launch_stream2d_pre(H.u[l], tau ? H.rc[l] : H.f[l], tau ? H.f[l] : nullptr, H.u2[l], H.u[l + 1],
                                        rc_next, L, p.nu1, l == 0 && zero_init, tau, seg, c->stream);
    if (e != cudaSuccess) return fail(FAS_ECUDA, std::string("stream2d pre: ") + cudaGetErrorString(e));
  }
  {
    const int64_t nc = c->shape[nf].cells();
    Prof pr(c, FAS_K_TAU, nf, (double)nc);
    k_tau<float, 2><<<grid_for(c, nc), kBlock, 0, c->stream>>>(H.f[nf], H.u[nf], H.desc[nf]);
  }
  // levels between the fused ones and the single-CTA level (narrow grids), then the small levels
  STATUS_TRY((vcycle_basic_from<float, 2>(c, H, nf, H.u[nf], H.f[nf])));
  for (int l = nf - 1; l >= 0; --l) {
    const LevelDesc<float>& L = H.desc[l];
    const int seg = seg_for_level(c, L.nx, L.ny);
    // the level-0 launch that also adds the result to the float64 solution is timed as an update
    Prof pr(c, (l == 0 && u64) ? FAS_K_UPDATE : FAS_K_PROLONG, l, (double)c->shape[l].cells());
    cudaError_t e = launch_stream2d_post(H.u2[l], H.f[l], H.u[l + 1], H.u[l], l == 0 ? u64 : nullptr, L, p.nu2, seg,
                                         c->stream);
    if (e != cudaSuccess) return fail(FAS_ECUDA, std::string("stream2d post: ") + cudaGetErrorString(e));
  }
  return FAS_OK;
}

template <typename T>
fas_status vcycle(fas_ctx* c, Hier<T>& H, T* u, const T* f) {
  if (c->p.dim == 2) return vcycle_basic_from<T, 2>(c, H, 0, u, f);
  return vcycle_basic_from<T, 3>(c, H, 0, u, f);
}

fas_status sync_read(fas_ctx* c, double* out) {
  CUDA_TRY(cudaMemcpyAsync(c->h_scalar, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  CUDA_TRY(cudaGetLastError());
  *out = c->h_scalar[0];
  return FAS_OK;
}

// ---------------------------------------------------------------------------------------------
// norms and the solve loop (Algorithm 1's outer loop). The stopping decision is computed on the
// device (SolveState); the host loop reads it after each cycle, the graph's while node reads it
// through its conditional handle.
// ---------------------------------------------------------------------------------------------

// ||x||_2 of a float64 level-0 field into *out (device), squares of the float-rounded values
void enqueue_norm(fas_ctx* c, const double* x, const float* nsp, double* out) {
  const int64_t n = c->shape[0].cells();
  const int g = grid_for(c, n);
  {
    Prof pr(c, FAS_K_NORM, 0, (double)n);
    k_norm2<double><<<g, kBlock, 0, c->stream>>>(x, n, nsp, c->partials);
  }
  Prof pr(c, FAS_K_NORM, 0, 0.0);
  k_finish_norm<<<1, kBlock, 0, c->stream>>>(c->partials, g, out, nsp);
}

// ||b - A u||_2 into *out; mixed precision also leaves r32 = (float)(b - A u) in h32.f[0]
// r32 = (float)(b - A u) on level 0 with per-block partials of its (nsp-scaled) squares; returns the
// number of partials.
int launch_ir_residual(fas_ctx* c, float* r32, const double* u, const double* b, const float* nsp) {
  const LevelDesc<double>& L = c->h64.desc[0];
  const int64_t n = c->shape[0].cells();
  int g = grid_for(c, n);
  Prof pr(c, FAS_K_IR, 0, (double)n);
  if (ir_strip_supported(L) &&
      launch_ir_strip(r32, u, b, L, nsp, c->partials, c->ir_ticket, c->sm_count, c->max_blocks, &g, c->stream,
                      Ir3Wait{g_wait_limit_ns.load(), take_withhold(1)}) == cudaSuccess)
    ;  // the strip kernels took the level
  else if (c->p.dim == 2)
    k_ir_residual<2><<<g, kBlock, 0, c->stream>>>(r32, u, b, L, nsp, c->partials);
  else
    k_ir_residual<3><<<g, kBlock, 0, c->stream>>>(r32, u, b, L, nsp, c->partials);
  return g;
}

void enqueue_residual_norm(fas_ctx* c, const double* u, const double* b, const float* nsp, double* out) {
  if (c->p.precision == FAS_MIXED) {
    const int g = launch_ir_residual(c, c->h32.f[0], u, b, nsp);
    Prof pr(c, FAS_K_NORM, 0, 0.0);
    k_finish_norm<<<1, kBlock, 0, c->stream>>>(c->partials, g, out, nsp);
  } else if (c->p.dim == 2) {
    launch_residual<double, 2>(c, c->h64.desc[0], 0, nullptr, u, b, nsp, out);
  } else {
    launch_residual<double, 3>(c, c->h64.desc[0], 0, nullptr, u, b, nsp, out);
  }
}

void enqueue_remove_mean(fas_ctx* c, double* x, const double* y) {
  const int64_t n = c->shape[0].cells();
  const int g = grid_for(c, n);
  {
    Prof pr(c, FAS_K_NORM, 0, (double)n);
    k_sum<double><<<g, kBlock, 0, c->stream>>>(y, n, c->partials);
  }
  {
    Prof pr(c, FAS_K_NORM, 0, 0.0);
    k_finish_sum<<<1, kBlock, 0, c->stream>>>(c->partials, g, c->d_scalar + 1);
  }
  Prof pr(c, FAS_K_OTHER, 0, (double)n);
  k_sub_mean<double><<<g, kBlock, 0, c->stream>>>(x, y, n, c->d_scalar + 1);
}

// One refinement step of the mixed solver: r32 (h32.f[0]) holds b - A u on entry; float32 V-cycles on
// A e = r32 from e = 0, then u += e in float64.
fas_status mixed_step(fas_ctx* c, double* u) {
  const int64_t n = c->shape[0].cells();
  const int inner = c->p.inner_cycles > 0 ? c->p.inner_cycles : 1;
  Hier<float>& H = c->h32;
  if (H.nfast > 0) {
    // the last cycle's post-smoothing kernel adds its result to u in float64
    for (int k = 0; k < inner; ++k) STATUS_TRY(vcycle_fast(c, H, k == 0, k == inner - 1 ? u : nullptr));
  } else {
    CUDA_TRY(cudaMemsetAsync(H.u[0], 0, n * sizeof(float), c->stream));
    for (int k = 0; k < inner; ++k) STATUS_TRY(vcycle<float>(c, H, H.u[0], H.f[0]));
    Prof pr(c, FAS_K_UPDATE, 0, (double)n);
    k_ir_update<<<grid_for(c, (n + 3) / 4), kBlock, 0, c->stream>>>(u, H.u[0], n);
  }
  return FAS_OK;
}

// The right-hand side the solve works with (the mean-free copy for singular problems).
const double* solve_rhs(fas_ctx* c, const double* f) { return c->singular ? c->fproj : f; }

// Enqueue everything before the first cycle. fn_ready: S->fn already holds ||f|| (heat steps).
fas_status enqueue_prologue(fas_ctx* c, double* u, const double* f_in, bool fn_ready, int max_cycles) {
  const fas_params& p = c->p;
  SolveState* S = c->S;
  const double* f = solve_rhs(c, f_in);
  if (c->singular) {
    enqueue_remove_mean(c, c->fproj, f_in);
    fn_ready = false;
  }
  if (!fn_ready) enqueue_norm(c, f, nullptr, &S->fn);
  const double w = p.tol_relative ? 1.0 : std::pow(c->shape[0].h, p.dim / 2.0);  // Eq. residual weight
  {
    Prof pr(c, FAS_K_OTHER, 0, 0.0);
    k_solve_begin<<<1, 1, 0, c->stream>>>(S, p.tol, max_cycles, w, (double)c->shape[0].cells());
  }
  enqueue_residual_norm(c, u, f, &S->nscale, &S->res0);
  Prof pr(c, FAS_K_OTHER, 0, 0.0);
  k_solve_ref<<<1, 1, 0, c->stream>>>(S, p.tol_relative);
  return FAS_OK;
}

// Enqueue one cycle, its residual norm and the stopping decision.
fas_status enqueue_body(fas_ctx* c, double* u, const double* f_in, cudaGraphConditionalHandle h, int set_cond) {
  const double* f = solve_rhs(c, f_in);
  if (c->p.precision == FAS_MIXED) {
    STATUS_TRY(mixed_step(c, u));
  } else {
    STATUS_TRY(vcycle<double>(c, c->h64, u, f));
  }
  if (c->singular) enqueue_remove_mean(c, u, u);
  enqueue_residual_norm(c, u, f, &c->S->nscale, &c->S->res);
  Prof pr(c, FAS_K_OTHER, 0, 0.0);
  k_solve_step<<<1, 1, 0, c->stream>>>(c->S, h, set_cond);
  return FAS_OK;
}

// Enqueue the read-back of the refinement residual's timeout word (the host copy is valid after the
// stream is synchronised; check_timeout reads it).
cudaError_t enqueue_timeout_read(fas_ctx* c, cudaStream_t st) {
  return cudaMemcpyAsync(c->h_flag, c->ir_ticket + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
}

// FAS_ETIMEOUT (and the word cleared) when a bounded wait of a kernel ran out since the last check.
fas_status check_timeout(fas_ctx* c, cudaStream_t st) {
  if (*c->h_flag == 0u) return FAS_OK;
  *c->h_flag = 0u;
  CUDA_TRY(cudaMemsetAsync(c->ir_ticket + 2, 0, sizeof(unsigned), st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return fail(FAS_ETIMEOUT, "a bounded wait for a tile copy ran out in the refinement residual");
}

fas_status read_state(fas_ctx* c) {
  CUDA_TRY(cudaMemcpyAsync(c->Sh, c->S, sizeof(SolveState), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(enqueue_timeout_read(c, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  CUDA_TRY(cudaGetLastError());
  return check_timeout(c, c->stream);
}

fas_status finish_info(fas_ctx* c, fas_info* info, int max_cycles) {
  const SolveState& S = *c->Sh;
  fas_info loc;
  std::memset(&loc, 0, sizeof(loc));
  loc.cycles = S.cycles;
  loc.converged = S.converged;
  loc.res0 = S.w * S.res0;
  loc.res = S.w * S.res;
  loc.rel = S.ref > 0.0 ? loc.res / S.ref : 0.0;
  loc.rho = (loc.cycles > 0 && loc.res0 > 0.0) ? std::pow(loc.res / loc.res0, 1.0 / loc.cycles) : 0.0;
  if (info) *info = loc;
  if (S.nonfinite) return fail(FAS_ENONFINITE, "fas_solve: residual is not finite");
  if (!S.converged && max_cycles == c->p.kmax)
    return fail(FAS_ENOTCONV, "fas_solve: tolerance not reached within kmax cycles");
  return FAS_OK;
}

// ---- the whole solve as one CUDA graph: prologue, then a while node whose body is one cycle ----

struct CaptureScope {  // switches the launch helpers to counting-only (no event records) while capturing
  fas_ctx* c;
  long long start;
  explicit CaptureScope(fas_ctx* ctx) : c(ctx), start(ctx->launches) { c->capturing = true; }
  long long count() const { return c->launches - start; }
  ~CaptureScope() { c->capturing = false; }
};

void destroy_graphs(fas_ctx* c) {
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  c->graphs.clear();
}

// Build (or find) the graph of a solve of u for f; kind 1 also forms the heat right-hand side
// b = u + dt fsrc (f = c->b) with its norm at the start.
fas_status solve_graph(fas_ctx* c, double* u, const double* f, const double* fsrc, double dt, int kind,
                       SolveGraph** out) {
  for (auto& g : c->graphs)
    if (g.u == u && g.f == f && g.fsrc == fsrc && g.dt == dt && g.kind == kind) {
      *out = &g;
      return FAS_OK;
    }
  SolveGraph g;
  g.u = u;
  g.f = f;
  g.fsrc = fsrc;
  g.dt = dt;
  g.kind = kind;
  CUDA_TRY(cudaGraphCreate(&g.graph, 0));
  // captured on the context's private streams (the caller's stream may be the legacy default stream,
  // which cannot be captured); the instantiated graph is launched on the caller's stream
  cudaStream_t user = c->stream;
  cudaStream_t main = c->side;
  fas_status st = FAS_OK;
  {
    CaptureScope cap(c);
    c->stream = main;
    cudaError_t eb = cudaStreamBeginCaptureToGraph(main, g.graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (eb != cudaSuccess) {
      c->stream = user;
      cudaGraphDestroy(g.graph);
      return fail(FAS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(eb));
    }
    const int64_t n = c->shape[0].cells();
    if (kind == 1) {
      const int gb = grid_for(c, n);
      {
        Prof pr(c, FAS_K_OTHER, 0, (double)n);
        k_heat_rhs<<<gb, kBlock, 0, main>>>(c->b, u, fsrc, dt, n, c->partials);
      }
      Prof pr(c, FAS_K_NORM, 0, 0.0);
      k_finish_norm<<<1, kBlock, 0, main>>>(c->partials, gb, &c->S->fn, nullptr);
    }
    st = enqueue_prologue(c, u, f, kind == 1, c->p.kmax);
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphConditionalHandle h = 0;
    cudaGraphNode_t cond_node = nullptr;
    cudaGraph_t body = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(main, &cs, nullptr, &cg, &deps, nullptr, &nd);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g.graph, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      e = cudaGraphAddNode(&cond_node, cg, deps, nullptr, nd, &np);
      if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(main, &cond_node, nullptr, 1, cudaStreamSetCaptureDependencies);
    cudaError_t e2 = cudaStreamEndCapture(main, &g.graph);
    if (e != cudaSuccess || e2 != cudaSuccess || st != FAS_OK) {
      c->stream = user;
      cudaGraphDestroy(g.graph);
      return st != FAS_OK ? st : fail(FAS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    g.n_pro = cap.count();
    // the while node's body: one cycle, its residual norm, the decision
    const long long before = c->launches;
    e = cudaStreamBeginCaptureToGraph(c->side2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      c->stream = user;
      cudaGraphDestroy(g.graph);
      return fail(FAS_ECUDA, std::string("graph body capture: ") + cudaGetErrorString(e));
    }
    c->stream = c->side2;
    st = enqueue_body(c, u, f, h, 1);
    c->stream = user;
    cudaGraph_t body_out = body;
    e = cudaStreamEndCapture(c->side2, &body_out);
    if (e != cudaSuccess || st != FAS_OK) {
      cudaGraphDestroy(g.graph);
      return st != FAS_OK ? st : fail(FAS_ECUDA, std::string("graph body capture: ") + cudaGetErrorString(e));
    }
    g.n_body = c->launches - before;
  }
  c->launches -= g.n_pro + g.n_body;  // counted when the graph runs
  cudaError_t e = cudaGraphInstantiate(&g.exec, g.graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g.graph);
    return fail(FAS_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  c->graphs.push_back(g);
  *out = &c->graphs.back();
  return FAS_OK;
}

// fn_ready: S->fn already holds ||f|| (set by the heat right-hand side kernel)
fas_status solve_impl(fas_ctx* c, double* u, const double* f, fas_info* info, int max_cycles,
                      bool fn_ready = false) {
  const bool graph = c->p.use_graph && !c->prof && max_cycles == c->p.kmax;
  if (graph) {
    SolveGraph* g = nullptr;
    STATUS_TRY(solve_graph(c, u, f, nullptr, 0.0, 0, &g));
    CUDA_TRY(cudaGraphLaunch(g->exec, c->stream));
    STATUS_TRY(read_state(c));
    c->launches += g->n_pro + (long long)c->Sh->cycles * g->n_body;
    return finish_info(c, info, max_cycles);
  }
  STATUS_TRY(enqueue_prologue(c, u, f, fn_ready, max_cycles));
  for (int k = 0; k < max_cycles; ++k) {
    STATUS_TRY(enqueue_body(c, u, f, 0, 0));
    STATUS_TRY(read_state(c));
    if (!c->Sh->cond) break;
  }
  CUDA_TRY(cudaGetLastError());
  return finish_info(c, info, max_cycles);
}

// ---------------------------------------------------------------------------------------------
// batched solves: one graph, one branch per problem
// ---------------------------------------------------------------------------------------------

__global__ void k_copy_state(SolveState* dst, const SolveState* src) { *dst = *src; }

struct BatchGraph {
  std::vector<fas_ctx*> ctxs;
  std::vector<double*> u;
  std::vector<const double*> f;
  std::vector<long long> n_pro, n_body;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  SolveState* d_states = nullptr;
  SolveState* h_states = nullptr;
};

std::mutex g_batch_mutex;
std::vector<BatchGraph*> g_batches;  // built batch graphs, dropped when one of their contexts is destroyed

void free_batch(BatchGraph* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_states) cudaFree(b->d_states);
  if (b->h_states) cudaFreeHost(b->h_states);
  delete b;
}

void drop_batches_of(const fas_ctx* c) {
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  for (size_t k = 0; k < g_batches.size();) {
    BatchGraph* b = g_batches[k];
    if (std::find(b->ctxs.begin(), b->ctxs.end(), c) != b->ctxs.end()) {
      free_batch(b);
      g_batches.erase(g_batches.begin() + k);
    } else {
      ++k;
    }
  }
}

fas_status build_batch(BatchGraph* B) {
  const int n = (int)B->ctxs.size();
  CUDA_TRY(cudaMalloc(&B->d_states, n * sizeof(SolveState)));
  CUDA_TRY(cudaMallocHost(&B->h_states, n * sizeof(SolveState)));
  CUDA_TRY(cudaGraphCreate(&B->graph, 0));
  cudaStream_t org = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins(n, nullptr);
  std::vector<cudaGraph_t> bodies(n, nullptr);
  std::vector<cudaGraphConditionalHandle> handles(n, 0);
  B->n_pro.assign(n, 0);
  B->n_body.assign(n, 0);
  fas_status st = FAS_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&org, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(org, B->graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(fork, org);
  // prologue and while node of every problem, each on its own context's capture stream
  for (int i = 0; i < n && e == cudaSuccess && st == FAS_OK; ++i) {
    fas_ctx* c = B->ctxs[i];
    cudaStream_t sv = c->stream;
    cudaStream_t cs = c->side;
    e = cudaStreamWaitEvent(cs, fork, 0);
    if (e != cudaSuccess) break;
    c->stream = cs;
    {
      CaptureScope cap(c);
      st = enqueue_prologue(c, B->u[i], B->f[i], false, c->p.kmax);
      B->n_pro[i] = cap.count() + 1;  // + the state copy below
    }
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphNode_t cond_node = nullptr;
    if (st == FAS_OK) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd);
    if (st == FAS_OK && e == cudaSuccess)
      e = cudaGraphConditionalHandleCreate(&handles[i], B->graph, 1, cudaGraphCondAssignDefault);
    if (st == FAS_OK && e == cudaSuccess) {
      cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
      np.conditional.handle = handles[i];
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      e = cudaGraphAddNode(&cond_node, cg, deps, nullptr, nd, &np);
      if (e == cudaSuccess) bodies[i] = np.conditional.phGraph_out[0];
    }
    if (st == FAS_OK && e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(cs, &cond_node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (st == FAS_OK && e == cudaSuccess) {
      k_copy_state<<<1, 1, 0, cs>>>(B->d_states + i, c->S);
      e = cudaEventRecord(joins[i], cs);
    }
    if (st == FAS_OK && e == cudaSuccess) e = cudaStreamWaitEvent(org, joins[i], 0);
    c->stream = sv;
  }
  cudaGraph_t g_out = B->graph;
  cudaError_t e2 = cudaStreamEndCapture(org, &g_out);
  if (e == cudaSuccess) e = e2;
  // bodies: one cycle, its residual norm and the decision, per problem
  for (int i = 0; i < n && e == cudaSuccess && st == FAS_OK; ++i) {
    fas_ctx* c = B->ctxs[i];
    cudaStream_t sv = c->stream;
    e = cudaStreamBeginCaptureToGraph(c->side2, bodies[i], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    c->stream = c->side2;
    {
      CaptureScope cap(c);
      st = enqueue_body(c, B->u[i], B->f[i], handles[i], 1);
      B->n_body[i] = cap.count();
    }
    c->stream = sv;
    cudaGraph_t b_out = bodies[i];
    e2 = cudaStreamEndCapture(c->side2, &b_out);
    if (e == cudaSuccess) e = e2;
  }
  for (int i = 0; i < n; ++i) B->ctxs[i]->launches -= B->n_pro[i] - 1 + B->n_body[i];  // counted at run time
  if (e == cudaSuccess && st == FAS_OK) e = cudaGraphInstantiate(&B->exec, B->graph, 0);
  for (auto ev : joins)
    if (ev) cudaEventDestroy(ev);
  if (fork) cudaEventDestroy(fork);
  if (org) cudaStreamDestroy(org);
  if (st != FAS_OK) return st;
  if (e != cudaSuccess) return fail(FAS_ECUDA, std::string("batched graph: ") + cudaGetErrorString(e));
  return FAS_OK;
}

// ---------------------------------------------------------------------------------------------
// autotuning: launch parameters chosen by timing whole solves, cached per size class
// ---------------------------------------------------------------------------------------------

struct TuneKey {
  int dim, nx, ny, nz, precision;
  bool operator==(const TuneKey& o) const {
    return dim == o.dim && nx == o.nx && ny == o.ny && nz == o.nz && precision == o.precision;
  }
};
struct TuneEntry {
  TuneKey key;
  fas_tune_result res;
};
std::mutex g_tune_mutex;
std::vector<TuneEntry> g_tune_cache;

fas_status check_ctx(const fas_ctx* c) {
  if (!c) return fail(FAS_EINVAL, "null context");
  return FAS_OK;
}

// A device field pointer: non-null where required, and 16-byte aligned (the kernels move fields in
// 16-byte vectors; a misaligned vector access would fault).
fas_status check_field(const void* p, bool required, const char* where) {
  if (!p) return required ? fail(FAS_EINVAL, std::string(where) + ": null field") : FAS_OK;
  if (reinterpret_cast<uintptr_t>(p) & 15u) return fail(FAS_EINVAL, std::string(where) + ": field not 16-byte aligned");
  return FAS_OK;
}

fas_status check_level(const fas_ctx* c, int level, bool needs_coarser) {
  STATUS_TRY(check_ctx(c));
  if (level < 0 || level >= c->nlev || (needs_coarser && level + 1 >= c->nlev))
    return fail(FAS_EINVAL, "level out of range");
  return FAS_OK;
}

// dst[i] = src[i], 16 bytes per thread and step (both 16-byte aligned, n even handled by the tail)
__global__ void k_copy_f64(double* __restrict__ dst, const double* __restrict__ src, int64_t n) {
  const int64_t n2 = n / 2;
  const double2* s2 = reinterpret_cast<const double2*>(src);
  double2* d2 = reinterpret_cast<double2*>(dst);
  for (int64_t i = gtid(); i < n2; i += gstride()) d2[i] = s2[i];
  if (gtid() == 0 && (n & 1)) dst[n - 1] = src[n - 1];
}

// f += 2 beta kappa_c g / h^2 on the cells next to each Dirichlet face with value g (dmask bit k:
// face k is Dirichlet), faces added in the order z, y, x, low side first.
struct FaceValues {
  double g[6];
};
__global__ void k_fold_dirichlet(double* __restrict__ f, const double* __restrict__ kappa, double kconst, double scale,
                                 int nx, int ny, int nz, FaceValues gv, int dmask) {
  const int64_t n = (int64_t)nx * ny * nz;
  for (int64_t idx = gtid(); idx < n; idx += gstride()) {
    const int i = (int)(idx % nx);
    const int64_t r = idx / nx;
    const int j = (int)(r % ny);
    const int l = (int)(r / ny);
    const bool edge = i == 0 || i == nx - 1 || j == 0 || j == ny - 1 || (nz > 1 && (l == 0 || l == nz - 1));
    if (!edge) continue;
    // product, then sum, each rounded (no contraction into an fma)
    const double sk = __dmul_rn(scale, kappa ? kappa[idx] : kconst);
    double v = f[idx];
    if (nz > 1) {
      if (l == 0 && (dmask & 16)) v = __dadd_rn(v, __dmul_rn(sk, gv.g[4]));
      if (l == nz - 1 && (dmask & 32)) v = __dadd_rn(v, __dmul_rn(sk, gv.g[5]));
    }
    if (j == 0 && (dmask & 4)) v = __dadd_rn(v, __dmul_rn(sk, gv.g[2]));
    if (j == ny - 1 && (dmask & 8)) v = __dadd_rn(v, __dmul_rn(sk, gv.g[3]));
    if (i == 0 && (dmask & 1)) v = __dadd_rn(v, __dmul_rn(sk, gv.g[0]));
    if (i == nx - 1 && (dmask & 2)) v = __dadd_rn(v, __dmul_rn(sk, gv.g[1]));
    f[idx] = v;
  }
}

// The device address of a host buffer the GPU may access directly (page-locked and mapped under
// unified addressing), or nullptr.
const void* mapped_host(const void* h) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();  // pageable memory may report an error on older drivers: clear it
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// n float64 values between a HOST buffer and a device buffer of the context, on its stream. Where the
// host buffer is page-locked and mapped (and 16-byte aligned), the GPU copies it with its own loads
// and stores over the host link, which moves data faster than one copy-engine transfer; otherwise a
// cudaMemcpyAsync.
cudaError_t copy_host(fas_ctx* c, void* dst, const void* src, int64_t n, bool to_device) {
  const void* h = to_device ? src : dst;
  const void* hd = mapped_host(h);
  if (hd && !(reinterpret_cast<uintptr_t>(hd) & 15u)) {
    const int g = grid_for(c, (n + 1) / 2);
    if (to_device)
      k_copy_f64<<<g, kBlock, 0, c->stream>>>(static_cast<double*>(dst), static_cast<const double*>(hd), n);
    else
      k_copy_f64<<<g, kBlock, 0, c->stream>>>(static_cast<double*>(const_cast<void*>(hd)),
                                               static_cast<const double*>(src), n);
    return cudaGetLastError();
  }
  return cudaMemcpyAsync(dst, src, n * sizeof(double), to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                         c->stream);
}

}  // namespace

void fasmg::set_last_error(const std::string& msg) { g_last_error = msg; }

// =============================================================================================
// C ABI
// =============================================================================================

// The single-CTA kernel's dynamic shared memory limit, for every unknown location.
template <typename T, int DIM>
cudaError_t coarse_attr() {
  cudaError_t e = cudaSuccess;
  for (cudaError_t ek : {cudaFuncSetAttribute(k_coarse_smem<T, DIM, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kCoarseSmemLimit),
                         cudaFuncSetAttribute(k_coarse_smem<T, DIM, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kCoarseSmemLimit),
                         cudaFuncSetAttribute(k_coarse_smem<T, DIM, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kCoarseSmemLimit),
                         cudaFuncSetAttribute(k_coarse_smem<T, DIM, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kCoarseSmemLimit)})
    if (e == cudaSuccess) e = ek;
  return e;
}

// Pseudo-random 64-bit patterns for the conversion self-test (SplitMix64 in counter mode).
__device__ __forceinline__ uint64_t st_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ bool same_or_both_nan_f(float a, float b) {
  return __float_as_uint(a) == __float_as_uint(b) || (a != a && b != b);
}

__device__ __forceinline__ bool same_or_both_nan_d(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b) || (a != a && b != b);
}

// For each k: a raw 64-bit pattern, a double in and around float32's exponent range (random, exact
// tie and tie +- 1 significands), and the low 32 bits as a float; both conversions of each checked
// against the hardware ones.
static __global__ void k_selftest_conv(long long count, unsigned long long seed, unsigned long long* bad) {
  unsigned long long nbad = 0;
  for (long long k = gtid(); k < count; k += gstride()) {
    const uint64_t z = st_mix(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(k + 1));
    const uint64_t z2 = st_mix(z ^ 0xD1B54A32D192ED03ull);
    uint64_t pats[4];
    pats[0] = z;
    const uint64_t E = 896 - 40 + (z2 % 300);  // float32 subnormals up to overflow
    const uint64_t sign = z2 & (1ull << 63);
    const uint64_t hiM = z & (((1ull << 23) - 1) << 29);
    pats[1] = sign | (E << 52) | (z & kMant52);
    pats[2] = sign | (E << 52) | hiM | (1ull << 28);                     // exact tie at float precision
    pats[3] = sign | (E << 52) | hiM | ((1ull << 28) + ((z2 >> 8) & 1 ? 1 : -1));
    for (int q = 0; q < 4; ++q) {
      const double d = __longlong_as_double((long long)pats[q]);
      if (!same_or_both_nan_f(f64_to_f32_rn_bits(d), __double2float_rn(d))) ++nbad;
      if (f32_normal_range(d) && !same_or_both_nan_f(f64_to_f32_rn_normal(d), __double2float_rn(d))) ++nbad;
    }
    const float fx = __uint_as_float((uint32_t)z);
    const float fy = __uint_as_float((uint32_t)(z2 >> 32) & 0x807FFFFFu);  // float32 subnormals
    if (!same_or_both_nan_d(f32_to_f64_bits(fx), (double)fx)) ++nbad;
    if (!same_or_both_nan_d(f32_to_f64_bits(fy), (double)fy)) ++nbad;
  }
  if (nbad) atomicAdd(bad, nbad);
}

static __global__ void k_selftest_specials(unsigned long long* bad) {
  const uint64_t dpat[] = {0ull, 1ull << 63, 0x7FF0000000000000ull, 0xFFF0000000000000ull, 0x7FF8000000000000ull,
                           0x47EFFFFFE0000000ull, 0x47EFFFFFF0000000ull, 0x47EFFFFFEFFFFFFFull,
                           0x3690000000000000ull, 0x3680000000000000ull, 0x3680000000000001ull,
                           0x36A0000000000000ull, 0x380FFFFFF0000000ull, 0x0000000000000001ull,
                           0x3FF0000000000000ull, 0xBFF0000010000000ull};
  const uint32_t fpat[] = {0u, 0x80000000u, 0x7F800000u, 0xFF800000u, 0x7FC00000u, 0x00000001u, 0x007FFFFFu,
                           0x00800000u, 0x7F7FFFFFu, 0x3F800000u, 0x80000001u, 0x00400000u};
  unsigned long long nbad = 0;
  for (uint64_t p : dpat) {
    const double d = __longlong_as_double((long long)p);
    if (!same_or_both_nan_f(f64_to_f32_rn_bits(d), __double2float_rn(d))) ++nbad;
    if (f32_normal_range(d) && !same_or_both_nan_f(f64_to_f32_rn_normal(d), __double2float_rn(d))) ++nbad;
  }
  for (uint32_t p : fpat) {
    const float f = __uint_as_float(p);
    if (!same_or_both_nan_d(f32_to_f64_bits(f), (double)f)) ++nbad;
  }
  *bad += nbad;
}

extern "C" {

void fas_default_params(fas_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->dim = 2;
  p->n[0] = p->n[1] = p->n[2] = 64;
  p->h = 1.0 / 64;
  p->alpha = 1.0;
  p->beta = 1.0;
  p->kappa = nullptr;
  p->kappa_const = 1.0;
  for (int k = 0; k < 6; ++k) p->bc[k] = FAS_BC_NEUMANN;
  p->nu1 = 2;
  p->nu2 = 2;
  p->nu_coarse = 0;
  p->kmax = 20;
  p->coarsest = 4;
  p->coarse_exact = 0;
  p->tol = 1e-10;
  p->tol_relative = 1;
  p->precision = FAS_FP64;
  p->inner_cycles = 1;
  p->use_graph = 1;
  p->path = 0;
  p->seg_rows = 0;
  p->location = FAS_CELL;
  p->ordering = FAS_ORDER_FORWARD;
}

fas_status fas_create(const fas_params* pin, void* stream, fas_ctx** out) {
  if (!pin || !out) return fail(FAS_EINVAL, "fas_create: null argument");
  *out = nullptr;
  const fas_params& p = *pin;
  if (p.dim != 2 && p.dim != 3) return fail(FAS_EINVAL, "dim must be 2 or 3");
  for (int a = 0; a < p.dim; ++a)
    if (!is_pow2(p.n[a]) || p.n[a] < 2) return fail(FAS_EINVAL, "every n must be a power of two >= 2");
  if (!(p.h > 0.0) || !std::isfinite(p.h)) return fail(FAS_EINVAL, "h must be positive");
  if (p.nu1 < 0 || p.nu2 < 0 || p.nu1 + p.nu2 < 1) return fail(FAS_EINVAL, "nu1, nu2 must be >= 0, sum >= 1");
  if (p.kmax < 1) return fail(FAS_EINVAL, "kmax must be >= 1");
  if (p.coarsest < 2 || !is_pow2(p.coarsest)) return fail(FAS_EINVAL, "coarsest must be a power of two >= 2");
  if (!(p.tol >= 0.0)) return fail(FAS_EINVAL, "tol must be >= 0");
  if (p.alpha < 0.0 || !(p.beta > 0.0)) return fail(FAS_EINVAL, "alpha must be >= 0 and beta > 0");
  if (!p.kappa && !(p.kappa_const > 0.0)) return fail(FAS_EINVAL, "kappa_const must be positive");
  STATUS_TRY(check_field(p.kappa, false, "fas_create (kappa)"));
  if (p.precision != FAS_FP64 && p.precision != FAS_MIXED) return fail(FAS_EINVAL, "unknown precision");
  if (p.ordering != FAS_ORDER_FORWARD && p.ordering != FAS_ORDER_SYMMETRIC) return fail(FAS_EINVAL, "unknown ordering");
  if (p.ordering != FAS_ORDER_FORWARD && p.location != FAS_CELL)
    return fail(FAS_EUNSUPPORTED, "the symmetric ordering is for cell-centred unknowns");
  for (int k = 0; k < 2 * p.dim; ++k)
    if (p.bc[k] != FAS_BC_NEUMANN && p.bc[k] != FAS_BC_DIRICHLET && p.bc[k] != FAS_BC_PERIODIC)
      return fail(FAS_EINVAL, "unknown bc kind");
  for (int a = 0; a < p.dim; ++a)
    if ((p.bc[2 * a] == FAS_BC_PERIODIC) != (p.bc[2 * a + 1] == FAS_BC_PERIODIC))
      return fail(FAS_EINVAL, "periodic faces come in pairs: both faces of an axis or neither");
  if (periodic_mask(p) && (p.kappa || p.location != FAS_CELL))
    return fail(FAS_EUNSUPPORTED, "periodic axes: cell-centred unknowns with a constant kappa only");
  if (p.location < FAS_CELL || p.location > p.dim) return fail(FAS_EINVAL, "location must be a cell or a face axis");
  if (p.path < 0 || p.path > 2) return fail(FAS_EINVAL, "path must be 0, 1 or 2");
  if (p.location != FAS_CELL) {
    for (int k = 0; k < 2 * p.dim; ++k)
      if (p.bc[k] != FAS_BC_DIRICHLET) return fail(FAS_EINVAL, "face grids have no-slip walls: bc must be Dirichlet");
    if (p.kappa || p.coarse_exact)
      return fail(FAS_EUNSUPPORTED, "face grids: constant kappa and a smoothed coarsest level only");
  }

  fas_ctx* c = new fas_ctx();
  c->p = p;
  if (c->p.dim == 2) c->p.n[2] = 1;
  if (c->p.inner_cycles < 1) c->p.inner_cycles = 1;
  c->stream = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
  c->max_blocks = c->sm_count * 16;
  bool no_dirichlet = true;  // Neumann and periodic faces leave the constants in the null space
  for (int k = 0; k < 2 * p.dim; ++k) no_dirichlet = no_dirichlet && p.bc[k] != FAS_BC_DIRICHLET;
  c->singular = p.alpha == 0.0 && no_dirichlet;
  // levels: halve every axis while the shortest exceeds `coarsest`
  LevelShape s{p.n[0], p.n[1], p.dim == 3 ? p.n[2] : 1, p.h};
  c->shape.push_back(s);
  auto shortest = [&](const LevelShape& q) { return p.dim == 3 ? std::min({q.nx, q.ny, q.nz}) : std::min(q.nx, q.ny); };
  while (shortest(c->shape.back()) > p.coarsest && (int)c->shape.size() < kMaxLevels) {
    LevelShape q = c->shape.back();
    q.nx /= 2;
    q.ny /= 2;
    if (p.dim == 3) q.nz /= 2;
    q.h *= 2.0;
    c->shape.push_back(q);
  }
  c->nlev = (int)c->shape.size();
  fas_status st = FAS_OK;
  auto bail = [&](fas_status s2) {
    fas_destroy(c);
    return s2;
  };
  if (cudaMalloc(&c->partials, c->max_blocks * sizeof(double)) != cudaSuccess) return bail(fail(FAS_ENOMEM, "partials"));
  if (cudaMalloc(&c->d_scalar, 8 * sizeof(double)) != cudaSuccess) return bail(fail(FAS_ENOMEM, "scalars"));
  if (cudaMalloc(&c->ir_ticket, 4 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->ir_ticket, 0, 4 * sizeof(unsigned)) != cudaSuccess)
    return bail(fail(FAS_ENOMEM, "work counter"));
  if (cudaMallocHost(&c->h_flag, sizeof(unsigned)) != cudaSuccess) return bail(fail(FAS_ENOMEM, "pinned flag"));
  *c->h_flag = 0u;
  if (cudaMallocHost(&c->h_scalar, 8 * sizeof(double)) != cudaSuccess) return bail(fail(FAS_ENOMEM, "pinned"));
  if (cudaMalloc(&c->S, sizeof(SolveState)) != cudaSuccess) return bail(fail(FAS_ENOMEM, "solve state"));
  if (cudaMallocHost(&c->Sh, sizeof(SolveState)) != cudaSuccess) return bail(fail(FAS_ENOMEM, "pinned state"));
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(FAS_ECUDA, "capture streams"));
  const bool mixed = p.precision == FAS_MIXED;
  st = build_hier<double>(c, c->h64, !mixed, false);
  if (st != FAS_OK) return bail(st);
  if (mixed) {
    st = build_hier<float>(c, c->h32, true, true);
    if (st != FAS_OK) return bail(st);
  }
  if (c->singular && cudaMalloc(&c->fproj, s.cells() * sizeof(double)) != cudaSuccess)
    return bail(fail(FAS_ENOMEM, "fproj"));
  // kernel attributes, set before any launch or stream capture
  cudaError_t e = stream2d_prepare();
  if (e == cudaSuccess) e = ir_strip_prepare();
  if (e == cudaSuccess) e = sweep3d_prepare();
  for (cudaError_t ek : {coarse_attr<double, 2>(), coarse_attr<double, 3>(), coarse_attr<float, 2>(),
                         coarse_attr<float, 3>()})
    if (e == cudaSuccess) e = ek;
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return bail(fail(FAS_ECUDA, std::string("fas_create: ") + cudaGetErrorString(e)));
  *out = c;
  return FAS_OK;
}

fas_status fas_destroy(fas_ctx* c) {
  if (!c) return FAS_OK;
  drop_batches_of(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_hier(c->h64);
  free_hier(c->h32);
  if (c->partials) cudaFree(c->partials);
  if (c->d_scalar) cudaFree(c->d_scalar);
  if (c->ir_ticket) cudaFree(c->ir_ticket);
  if (c->h_scalar) cudaFreeHost(c->h_scalar);
  if (c->h_flag) cudaFreeHost(c->h_flag);
  if (c->b) cudaFree(c->b);
  if (c->fproj) cudaFree(c->fproj);
  destroy_graphs(c);
  if (c->S) cudaFree(c->S);
  if (c->Sh) cudaFreeHost(c->Sh);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->side2) cudaStreamDestroy(c->side2);
  for (double* q : c->adj) cudaFree(q);
  if (c->host_u) cudaFree(c->host_u);
  if (c->host_f) cudaFree(c->host_f);
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  delete c;
  return FAS_OK;
}

int fas_num_levels(const fas_ctx* c) { return c ? c->nlev : 0; }

fas_status fas_vcycle(fas_ctx* c, double* u, const double* f, fas_info* info) {
  STATUS_TRY(check_ctx(c));
  STATUS_TRY(check_field(u, true, "fas_vcycle"));
  STATUS_TRY(check_field(f, true, "fas_vcycle"));
  return solve_impl(c, u, f, info, 1);
}

fas_status fas_solve(fas_ctx* c, double* u, const double* f, fas_info* info) {
  STATUS_TRY(check_ctx(c));
  STATUS_TRY(check_field(u, true, "fas_solve"));
  STATUS_TRY(check_field(f, true, "fas_solve"));
  return solve_impl(c, u, f, info, c->p.kmax);
}

fas_status fas_heat_run(fas_ctx* c, double* u, const double* fsrc, double dt, int nsteps, fas_info* infos) {
  STATUS_TRY(check_ctx(c));
  if (!u || nsteps < 0) return fail(FAS_EINVAL, "fas_heat_run: bad argument");
  STATUS_TRY(check_field(u, true, "fas_heat_run"));
  STATUS_TRY(check_field(fsrc, false, "fas_heat_run"));
  if (c->p.alpha != 1.0 || std::fabs(c->p.beta - dt) > 1e-15 * std::fabs(dt))
    return fail(FAS_EINVAL, "fas_heat_run: context must have alpha = 1 and beta = dt");
  const int64_t n = c->shape[0].cells();
  if (!c->b) CUDA_TRY(cudaMalloc(&c->b, n * sizeof(double)));
  fas_status worst = FAS_OK;
  const bool graph = c->p.use_graph && !c->prof;
  SolveGraph* g = nullptr;
  if (graph) STATUS_TRY(solve_graph(c, u, c->b, fsrc, dt, 1, &g));
  for (int s = 0; s < nsteps; ++s) {
    fas_info inf;
    fas_status st;
    if (graph) {
      // one graph per time step: b = u + dt fsrc with ||b||, then the solve to tolerance
      CUDA_TRY(cudaGraphLaunch(g->exec, c->stream));
      STATUS_TRY(read_state(c));
      c->launches += g->n_pro + (long long)c->Sh->cycles * g->n_body;
      st = finish_info(c, &inf, c->p.kmax);
    } else {
      const int gb = grid_for(c, n);
      {
        Prof pr(c, FAS_K_OTHER, 0, (double)n);
        k_heat_rhs<<<gb, kBlock, 0, c->stream>>>(c->b, u, fsrc, dt, n, c->partials);
      }
      {
        Prof pr(c, FAS_K_NORM, 0, 0.0);
        k_finish_norm<<<1, kBlock, 0, c->stream>>>(c->partials, gb, &c->S->fn, nullptr);
      }
      st = solve_impl(c, u, c->b, &inf, c->p.kmax, true);
    }
    if (infos) infos[s] = inf;
    if (st != FAS_OK && st != FAS_ENOTCONV) return st;
    if (st == FAS_ENOTCONV) worst = st;
  }
  return worst;
}

fas_status fas_heat_adjoint(fas_ctx* c, const double* u0, const double* fsrc, double dt, int nsteps,
                            const double* dL_duT, double* uT, double* g_u0, double* g_f, double* g_kappa,
                            int ckpt_every) {
  STATUS_TRY(check_ctx(c));
  if (!u0 || !dL_duT || nsteps < 1) return fail(FAS_EINVAL, "fas_heat_adjoint: bad argument");
  for (const void* q : {(const void*)u0, (const void*)fsrc, (const void*)dL_duT, (const void*)uT, (const void*)g_u0,
                        (const void*)g_f, (const void*)g_kappa})
    STATUS_TRY(check_field(q, false, "fas_heat_adjoint"));
  if (c->p.alpha != 1.0 || std::fabs(c->p.beta - dt) > 1e-15 * std::fabs(dt))
    return fail(FAS_EINVAL, "fas_heat_adjoint: context must have alpha = 1 and beta = dt");
  if (c->p.location != FAS_CELL) return fail(FAS_EUNSUPPORTED, "fas_heat_adjoint: cell-centred unknowns only");
  if (periodic_mask(c->p)) return fail(FAS_EUNSUPPORTED, "fas_heat_adjoint: periodic axes are not supported");
  const int64_t n = c->shape[0].cells();
  const size_t bytes = n * sizeof(double);
  const int K = ckpt_every > 0 ? std::min(ckpt_every, nsteps) : nsteps;
  const int nseg = (nsteps + K - 1) / K;
  // buffers: nseg checkpoints, K + 1 segment states, lambda, mu, work
  const size_t need = (size_t)nseg + K + 1 + 3;
  while (c->adj.size() < need) {
    double* q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) return fail(FAS_ENOMEM, "fas_heat_adjoint: buffers");
    c->adj.push_back(q);
  }
  double** ckpt = c->adj.data();
  double** seg = c->adj.data() + nseg;
  double* lam = c->adj[nseg + K + 1];
  double* mu = c->adj[nseg + K + 2];
  double* work = c->adj[nseg + K + 3];
  cudaStream_t st = c->stream;
  fas_status worst = FAS_OK;
  auto step = [&](double* u) -> fas_status {  // one backward-Euler step in place
    fas_info inf;
    fas_status s2 = fas_heat_run(c, u, fsrc, dt, 1, &inf);
    if (s2 == FAS_ENOTCONV) {
      worst = s2;
      return FAS_OK;
    }
    return s2;
  };
  // forward sweep, keeping every K-th state
  CUDA_TRY(cudaMemcpyAsync(work, u0, bytes, cudaMemcpyDeviceToDevice, st));
  for (int k = 0; k < nsteps; ++k) {
    if (k % K == 0) CUDA_TRY(cudaMemcpyAsync(ckpt[k / K], work, bytes, cudaMemcpyDeviceToDevice, st));
    STATUS_TRY(step(work));
  }
  if (uT) CUDA_TRY(cudaMemcpyAsync(uT, work, bytes, cudaMemcpyDeviceToDevice, st));
  // backward sweep
  CUDA_TRY(cudaMemcpyAsync(lam, dL_duT, bytes, cudaMemcpyDeviceToDevice, st));
  if (g_f) CUDA_TRY(cudaMemsetAsync(g_f, 0, bytes, st));
  if (g_kappa) CUDA_TRY(cudaMemsetAsync(g_kappa, 0, bytes, st));
  const LevelShape& s0 = c->shape[0];
  int dirmask = 0;
  for (int fc = 0; fc < 2 * c->p.dim; ++fc) dirmask |= (c->p.bc[fc] == FAS_BC_DIRICHLET) << fc;
  const double scale = c->p.beta / (s0.h * s0.h);
  const int lx = c->h64.desc[0].lx, ly = c->h64.desc[0].ly;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    const int n0 = sgi * K, n1 = std::min(n0 + K, nsteps);
    // recompute the segment's states u^{n0}..u^{n1}
    CUDA_TRY(cudaMemcpyAsync(work, ckpt[sgi], bytes, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(seg[0], work, bytes, cudaMemcpyDeviceToDevice, st));
    for (int j = 1; j <= n1 - n0; ++j) {
      STATUS_TRY(step(work));
      CUDA_TRY(cudaMemcpyAsync(seg[j], work, bytes, cudaMemcpyDeviceToDevice, st));
    }
    for (int k = n1 - 1; k >= n0; --k) {
      // mu = A^{-1} lambda (A symmetric), started from lambda
      CUDA_TRY(cudaMemcpyAsync(mu, lam, bytes, cudaMemcpyDeviceToDevice, st));
      fas_info inf;
      fas_status s2 = solve_impl(c, mu, lam, &inf, c->p.kmax);
      if (s2 == FAS_ENOTCONV) worst = s2;
      else if (s2 != FAS_OK) return s2;
      if (g_f) {
        Prof pr(c, FAS_K_OTHER, 0, (double)n);
        k_axpy<<<grid_for(c, n), kBlock, 0, st>>>(g_f, dt, mu, n);
      }
      if (g_kappa) {
        Prof pr(c, FAS_K_OTHER, 0, (double)n);
        if (c->p.dim == 2)
          k_kappa_grad<2><<<grid_for(c, n), kBlock, 0, st>>>(g_kappa, seg[k + 1 - n0], mu, s0.nx, s0.ny, s0.nz, lx,
                                                             ly, scale, dirmask);
        else
          k_kappa_grad<3><<<grid_for(c, n), kBlock, 0, st>>>(g_kappa, seg[k + 1 - n0], mu, s0.nx, s0.ny, s0.nz, lx,
                                                             ly, scale, dirmask);
      }
      std::swap(lam, mu);
    }
  }
  if (g_u0) CUDA_TRY(cudaMemcpyAsync(g_u0, lam, bytes, cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  CUDA_TRY(cudaGetLastError());
  if (worst != FAS_OK) return fail(worst, "fas_heat_adjoint: a solve missed its tolerance within kmax");
  return FAS_OK;
}

fas_status fas_fold_dirichlet(fas_ctx* c, double* f, const double values[6]) {
  STATUS_TRY(check_ctx(c));
  STATUS_TRY(check_field(f, true, "fas_fold_dirichlet"));
  if (!values) return fail(FAS_EINVAL, "fas_fold_dirichlet: null values");
  const fas_params& p = c->p;
  if (p.location != FAS_CELL) return fail(FAS_EUNSUPPORTED, "fas_fold_dirichlet: cell-centred unknowns only");
  FaceValues gv{};
  int dmask = 0;
  for (int k = 0; k < 2 * p.dim; ++k) {
    gv.g[k] = values[k];
    if (p.bc[k] == FAS_BC_DIRICHLET) dmask |= 1 << k;
  }
  const LevelShape& s = c->shape[0];
  const double scale = 2.0 * p.beta / (p.h * p.h);
  k_fold_dirichlet<<<grid_for(c, s.cells()), kBlock, 0, c->stream>>>(f, p.kappa, p.kappa_const, scale, s.nx, s.ny,
                                                                      s.nz, gv, dmask);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return FAS_OK;
}

fas_status fas_heat_run_host(fas_ctx* c, const double* u0_host, double* uT_host, const double* fsrc_host, double dt,
                             int nsteps, fas_info* infos) {
  STATUS_TRY(check_ctx(c));
  if (!u0_host || !uT_host) return fail(FAS_EINVAL, "fas_heat_run_host: null u");
  const int64_t n = c->shape[0].cells();
  if (!c->host_u) CUDA_TRY(cudaMalloc(&c->host_u, n * sizeof(double)));
  if (fsrc_host && !c->host_f) CUDA_TRY(cudaMalloc(&c->host_f, n * sizeof(double)));
  CUDA_TRY(copy_host(c, c->host_u, u0_host, n, true));
  if (fsrc_host) CUDA_TRY(copy_host(c, c->host_f, fsrc_host, n, true));
  fas_status st = fas_heat_run(c, c->host_u, fsrc_host ? c->host_f : nullptr, dt, nsteps, infos);
  CUDA_TRY(copy_host(c, uT_host, c->host_u, n, false));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return st;
}

fas_status fas_solve_batched(fas_ctx* const* ctxs, int count, double* const* u, const double* const* f,
                             fas_info* infos, void* stream) {
  if (!ctxs || !u || !f || count < 1) return fail(FAS_EINVAL, "fas_solve_batched: bad arguments");
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i] || !u[i] || !f[i]) return fail(FAS_EINVAL, "fas_solve_batched: null context or field");
    STATUS_TRY(check_field(u[i], true, "fas_solve_batched"));
    STATUS_TRY(check_field(f[i], true, "fas_solve_batched"));
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return fail(FAS_EINVAL, "fas_solve_batched: a context appears twice");
    if (ctxs[i]->prof) return fail(FAS_EINVAL, "fas_solve_batched: kernel timing is on for a context");
  }
  BatchGraph* B = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    for (BatchGraph* b : g_batches) {
      if ((int)b->ctxs.size() != count) continue;
      bool same = true;
      for (int i = 0; i < count && same; ++i) same = b->ctxs[i] == ctxs[i] && b->u[i] == u[i] && b->f[i] == f[i];
      if (same) {
        B = b;
        break;
      }
    }
  }
  if (!B) {
    B = new BatchGraph();
    B->ctxs.assign(ctxs, ctxs + count);
    B->u.assign(u, u + count);
    B->f.assign(f, f + count);
    fas_status st = build_batch(B);
    if (st != FAS_OK) {
      free_batch(B);
      return st;
    }
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    g_batches.push_back(B);
  }
  cudaStream_t st_ = (cudaStream_t)stream;
  CUDA_TRY(cudaGraphLaunch(B->exec, st_));
  CUDA_TRY(cudaMemcpyAsync(B->h_states, B->d_states, count * sizeof(SolveState), cudaMemcpyDeviceToHost, st_));
  for (int i = 0; i < count; ++i) CUDA_TRY(enqueue_timeout_read(ctxs[i], st_));
  CUDA_TRY(cudaStreamSynchronize(st_));
  CUDA_TRY(cudaGetLastError());
  fas_status worst = FAS_OK;
  for (int i = 0; i < count; ++i) STATUS_TRY(check_timeout(ctxs[i], st_));
  for (int i = 0; i < count; ++i) {
    fas_ctx* c = ctxs[i];
    *c->Sh = B->h_states[i];
    c->launches += B->n_pro[i] + (long long)B->h_states[i].cycles * B->n_body[i];
    fas_info inf;
    const fas_status st = finish_info(c, &inf, c->p.kmax);
    if (infos) infos[i] = inf;
    if (st == FAS_ENONFINITE || (st != FAS_OK && worst == FAS_OK)) worst = st;
  }
  if (worst == FAS_ENOTCONV) return fail(worst, "fas_solve_batched: a problem missed its tolerance within kmax");
  if (worst == FAS_ENONFINITE) return fail(worst, "fas_solve_batched: a residual is not finite");
  return worst;
}

fas_status fas_autotune(fas_ctx* c, double* u, const double* f, fas_tune_result* out) {
  STATUS_TRY(check_ctx(c));
  STATUS_TRY(check_field(u, true, "fas_autotune"));
  STATUS_TRY(check_field(f, true, "fas_autotune"));
  const TuneKey key{c->p.dim, c->shape[0].nx, c->shape[0].ny, c->shape[0].nz, c->p.precision};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (const TuneEntry& t : g_tune_cache)
      if (t.key == key) {
        c->p.inner_cycles = t.res.inner_cycles;
        c->p.seg_rows = t.res.seg_rows;
        destroy_graphs(c);
        drop_batches_of(c);
        if (out) {
          *out = t.res;
          out->candidates = 0;
        }
        return FAS_OK;
      }
  }
  const bool mixed = c->p.precision == FAS_MIXED;
  const bool fused = mixed && c->h32.nfast > 0;
  const int inners[3] = {1, 2, 3};
  const int segs[5] = {0, 16, 32, 64, 128};
  const int n_inner = mixed ? 3 : 1, n_seg = fused ? 5 : 1;
  const int64_t n = c->shape[0].cells();
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  fas_tune_result best{c->p.inner_cycles, c->p.seg_rows, 1e300, 0};
  const int keep_inner = c->p.inner_cycles, keep_seg = c->p.seg_rows;
  fas_status st = FAS_OK;
  for (int a = 0; a < n_inner && st == FAS_OK; ++a)
    for (int b = 0; b < n_seg && st == FAS_OK; ++b) {
      c->p.inner_cycles = mixed ? inners[a] : keep_inner;
      c->p.seg_rows = fused ? segs[b] : keep_seg;
      destroy_graphs(c);
      float ms = 0.f;
      for (int rep = 0; rep < 2 && st == FAS_OK; ++rep) {  // the first run captures the graph
        cudaMemsetAsync(u, 0, n * sizeof(double), c->stream);
        cudaEventRecord(e0, c->stream);
        fas_info inf;
        st = solve_impl(c, u, f, &inf, c->p.kmax);
        if (st == FAS_ENOTCONV) st = FAS_OK;  // a slow candidate still has a time
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
      }
      best.candidates++;
      if (st == FAS_OK && ms < best.ms) {
        best.ms = ms;
        best.inner_cycles = c->p.inner_cycles;
        best.seg_rows = c->p.seg_rows;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->p.inner_cycles = best.inner_cycles;
  c->p.seg_rows = best.seg_rows;
  destroy_graphs(c);
  drop_batches_of(c);
  if (st != FAS_OK) return st;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache.push_back(TuneEntry{key, best});
  }
  if (out) *out = best;
  return FAS_OK;
}

fas_status fas_residual(fas_ctx* c, int level, const double* u, const double* f, double* out, double* norm2) {
  STATUS_TRY(check_level(c, level, false));
  STATUS_TRY(check_field(u, true, "fas_residual"));
  STATUS_TRY(check_field(f, true, "fas_residual"));
  STATUS_TRY(check_field(out, false, "fas_residual"));
  const LevelDesc<double>& L = c->h64.desc[level];
  if (c->p.dim == 2)
    launch_residual<double, 2>(c, L, level, out, u, f, nullptr, c->d_scalar);
  else
    launch_residual<double, 3>(c, L, level, out, u, f, nullptr, c->d_scalar);
  double v = 0.0;
  STATUS_TRY(sync_read(c, &v));
  if (norm2) *norm2 = v;
  return FAS_OK;
}

fas_status fas_residual_ir(fas_ctx* c, const double* u, const double* f, float* r32, double* norm2) {
  STATUS_TRY(check_ctx(c));
  for (const void* q : {(const void*)u, (const void*)f, (const void*)r32})
    STATUS_TRY(check_field(q, true, "fas_residual_ir"));
  const int g = launch_ir_residual(c, r32, u, f, nullptr);
  {
    Prof pr(c, FAS_K_NORM, 0, 0.0);
    k_finish_norm<<<1, kBlock, 0, c->stream>>>(c->partials, g, c->d_scalar, nullptr);
  }
  CUDA_TRY(enqueue_timeout_read(c, c->stream));
  double v = 0.0;
  STATUS_TRY(sync_read(c, &v));
  STATUS_TRY(check_timeout(c, c->stream));
  if (norm2) *norm2 = v;
  return FAS_OK;
}

fas_status fas_selftest_conversions(long long count, unsigned long long seed, long long* mismatches) {
  if (count < 0 || !mismatches) return fail(FAS_EINVAL, "fas_selftest_conversions: bad argument");
  unsigned long long* d = nullptr;
  CUDA_TRY(cudaMalloc(&d, sizeof(unsigned long long)));
  cudaError_t e = cudaMemset(d, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) {
    k_selftest_specials<<<1, 1>>>(d);
    if (count > 0) k_selftest_conv<<<1024, 256>>>(count, seed, d);
    e = cudaGetLastError();
  }
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(FAS_ECUDA, std::string("fas_selftest_conversions: ") + cudaGetErrorString(e));
  *mismatches = (long long)h;
  return FAS_OK;
}

fas_status fas_smooth(fas_ctx* c, int level, double* u, const double* f, int sweeps) {
  STATUS_TRY(check_level(c, level, false));
  if (sweeps < 0) return fail(FAS_EINVAL, "sweeps must be >= 0");
  STATUS_TRY(check_field(u, true, "fas_smooth"));
  STATUS_TRY(check_field(f, true, "fas_smooth"));
  const LevelDesc<double>& L = c->h64.desc[level];
  if (c->p.dim == 2)
    launch_smooth<double, 2>(c, L, level, u, f, sweeps);
  else
    launch_smooth<double, 3>(c, L, level, u, f, sweeps);
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  CUDA_TRY(cudaGetLastError());
  return FAS_OK;
}

fas_status fas_restrict(fas_ctx* c, int level, const double* u, double* uc) {
  STATUS_TRY(check_level(c, level, true));
  STATUS_TRY(check_field(u, true, "fas_restrict"));
  STATUS_TRY(check_field(uc, true, "fas_restrict"));
  const LevelShape& s = c->shape[level];
  const int64_t nc = s.cells() >> c->p.dim;
  {
    Prof pr(c, FAS_K_RESTRICT, level, (double)s.cells());
    if (c->p.dim == 2)
      launch_restrict<double, 2>(c, nc, uc, nullptr, nullptr, u, nullptr, s.nx, s.ny, s.nz);
    else
      launch_restrict<double, 3>(c, nc, uc, nullptr, nullptr, u, nullptr, s.nx, s.ny, s.nz);
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  CUDA_TRY(cudaGetLastError());
  return FAS_OK;
}

fas_status fas_prolong_add(fas_ctx* c, int level, double* u, const double* cc) {
  STATUS_TRY(check_level(c, level, true));
  STATUS_TRY(check_field(u, true, "fas_prolong_add"));
  STATUS_TRY(check_field(cc, true, "fas_prolong_add"));
  const LevelShape& s = c->shape[level];
  const int64_t nc = s.cells() >> c->p.dim;
  {
    Prof pr(c, FAS_K_PROLONG, level, (double)s.cells());
    if (c->p.dim == 2)
      launch_prolong<double, 2>(c, s.cells(), u, cc, nullptr, s.nx, s.ny, s.nz);
    else
      launch_prolong<double, 3>(c, s.cells(), u, cc, nullptr, s.nx, s.ny, s.nz);
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  CUDA_TRY(cudaGetLastError());
  return FAS_OK;
}

fas_status fas_prof_enable(fas_ctx* c, int on) {
  STATUS_TRY(check_ctx(c));
  if (on) {
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->spans.clear();
    c->pool_next = 0;
  }
  c->prof = on != 0;
  return FAS_OK;
}

fas_status fas_prof_read(fas_ctx* c, fas_prof_record* out, int cap, int* count) {
  STATUS_TRY(check_ctx(c));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  std::vector<fas_prof_record> agg;
  for (const ProfSpan& sp : c->spans) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, sp.beg, sp.end));
    fas_prof_record* rec = nullptr;
    for (auto& a : agg)
      if (a.family == sp.family && a.level == sp.level) rec = &a;
    if (!rec) {
      fas_prof_record z;
      std::memset(&z, 0, sizeof(z));
      z.family = sp.family;
      z.level = sp.level;
      agg.push_back(z);
      rec = &agg.back();
    }
    rec->launches += 1;
    rec->ms += ms;
    rec->units += sp.units;
  }
  if (count) *count = (int)agg.size();
  for (int k = 0; k < (int)agg.size() && k < cap && out; ++k) out[k] = agg[k];
  return FAS_OK;
}

fas_status fas_debug_bounded_wait(long long limit_ns, int withhold_next) {
  if (limit_ns <= 0) return fail(FAS_EINVAL, "fas_debug_bounded_wait: limit_ns must be positive");
  if (withhold_next < 0 || withhold_next > 2) return fail(FAS_EINVAL, "fas_debug_bounded_wait: withhold_next is 0, 1 or 2");
  g_wait_limit_ns = (unsigned long long)limit_ns;
  g_withhold_copy = withhold_next;
  return FAS_OK;
}

const char* fas_last_error(void) { return g_last_error.c_str(); }

long long fas_launch_count(const fas_ctx* c, int reset) {
  if (!c) return 0;
  long long v = c->launches;
  if (reset) const_cast<fas_ctx*>(c)->launches = 0;
  return v;
}

}  // extern "C"
