// ns.cu -- first-order projection step for incompressible Navier-Stokes on the MAC grid (Sec. 4.2),
// with every linear solve done by the FAS multigrid (face grids for the velocity, cells for the
// pressure). The glue between the solves -- the explicit right-hand side with third-order WENO
// convection, the divergence, the projection -- is three float64 kernels, each one pass over the
// resident fields.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <type_traits>

#include "fas.h"
#include "ns.h"

namespace fasmg {
void set_last_error(const std::string& msg);  // fas_api.cu: the thread-local message of fas_last_error
}

namespace {

using fasmg::set_last_error;

constexpr int kNsBlock = 256;
constexpr double kWenoEps = 1e-6;

fas_status ns_fail(fas_status s, const std::string& msg) {
  set_last_error(msg);
  return s;
}

#define NS_CUDA_TRY(call)                                                                     \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return ns_fail(FAS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Grid geometry shared by the kernels: cells per axis, strides, and log2 of nx, ny for the index split.
struct NsGrid {
  int n[3];
  int64_t st[3];
  int lx, ly;
  int64_t cells;
  double h;
  double hinv;  // 1/h, exact when hpow2
  bool hpow2;   // h is a power of two
};

__device__ __forceinline__ int64_t ns_tid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t ns_stride() { return (int64_t)gridDim.x * blockDim.x; }

__device__ __forceinline__ void ns_coords(const NsGrid& G, int64_t idx, int* k) {
  k[0] = (int)(idx & (G.n[0] - 1));
  k[1] = (int)((idx >> G.lx) & (G.n[1] - 1));
  k[2] = (int)(idx >> (G.lx + G.ly));
}

// Value of a velocity component along its own axis a at face F (F may lie up to two faces beyond
// either wall): faces 0 and n are walls (0; face n is the stored slot n-1), beyond a wall the normal
// component is continued oddly, face -k = -face k and face n+k = -face n-k. `line` is the linear
// index of slot 0 on the line through the point.
__device__ __forceinline__ double normal_value(const double* __restrict__ phi, int64_t line, int64_t st, int n, int F) {
  double sgn = 1.0;
  if (F < 0) {
    F = -F;
    sgn = -1.0;
  } else if (F > n) {
    F = 2 * n - F;
    sgn = -1.0;
  }
  const double v = F == 0 ? 0.0 : phi[line + (int64_t)(F - 1) * st];
  return sgn * v;
}

// Value of a component along a tangential axis at cell c (up to two cells beyond either wall): a
// ghost cell mirrors the cell inside about the wall with ghost = 2 g - inside, g the wall's velocity.
__device__ __forceinline__ double tangential_value(const double* __restrict__ phi, int64_t line, int64_t st, int n,
                                                   int c, double g_lo, double g_hi) {
  if (c < 0) return 2.0 * g_lo - phi[line + (int64_t)(-c - 1) * st];
  if (c >= n) return 2.0 * g_hi - phi[line + (int64_t)(2 * n - 1 - c) * st];
  return phi[line + (int64_t)c * st];
}

// Third-order WENO of Jiang and Shu for a derivative from three consecutive first differences, the
// upwind one first: the two candidate slopes (3b - a)/2 and (b + c)/2 weighted by the ideal weights
// 1/3 and 2/3 over the square of eps + their smoothness (b - a)^2, (c - b)^2. With the weights
// alpha_k = d_k / q_k^2 brought to the common denominator 3 q0^2 q1^2 the combination is
// (q1^2 p0 + 2 q0^2 p1) / (q1^2 + 2 q0^2): one division instead of three (float64 division is a long
// sequence on the FP64 pipe).
__device__ __forceinline__ double weno3(double a, double b, double c) {
  const double p0 = 0.5 * (3.0 * b - a);
  const double p1 = 0.5 * (b + c);
  const double b0 = (b - a) * (b - a);
  const double b1 = (c - b) * (c - b);
  const double q0 = kWenoEps + b0, q1 = kWenoEps + b1;
  const double w0 = q1 * q1, w1 = 2.0 * (q0 * q0);
  return (w0 * p0 + w1 * p1) / (w0 + w1);
}

// x / h, as a multiplication by the exact reciprocal when h is a power of two (then bitwise equal)
struct InvH {
  double h, inv;
  bool pow2;
  __device__ __forceinline__ double operator()(double x) const { return pow2 ? x * inv : x / h; }
};

// f_C = c^n - dt (u^n . grad c^n)_WENO3 - dt (p^n_{s+1} - p^n_s)/h + dt F (F: body force at t^{n+1},
// optional), plus the lid's tangential wall velocity folded into the cells next to the top wall
// (2 beta g / h^2, the ghost 2g - inside of the viscous operator), 0 on the wall slot. C is the
// component (= its index axis).
template <int DIM, int C>
__global__ void k_ns_source(double* __restrict__ f, const double* __restrict__ U, const double* __restrict__ V,
                            const double* __restrict__ W, const double* __restrict__ P,
                            const double* __restrict__ F, NsGrid G, double dt, double beta, double lid_c) {
  const double* vel[3] = {U, V, W};
  const double* __restrict__ phi = vel[C];
  const double h = G.h;
  const InvH dh{G.h, G.hinv, G.hpow2};
  for (int64_t idx = ns_tid(); idx < G.cells; idx += ns_stride()) {
    int k[3];
    ns_coords(G, idx, k);
    if (k[C] == G.n[C] - 1) {
      f[idx] = 0.0;
      continue;
    }
    double conv = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int64_t st = G.st[a];
      const int64_t line = idx - (int64_t)k[a] * st;
      double v[5];
      if (a == C) {
#pragma unroll
        for (int s = -2; s <= 2; ++s) v[s + 2] = normal_value(phi, line, st, G.n[a], k[a] + 1 + s);
      } else {
        const double g_hi = a == DIM - 1 ? lid_c : 0.0;
#pragma unroll
        for (int s = -2; s <= 2; ++s) v[s + 2] = tangential_value(phi, line, st, G.n[a], k[a] + s, 0.0, g_hi);
      }
      double adv;
      if (a == C) {
        adv = phi[idx];
      } else {
        // component a at the point: its two faces around the cell along a, at the two cells on either
        // side of the point's face along C (face 0 along a is the wall, 0)
        const double* __restrict__ A = vel[a];
        const int64_t sa = G.st[a], sc = G.st[C];
        const bool in = k[a] > 0;
        const double lo = 0.5 * ((in ? A[idx - sa] : 0.0) + A[idx]);
        const double hi = 0.5 * ((in ? A[idx - sa + sc] : 0.0) + A[idx + sc]);
        adv = 0.5 * (lo + hi);
      }
      // only the upwind WENO3 derivative is used: the left-biased one (differences d1, d2, d3) where
      // the advecting velocity is positive, the right-biased one (d4, d3, d2) elsewhere
      const bool up = adv > 0.0;
      const double d2 = dh(v[2] - v[1]), d3 = dh(v[3] - v[2]);
      const double dx = up ? dh(v[1] - v[0]) : dh(v[4] - v[3]);
      const double dd = weno3(dx, up ? d2 : d3, up ? d3 : d2);
      conv = conv + adv * dd;
    }
    const double gp = dh(P[idx + G.st[C]] - P[idx]);
    double v = phi[idx] - dt * conv - dt * gp;
    if (F) v = v + dt * F[idx];
    if (C != DIM - 1 && k[DIM - 1] == G.n[DIM - 1] - 1) v = v + 2.0 * beta * lid_c / (h * h);
    f[idx] = v;
  }
}

// Second-order scheme (Scheme second-1..4, the lagged 8-field table): the right-hand side of
// (I - dt/2Re Lap) c~ = f_C with
//   f_C = c^n - dt (a . grad) cbar + (dt/2Re) Lap c^n - dt (p^n_{s+1} - p^n_s)/h + dt F (+ lid)
// where cbar = (3 c^n - c^{n-1})/2 is differentiated by WENO3, and the advecting component a is
// (a^n + a~^{n+1})/2 for a < C (already solved this step: a^n lagged into OLD, a~ in CUR) and
// (3 a^n - a^{n-1})/2 otherwise (CUR = a^n, OLD = a^{n-1}). The lid enters twice (implicit and
// explicit halves of the viscous term, 2 beta g / h^2 each, beta = dt/2Re).
template <int DIM, int C>
__global__ void k_ns_source2(double* __restrict__ f, const double* __restrict__ U, const double* __restrict__ Uo,
                             const double* __restrict__ V, const double* __restrict__ Vo,
                             const double* __restrict__ W, const double* __restrict__ Wo,
                             const double* __restrict__ P, const double* __restrict__ F, NsGrid G, double dt,
                             double beta, double lid_c) {
  const double* cur[3] = {U, V, W};
  const double* old[3] = {Uo, Vo, Wo};
  const double* __restrict__ cc = cur[C];
  const double* __restrict__ co = old[C];
  const double h = G.h;
  const InvH dh{G.h, G.hinv, G.hpow2};
  for (int64_t idx = ns_tid(); idx < G.cells; idx += ns_stride()) {
    int k[3];
    ns_coords(G, idx, k);
    if (k[C] == G.n[C] - 1) {
      f[idx] = 0.0;
      continue;
    }
    auto cbar = [&](int64_t q) { return 0.5 * (3.0 * cc[q] - co[q]); };
    double conv = 0.0, lap = 0.0;
    const double c0 = cc[idx];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int64_t st = G.st[a];
      const int64_t line = idx - (int64_t)k[a] * st;
      const int n = G.n[a];
      double v[5];
      if (a == C) {
#pragma unroll
        for (int s = -2; s <= 2; ++s) {
          int F2 = k[a] + 1 + s;  // face index, odd continuation beyond the walls
          double sg = 1.0;
          if (F2 < 0) {
            F2 = -F2;
            sg = -1.0;
          } else if (F2 > n) {
            F2 = 2 * n - F2;
            sg = -1.0;
          }
          v[s + 2] = F2 == 0 ? 0.0 : sg * cbar(line + (int64_t)(F2 - 1) * st);
        }
        const double lo = k[a] > 0 ? cc[idx - st] : 0.0;
        lap += (lo - 2.0 * c0) + cc[idx + st];
      } else {
        const double g_hi = a == DIM - 1 ? lid_c : 0.0;
#pragma unroll
        for (int s = -2; s <= 2; ++s) {
          const int cidx = k[a] + s;
          if (cidx < 0) v[s + 2] = -cbar(line + (int64_t)(-cidx - 1) * st);
          else if (cidx >= n) v[s + 2] = 2.0 * g_hi - cbar(line + (int64_t)(2 * n - 1 - cidx) * st);
          else v[s + 2] = cbar(line + (int64_t)cidx * st);
        }
        const double lo = k[a] > 0 ? cc[idx - st] : -c0;
        const double hi = k[a] < n - 1 ? cc[idx + st] : -c0;
        lap += (hi - c0) - (c0 - lo);
      }
      double adv;
      if (a == C) {
        adv = cbar(idx);
      } else {
        const double* __restrict__ Ac = cur[a];
        const double* __restrict__ Ao = old[a];
        auto A = [&](int64_t q) { return a < C ? 0.5 * (Ao[q] + Ac[q]) : 0.5 * (3.0 * Ac[q] - Ao[q]); };
        const int64_t sa = G.st[a], sc = G.st[C];
        const bool in = k[a] > 0;
        const double lo = 0.5 * ((in ? A(idx - sa) : 0.0) + A(idx));
        const double hi = 0.5 * ((in ? A(idx - sa + sc) : 0.0) + A(idx + sc));
        adv = 0.5 * (lo + hi);
      }
      // only the upwind WENO3 derivative is used: the left-biased one (differences d1, d2, d3) where
      // the advecting velocity is positive, the right-biased one (d4, d3, d2) elsewhere
      const bool up = adv > 0.0;
      const double d2 = dh(v[2] - v[1]), d3 = dh(v[3] - v[2]);
      const double dx = up ? dh(v[1] - v[0]) : dh(v[4] - v[3]);
      const double dd = weno3(dx, up ? d2 : d3, up ? d3 : d2);
      conv = conv + adv * dd;
    }
    const double gp = dh(P[idx + G.st[C]] - P[idx]);
    double v = c0 - dt * conv + beta * dh(dh(lap)) - dt * gp;
    if (F) v = v + dt * F[idx];
    if (C != DIM - 1 && k[DIM - 1] == G.n[DIM - 1] - 1) v = v + 2.0 * (2.0 * beta * lid_c / (h * h));
    f[idx] = v;
  }
}

// rhs = -div u over the cells, wall faces 0 (face k+1 of a cell is slot k, face k slot k-1).
template <int DIM>
__global__ void k_ns_neg_div(double* __restrict__ rhs, const double* __restrict__ U, const double* __restrict__ V,
                             const double* __restrict__ W, NsGrid G) {
  const double* vel[3] = {U, V, W};
  const InvH dh{G.h, G.hinv, G.hpow2};
  for (int64_t idx = ns_tid(); idx < G.cells; idx += ns_stride()) {
    int k[3];
    ns_coords(G, idx, k);
    double div = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const double* __restrict__ A = vel[a];
      const double lo = k[a] > 0 ? A[idx - G.st[a]] : 0.0;
      div = div + dh(A[idx] - lo);
    }
    rhs[idx] = -div;
  }
}

// c_old = c_new - dt (p_{s+1} - p_s)/h for every component (the wall slot keeps c_new, which is 0),
// p_old += p_new. One pass over the eight fields.
// (out may equal in: every element is read and written by the same thread.)
template <int DIM>
__global__ void k_ns_project(double* Uo, double* Vo, double* Wo, const double* Un, const double* Vn,
                             const double* Wn, double* __restrict__ Po, const double* __restrict__ Pn, NsGrid G,
                             double dt) {
  double* out[3] = {Uo, Vo, Wo};
  const double* in[3] = {Un, Vn, Wn};
  const InvH dh{G.h, G.hinv, G.hpow2};
  for (int64_t idx = ns_tid(); idx < G.cells; idx += ns_stride()) {
    int k[3];
    ns_coords(G, idx, k);
    const double pc = Pn[idx];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const double gp = k[a] < G.n[a] - 1 ? dh(Pn[idx + G.st[a]] - pc) : 0.0;
      out[a][idx] = in[a][idx] - dt * gp;
    }
    Po[idx] = Po[idx] + pc;
  }
}

// Per-block maximum of |div u| into partials[blockIdx.x].
template <int DIM>
__global__ void k_ns_div_max(const double* __restrict__ U, const double* __restrict__ V,
                             const double* __restrict__ W, NsGrid G, double* partials) {
  const double* vel[3] = {U, V, W};
  const InvH dh{G.h, G.hinv, G.hpow2};
  double m = 0.0;
  for (int64_t idx = ns_tid(); idx < G.cells; idx += ns_stride()) {
    int k[3];
    ns_coords(G, idx, k);
    double div = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const double* __restrict__ A = vel[a];
      const double lo = k[a] > 0 ? A[idx - G.st[a]] : 0.0;
      div = div + dh(A[idx] - lo);
    }
    m = fmax(m, fabs(div));
  }
  __shared__ double wm[32];
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? wm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) partials[blockIdx.x] = m;
  }
}

__global__ void k_ns_finish_max(const double* partials, int nb, double* out) {
  __shared__ double wm[32];
  double m = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = fmax(m, partials[b]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? wm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) out[0] = m;
  }
}

}  // namespace

struct ns_ctx {
  int dim = 2;
  NsGrid G{};
  double Re = 0.0, dt = 0.0, beta = 0.0;  // beta: dt/Re (first order) or dt/2Re (second order)
  int order = 1;
  double lid[3] = {0.0, 0.0, 0.0};
  cudaStream_t stream = nullptr;
  fas_ctx* vel[3] = {nullptr, nullptr, nullptr};
  fas_ctx* pres = nullptr;
  double* ftmp = nullptr;      // right-hand side of the current solve
  double* partials = nullptr;  // per-block maxima
  double* d_max = nullptr;
  double* h_max = nullptr;  // pinned
  int nblocks = 0;
  long long launches = 0;
};

namespace {

bool pow2_at_least(int v, int lo) { return v >= lo && (v & (v - 1)) == 0; }

template <int DIM, int C>
void source1(ns_ctx* c, double* const* un, const double* P, const double* F, double lid) {
  k_ns_source<DIM, C><<<c->nblocks, kNsBlock, 0, c->stream>>>(c->ftmp, un[0], un[1], DIM == 3 ? un[2] : nullptr, P, F,
                                                              c->G, c->dt, c->beta, lid);
}

void launch_source1(ns_ctx* c, int a, double* const* un, const double* P, const double* F, double lid) {
  if (c->dim == 2) {
    if (a == 0) source1<2, 0>(c, un, P, F, lid);
    else source1<2, 1>(c, un, P, F, lid);
  } else {
    if (a == 0) source1<3, 0>(c, un, P, F, lid);
    else if (a == 1) source1<3, 1>(c, un, P, F, lid);
    else source1<3, 2>(c, un, P, F, lid);
  }
}

template <int DIM, int C>
void source2(ns_ctx* c, double* const* cur, double* const* old, const double* P, const double* F, double lid) {
  k_ns_source2<DIM, C><<<c->nblocks, kNsBlock, 0, c->stream>>>(
      c->ftmp, cur[0], old[0], cur[1], old[1], DIM == 3 ? cur[2] : nullptr, DIM == 3 ? old[2] : nullptr, P, F, c->G,
      c->dt, c->beta, lid);
}

void launch_source2(ns_ctx* c, int a, double* const* cur, double* const* old, const double* P, const double* F,
                    double lid) {
  if (c->dim == 2) {
    if (a == 0) source2<2, 0>(c, cur, old, P, F, lid);
    else source2<2, 1>(c, cur, old, P, F, lid);
  } else {
    if (a == 0) source2<3, 0>(c, cur, old, P, F, lid);
    else if (a == 1) source2<3, 1>(c, cur, old, P, F, lid);
    else source2<3, 2>(c, cur, old, P, F, lid);
  }
}

fas_status ns_check_solve(fas_status st, const char* what, fas_status* first) {
  if (st == FAS_OK) return FAS_OK;
  if (st == FAS_ENOTCONV) {
    if (*first == FAS_OK) *first = st;
    return FAS_OK;
  }
  return ns_fail(st, std::string("ns_projection_step: ") + what + ": " + fas_last_error());
}

}  // namespace

extern "C" {

fas_status ns_create(int dim, const int n[3], double h, double Re, double dt, int order, const double lid[3],
                     const fas_params* solver, const fas_params* pressure, void* stream, ns_ctx** out) {
  if (!out || !n) return ns_fail(FAS_EINVAL, "ns_create: null argument");
  *out = nullptr;
  if (dim != 2 && dim != 3) return ns_fail(FAS_EINVAL, "ns_create: dim must be 2 or 3");
  for (int a = 0; a < dim; ++a)
    if (!pow2_at_least(n[a], 4)) return ns_fail(FAS_EINVAL, "ns_create: every n must be a power of two >= 4");
  if (!(h > 0.0) || !(Re > 0.0) || !(dt > 0.0) || !std::isfinite(h) || !std::isfinite(Re) || !std::isfinite(dt))
    return ns_fail(FAS_EINVAL, "ns_create: h, Re, dt must be positive");
  if (order != 1 && order != 2) return ns_fail(FAS_EUNSUPPORTED, "ns_create: order must be 1 or 2");
  ns_ctx* c = new ns_ctx();
  c->dim = dim;
  c->Re = Re;
  c->dt = dt;
  c->order = order;
  c->beta = order == 1 ? dt / Re : dt / (2.0 * Re);
  for (int a = 0; a < 3; ++a) c->lid[a] = lid ? lid[a] : 0.0;
  c->stream = (cudaStream_t)stream;
  NsGrid& G = c->G;
  G.n[0] = n[0];
  G.n[1] = n[1];
  G.n[2] = dim == 3 ? n[2] : 1;
  G.st[0] = 1;
  G.st[1] = G.n[0];
  G.st[2] = (int64_t)G.n[0] * G.n[1];
  G.lx = 0;
  while ((1 << G.lx) < G.n[0]) ++G.lx;
  G.ly = 0;
  while ((1 << G.ly) < G.n[1]) ++G.ly;
  G.cells = G.st[2] * G.n[2];
  G.h = h;
  {
    int e = 0;
    const double m = std::frexp(h, &e);  // h = m 2^e, m in [0.5, 1)
    G.hpow2 = m == 0.5;
    G.hinv = 1.0 / h;
  }
  auto bail = [&](fas_status s) {
    ns_destroy(c);
    return s;
  };
  // viscous solves: (I - dt/Re Lap) on the face grid of each component, no-slip walls
  fas_params pv;
  fas_default_params(&pv);
  pv.kmax = 40;
  if (solver) pv = *solver;
  pv.dim = dim;
  for (int a = 0; a < 3; ++a) pv.n[a] = G.n[a];
  pv.h = h;
  pv.alpha = 1.0;
  pv.beta = c->beta;
  pv.kappa = nullptr;
  pv.kappa_const = 1.0;
  for (int k = 0; k < 6; ++k) pv.bc[k] = FAS_BC_DIRICHLET;
  pv.coarse_exact = 0;
  pv.path = 1;
  for (int a = 0; a < dim; ++a) {
    pv.location = FAS_FACE_X + a;
    fas_status st = fas_create(&pv, stream, &c->vel[a]);
    if (st != FAS_OK) return bail(ns_fail(st, std::string("ns_create: velocity solver: ") + fas_last_error()));
  }
  // pressure: -dt Lap p = rhs, homogeneous Neumann (singular, mean fixed to 0)
  fas_params pp;
  fas_default_params(&pp);
  pp.kmax = 60;
  pp.coarse_exact = 1;
  if (pressure) pp = *pressure;
  pp.dim = dim;
  for (int a = 0; a < 3; ++a) pp.n[a] = G.n[a];
  pp.h = h;
  pp.alpha = 0.0;
  pp.beta = dt;
  pp.kappa = nullptr;
  pp.kappa_const = 1.0;
  for (int k = 0; k < 6; ++k) pp.bc[k] = FAS_BC_NEUMANN;
  pp.location = FAS_CELL;
  {
    fas_status st = fas_create(&pp, stream, &c->pres);
    if (st != FAS_OK) return bail(ns_fail(st, std::string("ns_create: pressure solver: ") + fas_last_error()));
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  c->nblocks = (int)std::min<int64_t>((G.cells + kNsBlock - 1) / kNsBlock, (int64_t)std::max(sms, 1) * 8);
  if (cudaMalloc(&c->ftmp, G.cells * sizeof(double)) != cudaSuccess) return bail(ns_fail(FAS_ENOMEM, "ns_create: rhs"));
  if (cudaMalloc(&c->partials, c->nblocks * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_max, sizeof(double)) != cudaSuccess || cudaMallocHost(&c->h_max, sizeof(double)) != cudaSuccess)
    return bail(ns_fail(FAS_ENOMEM, "ns_create: scratch"));
  *out = c;
  return FAS_OK;
}

fas_status ns_projection_step(ns_ctx* c, double* const fields[8], const double* const force[3], fas_info info[4],
                              double* div_max) {
  if (!c || !fields) return ns_fail(FAS_EINVAL, "ns_projection_step: null argument");
  const int dim = c->dim;
  double* cnew[3] = {fields[0], fields[2], dim == 3 ? fields[4] : nullptr};
  double* cold[3] = {fields[1], fields[3], dim == 3 ? fields[5] : nullptr};
  double* Pn = fields[6];
  double* Po = fields[7];
  for (int a = 0; a < dim; ++a)
    if (!cnew[a] || !cold[a]) return ns_fail(FAS_EINVAL, "ns_projection_step: missing velocity field");
  if (!Pn || !Po) return ns_fail(FAS_EINVAL, "ns_projection_step: missing pressure field");
  // every field moves through the solver's 16-byte vector accesses
  for (int k = 0; k < 8; ++k)
    if ((dim == 3 || (k != 4 && k != 5)) && (reinterpret_cast<uintptr_t>(fields[k]) & 15u))
      return ns_fail(FAS_EINVAL, "ns_projection_step: field not 16-byte aligned");
  if (force)
    for (int a = 0; a < dim; ++a)
      if (reinterpret_cast<uintptr_t>(force[a]) & 15u)
        return ns_fail(FAS_EINVAL, "ns_projection_step: force field not 16-byte aligned");
  if (info) std::memset(info, 0, 4 * sizeof(fas_info));
  const NsGrid& G = c->G;
  const size_t bytes = (size_t)G.cells * sizeof(double);
  fas_status first = FAS_OK;
  const bool second = c->order == 2;
  // viscous solves, one component at a time
  for (int a = 0; a < dim; ++a) {
    const double lid_a = c->lid[a];
    const double* Fa = force ? force[a] : nullptr;
    if (!second) {  // f from u^n (in C_old) and p^n; the solve starts from u^n copied into C_new
      launch_source1(c, a, cold, Po, Fa, lid_a);
    } else {  // f from c^n (C_new), c^{n-1} (C_old) and the solved a~ (C_new of a < C)
      launch_source2(c, a, cnew, cold, Po, Fa, lid_a);
    }
    c->launches += 1;
    NS_CUDA_TRY(cudaGetLastError());
    if (!second)
      NS_CUDA_TRY(cudaMemcpyAsync(cnew[a], cold[a], bytes, cudaMemcpyDeviceToDevice, c->stream));
    else  // the lagged update c^{n-1} <- c^n; C_new keeps c^n as the initial guess
      NS_CUDA_TRY(cudaMemcpyAsync(cold[a], cnew[a], bytes, cudaMemcpyDeviceToDevice, c->stream));
    fas_info inf;
    const fas_status st = fas_solve(c->vel[a], cnew[a], c->ftmp, &inf);
    if (info) info[a] = inf;
    if (ns_check_solve(st, "velocity solve", &first) != FAS_OK) return st;
  }
  // pressure increment: -dt Lap p~ = -div u~
  if (dim == 2)
    k_ns_neg_div<2><<<c->nblocks, kNsBlock, 0, c->stream>>>(c->ftmp, cnew[0], cnew[1], nullptr, G);
  else
    k_ns_neg_div<3><<<c->nblocks, kNsBlock, 0, c->stream>>>(c->ftmp, cnew[0], cnew[1], cnew[2], G);
  c->launches += 1;
  NS_CUDA_TRY(cudaGetLastError());
  NS_CUDA_TRY(cudaMemsetAsync(Pn, 0, bytes, c->stream));
  {
    fas_info inf;
    const fas_status st = fas_solve(c->pres, Pn, c->ftmp, &inf);
    if (info) info[3] = inf;
    if (ns_check_solve(st, "pressure solve", &first) != FAS_OK) return st;
  }
  // projection and pressure update: u^{n+1} into C_old (first order) or in place in C_new (second)
  double* const* out = second ? cnew : cold;
  if (dim == 2)
    k_ns_project<2><<<c->nblocks, kNsBlock, 0, c->stream>>>(out[0], out[1], nullptr, cnew[0], cnew[1], nullptr, Po,
                                                            Pn, G, c->dt);
  else
    k_ns_project<3><<<c->nblocks, kNsBlock, 0, c->stream>>>(out[0], out[1], out[2], cnew[0], cnew[1], cnew[2], Po,
                                                            Pn, G, c->dt);
  c->launches += 1;
  NS_CUDA_TRY(cudaGetLastError());
  if (div_max) {
    if (dim == 2)
      k_ns_div_max<2><<<c->nblocks, kNsBlock, 0, c->stream>>>(out[0], out[1], nullptr, G, c->partials);
    else
      k_ns_div_max<3><<<c->nblocks, kNsBlock, 0, c->stream>>>(out[0], out[1], out[2], G, c->partials);
    k_ns_finish_max<<<1, 1024, 0, c->stream>>>(c->partials, c->nblocks, c->d_max);
    c->launches += 2;
    NS_CUDA_TRY(cudaMemcpyAsync(c->h_max, c->d_max, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    NS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    *div_max = *c->h_max;
  } else {
    NS_CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  NS_CUDA_TRY(cudaGetLastError());
  return first;
}

long long ns_launch_count(ns_ctx* c, int reset) {
  if (!c) return 0;
  long long total = c->launches;
  for (int a = 0; a < 3; ++a)
    if (c->vel[a]) total += fas_launch_count(c->vel[a], reset);
  if (c->pres) total += fas_launch_count(c->pres, reset);
  if (reset) c->launches = 0;
  return total;
}

fas_status ns_destroy(ns_ctx* c) {
  if (!c) return FAS_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int a = 0; a < 3; ++a) fas_destroy(c->vel[a]);
  fas_destroy(c->pres);
  if (c->ftmp) cudaFree(c->ftmp);
  if (c->partials) cudaFree(c->partials);
  if (c->d_max) cudaFree(c->d_max);
  if (c->h_max) cudaFreeHost(c->h_max);
  delete c;
  return FAS_OK;
}

}  // extern "C"
