// stream2d.cu -- sweep-fused float32 multigrid kernels for 2D levels (register streaming).
//
// Each warp owns a strip of 128 columns (4 consecutive cells per lane, float4 loads) and a segment of
// rows, and streams down the rows with an 8-row window of the strip held in registers. Every step of
// the level's work is a pipeline stage one row behind the previous one:
//
//   pre-smoothing kernel  (Algorithm 1 pre-smoothing, residual, restriction, tau correction)
//     load row y  ->  [tau: f = R(r) + A u at row y-1]  ->  colour phase 1 .. 2*NS at rows y-1-t ..
//     -> residual r = f - A u at the next row -> on odd rows, the 2x2 averages R(u), R(r) (Appendix C)
//   post-smoothing kernel (coarse-grid correction and post-smoothing)
//     load row y -> on odd rows u += uc - R(u) for the row pair (Appendix C prolongation of the
//     correction, R(u) recomputed from the unchanged fine values) -> colour phases -> store; the
//     coarse values of a row pair travel in the row ring with the pair's second row. In the last
//     float32 cycle of a refinement step the store is u64 += e instead: the row is staged in shared
//     memory as float64 and added to u64 by a bulk reduction in the L2.
//
// A colour phase updates the cells of one X-MCGS colour (Sec. 2.3; colour 1 = cells whose 1-based
// i+j is odd, the paper's sets 1 and 2) from their four neighbours. A row's cells of one colour only
// see the other colour, so stage t at row y reads rows y-1, y, y+1 after stage t-1, which the
// pipeline guarantees. West/east neighbours come from the lane itself or by one warp shuffle.
//
// Strips and segments overlap (8 columns each side, 4 in the post-smoothing kernel with the float64
// update; 5-7 rows at the top and bottom) and recompute
// their halos; only the interior is written. Because neighbours read the halo, nothing a warp reads
// may be written by this kernel: u is read from one buffer and written to another, and the tau
// right-hand side is kept in registers and written to a buffer separate from R(r).
//
// Arithmetic per point is the same expression as in basic_kernels.cuh (same association and fma
// placement), so a V-cycle through these kernels is bit-for-bit the V-cycle of the per-operation
// float32 kernels.
#include <mutex>

#include "bits64.cuh"
#include "common.cuh"
#include "cp_async.cuh"
#include "stream2d.h"
#include "tma.cuh"

namespace fasmg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kWin = 8;  // register window rows (power of two, even)

struct StripGeo {
  int x0;   // first column of the strip (may be negative)
  int xl;   // first column of this lane's 4 cells
  int y0, y1;  // output rows [y0, y1)
  bool lane_in;   // the lane's 4 columns are inside the domain
  bool lane_out;  // the lane writes its 4 columns
};

// HALO recomputed columns on each side of a 128-column strip: the pre-smoothing kernel needs
// kStripHalo (its residual and restriction read one column beyond the last colour phase); the
// post-smoothing kernel, whose last stage is the last colour phase, needs one column per phase. Its
// float64-update variant uses 4 (0.33 -> 0.32 ms per 8192^2 launch); the plain variant measured
// slower with 4 than with 8 (0.158 -> 0.170 ms) and keeps 8.
template <bool UPD>
constexpr int post_halo() { return UPD ? 4 : kStripHalo; }

template <int HALO>
__device__ __forceinline__ StripGeo strip_geo(int nx, int ny, int seg) {
  constexpr int OUT = 128 - 2 * HALO;
  const int warp = (blockIdx.x * kWarps) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int nstrips = (nx + OUT - 1) / OUT;
  const int strip = warp % nstrips;
  const int sg = warp / nstrips;
  StripGeo g;
  g.x0 = strip * OUT - HALO;
  g.xl = g.x0 + 4 * lane;
  g.y0 = sg * seg;
  g.y1 = min(g.y0 + seg, ny);
  g.lane_in = g.xl >= 0 && g.xl < nx;  // nx is a multiple of 4, so all 4 or none
  g.lane_out = g.lane_in && lane >= HALO / 4 && lane < (HALO + OUT) / 4;
  return g;
}

__device__ __forceinline__ void st4(float* base, int64_t off, float4 v) {
  *reinterpret_cast<float4*>(base + off) = v;
}

// Per-lane stencil constants: the x-boundary flags of the lane's 4 cells and, for rows away from the
// y boundary, their class constants in registers (no indexed constant loads on the common path).
struct LaneCoef {
  int xf;  // x-boundary flags of the 4 cells, 2 bits each
  float a[4], b[4];
};

__device__ __forceinline__ LaneCoef lane_coef(int xl, const LevelDesc<float>& L) {
  LaneCoef q;
  q.xf = 0;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int x = xl + v;
    const int fl = (x == 0) | ((x == L.nx - 1) << 1);
    q.xf |= fl << (2 * v);
    q.a[v] = L.a[fl];
    q.b[v] = L.b[fl];
  }
  return q;
}

template <int V>
__device__ __forceinline__ int xflag(const LaneCoef& q) {
  return (q.xf >> (2 * V)) & 3;
}

__device__ __forceinline__ int yflags(int y, int ny) { return ((y == 0) << 2) | ((y == ny - 1) << 3); }

// Gauss-Seidel update of cell v of the lane from its neighbour sum nb (same expression as
// point_update in common.cuh).
template <bool FAST, int V>
__device__ __forceinline__ float gs(float nb, float fv, int yf, const LaneCoef& q, const LevelDesc<float>& L,
                                    bool in, float old) {
  float a = q.a[V], b = q.b[V];
  if (FAST) return fmaf(a, nb, b * fv);
  if (yf) {
    a = L.a[xflag<V>(q) | yf];
    b = L.b[xflag<V>(q) | yf];
  }
  const float val = fmaf(a, nb, b * fv);
  return in ? val : old;
}

template <bool FAST, int V>
__device__ __forceinline__ float dcoef(int yf, const LaneCoef& q, const LevelDesc<float>& L) {
  return FAST ? L.d[0] : L.d[xflag<V>(q) | yf];
}

// One colour phase on a row: PAR = 0 updates cells v = 0, 2 of the lane; PAR = 1 cells v = 1, 3.
// NBZ: every neighbour of the updated cells is zero (the first phase from a zero initial guess: the
// cells of the other colour have not been touched), so the neighbour sum is +0 without reading them.
template <bool FAST, int PAR, bool NBZ = false>
__device__ __forceinline__ void phase_row(float4& c, const float4& s, const float4& n, const float4& fv, int y,
                                          const LaneCoef& q, const LevelDesc<float>& L, bool in) {
  const int yf = FAST ? 0 : yflags(y, L.ny);
  if (PAR == 0) {
    const float wv = NBZ ? 0.f : __shfl_up_sync(kFull, c.w, 1);
    c.x = gs<FAST, 0>(NBZ ? 0.f : (wv + c.y) + (s.x + n.x), fv.x, yf, q, L, in, c.x);
    c.z = gs<FAST, 2>(NBZ ? 0.f : (c.y + c.w) + (s.z + n.z), fv.z, yf, q, L, in, c.z);
  } else {
    const float ev = NBZ ? 0.f : __shfl_down_sync(kFull, c.x, 1);
    c.y = gs<FAST, 1>(NBZ ? 0.f : (c.x + c.z) + (s.y + n.y), fv.y, yf, q, L, in, c.y);
    c.w = gs<FAST, 3>(NBZ ? 0.f : (c.z + ev) + (s.w + n.w), fv.w, yf, q, L, in, c.w);
  }
}

// (A u) on the 4 cells of a row (same expression as apply_point).
template <bool FAST>
__device__ __forceinline__ float4 apply_row(const float4& c, const float4& s, const float4& n, int y,
                                            const LaneCoef& q, const LevelDesc<float>& L) {
  const int yf = FAST ? 0 : yflags(y, L.ny);
  const float wv = __shfl_up_sync(kFull, c.w, 1);
  const float ev = __shfl_down_sync(kFull, c.x, 1);
  float4 o;
  o.x = fmaf(dcoef<FAST, 0>(yf, q, L), c.x, -L.c * ((wv + c.y) + (s.x + n.x)));
  o.y = fmaf(dcoef<FAST, 1>(yf, q, L), c.y, -L.c * ((c.x + c.z) + (s.y + n.y)));
  o.z = fmaf(dcoef<FAST, 2>(yf, q, L), c.z, -L.c * ((c.y + c.w) + (s.z + n.z)));
  o.w = fmaf(dcoef<FAST, 3>(yf, q, L), c.w, -L.c * ((c.z + ev) + (s.w + n.w)));
  return o;
}

// r = f - A u on the 4 cells of a row (same expression as residual_point).
template <bool FAST>
__device__ __forceinline__ float4 resid_row(const float4& c, const float4& s, const float4& n, const float4& fv,
                                            int y, const LaneCoef& q, const LevelDesc<float>& L) {
  const int yf = FAST ? 0 : yflags(y, L.ny);
  const float wv = __shfl_up_sync(kFull, c.w, 1);
  const float ev = __shfl_down_sync(kFull, c.x, 1);
  float4 o;
  o.x = fmaf(L.c, (wv + c.y) + (s.x + n.x), fmaf(-dcoef<FAST, 0>(yf, q, L), c.x, fv.x));
  o.y = fmaf(L.c, (c.x + c.z) + (s.y + n.y), fmaf(-dcoef<FAST, 1>(yf, q, L), c.y, fv.y));
  o.z = fmaf(L.c, (c.y + c.w) + (s.z + n.z), fmaf(-dcoef<FAST, 2>(yf, q, L), c.z, fv.z));
  o.w = fmaf(L.c, (c.z + ev) + (s.w + n.w), fmaf(-dcoef<FAST, 3>(yf, q, L), c.w, fv.w));
  return o;
}

// 2x2 averages of a row pair (lo = row 2J, hi = row 2J+1): coarse cells (v0,v1) and (v2,v3).
__device__ __forceinline__ float2 avg_pair(const float4& lo, const float4& hi) {
  return make_float2(((lo.x + lo.y) + (hi.x + hi.y)) * 0.25f, ((lo.z + lo.w) + (hi.z + hi.w)) * 0.25f);
}

// Rows are prefetched PF iterations before their first use with per-lane 16-byte cp.async copies into
// a shared-memory ring of PF rows per warp, one commit group per row; cells outside the domain are
// zero-filled by the copy. Row y is taken from the ring once cp.async.wait_group leaves at most PF-1
// newer groups pending. PF divides kWin. (Prefetching 8 rows ahead measured slower for every kernel.)
constexpr int kPF = 4;      // post-smoothing
constexpr int kPFPre = 4;   // pre-smoothing that reads u
constexpr int kPFZero = 4;  // pre-smoothing from a zero start (its ring holds f only)

template <int PF, bool HAS_U>
struct PreRing {
  static constexpr int kDepth = PF;
  static constexpr bool kHasC = false;
  float4 u[HAS_U ? PF : 1][32];
  float4 f[PF][32];
};

template <bool UPD>
struct Ring {
  static constexpr int kDepth = kPF;
  static constexpr bool kHasC = true;
  float4 u[kPF][32];
  float4 f[kPF][32];
  float2 c[kPF][32];  // the coarse values of the row pair that ends at the slot's row
};
// The post-smoothing kernel that also updates a float64 field stages each output row's correction e
// (converted to float64) in shared memory; one lane adds the row to the float64 field with a bulk
// reduction in the L2 (u64 += e, rounded to nearest), so the kernel never reads u64 itself.
constexpr int kStage = 2;  // staged rows per warp whose bulk reductions may still be reading
template <>
struct Ring<true> {
  static constexpr int kDepth = kPF;
  static constexpr bool kHasC = true;
  float4 u[kPF][32];
  float4 f[kPF][32];
  float2 c[kPF][32];
  double e[kStage][128];
};

// Issue the copies of row y (u only when LOAD_U) into ring slot `slot`, then commit the group. In
// the post-smoothing rings (kHasC), a group of an odd row y also holds the lane's two coarse values of
// the row pair (y - 1, y), zero outside 1 <= y <= min(yend, ny - 1).
template <bool FAST, bool LOAD_U, typename RingT>
__device__ __forceinline__ void prefetch_row(RingT& R, int slot, const float* __restrict__ u,
                                             const float* __restrict__ f, int y, int ny, const StripGeo& g, int nx,
                                             const float* __restrict__ uc = nullptr, int yend = 0) {
  const int lane = threadIdx.x & 31;
  const bool valid = FAST || (y >= 0 && y < ny && g.lane_in);
  const int64_t off = valid ? (int64_t)y * nx + g.xl : 0;
  if constexpr (LOAD_U) cp_async16(&R.u[slot][lane], u + off, valid);
  cp_async16(&R.f[slot][lane], f + off, valid);
  if constexpr (RingT::kHasC) {
    if (y & 1) {
      const bool vc = y <= yend && y >= 1 && y < ny && g.lane_in;
      const int64_t oc = vc ? (int64_t)(y >> 1) * (nx >> 1) + (g.xl >> 1) : 0;
      cp_async8z(&R.c[slot][lane], uc + oc, vc);
    }
  }
  cp_async_commit();
}

// A warp is "interior" when every row its stream touches (including the halo, the rounding of the
// loop to whole windows and the prefetch distance) lies in 1..ny-2 and its strip in 1..nx-2: then no
// row or column test is needed and every cell has the interior stencil constants. Interior warps run
// the FAST instantiation of the body; the others the general one. Both compute the same values.
__device__ __forceinline__ bool interior(const StripGeo& g, int ystart, int yend, int nx, int ny, int pf) {
  const int ylast = ystart + ((yend - ystart) / kWin + 1) * kWin - 1 + pf;
  return ystart >= 1 && ylast <= ny - 2 && g.x0 >= 1 && g.x0 + 32 * 4 - 1 <= nx - 2;
}

// ------------------------------------------------------------------------------------------------
// pre-smoothing
//   uin  : initial u (ignored when ZERO: the initial guess is 0)
//   fin  : right-hand side f, or R(r) from the finer level when TAU (f = R(r) + A u is formed here)
//   fout : TAU only: the formed right-hand side (output rows), for the post-smoothing kernel
//   uout : u after NS sweeps (output rows)
//   uc, rc : R(u), R(r) on the next coarser level (nullable: no residual / restriction stage)
// ------------------------------------------------------------------------------------------------
template <int NS, bool ZERO, bool TAU>
using PreRingOf = PreRing<ZERO ? kPFZero : kPFPre, !ZERO>;

template <int NS, bool ZERO, bool TAU, bool FAST>
__device__ __forceinline__ void pre_body(PreRingOf<NS, ZERO, TAU>& R, const StripGeo& g, int ystart, int yend,
                                         const float* __restrict__ uin, const float* __restrict__ fin,
                                         float* __restrict__ fout, float* __restrict__ uout, float* __restrict__ uc,
                                         float* __restrict__ rc, const LevelDesc<float>& L) {
  constexpr int NP = 2 * NS;
  constexpr int LT = TAU ? 1 : 0;  // lag of the tau stage
  constexpr int LR = NP + 1 + LT;  // lag of the residual stage
  constexpr int M = kWin - 1;
  const int nx = L.nx, ny = L.ny;
  const int lane = threadIdx.x & 31;
  const LaneCoef q = lane_coef(g.xl, L);
  const bool do_res = uc != nullptr;
  float4 U[kWin], F[kWin];
  float4 rprev = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < kWin; ++k) {
    U[k] = rprev;
    F[k] = rprev;
  }
  constexpr int PF = PreRingOf<NS, ZERO, TAU>::kDepth;
#pragma unroll
  for (int k = 0; k < PF; ++k) prefetch_row<FAST, !ZERO>(R, k, uin, fin, ystart + k, ny, g, nx);
  const int nxc = nx >> 1;
  for (int yb = ystart; yb <= yend; yb += kWin) {
#pragma unroll
    for (int it = 0; it < kWin; ++it) {
      const int y = yb + it;
      // ---- take row y from the ring, prefetch row y + PF into its slot
      cp_async_wait<PF - 1>();
      U[it] = ZERO ? make_float4(0.f, 0.f, 0.f, 0.f) : R.u[it % PF][lane];
      F[it] = R.f[it % PF][lane];
      prefetch_row<FAST, !ZERO>(R, it % PF, uin, fin, y + PF, ny, g, nx);
      // ---- tau: f = R(r) + A u at row y-1 (u still the restricted start)
      if (TAU) {
        const int yt = y - 1;
        if (FAST || (yt >= 0 && yt < ny)) {
          const int s = (it - 1) & M;
          const float4 au = apply_row<FAST>(U[s], U[(s - 1) & M], U[(s + 1) & M], yt, q, L);
          float4& fr = F[s];
          fr.x = fr.x + au.x;
          fr.y = fr.y + au.y;
          fr.z = fr.z + au.z;
          fr.w = fr.w + au.w;
          if (g.lane_out && yt >= g.y0 && yt < g.y1) st4(fout, (int64_t)yt * nx + g.xl, fr);
        }
      }
      // ---- colour phases t = 1..NP at rows y - LT - t
#pragma unroll
      for (int t = 1; t <= NP; ++t) {
        const int yp = y - LT - t;
        if (FAST || (yp >= 0 && yp < ny)) {
          const int s = (it - LT - t) & M;
          // colour 1 (t odd): cells with (x + y) odd, i.e. v = (y+1)&1; colour 0: v = y&1
          const int par = (t & 1) ? ((it - LT - t + 1) & 1) : ((it - LT - t) & 1);
          if (ZERO && t == 1) {  // colour 1 from a zero start: its neighbours are all still zero
            if (par == 0)
              phase_row<FAST, 0, true>(U[s], U[(s - 1) & M], U[(s + 1) & M], F[s], yp, q, L, g.lane_in);
            else
              phase_row<FAST, 1, true>(U[s], U[(s - 1) & M], U[(s + 1) & M], F[s], yp, q, L, g.lane_in);
          } else if (par == 0) {
            phase_row<FAST, 0>(U[s], U[(s - 1) & M], U[(s + 1) & M], F[s], yp, q, L, g.lane_in);
          } else {
            phase_row<FAST, 1>(U[s], U[(s - 1) & M], U[(s + 1) & M], F[s], yp, q, L, g.lane_in);
          }
        }
      }
      // ---- store u, residual and restriction at row y - LR
      {
        const int yr = y - LR;
        const int s = (it - LR) & M;
        if (FAST || (yr >= 0 && yr < ny)) {
          if (g.lane_out && yr >= g.y0 && yr < g.y1) st4(uout, (int64_t)yr * nx + g.xl, U[s]);
          if (do_res && yr >= g.y0 && yr < g.y1) {  // only the segment's own row pairs are restricted
            const float4 r = resid_row<FAST>(U[s], U[(s - 1) & M], U[(s + 1) & M], F[s], yr, q, L);
            if (((it - LR) & 1) == 1) {  // odd row: the pair (yr-1, yr) is complete
              if (g.lane_out && yr - 1 >= g.y0 && yr < g.y1) {
                const int64_t coff = (int64_t)(yr >> 1) * nxc + (g.xl >> 1);
                const float2 cu = avg_pair(U[(s - 1) & M], U[s]);
                const float2 cr = avg_pair(rprev, r);
                *reinterpret_cast<float2*>(uc + coff) = cu;
                *reinterpret_cast<float2*>(rc + coff) = cr;
              }
            }
            rprev = r;
          }
        }
      }
    }
  }
  cp_async_wait_all();
}

template <int NS, bool ZERO, bool TAU>
__global__ void __launch_bounds__(kThreads, 2)
    k_pre(const float* __restrict__ uin, const float* __restrict__ fin, float* __restrict__ fout,
          float* __restrict__ uout, float* __restrict__ uc, float* __restrict__ rc,
          const __grid_constant__ LevelDesc<float> L, int seg) {
  constexpr int NP = 2 * NS;
  constexpr int LT = TAU ? 1 : 0;
  extern __shared__ __align__(16) unsigned char ring_smem[];
  using RingT = PreRingOf<NS, ZERO, TAU>;
  RingT* rings = reinterpret_cast<RingT*>(ring_smem);
  const StripGeo g = strip_geo<kStripHalo>(L.nx, L.ny, seg);
  if (g.y0 >= L.ny) return;  // whole warp: surplus warps of the last block
  const int ytop = g.y0 - (NP + 1 + LT);                                    // first row that must be loaded
  const int ystart = (ytop >= 0 ? ytop : ytop - (kWin - 1)) / kWin * kWin;  // floor to kWin
  const int yend = g.y1 + (uc != nullptr ? NP + 1 + LT : NP + LT);         // last pipeline row
  RingT& R = rings[threadIdx.x >> 5];
  if (interior(g, ystart, yend, L.nx, L.ny, RingT::kDepth))
    pre_body<NS, ZERO, TAU, true>(R, g, ystart, yend, uin, fin, fout, uout, uc, rc, L);
  else
    pre_body<NS, ZERO, TAU, false>(R, g, ystart, yend, uin, fin, fout, uout, uc, rc, L);
}

// ------------------------------------------------------------------------------------------------
// post-smoothing: uout = S^NS(uin + P(uc - R(uin)))
// ------------------------------------------------------------------------------------------------
template <int NS, bool FAST, bool UPD>
__device__ __forceinline__ void post_body(Ring<UPD>& R, const StripGeo& g, int ystart, int yend,
                                          const float* __restrict__ uin, const float* __restrict__ f,
                                          const float* __restrict__ uc, float* __restrict__ uout,
                                          double* __restrict__ u64, const LevelDesc<float>& L) {
  constexpr int NP = 2 * NS;
  constexpr int LW = NP + 1;  // lag of the store stage; phase t runs at row y - 1 - t
  constexpr int M = kWin - 1;
  const int nx = L.nx, ny = L.ny;
  const int lane = threadIdx.x & 31;
  const LaneCoef q = lane_coef(g.xl, L);
  float4 U[kWin], F[kWin];
#pragma unroll
  for (int k = 0; k < kWin; ++k) {
    U[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    F[k] = U[k];
  }
#pragma unroll
  for (int k = 0; k < kPF; ++k) prefetch_row<FAST, true>(R, k, uin, f, ystart + k, ny, g, nx, uc, yend);
  // UPD: the output lanes are H/4 .. H/4 + nout - 1 (the strip's first output column x0 + H is >= 0)
  constexpr int H = post_halo<UPD>();
  const int nout = min((128 - H) / 4, (nx - g.x0) / 4) - H / 4;
  int stage = 0;
  for (int yb = ystart; yb <= yend; yb += kWin) {
#pragma unroll
    for (int it = 0; it < kWin; ++it) {
      const int y = yb + it;
      cp_async_wait<kPF - 1>();
      U[it] = R.u[it % kPF][lane];
      F[it] = R.f[it % kPF][lane];
      // coarse-grid correction values of the row pair (y-1, y) (ystart is even: y odd when it is odd)
      const float2 cv = (it & 1) ? R.c[it % kPF][lane] : make_float2(0.f, 0.f);
      prefetch_row<FAST, true>(R, it % kPF, uin, f, y + kPF, ny, g, nx, uc, yend);
      const int yw = y - LW;
      const bool row_out = yw >= g.y0 && yw < g.y1;  // warp-uniform
      const bool wr = row_out && g.lane_out;
      // coarse-grid correction of the row pair (y-1, y)
      if ((it & 1) == 1 && (FAST || (y < ny && y >= 1 && g.lane_in))) {
        float4& lo = U[(it - 1) & M];
        float4& hi = U[it];
        const float2 ru = avg_pair(lo, hi);
        const float d0 = cv.x - ru.x, d1 = cv.y - ru.y;
        lo.x += d0;
        lo.y += d0;
        hi.x += d0;
        hi.y += d0;
        lo.z += d1;
        lo.w += d1;
        hi.z += d1;
        hi.w += d1;
      }
#pragma unroll
      for (int t = 1; t <= NP; ++t) {
        const int yp = y - 1 - t;
        if (FAST || (yp >= 0 && yp < ny)) {
          const int s = (it - 1 - t) & M;
          const int par = (t & 1) ? ((it - 1 - t + 1) & 1) : ((it - 1 - t) & 1);
          if (par == 0)
            phase_row<FAST, 0>(U[s], U[(s - 1) & M], U[(s + 1) & M], F[s], yp, q, L, g.lane_in);
          else
            phase_row<FAST, 1>(U[s], U[(s - 1) & M], U[(s + 1) & M], F[s], yp, q, L, g.lane_in);
        }
      }
      if constexpr (UPD) {  // mixed precision: u64 += e, the float64 update of the refinement step
        if (row_out) {
          double* st = R.e[stage];
          stage = (stage + 1) & (kStage - 1);
          if (lane == 0) bulk_wait_read<kStage - 1>();  // the slot's previous reduction has read it
          __syncwarp();
          if (g.lane_out) {
            const float4 e = U[(it - LW) & M];
            double2* d = reinterpret_cast<double2*>(st + 4 * lane);
            d[0] = make_double2(f32_to_f64_bits(e.x), f32_to_f64_bits(e.y));
            d[1] = make_double2(f32_to_f64_bits(e.z), f32_to_f64_bits(e.w));
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) {
            bulk_reduce_add_f64(u64 + (int64_t)yw * nx + g.x0 + H, st + H, (uint32_t)nout * 32u);
            bulk_commit();
          }
        }
      } else if (wr) {
        st4(uout, (int64_t)yw * nx + g.xl, U[(it - LW) & M]);
      }
    }
  }
  cp_async_wait_all();
  if constexpr (UPD) {
    if (lane == 0) bulk_wait_all();
  }
}

template <int NS, bool UPD>
__global__ void __launch_bounds__(kThreads, 2)
    k_post(const float* __restrict__ uin, const float* __restrict__ f, const float* __restrict__ uc,
           float* __restrict__ uout, double* __restrict__ u64, const __grid_constant__ LevelDesc<float> L,
           int seg) {
  constexpr int NP = 2 * NS;
  extern __shared__ __align__(16) unsigned char ring_smem[];
  Ring<UPD>* rings = reinterpret_cast<Ring<UPD>*>(ring_smem);
  const StripGeo g = strip_geo<post_halo<UPD>()>(L.nx, L.ny, seg);
  if (g.y0 >= L.ny) return;
  const int ytop = g.y0 - NP;  // even, so correction pairs stay aligned
  const int ystart = (ytop >= 0 ? ytop : ytop - (kWin - 1)) / kWin * kWin;
  const int yend = g.y1 + NP + 1;
  Ring<UPD>& R = rings[threadIdx.x >> 5];
  if (interior(g, ystart, yend, L.nx, L.ny, Ring<UPD>::kDepth))
    post_body<NS, true, UPD>(R, g, ystart, yend, uin, f, uc, uout, u64, L);
  else
    post_body<NS, false, UPD>(R, g, ystart, yend, uin, f, uc, uout, u64, L);
}

template <int HALO>
int blocks_for(int nx, int ny, int seg) {
  const int nstrips = (nx + (128 - 2 * HALO) - 1) / (128 - 2 * HALO);
  const int nsegs = (ny + seg - 1) / seg;
  return (nstrips * nsegs + kWarps - 1) / kWarps;
}

}  // namespace

// The 8-row window holds the rows one pre-smoothing pass needs for nu <= 2 (2 nu + 4 rows with tau).
bool stream2d_supported(int nx, int ny, int nu) {
  return nx >= 128 && ny >= 16 && (nx % 4) == 0 && (ny % 2) == 0 && nu >= 1 && nu <= 2;
}

#define PRE_CASE(NSV, Z, T)                                                                      \
  k_pre<NSV, Z, T><<<blocks_for<kStripHalo>(L.nx, L.ny, seg), kThreads, sizeof(PreRingOf<NSV, Z, T>) * kWarps, stream>>>( \
      uin, fin, fout, uout, uc, rc, L, seg)

cudaError_t launch_stream2d_pre(const float* uin, const float* fin, float* fout, float* uout, float* uc, float* rc,
                                const LevelDesc<float>& L, int nu, bool zero_init, bool tau, int seg,
                                cudaStream_t stream) {
  if (zero_init && tau) return cudaErrorInvalidValue;
  switch (nu) {
    case 1:
      if (zero_init) PRE_CASE(1, true, false);
      else if (tau) PRE_CASE(1, false, true);
      else PRE_CASE(1, false, false);
      break;
    case 2:
      if (zero_init) PRE_CASE(2, true, false);
      else if (tau) PRE_CASE(2, false, true);
      else PRE_CASE(2, false, false);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int NS>
cudaError_t pre_attr() {
  const auto a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_pre<NS, true, false>, a, (int)(sizeof(PreRingOf<NS, true, false>) * kWarps));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_pre<NS, false, false>, a, (int)(sizeof(PreRingOf<NS, false, false>) * kWarps));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_pre<NS, false, true>, a, (int)(sizeof(PreRingOf<NS, false, true>) * kWarps));
  return e;
}

// Shared-memory size attributes of every fused kernel, set once before any launch or stream capture.
cudaError_t stream2d_prepare() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    const int big = (int)(sizeof(Ring<true>) * kWarps);
    cudaError_t e = cudaFuncSetAttribute(k_post<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_post<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = pre_attr<1>();
    if (e == cudaSuccess) e = pre_attr<2>();
    err = e;
  });
  return err;
}

template <int NS, bool UPD>
cudaError_t post_launch(const float* uin, const float* f, const float* uc, float* uout, double* u64,
                        const LevelDesc<float>& L, int seg, cudaStream_t stream) {
  constexpr size_t smem = sizeof(Ring<UPD>) * kWarps;  // > 48 KB for UPD: set by stream2d_prepare
  k_post<NS, UPD><<<blocks_for<post_halo<UPD>()>(L.nx, L.ny, seg), kThreads, smem, stream>>>(uin, f, uc, uout, u64,
                                                                                            L, seg);
  return cudaGetLastError();
}

cudaError_t launch_stream2d_post(const float* uin, const float* f, const float* uc, float* uout, double* u64,
                                 const LevelDesc<float>& L, int nu, int seg, cudaStream_t stream) {
  switch (nu * 2 + (u64 != nullptr)) {
    case 2: return post_launch<1, false>(uin, f, uc, uout, u64, L, seg, stream);
    case 3: return post_launch<1, true>(uin, f, uc, uout, u64, L, seg, stream);
    case 4: return post_launch<2, false>(uin, f, uc, uout, u64, L, seg, stream);
    case 5: return post_launch<2, true>(uin, f, uc, uout, u64, L, seg, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fasmg
