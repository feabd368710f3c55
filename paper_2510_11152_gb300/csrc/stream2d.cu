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
//     correction, R(u) recomputed from the unchanged fine values) -> colour phases -> store.
//
// A colour phase updates the cells of one X-MCGS colour (Sec. 2.3; colour 1 = cells whose 1-based
// i+j is odd, the paper's sets 1 and 2) from their four neighbours. A row's cells of one colour only
// see the other colour, so stage t at row y reads rows y-1, y, y+1 after stage t-1, which the
// pipeline guarantees. West/east neighbours come from the lane itself or by one warp shuffle.
//
// Strips and segments overlap (8 columns each side, 5-7 rows at the top and bottom) and recompute
// their halos; only the interior is written. Because neighbours read the halo, nothing a warp reads
// may be written by this kernel: u is read from one buffer and written to another, and the tau
// right-hand side is kept in registers and written to a buffer separate from R(r).
//
// Arithmetic per point is the same expression as in basic_kernels.cuh (same association and fma
// placement), so a V-cycle through these kernels is bit-for-bit the V-cycle of the per-operation
// float32 kernels.
#include "common.cuh"
#include "stream2d.h"

namespace fasmg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kWin = 8;  // register window rows (power of two, even)

__device__ __forceinline__ int cls2(int x, int y, int nx, int ny) {
  return (x == 0) | ((x == nx - 1) << 1) | ((y == 0) << 2) | ((y == ny - 1) << 3);
}

struct StripGeo {
  int x0;   // first column of the strip (may be negative)
  int xl;   // first column of this lane's 4 cells
  int y0, y1;  // output rows [y0, y1)
  bool lane_in;   // the lane's 4 columns are inside the domain
  bool lane_out;  // the lane writes its 4 columns
};

__device__ __forceinline__ StripGeo strip_geo(int nx, int ny, int seg) {
  const int warp = (blockIdx.x * kWarps) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int nstrips = (nx + kStripOut - 1) / kStripOut;
  const int strip = warp % nstrips;
  const int sg = warp / nstrips;
  StripGeo g;
  g.x0 = strip * kStripOut - kStripHalo;
  g.xl = g.x0 + 4 * lane;
  g.y0 = sg * seg;
  g.y1 = min(g.y0 + seg, ny);
  g.lane_in = g.xl >= 0 && g.xl < nx;  // nx is a multiple of 4, so all 4 or none
  g.lane_out = g.lane_in && lane >= kStripHalo / 4 && lane < (kStripHalo + kStripOut) / 4;
  return g;
}

__device__ __forceinline__ float4 ld4(const float* base, int64_t off) {
  return *reinterpret_cast<const float4*>(base + off);
}
__device__ __forceinline__ void st4(float* base, int64_t off, float4 v) {
  *reinterpret_cast<float4*>(base + off) = v;
}

// Gauss-Seidel update of one cell (same expression as point_update in common.cuh).
__device__ __forceinline__ float gs(float w, float e, float s, float n, float fv, int x, int y,
                                   const LevelDesc<float>& L, float old) {
  const float nb = (w + e) + (s + n);
  const int c = cls2(x, y, L.nx, L.ny);
  const float v = fmaf(L.a[c], nb, L.b[c] * fv);
  return (x >= 0 && x < L.nx) ? v : old;
}

// One colour phase on a row: PAR = 0 updates cells v = 0, 2 of the lane; PAR = 1 cells v = 1, 3.
template <int PAR>
__device__ __forceinline__ void phase_row(float4& c, const float4& s, const float4& n, const float4& fv, int xl,
                                          int y, const LevelDesc<float>& L) {
  if (PAR == 0) {
    const float wv = __shfl_up_sync(kFull, c.w, 1);
    c.x = gs(wv, c.y, s.x, n.x, fv.x, xl, y, L, c.x);
    c.z = gs(c.y, c.w, s.z, n.z, fv.z, xl + 2, y, L, c.z);
  } else {
    const float ev = __shfl_down_sync(kFull, c.x, 1);
    c.y = gs(c.x, c.z, s.y, n.y, fv.y, xl + 1, y, L, c.y);
    c.w = gs(c.z, ev, s.w, n.w, fv.w, xl + 3, y, L, c.w);
  }
}

// (A u) on the 4 cells of a row (same expression as apply_point).
__device__ __forceinline__ float4 apply_row(const float4& c, const float4& s, const float4& n, int xl, int y,
                                            const LevelDesc<float>& L) {
  const float wv = __shfl_up_sync(kFull, c.w, 1);
  const float ev = __shfl_down_sync(kFull, c.x, 1);
  float4 o;
  int k;
  k = cls2(xl, y, L.nx, L.ny);
  o.x = fmaf(L.d[k], c.x, -L.c * ((wv + c.y) + (s.x + n.x)));
  k = cls2(xl + 1, y, L.nx, L.ny);
  o.y = fmaf(L.d[k], c.y, -L.c * ((c.x + c.z) + (s.y + n.y)));
  k = cls2(xl + 2, y, L.nx, L.ny);
  o.z = fmaf(L.d[k], c.z, -L.c * ((c.y + c.w) + (s.z + n.z)));
  k = cls2(xl + 3, y, L.nx, L.ny);
  o.w = fmaf(L.d[k], c.w, -L.c * ((c.z + ev) + (s.w + n.w)));
  return o;
}

// r = f - A u on the 4 cells of a row (same expression as residual_point).
__device__ __forceinline__ float4 resid_row(const float4& c, const float4& s, const float4& n, const float4& fv,
                                            int xl, int y, const LevelDesc<float>& L) {
  const float wv = __shfl_up_sync(kFull, c.w, 1);
  const float ev = __shfl_down_sync(kFull, c.x, 1);
  float4 o;
  int k;
  k = cls2(xl, y, L.nx, L.ny);
  o.x = fmaf(L.c, (wv + c.y) + (s.x + n.x), fmaf(-L.d[k], c.x, fv.x));
  k = cls2(xl + 1, y, L.nx, L.ny);
  o.y = fmaf(L.c, (c.x + c.z) + (s.y + n.y), fmaf(-L.d[k], c.y, fv.y));
  k = cls2(xl + 2, y, L.nx, L.ny);
  o.z = fmaf(L.c, (c.y + c.w) + (s.z + n.z), fmaf(-L.d[k], c.z, fv.z));
  k = cls2(xl + 3, y, L.nx, L.ny);
  o.w = fmaf(L.c, (c.z + ev) + (s.w + n.w), fmaf(-L.d[k], c.w, fv.w));
  return o;
}

// 2x2 averages of a row pair (lo = row 2J, hi = row 2J+1): coarse cells (v0,v1) and (v2,v3).
__device__ __forceinline__ float2 avg_pair(const float4& lo, const float4& hi) {
  return make_float2(((lo.x + lo.y) + (hi.x + hi.y)) * 0.25f, ((lo.z + lo.w) + (hi.z + hi.w)) * 0.25f);
}

// ------------------------------------------------------------------------------------------------
// pre-smoothing kernel
//   uin  : initial u (ignored when ZERO: the initial guess is 0)
//   fin  : right-hand side f, or R(r) from the finer level when TAU (f = R(r) + A u is formed here)
//   fout : TAU only: the formed right-hand side (output rows), for the post-smoothing kernel
//   uout : u after NS sweeps (output rows)
//   uc, rc : R(u), R(r) on the next coarser level (nullable: no residual / restriction stage)
// ------------------------------------------------------------------------------------------------
template <int NS, bool ZERO, bool TAU>
__global__ void __launch_bounds__(kThreads) k_pre(const float* __restrict__ uin, const float* __restrict__ fin,
                                                  float* __restrict__ fout, float* __restrict__ uout,
                                                  float* __restrict__ uc, float* __restrict__ rc,
                                                  const __grid_constant__ LevelDesc<float> L, int seg) {
  constexpr int NP = 2 * NS;
  constexpr int LT = TAU ? 1 : 0;        // lag of the tau stage
  constexpr int LR = NP + 1 + LT;        // lag of the residual stage
  const int nx = L.nx, ny = L.ny;
  const StripGeo g = strip_geo(nx, ny, seg);
  if (g.y0 >= ny) return;  // whole warp: surplus warps of the last block
  const bool do_res = uc != nullptr;
  const int ytop = g.y0 - (NP + 1 + LT);            // first row that must be loaded
  const int ystart = (ytop >= 0 ? ytop : ytop - (kWin - 1)) / kWin * kWin;  // floor to kWin
  const int yend = g.y1 + (do_res ? LR : NP + LT);  // last pipeline row

  float4 U[kWin], F[kWin];
  float4 rprev = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < kWin; ++k) {
    U[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    F[k] = U[k];
  }
  const int nxc = nx >> 1;
  for (int yb = ystart; yb <= yend; yb += kWin) {
#pragma unroll
    for (int it = 0; it < kWin; ++it) {
      const int y = yb + it;
      // ---- load row y
      {
        float4 uv = make_float4(0.f, 0.f, 0.f, 0.f), fv = uv;
        if (y >= 0 && y < ny && g.lane_in) {
          const int64_t off = (int64_t)y * nx + g.xl;
          if (!ZERO) uv = ld4(uin, off);
          fv = ld4(fin, off);
        }
        U[it] = uv;
        F[it] = fv;
      }
      // ---- tau: f = R(r) + A u at row y-1 (u still the restricted start)
      if (TAU) {
        const int yt = y - 1;
        if (yt >= 0 && yt < ny) {
          const int s = (it - 1) & (kWin - 1);
          const float4 au = apply_row(U[s], U[(s - 1) & (kWin - 1)], U[(s + 1) & (kWin - 1)], g.xl, yt, L);
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
        if (yp >= 0 && yp < ny) {
          const int s = (it - LT - t) & (kWin - 1);
          // colour 1 (t odd): cells with (x + y) odd, i.e. v = (y+1)&1; colour 0: v = y&1
          const int par = (t & 1) ? ((it - LT - t + 1) & 1) : ((it - LT - t) & 1);
          if (par == 0)
            phase_row<0>(U[s], U[(s - 1) & (kWin - 1)], U[(s + 1) & (kWin - 1)], F[s], g.xl, yp, L);
          else
            phase_row<1>(U[s], U[(s - 1) & (kWin - 1)], U[(s + 1) & (kWin - 1)], F[s], g.xl, yp, L);
        }
      }
      // ---- store u, residual and restriction at row y - LR
      {
        const int yr = y - LR;
        const int s = (it - LR) & (kWin - 1);
        if (yr >= 0 && yr < ny) {
          if (g.lane_out && yr >= g.y0 && yr < g.y1) st4(uout, (int64_t)yr * nx + g.xl, U[s]);
          if (do_res) {
            const float4 r = resid_row(U[s], U[(s - 1) & (kWin - 1)], U[(s + 1) & (kWin - 1)], F[s], g.xl, yr, L);
            if (((it - LR) & 1) == 1) {  // odd row: the pair (yr-1, yr) is complete
              if (g.lane_out && yr - 1 >= g.y0 && yr < g.y1) {
                const int64_t coff = (int64_t)(yr >> 1) * nxc + (g.xl >> 1);
                const float2 cu = avg_pair(U[(s - 1) & (kWin - 1)], U[s]);
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
}

// ------------------------------------------------------------------------------------------------
// post-smoothing kernel: uout = S^NS(uin + P(uc - R(uin)))
// ------------------------------------------------------------------------------------------------
template <int NS>
__global__ void __launch_bounds__(kThreads) k_post(const float* __restrict__ uin, const float* __restrict__ f,
                                                   const float* __restrict__ uc, float* __restrict__ uout,
                                                   const __grid_constant__ LevelDesc<float> L, int seg) {
  constexpr int NP = 2 * NS;
  constexpr int LW = NP + 1;  // lag of the store stage; phase t runs at row y - 1 - t
  const int nx = L.nx, ny = L.ny;
  const StripGeo g = strip_geo(nx, ny, seg);
  if (g.y0 >= ny) return;
  const int ytop = g.y0 - NP;  // even, so correction pairs stay aligned
  const int ystart = (ytop >= 0 ? ytop : ytop - (kWin - 1)) / kWin * kWin;
  const int yend = g.y1 + LW;
  float4 U[kWin], F[kWin];
#pragma unroll
  for (int k = 0; k < kWin; ++k) {
    U[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    F[k] = U[k];
  }
  const int nxc = nx >> 1;
  for (int yb = ystart; yb <= yend; yb += kWin) {
#pragma unroll
    for (int it = 0; it < kWin; ++it) {
      const int y = yb + it;
      {
        float4 uv = make_float4(0.f, 0.f, 0.f, 0.f), fv = uv;
        if (y >= 0 && y < ny && g.lane_in) {
          const int64_t off = (int64_t)y * nx + g.xl;
          uv = ld4(uin, off);
          fv = ld4(f, off);
        }
        U[it] = uv;
        F[it] = fv;
      }
      // coarse-grid correction of the row pair (y-1, y)
      if ((it & 1) == 1 && y < ny && y >= 1 && g.lane_in) {
        float4& lo = U[(it - 1) & (kWin - 1)];
        float4& hi = U[it];
        const float2 cv = *reinterpret_cast<const float2*>(uc + (int64_t)(y >> 1) * nxc + (g.xl >> 1));
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
        if (yp >= 0 && yp < ny) {
          const int s = (it - 1 - t) & (kWin - 1);
          const int par = (t & 1) ? ((it - 1 - t + 1) & 1) : ((it - 1 - t) & 1);
          if (par == 0)
            phase_row<0>(U[s], U[(s - 1) & (kWin - 1)], U[(s + 1) & (kWin - 1)], F[s], g.xl, yp, L);
          else
            phase_row<1>(U[s], U[(s - 1) & (kWin - 1)], U[(s + 1) & (kWin - 1)], F[s], g.xl, yp, L);
        }
      }
      {
        const int yw = y - LW;
        const int s = (it - LW) & (kWin - 1);
        if (yw >= g.y0 && yw < g.y1 && g.lane_out) st4(uout, (int64_t)yw * nx + g.xl, U[s]);
      }
    }
  }
}

int blocks_for(int nx, int ny, int seg) {
  const int nstrips = (nx + kStripOut - 1) / kStripOut;
  const int nsegs = (ny + seg - 1) / seg;
  return (nstrips * nsegs + kWarps - 1) / kWarps;
}

}  // namespace

// The 8-row window holds the rows one pre-smoothing pass needs for nu <= 2 (2 nu + 4 rows with tau).
bool stream2d_supported(int nx, int ny, int nu) {
  return nx >= 128 && ny >= 16 && (nx % 4) == 0 && (ny % 2) == 0 && nu >= 1 && nu <= 2;
}

#define PRE_CASE(NSV, Z, T)                                                                      \
  k_pre<NSV, Z, T><<<blocks_for(L.nx, L.ny, seg), kThreads, 0, stream>>>(uin, fin, fout, uout, uc, rc, L, seg)

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

cudaError_t launch_stream2d_post(const float* uin, const float* f, const float* uc, float* uout,
                                 const LevelDesc<float>& L, int nu, int seg, cudaStream_t stream) {
  const int b = blocks_for(L.nx, L.ny, seg);
  switch (nu) {
    case 1: k_post<1><<<b, kThreads, 0, stream>>>(uin, f, uc, uout, L, seg); break;
    case 2: k_post<2><<<b, kThreads, 0, stream>>>(uin, f, uc, uout, L, seg); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fasmg
