// ir_strip.cu -- the float64 refinement residual r32 = (float)(b - A u) of the mixed-precision solve
// with a constant diffusivity, and its norm: 2D cell-centred levels, and 3D levels (cells or faces).
//
// GB300 runs float64 arithmetic at 1/64 of the float32 rate, which makes this kernel, not HBM, the
// bottleneck of a refinement step when evaluated as five float64 operations per cell. Here the
// stencil difference S = sum_nb u_nb - M u (M the diagonal's neighbour count plus boundary
// multiplicities) is summed exactly in 64-bit integers: each value's significand is unpacked once,
// aligned to the smallest exponent of the rows around the output row, and the point equation
// becomes r = fma(c, S, fma(-alpha, u, b)) (bits64.cuh). One warp owns a strip of 128 columns (four
// per lane) and walks a segment of rows (2D) or planes (3D) keeping the neighbouring ones unpacked in
// registers; horizontal neighbours come from the adjacent lanes, the strip's outer neighbours from
// two extra loads. Windows whose values span more than 2^kMaxExpSpread in magnitude, or hold a
// subnormal or non-finite value (2D: also a zero or values of both signs), take the float64 point
// equation instead (the warp decides per row).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "bits64.cuh"
#include "common.cuh"
#include "ir_strip.h"

namespace fasmg {
namespace {

constexpr int kIrWarps = 8;
constexpr int kIrThreads = 32 * kIrWarps;
constexpr int kIrCols = 128;  // columns per strip of the 3D kernel (4 per lane); 2D strips are 32 CPL wide
constexpr int kIrCpl2D = 4;   // cells per lane of the 2D kernel
constexpr int kIrMinBlocks2D = 2;
constexpr int kIrTasksPerWarp = 6;  // 2D work items per warp, taken dynamically
constexpr unsigned kAll = 0xffffffffu;
constexpr int kExpNone = 1 << 20;  // neutral bounds of an absent row; -kExpNone marks a bad value

// The same row as loaded from memory (bit patterns), before unpacking.
template <int CPL>
struct IrRaw {
  uint64_t v[CPL];
  uint64_t halo;  // lane 0: the cell left of the strip; lane 31: the cell right of it (else 0)
};

// One row of a lane's CPL cells (x0 .. x0+CPL-1) for the exact path of the 2D kernel: the magnitudes
// of the significands (implicit bit included) aligned to the row's smallest exponent, and
// t = fma(-alpha, u, b), the part of the point equation outside the stencil difference.
template <int CPL>
struct IrRowM {
  double t[CPL];
  uint64_t X[CPL];  // |significand| 2^(E - E_lo)
  uint64_t hX;      // lanes 0 / 31: the strip's outer neighbour, aligned likewise (0 where absent)
  int kmin, kmax;   // warp-wide min / max of key = (sign << 11) | E over the row and its halo
};
constexpr int kKeyNone = 1 << 20;  // kmin of an absent row (kmax: -1)

// The bit pattern of a normal float64 from its unpacked form.
__device__ __forceinline__ uint64_t repack(int64_t sig, int E) {
  const uint64_t neg = sig < 0 ? 1ull : 0ull;
  const uint64_t m = neg ? (uint64_t)(-sig) : (uint64_t)sig;
  return (neg << 63) | ((uint64_t)E << 52) | (m & kMant52);
}

__device__ __forceinline__ bool bad_exp(int E) { return (unsigned)(E - 1) >= 2046u; }

__device__ __forceinline__ double as_d(uint64_t v) { return __longlong_as_double((long long)v); }

// |significand| of the float64 with bit pattern v and key (sign << 11) | E, times 2^(E - lo) (the
// shift is taken mod 32: only rows whose exponents span at most kMaxExpSpread are used).
__device__ __forceinline__ uint64_t mag_aligned(uint64_t v, int key, int lo) {
  const uint32_t l = (uint32_t)v;
  const uint32_t m = ((uint32_t)(v >> 32) & 0xFFFFFu) | 0x100000u;
  const int sh = ((key & 0x7FF) - lo) & 31;
  return ((uint64_t)__funnelshift_l(l, m, sh) << 32) | (uint64_t)(l << sh);
}

// CPL consecutive float64 values from 16-byte aligned p (CPL = 2 or 4)
template <int CPL>
__device__ __forceinline__ void ld_vals(double (&v)[CPL], const double* __restrict__ p) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < CPL / 2; ++k) {
    const double2 t = q[k];
    v[2 * k] = t.x;
    v[2 * k + 1] = t.y;
  }
}

template <int CPL>
__device__ __forceinline__ void load_raw(IrRaw<CPL>& R, const double* __restrict__ u, int y, int nx, int ny, int x0,
                                         int lane) {
  R.halo = 0ull;
  if (y >= 0 && y < ny) {
    const int64_t base = (int64_t)y * nx + x0;
    double v[CPL];
    ld_vals<CPL>(v, u + base);
#pragma unroll
    for (int k = 0; k < CPL; ++k) R.v[k] = (uint64_t)__double_as_longlong(v[k]);
    if ((lane == 0 && x0 > 0) || (lane == 31 && x0 + CPL < nx))
      R.halo = (uint64_t)__double_as_longlong(u[lane == 0 ? base - 1 : base + CPL]);
  } else {
#pragma unroll
    for (int k = 0; k < CPL; ++k) R.v[k] = 0ull;
  }
}

// b of row y (zeros outside the grid)
template <int CPL>
__device__ __forceinline__ void load_b(double (&v)[CPL], const double* __restrict__ b, int y, int nx, int ny, int x0) {
  if (y >= 0 && y < ny) {
    ld_vals<CPL>(v, b + (int64_t)y * nx + x0);
  } else {
#pragma unroll
    for (int k = 0; k < CPL; ++k) v[k] = 0.0;
  }
}

template <int CPL>
__device__ __forceinline__ void unpack_rowM(IrRowM<CPL>& R, const IrRaw<CPL>& W, const double (&bw)[CPL], double alpha,
                                            bool present, int x0, int nx, int lane) {
  if (!present) {  // the same on every lane
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
      R.t[k] = 0.0;
      R.X[k] = 0ull;
    }
    R.hX = 0ull;
    R.kmin = kKeyNone;
    R.kmax = -1;
    return;
  }
  int key[CPL];
  int kmin = kKeyNone, kmax = -1;
#pragma unroll
  for (int k = 0; k < CPL; ++k) {
    key[k] = (int)(W.v[k] >> 52);
    kmin = min(kmin, key[k]);
    kmax = max(kmax, key[k]);
  }
  const bool has_halo = (lane == 0 && x0 > 0) || (lane == 31 && x0 + CPL < nx);
  const int hkey = (int)(W.halo >> 52);
  if (has_halo) {
    kmin = min(kmin, hkey);
    kmax = max(kmax, hkey);
  }
  R.kmin = __reduce_min_sync(kAll, kmin);
  R.kmax = __reduce_max_sync(kAll, kmax);
  const int lo = R.kmin & 0x7FF;
#pragma unroll
  for (int k = 0; k < CPL; ++k) {
    R.t[k] = fma(-alpha, as_d(W.v[k]), bw[k]);
    R.X[k] = mag_aligned(W.v[k], key[k], lo);
  }
  R.hX = has_halo ? mag_aligned(W.halo, hkey, lo) : 0ull;
}

template <int CPL>
__device__ __forceinline__ void store_r32(float* p, const float (&o)[CPL]) {
  if constexpr (CPL == 4)
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  else
    *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
}

// One output row y of the 2D kernel. P, C hold rows y-1, y; N receives row y+1 from `pend` (u) and
// `bnext` (b), which are refilled with row y+2.
//
// Exact path (decided per warp row): every value of the three rows (and the strip's outer
// neighbours) is a normal float64 of the same sign sigma, and their exponents span at most
// kMaxExpSpread binades. Then S = sum_nb u_nb - M u_c = sigma (sum_nb |u_nb| - M |u_c|) is summed
// exactly on the significand magnitudes aligned to the smallest exponent Eref of the window
// (|terms| < 2^58, |S| < 2^61) and rounded once; r = fma(c, S, fma(-alpha, u_c, b)). Otherwise the
// float64 point equation from the values in memory.
template <int CPL>
__device__ __forceinline__ void ir_row(const IrRowM<CPL>& P, const IrRowM<CPL>& C, IrRowM<CPL>& N, IrRaw<CPL>& pend,
                                       double (&bnext)[CPL], int y, float* __restrict__ r32, const double* __restrict__ u,
                                       const double* __restrict__ b, const LevelDesc<double>& L, int x0, int lane,
                                       float nscale, float& acc) {
  const int nx = L.nx, ny = L.ny;
  // row y+1 arrives from the loads issued one row earlier; row y+2 is requested now
  unpack_rowM<CPL>(N, pend, bnext, L.alpha, y + 1 < ny, x0, nx, lane);
  load_raw<CPL>(pend, u, y + 2, nx, ny, x0, lane);
  load_b<CPL>(bnext, b, y + 2, nx, ny, x0);
  const int64_t bb = (int64_t)y * nx + x0;
  double r[CPL];
  const int kmin = min(C.kmin, min(P.kmin, N.kmin));
  const int kmax = max(C.kmax, max(P.kmax, N.kmax));
  const int Eref = kmin & 0x7FF, Etop = kmax & 0x7FF;
  // the same on every lane: one sign, normal values, exponent spread
  bool exact = (kmin ^ kmax) < 0x800 && Eref >= 1 && Etop <= 2046 && Etop - Eref <= kMaxExpSpread;
  if (exact) {
    uint64_t xp[CPL], xc[CPL], xn[CPL];
    uint64_t hx = C.hX;
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
      xp[k] = P.X[k];
      xc[k] = C.X[k];
      xn[k] = N.X[k];
    }
    // rows whose smallest exponent is above Eref: shift them to it (absent rows hold zeros)
    const int dP = P.kmin < kKeyNone ? (P.kmin & 0x7FF) - Eref : 0;
    const int dC = (C.kmin & 0x7FF) - Eref;
    const int dN = N.kmin < kKeyNone ? (N.kmin & 0x7FF) - Eref : 0;
    if (dP | dC | dN) {
#pragma unroll
      for (int k = 0; k < CPL; ++k) {
        xp[k] <<= dP;
        xc[k] <<= dC;
        xn[k] <<= dN;
      }
      hx <<= dC;
    }
    uint64_t wl = (uint64_t)__shfl_up_sync(kAll, (long long)xc[CPL - 1], 1);
    uint64_t er = (uint64_t)__shfl_down_sync(kAll, (long long)xc[0], 1);
    if (lane == 0) wl = hx;
    if (lane == 31) er = hx;
    int64_t S[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
      const uint64_t Xw = k ? xc[k - 1] : wl;
      const uint64_t Xe = k < CPL - 1 ? xc[k + 1] : er;
      S[k] = (int64_t)((Xw + Xe) + (xp[k] + xn[k])) - (int64_t)(xc[k] << 2);
    }
    // boundary cells: absent neighbours are 0 above; the diagonal count is mt, not 4
    if (y == 0 || y == ny - 1) {
#pragma unroll
      for (int k = 0; k < CPL; ++k) {
        const int cls = bclass<2>(x0 + k, y, 0, nx, ny, 1);
        S[k] += (4 - (int64_t)L.mt[cls]) * (int64_t)xc[k];
      }
    } else {
      if (x0 == 0) S[0] += (4 - (int64_t)L.mt[bclass<2>(0, y, 0, nx, ny, 1)]) * (int64_t)xc[0];
      if (x0 + CPL == nx) S[CPL - 1] += (4 - (int64_t)L.mt[bclass<2>(nx - 1, y, 0, nx, ny, 1)]) * (int64_t)xc[CPL - 1];
    }
    uint64_t A[CPL];
    int pw[CPL];
    bool small = true;
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
      A[k] = S[k] < 0 ? (uint64_t)(-S[k]) : (uint64_t)S[k];
      pw[k] = 63 - __clzll((long long)A[k]);  // -1 for S = 0
      small = small && pw[k] <= 52;
    }
    const uint32_t sgm = (uint32_t)(kmin >> 11) << 31;  // sigma
    double Sd[CPL];
    bool ok = true;
    if (__all_sync(kAll, small)) {
      // |S| < 2^53: exact; |S| 2^(Eref - 1075) = A 2^(52 - p) with the implicit bit adding one to the
      // exponent field (Eref + p - 53)
#pragma unroll
      for (int k = 0; k < CPL; ++k) {
        const uint64_t q = A[k] << ((52 - pw[k]) & 63);
        const uint32_t sg = ((uint32_t)(S[k] < 0) << 31) ^ sgm;
        const uint32_t hw = ((uint32_t)(q >> 32) + ((uint32_t)(Eref + pw[k] - 53) << 20)) | sg;
        Sd[k] = A[k] ? __hiloint2double((int)hw, (int)(uint32_t)q) : 0.0;
        ok = ok && (A[k] == 0 || Eref + pw[k] >= 53);
      }
    } else {
#pragma unroll
      for (int k = 0; k < CPL; ++k) {
        ok = fixed_to_f64(S[k], Eref, &Sd[k]) && ok;
        Sd[k] = as_d((uint64_t)__double_as_longlong(Sd[k]) ^ ((uint64_t)sgm << 32));
      }
    }
#pragma unroll
    for (int k = 0; k < CPL; ++k) r[k] = fma(L.c, Sd[k], C.t[k]);
    exact = __all_sync(kAll, ok);
  }
  if (!exact) {  // the float64 point equation, as in residual_point, from the values in memory
    const double* __restrict__ uc = u + bb;
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
      const int x = x0 + k;
      const double w = x > 0 ? uc[k - 1] : 0.0;
      const double e = x < nx - 1 ? uc[k + 1] : 0.0;
      const double s = y > 0 ? uc[k - nx] : 0.0;
      const double n = y < ny - 1 ? uc[k + nx] : 0.0;
      const double nb = (w + e) + (s + n);
      const int cls = bclass<2>(x, y, 0, nx, ny, 1);
      r[k] = fma(L.c, nb, fma(-L.d[cls], uc[k], b[bb + k]));
    }
  }
  float o[CPL];
  bool nrm = true;
#pragma unroll
  for (int k = 0; k < CPL; ++k) nrm = nrm && f32_normal_range(r[k]);
  if (__all_sync(kAll, nrm)) {
#pragma unroll
    for (int k = 0; k < CPL; ++k) o[k] = f64_to_f32_rn_normal(r[k]);
  } else {
#pragma unroll
    for (int k = 0; k < CPL; ++k) o[k] = f64_to_f32_rn_bits(r[k]);
  }
  store_r32<CPL>(r32 + bb, o);
#pragma unroll
  for (int k = 0; k < CPL; ++k) {
    const float sk = o[k] * nscale;
    acc = fmaf(sk, sk, acc);
  }
}

// 2D: a warp takes tasks (a strip of 32 CPL columns and a segment of rows) from ticket[0] until none
// is left; the last block to finish sets both counters back to zero for the next launch. Segments near
// a sign change of u cost more (their rows take the float64 path), so tasks are handed out as warps
// become free instead of in a fixed share. r32 does not depend on that assignment; the per-block
// partial sums of its squares do, so the norm's last bits (float32 accumulation order) may differ
// from one launch to the next. (Writing one partial per task instead, in a fixed order, made the
// kernel 17 % slower.)
template <int CPL, int MINB>
__global__ void __launch_bounds__(kIrThreads, MINB)
    k_ir_strip(float* __restrict__ r32, const double* __restrict__ u, const double* __restrict__ b, LevelDesc<double> L,
               const float* nsp, double* partials, unsigned* ticket, int seg) {
  constexpr int COLS = 32 * CPL;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nx = L.nx, ny = L.ny;
  const int nstrips = nx / COLS;
  const int nseg = (ny + seg - 1) / seg;
  const int ntasks = nstrips * nseg;
  const float nscale = nsp ? *nsp : 1.f;
  float acc = 0.f;
  (void)warp;
  for (;;) {
    unsigned tk = 0;
    if (lane == 0) tk = atomicAdd(ticket, 1u);
    const int task = (int)__shfl_sync(kAll, tk, 0);
    if (task >= ntasks) break;
    const int sx = task % nstrips, sy = task / nstrips;
    const int x0 = sx * COLS + CPL * lane;
    const int y0 = sy * seg, y1 = min(ny, y0 + seg);
    IrRowM<CPL> R0, R1, R2;  // rows y-1, y, y+1
    IrRaw<CPL> pend;
    double bnext[CPL];
    load_raw<CPL>(pend, u, y0 - 1, nx, ny, x0, lane);
    load_b<CPL>(bnext, b, y0 - 1, nx, ny, x0);
    unpack_rowM<CPL>(R0, pend, bnext, L.alpha, y0 - 1 >= 0, x0, nx, lane);
    load_raw<CPL>(pend, u, y0, nx, ny, x0, lane);
    load_b<CPL>(bnext, b, y0, nx, ny, x0);
    unpack_rowM<CPL>(R1, pend, bnext, L.alpha, true, x0, nx, lane);
    load_raw<CPL>(pend, u, y0 + 1, nx, ny, x0, lane);
    load_b<CPL>(bnext, b, y0 + 1, nx, ny, x0);
    for (int y = y0; y < y1; ++y) {
      ir_row<CPL>(R0, R1, R2, pend, bnext, y, r32, u, b, L, x0, lane, nscale, acc);
      R0 = R1;
      R1 = R2;
    }
  }
  const double s = block_sum((double)acc);  // every warp of the block has left the task loop
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    if (atomicAdd(ticket + 1, 1u) == gridDim.x - 1) {  // the last block: no warp takes tasks any more
      ticket[0] = 0u;
      ticket[1] = 0u;
    }
  }
}

// ------------------------------------------------------------------------------------------------
// 3D (cell-centred or face grids, constant kappa): a warp owns a 128-column strip of one row y and
// walks a segment of planes z with the planes z-1, z, z+1 of its row unpacked in registers; the rows
// y-1 and y+1 of the current plane are read by the neighbouring warps of the block too (eight
// consecutive rows per block), so they come from L1. Exact zeros (the wall slots of face grids, a
// fluid at rest) are exact values here: significand 0, outside the exponent range. Each lane decides
// for its own four cells whether their stencils' values (its window of 22) qualify for the exact
// sum: a 3D row of 128 cells of a smooth field spans more than 2^5 far more often than that.
// ------------------------------------------------------------------------------------------------
constexpr int kIr3Rows = kIrWarps;  // rows y per block

struct IrRow3 {
  int64_t sig[4];
  int E[4];
  uint64_t halo;
  int lo, hi;
  bool present;
};

__device__ __forceinline__ void unpack_z(uint64_t raw, int64_t& sig, int& E, int& lo, int& hi, bool& bad) {
  E = (int)((raw >> 52) & 0x7FF);
  const bool zero = (raw << 1) == 0ull;
  const int64_t m = (int64_t)((raw & kMant52) | (1ull << 52));
  sig = zero ? 0 : ((raw >> 63) ? -m : m);
  if (!zero) {
    lo = min(lo, E);
    hi = max(hi, E);
    bad = bad || bad_exp(E);
  }
}

// sig 2^(E - Eref); zeros (sig 0) give 0 whatever their exponent field
__device__ __forceinline__ int64_t align_z(int64_t sig, int E, int Eref) {
  return (int64_t)((uint64_t)sig << ((E - Eref) & 63));
}

__device__ __forceinline__ void load_row3(IrRow3& R, const double* __restrict__ u, int64_t base, bool present,
                                          int x0, int nx, int lane, bool halos) {
  R.present = present;
  int lo = kExpNone, hi = -kExpNone;
  bool bad = false;
  R.halo = 0ull;
  if (present) {
    const double2 a = reinterpret_cast<const double2*>(u + base)[0];
    const double2 b = reinterpret_cast<const double2*>(u + base)[1];
    const uint64_t v[4] = {(uint64_t)__double_as_longlong(a.x), (uint64_t)__double_as_longlong(a.y),
                           (uint64_t)__double_as_longlong(b.x), (uint64_t)__double_as_longlong(b.y)};
#pragma unroll
    for (int k = 0; k < 4; ++k) unpack_z(v[k], R.sig[k], R.E[k], lo, hi, bad);
    if (halos && ((lane == 0 && x0 > 0) || (lane == 31 && x0 + 4 < nx))) {
      R.halo = (uint64_t)__double_as_longlong(u[lane == 0 ? base - 1 : base + 4]);
      int64_t hs;
      int Eh;
      unpack_z(R.halo, hs, Eh, lo, hi, bad);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      R.sig[k] = 0;
      R.E[k] = 0;
    }
  }
  R.lo = bad ? -kExpNone : lo;  // this lane's values only: the exact path is decided per lane
  R.hi = hi;
}

__global__ void __launch_bounds__(kIrThreads, 2)
    k_ir_strip3(float* __restrict__ r32, const double* __restrict__ u, const double* __restrict__ b,
                LevelDesc<double> L, const float* nsp, double* partials, int zseg) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  const int nstrips = nx / kIrCols;
  const int nyg = ny / kIr3Rows;
  const int nzs = (nz + zseg - 1) / zseg;
  const int ntasks = nstrips * nyg * nzs;
  const float nscale = nsp ? *nsp : 1.f;
  float acc = 0.f;
  for (int task = blockIdx.x; task < ntasks; task += gridDim.x) {
    const int sx = task % nstrips;
    const int rest = task / nstrips;
    const int y = (rest % nyg) * kIr3Rows + warp;
    const int z0 = (rest / nyg) * zseg, z1 = min(nz, z0 + zseg);
    const int x0 = sx * kIrCols + 4 * lane;
    const int64_t rowb = (int64_t)y * sy + x0;
    IrRow3 P, C, N;
    load_row3(P, u, rowb + (int64_t)(z0 - 1) * sz, z0 - 1 >= 0, x0, nx, lane, true);
    load_row3(C, u, rowb + (int64_t)z0 * sz, true, x0, nx, lane, true);
    for (int z = z0; z < z1; ++z) {
      load_row3(N, u, rowb + (int64_t)(z + 1) * sz, z + 1 < nz, x0, nx, lane, true);
      const int64_t cb = rowb + (int64_t)z * sz;
      IrRow3 S, T;  // rows y-1 and y+1 of plane z
      load_row3(S, u, cb - sy, y > 0, x0, nx, lane, false);
      load_row3(T, u, cb + sy, y < ny - 1, x0, nx, lane, false);
      const double2 b01 = reinterpret_cast<const double2*>(b + cb)[0];
      const double2 b23 = reinterpret_cast<const double2*>(b + cb)[1];
      const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
      double r[4];
      // The lane's window: its four cells in the five rows and their two horizontal neighbours (from
      // the adjacent lanes, or the strip's outer neighbours on lanes 0 and 31), unpacked.
      long long sw = __shfl_up_sync(kAll, (long long)C.sig[3], 1);
      int ew = __shfl_up_sync(kAll, C.E[3], 1);
      long long se = __shfl_down_sync(kAll, (long long)C.sig[0], 1);
      int ee = __shfl_down_sync(kAll, C.E[0], 1);
      if (lane == 0 || lane == 31) {
        int64_t hs = 0;
        int Eh = 0, l0 = 0, h0 = 0;
        bool bd = false;
        unpack_z(C.halo, hs, Eh, l0, h0, bd);  // 0 where the strip has no outer neighbour
        if (lane == 0) {
          sw = hs;
          ew = Eh;
        } else {
          se = hs;
          ee = Eh;
        }
      }
      int Eref = min(min(C.lo, min(P.lo, N.lo)), min(S.lo, T.lo));
      int Etop = max(max(C.hi, max(P.hi, N.hi)), max(S.hi, T.hi));
      if (sw != 0) {
        Eref = bad_exp(ew) ? -kExpNone : min(Eref, ew);
        Etop = max(Etop, ew);
      }
      if (se != 0) {
        Eref = bad_exp(ee) ? -kExpNone : min(Eref, ee);
        Etop = max(Etop, ee);
      }
      // an all-zero window has Eref = kExpNone: any exponent works, use 1
      const int Eb = Eref == kExpNone ? 1 : Eref;
      const bool want = Etop - Eref <= kMaxExpSpread || Eref == kExpNone;
      bool ok = want;
      if (want) {  // per lane; nothing below synchronises the warp
        int64_t Xc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) Xc[k] = align_z(C.sig[k], C.E[k], Eb);
        const int64_t wl = align_z(sw, ew, Eb), er = align_z(se, ee, Eb);
        const bool inner = y > 0 && y < ny - 1 && z > 0 && z < nz - 1;
        int64_t Sx[4];
        bool small = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int64_t Xw = k ? Xc[k - 1] : wl;
          const int64_t Xe = k < 3 ? Xc[k + 1] : er;
          const int64_t V = (align_z(S.sig[k], S.E[k], Eb) + align_z(T.sig[k], T.E[k], Eb)) +
                            (align_z(P.sig[k], P.E[k], Eb) + align_z(N.sig[k], N.E[k], Eb));
          int M = 6;
          if (!inner || (k == 0 && x0 == 0) || (k == 3 && x0 + 4 == nx)) {
            const int cls = bclass<3>(x0 + k, y, z, nx, ny, nz);
            M = (int)L.mt[cls];
          }
          Sx[k] = (Xw + Xe) + V - (int64_t)M * Xc[k];
          small = small && (uint64_t)(Sx[k] + ((1ll << 53) - 1)) < (1ull << 54) - 1ull;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          double Sd;
          ok = (small ? fixed_to_f64_small(Sx[k], Eb, &Sd) : fixed_to_f64(Sx[k], Eb, &Sd)) && ok;
          r[k] = fma(L.c, Sd, fma(-L.alpha, as_d(repack(C.sig[k], C.E[k])), bv[k]));
        }
      }
      if (!ok) {  // the float64 point equation, as in residual_point, from the values in memory
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int x = x0 + k;
          const int64_t q = cb + k;
          const double w = x > 0 ? u[q - 1] : 0.0;
          const double e = x < nx - 1 ? u[q + 1] : 0.0;
          const double sv = y > 0 ? u[q - sy] : 0.0;
          const double nv = y < ny - 1 ? u[q + sy] : 0.0;
          const double bo = z > 0 ? u[q - sz] : 0.0;
          const double to = z < nz - 1 ? u[q + sz] : 0.0;
          const double nb = ((w + e) + (sv + nv)) + (bo + to);
          const int cls = bclass<3>(x, y, z, nx, ny, nz);
          r[k] = fma(L.c, nb, fma(-L.d[cls], u[q], bv[k]));
        }
      }
      // frozen wall slots of a face grid: residual 0
      if (L.fax >= 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if ((L.fax == 0 && x0 + k == nx - 1) || (L.fax == 1 && y == ny - 1) || (L.fax == 2 && z == nz - 1))
            r[k] = 0.0;
      }
      float4 o;
      const bool nrm = f32_normal_range(r[0]) && f32_normal_range(r[1]) && f32_normal_range(r[2]) &&
                       f32_normal_range(r[3]);
      if (__all_sync(kAll, nrm)) {
        o.x = f64_to_f32_rn_normal(r[0]);
        o.y = f64_to_f32_rn_normal(r[1]);
        o.z = f64_to_f32_rn_normal(r[2]);
        o.w = f64_to_f32_rn_normal(r[3]);
      } else {
        o.x = f64_to_f32_rn_bits(r[0]);
        o.y = f64_to_f32_rn_bits(r[1]);
        o.z = f64_to_f32_rn_bits(r[2]);
        o.w = f64_to_f32_rn_bits(r[3]);
      }
      *reinterpret_cast<float4*>(r32 + cb) = o;
      const float s0 = o.x * nscale, s1 = o.y * nscale, s2 = o.z * nscale, s3 = o.w * nscale;
      acc = fmaf(s0, s0, acc);
      acc = fmaf(s1, s1, acc);
      acc = fmaf(s2, s2, acc);
      acc = fmaf(s3, s3, acc);
      P = C;
      C = N;
    }
  }
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

}  // namespace

bool ir_strip_supported(const LevelDesc<double>& L) {
  if (L.varkappa || L.per || L.nx % kIrCols != 0) return false;
  if (L.nz == 1) return L.fax < 0 && L.ny >= 1;
  return L.ny % kIr3Rows == 0;
}

cudaError_t launch_ir_strip(float* r32, const double* u, const double* b, const LevelDesc<double>& L,
                            const float* nsp, double* partials, unsigned* ticket, int sm_count, int max_blocks,
                            int* nblocks, cudaStream_t stream) {
  const int nstrips = L.nx / kIrCols;
  if (L.nz > 1) {
    // blocks of eight rows y; z segments sized for about four blocks per SM, 8..128 planes each
    const int64_t cols = (int64_t)nstrips * (L.ny / kIr3Rows);
    const int64_t per = std::max<int64_t>(1, ((int64_t)sm_count * 4) / cols);
    const int zseg = (int)std::min<int64_t>(128, std::max<int64_t>(8, (L.nz + per - 1) / per));
    const int64_t ntasks = cols * ((L.nz + zseg - 1) / zseg);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(max_blocks, ntasks));
    *nblocks = blocks;
    k_ir_strip3<<<blocks, kIrThreads, 0, stream>>>(r32, u, b, L, nsp, partials, zseg);
    return cudaGetLastError();
  }
  // one wave of kIrMinBlocks2D blocks of eight warps per SM; segments of 16..256 rows (two halo rows
  // each) sized for about kIrTasksPerWarp tasks per warp
  const int nstrips2 = L.nx / (32 * kIrCpl2D);
  const int64_t warps = (int64_t)sm_count * kIrMinBlocks2D * kIrWarps;
  const int64_t per_strip = std::max<int64_t>(1, warps * kIrTasksPerWarp / nstrips2);
  const int seg = (int)std::min<int64_t>(256, std::max<int64_t>(16, (L.ny + per_strip - 1) / per_strip));
  const int64_t ntasks = (int64_t)nstrips2 * ((L.ny + seg - 1) / seg);
  const int64_t want = (ntasks + kIrWarps - 1) / kIrWarps;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(max_blocks, want),
                                                                   (int64_t)sm_count * kIrMinBlocks2D));
  *nblocks = blocks;
  k_ir_strip<kIrCpl2D, kIrMinBlocks2D><<<blocks, kIrThreads, 0, stream>>>(r32, u, b, L, nsp, partials, ticket, seg);
  return cudaGetLastError();
}

}  // namespace fasmg
