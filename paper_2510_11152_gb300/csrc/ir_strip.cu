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
// two extra loads. Windows whose values span more than 2^kMaxExpSpread in magnitude, or hold a zero,
// a subnormal or non-finite value or values of both signs, take the float64 point equation instead
// (2D: the warp decides per row; 3D: each lane for its four cells).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "bits64.cuh"
#include "common.cuh"
#include "ir_strip.h"
#include "tma.cuh"

namespace fasmg {
namespace {

constexpr int kIrWarps = 8;
constexpr int kIrThreads = 32 * kIrWarps;
constexpr int kIrCols = 128;  // columns per strip of the 3D kernel (4 per lane); 2D strips are 32 CPL wide
constexpr int kIrCpl2D = 4;   // cells per lane of the 2D kernel
constexpr int kIrMinBlocks2D = 2;
constexpr int kIrTasksPerWarp = 6;  // 2D work items per warp, taken dynamically
constexpr unsigned kAll = 0xffffffffu;

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
// 3D (cell-centred or face grids, constant kappa): a block of eight warps owns a 128-column strip of
// eight consecutive rows y and walks a segment of planes z. The planes arrive in shared memory by TMA
// tile loads, up to three planes ahead: per plane a tile of 10 rows (y0-1 .. y0+8) by 132 columns
// (x0-2 .. x0+129; out-of-range cells read as zero) of u, in a ring of four slots, and the block's
// 8 x 128 cells of b, in a ring of three, each slot with an mbarrier that the copies complete; every
// wait on them is bounded (FAS_ETIMEOUT when a deadline passes).
//
// Every u value is unpacked once. Warp w owns row y0 + w; lane L owns its four cells x0 .. x0+3. When
// plane z+1 arrives, each lane takes the bit patterns of its four cells (and of their left and right
// neighbours) and turns them into signed significands aligned to the smallest exponent among them,
// its "row reference" (exact zeros count as 0 and take no part in the exponent range). The aligned
// row stays in the lane's registers for the planes z+1, z, z-1 of its own row, and goes to shared
// memory (three plane buffers) for the warps of the rows y-1 and y+1; warps 0 and 7 also unpack the
// tile's halo rows. The stencil of a cell then combines five rows, each already aligned to its own
// reference: with Eref the smallest of the five references and every exponent within kMaxExpSpread
// binades of it, each row's contribution is shifted left by (its reference - Eref) and
// S = sum_nb u_nb - M u_c is exact in 64-bit integers; it is rounded once, and
// r = fma(c, S, fma(-alpha, u, b)). A neighbour outside the grid takes the centre's own value in its
// slot and counts once more in M (M = 6 inside the grid; at a boundary the diagonal's multiplicity mt
// plus the number of absent neighbours). Windows with a subnormal or non-finite value or a wider
// exponent range take the float64 point equation, from u in memory.
// ------------------------------------------------------------------------------------------------
constexpr int kIr3Rows = kIrWarps;           // rows y per block
constexpr int kU3W = kIrCols + 4;            // u tile row: x0-2 .. x0+129
constexpr int kU3H = kIr3Rows + 2;           // u tile rows: y0-1 .. y0+8
constexpr int kU3Vals = kU3W * kU3H;         // 1320 values, 10560 bytes
constexpr int kU3Slot = 1328;                // slot stride in values (a multiple of 128 bytes)
constexpr int kB3Slot = kIrCols * kIr3Rows;  // 1024 values
constexpr int kDepthU = 4;                   // u tile slots: planes z-1 .. z+2 around the computed plane z
constexpr int kDepth = 3;                    // b tile slots and aligned-row buffers
constexpr int kA3Slot = kU3H * kIrCols;      // aligned rows of one plane: 10 x 128 int64
constexpr int kRefNone = 1 << 20;            // reference of a row holding only zeros
constexpr size_t kIr3Smem = (size_t)(kDepthU * kU3Slot + kDepth * kB3Slot) * sizeof(double) +
                            (size_t)kDepth * kA3Slot * sizeof(int64_t) +
                            (size_t)kDepth * kU3H * 32 * sizeof(int2) +      // per lane and row: reference, top
                            (kDepthU + kDepth) * sizeof(uint64_t) + 128;     // barriers, alignment

__device__ __forceinline__ uint32_t hiw(uint64_t v) { return (uint32_t)(v >> 32); }

// An aligned row of a lane: four signed significands times 2^(E - ref), the reference ref (the
// smallest exponent among the unpacked values; kRefNone when all are zero, -kRefNone when one is
// subnormal or non-finite) and the largest exponent top.
struct ARow {
  int64_t v[4];
  int ref, top;
};

__device__ __forceinline__ void exp_range(uint64_t v, int& lo, int& hi) {
  const int E = (int)((hiw(v) >> 20) & 0x7FFu);
  const bool zero = (v << 1) == 0ull;
  const bool bad = !zero && (unsigned)(E - 1) >= 2046u;
  lo = bad ? -kRefNone : (zero ? lo : min(lo, E));
  hi = zero ? hi : max(hi, E);
}

// v m for a small m (a power of two: a left shift) as a 64 x 32-bit multiplication on the integer
// multiply-add pipe instead of shifts on the ALU pipe (two's complement: also for negative v)
__device__ __forceinline__ int64_t mul_u32(int64_t v, uint32_t m) {
  const uint64_t lo = (uint64_t)(uint32_t)v * m;
  const uint32_t hi = (uint32_t)((uint64_t)v >> 32) * m + (uint32_t)(lo >> 32);
  return (int64_t)(((uint64_t)hi << 32) | (uint32_t)lo);
}

// The signed significand of the finite float64 with bit pattern v (0 for a zero), times 2^(E - ref),
// for E - ref in 0..31.
__device__ __forceinline__ int64_t sig_at(uint64_t v, int ref) {
  const uint32_t h = hiw(v), l = (uint32_t)v;
  const uint32_t m = (h & 0xFFFFFu) | 0x100000u;
  const int sh = (int)((h >> 20) & 0x7FFu) - ref;
  int64_t X = mul_u32((int64_t)(((uint64_t)m << 32) | l), 1u << (sh & 31));
  X = (v << 1) == 0ull ? 0 : X;
  const int64_t neg = (int64_t)((int32_t)h >> 31);  // 0 or -1
  return (X ^ neg) - neg;
}

__device__ __forceinline__ void lds_raw4(uint64_t (&v)[4], const double* p) {  // p 16-byte aligned
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 c = reinterpret_cast<const double2*>(p)[1];
  v[0] = (uint64_t)__double_as_longlong(a.x);
  v[1] = (uint64_t)__double_as_longlong(a.y);
  v[2] = (uint64_t)__double_as_longlong(c.x);
  v[3] = (uint64_t)__double_as_longlong(c.y);
}

// Align a lane's four values (and, when given, the two horizontal neighbours) to their reference.
__device__ __forceinline__ void align_row(ARow& R, const uint64_t (&v)[4], const uint64_t* wl, const uint64_t* er,
                                          int64_t* aw, int64_t* ae) {
  int lo = kRefNone, hi = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) exp_range(v[k], lo, hi);
  if (wl) {
    exp_range(*wl, lo, hi);
    exp_range(*er, lo, hi);
  }
  R.ref = lo;
  R.top = hi;
  const int ref = lo < 1 ? 1 : (lo == kRefNone ? 1 : lo);  // any shift works for zeros; bad rows are unused
#pragma unroll
  for (int k = 0; k < 4; ++k) R.v[k] = sig_at(v[k], ref);
  if (wl) {
    *aw = sig_at(*wl, ref);
    *ae = sig_at(*er, ref);
  }
}

__global__ void __launch_bounds__(kIrThreads, 2)
    k_ir_strip3(float* __restrict__ r32, const double* __restrict__ u, const __grid_constant__ CUtensorMap tu,
                const __grid_constant__ CUtensorMap tb, LevelDesc<double> L, const float* nsp, double* partials,
                unsigned* ticket, int zseg, Ir3Wait wt) {
  extern __shared__ __align__(128) unsigned char smem3[];
  // the rings start on a 128-byte boundary (tile copies land on 128-byte aligned slots)
  double* su = reinterpret_cast<double*>(smem3 + ((128u - (smem_u32(smem3) & 127u)) & 127u));
  double* sb = su + kDepthU * kU3Slot;
  int64_t* sa = reinterpret_cast<int64_t*>(sb + kDepth * kB3Slot);  // aligned rows per plane
  int2* sr = reinterpret_cast<int2*>(sa + kDepth * kA3Slot);          // (reference, top) per lane and row
  uint64_t* bar = reinterpret_cast<uint64_t*>(sr + kDepth * kU3H * 32);  // u slots, then b slots
  constexpr int kNBar = kDepthU + kDepth;
  __shared__ int s_task;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  const int nstrips = nx / kIrCols;
  const int nyg = ny / kIr3Rows;
  const int nzs = (nz + zseg - 1) / zseg;
  const int ntasks = nstrips * nyg * nzs;
  const float nscale = nsp ? *nsp : 1.f;
  if (tid == 0) {
    for (int k = 0; k < kNBar; ++k) mbar_init(bar + k, 1);
    mbar_init_fence();
  }
  __syncthreads();
  uint32_t par = 0u;   // per barrier: parity of the phase this thread waits for next
  uint32_t pend = 0u;  // thread 0: barriers with a copy issued and not yet waited for
  bool aborted = false;
  bool first_task = true;
  float acc = 0.f;
  auto wait_bar = [&](int k) -> bool {
    const bool ok = mbar_wait_bounded(bar + k, (par >> k) & 1u, wt.limit_ns);
    par ^= 1u << k;
    if (tid == 0 && ok) pend &= ~(1u << k);
    return ok;
  };
  while (!aborted) {
    if (tid == 0) s_task = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int task = s_task;
    __syncthreads();  // every thread has read s_task before it is written again
    if (task >= ntasks) break;
    const int sx = task % nstrips;
    const int rest = task / nstrips;
    const int y0 = (rest % nyg) * kIr3Rows;
    const int y = y0 + warp;
    const int z0 = (rest / nyg) * zseg, z1 = min(nz, z0 + zseg);
    const int xs = sx * kIrCols;
    const int x0 = xs + 4 * lane;
    auto issue_u = [&](int z) {
      const int k = z % kDepthU;
      mbar_expect_tx(bar + k, kU3Vals * (uint32_t)sizeof(double));
      tma_load_3d(su + k * kU3Slot, &tu, xs - 2, y0 - 1, z, bar + k);
      pend |= 1u << k;
    };
    auto issue_b = [&](int z) {
      const int k = kDepthU + z % kDepth;
      mbar_expect_tx(bar + k, kB3Slot * (uint32_t)sizeof(double));
      tma_load_3d(sb + (z % kDepth) * kB3Slot, &tb, xs, y0, z, bar + k);
      pend |= 1u << k;
    };
    // unpack plane z from its tile: this warp's row (with horizontal neighbours) into registers and
    // the plane's aligned-row buffer; warps 0 and 7 also the tile's halo rows y0-1 and y0+8
    auto unpack_plane = [&](int z, ARow& R, int64_t& aw, int64_t& ae) {
      const double* T = su + (z % kDepthU) * kU3Slot;
      int64_t* A = sa + (z % kDepth) * kA3Slot;
      int2* Rf = sr + (z % kDepth) * kU3H * 32;
      uint64_t v[4];
      const double* row = T + (warp + 1) * kU3W + 4 * lane + 2;
      lds_raw4(v, row);
      uint64_t wl = (uint64_t)__double_as_longlong(row[-1]), er = (uint64_t)__double_as_longlong(row[4]);
      if (x0 == 0) wl = v[0];  // absent: the centre's value
      if (x0 + 4 == nx) er = v[3];
      align_row(R, v, &wl, &er, &aw, &ae);
      longlong2* dst = reinterpret_cast<longlong2*>(A + (warp + 1) * kIrCols + 4 * lane);
      dst[0] = make_longlong2(R.v[0], R.v[1]);
      dst[1] = make_longlong2(R.v[2], R.v[3]);
      Rf[(warp + 1) * 32 + lane] = make_int2(R.ref, R.top);
      if ((warp == 0 && y0 > 0) || (warp == kIr3Rows - 1 && y0 + kIr3Rows < ny)) {
        const int hr = warp == 0 ? 0 : kU3H - 1;
        ARow H;
        lds_raw4(v, T + hr * kU3W + 4 * lane + 2);
        align_row(H, v, nullptr, nullptr, nullptr, nullptr);
        longlong2* hd = reinterpret_cast<longlong2*>(A + hr * kIrCols + 4 * lane);
        hd[0] = make_longlong2(H.v[0], H.v[1]);
        hd[1] = make_longlong2(H.v[2], H.v[3]);
        Rf[hr * 32 + lane] = make_int2(H.ref, H.top);
      }
    };
    // the test hook withholds one copy (block 0, first task): its waits must run out
    const bool withhold = wt.withhold && blockIdx.x == 0 && first_task;
    first_task = false;
    if (tid == 0) {
      fence_async_smem();  // the previous task's reads of the slots come before the new copies
      if (z0 > 0) issue_u(z0 - 1);
      if (!withhold) issue_u(z0);
      if (z0 + 1 < nz) issue_u(z0 + 1);
      issue_b(z0);
      if (z0 + 1 < z1) issue_b(z0 + 1);
    }
    ARow P, C, N;
    int64_t cw = 0, ce = 0, nw = 0, ne = 0, dw, de;
    bool ok = true;
    if (z0 > 0) {
      ok = wait_bar((z0 - 1) % kDepthU) && ok;
      if (ok) unpack_plane(z0 - 1, P, dw, de);
    }
    ok = wait_bar(z0 % kDepthU) && ok;
    if (ok) unpack_plane(z0, C, cw, ce);
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    if (z0 == 0) P = C;  // absent plane: the centre's values
    if (tid == 0) {
      fence_async_smem();
      if (z0 + 2 < nz && z0 + 2 <= z1) issue_u(z0 + 2);
    }
    for (int z = z0; z < z1; ++z) {
      ok = true;
      if (z + 1 < nz) {
        ok = wait_bar((z + 1) % kDepthU) && ok;
        if (ok) unpack_plane(z + 1, N, nw, ne);
      }
      ok = wait_bar(kDepthU + z % kDepth) && ok;
      // the aligned rows of plane z+1 are complete; plane z-1 (tile and b) is no longer read. A wait
      // that ran out anywhere in the block ends its work.
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      if (tid == 0) {
        fence_async_smem();
        if (z + 3 < nz && z + 3 <= z1) issue_u(z + 3);  // into the slot of plane z-1
        if (z + 2 < z1) issue_b(z + 2);                 // into the slot of plane z-1
      }
      if (z + 1 >= nz) {  // absent plane: the centre's values
        N = C;
        nw = cw;
        ne = ce;
      }
      // rows y-1 and y+1 of plane z (absent rows: the centre's values)
      ARow S, T;
      {
        const int64_t* A = sa + (z % kDepth) * kA3Slot;
        const int2* Rf = sr + (z % kDepth) * kU3H * 32;
        if (y > 0) {
          const longlong2* q = reinterpret_cast<const longlong2*>(A + warp * kIrCols + 4 * lane);
          const longlong2 a = q[0], c = q[1];
          S.v[0] = a.x, S.v[1] = a.y, S.v[2] = c.x, S.v[3] = c.y;
          const int2 rt = Rf[warp * 32 + lane];
          S.ref = rt.x, S.top = rt.y;
        } else {
          S = C;
        }
        if (y < ny - 1) {
          const longlong2* q = reinterpret_cast<const longlong2*>(A + (warp + 2) * kIrCols + 4 * lane);
          const longlong2 a = q[0], c = q[1];
          T.v[0] = a.x, T.v[1] = a.y, T.v[2] = c.x, T.v[3] = c.y;
          const int2 rt = Rf[(warp + 2) * 32 + lane];
          T.ref = rt.x, T.top = rt.y;
        } else {
          T = C;
        }
      }
      const double* bp = sb + (z % kDepth) * kB3Slot + warp * kIrCols + 4 * lane;
      const double2 b01 = reinterpret_cast<const double2*>(bp)[0];
      const double2 b23 = reinterpret_cast<const double2*>(bp)[1];
      const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
      uint64_t craw[4];  // this row of plane z, still in its tile slot
      lds_raw4(craw, su + (z % kDepthU) * kU3Slot + (warp + 1) * kU3W + 4 * lane + 2);
      const int eref = min(min(C.ref, min(P.ref, N.ref)), min(S.ref, T.ref));
      const int etop = max(max(C.top, max(P.top, N.top)), max(S.top, T.top));
      double r[4];
      bool ex = eref >= 1 && etop <= 2046 && (eref == kRefNone || etop - eref <= kMaxExpSpread);
      if (ex) {  // per lane; nothing below synchronises the warp
        const int e0 = eref == kRefNone ? 1 : eref;
        // each row's shift to the common reference (rows of zeros have any reference: shift 0)
        auto msh = [&](const ARow& R) { return 1u << (R.ref == kRefNone ? 0 : (R.ref < 1 ? 1 : R.ref) - e0); };
        const uint32_t mC = msh(C), mP = msh(P), mN = msh(N), mS = msh(S), mT = msh(T);
        const bool inner = y > 0 && y < ny - 1 && z > 0 && z < nz - 1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int64_t sw = k ? C.v[k - 1] : cw;
          const int64_t se = k < 3 ? C.v[k + 1] : ce;
          int M = 6;
          if (!inner || (k == 0 && x0 == 0) || (k == 3 && x0 + 4 == nx)) {
            const int cls = bclass<3>(x0 + k, y, z, nx, ny, nz);
            M = (int)L.mt[cls] + __popc(cls);
          }
          const int64_t cpart = (sw + se) - mul_u32(C.v[k], (uint32_t)M);
          const int64_t sum = mul_u32(cpart, mC) + (mul_u32(P.v[k], mP) + mul_u32(N.v[k], mN)) +
                              (mul_u32(S.v[k], mS) + mul_u32(T.v[k], mT));
          double Sd;
          // |sum| < 2^53 (the usual case: S is a second difference) converts without rounding
          const bool small = (uint64_t)(sum + ((1ll << 53) - 1)) < (1ull << 54) - 1ull;
          ex = (small ? fixed_to_f64_small(sum, e0, &Sd) : fixed_to_f64(sum, e0, &Sd)) && ex;
          r[k] = fma(L.c, Sd, fma(-L.alpha, as_d(craw[k]), bv[k]));
        }
      }
      if (!ex) {  // the float64 point equation, as in residual_point, from the values in memory
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int x = x0 + k;
          const int64_t q = (int64_t)z * sz + (int64_t)y * sy + x;
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
      *reinterpret_cast<float4*>(r32 + (int64_t)z * sz + (int64_t)y * sy + x0) = o;
      const float s0 = o.x * nscale, s1 = o.y * nscale, s2 = o.z * nscale, s3 = o.w * nscale;
      acc = fmaf(s0, s0, acc);
      acc = fmaf(s1, s1, acc);
      acc = fmaf(s2, s2, acc);
      acc = fmaf(s3, s3, acc);
      P = C;
      C = N;
      cw = nw;
      ce = ne;
    }
  }
  if (aborted && tid == 0) {
    atomicOr(ticket + 2, 1u);  // the host reports FAS_ETIMEOUT
    // copies still in flight must land before the block's shared memory is released
    for (int k = 0; k < kNBar; ++k)
      if ((pend >> k) & 1u) mbar_wait_bounded(bar + k, (par >> k) & 1u, wt.limit_ns);
  }
  const double s = block_sum((double)acc);  // every warp of the block has left the task loop
  if (tid == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    if (atomicAdd(ticket + 1, 1u) == gridDim.x - 1) {  // the last block: no block takes tasks any more
      ticket[0] = 0u;
      ticket[1] = 0u;
    }
  }
}

}  // namespace

cudaError_t ir_strip_prepare() {
  return cudaFuncSetAttribute(k_ir_strip3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kIr3Smem);
}

bool ir_strip_supported(const LevelDesc<double>& L) {
  if (L.varkappa || L.per || L.nx % kIrCols != 0) return false;
  if (L.nz == 1) return L.fax < 0 && L.ny >= 1;
  return L.ny % kIr3Rows == 0;
}

cudaError_t launch_ir_strip(float* r32, const double* u, const double* b, const LevelDesc<double>& L,
                            const float* nsp, double* partials, unsigned* ticket, int sm_count, int max_blocks,
                            int* nblocks, cudaStream_t stream, Ir3Wait wt) {
  const int nstrips = L.nx / kIrCols;
  if (L.nz > 1) {
    // one wave of two blocks of eight rows y per SM taking (strip, row group, plane segment) tasks;
    // segments of 16..128 planes (two halo planes each) sized for about kIrTasksPerWarp tasks per block
    const int64_t cols = (int64_t)nstrips * (L.ny / kIr3Rows);
    const int64_t wave = (int64_t)sm_count * 2;
    const int64_t per = std::max<int64_t>(1, (wave * kIrTasksPerWarp + cols - 1) / cols);
    const int zseg = (int)std::min<int64_t>(128, std::max<int64_t>(16, (L.nz + per - 1) / per));
    const int64_t ntasks = cols * ((L.nz + zseg - 1) / zseg);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(max_blocks, ntasks), wave));
    CUtensorMap tu, tb;
    cudaError_t e = tensor_map_3d(&tu, u, sizeof(double), L.nx, L.ny, L.nz, kU3W, kU3H, 1);
    if (e == cudaSuccess) e = tensor_map_3d(&tb, b, sizeof(double), L.nx, L.ny, L.nz, kIrCols, kIr3Rows, 1);
    if (e != cudaSuccess) return e;
    *nblocks = blocks;
    k_ir_strip3<<<blocks, kIrThreads, kIr3Smem, stream>>>(r32, u, tu, tb, L, nsp, partials, ticket, zseg, wt);
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
