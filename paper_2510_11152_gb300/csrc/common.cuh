// common.cuh -- level descriptors and the per-point arithmetic shared by every kernel.
//
// Operator (Sec. 2.2 generalised): A u = alpha u - beta div_h(kappa grad_h u) on cells of width h.
// Boundary conditions are folded into each boundary cell's point equation: multiplying the cell's
// equation by h^2,
//     D u_c - sum_{interior faces f} w_f u_nb = h^2 f_c,      w_f = beta kappa_f,
//     D = alpha h^2 + sum_f m_f w_f,   m_f = 1 interior face, 0 Neumann face (ghost = cell),
//                                      2 Dirichlet face (ghost = -cell).
// With constant kappa every cell of the same "boundary class" (which faces of the box it touches)
// has the same D, so the kernels look up per-class constants:
//     smoother (Eqs. FCGS-1..4)   u_c <- a[cls] * N + b[cls] * f_c,   a = beta kappa / D, b = h^2 / D
//     residual (Sec. 2.2)         r_c  = f_c - d[cls] u_c + c N,       d = D / h^2,       c = beta kappa / h^2
// where N is the plain sum of the existing neighbours. For alpha = beta = kappa = 1 in the interior
// the smoother is (sum of 4 neighbours + h^2 f) / (4 + h^2), the paper's update.
// With a per-cell kappa the face weights w_f (kappa_f = mean of the two cells) and 1/D, D/h^2 are
// stored per cell on every level.
// Periodic axes (the grain-growth example, Sec. 3.3.1): the grid wraps around, so the first and the
// last cell of the axis are neighbours across an interior face (m_f = 1). Their boundary classes then
// carry the interior constants, and the neighbour sums below fetch the wrapped cell.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fasmg {

constexpr int kMaxLevels = 24;
constexpr int kClasses = 64;  // 2^(2*dim) boundary classes, dim <= 3

template <typename T>
struct LevelDesc {
  int nx, ny, nz;  // cells per axis (nz = 1 in 2D), powers of two
  int lx, ly, lz;  // their base-2 logarithms (index decomposition by shifts)
  int varkappa;    // 1: use the per-cell arrays below
  int fax;         // -1: cell-centred unknowns; 0/1/2: face unknowns normal to x/y/z (staggered
                   // velocity component): slot s of that axis is face s+1, the last slot is the
                   // far wall (frozen at 0), the near wall face is implicit and 0
  int per;         // periodic axes: bit 0 x, bit 1 y, bit 2 z (constant kappa, cell-centred only)
  T h2, ih2;       // h^2, 1/h^2
  T c;             // beta kappa / h^2 (constant kappa)
  const T* wx;     // beta kappa_f of the face between cells i and i+1, stored at cell i (0 at i = nx-1)
  const T* wy;     // same along y (0 at j = ny-1)
  const T* wz;     // same along z (0 at l = nz-1)
  const T* rD;     // 1 / D
  const T* Dh;     // D / h^2
  T alpha;         // alpha of A u = alpha u - beta div(kappa grad u)
  T a[kClasses], b[kClasses], d[kClasses];
  unsigned char mt[kClasses];  // M of d = alpha + c M: neighbours plus boundary multiplicities
};

// boundary class: bit 0 x_lo, 1 x_hi, 2 y_lo, 3 y_hi, 4 z_lo, 5 z_hi
template <int DIM>
__device__ __forceinline__ int bclass(int i, int j, int l, int nx, int ny, int nz) {
  int fl = (i == 0) | ((i == nx - 1) << 1) | ((j == 0) << 2) | ((j == ny - 1) << 3);
  if (DIM == 3) fl |= ((l == 0) << 4) | ((l == nz - 1) << 5);
  return fl;
}

// True for the frozen wall slot of a face grid (never updated, residual 0).
template <typename T>
__device__ __forceinline__ bool frozen(const LevelDesc<T>& L, int i, int j, int l) {
  return (L.fax == 0 && i == L.nx - 1) || (L.fax == 1 && j == L.ny - 1) || (L.fax == 2 && l == L.nz - 1);
}

// Sum of the existing neighbours of cell (i, j, l) at linear index idx (constant kappa); on a periodic
// axis (bit of per) the neighbour across the boundary is the wrapped cell. PER = false is the code for
// levels without periodic axes.
template <typename T, int DIM, bool PER>
__device__ __forceinline__ T nbsum_t(const T* __restrict__ u, int64_t idx, int i, int j, int l, int nx, int ny,
                                     int nz, int per) {
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  if constexpr (!PER) {
    T w = i > 0 ? u[idx - 1] : T(0);
    T e = i < nx - 1 ? u[idx + 1] : T(0);
    T s = j > 0 ? u[idx - sy] : T(0);
    T n = j < ny - 1 ? u[idx + sy] : T(0);
    T acc = (w + e) + (s + n);
    if (DIM == 3) {
      T bo = l > 0 ? u[idx - sz] : T(0);
      T to = l < nz - 1 ? u[idx + sz] : T(0);
      acc = acc + (bo + to);
    }
    return acc;
  } else {
    // one load per neighbour: the address wraps on a periodic axis, the value is 0 where none exists
    T w = (i > 0 || (per & 1)) ? u[i > 0 ? idx - 1 : idx + (nx - 1)] : T(0);
    T e = (i < nx - 1 || (per & 1)) ? u[i < nx - 1 ? idx + 1 : idx - (nx - 1)] : T(0);
    T s = (j > 0 || (per & 2)) ? u[j > 0 ? idx - sy : idx + (ny - 1) * sy] : T(0);
    T n = (j < ny - 1 || (per & 2)) ? u[j < ny - 1 ? idx + sy : idx - (ny - 1) * sy] : T(0);
    T acc = (w + e) + (s + n);
    if (DIM == 3) {
      T bo = (l > 0 || (per & 4)) ? u[l > 0 ? idx - sz : idx + (nz - 1) * sz] : T(0);
      T to = (l < nz - 1 || (per & 4)) ? u[l < nz - 1 ? idx + sz : idx - (nz - 1) * sz] : T(0);
      acc = acc + (bo + to);
    }
    return acc;
  }
}

// Weighted neighbour sum sum_f w_f u_nb (per-cell kappa).
template <typename T, int DIM>
__device__ __forceinline__ T nbsum_w(const T* __restrict__ u, const LevelDesc<T>& L, int64_t idx, int i,
                                     int j, int l) {
  const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
  T acc = T(0);
  if (i > 0) acc = fma(L.wx[idx - 1], u[idx - 1], acc);
  if (i < L.nx - 1) acc = fma(L.wx[idx], u[idx + 1], acc);
  if (j > 0) acc = fma(L.wy[idx - sy], u[idx - sy], acc);
  if (j < L.ny - 1) acc = fma(L.wy[idx], u[idx + sy], acc);
  if (DIM == 3) {
    if (l > 0) acc = fma(L.wz[idx - sz], u[idx - sz], acc);
    if (l < L.nz - 1) acc = fma(L.wz[idx], u[idx + sz], acc);
  }
  return acc;
}

// Gauss-Seidel point update of cell (i, j, l): the new value from the current neighbours. PER: the
// level may have periodic axes (the kernels choose the instantiation once from the descriptor).
template <typename T, int DIM, bool PER = false>
__device__ __forceinline__ T point_update(const T* __restrict__ u, const T* __restrict__ f,
                                          const LevelDesc<T>& L, int64_t idx, int i, int j, int l) {
  if (L.varkappa) {
    T nw = nbsum_w<T, DIM>(u, L, idx, i, j, l);
    return fma(L.h2, f[idx], nw) * L.rD[idx];
  }
  const int cls = bclass<DIM>(i, j, l, L.nx, L.ny, L.nz);
  T nb = nbsum_t<T, DIM, PER>(u, idx, i, j, l, L.nx, L.ny, L.nz, L.per);
  return fma(L.a[cls], nb, L.b[cls] * f[idx]);
}

// (A u) at cell (i, j, l).
template <typename T, int DIM, bool PER = false>
__device__ __forceinline__ T apply_point(const T* __restrict__ u, const LevelDesc<T>& L, int64_t idx, int i,
                                         int j, int l) {
  if (L.varkappa) {
    T nw = nbsum_w<T, DIM>(u, L, idx, i, j, l);
    return fma(L.Dh[idx], u[idx], -L.ih2 * nw);
  }
  const int cls = bclass<DIM>(i, j, l, L.nx, L.ny, L.nz);
  T nb = nbsum_t<T, DIM, PER>(u, idx, i, j, l, L.nx, L.ny, L.nz, L.per);
  return fma(L.d[cls], u[idx], -L.c * nb);
}

// Residual f - A u at cell (i, j, l).
template <typename T, int DIM, bool PER = false>
__device__ __forceinline__ T residual_point(const T* __restrict__ u, const T* __restrict__ f,
                                            const LevelDesc<T>& L, int64_t idx, int i, int j, int l) {
  if (L.varkappa) {
    T nw = nbsum_w<T, DIM>(u, L, idx, i, j, l);
    return fma(L.ih2, nw, fma(-L.Dh[idx], u[idx], f[idx]));
  }
  const int cls = bclass<DIM>(i, j, l, L.nx, L.ny, L.nz);
  T nb = nbsum_t<T, DIM, PER>(u, idx, i, j, l, L.nx, L.ny, L.nz, L.per);
  return fma(L.c, nb, fma(-L.d[cls], u[idx], f[idx]));
}

// Block-wide sum of one double per thread; result valid in thread 0. blockDim.x <= 1024.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();  // protect warp_part against a previous use
  if (lane == 0) warp_part[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? warp_part[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace fasmg
