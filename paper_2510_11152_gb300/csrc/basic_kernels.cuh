// basic_kernels.cuh -- one-operation-per-launch kernels for every level, templated on the value type
// (double / float) and the dimension. Each operation is written as a range loop (start, stride) so
// that the same code serves a grid-stride launch and the single-CTA kernel that runs the whole
// V-cycle below a switch level (where every level is too small to fill the GPU).
//
// No pointer here is declared __restrict__ or read through the non-coherent path: the single-CTA
// kernel writes a level in one step and reads it in the next, separated only by __syncthreads.
#pragma once
#include <type_traits>

#include "bits64.cuh"
#include "common.cuh"

namespace fasmg {

// ---- X-MCGS colour phase (Sec. 2.3). colour 1: cells whose 1-based index sum i+j(+l) is odd (the
// paper's sets 1,2 in 2D, sets 1-4 in 3D); colour 0: even (sets 3,4 / 5-8). With the 0-based indices
// used here the 1-based sum is the 0-based sum plus DIM. Every cell of a colour has only other-colour
// neighbours, so all of them update at once from the current values.
template <typename T, int DIM, bool PER = false>
__device__ __forceinline__ void smooth_colour_range(T* u, const T* f, const LevelDesc<T>& L, int colour,
                                                    int64_t t0, int64_t stride) {
  const int lhx = L.lx - 1;
  const int64_t half = ((int64_t)1 << (lhx + L.ly + L.lz));
  for (int64_t t = t0; t < half; t += stride) {
    const int k = (int)(t & ((1 << lhx) - 1));
    const int j = (int)((t >> lhx) & (L.ny - 1));
    const int l = (int)(t >> (lhx + L.ly));
    const int i = 2 * k + ((colour + DIM + j + l) & 1);
    const int64_t idx = ((int64_t)l * L.ny + j) * L.nx + i;
    if (L.fax >= 0 && frozen(L, i, j, l)) continue;
    u[idx] = point_update<T, DIM, PER>(u, f, L, idx, i, j, l);
  }
}

// ---- r = f - A u (Sec. 2.2) over a range of cells; returns the thread's sum of (scale*r)^2.
template <typename T, int DIM, bool PER = false>
__device__ __forceinline__ float residual_range(T* r, const T* u, const T* f, const LevelDesc<T>& L,
                                                float nscale, int64_t t0, int64_t stride) {
  // nscale: power-of-two factor applied before squaring (keeps float squares in range)
  const int64_t n = (int64_t)L.nx * L.ny * L.nz;
  float acc = 0.f;
  for (int64_t idx = t0; idx < n; idx += stride) {
    const int i = (int)(idx & (L.nx - 1));
    const int j = (int)((idx >> L.lx) & (L.ny - 1));
    const int l = (int)(idx >> (L.lx + L.ly));
    const T rv = (L.fax >= 0 && frozen(L, i, j, l)) ? T(0) : residual_point<T, DIM, PER>(u, f, L, idx, i, j, l);
    if (r) r[idx] = rv;
    const float rs = (float)rv * nscale;
    acc = fmaf(rs, rs, acc);
  }
  return acc;
}

// ---- Appendix C restriction: coarse cell = average of its 2^d children. Writes uc (and uc0, a
// copy kept for the coarse-grid correction) from u, and fc = R(r) when r is given.
template <typename T, int DIM>
__device__ __forceinline__ T avg_children(const T* v, int64_t base, int64_t sy, int64_t sz) {
  T s = (v[base] + v[base + 1]) + (v[base + sy] + v[base + sy + 1]);
  if (DIM == 3) {
    const T s2 = (v[base + sz] + v[base + sz + 1]) + (v[base + sz + sy] + v[base + sz + sy + 1]);
    return (s + s2) * T(0.125);
  }
  return s * T(0.25);
}

template <typename T, int DIM>
__device__ __forceinline__ void restrict_range(T* uc, T* uc0, T* fc, const T* u, const T* r, int nxf, int nyf,
                                               int nzf, int64_t t0, int64_t stride) {
  const int nxc = nxf >> 1, nyc = nyf >> 1, nzc = DIM == 3 ? nzf >> 1 : 1;
  const int64_t nc = (int64_t)nxc * nyc * nzc;
  const int64_t sy = nxf, sz = (int64_t)nxf * nyf;
  const int lxc = __ffs(nxc) - 1, lyc = __ffs(nyc) - 1;
  for (int64_t I = t0; I < nc; I += stride) {
    const int ic = (int)(I & (nxc - 1));
    const int jc = (int)((I >> lxc) & (nyc - 1));
    const int lc = (int)(I >> (lxc + lyc));
    const int64_t base = ((int64_t)(DIM == 3 ? 2 * lc : 0) * nyf + 2 * jc) * nxf + 2 * ic;
    if (u) {
      const T v = avg_children<T, DIM>(u, base, sy, sz);
      uc[I] = v;
      if (uc0) uc0[I] = v;
    }
    if (r) fc[I] = avg_children<T, DIM>(r, base, sy, sz);
  }
}

// ---- tau correction (Algorithm 1, coarse source term): fc <- fc + A_c uc, fc holding R(r).
template <typename T, int DIM, bool PER = false>
__device__ __forceinline__ void tau_range(T* fc, const T* uc, const LevelDesc<T>& Lc, int64_t t0,
                                          int64_t stride) {
  const int64_t n = (int64_t)Lc.nx * Lc.ny * Lc.nz;
  for (int64_t idx = t0; idx < n; idx += stride) {
    const int i = (int)(idx & (Lc.nx - 1));
    const int j = (int)((idx >> Lc.lx) & (Lc.ny - 1));
    const int l = (int)(idx >> (Lc.lx + Lc.ly));
    if (Lc.fax >= 0 && frozen(Lc, i, j, l)) continue;
    fc[idx] = fc[idx] + apply_point<T, DIM, PER>(uc, Lc, idx, i, j, l);
  }
}

// ---- Appendix C prolongation of the correction: u += P(uc - uc0), every child gets its parent's.
template <typename T, int DIM>
__device__ __forceinline__ void prolong_range(T* u, const T* uc, const T* uc0, int nxf, int nyf, int nzf,
                                              int64_t t0, int64_t stride) {
  const int nxc = nxf >> 1, nyc = nyf >> 1, nzc = DIM == 3 ? nzf >> 1 : 1;
  const int64_t nc = (int64_t)nxc * nyc * nzc;
  const int64_t sy = nxf, sz = (int64_t)nxf * nyf;
  const int lxc = __ffs(nxc) - 1, lyc = __ffs(nyc) - 1;
  for (int64_t I = t0; I < nc; I += stride) {
    const int ic = (int)(I & (nxc - 1));
    const int jc = (int)((I >> lxc) & (nyc - 1));
    const int lc = (int)(I >> (lxc + lyc));
    const int64_t base = ((int64_t)(DIM == 3 ? 2 * lc : 0) * nyf + 2 * jc) * nxf + 2 * ic;
    const T c = uc0 ? uc[I] - uc0[I] : uc[I];
    u[base] += c;
    u[base + 1] += c;
    u[base + sy] += c;
    u[base + sy + 1] += c;
    if (DIM == 3) {
      u[base + sz] += c;
      u[base + sz + 1] += c;
      u[base + sz + sy] += c;
      u[base + sz + sy + 1] += c;
    }
  }
}

// ---- Appendix D transfers for face grids. FAX is the index axis normal to the faces (0 x, 1 y,
// 2 z); slot s along it is face s+1, the last slot the far wall (0), the near wall face is 0.
// Restriction: coarse slot S = fine slots 2S, 2S+1, 2S+2 weighted 1/4, 1/2, 1/4, times the average
// of the two fine cells along each tangential axis; the coarse wall slot is 0.
template <typename T, int DIM, int FAX, typename Get>
__device__ __forceinline__ T face_avg_of(Get get, int ic, int jc, int lc, int nxf, int nyf) {
  const int c3[3] = {ic, jc, lc};
  T acc = T(0);
#pragma unroll
  for (int w = 0; w < 3; ++w) {
    T s = T(0);
#pragma unroll
    for (int t = 0; t < (DIM == 3 ? 4 : 2); ++t) {
      int f3[3] = {0, 0, 0};
      int tb = 0;  // tangential bit
#pragma unroll
      for (int ax = 0; ax < DIM; ++ax) {
        if (ax == FAX) {
          f3[ax] = 2 * c3[ax] + w;
        } else {
          f3[ax] = 2 * c3[ax] + ((t >> tb) & 1);
          ++tb;
        }
      }
      s += get(((int64_t)f3[2] * nyf + f3[1]) * nxf + f3[0], f3[0], f3[1], f3[2]);
    }
    acc += (w == 1 ? T(0.5) : T(0.25)) * s;
  }
  return acc * (DIM == 3 ? T(0.25) : T(0.5));
}

template <typename T, int DIM, int FAX>
__device__ __forceinline__ T face_avg(const T* v, int ic, int jc, int lc, int nxf, int nyf) {
  return face_avg_of<T, DIM, FAX>([v](int64_t q, int, int, int) { return v[q]; }, ic, jc, lc, nxf, nyf);
}

template <int FAX>
__device__ __forceinline__ bool wall_slot(int i, int j, int l, int nx, int ny, int nz) {
  return FAX == 0 ? i == nx - 1 : (FAX == 1 ? j == ny - 1 : l == nz - 1);
}

template <typename T, int DIM, int FAX>
__device__ __forceinline__ void restrict_face_range(T* uc, T* uc0, T* fc, const T* u, const T* r, int nxf, int nyf,
                                                    int nzf, int64_t t0, int64_t stride) {
  const int nxc = nxf >> 1, nyc = nyf >> 1, nzc = DIM == 3 ? nzf >> 1 : 1;
  const int64_t nc = (int64_t)nxc * nyc * nzc;
  const int lxc = __ffs(nxc) - 1, lyc = __ffs(nyc) - 1;
  for (int64_t I = t0; I < nc; I += stride) {
    const int ic = (int)(I & (nxc - 1));
    const int jc = (int)((I >> lxc) & (nyc - 1));
    const int lc = (int)(I >> (lxc + lyc));
    const bool wall = wall_slot<FAX>(ic, jc, lc, nxc, nyc, nzc);
    if (u) {
      const T v = wall ? T(0) : face_avg<T, DIM, FAX>(u, ic, jc, lc, nxf, nyf);
      uc[I] = v;
      if (uc0) uc0[I] = v;
    }
    if (r) fc[I] = wall ? T(0) : face_avg<T, DIM, FAX>(r, ic, jc, lc, nxf, nyf);
  }
}

// Prolongation of the correction c = uc - uc0 (c = uc without uc0), added to every fine slot but
// the wall slot. Along each tangential axis the fine cell 2J takes (3 c_J + c_{J-1})/4 and 2J+1 takes
// (3 c_J + c_{J+1})/4, the coarse ghost beyond a wall being -c_J (no-slip walls). Along the face axis
// the odd fine slot 2S+1 coincides with coarse slot S; the even slot 2S lies halfway between coarse
// slots S-1 and S (slot -1 is the near wall, 0).
template <typename T, int DIM, int FAX>
__device__ __forceinline__ void prolong_face_range(T* u, const T* uc, const T* uc0, int nxf, int nyf, int nzf,
                                                   int64_t t0, int64_t stride) {
  const int nxc = nxf >> 1, nyc = nyf >> 1, nzc = DIM == 3 ? nzf >> 1 : 1;
  const int64_t n = (int64_t)nxf * nyf * nzf;
  const int lx = __ffs(nxf) - 1, ly = __ffs(nyf) - 1;
  for (int64_t idx = t0; idx < n; idx += stride) {
    const int f3[3] = {(int)(idx & (nxf - 1)), (int)((idx >> lx) & (nyf - 1)), DIM == 3 ? (int)(idx >> (lx + ly)) : 0};
    const int nf3[3] = {nxf, nyf, nzf};
    const int nc3[3] = {nxc, nyc, nzc};
    if (f3[FAX] == nf3[FAX] - 1) continue;
    // per axis two coarse positions and weights (weight 0: the term is absent)
    int cp[3][2];
    T cw[3][2];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      cp[ax][0] = cp[ax][1] = 0;
      cw[ax][0] = ax < DIM ? T(0) : T(1);
      cw[ax][1] = T(0);
    }
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
      const int fi = f3[ax], C = fi >> 1;
      if (ax == FAX) {
        if (fi & 1) {
          cp[ax][0] = C;
          cw[ax][0] = T(1);
        } else {
          // coarse slots C - 1 and C, each with weight 1/2 unless it is a wall (slot -1, or the
          // coarse wall slot nc - 1): a wall face contributes 0
          const bool lo = C >= 1, hi = C < nc3[ax] - 1;
          cp[ax][0] = hi ? C : 0;
          cw[ax][0] = hi ? T(0.5) : T(0);
          cp[ax][1] = lo ? C - 1 : 0;
          cw[ax][1] = lo ? T(0.5) : T(0);
        }
      } else {
        const int nb = (fi & 1) ? C + 1 : C - 1;
        const bool ghost = nb < 0 || nb >= nc3[ax];
        cp[ax][0] = C;
        cw[ax][0] = T(0.75);
        cp[ax][1] = ghost ? C : nb;
        cw[ax][1] = ghost ? T(-0.25) : T(0.25);
      }
    }
    T acc = T(0);
#pragma unroll
    for (int a0 = 0; a0 < 2; ++a0)
#pragma unroll
      for (int a1 = 0; a1 < 2; ++a1)
#pragma unroll
        for (int a2 = 0; a2 < (DIM == 3 ? 2 : 1); ++a2) {
          const T w = cw[0][a0] * cw[1][a1] * cw[2][a2];
          if (w != T(0)) {
            const int64_t I = ((int64_t)cp[2][a2] * nyc + cp[1][a1]) * nxc + cp[0][a0];
            const T cv = uc0 ? uc[I] - uc0[I] : uc[I];
            acc += w * cv;
          }
        }
    u[idx] += acc;
  }
}


// ------------------------------------------------------------------------------------------------
// grid-stride kernels
// ------------------------------------------------------------------------------------------------

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

template <typename T, int DIM>
__global__ void k_smooth_colour(T* u, const T* f, LevelDesc<T> L, int colour) {
  if (L.per)
    smooth_colour_range<T, DIM, true>(u, f, L, colour, gtid(), gstride());
  else
    smooth_colour_range<T, DIM, false>(u, f, L, colour, gtid(), gstride());
}

// One colour phase with a thread per group of 4 consecutive cells of a row (nx a multiple of 4,
// constant kappa): the group is read and written as 16-byte vectors and its 2 cells of the colour
// are updated with point_update's expression (the other 2, of the other colour, are written back
// unchanged; no thread writes them in this phase).
template <typename T>
struct Quad;
template <>
struct Quad<float> {
  float v[4];
  __device__ __forceinline__ void ld(const float* p) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  }
  __device__ __forceinline__ void st(float* p) const {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Quad<double> {
  double v[4];
  __device__ __forceinline__ void ld(const double* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
  __device__ __forceinline__ void st(double* p) const {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

template <typename T, int DIM, bool PER>
__device__ __forceinline__ void smooth_colour4_body(T* u, const T* f, const LevelDesc<T>& L, int colour) {
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  const int lg = L.lx - 2;  // groups per row: nx / 4 = 2^lg (every extent is a power of two)
  const int64_t ngroups = (int64_t)1 << (lg + L.ly + L.lz);
  for (int64_t g = gtid(); g < ngroups; g += gstride()) {
    const int x0 = (int)(g & ((1 << lg) - 1)) << 2;
    const int64_t rest = g >> lg;
    const int j = (int)(rest & (ny - 1));
    const int l = (int)(rest >> L.ly);
    const int64_t idx = ((int64_t)l * ny + j) * nx + x0;
    Quad<T> c, s4, n4, b4, t4, f4;
    c.ld(u + idx);
    f4.ld(f + idx);
    // neighbours across a boundary: the wrapped cells on a periodic axis, none otherwise
    const bool px = PER && (L.per & 1), py = PER && ((L.per >> 1) & 1), pz = PER && ((L.per >> 2) & 1);
    const T wedge = (x0 > 0 || px) ? u[x0 > 0 ? idx - 1 : idx + nx - 1] : T(0);
    const T eedge = (x0 + 4 < nx || px) ? u[x0 + 4 < nx ? idx + 4 : idx + 4 - nx] : T(0);
    if (j > 0 || py) s4.ld(u + (j > 0 ? idx - sy : idx + (ny - 1) * sy));
    if (j < ny - 1 || py) n4.ld(u + (j < ny - 1 ? idx + sy : idx - (ny - 1) * sy));
    if (DIM == 3) {
      if (l > 0 || pz) b4.ld(u + (l > 0 ? idx - sz : idx + (nz - 1) * sz));
      if (l < nz - 1 || pz) t4.ld(u + (l < nz - 1 ? idx + sz : idx - (nz - 1) * sz));
    }
    // cell x has the colour when (x + j + l + DIM + colour) is even; the same along a row
    auto upd = [&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const int i = x0 + k;
      if (L.fax >= 0 && frozen(L, i, j, l)) return;
      const T w = (i > 0 || px) ? (k > 0 ? c.v[k > 0 ? k - 1 : 0] : wedge) : T(0);
      const T e = (i < nx - 1 || px) ? (k < 3 ? c.v[k < 3 ? k + 1 : 3] : eedge) : T(0);
      const T sv = (j > 0 || py) ? s4.v[k] : T(0);
      const T nv = (j < ny - 1 || py) ? n4.v[k] : T(0);
      T acc = (w + e) + (sv + nv);
      if (DIM == 3) {
        const T bo = (l > 0 || pz) ? b4.v[k] : T(0);
        const T to = (l < nz - 1 || pz) ? t4.v[k] : T(0);
        acc = acc + (bo + to);
      }
      const int cls = bclass<DIM>(i, j, l, nx, ny, nz);
      c.v[k] = fma(L.a[cls], acc, L.b[cls] * f4.v[k]);
    };
    if (((x0 + j + l + DIM + colour) & 1) == 0) {
      upd(std::integral_constant<int, 0>());
      upd(std::integral_constant<int, 2>());
    } else {
      upd(std::integral_constant<int, 1>());
      upd(std::integral_constant<int, 3>());
    }
    c.st(u + idx);
  }
}

template <typename T, int DIM>
__global__ void k_smooth_colour4(T* u, const T* f, LevelDesc<T> L, int colour) {
  if (L.per)
    smooth_colour4_body<T, DIM, true>(u, f, L, colour);
  else
    smooth_colour4_body<T, DIM, false>(u, f, L, colour);
}

// r (nullable) = f - A u; per-block partial of sum (s r)^2 into partials[blockIdx.x], s = *nsp (or 1).
template <typename T, int DIM>
__global__ void k_residual(T* r, const T* u, const T* f, LevelDesc<T> L, const float* nsp, double* partials) {
  const float acc = L.per ? residual_range<T, DIM, true>(r, u, f, L, nsp ? *nsp : 1.f, gtid(), gstride())
                          : residual_range<T, DIM, false>(r, u, f, L, nsp ? *nsp : 1.f, gtid(), gstride());
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0 && partials) partials[blockIdx.x] = s;
}

// out[0] = sqrt(sum of partials) / s (s = *nsp, or 1), summed in a fixed order by one block.
static __global__ void k_finish_norm(const double* partials, int nblocks, double* out, const float* nsp) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[b];
  v = block_sum(v);
  if (threadIdx.x == 0) out[0] = sqrt(v) / (nsp ? (double)*nsp : 1.0);
}

// out[0] = sum of partials (no square root), used for means.
static __global__ void k_finish_sum(const double* partials, int nblocks, double* out) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[b];
  v = block_sum(v);
  if (threadIdx.x == 0) out[0] = v;
}

template <typename T, int DIM>
__global__ void k_restrict(T* uc, T* uc0, T* fc, const T* u, const T* r, int nxf, int nyf, int nzf) {
  restrict_range<T, DIM>(uc, uc0, fc, u, r, nxf, nyf, nzf, gtid(), gstride());
}

template <typename T, int DIM>
__global__ void k_tau(T* fc, const T* uc, LevelDesc<T> Lc) {
  if (Lc.per)
    tau_range<T, DIM, true>(fc, uc, Lc, gtid(), gstride());
  else
    tau_range<T, DIM, false>(fc, uc, Lc, gtid(), gstride());
}

template <typename T, int DIM>
__global__ void k_prolong(T* u, const T* uc, const T* uc0, int nxf, int nyf, int nzf) {
  prolong_range<T, DIM>(u, uc, uc0, nxf, nyf, nzf, gtid(), gstride());
}

template <typename T, int DIM, int FAX>
__global__ void k_restrict_face(T* uc, T* uc0, T* fc, const T* u, const T* r, int nxf, int nyf, int nzf) {
  restrict_face_range<T, DIM, FAX>(uc, uc0, fc, u, r, nxf, nyf, nzf, gtid(), gstride());
}

template <typename T, int DIM, int FAX>
__global__ void k_prolong_face(T* u, const T* uc, const T* uc0, int nxf, int nyf, int nzf) {
  prolong_face_range<T, DIM, FAX>(u, uc, uc0, nxf, nyf, nzf, gtid(), gstride());
}

// per-block partial sums of x (for means of singular problems)
template <typename T>
__global__ void k_sum(const T* x, int64_t n, double* partials) {
  double acc = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) acc += (double)x[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// x = y - mean, mean = sum[0] / n (y may equal x)
template <typename T>
__global__ void k_sub_mean(T* x, const T* y, int64_t n, const double* sum) {
  const T m = (T)(sum[0] / (double)n);
  for (int64_t i = gtid(); i < n; i += gstride()) x[i] = y[i] - m;
}

// heat step right-hand side: b = u + dt * fsrc (fsrc may be null: b = u), with the per-block partial
// sums of b^2 (float squares) for ||b||
static __global__ void k_heat_rhs(double* b, const double* u, const double* fsrc, double dt, int64_t n, double* partials) {
  float acc = 0.f;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double v = fsrc ? fma(dt, fsrc[i], u[i]) : u[i];
    b[i] = v;
    const float vf = f64_to_f32_rn_bits(v);
    acc = fmaf(vf, vf, acc);
  }
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// ---- mixed precision (iterative refinement): u += e, and r32 = (float)(b - A u) with its norm
static __global__ void k_ir_update(double* u, const float* e, int64_t n) {
  // four cells per iteration (one 16-byte load of e, two of u; both fields 16-byte aligned), then the
  // remaining n % 4 one by one
  const int64_t n4 = n >> 2;
  for (int64_t i = gtid(); i < n4; i += gstride()) {
    const float4 ev = reinterpret_cast<const float4*>(e)[i];
    double2* up = reinterpret_cast<double2*>(u) + 2 * i;
    double2 a = up[0], b = up[1];
    a.x += f32_to_f64_bits(ev.x);
    a.y += f32_to_f64_bits(ev.y);
    b.x += f32_to_f64_bits(ev.z);
    b.y += f32_to_f64_bits(ev.w);
    up[0] = a;
    up[1] = b;
  }
  for (int64_t i = 4 * n4 + gtid(); i < n; i += gstride()) u[i] += f32_to_f64_bits(e[i]);
}

// Bit patterns of the neighbours of cell (i, j, l) in the order x-, x+, y-, y+, z-, z+ (0 where a
// neighbour is missing; the wrapped cell across a periodic boundary) and the mask of the present ones.
template <int DIM>
__device__ __forceinline__ unsigned nb_bits(const double* __restrict__ u, int64_t idx, int i, int j, int l,
                                            const LevelDesc<double>& L, uint64_t (&nb)[2 * DIM]) {
  const unsigned long long* ub = reinterpret_cast<const unsigned long long*>(u);
  const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
  const bool px = L.per & 1, py = (L.per >> 1) & 1;
  const bool p0 = i > 0 || px, p1 = i < L.nx - 1 || px, p2 = j > 0 || py, p3 = j < L.ny - 1 || py;
  nb[0] = p0 ? ub[i > 0 ? idx - 1 : idx + L.nx - 1] : 0ull;
  nb[1] = p1 ? ub[i < L.nx - 1 ? idx + 1 : idx - (L.nx - 1)] : 0ull;
  nb[2] = p2 ? ub[j > 0 ? idx - sy : idx + (L.ny - 1) * sy] : 0ull;
  nb[3] = p3 ? ub[j < L.ny - 1 ? idx + sy : idx - (L.ny - 1) * sy] : 0ull;
  unsigned mask = (unsigned)p0 | ((unsigned)p1 << 1) | ((unsigned)p2 << 2) | ((unsigned)p3 << 3);
  if constexpr (DIM == 3) {
    const bool pz = (L.per >> 2) & 1;
    const bool p4 = l > 0 || pz, p5 = l < L.nz - 1 || pz;
    nb[4] = p4 ? ub[l > 0 ? idx - sz : idx + (L.nz - 1) * sz] : 0ull;
    nb[5] = p5 ? ub[l < L.nz - 1 ? idx + sz : idx - (L.nz - 1) * sz] : 0ull;
    mask |= ((unsigned)p4 << 4) | ((unsigned)p5 << 5);
  }
  return mask;
}

// r32 = (float)(b - A u) and the per-block partial of sum (nscale r32)^2. With constant kappa the
// point equation is evaluated as fma(c, S, fma(-alpha, u, b)) with S = sum_nb u_nb - M u exact
// (bits64.cuh); cells where that does not apply take the float64 point equation.
template <int DIM>
__global__ void k_ir_residual(float* r32, const double* u, const double* b, LevelDesc<double> L, const float* nsp,
                              double* partials) {
  const int64_t n = (int64_t)L.nx * L.ny * L.nz;
  const float nscale = nsp ? *nsp : 1.f;
  float acc = 0.f;
  for (int64_t idx = gtid(); idx < n; idx += gstride()) {
    const int i = (int)(idx & (L.nx - 1));
    const int j = (int)((idx >> L.lx) & (L.ny - 1));
    const int l = (int)(idx >> (L.lx + L.ly));
    float rv = 0.f;
    if (!(L.fax >= 0 && frozen(L, i, j, l))) {
      double r = 0.0, S = 0.0;
      bool done = false;
      if (!L.varkappa) {
        uint64_t nb[2 * DIM];
        const unsigned mask = nb_bits<DIM>(u, idx, i, j, l, L, nb);
        const double uc = u[idx];
        const int cls = bclass<DIM>(i, j, l, L.nx, L.ny, L.nz);
        if (stencil_diff_exact<2 * DIM>((uint64_t)__double_as_longlong(uc), nb, mask, L.mt[cls], &S)) {
          r = fma(L.c, S, fma(-L.alpha, uc, b[idx]));
          done = true;
        }
      }
      if (!done)
        r = L.per ? residual_point<double, DIM, true>(u, b, L, idx, i, j, l)
                  : residual_point<double, DIM, false>(u, b, L, idx, i, j, l);
      rv = f64_to_f32_rn_bits(r);
    }
    r32[idx] = rv;
    const float rs = rv * nscale;
    acc = fmaf(rs, rs, acc);
  }
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// per-block partial of sum (nscale x)^2, squares of the float-rounded values (norms for stopping
// tests need a few digits only, and the conversion keeps the work off the FP64 pipe)
template <typename T>
__global__ void k_norm2(const T* x, int64_t n, const float* nsp, double* partials) {
  const float nscale = nsp ? *nsp : 1.f;
  float acc = 0.f;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const float v = (float)x[i] * nscale;
    acc = fmaf(v, v, acc);
  }
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename T>
__global__ void k_fill(T* x, T v, int64_t n) {
  for (int64_t i = gtid(); i < n; i += gstride()) x[i] = v;
}

template <typename S, typename D>
__global__ void k_convert(D* out, const S* in, int64_t n) {
  for (int64_t i = gtid(); i < n; i += gstride()) out[i] = (D)in[i];
}

// ------------------------------------------------------------------------------------------------
// variable-kappa level set-up: face weights w_f = beta * kappa_f (kappa_f = mean of the two cells)
// and D = alpha h^2 + sum_f m_f w_f with boundary faces taking the cell's kappa (m_f: 0 Neumann,
// 2 Dirichlet). bcm[6] are the boundary multiplicities per face x_lo..z_hi.
// ------------------------------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void k_kappa_weights(T* wx, T* wy, T* wz, T* rD, T* Dh, const double* kappa, int nx, int ny, int nz,
                                double alpha, double beta, double h, int4 bcm_lo, int4 bcm_hi) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  const double h2 = h * h;
  for (int64_t idx = gtid(); idx < n; idx += gstride()) {
    const int i = (int)(idx % nx);
    const int64_t rest = idx / nx;
    const int j = (int)(rest % ny);
    const int l = (int)(rest / ny);
    const double kc = kappa[idx];
    double D = alpha * h2;
    // x faces
    double w;
    w = i > 0 ? beta * (0.5 * (kappa[idx - 1] + kc)) : bcm_lo.x * beta * kc;
    D += w;
    w = i < nx - 1 ? beta * (0.5 * (kc + kappa[idx + 1])) : bcm_hi.x * beta * kc;
    D += w;
    wx[idx] = (T)(i < nx - 1 ? beta * (0.5 * (kc + kappa[idx + 1])) : 0.0);
    w = j > 0 ? beta * (0.5 * (kappa[idx - sy] + kc)) : bcm_lo.y * beta * kc;
    D += w;
    w = j < ny - 1 ? beta * (0.5 * (kc + kappa[idx + sy])) : bcm_hi.y * beta * kc;
    D += w;
    wy[idx] = (T)(j < ny - 1 ? beta * (0.5 * (kc + kappa[idx + sy])) : 0.0);
    if (DIM == 3) {
      w = l > 0 ? beta * (0.5 * (kappa[idx - sz] + kc)) : bcm_lo.z * beta * kc;
      D += w;
      w = l < nz - 1 ? beta * (0.5 * (kc + kappa[idx + sz])) : bcm_hi.z * beta * kc;
      D += w;
      wz[idx] = (T)(l < nz - 1 ? beta * (0.5 * (kc + kappa[idx + sz])) : 0.0);
    }
    rD[idx] = (T)(1.0 / D);
    Dh[idx] = (T)(D / h2);
  }
}

// ------------------------------------------------------------------------------------------------
// Arguments of the single-CTA V-cycle over levels l0..nlev-1 (the small levels, which cannot fill the
// GPU): the same recursion as the host driver, with __syncthreads() between dependent steps. Level l0
// is read from and written back to (utop, ftop). The coarsest level is smoothed (paper) or, when cinv
// is given, solved exactly by the dense inverse (pseudo-inverse when singular).
// ------------------------------------------------------------------------------------------------
template <typename T>
struct CoarseArgs {
  const LevelDesc<T>* desc;  // device array, one per level
  T* const* u;               // per-level buffers (entry l0 replaced by utop)
  T* const* f;
  T* const* u0;
  const T* cinv;  // dense inverse of the coarsest operator, or null
  int l0, nlev, nu1, nu2, nuc;
  int ordering;  // fas_ordering
};

// Colour updated first by sweep s of a smoothing step: the odd index sums (sets 1-2 in 2D, 1-4 in
// 3D) for a forward sweep; a symmetric ordering runs every second sweep backward.
__host__ __device__ __forceinline__ int first_colour(int ordering, int s) { return (ordering == 1 && (s & 1)) ? 0 : 1; }

template <typename T, int DIM, bool PER>
__device__ void coarse_smooth(T* u, const T* f, const LevelDesc<T>& L, int sweeps, int ordering) {
  for (int s = 0; s < sweeps; ++s) {
    const int c0 = first_colour(ordering, s);
    smooth_colour_range<T, DIM, PER>(u, f, L, c0, threadIdx.x, blockDim.x);
    __syncthreads();
    smooth_colour_range<T, DIM, PER>(u, f, L, 1 - c0, threadIdx.x, blockDim.x);
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------------
// Single-CTA V-cycle with every level held in shared memory: levels l0..nlev-1 of u and f, and the
// restricted start u0 of the coarser ones. Same steps and same per-point arithmetic as the grid-wide
// kernels (the residual is evaluated per child inside the restriction instead of being stored
// first), so the results are identical; the latency of each dependent step is a shared-memory round
// trip instead of an L2 one.
// ------------------------------------------------------------------------------------------------
struct SmemLayout {
  int64_t off_u[kMaxLevels], off_f[kMaxLevels], off_u0[kMaxLevels];  // element offsets
  int64_t total;                                                      // elements
};

template <typename T, int DIM, bool PER = false>
__device__ __forceinline__ void restrict_resid_range(T* uc, T* uc0, T* fc, const T* u, const T* f,
                                                     const LevelDesc<T>& L, int64_t t0, int64_t stride) {
  const int nxf = L.nx, nyf = L.ny, nzf = L.nz;
  const int nxc = nxf >> 1, nyc = nyf >> 1, nzc = DIM == 3 ? nzf >> 1 : 1;
  const int64_t nc = (int64_t)nxc * nyc * nzc;
  const int64_t sy = nxf, sz = (int64_t)nxf * nyf;
  const int lxc = L.lx - 1, lyc = L.ly - 1;
  for (int64_t I = t0; I < nc; I += stride) {
    const int ic = (int)(I & (nxc - 1));
    const int jc = (int)((I >> lxc) & (nyc - 1));
    const int lc = (int)(I >> (lxc + lyc));
    const int i0 = 2 * ic, j0 = 2 * jc, l0 = DIM == 3 ? 2 * lc : 0;
    const int64_t base = ((int64_t)l0 * nyf + j0) * nxf + i0;
    const T v = avg_children<T, DIM>(u, base, sy, sz);
    uc[I] = v;
    uc0[I] = v;
    T r[8];
#pragma unroll
    for (int k = 0; k < (DIM == 3 ? 8 : 4); ++k) {
      const int di = k & 1, dj = (k >> 1) & 1, dl = (k >> 2) & 1;
      const int64_t idx = base + di + dj * sy + dl * sz;
      r[k] = residual_point<T, DIM, PER>(u, f, L, idx, i0 + di, j0 + dj, l0 + dl);
    }
    // same association as avg_children: (c00 + c01) + (c10 + c11) [+ the upper z layer]
    T sr = (r[0] + r[1]) + (r[2] + r[3]);
    if (DIM == 3) {
      const T s2 = (r[4] + r[5]) + (r[6] + r[7]);
      fc[I] = (sr + s2) * T(0.125);
    } else {
      fc[I] = sr * T(0.25);
    }
  }
}

// Face-grid counterpart: the fine residual is evaluated at each fine face the Appendix D weights
// touch (the three normal slots overlap between neighbouring coarse faces, so some are evaluated
// twice); the arithmetic per value equals that of k_residual followed by k_restrict_face.
template <typename T, int DIM, int FAX>
__device__ __forceinline__ void restrict_resid_face_range(T* uc, T* uc0, T* fc, const T* u, const T* f,
                                                          const LevelDesc<T>& L, int64_t t0, int64_t stride) {
  const int nxf = L.nx, nyf = L.ny;
  const int nxc = nxf >> 1, nyc = nyf >> 1, nzc = DIM == 3 ? L.nz >> 1 : 1;
  const int64_t nc = (int64_t)nxc * nyc * nzc;
  const int lxc = L.lx - 1, lyc = L.ly - 1;
  auto resid = [&](int64_t q, int i, int j, int l) {
    return frozen(L, i, j, l) ? T(0) : residual_point<T, DIM>(u, f, L, q, i, j, l);
  };
  for (int64_t I = t0; I < nc; I += stride) {
    const int ic = (int)(I & (nxc - 1));
    const int jc = (int)((I >> lxc) & (nyc - 1));
    const int lc = (int)(I >> (lxc + lyc));
    const bool wall = wall_slot<FAX>(ic, jc, lc, nxc, nyc, nzc);
    const T v = wall ? T(0) : face_avg<T, DIM, FAX>(u, ic, jc, lc, nxf, nyf);
    uc[I] = v;
    uc0[I] = v;
    fc[I] = wall ? T(0) : face_avg_of<T, DIM, FAX>(resid, ic, jc, lc, nxf, nyf);
  }
}

// Grid-wide restriction with the residual evaluated per child on the fly (never stored):
// uc = uc0 = R(u), fc = R(f - A u); the same per-point arithmetic and association as k_residual
// followed by k_restrict / k_restrict_face, so the results are identical.
template <typename T, int DIM, int FAX>
__global__ void k_restrict_resid(T* uc, T* uc0, T* fc, const T* u, const T* f, LevelDesc<T> L) {
  if constexpr (FAX < 0) {
    if (L.per)
      restrict_resid_range<T, DIM, true>(uc, uc0, fc, u, f, L, gtid(), gstride());
    else
      restrict_resid_range<T, DIM, false>(uc, uc0, fc, u, f, L, gtid(), gstride());
  } else
    restrict_resid_face_range<T, DIM, FAX>(uc, uc0, fc, u, f, L, gtid(), gstride());
}

// 3D float32 cell levels with constant kappa, no periodic axis and a multiple of 4 cells per row: the
// residual-restriction of k_restrict_resid with one thread per 4 x 2 x 2 block of fine cells (two
// coarse cells), every row of the block and of its y and z neighbours read as one 16-byte vector.
// Each residual is residual_point's expression and R(u), R(r) use avg_children's association, so the
// results are those of k_restrict_resid bit for bit.
static __global__ void __launch_bounds__(256) k_restrict_resid4_3d(float* __restrict__ uc, float* __restrict__ uc0,
                                                            float* __restrict__ fc, const float* __restrict__ u,
                                                            const float* __restrict__ f, const LevelDesc<float> L) {
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  const int lg = L.lx - 2;
  const int64_t ngroups = (int64_t)1 << (lg + L.ly - 1 + L.lz - 1);
  for (int64_t g = gtid(); g < ngroups; g += gstride()) {
    const int x0 = (int)(g & ((1 << lg) - 1)) << 2;
    const int64_t rest = g >> lg;
    const int j0 = (int)(rest & ((ny >> 1) - 1)) << 1;
    const int l0 = (int)(rest >> (L.ly - 1)) << 1;
    const int64_t base = ((int64_t)l0 * ny + j0) * nx + x0;
    Quad<float> c[2][2], fq[2][2], sq[2], nq[2], bq[2], tq[2];  // [dl][dj]; y neighbours per dl; z per dj
    float we[2][2], ee[2][2];
#pragma unroll
    for (int dl = 0; dl < 2; ++dl)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj) {
        const int64_t q = base + dl * sz + dj * sy;
        c[dl][dj].ld(u + q);
        fq[dl][dj].ld(f + q);
        we[dl][dj] = x0 > 0 ? u[q - 1] : 0.f;
        ee[dl][dj] = x0 + 4 < nx ? u[q + 4] : 0.f;
      }
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      sq[d].v[0] = sq[d].v[1] = sq[d].v[2] = sq[d].v[3] = 0.f;
      nq[d] = sq[d];
      bq[d] = sq[d];
      tq[d] = sq[d];
      if (j0 > 0) sq[d].ld(u + base + d * sz - sy);
      if (j0 + 2 < ny) nq[d].ld(u + base + d * sz + 2 * sy);
      if (l0 > 0) bq[d].ld(u + base + d * sy - sz);
      if (l0 + 2 < nz) tq[d].ld(u + base + d * sy + 2 * sz);
    }
    float r[2][2][4];
#pragma unroll
    for (int dl = 0; dl < 2; ++dl)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float w = k > 0 ? c[dl][dj].v[k > 0 ? k - 1 : 0] : we[dl][dj];
          const float e = k < 3 ? c[dl][dj].v[k < 3 ? k + 1 : 3] : ee[dl][dj];
          const float sv = dj == 0 ? sq[dl].v[k] : c[dl][0].v[k];
          const float nv = dj == 0 ? c[dl][1].v[k] : nq[dl].v[k];
          const float bo = dl == 0 ? bq[dj].v[k] : c[0][dj].v[k];
          const float to = dl == 0 ? c[1][dj].v[k] : tq[dj].v[k];
          const float acc = ((w + e) + (sv + nv)) + (bo + to);
          const int cls = bclass<3>(x0 + k, j0 + dj, l0 + dl, nx, ny, nz);
          r[dl][dj][k] = fmaf(L.c, acc, fmaf(-L.d[cls], c[dl][dj].v[k], fq[dl][dj].v[k]));
        }
    const int64_t I = ((int64_t)(l0 >> 1) * (ny >> 1) + (j0 >> 1)) * (nx >> 1) + (x0 >> 1);
#pragma unroll
    for (int qc = 0; qc < 2; ++qc) {
      const int a = 2 * qc, b = 2 * qc + 1;
      const float s1 = (c[0][0].v[a] + c[0][0].v[b]) + (c[0][1].v[a] + c[0][1].v[b]);
      const float s2 = (c[1][0].v[a] + c[1][0].v[b]) + (c[1][1].v[a] + c[1][1].v[b]);
      const float v = (s1 + s2) * 0.125f;
      uc[I + qc] = v;
      uc0[I + qc] = v;
      const float r1 = (r[0][0][a] + r[0][0][b]) + (r[0][1][a] + r[0][1][b]);
      const float r2 = (r[1][0][a] + r[1][0][b]) + (r[1][1][a] + r[1][1][b]);
      fc[I + qc] = (r1 + r2) * 0.125f;
    }
  }
}

// The tau correction fc += A_c uc on the same kind of 3D float32 level, 4 cells per thread
// (apply_point's expression per cell, so the results equal k_tau's).
static __global__ void __launch_bounds__(256) k_tau4_3d(float* __restrict__ fc, const float* __restrict__ uc,
                                                        const LevelDesc<float> L) {
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  const int lg = L.lx - 2;
  const int64_t ngroups = (int64_t)1 << (lg + L.ly + L.lz);
  for (int64_t g = gtid(); g < ngroups; g += gstride()) {
    const int x0 = (int)(g & ((1 << lg) - 1)) << 2;
    const int64_t rest = g >> lg;
    const int j = (int)(rest & (ny - 1));
    const int l = (int)(rest >> L.ly);
    const int64_t idx = ((int64_t)l * ny + j) * nx + x0;
    Quad<float> c, fq, sq, nq, bq, tq;
    c.ld(uc + idx);
    fq.ld(fc + idx);
    sq.v[0] = sq.v[1] = sq.v[2] = sq.v[3] = 0.f;
    nq = sq;
    bq = sq;
    tq = sq;
    if (j > 0) sq.ld(uc + idx - sy);
    if (j < ny - 1) nq.ld(uc + idx + sy);
    if (l > 0) bq.ld(uc + idx - sz);
    if (l < nz - 1) tq.ld(uc + idx + sz);
    const float we = x0 > 0 ? uc[idx - 1] : 0.f, ee = x0 + 4 < nx ? uc[idx + 4] : 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float w = k > 0 ? c.v[k > 0 ? k - 1 : 0] : we, e = k < 3 ? c.v[k < 3 ? k + 1 : 3] : ee;
      const float acc = ((w + e) + (sq.v[k] + nq.v[k])) + (bq.v[k] + tq.v[k]);
      const int cls = bclass<3>(x0 + k, j, l, nx, ny, nz);
      fq.v[k] = fq.v[k] + fmaf(L.d[cls], c.v[k], -L.c * acc);
    }
    fq.st(fc + idx);
  }
}

// The single-CTA V-cycle's work once its descriptors are in shared memory (sdesc, indexed by level).
template <typename T, int DIM, int FAX, bool PER>
__device__ __forceinline__ void coarse_body(const CoarseArgs<T>& A, const SmemLayout& S, T* utop, const T* ftop, T* sm,
                                            const LevelDesc<T>* sdesc) {
  const int last = A.nlev - 1;
  {
    const LevelDesc<T>& L = sdesc[A.l0];
    const int64_t n = (int64_t)L.nx * L.ny * L.nz;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      sm[S.off_u[A.l0] + i] = utop[i];
      sm[S.off_f[A.l0] + i] = ftop[i];
    }
  }
  __syncthreads();
  for (int l = A.l0; l < last; ++l) {
    const LevelDesc<T>& L = sdesc[l];
    T* u = sm + S.off_u[l];
    const T* f = sm + S.off_f[l];
    coarse_smooth<T, DIM, PER>(u, f, L, A.nu1, A.ordering);
    if constexpr (FAX < 0)
      restrict_resid_range<T, DIM, PER>(sm + S.off_u[l + 1], sm + S.off_u0[l + 1], sm + S.off_f[l + 1], u, f, L,
                                   threadIdx.x, blockDim.x);
    else
      restrict_resid_face_range<T, DIM, FAX>(sm + S.off_u[l + 1], sm + S.off_u0[l + 1], sm + S.off_f[l + 1], u, f,
                                             L, threadIdx.x, blockDim.x);
    __syncthreads();
    tau_range<T, DIM, PER>(sm + S.off_f[l + 1], sm + S.off_u[l + 1], sdesc[l + 1], threadIdx.x, blockDim.x);
    __syncthreads();
  }
  {
    const LevelDesc<T>& L = sdesc[last];
    T* u = sm + S.off_u[last];
    const T* f = sm + S.off_f[last];
    if (A.cinv) {  // coarsest level of at most 1024 cells (checked on the host): one cell per thread
      const int n = L.nx * L.ny * L.nz;
      const int p = threadIdx.x;
      if (p < n) {
        T acc = T(0);
        for (int q = 0; q < n; ++q) acc = fma(A.cinv[(int64_t)p * n + q], f[q], acc);
        u[p] = acc;
      }
      __syncthreads();
    } else {
      coarse_smooth<T, DIM, PER>(u, f, L, A.nuc, A.ordering);
    }
  }
  for (int l = last - 1; l >= A.l0; --l) {
    const LevelDesc<T>& L = sdesc[l];
    T* u = sm + S.off_u[l];
    const T* f = sm + S.off_f[l];
    if constexpr (FAX < 0)
      prolong_range<T, DIM>(u, sm + S.off_u[l + 1], sm + S.off_u0[l + 1], L.nx, L.ny, L.nz, threadIdx.x, blockDim.x);
    else
      prolong_face_range<T, DIM, FAX>(u, sm + S.off_u[l + 1], sm + S.off_u0[l + 1], L.nx, L.ny, L.nz, threadIdx.x,
                                      blockDim.x);
    __syncthreads();
    coarse_smooth<T, DIM, PER>(u, f, L, A.nu2, A.ordering);
  }
  {
    const LevelDesc<T>& L = sdesc[A.l0];
    const int64_t n = (int64_t)L.nx * L.ny * L.nz;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) utop[i] = sm[S.off_u[A.l0] + i];
  }
}

// FAX = -1: cell-centred levels; 0..2: face grids normal to that index axis.
template <typename T, int DIM, int FAX>
__global__ void __launch_bounds__(1024) k_coarse_smem(CoarseArgs<T> A, SmemLayout S, T* utop, const T* ftop) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  // level descriptors of levels l0..last, copied after the field arrays (every stencil reads them)
  LevelDesc<T>* sdesc = reinterpret_cast<LevelDesc<T>*>(smem_raw + S.total * sizeof(T)) - A.l0;
  {
    const int words = (int)((A.nlev - A.l0) * sizeof(LevelDesc<T>) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(A.desc + A.l0);
    int* dst = reinterpret_cast<int*>(sdesc + A.l0);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  if constexpr (FAX < 0) {
    if (sdesc[A.l0].per) {  // every level of a hierarchy has the same periodic axes
      coarse_body<T, DIM, FAX, true>(A, S, utop, ftop, sm, sdesc);
      return;
    }
  }
  coarse_body<T, DIM, FAX, false>(A, S, utop, ftop, sm, sdesc);
}

// ------------------------------------------------------------------------------------------------
// Adjoint of backward-Euler heat stepping: -(d(mu^T A u)/d kappa) per cell, added to g. Interior face
// c|nb: -(beta/h^2)(u_nb - u_c)(mu_nb - mu_c), half to each cell (face kappa = mean of the two
// cells); Dirichlet face: -(2 beta/h^2) mu_c u_c (face kappa = cell kappa); Neumann faces: nothing.
// scale = beta / h^2; dir[f] = 1 for a Dirichlet face f (x_lo, x_hi, y_lo, y_hi, z_lo, z_hi).
// ------------------------------------------------------------------------------------------------
template <int DIM>
__global__ void k_kappa_grad(double* g, const double* u, const double* mu, int nx, int ny, int nz, int lx, int ly,
                             double scale, int dirmask) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  for (int64_t idx = gtid(); idx < n; idx += gstride()) {
    const int i = (int)(idx & (nx - 1));
    const int j = (int)((idx >> lx) & (ny - 1));
    const int l = (int)(idx >> (lx + ly));
    const double uc = u[idx], mc = mu[idx];
    double acc = 0.0;
    if (i > 0) acc += (u[idx - 1] - uc) * (mu[idx - 1] - mc);
    if (i < nx - 1) acc += (u[idx + 1] - uc) * (mu[idx + 1] - mc);
    if (j > 0) acc += (u[idx - sy] - uc) * (mu[idx - sy] - mc);
    if (j < ny - 1) acc += (u[idx + sy] - uc) * (mu[idx + sy] - mc);
    if (DIM == 3) {
      if (l > 0) acc += (u[idx - sz] - uc) * (mu[idx - sz] - mc);
      if (l < nz - 1) acc += (u[idx + sz] - uc) * (mu[idx + sz] - mc);
    }
    double v = -0.5 * scale * acc;
    int nd = 0;  // Dirichlet faces of this cell
    nd += (i == 0) & (dirmask & 1);
    nd += (i == nx - 1) & ((dirmask >> 1) & 1);
    nd += (j == 0) & ((dirmask >> 2) & 1);
    nd += (j == ny - 1) & ((dirmask >> 3) & 1);
    if (DIM == 3) {
      nd += (l == 0) & ((dirmask >> 4) & 1);
      nd += (l == nz - 1) & ((dirmask >> 5) & 1);
    }
    if (nd) v -= 2.0 * scale * nd * mc * uc;
    g[idx] += v;
  }
}

// y += a x
static __global__ void k_axpy(double* y, double a, const double* x, int64_t n) {
  for (int64_t i = gtid(); i < n; i += gstride()) y[i] = fma(a, x[i], y[i]);
}

// ------------------------------------------------------------------------------------------------
// Device-side state of one solve (Algorithm 1's outer loop): the stopping decision is taken on the
// device, so that the same kernels serve a host-driven loop and a graph with a conditional node.
// ------------------------------------------------------------------------------------------------
struct SolveState {
  double fn;      // ||f||_2
  double res0;    // ||f - A u||_2 before the first cycle
  double res;     // after the last cycle
  double ref;     // reference of the relative test (||f||, or res0 when f = 0), 1 in absolute mode
  double w;       // 1 (relative test) or h^{d/2} (the paper's absolute h-weighted norm)
  double tol;
  float nscale;   // power of two applied to values before squaring them in float
  int kmax;
  int cycles;
  int converged;
  int nonfinite;
  int cond;       // 1: run another cycle
};

// After ||f|| is known: the norm scale (a power of two bringing the rms of f near 1).
static __global__ void k_solve_begin(SolveState* S, double tol, int kmax, double w, double ncells) {
  const double fn = S->fn;
  float s = 1.f;
  if (fn > 0.0 && isfinite(fn)) {
    const int e = (int)lrint(log2(fn / sqrt(ncells)));
    s = (float)ldexp(1.0, -max(-120, min(120, e)));
  }
  S->nscale = s;
  S->tol = tol;
  S->kmax = kmax;
  S->w = w;
  S->cycles = 0;
  S->converged = 0;
  S->nonfinite = 0;
  S->cond = 1;  // Algorithm 1 runs at least one cycle
}

// After the initial residual: the reference of the relative test.
static __global__ void k_solve_ref(SolveState* S, int relative) {
  S->ref = relative ? (S->fn > 0.0 ? S->fn : S->res0) : 1.0;
}

// After each cycle's residual norm (in S->res): count it and decide whether to continue. When
// set_cond, also set the graph's conditional (the kernel then runs inside the while node's body).
static __global__ void k_solve_step(SolveState* S, cudaGraphConditionalHandle h, int set_cond) {
  S->cycles += 1;
  const double res = S->w * S->res;
  int cond = 1;
  if (!isfinite(res)) {
    S->nonfinite = 1;
    cond = 0;
  } else if (res <= S->tol * S->ref) {
    S->converged = 1;
    cond = 0;
  } else if (S->cycles >= S->kmax) {
    cond = 0;
  }
  S->cond = cond;
  if (set_cond) cudaGraphSetConditional(h, (unsigned)cond);
}

}  // namespace fasmg
