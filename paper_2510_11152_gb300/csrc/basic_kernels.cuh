// basic_kernels.cuh -- one-operation-per-launch kernels for every level, templated on the value type
// (double / float) and the dimension. Each operation is written as a range loop (start, stride) so
// that the same code serves a grid-stride launch and the single-CTA kernel that runs the whole
// V-cycle below a switch level (where every level is too small to fill the GPU).
//
// No pointer here is declared __restrict__ or read through the non-coherent path: the single-CTA
// kernel writes a level in one step and reads it in the next, separated only by __syncthreads.
#pragma once
#include "common.cuh"

namespace fasmg {

// ---- X-MCGS colour phase (Sec. 2.3). colour 1: cells whose 1-based index sum i+j(+l) is odd (the
// paper's sets 1,2 in 2D, sets 1-4 in 3D); colour 0: even (sets 3,4 / 5-8). With the 0-based indices
// used here the 1-based sum is the 0-based sum plus DIM. Every cell of a colour has only other-colour
// neighbours, so all of them update at once from the current values.
template <typename T, int DIM>
__device__ __forceinline__ void smooth_colour_range(T* u, const T* f, const LevelDesc<T>& L, int colour,
                                                    int64_t t0, int64_t stride) {
  const int hx = L.nx >> 1;
  const int64_t half = (int64_t)hx * L.ny * L.nz;
  for (int64_t t = t0; t < half; t += stride) {
    const int k = (int)(t % hx);
    const int64_t rest = t / hx;
    const int j = (int)(rest % L.ny);
    const int l = (int)(rest / L.ny);
    const int i = 2 * k + ((colour + DIM + j + l) & 1);
    const int64_t idx = ((int64_t)l * L.ny + j) * L.nx + i;
    u[idx] = point_update<T, DIM>(u, f, L, idx, i, j, l);
  }
}

// ---- r = f - A u (Sec. 2.2) over a range of cells; returns the thread's sum of (scale*r)^2.
template <typename T, int DIM>
__device__ __forceinline__ float residual_range(T* r, const T* u, const T* f, const LevelDesc<T>& L,
                                                float nscale, int64_t t0, int64_t stride) {
  const int64_t n = (int64_t)L.nx * L.ny * L.nz;
  float acc = 0.f;
  for (int64_t idx = t0; idx < n; idx += stride) {
    const int i = (int)(idx % L.nx);
    const int64_t rest = idx / L.nx;
    const int j = (int)(rest % L.ny);
    const int l = (int)(rest / L.ny);
    const T rv = residual_point<T, DIM>(u, f, L, idx, i, j, l);
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
  for (int64_t I = t0; I < nc; I += stride) {
    const int ic = (int)(I % nxc);
    const int64_t rest = I / nxc;
    const int jc = (int)(rest % nyc);
    const int lc = (int)(rest / nyc);
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
template <typename T, int DIM>
__device__ __forceinline__ void tau_range(T* fc, const T* uc, const LevelDesc<T>& Lc, int64_t t0,
                                          int64_t stride) {
  const int64_t n = (int64_t)Lc.nx * Lc.ny * Lc.nz;
  for (int64_t idx = t0; idx < n; idx += stride) {
    const int i = (int)(idx % Lc.nx);
    const int64_t rest = idx / Lc.nx;
    const int j = (int)(rest % Lc.ny);
    const int l = (int)(rest / Lc.ny);
    fc[idx] = fc[idx] + apply_point<T, DIM>(uc, Lc, idx, i, j, l);
  }
}

// ---- Appendix C prolongation of the correction: u += P(uc - uc0), every child gets its parent's.
template <typename T, int DIM>
__device__ __forceinline__ void prolong_range(T* u, const T* uc, const T* uc0, int nxf, int nyf, int nzf,
                                              int64_t t0, int64_t stride) {
  const int nxc = nxf >> 1, nyc = nyf >> 1, nzc = DIM == 3 ? nzf >> 1 : 1;
  const int64_t nc = (int64_t)nxc * nyc * nzc;
  const int64_t sy = nxf, sz = (int64_t)nxf * nyf;
  for (int64_t I = t0; I < nc; I += stride) {
    const int ic = (int)(I % nxc);
    const int64_t rest = I / nxc;
    const int jc = (int)(rest % nyc);
    const int lc = (int)(rest / nyc);
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

// ------------------------------------------------------------------------------------------------
// grid-stride kernels
// ------------------------------------------------------------------------------------------------

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

template <typename T, int DIM>
__global__ void k_smooth_colour(T* u, const T* f, LevelDesc<T> L, int colour) {
  smooth_colour_range<T, DIM>(u, f, L, colour, gtid(), gstride());
}

// r (nullable) = f - A u; per-block partial of sum (nscale r)^2 into partials[blockIdx.x].
template <typename T, int DIM>
__global__ void k_residual(T* r, const T* u, const T* f, LevelDesc<T> L, float nscale, double* partials) {
  const float acc = residual_range<T, DIM>(r, u, f, L, nscale, gtid(), gstride());
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0 && partials) partials[blockIdx.x] = s;
}

// out[0] = sqrt(sum of partials) / nscale, summed in a fixed order by one block.
__global__ void k_finish_norm(const double* partials, int nblocks, double* out, double inv_scale) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[b];
  v = block_sum(v);
  if (threadIdx.x == 0) out[0] = sqrt(v) * inv_scale;
}

// out[0] = sum of partials (no square root), used for means.
__global__ void k_finish_sum(const double* partials, int nblocks, double* out) {
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
  tau_range<T, DIM>(fc, uc, Lc, gtid(), gstride());
}

template <typename T, int DIM>
__global__ void k_prolong(T* u, const T* uc, const T* uc0, int nxf, int nyf, int nzf) {
  prolong_range<T, DIM>(u, uc, uc0, nxf, nyf, nzf, gtid(), gstride());
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

// heat step right-hand side: b = u + dt * fsrc (fsrc may be null: b = u)
__global__ void k_heat_rhs(double* b, const double* u, const double* fsrc, double dt, int64_t n) {
  for (int64_t i = gtid(); i < n; i += gstride()) b[i] = fsrc ? fma(dt, fsrc[i], u[i]) : u[i];
}

// ---- mixed precision (iterative refinement): u += e, and r32 = (float)(b - A u) with its norm
__global__ void k_ir_update(double* u, const float* e, int64_t n) {
  for (int64_t i = gtid(); i < n; i += gstride()) u[i] += (double)e[i];
}

template <int DIM>
__global__ void k_ir_residual(float* r32, const double* u, const double* b, LevelDesc<double> L, float nscale,
                              double* partials) {
  const int64_t n = (int64_t)L.nx * L.ny * L.nz;
  float acc = 0.f;
  for (int64_t idx = gtid(); idx < n; idx += gstride()) {
    const int i = (int)(idx % L.nx);
    const int64_t rest = idx / L.nx;
    const int j = (int)(rest % L.ny);
    const int l = (int)(rest / L.ny);
    const float rv = (float)residual_point<double, DIM>(u, b, L, idx, i, j, l);
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
__global__ void k_norm2(const T* x, int64_t n, float nscale, double* partials) {
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
// Single-CTA V-cycle over levels l0..nlev-1 (the small levels, which cannot fill the GPU): the same
// recursion as the host driver, with __syncthreads() between dependent steps. Level l0 works on
// (utop, ftop); deeper levels on the context's buffers. The coarsest level is smoothed (paper) or,
// when cinv is given, solved exactly by the dense inverse (pseudo-inverse when singular).
// ------------------------------------------------------------------------------------------------
template <typename T>
struct CoarseArgs {
  const LevelDesc<T>* desc;  // device array, one per level
  T* const* u;               // per-level buffers (entry l0 replaced by utop)
  T* const* f;
  T* const* r;
  T* const* u0;
  const T* cinv;  // dense inverse of the coarsest operator, or null
  int l0, nlev, nu1, nu2, nuc;
};

template <typename T, int DIM>
__device__ void coarse_smooth(T* u, const T* f, const LevelDesc<T>& L, int sweeps) {
  for (int s = 0; s < sweeps; ++s) {
    smooth_colour_range<T, DIM>(u, f, L, 1, threadIdx.x, blockDim.x);
    __syncthreads();
    smooth_colour_range<T, DIM>(u, f, L, 0, threadIdx.x, blockDim.x);
    __syncthreads();
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(1024) k_coarse_vcycle(CoarseArgs<T> A, T* utop, const T* ftop) {
  const int last = A.nlev - 1;
  // descend
  for (int l = A.l0; l < last; ++l) {
    const LevelDesc<T>& L = A.desc[l];
    const LevelDesc<T>& Lc = A.desc[l + 1];
    T* u = l == A.l0 ? utop : A.u[l];
    const T* f = l == A.l0 ? ftop : A.f[l];
    coarse_smooth<T, DIM>(u, f, L, A.nu1);
    residual_range<T, DIM>(A.r[l], u, f, L, 1.f, threadIdx.x, blockDim.x);
    __syncthreads();
    restrict_range<T, DIM>(A.u[l + 1], A.u0[l + 1], A.f[l + 1], u, A.r[l], L.nx, L.ny, L.nz, threadIdx.x,
                           blockDim.x);
    __syncthreads();
    tau_range<T, DIM>(A.f[l + 1], A.u[l + 1], Lc, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  // coarsest level
  {
    const LevelDesc<T>& L = A.desc[last];
    T* u = last == A.l0 ? utop : A.u[last];
    const T* f = last == A.l0 ? ftop : A.f[last];
    if (A.cinv) {
      const int n = L.nx * L.ny * L.nz;
      for (int p = threadIdx.x; p < n; p += blockDim.x) {
        T acc = T(0);
        for (int q = 0; q < n; ++q) acc = fma(A.cinv[(int64_t)p * n + q], f[q], acc);
        A.r[last][p] = acc;
      }
      __syncthreads();
      for (int p = threadIdx.x; p < n; p += blockDim.x) u[p] = A.r[last][p];
      __syncthreads();
    } else {
      coarse_smooth<T, DIM>(u, f, L, A.nuc);
    }
  }
  // ascend
  for (int l = last - 1; l >= A.l0; --l) {
    const LevelDesc<T>& L = A.desc[l];
    T* u = l == A.l0 ? utop : A.u[l];
    const T* f = l == A.l0 ? ftop : A.f[l];
    prolong_range<T, DIM>(u, A.u[l + 1], A.u0[l + 1], L.nx, L.ny, L.nz, threadIdx.x, blockDim.x);
    __syncthreads();
    coarse_smooth<T, DIM>(u, f, L, A.nu2);
  }
}

}  // namespace fasmg
