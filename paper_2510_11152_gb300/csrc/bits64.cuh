// bits64.cuh -- float64 work moved off the FP64 pipe.
//
// GB300 issues float64 arithmetic and float32<->float64 conversions at a small fraction of its
// integer and float32 rates, so the float64 steps of the mixed-precision refinement (the fine-grid
// residual r = b - A u rounded to float32, and u += e) are bound by that pipe, not by HBM. These
// helpers do the same work with integer operations on the IEEE 754 bit patterns:
//   - exact float32 -> float64 and round-to-nearest-even float64 -> float32 conversions, field by
//     field from the binary32 / binary64 formats (IEEE 754-2008, Sec. 3.4);
//   - the stencil difference S = sum_nb u_nb - M u_c of the point equation, computed EXACTLY as an
//     integer sum of the significands aligned to the smallest exponent in the stencil, then rounded
//     once to float64. With it the residual f - (alpha + c M) u + c sum_nb u_nb is evaluated as
//     fma(c, S, fma(-alpha, u, f)): two float64 operations instead of five, and more accurate (the
//     cancellation inside S, large when beta/h^2 is large, happens without rounding).
#pragma once

#include <cstdint>

namespace fasmg {

constexpr uint64_t kMant52 = (1ull << 52) - 1;

// float32 -> float64, exact. Zero, subnormal, normal, infinity and NaN (payload kept, like the
// hardware conversion of a quiet NaN).
__device__ __forceinline__ double f32_to_f64_bits(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint32_t m = b & 0x7FFFFFu;
  uint64_t out;
  if (e == 0xFFu) {
    out = sign | (0x7FFull << 52) | ((uint64_t)m << 29);
  } else if (e != 0u) {
    out = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
  } else if (m == 0u) {
    out = sign;
  } else {  // subnormal: m 2^-149 with the leading one at bit p
    const int p = 31 - __clz(m);
    out = sign | ((uint64_t)(p + 874) << 52) | (((uint64_t)m << (52 - p)) & kMant52);
  }
  return __longlong_as_double((long long)out);
}

// float64 -> float32, round to nearest, ties to even; overflow to infinity, gradual underflow.
__device__ __forceinline__ float f64_to_f32_rn_bits(double x) {
  const uint64_t B = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(B >> 63) << 31;
  const int E = (int)((B >> 52) & 0x7FF);
  const uint64_t M = B & kMant52;
  if (E == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (M ? (0x400000u | (uint32_t)(M >> 29)) : 0u));
  const int e32 = E - 896;
  if (e32 >= 255) return __uint_as_float(sign | 0x7F800000u);
  if (e32 >= 1) {
    uint32_t q = ((uint32_t)e32 << 23) | (uint32_t)(M >> 29);
    const uint32_t rem = (uint32_t)(M & ((1u << 29) - 1u));
    if (rem > (1u << 28) || (rem == (1u << 28) && (q & 1u))) ++q;  // a carry moves into the exponent
    return __uint_as_float(sign | q);
  }
  // float32 subnormal or zero: value = (2^52 + M) 2^(E-1075) = q 2^-149 with q = Mf >> shift
  if (E == 0) return __uint_as_float(sign);  // float64 subnormals are far below float32's range
  const int shift = 30 - e32;                // 29 + (1 - e32), >= 30
  if (shift >= 54) return __uint_as_float(sign);
  const uint64_t Mf = M | (1ull << 52);
  uint32_t q = (uint32_t)(Mf >> shift);
  const uint64_t rem = Mf & ((1ull << shift) - 1ull);
  const uint64_t half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (q & 1u))) ++q;  // may become the smallest normal: still right
  return __uint_as_float(sign | q);
}

// Signed significand of a finite normal float64 with biased exponent E, scaled by 2^(E - Emin).
__device__ __forceinline__ int64_t aligned_sig(uint64_t bits, int E, int Emin) {
  const int64_t m = (int64_t)(((bits & kMant52) | (1ull << 52)) << (E - Emin));
  return (bits >> 63) ? -m : m;
}

// The float64 nearest (ties to even) to S 2^(E - 1075), i.e. S units of the last place of a float64
// of biased exponent E. Returns false when the result is not a normal float64 (or zero).
__device__ __forceinline__ bool fixed_to_f64(int64_t S, int E, double* out) {
  if (S == 0) {
    *out = 0.0;
    return true;
  }
  const uint64_t neg = S < 0 ? 1ull : 0ull;
  const uint64_t A = neg ? (uint64_t)(-S) : (uint64_t)S;
  const int p = 63 - __clzll((long long)A);
  uint64_t q;
  int ef;  // biased exponent of the result
  if (p <= 52) {
    q = A << (52 - p);
    ef = E + p - 52;
  } else {
    int sh = p - 52;
    q = A >> sh;
    const uint64_t rem = A & ((1ull << sh) - 1ull);
    const uint64_t half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) {
      ++q;
      if (q == (1ull << 53)) {
        q >>= 1;
        ++sh;
      }
    }
    ef = E + sh;
  }
  if ((unsigned)(ef - 1) >= 2046u) return false;
  *out = __longlong_as_double((long long)((neg << 63) | ((uint64_t)ef << 52) | (q & kMant52)));
  return true;
}

// fixed_to_f64 for |S| < 2^53, where the conversion is exact (no rounding step).
__device__ __forceinline__ bool fixed_to_f64_small(int64_t S, int E, double* out) {
  const uint64_t neg = S < 0 ? 1ull : 0ull;
  const uint64_t A = neg ? (uint64_t)(-S) : (uint64_t)S;
  const int p = 63 - __clzll((long long)A);
  const int ef = E + p - 52;
  const uint64_t bits = (neg << 63) | ((uint64_t)ef << 52) | ((A << (52 - p)) & kMant52);
  *out = S == 0 ? 0.0 : __longlong_as_double((long long)bits);
  return S == 0 || (unsigned)(ef - 1) < 2046u;
}

// f64_to_f32_rn_bits for a finite x whose float32 result is normal or rounds up to infinity
// (biased float64 exponent 897..1150).
__device__ __forceinline__ float f64_to_f32_rn_normal(double x) {
  const uint64_t B = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(B >> 32), lo = (uint32_t)B;
  // hi:lo shifted left by 3: bits 31..23 hold the low 9 bits of the float64 exponent E, bits 22..0
  // the top 23 significand bits. E - 896 lies in 1..254, and its low 8 bits are those of E plus 128.
  const uint32_t w = __funnelshift_l(lo, hi, 3);
  const uint32_t q = ((w + 0x40000000u) & 0x7FFFFFFFu) | (hi & 0x80000000u);
  // round to nearest even on the 29 dropped bits: +1 iff rem > 2^28, or rem == 2^28 and q is odd
  return __uint_as_float(q + (((lo & 0x1FFFFFFFu) + (w & 1u) + 0x0FFFFFFFu) >> 29));
}

// True if f64_to_f32_rn_normal applies to x.
__device__ __forceinline__ bool f32_normal_range(double x) {
  const uint32_t a = (uint32_t)((uint64_t)__double_as_longlong(x) >> 32) & 0x7FFFFFFFu;
  return a - (897u << 20) < (254u << 20);
}

// Largest exponent spread handled exactly: significands < 2^58, at most 6 neighbours plus M <= 9
// times the centre keep |S| < 2^62.
constexpr int kMaxExpSpread = 5;

// S = sum over the present neighbours of u_nb - M u_c, rounded once to float64 (round to nearest
// even) from its exact value. nb[k] are the neighbours' bit patterns, present bit k of `mask`.
// Returns false (S not computed) when a value is zero, subnormal, infinite or NaN, when the
// exponents in the stencil span more than kMaxExpSpread, or when S rounds outside the normal
// float64 range; the caller then evaluates the point equation in float64 arithmetic.
template <int NB>
__device__ __forceinline__ bool stencil_diff_exact(uint64_t c, const uint64_t (&nb)[NB], unsigned mask, int M,
                                                   double* out) {
  const int Ec = (int)((c >> 52) & 0x7FF);
  bool ok = (unsigned)(Ec - 1) < 2046u;
  int Emin = Ec, Emax = Ec;
  int E[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    E[k] = (int)((nb[k] >> 52) & 0x7FF);
    if ((mask >> k) & 1u) {
      ok = ok && (unsigned)(E[k] - 1) < 2046u;
      Emin = min(Emin, E[k]);
      Emax = max(Emax, E[k]);
    }
  }
  if (!ok || Emax - Emin > kMaxExpSpread) return false;
  int64_t S = -(int64_t)M * aligned_sig(c, Ec, Emin);
#pragma unroll
  for (int k = 0; k < NB; ++k)
    if ((mask >> k) & 1u) S += aligned_sig(nb[k], E[k], Emin);
  return fixed_to_f64(S, Emin, out);
}

}  // namespace fasmg
