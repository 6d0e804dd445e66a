// The non-physical-state check and the characteristic speeds of one Euler
// state, shared by every kernel that takes the Lax-Friedrichs alpha (Sec. 2:
// the maximum of |f'(u)| over the mesh): the state set by the caller, the
// last Runge-Kutta stage of each step, and the batched kernel.  One set of
// operations everywhere, so a run restarted from a saved state takes the
// same alpha as the uninterrupted run, bit for bit.
#pragma once

#include <cuda_runtime.h>

namespace enoao {

// Conversions between FP64 and FP32 on the integer units.  The hardware
// conversion instructions issue to the FP64 unit, which the FP32 bulk path
// otherwise leaves to the state update; these give the same bits for every
// value of normal FP32 magnitude.
// f32_rn: round to nearest even at mantissa bit 29 (the carry runs into the
// exponent); magnitudes below the smallest normal float give a signed zero,
// magnitudes from 2^128 up, infinities and NaN give NaN.
__device__ __forceinline__ float f32_rn(double x) {
  const unsigned lo = __double2loint(x), hi = __double2hiint(x);
  const unsigned long long b =
      ((static_cast<unsigned long long>(hi) << 32) | lo) + (0x0FFFFFFFull + ((lo >> 29) & 1u));
  unsigned r = static_cast<unsigned>(b >> 29) - (896u << 23);  // exponent bias 1023 -> 127
  r = (r & 0x7FFFFFFFu) | (hi & 0x80000000u);
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (e - 897u > 253u) r = e < 897u ? (hi & 0x80000000u) : 0x7FC00000u;
  return __uint_as_float(r);
}
// f64_of: exact widening; zero and subnormal floats give a signed zero,
// infinities and NaN give NaN.
__device__ __forceinline__ double f64_of(float x) {
  const unsigned u = __float_as_uint(x), a = u & 0x7FFFFFFFu;
  unsigned hi = (a >> 3) + (896u << 20), lo = u << 29;  // exponent bias 127 -> 1023
  if (a < 0x00800000u) hi = lo = 0u;
  if (a >= 0x7F800000u) hi = 0x7FF80000u, lo = 0u;
  return __hiloint2double(static_cast<int>(hi | (u & 0x80000000u)), static_cast<int>(lo));
}

// Speeds of one state u = (rho, m_1..m_{NV-2}, E) in conserved order: per axis
// d, s[d] = |u_d| + c, or with FIELD s[3 d + 0..2] = |u_d - c|, |u_d|,
// |u_d + c| (the constants of the per-field splitting).  Returns false for a
// non-physical state (rho <= 0, p <= 0 or NaN), leaving s untouched.
// FP64 arithmetic (the FP64 path, and the per-stage alphas of both paths).
template <int NV, bool FIELD>
__device__ __forceinline__ bool speeds64(const double (&u)[NV], double gamma,
                                         double (&s)[FIELD ? 9 : 3]) {
  const double rho = u[0], ir = 1.0 / rho;
  double m2 = 0.0;
#pragma unroll
  for (int c = 1; c < NV - 1; ++c) m2 += u[c] * u[c];
  const double p = (gamma - 1.0) * (u[NV - 1] - 0.5 * m2 * ir);
  if (!(rho > 0.0 && p > 0.0 && isfinite(p))) return false;
  const double cs = sqrt(gamma * p * ir);
#pragma unroll
  for (int d = 0; d < NV - 2; ++d) {
    if constexpr (FIELD) {
      const double v = u[1 + d] * ir;
      s[3 * d] = fabs(v - cs);
      s[3 * d + 1] = fabs(v);
      s[3 * d + 2] = fabs(v + cs);
    } else {
      s[d] = fabs(u[1 + d]) * ir + cs;
    }
  }
  return true;
}

// The same in the FP32 bulk arithmetic (the U^n alpha of FP32 bulk steps):
// density, momenta, kinetic energy, pressure and sound speed in FP32; only
// the energy difference E - ke stays FP64.
template <int NV, bool FIELD>
__device__ __forceinline__ bool speeds32(const double (&u)[NV], double gamma,
                                         double (&s)[FIELD ? 9 : 3]) {
  const float rho = f32_rn(u[0]);
  float m2 = 0.0f;
#pragma unroll
  for (int c = 1; c < NV - 1; ++c) {
    const float m = f32_rn(u[c]);
    m2 += m * m;
  }
  const float ke = __fdividef(0.5f * m2, rho);
  const float p = f32_rn((gamma - 1.0) * (u[NV - 1] - f64_of(ke)));
  if (!(rho > 0.0f && p > 0.0f && isfinite(p))) return false;
  const float ir = __fdividef(1.0f, rho);
  const float cs = sqrtf(f32_rn(gamma) * p * ir);
#pragma unroll
  for (int d = 0; d < NV - 2; ++d) {
    if constexpr (FIELD) {
      const float v = f32_rn(u[1 + d]) * ir;
      s[3 * d] = f64_of(fabsf(v - cs));
      s[3 * d + 1] = f64_of(fabsf(v));
      s[3 * d + 2] = f64_of(fabsf(v + cs));
    } else {
      s[d] = f64_of(fabsf(f32_rn(u[1 + d])) * ir + cs);
    }
  }
  return true;
}

}  // namespace enoao
