// Fused ENO-AO sweep kernel: one launch performs, for one axis and one
// Runge-Kutta stage, every step of the spatial operator of Shen's ENO-AO
// scheme (arXiv 2108.12742) and, on the last axis, the Runge-Kutta combine.
//
// Per tile (TA lines x TS cells along the swept axis, plus a halo of G cells
// on each side, G = 4 for ENO-AO5 and 5 for ENO-AO7):
//   phase 1  per pair of neighbouring cells: state difference dU (FP64),
//            flux difference dF in difference form, Lax-Friedrichs split
//            differences df+- = (dF +- alpha dU)/2 (Sec. 2, Eq. LF_Flux_Split);
//            per cell: Roe-average ingredients (sqrt rho, velocity, H).
//   phase 2  per face x_{j+1/2}: Roe average and eigenvectors (Sec. 4),
//            projection of the window differences onto each characteristic
//            field, indicators IS = MIN(delta_L, delta_R) as undivided
//            differences (Eq. New_Smoothness_Indicator, Tables 4-5), stencil
//            choice by the principle of Sec. 3.2 (ties to the higher
//            priority as in Appendix A), the chosen Table-1 value written as
//            f_j + sum_i b_i (f_{i+1} - f_i), the mirrored choice for f^-, and
//            the back-projection C_{j+1/2} = R (corr^+ + corr^-).
//   phase 3  per cell: L(u)_j = -(df+_{j-1} + df-_j + C_{j+1/2} - C_{j-1/2})/dx,
//            which equals -(F_{j+1/2} - F_{j-1/2})/dx of Eq. (1DWENOFD) because
//            F_{j+1/2} = f+_j + f-_{j+1} + C_{j+1/2}; then either store L(u)
//            for the next axis or add the earlier axes and apply the
//            third-order TVD Runge-Kutta combine in FP64, checking the new
//            state and accumulating the next step's alpha.
//
// Writing every quantity as a difference keeps FP32 rounding relative to the
// local variation |df| instead of |f|; the state and the combine stay FP64.
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "enoao_internal.h"
#include "state_speed.cuh"
#include "tma.cuh"

namespace enoao {

template <int ORDER>
struct Geo {
  static constexpr int G = ORDER / 2 + 2;       // halo cells per side
  static constexpr int NC = ORDER == 7 ? 9 : 6; // candidates
  static constexpr int LO = ORDER == 7 ? 0 : 1; // used window differences d[LO..HI]
  static constexpr int HI = ORDER == 7 ? 7 : 6;
};

// Chosen value minus the centre value, f^ - f_j = sum_i B[c][i] d[i], for the
// nine candidates in priority order, with d[i] = f_{j+i-3} - f_{j+i-4}
// (Table 1 rewritten in first differences).
__constant__ double kB64[9][8] = {
    {0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 1.0 / 2, 0, 0, 0},
    {0, 0, 0, 1.0 / 6, 1.0 / 3, 0, 0, 0},
    {0, 0, -1.0 / 12, 1.0 / 3, 1.0 / 4, 0, 0, 0},
    {0, 0, 0, 1.0 / 12, 1.0 / 2, -1.0 / 12, 0, 0},
    {0, 0, -1.0 / 30, 11.0 / 60, 2.0 / 5, -1.0 / 20, 0, 0},
    {0, 1.0 / 60, -1.0 / 10, 17.0 / 60, 1.0 / 3, -1.0 / 30, 0, 0},
    {0, 0, -1.0 / 60, 7.0 / 60, 1.0 / 2, -7.0 / 60, 1.0 / 60, 0},
    {0, 1.0 / 140, -11.0 / 210, 79.0 / 420, 3.0 / 7, -17.0 / 210, 1.0 / 105, 0},
};
__constant__ float kB32[9][8] = {
    {0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 1.0f / 2, 0, 0, 0},
    {0, 0, 0, 1.0f / 6, 1.0f / 3, 0, 0, 0},
    {0, 0, -1.0f / 12, 1.0f / 3, 1.0f / 4, 0, 0, 0},
    {0, 0, 0, 1.0f / 12, 1.0f / 2, -1.0f / 12, 0, 0},
    {0, 0, -1.0f / 30, 11.0f / 60, 2.0f / 5, -1.0f / 20, 0, 0},
    {0, 1.0f / 60, -1.0f / 10, 17.0f / 60, 1.0f / 3, -1.0f / 30, 0, 0},
    {0, 0, -1.0f / 60, 7.0f / 60, 1.0f / 2, -7.0f / 60, 1.0f / 60, 0},
    {0, 1.0f / 140, -11.0f / 210, 79.0f / 420, 3.0f / 7, -17.0f / 210, 1.0f / 105, 0},
};

template <typename R>
__device__ __forceinline__ R bcoef(int c, int i);
template <>
__device__ __forceinline__ double bcoef<double>(int c, int i) { return kB64[c][i]; }
template <>
__device__ __forceinline__ float bcoef<float>(int c, int i) { return kB32[c][i]; }

// Coefficient i of the top candidate (S_{j-2}^{j+2} of ENO-AO5, S_{j-3}^{j+3}
// of ENO-AO7), the same values as its row of kB32 / kB64, as immediates.
template <int ORDER, typename R>
__device__ __forceinline__ R bcoef_top(int i) {
  if constexpr (ORDER == 5) {
    constexpr R b[8] = {R(0), R(0), R(-1) / R(30), R(11) / R(60), R(2) / R(5), R(-1) / R(20), R(0),
                        R(0)};
    return b[i];
  } else {
    constexpr R b[8] = {R(0),         R(1) / R(140), R(-11) / R(210), R(79) / R(420),
                        R(3) / R(7), R(-17) / R(210), R(1) / R(105),  R(0)};
    return b[i];
  }
}

// Square root in the bulk precision (an unqualified sqrt on a float can
// resolve to the double routine, which runs on the slow FP64 unit).
__device__ __forceinline__ double bsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float bsqrt(float a) { return sqrtf(a); }
// Reciprocal and quotient in the bulk precision.  FP64 keeps correctly
// rounded division (parity with the FP64 oracle); the FP32 bulk path uses the
// fast hardware reciprocal (error of a few ulp, far inside the FP32-bulk
// tolerance) -- correctly rounded FP32 division is a long routine.
__device__ __forceinline__ double brcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float brcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double bdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float bdiv(float a, float b) { return __fdividef(a, b); }
// Absolute value (a sign-bit operation, no floating-point instruction).
__device__ __forceinline__ double rabs(double a) { return fabs(a); }
__device__ __forceinline__ float rabs(float a) { return fabsf(a); }
// Order key of a non-negative value: for doubles the bit pattern read as an
// integer orders exactly like the value (NaN above everything), so indicator
// comparisons and minima run on the integer units instead of the FP64 unit,
// which is 1/64 of the FP32 rate on this part.
__device__ __forceinline__ long long okey(double a) { return __double_as_longlong(a); }
__device__ __forceinline__ float okey(float a) { return a; }
template <typename R>
__device__ __forceinline__ R rmin(R a, R b) { return okey(a) < okey(b) ? a : b; }

// Narrowing of a phase-1 input (an FP64 state component or the difference of
// two) to FP32 in six integer operations: the exponent word is clamped at the
// smallest normal FP32 exponent (so zero needs no branch), half an FP32 ulp
// is added at mantissa bit 28 with the carry running into the exponent, and
// the word is shifted into place with the exponent rebased from 1023 to 127.
// Round to nearest for every magnitude in [2^-126, 2^128) (an exact tie
// rounds away from zero); zero keeps its sign; a magnitude below 2^-126 gives
// one below 2^-126.  Magnitudes of 2^128 and more are out of range: a state
// that large fails the state check of its step, which narrows with f32_rn.
// The hardware conversion issues to the FP64 unit and is slower here.
__device__ __forceinline__ float f32_near(double x) {
  const unsigned lo = __double2loint(x), hi = __double2hiint(x);
  const unsigned hc = max(hi & 0x7FFFFFFFu, 896u << 20);
  const unsigned long long w =
      ((static_cast<unsigned long long>(hc - (896u << 20)) << 32) | lo) + 0x10000000ull;
  return __uint_as_float(static_cast<unsigned>(w >> 29) | (hi & 0x80000000u));
}

// FP64 value in the bulk precision, and a bulk value widened to FP64.
template <typename R>
__device__ __forceinline__ R to_bulk(double x);
template <>
__device__ __forceinline__ double to_bulk<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_bulk<float>(double x) { return f32_near(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f64_of(x); }
// A constant of the sweep in the bulk precision: the FP64 argument, or its
// FP32 copy set on the host (SweepArgs, set_derived_constants).
template <typename R>
__device__ __forceinline__ R bconst(double d, float f);
template <>
__device__ __forceinline__ double bconst<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float bconst<float>(double, float f) { return f; }

// ENO-AO choice on one window of first differences d[LO..HI] (d[i] between
// offsets i-4 and i-3 of the centre cell).  Returns f^ - f_centre.  When
// CHECK is set, 'marginal' reports a decision that rounding of size tol_abs
// or a relative gap tie_rel could have changed.
// Rounding bound of the FP32 bulk indicators.  e[i] = sum_c |L_c| |df_c| is the
// magnitude of the terms whose FP32 sum gave d[i], so d[i] carries an error of
// at most feps * e[i] (feps = (NV + 8) eps32 covers the projection sum and the
// flux difference behind it).  An undivided difference of d sums its inputs
// with binomial weights, so the same Pascal sums of e bound its error; IS_c,
// the smaller of two such differences, is off by at most the larger bound.
template <int ORDER, typename R, bool CHECK>
__device__ __forceinline__ R eno_select(const R (&d)[8], R delta, R tie_rel, const R (&e)[8],
                                        R feps, int& pick_out, bool& marginal) {
  using GE = Geo<ORDER>;
  constexpr int LO = GE::LO, HI = GE::HI, NC = GE::NC;
  // Principle 1 first for the top candidate (highest priority): at or below
  // delta it is the pick whatever the other indicators are -- the smooth
  // case, most windows -- and only its indicator, its rounding bound and its
  // Table-1 value (compile-time coefficients) are needed.  Its two undivided
  // differences of order 5 (7) are formed directly with their binomial
  // weights; the difference table of the other candidates is built only when
  // the top one is above delta.
  const auto kdelta = okey(delta);
  R IS_top;
  if constexpr (ORDER == 7) {
    auto b6 = [&](int o) {  // sum_k (-1)^k C(6,k) d[o+k]
      R t = d[o] + d[o + 6];
      t = fma(R(-6), d[o + 1] + d[o + 5], t);
      t = fma(R(15), d[o + 2] + d[o + 4], t);
      return fma(R(-20), d[o + 3], t);
    };
    IS_top = rmin(rabs(b6(0)), rabs(b6(1)));
  } else {
    auto b4 = [&](int o) {  // sum_k (-1)^k C(4,k) d[o+k]
      R t = d[o] + d[o + 4];
      t = fma(R(-4), d[o + 1] + d[o + 3], t);
      return fma(R(6), d[o + 2], t);
    };
    IS_top = rmin(rabs(b4(1)), rabs(b4(2)));
  }
  int pick;
  R corr = R(0);
  if (okey(IS_top) <= kdelta) {
    pick = NC - 1;
    // its nonzero coefficients: d[2..5] (ENO-AO5), d[1..6] (ENO-AO7)
#pragma unroll
    for (int i = ORDER == 5 ? 2 : 1; i <= (ORDER == 5 ? 5 : 6); ++i)
      corr += bcoef_top<ORDER, R>(i) * d[i];
    if constexpr (CHECK) {
      // its bound: the Pascal sums of e over its two differences, written out
      R qa, qb;
      if constexpr (ORDER == 7) {
        qa = e[0] + e[6] + R(6) * (e[1] + e[5]) + R(15) * (e[2] + e[4]) + R(20) * e[3];
        qb = e[1] + e[7] + R(6) * (e[2] + e[6]) + R(15) * (e[3] + e[5]) + R(20) * e[4];
      } else {
        qa = e[1] + e[5] + R(4) * (e[2] + e[4]) + R(6) * e[3];
        qb = e[2] + e[6] + R(4) * (e[3] + e[5]) + R(6) * e[4];
      }
      marginal = rabs(IS_top - delta) <= tie_rel * delta + feps * fmaxf(qa, qb);
    }
  } else {
    R s2[8], s3[8], s4[8], s5[8], s6[8];
#pragma unroll
    for (int i = LO; i < HI; ++i) s2[i] = d[i + 1] - d[i];
#pragma unroll
    for (int i = LO; i < HI - 1; ++i) s3[i] = s2[i + 1] - s2[i];
#pragma unroll
    for (int i = LO; i < HI - 2; ++i) s4[i] = s3[i + 1] - s3[i];
#pragma unroll
    for (int i = LO; i < HI - 3; ++i) s5[i] = s4[i + 1] - s4[i];
    if constexpr (ORDER == 7) {
#pragma unroll
      for (int i = 0; i < 3; ++i) s6[i] = s5[i + 1] - s5[i];
    }
    R IS[9];
    // min(a/2, b/2) = min(a, b)/2 exactly (scaling by a power of two)
    IS[0] = R(0.5) * rmin(rabs(d[3]) + rabs(d[2]), rabs(d[4]) + rabs(d[5]));
    IS[1] = rmin(rabs(s2[3]), rabs(s2[4]));
    IS[2] = rmin(rabs(s3[2]), rabs(s3[3]));
    IS[3] = rmin(rabs(s4[1]), rabs(s4[2]));
    IS[4] = rmin(rabs(s4[2]), rabs(s4[3]));
    if constexpr (ORDER == 7) {
      IS[5] = rmin(rabs(s5[1]), rabs(s5[2]));
      IS[6] = rmin(rabs(s6[0]), rabs(s6[1]));
      IS[7] = rmin(rabs(s6[1]), rabs(s6[2]));
    }
    IS[NC - 1] = IS_top;
    // Principle 1 over the others (the top is above delta here).
    pick = -1;
#pragma unroll
    for (int c = 0; c < NC - 1; ++c)
      if (okey(IS[c]) <= kdelta) pick = c;
    const bool thr = pick >= 0;
    // Principle 2: otherwise the smallest IS, equal values to the higher priority.
    R best = IS[0];
    if (!thr) {
      pick = 0;
#pragma unroll
      for (int c = 1; c < NC; ++c)
        if (okey(IS[c]) <= okey(best)) {
          best = IS[c];
          pick = c;
        }
    }
    if constexpr (CHECK) {
      const R rel = tie_rel * delta;
      bool m = false;
      // per-candidate bounds: Pascal sums of e over each indicator's differences
      R q2[8], q3[8], q4[8], q5[8], q6[8], q7[8];
#pragma unroll
      for (int i = LO; i < HI; ++i) q2[i] = e[i] + e[i + 1];
#pragma unroll
      for (int i = LO; i < HI - 1; ++i) q3[i] = q2[i] + q2[i + 1];
#pragma unroll
      for (int i = LO; i < HI - 2; ++i) q4[i] = q3[i] + q3[i + 1];
#pragma unroll
      for (int i = LO; i < HI - 3; ++i) q5[i] = q4[i] + q4[i + 1];
      R tol[9];
      tol[0] = feps * R(0.5) * fmaxf(e[3] + e[2], e[4] + e[5]);
      tol[1] = feps * fmaxf(q2[3], q2[4]);
      tol[2] = feps * fmaxf(q3[2], q3[3]);
      tol[3] = feps * fmaxf(q4[1], q4[2]);
      tol[4] = feps * fmaxf(q4[2], q4[3]);
      tol[5] = feps * fmaxf(q5[1], q5[2]);
      if constexpr (ORDER == 7) {
#pragma unroll
        for (int i = 0; i < 3; ++i) q6[i] = q5[i] + q5[i + 1];
#pragma unroll
        for (int i = 0; i < 2; ++i) q7[i] = q6[i] + q6[i + 1];
        tol[6] = feps * fmaxf(q6[0], q6[1]);
        tol[7] = feps * fmaxf(q6[1], q6[2]);
        tol[8] = feps * fmaxf(q7[0], q7[1]);
      }
      if (thr) {
#pragma unroll
        for (int c = 0; c < NC; ++c) m |= (c >= pick) && (rabs(IS[c] - delta) <= rel + tol[c]);
      } else {
        R tp = tol[0];
#pragma unroll
        for (int c = 1; c < NC; ++c)
          if (c == pick) tp = tol[c];
        m = (best - delta) <= rel + tp;
        const R relA = tie_rel * best + tp;
        // Candidates 3 and 4 (and 6 and 7 of ENO-AO7) take the minimum over
        // two differences of which they share the middle one, b: with
        // IS_lo = min(a, b) and IS_hi = min(b, c), IS_lo wins exactly when
        // a < b and a < c, so the margin of the pair is max(a - b, a - c), not
        // IS_lo - IS_hi (which is zero whenever b is the smaller of both).
        R gap[9];
#pragma unroll
        for (int c = 0; c < NC; ++c) gap[c] = IS[c] - best;
        if (pick == 4) {
          const R a = rabs(s4[1]), b = rabs(s4[2]), c = rabs(s4[3]);
          gap[3] = fmaxf(a - b, a - c);
        }
        if constexpr (ORDER == 7) {
          if (pick == 7) {
            const R a = rabs(s6[0]), b = rabs(s6[1]), c = rabs(s6[2]);
            gap[6] = fmaxf(a - b, a - c);
          }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) m |= (c != pick) && (gap[c] <= relA + tol[c]);
      }
      marginal = m;
    }
#pragma unroll
    for (int i = LO; i <= HI; ++i) corr += bcoef<R>(pick, i) * d[i];
  }
  pick_out = pick;
  return corr;
}

// Conserved component stored at position c of the permuted state for a sweep
// along axis dir (momentum along dir first, tangential momenta cyclic).
template <int NV>
__device__ __forceinline__ int perm_comp(int c, int dir) {
  if (NV == 1 || c == 0 || c == NV - 1) return c;
  constexpr int ND = NV > 2 ? NV - 2 : 1;
  return 1 + (dir + c - 1) % ND;
}

// Conserved component k of a state held in permuted order, by selects (an
// index computed from the runtime axis would put the array in local memory).
template <int NV, typename T>
__device__ __forceinline__ T comp_of(const T (&up)[NV], int k, int dir) {
  if constexpr (NV < 3) {
    return up[k];
  } else {
    if (k == 0 || k == NV - 1) return up[k];
    T r = up[1];
#pragma unroll
    for (int c = 2; c < NV - 1; ++c) r = perm_comp<NV>(c, dir) == k ? up[c] : r;
    return r;
  }
}

// Flux difference F(qb) - F(qa) along the sweep axis, written in differences
// so that rounding scales with |dq| (Euler: F = [m, m u + p, m_t u, (E+p) u]).
template <int NV, typename T>
__device__ __forceinline__ void flux_diff(const T (&qa)[NV], const T (&qb)[NV], const T (&dq)[NV],
                                          T gm1, T adv, T (&dF)[NV]) {
  if constexpr (NV == 1) {
    dF[0] = adv * dq[0];
  } else {
    constexpr int NT = NV - 3;  // tangential components
    const T ia = brcp(qa[0]);
    const T ib = brcp(qb[0]);
    const T u = qa[1] * ia;
    T vt[NT > 0 ? NT : 1], dvt[NT > 0 ? NT : 1];
    const T du = (dq[1] - u * dq[0]) * ib;
    T v2 = u * u, vdv = u * du, dv2 = du * du;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      vt[t] = qa[2 + t] * ia;
      dvt[t] = (dq[2 + t] - vt[t] * dq[0]) * ib;
      v2 += vt[t] * vt[t];
      vdv += vt[t] * dvt[t];
      dv2 += dvt[t] * dvt[t];
    }
    const T ke_a = T(0.5) * qa[0] * v2;
    const T dke = T(0.5) * dq[0] * v2 + qb[0] * (vdv + T(0.5) * dv2);
    const T pa = gm1 * (qa[NV - 1] - ke_a);
    const T dp = gm1 * (dq[NV - 1] - dke);
    const T ub = u + du;
    dF[0] = dq[1];
    dF[1] = dq[1] * ub + qa[1] * du + dp;
#pragma unroll
    for (int t = 0; t < NT; ++t) dF[2 + t] = dq[2 + t] * ub + qa[2 + t] * du;
    dF[NV - 1] = (dq[NV - 1] + dp) * ub + (qa[NV - 1] + pa) * du;
  }
}

// Physical flux of a permuted state (used only for interface-flux output).
template <int NV>
__device__ __forceinline__ void phys_flux(const double (&q)[NV], double gm1, double adv,
                                          double (&F)[NV]) {
  if constexpr (NV == 1) {
    F[0] = adv * q[0];
  } else {
    double ke = 0.0;
#pragma unroll
    for (int i = 1; i < NV - 1; ++i) ke += q[i] * q[i];
    ke = 0.5 * ke / q[0];
    const double p = gm1 * (q[NV - 1] - ke);
    const double un = q[1] / q[0];
    F[0] = q[1];
    F[1] = q[1] * un + p;
#pragma unroll
    for (int i = 2; i < NV - 1; ++i) F[i] = q[i] * un;
    F[NV - 1] = (q[NV - 1] + p) * un;
  }
}

// Roe-average ingredients of one cell: sqrt(rho), velocity, total enthalpy.
template <int NV, typename T>
__device__ __forceinline__ void roe_prims(const T (&q)[NV], T gm1, T (&pr)[NV]) {
  if constexpr (NV > 1) {
    const T ir = brcp(q[0]);
    T ke = T(0);
#pragma unroll
    for (int i = 1; i < NV - 1; ++i) {
      pr[i] = q[i] * ir;
      ke += q[i] * pr[i];
    }
    const T p = gm1 * (q[NV - 1] - T(0.5) * ke);
    pr[0] = bsqrt(q[0]);
    pr[NV - 1] = (q[NV - 1] + p) * ir;
  }
}

// Eigen-system of the Euler flux Jacobian at the Roe state of a face.
template <int NV, typename T>
struct Eigen {
  T u, vt[NV > 3 ? NV - 3 : 1], H, c, ic, b1, b2, q2;
};

template <int NV, typename T>
__device__ __forceinline__ void roe_eigen(const T (&pl)[NV], const T (&prr)[NV], T gm1,
                                          Eigen<NV, T>& E) {
  constexpr int NT = NV - 3;
  const T inv = brcp(pl[0] + prr[0]);
  const T wl = pl[0] * inv, wr = prr[0] * inv;
  E.u = wl * pl[1] + wr * prr[1];
  T q2 = E.u * E.u;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    E.vt[t] = wl * pl[2 + t] + wr * prr[2 + t];
    q2 += E.vt[t] * E.vt[t];
  }
  E.H = wl * pl[NV - 1] + wr * prr[NV - 1];
  E.q2 = q2;
  const T c2 = gm1 * (E.H - T(0.5) * q2);
  E.c = bsqrt(c2);
  E.ic = brcp(E.c);
  E.b1 = bdiv(gm1, c2);
  E.b2 = T(0.5) * q2 * E.b1;
}

// The constant c ? 1 : 0 (and c ? 1 : -1) by an integer select: a
// floating-point select of constants can become a conversion instruction,
// which issues to the FP64 unit.
template <typename T>
__device__ __forceinline__ T one_if(bool c) {
  if constexpr (sizeof(T) == 4) return __int_as_float(c ? 0x3f800000 : 0);
  return c ? T(1) : T(0);
}
template <typename T>
__device__ __forceinline__ T sign_if(bool c) {
  if constexpr (sizeof(T) == 4) return __int_as_float(c ? 0x3f800000 : (int)0xbf800000u);
  return c ? T(1) : T(-1);
}

// Row v of L = R^{-1}; fields ordered (u-c, entropy, shear..., u+c).
template <int NV, typename T>
__device__ __forceinline__ void left_row(const Eigen<NV, T>& E, int v, T (&L)[NV]) {
  constexpr int NT = NV - 3;
  if (v == 0 || v == NV - 1) {
    const T s = sign_if<T>(v == 0);
    L[0] = T(0.5) * (E.b2 + s * E.u * E.ic);
    L[1] = T(0.5) * (-E.b1 * E.u - s * E.ic);
#pragma unroll
    for (int t = 0; t < NT; ++t) L[2 + t] = T(-0.5) * E.b1 * E.vt[t];
    L[NV - 1] = T(0.5) * E.b1;
  } else if (v == 1) {
    L[0] = T(1) - E.b2;
    L[1] = E.b1 * E.u;
#pragma unroll
    for (int t = 0; t < NT; ++t) L[2 + t] = E.b1 * E.vt[t];
    L[NV - 1] = -E.b1;
  } else {
    // shear field v: selects instead of indexing by v, so that L, E stay
    // in registers when the caller loops over v without unrolling
    T w = E.vt[0];
#pragma unroll
    for (int t = 1; t < NT; ++t) w = v - 2 == t ? E.vt[t] : w;
#pragma unroll
    for (int i = 1; i < NV; ++i) L[i] = one_if<T>(i == v);
    L[0] = -w;
  }
}

// Component v (a shear field, 2 <= v <= NV - 2) of a permuted vector, by
// selects so that the vector stays in registers.
template <int NV, typename T>
__device__ __forceinline__ T shear_comp(const T (&x)[NV], int v) {
  static_assert(NV >= 4, "shear fields exist for NV >= 4");
  T r = x[2];
#pragma unroll
  for (int c = 3; c < NV - 1; ++c) r = v == c ? x[c] : r;
  return r;
}

// Column v of R.
template <int NV, typename T>
__device__ __forceinline__ void right_col(const Eigen<NV, T>& E, int v, T (&Rc)[NV]) {
  constexpr int NT = NV - 3;
  if (v == 0 || v == NV - 1) {
    const T s = sign_if<T>(v != 0);
    Rc[0] = T(1);
    Rc[1] = E.u + s * E.c;
#pragma unroll
    for (int t = 0; t < NT; ++t) Rc[2 + t] = E.vt[t];
    Rc[NV - 1] = E.H + s * E.u * E.c;
  } else if (v == 1) {
    Rc[0] = T(1);
    Rc[1] = E.u;
#pragma unroll
    for (int t = 0; t < NT; ++t) Rc[2 + t] = E.vt[t];
    Rc[NV - 1] = T(0.5) * E.q2;
  } else {
    T w = E.vt[0];
#pragma unroll
    for (int t = 1; t < NT; ++t) w = v - 2 == t ? E.vt[t] : w;
#pragma unroll
    for (int i = 0; i < NV - 1; ++i) Rc[i] = one_if<T>(i == v);
    Rc[NV - 1] = w;
  }
}

// Ghost-cell map along the swept axis; s lies within one halo width of
// [0, n) (n is at least the halo width), so the periodic wrap is one add or
// subtract -- no integer division, whose 64-bit form runs on the FP64 unit.
// A sub-domain's split axis (kBcHalo) keeps its ghost layers in the arrays,
// next to the interior: positions outside [0, n) are read where they are.
__device__ __forceinline__ long long bc_map(long long s, long long n, int bc) {
  if (bc == 0) return s < 0 ? s + n : (s >= n ? s - n : s);
  if (bc == kBcHalo) return s;
  return s < 0 ? 0 : (s >= n ? n - 1 : s);
}

// Geometry of one tile: cell(a, s) = base + (a0 + a) * stride_a + s * stride_d.
struct TileGeo {
  long long s0, a0, base, stride_a, stride_d, na, nd;
  long long b;                             // index along the remaining axis (dir != 0)
  long long fbase, fstride_a, fstride_d;  // same for the face array (nd + 1 faces)
  int nts;                                 // valid cells of the tile along dir
};

__device__ __forceinline__ TileGeo tile_geo(const SweepArgs& A, long long tile) {
  TileGeo g;
  // tile counts fit 32 bits (checked on the host): 32-bit division only
  const unsigned t32 = (unsigned)tile, tsn = (unsigned)A.tiles_s, tan = (unsigned)A.tiles_a;
  const unsigned rest32 = t32 / tsn;
  const long long ts_i = t32 - rest32 * tsn;
  const long long b = rest32 / tan;
  const long long ta_i = rest32 - (unsigned)b * tan;
  const long long n0 = A.n[0], n1 = A.n[1], n2 = A.n[2];
  g.s0 = ts_i * A.ts;
  g.a0 = ta_i * A.ta;
  g.b = b;
  if (A.dir == 0) {
    g.nd = n0; g.na = n1 * n2;
    g.base = 0; g.stride_a = n0; g.stride_d = 1;
    g.fbase = 0; g.fstride_a = n0 + 1; g.fstride_d = 1;
  } else if (A.dir == 1) {
    g.nd = n1; g.na = n0;
    g.base = b * n1 * n0; g.stride_a = 1; g.stride_d = n0;
    g.fbase = b * (n1 + 1) * n0; g.fstride_a = 1; g.fstride_d = n0;
  } else {
    g.nd = n2; g.na = n0;
    g.base = b * n0; g.stride_a = 1; g.stride_d = n0 * n1;
    g.fbase = b * n0; g.fstride_a = 1; g.fstride_d = n0 * n1;
  }
  g.base += A.org;  // sub-domains: the interior starts after the low ghost layers
  const long long left = g.nd - g.s0;
  g.nts = (int)(left < A.ts ? left : A.ts);
  return g;
}

// Loads the permuted state of one cell.  COHERENT loads go through L2 (the
// batched kernel reads states it wrote itself); otherwise the read-only
// path is used (a sweep never writes the array it stencils from).
template <int NV, bool COHERENT = false>
__device__ __forceinline__ void load_state(const double* __restrict__ U, long long ncell,
                                           long long cell, int dir, double (&q)[NV]) {
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    const double* p = U + perm_comp<NV>(c, dir) * ncell + cell;
    q[c] = COHERENT ? __ldcg(p) : __ldg(p);
  }
}

// Lane group of W lanes (a power of two, at least the 2G window cells) that
// re-decides one choice in FP64 together: lane r holds window cell r, forms
// difference r with its neighbour's state, and the projected window is then
// gathered by shuffles; every lane of the group returns the same pick.  Groups
// of the same warp work on different choices at the same time, so the FP64
// unit (1/64 of the FP32 rate) runs on full warps instead of single lanes.
template <int NV, int ORDER, bool COHERENT, int W>
__device__ __forceinline__ int redo_group(const SweepArgs& A, const TileGeo& g, int a,
                                          long long sj, int v, int sgn, double alpha, int r) {
  constexpr int G = Geo<ORDER>::G;
  static_assert(W >= 2 * G, "a lane per window cell");
  const unsigned FULL = 0xffffffffu;
  const double gm1 = A.gm1;
  const long long line = g.base + (g.a0 + a) * g.stride_a;
  const int rr = r < 2 * G ? r : 2 * G - 1;
  double q[NV];
  load_state<NV, COHERENT>(A.u_in, A.cstride, line + bc_map(sj - G + 1 + rr, g.nd, A.bc) * g.stride_d,
                           A.dir, q);
  double L[NV];
  if constexpr (NV > 1) {
    double ql[NV], qr[NV], pl[NV], prr[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      ql[c] = __shfl_sync(FULL, q[c], G - 1, W);
      qr[c] = __shfl_sync(FULL, q[c], G, W);
    }
    roe_prims<NV, double>(ql, gm1, pl);
    roe_prims<NV, double>(qr, gm1, prr);
    Eigen<NV, double> E;
    roe_eigen<NV, double>(pl, prr, gm1, E);
    left_row<NV, double>(E, v, L);
  } else {
    L[0] = 1.0;
  }
  double qn[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) qn[c] = __shfl_down_sync(FULL, q[c], 1, W);
  double w = 0.0;
  {
    double dq[NV], dF[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) dq[c] = qn[c] - q[c];
    flux_diff<NV, double>(q, qn, dq, gm1, A.adv_speed, dF);
    const double sa = sgn == 0 ? alpha : -alpha;
#pragma unroll
    for (int c = 0; c < NV; ++c) w += L[c] * (0.5 * (dF[c] + sa * dq[c]));
  }
  // window difference k (between cells k and k+1) sits in group lane k
  double d[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) d[i] = 0.0;
#pragma unroll
  for (int i = Geo<ORDER>::LO; i <= Geo<ORDER>::HI; ++i) {
    const int k = sgn == 0 ? i - 4 + G - 1 : 4 - i + G - 1;
    const double wk = __shfl_sync(FULL, w, k, W);
    d[i] = sgn == 0 ? wk : -wk;
  }
  int pick;
  bool m;
  const double nomx[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  eno_select<ORDER, double, false>(d, A.delta, 0.0, nomx, 0.0, pick, m);
  return pick;
}

// The same FP64 re-decision by one thread alone: it walks the window cell by
// cell (two states live at a time).  Used when a warp has many flagged
// choices at once, so that all lanes work on their own choices in parallel
// instead of the warp serving them a few at a time.
template <int NV, int ORDER, bool COHERENT>
__device__ __forceinline__ int redo_lane(const SweepArgs& A, const TileGeo& g, int a, long long sj,
                                         int v, int sgn, double alpha) {
  using GE = Geo<ORDER>;
  constexpr int G = GE::G;
  const double gm1 = A.gm1;
  const long long line = g.base + (g.a0 + a) * g.stride_a;
  // window cell r (0..2G-1) is cell sj - G + 1 + r of the line; the face lies
  // between cells G-1 and G
  auto load_cell = [&](int r, double (&q)[NV]) {
    load_state<NV, COHERENT>(A.u_in, A.cstride, line + bc_map(sj - G + 1 + r, g.nd, A.bc) * g.stride_d,
                             A.dir, q);
  };
  double L[NV];
  if constexpr (NV > 1) {
    double ql[NV], qr[NV], pl[NV], prr[NV];
    load_cell(G - 1, ql);
    load_cell(G, qr);
    roe_prims<NV, double>(ql, gm1, pl);
    roe_prims<NV, double>(qr, gm1, prr);
    Eigen<NV, double> E;
    roe_eigen<NV, double>(pl, prr, gm1, E);
    left_row<NV, double>(E, v, L);
  } else {
    L[0] = 1.0;
  }
  const double sa = sgn == 0 ? alpha : -alpha;
  // d[i] is difference k = i + G - 5 (sign 0) or G + 3 - i (sign 1, negated),
  // between window cells k and k+1; consecutive i share one cell
  double d[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) d[i] = 0.0;
  double qlo[NV], qhi[NV];
  {
    const int k0 = sgn == 0 ? GE::LO + G - 5 : G + 3 - GE::LO;
    load_cell(k0, qlo);
    load_cell(k0 + 1, qhi);
  }
#pragma unroll
  for (int i = GE::LO; i <= GE::HI; ++i) {
    double dq[NV], dF[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) dq[c] = qhi[c] - qlo[c];
    flux_diff<NV, double>(qlo, qhi, dq, gm1, A.adv_speed, dF);
    double w = 0.0;
#pragma unroll
    for (int c = 0; c < NV; ++c) w += L[c] * (0.5 * (dF[c] + sa * dq[c]));
    d[i] = sgn == 0 ? w : -w;
    if (i < GE::HI) {
      const int k = sgn == 0 ? i + G - 5 : G + 3 - i;
      if (sgn == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) qlo[c] = qhi[c];
        load_cell(k + 2, qhi);
      } else {
#pragma unroll
        for (int c = 0; c < NV; ++c) qhi[c] = qlo[c];
        load_cell(k - 1, qlo);
      }
    }
  }
  int pick;
  bool m;
  const double nomx[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  eno_select<ORDER, double, false>(d, A.delta, 0.0, nomx, 0.0, pick, m);
  return pick;
}

// Position of the n-th (0-based) set bit of x, or -1.
__device__ __forceinline__ int nth_set_bit(unsigned x, int n) {
  for (int i = 0; i < n && x; ++i) x &= x - 1;
  return x ? __ffs(x) - 1 : -1;
}

template <int NV>
struct NPrim {
  static constexpr int value = NV > 1 ? NV : 0;
};

// Runs body(a, e) over the items of a TA x cnt tile.  x sweeps (sfast):
// each thread keeps one line a and strides along e (lanes along the line);
// y/z sweeps: each thread keeps one line a (lanes across lines, i.e. along x)
// and strides along e.  TA is a power of two dividing the block size, so the
// mapping is shifts and masks -- no per-item integer division.
template <typename F>
__device__ __forceinline__ void for_items(int lgTA, int cnt, bool sfast, F&& body) {
  const int bd = blockDim.x, tid = threadIdx.x;
  if (sfast) {
    const int lgTpl = __ffs(bd) - 1 - lgTA;  // threads per line = bd / TA
    const int a = tid >> lgTpl, tpl = 1 << lgTpl;
    for (int e = tid & (tpl - 1); e < cnt; e += tpl) body(a, e);
  } else {
    const int a = tid & ((1 << lgTA) - 1);
    const int step = bd >> lgTA;
    for (int e = tid >> lgTA; e < cnt; e += step) body(a, e);
  }
}

// The mapping of for_items as values: this thread's line a, its first item
// e0 and the stride between its items.
__device__ __forceinline__ void item_start(int lgTA, bool sfast, int& a, int& e0, int& step) {
  const int bd = blockDim.x, tid = threadIdx.x;
  if (sfast) {
    const int lgTpl = __ffs(bd) - 1 - lgTA;
    a = tid >> lgTpl;
    step = 1 << lgTpl;
    e0 = tid & (step - 1);
  } else {
    a = tid & ((1 << lgTA) - 1);
    step = bd >> lgTA;
    e0 = tid >> lgTA;
  }
}

// Per-cell vectors in shared memory.  FP32 four-component states (2D Euler)
// are stored as one float4 per cell, so a cell moves in one 128-bit access;
// every other case keeps one plane per component.  Both layouts take NV
// values of R per cell slot.
template <int NV, typename R>
struct CellVec {
  static constexpr bool kAoS = sizeof(R) == 4 && NV == 4;
  __device__ __forceinline__ static void load(const R* base, int cells, int i, R (&v)[NV]) {
    if constexpr (kAoS) {
      const float4 t = reinterpret_cast<const float4*>(base)[i];
      v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    } else {
#pragma unroll
      for (int c = 0; c < NV; ++c) v[c] = base[c * cells + i];
    }
  }
  __device__ __forceinline__ static void store(R* base, int cells, int i, const R (&v)[NV]) {
    if constexpr (kAoS) {
      reinterpret_cast<float4*>(base)[i] = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int c = 0; c < NV; ++c) base[c * cells + i] = v[c];
    }
  }
};

// Lax-Friedrichs split differences of one pair of neighbouring cells in the
// bulk precision (phase 1): dq = qb - qa rounded once from FP64, the flux
// difference in difference form, and (dF +- alpha dq)/2 written as
// dF/2 +- (alpha/2) dq (the same bits: halving is exact).
template <int NV, typename R>
__device__ __forceinline__ void split_diff(const double (&qa64)[NV], const double (&qb64)[NV],
                                           const R (&qa)[NV], const R (&qb)[NV], R gm1, R adv,
                                           R halpha, R (&fp)[NV], R (&fm)[NV]) {
  R dq[NV], dF[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) dq[c] = to_bulk<R>(qb64[c] - qa64[c]);
  flux_diff<NV, R>(qa, qb, dq, gm1, adv, dF);
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    const R hdF = R(0.5) * dF[c];
    fp[c] = fma(halpha, dq[c], hdF);
    fm[c] = fma(-halpha, dq[c], hdF);
  }
}

// The same pair of cells for per-field splitting: dF/2 and dq/2 (exact
// halvings), to be split per characteristic field after the projection.
template <int NV, typename R>
__device__ __forceinline__ void split_parts(const double (&qa64)[NV], const double (&qb64)[NV],
                                            const R (&qa)[NV], const R (&qb)[NV], R gm1, R adv,
                                            R (&hdF)[NV], R (&hdq)[NV]) {
  R dq[NV], dF[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) dq[c] = to_bulk<R>(qb64[c] - qa64[c]);
  flux_diff<NV, R>(qa, qb, dq, gm1, adv, dF);
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    hdF[c] = R(0.5) * dF[c];
    hdq[c] = R(0.5) * dq[c];
  }
}

// Per-field splitting constant of characteristic field v (u-c, entropy,
// shear..., u+c) along axis dir: max |u_d - c|, max |u_d|, max |u_d + c|.
template <int NV>
__device__ __forceinline__ double field_alpha(const StepState* st, int dir, int v) {
  return st->alpha_f[dir][v == 0 ? 0 : (v == NV - 1 ? 2 : 1)];
}

// FP32 bulk: the state is checked, and the next step's alpha taken, on each
// step's final state; the kinetic energy, sound speed and |u| + c are FP32,
// the energy difference E - ke stays FP64.  The alpha of a later stage of the
// same step (per-stage alpha) is taken in FP64 like the FP64 path's: the
// stage's stencil choices must not depend on FP32 rounding of the splitting
// constant.  unew is the combined state of cell in conserved order.
template <int NV>
__device__ __forceinline__ void bulk_state_check(const SweepArgs& A, long long cell,
                                                 const double (&unew)[NV], int mode,
                                                 double (&amax)[3]) {
  StepState* st = A.st;
  if constexpr (NV > 1) {
    if (A.stage < 2 && (mode & kModeAlpha)) {
      double s[3];
      if (!speeds64<NV, false>(unew, A.gamma, s)) {
        atomicOr(&st->err, kErrNonPhys);
        atomicMin(&st->err_cell, cell);
      } else {
#pragma unroll
        for (int d = 0; d < NV - 2; ++d) amax[d] = fmax(amax[d], s[d]);
      }
      return;
    }
  }
  if (A.stage == 2) {
    if constexpr (NV > 1) {
      double s[3];
      if (!speeds32<NV, false>(unew, A.gamma, s)) {
        atomicOr(&st->err, kErrNonPhys);
        atomicMin(&st->err_cell, cell);
      } else if (mode & kModeAlpha) {
#pragma unroll
        for (int d = 0; d < NV - 2; ++d)
          if (okey(s[d]) > okey(amax[d])) amax[d] = s[d];  // non-negative: bits order like values
      }
    } else if (!isfinite(unew[0])) {
      atomicOr(&st->err, kErrNonPhys);
      atomicMin(&st->err_cell, cell);
    }
  }
}

// Per-field variant (last stage only): the state check, and per axis the
// maxima of |u_d - c|, |u_d| and |u_d + c| in amax[3 d + 0..2], in FP32 like
// the one-alpha path's |u_d| + c.
template <int NV>
__device__ __forceinline__ void bulk_state_check(const SweepArgs& A, long long cell,
                                                 const double (&unew)[NV], int mode,
                                                 double (&amax)[9]) {
  StepState* st = A.st;
  if (A.stage != 2) return;
  if constexpr (NV > 1) {
    double s[9];
    if (!speeds32<NV, true>(unew, A.gamma, s)) {
      atomicOr(&st->err, kErrNonPhys);
      atomicMin(&st->err_cell, cell);
    } else if (mode & kModeAlpha) {
#pragma unroll
      for (int k = 0; k < 3 * (NV - 2); ++k)
        if (okey(s[k]) > okey(amax[k])) amax[k] = s[k];
    }
  }
}

// Number of alpha maxima a sweep accumulates: |u_d| + c per axis, or with
// per-field constants |u_d - c|, |u_d|, |u_d + c| per axis.
template <bool FIELD>
constexpr int kAmax = FIELD ? 9 : 3;

// The shared-memory planes of a tile (per extended cell: the split
// differences df+ and df-, the face correction C, the Roe ingredients and,
// in FP32 bulk, one word of near-tie flags) and the projected windows of its
// faces, shared by the tile's phases and the out-of-line re-decision.
template <int NV, int ORDER, typename R, bool FIELD>
struct TileView {
  using GE = Geo<ORDER>;
  using CV = CellVec<NV, R>;
  static constexpr bool FP32 = sizeof(R) == 4;
  R* dfp;
  R* dfm;
  R* Cf;
  R* prim;
  unsigned* fixmask;
  int cells, SE;
  __device__ __forceinline__ TileView(unsigned char* smem_raw, int ta, int se) : cells(ta * se), SE(se) {
    dfp = reinterpret_cast<R*>(smem_raw);
    dfm = dfp + NV * cells;
    Cf = dfm + NV * cells;
    prim = Cf + NV * cells;
    fixmask = reinterpret_cast<unsigned*>(prim + NPrim<NV>::value * cells);
  }
  __device__ __forceinline__ int sidx(int a, int e) const { return a * SE + e; }
  // Projected window of face j (extended cells) onto the field with left
  // eigenvector row L: sign 0 is the f^+ window centred on cell j, sign 1 the
  // mirrored f^- window centred on cell j+1 (d[i] = -(L df^-) at j+4-i).
  __device__ __forceinline__ void window(int a, int j, int sgn, const R (&L)[NV], R (&d)[8]) const {
    const R* src = sgn == 0 ? dfp : dfm;
#pragma unroll
    for (int i = 0; i < 8; ++i) d[i] = R(0);
#pragma unroll
    for (int i = GE::LO; i <= GE::HI; ++i) {
      const int e = sidx(a, sgn == 0 ? j - 4 + i : j + 4 - i);
      R x[NV];
      CV::load(src, cells, e, x);
      R acc = R(0);
#pragma unroll
      for (int c = 0; c < NV; ++c) acc += L[c] * x[c];
      d[i] = sgn == 0 ? acc : -acc;
    }
  }
  // the same window with the magnitudes sum_c |L_c| |df_c| of its terms
  __device__ __forceinline__ void window_mag(int a, int j, int sgn, const R (&L)[NV], R (&d)[8],
                                             R (&m)[8]) const {
    const R* src = sgn == 0 ? dfp : dfm;
#pragma unroll
    for (int i = 0; i < 8; ++i) d[i] = m[i] = R(0);
#pragma unroll
    for (int i = GE::LO; i <= GE::HI; ++i) {
      const int e = sidx(a, sgn == 0 ? j - 4 + i : j + 4 - i);
      R x[NV];
      CV::load(src, cells, e, x);
      R acc = R(0), mag = R(0);
#pragma unroll
      for (int c = 0; c < NV; ++c) {
        acc += L[c] * x[c];
        mag += rabs(L[c]) * rabs(x[c]);
      }
      d[i] = sgn == 0 ? acc : -acc;
      m[i] = mag;
    }
  }
  // The same for shear field v, whose left row is e_v - w e_0 (w its
  // tangential Roe velocity): one multiply-add per difference instead of NV.
  __device__ __forceinline__ void window_shear(int a, int j, int sgn, int v, R w, R (&d)[8],
                                               R (&m)[8]) const {
    if constexpr (NV >= 4) {
      const R* src = sgn == 0 ? dfp : dfm;
#pragma unroll
      for (int i = 0; i < 8; ++i) d[i] = m[i] = R(0);
#pragma unroll
      for (int i = GE::LO; i <= GE::HI; ++i) {
        const int e = sidx(a, sgn == 0 ? j - 4 + i : j + 4 - i);
        R x[NV];
        CV::load(src, cells, e, x);
        const R xv = shear_comp<NV>(x, v);
        const R acc = xv - w * x[0];
        d[i] = sgn == 0 ? acc : -acc;
        if constexpr (FP32) m[i] = rabs(xv) + rabs(w) * rabs(x[0]);
      }
    }
  }
  // Per-field windows: dfp / dfm hold dF/2 and dq/2; field v splits after the
  // projection, d = L dF/2 +- alpha_v L dq/2 (sign 0: +, sign 1: mirrored -),
  // with magnitude sum |L||dF/2| + alpha_v sum |L||dq/2| for the near-tie bound.
  __device__ __forceinline__ void window_field(int a, int j, int sgn, int v, const R (&L)[NV], R w,
                                               R av, R (&d)[8], R (&m)[8]) const {
    const bool shear = NV >= 4 && v >= 2 && v <= NV - 2;
    const R sa = sgn == 0 ? av : -av;
#pragma unroll
    for (int i = 0; i < 8; ++i) d[i] = m[i] = R(0);
#pragma unroll
    for (int i = GE::LO; i <= GE::HI; ++i) {
      const int e = sidx(a, sgn == 0 ? j - 4 + i : j + 4 - i);
      R xF[NV], xq[NV];
      CV::load(dfp, cells, e, xF);
      CV::load(dfm, cells, e, xq);
      R aF = R(0), aq = R(0), mF = R(0), mq = R(0);
      if constexpr (NV >= 4) {
        if (shear) {
          const R fv = shear_comp<NV>(xF, v), qv = shear_comp<NV>(xq, v);
          aF = fv - w * xF[0];
          aq = qv - w * xq[0];
          if constexpr (FP32) {
            mF = rabs(fv) + rabs(w) * rabs(xF[0]);
            mq = rabs(qv) + rabs(w) * rabs(xq[0]);
          }
        }
      }
      if (!shear) {
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          aF += L[c] * xF[c];
          aq += L[c] * xq[c];
          if constexpr (FP32) {
            mF += rabs(L[c]) * rabs(xF[c]);
            mq += rabs(L[c]) * rabs(xq[c]);
          }
        }
      }
      const R acc = fma(sa, aq, aF);
      d[i] = sgn == 0 ? acc : -acc;
      m[i] = fma(av, mq, mF);
    }
  }
  // Projected window of field v (the same arithmetic in phase 2 and in the
  // phase-2b check of a flagged choice, which must reproduce its pick).
  __device__ __forceinline__ void field_window(int a, int j, int sgn, int v, const R (&L)[NV], R w,
                                               R av, R (&d)[8], R (&mag)[8]) const {
    const bool shear = NV >= 4 && v >= 2 && v <= NV - 2;
    if constexpr (FIELD) {
      window_field(a, j, sgn, v, L, w, av, d, mag);
      return;
    }
    (void)av;
    if (shear) {
      window_shear(a, j, sgn, v, w, d, mag);
    } else if constexpr (FP32) {
      window_mag(a, j, sgn, L, d, mag);
    } else {
      window(a, j, sgn, L, d);
#pragma unroll
      for (int i = 0; i < 8; ++i) mag[i] = R(0);
    }
  }
};

// The raw state of a tile staged in shared memory by TMA: conserved
// component c of line a at extended cell e is p[c rc + a ra + (e + xoff) re]
// (the layout of the copied box; xoff is the alignment slack of x boxes).
struct RawTile {
  const double* p = nullptr;
  int rc = 0, ra = 0, re = 0, xoff = 0;
};
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// One tile of a sweep (phases 1-3 above).  alpha_d and dt are the splitting
// constant of the swept axis and the step size; amax accumulates |u_d| + c of
// combined states (last stage), nfall counts FP64 re-decisions.  FIELD: each
// characteristic field splits with its own constant (st->alpha_f): phase 1
// keeps dF/2 and dq/2, the split follows the projection, and the face's
// centre part 1/2 R diag(alpha) L dq moves into its correction C.
// Phase 2b of a tile (FP32 bulk, near-ties re-decided in the sweep): the
// flagged choices are re-decided from the FP64 state by lane groups of the
// warp (redo_group), or lane by lane when a warp has many (redo_lane), then
// each face applies the changes of its chosen values to its correction C in a
// fixed field/sign order.  Out of line: only tiles with flagged choices call
// it, and its FP64 code does not raise the register footprint of the common
// path.  Ends with a block barrier.
template <int NV, int ORDER, bool COHERENT, bool FIELD>
__device__ __forceinline__ void redecide_tile(const SweepArgs& A, const TileGeo& g,
                                              unsigned char* smem_raw, double alpha_d,
                                              unsigned long long& nfall) {
  using R = float;
  using GE = Geo<ORDER>;
  using CV = CellVec<NV, R>;
  constexpr int G = GE::G;
  StepState* st = A.st;
  const int TA = A.ta, SE = A.se;
  const TileView<NV, ORDER, R, FIELD> tv(smem_raw, TA, SE);
  R* Cf = tv.Cf;
  R* prim = tv.prim;
  unsigned* fixmask = tv.fixmask;
  const int cells = tv.cells;
  auto sidx = [&](int a, int e) { return a * SE + e; };
  const bool sfast = A.dir == 0;
  const int lgTA = __ffs(TA) - 1;
  const int nts = g.nts;
  const int mode = A.mode;
  const R gm1 = bconst<R>(A.gm1, A.gm1_f);
  const R delta = bconst<R>(A.delta, A.delta_f);
  const R tie_rel = bconst<R>(A.tie_rel, A.tie_rel_f);
  const R alpha = (R)alpha_d;
  R alo = alpha, amid = alpha, ahi = alpha;
  if constexpr (FIELD) {
    alo = (R)st->alpha_f[A.dir][0];
    amid = (R)st->alpha_f[A.dir][1];
    ahi = (R)st->alpha_f[A.dir][2];
  }
  auto afield = [&](int v) { return v == 0 ? alo : (v == NV - 1 ? ahi : amid); };
  auto alpha64 = [&](int v) {
    if constexpr (FIELD) return field_alpha<NV>(st, A.dir, v);
    return alpha_d;
  };
  auto field_window = [&](int a, int j, int sgn, int v, const R (&L)[NV], R w, R av, R (&d)[8],
                          R (&mag)[8]) { tv.field_window(a, j, sgn, v, L, w, av, d, mag); };
    constexpr int W = 2 * G <= 8 ? 8 : 16;  // lanes per re-decision group
    const unsigned FULL = 0xffffffffu;
    const int cnt = nts + 1;
    const int bd = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    int al, e0, estep;  // this thread's line, first face and face stride (as for_items)
    if (sfast) {
      const int lgTpl = __ffs(bd) - 1 - lgTA;
      al = tid >> lgTpl;
      e0 = tid & ((1 << lgTpl) - 1);
      estep = 1 << lgTpl;
    } else {
      al = tid & (TA - 1);
      e0 = tid >> lgTA;
      estep = bd >> lgTA;
    }
    // estep is a power of two (blocks of 128 threads): no integer division,
    // which runs partly on the FP64 unit
    const int rounds = (cnt + estep - 1) >> (__ffs(estep) - 1);  // the same for every lane
    for (int rd = 0; rd < rounds; ++rd) {
      const int f = e0 + rd * estep;
      const bool valid = f < cnt && g.a0 + al < g.na;
      const int j = G - 1 + f;
      unsigned fix = valid ? fixmask[sidx(al, j)] : 0u;
      if (!__any_sync(FULL, fix != 0u)) continue;
      // Re-decide every flagged choice of the warp: in each pass, group gi
      // takes the lowest flagged choice of the gi-th lane that still has one,
      // and that lane collects the result from group gi.  Every pass clears at
      // least one of the at most 32 * 2 NV flags, so the default bound (64 NV
      // passes) is never reached; a smaller bound (a test knob) can be: then
      // the error word says so and the choices left keep their FP32 pick.
      constexpr int NG = 32 / W;
      unsigned todo = fix;
      unsigned long long picks = 0ull;
      // Many flags in the warp: each lane re-decides its own choices alone
      // (as many rounds as the busiest lane has flags) instead of the warp
      // serving NG choices per pass; a lone re-decision costs about 2.5x
      // (ENO-AO5) or 3x (ENO-AO7) a cooperative pass.
      const unsigned total = __reduce_add_sync(FULL, (unsigned)__popc(fix));
      const unsigned most = __reduce_max_sync(FULL, (unsigned)__popc(fix));
      if (most * (ORDER == 7 ? 6u : 5u) < 2u * ((total + NG - 1) / NG)) {
        while (todo) {
          const int kk = __ffs(todo) - 1;
          todo &= todo - 1;
          const int pick = redo_lane<NV, ORDER, COHERENT>(A, g, al, g.s0 + f - 1, kk >> 1, kk & 1,
                                                          alpha64(kk >> 1));
          picks |= (unsigned long long)pick << (4 * kk);
          ++nfall;
        }
      }
      const int pass_limit = A.redo_passes;
      for (int pass = 0; pass <= pass_limit; ++pass) {
        const unsigned have = __ballot_sync(FULL, todo != 0u);
        if (!have) break;
        if (pass == pass_limit) {
          if (lane == 0) atomicOr(&st->err, kErrTimeout);
          break;
        }
        const int src = nth_set_bit(have, lane / W);
        const int srcl = src < 0 ? 0 : src;
        const int k = __shfl_sync(FULL, todo ? __ffs(todo) - 1 : 0, srcl);
        int ga = __shfl_sync(FULL, al, srcl);
        int gf = __shfl_sync(FULL, f, srcl);
        if (src < 0) {  // idle group: a valid face of the tile, result unused
          ga = 0;
          gf = 0;
        }
        const int pick = redo_group<NV, ORDER, COHERENT, W>(A, g, ga, g.s0 + gf - 1, k >> 1, k & 1,
                                                            alpha64(k >> 1), lane & (W - 1));
        // my rank among the lanes with work tells which group (if any) took it
        const int rank = __popc(have & ((1u << lane) - 1u));
        const int mine = __shfl_sync(FULL, pick, (rank < NG ? rank : 0) * W);
        if (todo != 0u && rank < NG) {
          const int kk = __ffs(todo) - 1;
          todo &= ~(1u << kk);
          picks |= (unsigned long long)mine << (4 * kk);
          ++nfall;
        }
      }
      fix &= ~todo;  // choices left by a pass bound keep their FP32 pick
      if (!fix) continue;
      // apply the changed choices of this face
      Eigen<NV, R> E;
      if constexpr (NV > 1) {
        R pl[NV], prr[NV];
        CV::load(prim, cells, sidx(al, j), pl);
        CV::load(prim, cells, sidx(al, j + 1), prr);
        roe_eigen<NV, R>(pl, prr, gm1, E);
      }
      const long long gface = g.s0 + f;
      const bool own = (gface <= g.nd) && (f < A.ts || gface == g.nd);
      R dC[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) dC[c] = R(0);
#pragma unroll 1
      for (int k = 0; k < 2 * NV; ++k) {
        if (!(fix & (1u << k))) continue;
        const int v = k >> 1, sgn = k & 1;
        const int pick = (int)((picks >> (4 * k)) & 15ull);
        const bool shear = NV >= 4 && v >= 2 && v <= NV - 2;
        R L[NV], w = R(0);
        if constexpr (NV > 1) {
          left_row<NV, R>(E, v, L);
          if constexpr (NV >= 4) w = -L[0];
        } else {
          L[0] = R(1);
        }
        R d[8], mag[8];
        field_window(al, j, sgn, v, L, w, afield(v), d, mag);
        int pick_old;
        bool m;
        const R nomx[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
        const R corr_old = eno_select<ORDER, R, false>(d, delta, tie_rel, nomx, R(0), pick_old, m);
        if (pick != pick_old) {
          R corr = R(0);
#pragma unroll
          for (int i = GE::LO; i <= GE::HI; ++i) corr += bcoef<R>(pick, i) * d[i];
          const R dv = corr - corr_old;
          if (shear) {
#pragma unroll
            for (int c = 2; c < NV - 1; ++c) dC[c] += c == v ? dv : R(0);
            dC[NV - 1] += w * dv;
          } else if constexpr (NV > 1) {
            R Rc[NV];
            right_col<NV, R>(E, v, Rc);
#pragma unroll
            for (int c = 0; c < NV; ++c) dC[c] += Rc[c] * dv;
          } else {
            dC[0] += dv;
          }
        }
        if ((mode & kModeFlux) && A.idx_out && own) {
          const long long nf = A.nfaces;
          const long long fc = g.fbase + (g.a0 + al) * g.fstride_a + gface * g.fstride_d;
          A.idx_out[(v * 2 + sgn) * nf + fc] = (int8_t)pick;
        }
      }
      const int sj = sidx(al, j);
      R Cv[NV];
      CV::load(Cf, cells, sj, Cv);
#pragma unroll
      for (int c = 0; c < NV; ++c) Cv[c] += dC[c];
      CV::store(Cf, cells, sj, Cv);
    }
  __syncthreads();
}

// The same, not inlined (only one copy of the code, called by the tiles that
// have flags): where the FP64 re-decision code would otherwise set the
// register budget of the whole tile.
template <int NV, int ORDER, bool COHERENT, bool FIELD>
__device__ __noinline__ void redecide_tile_call(const SweepArgs& A, const TileGeo& g,
                                                unsigned char* smem_raw, double alpha_d,
                                                unsigned long long& nfall) {
  redecide_tile<NV, ORDER, COHERENT, FIELD>(A, g, smem_raw, alpha_d, nfall);
}

// TMA: phase 1 reads the tile's raw state from rt instead of global memory,
// and hook() runs once every thread is past phase 1 (the raw buffer is then
// free for the next tile's copy).
template <int NV, int ORDER, typename R, bool COHERENT = false, bool DEFER = false,
          bool FIELD = false, bool TMA = false, typename Hook = NoHook, bool LEAN = false>
__device__ __forceinline__ void sweep_tile(const SweepArgs& A, const TileGeo& g,
                                           unsigned char* smem_raw, double alpha_d, double dt,
                                           double (&amax)[kAmax<FIELD>],
                                           unsigned long long& nfall, const RawTile& rt = RawTile{},
                                           Hook hook = Hook{}) {
  static_assert(!FIELD || NV >= 3, "per-field constants are for the Euler equations");
  using GE = Geo<ORDER>;
  constexpr int G = GE::G;
  constexpr bool FP32 = sizeof(R) == 4;
  constexpr int NP = NPrim<NV>::value;
  StepState* st = A.st;
  const int TA = A.ta, TS = A.ts;
  const int SE = A.se;  // row pitch (>= TS + 2G), chosen on the host for conflict-free banks
  const int cells = TA * SE;
  R* dfp = reinterpret_cast<R*>(smem_raw);
  R* dfm = dfp + NV * cells;
  R* Cf = dfm + NV * cells;
  R* prim = Cf + NV * cells;
  // FP32 only: near-tie flags per face (one word per cell slot)
  unsigned* fixmask = reinterpret_cast<unsigned*>(prim + NP * cells);

  const int dir = A.dir;
  const bool sfast = dir == 0;
  const R alpha = (R)alpha_d;
  const R halpha = R(0.5) * alpha;
  // splitting constant of field v: alpha, or per field max |u_d - c|, |u_d|, |u_d + c|
  R alo = alpha, amid = alpha, ahi = alpha;
  if constexpr (FIELD) {
    alo = (R)st->alpha_f[A.dir][0];
    amid = (R)st->alpha_f[A.dir][1];
    ahi = (R)st->alpha_f[A.dir][2];
  }
  auto afield = [&](int v) { return v == 0 ? alo : (v == NV - 1 ? ahi : amid); };
  // the same in FP64, for the re-decisions of near-ties
  auto alpha64 = [&](int v) {
    if constexpr (FIELD) return field_alpha<NV>(st, A.dir, v);
    return alpha_d;
  };
  const R gm1 = bconst<R>(A.gm1, A.gm1_f);
  const R adv = bconst<R>(A.adv_speed, A.adv_f);
  const R delta = bconst<R>(A.delta, A.delta_f);
  const R tie_rel = bconst<R>(A.tie_rel, A.tie_rel_f);
  const int mode = A.mode;
  const double inv_dx = A.inv_dx;
  const R inv_dx_r = bconst<R>(inv_dx, A.inv_dx_f);
  // FP32 bulk combine: dt and the stage's weight of dt L in FP32
  const float dt32 = f32_rn(dt);
  const float wdt32 = f32_rn((A.stage == 0 ? 1.0 : (A.stage == 1 ? 0.25 : 2.0 / 3.0)) * dt);
  const float inc_w = A.stage == 1 ? -0.75f : -f32_rn(1.0 / 12.0);  // weight of the carried increment
  // Shared-memory rows of SE cells per line for every axis: unit stride
  // along the swept axis (window offsets are immediates); SE is odd, so the
  // y/z sweeps, whose lanes run across lines, hit distinct banks.
  auto sidx = [&](int a, int e) { return a * SE + e; };
  using CV = CellVec<NV, R>;
  const int lgTA = __ffs(TA) - 1;  // TA is a power of two (checked on the host)
  (void)TS;
  const TileView<NV, ORDER, R, FIELD> tv(smem_raw, TA, SE);
  // Projected window of field v (the same arithmetic in phase 2 and in the
  // phase-2b check of a flagged choice, which must reproduce its pick).
  auto field_window = [&](int a, int j, int sgn, int v, const R (&L)[NV], R w, R av, R (&d)[8],
                          R (&mag)[8]) { tv.field_window(a, j, sgn, v, L, w, av, d, mag); };
  const int nts = g.nts;
  const int sext = nts + 2 * G;  // extended cells in use

  // ---------------- phase 1: split differences and Roe ingredients
  {
    const int cnt = sext;
    // the tile's raw state: staged by TMA, or straight from global memory
    auto cell_state = [&](int a, int ee, double (&q)[NV]) {
      if constexpr (TMA) {
        const double* p = rt.p + a * rt.ra + (ee + rt.xoff) * rt.re;
#pragma unroll
        for (int c = 0; c < NV; ++c) q[c] = p[perm_comp<NV>(c, dir) * rt.rc];
      } else {
        const long long la = g.base + (g.a0 + a) * g.stride_a;
        load_state<NV, COHERENT>(A.u_in, A.cstride,
                                 la + bc_map(g.s0 - G + ee, g.nd, A.bc) * g.stride_d, dir, q);
      }
    };
    // cell e's Roe ingredients, and the split differences of the pair (e, e+1)
    auto prim_out = [&](int a, int e, const R (&qa)[NV]) {
      if constexpr (NP > 0) {
        if (e >= G - 1 && e <= G + nts) {
          R pr[NV];
          roe_prims<NV, R>(qa, gm1, pr);
          CV::store(prim, cells, sidx(a, e), pr);
        }
      }
    };
    auto pair_out = [&](int a, int e, const double (&qa64)[NV], const R (&qa)[NV],
                        const double (&qb64)[NV], const R (&qb)[NV]) {
      R fp[NV], fm[NV];
      if constexpr (FIELD)
        split_parts<NV, R>(qa64, qb64, qa, qb, gm1, adv, fp, fm);  // dF/2, dq/2
      else
        split_diff<NV, R>(qa64, qb64, qa, qb, gm1, adv, halpha, fp, fm);
      CV::store(dfp, cells, sidx(a, e), fp);
      CV::store(dfm, cells, sidx(a, e), fm);
    };
    if (sfast) {
      // x sweeps: lanes along the line (coalesced), one pair per item
      for_items(lgTA, cnt, sfast, [&](const int a, const int e) {
        if (g.a0 + a >= g.na) return;
        double qa64[NV];
        cell_state(a, e, qa64);
        R qa[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) qa[c] = to_bulk<R>(qa64[c]);
        prim_out(a, e, qa);
        if (e + 1 < cnt) {
          double qb64[NV];
          cell_state(a, e + 1, qb64);
          R qb[NV];
#pragma unroll
          for (int c = 0; c < NV; ++c) qb[c] = to_bulk<R>(qb64[c]);
          pair_out(a, e, qa64, qa, qb64, qb);
        }
      });
    } else {
      // y/z sweeps: lanes across lines, so a thread can take a run of
      // consecutive cells of its line without losing coalescing; each cell
      // is then loaded and narrowed once (the right cell of one pair is the
      // left cell of the next), the run's last pair reaching one cell on
      int a, j0, step;
      item_start(lgTA, false, a, j0, step);
      const int run = (cnt + step - 1) / step;
      int e = j0 * run;
      const int e_end = min(e + run, cnt);
      if (g.a0 + a < g.na && e < e_end) {
        double q64[NV];
        cell_state(a, e, q64);
        R q[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) q[c] = to_bulk<R>(q64[c]);
        for (;; ++e) {
          prim_out(a, e, q);
          if (e + 1 >= cnt) break;
          double n64[NV];
          cell_state(a, e + 1, n64);
          R n[NV];
#pragma unroll
          for (int c = 0; c < NV; ++c) n[c] = to_bulk<R>(n64[c]);
          pair_out(a, e, q64, q, n64, n);
          if (e + 1 >= e_end) break;
#pragma unroll
          for (int c = 0; c < NV; ++c) {
            q64[c] = n64[c];
            q[c] = n[c];
          }
        }
      }
    }
  }
  __syncthreads();
  hook();

  // ---------------- phase 2: per face choice and back-projection
  bool any_fix = false;  // FP32 bulk: this thread flagged a near-tie
  {
    const int cnt = nts + 1;
    for_items(lgTA, cnt, sfast, [&](const int a, const int f) {
      if (g.a0 + a >= g.na) return;
      const int j = G - 1 + f;  // face j+1/2 in extended cells
      Eigen<NV, R> E;
      if constexpr (NV > 1) {
        R pl[NV], prr[NV];
        CV::load(prim, cells, sidx(a, j), pl);
        CV::load(prim, cells, sidx(a, j + 1), prr);
        roe_eigen<NV, R>(pl, prr, gm1, E);
      }
      const long long gface = g.s0 + f;  // face index between cells gface-1 and gface
      const bool own = (gface <= g.nd) && (f < A.ts || gface == g.nd);
      R C[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) C[c] = R(0);
      unsigned fix = 0;
#pragma unroll 1
      for (int v = 0; v < NV; ++v) {
        // shear fields (2D/3D Euler) have a sparse left row e_v - w e_0
        const bool shear = NV >= 4 && v >= 2 && v <= NV - 2;
        R L[NV], w = R(0);
        if constexpr (NV > 1) {
          left_row<NV, R>(E, v, L);
          if constexpr (NV >= 4) w = -L[0];
        } else {
          L[0] = R(1);
        }
        // f^+ then mirrored f^- window, one live at a time
        R cv = R(0);
        const R av = afield(v);
        if constexpr (FIELD) {
          // the face's centre part: - alpha_v L dq/2 of the face's own pair
          R xq[NV];
          CV::load(dfm, cells, sidx(a, j), xq);
          R aq = R(0);
          if constexpr (NV >= 4) {
            if (shear) aq = shear_comp<NV>(xq, v) - w * xq[0];
          }
          if (!shear) {
#pragma unroll
            for (int c = 0; c < NV; ++c) aq += L[c] * xq[c];
          }
          cv = -av * aq;
        }
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
          R d[8], mag[8];
          field_window(a, j, sgn, v, L, w, av, d, mag);
          int pick;
          bool marg = false;
          R corr = eno_select<ORDER, R, FP32>(d, delta, tie_rel, mag, R(NV + 8) * R(FLT_EPSILON),
                                              pick, marg);
          if constexpr (FP32) {
            if (marg) fix |= 1u << (v * 2 + sgn);  // re-decided in FP64 (phase 2b or the pass)
          }
          if ((mode & kModeFlux) && A.idx_out && own) {
            const long long nf = A.nfaces;
            const long long fc = g.fbase + (g.a0 + a) * g.fstride_a + gface * g.fstride_d;
            A.idx_out[(v * 2 + sgn) * nf + fc] = (int8_t)pick;
          }
          cv += corr;
        }
        if constexpr (NV >= 4) {
          if (shear) {
            // column v of R is e_v + w e_{NV-1}
#pragma unroll
            for (int c = 2; c < NV - 1; ++c) C[c] += c == v ? cv : R(0);
            C[NV - 1] += w * cv;
            continue;
          }
        }
        if constexpr (NV > 1) {
          R Rc[NV];
          right_col<NV, R>(E, v, Rc);
#pragma unroll
          for (int c = 0; c < NV; ++c) C[c] += Rc[c] * cv;
        } else {
          C[0] += cv;
        }
      }
      const int sj = sidx(a, j);
      CV::store(Cf, cells, sj, C);
      if constexpr (FP32) {
        fixmask[sj] = fix;
        any_fix |= fix != 0u;
      }
    });
  }
  if constexpr (!(FP32 && !DEFER)) __syncthreads();  // else the barrier of phase 2b's test

  // ---------------- phase 2b (FP32 bulk, re-decision list): list the faces
  // with flagged choices that this tile owns; the grid-wide pass corrects both
  // cells of each, whichever tiles they lie in, so results do not depend on
  // tiles.  Nothing here changes Cf: phase 3 uses the FP32 choices.
  if constexpr (FP32 && DEFER) {
    for_items(lgTA, nts + 1, sfast, [&](const int a, const int f) {
      if (g.a0 + a >= g.na) return;
      const unsigned fix = fixmask[sidx(a, G - 1 + f)];
      const long long gface = g.s0 + f;
      if (!fix || !((gface <= g.nd) && (f < A.ts || gface == g.nd))) return;
      const unsigned slot = atomicAdd(&st->redo_n, 1u);
      if (slot < A.redo_cap) {
        const long long fc = g.fbase + (g.a0 + a) * g.fstride_a + gface * g.fstride_d;
        A.redo[slot] = ((unsigned long long)fc << 16) | fix;
      } else {
        atomicOr(&st->err, kErrRedoFull);
      }
    });
  }

  // ---------------- phase 2b (FP32 bulk, no list): FP64 re-decision of near-ties
  // Only tiles with flagged choices run it.  LEAN kernels call it out of line,
  // so that its FP64 code does not set the register budget of every tile.
  if constexpr (FP32 && !DEFER) {
    if (__syncthreads_or(any_fix)) {
      if constexpr (LEAN)
        redecide_tile_call<NV, ORDER, COHERENT, FIELD>(A, g, smem_raw, alpha_d, nfall);
      else
        redecide_tile<NV, ORDER, COHERENT, FIELD>(A, g, smem_raw, alpha_d, nfall);
    }
  }

  // ---------------- phase 3: flux difference and Runge-Kutta combine
  if (mode & kModeFlux) {
    const int cnt = nts + 1;
    const long long nf = A.nfaces;
    for_items(lgTA, cnt, sfast, [&](const int a, const int f) {
      if (g.a0 + a >= g.na) return;
      const long long gface = g.s0 + f;
      if (!((gface <= g.nd) && (f < A.ts || gface == g.nd))) return;
      const int j = G - 1 + f;
      const long long la = g.base + (g.a0 + a) * g.stride_a;
      double ql[NV], qr[NV], Fl[NV], Fr[NV];
      load_state<NV, COHERENT>(A.u_in, A.cstride, la + bc_map(gface - 1, g.nd, A.bc) * g.stride_d, dir, ql);
      load_state<NV, COHERENT>(A.u_in, A.cstride, la + bc_map(gface, g.nd, A.bc) * g.stride_d, dir, qr);
      phys_flux<NV>(ql, A.gm1, A.adv_speed, Fl);
      phys_flux<NV>(qr, A.gm1, A.adv_speed, Fr);
      const long long fc = g.fbase + (g.a0 + a) * g.fstride_a + gface * g.fstride_d;
      R Cv[NV];
      CV::load(Cf, cells, sidx(a, j), Cv);
#pragma unroll
      for (int c = 0; c < NV; ++c) {
        if constexpr (FIELD) {
          // F^ = (F_l + F_r)/2 + C, the split's centre part being inside C
          A.fhat[perm_comp<NV>(c, dir) * nf + fc] = 0.5 * (Fl[c] + Fr[c]) + to_f64(Cv[c]);
        } else {
          const double fp = 0.5 * (Fl[c] + alpha_d * ql[c]);
          const double fm = 0.5 * (Fr[c] - alpha_d * qr[c]);
          A.fhat[perm_comp<NV>(c, dir) * nf + fc] = fp + fm + to_f64(Cv[c]);
        }
      }
    });
  } else {
    const int cnt = nts;
    for_items(lgTA, cnt, sfast, [&](const int a, const int t) {
      if (g.a0 + a >= g.na) return;
      const int e = G + t;
      const long long cell = g.base + (g.a0 + a) * g.stride_a + (g.s0 + t) * g.stride_d;
      R r[NV];
      {
        R p0[NV], m1[NV], c1[NV], c0[NV];
        // per field: dF/2 of both of the cell's pairs (the centre part is in C)
        CV::load(dfp, cells, sidx(a, e - 1), p0);
        CV::load(FIELD ? dfp : dfm, cells, sidx(a, e), m1);
        CV::load(Cf, cells, sidx(a, e), c1);
        CV::load(Cf, cells, sidx(a, e - 1), c0);
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          const R s = p0[c] + m1[c] + (c1[c] - c0[c]);
          r[c] = -s * inv_dx_r;
        }
      }
      // Every store of the cell comes after all its loads: the stores could
      // alias the inputs as far as the compiler knows, so a load after a
      // store would wait for it (one memory round trip per component).
      if (!(mode & kModeCombine)) {
        R* rb = reinterpret_cast<R*>(A.rhs);
        R v[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          const long long k = perm_comp<NV>(c, dir) * A.cstride + cell;
          v[c] = (mode & kModeRhsAdd) ? rb[k] + r[c] : r[c];
        }
#pragma unroll
        for (int c = 0; c < NV; ++c) rb[perm_comp<NV>(c, dir) * A.cstride + cell] = v[c];
        return;
      }
      auto u0v = [&](const double* p) { return COHERENT ? __ldcg(p) : __ldg(p); };
      double up[NV], unew[NV];
      float inc[NV];  // FP32 bulk: the increment this stage carries on
#pragma unroll
      for (int c = 0; c < NV; ++c) {
        const long long k = perm_comp<NV>(c, dir) * A.cstride + cell;
        // L(u) summed over the axes in the bulk precision, then one rounding
        // to FP64 for the Runge-Kutta combine
        R Lsum = r[c];
        if (mode & kModeRhsAdd) Lsum = reinterpret_cast<const R*>(A.rhs)[k] + r[c];
        // (the batched kernel reads stage states it wrote itself: through L2)
        const double ui = COHERENT ? __ldcg(A.u_in + k) : __ldg(A.u_in + k);
        const double* u0p = A.u0 + k;
        double un;
        if constexpr (FP32) {
          // Each stage as its own input u_i plus an FP32 increment, the
          // step's increments so far carried in FP32 (each is dt times an
          // FP32-bulk L(u)): with I0 = dt L(u0) and I1 = I0 + dt L(u1),
          //   u1 = u0 + I0
          //   u2 = u1 + (1/4 dt L(u1) - 3/4 I0)
          //   u3 = u2 + (2/3 dt L(u2) - 1/12 I1),
          // which are 3/4 u0 + 1/4 (u1 + dt L(u1)) and 1/3 u0 + 2/3 (u2 +
          // dt L(u2)) because u1 - u0 = I0 and u2 - u0 = I1 / 4 (up to FP64
          // rounding of u1 and u2).  One FP64 add per component (the FP64
          // unit runs at 1/64 of the FP32 rate) and no read of U^n: the
          // increments take the bytes U^n took, and u_i was just read by
          // phase 1.
          float t = wdt32 * Lsum;
          if (A.stage > 0) {
            const float I = COHERENT ? __ldcg(A.inc_in + k) : __ldg(A.inc_in + k);
            inc[c] = fmaf(dt32, Lsum, I);  // I1 (stored by stage 1 only)
            t = fmaf(inc_w, I, t);
          } else {
            inc[c] = t;  // I0
          }
          un = ui + f64_of(t);
        } else {
          const double Lk = to_f64(Lsum);
          if (A.stage == 0) {
            un = ui + dt * Lk;
          } else if (A.stage == 1) {
            un = 0.75 * u0v(u0p) + 0.25 * (ui + dt * Lk);
          } else {
            un = (1.0 / 3.0) * u0v(u0p) + (2.0 / 3.0) * (ui + dt * Lk);
          }
        }
        up[c] = un;
      }
#pragma unroll
      for (int c = 0; c < NV; ++c) A.u_out[perm_comp<NV>(c, dir) * A.cstride + cell] = up[c];
      if constexpr (FP32) {
        if (A.stage < 2) {
#pragma unroll
          for (int c = 0; c < NV; ++c) A.inc_out[perm_comp<NV>(c, dir) * A.cstride + cell] = inc[c];
        }
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) unew[k] = comp_of<NV>(up, k, dir);  // conserved order
      if constexpr (FP32) {
        bulk_state_check<NV>(A, cell, unew, mode, amax);
      } else if constexpr (NV > 1) {
        // non-physical check and next-step alpha on the new state
        double s[kAmax<FIELD>];
        if (!speeds64<NV, FIELD>(unew, A.gamma, s)) {
          atomicOr(&st->err, kErrNonPhys);
          atomicMin(&st->err_cell, cell);
        } else if (mode & kModeAlpha) {
#pragma unroll
          for (int k = 0; k < (FIELD ? 3 : 1) * (NV - 2); ++k) amax[k] = fmax(amax[k], s[k]);
        }
      } else {
        if (!isfinite(unew[0])) {
          atomicOr(&st->err, kErrNonPhys);
          atomicMin(&st->err_cell, cell);
        }
      }
    });
  }
  __syncthreads();
}

// Minimum resident blocks per SM asked of the compiler for the FP32-bulk
// sweep (caps its registers at 65536 / (128 * min blocks)): the sweep is
// latency-bound, so six blocks (80 registers, a few spilled) beat four
// without spills for ENO-AO5; ENO-AO7 keeps more live values and takes five.
#ifndef ENOAO_FP32_MIN_BLOCKS_AO5
#define ENOAO_FP32_MIN_BLOCKS_AO5 6
#endif
#ifndef ENOAO_FP32_MIN_BLOCKS_AO7
#define ENOAO_FP32_MIN_BLOCKS_AO7 5
#endif
// Per-field splitting keeps two projections per window cell live and takes
// four blocks (128 registers).
// With a TMA-staged raw tile a block needs more shared memory, and four of
// them fill an SM: they get the registers (128, no spills; at 96 the
// thread-0 copy issue spills).
// LEAN (ENO-AO5 in-sweep re-decision, re-decisions out of line): 64
// registers (no more spills than at 72), for tiles whose shared memory lets
// seven or eight blocks share an SM.
template <int ORDER, typename R, bool FIELD = false, bool TMA = false, bool LEAN = false>
constexpr int sweep_min_blocks() {
  return sizeof(R) == 8 ? 1
                        : (FIELD ? 4
                                 : (TMA ? 4
                                        : (LEAN ? 8
                                                : (ORDER == 5 ? ENOAO_FP32_MIN_BLOCKS_AO5
                                                              : ENOAO_FP32_MIN_BLOCKS_AO7))));
}

// Bound on the polls of a TMA completion barrier (a copy of a few tens of KB
// lands in microseconds; this is about a second): beyond it the kernel sets
// the error word and returns instead of spinning on.
constexpr long long kTmaPollLimit = 1ll << 24;

// TMA: the tile's raw state (every component, the tile's lines, its cells and
// halo along the swept axis) is one box of the tensor map tmap, copied into
// the first A.tma_raw_bytes of dynamic shared memory by thread 0; the copy of
// the next tile is issued as soon as phase 1 of the current one is done, so
// it lands while phases 2 and 3 run.  Ghost cells outside the grid (the box
// reads zeros there) are then filled from the boundary map with plain loads.
// The end of a sweep launch, for every block: the last block to leave resets
// the tile queue (and the re-decision epoch), the FP64 re-decision count is
// added up, and the block's maxima of the new state's speeds go to alpha.
template <int NV, typename R, bool DEFER, bool FIELD>
__device__ __forceinline__ void sweep_epilogue(const SweepArgs& A, double (&amax)[kAmax<FIELD>],
                                               unsigned long long nfall) {
  constexpr int KA = kAmax<FIELD>;
  StepState* st = A.st;
  const int mode = A.mode;
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1) {
      st->tile_next = 0ull;
      st->blocks_done = 0u;
      if (DEFER) {
        // a new tag for the faces this sweep's re-decision pass marks (never 0,
        // the value of an unmarked face)
        const unsigned e = st->redo_epoch + 1u;
        st->redo_epoch = e ? e : 1u;
      }
      __threadfence();
    }
  }

  if constexpr (sizeof(R) == 4) {
    if (nfall) atomicAdd(&st->fallbacks, nfall);
  }
  if (NV > 1 && (mode & kModeAlpha)) {
    // block max of |u_d| + c (per field: |u_d - c|, |u_d|, |u_d + c|), then
    // one atomic per block and value
    __shared__ double red[KA][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < KA; ++d) {
      double v = amax[d];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0) red[d][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
      for (int d = 0; d < KA; ++d) {
        double v = threadIdx.x < nw ? red[d][threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        unsigned long long* acc;
        int axis;
        if constexpr (FIELD) {  // last stage only (per-field runs with per-step alpha)
          acc = &st->alpha_acc_f[st->par][0][0] + d;
          axis = d / 3;
        } else {
          acc = (A.stage == 2 ? st->alpha_acc[st->par] : st->alpha_stage) + d;
          axis = d;
        }
        if (threadIdx.x == 0 && axis < A.ndim && v > 0.0)
          atomicMax(acc, (unsigned long long)__double_as_longlong(v));
      }
    }
  }
}

template <int NV, int ORDER, typename R, bool DEFER = false, bool FIELD = false, bool TMA = false,
          bool LEAN = false>
__global__ void __launch_bounds__(128, sweep_min_blocks<ORDER, R, FIELD, TMA, LEAN>())
    sweep_kernel(const __grid_constant__ SweepArgs A, const __grid_constant__ CUtensorMap tmap) {
  constexpr bool FP32 = sizeof(R) == 4;
  constexpr int G = Geo<ORDER>::G;
  StepState* st = A.st;
  if (st->skip) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int mode = A.mode;
  const double alpha_d = st->alpha[A.dir];
  const double dt = st->dt;
  constexpr int KA = kAmax<FIELD>;
  double amax[KA];
#pragma unroll
  for (int i = 0; i < KA; ++i) amax[i] = 0.0;
  unsigned long long nfall = 0;
  // Dynamic tile queue: tiles differ in cost (FP64 re-decisions cluster at
  // discontinuities), so blocks pull the next tile instead of striding.  The
  // last block to leave resets the queue for the next launch on the stream.
  __shared__ long long s_tile;
  if constexpr (!TMA) {
    for (;;) {
      if (threadIdx.x == 0) s_tile = (long long)atomicAdd(&st->tile_next, 1ull);
      __syncthreads();
      const long long tile = s_tile;
      if (tile >= A.ntiles) break;
      sweep_tile<NV, ORDER, R, false, DEFER, FIELD, false, NoHook, LEAN>(
          A, tile_geo(A, tile), smem_raw, alpha_d, dt, amax, nfall);
    }
  } else {
    __shared__ __align__(8) unsigned long long s_bar;
    double* raw = reinterpret_cast<double*>(smem_raw);
    unsigned char* smem = smem_raw + A.tma_raw_bytes;
    const int bx = A.tma_box;  // box extent along the swept axis
    RawTile rt;
    rt.p = raw;
    if (A.dir == 0) {  // box (x, lines, components)
      rt.re = 1, rt.ra = bx, rt.rc = bx * A.ta;
    } else {           // box (x = lines, [y,] swept axis, [z,] components)
      rt.re = A.ta, rt.ra = 1, rt.rc = A.ta * bx;
    }
    // thread 0: tile t's box on its way (x boxes start on the even x at or
    // below the tile's first extended cell, 16-byte aligned)
    auto issue = [&](long long t) {
      const TileGeo gg = tile_geo(A, t);
      const long long s_lo = gg.s0 - G;  // first extended cell along the swept axis
      fence_proxy_async();
      mbar_arrive_expect_tx(&s_bar, A.tma_bytes);
      if (A.dir == 0)
        tma_load_3d(raw, &tmap, (int)(s_lo - (s_lo & 1)), (int)gg.a0, 0, &s_bar);
      else if (A.dir == 1)
        tma_load_4d(raw, &tmap, (int)gg.a0, (int)s_lo, (int)gg.b, 0, &s_bar);
      else
        tma_load_4d(raw, &tmap, (int)gg.a0, (int)gg.b, (int)s_lo, 0, &s_bar);
    };
    if (threadIdx.x == 0) {
      mbar_init(&s_bar, 1);
      const long long t = (long long)atomicAdd(&st->tile_next, 1ull);
      s_tile = t;
      if (t < A.ntiles) issue(t);
    }
    __syncthreads();
    unsigned phase = 0;
    for (;;) {
      const long long tile = s_tile;
      if (tile >= A.ntiles) break;
      // the tile's box: a bounded wait, the same decision for the whole block
      bool late = true;
      for (long long it = 0; it < kTmaPollLimit; ++it)
        if (mbar_try_wait(&s_bar, phase)) {
          late = false;
          break;
        }
      if (__syncthreads_or(late)) {
        if (threadIdx.x == 0) atomicOr(&st->err, kErrTimeout);
        // the copy may still be in flight into this block's shared memory:
        // wait for it once more, again bounded, before leaving
        for (long long it = 0; it < kTmaPollLimit && !mbar_try_wait(&s_bar, phase); ++it) {
        }
        break;
      }
      phase ^= 1;
      const TileGeo g = tile_geo(A, tile);
      rt.xoff = A.dir == 0 ? (int)((g.s0 - G) & 1) : 0;
      // ghost cells beyond the grid along the swept axis (edge tiles only)
      if (g.s0 - G < 0 || g.s0 + g.nts + G > g.nd) {
        const int lgTA = __ffs(A.ta) - 1;
        for_items(lgTA, 2 * G, A.dir == 0, [&](const int a, const int k) {
          if (g.a0 + a >= g.na) return;
          const int e = k < G ? k : g.nts + k;
          const long long sg = g.s0 - G + e;
          if (sg >= 0 && sg < g.nd) return;
          double q[NV];
          load_state<NV, false>(A.u_in, A.cstride,
                                g.base + (g.a0 + a) * g.stride_a + bc_map(sg, g.nd, A.bc) * g.stride_d,
                                A.dir, q);
          double* p = raw + a * rt.ra + (e + rt.xoff) * rt.re;
#pragma unroll
          for (int c = 0; c < NV; ++c) p[perm_comp<NV>(c, A.dir) * rt.rc] = q[c];
        });
        __syncthreads();
      }
      auto hook = [&]() {
        if (threadIdx.x == 0) {
          const long long t = (long long)atomicAdd(&st->tile_next, 1ull);
          s_tile = t;
          if (t < A.ntiles) issue(t);
        }
      };
      sweep_tile<NV, ORDER, R, false, DEFER, FIELD, true>(A, g, smem, alpha_d, dt, amax, nfall, rt,
                                                          hook);
    }
  }
  sweep_epilogue<NV, R, DEFER, FIELD>(A, amax, nfall);
}

// One Runge-Kutta stage of a 2D problem in one launch (FP32 bulk, one alpha,
// in-sweep re-decisions; Sec. 2's unsplit sum of the two axes' flux
// differences).  A block takes a 2D tile of Ax.ts x Ay.ts cells: first the x
// part of L(u) on it, as sub-tiles of Ax.ta rows that store it in the
// right-hand-side array like the x sweep, then, after the barrier that ends
// every sub-tile, the y part as sub-tiles of Ay.ta columns that add the
// stored x part and combine, like the y sweep.  A cell's x part is read back
// only by the block that wrote it, straight after writing it (from L2), so
// blocks never wait on one another.  Ax and Ay are the two axes' arguments
// as separate launches would take them; the host makes the 2D tile a whole
// number of both axes' sub-tiles (Ay.ts % Ax.ta == 0, Ax.ts % Ay.ta == 0).
template <int NV, int ORDER, bool LEAN>
__global__ void __launch_bounds__(128, sweep_min_blocks<ORDER, float, false, false, LEAN>())
    fused2d_kernel(const __grid_constant__ SweepArgs Ax, const __grid_constant__ SweepArgs Ay) {
  using R = float;
  StepState* st = Ay.st;
  if (st->skip) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const double alpha_x = st->alpha[0], alpha_y = st->alpha[1];
  const double dt = st->dt;
  double amax[3] = {0.0, 0.0, 0.0};
  unsigned long long nfall = 0;
  const long long tx = Ax.tiles_s, ty = Ay.tiles_s;  // 2D tiles along x and y
  const int kx = Ay.ts / Ax.ta, ky = Ax.ts / Ay.ta;   // sub-tiles per 2D tile
  __shared__ long long s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(&st->tile_next, 1ull);
    __syncthreads();
    const long long T = s_tile;
    if (T >= tx * ty) break;
    const long long X = T % tx, Y = T / tx;
    for (int k = 0; k < kx; ++k) {
      const long long rows = Y * kx + k;  // row group of Ax.ta rows
      if (rows >= Ax.tiles_a) break;
      sweep_tile<NV, ORDER, R, false, false, false, false, NoHook, LEAN>(
          Ax, tile_geo(Ax, X + Ax.tiles_s * rows), smem_raw, alpha_x, dt, amax, nfall);
    }
    for (int m = 0; m < ky; ++m) {
      const long long cols = X * ky + m;  // column group of Ay.ta columns
      if (cols >= Ay.tiles_a) break;
      sweep_tile<NV, ORDER, R, false, false, false, false, NoHook, LEAN>(
          Ay, tile_geo(Ay, Y + Ay.tiles_s * cols), smem_raw, alpha_y, dt, amax, nfall);
    }
  }
  sweep_epilogue<NV, R, false, false>(Ay, amax, nfall);
}

// ------------------------------------------------ grid-wide FP64 re-decisions
// Near-tie choices cluster at discontinuities and slip lines, in a few tiles
// whose SMs' FP64 units would then set a sweep's length.  With a list, the
// sweep instead lists every face that has flagged choices (its owner tile
// does), uses the FP32 choices throughout, and two passes over the whole grid
// follow it: redo_kernel re-decides the listed choices in FP64, one face per
// thread, and applies a change to the face's right cell; redo_apply_kernel
// then applies it to the face's left cell.  L(u) is linear in the face
// correction C, so a change dC of face F adds -dC/dx to cell F - 1 and +dC/dx
// to cell F.  Each cell takes its left face's change first, then its right
// face's, whatever tiles its faces fell in: the result does not depend on
// tiles.

// The line and the position along it of face fc (the face layout of the
// swept axis: nd + 1 faces per line, as tile_geo numbers them).
__device__ __forceinline__ void face_line(const SweepArgs& A, long long fc, long long& line,
                                          long long& F, long long& nd, long long& stride_d,
                                          long long& fstride_d) {
  const long long n0 = A.n[0], n1 = A.n[1];
  if (A.dir == 0) {
    nd = n0; stride_d = 1; fstride_d = 1;
    const long long li = fc / (n0 + 1);
    F = fc - li * (n0 + 1);
    line = li * n0;
  } else if (A.dir == 1) {
    nd = n1; stride_d = n0; fstride_d = n0;
    const long long b = fc / ((n1 + 1) * n0);
    const long long r = fc - b * (n1 + 1) * n0;
    F = r / n0;
    line = b * n1 * n0 + (r - F * n0);
  } else {
    nd = A.n[2]; stride_d = n0 * n1; fstride_d = n0 * n1;
    F = fc / (n0 * n1);
    line = fc - F * (n0 * n1);
  }
}

// Change of face F's correction C (sweep component order) when the choice of
// field v, sign sgn moves from the FP32 pick to pick64, added into dC: the
// FP32 window is rebuilt from the state with the arithmetic of phases 1 and
// 2, and the FP32 pick and value re-derived from it as phase 2b does.
template <int NV, int ORDER>
__device__ __forceinline__ void face_change32(const SweepArgs& A, const TileGeo& g, long long F,
                                              int v, int sgn, int pick64, double alpha_d,
                                              float (&dC)[NV], bool& changed) {
  using GE = Geo<ORDER>;
  const float gm1 = A.gm1_f, adv = A.adv_f;
  const float halpha = 0.5f * (float)alpha_d;
  auto cell = [&](long long gi, double (&q)[NV]) {
    load_state<NV, false>(A.u_in, A.cstride, g.base + bc_map(gi, g.nd, A.bc) * g.stride_d, A.dir, q);
  };
  const bool shear = NV >= 4 && v >= 2 && v <= NV - 2;
  float L[NV], Rc[NV], w = 0.0f;
  if constexpr (NV > 1) {
    double ql64[NV], qr64[NV];
    cell(F - 1, ql64);
    cell(F, qr64);
    float ql[NV], qr[NV], pl[NV], prr[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      ql[c] = to_bulk<float>(ql64[c]);  // the sweep's phase-1 narrowing
      qr[c] = to_bulk<float>(qr64[c]);
    }
    roe_prims<NV, float>(ql, gm1, pl);
    roe_prims<NV, float>(qr, gm1, prr);
    Eigen<NV, float> E;
    roe_eigen<NV, float>(pl, prr, gm1, E);
    left_row<NV, float>(E, v, L);
    right_col<NV, float>(E, v, Rc);
    if constexpr (NV >= 4) w = -L[0];
  } else {
    L[0] = 1.0f;
    Rc[0] = 1.0f;
  }
  // sign 0: d[i] is f^+ of cells (F-5+i, F-4+i); sign 1: -(f^- of (F+3-i, F+4-i))
  float d[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) d[i] = 0.0f;
#pragma unroll
  for (int i = GE::LO; i <= GE::HI; ++i) {
    const long long c0 = sgn == 0 ? F - 5 + i : F + 3 - i;
    double qa64[NV], qb64[NV];
    cell(c0, qa64);
    cell(c0 + 1, qb64);
    float qa[NV], qb[NV], fp[NV], fm[NV], x[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      qa[c] = to_bulk<float>(qa64[c]);
      qb[c] = to_bulk<float>(qb64[c]);
    }
    split_diff<NV, float>(qa64, qb64, qa, qb, gm1, adv, halpha, fp, fm);
#pragma unroll
    for (int c = 0; c < NV; ++c) x[c] = sgn == 0 ? fp[c] : fm[c];
    float acc = 0.0f;
    if constexpr (NV >= 4) {
      if (shear) {
        acc = shear_comp<NV>(x, v) - w * x[0];
      } else {
#pragma unroll
        for (int c = 0; c < NV; ++c) acc += L[c] * x[c];
      }
    } else {
#pragma unroll
      for (int c = 0; c < NV; ++c) acc += L[c] * x[c];
    }
    d[i] = sgn == 0 ? acc : -acc;
  }
  int pick32;
  bool m;
  const float nomx[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  const float corr_old = eno_select<ORDER, float, false>(d, A.delta_f, A.tie_rel_f, nomx,
                                                         0.0f, pick32, m);
  if (pick64 == pick32) return;
  changed = true;
  float corr = 0.0f;
#pragma unroll
  for (int i = GE::LO; i <= GE::HI; ++i) corr += bcoef<float>(pick64, i) * d[i];
  const float dv = corr - corr_old;
  if constexpr (NV >= 4) {
    if (shear) {  // column v of R is e_v + w e_{NV-1}
#pragma unroll
      for (int c = 2; c < NV - 1; ++c) dC[c] += c == v ? dv : 0.0f;
      dC[NV - 1] += w * dv;
      return;
    }
  }
#pragma unroll
  for (int c = 0; c < NV; ++c) dC[c] += Rc[c] * dv;
}

// Adds s * dC (s = +-1/dx) to L(u) of one cell: to the stored L(u) of a
// non-final axis, or, on the final axis, to the combined state through the
// stage's weight of dt L (redo_coef) and to the FP32 increment the stage
// carries on (I0, I1: weight dt).
template <int NV>
__device__ __forceinline__ void apply_change(const SweepArgs& A, long long cell, float s,
                                             const float (&dC)[NV]) {
  const bool combine = (A.mode & kModeCombine) != 0;
  const double w = A.redo_coef * A.st->dt;
  const float dt32 = f32_rn(A.st->dt);
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    const long long k = perm_comp<NV>(c, A.dir) * A.cstride + cell;
    const float dL = s * dC[c];
    if (combine) {
      A.u_out[k] += w * (double)dL;
      if (A.inc_out) A.inc_out[k] = fmaf(dt32, dL, A.inc_out[k]);  // I0, I1 carry dt L
    } else {
      reinterpret_cast<float*>(A.rhs)[k] += dL;
    }
  }
}

// The re-decision pass.  A warp takes CF listed faces at a time and spreads
// their flagged choices over its lanes, one choice per lane (32 per round):
// each lane re-decides its choice in FP64 alone (redo_lane), so that one warp
// instruction of the FP64 unit, whose cost does not shrink with fewer active
// lanes, serves up to 32 choices; it then re-derives the choice's FP32 pick
// and value, and each face's lane adds the changes of its choices in field /
// sign order.  A changed face stores its dC, marks itself with the sweep's
// epoch and applies the change to its right cell F.
template <int NV, int ORDER>
__global__ void __launch_bounds__(128) redo_kernel(const SweepArgs A) {
  constexpr int CF = 8;  // listed faces per warp round
  const unsigned FULL = 0xffffffffu;
  StepState* st = A.st;
  if (st->skip) return;
  const unsigned n = st->redo_n < A.redo_cap ? st->redo_n : (unsigned)A.redo_cap;
  const unsigned epoch = st->redo_epoch;
  const double alpha_d = st->alpha[A.dir];
  const float inv_dx = A.inv_dx_f;
  const int lane = threadIdx.x & 31;
  const unsigned nwarps = gridDim.x * (blockDim.x >> 5);
  unsigned long long nf = 0;
  for (unsigned base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * CF; base < n;
       base += nwarps * CF) {
    // lane j < CF holds listed face base + j
    const unsigned i = base + lane;
    const bool hasf = lane < CF && i < n;
    const unsigned long long rec = hasf ? A.redo[i] : 0ull;
    const unsigned mask = (unsigned)(rec & 0xffffull);
    long long line, F, nd, stride_d, fstride_d;
    face_line(A, (long long)(rec >> 16), line, F, nd, stride_d, fstride_d);
    // choices of face j are numbers pre_j .. pre_j + m_j - 1 of the round
    const int m = __popc(mask);
    int incl = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += t;
    }
    const int pre = incl - m;
    const int T = __shfl_sync(FULL, incl, 31);
    float dC[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) dC[c] = 0.0f;
    bool changed = false;
    for (int c0 = 0; c0 < T; c0 += 32) {
      // lane l takes choice c0 + l: face j, field * 2 + sign k
      const int ci = c0 + lane;
      int j = 0;
#pragma unroll
      for (int q = 1; q < CF; ++q) {
        const int pq = __shfl_sync(FULL, pre, q);
        if (ci >= pq) j = q;
      }
      // every lane takes part in each shuffle (none inside a condition)
      const unsigned mj = __shfl_sync(FULL, mask, j);
      const int prej = __shfl_sync(FULL, pre, j);
      const long long lj = __shfl_sync(FULL, line, j), Fj = __shfl_sync(FULL, F, j);
      const int kb = ci < T ? nth_set_bit(mj, ci - prej) : -1;
      const bool valid = kb >= 0;
      const int k = valid ? kb : 0;
      const int cnt = T - c0 < 32 ? T - c0 : 32;
      float dk[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) dk[c] = 0.0f;
      bool ch = false;
      if (valid) {
        TileGeo g;  // the face's line, as redo_lane reads it
        g.base = lj;
        g.a0 = 0;
        g.stride_a = 0;
        g.stride_d = stride_d;
        g.nd = nd;
        const int pick64 = redo_lane<NV, ORDER, false>(A, g, 0, Fj - 1, k >> 1, k & 1, alpha_d);
        face_change32<NV, ORDER>(A, g, Fj, k >> 1, k & 1, pick64, alpha_d, dk, ch);
        ++nf;
      }
      // each face's lane adds its choices' changes in field / sign order
      for (int l = 0; l < cnt; ++l) {
        const int jl = __shfl_sync(FULL, j, l);
        const int chl = __shfl_sync(FULL, (int)ch, l);
        float v[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) v[c] = __shfl_sync(FULL, dk[c], l);
        if (lane == jl && chl) {
#pragma unroll
          for (int c = 0; c < NV; ++c) dC[c] += v[c];
          changed = true;
        }
      }
    }
    if (hasf) {
      const long long fc = (long long)(rec >> 16);
      A.redo_mark[fc] = changed ? epoch : 0u;
      if (changed) {
#pragma unroll
        for (int c = 0; c < NV; ++c) A.redo_dc[(long long)i * NV + c] = dC[c];
        if (F < nd) apply_change<NV>(A, line + F * stride_d, inv_dx, dC);
      }
    }
  }
  if (nf) atomicAdd(&st->fallbacks, nf);
}

// Second pass: each changed face applies its change to its left cell F - 1.
// On the final axis the cells a change touched are then checked and enter
// the next alpha (a cell whose right face also changed is checked by that
// face's thread, after both of its changes).  The last block to leave empties
// the list for the next sweep.
template <int NV>
__global__ void __launch_bounds__(128) redo_apply_kernel(const SweepArgs A) {
  StepState* st = A.st;
  const unsigned n = st->skip ? 0u : (st->redo_n < A.redo_cap ? st->redo_n : (unsigned)A.redo_cap);
  const unsigned epoch = st->redo_epoch;
  const float inv_dx = A.inv_dx_f;
  const bool check = (A.mode & kModeCombine) != 0;
  double amax[3] = {0.0, 0.0, 0.0};
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long fc = (long long)(A.redo[i] >> 16);
    if (A.redo_mark[fc] != epoch) continue;
    long long line, F, nd, stride_d, fstride_d;
    face_line(A, fc, line, F, nd, stride_d, fstride_d);
    float dC[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) dC[c] = A.redo_dc[(long long)i * NV + c];
    auto check_cell = [&](long long cell) {
      double u[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) u[c] = A.u_out[c * A.cstride + cell];
      bulk_state_check<NV>(A, cell, u, A.mode, amax);
    };
    if (F >= 1) {
      apply_change<NV>(A, line + (F - 1) * stride_d, -inv_dx, dC);
      if (check) check_cell(line + (F - 1) * stride_d);
    }
    if (check && F < nd && !(F + 1 <= nd && A.redo_mark[fc + fstride_d] == epoch))
      check_cell(line + F * stride_d);
  }
  if constexpr (NV > 1) {
    if (check && (A.mode & kModeAlpha)) {
      unsigned long long* acc = A.stage == 2 ? st->alpha_acc[st->par] : st->alpha_stage;
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (d < A.ndim && amax[d] > 0.0)
          atomicMax(&acc[d], (unsigned long long)__double_as_longlong(amax[d]));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&st->redo_done, 1u) == gridDim.x - 1) {
      st->redo_n = 0u;
      st->redo_done = 0u;
      __threadfence();
    }
  }
}

}  // namespace enoao
