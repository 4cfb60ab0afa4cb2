// weno_device.cuh -- device building blocks of the WENO-ZA6 right-hand side.
//
// Method: Gu, Wang, Don, Jung, arXiv 2603.26272 (WENO-ZA6, Section 3; the
// general framework of Section 2; the Euler systems of Section 4).
//
// Arithmetic economy.  On GB300 the FP64 pipe is ~1/64 of the FP32 rate, so
// this path is bound by FP64 instruction issue, not by HBM.  Every formula
// below is an algebraically exact rewrite of the paper's, chosen to use few
// FP64 operations and to round relative to the stencil's variation:
//  * the smoothness indicators of eq. (15) in terms of first and second
//    differences (equal to the quadratic forms <f_k, B_k f_k>),
//  * tau of eq. (17) as a third difference of second differences,
//  * the candidate fluxes of eq. (11) as f_i plus a difference correction,
//  * the left eigenvectors of the Roe matrix in closed form with shared
//    sub-expressions, two of their rows and the 1/2 of eq. (6) folded into
//    the back-projection.
#pragma once
#include <cstdint>

namespace weno {

// Parameters of eqs. (21)-(22) for one characteristic field.  The field's
// split fluxes reach the reconstruction multiplied by `scale` (2 or 4, see
// the projection below), so mu_0 and, without Ai, epsilon are scaled to keep
// Gamma_k exactly the paper's.
struct ReconParams {
  double eps4;   // 4 * eps            (indicators are carried as 4*beta, 4*tau)
  double mu0s;   // scale * mu_0       (Ai)
  double efix;   // 4 * eps * scale^2  (no Ai: mu = 1)
  double p;      // power parameter of eq. (21)
  double me;     // sqrt(4 eps) / 6    (Ai: 4 eps mu^2 = (me * dev + mo)^2, dev =
  double mo;     // sqrt(4 eps) * scale * mu_0   the sum of |v_j - mean v|)
  double e0;     // mo^2: the term of a flat stencil (dev = 0)
  float mef;     // me^2 = eps / 9 = mef 2^eme, mef in [1, 2) (FP32)
  int eme;
  int lthr;      // dev >= 2^(lthr - 1019) implies me dev >= 2^30 mo (mo negligible)
};

// ---------------------------------------------------------------------------
// Format changes on the integer pipe.  An FP64 <-> FP32 conversion issues to
// the FP64 pipe, the one these kernels are bound by; where a value only needs
// FP32 accuracy the helpers below move between the formats with integer
// instructions on the bit patterns instead.
// ---------------------------------------------------------------------------

// x 2^(1019 - es) as FP32 with the mantissa truncated to 23 bits, where es is
// at least the biased exponent of x (so the result is below 2^-3 in
// magnitude); 0 where the result would fall below FP32's normal range.
__device__ __forceinline__ float f32_scaled(double x, int es) {
  const int hi = __double2hiint(x);
  const int fe = ((hi >> 20) & 0x7FF) - es + 123;
  const unsigned m = __funnelshift_r((unsigned)__double2loint(x), (unsigned)hi, 29) & 0x7FFFFFu;
  const unsigned b = ((unsigned)hi & 0x80000000u) | ((unsigned)fe << 23) | m;
  return (fe > 0 && (hi & 0x7FF00000) != 0) ? __uint_as_float(b) : 0.0f;
}

// x 2^(1019 - es) rounded to FP32 (to nearest, ties away from zero), with es
// at least the biased exponent of x; 0 below FP32's normal range.
__device__ __forceinline__ float f32_scaled_rn(double x, int es) {
  const unsigned lo = (unsigned)__double2loint(x), lor = lo + 0x10000000u;
  const int hi = __double2hiint(x) + (lor < lo ? 1 : 0);  // a carry into the exponent is exact
  const int fe = ((hi >> 20) & 0x7FF) - es + 123;
  const unsigned m = __funnelshift_r(lor, (unsigned)hi, 29) & 0x7FFFFFu;
  const unsigned b = ((unsigned)hi & 0x80000000u) | ((unsigned)fe << 23) | m;
  return (fe > 0 && (__double2hiint(x) & 0x7FF00000) != 0) ? __uint_as_float(b) : 0.0f;
}

// x rounded to FP32 (to nearest, ties away from zero): 0 below FP32's normal
// range, infinite above it.
__device__ __forceinline__ float f32_rn(double x) {
  const unsigned lo = (unsigned)__double2loint(x), lor = lo + 0x10000000u;
  const int hi = __double2hiint(x) + (lor < lo ? 1 : 0);
  const int fe = ((hi >> 20) & 0x7FF) - 896;
  const unsigned sg = (unsigned)hi & 0x80000000u;
  const unsigned m = __funnelshift_r(lor, (unsigned)hi, 29) & 0x7FFFFFu;
  const unsigned b = fe <= 0 ? sg : (fe >= 255 ? (sg | 0x7F800000u) : (sg | ((unsigned)fe << 23) | m));
  return __uint_as_float(b);
}

// y 2^k as FP64 for any FP32 y: exact for a normal y whose image is a normal
// double; 0 for a zero or subnormal y or below FP64's normal range; infinite
// above it (and for an infinite or NaN y).
__device__ __forceinline__ double f64_of_f32(float y, int k) {
  const unsigned b = __float_as_uint(y), sg = b & 0x80000000u;
  const int fe = (int)((b >> 23) & 0xFFu);
  const int F = fe + 896 + k;
  const unsigned hi = (fe == 0 || F <= 0)  ? sg
                      : (fe == 255 || F >= 2047) ? (sg | 0x7FF00000u)
                      : (sg | ((unsigned)(F << 20) + ((b >> 3) & 0xFFFFFu)));
  const unsigned lo = (fe == 0 || F <= 0 || fe == 255 || F >= 2047) ? 0u : (b << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// y 2^k as FP64 for a positive normal FP32 y, exactly (the caller keeps the
// result inside FP64's normal range).
__device__ __forceinline__ double f64_of_f32_pos(float y, int k) {
  const unsigned b = __float_as_uint(y);
  return __hiloint2double((int)(b >> 3) + ((896 + k) << 20), (int)(b << 29));
}

// f > 0 and finite, by the bit pattern (integer pipe only).
__device__ __forceinline__ bool pos_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7FF0000000000000LL;
}

// Order-preserving map of any double to an unsigned integer (and back), so
// signed minima and maxima can be reduced with integer atomicMax.
__device__ __forceinline__ unsigned long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? ((unsigned long long)b | 0x8000000000000000ull) : ~(unsigned long long)b;
}
__device__ __forceinline__ double okey_inv(unsigned long long k) {
  return __longlong_as_double((k & 0x8000000000000000ull) ? (long long)(k & 0x7FFFFFFFFFFFFFFFull)
                                                           : (long long)~k);
}

// Scalar fluxes (Section 4.1): system 0 linear advection f = a u, 2 Burgers
// f = u^2/2, 3 Buckley-Leverett f = u^2 / (u^2 + 0.25 (1-u)^2); f' below.
__device__ __forceinline__ double scalar_flux(int system, double a, double u) {
  if (system == 2) return 0.5 * (u * u);
  if (system == 3) {
    const double q = 1.0 - u;
    const double uu = u * u;
    return uu / fma(0.25 * q, q, uu);
  }
  return a * u;
}
__device__ __forceinline__ double scalar_speed(int system, double a, double u) {
  if (system == 2) return u;
  if (system == 3) {
    const double q = 1.0 - u;
    const double D = fma(0.25 * q, q, u * u);
    return (0.5 * u * q) / (D * D);
  }
  return a;
}
// GLF speed of eq. (6) for a scalar flux over the data range [umin, umax]:
// the largest |f'| there (for Buckley-Leverett f' peaks inside (0, 1) at
// ustar, which the host supplies).
__device__ __forceinline__ double scalar_alpha(int system, double a, double umin, double umax,
                                               double ustar) {
  if (system == 0) return fabs(a);
  double s = fmax(fabs(scalar_speed(system, a, umin)), fabs(scalar_speed(system, a, umax)));
  if (system == 3 && umin <= ustar && ustar <= umax)
    s = fmax(s, fabs(scalar_speed(system, a, ustar)));
  return s;
}

// Bit pattern of |x| as an ordered integer: for non-negative doubles the
// integer order is the numeric order (NaN sorts above +inf).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL);
}

// 1/x for a positive normal x (the divisions of the stage kernels: the Roe
// weights, the weight denominators, 1/rho), by Newton-Raphson.  With
// x = m 2^E, m in [1, 2), the seed is the FP32 approximate reciprocal of m
// (rcp.approx.ftz.f32 on the special-function unit, within about 2^-22
// of 1/m after m is truncated to FP32's 23 mantissa bits), made an FP64
// number scaled by 2^-E on the integer pipe; one cubic Newton-Raphson step,
// r <- r + r (e + e^2) with e = 1 - x r, leaves a relative error of about
// e^3 < 2^-64, so the result is 1/x to within the FP64 rounding of its three
// fused multiply-adds (about 1 ulp).  Three FP64 operations instead of the
// ~8 pipe slots of an IEEE division.  (Inputs outside the positive normal
// range, or so large that 1/x is subnormal -- a nonphysical state, which the
// kernels report separately -- give a meaningless but finite value.)
__device__ __forceinline__ double rcp_pos(double x) {
  const int hi = __double2hiint(x);
  const int ex = (hi >> 20) & 0x7FF;
  const float mf = __uint_as_float(
      0x3F800000u | (__funnelshift_r((unsigned)__double2loint(x), (unsigned)hi, 29) & 0x7FFFFFu));
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));
  const double r = f64_of_f32_pos(rf, 1023 - ex);
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// 1/sqrt(x) for a positive normal x, by the same route as rcp_pos: with
// x = m' 2^(2q), m' in [1, 4), the FP32 approximate reciprocal square root of
// m' (rsqrt.approx.ftz.f32, within about 2^-22 after m' is truncated to FP32)
// scaled by 2^-q on the integer pipe, then one step of the third-order
// iteration r <- r (1 + e/2 + 3 e^2 / 8), e = 1 - x r^2 (the series of
// (1 - e)^(-1/2)), which leaves a relative error of about 2.5 e^3 / 8 <
// 2^-64: five FP64 operations.  (Outside the positive normal range -- a
// nonphysical state, reported separately -- the value is meaningless.)
__device__ __forceinline__ double rsqrt_pos(double x) {
  const int hi = __double2hiint(x);
  const int ex = (hi >> 20) & 0x7FF;
  const int odd = (ex & 1) ^ 1;  // the unbiased exponent ex - 1023 is odd
  const float mf = __uint_as_float(((unsigned)(127 + odd) << 23) |
                                   (__funnelshift_r((unsigned)__double2loint(x), (unsigned)hi, 29) &
                                    0x7FFFFFu));
  float rf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));
  const double r = f64_of_f32_pos(rf, (1023 + odd - ex) / 2);  // times 2^-q, q = (ex - 1023 - odd) / 2
  const double e = fma(-x, r * r, 1.0);
  return fma(r * fma(0.375, e, 0.5), e, r);
}

// sqrt(x) = x / sqrt(x) for a positive normal x (six FP64 operations).
__device__ __forceinline__ double sqrt_pos(double x) { return x * rsqrt_pos(x); }

// ---------------------------------------------------------------------------
// WENO-ZA6 numerical flux at x_{i+1/2} from v0..v5 = f_{i-2}..f_{i+3}
// (positive flux; the negative flux is this routine on the mirrored stencil).
//
// With d_j = v_{j+1} - v_j and s_k = d_{k+1} - d_k:
//   4 beta_k = 13/3 s_k^2 + t_k^2, t = (3d1 - d0, d1 + d2, 3d2 - d3, 3d4 - 5d3)
//       (eq. (15) with the matrices B_0, B_1, B_2 = rev(B_0), B_d),
//   4 beta_3 = mean of the four (eq. (16)),
//   4 tau = 4 (s3 - s0 + 3 (s1 - s2))^2 (eq. (17): the fifth difference),
//   f^k = v2 + r_k / 6, r = (5d1 - 2d0, d1 + 2d2, 4d2 - d3, 6d2 - 5d3 + 2d4)
//       = (2 t0 - d1, d1 + 2d2, 4d2 - d3, 6d2 + (t3 - d4))  (eq. (11)),
//   mu = mean |v_j - mean v| + mu_0 (eq. (22)), Gamma_k = (tau/(beta_k +
//   eps mu^2))^p (eq. (21)), alpha_k = d_k (1 + Gamma_k) (eq. (20), L = q = 1),
//   f = sum alpha_k f^k / sum alpha_k (eqs. (14), (19)), d = (1, 9, 9, 1)/20.
//
// The routine takes the five differences d_j (it never needs the values
// themselves) and returns num = sum a_k r_k and den = sum a_k with a_k
// proportional to alpha_k, so f = v2 + num / (6 den); field_flux below forms
// the differences of a field's positive and mirrored negative fluxes and
// adds the two reconstructions with one reciprocal.
// b_k = 4 beta_k + 4 eps mu^2 is formed as 13/3 s_k^2 + (t_k^2 + e), and
// b_3 = mean of b_0, b_1, b_2, b_d (the same number as 4 beta_3 + e).
// (The bound on the spread of the b_k with Ai: each 4 beta_k is at most ~1e4
// mu^2 and e = 4e-40 mu^2, so min b / max b > ~1e-44.)
//
// For p = 1 the four divisions tau/b_k are removed: a_k is proportional to
// (b_k + 4 tau) prod_{j != k} b_j, formed pairwise: with p01 = b0 b1 and
// p23 = b2 b3, a_0 = p23 (p01 + 4 tau b1), a_1 = p23 (p01 + 4 tau b0),
// a_2 = p01 (p23 + 4 tau b3), a_3 = p01 (p23 + 4 tau b2), and the sums over
// k = 0, 1 and k = 2, 3 are taken before their factors p23, p01.  Before the
// products, the b_k and 4 tau are multiplied by the power of two that brings
// their maximum into [1, 2) (built from the exponent bits), and the scaled
// b_k are floored at 2^-166, so the products -- and the product of two
// denominators in pair_flux, at least 2^-996 -- can neither overflow nor
// underflow.  The floor acts only on a substencil flatter than 2^-166 of the
// largest indicator (never with Ai and eps >= 1e-40, where the spread is
// below 2^-142; possible with a tiny eps or without Ai on large data).  Such
// substencils' candidates differ from one another by less than 2^-80 of the
// stencil's variation, and 4 tau, when not 0, is above 2^-104 of the largest
// indicator (it is the square of a difference of the d_j, which is 0 or at
// least an ulp of them), so their weights keep dominating the others and
// the flux moves by less than that 2^-80.
//
// mu is formed in FP32 from the FP64 differences (truncated to FP32 after a
// common power-of-two scaling, so no data magnitude overflows it), and
// eps mu^2 from it to FP32 accuracy: it enters only through eps mu^2 with
// eps = 1e-40, which matters only for a substencil whose indicator is below
// ~1e-30 mu^2, where a relative error of ~1e-6 in eps mu^2 moves Gamma_k by
// the same relative amount and the weights by less than 1e-30.  The rescale
// below relies on eps mu^2 being right to within that 1e-6.
// ---------------------------------------------------------------------------
// The sensitivity term 4 eps mu^2 = (me dev + mo)^2 of eqs. (21)-(22) from
// the FP32 deviation sum devf of a stencil scaled by 2^(1019 - es)
// (dev = devf 2^(es - 1019)).  Flat stencil (devf = 0): mo^2.  Where
// me dev >= 2^30 mo it is me^2 dev^2 to FP32 accuracy: with devf = mdf 2^edf,
// the FP32 product y = mef mdf^2 in [1, 8) times 2^(eme + 2 edf +
// 2 (es - 1019)), assembled on the integer pipe.  Otherwise (a variation below
// ~1e-29 of the data, or exponents beyond FP64's range) dev64() -- the same
// deviation sum in FP64 -- in a branch only the warps that need it run.
template <class Dev64>
__device__ __forceinline__ double sens_term(float devf, int es, const ReconParams &P,
                                            Dev64 dev64) {
  const unsigned db = __float_as_uint(devf);
  const int edf = (int)(db >> 23) - 127;
  const float mdf = __uint_as_float((db & 0x7FFFFFu) | 0x3F800000u);
  const float y = P.mef * (mdf * mdf);
  const int k = P.eme + 2 * (edf + es - 1019);
  const int fexp = (int)(__float_as_uint(y) >> 23) + 896 + k;  // biased exponent of the result
  const bool flat = (devf == 0.0f);
  const bool fast = flat || (edf + es >= P.lthr && fexp > 0 && fexp < 2047);
  double e = flat ? P.e0 : f64_of_f32_pos(y, fast ? k : 0);
  if (__any_sync(__activemask(), !fast)) {
    if (!fast) {
      const double sm = fma(dev64(), P.me, P.mo);  // sqrt(4 eps) mu
      e = sm * sm;
    }
  }
  return e;
}

struct ZA6Part {
  double num, den;  // f = v2 + num / (6 den)
};

template <bool AI, bool P1>
__device__ __forceinline__ ZA6Part za6d(double d0, double d1, double d2, double d3, double d4,
                                        const ReconParams &P) {
  const double s0 = d1 - d0, s1 = d2 - d1, s2 = d3 - d2, s3 = d4 - d3;
  const double t0 = fma(3.0, d1, -d0);
  const double t1 = d1 + d2;
  const double t2 = fma(3.0, d2, -d3);
  const double t3 = fma(3.0, d4, -5.0 * d3);
  const double r5 = fma(3.0, s1 - s2, s3 - s0);
  double e;
  if (AI) {
    // deviations from v2, then from their mean, in FP32, on the differences
    // scaled by 2^(1019 - es) with es the largest of their exponents (so no
    // data range overflows FP32): dev = devf 2^(es - 1019)
    const int es = max(max(max(__double2hiint(d0) & 0x7FFFFFFF, __double2hiint(d1) & 0x7FFFFFFF),
                           max(__double2hiint(d2) & 0x7FFFFFFF, __double2hiint(d3) & 0x7FFFFFFF)),
                       __double2hiint(d4) & 0x7FFFFFFF) >> 20;
    const float f0 = f32_scaled(d0, es), f1 = f32_scaled(d1, es), f2 = f32_scaled(d2, es),
                f3 = f32_scaled(d3, es), f4 = f32_scaled(d4, es);
    const float fa0 = -(f0 + f1), fa1 = -f1, fa3 = f2, fa4 = f2 + f3, fa5 = fa4 + f4;
    const float fm = ((fa0 + fa1) + (fa3 + fa4) + fa5) * (1.0f / 6.0f);
    const float devf = fabsf(fa0 - fm) + fabsf(fa1 - fm) + fabsf(fm) + fabsf(fa3 - fm) +
                       fabsf(fa4 - fm) + fabsf(fa5 - fm);
    e = sens_term(devf, es, P, [&]() {
      const double a0 = -(d0 + d1), a1 = -d1, a3 = d2, a4 = d2 + d3, a5 = a4 + d4;
      const double m = ((a0 + a1) + (a3 + a4) + a5) * (1.0 / 6.0);
      return fabs(a0 - m) + fabs(a1 - m) + fabs(m) + fabs(a3 - m) + fabs(a4 - m) + fabs(a5 - m);
    });
  } else {
    e = P.efix;
  }
  const double c13 = 13.0 / 3.0;
  double b0 = fma(c13 * s0, s0, fma(t0, t0, e));
  double b1 = fma(c13 * s1, s1, fma(t1, t1, e));
  double b2 = fma(c13 * s2, s2, fma(t2, t2, e));
  const double bd = fma(c13 * s3, s3, fma(t3, t3, e));
  const double bsum = (b0 + b1) + (b2 + bd);  // 4 b_3
  const double r0 = fma(2.0, t0, -d1);
  const double r1 = fma(2.0, d2, d1);
  const double r2 = fma(4.0, d2, -d3);
  const double r3 = fma(6.0, d2, t3 - d4);
  const double T0 = r5 * r5;  // tau
  double a0, a1, a2, a3;
  if (P1) {
    // largest exponent among b_k and 4 tau (bit patterns of positives order
    // as the numbers; 4 tau by adding 2 to the exponent field; b_3 is a mean
    // of the others and never the largest)
    unsigned long long mb = max(max(__double_as_longlong(b0), __double_as_longlong(b1)),
                                max(__double_as_longlong(b2), __double_as_longlong(bd)));
    mb = max(mb, (unsigned long long)(__double_as_longlong(T0) + (2LL << 52)));
    const int ex = (int)((mb >> 52) & 0x7FF);
    double b3;
    if (AI) {
      // With the affine-invariant e every b_k is within a factor ~1e-44 of
      // the largest, so the scaled values stay normal and the scaling by
      // 2^(1023 - ex) is an exact add to the exponent field (integer pipe);
      // b_3 = bsum / 4 takes exponent - 2 in the same add.
      const int k = (1023 - ex) << 20;
      b0 = __hiloint2double(__double2hiint(b0) + k, __double2loint(b0));
      b1 = __hiloint2double(__double2hiint(b1) + k, __double2loint(b1));
      b2 = __hiloint2double(__double2hiint(b2) + k, __double2loint(b2));
      b3 = __hiloint2double(__double2hiint(bsum) + k - (2 << 20), __double2loint(bsum));
    } else {
      const double sc = __longlong_as_double((2046LL - ex) << 52);
      b0 *= sc;
      b1 *= sc;
      b2 *= sc;
      b3 = bsum * (0.25 * sc);
    }
    // 4 tau, scaled by the same 2^(1023 - ex) (T0 times 2^(1025 - ex)): an add
    // to the exponent field for a normal T0; 0 when the scaled value falls
    // below the normal range (it is then under 2^-1022 of the largest b_k and
    // moves no weight); a subnormal T0 takes the multiplication, in a branch
    // only the warps that need it run.
    const long long tb = __double_as_longlong(T0);
    const int t0e = (int)(tb >> 52);
    double T = (t0e > 0 && t0e + 1025 - ex > 0)
                   ? __longlong_as_double(tb + ((long long)(1025 - ex) << 52))
                   : 0.0;
    const bool sub = (t0e == 0 && tb != 0);
    if (__any_sync(__activemask(), sub)) {
      if (sub) T = T0 * __longlong_as_double((2048LL - ex) << 52);
    }
    const long long floor_bits = (1023LL - 166) << 52;  // 2^-166 (b_3 >= max / 4 needs none)
    b0 = __longlong_as_double(max(__double_as_longlong(b0), floor_bits));
    b1 = __longlong_as_double(max(__double_as_longlong(b1), floor_bits));
    b2 = __longlong_as_double(max(__double_as_longlong(b2), floor_bits));
    // a_0 = p23 x0, a_1 = p23 x1, a_2 = p01 x2, a_3 = p01 x3 with p01 = b0 b1,
    // p23 = b2 b3 and x0 = b1 (b0 + T) = p01 + T b1, x1 = p01 + T b0,
    // x2 = p23 + T b3, x3 = p23 + T b2; the linear weights 1 : 9 : 9 : 1 go
    // on x1, x2, and each half's sums are taken before its common factor
    const double p01 = b0 * b1, p23 = b2 * b3;
    const double x0 = fma(T, b1, p01), y1 = 9.0 * fma(T, b0, p01);
    const double y2 = 9.0 * fma(T, b3, p23), x3 = fma(T, b2, p23);
    ZA6Part o;
    o.num = fma(p23, fma(y1, r1, x0 * r0), p01 * fma(y2, r2, x3 * r3));
    o.den = fma(p23, x0 + y1, p01 * (y2 + x3));
    return o;
  } else {
    const double T = 4.0 * T0;
    const double b3 = 0.25 * bsum;
    a0 = 1.0 + pow(T / b0, P.p);
    a1 = 1.0 + pow(T / b1, P.p);
    a2 = 1.0 + pow(T / b2, P.p);
    a3 = 1.0 + pow(T / b3, P.p);
  }
  ZA6Part o;  // the linear weights 1 : 9 : 9 : 1 applied here
  o.num = fma(9.0, fma(a1, r1, a2 * r2), fma(a0, r0, a3 * r3));
  o.den = fma(9.0, a1 + a2, a0 + a3);
  return o;
}

// f^+_{i+1/2} + f^-_{i+1/2} of one field from its two reconstructions, with
// one reciprocal: base + (n+ d- + n- d+) / (6 d+ d-), where base = v2+ + v2-
// is the sum of the two stencils' centre values.
__device__ __forceinline__ double pair_flux(double base, const ZA6Part &p, const ZA6Part &m) {
  const double q = fma(p.num, m.den, m.num * p.den) * rcp_pos(p.den * m.den);
  return fma(q, 1.0 / 6.0, base);
}

// One characteristic field of one face (FP64): w[j], g[j] are the projected
// states and fluxes of the six stencil cells i-2 .. i+3 and A the field's GLF
// speed.  The split of eq. (6) (kernel scaling: without the 1/2) is applied
// to the differences: f+ = g + A w has differences dg + A dw, and the
// mirrored f- = g - A w, read from i+3 down to i-2, has differences
// A dw - dg in reverse order; the two centre values add up to
// (g_i + g_{i+1}) - A (w_{i+1} - w_i).  Returns h = f^+ + f^- at i+1/2.
template <bool AI, bool P1>
__device__ __forceinline__ double field_flux(const double (&w)[6], const double (&g)[6], double A,
                                             const ReconParams &P) {
  double dp[5], dm[5], dw2 = 0.0;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const double dw = w[j + 1] - w[j], dg = g[j + 1] - g[j];
    dp[j] = fma(A, dw, dg);
    dm[4 - j] = fma(A, dw, -dg);
    if (j == 2) dw2 = dw;
  }
  const double base = fma(-A, dw2, g[2] + g[3]);
  return pair_flux(base, za6d<AI, P1>(dp[0], dp[1], dp[2], dp[3], dp[4], P),
                   za6d<AI, P1>(dm[0], dm[1], dm[2], dm[3], dm[4], P));
}

// The same from the differences alone: dw[j] = w_{j+1} - w_j and
// dg[j] = g_{j+1} - g_j over the six stencil cells.  Returns h less the
// centre values g_i + g_{i+1}, i.e. the dissipation -A (w_{i+1} - w_i) plus
// the two reconstructions' corrections; the caller adds the centre values
// back (the 2D kernel in physical form after the back-projection, where
// R (g_i + g_{i+1}) is the physical F_i + F_{i+1}).
template <bool AI, bool P1>
__device__ __forceinline__ double field_flux_d(const double (&dw)[5], const double (&dg)[5],
                                               double A, const ReconParams &P) {
  double dp[5], dm[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    dp[j] = fma(A, dw[j], dg[j]);
    dm[4 - j] = fma(A, dw[j], -dg[j]);
  }
  return pair_flux(-A * dw[2], za6d<AI, P1>(dp[0], dp[1], dp[2], dp[3], dp[4], P),
                   za6d<AI, P1>(dm[0], dm[1], dm[2], dm[3], dm[4], P));
}

// ---------------------------------------------------------------------------
// Central-upwind WENO of order 2R for R = 2, 4, 5 (the Appendix schemes; R = 3
// uses za6 above).  Tables as printed in the Appendix, divided out; rows the
// paper writes as rev(.) are spelled out reversed.  The candidate fluxes are
// formed as v_{R-1} plus a correction (every c_k sums to 1); each indicator
// beta_k = <f_k, B_k f_k> is evaluated on f_k minus its first entry (B_k
// annihilates constants, so this is the same number with rounding relative to
// the substencil's variation) and clamped at 0 against rounding; tau from
// c_tau on the stencil relative to v_{R-1} (c_tau sums to 0).  The weights
// follow eqs. (16)-(22); for p = 1 without divisions per candidate, as in
// za6: a_k = d_k (b_k + 4 tau) prod_{j != k} b_j after a power-of-two
// rescale, in the "4 beta" units of za6 (b_k = 4 beta_k + 4 eps mu^2).
// ---------------------------------------------------------------------------
template <int R> struct OrderTab;

template <> struct OrderTab<2> {
  __device__ static double dn(int k) {  // d_k times its common denominator
    const double v[3] = {1, 4, 1};
    return v[k];
  }
  __device__ static double ck(int k, int m) {
    const double c[3][2] = {{-1, 3}, {1, 1}, {3, -1}};
    return c[k][m] / 2.0;
  }
  __device__ static double d(int k) {
    const double v[3] = {1, 4, 1};
    return v[k] / 6.0;
  }
  __device__ static double B(int k, int a, int b) {  // B_0 = B_1 = B_d
    return (a == b) ? 1.0 : -1.0;
  }
  __device__ static double ctau(int j) {
    const double v[4] = {-1, 3, -3, 1};
    return v[j];
  }
};

template <> struct OrderTab<4> {
  __device__ static double dn(int k) {  // d_k times its common denominator
    const double v[5] = {1, 16, 36, 16, 1};
    return v[k];
  }
  __device__ static double ck(int k, int m) {
    const double c[5][4] = {{-3, 13, -23, 25}, {1, -5, 13, 3}, {-1, 7, 7, -1}, {3, 13, -5, 1},
                            {25, -23, 13, -3}};
    return c[k][m] / 12.0;
  }
  __device__ static double d(int k) {
    const double v[5] = {1, 16, 36, 16, 1};
    return v[k] / 70.0;
  }
  __device__ static double B(int k, int a, int b) {
    const double B0[4][4] = {{547, -1941, 2321, -927}, {-1941, 7043, -8623, 3521},
                             {2321, -8623, 11003, -4701}, {-927, 3521, -4701, 2107}};
    const double B1[4][4] = {{267, -821, 801, -247}, {-821, 2843, -2983, 961},
                             {801, -2983, 3443, -1261}, {-247, 961, -1261, 547}};
    const double Bd[4][4] = {{7107, -16901, 13521, -3727}, {-16901, 40643, -32863, 9121},
                             {13521, -32863, 26843, -7501}, {-3727, 9121, -7501, 2107}};
    double v;
    if (k == 0) v = B0[a][b];
    else if (k == 1) v = B1[a][b];
    else if (k == 2) v = B1[3 - a][3 - b];
    else if (k == 3) v = B0[3 - a][3 - b];
    else v = Bd[a][b];
    return v / 240.0;
  }
  __device__ static double ctau(int j) {
    const double v[8] = {-1, 7, -21, 35, -35, 21, -7, 1};
    return v[j];
  }
};

template <> struct OrderTab<5> {
  __device__ static double dn(int k) {  // d_k times its common denominator
    const double v[6] = {1, 25, 100, 100, 25, 1};
    return v[k];
  }
  __device__ static double ck(int k, int m) {
    const double c[6][5] = {{12, -63, 137, -163, 137}, {-3, 17, -43, 77, 12},
                            {2, -13, 47, 27, -3},      {-3, 27, 47, -13, 2},
                            {12, 77, -43, 17, -3},     {137, -163, 137, -63, 12}};
    return c[k][m] / 60.0;
  }
  __device__ static double d(int k) {
    const double v[6] = {1, 25, 100, 100, 25, 1};
    return v[k] / 252.0;
  }
  __device__ static double B(int k, int a, int b) {
    const double B0[5][5] = {{45316, -208501, 364863, -288007, 86329},
                             {-208501, 965926, -1704396, 1358458, -411487},
                             {364863, -1704396, 3042786, -2462076, 758823},
                             {-288007, 1358458, -2462076, 2041126, -649501},
                             {86329, -411487, 758823, -649501, 215836}};
    const double B1[5][5] = {{13816, -60871, 99213, -70237, 18079},
                             {-60871, 277126, -464976, 337018, -88297},
                             {99213, -464976, 812586, -611976, 165153},
                             {-70237, 337018, -611976, 485446, -140251},
                             {18079, -88297, 165153, -140251, 45316}};
    const double B2[5][5] = {{13816, -51001, 67923, -38947, 8209},
                             {-51001, 209926, -299076, 179098, -38947},
                             {67923, -299076, 462306, -299076, 67923},
                             {-38947, 179098, -299076, 209926, -51001},
                             {8209, -38947, 67923, -51001, 13816}};
    const double Bd[5][5] = {{942016, -2964751, 3597813, -2004757, 429679},
                             {-2964751, 9449926, -11584896, 6499258, -1399537},
                             {3597813, -11584896, 14319786, -8079576, 1746873},
                             {-2004757, 6499258, -8079576, 4577926, -992851},
                             {429679, -1399537, 1746873, -992851, 215836}};
    double v;
    if (k == 0) v = B0[a][b];
    else if (k == 1) v = B1[a][b];
    else if (k == 2) v = B2[a][b];
    else if (k == 3) v = B1[4 - a][4 - b];
    else if (k == 4) v = B0[4 - a][4 - b];
    else v = Bd[a][b];
    return v / 10080.0;
  }
  __device__ static double ctau(int j) {
    const double v[10] = {-1, 9, -36, 84, -126, 126, -84, 36, -9, 1};
    return v[j];
  }
};

// Partial result of a reconstruction of order 2R: the flux is vc + num / den.
struct RPart {
  double vc, num, den;
};

template <int R, bool AI, bool P1>
__device__ __forceinline__ RPart za_r(const double (&v)[2 * R], const ReconParams &P) {
  using Tb = OrderTab<R>;
  constexpr int N = 2 * R;
  const double vc = v[R - 1];
  double w[N];  // the stencil relative to v_{R-1}
#pragma unroll
  for (int j = 0; j < N; ++j) w[j] = (j == R - 1) ? 0.0 : v[j] - vc;
  double e;
  if (AI) {  // mu from FP32 deviations, as in za6d (dev = 6/N of the sum over N points)
    int es = 0;
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (j != R - 1) es = max(es, __double2hiint(w[j]) & 0x7FFFFFFF);
    es >>= 20;
    float wf[N], mf = 0.0f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      wf[j] = (j == R - 1) ? 0.0f : f32_scaled(w[j], es);
      mf += wf[j];
    }
    mf *= 1.0f / N;
    float df = 0.0f;
#pragma unroll
    for (int j = 0; j < N; ++j) df += fabsf(wf[j] - mf);
    e = sens_term(df * (6.0f / N), es, P, [&]() {
      double m = 0.0, dev = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) m += w[j];
      m *= 1.0 / N;
#pragma unroll
      for (int j = 0; j < N; ++j) dev += fabs(w[j] - m);
      return dev * (6.0 / N);
    });
  } else {
    e = P.efix;
  }
  // b_k = 4 beta_k + e on f_k minus its first entry (symmetric form: each
  // off-diagonal pair once); k = R is the downwind substencil's beta_d
  double b[R + 1];
  double bd = 0.0, bsum = 0.0;
#pragma unroll
  for (int k = 0; k <= R; ++k) {
    double g[R];
#pragma unroll
    for (int m = 1; m < R; ++m) g[m] = (k == R - 1) ? w[k + m] : w[k + m] - w[k];
    double q = 0.0;
#pragma unroll
    for (int a = 1; a < R; ++a) {
      double row = (4.0 * Tb::B(k, a, a)) * g[a];
#pragma unroll
      for (int c = a + 1; c < R; ++c) row = fma(8.0 * Tb::B(k, a, c), g[c], row);
      q = fma(g[a], row, q);
    }
    q = fmax(q, 0.0) + e;  // the form is positive semidefinite; clamp its rounding
    if (k < R) b[k] = q; else bd = q;
    bsum += q;
  }
  b[R] = bsum * (1.0 / (R + 1));  // eq. (16): the mean, with e included once
  double tr = 0.0;                // 2 (c_tau . f): T = 4 tau
#pragma unroll
  for (int j = 0; j < N; ++j)
    if (j != R - 1) tr = fma(2.0 * Tb::ctau(j), w[j], tr);
  const double T0 = tr * tr;
  double a[R + 1];
  if (P1) {
    unsigned long long mb = (unsigned long long)__double_as_longlong(bd);
#pragma unroll
    for (int k = 0; k < R; ++k) mb = max(mb, (unsigned long long)__double_as_longlong(b[k]));
    mb = max(mb, (unsigned long long)__double_as_longlong(T0));
    const int ex = (int)((mb >> 52) & 0x7FF);
    if (AI) {  // exact exponent add, as in za6 (the b_k lie within ~1e-46 of the largest)
      const int sh = (1023 - ex) << 20;
#pragma unroll
      for (int k = 0; k <= R; ++k)
        b[k] = __hiloint2double(__double2hiint(b[k]) + sh, __double2loint(b[k]));
    } else {
      const double sc = __longlong_as_double((2046LL - ex) << 52);
#pragma unroll
      for (int k = 0; k <= R; ++k) b[k] *= sc;
    }
    const double T = T0 * __longlong_as_double((2046LL - ex) << 52);
    // floor of the scaled indicators, as in za6d: 2^(-1000 / 2R) up to R = 4,
    // where the product of two denominators holds 2R of them, 2^-200 at R = 5
    // (no product of denominators; a Q_k holds 5)
    constexpr long long kFloorExp = (R == 5) ? 200 : 1000 / (2 * R);
    const long long floor_bits = (1023LL - kFloorExp) << 52;
#pragma unroll
    for (int k = 0; k <= R; ++k)
      b[k] = __longlong_as_double(max(__double_as_longlong(b[k]), floor_bits));
    // a_k = (b_k + T) prod_{j != k} b_j from prefix and suffix products
    double pre[R + 1], suf[R + 1];
    pre[0] = 1.0;
    suf[R] = 1.0;
#pragma unroll
    for (int k = 1; k <= R; ++k) pre[k] = (k == 1) ? b[0] : pre[k - 1] * b[k - 1];
#pragma unroll
    for (int k = R - 1; k >= 0; --k) suf[k] = (k == R - 1) ? b[R] : suf[k + 1] * b[k + 1];
    const double Pall = pre[R] * b[R];  // prod of all b_j
#pragma unroll
    for (int k = 0; k <= R; ++k) {
      const double pk = (k == 0) ? suf[0] : (k == R ? pre[R] : pre[k] * suf[k]);
      a[k] = fma(T, pk, Pall);  // (b_k + T) prod_{j != k} b_j
    }
  } else {
    const double T = T0;
#pragma unroll
    for (int k = 0; k <= R; ++k) a[k] = 1.0 + pow(T / b[k], P.p);
  }
  double num = 0.0, den = 0.0;
#pragma unroll
  for (int k = 0; k <= R; ++k) {
    double corr = 0.0;  // f^k - v_{R-1}
#pragma unroll
    for (int m = 0; m < R; ++m)
      if (k + m != R - 1) corr = fma(Tb::ck(k, m), w[k + m], corr);
    const double ak = (Tb::dn(k) == 1.0) ? a[k] : Tb::dn(k) * a[k];
    num = fma(ak, corr, num);
    den += ak;
  }
  return RPart{vc, num, den};
}

// f^+ + f^- of one field from two reconstructions of order 2R.  Up to R = 4
// the two denominators share one division; at R = 5 a single discontinuity
// at the edge of the stencil leaves five flat substencils, whose products
// reach ~1e-170 (in the rescaled units), and the product of two such
// denominators would underflow, so each keeps its own division there.
template <int R>
__device__ __forceinline__ double pair_flux_r(const RPart &p, const RPart &m) {
  if (R <= 4) {
    const double q = fma(p.num, m.den, m.num * p.den) * rcp_pos(p.den * m.den);
    return (p.vc + m.vc) + q;
  }
  return (p.vc + p.num * rcp_pos(p.den)) + (m.vc + m.num * rcp_pos(m.den));
}

// ---------------------------------------------------------------------------
// FP32 reconstruction (precision mode WENO_PREC_FP32_RECON).
//
// Input: the five FP64 stencil differences d_j = v_{j+1} - v_j already
// rounded to FP32.  Output: the FP32 correction c with f_hat = v2 + c.
// The stencil is normalised by its descaler, d_j / mu with
// mu = mean |v_j - mean v| + mu_0 (eq. (22)); with the affine-invariant
// weights this is an exact symmetry (Gamma_k of eq. (21) is unchanged when the
// data are scaled), so all indicators are O(1) numbers in FP32.  In normalised
// units the sensitivity term eps mu^2 becomes eps; it is replaced by
// eps32 = 1e-30 (1e-40 is below FP32's normal range); this changes Gamma_k
// only for substencils flat to 1e-15 of the stencil's variation, whose rivals'
// weights then fall to 1e-30 instead of 1e-40 -- far below FP32 resolution.
// Weights are normalised before the products with the candidates, so no
// intermediate can overflow.
// ---------------------------------------------------------------------------
struct Recon32 {
  float eps4;   // 4 * eps32
  float p;      // power parameter
};

template <bool P1>
__device__ __forceinline__ float za6_f32(float e0, float e1, float e2, float e3, float e4,
                                         const Recon32 &P) {
  const float a0 = -(e0 + e1), a1 = -e1, a3 = e2, a4 = e2 + e3, a5 = a4 + e4;
  const float m = ((a0 + a1) + (a3 + a4) + a5) * (1.0f / 6.0f);
  const float dev = fabsf(a0 - m) + fabsf(a1 - m) + fabsf(m) + fabsf(a3 - m) + fabsf(a4 - m) +
                    fabsf(a5 - m);
  // mu_0 only guards the normalisation against 0/0; in FP32 its reciprocal
  // would overflow, so mu is floored at 1e-30 instead (the weights do not
  // depend on the normalisation).
  const float mu = fmaxf(dev * (1.0f / 6.0f), 1e-30f);
  const float im = 1.0f / mu;
  const float d0 = e0 * im, d1 = e1 * im, d2 = e2 * im, d3 = e3 * im, d4 = e4 * im;
  const float s0 = d1 - d0, s1 = d2 - d1, s2 = d3 - d2, s3 = d4 - d3;
  const float t0 = fmaf(3.0f, d1, -d0);
  const float t1 = d1 + d2;
  const float t2 = fmaf(3.0f, d2, -d3);
  const float t3 = fmaf(3.0f, d4, -5.0f * d3);
  const float c13 = 13.0f / 3.0f;
  const float B0 = fmaf(c13 * s0, s0, t0 * t0);
  const float B1 = fmaf(c13 * s1, s1, t1 * t1);
  const float B2 = fmaf(c13 * s2, s2, t2 * t2);
  const float Bd = fmaf(c13 * s3, s3, t3 * t3);
  const float B3 = 0.25f * ((B0 + B1) + (B2 + Bd));
  const float r5 = fmaf(3.0f, s1 - s2, s3 - s0);
  const float T = 4.0f * (r5 * r5);
  const float b0 = B0 + P.eps4, b1 = B1 + P.eps4, b2 = B2 + P.eps4, b3 = B3 + P.eps4;
  float a0w, a1w, a2w, a3w;
  if (P1) {
    a0w = 1.0f + T / b0;
    a1w = 9.0f * (1.0f + T / b1);
    a2w = 9.0f * (1.0f + T / b2);
    a3w = 1.0f + T / b3;
  } else {
    // (T / b_k)^p overflows FP32 next to a flat substencil (T / eps32 ~ 1e33),
    // so with b_min the smallest b_k every alpha_k is taken times
    // (b_min / T)^p when T > b_min: alpha_k ~ d_k ((b_min/T)^p + (b_min/b_k)^p),
    // the same weights, and no term above 1.
    const float bmin = fminf(fminf(b0, b1), fminf(b2, b3));
    const float q0 = powf(bmin / b0, P.p), q1 = powf(bmin / b1, P.p),
                q2 = powf(bmin / b2, P.p), q3 = powf(bmin / b3, P.p);
    float base = 1.0f, M = 0.0f;
    if (T <= bmin) {
      M = powf(T / bmin, P.p);  // alpha_k = d_k (1 + M q_k)
    } else {
      base = powf(bmin / T, P.p);  // alpha_k ~ d_k ((b_min/T)^p + q_k)
      M = 1.0f;
    }
    a0w = fmaf(M, q0, base);
    a1w = 9.0f * fmaf(M, q1, base);
    a2w = 9.0f * fmaf(M, q2, base);
    a3w = fmaf(M, q3, base);
  }
  const float is = 1.0f / ((a0w + a1w) + (a2w + a3w));
  const float r0 = fmaf(5.0f, d1, -2.0f * d0);
  const float r1 = fmaf(2.0f, d2, d1);
  const float r2 = fmaf(4.0f, d2, -d3);
  const float r3 = fmaf(6.0f, d2, fmaf(-5.0f, d3, 2.0f * d4));
  const float c = fmaf(a0w * is, r0, fmaf(a1w * is, r1, fmaf(a2w * is, r2, (a3w * is) * r3)));
  return (c * (1.0f / 6.0f)) * mu;
}

// The FP32 part from the FP64 differences dw[j] = w_{j+1} - w_j, dg[j]:
// the corrections of both reconstructions, c+ + c-, as an FP64 number.  The
// differences go to FP32 scaled by the common power of two 2^(1019 - es)
// (es: their largest exponent; the reconstruction is homogeneous of degree
// one in the data, so the correction comes back times 2^(es - 1019)), with
// the format changes on the integer pipe.
template <bool P1>
__device__ __forceinline__ double recon_pair_f32(const double (&dw)[5], const double (&dg)[5],
                                                 double A, const Recon32 &P) {
  const float Af = f32_rn(A);
  int es = 0;
#pragma unroll
  for (int j = 0; j < 5; ++j)
    es = max(es, max(__double2hiint(dw[j]) & 0x7FFFFFFF, __double2hiint(dg[j]) & 0x7FFFFFFF));
  es >>= 20;
  float dp[5], dm[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const float fw = f32_scaled_rn(dw[j], es), fg = f32_scaled_rn(dg[j], es);
    dp[j] = fmaf(Af, fw, fg);
    dm[j] = fmaf(-Af, fw, fg);
  }
  // f^+ on (i-2..i+3) around v2 = f^+_i; f^- mirrored (i+3..i-2) around f^-_{i+1},
  // whose differences are -dm[4], ..., -dm[0].
  const float cp = za6_f32<P1>(dp[0], dp[1], dp[2], dp[3], dp[4], P);
  const float cm = za6_f32<P1>(-dm[4], -dm[3], -dm[2], -dm[1], -dm[0], P);
  return f64_of_f32(cp + cm, es - 1019);
}

// One characteristic field in FP32-reconstruction mode: w[j], g[j] are the
// FP64 projections of the six stencil states and fluxes, A the field's GLF
// speed.  Returns h = f_hat^+ + f_hat^- (kernel scaling: split without 1/2).
// FP64 work: the ten differences, the base f+_i + f-_{i+1} and one add.
template <bool P1>
__device__ __forceinline__ double field_flux_f32(const double (&w)[6], const double (&g)[6],
                                                 double A, const Recon32 &P) {
  double dw[5], dg[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    dw[j] = w[j + 1] - w[j];
    dg[j] = g[j + 1] - g[j];
  }
  const double base = fma(A, w[2] - w[3], g[2] + g[3]);
  return base + recon_pair_f32<P1>(dw, dg, A, P);
}

// field_flux_f32 from the differences alone, less the centre values
// g_i + g_{i+1} (as field_flux_d).
template <bool P1>
__device__ __forceinline__ double field_flux_f32d(const double (&dw)[5], const double (&dg)[5],
                                                  double A, const Recon32 &P) {
  return fma(-A, dw[2], recon_pair_f32<P1>(dw, dg, A, P));
}

// ---------------------------------------------------------------------------
// Characteristic-wise Lax-Friedrichs flux of the Euler equations at one face
// (Section 4.2), in the face's normal frame: components (rho, m_n, m_t, E)
// with normal flux (F0..F3), face-normal velocity u_n, tangential u_t.
//
// Roe average of the cells on both sides; right eigenvectors
//   r1 = (1, un-c, ut, H-un c), r2 = (1, un, ut, q^2/2), r3 = (0, 0, 1, ut),
//   r4 = (1, un+c, ut, H+un c);
// with b1 = (gamma-1)/c^2, b2 = b1 q^2/2, the left eigenvectors are
//   l1 = 1/2 (b2 + un/c, -(b1 un + 1/c), -b1 ut, b1),  l2 = (1-b2, b1 un, b1 ut, -b1),
//   l3 = (-ut, 0, 1, 0),  l4 = 1/2 (b2 - un/c, -(b1 un - 1/c), -b1 ut, b1).
// The kernel projects with 2 l1, l2, l3, 2 l4 and splits without the 1/2 of
// eq. (6), so field m reaches the reconstruction scaled by k = (4, 2, 2, 4);
// the back-projection divides again.
// ---------------------------------------------------------------------------
struct FaceState {
  double un, ut, H, c, ic, b1, b2, hq2, q2;  // Roe-averaged face state
};

__device__ __forceinline__ bool roe_face(double sl, double unl, double utl, double Hl, double sr,
                                         double unr, double utr, double Hr, double gm1,
                                         FaceState &f) {
  const double inv = rcp_pos(sl + sr);
  const double wl = sl * inv, wr = sr * inv;
  f.un = fma(wl, unl, wr * unr);
  f.ut = fma(wl, utl, wr * utr);
  f.H = fma(wl, Hl, wr * Hr);
  const double q2 = fma(f.un, f.un, f.ut * f.ut);
  f.q2 = q2;
  f.hq2 = 0.5 * q2;
  const double c2 = gm1 * (f.H - f.hq2);
  if (!pos_finite(c2)) return false;
  f.ic = rsqrt_pos(c2);
  f.c = c2 * f.ic;
  f.b1 = gm1 * (f.ic * f.ic);
  f.b2 = f.b1 * f.hq2;
  return true;
}

// Characteristic values (2 l1.V, l2.V, l3.V, 2 l4.V) of a vector V in the
// normal frame (rho-like, mn-like, mt-like, E-like).
__device__ __forceinline__ void project4(const FaceState &f, double r, double mn, double mt,
                                         double E, double &w1, double &w2, double &w3,
                                         double &w4) {
  const double s = fma(f.un, mn, fma(f.ut, mt, -E));
  const double z = fma(f.b2, r, -(f.b1 * s));
  const double tc = fma(f.un, r, -mn) * f.ic;
  w1 = z + tc;
  w4 = z - tc;
  w2 = r - z;
  w3 = fma(-f.ut, r, mt);
}

// Characteristic values of the physical flux of a cell from those of its
// state: in the normal frame F = un_j U + p_j (0, 1, 0, un_j) (eq. (25)), and
// the projection is linear, so g = un_j w + p_j project4(0, 1, 0, un_j), where
// project4(0, 1, 0, un_j) = (z - 1/c, -z, 0, z + 1/c) with z = b1 (un_j - un).
// Same operation count as projecting F, but F need not be staged.
__device__ __forceinline__ void project_flux4(const FaceState &f, double unj, double pj,
                                              double w1, double w2, double w3, double w4,
                                              double &g1, double &g2, double &g3, double &g4) {
  const double z = f.b1 * (unj - f.un);
  const double pz = pj * z, pc = pj * f.ic;
  g1 = fma(unj, w1, pz - pc);
  g2 = fma(unj, w2, -pz);
  g3 = unj * w3;
  g4 = fma(unj, w4, pz + pc);
}

// Four times the physical flux from h = (h1, h2, h3, h4) reconstructed in
// the scaled characteristic fields: with e = (h1/4, h2/2, h3/2, h4/4),
// 4 F = 4 R e = R (h1, 2 h2, 2 h3, h4); the 1/4 is applied with 1/dx in the
// flux difference, so no multiplication by it is spent here.
__device__ __forceinline__ void backproject4(const FaceState &f, double h1, double h2, double h3,
                                             double h4, double &F0, double &F1, double &F2,
                                             double &F3) {
  const double h14 = h1 + h4;
  const double S = fma(2.0, h2, h14);  // 4 (e1 + e2 + e4)
  const double D = h4 - h1;            // 4 (e4 - e1)
  const double h3x2 = h3 + h3;         // 4 e3
  F0 = S;
  F1 = fma(f.un, S, f.c * D);
  F2 = fma(f.ut, S, h3x2);
  F3 = fma(f.H, h14, fma(f.un * f.c, D, fma(f.q2, h2, f.ut * h3x2)));
}

// 1D Euler (rho, m, E): R = [(1, u-c, H-uc), (1, u, u^2/2), (1, u+c, H+uc)],
// L rows 1/2 (b2 + u/c, -(b1 u + 1/c), b1), (1-b2, b1 u, -b1),
// 1/2 (b2 - u/c, -(b1 u - 1/c), b1); fields scaled by k = (4, 2, 4).
// (Written with explicit FMAs only, so the compiler has nothing to contract
// and project3_field below computes every field bit for bit as project3.)
__device__ __forceinline__ void project3(const FaceState &f, double r, double m, double E,
                                         double &w1, double &w2, double &w3) {
  const double s = fma(f.un, m, -E);
  const double z = fma(f.b2, r, -(f.b1 * s));
  const double t = fma(f.un, r, -m);
  w1 = fma(t, f.ic, z);
  w3 = fma(-t, f.ic, z);
  w2 = r - z;
}

// Field q of project3 alone (the same operations as its q-th output).
__device__ __forceinline__ double project3_field(const FaceState &f, int q, double r, double m,
                                                 double E) {
  const double s = fma(f.un, m, -E);
  const double z = fma(f.b2, r, -(f.b1 * s));
  if (q == 1) return r - z;
  const double t = fma(f.un, r, -m);
  return fma(q == 0 ? t : -t, f.ic, z);
}

// Four times the 1D physical flux, 4 F = R (h1, 2 h2, h3), as backproject4.
__device__ __forceinline__ void backproject3(const FaceState &f, double h1, double h2, double h3,
                                             double &F0, double &F1, double &F2) {
  const double h13 = h1 + h3;
  const double S = fma(2.0, h2, h13);
  const double D = h3 - h1;
  F0 = S;
  F1 = fma(f.un, S, f.c * D);
  F2 = fma(f.H, h13, fma(f.un * f.c, D, f.q2 * h2));
}

}  // namespace weno
