// wos_math.cuh -- scalar math of one walk-on-spheres step, for FP32 and FP64.
//
//   * Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the
//     conversion of its words to uniforms in (0,1).
//   * Modified Bessel functions I0, I1, K0, K1.  FP32: the polynomial
//     approximations of Abramowitz & Stegun 9.8.1-9.8.8.  FP64: power series
//     (DLMF 10.25.2, 10.31.1-2), the large-argument expansion (DLMF 10.40.1)
//     and the trapezoidal rule on K_nu(x) = int_0^inf e^{-x cosh t} cosh(nu t) dt
//     (DLMF 10.32.9), which converges geometrically for this integrand.
//   * The centred screened-Poisson Green's function of a ball (Supplemental
//     Sec. 1.1): P^B = sigma_bar |G|, |G|, and the radius of y ~ G/|G| by
//     safeguarded Newton on the radial CDF.
//
// Everything is __host__ __device__ so the same code can be checked on a CPU.
#pragma once

#if defined(__CUDACC_RTC__)
// runtime compilation (the problem-specialised walk kernel): device built-ins only
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#define INFINITY __int_as_float(0x7f800000)
#define NAN __int_as_float(0x7fffffff)
#else
#include <stdint.h>

#include <cmath>
#include <cstring>
#endif

#if defined(__CUDACC__)
#define WOS_HD __host__ __device__ __forceinline__
#else
#define WOS_HD inline
#endif

namespace wos {

// ---------------------------------------------------------------------------
// real-type helpers
// ---------------------------------------------------------------------------
// FP32 on the device uses the special-function unit (ex2/lg2/sin/cos.approx):
// relative errors ~1e-6 over the argument ranges of a walk step, far below the
// statistical error of any estimate, and no slow-path code in the kernel.
WOS_HD float w_exp(float x) {
#if defined(__CUDA_ARCH__)
  return __expf(x);
#else
  return expf(x);
#endif
}
WOS_HD double w_exp(double x) { return exp(x); }
WOS_HD float w_log(float x) {
#if defined(__CUDA_ARCH__)
  return __logf(x);
#else
  return logf(x);
#endif
}
WOS_HD double w_log(double x) { return log(x); }
WOS_HD float w_div(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
WOS_HD double w_div(double a, double b) { return a / b; }
WOS_HD float w_sqrt(float x) { return sqrtf(x); }
WOS_HD double w_sqrt(double x) { return sqrt(x); }
WOS_HD float w_rsqrt(float x) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}
WOS_HD double w_rsqrt(double x) { return 1.0 / sqrt(x); }
// sqrt(x) for x >= 0 as x * rsqrt(x) on the device (two instructions against the IEEE-rounded
// square root's longer sequence; a few ulp, where the walk's uses need ~1e-6).  x below the
// smallest normal float is raised to it, so x = 0 gives ~1e-19 instead of 0 * inf.
WOS_HD float w_sqrt_fast(float x) {
#if defined(__CUDA_ARCH__)
  x = fmaxf(x, 1.17549435e-38f);
  return x * rsqrtf(x);
#else
  return sqrtf(x);
#endif
}
WOS_HD double w_sqrt_fast(double x) { return sqrt(x); }
WOS_HD float w_sin(float x) {
#if defined(__CUDA_ARCH__)
  return __sinf(x);
#else
  return sinf(x);
#endif
}
WOS_HD double w_sin(double x) { return sin(x); }
WOS_HD float w_cos(float x) {
#if defined(__CUDA_ARCH__)
  return __cosf(x);
#else
  return cosf(x);
#endif
}
WOS_HD double w_cos(double x) { return cos(x); }
WOS_HD void w_sincos(float x, float* s, float* c) {
#if defined(__CUDA_ARCH__)
  __sincosf(x, s, c);
#else
  *s = sinf(x);
  *c = cosf(x);
#endif
}
WOS_HD void w_sincos(double x, double* s, double* c) {
#if defined(__CUDA_ARCH__)
  sincos(x, s, c);
#else
  *s = sin(x);
  *c = cos(x);
#endif
}
// sin(2 pi u), cos(2 pi u) for u in (0,1)
WOS_HD void w_sincospi2(float u, float* s, float* c) {
#if defined(__CUDA_ARCH__)
  __sincosf(6.2831853071795865f * u - 3.1415926535897932f, s, c);  // angle in (-pi, pi)
  *s = -*s;
  *c = -*c;
#else
  *s = sinf(6.283185307179586f * u);
  *c = cosf(6.283185307179586f * u);
#endif
}
WOS_HD void w_sincospi2(double u, double* s, double* c) {
#if defined(__CUDA_ARCH__)
  sincospi(2.0 * u, s, c);
#else
  *s = sin(6.283185307179586476925 * u);
  *c = cos(6.283185307179586476925 * u);
#endif
}
WOS_HD float w_cbrt(float x) { return cbrtf(x); }
WOS_HD double w_cbrt(double x) { return cbrt(x); }
WOS_HD float w_expm1(float x) { return expm1f(x); }
WOS_HD double w_expm1(double x) { return expm1(x); }
WOS_HD float w_asin(float x) { return asinf(x); }
WOS_HD double w_asin(double x) { return asin(x); }
WOS_HD float w_fabs(float x) { return fabsf(x); }
WOS_HD double w_fabs(double x) { return fabs(x); }
WOS_HD float w_fmax(float a, float b) { return fmaxf(a, b); }
WOS_HD double w_fmax(double a, double b) { return fmax(a, b); }
WOS_HD float w_fmin(float a, float b) { return fminf(a, b); }
WOS_HD double w_fmin(double a, double b) { return fmin(a, b); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

WOS_HD void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
#if defined(__CUDA_ARCH__)
  *hi = __umulhi(a, b);
  *lo = a * b;
#else
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
#endif
}

WOS_HD U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c.x, &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c.z, &hi1, &lo1);
    U4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The same generator with its ten rounds' keys given: rk[2r], rk[2r + 1] = (k0, k1) plus r
// times the two Weyl increments, as the loop above advances them.
WOS_HD void philox_round_keys(uint64_t seed, uint32_t rk[20]) {
  uint32_t k0 = (uint32_t)(seed & 0xffffffffull), k1 = (uint32_t)(seed >> 32);
  for (int round = 0; round < 10; ++round) {
    rk[2 * round] = k0;
    rk[2 * round + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}
WOS_HD U4 philox4x32_10_rk(U4 c, const uint32_t (&rk)[20]) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c.x, &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c.z, &hi1, &lo1);
    U4 n;
    n.x = hi1 ^ c.y ^ rk[2 * round];
    n.y = lo1;
    n.z = hi0 ^ c.w ^ rk[2 * round + 1];
    n.w = lo0;
    c = n;
  }
  return c;
}

// uniforms in (0,1): FP32 keeps the top 24 bits, FP64 all 32
template <typename R>
WOS_HD R to_uniform(uint32_t x);
// FP32: ((x >> 9) + 1/2) 2^-23, built from the bits -- the 23 high bits as the mantissa of
// a float in [1, 2), minus (1 - 2^-24), both exact -- with an OR and a subtraction instead
// of an integer-to-float conversion.  The FP32 walks' parity with the oracle is
// statistical, so their uniforms need not be the FP64 ones rounded.
WOS_HD float u32_bits_as_float(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
WOS_HD int32_t f_as_i_bits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_int(f);
#else
  int32_t i;
  memcpy(&i, &f, 4);
  return i;
#endif
}
template <>
WOS_HD float to_uniform<float>(uint32_t x) {
  return u32_bits_as_float(0x3f800000u | (x >> 9)) - 0.99999994039535522461f;
}
template <>
WOS_HD double to_uniform<double>(uint32_t x) {
  return ((double)x + 0.5) * 2.3283064365386962890625e-10;
}

// 3D steps draw six uniforms from one Philox block: the top 21 bits of each word, and two
// more fields of 21 bits from the words' low bits, ((w0 & 0x7ff) << 10) | (w2 & 0x3ff) and
// ((w1 & 0x7ff) << 10) | (w3 & 0x3ff) -- disjoint bits, so the six are independent.  A
// field f gives (f + 1/2) 2^-21 in (0, 1), exact and equal in FP32 and FP64.
template <typename R>
WOS_HD R u21(uint32_t f);
template <>
WOS_HD float u21<float>(uint32_t f) {
  return u32_bits_as_float(0x3f800000u | (f << 2)) - 0.99999976158142089844f;  // 1 + f 2^-21, minus 1 - 2^-22
}
template <>
WOS_HD double u21<double>(uint32_t f) {
  return ((double)f + 0.5) * 4.76837158203125e-07;
}
WOS_HD void split21(U4 r, uint32_t* f) {
  f[0] = r.x >> 11;
  f[1] = r.y >> 11;
  f[2] = r.z >> 11;
  f[3] = r.w >> 11;
  f[4] = ((r.x & 0x7ffu) << 10) | (r.z & 0x3ffu);
  f[5] = ((r.y & 0x7ffu) << 10) | (r.w & 0x3ffu);
}

// ---------------------------------------------------------------------------
// Bessel functions, FP32: Abramowitz & Stegun 9.8.1-9.8.8 (|error| <~ 2e-7 on
// the scaled quantities).  *_s are exponentially scaled: i0s(x) = e^{-x} I0(x),
// k0s(x) = e^{x} K0(x).
// ---------------------------------------------------------------------------
WOS_HD float as_i0_small(float x) {  // x <= 3.75
  float t = x * (1.0f / 3.75f);
  t *= t;
  return 1.0f + t * (3.5156229f + t * (3.0899424f + t * (1.2067492f + t * (0.2659732f +
         t * (0.0360768f + t * 0.0045813f)))));
}
WOS_HD float as_i1_small(float x) {  // x <= 3.75
  float t = x * (1.0f / 3.75f);
  t *= t;
  return x * (0.5f + t * (0.87890594f + t * (0.51498869f + t * (0.15084934f + t * (0.02658733f +
              t * (0.00301532f + t * 0.00032411f))))));
}
WOS_HD float as_i0s_large(float x) {  // x >= 3.75: e^{-x} I0(x)
  float t = w_div(3.75f, x);
  float p = 0.39894228f + t * (0.01328592f + t * (0.00225319f + t * (-0.00157565f + t * (0.00916281f +
            t * (-0.02057706f + t * (0.02635537f + t * (-0.01647633f + t * 0.00392377f)))))));
  return p * w_rsqrt(x);
}
WOS_HD float as_i1s_large(float x) {  // x >= 3.75: e^{-x} I1(x)
  float t = w_div(3.75f, x);
  float p = 0.39894228f + t * (-0.03988024f + t * (-0.00362018f + t * (0.00163801f + t * (-0.01031555f +
            t * (0.02282967f + t * (-0.02895312f + t * (0.01787654f - t * 0.00420059f)))))));
  return p * w_rsqrt(x);
}
// K0(x) + ln(x/2) I0(x), x <= 2
WOS_HD float as_k0_poly(float x) {
  float t = 0.25f * x * x;
  return -0.57721566f + t * (0.42278420f + t * (0.23069756f + t * (0.03488590f + t * (0.00262698f +
         t * (0.00010750f + t * 0.0000074f)))));
}
// x K1(x) - x ln(x/2) I1(x) - 1, x <= 2
WOS_HD float as_k1_poly(float x) {
  float t = 0.25f * x * x;
  return t * (0.15443144f + t * (-0.67278579f + t * (-0.18156897f + t * (-0.01919402f +
         t * (-0.00110404f - t * 0.00004686f)))));
}
WOS_HD float as_k0s_large(float x) {  // x >= 2: e^{x} K0(x)
  float t = w_div(2.0f, x);
  float p = 1.25331414f + t * (-0.07832358f + t * (0.02189568f + t * (-0.01062446f + t * (0.00587872f +
            t * (-0.00251540f + t * 0.00053208f)))));
  return p * w_rsqrt(x);
}
WOS_HD float as_k1s_large(float x) {  // x >= 2: e^{x} K1(x)
  float t = w_div(2.0f, x);
  float p = 1.25331414f + t * (0.23498619f + t * (-0.03655620f + t * (0.01504268f + t * (-0.00780353f +
            t * (0.00325614f - t * 0.00068245f)))));
  return p * w_rsqrt(x);
}

// ---------------------------------------------------------------------------
// Bessel functions, FP64
// ---------------------------------------------------------------------------
// sum_k (x^2/4)^k / (k! (k+nu)!) for nu = 0, 1
WOS_HD double ser_i(int nu, double x) {
  double q = 0.25 * x * x, term = 1.0, acc = 1.0;
  for (int k = 1; k < 200; ++k) {
    term *= q / ((double)k * (double)(k + nu));
    acc += term;
    if (term < 1e-18 * acc) break;
  }
  return acc;
}
// e^{-x} I_nu(x) sqrt(2 pi x) by the large-argument expansion, x >= 20
WOS_HD double asym_is(int nu, double x) {
  double mu = 4.0 * nu * nu, term = 1.0, acc = 1.0;
  for (int k = 1; k < 60; ++k) {
    double f = (2.0 * k - 1.0);
    double nt = -term * (mu - f * f) / (k * 8.0 * x);
    if (fabs(nt) > fabs(term)) break;
    term = nt;
    acc += term;
    if (fabs(term) < 1e-18 * fabs(acc)) break;
  }
  return acc;
}
WOS_HD double d_i0s(double x) {  // e^{-x} I0(x)
  if (x < 20.0) return exp(-x) * ser_i(0, x);
  return asym_is(0, x) / sqrt(6.283185307179586476925 * x);
}
WOS_HD double d_i1s(double x) {  // e^{-x} I1(x)
  if (x < 20.0) return exp(-x) * 0.5 * x * ser_i(1, x);
  return asym_is(1, x) / sqrt(6.283185307179586476925 * x);
}
WOS_HD double d_i0(double x) { return (x < 20.0) ? ser_i(0, x) : exp(x) * d_i0s(x); }
WOS_HD double d_i1(double x) { return (x < 20.0) ? 0.5 * x * ser_i(1, x) : exp(x) * d_i1s(x); }
// e^{x} K_nu(x) = int_0^inf e^{-x (cosh t - 1)} cosh(nu t) dt, trapezoid with step h
// The integrand is analytic in a strip whose useful width shrinks like 1/sqrt(x),
// so the step is h = min(1/8, 0.6/sqrt(x)) for an error below e^{-50}.
WOS_HD double trap_ks(int nu, double x) {
  const double h = fmin(0.125, 0.6 / sqrt(x));
  double acc = 0.5;
  for (int j = 1; j < 2000; ++j) {
    double t = j * h;
    double e = exp(-x * (cosh(t) - 1.0));
    acc += e * (nu ? cosh(t) : 1.0);
    if (e < 1e-19) break;
  }
  return acc * h;
}
// K0(x) + ln(x/2) I0(x) = -gamma I0(x) + sum_{k>=1} H_k (x^2/4)^k/(k!)^2 (DLMF 10.31.2)
WOS_HD double d_k0_small(double x) {
  const double eg = 0.57721566490153286061;
  double q = 0.25 * x * x, term = 1.0, H = 0.0, s = 0.0, i0 = 1.0;
  for (int k = 1; k < 100; ++k) {
    term *= q / ((double)k * k);
    H += 1.0 / k;
    s += H * term;
    i0 += term;
    if (term < 1e-19) break;
  }
  return -(log(0.5 * x) + eg) * i0 + s;
}
// 1 - x K1(x) by DLMF 10.31.1 (n = 1), x <= 2:
//   1 - x K1(x) = -x ln(x/2) I1(x) + (x^2/4) sum_k (psi(k+1) + psi(k+2)) (x^2/4)^k / (k!(k+1)!)
WOS_HD double d_1m_xk1_small(double x) {
  const double eg = 0.57721566490153286061;
  double q = 0.25 * x * x, term = 1.0, H = 0.0, acc = 0.0, i1s = 0.0;
  for (int k = 0; k < 100; ++k) {
    if (k > 0) {
      term *= q / ((double)k * (k + 1));
      H += 1.0 / k;
    }
    double psi1 = -eg + H, psi2 = -eg + H + 1.0 / (k + 1);
    acc += (psi1 + psi2) * term;
    i1s += term;
    if (k > 2 && term < 1e-20) break;
  }
  double i1 = 0.5 * x * i1s;
  return -x * log(0.5 * x) * i1 + q * acc;
}
WOS_HD double d_k0(double x) { return (x <= 2.0) ? d_k0_small(x) : exp(-x) * trap_ks(0, x); }
WOS_HD double d_k1(double x) { return (x <= 2.0) ? (1.0 - d_1m_xk1_small(x)) / x : exp(-x) * trap_ks(1, x); }

// ---------------------------------------------------------------------------
// 1/n! as a compile-time constant, and sum_{k<NT} t^k / (2k + OFF)! by Horner's rule with
// the coefficients folded in (one FMA per term).
// ---------------------------------------------------------------------------
template <int N>
struct RFact {
  static constexpr double v = RFact<N - 1>::v / N;
};
template <>
struct RFact<0> {
  static constexpr double v = 1.0;
};
template <typename R, int OFF, int K, int NT, bool LAST = (K + 1 >= NT)>
struct FactPoly {
  static WOS_HD R eval(R t) { return R(RFact<2 * K + OFF>::v) + t * FactPoly<R, OFF, K + 1, NT>::eval(t); }
};
template <typename R, int OFF, int K, int NT>
struct FactPoly<R, OFF, K, NT, true> {
  static WOS_HD R eval(R) { return R(RFact<2 * K + OFF>::v); }
};

// ---------------------------------------------------------------------------
// Green's function of Lap - sb on a ball of radius R centred at x
// (Supplemental 1.1).  a = sqrt(sb) R.
//   |G| = R^2 q(a) with 3D q = (1 - a/sinh a)/a^2, 2D q = (1 - 1/I0(a))/a^2,
//   P^B = sb |G| = a^2 q(a).
// ---------------------------------------------------------------------------
WOS_HD float green_q3(float a) {
  // q = (1 - a/sinh a)/a^2 = S(a) / (a^2 sinh a), S(a) = sinh a - a.  a < 1: S(a) = a^3 P(a^2)
  // and sinh a = a (1 + a^2 P(a^2)), P(t) = sum t^k/(2k+3)! (the radial CDF's series, which
  // shares P(a^2) and e^{-a} with this); a >= 1: exponentials scaled by 2e^{-a}.  Chosen by a
  // select, not a branch.
  const float t = a * a;
  const float P = FactPoly<float, 3, 0, 5>::eval(t);
  const float e = w_exp(-a);
  const float qs = w_div(P, 1.0f + t * P);
  const float ql = w_div((1.0f - e * e) - 2.0f * a * e, t * (1.0f - e * e));
  return (a < 1.0f) ? qs : ql;
}
WOS_HD double green_q3(double a) {
  if (a < 1.0) {  // (sinh a - a)/(a^2 sinh a) by the series of sinh a - a
    double t = a * a, term = a, s = 0.0;
    for (int k = 1; k < 30; ++k) {
      term *= t / ((2.0 * k) * (2.0 * k + 1.0));
      s += term;
      if (term < 1e-19 * s) break;
    }
    if (a == 0.0) return 1.0 / 6.0;
    return s / (t * sinh(a));
  }
  double e = exp(-a);
  double ratio = 2.0 * a * e / (1.0 - e * e);
  return (1.0 - ratio) / (a * a);
}
WOS_HD float green_q2(float a) {
  if (a < 3.75f) {  // (I0 - 1)/a^2 / I0 with the series of I0 - 1
    float q = 0.25f * a * a;
    float s = 0.25f, term = 0.25f;  // (I0-1)/a^2 = 1/4 sum_{k>=1} q^(k-1)/(k!)^2
#pragma unroll
    for (int k = 2; k < 12; ++k) {
      term *= q * (1.0f / (float)(k * k));
      s += term;
    }
    return w_div(s, 1.0f + a * a * s);
  }
  float inv_i0 = w_div(w_exp(-a), as_i0s_large(a));  // 1/I0(a)
  return w_div(1.0f - inv_i0, a * a);
}
WOS_HD double green_q2(double a) {
  if (a == 0.0) return 0.25;
  if (a < 2.0) {
    double q = 0.25 * a * a, term = 1.0, s = 0.0;
    for (int k = 1; k < 60; ++k) {
      term *= q / ((double)k * k);
      s += term;
      if (term < 1e-19 * s) break;
    }
    return (s / (a * a)) / (1.0 + s);
  }
  return (1.0 - exp(-a) / d_i0s(a)) / (a * a);
}

template <int DIM, typename R>
WOS_HD R green_q(R a) {
  return DIM == 2 ? green_q2(a) : green_q3(a);
}

// ---------------------------------------------------------------------------
// Exponentially scaled I0, I1, K0, K1 at one argument:
//   i0s = e^{-x} I0(x), i1s = e^{-x} I1(x), k0s = e^{x} K0(x), k1s = e^{x} K1(x).
// ---------------------------------------------------------------------------
WOS_HD void bessel_scaled(float x, float* i0s, float* i1s, float* k0s, float* k1s) {
  float ex = w_exp(-x);
  if (x < 3.75f) {
    *i0s = as_i0_small(x) * ex;
    *i1s = as_i1_small(x) * ex;
  } else {
    *i0s = as_i0s_large(x);
    *i1s = as_i1s_large(x);
  }
  if (x <= 2.0f) {
    float lt = w_log(0.5f * x);
    float k0 = as_k0_poly(x) - lt * as_i0_small(x);
    float k1 = w_div(1.0f + as_k1_poly(x) + x * lt * as_i1_small(x), x);
    *k0s = w_div(k0, ex);
    *k1s = w_div(k1, ex);
  } else {
    *k0s = as_k0s_large(x);
    *k1s = as_k1s_large(x);
  }
}
WOS_HD void bessel_scaled(double x, double* i0s, double* i1s, double* k0s, double* k1s) {
  *i0s = d_i0s(x);
  *i1s = d_i1s(x);
  if (x <= 2.0) {
    double ex = exp(x);
    *k0s = d_k0_small(x) * ex;
    *k1s = (1.0 - d_1m_xk1_small(x)) / x * ex;
  } else {
    *k0s = trap_ks(0, x);
    *k1s = trap_ks(1, x);
  }
}

// ---------------------------------------------------------------------------
// Gradients at the centre of the ball (Supplemental 1.3) as ratios to the centred
// densities:  grad_x G(x, y) = gG G(x, y) (y - x)/r,  grad_x P(x, z) = gP P(x, z) (z - x)/R.
// Returned scaled by the radius, gGR = R gG and gPR = R gP, for a = sqrt(sb) R and
// rho = r/R (t = a rho).  Supplemental Sec. 2 weights the first ball's samples by them.
// 3D, with c(z) = cosh z - sinh z/z and kk(z) = e^{-z}(1 + 1/z), the printed
// expressions give
//   4 pi G = sinh(a - t)/(r sinh a),     4 pi |grad G| = (s/r)(kk(t) - c(t) kk(a)/c(a)),
//   4 pi R^2 P = a/sinh a,               4 pi R^2 |grad P| = s a/c(a),
// so gPR = a sinh(a)/c(a) and gGR = gPR (kk(t) c(a) - c(t) kk(a))/sinh(a - t), written
// below with e^{-z}-scaled c^ = e^{-z} c, s^ = e^{-z} sinh (no overflow at large a):
//   gGR = gPR [(1 + 1/t) c^(a) - e^{-2(a-t)} c^(t)(1 + 1/a)] / s^(a - t).
// c(z) is summed as its series sum_{n>=1} 2n z^{2n}/(2n+1)! below z = 1/2, where
// cosh z - sinh z/z cancels.  2D, from the printed K1/I1 forms:
//   gPR = a I0(a)/I1(a),
//   gGR = a [K1(t) - K1(a) I1(t)/I1(a)] / [K0(t) - K0(a) I0(t)/I0(a)].
// For a -> 0 (Laplace ball) they tend to gPR = DIM and gGR = (1 + rho + rho^2)/rho (3D),
// (1/rho - rho)/ln(1/rho) (2D); used below a = 1e-4.
// ---------------------------------------------------------------------------
template <typename R>
WOS_HD R grad_chat(R z) {  // e^{-z} (cosh z - sinh z / z)
  if (z < R(0.5)) {
    R z2 = z * z, term = z2 * R(1.0 / 3.0), acc = term;
#pragma unroll
    for (int n = 1; n < 8; ++n) {
      term *= z2 / R((2 * n) * (2 * n + 3));
      acc += term;
    }
    return acc * w_exp(-z);
  }
  R e2 = w_exp(R(-2) * z);
  return R(0.5) * (R(1) + e2) - R(0.5) * (R(1) - e2) / z;
}

template <int DIM, typename R>
WOS_HD void grad_ratios(R a, R rho, R* gGR, R* gPR) {
  if (DIM == 3) {
    if (a < R(1e-4)) {
      *gPR = R(3);
      *gGR = (R(1) + rho + rho * rho) / rho;
      return;
    }
    R t = a * rho;
    R ca = grad_chat(a), ct = grad_chat(t);
    R sa = R(-0.5) * w_expm1(R(-2) * a);
    R sat = R(-0.5) * w_expm1(R(-2) * (a - t));
    R gp = a * sa / ca;
    R num = (R(1) + R(1) / t) * ca - w_exp(R(-2) * (a - t)) * ct * (R(1) + R(1) / a);
    *gPR = gp;
    *gGR = gp * num / sat;
    return;
  }
  if (a < R(1e-4)) {
    *gPR = R(2);
    *gGR = (R(1) / rho - rho) / (-w_log(rho));
    return;
  }
  R t = a * rho;
  R i0a, i1a, k0a, k1a, i0t, i1t, k0t, k1t;
  bessel_scaled(a, &i0a, &i1a, &k0a, &k1a);
  bessel_scaled(t, &i0t, &i1t, &k0t, &k1t);
  R e = w_exp(R(-2) * (a - t));
  *gPR = a * i0a / i1a;
  *gGR = a * (k1t - k1a * i1t / i1a * e) / (k0t - k0a * i0t / i0a * e);
}

// ---------------------------------------------------------------------------
// R |G'(r)/G(r)| of the centred Green's function (Supplemental 1.1), rho = r/R,
// a = sqrt(sb) R, t = a rho: the weight of an extra drift (see coeffs).
//   3D: G ~ sinh(a - t)/r          -> a / tanh(a - t) + 1/rho   (Laplace: 1/(1 - rho) + 1/rho)
//   2D: G ~ K0(t) - cK I0(t) ...   -> a (k1s(t) + cK e^{2(t-a)} i1s(t)) / (k0s(t) - cK e^{2(t-a)} i0s(t))
//                                      (Laplace: 1/(rho ln(1/rho)))
// ---------------------------------------------------------------------------
template <int DIM, typename R>
WOS_HD R green_dlog_r(R a, R rho) {
  if (DIM == 3) {
    if (a < R(1e-4)) return R(1) / (R(1) - rho) + R(1) / rho;
    R dl = a * (R(1) - rho);
    R th = (dl < R(20)) ? (-w_expm1(R(-2) * dl)) / (R(1) + w_exp(R(-2) * dl)) : R(1);  // tanh(dl)
    return a / th + R(1) / rho;
  }
  if (a < R(1e-4)) return R(1) / (rho * (-w_log(rho)));
  R t = a * rho;
  R i0a, i1a, k0a, k1a, i0t, i1t, k0t, k1t;
  bessel_scaled(a, &i0a, &i1a, &k0a, &k1a);
  bessel_scaled(t, &i0t, &i1t, &k0t, &k1t);
  R cK = k0a / i0a, e = w_exp(R(-2) * (a - t));
  return a * (k1t + cK * e * i1t) / (k0t - cK * e * i0t);
}

// ---------------------------------------------------------------------------
// Next-flight kernels (Sec. 5.2): the approximate off-centred Green's function and
// Poisson kernel of Supplemental 1.2 on a ball of radius R (centre c), in terms of
//   Q(r): the bracket of the centred G (G = Q/(2 pi) in 2D, Q/(4 pi) in 3D), any r > 0,
//   V(r) = -Q'(r):
//   G(x, y) = (Q(|w|) - Q(rho')) / (2 pi | 4 pi),
//   P(x, z) = (V(|w|)(R^2 - u.v)/(|w| R) + V(rho') u.v / R^2) / (2 pi | 4 pi),
// with u = x - c, v = y - c (|v| = R for P), w = v - u, rho' = (R^2 - u.v)/R.
// Overflow-free forms (t = s r, a = s R):
//   3D  Q = (e^{-t} - e^{t-2a}) / (r (1 - e^{-2a}))             [= sinh(a-t)/(r sinh a)]
//       V = (s/r)(e^{-t}(1 + 1/t) + 2 e^{t-2a} c^(t) / (1 - e^{-2a})),  c^ = e^{-t}(cosh t - sinh t/t)
//   2D  Q = e^{-t} k0s(t) - cK e^{t-2a} i0s(t),   V = s (e^{-t} k1s(t) + cK e^{t-2a} i1s(t)),
//       cK = k0s(a)/i0s(a)  (e^{-x}-scaled I, e^{x}-scaled K)
// and the Laplace forms (3D 1/r - 1/R, 1/r^2; 2D ln(R/r), 1/r) for a < 1e-7.
// ---------------------------------------------------------------------------
template <int DIM, typename R>
struct NfBall {
  R s, a, Rb;
  R inv_den;  // 3D: 1 / (1 - e^{-2a})
  R cK;       // 2D: k0s(a) / i0s(a)
  bool lap;
  R pcentre;  // P^dB of the centred ball: P(c, z) |dB|

  WOS_HD void init(R s_, R Rb_) {
    s = s_;
    Rb = Rb_;
    a = s * Rb;
    lap = !(a >= R(1e-7));
    inv_den = R(0);
    cK = R(0);
    if (lap) {
      pcentre = R(1);
      return;
    }
    if (DIM == 3) {
      inv_den = R(1) / (-w_expm1(R(-2) * a));
      pcentre = R(2) * a * w_exp(-a) * inv_den;  // a / sinh a
    } else {
      R i0s, i1s, k0s, k1s;
      bessel_scaled(a, &i0s, &i1s, &k0s, &k1s);
      cK = k0s / i0s;
      pcentre = w_exp(-a) / i0s;                 // 1 / I0(a)
    }
  }
  WOS_HD R Q(R r) const {
    if (DIM == 3) {
      if (lap) return R(1) / r - R(1) / Rb;
      R t = s * r;
      // e^{-t} - e^{t-2a}, factored on the side that cannot overflow
      R num = (t <= a) ? w_exp(-t) * (-w_expm1(R(-2) * (a - t))) : -w_exp(t - R(2) * a) * (-w_expm1(R(-2) * (t - a)));
      return num * inv_den / r;
    }
    if (lap) return w_log(Rb / r);
    R t = s * r;
    R i0s, i1s, k0s, k1s;
    bessel_scaled(t, &i0s, &i1s, &k0s, &k1s);
    return w_exp(-t) * k0s - cK * w_exp(t - R(2) * a) * i0s;
  }
  WOS_HD R V(R r) const {
    if (DIM == 3) {
      if (lap) return R(1) / (r * r);
      R t = s * r;
      return s / r * (w_exp(-t) * (R(1) + R(1) / t) + R(2) * w_exp(t - R(2) * a) * grad_chat(t) * inv_den);
    }
    if (lap) return R(1) / r;
    R t = s * r;
    R i0s, i1s, k0s, k1s;
    bessel_scaled(t, &i0s, &i1s, &k0s, &k1s);
    return s * (w_exp(-t) * k1s + cK * w_exp(t - R(2) * a) * i1s);
  }
  // G(c + u, c + v)
  WOS_HD R G(const R* u, const R* v) const {
    R w2 = R(0), uv = R(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      R wi = v[i] - u[i];
      w2 += wi * wi;
      uv += u[i] * v[i];
    }
    const R cd = (DIM == 2) ? R(0.15915494309189533577) : R(0.07957747154594766788);
    return cd * (Q(w_sqrt(w2)) - Q((Rb * Rb - uv) / Rb));
  }
  // P(c + u, c + v), |v| = R
  WOS_HD R P(const R* u, const R* v) const {
    R w2 = R(0), uv = R(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      R wi = v[i] - u[i];
      w2 += wi * wi;
      uv += u[i] * v[i];
    }
    const R cd = (DIM == 2) ? R(0.15915494309189533577) : R(0.07957747154594766788);
    R nw = w_sqrt(w2), r2 = Rb * Rb;
    return cd * (V(nw) * (r2 - uv) / (nw * Rb) + V((r2 - uv) / Rb) * uv / r2);
  }
};

// ---------------------------------------------------------------------------
// Next-flight kernels as the series of Supplemental 1.2 (the exact off-centred kernels,
// truncated at N terms), for a ball of radius R centred at c, k = sqrt(sigma_bar),
// a = kR, u = x - c, v = y - c:
//   G(x, y) = Phi(|v - u|) - H(u, v),  Phi = e^{-kd}/(4 pi d) (3D), K_0(kd)/(2 pi) (2D),
//   H = 1/(4 pi R) sum_{n<N} (2n+1) P_n(cos) p_n t_n(k|u|) t_n(k|v|)            (3D)
//     = 1/(2 pi)   sum_{|n|<N} cos(n th) p_n t_n(k|u|) t_n(k|v|)                 (2D)
//   P(y, z) = 1/(4 pi R^2) sum_{n<N} (2n+1) P_n(cos) t_n(k|v|)                   (3D)
//           = 1/(2 pi R)   sum_{|n|<N} cos(n th) t_n(k|v|)                        (2D)
// with t_n(z) = i_n(z)/i_n(a) (modified spherical Bessel; 2D I_n(z)/I_n(a)) and
// p_n = a k_n(a) i_n(a) (2D I_n(a) K_n(a)).  The free-space kernel in closed form keeps
// G's singularity exact; the regular part H and the whole P are truncated, i.e. projected
// on the angular harmonics of degree < N.
// Evaluation:
//  * the ratios rho_n(z) = i_n(z)/i_{n-1}(z) by the backward recurrence
//    rho_n = 1 / ((2n+1)/z + rho_{n+1}) (2D: 2n/z), the stable direction for i_n, started
//    with rho = 0 at n0 = N + 12 + a or above (the error shrinks by rho_n^2 per step);
//  * t_{n-1} = t_n rho_n(a) / rho_n(z), run downwards from an arbitrary t at the top and
//    rescaled at the end by the closed form t_0 (3D (a/z) sinh z / sinh a, 2D I_0(z)/I_0(a));
//  * p_n upwards from p_0 (3D (1 - e^{-2a})/(2a), 2D I_0(a) K_0(a)) by
//    p_n = rho_n(a) (1/a - rho_n(a) p_{n-1}), which follows from the cross products
//    i_{n-1} k_n + i_n k_{n-1} = 1/a^2 (2D: I_{n-1} K_n + I_n K_{n-1} = 1/a) and damps
//    errors (factor rho_n^2 per step);
//  * the Legendre / cosine sums by Clenshaw's recurrence, downwards with the t's.
// p_n and rho_n(a) depend on the ball only: nf_series_ball fills them once per ball.
// ---------------------------------------------------------------------------
constexpr int kNfSeriesMax = 64;  // largest N

// (2n+1) in 3D, 2n in 2D: the recurrence coefficient of the ratios
template <int DIM, typename R>
WOS_HD R nf_rec_coef(int n) {
  return (DIM == 3) ? R(2 * n + 1) : R(2 * n);
}

// rho_n(a) for 1 <= n < N into ra[n], p_n for 0 <= n < N into pn[n]
template <int DIM, typename R>
WOS_HD void nf_series_ball(R a, int N, R* pn, R* ra) {
  const R inv_a = w_div(R(1), a);
  const int n0 = N + 12 + (int)w_fmin(a, R(4096));
  R rho = R(0);
  for (int n = n0; n >= 1; --n) {
    rho = w_div(R(1), nf_rec_coef<DIM, R>(n) * inv_a + rho);
    if (n < N) ra[n] = rho;
  }
  if (DIM == 3) {
    pn[0] = R(-0.5) * w_expm1(R(-2) * a) * inv_a;
  } else {
    R i0s, i1s, k0s, k1s;
    bessel_scaled(a, &i0s, &i1s, &k0s, &k1s);
    pn[0] = i0s * k0s;
  }
  for (int n = 1; n < N; ++n) pn[n] = ra[n] * (inv_a - ra[n] * pn[n - 1]);
}

// t_0(z) = i_0(z)/i_0(a) (2D I_0(z)/I_0(a)), 0 <= z <= a
template <int DIM, typename R>
WOS_HD R nf_series_t0(R z, R a) {
  if (DIM == 3) {
    // (a/z) sinh z / sinh a = (a/z) e^{z-a} (1 - e^{-2z}) / (1 - e^{-2a}); a/sinh a at z = 0
    const R den = -w_expm1(R(-2) * a);
    if (!(z > R(0))) return R(2) * a * w_exp(-a) / den;
    return a / z * w_exp(z - a) * (-w_expm1(R(-2) * z)) / den;
  }
  R i0z, i1z, k0z, k1z, i0a, i1a, k0a, k1a;
  bessel_scaled(z, &i0z, &i1z, &k0z, &k1z);
  bessel_scaled(a, &i0a, &i1a, &k0a, &k1a);
  return i0z / i0a * w_exp(z - a);
}

// the last index whose terms matter at geometric rate q (terms shrink like q^n; below
// 2^-40 relative (2^-64 for FP64) they are dropped), capped at N - 1
template <typename R>
WOS_HD int nf_series_last(R q, int N) {
  if (!(q > R(0))) return 0;
  if (q > R(0.5)) return N - 1;
  const R bits = (sizeof(R) == 4) ? R(40) : R(64);
  const R m = bits / (-w_log(q) * R(1.44269504088896340736));  // bits / -log2(q)
  return (m < R(N - 1)) ? (int)m + 1 : N - 1;
}

// For G(c + u, c + v) = Phi - H: its regular part H and the free-space kernel Phi(|v - u|);
// and P(c + v, c + zp) (|zp| = R); from one downward sweep.  n0 >= the ball's N + 12 + a
// (the caller may pass a larger one, e.g. the largest of its warp, so that the sweep's
// index is the same on every lane).
template <int DIM, typename R>
WOS_HD void nf_series_eval(R k, R a, R Rb, int N, int n0, const R* pn, const R* ra, const R* u, const R* v,
                           const R* zp, R* H, R* Phi, R* P) {
  R r1s = R(0), r2s = R(0), uv = R(0), vz = R(0), d2 = R(0);
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    r1s += u[i] * u[i];
    r2s += v[i] * v[i];
    uv += u[i] * v[i];
    vz += v[i] * zp[i];
    const R w = v[i] - u[i];
    d2 += w * w;
  }
  const R r1 = w_sqrt(r1s), r2 = w_sqrt(r2s), d = w_sqrt(d2);
  const R muH = (r1 > R(0) && r2 > R(0)) ? w_fmax(R(-1), w_fmin(R(1), uv / (r1 * r2))) : R(0);
  const R muP = (r2 > R(0)) ? w_fmax(R(-1), w_fmin(R(1), vz / (r2 * Rb))) : R(0);
  const R z1 = k * r1, z2 = k * r2;
  // 1/z, 0 at the centre (only the n = 0 terms remain there: the sweep leaves t alone)
  const R iz1 = (z1 > R(0)) ? w_div(R(1), z1) : R(0), iz2 = (z2 > R(0)) ? w_div(R(1), z2) : R(0);
  const int lastH = nf_series_last<R>(r1 * r2 / (Rb * Rb), N);
  const int lastP = nf_series_last<R>(r2 / Rb, N);
  const R big = R(1073741824.0), small = R(1.0 / 1073741824.0);  // 2^30, 2^-30
  R rho1 = R(0), rho2 = R(0), t1 = R(1), t2 = R(1);
  R bH1 = R(0), bH2 = R(0), bP1 = R(0), bP2 = R(0);
  R inv_n2 = w_div(R(1), R(n0 + 2));  // 1/(n+2) of the first step
  for (int n = n0; n >= 1; --n) {
    const R c = nf_rec_coef<DIM, R>(n);
    const R s1 = (z1 > R(0)) ? c * iz1 + rho1 : R(1), s2 = (z2 > R(0)) ? c * iz2 + rho2 : R(1);
    rho1 = w_div(R(1), s1);
    rho2 = w_div(R(1), s2);
    const R inv_n1 = w_div(R(1), R(n + 1));
    // Clenshaw coefficients of term n: 3D Legendre alpha_n = (2n+1) mu/(n+1), beta_{n+1} =
    // -(n+1)/(n+2); 2D cosines alpha_n = 2 mu, beta = -1
    const R aH = (DIM == 3) ? R(2 * n + 1) * muH * inv_n1 : R(2) * muH;
    const R aP = (DIM == 3) ? R(2 * n + 1) * muP * inv_n1 : R(2) * muP;
    const R bt = (DIM == 3) ? -R(n + 1) * inv_n2 : R(-1);
    const R wn = (DIM == 3) ? R(2 * n + 1) : R(2);  // weight of term n (2D: n and -n)
    if (n <= lastP) {
      const R b0 = wn * t2 + aP * bP1 + bt * bP2;
      bP2 = bP1;
      bP1 = b0;
    }
    if (n <= lastH) {
      const R b0 = wn * pn[n] * t1 * t2 + aH * bH1 + bt * bH2;
      bH2 = bH1;
      bH1 = b0;
      t1 *= ra[n] * s1;  // t_{n-1}(z1)
      if (t1 > big) {
        t1 *= small;
        bH1 *= small;
        bH2 *= small;
      }
    }
    if (n <= lastP) {
      t2 *= ra[n] * s2;  // t_{n-1}(z2)
      if (t2 > big) {
        t2 *= small;
        bP1 *= small;
        bP2 *= small;
        bH1 *= small;
        bH2 *= small;
      }
    }
    inv_n2 = inv_n1;
  }
  // n = 0: alpha_0 = mu (both), beta_1 = -1/2 (3D) or -1 (2D)
  const R b1 = (DIM == 3) ? R(-0.5) : R(-1);
  const R SP = t2 + muP * bP1 + b1 * bP2;
  const R SH = pn[0] * t1 * t2 + muH * bH1 + b1 * bH2;
  const R n2 = nf_series_t0<DIM, R>(z2, a) / t2;
  const R n1 = nf_series_t0<DIM, R>(z1, a) / t1;
  if (DIM == 3) {
    const R c4 = R(0.07957747154594766788);  // 1/(4 pi)
    *P = c4 * SP * n2 / (Rb * Rb);
    *H = c4 * SH * n1 * n2 / Rb;
    *Phi = c4 * w_exp(-k * d) / d;
  } else {
    const R c2 = R(0.15915494309189533577);  // 1/(2 pi)
    R i0s, i1s, k0s, k1s;
    bessel_scaled(k * d, &i0s, &i1s, &k0s, &k1s);
    *P = c2 * SP * n2 / Rb;
    *H = c2 * SH * n1 * n2;
    *Phi = c2 * k0s * w_exp(-k * d);
  }
}

// In-ball points of the series walk: y = x + r w, w uniform on the unit sphere (circle),
// r in [0, r_m] (r_m the distance from x to the sphere along w) with density proportional
// to Phi(r) r^{d-1}.  Then p(y) = Phi(r) k^2 / h(k r_m) with
//   h(t) = 1 - e^{-t}(1 + t) (3D),  1 - t K_1(t) (2D),   h'(t) = t e^{-t},  t K_0(t),
// and G(x, y)/p(y) = (1 - H/Phi) h(k r_m) / sigma_bar <= 1/sigma_bar (0 <= G <= Phi): the
// throughput factor G/p (sigma_bar - sigma') stays at most 1 - sigma'/sigma_bar.
// Small t: 3D sum_{n>=2} (-1)^n (n-1) t^n / n!; 2D (DLMF 10.31.1 at n = 1)
//   1 - t K_1(t) = -t ln(t/2) I_1(t) + (t^2/4) sum_k (psi(k+1) + psi(k+2)) (t^2/4)^k / (k! (k+1)!).
template <int DIM, typename R>
WOS_HD R nf_free_h(R t) {
  if (DIM == 3) {
    if (t < R(0.5)) {
      R term = R(0.5) * t * t, sum = R(0);
      const int nmax = (sizeof(R) == 4) ? 12 : 24;
      for (int n = 2; n <= nmax; ++n) {
        sum += R(n - 1) * term;
        term *= -t / R(n + 1);
      }
      return sum;
    }
    return -w_expm1(-t) - t * w_exp(-t);
  }
  if (t < R(2)) {
    if (!(t > R(0))) return R(0);
    const R q = R(0.25) * t * t;
    R c = R(1), i1 = R(0), ps = R(0);
    R psi1 = R(-0.57721566490153286061), psi2 = R(0.42278433509846713939);  // psi(1), psi(2)
    const int kmax = (sizeof(R) == 4) ? 9 : 18;
    for (int kk = 0; kk <= kmax; ++kk) {
      i1 += c;
      ps += (psi1 + psi2) * c;
      psi1 += R(1) / R(kk + 1);
      psi2 += R(1) / R(kk + 2);
      c *= q / (R(kk + 1) * R(kk + 2));
    }
    return -t * w_log(R(0.5) * t) * (R(0.5) * t * i1) + q * ps;
  }
  R i0s, i1s, k0s, k1s;
  bessel_scaled(t, &i0s, &i1s, &k0s, &k1s);
  return R(1) - t * k1s * w_exp(-t);
}
template <int DIM, typename R>
WOS_HD R nf_free_hp(R t) {
  if (DIM == 3) return t * w_exp(-t);
  R i0s, i1s, k0s, k1s;
  bessel_scaled(t, &i0s, &i1s, &k0s, &k1s);
  return t * k0s * w_exp(-t);
}
// r in [0, rm] with h(k r) = U h(k rm): safeguarded Newton on t = k r (bracketed;
// FP64 runs to convergence, FP32 to a step of 1e-6 of t)
template <int DIM, typename R>
WOS_HD R nf_free_radius(R k, R rm, R U) {
  const R tm = k * rm, c = U * nf_free_h<DIM, R>(tm);
  const R tol = (sizeof(R) == 4) ? R(1e-6) : R(4e-16);
  const int itmax = (sizeof(R) == 4) ? 30 : 200;
  R lo = R(0), hi = tm, t = tm * w_sqrt(U);
  for (int it = 0; it < itmax; ++it) {
    const R f = nf_free_h<DIM, R>(t) - c;
    if (f == R(0)) break;
    if (f > R(0)) hi = t; else lo = t;
    const R dh = nf_free_hp<DIM, R>(t);
    R nt = (dh > R(0)) ? t - f / dh : R(0.5) * (lo + hi);
    if (!(nt >= lo && nt <= hi)) nt = R(0.5) * (lo + hi);
    const R step = w_fabs(nt - t);
    t = nt;
    if (step <= tol * t || hi - lo <= tol * t) break;
  }
  return t / k;
}

// ---------------------------------------------------------------------------
// Radial CDF F(rho) of y ~ G/|G|, rho = r/R, and its density, 3D.
//   N(rho) = a^2 int_0^rho s sinh(a(1-s)) ds, F = N(rho)/N(1).
// Integrating by parts, with v = 1 - rho, y = a v, x = a rho and S(y) = sinh y - y:
//   1 - F = [S(y) + x (cosh y - 1)] / S(a),   dF/drho = a x sinh(y) / S(a).
// Both terms of the numerator are >= 0, so 1 - F carries the relative accuracy of its
// parts at every a and rho.  Each part has two forms, and a select on its own argument
// (not a branch: every lane of a warp runs the same instructions) picks one:
//   y < 1:  Taylor series of positive terms, S(y) = y^3 P(t), cosh y - 1 = y^2 C(t),
//           sinh y = y (1 + t P(t)), t = y^2, P(t) = sum t^k/(2k+3)!, C(t) = sum t^k/(2k+2)!
//           (NC terms: the first one left out is below the type's rounding for t < 1);
//   y >= 1: exponentials, everything scaled by 2e^{-a} (no overflow at any a), with
//           e1 = e^{-x}, e2 = e^{-a(1+v)}:  2e^{-a} S(y) = e1 - e2 - 2y e^{-a},
//           2e^{-a} (cosh y - 1) = e1 + e2 - 2e^{-a},  2e^{-a} sinh y = e1 - e2.
// The denominator takes the same choice on a: P(a^2) for a < 1 (the a^3 common to the
// numerator and S(a) cancels, so a -> 0 needs no care), 1 - e^{-2a} - 2a e^{-a} for a >= 1.
// The numerator's series form is multiplied by K = 1 (a < 1) or 2e^{-a} a^3 (a >= 1) to
// put it in the denominator's units.  At a = 0 this is the Beta(2,2) law,
// 1 - F = v^2 (3 - 2v).
// ---------------------------------------------------------------------------
template <typename R>
struct Radial3 {
  static constexpr int NC = (sizeof(R) == 4) ? 5 : 10;  // series terms
  R a;
  R ea;    // e^{-a}
  R K;     // units of the series form of the numerator
  R invD;  // 1 / denominator

  WOS_HD void init(R a_) {
    a = a_;
    ea = w_exp(-a);
    const R a2 = a * a;
    const bool sm = a < R(1);
    const R dsm = FactPoly<R, 3, 0, NC>::eval(a2);
    const R dlg = (R(1) - ea * ea) - R(2) * a * ea;
    K = sm ? R(1) : R(2) * ea * a2 * a;
    invD = w_div(R(1), sm ? dsm : dlg);
  }
  // F(rho) and dF/drho
  WOS_HD void eval(R rho, R* F, R* pdf) const {
    const R v = R(1) - rho;
    const R y = a * v;
    const R x = a * rho;
    const R t = y * y;
    const R e1 = w_exp(-x);
    const R e2 = w_exp(-a - y);
    const R P = FactPoly<R, 3, 0, NC>::eval(t);
    const R C = FactPoly<R, 2, 0, NC>::eval(t);
    const bool sm = y < R(1);
    // series forms in units of K: S(y) + x (cosh y - 1) = a^3 v^2 (v P + rho C), and
    // a x sinh y = a^3 rho v (1 + t P)
    const R nsm = K * (v * v) * (v * P + rho * C);
    const R ssm = K * (rho * v) * (R(1) + t * P);
    const R nlg = ((e1 - e2) - R(2) * y * ea) + x * ((e1 + e2) - R(2) * ea);
    const R slg = a * x * (e1 - e2);
    *F = R(1) - (sm ? nsm : nlg) * invD;
    *pdf = (sm ? ssm : slg) * invD;
  }
};

// ---------------------------------------------------------------------------
// Radial CDF, 2D.  N(rho) = 1 - t K1(t) - c t I1(t), t = a rho, c = K0(a)/I0(a),
// N(1) = 1 - 1/I0(a);  dN/drho = a^2 rho (K0(t) - c I0(t)).
// For a < 2 the power series of I0, K0 gives (logs of a cancel)
//   N/a^2 = rho^2 [B(rho^2) - ln(rho) A(rho^2)],
//   A_k = b_k / (2k+2),  B_k = b_k [1/(2k+2)^2 + (H_k - beta)/(2k+2)],
//   dN/drho / a^2 = rho [C(rho^2) - ln(rho) D(rho^2)], D_k = b_k, C_k = b_k (H_k - beta),
// b_k = (a^2/4)^k / (k!)^2, beta = S(a)/I0(a), S(a) = sum_{k>=1} H_k b_k.
// ---------------------------------------------------------------------------
template <typename R>
struct Radial2;

template <>
struct Radial2<float> {
  float a;
  int small;
  float q, beta, invN1;  // a < 2: the series' parameters (coefficients are formed as summed)
  float c_scaled;        // K0(a)/I0(a) times e^{2a}: k0s(a)/i0s(a)
  float e2a;

  // For a < 2 no coefficient arrays are kept (they cost registers and a stack frame in the
  // walk kernels): init sums N(1) and beta in one pass, eval the four series at rho in
  // another, with the beta terms factored out as in radial2_once below.
  WOS_HD void init(float a_) {
    a = a_;
    small = (a < 2.0f);
    if (small) {
      q = 0.25f * a * a;
      float b = 1.0f, H = 0.0f, I0 = 0.0f, S = 0.0f, n1 = 0.0f, n2 = 0.0f, n3 = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k > 0) {
          b *= q * (1.0f / (float)(k * k));
          H += 1.0f / (float)k;
        }
        const float im = 1.0f / (2.0f * k + 2.0f);
        I0 += b;
        S += H * b;
        n1 += b * im * im;
        n2 += b * H * im;
        n3 += b * im;
      }
      beta = w_div(S, I0);
      invN1 = w_div(1.0f, n1 + n2 - beta * n3);  // N(1)/a^2 = B(1)
    } else {
      float ea = w_exp(-a);
      e2a = ea * ea;
      float i0s = (a < 3.75f) ? as_i0_small(a) * ea : as_i0s_large(a);
      float k0s = as_k0s_large(a);  // a >= 2
      c_scaled = w_div(k0s, i0s);   // c = c_scaled e^{-2a}
      invN1 = w_div(1.0f, 1.0f - w_div(ea, i0s));
    }
  }
  WOS_HD void eval(float rho, float* F, float* pdf) const {
    if (small) {
      if (rho <= 0.0f) { *F = 0.0f; *pdf = 0.0f; return; }
      const float r2 = rho * rho, lr = w_log(rho);
      float b = 1.0f, H = 0.0f, rk = 1.0f, pa = 0.0f, pb1 = 0.0f, pb2 = 0.0f, pc1 = 0.0f, pd = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k > 0) {
          b *= q * (1.0f / (float)(k * k));
          H += 1.0f / (float)k;
          rk *= r2;
        }
        const float im = 1.0f / (2.0f * k + 2.0f), brk = b * rk;
        pa += brk * im;
        pb1 += brk * im * im;
        pb2 += brk * H * im;
        pc1 += brk * H;
        pd += brk;
      }
      const float pb = pb1 + pb2 - beta * pa, pc = pc1 - beta * pd;
      *F = r2 * (pb - lr * pa) * invN1;
      *pdf = rho * (pc - lr * pd) * invN1;
      return;
    }
    float t = a * rho;
    if (t <= 0.0f) { *F = 0.0f; *pdf = 0.0f; return; }
    float one_m_tk1, k0t, i0t, ti1t;  // c I0(t), c t I1(t) carry the factor e^{-2a}
    if (t < 2.0f) {
      float lt = w_log(0.5f * t);
      float i1 = as_i1_small(t), i0 = as_i0_small(t);
      one_m_tk1 = -t * lt * i1 - as_k1_poly(t);
      k0t = as_k0_poly(t) - lt * i0;
      i0t = c_scaled * e2a * i0;
      ti1t = c_scaled * e2a * t * i1;
    } else {
      float et = w_exp(-t);
      one_m_tk1 = 1.0f - t * as_k1s_large(t) * et;
      k0t = as_k0s_large(t) * et;
      if (t < 3.75f) {
        i0t = c_scaled * e2a * as_i0_small(t);
        ti1t = c_scaled * e2a * t * as_i1_small(t);
      } else {
        float g = c_scaled * w_exp(t - 2.0f * a);  // c e^{t}
        i0t = g * as_i0s_large(t);
        ti1t = g * t * as_i1s_large(t);
      }
    }
    *F = (one_m_tk1 - ti1t) * invN1;
    *pdf = a * t * (k0t - i0t) * invN1;
  }
};

template <>
struct Radial2<double> {
  double a;
  int small;
  double A[24], B[24], Cc[24], Dd[24];
  int n;
  double invN1;
  double c;  // K0(a)/I0(a)

  WOS_HD void init(double a_) {
    a = a_;
    small = (a <= 2.0);
    if (small) {
      double q = 0.25 * a * a, b = 1.0, H = 0.0, I0 = 0.0, S = 0.0;
      double bk[24], Hk[24];
      n = 24;
      for (int k = 0; k < 24; ++k) {
        if (k > 0) {
          b *= q / ((double)k * k);
          H += 1.0 / k;
        }
        bk[k] = b;
        Hk[k] = H;
        I0 += b;
        S += H * b;
      }
      double beta = S / I0, N1 = 0.0;
      for (int k = 0; k < 24; ++k) {
        double m = 2.0 * k + 2.0;
        A[k] = bk[k] / m;
        B[k] = bk[k] * (1.0 / (m * m) + (Hk[k] - beta) / m);
        Dd[k] = bk[k];
        Cc[k] = bk[k] * (Hk[k] - beta);
        N1 += B[k];
      }
      invN1 = 1.0 / N1;
    } else {
      c = d_k0(a) / d_i0(a);
      invN1 = 1.0 / (1.0 - 1.0 / d_i0(a));
    }
  }
  WOS_HD void eval(double rho, double* F, double* pdf) const {
    if (rho <= 0.0) { *F = 0.0; *pdf = 0.0; return; }
    if (small) {
      double r2 = rho * rho, lr = log(rho);
      double pa = 0, pb = 0, pc = 0, pd = 0;
      for (int k = n - 1; k >= 0; --k) {
        pa = pa * r2 + A[k];
        pb = pb * r2 + B[k];
        pc = pc * r2 + Cc[k];
        pd = pd * r2 + Dd[k];
      }
      *F = r2 * (pb - lr * pa) * invN1;
      *pdf = rho * (pc - lr * pd) * invN1;
      return;
    }
    double t = a * rho;
    double one_m_tk1 = (t <= 2.0) ? d_1m_xk1_small(t) : 1.0 - t * d_k1(t);
    *F = (one_m_tk1 - c * t * d_i1(t)) * invN1;
    *pdf = a * t * (d_k0(t) - c * d_i0(t)) * invN1;
  }
};

// One evaluation of the 2D radial CDF and density (the one-step sampler).  For a < 2 the
// series of Radial2<float> is summed in a single pass: with B_k = b_k/m^2 + b_k H_k/m
// - beta b_k/m and C_k = b_k H_k - beta b_k, the beta terms factor out of the sums, so
// no coefficient arrays are formed (they cost registers and spills in the walk kernel).
WOS_HD void radial2_once(float a, float rho, float* F, float* pdf) {
  if (a >= 2.0f) {
    Radial2<float> rad;
    rad.init(a);
    rad.eval(rho, F, pdf);
    return;
  }
  if (rho <= 0.0f) {
    *F = 0.0f;
    *pdf = 0.0f;
    return;
  }
  const float q = 0.25f * a * a, r2 = rho * rho;
  float b = 1.0f, H = 0.0f, rk = 1.0f;
  float I0 = 0.0f, S = 0.0f, pa = 0.0f, pb1 = 0.0f, pb2 = 0.0f, pc1 = 0.0f, pd = 0.0f;
  float n1 = 0.0f, n2 = 0.0f, n3 = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k > 0) {
      b *= q * (1.0f / (float)(k * k));
      H += 1.0f / (float)k;
      rk *= r2;
    }
    const float im = 1.0f / (2.0f * k + 2.0f);
    const float bi = b * im, bh = b * H;
    I0 += b;
    S += bh;
    n1 += bi * im;
    n2 += bh * im;
    n3 += bi;
    pa += bi * rk;
    pb1 += bi * im * rk;
    pb2 += bh * im * rk;
    pc1 += bh * rk;
    pd += b * rk;
  }
  const float beta = w_div(S, I0);
  const float invN1 = w_div(1.0f, n1 + n2 - beta * n3);
  const float pb = pb1 + pb2 - beta * pa, pc = pc1 - beta * pd;
  const float lr = w_log(rho);
  *F = r2 * (pb - lr * pa) * invN1;
  *pdf = rho * (pc - lr * pd) * invN1;
}
WOS_HD void radial2_once(double a, double rho, double* F, double* pdf) {
  Radial2<double> rad;
  rad.init(a);
  rad.eval(rho, F, pdf);
}

// ---------------------------------------------------------------------------
// Radius of y ~ G/|G| on the centred ball: r = R F^{-1}(u), safeguarded Newton.
// FP32 runs a fixed number of iterations from a closed-form starting point;
// FP64 iterates to convergence.
// ---------------------------------------------------------------------------
// Stops when the step is below tol or the CDF residual is below ftol (FP32: a few
// ulps of u, the level at which rounding noise in F would make Newton oscillate).
template <typename Rad, typename R>
WOS_HD R newton_inverse(const Rad& rad, R u, R rho, int iters, R tol, R ftol, int* iters_used = nullptr) {
  R lo = R(0), hi = R(1);
  int it = 0;
  for (; it < iters; ++it) {
    R F, p;
    rad.eval(rho, &F, &p);
    R res = F - u;
    if (w_fabs(res) <= ftol) break;
    if (res > R(0)) hi = rho; else lo = rho;
    R nr = (p > R(0)) ? rho - w_div(res, p) : R(0.5) * (lo + hi);
    // Newton may land on the bracket end it started from once converged; only
    // a step that leaves [lo, hi] falls back to bisection
    if (!(nr >= lo && nr <= hi)) nr = R(0.5) * (lo + hi);
    R step = w_fabs(nr - rho);
    rho = nr;
    if (step <= tol) break;
  }
  if (iters_used) *iters_used = it;
  return rho;
}

// starting points: Beta(2,2) quantile (3D, a -> 0), the equation
// L - ln(1+L) = -ln u for L = -2 ln rho (2D, a -> 0), and the Gamma(2)
// quantile t - ln(1+t) = -ln(1-u) (large a), each with L0 = m + sqrt(2m).
template <int DIM, typename R>
WOS_HD R radial_guess(R a, R u) {
  if (DIM == 3 && a < R(2)) {
    return R(0.5) + w_sin(w_asin(R(2) * u - R(1)) * R(0.3333333333333333));
  }
  if (DIM == 2 && a < R(2)) {
    R m = -w_log(u);
    R L = m + w_sqrt(R(2) * m);
    return w_exp(R(-0.5) * L);
  }
  R m = -w_log(R(1) - u);
  R t = m + w_sqrt(R(2) * m);
  return w_fmin(t / a, R(0.999));
}

// Tabulated inverse radial CDF rho(u; a), filled in FP64 by the sampler below, on a
// uniform grid a = i * kTabDA (i < kTabA) and t = j / (kTabU - 1), where
//   u = 2 t^2 (t <= 1/2),  u = 1 - 2 (1 - t)^2 (t >= 1/2).
// The radial density vanishes linearly at rho = 0 (3D; with a log factor in 2D) and
// at rho = 1, so rho ~ sqrt(u) and 1 - rho ~ sqrt(1 - u) at the ends: in t both are
// linear and bilinear interpolation is accurate up to the ends.  From the
// interpolated start one Newton step leaves |F(rho) - u| at the FP32 rounding level
// (max 1.3e-7 over a < 32, measured against the FP64 sampler), so the FP32 sampler
// takes exactly one step there: no data-dependent loop, no divergence in a warp.
constexpr int kTabA = 129;
constexpr int kTabU = 513;
constexpr float kTabDA = 0.25f;
constexpr int kTabSize = kTabA * kTabU;
// u beyond the last t interval (probability 7.6e-6): rho jumps there from ~0.5 to 1 at
// large a, so these few samples take the safeguarded Newton loop instead
constexpr double kTabUHi = 1.0 - 2.0 / ((double)(kTabU - 1) * (double)(kTabU - 1));

WOS_HD double tab_u_of_t(double t) { return (t <= 0.5) ? 2.0 * t * t : 1.0 - 2.0 * (1.0 - t) * (1.0 - t); }
WOS_HD float tab_t_of_u(float u) {
  const float r = w_sqrt_fast(0.5f * fminf(u, 1.0f - u));
  return (u <= 0.5f) ? r : 1.0f - r;
}

WOS_HD float load_tab(const float* p) {
#if defined(__CUDA_ARCH__)
  return __ldg(p);
#else
  return *p;
#endif
}

// floor of v in [0, 2^22) as (index, v - index) by the float magic number 1.5 * 2^23: adding
// it rounds v - 1/2 to an integer held in the mantissa (at an integer v a tie may round one
// down, leaving a fraction of exactly 1: the interpolation is continuous there).  No
// float-integer conversion instruction.
WOS_HD int floor_split(float v, float* frac) {
  const float m = (v - 0.5f) + 12582912.0f;
  const float fl = m - 12582912.0f;
  *frac = v - fl;
  return (int)(f_as_i_bits(m) - f_as_i_bits(12582912.0f));
}
WOS_HD float table_guess(const float* tab, float a, float u) {
  const float fa = a * (1.0f / kTabDA);  // a < (kTabA - 1) kTabDA when the table is used
  float ta;
  int ia = floor_split(fa, &ta);
  if (ia > kTabA - 2) {  // a at the table's upper edge
    ta += (float)(ia - (kTabA - 2));
    ia = kTabA - 2;
  }
  float tt;
  int it = floor_split(tab_t_of_u(u) * (float)(kTabU - 1), &tt);
  if (it > kTabU - 2) {  // t = 1
    tt += 1.0f;
    it = kTabU - 2;
  }
  const float* r0 = tab + ia * kTabU + it;
  const float* r1 = r0 + kTabU;
  float v0 = load_tab(r0) + tt * (load_tab(r0 + 1) - load_tab(r0));
  float v1 = load_tab(r1) + tt * (load_tab(r1 + 1) - load_tab(r1));
  return v0 + ta * (v1 - v0);
}

template <int DIM, typename R>
WOS_HD R sample_radius(R a, R u, int* iters_used = nullptr, const float* tab = nullptr) {
  // FP32: the loop serves only the rare samples outside the table's one-step range (the
  // last t interval, a >= 32); in the flat tail near rho = 1 it may need bisection steps
  const int iters = (sizeof(R) == 4) ? 40 : 200;
  const R tol = (sizeof(R) == 4) ? R(1e-7) : R(1e-16);
  const R ftol = (sizeof(R) == 4) ? R(1e-6) : R(0);
  const bool tabled = tab != nullptr && a < R((kTabA - 1) * kTabDA);
  R g;
  if (tabled) {
    g = R(table_guess(tab, (float)a, (float)u));
    g = w_fmin(w_fmax(g, R(1e-6)), R(1) - R(1e-6));
  } else {
    g = radial_guess<DIM, R>(a, u);
  }
  if (tabled && u < R(kTabUHi)) {
    // one Newton step from the table (see above).  The start is kept where it already meets
    // the FP32 tolerance (near rho = 1, where the density is tiny, F - u is rounding noise
    // and a step would jump far), and where the step is larger than the table's error
    // (at most 6e-3 in rho) or leaves (0, 1).
    R F, p;
    if (DIM == 3) {
      Radial3<R> rad;
      rad.init(a);
      rad.eval(g, &F, &p);
    } else {
      radial2_once(a, g, &F, &p);
    }
    const R res = F - u;
    const R step = (p > R(0)) ? w_div(res, p) : R(0);
    const R nr = g - step;
    if (iters_used) *iters_used = 1;
    return (w_fabs(res) > ftol && w_fabs(step) <= R(0.02) && nr > R(0) && nr < R(1)) ? nr : g;
  }
  if (DIM == 3) {
    Radial3<R> rad;
    rad.init(a);
    return newton_inverse(rad, u, g, iters, tol, ftol, iters_used);
  } else {
    Radial2<R> rad;
    rad.init(a);
    return newton_inverse(rad, u, g, iters, tol, ftol, iters_used);
  }
}

// density f(rho) = dF/drho of rho = r/R under y ~ G/|G|
template <int DIM, typename R>
WOS_HD R radial_pdf(R a, R rho) {
  R F, p;
  if (DIM == 3) {
    Radial3<R> rad;
    rad.init(a);
    rad.eval(rho, &F, &p);
  } else {
    radial2_once(a, rho, &F, &p);
  }
  return p;
}

// Mixture ball sample for weights that carry |G'(r)/G(r)| (the extra drift's null weight,
// the gradient's first ball), which has an infinite second moment under G/|G|: a fraction
// lam of the radius uniform's range draws from G/|G| (u < lam, rescaled to u / lam), the
// rest a uniform radius (rho = (u - lam) / (1 - lam)).  The source term and the null
// weight are then multiplied by *mixw = f / (lam f + 1 - lam), the density ratio of G/|G|
// to the mixture, which keeps their expectations and bounds the weight at both ends.
// The radius of a mixture lane from the inverse-CDF radius rho_g (drawn with u / lam when
// u < lam, the part of G/|G|) and the uniform u; sets *mixw.  FP32 uniforms are rounded
// to 24 bits, so u can equal lam and u / lam can round to 1: rho is kept inside the
// uniform's resolution, where the weight and the |G'/G| factor are finite (at rho = 0 or
// 1 the weight vanishes and the factor is infinite; their product has a finite limit).
template <int DIM, typename R>
WOS_HD R mix_radius_weight(R a, R u, R rho_g, R lam, R* mixw) {
  R rho = (u < lam) ? rho_g : (u - lam) / (R(1) - lam);
  if (sizeof(R) == 4) rho = w_fmin(w_fmax(rho, R(1e-7)), R(1) - R(6e-8));
  const R f = radial_pdf<DIM, R>(a, rho);
  *mixw = f / (lam * f + (R(1) - lam));
  return rho;
}

template <int DIM, typename R>
WOS_HD R mix_sample_radius(R a, R u, const float* tab, R lam, R* mixw) {
  const R rho_g = sample_radius<DIM, R>(a, (u < lam) ? u / lam : R(0.5), nullptr, tab);
  return mix_radius_weight<DIM, R>(a, u, rho_g, lam, mixw);
}

}  // namespace wos
