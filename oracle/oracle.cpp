// oracle.cpp -- plain FP64 CPU oracle for delta-tracking walk on spheres.
//
// TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
// CPU-baseline leg of the benchmark.  The product library never includes,
// links or calls it, and it shares no source with the CUDA path.
//
// Every function follows one passage of Sawhney, Seyb, Jarosz, Crane,
// "Grid-Free Monte Carlo for PDEs with Spatially Varying Coefficients"
// (SIGGRAPH 2022); the passage is named above the function.  Speed is not a
// goal: closed forms are evaluated as printed, with a power series only where
// the printed form cancels catastrophically in double precision, and roots
// are found by safeguarded Newton iteration run to convergence.
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <omp.h>

namespace {

const double kPi = 3.14159265358979323846;
const double kEulerGamma = 0.57721566490153286061;

// ---------------------------------------------------------------------------
// Bessel functions: the C++17 special functions of libstdc++ (library step).
// ---------------------------------------------------------------------------
double bI0(double x) { return std::cyl_bessel_i(0.0, x); }
double bI1(double x) { return std::cyl_bessel_i(1.0, x); }
double bK0(double x) { return std::cyl_bessel_k(0.0, x); }
double bK1(double x) { return std::cyl_bessel_k(1.0, x); }

// ---------------------------------------------------------------------------
// Supplemental Sec. 1.1, 2D.  Small-argument forms from the power series of
// I0 and K0 (DLMF 10.25.2 and 10.31.2): with b_k = (a^2/4)^k / (k!)^2 and
// H_k the harmonic numbers,
//   I0(a) = sum_k b_k,   K0(a) = -(ln(a/2) + gamma_E) I0(a) + S(a),
//   S(a) = sum_{k>=1} H_k b_k.
// Substituting into Q2D(a rho) = K0(a rho) - K0(a) I0(a rho) / I0(a) the
// logarithms of a cancel, leaving
//   Q2D(a rho) = -ln(rho) I0(a rho) + S(a rho) - beta I0(a rho),
//   beta = S(a) / I0(a),
// and the radial integral N(rho) = a^2 int_0^rho t Q2D(a t) dt term by term:
//   N(rho)/a^2 = sum_k b_k rho^(2k+2) [1/(2k+2)^2 - ln(rho)/(2k+2)
//                                       + (H_k - beta)/(2k+2)].
// ---------------------------------------------------------------------------
struct Series2D {
  double b[40];
  double H[40];
  int n;
  double beta;
};

void series2d_init(double a, Series2D* s) {
  double q = a * a / 4.0;
  double bk = 1.0, Hk = 0.0, I0 = 0.0, S = 0.0;
  int k = 0;
  for (; k < 40; ++k) {
    if (k > 0) {
      bk *= q / ((double)k * (double)k);
      Hk += 1.0 / k;
    }
    s->b[k] = bk;
    s->H[k] = Hk;
    I0 += bk;
    S += Hk * bk;
    if (k > 2 && bk < 1e-20 * I0) { ++k; break; }
  }
  s->n = k;
  s->beta = S / I0;
}

// N(rho) / a^2 from the series
double series2d_N(const Series2D& s, double rho) {
  if (rho <= 0.0) return 0.0;
  double lr = std::log(rho);
  double r2 = rho * rho, rp = r2, acc = 0.0;
  for (int k = 0; k < s.n; ++k) {
    double m = 2.0 * k + 2.0;
    acc += s.b[k] * rp * (1.0 / (m * m) - lr / m + (s.H[k] - s.beta) / m);
    rp *= r2;
  }
  return acc;
}

// Q2D(a rho) from the series
double series2d_Q(const Series2D& s, double rho) {
  double lr = std::log(rho);
  double r2 = rho * rho, rp = 1.0, I0 = 0.0, S = 0.0;
  for (int k = 0; k < s.n; ++k) {
    I0 += s.b[k] * rp;
    S += s.H[k] * s.b[k] * rp;
    rp *= r2;
  }
  return -lr * I0 + S - s.beta * I0;
}

// 1 - t K1(t) for t < 2, from DLMF 10.31.1 (n = 1), no cancellation:
//   1 - t K1(t) = -t ln(t/2) I1(t)
//                 + (t^2/4) sum_k (psi(k+1) + psi(k+2)) (t^2/4)^k / (k! (k+1)!)
double one_minus_tK1_small(double t) {
  double q = t * t / 4.0;
  double term = 1.0;  // (t^2/4)^k / (k! (k+1)!)
  double Hk = 0.0;    // H_k
  double acc = 0.0;
  for (int k = 0; k < 40; ++k) {
    if (k > 0) {
      term *= q / ((double)k * (double)(k + 1));
      Hk += 1.0 / k;
    }
    double psi1 = -kEulerGamma + Hk;
    double psi2 = -kEulerGamma + Hk + 1.0 / (k + 1);
    acc += (psi1 + psi2) * term;
    if (k > 2 && std::fabs(term) < 1e-22) break;
  }
  return -t * std::log(t / 2.0) * bI1(t) + q * acc;
}

// ---------------------------------------------------------------------------
// Supplemental Sec. 1.1, 3D.  N(rho) = a^2 int_0^rho t sinh(a(1-t)) dt with
//   N(rho) = sinh a - sinh(a(1-rho)) - a rho cosh(a(1-rho)),
//   D = N(1) = sinh a - a.
// For a < 1 the Taylor series of sinh in a is integrated term by term:
//   N(rho) = a^3 sum_j a^(2j)/(2j+1)! J_{2j+1}(rho),
//   J_m(rho) = int_0^rho t (1-t)^m dt = [1 - (1-rho)^(m+1)(1+(m+1)rho)] / ((m+1)(m+2)).
// For a >= 1 both N and D are multiplied by 2 e^{-a} (no overflow):
//   N~(rho) = h(-a rho) - e^{-2a} h(a rho),  h(x) = 1 - e^x (1 - x),
//   D~ = 1 - 2 a e^{-a} - e^{-2a}.
// ---------------------------------------------------------------------------
double J_m(int m, double rho) {
  if (rho < 0.25) {
    // sum_i C(m,i) (-1)^i rho^(i+2) / (i+2)
    double acc = 0.0, c = 1.0, rp = rho * rho;
    for (int i = 0; i <= m; ++i) {
      acc += ((i & 1) ? -c : c) * rp / (i + 2);
      c = c * (m - i) / (i + 1);
      rp *= rho;
    }
    return acc;
  }
  double om = 1.0 - rho;
  return (1.0 - std::pow(om, m + 1) * (1.0 + (m + 1) * rho)) / ((m + 1.0) * (m + 2.0));
}

// h(x) = 1 - e^x (1 - x) = sum_{m>=2} x^m (m-1)/m!  (h(-x) = 1 - e^{-x}(1+x))
double h_fn(double x) {
  if (std::fabs(x) < 0.5) {
    double acc = 0.0, term = x;  // x^m / m!
    for (int m = 2; m < 30; ++m) {
      term *= x / m;
      acc += term * (m - 1);
      if (std::fabs(term) < 1e-20) break;
    }
    return acc;
  }
  return 1.0 - std::exp(x) * (1.0 - x);
}

// e^{-2a} h(a rho), written without overflow
double e2a_h(double a, double rho) {
  double x = a * rho;
  if (x < 0.5) return std::exp(-2.0 * a) * h_fn(x);
  return std::exp(-2.0 * a) - std::exp(-a * (2.0 - rho)) * (1.0 - x);
}

double cdf3(double a, double rho) {
  if (rho <= 0.0) return 0.0;
  if (rho >= 1.0) return 1.0;
  if (a < 1.0) {
    double num = 0.0, den = 0.0, c = 1.0;  // c = a^(2j)/(2j+1)!
    for (int j = 0; j < 30; ++j) {
      int m = 2 * j + 1;
      num += c * J_m(m, rho);
      den += c / ((m + 1.0) * (m + 2.0));
      c *= a * a / ((2.0 * j + 2.0) * (2.0 * j + 3.0));
      if (c < 1e-22) break;
    }
    return num / den;
  }
  double num = h_fn(-a * rho) - e2a_h(a, rho);
  double den = 1.0 - 2.0 * a * std::exp(-a) - std::exp(-2.0 * a);
  return num / den;
}

// dF/drho
double pdf3(double a, double rho) {
  if (rho <= 0.0 || rho >= 1.0) return 0.0;
  if (a < 1.0) {
    double num = 0.0, den = 0.0, c = 1.0;
    for (int j = 0; j < 30; ++j) {
      int m = 2 * j + 1;
      num += c * rho * std::pow(1.0 - rho, m);
      den += c / ((m + 1.0) * (m + 2.0));
      c *= a * a / ((2.0 * j + 2.0) * (2.0 * j + 3.0));
      if (c < 1e-22) break;
    }
    return num / den;
  }
  double num = a * a * rho * (std::exp(-a * rho) - std::exp(-a * (2.0 - rho)));
  double den = 1.0 - 2.0 * a * std::exp(-a) - std::exp(-2.0 * a);
  return num / den;
}

// 2D radial CDF: F = N(rho) / N(1),
//   N(rho) = 1 - t K1(t) - (K0(a)/I0(a)) t I1(t),  t = a rho,  N(1) = 1 - 1/I0(a)
double cdf2(double a, double rho) {
  if (rho <= 0.0) return 0.0;
  if (rho >= 1.0) return 1.0;
  if (a <= 2.0) {
    Series2D s;
    series2d_init(a, &s);
    return series2d_N(s, rho) / series2d_N(s, 1.0);
  }
  double t = a * rho;
  double c = bK0(a) / bI0(a);
  double first = (t < 2.0) ? one_minus_tK1_small(t) : 1.0 - t * bK1(t);
  double num = first - c * t * bI1(t);
  double den = 1.0 - 1.0 / bI0(a);
  return num / den;
}

double pdf2(double a, double rho) {
  if (rho <= 0.0 || rho >= 1.0) return 0.0;
  if (a <= 2.0) {
    Series2D s;
    series2d_init(a, &s);
    return rho * series2d_Q(s, rho) / series2d_N(s, 1.0);
  }
  double t = a * rho;
  double c = bK0(a) / bI0(a);
  double den = 1.0 - 1.0 / bI0(a);
  return a * a * rho * (bK0(t) - c * bI0(t)) / den;
}

// ---------------------------------------------------------------------------
// Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11.  Round: two 32x32->64 products of counter words 0 and 2
// with the round multipliers, outputs (hi1^c1^k0, lo1, hi0^c3^k1, lo0); the
// key is bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
void philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

double uniform01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

// Reading R12: a 3D step takes its six uniforms (mu, the radius uniform, two per direction)
// from one Philox block: 21-bit fields -- each word's top 21 bits, then the low 11 bits of
// words 0 and 1 each followed by the low 10 bits of words 2 and 3 -- as (f + 1/2) / 2^21.
void uniforms21(const uint32_t* o, double* u) {
  const uint32_t f[6] = {o[0] >> 11, o[1] >> 11, o[2] >> 11, o[3] >> 11,
                         ((o[0] & 0x7ffu) << 10) | (o[2] & 0x3ffu), ((o[1] & 0x7ffu) << 10) | (o[3] & 0x3ffu)};
  for (int i = 0; i < 6; ++i) u[i] = ((double)f[i] + 0.5) / 2097152.0;
}

// The step's mu, radius uniform and the two directions (y's and z's), dim 2 or 3
void step_randoms(int dim, const uint32_t* o0, double* mu, double* ur, double* dy, double* dz) {
  if (dim == 2) {
    *mu = uniform01(o0[0]);
    *ur = uniform01(o0[1]);
    double ty = 2.0 * kPi * uniform01(o0[2]), tz = 2.0 * kPi * uniform01(o0[3]);
    dy[0] = std::cos(ty); dy[1] = std::sin(ty);
    dz[0] = std::cos(tz); dz[1] = std::sin(tz);
    return;
  }
  double u6[6];
  uniforms21(o0, u6);
  *mu = u6[0];
  *ur = u6[1];
  // uniform direction on the sphere from two uniforms (Archimedes' projection)
  double cy = 1.0 - 2.0 * u6[2], py = 2.0 * kPi * u6[3];
  double sy = std::sqrt(std::fmax(0.0, 1.0 - cy * cy));
  dy[0] = sy * std::cos(py); dy[1] = sy * std::sin(py); dy[2] = cy;
  double cz = 1.0 - 2.0 * u6[4], pz = 2.0 * kPi * u6[5];
  double sz = std::sqrt(std::fmax(0.0, 1.0 - cz * cz));
  dz[0] = sz * std::cos(pz); dz[1] = sz * std::sin(pz); dz[2] = cz;
}

// ---------------------------------------------------------------------------
// Fields: sum of separable terms, grids, manufactured source.
// ---------------------------------------------------------------------------
void atom(int type, double k, double phi, double x, double* h, double* h1, double* h2) {
  double t = k * x + phi;
  switch (type) {
    case ORC_ONE: *h = 1.0; *h1 = 0.0; *h2 = 0.0; break;
    case ORC_SIN: *h = std::sin(t); *h1 = k * std::cos(t); *h2 = -k * k * std::sin(t); break;
    case ORC_COS: *h = std::cos(t); *h1 = -k * std::sin(t); *h2 = -k * k * std::cos(t); break;
    case ORC_EXP: *h = std::exp(t); *h1 = k * std::exp(t); *h2 = k * k * std::exp(t); break;
    case ORC_SINH: *h = std::sinh(t); *h1 = k * std::cosh(t); *h2 = k * k * std::sinh(t); break;
    case ORC_COSH: *h = std::cosh(t); *h1 = k * std::sinh(t); *h2 = k * k * std::cosh(t); break;
    case ORC_LIN: *h = t; *h1 = k; *h2 = 0.0; break;
    case ORC_QUAD: *h = t * t; *h1 = 2.0 * k * t; *h2 = 2.0 * k * k; break;
    default: *h = NAN; *h1 = NAN; *h2 = NAN; break;
  }
}

void sst_eval(int dim, const orc_field* fl, const double* x, double* v, double* g, double* lap) {
  *v = 0.0;
  *lap = 0.0;
  for (int i = 0; i < 3; ++i) g[i] = 0.0;
  for (int n = 0; n < fl->nterms; ++n) {
    const orc_term& tm = fl->terms[n];
    double h[3], h1[3], h2[3];
    for (int i = 0; i < 3; ++i) { h[i] = 1.0; h1[i] = 0.0; h2[i] = 0.0; }
    for (int i = 0; i < dim; ++i) atom(tm.type[i], tm.k[i], tm.phi[i], x[i], &h[i], &h1[i], &h2[i]);
    *v += tm.c * h[0] * h[1] * h[2];
    g[0] += tm.c * h1[0] * h[1] * h[2];
    g[1] += tm.c * h[0] * h1[1] * h[2];
    g[2] += tm.c * h[0] * h[1] * h1[2];
    *lap += tm.c * (h2[0] * h[1] * h[2] + h[0] * h2[1] * h[2] + h[0] * h[1] * h2[2]);
  }
}

// node-centred multilinear interpolation, coordinates clamped to the grid box
void grid_linear(int dim, const orc_field* fl, const double* x, double* v, double* g, double* lap) {
  int i0[3] = {0, 0, 0};
  double t[3] = {0, 0, 0}, hh[3] = {1, 1, 1};
  for (int d = 0; d < dim; ++d) {
    hh[d] = (fl->hi[d] - fl->lo[d]) / (fl->res[d] - 1);
    double s = (x[d] - fl->lo[d]) / hh[d];
    if (s < 0.0) s = 0.0;
    if (s > fl->res[d] - 1) s = fl->res[d] - 1;
    int i = (int)std::floor(s);
    if (i > fl->res[d] - 2) i = fl->res[d] - 2;
    i0[d] = i;
    t[d] = s - i;
  }
  *v = 0.0;
  *lap = 0.0;
  for (int d = 0; d < 3; ++d) g[d] = 0.0;
  int nc = (dim == 3) ? 8 : 4;
  for (int c = 0; c < nc; ++c) {
    int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    long idx = 0, stride = 1;
    double w = 1.0, dw[3] = {1, 1, 1};
    for (int d = 0; d < dim; ++d) {
      idx += (long)(i0[d] + o[d]) * stride;
      stride *= fl->res[d];
      double wd = o[d] ? t[d] : 1.0 - t[d];
      double dd = (o[d] ? 1.0 : -1.0) / hh[d];
      for (int e = 0; e < dim; ++e) dw[e] *= (e == d) ? dd : wd;
      w *= wd;
    }
    double val = fl->data[idx];
    *v += w * val;
    for (int d = 0; d < dim; ++d) g[d] += dw[d] * val;
  }
}

// uniform cubic B-spline basis and derivatives at fraction t
void bspline_basis(double t, double B[4], double B1[4], double B2[4]) {
  double u = 1.0 - t;
  B[0] = u * u * u / 6.0;
  B[1] = (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0;
  B[2] = (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0;
  B[3] = t * t * t / 6.0;
  B1[0] = -u * u / 2.0;
  B1[1] = (3.0 * t * t - 4.0 * t) / 2.0;
  B1[2] = (-3.0 * t * t + 2.0 * t + 1.0) / 2.0;
  B1[3] = t * t / 2.0;
  B2[0] = u;
  B2[1] = 3.0 * t - 2.0;
  B2[2] = -3.0 * t + 1.0;
  B2[3] = t;
}

// cubic B-spline with the grid values as control points at the nodes; control
// indices are clamped to the grid (constant extension), which keeps it C^2.
void grid_bspline(int dim, const orc_field* fl, const double* x, double* v, double* g, double* lap) {
  int ib[3] = {0, 0, 0};
  double B[3][4], B1[3][4], B2[3][4], hh[3] = {1, 1, 1};
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < 4; ++a) { B[d][a] = (a == 0); B1[d][a] = 0; B2[d][a] = 0; }
  for (int d = 0; d < dim; ++d) {
    hh[d] = (fl->hi[d] - fl->lo[d]) / (fl->res[d] - 1);
    double s = (x[d] - fl->lo[d]) / hh[d];
    double fs = std::floor(s);
    ib[d] = (int)fs - 1;
    bspline_basis(s - fs, B[d], B1[d], B2[d]);
    for (int a = 0; a < 4; ++a) { B1[d][a] /= hh[d]; B2[d][a] /= hh[d] * hh[d]; }
  }
  *v = 0.0;
  *lap = 0.0;
  for (int d = 0; d < 3; ++d) g[d] = 0.0;
  int n2 = (dim == 3) ? 4 : 1;
  for (int c2 = 0; c2 < n2; ++c2)
    for (int c1 = 0; c1 < 4; ++c1)
      for (int c0 = 0; c0 < 4; ++c0) {
        int c[3] = {c0, c1, c2};
        long idx = 0, stride = 1;
        for (int d = 0; d < dim; ++d) {
          int j = ib[d] + c[d];
          if (j < 0) j = 0;
          if (j > fl->res[d] - 1) j = fl->res[d] - 1;
          idx += (long)j * stride;
          stride *= fl->res[d];
        }
        double val = fl->data[idx];
        double b0 = B[0][c0], b1 = B[1][c1], b2 = B[2][c2];
        *v += val * b0 * b1 * b2;
        g[0] += val * B1[0][c0] * b1 * b2;
        g[1] += val * b0 * B1[1][c1] * b2;
        g[2] += val * b0 * b1 * B1[2][c2];
        *lap += val * (B2[0][c0] * b1 * b2 + b0 * B2[1][c1] * b2 + b0 * b1 * B2[2][c2]);
      }
}

int field_eval(const orc_problem* P, const orc_field* fl, const double* x, double* v, double* g,
               double* lap) {
  int dim = P->dim;
  switch (fl->kind) {
    case ORC_FIELD_ZERO:
      *v = 0.0; *lap = 0.0; g[0] = g[1] = g[2] = 0.0;
      return 0;
    case ORC_FIELD_CONST:
      *v = fl->value; *lap = 0.0; g[0] = g[1] = g[2] = 0.0;
      return 0;
    case ORC_FIELD_SST:
      sst_eval(dim, fl, x, v, g, lap);
      return 0;
    case ORC_FIELD_GRID_LINEAR:
      grid_linear(dim, fl, x, v, g, lap);
      return 0;
    case ORC_FIELD_GRID_BSPLINE:
      grid_bspline(dim, fl, x, v, g, lap);
      return 0;
    case ORC_FIELD_MANUFACTURED: {
      // eq. 1 solved for f at a known u:  f = -div(alpha grad u) - omega.grad u + sigma u,
      // div(alpha grad u) = alpha Lap u + grad alpha . grad u,  omega = alpha grad Phi.
      double u, gu[3], lu, a, ga[3], la, ph, gp[3], lp, s, gs[3], ls;
      if (field_eval(P, &P->um, x, &u, gu, &lu)) return -1;
      if (field_eval(P, &P->alpha, x, &a, ga, &la)) return -1;
      if (field_eval(P, &P->phi, x, &ph, gp, &lp)) return -1;
      if (field_eval(P, &P->sigma, x, &s, gs, &ls)) return -1;
      double dot_a = 0.0, dot_p = 0.0, dot_w = 0.0;
      for (int d = 0; d < dim; ++d) {
        dot_a += ga[d] * gu[d];
        dot_p += gp[d] * gu[d];
        double w, gw[3], lw;
        if (field_eval(P, &P->omega[d], x, &w, gw, &lw)) return -1;
        dot_w += w * gu[d];
      }
      *v = -(a * lu + dot_a) - a * dot_p - dot_w + s * u;
      *lap = NAN;
      g[0] = g[1] = g[2] = NAN;
      return 0;
    }
    default:
      return -1;
  }
}

// Sec. 4.1 (eq. 7-8) and App. A: gamma = 1/2 ln(alpha) + 1/2 Phi,
// sigma' = sigma/alpha + Lap(gamma) + |grad gamma|^2, f' = e^gamma f / alpha.
bool has_drift(const orc_problem* P) {
  for (int d = 0; d < P->dim; ++d)
    if (P->omega[d].kind != ORC_FIELD_ZERO) return true;
  return false;
}

void coeffs(const orc_problem* P, const double* x, double* gamma, double* sp, double* fp,
            double* fv, double* av, double* bout = nullptr) {
  int dim = P->dim;
  double a, ga[3], la, ph, gp[3], lp, s, gs[3], ls, f, gf[3], lf;
  field_eval(P, &P->alpha, x, &a, ga, &la);
  field_eval(P, &P->phi, x, &ph, gp, &lp);
  field_eval(P, &P->sigma, x, &s, gs, &ls);
  field_eval(P, &P->f, x, &f, gf, &lf);
  double ggam[3] = {0, 0, 0}, na2 = 0.0;
  for (int d = 0; d < dim; ++d) {
    ggam[d] = 0.5 * (ga[d] / a + gp[d]);
    na2 += ga[d] * ga[d];
  }
  double lgam = 0.5 * (la / a - na2 / (a * a) + lp);
  double ng2 = 0.0;
  for (int d = 0; d < dim; ++d) ng2 += ggam[d] * ggam[d];
  *gamma = 0.5 * std::log(a) + 0.5 * ph;
  *sp = s / a + lgam + ng2;
  *fp = std::exp(*gamma) * f / a;
  *fv = f;
  *av = a;
  if (bout) bout[0] = bout[1] = bout[2] = 0.0;
  if (has_drift(P)) {
    // b = omega_extra / alpha: sigma'' = sigma' + b . grad gamma, plus div b from the parts
    double divw = 0.0, wga = 0.0, bg = 0.0, b[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
      double w, gw[3], lw;
      field_eval(P, &P->omega[d], x, &w, gw, &lw);
      divw += gw[d];
      wga += w * ga[d];
      b[d] = w / a;
      bg += b[d] * ggam[d];
    }
    double divb = divw / a - wga / (a * a);
    *sp += bg + divb;
    if (bout)
      for (int d = 0; d < dim; ++d) bout[d] = b[d];
  }
}

// |G'(r) / G(r)| of the centred Green's function on a ball of radius R (Supplemental 1.1):
// 3D G ~ sinh(s(R - r)) / r, 2D G ~ K0(sr) - K0(sR) I0(sr) / I0(sR).
double green_dlog(int dim, double R, double sb, double r) {
  double s = std::sqrt(sb);
  if (dim == 3) {
    if (sb == 0.0) return 1.0 / r + 1.0 / (R - r);
    return s / std::tanh(s * (R - r)) + 1.0 / r;
  }
  if (sb == 0.0) return 1.0 / (r * std::log(R / r));
  double t = s * r, a = s * R;
  return s * (bK1(t) + bK0(a) / bI0(a) * bI1(t)) / (bK0(t) - bK0(a) / bI0(a) * bI0(t));
}

double gamma_at(const orc_problem* P, const double* x) {
  double a, ga[3], la, ph, gp[3], lp;
  field_eval(P, &P->alpha, x, &a, ga, &la);
  field_eval(P, &P->phi, x, &ph, gp, &lp);
  return 0.5 * std::log(a) + 0.5 * ph;
}

// ---------------------------------------------------------------------------
// Triangle meshes: closest point on a triangle and a plain BVH (Sec. 7.1: the
// distance query on a mesh is accelerated by a bounding volume hierarchy).
// ---------------------------------------------------------------------------
struct V3 {
  double x, y, z;
};
V3 v3sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 v3add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V3 v3mul(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
double v3dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 v3cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }

V3 closest_on_segment(V3 p, V3 a, V3 b) {
  V3 ab = v3sub(b, a);
  double l2 = v3dot(ab, ab);
  double t = (l2 > 0.0) ? v3dot(v3sub(p, a), ab) / l2 : 0.0;
  t = std::min(1.0, std::max(0.0, t));
  return v3add(a, v3mul(ab, t));
}

// The closest point of a triangle: the projection onto its plane when that
// falls inside the triangle, else the closest of the closest points of its edges.
V3 closest_on_triangle(V3 p, V3 a, V3 b, V3 c) {
  V3 n = v3cross(v3sub(b, a), v3sub(c, a));
  double n2 = v3dot(n, n);
  if (n2 > 0.0) {
    V3 q = v3sub(p, v3mul(n, v3dot(v3sub(p, a), n) / n2));
    bool in = v3dot(v3cross(v3sub(b, a), v3sub(q, a)), n) >= 0.0 &&
              v3dot(v3cross(v3sub(c, b), v3sub(q, b)), n) >= 0.0 &&
              v3dot(v3cross(v3sub(a, c), v3sub(q, c)), n) >= 0.0;
    if (in) return q;
  }
  V3 best = closest_on_segment(p, a, b);
  double bd = v3dot(v3sub(p, best), v3sub(p, best));
  V3 e[2] = {closest_on_segment(p, b, c), closest_on_segment(p, c, a)};
  for (V3 q : e) {
    double dq = v3dot(v3sub(p, q), v3sub(p, q));
    if (dq < bd) { bd = dq; best = q; }
  }
  return best;
}

V3 mesh_vertex(const orc_domain& D, int64_t i) {
  return {D.verts[3 * i], D.verts[3 * i + 1], D.verts[3 * i + 2]};
}

struct OrcNode {
  double lo[3], hi[3];
  int left, right;  // children (-1 for a leaf)
  int first, count;  // leaf: range of the permuted triangle list
};

struct OrcBVH {
  std::vector<OrcNode> nodes;
  std::vector<int64_t> tri;  // permuted triangle indices
  // optional distance grid
  int n = 0;
  double lo[3] = {0, 0, 0}, h[3] = {0, 0, 0}, thresh = 0.0;
  std::vector<double> dist;
};

int bvh_build(const orc_domain& D, OrcBVH& B, std::vector<V3>& cent, int first, int count) {
  OrcNode nd;
  for (int d = 0; d < 3; ++d) { nd.lo[d] = INFINITY; nd.hi[d] = -INFINITY; }
  for (int i = first; i < first + count; ++i) {
    const int32_t* t = D.tris + 3 * B.tri[i];
    for (int k = 0; k < 3; ++k) {
      V3 v = mesh_vertex(D, t[k]);
      double c[3] = {v.x, v.y, v.z};
      for (int d = 0; d < 3; ++d) {
        nd.lo[d] = std::min(nd.lo[d], c[d]);
        nd.hi[d] = std::max(nd.hi[d], c[d]);
      }
    }
  }
  nd.left = nd.right = -1;
  nd.first = first;
  nd.count = count;
  int idx = (int)B.nodes.size();
  B.nodes.push_back(nd);
  if (count <= 4) return idx;
  // split at the median centroid along the longest axis of the box
  int ax = 0;
  for (int d = 1; d < 3; ++d)
    if (nd.hi[d] - nd.lo[d] > nd.hi[ax] - nd.lo[ax]) ax = d;
  auto key = [&](int64_t t) { V3 c = cent[t]; return ax == 0 ? c.x : (ax == 1 ? c.y : c.z); };
  int mid = first + count / 2;
  std::nth_element(B.tri.begin() + first, B.tri.begin() + mid, B.tri.begin() + first + count,
                   [&](int64_t a, int64_t b) { return key(a) < key(b); });
  int l = bvh_build(D, B, cent, first, mid - first);
  int r = bvh_build(D, B, cent, mid, first + count - mid);
  B.nodes[idx].left = l;
  B.nodes[idx].right = r;
  return idx;
}

double box_dist2(const OrcNode& n, V3 p) {
  double c[3] = {p.x, p.y, p.z}, s = 0.0;
  for (int d = 0; d < 3; ++d) {
    double e = std::max(0.0, std::max(n.lo[d] - c[d], c[d] - n.hi[d]));
    s += e * e;
  }
  return s;
}

void bvh_query(const orc_domain& D, const OrcBVH& B, int ni, V3 p, double* best2, V3* bestq) {
  const OrcNode& n = B.nodes[ni];
  if (box_dist2(n, p) >= *best2) return;
  if (n.left < 0) {
    for (int i = n.first; i < n.first + n.count; ++i) {
      const int32_t* t = D.tris + 3 * B.tri[i];
      V3 q = closest_on_triangle(p, mesh_vertex(D, t[0]), mesh_vertex(D, t[1]), mesh_vertex(D, t[2]));
      double d2 = v3dot(v3sub(p, q), v3sub(p, q));
      if (d2 < *best2) { *best2 = d2; *bestq = q; }
    }
    return;
  }
  double dl = box_dist2(B.nodes[n.left], p), dr = box_dist2(B.nodes[n.right], p);
  if (dl <= dr) {
    bvh_query(D, B, n.left, p, best2, bestq);
    bvh_query(D, B, n.right, p, best2, bestq);
  } else {
    bvh_query(D, B, n.right, p, best2, bestq);
    bvh_query(D, B, n.left, p, best2, bestq);
  }
}

double mesh_distance(const orc_domain& D, const double* x, double* xb) {
  V3 p = {x[0], x[1], x[2]}, q = p;
  double best2 = INFINITY;
  const OrcBVH* B = static_cast<const OrcBVH*>(D.bvh);
  if (B) {
    bvh_query(D, *B, 0, p, &best2, &q);
  } else {
    for (int64_t i = 0; i < D.ntris; ++i) {
      const int32_t* t = D.tris + 3 * i;
      V3 c = closest_on_triangle(p, mesh_vertex(D, t[0]), mesh_vertex(D, t[1]), mesh_vertex(D, t[2]));
      double d2 = v3dot(v3sub(p, c), v3sub(p, c));
      if (d2 < best2) { best2 = d2; q = c; }
    }
  }
  xb[0] = q.x;
  xb[1] = q.y;
  xb[2] = q.z;
  return std::sqrt(best2);
}

// ---------------------------------------------------------------------------
// Distance to the boundary (Alg. 1 "DistanceToBoundary"), analytic shapes.
// ---------------------------------------------------------------------------
// Signed distance of one CSG primitive and its gradient (standard exact distances).
double csg_one(const orc_csg_node& n, int dim, const double* x, double* grad) {
  const double* p = n.p;
  for (int d = 0; d < 3; ++d) grad[d] = 0.0;
  if (n.prim == 0 || n.prim == 2) {
    // sphere: distance to the centre; capsule: distance to the segment a-b
    double c[3] = {p[0], p[1], p[2]};
    double rad = p[3];
    if (n.prim == 2) {
      double ab[3] = {0, 0, 0}, t = 0.0, l2 = 0.0;
      for (int d = 0; d < dim; ++d) {
        ab[d] = p[3 + d] - p[d];
        t += ab[d] * (x[d] - p[d]);
        l2 += ab[d] * ab[d];
      }
      t = l2 > 0.0 ? std::min(1.0, std::max(0.0, t / l2)) : 0.0;
      for (int d = 0; d < dim; ++d) c[d] = p[d] + t * ab[d];
      rad = p[6];
    }
    double r2 = 0.0;
    for (int d = 0; d < dim; ++d) r2 += (x[d] - c[d]) * (x[d] - c[d]);
    double r = std::sqrt(r2);
    if (r > 0.0) {
      for (int d = 0; d < dim; ++d) grad[d] = (x[d] - c[d]) / r;
    } else {
      grad[0] = 1.0;
    }
    return r - rad;
  }
  if (n.prim == 1) {
    // rounded box: the inner box (half extents - corner) grown by the corner radius
    double rc = p[6], q[3] = {0, 0, 0}, out2 = 0.0, qmax = -INFINITY;
    int imax = 0;
    for (int d = 0; d < dim; ++d) {
      q[d] = std::fabs(x[d] - p[d]) - (p[3 + d] - rc);
      if (q[d] > 0.0) out2 += q[d] * q[d];
      if (q[d] > qmax) { qmax = q[d]; imax = d; }
    }
    if (out2 > 0.0) {
      double od = std::sqrt(out2);
      for (int d = 0; d < dim; ++d)
        grad[d] = q[d] > 0.0 ? ((x[d] >= p[d]) ? 1.0 : -1.0) * q[d] / od : 0.0;
      return od - rc;
    }
    grad[imax] = (x[imax] >= p[imax]) ? 1.0 : -1.0;
    return qmax - rc;
  }
  if (n.prim == 3) {
    double v0 = x[0] - p[0], v1 = x[1] - p[1];
    double rr = std::sqrt(v0 * v0 + v1 * v1);
    if (dim == 2) {
      double q = rr - p[3];
      double sg = q >= 0.0 ? 1.0 : -1.0;
      if (rr > 0.0) { grad[0] = sg * v0 / rr; grad[1] = sg * v1 / rr; } else { grad[0] = -1.0; }
      return std::fabs(q) - p[4];
    }
    double q0 = rr - p[3], q1 = x[2] - p[2];
    double ql = std::sqrt(q0 * q0 + q1 * q1);
    if (ql > 0.0 && rr > 0.0) {
      grad[0] = q0 / ql * v0 / rr;
      grad[1] = q0 / ql * v1 / rr;
      grad[2] = q1 / ql;
    }
    return ql - p[4];
  }
  // half-space with unit outward normal
  double nn = 0.0;
  for (int d = 0; d < dim; ++d) nn += p[3 + d] * p[3 + d];
  nn = std::sqrt(nn);
  double sd = 0.0;
  for (int d = 0; d < dim; ++d) {
    grad[d] = p[3 + d] / nn;
    sd += grad[d] * (x[d] - p[d]);
  }
  return sd;
}

double csg_eval(const orc_problem* P, const double* x, double* grad) {
  const orc_domain& D = P->domain;
  double d = csg_one(D.csg[0], P->dim, x, grad);
  for (int i = 1; i < D.ncsg; ++i) {
    double g[3];
    double s = csg_one(D.csg[i], P->dim, x, g);
    int op = D.csg[i].op;
    if (op == 2) {
      s = -s;
      for (int k = 0; k < 3; ++k) g[k] = -g[k];
    }
    bool take = (op == 0) ? (s < d) : (s > d);
    if (take) {
      d = s;
      for (int k = 0; k < 3; ++k) grad[k] = g[k];
    }
  }
  return d;
}

double distance(const orc_problem* P, const double* x, double* xb) {
  int dim = P->dim;
  const double* p = P->domain.p;
  for (int d = 0; d < 3; ++d) xb[d] = (d < dim) ? x[d] : 0.0;
  switch (P->domain.kind) {
    case ORC_DOM_BOX: {
      double best = INFINITY;
      int bd = 0;
      double bv = 0.0;
      for (int d = 0; d < dim; ++d) {
        double dl = x[d] - p[d], dh = p[3 + d] - x[d];
        if (dl < best) { best = dl; bd = d; bv = p[d]; }
        if (dh < best) { best = dh; bd = d; bv = p[3 + d]; }
      }
      xb[bd] = bv;
      return best;
    }
    case ORC_DOM_BALL: {
      double v[3] = {0, 0, 0}, r2 = 0.0;
      for (int d = 0; d < dim; ++d) { v[d] = x[d] - p[d]; r2 += v[d] * v[d]; }
      double r = std::sqrt(r2);
      if (r == 0.0) { v[0] = 1.0; r = 1.0; }
      for (int d = 0; d < dim; ++d) xb[d] = p[d] + v[d] / r * p[3];
      return p[3] - std::sqrt(r2);
    }
    case ORC_DOM_ANNULUS: {
      double v[3] = {0, 0, 0}, r2 = 0.0;
      for (int d = 0; d < dim; ++d) { v[d] = x[d] - p[d]; r2 += v[d] * v[d]; }
      double r = std::sqrt(r2);
      double din = r - p[3], dout = p[4] - r;
      double rad = (din < dout) ? p[3] : p[4];
      if (r == 0.0) { v[0] = 1.0; r = 1.0; }
      for (int d = 0; d < dim; ++d) xb[d] = p[d] + v[d] / r * rad;
      return (din < dout) ? din : dout;
    }
    case ORC_DOM_CSG: {
      double g[3];
      double sd = csg_eval(P, x, g);
      for (int d = 0; d < dim; ++d) xb[d] = x[d] - sd * g[d];
      return -sd;
    }
    case ORC_DOM_ROUNDED_BOX: {
      // Minkowski sum of the inner box (half extents b - rc) and a ball of radius rc
      double rc = p[6];
      double q[3] = {0, 0, 0}, rel[3] = {0, 0, 0}, inner[3] = {0, 0, 0};
      double outside2 = 0.0, qmax = -INFINITY;
      int imax = 0;
      for (int d = 0; d < dim; ++d) {
        rel[d] = x[d] - p[d];
        inner[d] = p[3 + d] - rc;
        q[d] = std::fabs(rel[d]) - inner[d];
        if (q[d] > 0.0) outside2 += q[d] * q[d];
        if (q[d] > qmax) { qmax = q[d]; imax = d; }
      }
      if (outside2 > 0.0) {
        double od = std::sqrt(outside2);
        for (int d = 0; d < dim; ++d) {
          double c = rel[d];
          if (c > inner[d]) c = inner[d];
          if (c < -inner[d]) c = -inner[d];
          xb[d] = p[d] + c + (rel[d] - c) / od * rc;
        }
        return rc - od;
      }
      xb[imax] = p[imax] + ((rel[imax] >= 0.0) ? p[3 + imax] : -p[3 + imax]);
      return rc - qmax;
    }
    case ORC_DOM_MESH: {
      const OrcBVH* B = static_cast<const OrcBVH*>(P->domain.bvh);
      if (B && B->n > 0) {
        // 1-Lipschitz bound from the corners of the point's cell
        int i0[3];
        for (int d = 0; d < 3; ++d) {
          double sg = std::floor((x[d] - B->lo[d]) / B->h[d]);
          i0[d] = (int)std::min(std::max(sg, 0.0), (double)(B->n - 2));
        }
        double lb = -INFINITY;
        for (int c = 0; c < 8; ++c) {
          int ii = i0[0] + (c & 1), jj = i0[1] + ((c >> 1) & 1), kk = i0[2] + ((c >> 2) & 1);
          double e[3] = {x[0] - (B->lo[0] + ii * B->h[0]), x[1] - (B->lo[1] + jj * B->h[1]),
                         x[2] - (B->lo[2] + kk * B->h[2])};
          double dc = B->dist[ii + (int64_t)B->n * (jj + (int64_t)B->n * kk)];
          lb = std::max(lb, dc - std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]));
        }
        if (lb >= B->thresh) return lb;
      }
      return mesh_distance(P->domain, x, xb);
    }
    default:
      return NAN;
  }
}

void domain_bbox(const orc_problem* P, double lo[3], double hi[3]) {
  const double* p = P->domain.p;
  for (int d = 0; d < 3; ++d) { lo[d] = 0.0; hi[d] = 0.0; }
  for (int d = 0; d < P->dim; ++d) {
    switch (P->domain.kind) {
      case ORC_DOM_BOX:
      case ORC_DOM_CSG: lo[d] = p[d]; hi[d] = p[3 + d]; break;
      case ORC_DOM_BALL: lo[d] = p[d] - p[3]; hi[d] = p[d] + p[3]; break;
      case ORC_DOM_ANNULUS: lo[d] = p[d] - p[4]; hi[d] = p[d] + p[4]; break;
      case ORC_DOM_ROUNDED_BOX: lo[d] = p[d] - p[3 + d]; hi[d] = p[d] + p[3 + d]; break;
      case ORC_DOM_MESH:
        lo[d] = INFINITY;
        hi[d] = -INFINITY;
        for (int64_t i = 0; i < P->domain.nverts; ++i) {
          lo[d] = std::min(lo[d], (double)P->domain.verts[3 * i + d]);
          hi[d] = std::max(hi[d], (double)P->domain.verts[3 * i + d]);
        }
        break;
    }
  }
}

// ---------------------------------------------------------------------------
// Centred Green's function of Lap - sigma_bar on a ball (Supplemental 1.1).
// ---------------------------------------------------------------------------
double green_norm(int dim, double R, double sb) {
  double a = std::sqrt(sb) * R;
  if (dim == 2) {
    // |G| = (1/sb)(1 - 1/I0(a)) = R^2 (I0(a) - 1) / (a^2 I0(a))
    if (a == 0.0) return R * R / 4.0;
    if (a < 2.0) {
      double q = a * a / 4.0, bk = 1.0, s = 0.0;  // s = I0(a) - 1 = sum_{k>=1} b_k
      for (int k = 1; k < 40; ++k) {
        bk *= q / ((double)k * k);
        s += bk;
        if (bk < 1e-22 * s) break;
      }
      return R * R * (s / (a * a)) / (1.0 + s);
    }
    return (1.0 - 1.0 / bI0(a)) / sb;
  }
  // |G| = (1/sb)(1 - a/sinh a) = R^2 (sinh a - a) / (a^2 sinh a)
  if (a == 0.0) return R * R / 6.0;
  if (a < 1.0) {
    double term = a, s = 0.0;  // sinh a - a = sum_{k>=1} a^(2k+1)/(2k+1)!
    for (int k = 1; k < 30; ++k) {
      term *= a * a / ((2.0 * k) * (2.0 * k + 1.0));
      s += term;
      if (term < 1e-22 * s) break;
    }
    return R * R * s / (a * a * std::sinh(a));
  }
  if (a > 30.0) return (1.0 - 2.0 * a * std::exp(-a) / (1.0 - std::exp(-2.0 * a))) / sb;
  return (1.0 - a / std::sinh(a)) / sb;
}

}  // namespace

// ===========================================================================
// exported API
// ===========================================================================
extern "C" {

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox(ctr, key, out);
}

double orc_uniform(uint32_t x) { return uniform01(x); }
void orc_uniforms21(const uint32_t* o, double* u) { uniforms21(o, u); }

void orc_bessel(double x, double out[4]) {
  out[0] = bI0(x);
  out[1] = bI1(x);
  out[2] = bK0(x);
  out[3] = bK1(x);
}

// Supplemental 1.1: G^sigma(x, y) at |y - x| = r on the centred ball, as printed
// (Q2D / 2pi, Q3D / 4pi); sigma -> 0 gives the harmonic Green's function.
double orc_green_G(int dim, double R, double sb, double r) {
  double s = std::sqrt(sb);
  if (dim == 2) {
    if (sb == 0.0) return std::log(R / r) / (2.0 * kPi);
    return (bK0(r * s) - bK0(R * s) / bI0(R * s) * bI0(r * s)) / (2.0 * kPi);
  }
  if (sb == 0.0) return (1.0 / r - 1.0 / R) / (4.0 * kPi);
  double q = std::exp(-r * s) / r -
             std::exp(-R * s) / R * (std::sinh(r * s) / (r * s)) * ((R * s) / std::sinh(R * s));
  return q / (4.0 * kPi);
}

double orc_green_norm(int dim, double R, double sb) { return green_norm(dim, R, sb); }

// Supplemental 1.1: P^sigma on the sphere of the centred ball, as printed.
double orc_green_poisson(int dim, double R, double sb) {
  double a = std::sqrt(sb) * R;
  if (dim == 2) return 1.0 / (2.0 * kPi * R) / bI0(a);
  double ratio = (a == 0.0) ? 1.0 : a / std::sinh(a);
  return ratio / (4.0 * kPi * R * R);
}

double orc_green_cdf(int dim, double R, double sb, double r) {
  double a = std::sqrt(sb) * R, rho = r / R;
  return (dim == 2) ? cdf2(a, rho) : cdf3(a, rho);
}

double orc_green_pdf(int dim, double R, double sb, double r) {
  double a = std::sqrt(sb) * R, rho = r / R;
  return ((dim == 2) ? pdf2(a, rho) : pdf3(a, rho)) / R;
}

// F^{-1}(u): safeguarded Newton on rho in [0,1], run to convergence.
double orc_green_inv(int dim, double R, double sb, double u) {
  double a = std::sqrt(sb) * R;
  double lo = 0.0, hi = 1.0, rho = 0.5;
  for (int it = 0; it < 200; ++it) {
    double F = (dim == 2) ? cdf2(a, rho) : cdf3(a, rho);
    double fres = F - u;
    if (fres == 0.0) break;
    if (fres > 0.0) hi = rho; else lo = rho;
    double p = (dim == 2) ? pdf2(a, rho) : pdf3(a, rho);
    double nr = (p > 0.0) ? rho - fres / p : 0.5 * (lo + hi);
    if (!(nr >= lo && nr <= hi)) nr = 0.5 * (lo + hi);
    double step = std::fabs(nr - rho);
    rho = nr;
    if (step < 1e-16 || hi - lo < 1e-16) break;
  }
  return rho * R;
}

// Reading R23 (not in the paper).  Near the boundary the balls shrink to eps, and the
// extra drift's null weight (about 2n |b| / (R sigma_bar) for a small ball) grows like 1/R
// while the null event's probability sigma_bar |G| ~ sigma_bar R^2 / (2n) shrinks: rare,
// huge weights, a heavy tail.  The bound of delta tracking may differ from ball to ball
// (the ball's integral identity holds for any constant sigma_B > 0), so a ball of radius R
// takes sigma_B = max(sigma_bar, 10 B / R), B >= max |b| the problem's drift bound: its
// drift weight stays bounded and the null events near the boundary stay rare (~ B R).
static const double kDriftBallScale = 10.0;
static double ball_bound(const orc_problem* P, double sb, double R) {
  if (P->drift_bound > 0.0) return std::fmax(sb, kDriftBallScale * P->drift_bound / R);
  return sb;
}

// Reading R22 (ball sample for weights that carry |G'/G|, not in the paper).  A weight with
// the factor |G'(r)/G(r)| (the extra drift's null weight; the gradient's first ball) has an
// infinite second moment when r is drawn from G/|G|: the ratio grows like 1/r at the centre
// (a real log divergence in 3D) and like 1/(R - r) at the sphere.  The sample is drawn
// instead from the mixture q = lambda G/|G| + (1 - lambda) p2, p2 uniform in r (direction
// uniform): the radius uniform picks the part (ur < lambda) and is rescaled to [0, 1) for
// it.  Weighting the source term and the null weight by (G/|G|) / q = f / (lambda f + 1 -
// lambda), f the density of rho = r/R under G/|G|, keeps every expectation and bounds the
// weight (near both ends the uniform part dominates q).  The ratio also reaches 1/lambda
// where G/|G| is dense, and along a walk those factors multiply: every drift ball takes
// lambda = 0.97 (measured on the oracle: the literal 3D drift's per-walk spread 2.5x lower
// and its rare huge walks gone; a 2D drift with ~450 null events per walk 8% noisier), the
// gradient's first ball, a single factor, lambda = 1/2.
static const double kDriftMixLambda = 0.97;
static const double kGradMixLambda = 0.5;
static double mix_radius(int dim, double R, double sb, double ur, double lam, double* mixw) {
  double r;
  if (ur < lam) r = orc_green_inv(dim, R, sb, ur / lam);
  else r = R * ((ur - lam) / (1.0 - lam));
  double a = std::sqrt(sb) * R, rho = r / R;
  double f = (dim == 2) ? pdf2(a, rho) : pdf3(a, rho);
  *mixw = f / (lam * f + (1.0 - lam));
  return r;
}

double orc_mix_radius(int dim, double R, double sb, double ur, double lam, double* mixw) {
  return mix_radius(dim, R, sb, ur, lam, mixw);
}

int orc_field_eval(const orc_problem* prob, const orc_field* fld, const double* x, double* v,
                   double* grad, double* lap) {
  double g[3];
  int rc = field_eval(prob, fld, x, v, g, lap);
  for (int d = 0; d < prob->dim; ++d) grad[d] = g[d];
  return rc;
}

int orc_coeffs(const orc_problem* prob, const double* x, double out[5]) {
  coeffs(prob, x, &out[0], &out[1], &out[2], &out[3], &out[4]);
  return 0;
}

int orc_mesh_prepare(orc_problem* prob) {
  orc_domain& D = prob->domain;
  if (D.kind != ORC_DOM_MESH || prob->dim != 3 || !D.verts || !D.tris || D.ntris < 1) return -1;
  if (D.bvh) return 0;
  OrcBVH* B = new OrcBVH();
  std::vector<V3> cent(D.ntris);
  B->tri.resize(D.ntris);
  for (int64_t i = 0; i < D.ntris; ++i) {
    const int32_t* t = D.tris + 3 * i;
    V3 a = mesh_vertex(D, t[0]), b = mesh_vertex(D, t[1]), c = mesh_vertex(D, t[2]);
    cent[i] = v3mul(v3add(v3add(a, b), c), 1.0 / 3.0);
    B->tri[i] = i;
  }
  bvh_build(D, *B, cent, 0, (int)D.ntris);
  D.bvh = B;
  if (D.grid_res > 0) {
    int n = D.grid_res;
    double vlo[3] = {INFINITY, INFINITY, INFINITY}, vhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < 3 * D.ntris; ++i) {
      V3 v = mesh_vertex(D, D.tris[i]);
      double c[3] = {v.x, v.y, v.z};
      for (int k = 0; k < 3; ++k) { vlo[k] = std::min(vlo[k], c[k]); vhi[k] = std::max(vhi[k], c[k]); }
    }
    double ext = std::max(vhi[0] - vlo[0], std::max(vhi[1] - vlo[1], vhi[2] - vlo[2]));
    double diag2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      B->lo[k] = vlo[k] - 0.02 * ext;
      B->h[k] = (vhi[k] - vlo[k] + 0.04 * ext) / (n - 1);
      diag2 += B->h[k] * B->h[k];
    }
    B->thresh = 0.5 * std::sqrt(diag2);
    B->dist.resize((size_t)n * n * n);
    int64_t total = (int64_t)n * n * n;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < total; ++i) {
      double x[3] = {B->lo[0] + (double)(i % n) * B->h[0], B->lo[1] + (double)((i / n) % n) * B->h[1],
                     B->lo[2] + (double)(i / ((int64_t)n * n)) * B->h[2]};
      double xb[3];
      B->dist[i] = mesh_distance(D, x, xb);
    }
    B->n = n;
  }
  return 0;
}

void orc_mesh_release(orc_problem* prob) {
  delete static_cast<OrcBVH*>(prob->domain.bvh);
  prob->domain.bvh = nullptr;
}

double orc_mesh_distance_brute(const orc_problem* prob, const double* x, double* xbar) {
  orc_domain D = prob->domain;
  D.bvh = nullptr;
  return mesh_distance(D, x, xbar);
}

double orc_distance(const orc_problem* prob, const double* x, double* xbar) {
  double xb[3];
  double d = distance(prob, x, xb);
  for (int i = 0; i < prob->dim; ++i) xbar[i] = xb[i];
  return d;
}

// Supplemental Algorithm 1 (delta-tracking WoS), unrolled into a loop.  The
// recursion multiplies the estimate of the next point by sqrt(alpha(next) /
// alpha(current)) -- in general e^{gamma(next) - gamma(current)} -- and, on a
// null event, by (1 - sigma'(y)/sigma_bar); the source term
// |G| f(y) / sqrt(alpha(x) alpha(y)) (in general |G| f'(y) e^{-gamma(x)}) is
// added at every step.  The exponentials telescope, so the walk carries the
// product W of null weights, accumulates W |G| f'(y) and W e^{gamma(x_n)} g(xbar_n)
// on termination, and multiplies the sum by e^{-gamma(x_0)} at the end.
double orc_walk(const orc_problem* P, const double* x0, uint32_t point, uint32_t walk,
                uint64_t seed, double eps, double sb, int64_t max_steps, int64_t* steps_out,
                int32_t* flags_out) {
  int dim = P->dim;
  double x[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) x[d] = x0[d];
  double W = 1.0, acc = 0.0;
  double g0 = gamma_at(P, x);
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  int64_t k = 0;
  int32_t flags = 0;
  for (;;) {
    double xb[3];
    double d = distance(P, x, xb);
    if (d < eps) {
      // epsilon shell: read g at the closest boundary point (Alg. 1, first branch)
      double gv, gg[3], gl;
      field_eval(P, &P->g, xb, &gv, gg, &gl);
      acc += W * std::exp(gamma_at(P, x)) * gv;
      break;
    }
    if (k >= max_steps) {
      flags |= 1;
      break;
    }
    double R = d;
    uint32_t ctr[4] = {point, walk, (uint32_t)k, 0u}, o0[4];
    philox(ctr, key, o0);
    double mu, ur, dy[3] = {0, 0, 0}, dz[3] = {0, 0, 0};
    step_randoms(dim, o0, &mu, &ur, dy, dz);
    // the extra drift: the ball's own bound (reading R23) and the mixture sample (R22)
    const bool drift = has_drift(P);
    const double sbk = drift ? ball_bound(P, sb, R) : sb;
    double Gn = green_norm(dim, R, sbk);
    double mixw = 1.0;
    double r = drift ? mix_radius(dim, R, sbk, ur, kDriftMixLambda, &mixw) : orc_green_inv(dim, R, sbk, ur);
    double y[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) y[i] = x[i] + r * dy[i];
    double gam_y, sp_y, fp_y, f_y, a_y, b_y[3];
    coeffs(P, y, &gam_y, &sp_y, &fp_y, &f_y, &a_y, b_y);
    acc += W * Gn * fp_y * mixw;                // source term, every step
    if (mu <= sbk * Gn) {                       // volume term: null event at y
      double wn = 1.0 - sp_y / sbk;
      if (drift) {
        double db = 0.0;
        for (int i = 0; i < dim; ++i) db += dy[i] * b_y[i];
        wn += green_dlog(dim, R, sbk, r) * db / sbk;
        wn *= mixw;
      }
      W *= wn;
      for (int i = 0; i < dim; ++i) x[i] = y[i];
    } else {                                    // boundary term: z uniform on the sphere
      for (int i = 0; i < dim; ++i) x[i] = x[i] + R * dz[i];
    }
    ++k;
  }
  double u = acc * std::exp(-g0);
  if (!std::isfinite(u)) flags |= 2;
  if (steps_out) *steps_out = k;
  if (flags_out) *flags_out = flags;
  return u;
}

// cosh z - sinh z / z; below z = 1 by its Taylor series sum_{n>=1} 2n z^{2n} / (2n+1)!,
// where the two terms of the closed form cancel.
double cosh_m_sinhc(double z) {
  if (z >= 1.0) return std::cosh(z) - std::sinh(z) / z;
  double z2 = z * z, term = z2 / 3.0, acc = term;
  for (int n = 1; n < 30 && term > 1e-18 * acc; ++n) {
    term *= z2 / ((2.0 * n) * (2.0 * n + 3.0));
    acc += term;
  }
  return acc;
}

// Supplemental 1.3: grad_x G and grad_x P at the centre, as printed, over G and P.
void grad_ratios(int dim, double R, double sb, double r, double* gG, double* gP) {
  double s = std::sqrt(sb), a = s * R, t = s * r;
  if (dim == 2) {
    if (sb == 0.0) {
      // harmonic: G = ln(R/r)/(2 pi), grad_x G = (y - x)(1/r^2 - 1/R^2)/(2 pi), P = 1/(2 pi R)
      *gG = (1.0 / (r * r) - 1.0 / (R * R)) * r / std::log(R / r);
      *gP = 2.0 / R;
      return;
    }
    double G = bK0(t) - bK0(a) / bI0(a) * bI0(t);                     // 2 pi G
    double dG = s / r * (bK1(t) - bK1(a) / bI1(a) * bI1(t));          // 2 pi |grad G| / |y - x|
    *gG = dG * r / G;
    double P = 1.0 / (R * bI0(a));                                     // 2 pi P
    double dP = sb / R * (1.0 / (a * bI1(a)));                        // 2 pi |grad P| / |z - x|
    *gP = dP * R / P;
    return;
  }
  if (sb == 0.0) {
    *gG = (1.0 / (r * r * r) - 1.0 / (R * R * R)) * r / (1.0 / r - 1.0 / R);
    *gP = 3.0 / R;
    return;
  }
  double G = std::exp(-t) / r - std::exp(-a) / R * (std::sinh(t) / t) * (a / std::sinh(a));   // 4 pi G
  double br = std::exp(-t) * (1.0 + 1.0 / t) -
              cosh_m_sinhc(t) * (std::exp(-a) * (1.0 + 1.0 / a)) / cosh_m_sinhc(a);
  double dG = s / (r * r) * br;                                       // 4 pi |grad G| / |y - x|
  *gG = dG * r / G;
  double P = (a / std::sinh(a)) / (R * R);                            // 4 pi P
  double dP = sb / (R * R) / cosh_m_sinhc(a);                          // 4 pi |grad P| / |z - x|
  *gP = dP * R / P;
}

// Sec. 6 weight window on top of Supplemental Algorithm 1 (see oracle.h for the
// random-number contract).  Branches of one walk share its estimate: every branch
// adds its own weighted source terms and boundary value to the walk's sum.
double orc_walk_ww(const orc_problem* P, const double* x0, uint32_t point, uint32_t walk,
                   uint64_t seed, double eps, double sb, int64_t max_steps, double ww_lo,
                   double ww_hi, int depth, int64_t* steps_out, int32_t* flags_out) {
  int dim = P->dim;
  struct Branch {
    double x[3];
    double W;
    int64_t k;
    uint32_t id;
  };
  std::vector<Branch> pending;
  uint32_t next_id = 1;
  double acc = 0.0;
  double g0 = gamma_at(P, x0);
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  int64_t steps = 0;
  int32_t flags = 0;
  Branch b;
  for (int d = 0; d < 3; ++d) b.x[d] = (d < dim) ? x0[d] : 0.0;
  b.W = 1.0;
  b.k = 0;
  b.id = 0;
  for (;;) {
    // run branch b until it ends
    for (;;) {
      double xb[3];
      double d = distance(P, b.x, xb);
      if (d < eps) {
        double gv, gg[3], gl;
        field_eval(P, &P->g, xb, &gv, gg, &gl);
        acc += b.W * std::exp(gamma_at(P, b.x)) * gv;
        break;
      }
      if (b.k >= max_steps) {
        flags |= 1;
        break;
      }
      double R = d;
      uint32_t blk0 = b.id << 2;
      uint32_t ctr[4] = {point, walk, (uint32_t)b.k, blk0}, o0[4], o1[4];
      philox(ctr, key, o0);
      ctr[3] = blk0 | 1u;
      philox(ctr, key, o1);
      double mu, ur, dy[3] = {0, 0, 0}, dz[3] = {0, 0, 0};
      step_randoms(dim, o0, &mu, &ur, dy, dz);
      const double uww = uniform01(o1[(dim == 2) ? 0 : 2]);  // the window's: block 1, word 0 (2D) or 2 (3D)
      const bool drift = has_drift(P);
      const double sbk = drift ? ball_bound(P, sb, R) : sb;  // readings R22, R23
      double Gn = green_norm(dim, R, sbk);
      double mixw = 1.0;
      double r = drift ? mix_radius(dim, R, sbk, ur, kDriftMixLambda, &mixw) : orc_green_inv(dim, R, sbk, ur);
      double y[3] = {0, 0, 0};
      for (int i = 0; i < dim; ++i) y[i] = b.x[i] + r * dy[i];
      double gam_y, sp_y, fp_y, f_y, a_y, b_y[3];
      coeffs(P, y, &gam_y, &sp_y, &fp_y, &f_y, &a_y, b_y);
      acc += b.W * Gn * fp_y * mixw;
      ++steps;
      ++b.k;
      if (mu <= sbk * Gn) {
        double wn = 1.0 - sp_y / sbk;
        if (drift) {
          double db = 0.0;
          for (int i = 0; i < dim; ++i) db += dy[i] * b_y[i];
          wn += green_dlog(dim, R, sbk, r) * db / sbk;
          wn *= mixw;
        }
        b.W *= wn;
        for (int i = 0; i < dim; ++i) b.x[i] = y[i];
        double aw = std::fabs(b.W);
        if (ww_lo > 0.0 && aw < ww_lo) {
          if (uww < aw / ww_lo) {
            b.W = (b.W < 0.0 ? -ww_lo : ww_lo);
          } else {
            break;  // the branch ends without a boundary value
          }
        } else if (ww_lo > 0.0 && aw > ww_hi) {
          // expected-value splitting: N copies of weight W/m with E[N] = m, N in
          // {floor(m), floor(m) + 1}; m is capped by the room for waiting copies
          // (an integer m then gives exactly m copies, so the split stays unbiased)
          double m = aw / ww_hi;
          double room = (double)(depth - (int64_t)pending.size());
          if (m > room + 1.0) m = room + 1.0;
          double fl = std::floor(m);
          int64_t n = (int64_t)fl + ((uww < fl + 1.0 - m) ? 0 : 1);
          b.W /= m;
          for (int64_t c = 1; c < n; ++c) {
            Branch nb = b;
            nb.id = next_id++;
            pending.push_back(nb);
          }
        }
      } else {
        for (int i = 0; i < dim; ++i) b.x[i] = b.x[i] + R * dz[i];
      }
    }
    if (pending.empty()) break;
    b = pending.back();
    pending.pop_back();
  }
  double u = acc * std::exp(-g0);
  if (!std::isfinite(u)) flags |= 2;
  if (steps_out) *steps_out = steps;
  if (flags_out) *flags_out = flags;
  return u;
}

int orc_solve_ww(const orc_problem* P, const double* pts, int64_t npts, int32_t walks_uniform,
                 uint64_t walk_offset, uint64_t seed, double eps, double sb, int64_t max_steps,
                 double ww_lo, double ww_hi, int depth, double* sum, double* sumsq, int64_t* count,
                 int64_t* stats, int nthreads) {
  if (!(sb > 0.0) || !(eps > 0.0) || !(ww_hi > ww_lo)) return -1;
  int dim = P->dim;
  int64_t st_steps = 0, st_walks = 0, st_capped = 0, st_nonfinite = 0;
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) \
    reduction(+ : st_steps, st_walks, st_capped, st_nonfinite)
  for (int64_t p = 0; p < npts; ++p) {
    double x0[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) x0[d] = pts[d * npts + p];
    double s1 = 0.0, s2 = 0.0;
    for (int32_t j = 0; j < walks_uniform; ++j) {
      int64_t k;
      int32_t fl;
      double u = orc_walk_ww(P, x0, (uint32_t)p, (uint32_t)(walk_offset + (uint64_t)j), seed, eps, sb,
                             max_steps, ww_lo, ww_hi, depth, &k, &fl);
      s1 += u;
      s2 += u * u;
      st_steps += k;
      st_walks += 1;
      st_capped += (fl & 1) ? 1 : 0;
      st_nonfinite += (fl & 2) ? 1 : 0;
    }
    sum[p] += s1;
    sumsq[p] += s2;
    count[p] += walks_uniform;
  }
  if (stats) {
    stats[0] += st_steps;
    stats[1] += st_walks;
    stats[2] += st_capped;
    stats[3] += st_nonfinite;
  }
  return 0;
}

double orc_green_dlog(int dim, double R, double sb, double r) { return green_dlog(dim, R, sb, r); }

void orc_green_grad_ratios(int dim, double R, double sb, double r, double out[2]) {
  grad_ratios(dim, R, sb, r, &out[0], &out[1]);
}

// Supplemental Sec. 2 with the delta-tracking walk: the walk of orc_walk, plus the
// first ball's gradient weights.
double orc_walk_grad(const orc_problem* P, const double* x0, uint32_t point, uint32_t walk,
                     uint64_t seed, double eps, double sb, int64_t max_steps, double* grad_out,
                     int64_t* steps_out, int32_t* flags_out) {
  int dim = P->dim;
  if (has_drift(P)) return NAN;  // the first-ball gradient here has no extra-drift term
  double x[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) x[d] = x0[d];
  double W = 1.0, acc = 0.0, S0 = 0.0;
  double gradG[3] = {0, 0, 0}, gradB[3] = {0, 0, 0};
  double g0 = gamma_at(P, x);
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  int64_t k = 0;
  int32_t flags = 0;
  for (;;) {
    double xb[3];
    double d = distance(P, x, xb);
    if (d < eps) {
      double gv, gg[3], gl;
      field_eval(P, &P->g, xb, &gv, gg, &gl);
      acc += W * std::exp(gamma_at(P, x)) * gv;
      break;
    }
    if (k >= max_steps) {
      flags |= 1;
      break;
    }
    double R = d;
    uint32_t ctr[4] = {point, walk, (uint32_t)k, 0u}, o0[4];
    philox(ctr, key, o0);
    double mu, ur, dy[3] = {0, 0, 0}, dz[3] = {0, 0, 0};
    step_randoms(dim, o0, &mu, &ur, dy, dz);
    double Gn = green_norm(dim, R, sb);
    // the first ball's sample weights grad G / G (~ 1/r at the centre): the mixture sample
    // of reading R22 bounds it (mixw = 1 on the later balls)
    double mixw = 1.0;
    double r = (k == 0) ? mix_radius(dim, R, sb, ur, kGradMixLambda, &mixw) : orc_green_inv(dim, R, sb, ur);
    double y[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) y[i] = x[i] + r * dy[i];
    double gam_y, sp_y, fp_y, f_y, a_y;
    coeffs(P, y, &gam_y, &sp_y, &fp_y, &f_y, &a_y);
    acc += W * Gn * fp_y * mixw;
    bool null_event = mu <= sb * Gn;
    if (k == 0) {
      double gG, gP;
      grad_ratios(dim, R, sb, r, &gG, &gP);
      S0 = Gn * fp_y * mixw;
      for (int i = 0; i < dim; ++i) {
        gradG[i] = gG * dy[i];
        gradB[i] = null_event ? gG * dy[i] : gP * dz[i];
      }
    }
    if (null_event) {
      W *= (1.0 - sp_y / sb) * mixw;
      for (int i = 0; i < dim; ++i) x[i] = y[i];
    } else {
      for (int i = 0; i < dim; ++i) x[i] = x[i] + R * dz[i];
    }
    ++k;
  }
  double e0 = std::exp(-g0);
  double u = acc * e0;
  // grad gamma(x0) = (grad alpha / alpha + grad Phi) / 2
  double av, ga[3], la, pv, gp[3], lp;
  field_eval(P, &P->alpha, x0, &av, ga, &la);
  field_eval(P, &P->phi, x0, &pv, gp, &lp);
  for (int i = 0; i < dim; ++i) {
    double gU = S0 * gradG[i] + (acc - S0) * gradB[i];
    double ggam = 0.5 * (ga[i] / av + gp[i]);
    grad_out[i] = (k == 0) ? NAN : e0 * (gU - acc * ggam);
  }
  if (!std::isfinite(u)) flags |= 2;
  if (steps_out) *steps_out = k;
  if (flags_out) *flags_out = flags;
  return u;
}

// ---------------------------------------------------------------------------
// Next-flight variant (Sec. 5.2; Supplemental 1.2 and Algorithm 2)
// ---------------------------------------------------------------------------
// Q(r): the bracket of the centred G of Supplemental 1.1 (G = Q / (2 pi) in 2D,
// Q / (4 pi) in 3D) on a ball of radius R, taken at any r > 0; V(r) = -Q'(r), the
// bracket of Supplemental 1.2's V.  sigma_bar = 0 gives the Laplace forms.
double nf_Q(int dim, double R, double sb, double r) {
  double s = std::sqrt(sb);
  if (dim == 2) {
    if (sb == 0.0) return std::log(R / r);
    return bK0(r * s) - bK0(R * s) / bI0(R * s) * bI0(r * s);
  }
  if (sb == 0.0) return 1.0 / r - 1.0 / R;
  double a = R * s, t = r * s;
  // e^{-t}/r - e^{-a} sinh(t) / (r sinh(a)) = sinh(a - t) / (r sinh(a)), the form
  // that does not cancel for r near R
  if (a < 300.0) return std::sinh(a - t) / (r * std::sinh(a));
  return std::exp(-t) * (1.0 - std::exp(-2.0 * (a - t))) / (r * (1.0 - std::exp(-2.0 * a)));
}

double nf_V(int dim, double R, double sb, double r) {
  double s = std::sqrt(sb);
  if (dim == 2) {
    if (sb == 0.0) return 1.0 / r;
    return s * (bK1(r * s) + bK0(R * s) / bI0(R * s) * bI1(r * s));
  }
  if (sb == 0.0) return 1.0 / (r * r);
  double a = R * s, t = r * s;
  double em = 2.0 * std::exp(-2.0 * a) / (1.0 - std::exp(-2.0 * a));
  return s / r * (std::exp(-t) * (1.0 + 1.0 / t) + em * cosh_m_sinhc(t));
}

double dot3(const double* a, const double* b, int dim) {
  double acc = 0.0;
  for (int i = 0; i < dim; ++i) acc += a[i] * b[i];
  return acc;
}

double orc_offcentre_G(int dim, double R, double sb, const double* u, const double* v) {
  double w[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i) w[i] = v[i] - u[i];
  double nw = std::sqrt(dot3(w, w, dim));
  double img = (R * R - dot3(u, v, dim)) / R;
  double c = (dim == 2) ? 1.0 / (2.0 * kPi) : 1.0 / (4.0 * kPi);
  return c * (nf_Q(dim, R, sb, nw) - nf_Q(dim, R, sb, img));
}

double orc_offcentre_P(int dim, double R, double sb, const double* u, const double* v) {
  double w[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i) w[i] = v[i] - u[i];
  double nw = std::sqrt(dot3(w, w, dim)), nv = std::sqrt(dot3(v, v, dim));
  double uv = dot3(u, v, dim);
  double img = (R * R - uv) / R;
  double c = (dim == 2) ? 1.0 / (2.0 * kPi) : 1.0 / (4.0 * kPi);
  return c * (nf_V(dim, R, sb, nw) * (nv * nv - uv) / (nw * nv) + nf_V(dim, R, sb, img) * uv / (R * nv));
}

// ---------------------------------------------------------------------------
// Supplemental Sec. 1.2, the off-centred Green's function and Poisson kernel as the
// printed infinite series (Legendre polynomials in 3D, cosines in 2D, with modified
// Bessel functions of the two distances and of R sqrt(sigma_bar)).  Written here in
// the form G = Phi(|x - y|) - H(x, y): the free-space kernel Phi (its addition
// theorem is the part of the printed series in I(r<) K(r>)) in closed form, and the
// regular part H (the part in K(R)/I(R)) as the series, whose terms shrink like
// (r1 r2 / R^2)^n.  With k = sqrt(sigma_bar), a = kR, z = k r:
//   3D: Phi = e^{-kd} / (4 pi d),  H = 1/(4 pi R) sum_n (2n+1) P_n(cos theta) p_n t_n(z1) t_n(z2),
//   2D: Phi = K_0(kd) / (2 pi),    H = 1/(2 pi) sum_{n in Z} cos(n theta) p_n t_n(z1) t_n(z2),
// t_n(z) = i_n(z)/i_n(a) (3D, modified spherical Bessel) or I_n(z)/I_n(a) (2D), and
// p_n = a k_n(a) i_n(a) (3D) or I_n(a) K_n(a) (2D).  The Poisson kernel is the inward
// normal derivative of G at |y - c| = R; term by term the Wronskians
// i_n k_n' - i_n' k_n = -1/z^2 and I_n K_n' - I_n' K_n = -1/z leave
//   3D: P = 1/(4 pi R^2) sum_n (2n+1) P_n(cos theta) t_n(k |x - c|),
//   2D: P = 1/(2 pi R) sum_{n in Z} cos(n theta) t_n(k |x - c|).
// nterms > 0 keeps n = 0 .. nterms - 1 (2D: |n| < nterms); nterms = 0 sums until
// the terms are below rounding.  sigma_bar = 0 takes the Laplace coefficients
// (t_n = (r/R)^n, 3D p_n = 1/(2n+1); 2D: Phi = -ln(d)/(2 pi), the n = 0 term of H
// -ln(R)/(2 pi), p_n = 1/(2|n|)).
// Every Bessel value comes from its defining power series, summed in logarithms
// (no cancellation: all terms are positive), except K_n of 2D, which runs the
// three-term recurrence upwards from the library's K_0 and K_1 (the stable
// direction for K).
namespace {

// ln I_n(z) (2D) or ln i_n(z) (3D), z > 0:
//   I_n(z) = (z/2)^n sum_m (z^2/4)^m / (m! (n+m)!),
//   i_n(z) = z^n / (2n+1)!! sum_m (z^2/2)^m / (m! (2n+3)(2n+5)...(2n+2m+1)).
double ln_bessel_i(int dim, int n, double z) {
  double sum = 1.0, term = 1.0;
  for (int m = 1; m < 1000000; ++m) {
    if (dim == 2) term *= (z * z / 4.0) / ((double)m * (double)(n + m));
    else term *= (z * z / 2.0) / ((double)m * (double)(2 * n + 2 * m + 1));
    sum += term;
    if ((double)m > z && term < 1e-18 * sum) break;
  }
  if (dim == 2) return n * std::log(z / 2.0) - std::lgamma(n + 1.0) + std::log(sum);
  const double ln_dfact = std::lgamma(2.0 * n + 2.0) - n * std::log(2.0) - std::lgamma(n + 1.0);  // (2n+1)!!
  return n * std::log(z) - ln_dfact + std::log(sum);
}

// ln k_n(z), 3D: k_n(z) = e^{-z}/z sum_{j=0}^{n} (n+j)! / (j! (n-j)!) (2z)^{-j}
double ln_sph_k(int n, double z) {
  std::vector<double> lt(n + 1);
  double mx = -INFINITY;
  for (int j = 0; j <= n; ++j) {
    lt[j] = std::lgamma(n + j + 1.0) - std::lgamma(j + 1.0) - std::lgamma(n - j + 1.0) - j * std::log(2.0 * z);
    mx = std::max(mx, lt[j]);
  }
  double s = 0.0;
  for (int j = 0; j <= n; ++j) s += std::exp(lt[j] - mx);
  return -z - std::log(z) + mx + std::log(s);
}

// ln p_n for n = 0 .. N-1 on a ball with a = k R
std::vector<double> series_ln_p(int dim, double a, int N) {
  std::vector<double> lp(N);
  if (dim == 3) {
    for (int n = 0; n < N; ++n) lp[n] = std::log(a) + ln_sph_k(n, a) + ln_bessel_i(3, n, a);
    return lp;
  }
  // K_{n+1} = K_{n-1} + (2n/a) K_n, carried as the ratio K_{n+1}/K_n and ln K_n
  double lnK = std::log(bK0(a)), ratio = bK1(a) / bK0(a);
  for (int n = 0; n < N; ++n) {
    lp[n] = ln_bessel_i(2, n, a) + lnK;
    lnK += std::log(ratio);
    ratio = 2.0 * (n + 1) / a + 1.0 / ratio;
  }
  return lp;
}

struct SeriesGeom {
  double r1, r2, d, mu;
};
SeriesGeom series_geom(int dim, const double* u, const double* v) {
  SeriesGeom g;
  double w[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i) w[i] = v[i] - u[i];
  g.r1 = std::sqrt(dot3(u, u, dim));
  g.r2 = std::sqrt(dot3(v, v, dim));
  g.d = std::sqrt(dot3(w, w, dim));
  g.mu = (g.r1 > 0.0 && g.r2 > 0.0) ? std::fmax(-1.0, std::fmin(1.0, dot3(u, v, dim) / (g.r1 * g.r2))) : 1.0;
  return g;
}

// angular factor of term n: 3D (2n+1) P_n(mu); 2D cos(n theta), doubled for n >= 1 (n and -n)
double series_angle(int dim, int n, double mu) {
  if (dim == 3) return (2.0 * n + 1.0) * std::legendre((unsigned)n, mu);
  return (n == 0 ? 1.0 : 2.0) * std::cos(n * std::acos(mu));
}

// t_n(z) = i_n(z)/i_n(a) (or I_n), with t_n(0) = 0 for n >= 1
double series_t(int dim, int n, double z, double ln_ia) {
  if (z <= 0.0) return (n == 0) ? std::exp(-ln_ia) : 0.0;  // i_0(0) = I_0(0) = 1
  return std::exp(ln_bessel_i(dim, n, z) - ln_ia);
}

const int kSeriesMaxTerms = 100000;

// The regular part H of the series G (G = Phi - H), for the in-ball sampling below.
double series_H(int dim, double R, double sb, const double* u, const double* v, int nterms, double* phi_out);

// ---------------------------------------------------------------------------
// In-ball points of the series walk (reading R24, not in the paper).  Sec. 5.2 leaves the
// in-ball density p^B free (Supplemental 1.4: uniform suffices).  Uniform points make the
// throughput factor theta = G |B| (sigma_bar - sigma') unbounded near the current point
// (G ~ Phi there), and the series' variance infinite once (sigma_bar - sigma')^2 R^4 is of
// order one.  The series walk draws y = x + r w instead: w uniform on the unit sphere
// (circle), r in [0, r_m(w)] (r_m the distance from x to the sphere along w) with density
// proportional to Phi(r) r^{d-1}, Phi the free-space kernel.  With k = sqrt(sigma_bar),
//   p(y) = Phi(r) k^2 / h(k r_m),  h(t) = 1 - e^{-t}(1 + t) (3D),  1 - t K_1(t) (2D)
// (k^2 times the free-space kernel's mass within radius t/k), and since 0 <= G <= Phi,
//   G(x, y) / p(y) = (1 - H/Phi) h(k r_m) / sigma_bar <= 1 / sigma_bar,
// so theta <= 1 - sigma'/sigma_bar: the throughput no longer grows.
// ---------------------------------------------------------------------------
// h and h' = t e^{-t} (3D), t K_0(t) (2D)
double nf_h(int dim, double t) {
  if (dim == 3) {
    if (t < 0.5) {  // sum_{n>=2} (-1)^n (n-1) t^n / n!
      double term = t * t / 2.0, sum = 0.0;
      for (int n = 2; n < 60 && std::fabs(term) > 1e-300; ++n) {
        sum += (n - 1) * term;
        term *= -t / (n + 1);
      }
      return sum;
    }
    return 1.0 - std::exp(-t) * (1.0 + t);
  }
  if (t < 2.0) {
    // DLMF 10.31.1 (n = 1): 1 - t K_1(t) = -t ln(t/2) I_1(t)
    //   + (t^2/4) sum_k (psi(k+1) + psi(k+2)) (t^2/4)^k / (k! (k+1)!)
    if (t == 0.0) return 0.0;
    const double q = t * t / 4.0;
    double c = 1.0, i1 = 0.0, ps = 0.0;  // c = q^k / (k! (k+1)!)
    double psi1 = -kEulerGamma, psi2 = 1.0 - kEulerGamma;  // psi(k+1), psi(k+2)
    for (int k = 0; k < 60; ++k) {
      i1 += c;
      ps += (psi1 + psi2) * c;
      psi1 += 1.0 / (k + 1);
      psi2 += 1.0 / (k + 2);
      c *= q / ((k + 1.0) * (k + 2.0));
      if (c < 1e-20) break;
    }
    i1 *= t / 2.0;
    return -t * std::log(t / 2.0) * i1 + q * ps;
  }
  return 1.0 - t * bK1(t);
}
double nf_hprime(int dim, double t) { return (dim == 3) ? t * std::exp(-t) : t * bK0(t); }

// r in [0, rm] with h(k r) = U h(k rm): safeguarded Newton on t = k r, run to convergence
double nf_free_radius(int dim, double k, double rm, double U) {
  const double tm = k * rm, c = U * nf_h(dim, tm);
  double lo = 0.0, hi = tm, t = tm * std::sqrt(U);
  for (int it = 0; it < 200; ++it) {
    const double f = nf_h(dim, t) - c;
    if (f == 0.0) break;
    if (f > 0.0) hi = t; else lo = t;
    const double d = nf_hprime(dim, t);
    double nt = (d > 0.0) ? t - f / d : 0.5 * (lo + hi);
    if (!(nt >= lo && nt <= hi)) nt = 0.5 * (lo + hi);
    const double step = std::fabs(nt - t);
    t = nt;
    if (step <= 1e-16 * tm || hi - lo <= 1e-16 * tm) break;
  }
  return t / k;
}
}  // namespace

double orc_series_G(int dim, double R, double sb, const double* u, const double* v, int nterms) {
  double phi;
  const double H = series_H(dim, R, sb, u, v, nterms, &phi);
  return phi - H;
}

namespace {
double series_H(int dim, double R, double sb, const double* u, const double* v, int nterms, double* phi_out) {
  const SeriesGeom g = series_geom(dim, u, v);
  const double cd = (dim == 2) ? 1.0 / (2.0 * kPi) : 1.0 / (4.0 * kPi);
  const int N = (nterms > 0) ? nterms : kSeriesMaxTerms;
  double H = 0.0, phi;
  if (sb == 0.0) {
    const double t = g.r1 * g.r2 / (R * R);
    phi = (dim == 2) ? -cd * std::log(g.d) : cd / g.d;
    for (int n = 0; n < N; ++n) {
      double c;
      if (dim == 3) c = std::legendre((unsigned)n, g.mu) * std::pow(t, n) / R;
      else c = (n == 0) ? -std::log(R) : std::cos(n * std::acos(g.mu)) * std::pow(t, n) / n;
      H += cd * c;
      if (nterms == 0 && n > 8 && std::pow(t, n) < 1e-18) break;
    }
    *phi_out = phi;
    return H;
  }
  const double k = std::sqrt(sb), a = k * R, z1 = k * g.r1, z2 = k * g.r2;
  phi = (dim == 2) ? cd * bK0(k * g.d) : cd * std::exp(-k * g.d) / g.d;
  int n_lp = std::min(N, 4096);
  std::vector<double> lp = series_ln_p(dim, a, n_lp);
  for (int n = 0; n < N; ++n) {
    if (n >= n_lp) {  // long sums (nterms = 0 near the sphere): extend p_n
      n_lp = std::min(N, 2 * n_lp);
      lp = series_ln_p(dim, a, n_lp);
    }
    const double ln_ia = ln_bessel_i(dim, n, a);
    const double tt = series_t(dim, n, z1, ln_ia) * series_t(dim, n, z2, ln_ia);
    const double term = series_angle(dim, n, g.mu) * std::exp(lp[n]) * tt;
    H += term * ((dim == 3) ? cd / R : cd);
    if (nterms == 0 && n > 8 && std::fabs(term) * (2.0 * n + 1.0) < 1e-18 * std::fabs(H)) break;
    if (tt == 0.0 && n > 0) break;
  }
  *phi_out = phi;
  return H;
}
}  // namespace

double orc_nf_h(int dim, double t) { return nf_h(dim, t); }
double orc_nf_free_radius(int dim, double sb, double rm, double U) { return nf_free_radius(dim, std::sqrt(sb), rm, U); }

double orc_series_P(int dim, double R, double sb, const double* u, const double* v, int nterms) {
  const SeriesGeom g = series_geom(dim, u, v);
  const double cd = (dim == 2) ? 1.0 / (2.0 * kPi * R) : 1.0 / (4.0 * kPi * R * R);
  const int N = (nterms > 0) ? nterms : kSeriesMaxTerms;
  const double k = std::sqrt(sb), a = k * R, z1 = k * g.r1, s = g.r1 / R;
  double P = 0.0;
  for (int n = 0; n < N; ++n) {
    const double t = (sb == 0.0) ? std::pow(s, n) : series_t(dim, n, z1, ln_bessel_i(dim, n, a));
    const double term = series_angle(dim, n, g.mu) * t;
    P += cd * term;
    if (nterms == 0 && n > 8 && std::fabs(term) < 1e-18 * std::fabs(P / cd)) break;
    if (t == 0.0 && n > 0) break;
  }
  return P;
}

double orc_walk_nf(const orc_problem* P, const double* x0, uint32_t point, uint32_t walk, uint64_t seed,
                   double eps, double sb, int64_t max_steps, int64_t max_inner, int32_t series_terms,
                   int64_t* steps_out, int64_t* inner_out, int32_t* flags_out) {
  int dim = P->dim;
  if (has_drift(P)) return NAN;  // the off-centred series here has no extra-drift term
  double x[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) x[d] = x0[d];
  double W = 1.0, acc = 0.0;
  double g0 = gamma_at(P, x);
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  int64_t k = 0, inner = 0;
  int32_t flags = 0;
  for (;;) {
    double xb[3];
    double d = distance(P, x, xb);
    if (d < eps) {
      double gv, gg[3], gl;
      field_eval(P, &P->g, xb, &gv, gg, &gl);
      acc += W * std::exp(gamma_at(P, x)) * gv;
      break;
    }
    if (k >= max_steps) {
      flags |= 1;
      break;
    }
    double R = d;
    // exit point z, uniform on the sphere, shared by every term of the boundary series
    uint32_t ctr[4] = {point, walk, (uint32_t)k, 0u}, o[4];
    philox(ctr, key, o);
    double dz[3] = {0, 0, 0};
    if (dim == 2) {
      double tz = 2.0 * kPi * uniform01(o[0]);
      dz[0] = std::cos(tz); dz[1] = std::sin(tz);
    } else {
      double cz = 1.0 - 2.0 * uniform01(o[0]), pz = 2.0 * kPi * uniform01(o[1]);
      double sz = std::sqrt(std::fmax(0.0, 1.0 - cz * cz));
      dz[0] = sz * std::cos(pz); dz[1] = sz * std::sin(pz); dz[2] = cz;
    }
    double vz[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) vz[i] = R * dz[i];
    double area = (dim == 2) ? 2.0 * kPi * R : 4.0 * kPi * R * R;
    double vol = (dim == 2) ? kPi * R * R : 4.0 / 3.0 * kPi * R * R * R;
    double uc[3] = {0, 0, 0};  // current sample point minus the ball centre
    double T = 1.0, Ttr = 0.0, Tsrc = 0.0;
    for (int64_t j = 0;; ++j) {
      // P(x_c, z) / p(z): the printed approximation, or the series of series_terms terms
      const double Pv = (series_terms > 0) ? orc_series_P(dim, R, sb, uc, vz, series_terms)
                                           : orc_offcentre_P(dim, R, sb, uc, vz);
      Ttr += Pv * area * T;
      ctr[3] = (uint32_t)(j + 1);
      philox(ctr, key, o);
      double pRR = std::fmin(1.0, std::fabs(T));
      if (pRR < uniform01(o[0])) break;
      T /= pRR;
      if (j >= max_inner) {
        flags |= 4;
        break;
      }
      ++inner;
      // next in-ball point: uniform (printed approximations), or along a uniform direction
      // w at a free-space-kernel distance from the current point (series, reading R24)
      double vn[3] = {0, 0, 0}, w[3] = {0, 0, 0}, Gv;
      if (dim == 2) {
        double th = 2.0 * kPi * uniform01(o[2]);
        w[0] = std::cos(th); w[1] = std::sin(th);
      } else {
        double cn = 1.0 - 2.0 * uniform01(o[2]), pn = 2.0 * kPi * uniform01(o[3]);
        double sn = std::sqrt(std::fmax(0.0, 1.0 - cn * cn));
        w[0] = sn * std::cos(pn); w[1] = sn * std::sin(pn); w[2] = cn;
      }
      if (series_terms > 0) {
        const double k = std::sqrt(sb), uw = dot3(uc, w, dim);
        const double rm = -uw + std::sqrt(std::fmax(0.0, uw * uw + R * R - dot3(uc, uc, dim)));
        const double r = nf_free_radius(dim, k, rm, uniform01(o[1]));
        for (int i = 0; i < dim; ++i) vn[i] = uc[i] + r * w[i];
        double phi;
        const double H = series_H(dim, R, sb, uc, vn, series_terms, &phi);
        Gv = (1.0 - H / phi) * nf_h(dim, k * rm) / sb;  // G(x_c, x_n) / p(x_n)
      } else {
        double rr = (dim == 2) ? R * std::sqrt(uniform01(o[1])) : R * std::cbrt(uniform01(o[1]));
        for (int i = 0; i < dim; ++i) vn[i] = rr * w[i];
        Gv = orc_offcentre_G(dim, R, sb, uc, vn) * vol;  // G(x_c, x_n) / p(x_n)
      }
      double y[3] = {0, 0, 0};
      for (int i = 0; i < dim; ++i) y[i] = x[i] + vn[i];
      double gam_y, sp_y, fp_y, f_y, a_y;
      coeffs(P, y, &gam_y, &sp_y, &fp_y, &f_y, &a_y);
      // source: f'(x_n) / (sigma_bar - sigma'(x_n)) times the updated throughput
      Tsrc += fp_y * Gv * T;
      T *= Gv * (sb - sp_y);
      for (int i = 0; i < dim; ++i) uc[i] = vn[i];
    }
    acc += W * Tsrc;
    W *= Ttr;
    for (int i = 0; i < dim; ++i) x[i] += vz[i];
    ++k;
  }
  double u = acc * std::exp(-g0);
  if (!std::isfinite(u)) flags |= 2;
  if (steps_out) *steps_out = k;
  if (inner_out) *inner_out = inner;
  if (flags_out) *flags_out = flags;
  return u;
}

int orc_walks_nf(const orc_problem* P, const double* pts, int64_t npts, int32_t wpp, uint64_t walk_offset,
                 uint64_t seed, double eps, double sb, int64_t max_steps, int64_t max_inner, int32_t series_terms,
                 double* uhat, int64_t* steps, int64_t* inner, int nthreads) {
  if (!(sb > 0.0) || !(eps > 0.0) || series_terms < 0) return -1;
  int dim = P->dim;
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int64_t p = 0; p < npts; ++p) {
    double x0[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) x0[d] = pts[d * npts + p];
    for (int32_t j = 0; j < wpp; ++j) {
      int64_t i = p * wpp + j, k, m;
      int32_t fl;
      uhat[i] = orc_walk_nf(P, x0, (uint32_t)p, (uint32_t)(walk_offset + j), seed, eps, sb, max_steps, max_inner,
                            series_terms, &k, &m, &fl);
      steps[i] = k;
      inner[i] = m;
    }
  }
  return 0;
}

int orc_solve(const orc_problem* P, const double* pts, int64_t npts, const int32_t* walks,
              int32_t walks_uniform, uint64_t walk_offset, uint64_t seed, double eps, double sb,
              int64_t max_steps, double* sum, double* sumsq, int64_t* count, int64_t* stats,
              int nthreads) {
  if (P->dim != 2 && P->dim != 3) return -1;
  if (!(sb > 0.0) || !(eps > 0.0)) return -1;
  int dim = P->dim;
  int64_t st_steps = 0, st_walks = 0, st_capped = 0, st_nonfinite = 0;
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) \
    reduction(+ : st_steps, st_walks, st_capped, st_nonfinite)
  for (int64_t p = 0; p < npts; ++p) {
    double x0[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) x0[d] = pts[d * npts + p];
    int32_t nw = walks ? walks[p] : walks_uniform;
    double s1 = 0.0, s2 = 0.0;
    for (int32_t j = 0; j < nw; ++j) {
      int64_t k;
      int32_t fl;
      double u = orc_walk(P, x0, (uint32_t)p, (uint32_t)(walk_offset + (uint64_t)j), seed, eps, sb,
                          max_steps, &k, &fl);
      s1 += u;
      s2 += u * u;
      st_steps += k;
      st_walks += 1;
      st_capped += (fl & 1) ? 1 : 0;
      st_nonfinite += (fl & 2) ? 1 : 0;
    }
    sum[p] += s1;
    sumsq[p] += s2;
    count[p] += nw;
  }
  if (stats) {
    stats[0] += st_steps;
    stats[1] += st_walks;
    stats[2] += st_capped;
    stats[3] += st_nonfinite;
  }
  return 0;
}

int orc_walks_grad(const orc_problem* P, const double* pts, int64_t npts, int32_t wpp,
                   uint64_t walk_offset, uint64_t seed, double eps, double sb, int64_t max_steps,
                   double* u, double* grad, int64_t* steps, int nthreads) {
  if (!(sb > 0.0) || !(eps > 0.0)) return -1;
  int dim = P->dim;
  int64_t n = npts * (int64_t)wpp;
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int64_t p = 0; p < npts; ++p) {
    double x0[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) x0[d] = pts[d * npts + p];
    for (int32_t j = 0; j < wpp; ++j) {
      int64_t k;
      int32_t fl;
      double g[3];
      int64_t i = p * wpp + j;
      u[i] = orc_walk_grad(P, x0, (uint32_t)p, (uint32_t)(walk_offset + j), seed, eps, sb, max_steps, g, &k, &fl);
      for (int d = 0; d < dim; ++d) grad[d * n + i] = g[d];
      steps[i] = k;
    }
  }
  return 0;
}

int orc_walks(const orc_problem* P, const double* pts, int64_t npts, int32_t wpp,
              uint64_t walk_offset, uint64_t seed, double eps, double sb, int64_t max_steps,
              double* uhat, int64_t* steps, int nthreads) {
  if (!(sb > 0.0) || !(eps > 0.0)) return -1;
  int dim = P->dim;
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int64_t p = 0; p < npts; ++p) {
    double x0[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) x0[d] = pts[d * npts + p];
    for (int32_t j = 0; j < wpp; ++j) {
      int64_t k;
      int32_t fl;
      uhat[p * wpp + j] = orc_walk(P, x0, (uint32_t)p, (uint32_t)(walk_offset + (uint64_t)j), seed,
                                   eps, sb, max_steps, &k, &fl);
      if (steps) steps[p * wpp + j] = k;
    }
  }
  return 0;
}

// Sec. 5.1 / Sec. 7.1: sigma_bar bounds sigma' over the domain.  The paper's
// default is max(sigma') - min(sigma'); this oracle returns
// max(max - min, max, 1e-3 / diam^2), which equals the paper's value whenever
// min(sigma') < 0 and stays positive otherwise.
int orc_sigma_bar(const orc_problem* P, int m, double* sigma_bar, double* smin, double* smax) {
  int dim = P->dim;
  double lo[3], hi[3];
  domain_bbox(P, lo, hi);
  double mn = INFINITY, mx = -INFINITY, b2max = 0.0;
  int64_t total = 1;
  for (int d = 0; d < dim; ++d) total *= m;
  for (int64_t idx = 0; idx < total; ++idx) {
    double x[3] = {0, 0, 0}, xb[3];
    int64_t r = idx;
    for (int d = 0; d < dim; ++d) {
      x[d] = lo[d] + (r % m + 0.5) * (hi[d] - lo[d]) / m;
      r /= m;
    }
    if (!(distance(P, x, xb) > 0.0)) continue;
    double gm, sp, fp, fv, av, b[3];
    coeffs(P, x, &gm, &sp, &fp, &fv, &av, b);
    if (sp < mn) mn = sp;
    if (sp > mx) mx = sp;
    double b2 = 0.0;
    for (int d = 0; d < dim; ++d) b2 += b[d] * b[d];
    if (b2 > b2max) b2max = b2;
  }
  double diam2 = 0.0;
  for (int d = 0; d < dim; ++d) diam2 += (hi[d] - lo[d]) * (hi[d] - lo[d]);
  double sbv = mx - mn;
  if (mx > sbv) sbv = mx;
  if (1e-3 / diam2 > sbv) sbv = 1e-3 / diam2;
  // extra drift: the variance of its weight term falls like |b|^2 / sigma_bar
  if (50.0 * b2max > sbv) sbv = 50.0 * b2max;
  *sigma_bar = sbv;
  *smin = mn;
  *smax = mx;
  return 0;
}

}  // extern "C"
