// wos_hostcheck.cpp -- host build of the device step math, for CPU-side checks.
//
// Compiled with a plain C++ compiler from the same header the kernels use, so
// the FP32 and FP64 Green's-function sampling, Bessel approximations and the
// Philox stream can be compared with independent references without a GPU.
// It is a test aid of the product library and never part of a solve.
#include <stdint.h>

#include "wos_math.cuh"

extern "C" {

// which: 0 I0, 1 I1, 2 K0, 3 K1
void wos_hc_bessel_f32(int which, const double* x, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    float v = (float)x[i], r = 0.0f;
    switch (which) {
      case 0: r = (v <= 3.75f) ? wos::as_i0_small(v) : wos::as_i0s_large(v) * expf(v); break;
      case 1: r = (v <= 3.75f) ? wos::as_i1_small(v) : wos::as_i1s_large(v) * expf(v); break;
      case 2:
        r = (v <= 2.0f) ? wos::as_k0_poly(v) - logf(0.5f * v) * wos::as_i0_small(v)
                        : wos::as_k0s_large(v) * expf(-v);
        break;
      case 3:
        r = (v <= 2.0f) ? (1.0f + wos::as_k1_poly(v) + v * logf(0.5f * v) * wos::as_i1_small(v)) / v
                        : wos::as_k1s_large(v) * expf(-v);
        break;
    }
    out[i] = r;
  }
}

void wos_hc_bessel_f64(int which, const double* x, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    double v = x[i];
    switch (which) {
      case 0: out[i] = wos::d_i0(v); break;
      case 1: out[i] = wos::d_i1(v); break;
      case 2: out[i] = wos::d_k0(v); break;
      case 3: out[i] = wos::d_k1(v); break;
    }
  }
}

// |G| / R^2 = q(a)
void wos_hc_green_q(int dim, int fp64, const double* a, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    if (fp64) out[i] = (dim == 2) ? wos::green_q2(a[i]) : wos::green_q3(a[i]);
    else out[i] = (dim == 2) ? wos::green_q2((float)a[i]) : wos::green_q3((float)a[i]);
  }
}

// radial CDF and density at rho for a
void wos_hc_radial(int dim, int fp64, double a, const double* rho, int64_t n, double* F, double* pdf) {
  if (fp64) {
    wos::Radial3<double> r3;
    wos::Radial2<double> r2;
    if (dim == 3) r3.init(a); else r2.init(a);
    for (int64_t i = 0; i < n; ++i) {
      if (dim == 3) r3.eval(rho[i], &F[i], &pdf[i]); else r2.eval(rho[i], &F[i], &pdf[i]);
    }
  } else {
    wos::Radial3<float> r3;
    wos::Radial2<float> r2;
    if (dim == 3) r3.init((float)a); else r2.init((float)a);
    for (int64_t i = 0; i < n; ++i) {
      float f, p;
      if (dim == 3) r3.eval((float)rho[i], &f, &p); else r2.eval((float)rho[i], &f, &p);
      F[i] = f;
      pdf[i] = p;
    }
  }
}

// rho = F^{-1}(u) as the walk computes it
void wos_hc_sample_radius(int dim, int fp64, double a, const double* u, int64_t n, double* rho) {
  for (int64_t i = 0; i < n; ++i) {
    if (fp64) rho[i] = (dim == 2) ? wos::sample_radius<2, double>(a, u[i]) : wos::sample_radius<3, double>(a, u[i]);
    else rho[i] = (dim == 2) ? wos::sample_radius<2, float>((float)a, (float)u[i])
                             : wos::sample_radius<3, float>((float)a, (float)u[i]);
  }
}

void wos_hc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  wos::U4 c = {ctr[0], ctr[1], ctr[2], ctr[3]};
  wos::U4 o = wos::philox4x32_10(c, key[0], key[1]);
  out[0] = o.x;
  out[1] = o.y;
  out[2] = o.z;
  out[3] = o.w;
}

// the walk kernels' form: round keys precomputed from the 64-bit seed (key[0] low word)
void wos_hc_philox_rk(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  uint32_t rk[20];
  wos::philox_round_keys(((uint64_t)key[1] << 32) | key[0], rk);
  wos::U4 c = {ctr[0], ctr[1], ctr[2], ctr[3]};
  wos::U4 o = wos::philox4x32_10_rk(c, rk);
  out[0] = o.x;
  out[1] = o.y;
  out[2] = o.z;
  out[3] = o.w;
}

// the inverse-CDF table the library builds on the device, built here on the host
static float g_tab[2][wos::kTabSize];
static int g_tab_ready[2] = {0, 0};
static const float* host_table(int dim) {
  int k = dim - 2;
  if (!g_tab_ready[k]) {
    for (int i = 0; i < wos::kTabSize; ++i) {
      int ia = i / wos::kTabU, iu = i % wos::kTabU;
      double a = ia * (double)wos::kTabDA, u = wos::tab_u_of_t((double)iu / (wos::kTabU - 1));
      double r = (iu == 0) ? 0.0 : (iu == wos::kTabU - 1) ? 1.0
               : (dim == 2 ? wos::sample_radius<2, double>(a, u) : wos::sample_radius<3, double>(a, u));
      g_tab[k][i] = (float)r;
    }
    g_tab_ready[k] = 1;
  }
  return g_tab[k];
}

// rho and the number of Newton iterations of the FP32 sampler; use_table selects the
// tabulated start (as the kernels do) instead of the closed-form one
void wos_hc_sample_f32(int dim, int use_table, double a, const double* u, int64_t n, double* rho, double* iters) {
  const float* tab = use_table ? host_table(dim) : nullptr;
  for (int64_t i = 0; i < n; ++i) {
    int it = 0;
    float r = (dim == 2) ? wos::sample_radius<2, float>((float)a, (float)u[i], &it, tab)
                         : wos::sample_radius<3, float>((float)a, (float)u[i], &it, tab);
    rho[i] = r;
    iters[i] = it;
  }
}

// gradient ratios at the ball centre, scaled by R: out[2i] = R gG, out[2i+1] = R gP
void wos_hc_grad_ratios(int dim, int fp64, double a, const double* rho, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    if (fp64) {
      double g, p;
      if (dim == 2) wos::grad_ratios<2, double>(a, rho[i], &g, &p);
      else wos::grad_ratios<3, double>(a, rho[i], &g, &p);
      out[2 * i] = g;
      out[2 * i + 1] = p;
    } else {
      float g, p;
      if (dim == 2) wos::grad_ratios<2, float>((float)a, (float)rho[i], &g, &p);
      else wos::grad_ratios<3, float>((float)a, (float)rho[i], &g, &p);
      out[2 * i] = g;
      out[2 * i + 1] = p;
    }
  }
}

// next-flight kernels: out[2i] = G(c + u_i, c + v_i), out[2i+1] = P(c + u_i, c + z_i) (|z_i| = R)
void wos_hc_offcentre(int dim, int fp64, double Rb, double sb, const double* u, const double* v, const double* z,
                      int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    if (fp64) {
      double uu[3] = {u[3 * i], u[3 * i + 1], u[3 * i + 2]}, vv[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
      double zz[3] = {z[3 * i], z[3 * i + 1], z[3 * i + 2]};
      if (dim == 2) {
        wos::NfBall<2, double> b;
        b.init(std::sqrt(sb), Rb);
        out[2 * i] = b.G(uu, vv);
        out[2 * i + 1] = b.P(uu, zz);
      } else {
        wos::NfBall<3, double> b;
        b.init(std::sqrt(sb), Rb);
        out[2 * i] = b.G(uu, vv);
        out[2 * i + 1] = b.P(uu, zz);
      }
    } else {
      float uu[3] = {(float)u[3 * i], (float)u[3 * i + 1], (float)u[3 * i + 2]};
      float vv[3] = {(float)v[3 * i], (float)v[3 * i + 1], (float)v[3 * i + 2]};
      float zz[3] = {(float)z[3 * i], (float)z[3 * i + 1], (float)z[3 * i + 2]};
      if (dim == 2) {
        wos::NfBall<2, float> b;
        b.init(std::sqrt((float)sb), (float)Rb);
        out[2 * i] = b.G(uu, vv);
        out[2 * i + 1] = b.P(uu, zz);
      } else {
        wos::NfBall<3, float> b;
        b.init(std::sqrt((float)sb), (float)Rb);
        out[2 * i] = b.G(uu, vv);
        out[2 * i + 1] = b.P(uu, zz);
      }
    }
  }
}

}  // extern "C"

// next-flight series kernels (N terms): out[2i] = G(c + u_i, c + v_i), out[2i+1] = P(c + v_i, c + z_i)
template <int DIM, typename R>
static void hc_nf_series(double Rb, double sb, int N, const double* u, const double* v, const double* z, int64_t n,
                         double* out) {
  const R k = (R)std::sqrt(sb), rb = (R)Rb, a = k * rb;
  R pn[wos::kNfSeriesMax], ra[wos::kNfSeriesMax];
  wos::nf_series_ball<DIM, R>(a, N, pn, ra);
  const int n0 = N + 12 + (int)std::fmin((double)a, 4096.0);
  for (int64_t i = 0; i < n; ++i) {
    R uu[3], vv[3], zz[3];
    for (int d = 0; d < 3; ++d) {
      uu[d] = (R)u[3 * i + d];
      vv[d] = (R)v[3 * i + d];
      zz[d] = (R)z[3 * i + d];
    }
    R H, Phi, P;
    wos::nf_series_eval<DIM, R>(k, a, rb, N, n0, pn, ra, uu, vv, zz, &H, &Phi, &P);
    out[2 * i] = (double)(Phi - H);
    out[2 * i + 1] = (double)P;
  }
}

extern "C" {

int wos_hc_nf_series(int dim, int fp64, double Rb, double sb, int N, const double* u, const double* v,
                     const double* z, int64_t n, double* out) {
  if (N < 1 || N > wos::kNfSeriesMax) return -1;
  if (dim == 2) {
    if (fp64) hc_nf_series<2, double>(Rb, sb, N, u, v, z, n, out);
    else hc_nf_series<2, float>(Rb, sb, N, u, v, z, n, out);
  } else {
    if (fp64) hc_nf_series<3, double>(Rb, sb, N, u, v, z, n, out);
    else hc_nf_series<3, float>(Rb, sb, N, u, v, z, n, out);
  }
  return 0;
}

// series walk sampling: out[i] = h(t_i) (which = 0) or the radius r with h(k r) = U_i h(k rm) (which = 1)
int wos_hc_nf_free(int dim, int fp64, int which, double sb, double rm, const double* x, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    if (which == 0) {
      out[i] = (dim == 2) ? (fp64 ? wos::nf_free_h<2, double>(x[i]) : (double)wos::nf_free_h<2, float>((float)x[i]))
                          : (fp64 ? wos::nf_free_h<3, double>(x[i]) : (double)wos::nf_free_h<3, float>((float)x[i]));
    } else {
      const double k = std::sqrt(sb);
      out[i] = (dim == 2)
                   ? (fp64 ? wos::nf_free_radius<2, double>(k, rm, x[i])
                           : (double)wos::nf_free_radius<2, float>((float)k, (float)rm, (float)x[i]))
                   : (fp64 ? wos::nf_free_radius<3, double>(k, rm, x[i])
                           : (double)wos::nf_free_radius<3, float>((float)k, (float)rm, (float)x[i]));
    }
  }
  return 0;
}

// the 3D step's six 21-bit uniforms of Philox blocks w[4 i .. 4 i + 3] (out[6 i + j])
void wos_hc_uniforms21(int fp64, const uint32_t* w, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    uint32_t f[6];
    wos::split21(wos::U4{w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]}, f);
    for (int j = 0; j < 6; ++j) out[6 * i + j] = fp64 ? wos::u21<double>(f[j]) : (double)wos::u21<float>(f[j]);
  }
}

// R |G'/G| of the centred Green's function at rho = r/R
void wos_hc_green_dlog(int dim, int fp64, double a, const double* rho, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    if (fp64) out[i] = (dim == 2) ? wos::green_dlog_r<2, double>(a, rho[i]) : wos::green_dlog_r<3, double>(a, rho[i]);
    else out[i] = (dim == 2) ? wos::green_dlog_r<2, float>((float)a, (float)rho[i])
                             : wos::green_dlog_r<3, float>((float)a, (float)rho[i]);
  }
}

// the mixture ball sample: out[2i] = rho, out[2i+1] = its weight, for radius uniforms u
void wos_hc_mix_radius(int dim, int fp64, double a, double lam, const double* u, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    if (fp64) {
      double w = 0.0;
      double rho = (dim == 2) ? wos::mix_sample_radius<2, double>(a, u[i], nullptr, lam, &w)
                              : wos::mix_sample_radius<3, double>(a, u[i], nullptr, lam, &w);
      out[2 * i] = rho;
      out[2 * i + 1] = w;
    } else {
      float w = 0.0f;
      float rho = (dim == 2) ? wos::mix_sample_radius<2, float>((float)a, (float)u[i], nullptr, (float)lam, &w)
                             : wos::mix_sample_radius<3, float>((float)a, (float)u[i], nullptr, (float)lam, &w);
      out[2 * i] = rho;
      out[2 * i + 1] = w;
    }
  }
}

// FP32 uniforms of the walk kernels from Philox words
void wos_hc_uniform_f32(const uint32_t* x, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = (double)wos::to_uniform<float>(x[i]);
}

}  // extern "C"
