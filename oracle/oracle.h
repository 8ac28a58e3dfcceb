/*
 * oracle.h -- plain FP64 CPU oracle for delta-tracking walk on spheres.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links or
 * calls this code.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no source with the CUDA path.
 *
 * It computes, slowly and in double precision, what the paper's method defines
 * (Sawhney, Seyb, Jarosz, Crane, "Grid-Free Monte Carlo for PDEs with Spatially
 * Varying Coefficients", SIGGRAPH 2022):
 *
 *   PDE (eq. 1):   div(alpha grad u) + omega . grad u - sigma u = -f  in Omega,
 *                  u = g on the boundary,   with omega = alpha grad(Phi).
 *   Transform (Sec. 4.1 eq. 7-8 and App. A):
 *                  gamma = 1/2 ln alpha + 1/2 Phi,   U = e^gamma u,
 *                  sigma' = sigma/alpha + Lap(gamma) + |grad gamma|^2,
 *                  f' = e^gamma f / alpha,           g' = e^gamma g,
 *                  Lap U - sigma' U = -f'.
 *   Delta tracking (eq. 11) and the mean-value estimator (eq. 14, Sec. 5.1,
 *   Supplemental Algorithm 1) with centred Green's functions (Supplemental 1.1).
 *
 * All arrays are HOST memory owned by the caller.  Functions never allocate
 * memory that outlives the call.  Errors are reported by return value < 0.
 */
#ifndef WOS_ORACLE_H
#define WOS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* atom types of a separable term: h(t) with t = k*x_i + phi */
enum { ORC_ONE = 0, ORC_SIN = 1, ORC_COS = 2, ORC_EXP = 3, ORC_SINH = 4,
       ORC_COSH = 5, ORC_LIN = 6, ORC_QUAD = 7 };

/* value = c * prod_i h_{type[i]}(k[i] * x_i + phi[i]) */
typedef struct {
  double c;
  int32_t type[3];
  double k[3];
  double phi[3];
} orc_term;

enum { ORC_FIELD_ZERO = 0, ORC_FIELD_CONST = 1, ORC_FIELD_SST = 2,
       ORC_FIELD_MANUFACTURED = 3, ORC_FIELD_GRID_LINEAR = 4,
       ORC_FIELD_GRID_BSPLINE = 5 };

typedef struct {
  int32_t kind;
  int32_t nterms;
  const orc_term* terms;   /* SST: nterms terms */
  double value;            /* CONST */
  int32_t res[3];          /* GRID: nodes per axis, node i at lo + i*(hi-lo)/(res-1) */
  double lo[3];
  double hi[3];
  const float* data;       /* GRID: x fastest, [res2][res1][res0] */
} orc_field;

enum { ORC_DOM_BOX = 0, ORC_DOM_BALL = 1, ORC_DOM_ANNULUS = 2,
       ORC_DOM_ROUNDED_BOX = 3, ORC_DOM_MESH = 4, ORC_DOM_CSG = 5 };

/* one signed-distance CSG node (Sec. 7.2): prim 0 sphere (centre, radius), 1 box
   (centre, half extents, corner radius), 2 capsule (a, b, radius), 3 torus (centre,
   major, minor radius; axis z; 2D: a ring), 4 half-space (point, outward normal);
   op 0 union (min), 1 intersection (max), 2 subtraction (max(d, -s)). */
typedef struct {
  int32_t prim;
  int32_t op;
  double p[8];
} orc_csg_node;

typedef struct {
  int32_t kind;
  double p[16];
  /* BOX: lo p[0..2], hi p[3..5]
     BALL: centre p[0..2], radius p[3]
     ANNULUS: centre p[0..2], inner radius p[3], outer radius p[4]
     ROUNDED_BOX: centre p[0..2], half extents p[3..5], corner radius p[6]
     MESH (3D): closed triangle mesh, host arrays verts [nverts][3], tris [ntris][3];
                orc_mesh_prepare builds the oracle's own BVH into `bvh`. */
  const float* verts;
  int64_t nverts;
  const int32_t* tris;
  int64_t ntris;
  void* bvh;
  /* CSG: nodes combined left to right; p[0..5] bound the domain.  The ball radius is
     -sdf(x) and the closest point x - sdf(x) grad sdf(x). */
  const orc_csg_node* csg;
  int32_t ncsg;
  /* MESH: grid_res > 0 asks orc_mesh_prepare for a grid_res^3 grid of exact distances
     over the triangles' vertex bounds plus 2% of the largest extent; the walk radius is
     then L = max over the cell corners c of (d(c) - |x - c|) when L >= half the cell
     diagonal, else the exact distance. */
  int32_t grid_res;
} orc_domain;

typedef struct {
  int32_t dim;          /* 2 or 3 */
  orc_domain domain;
  orc_field alpha;      /* diffusion coefficient, > 0 */
  orc_field phi;        /* drift potential: omega = alpha * grad(phi) */
  orc_field sigma;      /* screening coefficient */
  orc_field f;          /* source; MANUFACTURED: f = -div(alpha grad um) - omega.grad um + sigma um */
  orc_field g;          /* Dirichlet data, read at the closest boundary point */
  orc_field um;         /* manufactured solution used by f when f.kind == MANUFACTURED */
  /* A further drift, any vector field (the non-conservative part): the PDE's drift is
     omega = alpha grad(phi) + (omega_x, omega_y, omega_z).  Not in the paper: with
     b = omega_extra / alpha the transformed equation gains b . grad U, which is moved
     onto the Green's function by parts on each ball (G = 0 on the sphere), giving
     null weights 1 - (sigma' + b . grad gamma + div b) / sigma_bar
     + |G'(r)/G(r)| (dir_y . b(y)) / sigma_bar.  ZERO fields: no extra drift. */
  orc_field omega[3];
  /* With an extra drift: B >= max |omega_extra / alpha| over the domain, or 0.  B > 0 gives
     each ball its own bound sigma_B = max(sigma_bar, 10 B / R) (reading R23). */
  double drift_bound;
} orc_problem;

/* Philox4x32-10 block (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* uniform in (0,1): (x + 1/2) 2^-32 */
double orc_uniform(uint32_t x);
/* Reading R12, 3D steps: the six uniforms (mu, radius, two per direction) of one Philox
   block o[4] as 21-bit fields (see oracle.cpp). */
void orc_uniforms21(const uint32_t* o, double* u);

/* Bessel I0, I1, K0, K1 as used by the oracle (C++17 special functions). */
void orc_bessel(double x, double out[4]);

/* Centred screened-Poisson Green's function on a ball of radius R, sigma_bar >= 0
   (Supplemental 1.1).  G(r) density value, |G| its integral over the ball,
   F(r) the radial CDF of y ~ G/|G|, pdf = dF/dr, inv = F^{-1}(u). */
double orc_green_G(int dim, double R, double sigma_bar, double r);
double orc_green_norm(int dim, double R, double sigma_bar);
double orc_green_poisson(int dim, double R, double sigma_bar);
double orc_green_cdf(int dim, double R, double sigma_bar, double r);
double orc_green_pdf(int dim, double R, double sigma_bar, double r);
double orc_green_inv(int dim, double R, double sigma_bar, double u);
/* Reading R22: radius r from the uniform ur under the mixture lam G/|G| (ur < lam, rescaled)
   + (1 - lam) uniform radius (ur >= lam, rescaled); *mixw = (G/|G|)/mixture density at r. */
double orc_mix_radius(int dim, double R, double sigma_bar, double ur, double lam, double* mixw);

/* Field value, gradient and Laplacian at x (MANUFACTURED needs the problem). */
int orc_field_eval(const orc_problem* prob, const orc_field* fld, const double* x,
                   double* v, double* grad, double* lap);

/* Transformed coefficients at x: out = {gamma, sigma', f', f, alpha}. */
int orc_coeffs(const orc_problem* prob, const double* x, double out[5]);

/* Distance to the boundary (positive inside) and closest boundary point.  For a
   mesh the distance is unsigned (points are assumed inside the closed surface). */
double orc_distance(const orc_problem* prob, const double* x, double* xbar);

/* Mesh domains: build / free the oracle's BVH (median split of triangle
   centroids, <= 4 triangles per leaf), and the brute-force distance over all
   triangles that pins it. */
int orc_mesh_prepare(orc_problem* prob);
void orc_mesh_release(orc_problem* prob);
double orc_mesh_distance_brute(const orc_problem* prob, const double* x, double* xbar);

/* One delta-tracking walk from x0.  Randoms: Philox4x32-10, key = (seed lo, seed hi),
   counter = (point, walk, step, block).  Returns the estimate of u(x0).
   steps_out: number of sampling steps; flags_out: bit0 capped, bit1 non-finite. */
double orc_walk(const orc_problem* prob, const double* x0, uint32_t point, uint32_t walk,
                uint64_t seed, double eps, double sigma_bar, int64_t max_steps,
                int64_t* steps_out, int32_t* flags_out);

/* Weight window (Sec. 6): after every null event, |W| < lo is Russian roulette
   (survive with |W|/lo, then |W| = lo) and |W| > hi expected-value splitting into
   floor(m) or floor(m)+1 copies (E = m = |W|/hi) of weight W/m.  Copies continue
   depth-first within the walk (last created first); copy b draws its randoms with
   Philox block word (b << 2) | block.  The window's own uniform: 3D block 1 word 2,
   2D block 1 word 0.  At most `depth` copies wait at a time (fewer splits when full,
   which stays unbiased).  lo <= 0 disables it. */
double orc_walk_ww(const orc_problem* prob, const double* x0, uint32_t point, uint32_t walk,
                   uint64_t seed, double eps, double sigma_bar, int64_t max_steps, double ww_lo,
                   double ww_hi, int depth, int64_t* steps_out, int32_t* flags_out);
int orc_solve_ww(const orc_problem* prob, const double* pts, int64_t npts, int32_t walks_uniform,
                 uint64_t walk_offset, uint64_t seed, double eps, double sigma_bar, int64_t max_steps,
                 double ww_lo, double ww_hi, int depth, double* sum, double* sumsq, int64_t* count,
                 int64_t* stats, int nthreads);

/* |G'(r)/G(r)| of the centred Green's function on a ball of radius R (Supplemental 1.1). */
double orc_green_dlog(int dim, double R, double sigma_bar, double r);

/* Gradient of the Green's function and Poisson kernel at the centre of the ball
   (Supplemental 1.3, as printed), divided by the centred G(r) resp. P:
   out[0] = |grad_x G| / G at distance r (the gradient points along y - x),
   out[1] = |grad_x P| / P (along z - x). */
void orc_green_grad_ratios(int dim, double R, double sigma_bar, double r, double out[2]);

/* One walk estimating u(x0) and grad u(x0) (Supplemental Sec. 2): the first ball's
   source sample and branch give grad U(x0) = S0 gG(y0) + (A - S0) g_branch, with
   gG = grad_x G / G (y - x direction) and g_branch = gG on a null event or
   grad_x P / P on a boundary step; grad u = e^{-gamma(x0)} (grad U - U grad gamma(x0)).
   grad_out[dim]; NaN if x0 lies within eps of the boundary. */
double orc_walk_grad(const orc_problem* prob, const double* x0, uint32_t point, uint32_t walk,
                     uint64_t seed, double eps, double sigma_bar, int64_t max_steps, double* grad_out,
                     int64_t* steps_out, int32_t* flags_out);

/* Many gradient walks: u[npts * wpp], grad[dim][npts * wpp] (SoA), steps[npts * wpp]. */
int orc_walks_grad(const orc_problem* prob, const double* pts, int64_t npts, int32_t wpp,
                   uint64_t walk_offset, uint64_t seed, double eps, double sigma_bar, int64_t max_steps,
                   double* u, double* grad, int64_t* steps, int nthreads);

/* Next-flight variant (Sec. 5.2, Supplemental Algorithm 2) on the transformed
   problem.  The approximate off-centred Green's function and Poisson kernel of
   Supplemental 1.2 on a ball of radius R centred at c, with u = x - c, v = y - c
   (v = z - c on the sphere for P); full G and P (not divided by 2 pi / 4 pi).
   Exact at u = 0. */
double orc_offcentre_G(int dim, double R, double sigma_bar, const double* u, const double* v);
double orc_offcentre_P(int dim, double R, double sigma_bar, const double* u, const double* v);
/* The off-centred G and P as the series of Supplemental 1.2 (Legendre polynomials in
   3D, cosines in 2D, modified Bessel functions), G written as the closed-form
   free-space kernel minus the series of its regular part; nterms > 0 keeps the
   terms n < nterms (2D: |n| < nterms), nterms = 0 sums to rounding.  Same
   arguments and scaling as orc_offcentre_G / _P; sigma_bar = 0 gives Laplace's. */
double orc_series_G(int dim, double R, double sigma_bar, const double* u, const double* v, int nterms);
double orc_series_P(int dim, double R, double sigma_bar, const double* u, const double* v, int nterms);
/* The series walk's in-ball sampling (reading R24): h(t) = 1 - e^{-t}(1 + t) (3D) or
   1 - t K_1(t) (2D), and the distance r in [0, rm] with h(sqrt(sigma_bar) r) =
   U h(sqrt(sigma_bar) rm) (density proportional to the free-space kernel times r^{d-1}). */
double orc_nf_h(int dim, double t);
double orc_nf_free_radius(int dim, double sigma_bar, double rm, double U);
/* One next-flight walk.  Randoms: outer step k draws the exit point z from Philox
   block (point, walk, k, 0); inner iteration j of that ball draws its roulette
   uniform and its uniform in-ball point from block (point, walk, k, j + 1).
   steps_out = outer steps (distance queries), inner_out = inner iterations; flags
   bit 0 = outer step cap, bit 1 = non-finite, bit 2 = inner cap hit.
   series_terms = 0: the printed approximate G and P with uniform in-ball points; > 0:
   the series with that many terms (orc_series_G / _P), in-ball points drawn along a
   uniform direction at a distance from the current point with density proportional to
   the free-space kernel (orc_nf_free_radius; the uniforms of the uniform point: word 1
   the distance, words 2, 3 the direction). */
double orc_walk_nf(const orc_problem* prob, const double* x0, uint32_t point, uint32_t walk, uint64_t seed,
                   double eps, double sigma_bar, int64_t max_steps, int64_t max_inner, int32_t series_terms,
                   int64_t* steps_out, int64_t* inner_out, int32_t* flags_out);
int orc_walks_nf(const orc_problem* prob, const double* pts, int64_t npts, int32_t wpp, uint64_t walk_offset,
                 uint64_t seed, double eps, double sigma_bar, int64_t max_steps, int64_t max_inner,
                 int32_t series_terms, double* uhat, int64_t* steps, int64_t* inner, int nthreads);

/* Many walks: pts SoA [dim][npts].  walks[p] (or walks_uniform if walks == NULL)
   walks per point with ids walk_offset .. walk_offset + walks - 1, accumulated
   into sum / sumsq / count (FP64, caller-initialised).  stats: {steps, walks,
   capped, nonfinite} added.  nthreads <= 0: all OpenMP threads. */
int orc_solve(const orc_problem* prob, const double* pts, int64_t npts,
              const int32_t* walks, int32_t walks_uniform, uint64_t walk_offset,
              uint64_t seed, double eps, double sigma_bar, int64_t max_steps,
              double* sum, double* sumsq, int64_t* count, int64_t* stats, int nthreads);

/* Per-walk estimates uhat[p * walks_per_point + j] and step counts. */
int orc_walks(const orc_problem* prob, const double* pts, int64_t npts,
              int32_t walks_per_point, uint64_t walk_offset, uint64_t seed, double eps,
              double sigma_bar, int64_t max_steps, double* uhat, int64_t* steps,
              int nthreads);

/* Range of sigma' over interior nodes of an m^dim lattice on the domain's bounding box,
   and the bound sigma_bar = max(max - min, max, 1e-3 / diam^2). */
int orc_sigma_bar(const orc_problem* prob, int m, double* sigma_bar, double* smin,
                  double* smax);

#ifdef __cplusplus
}
#endif
#endif
