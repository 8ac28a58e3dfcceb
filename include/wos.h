/*
 * wos.h -- C interface of the GB300 delta-tracking walk-on-spheres library.
 *
 * The library estimates, at user-given points, the solution of the linear
 * elliptic PDE of Sawhney, Seyb, Jarosz, Crane, "Grid-Free Monte Carlo for PDEs
 * with Spatially Varying Coefficients" (SIGGRAPH 2022), Sec. 3 eq. 1:
 *
 *     div(alpha grad u) + omega . grad u - sigma u = -f   in Omega,
 *     u = g                                               on the boundary,
 *
 * with alpha > 0, omega = alpha grad(Phi) (a drift the paper removes exactly,
 * App. A), by independent random walks of the delta-tracking walk on spheres
 * (Sec. 5.1, eq. 11; Supplemental Algorithm 1) on the transformed screened
 * Poisson equation Lap U - sigma_bar U = -(f' + (sigma_bar - sigma') U) with
 * U = e^gamma u, gamma = (ln alpha + Phi)/2 (Sec. 4.1, eq. 7-8).
 *
 * Conventions
 *   - Every call returns an int status: WOS_OK (0) or a negative WOS_E* code.
 *     No C++ exception crosses this interface.  wos_last_error() returns a
 *     message for the last failure on a context (valid until the next call).
 *   - Arrays marked "device" are CUDA device pointers owned by the caller;
 *     arrays marked "host" are host pointers owned by the caller.  Opaque
 *     handles (wos_ctx, wos_problem) are owned by the library and freed by
 *     their destroy call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device-pointer calls are asynchronous on that stream unless
 *     stated otherwise.
 *   - Points are SoA float32: x coordinates of all points, then y, then z.
 *   - Randomness: Philox4x32-10 with key = (seed low word, seed high word) and
 *     counter = (point index, walk id, step, block); walk ids of one call are
 *     walk_offset .. walk_offset + walks - 1, so a later call with a larger
 *     walk_offset continues the same streams (the accumulators are the
 *     checkpoint state).
 */
#ifndef WOS_H
#define WOS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define WOS_OK 0
#define WOS_EINVAL (-1)       /* invalid argument or problem description */
#define WOS_ENOMEM (-2)       /* device or host allocation failed */
#define WOS_ECUDA (-3)        /* a CUDA runtime call failed (message has details) */
#define WOS_ETIMEOUT (-4)     /* reserved: a bounded device wait gave up */
#define WOS_EUNSUPPORTED (-5) /* valid request the library does not handle */

/* ---- statistics words (device uint64 array of WOS_STATS_WORDS, added to) ---- */
#define WOS_STAT_STEPS 0     /* walk steps: distance query + Green's sample */
#define WOS_STAT_WALKS 1     /* finished walks */
#define WOS_STAT_CAPPED 2    /* walks stopped by max_steps (biased; should be 0) */
#define WOS_STAT_NONFINITE 3 /* walks whose estimate is not finite */
#define WOS_STAT_OUTSIDE 4   /* walks started at a point with distance <= 0 */
#define WOS_STAT_INNER 5     /* next-flight walks: inner (in-ball) iterations; steps count balls */
#define WOS_STAT_MESH_NODES 6 /* mesh walks: BVH nodes visited by the distance queries */
#define WOS_STAT_MESH_TRIS 7  /* mesh walks: triangles tested by the distance queries */
#define WOS_STAT_EXHAUSTED 8  /* mesh walks: queries that found no boundary point (the walk ends
                                 there, at distance 0; should be 0) */
#define WOS_STATS_WORDS 9

/* ---- problem description ---- */

/* atom h(t), t = k x_i + phi, of a separable term */
enum {
  WOS_ATOM_ONE = 0, WOS_ATOM_SIN = 1, WOS_ATOM_COS = 2, WOS_ATOM_EXP = 3,
  WOS_ATOM_SINH = 4, WOS_ATOM_COSH = 5, WOS_ATOM_LIN = 6 /* t */, WOS_ATOM_QUAD = 7 /* t^2 */
};

/* one separable term: c * prod_{i < dim} h_{type[i]}(k[i] * x_i + phi[i]) */
typedef struct {
  double c;
  int32_t type[3];
  double k[3];
  double phi[3];
} wos_term;

enum {
  WOS_FIELD_ZERO = 0,
  WOS_FIELD_CONST = 1,        /* value */
  WOS_FIELD_SST = 2,          /* sum of nterms separable terms (host array, copied) */
  WOS_FIELD_MANUFACTURED = 3, /* source only: f = -div(alpha grad um) - omega.grad um + sigma um */
  WOS_FIELD_GRID_LINEAR = 4,  /* node grid, multilinear interpolation (C^0) */
  WOS_FIELD_GRID_BSPLINE = 5  /* node values as control points of a uniform cubic B-spline (C^2) */
};

/* A scalar field.  Grids: res[i] nodes on [lo[i], hi[i]] (node j at lo + j (hi-lo)/(res-1)),
   float32 values with x fastest, in DEVICE memory owned by the caller, which must keep
   them alive while the problem exists.  Linear grids clamp points to the box; B-spline
   grids clamp control indices (constant extension).  Fields differentiated by the
   method (alpha and Phi: value, gradient, Laplacian) must be CONST, SST or GRID_BSPLINE. */
typedef struct {
  int32_t kind;
  int32_t nterms;
  const wos_term* terms; /* host */
  double value;
  int32_t res[3];
  double lo[3];
  double hi[3];
  const float* data; /* device */
} wos_field_desc;

enum {
  WOS_DOMAIN_BOX = 0,         /* p[0..2] lower corner, p[3..5] upper corner */
  WOS_DOMAIN_BALL = 1,        /* p[0..2] centre, p[3] radius (a disk in 2D) */
  WOS_DOMAIN_ANNULUS = 2,     /* p[0..2] centre, p[3] inner radius, p[4] outer radius */
  WOS_DOMAIN_ROUNDED_BOX = 3, /* p[0..2] centre, p[3..5] half extents, p[6] corner radius */
  WOS_DOMAIN_MESH = 4,        /* 3D closed triangle mesh: verts / tris below */
  WOS_DOMAIN_CSG = 5          /* signed-distance CSG list: csg / ncsg below; p[0..5] a bounding box */
};

/* CSG primitives (signed distance, negative inside) and operations for WOS_DOMAIN_CSG
   (Sec. 7.2: domains given as a list of signed-distance CSG operations).  Node 0 starts
   the list (its op is ignored); node i then combines d = op(d, prim_i):
   UNION min(d, s), INTERSECT max(d, s), SUBTRACT max(d, -s). */
enum {
  WOS_CSG_SPHERE = 0,    /* p[0..2] centre, p[3] radius (a disk in 2D) */
  WOS_CSG_BOX = 1,       /* p[0..2] centre, p[3..5] half extents, p[6] corner radius (0: sharp) */
  WOS_CSG_CAPSULE = 2,   /* p[0..2] end a, p[3..5] end b, p[6] radius */
  WOS_CSG_TORUS = 3,     /* p[0..2] centre, p[3] major radius, p[4] minor radius; axis z (2D: a ring) */
  WOS_CSG_HALFSPACE = 4  /* p[0..2] a point on the plane, p[3..5] outward normal: the side it points away from */
};
enum { WOS_CSG_UNION = 0, WOS_CSG_INTERSECT = 1, WOS_CSG_SUBTRACT = 2 };
typedef struct {
  int32_t prim;
  int32_t op;
  double p[8];
} wos_csg_node;
#define WOS_CSG_MAX_NODES 16

/* Domain.  For WOS_DOMAIN_MESH, verts (HOST float32 [nverts][3]) and tris (HOST int32
   [ntris][3], indices into verts) describe a closed surface; wos_problem_create builds
   a bounding volume hierarchy for closest-point queries (Sec. 7.1) and keeps its own
   copy, so the arrays may be freed afterwards.  Distances to a mesh are unsigned:
   points must lie inside the surface (the library cannot tell).
   For WOS_DOMAIN_CSG, csg (HOST, ncsg in 1..WOS_CSG_MAX_NODES nodes, copied) lists the
   operations and p[0..2], p[3..5] the corners of a box containing the domain (used for the
   sigma_bar lattice).  The walk's ball radius is -sdf(x): for a CSG of exact primitive
   distances this is a lower bound of the distance to the boundary, so the ball lies in the
   domain (any such ball keeps the estimator unbiased; a smaller one only costs steps).
   The closest point is x - sdf(x) grad sdf(x) with the active primitive's gradient. */
typedef struct {
  int32_t kind;
  double p[16];
  const float* verts;
  int64_t nverts;
  const int32_t* tris;
  int64_t ntris;
  const wos_csg_node* csg;
  int32_t ncsg;
  /* WOS_DOMAIN_MESH only: 0 (default) takes every ball radius from an exact closest-point
     query.  n >= 4 builds, at problem creation, an n^3 grid of exact distances to the
     mesh over its bounding box (2% margin) and then takes the radius
     L = max over the 8 corners c of the point's cell of (d(c) - |x - c|), a lower bound of
     the distance (distances are 1-Lipschitz), whenever L >= |cell diagonal| / 2; nearer the
     boundary the exact query runs, bounded by min over the corners of (d(c) + |x - c|).
     A ball inside the domain keeps the estimator unbiased; interior steps then cost eight
     loads instead of a BVH traversal.  Not in the paper (a distance acceleration structure
     in the sense of Sec. 7.1). */
  int32_t mesh_grid_res;
  /* WOS_DOMAIN_MESH only: 0 (default) makes every ball radius the exact distance.  tol in
     (0, 0.5] lets a query stop once it has certified a radius between (1 - tol) d and d (d the
     exact distance): a box is opened only while its distance is below (1 - tol) times the
     best triangle's, and the radius is (1 - tol) times that triangle's distance, a lower
     bound of d.  Any ball inside the domain keeps the estimator unbiased (Sec. 2.2); smaller
     balls cost steps only.  Where the radius falls below eps the exact query runs, so the
     eps-shell test and the closest point for g are those of the exact walk.  Not in the paper
     (Sec. 5.2 names distance queries as the main cost; this bounds their work). */
  double mesh_tol;
} wos_domain_desc;

/* The PDE of Sec. 3 eq. 1 on a domain.  alpha > 0 (diffusion), phi the drift
   potential (omega = alpha grad phi, App. A), sigma (screening), f (source),
   g (Dirichlet data, read at the closest boundary point), um (the manufactured
   solution used when f.kind == WOS_FIELD_MANUFACTURED, else ignored).
   omega[0..dim-1]: a further drift, any vector field (ZERO kinds: none), so the drift
   of eq. 1 is alpha grad phi + omega.  Not in the paper, whose estimator needs
   omega / alpha to be a gradient: with b = omega / alpha the transformed equation keeps
   b . grad U, moved onto the Green's function by parts on each ball (G vanishes on the
   sphere), so a null event at y = x + r dir_y carries the weight
   1 - (sigma' + b . grad gamma + div b)/sigma_bar + |G'(r)/G(r)| (dir_y . b(y))/sigma_bar.
   The components need first derivatives (not WOS_FIELD_GRID_LINEAR).  Supported by
   wos_solve, wos_walk_estimates, wos_solve_host and wos_sigma_bar on analytic domains;
   the other entry points return WOS_EUNSUPPORTED for such a problem. */
typedef struct {
  int32_t dim; /* 2 or 3 */
  wos_domain_desc domain;
  wos_field_desc alpha, phi, sigma, f, g, um;
  wos_field_desc omega[3];
  /* With an extra drift: 0, or B >= max |omega / alpha| over the domain.  The extra drift's
     null weight then uses a mixture sample (half of the radius uniform's range draws from
     G/|G|, half a uniform radius; the source and null weights carry the density ratio),
     which bounds the |G'/G| factor, and each ball of radius R delta-tracks with its own
     bound max(sigma_bar, 10 B / R), which bounds the drift weight of small balls near the
     boundary.  Both keep the expectation (any positive bound per ball is unbiased). */
  double drift_bound;
} wos_problem_desc;

enum { WOS_FP32 = 0, WOS_FP64 = 1 };

/* Parameters of one solve.
   eps:        epsilon-shell width (Sec. 2.1 notation; Alg. 1 stops when d < eps), > 0.
   sigma_bar:  delta-tracking bound (Sec. 5.1), > 0; any positive value is unbiased.
   seed:       Philox key.
   walk_offset: walk id of the first walk of every point.
   max_steps:  step cap per walk (capped walks are counted, not hidden), >= 1.
   precision:  WOS_FP32 walk state (production) or WOS_FP64 (replays the FP64
               reference arithmetic on the same random streams).
   ww_lo, ww_hi, ww_depth: the weight window of Sec. 6 (the paper uses [0.5, 1.5]);
               ww_lo = 0 turns it off.  After every null event the product W of null
               weights is windowed: |W| < ww_lo plays Russian roulette (survive with
               |W|/ww_lo, then |W| = ww_lo); |W| > ww_hi splits the walk into floor(m) or
               floor(m)+1 copies (mean m = |W|/ww_hi) of weight W/m.  Copies run after
               the branch that made them, in the same lane, so each walk's estimate is
               still one sample; at most ww_depth (<= 8) copies wait at a time (m is
               capped by the free room, which keeps the estimator unbiased).  Copy b of a
               walk draws its randoms with block word (b << 2) | block; the window's own
               uniform is block 1 word 2 (3D) or block 1 word 0 (2D).  Only wos_solve and
               wos_walk_estimates support it. */
typedef struct {
  double eps;
  double sigma_bar;
  uint64_t seed;
  uint64_t walk_offset;
  int64_t max_steps;
  int32_t precision;
  int32_t ww_depth;
  double ww_lo;
  double ww_hi;
} wos_params;

typedef struct wos_ctx wos_ctx;
typedef struct wos_problem wos_problem;
typedef struct wos_batch wos_batch;

/* Create a context on CUDA device `device` (allocates a small scratch buffer).
   Errors: WOS_EINVAL (null out pointer), WOS_ECUDA (device not usable). */
int wos_create(wos_ctx** ctx, int device);
/* Free the context and its scratch; problems must be destroyed first. */
int wos_destroy(wos_ctx* ctx);
/* Message of the last failure on ctx ("" if none); never NULL. */
const char* wos_last_error(const wos_ctx* ctx);
/* Library version string. */
const char* wos_version(void);

/* Validate and upload a problem (Sec. 3 eq. 1).  Copies the description; grid data
   stays with the caller; a mesh boundary gets its BVH built here.  Errors: WOS_EINVAL
   (bad dim, kind, term count, grid size, null grid data, alpha/phi given as linear
   grids, mesh not 3D or with an out-of-range index or a non-finite vertex),
   WOS_ENOMEM, WOS_ECUDA. */
int wos_problem_create(wos_ctx* ctx, const wos_problem_desc* desc, wos_problem** prob);
int wos_problem_destroy(wos_problem* prob);

/* The delta-tracking bound (Sec. 5.1, Sec. 7.1: the paper's default is
   max sigma' - min sigma'): sigma' is sampled at the interior nodes of an
   m^dim lattice of cell centres over the domain's bounding box; returns (host)
   sigma_bar = max(max - min, max, 1e-3 / diam^2), min sigma' and max sigma'.  With an extra
   drift omega, sigma' includes b . grad gamma + div b (b = omega/alpha) and sigma_bar is
   at least 50 max |b|^2 (the drift weight's variance falls like |b|^2 / sigma_bar).
   Synchronises `stream`.  Errors: WOS_EINVAL if m < 2 or alpha <= 0 at a node. */
int wos_sigma_bar(wos_ctx* ctx, const wos_problem* prob, int32_t m, double* sigma_bar,
                  double* sigma_prime_min, double* sigma_prime_max, void* stream);

/* Run walks and ADD their estimates to per-point FP64 accumulators.
   pts:    device float32 SoA [dim][npts].
   walks:  device int32 [npts] walks per point, or NULL to use walks_uniform.
   sum, sumsq: device double [npts]; count: device int64 [npts] (zero them to start).
   stats:  device uint64 [WOS_STATS_WORDS] added to, or NULL.
   npts == 0 or zero walks is a no-op.  Points within eps of the boundary return
   g at the closest point (Alg. 1).  Errors: WOS_EINVAL (null pointers, eps or
   sigma_bar not > 0 and finite, max_steps < 1, walks per point > 2^32), WOS_ECUDA. */
int wos_solve(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts,
              const int32_t* walks, int32_t walks_uniform, const wos_params* params,
              double* sum, double* sumsq, int64_t* count, uint64_t* stats, void* stream);

/* As wos_solve with walks_per_point walks per point, also writing every walk's
   estimate uhat[p * walks_per_point + j] and step count steps[...] (device
   arrays of npts * walks_per_point).  For tests and custom estimators. */
int wos_walk_estimates(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts,
                       int32_t walks_per_point, const wos_params* params, double* uhat,
                       int64_t* steps, uint64_t* stats, void* stream);

/* Spatial gradient (Supplemental Sec. 2, with the centre gradients of G and P of
   Supplemental 1.3): as wos_solve, and also ADD every walk's estimate of grad u at
   its point to grad_sum / grad_sumsq, device double SoA [dim][npts] (component d of
   point p at d * npts + p; zero them to start; the count is `count`).  A walk weights
   its first ball's source sample by grad_x G / G at y_0, and the rest of its estimate
   by grad_x G / G (null event) or grad_x P / P at z_0 (boundary step); then
   grad u = e^{-gamma(x_0)} (grad U - U grad gamma(x_0)) with gamma = (ln alpha + Phi)/2.
   The first ball's radius comes from a mixture (half of the radius uniform's range draws
   from G/|G|, half a uniform radius) and its source and null weights carry the density
   ratio of G/|G| to the mixture: this bounds the grad G / G factor, whose second moment
   under G/|G| is infinite, and keeps the expectation of the value and the gradient.  The
   value estimate therefore has wos_solve's expectation, not its walks.
   A point within eps of the boundary has no first ball: its gradient sums are NaN.
   wos_finalize(grad_sum + d * npts, grad_sumsq + d * npts, count, ...) gives
   component d.  Errors: as wos_solve; WOS_EUNSUPPORTED with a weight window. */
int wos_solve_grad(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts,
                   const int32_t* walks, int32_t walks_uniform, const wos_params* params,
                   double* sum, double* sumsq, int64_t* count, double* grad_sum, double* grad_sumsq,
                   uint64_t* stats, void* stream);

/* As wos_walk_estimates, also writing every walk's gradient estimate to grad_hat,
   device double SoA [dim][npts * walks_per_point] (component d of walk
   p * walks_per_point + j at d * npts * walks_per_point + p * walks_per_point + j).
   For tests and custom estimators.  Errors: as wos_walk_estimates; WOS_EUNSUPPORTED
   with a weight window. */
int wos_walk_grad_estimates(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts,
                            int32_t walks_per_point, const wos_params* params, double* uhat,
                            double* grad_hat, int64_t* steps, uint64_t* stats, void* stream);

/* Next-flight walk on spheres (Sec. 5.2, Supplemental Algorithm 2).
   One distance query per ball; in ball B(x) of radius R the walk draws one exit
   point z uniform on the sphere and sums the boundary series
   T_tr = sum_j P(x^j, z)|dB| prod_{l<j} theta_l and the source series
   T_src = sum_{j>=1} f'(x^j) G(x^{j-1}, x^j)|B| prod_{l<j-1} theta_l over uniform
   in-ball points x^j, theta_l = G(x^l, x^{l+1}) |B| (sigma_bar - sigma'(x^{l+1})),
   with Russian roulette of probability min(1, |throughput|) ending the series; the
   walk adds W T_src, sets W *= T_tr and moves to z.  Randoms: ball k of walk (p, w)
   uses Philox block (p, w, k, 0) for z and block (p, w, k, j + 1) for inner
   iteration j.  max_inner (>= 1) caps a ball's iterations (the walk is then counted
   as capped).
   series_terms selects the off-centred G and P (Supplemental 1.2):
     0      the printed approximations: exact at the ball centre only, so the estimate
            is biased where sigma' < sigma_bar (exact when sigma' = sigma_bar
            everywhere), and the approximate P is not integrable near the exit point;
     1..WOS_NF_SERIES_MAX  the printed series with that many terms (n < N in 3D,
            |n| < N in 2D), G as the closed-form free-space kernel minus its regular
            part's series: the exact kernels projected on angular harmonics of degree
            < N, so the estimate's mean is exact for boundary values and sources
            without higher harmonics on the balls' spheres, and P stays bounded
            (about N^2 / |dB|), which keeps the variance finite.  Each inner iteration
            then sums both series in one sweep of about N + 12 + sqrt(sigma_bar) R
            terms.
   Arguments and results as wos_solve (stats: steps = balls, WOS_STAT_INNER = inner
   iterations).  Errors: as wos_solve; WOS_EINVAL if max_inner < 1 or series_terms
   is outside [0, WOS_NF_SERIES_MAX]; WOS_EUNSUPPORTED with a weight window. */
#define WOS_NF_SERIES_MAX 64
int wos_solve_nf(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts,
                 const int32_t* walks, int32_t walks_uniform, const wos_params* params, int64_t max_inner,
                 int32_t series_terms, double* sum, double* sumsq, int64_t* count, uint64_t* stats,
                 void* stream);

/* As wos_walk_estimates for next-flight walks (uhat, steps = balls per walk). */
int wos_walk_estimates_nf(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts,
                          int32_t walks_per_point, const wos_params* params, int64_t max_inner,
                          int32_t series_terms, double* uhat, int64_t* steps, uint64_t* stats, void* stream);

/* Per-point mean, unbiased sample variance of one walk's estimate, and standard
   error of the mean from the accumulators (Sec. 2.2: the estimate is the average
   of single-sample estimates).  All device arrays of npts; any output may be NULL. */
int wos_finalize(wos_ctx* ctx, const double* sum, const double* sumsq, const int64_t* count,
                 int64_t npts, double* mean, double* var, double* stderr_out, void* stream);

/* Gradient of sum_p grad_u[p] * mean_p with respect to the node values of the
   screening field sigma, where mean_p is the estimate wos_solve returns for point p
   with the same points, walks_uniform and params (same seed and walk ids).  Not in
   the paper: the walks are replayed from their Philox streams (no stored paths).
   Given sigma_bar, a walk's path does not depend on sigma; sigma enters only the
   null weights w = 1 - sigma'(y)/sigma_bar with d sigma'/d sigma_m = N_m(y)/alpha(y)
   (Sec. 4.1, Sec. 5.1), so each walk runs twice: once for its total, once adding
   (total - prefix)/w * dw/dsigma_m at every null event.  The two runs are two kernel
   launches on `stream` (per 2^24 walks); the totals between them live in a
   context-owned buffer of 4 (FP32) or 8 (FP64) bytes per walk, grown with cudaMalloc
   when a call needs more (after a device synchronisation), so calls on one context
   are not concurrent.
   grad_u: device double [npts]; grad_sigma: device double [sigma grid nodes], ADDED to.
   Errors: WOS_EUNSUPPORTED unless sigma is WOS_FIELD_GRID_LINEAR and f is not
   WOS_FIELD_MANUFACTURED; WOS_EINVAL as wos_solve. */
int wos_adjoint_sigma(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts,
                      int32_t walks_uniform, const wos_params* params, const double* grad_u,
                      double* grad_sigma, uint64_t* stats, void* stream);

/* Gradient of sum_p grad_u[p] * mean_p with respect to the control values of the cubic
   B-spline alpha grid, by the same path replay as wos_adjoint_sigma (the walks do
   not move with alpha either: sampling uses only the geometry, sigma_bar and the
   randoms).  alpha enters through gamma = (ln alpha + Phi)/2, i.e. through
   e^{-gamma(x_0)}, the sources f' = e^{gamma} f / alpha, the null weights via
   sigma' = sigma/alpha + Lap gamma + |grad gamma|^2, and e^{gamma(x_n)} at the
   boundary (Sec. 4.1, App. A).  grad_alpha: device double [alpha grid nodes], ADDED
   to.  Grids of up to 8192 nodes are accumulated per CTA in shared memory first.
   Launches and the totals buffer as wos_adjoint_sigma.
   Errors: WOS_EUNSUPPORTED unless alpha is WOS_FIELD_GRID_BSPLINE and f is not
   WOS_FIELD_MANUFACTURED; WOS_EINVAL as wos_solve. */
int wos_adjoint_alpha(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts,
                      int32_t walks_uniform, const wos_params* params, const double* grad_u,
                      double* grad_alpha, uint64_t* stats, void* stream);

/* ---- batches of independent problems (not in the paper; many small solves in one launch) ----
   wos_batch_create uploads nprob problems of one dimension (no mesh domains) with HOST
   point offsets [nprob + 1] (points of problem i are offsets[i] .. offsets[i+1]-1 of the
   batch's point array; offsets[0] = 0, non-decreasing) and HOST per-problem sigma_bar
   [nprob] (> 0).  The batch keeps device copies of the problem descriptions (grid data
   stays with the caller) and a prefix-sum buffer for per-point walk counts.
   wos_solve_batch runs every walk of every problem in ONE persistent launch, claiming
   (point, walk) items across problems as walks finish; it allocates nothing and does not
   synchronise, so it can be captured in a CUDA graph.  Arguments and results as
   wos_solve (pts: device SoA [dim][npts of the batch]); params->sigma_bar is ignored.
   Walk streams are keyed by the point's index in the batch. */
int wos_batch_create(wos_ctx* ctx, const wos_problem* const* probs, int32_t nprob, const int64_t* pt_offsets,
                     const double* sigma_bars, wos_batch** batch);
int wos_batch_destroy(wos_batch* batch);
int wos_solve_batch(wos_ctx* ctx, const wos_batch* batch, const float* pts, const int32_t* walks,
                    int32_t walks_uniform, const wos_params* params, double* sum, double* sumsq, int64_t* count,
                    uint64_t* stats, void* stream);

/* Launch schedule of a batch's persistent launch (not in the paper).  The work queue
   hands each warp `chunk` consecutive (point, walk) items at a time: small chunks balance
   the tail, large ones keep a lane on one point (fewer partial-sum flushes).
     chunk          0 = the kernel's rule (total / (warps x 64), 128..2048), else a
                    multiple of 32 in 32..65536
     blocks_per_sm  0 = as many 128-thread blocks as fit, else 1..32 (capped by what fits)
     regs_variant   0 = the default register cap, 1 = 64 registers (8 blocks per SM)
     reserved       0
   The schedule changes which lane runs which walk, not the walks: the same seed gives the
   same walk estimates, and sums that differ only in the order of additions. */
typedef struct {
  int32_t chunk;
  int32_t blocks_per_sm;
  int32_t regs_variant;
  int32_t reserved;
} wos_schedule;

/* Set (sched NULL = default) or read a batch's schedule; WOS_EINVAL for a value out of range. */
int wos_batch_set_schedule(wos_batch* batch, const wos_schedule* sched);
int wos_batch_get_schedule(const wos_batch* batch, wos_schedule* sched);

/* Autotuner: times trial launches of this batch over candidate schedules (the kernel's
   chunk rule and chunks 64..2048, at both register caps), each with walks per point
   reduced to max(1, walks >> trial_shift) (0..16; 4 is a sixteenth), keeps the fastest in the
   batch and returns it with its trial time (*best_ms) and the default schedule's
   (*default_ms; either pointer may be NULL).  It allocates trial accumulators on the device,
   synchronises `stream` after every trial and frees them before returning: call it before
   capturing the batch's solve in a CUDA graph, not inside one.  Arguments as
   wos_solve_batch; the trial sums are discarded. */
int wos_batch_autotune(wos_ctx* ctx, wos_batch* batch, const float* pts, const int32_t* walks,
                       int32_t walks_uniform, const wos_params* params, int32_t trial_shift,
                       wos_schedule* best, double* best_ms, double* default_ms, void* stream);

/* Batch specialisation (not in the paper): compile, with NVRTC for sm_103a, the batched walk
   kernel with every field that all problems of the batch share (the same kind and, for
   CONST and SST fields, the same value or terms) written out as code; grid fields read the
   walk's own problem's grid as before, and fields that differ between problems keep the
   field interpreter.  Both register caps of wos_schedule are compiled, so schedules and
   the autotuner apply unchanged; later wos_solve_batch calls launch these kernels.
   flags: WOS_SPEC_FP32 and/or WOS_SPEC_FP64 (neither = FP32), optionally WOS_SPEC_PLAIN.
   Blocks for the compilation.  Errors: WOS_EINVAL (unknown flag), WOS_EUNSUPPORTED (no
   libnvrtc, a compile error, or problems whose sources differ in being manufactured),
   WOS_ECUDA.  wos_batch_specialized: WOS_SPEC_* bits of the loaded kernels and (if
   uniform_fields is not NULL) the shared fields as bits alpha 1, Phi 2, sigma 4, f 8,
   g 16, u_m 32. */
int wos_batch_specialize(wos_ctx* ctx, wos_batch* batch, int32_t flags);
int wos_batch_specialized(const wos_batch* batch, int32_t* flags_out, int32_t* uniform_fields);

/* End-to-end convenience: HOST points in, HOST mean / variance / stderr out (and
   HOST stats if non-NULL).  Copies the inputs to device buffers owned by the
   context (grown as needed), runs wos_solve on fresh accumulators and
   wos_finalize, copies the results back and synchronises `stream`. */
int wos_solve_host(wos_ctx* ctx, const wos_problem* prob, const float* pts_host, int64_t npts,
                   int32_t walks_uniform, const wos_params* params, double* mean_host,
                   double* var_host, double* stderr_host, uint64_t* stats_host, void* stream);

/* ---- problem-specialised walk kernels (runtime compilation) ----
   The walk (Supplemental Alg. 1) evaluates alpha, Phi, sigma, f, g (and the
   manufactured u, omega) with their gradients and Laplacians at every step
   (Sec. 4.1, App. A).  wos_problem_specialize compiles, with NVRTC for sm_103a,
   the walk kernel of this problem with those fields written out as code (the
   problem's constants folded in); the domain, grids and every other part of the
   walk are the same source as the generic kernel, and the estimates are the
   same up to floating-point rounding.  It blocks for the compilation (seconds)
   and loads the kernels on the problem's device.  Afterwards wos_solve,
   wos_walk_estimates, wos_solve_grad, wos_walk_grad_estimates and
   wos_solve_host on this problem launch the specialised kernel of the matching
   precision and variant, and wos_adjoint_sigma, wos_adjoint_alpha and wos_adjoint
   the specialised adjoint kernels once WOS_SPEC_ADJOINT was asked for; the
   next-flight walks keep the generic kernels (batches: wos_batch_specialize).
   flags: WOS_SPEC_FP32 and/or WOS_SPEC_FP64 (neither = FP32), and the variants
   WOS_SPEC_PLAIN, WOS_SPEC_WINDOW (weight window), WOS_SPEC_GRAD (spatial
   gradient), WOS_SPEC_ADJOINT (both replay adjoints; analytic domains) (none = PLAIN).  Calling it again adds variants; loaded kernels are
   kept until wos_problem_destroy.
   Errors: WOS_EINVAL (null handle, unknown flag); WOS_EUNSUPPORTED (libnvrtc
   not found, a compilation error -- message in wos_last_error -- or a variant
   the problem cannot run, e.g. a window with an extra drift); WOS_ECUDA (load). */
#define WOS_SPEC_FP32 0x1
#define WOS_SPEC_FP64 0x2
#define WOS_SPEC_PLAIN 0x10
#define WOS_SPEC_WINDOW 0x20
#define WOS_SPEC_GRAD 0x40
#define WOS_SPEC_ADJOINT 0x80 /* the path-replay adjoint kernels of wos_adjoint_sigma / _alpha / wos_adjoint */
int wos_problem_specialize(wos_ctx* ctx, wos_problem* prob, int32_t flags);

/* Which specialised kernels a problem holds: OR of the WOS_SPEC_* bits of the
   loaded (precision, variant) pairs.  Host only. */
int wos_problem_specialized(const wos_problem* prob, int32_t* flags_out);

/* The generated program of a description (host only, no device): the field
   code placed after the walk kernel's headers.  Writes up to cap-1 bytes and a
   NUL to buf (may be NULL to query *len = full length).  WOS_EINVAL for an
   invalid description (the reason is written to buf). */
int wos_jit_source(const wos_problem_desc* desc, char* buf, int64_t cap, int64_t* len);

/* Compile (no device, no load) the specialised kernels that flags select for a
   description; *cubin_bytes = size of the sm_103a image.  The compiler log (or
   the reason for a failure) is written to log (cap bytes, NUL-terminated). */
int wos_jit_compile(const wos_problem_desc* desc, int32_t flags, char* log, int64_t log_cap,
                    int64_t* cubin_bytes);

/* The same two for a batch of n descriptions (host only): the generated program of
   wos_batch_specialize, and its NVRTC compile of one precision (both register caps). */
int wos_jit_batch_source(const wos_problem_desc* descs, int32_t n, char* buf, int64_t cap, int64_t* len);
int wos_jit_batch_compile(const wos_problem_desc* descs, int32_t n, int32_t flags, char* log, int64_t log_cap,
                          int64_t* cubin_bytes);

/* ---- progressive slice view (Sec. 7.2) ----
   The paper's interactive path: a solve on the points of a slice plane that adds one walk
   per point per frame to the accumulators (discarding them when the problem is edited),
   and a sphere-traced view of the domain cut by the plane.  Headless: the image goes to a
   device buffer.  3D: a pinhole camera (eye, look-at point, up vector, vertical field of
   view in degrees) and a slice rectangle plane_origin + a plane_u + b plane_v, a, b in
   [0, 1), with plane_u orthogonal to plane_v.  2D: the rectangle is axis-aligned
   (plane_u along x, plane_v along y) and fills the image; the camera is ignored.  The
   slice grid is slice_nu x slice_nv cell centres, point index iv * slice_nu + iu.
   Values are mapped linearly from [value_lo, value_hi] onto a blue-white-red scale. */
typedef struct {
  double eye[3], look[3], up[3];
  double fov_y_deg;
  double plane_origin[3], plane_u[3], plane_v[3];
  int32_t slice_nu, slice_nv;
  int32_t width, height;
  double value_lo, value_hi;
} wos_view;

/* Write the slice grid's points, device float32 SoA [dim][slice_nu * slice_nv], for the
   solve entry points.  Errors: WOS_EINVAL (degenerate rectangle or camera). */
int wos_slice_points(wos_ctx* ctx, const wos_problem* prob, const wos_view* view, float* pts, void* stream);

/* Render the view: per pixel a ray sphere-traced against the domain with the part on the
   eye's side of the plane cut away (3D).  Where the ray meets the plane inside the domain
   the pixel shows mean = sum / count of its slice cell (grey if count is 0); where it meets
   the boundary it shows g there, Lambert-shaded by the normal of the signed distance.
   rgba: device uint8 [height][width][4]; value: device float [height][width] with the
   shown mean (NaN elsewhere), or NULL; depth: device float [height][width] ray parameter
   of the hit (INFINITY on a miss; 3D only), or NULL.  sum, count: the slice points'
   accumulators.  Errors: WOS_EINVAL (bad view, value_hi <= value_lo), WOS_EUNSUPPORTED
   (mesh domains: their distance is unsigned). */
int wos_render_slice(wos_ctx* ctx, const wos_problem* prob, const wos_view* view, const double* sum,
                     const int64_t* count, uint8_t* rgba, float* value, float* depth, void* stream);

/* ---- problem handles: the problem statement of Sec. 3 piece by piece ----
   The calls below build a problem from separate handles for the domain Omega and the
   scalar fields of eq. 1 (alpha > 0, sigma, the drift potential Phi with
   omega = alpha grad Phi, the source f and the Dirichlet data g), and return per-point
   means and variances directly.  They are layered on wos_problem_desc / wos_solve and
   give the same estimates for the same problem, seed and walks.  A handle is owned by
   the library until its destroy call; a problem keeps no reference to the handles it
   was assembled from (grid data stay with the caller and must outlive the problem).
   ctx may be NULL for the domain and field constructors (errors are then reported by
   the return code only). */
typedef struct wos_domain wos_domain;
typedef struct wos_field wos_field;

/* Axis-aligned box [lo, hi] (dim = 2 or 3; host arrays of dim values).  WOS_EINVAL
   unless hi > lo in every axis and all values are finite. */
int wos_domain_box(wos_ctx* ctx, int32_t dim, const double* lo, const double* hi, wos_domain** out);
/* Analytic signed-distance domain: kind WOS_DOMAIN_BALL (a disk in 2D), WOS_DOMAIN_ANNULUS
   or WOS_DOMAIN_ROUNDED_BOX, params (host) laid out as wos_domain_desc.p for that kind
   (ball 4 values, annulus 5, rounded box 7).  WOS_EINVAL for another kind, a non-positive
   radius or extent, or a corner radius beyond a half extent. */
int wos_domain_sdf(wos_ctx* ctx, int32_t dim, int32_t kind, const double* params, wos_domain** out);
/* Closed triangle mesh (3D, Sec. 7.1): verts DEVICE float32 [nverts][3], tris DEVICE int32
   [ntris][3].  The arrays are copied to the host here (this call synchronises the legacy
   default stream); the bounding volume hierarchy is built when a problem is assembled on
   the domain.  WOS_EINVAL for an index out of range, a non-finite vertex, or a surface that
   is not closed (some edge not shared by exactly two triangles).  Points must lie inside. */
int wos_domain_mesh(wos_ctx* ctx, const float* verts, int64_t nverts, const int32_t* tris, int64_t ntris,
                    wos_domain** out);
int wos_domain_destroy(wos_domain* dom);

/* Analytic field of a family:
     WOS_FIELD_ZERO          nparams 0;
     WOS_FIELD_CONST         params[0] = the value (nparams 1);
     WOS_FIELD_SST           a sum of nparams / 10 separable terms, each packed as 10
                             doubles (c, type[0..2], k[0..2], phi[0..2]; see wos_term);
     WOS_FIELD_MANUFACTURED  the manufactured solution u_m packed as for SST: used as the
                             source f, it stands for f = -div(alpha grad u_m) - omega.grad u_m
                             + sigma u_m with the problem's own alpha, Phi and sigma.
   WOS_EINVAL for another family, a bad term count or atom type, or non-finite values. */
int wos_field_analytic(wos_ctx* ctx, int32_t family_id, const double* params, int32_t nparams, wos_field** out);
/* Grid field: res[i] >= 2 nodes on [lo[i], hi[i]] (host arrays of dim values), DEVICE
   float32 node values (x fastest) owned by the caller, interp WOS_FIELD_GRID_LINEAR
   (multilinear) or WOS_FIELD_GRID_BSPLINE (node values as cubic B-spline control points;
   alpha and Phi need this one). */
int wos_field_grid(wos_ctx* ctx, int32_t dim, const int32_t* res, const double* lo, const double* hi,
                   const float* data, int32_t interp, wos_field** out);
int wos_field_destroy(wos_field* field);

/* Assemble the problem of eq. 1 on a domain: alpha, sigma, f and g are required, Phi may
   be NULL (no drift).  The fields' dimension must match the domain's.  Then as
   wos_problem_create (validation, upload, BVH of a mesh domain). */
int wos_problem_assemble(wos_ctx* ctx, const wos_domain* dom, const wos_field* alpha, const wos_field* sigma,
                         const wos_field* phi, const wos_field* f, const wos_field* g, wos_problem** prob);

/* The paper's default delta-tracking bound (Sec. 5.1, Sec. 7.1) with the library's lattice:
   wos_sigma_bar with m = 256 in 2D and 128 in 3D, on the legacy default stream
   (synchronised).  Any output pointer but sigma_bar may be NULL. */
int wos_problem_sigma_bar(wos_ctx* ctx, const wos_problem* prob, double* sigma_bar, double* sigma_prime_min,
                          double* sigma_prime_max);

/* Run walks and return per-point estimates (Sec. 2.2: the mean of single-walk estimates):
   mean, var (unbiased sample variance of one walk's estimate) and count, DEVICE arrays of
   npts.  If count[p] > 0 on entry, the new walks are merged with (mean[p], var[p],
   count[p]) by the pairwise update of Chan, Golub and LeVeque, so a call with a later
   walk_offset continues an estimate (pass zeroed counts to start).  Walks go to
   context-owned FP64 accumulators first (grown with cudaMalloc when npts exceeds their
   size; otherwise nothing is allocated).  Other arguments and errors as wos_solve. */
int wos_solve_mean(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts, const int32_t* walks,
                   int32_t walks_uniform, const wos_params* params, double* mean, double* var, int64_t* count,
                   uint64_t* stats, void* stream);

/* Solve many problems of one dimension in one persistent launch and return per-point
   estimates as wos_solve_mean.  pt_offsets: HOST [nprob + 1] (points of problem i are
   pt_offsets[i] .. pt_offsets[i+1]-1 of pts); sigma_bars: HOST [nprob] or NULL (then each
   problem's wos_problem_sigma_bar).  A batch is created, run and freed inside the call,
   which therefore allocates and synchronises `stream`; for repeated solves of one batch
   (and CUDA graphs) use wos_batch_create and wos_solve_batch. */
int wos_solve_batched(wos_ctx* ctx, const wos_problem* const* probs, int32_t nprob, const int64_t* pt_offsets,
                      const double* sigma_bars, const float* pts, const int32_t* walks, int32_t walks_uniform,
                      const wos_params* params, double* mean, double* var, int64_t* count, uint64_t* stats,
                      void* stream);

/* Gradient of sum_p grad_u[p] * mean_p with respect to the sigma grid's node values
   (grad_sigma, DEVICE float32 [sigma nodes]) and to the alpha B-spline grid's control
   values (grad_alpha, DEVICE float32 [alpha nodes]), WRITTEN (not added), by the path
   replay of wos_adjoint_sigma and wos_adjoint_alpha (FP64 accumulation, then rounded).
   Either output may be NULL; a non-NULL one needs that field to be a grid of the kind
   those calls accept (else WOS_EUNSUPPORTED).  Uses context-owned FP64 buffers (grown
   with cudaMalloc as needed). */
int wos_adjoint(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts, int32_t walks_uniform,
                const wos_params* params, const double* grad_u, float* grad_sigma, float* grad_alpha,
                uint64_t* stats, void* stream);

/* ---- measurement utilities (not part of the method) ----
   Sustained rates of the units the walk kernels use, measured on the context's device
   (which must be current) with CUDA events around five launches after one warm-up:
     WOS_PEAK_FP32_LANES  FP32 fused multiply-add lane operations per second (independent
                          chains; the lanes' rate also bounds the issue of every instruction);
     WOS_PEAK_MUFU        special-function lane operations per second (approximate
                          reciprocal square roots, independent chains);
     WOS_PEAK_L2_READ     bytes per second read by 16-byte cache-global loads (L1 bypassed)
                          from buf, a zero-filled 16-byte aligned DEVICE buffer of `bytes`
                          (>= 1 MiB) small enough to stay in L2, read about 40 GB per launch.
   *rate receives the rate, *ms (may be NULL) one launch's duration.  Synchronises `stream`. */
#define WOS_PEAK_FP32_LANES 0
#define WOS_PEAK_MUFU 1
#define WOS_PEAK_L2_READ 2
int wos_measure_peak(wos_ctx* ctx, int32_t which, void* buf, int64_t bytes, double* rate, double* ms, void* stream);

/* ---- allocation-free solve ----
   The paper has no counterpart: this entry point exists for callers that cannot
   allocate device memory -- code running inside an allocator hook or a memory-pool
   callback (allocating there would re-enter the allocator), plugins whose host program
   owns every allocation and forbids cudaMalloc/cudaFree, and programs that must not
   synchronise the device (cudaFree does).  It needs no context and no wos_problem: the
   problem description is passed directly, and the walk kernel's scratch (work counter,
   default statistics, the problem description and the per-point walk prefix sums)
   lives in one static device array of WOS_NOALLOC_SCRATCH_BYTES that the library's
   module image carries, so every GPU that loads this library holds it until the process
   exits.  The call performs no cudaMalloc, cudaFree or other allocating routine, and
   it does not block the host: the description reaches the device as a kernel argument.

   Same arguments and results as wos_solve, on the CURRENT CUDA device, except:
     - desc: host problem description (validated on every call; grid data are device
       pointers owned by the caller).  Only analytic domains (box, ball, annulus,
       rounded box) without an extra drift: mesh domains need a BVH built and stored at
       problem creation, CSG lists do not fit the static description, and both return
       WOS_EINVAL here, as does a non-ZERO omega;
     - walks (per-point counts) is limited to npts <= WOS_NOALLOC_MAX_VAR_POINTS, the
       capacity of the static prefix-sum buffer; larger npts with walks != NULL returns
       WOS_EINVAL (uniform walk counts have no point limit);
     - no weight window (WOS_EUNSUPPORTED when ww_lo != 0);
     - errors are reported by the return code only (WOS_EINVAL, WOS_ECUDA);
     - FP32 walks start Newton from the closed-form guess instead of the context's
       inverse-CDF table: same distribution, somewhat slower.
   Every call asks the runtime for the static array's address on the current device
   (cudaGetSymbolAddress); the first call on a device also loads the library's module
   there, so make that first call before any CUDA stream capture.  Every call on a
   device shares the one array and resets what must start at zero; the array keeps the
   last call's contents otherwise.  Calls whose work overlaps on the GPU (other streams,
   other host threads) race on it and must be serialised by the caller. */
#define WOS_NOALLOC_MAX_VAR_POINTS 65536
#define WOS_NOALLOC_SCRATCH_BYTES (16640 + 8 * WOS_NOALLOC_MAX_VAR_POINTS)
int wos_solve_noalloc(const wos_problem_desc* desc, const float* pts, int64_t npts, const int32_t* walks,
                      int32_t walks_uniform, const wos_params* params, double* sum, double* sumsq,
                      int64_t* count, uint64_t* stats, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* WOS_H */
