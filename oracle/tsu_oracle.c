/*
 * tsu_oracle.c -- plain, slow, FP64 CPU oracle for the regularised 2D tsunami
 * wave equation stepped by explicit leapfrog.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the bench's CPU
 * baseline may load this library.  It shares no code, header, constant or
 * helper with the CUDA path and must never be used as a fallback for it.
 *
 * What it computes (paper: "Tsunami propagation for singular topographies"):
 *   PDE      u_tt = d_x(h_x d_x u) + d_y(h_y d_y u)           -- Sec. 2, eq. (2.1)
 *                                                               (vector depth h = (h_1, h_2))
 *   box      [0,1]^2 with zero Dirichlet data on its edges    -- Sec. 3.3 (2D BVP)
 *   grid     x_i = i dx, y_j = j dy, i = 0..nx-1, j = 0..ny-1  -- Sec. 3.3, grid omega (2dwave_2)
 *   depth    h_eps = background + sum_s amp_s * phi_eps(dist_s)^p_s,
 *            phi_eps a unit-mass mollifier of width eps        -- Sec. 2.1 (h * psi_eps), Sec. 3.1
 *   energy   d/dt (||u_t||^2 + sum_j ||h_j^1/2 d_j u||^2) = 0   -- Theorem 2.1, identity (CL-01)
 *   d h_eps / d eps, the depth's derivative in the regularisation width  -- Sec. 2.1
 *   an FP32 emulation of the stepping in both forms (rounding study only)
 *   and the implicit comparator: a factorized scheme with line-wise tridiagonal
 *   systems (Sec. 3.3 names an implicit scheme solved along lines; the scheme
 *   itself is a reading, written out at its section below)
 *
 * The scheme is the explicit leapfrog written out exactly as defined:
 *   fx(u)_ij = hx_ij (u_i+1,j - u_ij) - hx_i-1,j (u_ij - u_i-1,j)
 *   fy(u)_ij = hy_ij (u_i,j+1 - u_ij) - hy_i,j-1 (u_ij - u_i,j-1)
 *   B u      = cx fx(u) + cy fy(u),   cx = tau^2/dx^2,  cy = tau^2/dy^2   (B = tau^2 L_h)
 *   u^1      = (u^0 + tau u1) + B u^0 / 2                       (Taylor start)
 *   u^{n+1}  = (2 u^n - u^{n-1}) + B u^n                         (leapfrog)
 * with hx_ij = h(x_i + dx/2, y_j) and hy_ij = h(x_i, y_j + dy/2) sampled at
 * cell faces.  Boundary nodes hold 0 and are never updated.  Arrays are
 * row-major, x fastest: a[j*ld + i], ld >= nx.
 *
 * Compiled with -ffp-contract=off so that no multiply-add is fused: every
 * expression is rounded in the order written.  OpenMP only splits rows between
 * threads; the arithmetic of every node, and the order of every sum, is the
 * same for any thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { int32_t nx, ny; int64_t ld; double dx, dy; } orc_grid;
typedef struct { int32_t kind, power; double amp, cx, cy; } orc_sing;
typedef struct {
  double background, eps;
  int32_t mollifier, nsing;
  const orc_sing* sing;
} orc_depth;

enum { ORC_LINE_X = 0, ORC_LINE_Y = 1, ORC_POINT = 2, ORC_STEP_X = 3, ORC_STEP_Y = 4 };
enum { ORC_GAUSS = 0, ORC_FRIEDRICHS = 1 };

#define IDX(g, i, j) ((int64_t)(j) * (g)->ld + (i))

/* ------------------------------------------------------------------------- */
/* threads                                                                   */
/* ------------------------------------------------------------------------- */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Mollifiers (Sec. 2.1: psi_eps(x) = eps^-d psi(x/eps), int psi = 1;        */
/* Sec. 3.1: the bump c exp(1/(x^2-1)) on |x| < 1, c ~ 2.2523).              */
/* ------------------------------------------------------------------------- */
static double bump(double x) { return (fabs(x) < 1.0) ? exp(1.0 / (x * x - 1.0)) : 0.0; }

/* c1 = 1 / int_{-1}^{1} bump(x) dx, by composite Simpson's rule. */
double orc_friedrichs_c1(void) {
  const int n = 400000; /* even */
  const double a = -1.0, h = 2.0 / n;
  double s = bump(a) + bump(1.0);
  for (int k = 1; k < n; ++k) s += ((k & 1) ? 4.0 : 2.0) * bump(a + k * h);
  return 1.0 / (s * h / 3.0);
}

/* c2 = 1 / int_{R^2} bump(|r|) dA = 1 / (2 pi int_0^1 r bump(r) dr), Simpson. */
double orc_friedrichs_c2(void) {
  const int n = 400000;
  const double h = 1.0 / n;
  double s = 0.0 * bump(0.0) + 1.0 * bump(1.0);
  for (int k = 1; k < n; ++k) {
    double r = k * h;
    s += ((k & 1) ? 4.0 : 2.0) * r * bump(r);
  }
  return 1.0 / (2.0 * M_PI * s * h / 3.0);
}

/* Cumulative mass of the 1D Friedrichs bump: c1 * int_{-1}^{t} bump, Simpson. */
static double friedrichs_cdf(double c1, double t) {
  if (t <= -1.0) return 0.0;
  if (t >= 1.0) return 1.0;
  const int n = 20000;
  const double h = (t + 1.0) / n;
  double s = bump(-1.0) + bump(t);
  for (int k = 1; k < n; ++k) s += ((k & 1) ? 4.0 : 2.0) * bump(-1.0 + k * h);
  return c1 * s * h / 3.0;
}

/* 1D unit-mass mollifier of width eps evaluated at s. */
static double phi1(int moll, double c1, double eps, double s) {
  if (moll == ORC_GAUSS) return exp(-(s / eps) * (s / eps)) / (eps * sqrt(M_PI));
  return c1 / eps * bump(s / eps);
}

/* 2D unit-mass radial mollifier of width eps at distance r (eps^-2 scaling). */
static double phi2(int moll, double c2, double eps, double r) {
  if (moll == ORC_GAUSS) return exp(-(r / eps) * (r / eps)) / (M_PI * eps * eps);
  return c2 / (eps * eps) * bump(r / eps);
}

/* Mollified Heaviside H(c - x) (depth amp on the side x < c): the mollifier's
 * mass on (-inf, (c - x)/eps]. */
static double step1(int moll, double c1, double eps, double s) {
  if (moll == ORC_GAUSS) return 0.5 * erfc(-s / eps);
  return friedrichs_cdf(c1, s / eps);
}

static double depth_at(const orc_depth* d, double c1, double c2, double x, double y) {
  double h = d->background;
  for (int k = 0; k < d->nsing; ++k) {
    const orc_sing* s = &d->sing[k];
    double v;
    switch (s->kind) {
      case ORC_LINE_X: v = phi1(d->mollifier, c1, d->eps, x - s->cx); break;
      case ORC_LINE_Y: v = phi1(d->mollifier, c1, d->eps, y - s->cy); break;
      case ORC_POINT: {
        double r = sqrt((x - s->cx) * (x - s->cx) + (y - s->cy) * (y - s->cy));
        v = phi2(d->mollifier, c2, d->eps, r);
        break;
      }
      case ORC_STEP_X: v = step1(d->mollifier, c1, d->eps, s->cx - x); break;
      case ORC_STEP_Y: v = step1(d->mollifier, c1, d->eps, s->cy - y); break;
      default: return NAN;
    }
    double p = v;
    for (int q = 1; q < s->power; ++q) p = p * v; /* phi_eps^power (power 2: the delta^2 case, Sec. 3.1) */
    h = h + s->amp * p;
  }
  return h;
}

/* Face coefficients: hx[j][i] = h(x_i + dx/2, y_j) for i <= nx-2,
 * hy[j][i] = h(x_i, y_j + dy/2) for j <= ny-2; every other entry is 0.
 * ext[4] = {min hx, max hx, min hy, max hy} over the defined faces.
 * Returns 0, or 1 on bad arguments. */
int orc_make_depth(const orc_grid* g, const orc_depth* d, double* hx, double* hy, double* ext) {
  if (g->nx < 3 || g->ny < 3 || g->ld < g->nx || !(d->eps > 0.0)) return 1;
  if (d->nsing > 0 && !d->sing) return 1;
  for (int k = 0; k < d->nsing; ++k) {
    if (d->sing[k].kind < 0 || d->sing[k].kind > 4 || d->sing[k].power < 1) return 1;
  }
  const double c1 = orc_friedrichs_c1(), c2 = orc_friedrichs_c2();
  const int64_t n = (int64_t)g->ny * g->ld;
  memset(hx, 0, sizeof(double) * n);
  memset(hy, 0, sizeof(double) * n);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < g->ny; ++j) {
    for (int i = 0; i < g->nx; ++i) {
      double x = i * g->dx, y = j * g->dy;
      if (i <= g->nx - 2) hx[IDX(g, i, j)] = depth_at(d, c1, c2, (i + 0.5) * g->dx, y);
      if (j <= g->ny - 2) hy[IDX(g, i, j)] = depth_at(d, c1, c2, x, (j + 0.5) * g->dy);
    }
  }
  double mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
  for (int j = 0; j < g->ny; ++j)
    for (int i = 0; i < g->nx; ++i) {
      if (i <= g->nx - 2) {
        double v = hx[IDX(g, i, j)];
        mnx = fmin(mnx, v);
        mxx = fmax(mxx, v);
      }
      if (j <= g->ny - 2) {
        double v = hy[IDX(g, i, j)];
        mny = fmin(mny, v);
        mxy = fmax(mxy, v);
      }
    }
  ext[0] = mnx;
  ext[1] = mxx;
  ext[2] = mny;
  ext[3] = mxy;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* FP32 emulation: the same start and leapfrog in float arithmetic, in the   */
/* order written (no fused multiply-add), in the standard form               */
/*   u^{n+1} = (2 u^n - u^{n-1}) + B u^n                                     */
/* or the increment form                                                     */
/*   v^1 = tau u1 + B u^0 / 2,  u^1 = u^0 + v^1,  v^{n+1} = v^n + B u^n,     */
/*   u^{n+1} = u^n + v^{n+1}                                                 */
/* (algebraically the same scheme).  It shows how FP32 rounding grows in     */
/* each form, independently of any GPU code.  Inputs are FP64 and rounded to */
/* float once; the final u^S is returned widened to double.                  */
/* ------------------------------------------------------------------------- */
static inline float fxf(const orc_grid* g, const float* hx, const float* u, int i, int j) {
  return hx[IDX(g, i, j)] * (u[IDX(g, i + 1, j)] - u[IDX(g, i, j)]) -
         hx[IDX(g, i - 1, j)] * (u[IDX(g, i, j)] - u[IDX(g, i - 1, j)]);
}
static inline float fyf(const orc_grid* g, const float* hy, const float* u, int i, int j) {
  return hy[IDX(g, i, j)] * (u[IDX(g, i, j + 1)] - u[IDX(g, i, j)]) -
         hy[IDX(g, i, j - 1)] * (u[IDX(g, i, j)] - u[IDX(g, i, j - 1)]);
}

int orc_forward_f32(const orc_grid* g, double tau, const double* hx, const double* hy, const double* u0,
                    const double* u1, int64_t S, int increment, double* u_out) {
  if (S < 1) return 1;
  const int64_t n = (int64_t)g->ny * g->ld;
  float* fhx = (float*)calloc(n, sizeof(float));
  float* fhy = (float*)calloc(n, sizeof(float));
  float* a = (float*)calloc(n, sizeof(float)); /* u^{n-1} (standard) or v^n (increment) */
  float* b = (float*)calloc(n, sizeof(float)); /* u^n */
  if (!fhx || !fhy || !a || !b) {
    free(fhx); free(fhy); free(a); free(b);
    return 2;
  }
  for (int64_t k = 0; k < n; ++k) {
    fhx[k] = (float)hx[k];
    fhy[k] = (float)hy[k];
  }
  const float cx = (float)(tau * tau / (g->dx * g->dx)), cy = (float)(tau * tau / (g->dy * g->dy));
  const float ftau = (float)tau;
  /* u^0 with zero boundary into a (standard: u^{n-1} slot) or b (increment: u slot) */
  float* u = increment ? b : a;
  for (int j = 1; j < g->ny - 1; ++j)
    for (int i = 1; i < g->nx - 1; ++i) u[IDX(g, i, j)] = (float)u0[IDX(g, i, j)];
  /* start */
  if (increment) {
    for (int j = 1; j < g->ny - 1; ++j)
      for (int i = 1; i < g->nx - 1; ++i) {
        const float bu = cx * fxf(g, fhx, b, i, j) + cy * fyf(g, fhy, b, i, j);
        const float v1 = u1 ? (float)u1[IDX(g, i, j)] : 0.0f;
        a[IDX(g, i, j)] = ftau * v1 + 0.5f * bu;
      }
    for (int j = 1; j < g->ny - 1; ++j)
      for (int i = 1; i < g->nx - 1; ++i) b[IDX(g, i, j)] = b[IDX(g, i, j)] + a[IDX(g, i, j)];
  } else {
    for (int j = 1; j < g->ny - 1; ++j)
      for (int i = 1; i < g->nx - 1; ++i) {
        const float bu = cx * fxf(g, fhx, a, i, j) + cy * fyf(g, fhy, a, i, j);
        const float v1 = u1 ? (float)u1[IDX(g, i, j)] : 0.0f;
        b[IDX(g, i, j)] = (a[IDX(g, i, j)] + ftau * v1) + 0.5f * bu;
      }
  }
  /* steps 2..S */
  float* bu = (float*)calloc(n, sizeof(float));
  if (!bu) {
    free(fhx); free(fhy); free(a); free(b);
    return 2;
  }
  for (int64_t step = 2; step <= S; ++step) {
#pragma omp parallel for schedule(static)
    for (int j = 1; j < g->ny - 1; ++j)
      for (int i = 1; i < g->nx - 1; ++i) bu[IDX(g, i, j)] = cx * fxf(g, fhx, b, i, j) + cy * fyf(g, fhy, b, i, j);
#pragma omp parallel for schedule(static)
    for (int j = 1; j < g->ny - 1; ++j)
      for (int i = 1; i < g->nx - 1; ++i) {
        const int64_t k = IDX(g, i, j);
        if (increment) {
          a[k] = a[k] + bu[k];
          b[k] = b[k] + a[k];
        } else {
          const float next = (2.0f * b[k] - a[k]) + bu[k];
          a[k] = b[k];
          b[k] = next;
        }
      }
  }
  for (int64_t k = 0; k < n; ++k) u_out[k] = (double)b[k];
  free(fhx); free(fhy); free(a); free(b); free(bu);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* d h_eps / d eps at the faces: how the regularised depth moves with the    */
/* regularisation width (Sec. 2.1, h_eps = h * psi_eps).  Differentiating    */
/* psi_eps(s) = eps^-d psi(s/eps) in eps (t = s/eps):                        */
/*   d/deps [eps^-d psi(t)] = -eps^-(d+1) [d psi(t) + t psi'(t)],            */
/* with psi the Gaussian exp(-t^2)/sqrt(pi)^d or c_d bump(t),                */
/*   Gaussian: t psi' = -2 t^2 psi;   bump: t psi' = -2 t^2/(t^2-1)^2 psi,   */
/* and for the mollified step S = int_{-inf}^{s/eps} psi: dS/deps = -t/eps   */
/* psi(t).  A power p > 1 brings the factor p phi^{p-1}.                     */
/* ------------------------------------------------------------------------- */
static double dphi_deps(int moll, double c, int d, double eps, double s) {
  const double t = s / eps;
  double psi, tdpsi;
  if (moll == ORC_GAUSS) {
    psi = exp(-t * t) / (d == 1 ? sqrt(M_PI) : M_PI);
    tdpsi = -2.0 * t * t * psi;
  } else {
    if (!(fabs(t) < 1.0)) return 0.0;
    psi = c * bump(t);
    const double w = t * t - 1.0;
    tdpsi = -2.0 * t * t / (w * w) * psi;
  }
  return -(d * psi + tdpsi) / pow(eps, d + 1);
}

static double dstep_deps(int moll, double c1, double eps, double s) {
  const double t = s / eps;
  double psi;
  if (moll == ORC_GAUSS)
    psi = exp(-t * t) / sqrt(M_PI);
  else
    psi = (fabs(t) < 1.0) ? c1 * bump(t) : 0.0;
  return -t / eps * psi;
}

static double depth_deps_at(const orc_depth* d, double c1, double c2, double x, double y) {
  double acc = 0.0;
  for (int k = 0; k < d->nsing; ++k) {
    const orc_sing* s = &d->sing[k];
    double v, dv;
    switch (s->kind) {
      case ORC_LINE_X:
        v = phi1(d->mollifier, c1, d->eps, x - s->cx);
        dv = dphi_deps(d->mollifier, c1, 1, d->eps, x - s->cx);
        break;
      case ORC_LINE_Y:
        v = phi1(d->mollifier, c1, d->eps, y - s->cy);
        dv = dphi_deps(d->mollifier, c1, 1, d->eps, y - s->cy);
        break;
      case ORC_POINT: {
        double r = sqrt((x - s->cx) * (x - s->cx) + (y - s->cy) * (y - s->cy));
        v = phi2(d->mollifier, c2, d->eps, r);
        dv = dphi_deps(d->mollifier, c2, 2, d->eps, r);
        break;
      }
      case ORC_STEP_X:
        v = step1(d->mollifier, c1, d->eps, s->cx - x);
        dv = dstep_deps(d->mollifier, c1, d->eps, s->cx - x);
        break;
      case ORC_STEP_Y:
        v = step1(d->mollifier, c1, d->eps, s->cy - y);
        dv = dstep_deps(d->mollifier, c1, d->eps, s->cy - y);
        break;
      default: return NAN;
    }
    double pw = 1.0; /* v^(power-1) */
    for (int q = 1; q < s->power; ++q) pw = pw * v;
    acc = acc + s->amp * (s->power * pw) * dv;
  }
  return acc;
}

/* dhx[j][i] = d h_eps / d eps at the x-face (x_i + dx/2, y_j), i <= nx-2, and dhy likewise;
 * every other entry 0.  Returns 0, or 1 on bad arguments. */
int orc_depth_deps(const orc_grid* g, const orc_depth* d, double* dhx, double* dhy) {
  if (g->nx < 3 || g->ny < 3 || g->ld < g->nx || !(d->eps > 0.0)) return 1;
  if (d->nsing > 0 && !d->sing) return 1;
  for (int k = 0; k < d->nsing; ++k) {
    if (d->sing[k].kind < 0 || d->sing[k].kind > 4 || d->sing[k].power < 1) return 1;
  }
  const double c1 = orc_friedrichs_c1(), c2 = orc_friedrichs_c2();
  const int64_t n = (int64_t)g->ny * g->ld;
  memset(dhx, 0, sizeof(double) * n);
  memset(dhy, 0, sizeof(double) * n);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < g->ny; ++j) {
    for (int i = 0; i < g->nx; ++i) {
      double x = i * g->dx, y = j * g->dy;
      if (i <= g->nx - 2) dhx[IDX(g, i, j)] = depth_deps_at(d, c1, c2, (i + 0.5) * g->dx, y);
      if (j <= g->ny - 2) dhy[IDX(g, i, j)] = depth_deps_at(d, c1, c2, x, (j + 0.5) * g->dy);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* The discrete operator B = tau^2 L_h (interior nodes; 0 on the boundary).  */
/* ------------------------------------------------------------------------- */
static inline double fx_at(const orc_grid* g, const double* hx, const double* u, int i, int j) {
  return hx[IDX(g, i, j)] * (u[IDX(g, i + 1, j)] - u[IDX(g, i, j)]) -
         hx[IDX(g, i - 1, j)] * (u[IDX(g, i, j)] - u[IDX(g, i - 1, j)]);
}
static inline double fy_at(const orc_grid* g, const double* hy, const double* u, int i, int j) {
  return hy[IDX(g, i, j)] * (u[IDX(g, i, j + 1)] - u[IDX(g, i, j)]) -
         hy[IDX(g, i, j - 1)] * (u[IDX(g, i, j)] - u[IDX(g, i, j - 1)]);
}

/* out = B u = cx fx(u) + cy fy(u) on interior nodes, 0 on boundary nodes. */
void orc_apply_B(const orc_grid* g, double cx, double cy, const double* hx, const double* hy,
                 const double* u, double* out) {
  memset(out, 0, sizeof(double) * (int64_t)g->ny * g->ld);
#pragma omp parallel for schedule(static)
  for (int j = 1; j < g->ny - 1; ++j)
    for (int i = 1; i < g->nx - 1; ++i)
      out[IDX(g, i, j)] = cx * fx_at(g, hx, u, i, j) + cy * fy_at(g, hy, u, i, j);
}

static void zero_boundary(const orc_grid* g, double* u) {
  for (int i = 0; i < g->nx; ++i) {
    u[IDX(g, i, 0)] = 0.0;
    u[IDX(g, i, g->ny - 1)] = 0.0;
  }
  for (int j = 0; j < g->ny; ++j) {
    u[IDX(g, 0, j)] = 0.0;
    u[IDX(g, g->nx - 1, j)] = 0.0;
  }
}

/* Taylor start: u_prev <- u^0 (boundary zeroed), u_cur <- u^1 =
 * (u^0 + tau u1) + B u^0 / 2.  u1 may be NULL (zero initial velocity). */
void orc_init(const orc_grid* g, double tau, const double* hx, const double* hy, const double* u0,
              const double* u1, double* u_prev, double* u_cur) {
  const double cx = tau * tau / (g->dx * g->dx), cy = tau * tau / (g->dy * g->dy);
  const int64_t n = (int64_t)g->ny * g->ld;
  memcpy(u_prev, u0, sizeof(double) * n);
  zero_boundary(g, u_prev);
  memset(u_cur, 0, sizeof(double) * n);
#pragma omp parallel for schedule(static)
  for (int j = 1; j < g->ny - 1; ++j)
    for (int i = 1; i < g->nx - 1; ++i) {
      double b = cx * fx_at(g, hx, u_prev, i, j) + cy * fy_at(g, hy, u_prev, i, j);
      double v = u1 ? u1[IDX(g, i, j)] : 0.0;
      u_cur[IDX(g, i, j)] = (u_prev[IDX(g, i, j)] + tau * v) + 0.5 * b;
    }
}

/* One leapfrog step: u_prev holds u^{n-1} on entry and u^{n+1} on return. */
void orc_step(const orc_grid* g, double tau, const double* hx, const double* hy, double* u_prev,
              const double* u_cur) {
  const double cx = tau * tau / (g->dx * g->dx), cy = tau * tau / (g->dy * g->dy);
#pragma omp parallel for schedule(static)
  for (int j = 1; j < g->ny - 1; ++j)
    for (int i = 1; i < g->nx - 1; ++i) {
      int64_t k = IDX(g, i, j);
      double b = cx * fx_at(g, hx, u_cur, i, j) + cy * fy_at(g, hy, u_cur, i, j);
      u_prev[k] = (2.0 * u_cur[k] - u_prev[k]) + b;
    }
}

/* ------------------------------------------------------------------------- */
/* Discrete energy of the pair (u^n, u^{n+1}) -- the leapfrog analogue of    */
/* (CL-01), Theorem 2.1:                                                      */
/*   E^{n+1/2} = 1/2 sum_nodes ((u^{n+1}-u^n)/tau)^2 dxdy                      */
/*             + 1/2 sum_x-faces hx (D_x u^{n+1})(D_x u^n) dxdy                */
/*             + 1/2 sum_y-faces hy (D_y u^{n+1})(D_y u^n) dxdy                */
/* with D_x u = (u_{i+1}-u_i)/dx.  Every sum is compensated (Neumaier).       */
/* ------------------------------------------------------------------------- */
typedef struct { double s, c; } nsum;
static inline void nadd(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}
static inline double nval(const nsum* a) { return a->s + a->c; }

double orc_energy(const orc_grid* g, double tau, const double* hx, const double* hy,
                  const double* u_n, const double* u_n1) {
  double* rows = (double*)malloc(sizeof(double) * 3 * g->ny);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < g->ny; ++j) {
    nsum kin = {0, 0}, px = {0, 0}, py = {0, 0};
    for (int i = 0; i < g->nx; ++i) {
      int64_t k = IDX(g, i, j);
      double v = u_n1[k] - u_n[k];
      nadd(&kin, v * v);
      if (i <= g->nx - 2)
        nadd(&px, hx[k] * (u_n1[k + 1] - u_n1[k]) * (u_n[k + 1] - u_n[k]));
      if (j <= g->ny - 2)
        nadd(&py, hy[k] * (u_n1[k + g->ld] - u_n1[k]) * (u_n[k + g->ld] - u_n[k]));
    }
    rows[3 * j + 0] = nval(&kin);
    rows[3 * j + 1] = nval(&px);
    rows[3 * j + 2] = nval(&py);
  }
  nsum kin = {0, 0}, px = {0, 0}, py = {0, 0};
  for (int j = 0; j < g->ny; ++j) {
    nadd(&kin, rows[3 * j + 0]);
    nadd(&px, rows[3 * j + 1]);
    nadd(&py, rows[3 * j + 2]);
  }
  free(rows);
  const double dxdy = g->dx * g->dy;
  return 0.5 * dxdy * (nval(&kin) / (tau * tau) + nval(&px) / (g->dx * g->dx) + nval(&py) / (g->dy * g->dy));
}

/* ------------------------------------------------------------------------- */
/* Whole forward run: Taylor start then S-1 leapfrog steps, final u^S.        */
/*   energy[n] = E^{n+1/2}, n = 0..S-1          (may be NULL)                  */
/*   traces[(n-1)*nrec + r] = u^n[rec_idx[r]], n = 1..S   (may be NULL)        */
/* On return u_prev = u^{S-1}, u_cur = u^S.  Requires S >= 1.                  */
/* ------------------------------------------------------------------------- */
int orc_forward(const orc_grid* g, double tau, const double* hx, const double* hy, const double* u0,
                const double* u1, int64_t S, double* energy, int32_t nrec, const int64_t* rec_idx,
                double* traces, double* u_prev, double* u_cur) {
  if (S < 1) return 1;
  orc_init(g, tau, hx, hy, u0, u1, u_prev, u_cur);
  for (int64_t n = 1;; ++n) { /* state holds (u^{n-1}, u^n) */
    if (energy) energy[n - 1] = orc_energy(g, tau, hx, hy, u_prev, u_cur);
    if (traces)
      for (int r = 0; r < nrec; ++r) traces[(n - 1) * nrec + r] = u_cur[rec_idx[r]];
    if (n == S) break;
    orc_step(g, tau, hx, hy, u_prev, u_cur);
    double* t = u_prev;
    u_prev = u_cur;
    u_cur = t;
  }
  /* the pointers were swapped S-1 times: put u^{S-1}, u^S in the caller's order */
  if ((S - 1) & 1) {
    const int64_t m = (int64_t)g->ny * g->ld;
    double* tmp = (double*)malloc(sizeof(double) * m);
    memcpy(tmp, u_prev, sizeof(double) * m);
    memcpy(u_prev, u_cur, sizeof(double) * m);
    memcpy(u_cur, tmp, sizeof(double) * m);
    free(tmp);
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Discrete adjoint of orc_forward for a receiver functional J(traces).      */
/* (Not in the paper; the exact reverse of the scheme above.)                */
/*   g^n  = S^T dJ/dtrace^n  (scatter-add of dtr[(n-1)*nrec + r] to rec_idx)  */
/*   lam^n = g^n + (2I + B) lam^{n+1} - lam^{n+2},  n = S..1,                 */
/*           lam^{S+1} = lam^{S+2} = 0                                        */
/*   dJ/du0 = (I + B/2) lam^1 - lam^2,   dJ/du1 = tau lam^1                   */
/*   dJ/dhx_ij = -cx [ sum_{n=1}^{S-1} (lam^{n+1}_{i+1,j}-lam^{n+1}_ij)       */
/*                                     (u^n_{i+1,j}-u^n_ij)                   */
/*                 + 1/2 (lam^1_{i+1,j}-lam^1_ij)(u^0_{i+1,j}-u^0_ij) ]        */
/*   dJ/dhy likewise with cy and j+1.  lam = 0 on boundary nodes.             */
/* The whole forward history is stored (tiny problems only).                  */
/* ------------------------------------------------------------------------- */
static void add_face_grads(const orc_grid* g, double wx, double wy, const double* lam, const double* u,
                           double* ghx, double* ghy) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < g->ny; ++j)
    for (int i = 0; i < g->nx; ++i) {
      int64_t k = IDX(g, i, j);
      if (i <= g->nx - 2 && j >= 1 && j <= g->ny - 2)
        ghx[k] += wx * ((lam[k + 1] - lam[k]) * (u[k + 1] - u[k]));
      if (j <= g->ny - 2 && i >= 1 && i <= g->nx - 2)
        ghy[k] += wy * ((lam[k + g->ld] - lam[k]) * (u[k + g->ld] - u[k]));
    }
}

int orc_adjoint(const orc_grid* g, double tau, const double* hx, const double* hy, const double* u0,
                const double* u1, int64_t S, int32_t nrec, const int64_t* rec_idx, const double* dtr,
                double* g_hx, double* g_hy, double* g_u0, double* g_u1) {
  if (S < 1) return 1;
  const int64_t m = (int64_t)g->ny * g->ld;
  const double cx = tau * tau / (g->dx * g->dx), cy = tau * tau / (g->dy * g->dy);
  double* U = (double*)malloc(sizeof(double) * m * (S + 1)); /* U[n] = u^n */
  double* lam1 = (double*)calloc(m, sizeof(double));         /* lam^{n+1} */
  double* lam2 = (double*)calloc(m, sizeof(double));         /* lam^{n+2} */
  double* lam = (double*)calloc(m, sizeof(double));          /* lam^n */
  double* Bl = (double*)malloc(sizeof(double) * m);
  if (!U || !lam1 || !lam2 || !lam || !Bl) {
    free(U); free(lam1); free(lam2); free(lam); free(Bl);
    return 2;
  }
  /* forward history */
  orc_init(g, tau, hx, hy, u0, u1, U + 0 * m, U + 1 * m);
  for (int64_t n = 1; n < S; ++n) {
    memcpy(U + (n + 1) * m, U + (n - 1) * m, sizeof(double) * m);
    orc_step(g, tau, hx, hy, U + (n + 1) * m, U + n * m);
  }
  memset(g_hx, 0, sizeof(double) * m);
  memset(g_hy, 0, sizeof(double) * m);
  for (int64_t n = S; n >= 1; --n) {
    /* lam^n = g^n + (2I + B) lam^{n+1} - lam^{n+2} */
    orc_apply_B(g, cx, cy, hx, hy, lam1, Bl);
    for (int64_t k = 0; k < m; ++k) lam[k] = (2.0 * lam1[k] - lam2[k]) + Bl[k];
    for (int r = 0; r < nrec; ++r) lam[rec_idx[r]] += dtr[(n - 1) * nrec + r];
    zero_boundary(g, lam);
    /* face terms of equation n+1 (u^{n+1} = 2u^n - u^{n-1} + B u^n), multiplier lam^{n+1} */
    if (n <= S - 1) add_face_grads(g, -cx, -cy, lam1, U + n * m, g_hx, g_hy);
    double* t = lam2;
    lam2 = lam1;
    lam1 = lam;
    lam = t;
  }
  /* now lam1 = lam^1, lam2 = lam^2 */
  orc_apply_B(g, cx, cy, hx, hy, lam1, Bl);
  for (int64_t k = 0; k < m; ++k) {
    g_u0[k] = (lam1[k] - lam2[k]) + 0.5 * Bl[k];
    g_u1[k] = tau * lam1[k];
  }
  zero_boundary(g, g_u0);
  zero_boundary(g, g_u1);
  add_face_grads(g, -0.5 * cx, -0.5 * cy, lam1, U + 0 * m, g_hx, g_hy);
  free(U); free(lam1); free(lam2); free(lam); free(Bl);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Implicit comparator.  Sec. 3.3 solves the 2D problem with an implicit       */
/* finite-difference scheme whose systems are tridiagonal along grid lines     */
/* (cyclic reduction), without writing the scheme out.  The reading taken     */
/* here is the factorized scheme with weight sigma (sigma = 1/4: stable for    */
/* every tau):                                                                 */
/*   (I - sigma B_x)(I - sigma B_y) w^n = B u^n,   B_x u = cx fx(u),           */
/*                                                 B_y u = cy fy(u)            */
/* in increment form                                                           */
/*   v^{n+1} = v^n + w^n,   u^{n+1} = u^n + v^{n+1},                            */
/* started by w^0 from the same systems with B u^0 and                          */
/*   v^1 = tau u1 + w^0 / 2,   u^1 = u^0 + v^1.                                 */
/* Each factor is one independent tridiagonal system per grid line over the    */
/* interior nodes (zero Dirichlet ends), solved by plain Thomas elimination.   */
/* ------------------------------------------------------------------------- */

/* Thomas elimination of a tridiagonal system of n >= 1 rows: sub-diagonal a   */
/* (a[0] unused), diagonal b, super-diagonal c (c[n-1] unused); d holds the     */
/* right-hand side on entry and the solution on return; cp is scratch.        */
static void thomas(int n, const double* a, const double* b, const double* c, double* d, double* cp) {
  cp[0] = c[0] / b[0];
  d[0] = d[0] / b[0];
  for (int k = 1; k < n; ++k) {
    const double p = b[k] - a[k] * cp[k - 1];
    cp[k] = c[k] / p;
    d[k] = (d[k] - a[k] * d[k - 1]) / p;
  }
  for (int k = n - 2; k >= 0; --k) d[k] = d[k] - cp[k] * d[k + 1];
}

static int team_size(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
static int team_rank(void) {
#ifdef _OPENMP
  return omp_get_thread_num();
#else
  return 0;
#endif
}

/* r <- (I - s B_x)^{-1} r on every interior row (s = sigma): the system of row */
/* j couples the interior nodes i = 1..nx-2 through the x faces of that row.    */
static int solve_x(const orc_grid* g, double s, double cx, const double* hx, double* r) {
  const int n = g->nx - 2, nt = team_size();
  double* all = (double*)malloc(sizeof(double) * 5 * (size_t)n * (size_t)nt);
  if (!all) return 1;
#pragma omp parallel num_threads(nt)
  {
    double* a = all + (size_t)5 * n * team_rank();
    double *b = a + n, *c = a + 2 * n, *d = a + 3 * n, *cp = a + 4 * n;
#pragma omp for schedule(static)
    for (int j = 1; j < g->ny - 1; ++j) {
      for (int k = 0; k < n; ++k) {
        const int i = k + 1;
        const double hl = hx[IDX(g, i - 1, j)], hr = hx[IDX(g, i, j)];
        a[k] = -(s * cx * hl);
        b[k] = 1.0 + s * cx * (hl + hr);
        c[k] = -(s * cx * hr);
        d[k] = r[IDX(g, i, j)];
      }
      thomas(n, a, b, c, d, cp);
      for (int k = 0; k < n; ++k) r[IDX(g, k + 1, j)] = d[k];
    }
  }
  free(all);
  return 0;
}

/* r <- (I - s B_y)^{-1} r on every interior column. */
static int solve_y(const orc_grid* g, double s, double cy, const double* hy, double* r) {
  const int n = g->ny - 2, nt = team_size();
  double* all = (double*)malloc(sizeof(double) * 5 * (size_t)n * (size_t)nt);
  if (!all) return 1;
#pragma omp parallel num_threads(nt)
  {
    double* a = all + (size_t)5 * n * team_rank();
    double *b = a + n, *c = a + 2 * n, *d = a + 3 * n, *cp = a + 4 * n;
#pragma omp for schedule(static)
    for (int i = 1; i < g->nx - 1; ++i) {
      for (int k = 0; k < n; ++k) {
        const int j = k + 1;
        const double hd = hy[IDX(g, i, j - 1)], hu = hy[IDX(g, i, j)];
        a[k] = -(s * cy * hd);
        b[k] = 1.0 + s * cy * (hd + hu);
        c[k] = -(s * cy * hu);
        d[k] = r[IDX(g, i, j)];
      }
      thomas(n, a, b, c, d, cp);
      for (int k = 0; k < n; ++k) r[IDX(g, i, k + 1)] = d[k];
    }
  }
  free(all);
  return 0;
}

/* w <- A^{-1} B u with A = (I - s B_x)(I - s B_y): first z = (I - s B_x)^{-1}  */
/* B u, then w = (I - s B_y)^{-1} z.                                            */
static int implicit_w(const orc_grid* g, double s, double cx, double cy, const double* hx, const double* hy,
                      const double* u, double* w) {
  orc_apply_B(g, cx, cy, hx, hy, u, w);
  if (solve_x(g, s, cx, hx, w)) return 2;
  if (solve_y(g, s, cy, hy, w)) return 2;
  return 0;
}

/* The start and S - 1 steps of the factorized scheme; u_out = u^S, and, when  */
/* v_out is not NULL, v_out = v^S = u^S - u^{S-1}.                              */
int orc_implicit_forward(const orc_grid* g, double tau, double sigma, const double* hx, const double* hy,
                         const double* u0, const double* u1, int64_t S, double* u_out, double* v_out) {
  if (S < 1 || g->nx < 3 || g->ny < 3 || !(sigma >= 0.0)) return 1;
  const int64_t n = (int64_t)g->ny * g->ld;
  const double cx = tau * tau / (g->dx * g->dx), cy = tau * tau / (g->dy * g->dy);
  double* u = (double*)calloc(n, sizeof(double));
  double* v = (double*)calloc(n, sizeof(double));
  double* w = (double*)calloc(n, sizeof(double));
  int rc = 0;
  if (!u || !v || !w) {
    rc = 2;
    goto out;
  }
  memcpy(u, u0, sizeof(double) * n);
  zero_boundary(g, u);
  if ((rc = implicit_w(g, sigma, cx, cy, hx, hy, u, w))) goto out;
  for (int j = 1; j < g->ny - 1; ++j)
    for (int i = 1; i < g->nx - 1; ++i) {
      const int64_t k = IDX(g, i, j);
      v[k] = tau * (u1 ? u1[k] : 0.0) + 0.5 * w[k];
      u[k] = u[k] + v[k];
    }
  for (int64_t step = 2; step <= S; ++step) {
    if ((rc = implicit_w(g, sigma, cx, cy, hx, hy, u, w))) goto out;
#pragma omp parallel for schedule(static)
    for (int j = 1; j < g->ny - 1; ++j)
      for (int i = 1; i < g->nx - 1; ++i) {
        const int64_t k = IDX(g, i, j);
        v[k] = v[k] + w[k];
        u[k] = u[k] + v[k];
      }
  }
  memcpy(u_out, u, sizeof(double) * n);
  if (v_out) memcpy(v_out, v, sizeof(double) * n);
out:
  free(u);
  free(v);
  free(w);
  return rc;
}
