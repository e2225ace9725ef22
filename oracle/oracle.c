/*
 * Plain FP64 CPU oracle — TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Paper: "PDHCG-CQP", arXiv 2608.09159.  Section numbers, equations and
 * tables cited below are the paper's.  Where the paper is silent the reading
 * taken is stated at the point of use.
 *
 * The same source builds twice: single-threaded (liboracle.so) and with OpenMP
 * (liboracle_omp.so, -fopenmp), the latter only to time the CPU baseline on all
 * host cores.  Parallel loops touch independent rows, coordinates or blocks, and
 * every long sum is taken in fixed chunks of ORC_CHUNK terms whose totals are then
 * added in index order, so both builds perform the same additions in the same order
 * and return identical iterates with any thread count.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EULER_E 2.718281828459045235360287
#define ORC_CHUNK 4096

static double* dalloc(int64_t n) { return (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

/* fixed-order sums (see the header comment): kind 0: sum a_i b_i, 1: sum (a_i - b_i)^2,
 * 2: sum a_i w_i b_i, 3: sum a_i (b_i - w_i) */
static double csum(int kind, int64_t n, const double* a, const double* b, const double* w) {
  const int64_t nc = (n + ORC_CHUNK - 1) / ORC_CHUNK;
  double part1[1];
  double* part = nc <= 1 ? part1 : (double*)malloc((size_t)nc * sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (nc > 1)
#endif
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t i1 = (c + 1) * ORC_CHUNK < n ? (c + 1) * ORC_CHUNK : n;
    double t = 0.0;
    for (int64_t i = c * ORC_CHUNK; i < i1; ++i) {
      if (kind == 0) t += a[i] * b[i];
      else if (kind == 1) { const double d = a[i] - b[i]; t += d * d; }
      else if (kind == 2) t += a[i] * w[i] * b[i];
      else t += a[i] * (b[i] - w[i]);
    }
    part[c] = t;
  }
  double s = 0.0;
  for (int64_t c = 0; c < nc; ++c) s += part[c];
  if (part != part1) free(part);
  return s;
}
static double dot(int64_t n, const double* a, const double* b) { return csum(0, n, a, b, NULL); }
static double dist2(int64_t n, const double* a, const double* b) { return csum(1, n, a, b, NULL); }

void orc_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
static double nrm2(int64_t n, const double* a) { return sqrt(dot(n, a, a)); }
static double sq(double a) { return a * a; }

/* ------------------------------------------------------------------------- */
/* Sparse and structured products (Sec. 1: A, A*, Q applications)            */
/* ------------------------------------------------------------------------- */

void orc_spmv(int64_t m, const int64_t* rowptr, const int64_t* colind, const double* val,
              const double* x, double* y) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 512)
#endif
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[colind[k]];
    y[i] = s;
  }
}

void orc_spmv_t(int64_t m, int64_t n, const int64_t* rowptr, const int64_t* colind, const double* val,
                const double* y, double* out) {
  for (int64_t j = 0; j < n; ++j) out[j] = 0.0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) out[colind[k]] += val[k] * y[i];
}

/* Q x with Q = diag(q) + P + R' D R, never forming Q (Sec. 4.1, "Products with a
 * structured operator"). */
static void q_apply_parts(int64_t n, const double* qd, const int64_t* pr, const int64_t* pc, const double* pv,
                          int64_t k, const double* R, const double* D, const double* x, double* out) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < n; ++i) out[i] = qd ? qd[i] * x[i] : 0.0;
  if (pr) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 512)
#endif
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t t = pr[i]; t < pr[i + 1]; ++t) s += pv[t] * x[pc[t]];
      out[i] += s;
    }
  }
  if (k > 0) {
    double* t1 = dalloc(k);
    double* t2 = dalloc(k);
    for (int64_t l = 0; l < k; ++l) t1[l] = dot(n, R + l * n, x);
    for (int64_t l = 0; l < k; ++l) {
      double s = 0.0;
      for (int64_t j = 0; j < k; ++j) s += D[l * k + j] * t1[j];
      t2[l] = s;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i)
      for (int64_t l = 0; l < k; ++l) out[i] += R[l * n + i] * t2[l];
    free(t1);
    free(t2);
  }
}

void orc_q_apply(const orc_problem* p, const double* x, double* out) {
  q_apply_parts(p->n, p->q_diag, p->p_rowptr, p->p_colind, p->p_val, p->q_rank, p->q_R, p->q_D, x, out);
}

/* ------------------------------------------------------------------------- */
/* Cone membership (used for the trivial cases of every projection, App. A)   */
/* ------------------------------------------------------------------------- */

static double pow_geo(double x, double y, double a) {
  /* x^a y^(1-a) for x, y >= 0 */
  if (x <= 0.0 || y <= 0.0) return 0.0;
  return exp(a * log(x) + (1.0 - a) * log(y));
}

int orc_in_cone(int type, int64_t d, double alpha, const double* r, double tol) {
  switch (type) {
    case ORC_FREE: return 1;
    case ORC_NONNEG:
      for (int64_t i = 0; i < d; ++i) if (r[i] < -tol) return 0;
      return 1;
    case ORC_SOC: return nrm2(d - 1, r) <= r[d - 1] + tol;
    case ORC_RSOC: {
      double s = r[d - 2], t = r[d - 1];
      return s >= -tol && t >= -tol && dot(d - 2, r, r) <= 2.0 * s * t + tol;
    }
    case ORC_EXP: {
      double r0 = r[0], s0 = r[1], t0 = r[2];
      if (s0 > 0.0 && s0 * exp(r0 / s0) <= t0 + tol) return 1;
      return r0 <= tol && fabs(s0) <= tol && t0 >= -tol;
    }
    case ORC_POW:
      return r[0] >= -tol && r[1] >= -tol && pow_geo(r[0], r[1], alpha) + tol >= fabs(r[2]);
    case ORC_EXP1:
      return fabs(r[1] - 1.0) <= tol && exp(r[0]) <= r[2] + tol;
    case ORC_POW1:
      return fabs(r[1] - 1.0) <= tol && r[0] >= -tol && pow(fmax(r[0], 0.0), alpha) + tol >= fabs(r[2]);
  }
  return 0;
}

/* Dual cones: nonneg, SOC, RSOC are self-dual; free -> {0}.  Exponential dual
 * in the (r,s,t) ordering: cl{(u,v,w): u < 0, -u exp(v/u) <= e w}.  Power dual
 * as printed in App. A (three-dimensional power cone). */
int orc_in_dual_cone(int type, int64_t d, double alpha, const double* r, double tol) {
  switch (type) {
    case ORC_FREE:
      for (int64_t i = 0; i < d; ++i) if (fabs(r[i]) > tol) return 0;
      return 1;
    case ORC_NONNEG: case ORC_SOC: case ORC_RSOC:
      return orc_in_cone(type, d, alpha, r, tol);
    case ORC_EXP: {
      double u = r[0], v = r[1], w = r[2];
      if (u < 0.0 && -u * exp(v / u) <= EULER_E * w + tol) return 1;
      return fabs(u) <= tol && v >= -tol && w >= -tol;
    }
    case ORC_POW: {
      double p = r[0], q = r[1], w = r[2];
      if (p < -tol || q < -tol) return 0;
      return pow_geo(fmax(p, 0.0) / alpha, fmax(q, 0.0) / (1.0 - alpha), alpha) + tol >= fabs(w);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Projections (App. A, Table "cone-projection-methods")                      */
/* ------------------------------------------------------------------------- */

/* Bisection on a bracket [lo, hi] with f(lo) and f(hi) of opposite sign given
 * as sign_lo; runs until the midpoint no longer moves. */
typedef double (*scalar_fn)(double, const void*);
static double bisect(scalar_fn f, const void* ctx, double lo, double hi, int lo_positive) {
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double v = f(mid, ctx);
    if (v == 0.0) return mid;
    if ((v > 0.0) == (lo_positive != 0)) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* --- second-order cone K = {(v,t): ||v|| <= t}, t last (Sec. 4 standard form) --- */

static void proj_soc(int64_t d, const double* r, double* out) {
  /* Euclidean closed form (App. A.2, eq. soc-euclidean-projection) */
  int64_t nv = d - 1;
  double t = r[nv], a = nrm2(nv, r);
  if (a <= t) { memcpy(out, r, (size_t)d * sizeof(double)); return; }
  if (a <= -t) { memset(out, 0, (size_t)d * sizeof(double)); return; }
  double coef = (a + t) / (2.0 * a);
  for (int64_t i = 0; i < nv; ++i) out[i] = coef * r[i];
  out[nv] = 0.5 * (a + t);
}

typedef struct { int64_t nv; const double* r; const double* m; } soc_ctx;
static double soc_f(double lam, const void* vctx) {
  /* ||v(lam)||^2 - t(lam)^2 with v_i = m_i r_i/(m_i+lam), t = m_t r_t/(m_t-lam)
   * (App. A.2, eq. soc-metric-projection) */
  const soc_ctx* c = (const soc_ctx*)vctx;
  double s = 0.0;
  for (int64_t i = 0; i < c->nv; ++i) s += sq(c->m[i] * c->r[i] / (c->m[i] + lam));
  double mt = c->m[c->nv], rt = c->r[c->nv];
  return s - sq(mt * rt / (mt - lam));
}

static void proj_soc_m(int64_t d, const double* r, const double* m, double* out) {
  int64_t nv = d - 1;
  double t = r[nv], mt = m[nv];
  if (nrm2(nv, r) <= t) { memcpy(out, r, (size_t)d * sizeof(double)); return; }
  double A = 0.0, mmax = 0.0;
  for (int64_t i = 0; i < nv; ++i) { A += sq(m[i] * r[i]); if (m[i] > mmax) mmax = m[i]; }
  A = sqrt(A);
  double B = mt * fabs(t);
  if (t <= 0.0 && A <= B) { memset(out, 0, (size_t)d * sizeof(double)); return; } /* -Mr in K* = K */
  double lam;
  if (t == 0.0) {
    lam = mt;  /* singular case: v_i = m_i r_i/(m_i+m_t), t = ||v|| */
  } else {
    soc_ctx c = {nv, r, m};
    if (t > 0.0) {
      /* root in (0, m_t): f(0) = ||r_v||^2 - r_t^2 > 0, f -> -inf at m_t */
      lam = bisect(soc_f, &c, 0.0, mt, 1);
    } else {
      /* root in (m_t, lam_U]: f -> -inf at m_t; f(lam_U) >= 0 for
       * lam_U = (A m_t + B m_max)/(A - B), from ||v||^2 >= A^2/(m_max+lam)^2
       * and t^2 = B^2/(lam-m_t)^2.  (Bracket derived here; the paper defers it.) */
      double hi = (A * mt + B * mmax) / (A - B);
      hi = hi * (1.0 + 1e-12) + 1e-300;
      while (soc_f(hi, &c) < 0.0) hi *= 2.0;
      lam = bisect(soc_f, &c, mt, hi, 0);
    }
  }
  double nv2 = 0.0;
  for (int64_t i = 0; i < nv; ++i) { out[i] = m[i] * r[i] / (m[i] + lam); nv2 += sq(out[i]); }
  out[nv] = sqrt(nv2);
}

/* --- rotated SOC K = {(v,s,t): ||v||^2 <= 2 s t, s,t >= 0} --- */

static void proj_rsoc(int64_t d, const double* r, double* out) {
  /* Euclidean: U^{-1} Pi_soc(U r), U(v,s,t) = ((v,(s-t)/sqrt2),(s+t)/sqrt2) (App. A.3) */
  const double h = 1.0 / sqrt(2.0);
  double* w = dalloc(d);
  double* p = dalloc(d);
  int64_t nv = d - 2;
  for (int64_t i = 0; i < nv; ++i) w[i] = r[i];
  w[nv] = (r[nv] - r[nv + 1]) * h;
  w[nv + 1] = (r[nv] + r[nv + 1]) * h;
  proj_soc(d, w, p);
  for (int64_t i = 0; i < nv; ++i) out[i] = p[i];
  out[nv] = (p[nv] + p[nv + 1]) * h;
  out[nv + 1] = (p[nv + 1] - p[nv]) * h;
  free(w);
  free(p);
}

typedef struct { int64_t nv; const double* r; const double* m; } rsoc_ctx;
static void rsoc_st(const rsoc_ctx* c, double xi, double* s, double* t) {
  /* the 2x2 system of App. A.3, eq. rsoc-metric-projection */
  double ms = c->m[c->nv], mt = c->m[c->nv + 1], rs = c->r[c->nv], rt = c->r[c->nv + 1];
  double det = ms * mt - 4.0 * xi * xi;
  *s = mt * (ms * rs + 2.0 * xi * rt) / det;
  *t = ms * (mt * rt + 2.0 * xi * rs) / det;
}
static double rsoc_f(double xi, const void* vctx) {
  const rsoc_ctx* c = (const rsoc_ctx*)vctx;
  double v2 = 0.0, s, t;
  for (int64_t i = 0; i < c->nv; ++i) v2 += sq(c->m[i] * c->r[i] / (c->m[i] + 2.0 * xi));
  rsoc_st(c, xi, &s, &t);
  return v2 - 2.0 * s * t;
}

static void proj_rsoc_m(int64_t d, const double* r, const double* m, double* out) {
  int64_t nv = d - 2;
  double rs = r[nv], rt = r[nv + 1], ms = m[nv], mt = m[nv + 1];
  double v2 = dot(nv, r, r), mv2 = 0.0;
  for (int64_t i = 0; i < nv; ++i) mv2 += sq(m[i] * r[i]);
  if (rs >= 0.0 && rt >= 0.0 && v2 <= 2.0 * rs * rt) { memcpy(out, r, (size_t)d * sizeof(double)); return; }
  if (rs <= 0.0 && rt <= 0.0 && mv2 <= 2.0 * (ms * rs) * (mt * rt)) {  /* -Mr in K* = K */
    memset(out, 0, (size_t)d * sizeof(double));
    return;
  }
  if (v2 == 0.0) {
    /* with v = 0 the cone reduces to the quadrant s, t >= 0 */
    for (int64_t i = 0; i < nv; ++i) out[i] = 0.0;
    out[nv] = fmax(rs, 0.0);
    out[nv + 1] = fmax(rt, 0.0);
    return;
  }
  double q = sqrt(ms * mt);
  double kappa = sqrt(ms) * rs + sqrt(mt) * rt;
  double kscale = sqrt(ms) * fabs(rs) + sqrt(mt) * fabs(rt);
  if (fabs(kappa) <= 1e-14 * kscale) {
    /* singular, consistent case 2 xi = q (eq. rsoc-metric-singular-projection) */
    double delta = sqrt(ms) * rs, vv = 0.0;
    for (int64_t i = 0; i < nv; ++i) { out[i] = m[i] * r[i] / (m[i] + q); vv += sq(out[i]); }
    double chi = sqrt(delta * delta + 2.0 * q * vv);
    out[nv] = (delta + chi) / (2.0 * sqrt(ms));
    out[nv + 1] = (-delta + chi) / (2.0 * sqrt(mt));
    return;
  }
  /* Branch choice (derived here): on 0 < xi < q/2 the constraints s, t >= 0 read
   * ms rs + 2 xi rt >= 0 and mt rt + 2 xi rs >= 0; at xi = q/2 both equal a
   * positive multiple of kappa.  f -> -inf at the pole from the side on which
   * s, t >= 0 hold, and f > 0 at the other end of that side's interval, so the
   * admissible root lies below q/2 when kappa > 0 and above q/2 when kappa < 0. */
  rsoc_ctx c = {nv, r, m};
  double xi;
  if (kappa > 0.0) {
    double lo = 0.0;
    double al[2] = {ms * rs, mt * rt}, be[2] = {rt, rs};
    for (int j = 0; j < 2; ++j)
      if (al[j] < 0.0) { double z = -al[j] / (2.0 * be[j]); if (z > lo) lo = z; }
    xi = bisect(rsoc_f, &c, lo, 0.5 * q, 1);
  } else {
    double hi = INFINITY;
    double al[2] = {ms * rs, mt * rt}, be[2] = {rt, rs};
    for (int j = 0; j < 2; ++j)
      if (be[j] > 0.0) { double z = -al[j] / (2.0 * be[j]); if (z < hi) hi = z; }
    if (!isfinite(hi)) {
      hi = q;
      while (rsoc_f(hi, &c) <= 0.0 && hi < 1e300) hi *= 2.0;
    }
    xi = bisect(rsoc_f, &c, 0.5 * q, hi, 0);
  }
  double s, t;
  for (int64_t i = 0; i < nv; ++i) out[i] = m[i] * r[i] / (m[i] + 2.0 * xi);
  rsoc_st(&c, xi, &s, &t);
  out[nv] = fmax(s, 0.0);
  out[nv + 1] = fmax(t, 0.0);
}

/* --- exponential cone K = cl{(r,s,t): s > 0, s exp(r/s) <= t} --- */

/* Decomposition used for both metrics (derived here from the paper's boundary
 * parameterisation eta (rho, 1, e^rho), App. A.4): at the projection p of r,
 * p = eta a(rho) with a = (rho, 1, e^rho), and M(p - r) = mu c(rho) with
 * c = (-1, rho - 1, e^-rho) the dual-cone boundary ray normal to K at p;
 * eta, mu > 0 and r = eta a - mu M^{-1} c.  The scalar rho is a zero of
 *   G(rho) = m_t e^rho (m_s s0 + m_r (rho-1) r0) + m_r m_s e^-rho (rho s0 - r0)
 *            - m_t t0 (m_r rho (rho-1) + m_s),
 * (r in span{a, M^{-1} c}); at the admissible zero G crosses from negative to
 * positive. */
typedef struct { double r0, s0, t0, mr, ms, mt; } exp_ctx;
static double exp_G(double rho, const void* vctx) {
  /* evaluated as e^{-|rho|} G(rho): same sign, no overflow for large |rho| */
  const exp_ctx* c = (const exp_ctx*)vctx;
  double a = c->mt * (c->ms * c->s0 + c->mr * (rho - 1.0) * c->r0);
  double b = c->mr * c->ms * (rho * c->s0 - c->r0);
  double p = c->mt * c->t0 * (c->mr * rho * (rho - 1.0) + c->ms);
  if (rho >= 0.0) {
    double e1 = exp(-rho);
    return a + b * e1 * e1 - p * e1;
  }
  double e1 = exp(rho);
  return a * e1 * e1 + b - p * e1;
}
static double exp_N(double rho, const void* vctx) {  /* numerator of eta_M, scaled by e^{-rho} for rho > 0 */
  const exp_ctx* c = (const exp_ctx*)vctx;
  if (rho > 0.0) {
    double e1 = exp(-rho);
    return (c->mr * rho * c->r0 + c->ms * c->s0) * e1 + c->mt * c->t0;
  }
  return c->mr * rho * c->r0 + c->ms * c->s0 + c->mt * exp(rho) * c->t0;
}
static double exp_g2(double rho, const void* vctx) {  /* -<r, c(rho)>: positive iff mu > 0; scaled by e^{rho} for rho < 0 */
  const exp_ctx* c = (const exp_ctx*)vctx;
  if (rho < 0.0) {
    double e1 = exp(rho);
    return (c->r0 + (1.0 - rho) * c->s0) * e1 - c->t0;
  }
  return c->r0 + (1.0 - rho) * c->s0 - exp(-rho) * c->t0;
}

static int exp_trivial(double r0, double s0, double t0, double mr, double ms, double mt, double* out) {
  /* r in K */
  if ((s0 > 0.0 && s0 * exp(r0 / s0) <= t0) || (r0 <= 0.0 && s0 == 0.0 && t0 >= 0.0)) {
    out[0] = r0; out[1] = s0; out[2] = t0; return 1;
  }
  /* -Mr in K* */
  double u = -mr * r0, v = -ms * s0, w = -mt * t0;
  if ((u < 0.0 && -u * exp(v / u) <= EULER_E * w) || (u == 0.0 && v >= 0.0 && w >= 0.0)) {
    out[0] = out[1] = out[2] = 0.0; return 1;
  }
  /* r0 <= 0, s0 <= 0: projection onto the face {s = 0} (App. A.4) */
  if (r0 <= 0.0 && s0 <= 0.0) {
    out[0] = r0; out[1] = 0.0; out[2] = fmax(t0, 0.0); return 1;
  }
  return 0;
}

static void exp_finish(double rho, const exp_ctx* c, double* out) {
  /* eta_M(rho) (rho, 1, e^rho), App. A.4 eq. exp-metric-projection; for rho > 0 the
   * point is formed as (eta e^rho)(rho e^-rho, e^-rho, 1) to avoid overflow */
  if (rho <= 0.0) {
    double ep = exp(rho);
    double eta = (c->mr * rho * c->r0 + c->ms * c->s0 + c->mt * ep * c->t0) /
                 (c->mr * rho * rho + c->ms + c->mt * ep * ep);
    out[0] = eta * rho;
    out[1] = eta;
    out[2] = eta * ep;
  } else {
    double em = exp(-rho);
    double te = (c->mr * rho * c->r0 * em + c->ms * c->s0 * em + c->mt * c->t0) /
                (c->mr * rho * rho * em * em + c->ms * em * em + c->mt);   /* eta e^rho */
    out[0] = te * rho * em;
    out[1] = te * em;
    out[2] = te;
  }
}

static void proj_exp(const double* r, double* out) {
  /* Euclidean metric.  With M = I the first two components of r = eta a + mu b,
   * b = (1, 1-rho, -e^-rho), give eta = (s0 + (rho-1) r0)/(rho^2-rho+1) and
   * mu = (r0 - rho s0)/(rho^2-rho+1) (denominator > 0), so the admissible set
   * {eta > 0, mu > 0} is an interval cut out by two linear inequalities in rho.
   * G < 0 at its left end and > 0 at its right end. */
  double r0 = r[0], s0 = r[1], t0 = r[2];
  if (exp_trivial(r0, s0, t0, 1.0, 1.0, 1.0, out)) return;
  exp_ctx c = {r0, s0, t0, 1.0, 1.0, 1.0};
  double lo = -INFINITY, hi = INFINITY;
  if (r0 > 0.0) lo = fmax(lo, 1.0 - s0 / r0);
  if (r0 < 0.0) hi = fmin(hi, 1.0 - s0 / r0);
  if (s0 > 0.0) hi = fmin(hi, r0 / s0);
  if (s0 < 0.0) lo = fmax(lo, r0 / s0);
  if (!isfinite(lo)) {
    double step = 1.0;
    lo = hi - step;
    while (exp_G(lo, &c) >= 0.0 && step < 1e8) { step *= 2.0; lo = hi - step; }
  }
  if (!isfinite(hi)) {
    double step = 1.0;
    hi = lo + step;
    while (exp_G(hi, &c) <= 0.0 && step < 1e8) { step *= 2.0; hi = lo + step; }
  }
  double rho = bisect(exp_G, &c, lo, hi, 0);
  exp_finish(rho, &c, out);
}

/* zeros (at most two) of a function that is convex or concave in rho, with
 * stationary point rho_c (NaN if monotone): sign changes located on each
 * monotone piece by outward doubling, then bisection. */
static int piece_roots(scalar_fn f, const void* c, double rho_c, double* roots) {
  int nr = 0;
  double anchors[2];
  int na = 0;
  if (isnan(rho_c)) { anchors[na++] = 0.0; } else { anchors[na++] = rho_c; }
  /* left piece (-inf, a0] and right piece [a_last, inf); if monotone everywhere
   * both pieces share the anchor 0 */
  double a = anchors[0];
  double fa = f(a, c);
  if (fa == 0.0) { roots[nr++] = a; return nr; }
  /* search left */
  {
    double step = 1.0, x = a - step;
    while (step < 1e8) {
      double fx = f(x, c);
      if ((fx > 0.0) != (fa > 0.0)) { roots[nr++] = bisect(f, c, x, a, fx > 0.0); break; }
      step *= 2.0; x = a - step;
    }
  }
  {
    double step = 1.0, x = a + step;
    while (step < 1e8) {
      double fx = f(x, c);
      if ((fx > 0.0) != (fa > 0.0)) { roots[nr++] = bisect(f, c, a, x, fa > 0.0); break; }
      step *= 2.0; x = a + step;
    }
  }
  return nr;
}

static void proj_exp_m(const double* r, const double* m, double* out) {
  /* M-norm (App. A.4 eq. exp-metric-projection).  The admissible zero of G has
   * eta_M > 0 (N > 0) and mu > 0 (g2 > 0).  N and g2 are each convex or concave,
   * so {N > 0, g2 > 0} is a union of at most a few intervals bounded by their
   * zeros; on each such interval G has no zero other than the admissible one,
   * which is an up-crossing.  We enumerate the intervals, keep those with a
   * negative-to-positive sign change of G and bisect. */
  double r0 = r[0], s0 = r[1], t0 = r[2], mr = m[0], ms = m[1], mt = m[2];
  if (exp_trivial(r0, s0, t0, mr, ms, mt, out)) return;
  exp_ctx c = {r0, s0, t0, mr, ms, mt};
  double br[4];
  int nb = 0;
  double rc = NAN;
  if (t0 != 0.0 && -mr * r0 / (mt * t0) > 0.0) rc = log(-mr * r0 / (mt * t0));
  nb += piece_roots(exp_N, &c, rc, br + nb);
  rc = NAN;
  if (s0 != 0.0 && t0 / s0 > 0.0) rc = log(t0 / s0);
  nb += piece_roots(exp_g2, &c, rc, br + nb);
  /* sort breakpoints */
  for (int i = 1; i < nb; ++i)
    for (int j = i; j > 0 && br[j] < br[j - 1]; --j) { double tmp = br[j]; br[j] = br[j - 1]; br[j - 1] = tmp; }
  double ends[6];
  int ne = 0;
  ends[ne++] = -INFINITY;
  for (int i = 0; i < nb; ++i) ends[ne++] = br[i];
  ends[ne++] = INFINITY;
  double best_rho = NAN;
  for (int iv = 0; iv + 1 < ne; ++iv) {
    double a = ends[iv], b = ends[iv + 1];
    if (!(b > a)) continue;
    double p;
    if (isfinite(a) && isfinite(b)) p = 0.5 * (a + b);
    else if (isfinite(a)) p = a + 1.0;
    else if (isfinite(b)) p = b - 1.0;
    else p = 0.0;
    if (!(exp_N(p, &c) > 0.0 && exp_g2(p, &c) > 0.0)) continue;
    double gp = exp_G(p, &c);
    double lo = NAN, hi = NAN;
    if (gp == 0.0) { best_rho = p; break; }
    if (gp < 0.0) {
      lo = p;
      if (isfinite(b)) { if (exp_G(b, &c) > 0.0) hi = b; }
      else {
        double step = 1.0;
        while (step < 1e8) { if (exp_G(p + step, &c) > 0.0) { hi = p + step; break; } step *= 2.0; }
      }
    } else {
      hi = p;
      if (isfinite(a)) { if (exp_G(a, &c) < 0.0) lo = a; }
      else {
        double step = 1.0;
        while (step < 1e8) { if (exp_G(p - step, &c) < 0.0) { lo = p - step; break; } step *= 2.0; }
      }
    }
    if (!isnan(lo) && !isnan(hi)) { best_rho = bisect(exp_G, &c, lo, hi, 0); break; }
  }
  if (isnan(best_rho)) {  /* not expected; fall back to the Euclidean root as a guess */
    double tmp[3];
    proj_exp(r, tmp);
    best_rho = tmp[1] > 0.0 ? log(fmax(tmp[2] / tmp[1], 1e-300)) : 0.0;
  }
  exp_finish(best_rho, &c, out);
}

/* --- power cone K = {(x,y,z): x,y >= 0, x^a y^(1-a) >= |z|} (App. A.5) --- */

static double qroot(double s, double c) {
  /* positive root of u^2 - s u - c = 0 without cancellation (eq. power-cone-stable-quadratic-root) */
  double d = sqrt(s * s + 4.0 * c);
  return s >= 0.0 ? 0.5 * (s + d) : 2.0 * c / (d - s);
}
typedef struct { double rx, ry, R, a, kx, ky; } pow_ctx;
static double pow_g(double rho, const void* vctx) {
  /* g_M(rho) = a log x_M + (1-a) log y_M - log rho (eq. power-projection-root) */
  const pow_ctx* c = (const pow_ctx*)vctx;
  double w = rho * (c->R - rho);
  double x = qroot(c->rx, c->a * c->kx * w);
  double y = qroot(c->ry, (1.0 - c->a) * c->ky * w);
  return c->a * log(x) + (1.0 - c->a) * log(y) - log(rho);
}

static void proj_pow_m(const double* r, const double* m, double alpha, double* out) {
  double rx = r[0], ry = r[1], rz = r[2];
  double mx = m ? m[0] : 1.0, my = m ? m[1] : 1.0, mz = m ? m[2] : 1.0;
  if (rx >= 0.0 && ry >= 0.0 && pow_geo(rx, ry, alpha) >= fabs(rz)) { out[0] = rx; out[1] = ry; out[2] = rz; return; }
  {
    double p = -mx * rx, q = -my * ry, w = -mz * rz;
    if (p >= 0.0 && q >= 0.0 && pow_geo(p / alpha, q / (1.0 - alpha), alpha) >= fabs(w)) {
      out[0] = out[1] = out[2] = 0.0; return;
    }
  }
  if (rz == 0.0) { out[0] = fmax(rx, 0.0); out[1] = fmax(ry, 0.0); out[2] = 0.0; return; }
  double R = fabs(rz);
  pow_ctx c = {rx, ry, R, alpha, mz / mx, mz / my};
  /* Proposition "power-cone-bisection": unique zero in (0, R), g > 0 near 0,
   * g < 0 near R.  The oracle bisects until the midpoint stops moving (a
   * tighter version of the printed eps_bis max{1,R} rule). */
  double rho = bisect(pow_g, &c, 0.0, R, 1);
  double w = rho * (R - rho);
  out[0] = qroot(rx, alpha * c.kx * w);
  out[1] = qroot(ry, (1.0 - alpha) * c.ky * w);
  out[2] = rz > 0.0 ? rho : -rho;
}

/* --- slices with the middle coordinate fixed (Sec. 5.4, eq. fisher-conic) ---
 * X_f = {(r, f, t): f e^{r/f} <= t} (exponential) and {(x, f, z): x^a f^(1-a) >= |z|, x >= 0}
 * (power) for a fixed f > 0.  Both equal f X_1 with X_1 the slice at f = 1, and a projection in a
 * diagonal metric commutes with a positive scalar: argmin_{u in f X_1} ||u - r||_M
 * = f argmin_{v in X_1} ||v - r/f||_M.  On X_1 the middle coordinate is fixed, so the projection
 * is that of the remaining pair onto a 2-D convex set, found from its normal-cone condition as
 * the zero of a monotone scalar function (derived here; the paper gives no formula). */

/* Exponential slice X_1 = {(a, 1, c): e^a <= c}.  Outside X_1 the projection (a, e^a) satisfies
 * M (r - u) = lambda (e^a, -1) with lambda >= 0 (outward normal of e^a - c <= 0), i.e.
 *   phi(a) = m_a (a0 - a) - m_c (e^a - c0) e^a = 0,   a <= a0,  e^a >= c0.
 * On that range phi' = -m_a - m_c e^a (2 e^a - c0) < 0, so the zero is unique.  Bracket:
 * lo = log c0 for c0 > 0 (phi = m_a (a0 - log c0) > 0 there), else the first of
 * min(a0, 0) - 2^k with phi >= 0 (phi -> +inf as a -> -inf); hi = min(a0, log(S + max(c0, 0)))
 * with S^2 = (m_a/m_c)(a0 - lo): there e^a (e^a - c0) >= S^2 >= (m_a/m_c)(a0 - a), so phi <= 0.
 * (The bracket stays a few units wide even when e^{a0} is huge.) */
typedef struct { double a0, c0, ma, mc; } eslice_ctx;
static double eslice_phi(double a, const void* vctx) {
  const eslice_ctx* c = (const eslice_ctx*)vctx;
  double ea = exp(a);
  return c->ma * (c->a0 - a) - c->mc * (ea - c->c0) * ea;
}

/* Power slice X_1 = {(x, 1, z): x^a >= |z|, x >= 0}.  For z0 != 0 outside X_1 the projection is
 * (x, sign(z0) x^a) with x in (max(x0, 0), |z0|^{1/a}) the zero of
 *   psi(x) = m_x (x - x0) - m_z (|z0| - x^a) a x^{a-1},
 * which tends to -infinity at 0+ (or is < 0 at x0 > 0) and is m_x (|z0|^{1/a} - x0) > 0 at the
 * right end; psi' >= m_x > 0 there, so the zero is unique.  At the zero |z0| - x^a <= |z0|, so
 * x^{1-a} (x - x0) <= k = (m_z/m_x) a |z0|: the right end can be lowered to k^{1/(2-a)} (x0 <= 0)
 * or x0 + k x0^{a-1} (x0 > 0).  For z0 = 0 the projection is (max(x0, 0), 0). */
typedef struct { double x0, Z, a, mx, mz; } pslice_ctx;
static double pslice_psi(double x, const void* vctx) {
  const pslice_ctx* c = (const pslice_ctx*)vctx;
  return c->mx * (x - c->x0) - c->mz * (c->Z - pow(x, c->a)) * c->a * pow(x, c->a - 1.0);
}

int orc_proj_slice(int type, double alpha, double f, const double* r, const double* m, double* out) {
  if (!(f > 0.0) || !isfinite(f)) return -1;
  double m0 = m ? m[0] : 1.0, m2 = m ? m[2] : 1.0;
  double a0 = r[0] / f, c0 = r[2] / f;
  double u0, u2;
  if (type == ORC_EXP1) {
    if (exp(a0) <= c0) {
      u0 = a0; u2 = c0;
    } else {
      eslice_ctx c = {a0, c0, m0, m2};
      double lo;
      if (c0 > 0.0) {
        lo = log(c0);
      } else {
        double top = fmin(a0, 0.0), step = 1.0;
        lo = top - step;
        while (eslice_phi(lo, &c) < 0.0 && step < 1e300) { step *= 2.0; lo = top - step; }
      }
      double hi = fmin(a0, log(sqrt((m0 / m2) * (a0 - lo)) + fmax(c0, 0.0)));
      if (!(hi > lo)) hi = a0;
      double a = bisect(eslice_phi, &c, lo, hi, 1);
      u0 = a; u2 = exp(a);
    }
  } else if (type == ORC_POW1) {
    if (!(alpha > 0.0 && alpha < 1.0)) return -1;
    if (a0 >= 0.0 && pow(a0, alpha) >= fabs(c0)) {
      u0 = a0; u2 = c0;
    } else if (c0 == 0.0) {
      u0 = fmax(a0, 0.0); u2 = 0.0;
    } else {
      pslice_ctx c = {a0, fabs(c0), alpha, m0, m2};
      double lo = fmax(a0, 0.0), hi = pow(fabs(c0), 1.0 / alpha);
      double k = (m2 / m0) * alpha * fabs(c0);
      double hb = a0 > 0.0 ? a0 + k * pow(a0, alpha - 1.0) : pow(k, 1.0 / (2.0 - alpha));
      if (hb > lo && hb < hi) hi = hb;
      double x = bisect(pslice_psi, &c, lo, hi, 0);
      u0 = x; u2 = (c0 > 0.0 ? 1.0 : -1.0) * pow(x, alpha);
    }
  } else {
    return -1;
  }
  out[0] = f * u0;
  out[1] = f;
  out[2] = f * u2;
  return 0;
}

int orc_proj_block(int type, int64_t d, double alpha, const double* r, const double* m, double* out) {
  switch (type) {
    case ORC_FREE: memcpy(out, r, (size_t)d * sizeof(double)); return 0;
    case ORC_NONNEG:
      /* App. A.1: metric-independent */
      for (int64_t i = 0; i < d; ++i) out[i] = r[i] > 0.0 ? r[i] : 0.0;
      return 0;
    case ORC_SOC:
      if (d < 2) return -1;
      if (m) proj_soc_m(d, r, m, out); else proj_soc(d, r, out);
      return 0;
    case ORC_RSOC:
      if (d < 3) return -1;
      if (m) proj_rsoc_m(d, r, m, out); else proj_rsoc(d, r, out);
      return 0;
    case ORC_EXP:
      if (d != 3) return -1;
      if (m) proj_exp_m(r, m, out); else proj_exp(r, out);
      return 0;
    case ORC_POW:
      if (d != 3 || !(alpha > 0.0 && alpha < 1.0)) return -1;
      proj_pow_m(r, m, alpha, out);
      return 0;
    case ORC_EXP1: case ORC_POW1:
      if (d != 3) return -1;
      return orc_proj_slice(type, alpha, 1.0, r, m, out);
  }
  return -1;
}

void orc_proj_product(const orc_problem* p, const double* r, const double* m, double* out) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int64_t j = 0; j < p->nblocks; ++j) {
    int64_t s = p->blk_start[j], d = p->blk_dim[j];
    if (p->blk_type[j] == ORC_BOX) {   /* coordinatewise clip: metric-independent (App. A.1) */
      for (int64_t i = s; i < s + d; ++i) out[i] = fmin(fmax(r[i], p->x_lo[i]), p->x_hi[i]);
      continue;
    }
    if (p->blk_type[j] == ORC_EXP1 || p->blk_type[j] == ORC_POW1) {
      orc_proj_slice(p->blk_type[j], p->blk_alpha[j], p->blk_fix ? p->blk_fix[j] : 1.0, r + s, m ? m + s : NULL,
                     out + s);
      continue;
    }
    orc_proj_block(p->blk_type[j], d, p->blk_alpha[j], r + s, m ? m + s : NULL, out + s);
  }
}

/* bounds of row i: [row_lo, row_hi], or [b, b] for an equality row */
static void row_bounds(const orc_problem* p, int64_t i, double* lo, double* hi) {
  if (p->row_lo) { *lo = p->row_lo[i]; *hi = p->row_hi[i]; }
  else { *lo = p->b[i]; *hi = p->b[i]; }
}

/* size of the right-hand side used to normalise primal residuals and in the bound
 * scaling (reading): per row the largest finite bound magnitude (|b_i| for equalities) */
static double bound_norm(const orc_problem* p) {
  double s = 0.0;
  for (int64_t i = 0; i < p->m; ++i) {
    double lo, hi, a = 0.0;
    row_bounds(p, i, &lo, &hi);
    if (isfinite(lo)) a = fmax(a, fabs(lo));
    if (isfinite(hi)) a = fmax(a, fabs(hi));
    s += a * a;
  }
  return sqrt(s);
}

/* ------------------------------------------------------------------------- */
/* KKT report (eq. kkt-cqp; relative measures as read in the build notes R1)  */
/* ------------------------------------------------------------------------- */

/* Support term of a slice block at f = 1: inf over X_1 of sl'x for the dual slack sl.
 * Exponential, X_1 = {(r, 1, t): e^r <= t}: inf = sl_1 + inf_r (sl_0 r + sl_2 e^r), finite only for
 * sl_0 <= 0 <= sl_2; then it is sl_1 + sl_0 (log(-sl_0/sl_2) - 1) (the minimiser e^r = -sl_0/sl_2),
 * sl_1 for sl_0 = 0, and -infinity for sl_0 < 0 = sl_2.  Power, X_1 = {(x, 1, z): x^a >= |z|, x >= 0}:
 * inf = sl_1 + inf_{x >= 0} (sl_0 x - |sl_2| x^a), finite only for sl_0 >= 0; with
 * x* = (a |sl_2| / sl_0)^{1/(1-a)} it is sl_1 - (1-a)/a sl_0 x*, sl_1 for sl_2 = 0, and -infinity
 * for sl_0 = 0 != sl_2.  D = {sl_0 <= 0, sl_2 >= 0} (exp) or {sl_0 >= 0} (pow) is the closed cone
 * of slacks with a finite (or limiting) term; res receives sl - Pi_D(sl), the part counted as dual
 * residual, and the term is evaluated at Pi_D(sl). */
static double slice_support(int type, double alpha, const double* sl, double* res) {
  res[0] = res[1] = res[2] = 0.0;
  if (type == ORC_EXP1) {
    double a = sl[0], c = sl[2];
    if (a > 0.0) { res[0] = a; a = 0.0; }
    if (c < 0.0) { res[2] = c; c = 0.0; }
    if (a == 0.0) return sl[1];
    if (c == 0.0) return -INFINITY;
    return sl[1] + a * (log(-a / c) - 1.0);
  }
  double p = sl[0], w = fabs(sl[2]);
  if (p < 0.0) { res[0] = p; p = 0.0; }
  if (w == 0.0) return sl[1];
  if (p == 0.0) return -INFINITY;
  double xs = pow(alpha * w / p, 1.0 / (1.0 - alpha));
  return sl[1] - (1.0 - alpha) / alpha * p * xs;
}

void orc_kkt(const orc_problem* p, const double* x, const double* y, orc_kkt_report* rep) {
  int64_t m = p->m, n = p->n;
  double* ax = dalloc(m);
  double* aty = dalloc(n);
  double* qx = dalloc(n);
  double* s = dalloc(n);
  double* ps = dalloc(n);
  orc_spmv(m, p->a_rowptr, p->a_colind, p->a_val, x, ax);
  orc_spmv_t(m, n, p->a_rowptr, p->a_colind, p->a_val, y, aty);
  orc_q_apply(p, x, qx);
  /* primal: distance of Ax to [row_lo, row_hi]; dual objective term min_{z in [lo,hi]} y'z,
   * whose finiteness (y_i <= 0 when lo_i = -inf, y_i >= 0 when hi_i = +inf) joins the dual
   * residual; equality rows give |Ax - b| and b'y as before */
  double rp = 0.0, by = 0.0, rd2 = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    double lo, hi;
    row_bounds(p, i, &lo, &hi);
    rp += sq(ax[i] - fmin(fmax(ax[i], lo), hi));
    if (y[i] > 0.0) { if (isfinite(lo)) by += y[i] * lo; else rd2 += sq(y[i]); }
    else if (y[i] < 0.0) { if (isfinite(hi)) by += y[i] * hi; else rd2 += sq(y[i]); }
  }
  rp = sqrt(rp);
  /* s = Qx + c - A'y; on cone blocks dist(s, K*) = ||Pi_K(-s)|| by the Moreau decomposition;
   * on box blocks min_{x_j in [lo,hi]} s_j x_j joins the dual objective and is finite only if
   * s_j <= 0 when lo_j = -inf and s_j >= 0 when hi_j = +inf */
  for (int64_t i = 0; i < n; ++i) s[i] = -(qx[i] + p->c[i] - aty[i]);
  orc_proj_product(p, s, NULL, ps);
  double boxterm = 0.0;
  for (int64_t j = 0; j < p->nblocks; ++j) {
    if (p->blk_type[j] != ORC_BOX) continue;
    for (int64_t i = p->blk_start[j]; i < p->blk_start[j] + p->blk_dim[j]; ++i) {
      double sj = -s[i], lo = p->x_lo[i], hi = p->x_hi[i], r = 0.0;
      if (sj > 0.0) { if (isfinite(lo)) boxterm += sj * lo; else r = sj; }
      else if (sj < 0.0) { if (isfinite(hi)) boxterm += sj * hi; else r = sj; }
      ps[i] = r;
    }
  }
  /* slice blocks (ORC_EXP1 / ORC_POW1, a convex set X_f = f X_1, not a cone): the dual objective
   * gains inf_{x in X_f} s'x = f (s_mid + h(s)), which is finite only on a cone D of dual slacks;
   * the distance of s to D joins the dual residual and h is taken at the projection onto D
   * (reading, the slice analogue of the box terms above; derivation at slice_support) */
  double sliceterm = 0.0;
  for (int64_t j = 0; j < p->nblocks; ++j) {
    int t = p->blk_type[j];
    if (t != ORC_EXP1 && t != ORC_POW1) continue;
    int64_t b0 = p->blk_start[j];
    double sl[3] = {-s[b0], -s[b0 + 1], -s[b0 + 2]};   /* the slack Qx + c - A'y */
    double res[3];
    sliceterm += (p->blk_fix ? p->blk_fix[j] : 1.0) * slice_support(t, p->blk_alpha[j], sl, res);
    for (int q = 0; q < 3; ++q) ps[b0 + q] = res[q];
  }
  double rd = sqrt(dot(n, ps, ps) + rd2);
  double xqx = dot(n, x, qx), cx = dot(n, p->c, x);
  double pobj = 0.5 * xqx + cx, dobj = by + boxterm + sliceterm - 0.5 * xqx;
  rep->norm_res_p = rp;
  rep->norm_res_d = rd;
  rep->eps_p = rp / (1.0 + bound_norm(p));
  rep->eps_d = rd / (1.0 + nrm2(n, p->c));
  /* an infinite support term (dual objective -inf) is the limit eps_g -> 1 */
  rep->eps_g = isfinite(dobj) ? fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj)) : 1.0;
  rep->pobj = pobj;
  rep->dobj = dobj;
  rep->rel_kkt = fmax(rep->eps_p, fmax(rep->eps_d, rep->eps_g));
  free(ax); free(aty); free(qx); free(s); free(ps);
}

/* ------------------------------------------------------------------------- */
/* Working (possibly scaled) copy of the problem                              */
/* ------------------------------------------------------------------------- */

typedef struct {
  int64_t m, n, nnz;
  int64_t *ar, *ac; double* av;      /* A, CSR */
  int64_t *tr, *tc; double* tv;      /* A', CSR (n rows), built by a stable counting sort */
  double* qd;                        /* diag(Q) part, n (zeros if absent) */
  int64_t *pr, *pc; double* pv; int64_t pnnz;   /* sparse P or NULL */
  int64_t k; double *R, *D;          /* low-rank part */
  double *c, *b;
  double *lo, *hi;                   /* row bounds (NULL: equality rows, b) */
  double *xlo, *xhi;                 /* box bounds (NULL: no box blocks) */
  double* csc;                       /* rescaled-cone mode: S_x on cone coordinates (NULL: blocks are cones) */
  double* fix;                       /* per block: fixed middle coordinate of slice blocks (scaled) */
  double beta_b;                     /* bound-objective factor of x (1 before rescaling) */
  orc_problem view;                  /* problem struct pointing at the arrays above */
} wprob;

static void build_transpose(wprob* w) {
  int64_t m = w->m, n = w->n, nnz = w->nnz;
  w->tr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  w->tc = (int64_t*)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(int64_t));
  w->tv = dalloc(nnz);
  for (int64_t k = 0; k < nnz; ++k) w->tr[w->ac[k] + 1]++;
  for (int64_t j = 0; j < n; ++j) w->tr[j + 1] += w->tr[j];
  int64_t* cur = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  memcpy(cur, w->tr, (size_t)n * sizeof(int64_t));
  for (int64_t i = 0; i < m; ++i)
    for (int64_t k = w->ar[i]; k < w->ar[i + 1]; ++k) {
      int64_t j = w->ac[k], pos = cur[j]++;
      w->tc[pos] = i;
      w->tv[pos] = w->av[k];
    }
  free(cur);
}

static void refresh_transpose_values(wprob* w) {
  int64_t* cur = (int64_t*)calloc((size_t)w->n + 1, sizeof(int64_t));
  memcpy(cur, w->tr, (size_t)w->n * sizeof(int64_t));
  for (int64_t i = 0; i < w->m; ++i)
    for (int64_t k = w->ar[i]; k < w->ar[i + 1]; ++k) w->tv[cur[w->ac[k]]++] = w->av[k];
  free(cur);
}

static void wprob_init(wprob* w, const orc_problem* p) {
  memset(w, 0, sizeof(*w));
  w->m = p->m; w->n = p->n; w->nnz = p->a_rowptr[p->m];
  w->ar = (int64_t*)malloc((size_t)(w->m + 1) * sizeof(int64_t));
  memcpy(w->ar, p->a_rowptr, (size_t)(w->m + 1) * sizeof(int64_t));
  w->ac = (int64_t*)malloc((size_t)(w->nnz > 0 ? w->nnz : 1) * sizeof(int64_t));
  memcpy(w->ac, p->a_colind, (size_t)w->nnz * sizeof(int64_t));
  w->av = dalloc(w->nnz);
  memcpy(w->av, p->a_val, (size_t)w->nnz * sizeof(double));
  w->qd = dalloc(w->n);
  if (p->q_diag) memcpy(w->qd, p->q_diag, (size_t)w->n * sizeof(double));
  if (p->p_rowptr) {
    w->pnnz = p->p_rowptr[p->n];
    w->pr = (int64_t*)malloc((size_t)(w->n + 1) * sizeof(int64_t));
    memcpy(w->pr, p->p_rowptr, (size_t)(w->n + 1) * sizeof(int64_t));
    w->pc = (int64_t*)malloc((size_t)(w->pnnz > 0 ? w->pnnz : 1) * sizeof(int64_t));
    memcpy(w->pc, p->p_colind, (size_t)w->pnnz * sizeof(int64_t));
    w->pv = dalloc(w->pnnz);
    memcpy(w->pv, p->p_val, (size_t)w->pnnz * sizeof(double));
  }
  w->k = p->q_rank;
  if (w->k > 0) {
    w->R = dalloc(w->k * w->n);
    memcpy(w->R, p->q_R, (size_t)(w->k * w->n) * sizeof(double));
    w->D = dalloc(w->k * w->k);
    memcpy(w->D, p->q_D, (size_t)(w->k * w->k) * sizeof(double));
  }
  w->c = dalloc(w->n);
  memcpy(w->c, p->c, (size_t)w->n * sizeof(double));
  w->b = dalloc(w->m);
  if (p->b) memcpy(w->b, p->b, (size_t)w->m * sizeof(double));
  if (p->row_lo) {
    w->lo = dalloc(w->m);
    w->hi = dalloc(w->m);
    memcpy(w->lo, p->row_lo, (size_t)w->m * sizeof(double));
    memcpy(w->hi, p->row_hi, (size_t)w->m * sizeof(double));
  }
  if (p->x_lo) {
    w->xlo = dalloc(w->n);
    w->xhi = dalloc(w->n);
    memcpy(w->xlo, p->x_lo, (size_t)w->n * sizeof(double));
    memcpy(w->xhi, p->x_hi, (size_t)w->n * sizeof(double));
  }
  w->fix = dalloc(p->nblocks);
  for (int64_t j = 0; j < p->nblocks; ++j) w->fix[j] = p->blk_fix ? p->blk_fix[j] : 1.0;
  w->beta_b = 1.0;
  build_transpose(w);
  w->view = *p;
  w->view.a_rowptr = w->ar; w->view.a_colind = w->ac; w->view.a_val = w->av;
  w->view.q_diag = w->qd;
  w->view.p_rowptr = w->pr; w->view.p_colind = w->pc; w->view.p_val = w->pv;
  w->view.q_R = w->R; w->view.q_D = w->D;
  w->view.c = w->c; w->view.b = w->b;
  w->view.row_lo = w->lo; w->view.row_hi = w->hi; w->view.x_lo = w->xlo; w->view.x_hi = w->xhi;
  w->view.blk_fix = w->fix;
}

static void wprob_free(wprob* w) {
  free(w->ar); free(w->ac); free(w->av); free(w->tr); free(w->tc); free(w->tv);
  free(w->qd); free(w->pr); free(w->pc); free(w->pv); free(w->R); free(w->D); free(w->c); free(w->b);
  free(w->lo); free(w->hi); free(w->xlo); free(w->xhi); free(w->csc); free(w->fix);
}

static int q_is_diagonal(const wprob* w) { return w->pr == NULL && w->k == 0; }

static void w_q_apply(const wprob* w, const double* x, double* out) {
  q_apply_parts(w->n, w->qd, w->pr, w->pc, w->pv, w->k, w->R, w->D, x, out);
}

/* ------------------------------------------------------------------------- */
/* Rescaling (Sec. 4.2.2, eqs. problem-rescaling, cone-scaling-candidates,    */
/* cone-preserving-scaling; defaults of Table practical-defaults)             */
/* ------------------------------------------------------------------------- */

typedef struct {
  double* col;   /* x_scaled = col .* x / beta_b */
  double* row;   /* A_scaled = diag(1/row) A diag(1/col) */
  double beta_b, beta_c;
} scaling;

/* Cone-preserving aggregation of column candidates: max over the block for
 * Ruiz, root-mean-square over the block for Pock-Chambolle; nonnegative, free
 * and box coordinates stay coordinatewise. */
static void aggregate_blocks(const orc_problem* p, double* cand, int use_rms) {
  for (int64_t j = 0; j < p->nblocks; ++j) {
    int t = p->blk_type[j];
    if (t == ORC_FREE || t == ORC_NONNEG || t == ORC_BOX) continue;
    int64_t s = p->blk_start[j], d = p->blk_dim[j];
    double agg = 0.0;
    if (use_rms) {
      for (int64_t i = 0; i < d; ++i) agg += cand[s + i] * cand[s + i];
      agg = sqrt(agg / (double)d);
    } else {
      for (int64_t i = 0; i < d; ++i) agg = fmax(agg, cand[s + i]);
    }
    for (int64_t i = 0; i < d; ++i) cand[s + i] = agg;
  }
}

static void apply_scaling_step(wprob* w, const double* colf, const double* rowf, double* col, double* row) {
  for (int64_t i = 0; i < w->m; ++i)
    for (int64_t k = w->ar[i]; k < w->ar[i + 1]; ++k) w->av[k] /= rowf[i] * colf[w->ac[k]];
  for (int64_t j = 0; j < w->n; ++j) col[j] *= colf[j];
  for (int64_t i = 0; i < w->m; ++i) row[i] *= rowf[i];
}

static void do_rescale(wprob* w, const orc_problem* p, const orc_options* o, scaling* sc) {
  int64_t m = w->m, n = w->n;
  sc->col = dalloc(n);
  sc->row = dalloc(m);
  for (int64_t j = 0; j < n; ++j) sc->col[j] = 1.0;
  for (int64_t i = 0; i < m; ++i) sc->row[i] = 1.0;
  double* colf = dalloc(n);
  double* rowf = dalloc(m);
  /* Ruiz l_inf: r_i = (max_l |A_li|)^(1/2) per column, same per row */
  for (int it = 0; it < o->ruiz_iters; ++it) {
    for (int64_t j = 0; j < n; ++j) colf[j] = 0.0;
    for (int64_t i = 0; i < m; ++i) {
      double mx = 0.0;
      for (int64_t k = w->ar[i]; k < w->ar[i + 1]; ++k) {
        double a = fabs(w->av[k]);
        if (a > mx) mx = a;
        if (a > colf[w->ac[k]]) colf[w->ac[k]] = a;
      }
      rowf[i] = mx > 0.0 ? sqrt(mx) : 1.0;
    }
    for (int64_t j = 0; j < n; ++j) colf[j] = colf[j] > 0.0 ? sqrt(colf[j]) : 1.0;
    if (!o->rescaled_cones) aggregate_blocks(p, colf, 0);
    apply_scaling_step(w, colf, rowf, sc->col, sc->row);
  }
  /* Pock-Chambolle: p_i = (sum_l |A_li|^(2-alpha))^(1/2) per column and
   * (sum_i |A_li|^alpha)^(1/2) per row */
  if (o->pc_alpha >= 0.0) {
    double al = o->pc_alpha;
    for (int64_t j = 0; j < n; ++j) colf[j] = 0.0;
    for (int64_t i = 0; i < m; ++i) {
      double sr = 0.0;
      for (int64_t k = w->ar[i]; k < w->ar[i + 1]; ++k) {
        double a = fabs(w->av[k]);
        sr += pow(a, al);
        colf[w->ac[k]] += pow(a, 2.0 - al);
      }
      rowf[i] = sr > 0.0 ? sqrt(sr) : 1.0;
    }
    for (int64_t j = 0; j < n; ++j) colf[j] = colf[j] > 0.0 ? sqrt(colf[j]) : 1.0;
    if (!o->rescaled_cones) aggregate_blocks(p, colf, 1);
    apply_scaling_step(w, colf, rowf, sc->col, sc->row);
  }
  free(colf);
  free(rowf);
  /* data in the scaled variables: c~ = c/col, b~ = b/row, Q~ = S^-1 Q S^-1 */
  for (int64_t j = 0; j < n; ++j) w->c[j] /= sc->col[j];
  for (int64_t i = 0; i < m; ++i) w->b[i] /= sc->row[i];
  if (w->lo)   /* bounds scale like b (rows) and like x (boxes); infinities stay */
    for (int64_t i = 0; i < m; ++i) { w->lo[i] /= sc->row[i]; w->hi[i] /= sc->row[i]; }
  if (w->xlo)
    for (int64_t j = 0; j < n; ++j) { w->xlo[j] *= sc->col[j]; w->xhi[j] *= sc->col[j]; }
  for (int64_t j = 0; j < n; ++j) w->qd[j] /= sc->col[j] * sc->col[j];
  if (w->pr)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t t = w->pr[i]; t < w->pr[i + 1]; ++t) w->pv[t] /= sc->col[i] * sc->col[w->pc[t]];
  for (int64_t l = 0; l < w->k; ++l)
    for (int64_t j = 0; j < n; ++j) w->R[l * n + j] /= sc->col[j];
  /* bound-objective: b~ /= beta_b, c~ /= beta_c with beta = ||.||_2 + 1; x scales by
   * 1/beta_b, y by 1/beta_c and Q~ by beta_b/beta_c so the problem stays equivalent */
  sc->beta_b = 1.0;
  sc->beta_c = 1.0;
  if (o->bound_obj) {
    sc->beta_b = bound_norm(&w->view) + 1.0;
    sc->beta_c = nrm2(n, w->c) + 1.0;
    for (int64_t i = 0; i < m; ++i) w->b[i] /= sc->beta_b;
    if (w->lo)
      for (int64_t i = 0; i < m; ++i) { w->lo[i] /= sc->beta_b; w->hi[i] /= sc->beta_b; }
    if (w->xlo)
      for (int64_t j = 0; j < n; ++j) { w->xlo[j] /= sc->beta_b; w->xhi[j] /= sc->beta_b; }
    for (int64_t j = 0; j < n; ++j) w->c[j] /= sc->beta_c;
    double qs = sc->beta_b / sc->beta_c;
    for (int64_t j = 0; j < n; ++j) w->qd[j] *= qs;
    if (w->pr) for (int64_t t = 0; t < w->pnnz; ++t) w->pv[t] *= qs;
    for (int64_t t = 0; t < w->k * w->k; ++t) w->D[t] *= qs;
  }
  refresh_transpose_values(w);
  /* a slice block X_f holds x~ = col x / beta_b; with one factor per block (cone-preserving mode)
   * that is the slice with f~ = f col / beta_b (the set is f X_1 and scales as a whole) */
  w->beta_b = sc->beta_b;
  for (int64_t j = 0; j < p->nblocks; ++j)
    if (!o->rescaled_cones && (p->blk_type[j] == ORC_EXP1 || p->blk_type[j] == ORC_POW1))
      w->fix[j] *= sc->col[p->blk_start[j] + 1] / sc->beta_b;
  /* rescaled-cone mode: the scaled variable x~ = S_x x / beta_b lies in S_j K_j on each
   * cone block (beta_b is a positive scalar and drops out of the cone) */
  if (o->rescaled_cones) {
    w->csc = dalloc(n);
    memcpy(w->csc, sc->col, (size_t)n * sizeof(double));
  }
}

void orc_rescale(const orc_problem* p, const orc_options* o, double* col_scale, double* row_scale, double* beta_bc,
                 double* a_val_out, double* c_out, double* b_out) {
  wprob w;
  scaling sc;
  wprob_init(&w, p);
  do_rescale(&w, p, o, &sc);
  memcpy(col_scale, sc.col, (size_t)p->n * sizeof(double));
  memcpy(row_scale, sc.row, (size_t)p->m * sizeof(double));
  beta_bc[0] = sc.beta_b;
  beta_bc[1] = sc.beta_c;
  if (a_val_out) memcpy(a_val_out, w.av, (size_t)w.nnz * sizeof(double));
  if (c_out) memcpy(c_out, w.c, (size_t)p->n * sizeof(double));
  if (b_out) memcpy(b_out, w.b, (size_t)p->m * sizeof(double));
  free(sc.col); free(sc.row);
  wprob_free(&w);
}

/* Start vector of the norm estimate (reading): entry j is 1/2 + U_j with U_j in [0, 1)
 * the top 53 bits of output j+1 of SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) from state 0, i.e. the finaliser applied to
 * (j+1) times the golden-ratio increment.  An all-ones start can be orthogonal to the top
 * singular subspace (the estimate then converges to a smaller singular value); a positive
 * perturbation of it keeps all-ones' overlap with the leading direction of scaled matrices. */
static double power_start(uint64_t j) {
  uint64_t z = (j + 1) * 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  z = z ^ (z >> 31);
  return 0.5 + (double)(z >> 11) / 9007199254740992.0;
}

void orc_power_start(int64_t n, double* out) {
  for (int64_t j = 0; j < n; ++j) out[j] = power_start((uint64_t)j);
}

/* Largest eigenvalue of the symmetric tridiagonal matrix with diagonal a[0..k) and
 * off-diagonal b[0..k-1), by bisection on the Sturm count (Golub and Van Loan, Matrix
 * Computations, Sec. 8.4.1): below(x) = number of negative pivots of the LDL' factorisation
 * of T - x I = number of eigenvalues below x.  The bracket starts at the Gershgorin bound. */
static double tridiag_max_eig(const double* a, const double* b, int k) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
    if (a[i] - r < lo) lo = a[i] - r;
    if (a[i] + r > hi) hi = a[i] + r;
  }
  for (int step = 0; step < 200 && hi - lo > 1e-15 * fabs(hi); ++step) {
    const double x = 0.5 * (lo + hi);
    int below = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
      d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;      /* an exact zero pivot counts as negative */
      if (d < 0.0) ++below;
    }
    if (below == k) hi = x; else lo = x;
  }
  return hi;
}

double orc_tridiag_max_eig(const double* a, const double* b, int k) { return tridiag_max_eig(a, b, k); }

/* ||A||_2 (needed for eta = 0.998/||A||_2, eq. practical-stepsizes).  The paper does not
 * say how it is estimated; reading: the Lanczos process on A'A (Lanczos 1950; Golub and
 * Van Loan, Sec. 9.1) from the normalised SplitMix64 start above, without
 * reorthogonalisation.  Step j: alpha_j = ||A v_j||^2 (= v_j'A'A v_j),
 * w = A'A v_j - alpha_j v_j - beta_{j-1} v_{j-1}, beta_j = ||w||, v_{j+1} = w / beta_j;
 * sigma_j = sqrt of the largest eigenvalue of the tridiagonal T_j.  Stop when sigma changes
 * by <= tol relative, when beta_j = 0 (an invariant subspace: sigma is exact), or after
 * `iters` steps. */
double orc_norm_est(int64_t m, int64_t n, const int64_t* rowptr, const int64_t* colind, const double* val,
                    int iters, double tol, int* iters_used) {
  double* v = dalloc(n);
  double* vprev = dalloc(n);
  double* av = dalloc(m);
  double* z = dalloc(n);
  double* al = dalloc(iters > 0 ? iters : 1);
  double* be = dalloc(iters > 0 ? iters : 1);
  double vn = 0.0;
  for (int64_t j = 0; j < n; ++j) { v[j] = power_start((uint64_t)j); vn += v[j] * v[j]; }
  vn = sqrt(vn);
  for (int64_t j = 0; j < n; ++j) v[j] = vn > 0.0 ? v[j] / vn : 0.0;
  double sig = 0.0, beta_prev = 0.0;
  int it;
  for (it = 0; it < iters; ++it) {
    orc_spmv(m, rowptr, colind, val, v, av);
    const double alpha = dot(m, av, av);
    orc_spmv_t(m, n, rowptr, colind, val, av, z);
    for (int64_t j = 0; j < n; ++j) z[j] -= alpha * v[j] + beta_prev * vprev[j];
    const double beta = nrm2(n, z);
    al[it] = alpha;
    const double s_new = sqrt(fmax(tridiag_max_eig(al, be, it + 1), 0.0));
    if ((it > 0 && fabs(s_new - sig) <= tol * s_new) || beta == 0.0) { sig = s_new; ++it; break; }
    sig = s_new;
    be[it] = beta;
    for (int64_t j = 0; j < n; ++j) {
      vprev[j] = v[j];
      v[j] = z[j] / beta;
    }
    beta_prev = beta;
  }
  if (iters_used) *iters_used = it;
  free(v); free(vprev); free(av); free(z); free(al); free(be);
  return sig;
}

/* ------------------------------------------------------------------------- */
/* Primal prox (eq. prox-subproblem)                                         */
/* ------------------------------------------------------------------------- */

int orc_proj_block_scaled(int type, int64_t d, double alpha, const double* sc, const double* r, const double* m,
                          double* out) {
  double* rs = dalloc(d);
  double* ms = dalloc(d);
  double* os = dalloc(d);
  for (int64_t i = 0; i < d; ++i) {
    rs[i] = r[i] / sc[i];
    ms[i] = (m ? m[i] : 1.0) * sc[i] * sc[i];
  }
  int rc = orc_proj_block(type, d, alpha, rs, ms, os);
  for (int64_t i = 0; i < d; ++i) out[i] = sc[i] * os[i];
  free(rs); free(ms); free(os);
  return rc;
}

/* Projection of the scaled variable onto the product set in the diagonal metric m
 * (NULL: Euclidean).  In the rescaled-cone mode a cone block is S K with S = diag(csc)
 * on the block; the change of variables u = S w turns the m-metric projection onto S K
 * into S Pi_K^{S m S}(S^-1 r), the metric form of eq. scaling-induced-metric (and of
 * eq. metric-rescaled-cone-equivalence).  Free, nonnegative and box coordinates are
 * projected coordinatewise as in the cone-preserving mode (S R+ = R+). */
static void proj_scaled(const wprob* w, const double* r, const double* m, double* out) {
  if (!w->csc) { orc_proj_product(&w->view, r, m, out); return; }
  const orc_problem* p = &w->view;
  for (int64_t j = 0; j < p->nblocks; ++j) {
    int64_t s = p->blk_start[j], d = p->blk_dim[j];
    int t = p->blk_type[j];
    if (t == ORC_FREE || t == ORC_NONNEG || t == ORC_BOX) {
      orc_problem one = *p;
      one.nblocks = 1;
      one.blk_type = p->blk_type + j; one.blk_start = p->blk_start + j; one.blk_dim = p->blk_dim + j;
      one.blk_alpha = p->blk_alpha + j;
      orc_proj_product(&one, r, m, out);
      continue;
    }
    if (t == ORC_EXP1 || t == ORC_POW1) {
      /* a slice is not a cone, so beta_b stays: x~ lies in S X_f / beta_b, projected as
       * S' Pi_{X_f}^{S' m S'}(S'^-1 r) with S' = S / beta_b (w->fix keeps the original f in
       * this mode) */
      double sc3[3], r3[3], m3[3], o3[3];
      for (int q = 0; q < 3; ++q) {
        sc3[q] = w->csc[s + q] / w->beta_b;
        r3[q] = r[s + q] / sc3[q];
        m3[q] = (m ? m[s + q] : 1.0) * sc3[q] * sc3[q];
      }
      orc_proj_slice(t, p->blk_alpha[j], w->fix[j], r3, m3, o3);
      for (int q = 0; q < 3; ++q) out[s + q] = sc3[q] * o3[q];
      continue;
    }
    orc_proj_block_scaled(t, d, p->blk_alpha[j], w->csc + s, r + s, m ? m + s : NULL, out + s);
  }
}

/* Diagonal Q: single metric projection p = Pi^{M}(x~), M = I + tau diag(q),
 * x~ = M^{-1}(v - tau c) with v = x + tau A'y (eqs. diagonal-q-metric,
 * diagonal-q-metric-projection).  The scaled variable is used directly, so M_sc = I here;
 * in the rescaled-cone mode the cone scaling enters through proj_scaled, which is the
 * same projection written in the scaled coordinates. */
static void prox_diag(const wprob* w, double tau, const double* v, double* out) {
  int64_t n = w->n;
  double* mm = dalloc(n);
  double* xt = dalloc(n);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < n; ++i) {
    mm[i] = 1.0 + tau * w->qd[i];
    xt[i] = (v[i] - tau * w->c[i]) / mm[i];
  }
  proj_scaled(w, xt, mm, out);
  free(mm); free(xt);
}

/* Projected Barzilai-Borwein with the Jacobi metric J = diag(Q) + I/tau
 * (eqs. bb-inner-gradient, jacobi-bb-step), stopping when the Euclidean norm of
 * the last projected update is <= eps_in (eqs. current-inner-step-stop,
 * jacobi-stop-unscale).  Readings: first step alpha = 1 (a plain Jacobi step;
 * for the Euclidean variant alpha_0 = 1/max_i J_ii); if <s, dg> <= 1e-30 the
 * previous alpha is kept; alpha clipped to [1e-10, 1e10]. */
static int prox_bb(const wprob* w, double tau, const double* v, const double* u0, double eps_in, int max_inner,
                   int jacobi, double* u_out, double* last_du) {
  int64_t n = w->n;
  double* J = dalloc(n);
  double* u = dalloc(n);
  double* un = dalloc(n);
  double* g = dalloc(n);
  double* gn = dalloc(n);
  double* q = dalloc(n);
  double* trial = dalloc(n);
  double jmax = 0.0;
  /* J = diag(Q) + I/tau with the full diagonal of Q = diag(q) + P + R'DR (eq. jacobi-inner-metric) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(max : jmax)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double qi = w->qd[i];
    if (w->pr)
      for (int64_t t = w->pr[i]; t < w->pr[i + 1]; ++t)
        if (w->pc[t] == i) qi += w->pv[t];
    for (int64_t l = 0; l < w->k; ++l)
      for (int64_t l2 = 0; l2 < w->k; ++l2) qi += w->R[l * n + i] * w->D[l * w->k + l2] * w->R[l2 * n + i];
    J[i] = jacobi ? qi + 1.0 / tau : 1.0;
    if (qi + 1.0 / tau > jmax) jmax = qi + 1.0 / tau;
  }
  memcpy(u, u0, (size_t)n * sizeof(double));
  w_q_apply(w, u, q);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < n; ++i) g[i] = q[i] + w->c[i] + (u[i] - v[i]) / tau;
  double alpha = jacobi ? 1.0 : 1.0 / jmax;
  int it;
  double du = 0.0;
  for (it = 0; it < max_inner; ++it) {
    #ifdef _OPENMP
    #pragma omp parallel for schedule(static)
    #endif
    for (int64_t i = 0; i < n; ++i) trial[i] = u[i] - alpha * g[i] / J[i];
    proj_scaled(w, trial, jacobi ? J : NULL, un);
    du = sqrt(dist2(n, un, u));
    if (du <= eps_in) { memcpy(u, un, (size_t)n * sizeof(double)); ++it; break; }
    w_q_apply(w, un, q);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) {
      gn[i] = q[i] + w->c[i] + (un[i] - v[i]) / tau;
      trial[i] = un[i] - u[i];          /* s = u^{j+1} - u^j */
    }
    /* <s, J s> and <s, dg> with dg = g^{j+1} - g^j */
    double sjs = csum(2, n, trial, trial, J), sdg = csum(3, n, trial, gn, g);
    if (sdg > 1e-30) alpha = sjs / sdg;
    if (alpha < 1e-10) alpha = 1e-10;
    if (alpha > 1e10) alpha = 1e10;
    memcpy(u, un, (size_t)n * sizeof(double));
    memcpy(g, gn, (size_t)n * sizeof(double));
  }
  memcpy(u_out, u, (size_t)n * sizeof(double));
  if (last_du) *last_du = du;
  free(J); free(u); free(un); free(g); free(gn); free(q); free(trial);
  return it;
}

static int do_prox(const wprob* w, double tau, const double* v, const double* u0, double eps_in, int max_inner,
                   int jacobi, int force_inner, double* out) {
  if (q_is_diagonal(w) && !force_inner) { prox_diag(w, tau, v, out); return 1; }
  return prox_bb(w, tau, v, u0, eps_in, max_inner, jacobi, out, NULL);
}

/* One primal-first PDHG operator evaluation T(z) (eq. theory-pdhg-map). */
static int pdhg_operator(const wprob* w, double tau, double sigma, const double* x, const double* y, double eps_in,
                         int max_inner, int jacobi, int force_inner, double* xo, double* yo, double* scratch_n,
                         double* scratch_m) {
  int64_t m = w->m, n = w->n;
  double* v = scratch_n;
  orc_spmv(n, w->tr, w->tc, w->tv, y, v);            /* A'y via the transpose CSR */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < n; ++i) v[i] = x[i] + tau * v[i];
  int inner = do_prox(w, tau, v, x, eps_in, max_inner, jacobi, force_inner, xo);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < n; ++i) v[i] = 2.0 * xo[i] - x[i];
  orc_spmv(m, w->ar, w->ac, w->av, v, scratch_m);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < m; ++i) {
    double lo, hi;
    row_bounds(&w->view, i, &lo, &hi);
    if (lo == hi) {
      yo[i] = y[i] + sigma * (lo - scratch_m[i]);
    } else {
      /* prox of the support function of [lo, hi] (Moreau): y - sigma v + sigma Pi(v - y/sigma) */
      const double v = scratch_m[i];
      yo[i] = y[i] - sigma * v + sigma * fmin(fmax(v - y[i] / sigma, lo), hi);
    }
  }
  return inner;
}

int orc_pdhg_operator(const orc_problem* p, double tau, double sigma, const double* x, const double* y, double eps_in,
                      int max_inner, int jacobi, int force_inner, double* x_out, double* y_out) {
  wprob w;
  wprob_init(&w, p);
  double* sn = dalloc(p->n);
  double* sm = dalloc(p->m);
  int it = pdhg_operator(&w, tau, sigma, x, y, eps_in, max_inner, jacobi, force_inner, x_out, y_out, sn, sm);
  free(sn); free(sm);
  wprob_free(&w);
  return it;
}

int orc_prox(const orc_problem* p, double tau, const double* v, const double* u0, double eps_in, int max_inner,
             int jacobi, int force_inner, double* u_out) {
  wprob w;
  wprob_init(&w, p);
  int it = do_prox(&w, tau, v, u0, eps_in, max_inner, jacobi, force_inner, u_out);
  wprob_free(&w);
  return it;
}

/* ------------------------------------------------------------------------- */
/* Restarted PDHG (Alg. "pdhcq1"; Sec. 4.2.1 reflected Halpern, 4.2.3 adaptive */
/* inner accuracy, 4.2.5 step sizes, PID primal weight and adaptive restart)  */
/* ------------------------------------------------------------------------- */

void orc_default_options(orc_options* o) {
  memset(o, 0, sizeof(*o));
  o->ruiz_iters = 10; o->pc_alpha = 1.0; o->bound_obj = 1;
  o->eps0_in = 1e-3; o->gamma_in = 5e-4; o->eps_min_in = 1e-9;
  o->jacobi = 1; o->rho = 1.0;
  o->beta_s = 0.2; o->beta_n = 0.8; o->beta_a = 0.36;
  o->beta_I = 0.3; o->K_P = 0.99; o->K_I = 0.01; o->K_D = 0.0;
  o->check_every = 64; o->max_iter = 100000; o->max_inner = 1000; o->tol = 1e-4;
  o->update = 0; o->avg_epoch = 64;
  o->power_iters = 200; o->power_tol = 1e-6; o->step_factor = 0.998;
  o->force_inner = 0; o->pid = 1; o->hist_cap = 0; o->rescaled_cones = 0;
}

static void unscale(const wprob* w, const scaling* sc, const double* xs, const double* ys, double* x, double* y) {
  for (int64_t j = 0; j < w->n; ++j) x[j] = sc->beta_b * xs[j] / sc->col[j];
  for (int64_t i = 0; i < w->m; ++i) y[i] = sc->beta_c * ys[i] / sc->row[i];
}

/* E^2 = w ||dx||^2 + ||dy||^2/w + 2 eta <A dx, dy> (eq. practical-fixed-point-movement) */
static double fixed_point_error(const wprob* w, double omega, double eta, const double* hx, const double* hy,
                                const double* wx, const double* wy, double* dxn, double* adx) {
  int64_t m = w->m, n = w->n;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t j = 0; j < n; ++j) dxn[j] = hx[j] - wx[j];
  orc_spmv(m, w->ar, w->ac, w->av, dxn, adx);
  double dx2 = dot(n, dxn, dxn), dy2 = dist2(m, hy, wy), cross = csum(3, m, adx, hy, wy);
  double e2 = omega * dx2 + dy2 / omega + 2.0 * eta * cross;
  return sqrt(fmax(e2, 0.0));
}

/* Adaptive restart (eq. practical-restart-rule): sufficient decay, necessary decay without local
 * progress, or the artificial limit, tested from the epoch's second iteration on. */
int orc_restart_rule(double E, double E0, double Eprev, int64_t k, int64_t ktot, const orc_options* o) {
  if (k < 1) return 0;
  if (E <= o->beta_s * E0) return 1;
  if (E <= o->beta_n * E0 && E > Eprev) return 1;
  if ((double)k >= o->beta_a * (double)ktot) return 1;
  return 0;
}

/* PID primal weight (eqs. pid-error, pid-weight):
 *   e_n = log(||dy|| / (omega_n ||dx||)),  I_n = beta_I I_{n-1} + e_n,
 *   log omega_{n+1} = log omega_n + K_P e_n + K_I I_n + K_D (e_n - e_{n-1}). */
double orc_pid_update(double omega, double dx, double dy, const orc_options* o, double* state) {
  if (!o->pid || !(dx > 1e-10) || !(dy > 1e-10)) return omega;
  double e = log(dy / (omega * dx));
  state[0] = o->beta_I * state[0] + e;
  double lw = log(omega) + o->K_P * e + o->K_I * state[0] + o->K_D * (e - state[1]);
  state[1] = e;
  return exp(lw);
}

/* Adaptive inner tolerance (eq. monotone-primal-inner-tol):
 *   eps_k = min{eps_{k-1}, max{gamma_in ||x^{n,k} - x^{n,k-1}|| / tau_n, eps_min}}. */
double orc_inner_tol(double eps_prev, double mov, double tau, const orc_options* o) {
  return fmin(eps_prev, fmax(o->gamma_in * mov / tau, o->eps_min_in));
}

int orc_solve(const orc_problem* p, const orc_options* o, const double* x0, const double* y0, double* x_out,
              double* y_out, orc_info* info) {
  int64_t m = p->m, n = p->n;
  for (int64_t j = 0; j < p->nblocks; ++j)
    if ((p->blk_type[j] == ORC_EXP1 || p->blk_type[j] == ORC_POW1) && p->blk_fix && !(p->blk_fix[j] > 0.0))
      return -1;
  wprob w;
  scaling sc;
  wprob_init(&w, p);
  do_rescale(&w, p, o, &sc);
  int pits = 0;
  double normA = orc_norm_est(m, n, w.ar, w.ac, w.av, o->power_iters, o->power_tol, &pits);
  double eta = o->step_factor / (normA > 0.0 ? normA : 1.0);
  /* initial primal weight (reading): ||c~||/||b~|| when both are positive, else 1 */
  double cn = nrm2(n, w.c), bn = bound_norm(&w.view);
  double omega = (cn > 1e-10 && bn > 1e-10) ? cn / bn : 1.0;
  double tau = eta / omega, sigma = eta * omega;

  double *hx = dalloc(n), *hy = dalloc(m), *ax = dalloc(n), *ay = dalloc(m);
  double *wx = dalloc(n), *wy = dalloc(m), *xprev = dalloc(n);
  double *sn = dalloc(n), *sm = dalloc(m), *sn2 = dalloc(n);
  double *ux = dalloc(n), *uy = dalloc(m);
  double *avx = dalloc(n), *avy = dalloc(m);   /* running averages (averaged variant) */
  /* warm start in scaled variables */
  for (int64_t j = 0; j < n; ++j) hx[j] = x0 ? x0[j] * sc.col[j] / sc.beta_b : 0.0;
  for (int64_t i = 0; i < m; ++i) hy[i] = y0 ? y0[i] * sc.row[i] / sc.beta_c : 0.0;
  memcpy(ax, hx, (size_t)n * sizeof(double));
  memcpy(ay, hy, (size_t)m * sizeof(double));
  memcpy(xprev, hx, (size_t)n * sizeof(double));
  double eps_in = o->eps0_in;
  double pid_state[2] = {0.0, 0.0};   /* I_{n-1}, e_{n-1}; reading: both start at 0 */
  double E0 = 0.0, Eprev = 0.0;
  int64_t k = 0, ktot = 0, restarts = 0, inner_total = 0;
  double mov = 0.0;
  int status = 1;
  orc_kkt_report rep;
  memset(&rep, 0, sizeof(rep));
  int hist_len = 0;
  int averaged = (o->update == 1);

  while (ktot < o->max_iter) {
    /* adaptive inner tolerance (eq. monotone-primal-inner-tol) for k >= 1, with
     * x^{n,k} - x^{n,k-1} read as consecutive stored candidates */
    if (k >= 1) eps_in = orc_inner_tol(eps_in, mov, tau, o);
    int inner = pdhg_operator(&w, tau, sigma, hx, hy, eps_in, o->max_inner, o->jacobi, o->force_inner, wx, wy, sn,
                              sm);
    inner_total += inner;
    mov = sqrt(dist2(n, wx, xprev));
    memcpy(xprev, wx, (size_t)n * sizeof(double));
    ktot += 1;
    int check = (ktot % o->check_every) == 0 || ktot >= o->max_iter;

    if (averaged) {
      /* Cesaro average of the epoch's iterates z^{n,k+1} (Alg. 1, averaged branch) */
      for (int64_t j = 0; j < n; ++j) avx[j] = (k * avx[j] + wx[j]) / (double)(k + 1);
      for (int64_t i = 0; i < m; ++i) avy[i] = (k * avy[i] + wy[i]) / (double)(k + 1);
      memcpy(hx, wx, (size_t)n * sizeof(double));
      memcpy(hy, wy, (size_t)m * sizeof(double));
      k += 1;
      if (check) {
        unscale(&w, &sc, avx, avy, ux, uy);
        orc_kkt(p, ux, uy, &rep);
        if (info && info->hist_iter && hist_len < o->hist_cap) {
          info->hist_iter[hist_len] = ktot; info->hist_kkt[hist_len] = rep.rel_kkt;
          info->hist_gap[hist_len] = fabs(rep.pobj - rep.dobj); info->hist_E[hist_len] = 0.0;
          info->hist_restart[hist_len] = 0; hist_len++;
        }
        if (rep.rel_kkt <= o->tol) { status = 0; memcpy(wx, avx, (size_t)n * 8); memcpy(wy, avy, (size_t)m * 8); break; }
      }
      if (k >= o->avg_epoch) {  /* restart from the epoch average */
        memcpy(hx, avx, (size_t)n * sizeof(double));
        memcpy(hy, avy, (size_t)m * sizeof(double));
        k = 0; restarts++;
      }
      continue;
    }

    double E = -1.0;
    if (k == 0) {
      E = fixed_point_error(&w, omega, eta, hx, hy, wx, wy, sn2, sm);
      E0 = E;
      Eprev = E;
    }
    int do_restart = 0;
    if (check) {
      if (E < 0.0) E = fixed_point_error(&w, omega, eta, hx, hy, wx, wy, sn2, sm);
      unscale(&w, &sc, wx, wy, ux, uy);
      orc_kkt(p, ux, uy, &rep);
      if (rep.rel_kkt <= o->tol) {
        status = 0;
        if (info && info->hist_iter && hist_len < o->hist_cap) {
          info->hist_iter[hist_len] = ktot; info->hist_kkt[hist_len] = rep.rel_kkt;
          info->hist_gap[hist_len] = fabs(rep.pobj - rep.dobj); info->hist_E[hist_len] = E;
          info->hist_restart[hist_len] = 0; hist_len++;
        }
        break;
      }
      /* restart rule (eq. practical-restart-rule) */
      do_restart = orc_restart_rule(E, E0, Eprev, k, ktot, o);
      Eprev = E;
      if (info && info->hist_iter && hist_len < o->hist_cap) {
        info->hist_iter[hist_len] = ktot; info->hist_kkt[hist_len] = rep.rel_kkt;
        info->hist_gap[hist_len] = fabs(rep.pobj - rep.dobj); info->hist_E[hist_len] = E;
        info->hist_restart[hist_len] = do_restart; hist_len++;
      }
    }
    if (do_restart) {
      /* PID primal weight (eqs. pid-error, pid-weight) from the accepted endpoint
       * w^{n,N} against the epoch start z^{n,0} = a^n.  Reading: skipped when either
       * movement is below 1e-10. */
      double dxn = sqrt(dist2(n, wx, ax)), dyn = sqrt(dist2(m, wy, ay));
      omega = orc_pid_update(omega, dxn, dyn, o, pid_state);
      tau = eta / omega;
      sigma = eta * omega;
      /* restart from the final stored candidate (eq. restart-output) */
      memcpy(ax, wx, (size_t)n * sizeof(double));
      memcpy(ay, wy, (size_t)m * sizeof(double));
      memcpy(hx, wx, (size_t)n * sizeof(double));
      memcpy(hy, wy, (size_t)m * sizeof(double));
      k = 0;
      restarts++;
    } else {
      /* anchored reflected-Halpern step (eq. rh-update) */
      double c1 = (double)(k + 1) / (double)(k + 2), c2 = 1.0 / (double)(k + 2), r2 = 2.0 * o->rho,
             r1 = 1.0 - 2.0 * o->rho;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
      for (int64_t j = 0; j < n; ++j) hx[j] = c1 * (r2 * wx[j] + r1 * hx[j]) + c2 * ax[j];
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
      for (int64_t i = 0; i < m; ++i) hy[i] = c1 * (r2 * wy[i] + r1 * hy[i]) + c2 * ay[i];
      k += 1;
    }
  }
  if (status != 0) {
    unscale(&w, &sc, averaged ? avx : wx, averaged ? avy : wy, ux, uy);
    orc_kkt(p, ux, uy, &rep);
  } else {
    unscale(&w, &sc, wx, wy, ux, uy);
  }
  if (x_out) memcpy(x_out, ux, (size_t)n * sizeof(double));
  if (y_out) memcpy(y_out, uy, (size_t)m * sizeof(double));
  if (info) {
    info->status = status; info->iters = ktot; info->restarts = restarts; info->inner_total = inner_total;
    info->eta = eta; info->norm_A = normA; info->omega = omega; info->beta_b = sc.beta_b; info->beta_c = sc.beta_c;
    info->kkt = rep; info->hist_len = hist_len;
  }
  free(hx); free(hy); free(ax); free(ay); free(wx); free(wy); free(xprev); free(sn); free(sm); free(sn2);
  free(ux); free(uy); free(avx); free(avy);
  free(sc.col); free(sc.row);
  wprob_free(&w);
  return status;
}
