// Cone projections on the GPU (paper App. "cone-projections", Table
// "cone-projection-methods").  Conventions of the standard form (Sec. 4):
//   SOC  (v, t), t last;  RSOC (v, s, t), ||v||^2 <= 2 s t, s, t last;
//   EXP  (r, s, t), s exp(r/s) <= t;  POW (r, s, t), r^a s^(1-a) >= |t|.
// Metric projections Pi^M_K(z) = argmin_{u in K} ||u - z||_M^2 with diagonal M.
//
// SOC / RSOC blocks are projected by one warp: the block's coordinates are
// strided over the lanes, norms and root-function sums are warp reductions,
// and the scalar root iteration runs on lane 0, which broadcasts each iterate.
// EXP / POW blocks are projected by one thread in FP64.
#pragma once

#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace cqp {

template <typename T> struct Tol;
template <> struct Tol<float> { static constexpr double rel = 4e-7; };
template <> struct Tol<double> { static constexpr double rel = 4e-16; };
// unit roundoff of the element sums' precision
template <typename T> struct Unit;
template <> struct Unit<float> { static constexpr double u = 5.9604644775390625e-08; };
template <> struct Unit<double> { static constexpr double u = 1.1102230246251565e-16; };

// FP64 on this GPU runs at about 1/57 of the FP32 rate, so the warp-level
// projections keep element work and warp trees in the iterate precision T and
// run the FP64 scalar iteration on lane 0 only, broadcasting its result.

__device__ __forceinline__ double bcast(double v) { return __shfl_sync(0xffffffffu, v, 0); }

// --------------------------------------------------------------------------
// Second-order cone, Euclidean (App. A.2, eq. soc-euclidean-projection).
// x holds the d coordinates (v_1..v_{d-1}, t); projected in place.
// --------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ void warp_soc_euclid(T* x, int d, int lane) {
  T s = T(0);
  for (int i = lane; i < d - 1; i += 32) s += x[i] * x[i];
  const T t = x[d - 1];
  s = warp_sum(s);
  const T a = sqrt(s);
  if (a <= t) return;
  if (a <= -t) {
    for (int i = lane; i < d; i += 32) x[i] = T(0);
    __syncwarp();
    return;
  }
  const T coef = (a + t) / (T(2) * a);
  for (int i = lane; i < d - 1; i += 32) x[i] = coef * x[i];
  if (lane == 0) x[d - 1] = T(0.5) * (a + t);
  __syncwarp();
}

// --------------------------------------------------------------------------
// Second-order cone in the metric M = diag(m) (App. A.2, eq.
// soc-metric-projection): v_i(l) = m_i z_i/(m_i + l), t(l) = m_t z_t/(m_t - l).
// The admissible root solves psi(l) = 1/t(l) - 1/||v(l)|| = 0 (the same root as
// ||v||^2 - t^2, nearly linear in l so Newton needs few steps), with
// psi' = -1/(m_t z_t) - S3/S^{3/2}, S = sum a_i/(m_i+l)^2, S3 = sum a_i/(m_i+l)^3,
// a_i = (m_i z_i)^2.  Bracket: (0, m_t) when z_t > 0 (psi > 0 at 0, < 0 at m_t);
// (m_t, l_U] when z_t < 0 with l_U = (A m_t + B m_max)/(A - B), A = ||M_v z_v||,
// B = m_t |z_t| (||v||^2 >= A^2/(m_max + l)^2 gives psi(l_U) >= 0).  Singular
// z_t = 0: l = m_t, t = ||v||.
// --------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ void warp_soc_metric(T* x, const T* m, int d, int lane, float* guess = nullptr) {
  const int nv = d - 1;
  T v2 = T(0), A2 = T(0), mmax = T(0);
  for (int i = lane; i < nv; i += 32) {
    const T xi = x[i], mi = m[i];
    v2 += xi * xi;
    A2 += (mi * xi) * (mi * xi);
    mmax = mi > mmax ? mi : mmax;
  }
  const T zt = x[nv], mt = m[nv];
  v2 = warp_sum(v2);
  A2 = warp_sum(A2);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) { const T q = __shfl_xor_sync(0xffffffffu, mmax, o); mmax = q > mmax ? q : mmax; }
  if (sqrt(v2) <= zt) return;                          // z in K
  const T A = sqrt(A2), B = mt * (zt < T(0) ? -zt : zt);
  if (zt <= T(0) && A <= B) {                          // -Mz in K* = K
    for (int i = lane; i < d; i += 32) x[i] = T(0);
    __syncwarp();
    return;
  }
  T lam = mt;
  if (zt != T(0)) {
    // lane 0 holds the bracket and the Newton state (scalars in the iterate precision T)
    T lo, hi;
    if (zt > T(0)) { lo = T(0); hi = mt; }
    else { lo = mt; hi = (A * mt + B * mmax) / (A - B) * T(1.000001) + T(1e-30); }
    const bool lo_pos = zt > T(0);
    const T inv_mtzt = T(1) / (mt * zt);
    lam = T(0.5) * (lo + hi);
    // warm start from the previous root of this block when it lies in the bracket
    if (guess) {
      const T g0 = T(*guess);
      if (g0 > lo && g0 < hi) lam = g0;
    }
    for (int it = 0; it < 100; ++it) {
      T s2t = T(0), s3t = T(0);
      for (int i = lane; i < nv; i += 32) {
        const T mi = m[i], xi = x[i];
        const T ai = (mi * xi) * (mi * xi);
        const T den = mi + lam;
        const T q = ai / (den * den);
        s2t += q;
        s3t += q / den;
      }
      s2t = warp_sum(s2t);
      s3t = warp_sum(s3t);
      int done = 0;
      if (lane == 0) {
        const T nrm = sqrt(s2t);
        const T a = (mt - lam) * inv_mtzt, b = T(1) / nrm;
        const T psi = a - b;
        const T dpsi = -inv_mtzt - s3t / (s2t * nrm);
        // psi within a few roundings of its terms is noise: its sign no longer tells the side of
        // the root, so the iteration stops
        const T noise = T(8.0 * Unit<T>::u) * ((a < T(0) ? -a : a) + b);
        if (psi == T(0) || (psi < T(0) ? -psi : psi) <= noise) {
          done = 1;
        } else {
          if ((psi > T(0)) == lo_pos) lo = lam; else hi = lam;
          T nx = (dpsi != T(0)) ? lam - psi / dpsi : T(0.5) * (lo + hi);
          if (!(nx > lo && nx < hi)) nx = T(0.5) * (lo + hi);
          const T step = nx > lam ? nx - lam : lam - nx;
          lam = nx;
          const T tol = T(Tol<T>::rel) * (lam > T(1e-30) ? lam : T(1e-30));
          done = (step <= tol || (hi - lo) <= tol) ? 1 : 0;
        }
      }
      lam = __shfl_sync(0xffffffffu, lam, 0);
      if (__shfl_sync(0xffffffffu, done, 0)) break;
    }
  }
  if (guess && lane == 0 && zt != T(0)) *guess = (float)lam;
  const T lt = lam;
  T vv = T(0);
  for (int i = lane; i < nv; i += 32) {
    const T mi = m[i];
    const T vi = mi * x[i] / (mi + lt);
    x[i] = vi;
    vv += vi * vi;
  }
  vv = warp_sum(vv);
  if (lane == 0) x[nv] = sqrt(vv);
  __syncwarp();
}

// --------------------------------------------------------------------------
// Rotated SOC, Euclidean: U^{-1} Pi_soc(U z), U(v,s,t) = ((v,(s-t)/sqrt2),(s+t)/sqrt2)
// (App. A.3, eq. rsoc-via-soc).
// --------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ void warp_rsoc_euclid(T* x, int d, int lane) {
  const int nv = d - 2;
  const T h = T(0.70710678118654752440);
  T s = T(0);
  for (int i = lane; i < nv; i += 32) s += x[i] * x[i];
  const T zs = x[nv], zt = x[nv + 1];
  s = warp_sum(s);
  const T w = (zs - zt) * h, tt = (zs + zt) * h;
  const T a = sqrt(s + w * w);
  if (a <= tt) return;
  if (a <= -tt) {
    for (int i = lane; i < d; i += 32) x[i] = T(0);
    __syncwarp();
    return;
  }
  const T coef = (a + tt) / (T(2) * a);
  for (int i = lane; i < nv; i += 32) x[i] = coef * x[i];
  if (lane == 0) {
    const T wp = coef * w, tp = T(0.5) * (a + tt);
    x[nv] = (wp + tp) * h;
    x[nv + 1] = (tp - wp) * h;
  }
  __syncwarp();
}

// --------------------------------------------------------------------------
// Rotated SOC in the metric M (App. A.3, eq. rsoc-metric-projection):
// v_i(xi) = m_i z_i/(m_i + 2 xi); [m_s, -2xi; -2xi, m_t][s; t] = [m_s z_s; m_t z_t];
// f(xi) = ||v||^2 - 2 s t.  Singular 2 xi = q = sqrt(m_s m_t) with consistent
// right-hand side handled by eq. rsoc-metric-singular-projection.  Branch: with
// kappa = sqrt(m_s) z_s + sqrt(m_t) z_t the admissible root (s, t >= 0) lies in
// (l, q/2) when kappa > 0 and in (q/2, u) when kappa < 0, where l, u are the
// points at which s or t changes sign; f > 0 at l (or u, or infinity) and
// f -> -inf at the pole.  Safeguarded Newton on f inside that bracket.
// --------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ void warp_rsoc_metric(T* x, const T* m, int d, int lane, float* guess = nullptr) {
  const int nv = d - 2;
  T v2 = T(0), mv2 = T(0);
  for (int i = lane; i < nv; i += 32) {
    const T xi = x[i], mi = m[i];
    v2 += xi * xi;
    mv2 += (mi * xi) * (mi * xi);
  }
  const double zs = (double)x[nv], zt = (double)x[nv + 1];
  const double ms = (double)m[nv], mt = (double)m[nv + 1];
  v2 = warp_sum(v2);
  mv2 = warp_sum(mv2);
  if (zs >= 0.0 && zt >= 0.0 && (double)v2 <= 2.0 * zs * zt) return;
  if (zs <= 0.0 && zt <= 0.0 && (double)mv2 <= 2.0 * (ms * zs) * (mt * zt)) {
    for (int i = lane; i < d; i += 32) x[i] = T(0);
    __syncwarp();
    return;
  }
  if (v2 == T(0)) {  // cone reduces to the quadrant s, t >= 0
    __syncwarp();
    if (lane == 0) {
      x[nv] = T(fmax(zs, 0.0));
      x[nv + 1] = T(fmax(zt, 0.0));
    }
    __syncwarp();
    return;
  }
  const double sms = sqrt(ms), smt = sqrt(mt), q = sms * smt;
  const double kappa = sms * zs + smt * zt;
  const double kscale = sms * fabs(zs) + smt * fabs(zt);
  double s_out = 0.0, t_out = 0.0, xi = 0.5 * q;
  // sums of the element terms at xi (warp-wide, in T); every lane gets them
  auto sums = [&](double xx, T& sv, T& sv3) {
    const T tx = T(2.0 * xx);
    sv = T(0);
    sv3 = T(0);
    for (int i = lane; i < nv; i += 32) {
      const T mi = m[i], zi = x[i];
      const T a = (mi * zi) * (mi * zi);
      const T den = mi + tx;
      const T qq = a / (den * den);
      sv += qq;
      sv3 += qq / den;
    }
    sv = warp_sum(sv);
    sv3 = warp_sum(sv3);
  };
  // f and f' from the sums (lane 0)
  auto fval = [&](double xx, double sv, double sv3, double* df) {
    const double det = ms * mt - 4.0 * xx * xx;
    const double id = 1.0 / det;   // the only FP64 division of the iteration
    const double ns = ms * zs + 2.0 * xx * zt, nt = mt * zt + 2.0 * xx * zs;
    const double s = mt * ns * id, t = ms * nt * id;
    const double ds = mt * (2.0 * zt + 8.0 * xx * ns * id) * id;
    const double dt = ms * (2.0 * zs + 8.0 * xx * nt * id) * id;
    *df = -4.0 * sv3 - 2.0 * (ds * t + s * dt);
    return sv - 2.0 * s * t;
  };
  if (fabs(kappa) <= 64.0 * Tol<T>::rel * kscale) {
    T sv, sv3;
    sums(0.5 * q, sv, sv3);   // sum of v_i^2 at 2 xi = q
    const double delta = sms * zs;
    const double chi = sqrt(delta * delta + 2.0 * q * (double)sv);
    s_out = (delta + chi) / (2.0 * sms);
    t_out = (-delta + chi) / (2.0 * smt);
  } else {
    double lo, hi;
    const double al[2] = {ms * zs, mt * zt}, be[2] = {zt, zs};
    if (kappa > 0.0) {
      lo = 0.0;
      hi = 0.5 * q;
      for (int j = 0; j < 2; ++j)
        if (al[j] < 0.0) lo = fmax(lo, -al[j] / (2.0 * be[j]));
    } else {
      lo = 0.5 * q;
      hi = INFINITY;
      for (int j = 0; j < 2; ++j)
        if (be[j] > 0.0) hi = fmin(hi, -al[j] / (2.0 * be[j]));
    }
    double dfv;
    if (!isfinite(hi)) {
      // f xi^2 tends to (||M z_v||^2 - 2 m_s m_t z_s z_t)/4 > 0; when rounding hides that
      // margin the input lies within rounding of -K* and the projection is the origin
      hi = q;
      int it = 0, pos = 0;
      for (; it < 128; ++it) {
        T sv, sv3;
        sums(hi, sv, sv3);
        if (lane == 0) pos = fval(hi, (double)sv, (double)sv3, &dfv) > 0.0 ? 1 : 0;
        if (__shfl_sync(0xffffffffu, pos, 0)) break;
        hi *= 2.0;
      }
      if (it == 128) {
        for (int i = lane; i < d; i += 32) x[i] = T(0);
        __syncwarp();
        return;
      }
    }
    const bool lo_pos = kappa > 0.0;
    double xx = 0.5 * (lo + hi);
    if (guess) {
      const double g0 = (double)*guess;
      if (g0 > lo && g0 < hi) xx = g0;
    }
    for (int it = 0; it < 200; ++it) {
      T sv, sv3;
      sums(xx, sv, sv3);
      int done = 0;
      if (lane == 0) {
        const double f = fval(xx, (double)sv, (double)sv3, &dfv);
        // f = sv - 2 s t with sv a sum in T: within a few roundings of its terms f is noise
        const double noise = 8.0 * Unit<T>::u * ((double)sv + fabs((double)sv - f));
        if (f == 0.0 || fabs(f) <= noise) {
          done = 1;
        } else {
          if ((f > 0.0) == lo_pos) lo = xx; else hi = xx;
          double nx = (dfv != 0.0 && isfinite(dfv)) ? xx - f / dfv : 0.5 * (lo + hi);
          if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
          const double step = fabs(nx - xx);
          xx = nx;
          done = (step <= Tol<T>::rel * xx || (hi - lo) <= Tol<T>::rel * xx) ? 1 : 0;
        }
      }
      xx = bcast(xx);
      if (__shfl_sync(0xffffffffu, done, 0)) break;
    }
    xi = xx;
    if (guess && lane == 0) *guess = (float)xi;
    const double id = 1.0 / (ms * mt - 4.0 * xi * xi);
    s_out = fmax(mt * (ms * zs + 2.0 * xi * zt) * id, 0.0);
    t_out = fmax(ms * (mt * zt + 2.0 * xi * zs) * id, 0.0);
  }
  const T tx = T(2.0 * xi);
  for (int i = lane; i < nv; i += 32) {
    const T mi = m[i];
    x[i] = mi * x[i] / (mi + tx);
  }
  __syncwarp();
  if (lane == 0) {
    x[nv] = T(s_out);
    x[nv + 1] = T(t_out);
  }
  __syncwarp();
}

// --------------------------------------------------------------------------
// Exponential cone.  At the projection p = eta a(rho), a = (rho, 1, e^rho), and
// M(p - z) = mu c(rho) with c = (-1, rho - 1, e^-rho) (the dual-cone ray normal to
// K at p), eta, mu > 0; rho is a zero of
//   G(rho) = m_t e^rho (m_s s0 + m_r (rho-1) r0) + m_r m_s e^-rho (rho s0 - r0)
//            - m_t t0 (m_r rho (rho-1) + m_s)
// (z in span{a, M^{-1} c}) at which G crosses from negative to positive.  All
// scalar functions are evaluated times e^{-|rho|} (same sign, no overflow).
// --------------------------------------------------------------------------
struct ExpData {
  double r0, s0, t0, mr, ms, mt;
};

__device__ __forceinline__ double exp_G(const ExpData& c, double rho, double* dG) {
  // returns e^{-|rho|} G(rho); *dG receives e^{-|rho|} G'(rho)
  const double a = c.mt * (c.ms * c.s0 + c.mr * (rho - 1.0) * c.r0);
  const double da = c.mt * c.mr * c.r0;
  const double b = c.mr * c.ms * (rho * c.s0 - c.r0);
  const double db = c.mr * c.ms * c.s0;
  const double p = c.mt * c.t0 * (c.mr * rho * (rho - 1.0) + c.ms);
  const double dp = c.mt * c.t0 * c.mr * (2.0 * rho - 1.0);
  if (rho >= 0.0) {
    const double e1 = exp(-rho), e2 = e1 * e1;
    // G = e^rho a + e^-rho b - p; G' = e^rho (a + da) + e^-rho (db - b) - dp
    *dG = (a + da) + (db - b) * e2 - dp * e1;
    return a + b * e2 - p * e1;
  }
  const double e1 = exp(rho), e2 = e1 * e1;
  *dG = (a + da) * e2 + (db - b) - dp * e1;
  return a * e2 + b - p * e1;
}

__device__ __forceinline__ double exp_N(const ExpData& c, double rho) {  // eta_M numerator, scaled for rho > 0
  if (rho > 0.0) {
    const double e1 = exp(-rho);
    return (c.mr * rho * c.r0 + c.ms * c.s0) * e1 + c.mt * c.t0;
  }
  return c.mr * rho * c.r0 + c.ms * c.s0 + c.mt * exp(rho) * c.t0;
}
__device__ __forceinline__ double exp_g2(const ExpData& c, double rho) {  // > 0 iff mu > 0, scaled for rho < 0
  if (rho < 0.0) {
    const double e1 = exp(rho);
    return (c.r0 + (1.0 - rho) * c.s0) * e1 - c.t0;
  }
  return c.r0 + (1.0 - rho) * c.s0 - exp(-rho) * c.t0;
}

// safeguarded Newton on G over [lo, hi] with G(lo) < 0 < G(hi)
static __device__ __noinline__ double exp_root(const ExpData& c, double lo, double hi, double start) {
  double rho = (start > lo && start < hi) ? start : 0.5 * (lo + hi);
  for (int it = 0; it < 300; ++it) {
    double dG;
    const double G = exp_G(c, rho, &dG);
    if (G == 0.0) return rho;
    if (G < 0.0) lo = rho; else hi = rho;
    double nx = (dG != 0.0) ? rho - G / dG : 0.5 * (lo + hi);
    if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
    const double step = fabs(nx - rho);
    rho = nx;
    if (step <= 4e-16 * fmax(1.0, fabs(rho)) || (hi - lo) <= 4e-16 * fmax(1.0, fabs(rho))) break;
  }
  return rho;
}

static __device__ void exp_finish(const ExpData& c, double rho, double* out) {
  if (rho <= 0.0) {
    const double ep = exp(rho);
    const double eta = (c.mr * rho * c.r0 + c.ms * c.s0 + c.mt * ep * c.t0) / (c.mr * rho * rho + c.ms + c.mt * ep * ep);
    out[0] = eta * rho;
    out[1] = eta;
    out[2] = eta * ep;
  } else {
    const double em = exp(-rho);
    const double te = (c.mr * rho * c.r0 * em + c.ms * c.s0 * em + c.mt * c.t0) /
                      (c.mr * rho * rho * em * em + c.ms * em * em + c.mt);   // eta e^rho
    out[0] = te * rho * em;
    out[1] = te * em;
    out[2] = te;
  }
}

// returns true if one of the closed-form cases applied (App. A.4)
static __device__ bool exp_trivial(const ExpData& c, double* out) {
  const double r0 = c.r0, s0 = c.s0, t0 = c.t0;
  if ((s0 > 0.0 && r0 <= s0 * log(fmax(t0, 0.0) / s0)) || (r0 <= 0.0 && s0 == 0.0 && t0 >= 0.0)) {
    out[0] = r0; out[1] = s0; out[2] = t0;       // z in K
    return true;
  }
  const double u = -c.mr * r0, v = -c.ms * s0, w = -c.mt * t0;   // -Mz in K*?
  if ((u < 0.0 && w > 0.0 && log(-u) + v / u <= 1.0 + log(w)) || (u == 0.0 && v >= 0.0 && w >= 0.0)) {
    out[0] = out[1] = out[2] = 0.0;
    return true;
  }
  if (r0 <= 0.0 && s0 <= 0.0) {                  // face {s = 0}
    out[0] = r0; out[1] = 0.0; out[2] = fmax(t0, 0.0);
    return true;
  }
  return false;
}

// Euclidean exponential-cone projection.  With M = I the first two components
// of z = eta a + mu b (b = -c) give eta = (s0 + (rho-1) r0)/(rho^2-rho+1) and
// mu = (r0 - rho s0)/(rho^2-rho+1), so {eta > 0, mu > 0} is an interval cut out
// by two linear inequalities in rho, with G < 0 at its left end and G > 0 at
// its right end.
static __device__ __noinline__ void exp_proj_euclid(double r0, double s0, double t0, double* out,
                                                    float* guess = nullptr) {
  const ExpData c{r0, s0, t0, 1.0, 1.0, 1.0};
  if (exp_trivial(c, out)) return;
  double lo = -INFINITY, hi = INFINITY;
  if (r0 > 0.0) lo = fmax(lo, 1.0 - s0 / r0);
  if (r0 < 0.0) hi = fmin(hi, 1.0 - s0 / r0);
  if (s0 > 0.0) hi = fmin(hi, r0 / s0);
  if (s0 < 0.0) lo = fmax(lo, r0 / s0);
  double dG;
  // a warm start inside the admissible interval tightens one end of the bracket
  double g0 = guess ? (double)*guess : NAN;
  if (isfinite(g0) && g0 > lo && g0 < hi) {
    if (exp_G(c, g0, &dG) < 0.0) lo = g0; else hi = g0;
  } else {
    g0 = NAN;
  }
  if (!isfinite(lo)) {
    double step = 1.0;
    lo = hi - step;
    while (exp_G(c, lo, &dG) >= 0.0 && step < 1e8) { step *= 2.0; lo = hi - step; }
  }
  if (!isfinite(hi)) {
    double step = 1.0;
    hi = lo + step;
    while (exp_G(c, hi, &dG) <= 0.0 && step < 1e8) { step *= 2.0; hi = lo + step; }
  }
  const double rho = exp_root(c, lo, hi, g0);
  if (guess) *guess = (float)rho;
  exp_finish(c, rho, out);
}

// zeros of a function that is convex or concave with stationary point rc (NaN:
// monotone), located by outward doubling from the anchor and bisection
template <typename F>
static __device__ int exp_piece_roots(F f, double rc, double* roots) {
  int nr = 0;
  const double a = isnan(rc) ? 0.0 : rc;
  const double fa = f(a);
  if (fa == 0.0) { roots[nr++] = a; return nr; }
  for (int dir = -1; dir <= 1; dir += 2) {
    for (double step = 1.0; step < 1e8; step *= 2.0) {
      const double xx = a + dir * step;
      const double fx = f(xx);
      if ((fx > 0.0) != (fa > 0.0)) {
        double lo = dir < 0 ? xx : a, hi = dir < 0 ? a : xx;
        const bool lo_pos = (dir < 0 ? fx : fa) > 0.0;
        for (int it = 0; it < 200; ++it) {
          const double mid = 0.5 * (lo + hi);
          if (mid <= lo || mid >= hi) break;
          if ((f(mid) > 0.0) == lo_pos) lo = mid; else hi = mid;
        }
        roots[nr++] = 0.5 * (lo + hi);
        break;
      }
    }
  }
  return nr;
}

// Exponential-cone projection in the metric M (App. A.4, eq. exp-metric-projection).
// The admissible zero of G has N > 0 (eta_M > 0) and g2 > 0 (mu > 0).  N and g2
// are each convex or concave in rho, so {N > 0, g2 > 0} is a union of a few
// intervals bounded by their zeros; on each interval G has no zero but the
// admissible one, an up-crossing.  The intervals are enumerated and the one
// with a sign change of G is solved by the safeguarded Newton iteration.
static __device__ __noinline__ void exp_proj_metric(double r0, double s0, double t0, double mr, double ms, double mt, double* out) {
  const ExpData c{r0, s0, t0, mr, ms, mt};
  if (exp_trivial(c, out)) return;
  double br[4];
  int nb = 0;
  double rc = NAN;
  if (t0 != 0.0 && -mr * r0 / (mt * t0) > 0.0) rc = log(-mr * r0 / (mt * t0));
  nb += exp_piece_roots([&](double x) { return exp_N(c, x); }, rc, br + nb);
  rc = NAN;
  if (s0 != 0.0 && t0 / s0 > 0.0) rc = log(t0 / s0);
  nb += exp_piece_roots([&](double x) { return exp_g2(c, x); }, rc, br + nb);
  for (int i = 1; i < nb; ++i)
    for (int j = i; j > 0 && br[j] < br[j - 1]; --j) { const double tmp = br[j]; br[j] = br[j - 1]; br[j - 1] = tmp; }
  double rho = NAN, dG;
  for (int iv = 0; iv <= nb && isnan(rho); ++iv) {
    const double a = iv == 0 ? -INFINITY : br[iv - 1];
    const double b = iv == nb ? INFINITY : br[iv];
    if (!(b > a)) continue;
    double p;
    if (isfinite(a) && isfinite(b)) p = 0.5 * (a + b);
    else if (isfinite(a)) p = a + 1.0;
    else if (isfinite(b)) p = b - 1.0;
    else p = 0.0;
    if (!(exp_N(c, p) > 0.0 && exp_g2(c, p) > 0.0)) continue;
    const double gp = exp_G(c, p, &dG);
    if (gp == 0.0) { rho = p; break; }
    double lo = NAN, hi = NAN;
    if (gp < 0.0) {
      lo = p;
      if (isfinite(b)) { if (exp_G(c, b, &dG) > 0.0) hi = b; }
      else for (double st = 1.0; st < 1e8; st *= 2.0) if (exp_G(c, p + st, &dG) > 0.0) { hi = p + st; break; }
    } else {
      hi = p;
      if (isfinite(a)) { if (exp_G(c, a, &dG) < 0.0) lo = a; }
      else for (double st = 1.0; st < 1e8; st *= 2.0) if (exp_G(c, p - st, &dG) < 0.0) { lo = p - st; break; }
    }
    if (!isnan(lo) && !isnan(hi)) rho = exp_root(c, lo, hi, NAN);
  }
  if (isnan(rho)) {          // not expected: fall back to the Euclidean direction
    double e[3];
    exp_proj_euclid(r0, s0, t0, e);
    rho = e[1] > 0.0 ? log(fmax(e[2] / e[1], 1e-300)) : 0.0;
  }
  exp_finish(c, rho, out);
}

// --------------------------------------------------------------------------
// Three-dimensional power cone (App. A.5, eqs. power-projection-root,
// power-cone-stable-quadratic-root, Prop. power-cone-bisection): the unique
// zero of g(rho) = a log x(rho) + (1-a) log y(rho) - log rho in (0, R), R = |z_t|,
// with g > 0 near 0 and g < 0 near R, found by Newton steps kept inside the
// bisection bracket.
// --------------------------------------------------------------------------
__device__ __forceinline__ double pow_qroot(double s, double c) {
  const double d = sqrt(s * s + 4.0 * c);
  return s >= 0.0 ? 0.5 * (s + d) : 2.0 * c / (d - s);
}

static __device__ __noinline__ void pow_proj(double rx, double ry, double rz, double al, double mx, double my, double mz,
                                            double* out, float* guess = nullptr) {
  auto geo = [&](double xx, double yy) { return (xx <= 0.0 || yy <= 0.0) ? 0.0 : exp(al * log(xx) + (1.0 - al) * log(yy)); };
  if (rx >= 0.0 && ry >= 0.0 && geo(rx, ry) >= fabs(rz)) { out[0] = rx; out[1] = ry; out[2] = rz; return; }
  {
    const double p = -mx * rx, q = -my * ry, w = -mz * rz;
    if (p >= 0.0 && q >= 0.0 && geo(p / al, q / (1.0 - al)) >= fabs(w)) { out[0] = out[1] = out[2] = 0.0; return; }
  }
  if (rz == 0.0) { out[0] = fmax(rx, 0.0); out[1] = fmax(ry, 0.0); out[2] = 0.0; return; }
  const double R = fabs(rz), kx = al * mz / mx, ky = (1.0 - al) * mz / my;
  double lo = 0.0, hi = R, rho = 0.5 * R;
  if (guess && *guess > 0.0f && *guess < 1.0f) rho = (double)*guess * R;   // warm start: previous rho/R
  for (int it = 0; it < 300; ++it) {
    const double w = rho * (R - rho), dw = R - 2.0 * rho;
    const double cx = kx * w, cy = ky * w;
    const double dx = sqrt(rx * rx + 4.0 * cx), dy = sqrt(ry * ry + 4.0 * cy);
    const double xx = rx >= 0.0 ? 0.5 * (rx + dx) : 2.0 * cx / (dx - rx);
    const double yy = ry >= 0.0 ? 0.5 * (ry + dy) : 2.0 * cy / (dy - ry);
    const double g = al * log(xx) + (1.0 - al) * log(yy) - log(rho);
    if (g == 0.0) break;
    if (g > 0.0) lo = rho; else hi = rho;
    // d/drho of the positive root u of u^2 - s u - c: du = dc / (2u - s) = dc / sqrt(s^2 + 4c)
    const double gx = kx * dw / dx, gy = ky * dw / dy;
    const double dg = al * gx / xx + (1.0 - al) * gy / yy - 1.0 / rho;
    double nx = (dg != 0.0 && isfinite(dg)) ? rho - g / dg : 0.5 * (lo + hi);
    if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
    const double step = fabs(nx - rho);
    rho = nx;
    if (step <= 4e-16 * fmax(rho, 1e-300) || (hi - lo) <= 4e-16 * fmax(1.0, R)) break;
  }
  if (guess) *guess = (float)(rho / R);
  const double w = rho * (R - rho);
  out[0] = pow_qroot(rx, kx * w);
  out[1] = pow_qroot(ry, ky * w);
  out[2] = rz > 0.0 ? rho : -rho;
}

// --------------------------------------------------------------------------
// Slices with the middle coordinate fixed (Sec. 5.4, eq. fisher-conic: each buyer's
// (z, 1, t) block of the Fisher model stores the one and has no row for it):
//   exponential X_f = {(r, f, t): f e^{r/f} <= t},
//   power       X_f = {(x, f, z): x^a f^{1-a} >= |z|, x >= 0},   f > 0 fixed.
// X_f = f X_1, and a projection in a diagonal metric commutes with the positive scalar
// f, so the outer pair is divided by f, projected onto the 2-D set X_1 and scaled back.
// Outside X_1 the projection is the zero of a monotone scalar function obtained from
// the normal-cone condition M (z - u) = lambda * (outward normal); it is found in FP64
// by Newton steps kept inside a sign-change bracket.  `guess` (optional) holds the
// previous root of the block (exp: a, pow: x / |z|^{1/a}) and is updated.
// --------------------------------------------------------------------------

// Newton steps on a monotone function inside a sign-change bracket [lo, hi], with a
// bisection step whenever two Newton steps have not halved the bracket (so far starts and
// flat or steep stretches cannot stall it).  f(x, &df) returns the value and derivative;
// up_at_lo: the function is negative at lo (increasing) or positive at lo (decreasing).
// rtol: stop once a step or the bracket is below rtol max(1, |x|).  f(x, &d, &sc) also returns
// the size sc of the terms it sums: once |f| <= 8 u sc (u the unit roundoff of R) the value is
// rounding noise and further steps cannot improve x, so the iteration stops there too.
template <typename R, typename F>
static __device__ R bracketed_newton(F f, R lo, R hi, R x, bool neg_at_lo, R rtol) {
  const R u = sizeof(R) == 4 ? R(5.9604645e-08) : R(1.1102230246251565e-16);
  if (!(x > lo && x < hi)) x = R(0.5) * (lo + hi);
  R w_old = hi - lo, step_old = hi - lo;
  for (int it = 0; it < 200; ++it) {
    R d, sc;
    const R v = f(x, &d, &sc);
    if (v == R(0) || fabs(v) <= R(8) * u * sc) break;
    if ((v < R(0)) == neg_at_lo) lo = x; else hi = x;
    R nx = (d != R(0) && isfinite(d)) ? x - v / d : R(0.5) * (lo + hi);
    if (!(nx > lo && nx < hi)) nx = R(0.5) * (lo + hi);
    // bisect when two steps have not halved the bracket and Newton is not converging fast
    if ((it & 1) == 1) {
      if (hi - lo > R(0.5) * w_old && fabs(nx - x) > R(0.25) * step_old) nx = R(0.5) * (lo + hi);
      w_old = hi - lo;
    }
    const R step = fabs(nx - x);
    step_old = step;
    x = nx;
    if (step <= rtol * fmax(R(1), fabs(x)) || (hi - lo) <= rtol * fmax(R(1), fabs(x))) break;
  }
  return x;
}

// exp: u = (a, 1, e^a) with phi(a) = m_r (a0 - a) - m_t (e^a - c0) e^a = 0; phi is
// decreasing where e^a >= c0.  Bracket: lo = log c0 for c0 > 0 (phi = m_r (a0 - log c0) > 0
// there), else the first of min(a0, 0) - 2^k with phi >= 0 (phi grows without bound as
// a -> -inf); hi = min(a0, log(S + max(c0, 0))) with S = sqrt((m_r/m_t)(a0 - lo)), where
// e^a (e^a - c0) >= S^2 >= (m_r/m_t)(a0 - a) makes phi <= 0.
static __device__ __noinline__ void exp_slice_proj(double r0, double t0, double f, double mr, double mt, double* out,
                                                  float* guess = nullptr) {
  const double a0 = r0 / f, c0 = t0 / f;
  out[1] = f;
  if (exp(a0) <= c0) { out[0] = r0; out[2] = t0; return; }
  auto phi = [&](double a, double* dphi, double* sc) {
    const double ea = exp(a);
    *dphi = -mr - mt * ea * (2.0 * ea - c0);
    *sc = mr * (fabs(a0) + fabs(a)) + mt * ea * (ea + fabs(c0));
    return mr * (a0 - a) - mt * (ea - c0) * ea;
  };
  double d, sc, lo;
  if (c0 > 0.0) {
    lo = log(c0);
  } else {
    const double top = fmin(a0, 0.0);
    double step = 1.0;
    lo = top - step;
    while (phi(lo, &d, &sc) < 0.0 && step < 1e300) { step *= 2.0; lo = top - step; }
  }
  double hi = fmin(a0, log(sqrt((mr / mt) * (a0 - lo)) + fmax(c0, 0.0)));
  if (!(hi > lo)) hi = a0;
  const double g0 = guess ? (double)*guess : NAN;
  double start = (isfinite(g0) && g0 > lo && g0 < hi) ? g0 : hi;
  // the bulk of the iteration in FP32 (GB300's FP64 rate is a small fraction of its FP32
  // rate), then FP64 Newton steps from its result inside the FP64 bracket
  if (fabs(lo) < 60.0 && fabs(hi) < 60.0 && fabs(a0) < 1e6 && fabs(c0) < 1e30) {
    const float a0f = (float)a0, c0f = (float)c0, mrf = (float)mr, mtf = (float)mt;
    auto phif = [&](float a, float* dphi, float* scf) {
      const float ea = expf(a);
      *dphi = -mrf - mtf * ea * (2.0f * ea - c0f);
      *scf = mrf * (fabsf(a0f) + fabsf(a)) + mtf * ea * (ea + fabsf(c0f));
      return mrf * (a0f - a) - mtf * (ea - c0f) * ea;
    };
    const float af = bracketed_newton<float>(phif, (float)lo, (float)hi, (float)start, false, 2e-6f);
    if (isfinite(af) && (double)af > lo && (double)af < hi) start = (double)af;
  }
  const double a = bracketed_newton<double>(phi, lo, hi, start, false, 4e-16);
  if (guess) *guess = (float)a;
  out[0] = f * a;
  out[2] = f * exp(a);
}

// pow: u = (x, 1, sign(c0) x^a) with psi(x) = m_x (x - x0) - m_z (Z - x^a) a x^{a-1} = 0,
// Z = |c0|; psi is increasing on (max(x0, 0), Z^{1/a}), negative at its left end (or
// tending to -inf at 0+) and positive at its right end.  Since Z - x^a <= Z at the root,
// x^{1-a} (x - x0) <= (m_z/m_x) a Z there, which bounds it by ((m_z/m_x) a Z)^{1/(2-a)} for
// x0 <= 0 and by x0 + (m_z/m_x) a Z x0^{a-1} for x0 > 0.
static __device__ __noinline__ void pow_slice_proj(double rx, double rz, double al, double f, double mx, double mz,
                                                  double* out, float* guess = nullptr) {
  const double x0 = rx / f, c0 = rz / f;
  out[1] = f;
  const double Z = fabs(c0);
  if (x0 >= 0.0 && (Z == 0.0 || (x0 > 0.0 && al * log(x0) >= log(Z)))) { out[0] = rx; out[2] = rz; return; }
  if (Z == 0.0) { out[0] = f * fmax(x0, 0.0); out[2] = 0.0; return; }
  const double lo = fmax(x0, 0.0);
  const double k = (mz / mx) * al * Z;
  double hi = exp(log(Z) / al);
  const double hb = x0 > 0.0 ? x0 + k * exp((al - 1.0) * log(x0)) : exp(log(k) / (2.0 - al));
  if (hb > lo && hb < hi) hi = hb;
  auto psi = [&](double x, double* dpsi, double* sc) {
    const double lx = log(x);
    const double xa = exp(al * lx), xam1 = exp((al - 1.0) * lx);
    *dpsi = mx + mz * al * ((1.0 - al) * Z * xam1 / x + (2.0 * al - 1.0) * xam1 * xam1);
    *sc = mx * (fabs(x) + fabs(x0)) + mz * (Z + xa) * al * xam1;
    return mx * (x - x0) - mz * (Z - xa) * al * xam1;
  };
  const double g0 = guess ? (double)*guess : NAN;
  double start = (isfinite(g0) && g0 > 0.0 && g0 * hi > lo && g0 < 1.0) ? g0 * hi : 0.5 * (lo + hi);
  // FP32 bulk, FP64 finish (as for the exponential slice)
  if (hi < 1e30 && fabs(x0) < 1e30 && Z < 1e30 && lo < 1e30) {
    const float x0f = (float)x0, Zf = (float)Z, alf = (float)al, mxf = (float)mx, mzf = (float)mz;
    auto psif = [&](float x, float* dpsi, float* scf) {
      const float lx = logf(x);
      const float xa = expf(alf * lx), xam1 = expf((alf - 1.0f) * lx);
      *dpsi = mxf + mzf * alf * ((1.0f - alf) * Zf * xam1 / x + (2.0f * alf - 1.0f) * xam1 * xam1);
      *scf = mxf * (fabsf(x) + fabsf(x0f)) + mzf * (Zf + xa) * alf * xam1;
      return mxf * (x - x0f) - mzf * (Zf - xa) * alf * xam1;
    };
    const float xf = bracketed_newton<float>(psif, (float)lo, (float)hi, (float)start, true, 2e-6f);
    if (isfinite(xf) && (double)xf > lo && (double)xf < hi) start = (double)xf;
  }
  const double x = bracketed_newton<double>(psi, lo, hi, start, true, 4e-16);
  if (guess) *guess = (float)(x / hi);
  out[0] = f * x;
  out[2] = (c0 > 0.0 ? f : -f) * exp(al * log(x));
}

// Dual side of a slice block (unscaled, f = 1): the dual objective of the KKT report
// gains inf_{x in X_1} sl'x, finite only when the slack sl lies in a closed cone D
// (exp: sl_0 <= 0 <= sl_2, pow: sl_0 >= 0); res receives sl - Pi_D(sl), which counts as
// dual residual, and the term is taken at Pi_D(sl):
//   exp: sl_1 + sl_0 (log(-sl_0 / sl_2) - 1) (minimiser e^r = -sl_0 / sl_2), sl_1 at
//        sl_0 = 0, -inf at sl_0 < 0 = sl_2;
//   pow: sl_1 - (1-a)/a sl_0 x* with x* = (a |sl_2| / sl_0)^{1/(1-a)}, sl_1 at sl_2 = 0,
//        -inf at sl_0 = 0 != sl_2.
static __device__ double slice_support(bool is_pow, double al, const double* sl, double* res) {
  res[0] = res[1] = res[2] = 0.0;
  if (!is_pow) {
    double a = sl[0], c = sl[2];
    if (a > 0.0) { res[0] = a; a = 0.0; }
    if (c < 0.0) { res[2] = c; c = 0.0; }
    if (a == 0.0) return sl[1];
    if (c == 0.0) return -INFINITY;
    return sl[1] + a * (log(-a / c) - 1.0);
  }
  double p = sl[0];
  const double w = fabs(sl[2]);
  if (p < 0.0) { res[0] = p; p = 0.0; }
  if (w == 0.0) return sl[1];
  if (p == 0.0) return -INFINITY;
  const double xs = exp(log(al * w / p) / (1.0 - al));
  return sl[1] - (1.0 - al) / al * p * xs;
}

}  // namespace cqp
