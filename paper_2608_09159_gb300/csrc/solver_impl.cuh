// Bodies of the Solver phases declared in solver.cuh.
#pragma once

#include "solver.cuh"

namespace cqp {

// rows [r0, r1) with groups of G lanes computing two row products at once
template <int G, typename Acc, typename T, typename X1, typename X2, typename F>
__device__ __forceinline__ void rows_loop2(const int* rp, const int* ci, const T* v, int64_t r0, int64_t r1, X1 x1,
                                           X2 x2, F f) {
  const int lane = threadIdx.x & 31, gl = lane & (G - 1);
  const int64_t per_warp = 32 / G, nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5;
  for (int64_t base = warp * per_warp; base < r1 - r0; base += nwarps * per_warp) {
    const int64_t r = r0 + base + lane / G;
    const bool ok = r < r1;
    Acc s1 = Acc(0), s2 = Acc(0);
    if (ok) {
      const int beg = rp[r], end = rp[r + 1];
      constexpr int U = RowBatch<G>::value;
      for (int k = beg + gl; k < end; k += U * G) {
        int j[U];
        Acc a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int kk = k + u * G;
          const bool okk = kk < end;
          j[u] = okk ? __ldg(ci + kk) : -1;
          a[u] = okk ? ld_val<Acc>(v + kk) : Acc(0);
        }
        Acc g1[U], g2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          g1[u] = j[u] >= 0 ? (Acc)x1(j[u]) : Acc(0);
          g2[u] = j[u] >= 0 ? (Acc)x2(j[u]) : Acc(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          s1 += a[u] * g1[u];
          s2 += a[u] * g2[u];
        }
      }
    }
    s1 = group_sum<G>(s1);
    s2 = group_sum<G>(s2);
    if (ok) f(r, gl, s1, s2);
  }
}

template <typename Acc, typename T, typename X1, typename X2, typename F>
__device__ __forceinline__ void rows_loop2_tpr(int tpr, const int* rp, const int* ci, const T* v, int64_t r0, int64_t r1,
                                               X1 x1, X2 x2, F f) {
  switch (tpr) {
    case kRowsBatched:
    case 1: rows_loop2<1, Acc>(rp, ci, v, r0, r1, x1, x2, f); break;
    case 2: rows_loop2<2, Acc>(rp, ci, v, r0, r1, x1, x2, f); break;
    case 4: rows_loop2<4, Acc>(rp, ci, v, r0, r1, x1, x2, f); break;
    case 8: rows_loop2<8, Acc>(rp, ci, v, r0, r1, x1, x2, f); break;
    case 16: rows_loop2<16, Acc>(rp, ci, v, r0, r1, x1, x2, f); break;
    default: rows_loop2<32, Acc>(rp, ci, v, r0, r1, x1, x2, f); break;
  }
}

// w = D~ t (k entries), threads l < k; wf (optional) receives an FP32 copy
template <typename T>
__device__ __forceinline__ void apply_D(const Prob<T>& P, const double* t, double* w, float* wf = nullptr) {
  __syncthreads();
  for (int l = threadIdx.x; l < P.k; l += blockDim.x) {
    double s = 0.0;
    if (P.d_scale > 0.0) {
      s = P.d_scale * t[l];
    } else {
      for (int l2 = 0; l2 < P.k; ++l2) s += P.D[l * P.k + l2] * t[l2];
    }
    w[l] = s;
    if (wf) wf[l] = (float)s;
  }
  for (int l = P.k + threadIdx.x; l < P.kpad; l += blockDim.x) {   // zero padding read by the inner step
    w[l] = 0.0;
    if (wf) wf[l] = 0.0f;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// prox for diagonal Q: one metric projection (eqs. diagonal-q-metric,
// diagonal-q-metric-projection, M_sc = I): u = Pi^M((v - tau c)/(1 + tau q)),
// M = I + tau diag(q).  Result in W.u[0].
// ---------------------------------------------------------------------------
template <typename T, class Team, bool GEN>
__device__ bool Solver<T, Team, GEN>::prox_diag(const T* hx) {
  using S = Solver<T, Team, GEN>;
  const double tau = C.s.tau;
  if (!phase_aty(hx, W.hy[C.s.hb], tau)) return false;
  tick(0);
  T* u = W.u[0];
  const T tt = T(tau);
  for (int seg = 0; seg < 6; ++seg)
    for (int64_t i = own.x0[seg] + threadIdx.x; i < own.x1[seg]; i += blockDim.x) {
      const T z = (W.v[i] - tt * P.c[i]) / (T(1) + tt * P.qd[i]);
      u[i] = seg < 2 ? proj_elem(i, z) : z;
    }
  __syncthreads();
  project_owned_cones(u, P.euclid_cones ? S::kEuclid : S::kDiagQ, tau);
  if (threadIdx.x == 0) C.inner_j = 1;
  tick(1);
  const bool ok = team.sync();
  tick(2);
  return ok;
}

// ---------------------------------------------------------------------------
// prox for general Q: Jacobi projected BB from u^0 = h_x (warm start), first
// step alpha = 1, stop when ||u^{j+1} - u^j||_2 <= eps_in or max_inner steps.
// Returns the buffer index of the final iterate in ub.
// ---------------------------------------------------------------------------
template <typename T, class Team, bool GEN>
__device__ bool Solver<T, Team, GEN>::prox_bb(const T* hx, int& ub) {
  const double tau = C.s.tau;
  const int k = P.k;
  const bool sparse = P.qmode == kQSparse;
  if (!phase_aty(hx, W.hy[C.s.hb], tau)) return false;
  tick(0);
  // t = R h_x from the state; w = D t
  for (int l = threadIdx.x; l < k; l += blockDim.x) C.tcur[l] = C.s.t_h[l];
  apply_D(P, C.tcur, C.w, C.wf);
  T v3[4];
  int gb = 0;
  // ||u^{j+1} - u^j|| cannot fall below the rounding level of u: the stop test compares it
  // with max(eps_in, 4 eps_T ||u||) (precision floor; eps_T = 2^-24 or 2^-53)
  const double eps_T = sizeof(T) == 4 ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
  if (sparse) {
    double v2[2];
    grad_pass(hx, nullptr, nullptr, W.g[0], tau, v2, true);
    inner_step(hx, W.u[0], W.g[0], 1.0, tau, v3);
  } else {
    inner_step(hx, W.u[0], nullptr, 1.0, tau, v3);
  }
  publish_t<4>(v3, 0, k > 0);
  if (!sync_gather(4 + k, 1, 2)) return false;
  int cur = 0;
  long long j = 1;
  const T* uprev = hx;
  for (;;) {
    const double du = sqrt(fmax(C.red[0], 0.0));
    const double floor_u = 4.0 * eps_T * sqrt(fmax(C.red[3], 0.0));
    if (!(du > fmax(C.s.eps_in, floor_u)) || j >= O.max_inner) break;
    if (!isfinite(du)) break;
    const double sJs = O.jacobi ? C.red[1] : C.red[0];
    double sdg;
    __syncthreads();
    if (threadIdx.x == 0) C.sJs = sJs;
    // t_{j} = R u^{j} from the reduction; dt = t_j - t_{j-1}
    if (!sparse) {
      // <s, dg> = sum (qd + 1/tau) s^2 + (R s)' D (R s), R s = t_new - t_old (warp 0)
      if (threadIdx.x < 32) {
        double part = 0.0;
        for (int l = threadIdx.x; l < k; l += 32) {
          const double dl = C.red[4 + l] - C.tcur[l];
          double ddl;
          if (P.d_scale > 0.0) {
            ddl = P.d_scale * dl;
          } else {
            ddl = 0.0;
            for (int l2 = 0; l2 < k; ++l2) ddl += P.D[l * k + l2] * (C.red[4 + l2] - C.tcur[l2]);
          }
          part += dl * ddl;
        }
        part = warp_sum(part);
        if (threadIdx.x == 0) C.alpha = C.red[2] + part;
      }
      __syncthreads();
      sdg = C.alpha;
      for (int l = threadIdx.x; l < k; l += blockDim.x) C.tcur[l] = C.red[4 + l];
      apply_D(P, C.tcur, C.w, C.wf);
    } else {
      for (int l = threadIdx.x; l < k; l += blockDim.x) C.tcur[l] = C.red[4 + l];
      apply_D(P, C.tcur, C.w, C.wf);
      double v2[2];
      grad_pass(W.u[cur], uprev, W.g[gb], W.g[gb ^ 1], tau, v2, false);
      publish<2>(v2, 0, false);
      if (!sync_gather(2, 1, 2)) return false;
      sdg = C.red[0];
      gb ^= 1;
    }
    // Barzilai-Borwein step (eqs. bb-step / jacobi-bb-step); readings: keep the previous
    // alpha when <s, dg> <= 1e-30, clip to [1e-10, 1e10]
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = C.alpha;
      if (j == 1) a = 1.0;
      if (sdg > 1e-30) a = C.sJs / sdg;
      a = fmin(fmax(a, 1e-10), 1e10);
      C.alpha = a;
    }
    __syncthreads();
    const double alpha = C.alpha;
    inner_step(W.u[cur], W.u[cur ^ 1], sparse ? W.g[gb] : nullptr, alpha, tau, v3);
    publish_t<4>(v3, 0, k > 0);
    if (!sync_gather(4 + k, 1, 2)) return false;
    uprev = W.u[cur];
    cur ^= 1;
    ++j;
  }
  // R u_final for later use (restart to the candidate, KKT)
  __syncthreads();
  for (int l = threadIdx.x; l < k; l += blockDim.x) C.tcur[l] = C.red[4 + l];
  if (threadIdx.x == 0) C.inner_j = j;
  __syncthreads();
  ub = cur;
  return true;
}

// ---------------------------------------------------------------------------
// FP64 KKT report of the scaled point (x, y), measured on the unscaled problem
// (reading of the "relative KKT" of Sec. 4.2.2: eps_p = ||Ax-b||/(1+||b||),
// eps_d = ||Pi_K(-s)||/(1+||c||), s = Qx + c - A'y, eps_g = |p-d|/(1+|p|+|d|)).
// have_rx: C.tcur already holds R~ x.
// ---------------------------------------------------------------------------
template <typename T, class Team, bool GEN>
__device__ bool Solver<T, Team, GEN>::kkt(const T* x, const T* y, bool have_rx) {
  const int k = P.k;
  const bool sparse = P.qmode == kQSparse;
  __shared__ double tk[kMaxRank], wk[kMaxRank];
  // K1: rows (primal residual, b'y) and x-part (c'x, sum qd x^2, R x).  General form:
  // distance of Ax to [lo, hi], the dual objective term min_{z in [lo,hi]} y'z, and the
  // dual-sign residual of rows with an infinite side (added to the dual residual in K2)
  double v4[4] = {0.0, 0.0, 0.0, 0.0};
  double rd_rows = 0.0;
  vals(P.a_v, P.a_vb, [&](auto av) {
    rows_loop_tpr_plain<double>(own.g_a, P.a_rp, P.a_ci, av, own.row0, own.row1, [&](int j) { return x[j]; },
                          [&](int64_t r, int gl, double ax) {
                            if (gl == 0) {
                              if (GEN && P.rhi) {
                                const double lo = (double)P.b[r], hi = (double)P.rhi[r];
                                const double res = P.beta_b * P.row[r] * (ax - fmin(fmax(ax, lo), hi));
                                v4[0] += res * res;
                                const double yr = (double)y[r];
                                if (lo == hi) {
                                  v4[1] += lo * yr;
                                } else if (yr != 0.0) {
                                  const double bd = yr > 0.0 ? lo : hi;
                                  if (isfinite(bd)) v4[1] += bd * yr;
                                  else { const double yu = P.beta_c * yr / P.row[r]; rd_rows += yu * yu; }
                                }
                              } else {
                                const double res = P.beta_b * P.row[r] * (ax - (double)P.b[r]);
                                v4[0] += res * res;
                                v4[1] += (double)P.b[r] * (double)y[r];
                              }
                            }
                          });
  });
  const bool need_r = k > 0 && !have_rx;
  const int lane = threadIdx.x & 31;
  for (int seg = 0; seg < 6; ++seg) {
    const int64_t a = own.x0[seg], b = own.x1[seg];
    for (int64_t base = a + (threadIdx.x - lane); base < b; base += blockDim.x) {
      const int64_t i = base + lane;
      const bool ok = i < b;
      T xi = T(0);
      if (ok) {
        xi = x[i];
        v4[2] += (double)P.c[i] * (double)xi;
        v4[3] += (double)P.qd[i] * (double)xi * (double)xi;
      }
    }
  }
  if (need_r) rx_lmajor(x);
  double v5[5] = {v4[0], v4[1], v4[2], v4[3], 0.0};
  if (sparse) {
    // (P~ x)_i on the owned coordinates, kept in W.sd until K2 reads it
    for (int seg = 0; seg < 6; ++seg)
      vals(P.p_v, P.p_vb, [&](auto pv) {
        rows_loop_tpr_plain<double>(own.g_p, P.p_rp, P.p_ci, pv, own.x0[seg], own.x1[seg], [&](int j) { return x[j]; },
                              [&](int64_t i, int gl, double px) {
                                if (gl == 0) {
                                  W.sd[i] = px;
                                  v5[4] += (double)x[i] * px;
                                }
                              });
      });
  }
  __syncthreads();
  publish<5>(v5, 0, need_r);
  if (!sync_gather(5 + (need_r ? k : 0))) return false;
  const double rp2 = C.red[0], by = C.red[1], cx = C.red[2], xqdx = C.red[3], xpx = C.red[4];
  for (int l = threadIdx.x; l < k; l += blockDim.x) tk[l] = need_r ? C.red[5 + l] : C.tcur[l];
  apply_D(P, tk, wk);
  // K2: s~ = Q~x + c~ - A~'y on the owned coordinates, unscaled s = beta_c col s~,
  // ||Pi_K(-s)||^2 (free: K* = {0}; nonneg: max(-s, 0); cones below)
  // dual residual^2, box term of the dual objective (scaled), slice term (unscaled)
  double v2[3] = {rd_rows, 0.0, 0.0};
  for (int seg = 0; seg < 6; ++seg) {
    vals(P.t_v, P.t_vb, [&](auto tv) {
      rows_loop_tpr_plain<double>(
          own.g_t, P.t_rp, P.t_ci, tv, own.x0[seg], own.x1[seg], [&](int j) { return y[j]; },
          [&](int64_t i, int gl, double aty) {
            if (gl == 0) {
              double qx = (double)P.qd[i] * (double)x[i];
              if (k > 0) qx += rtw_d(i, wk);
              if (sparse) qx += W.sd[i];
              const double st = qx + (double)P.c[i] - aty;
              const double ss = P.beta_c * P.col[i] * st;
              if (seg == 0 && GEN && P.xlo) {
                // box coordinate: min_{x in [lo,hi]} s x joins the dual objective; an infinite
                // side demands the matching sign of s
                if (st != 0.0) {
                  const double bd = st > 0.0 ? (double)P.xlo[i] : (double)P.xhi[i];
                  if (isfinite(bd)) v2[1] += st * bd;
                  else v2[0] += ss * ss;
                }
              } else if (seg == 0) v2[0] += ss * ss;
              else if (seg == 1) { const double t = fmax(-ss, 0.0); v2[0] += t * t; }
              else W.sd[i] = -ss;
            }
          });
    });
  }
  __syncthreads();
  // cone coordinates: project -s onto each cone (Euclidean, FP64, in place in W.sd)
  {
    const int warp = threadIdx.x >> 5, nw = nwarps();
    for (int pass = 0; pass < 2; ++pass) {
      const int64_t b0 = pass == 0 ? own.s0 : own.r0, b1 = pass == 0 ? own.s1 : own.r1;
      const int64_t* off = pass == 0 ? P.soc_off : P.rsoc_off;
      for (int64_t blk = b0 + warp; blk < b1; blk += nw) {
        const int64_t s = off[blk];
        const int d = (int)(off[blk + 1] - s);
        if (pass == 0) warp_soc_euclid<double>(W.sd + s, d, lane);
        else warp_rsoc_euclid<double>(W.sd + s, d, lane);
      }
    }
    // slices (unscaled middle coordinate 1): the support term joins the dual objective and
    // the part of the slack outside its domain is left in W.sd as dual residual
    for (int64_t e = own.e0 + threadIdx.x; e < own.e1; e += blockDim.x) {
      double* z = W.sd + P.exp_base + 3 * e;
      double o[3];
      if (P.exp_fix && P.exp_fix[e] > 0.0) {
        const double sl[3] = {-z[0], -z[1], -z[2]};
        v2[2] += slice_support(false, 0.0, sl, o);
      } else {
        exp_proj_euclid(z[0], z[1], z[2], o);
      }
      z[0] = o[0]; z[1] = o[1]; z[2] = o[2];
    }
    for (int64_t e = own.p0 + threadIdx.x; e < own.p1; e += blockDim.x) {
      double* z = W.sd + P.pow_base + 3 * e;
      double o[3];
      if (P.pow_fix && P.pow_fix[e] > 0.0) {
        const double sl[3] = {-z[0], -z[1], -z[2]};
        v2[2] += slice_support(true, P.pow_alpha[e], sl, o);
      } else {
        pow_proj(z[0], z[1], z[2], P.pow_alpha[e], 1.0, 1.0, 1.0, o);
      }
      z[0] = o[0]; z[1] = o[1]; z[2] = o[2];
    }
    __syncthreads();
    for (int seg = 2; seg < 6; ++seg)
      for (int64_t i = own.x0[seg] + threadIdx.x; i < own.x1[seg]; i += blockDim.x) v2[0] += W.sd[i] * W.sd[i];
  }
  publish<3>(v2, 0, false);
  if (!sync_gather(3)) return false;
  if (threadIdx.x == 0) {
    double rqr = 0.0;
    for (int l = 0; l < k; ++l) rqr += tk[l] * wk[l];
    const double xqx = xqdx + rqr + xpx;
    const double sc = P.beta_b * P.beta_c;
    const double pobj = sc * (0.5 * xqx + cx), dobj = sc * (by + (GEN ? C.red[1] : 0.0) - 0.5 * xqx) + C.red[2];
    const double nrp = sqrt(rp2), nrd = sqrt(C.red[0]);
    double* K = C.s.kkt;
    K[0] = nrp / (1.0 + P.norm_b);
    K[1] = nrd / (1.0 + P.norm_c);
    // an infinite slice support term (dual objective -inf) is the limit eps_g -> 1
    K[2] = isfinite(dobj) ? fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj)) : 1.0;
    K[3] = fmax(K[0], fmax(K[1], K[2]));
    K[4] = pobj; K[5] = dobj; K[6] = nrp; K[7] = nrd;
    if (!isfinite(K[3])) C.s.err = kErrNumeric;
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// main loop: `budget` outer iterations at most (the host relaunches)
// ---------------------------------------------------------------------------
template <typename T, class Team, bool GEN>
__device__ void Solver<T, Team, GEN>::run(long long budget) {
  const int k = P.k;
  const bool avg = O.update == 1;
  const int lane = threadIdx.x & 31;
  if (O.profile && team.bid() == 0 && threadIdx.x == 0) C.t_last = now_ns();
  const unsigned long long t_begin = C.t_last;
  for (long long it = 0; it < budget; ++it) {
    if (C.s.status != 0 || C.s.err != 0) break;
    // adaptive inner tolerance (eq. monotone-primal-inner-tol), movement of consecutive candidates
    if (threadIdx.x == 0 && C.s.k >= 1) {
      const double cand = fmax(O.gamma_in * C.s.mov / C.s.tau, O.eps_min_in);
      if (cand < C.s.eps_in) C.s.eps_in = cand;
    }
    __syncthreads();
    const int hb = C.s.hb, wb = C.s.wb;
    const T* hx = W.hx[hb];
    const T* hy = W.hy[hb];
    int ub = 0;
    const bool ok = (P.qmode == kQDiag) ? prox_diag(hx) : prox_bb(hx, ub);
    if (!ok) return;
    const T* wxn = W.u[ub];
    const long long ktot1 = C.s.ktot + 1;
    const bool check = (ktot1 % O.check_every) == 0 || ktot1 >= O.max_iter;
    const bool needE = !avg && (C.s.k == 0 || check);
    const bool halpern_now = !avg && !check;
    const double tau = C.s.tau, sigma = C.s.sigma;
    const double kk = (double)C.s.k;
    const double c1 = (kk + 1.0) / (kk + 2.0), c2 = 1.0 / (kk + 2.0), r2 = 2.0 * O.rho, r1 = 1.0 - 2.0 * O.rho;
    // ---- P5: dual step on the owned rows, candidate bookkeeping on the owned coordinates.
    // Every-iteration work in the iterate precision T; the check-time quantities
    // (E^2 parts, PID movements) in FP64.
    double v6[6] = {0, 0, 0, 0, 0, 0};
    T mov_acc = T(0);
    T* hyn = W.hy[hb ^ 1];
    const T sg = T(sigma), tc1 = T(c1), tc2 = T(c2), tr1 = T(r1), tr2 = T(r2), tkk = T(kk);
    auto dual_row = [&](int64_t r, int gl, T s1, T s2) {
      if (gl != 0) return;
      const T h = hy[r];
      T wy = h + sg * (P.b[r] - s1);   // eq. stored-pdhg-candidate
      if (GEN && P.rhi) {   // general form: prox of the support function of [lo, hi] (Moreau)
        const T lo = P.b[r], hi = P.rhi[r];
        if (lo != hi) {
          const T z = s1 - h / sg;
          wy = h - sg * s1 + sg * (z < lo ? lo : (z > hi ? hi : z));
        }
      }
      W.wy[r] = wy;
      if (halpern_now) hyn[r] = tc1 * (tr2 * wy + tr1 * h) + tc2 * W.ay[r];   // eq. rh-update
      if (avg) {
        hyn[r] = wy;
        W.avy[r] = (tkk * W.avy[r] + wy) / (tkk + T(1));
      }
      if (needE) {
        const double dy = (double)h - (double)wy;
        v6[2] += dy * dy;
        v6[3] += (double)s2 * dy;
      }
      if (check) {
        const double e = (double)wy - (double)W.ay[r];
        v6[5] += e * e;
      }
    };
    unsigned long long tsub = (O.profile && team.bid() == 0 && threadIdx.x == 0) ? now_ns() : 0ull;
    if (needE) {
      vals(P.a_v, P.a_vb, [&](auto av) {
        rows_loop2_tpr<T>(own.g_a, P.a_rp, P.a_ci, av, own.row0, own.row1,
                          [&](int j) { return T(2) * wxn[j] - hx[j]; }, [&](int j) { return hx[j] - wxn[j]; },
                          dual_row);
      });
    } else {
      // between checks the row products need only 2 w_x - h_x: written once for the owned
      // coordinates, it is gathered as one operand instead of two
      T* zv = W.z;
      for (int seg = 0; seg < 6; ++seg)
        for (int64_t i0 = own.x0[seg] + threadIdx.x; i0 < own.x1[seg]; i0 += 4 * (int64_t)blockDim.x) {
          T w4[4], h4[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int64_t i = i0 + e * (int64_t)blockDim.x;
            w4[e] = i < own.x1[seg] ? wxn[i] : T(0);
            h4[e] = i < own.x1[seg] ? hx[i] : T(0);
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int64_t i = i0 + e * (int64_t)blockDim.x;
            if (i < own.x1[seg]) zv[i] = T(2) * w4[e] - h4[e];
          }
        }
      if (!team.sync()) return;
      subtick(12, tsub);
      if (P.cb_n > 1) {
        // column blocks: every block of the team works on the same slice of z (one barrier per
        // slice), so the slice stays in L2 while its entries stream past; a row keeps its lane
        // in every slice, which adds its partial sums in slice order
        T* acc = W.cb_acc;
        for (int b = 0; b < P.cb_n; ++b) {
          const bool first = b == 0, last = b == P.cb_n - 1;
          vals(P.cb_v, P.cb_vb, [&](auto cbv) {
            rows_loop_multi<kMultiRows, T, kMultiU, true>(P.cb_rp + (int64_t)b * P.m, P.cb_ci, cbv, own.row0, own.row1,
                             [&](int j) { return zv[j]; }, [&](int64_t r, int gl, T s1) {
                               if (gl != 0) return;
                               if (last) dual_row(r, 0, first ? s1 : acc[r] + s1, T(0));
                               else acc[r] = first ? s1 : acc[r] + s1;
                             });
          });
          if (!last && !team.sync()) return;
        }
      } else {
        vals(P.a_v, P.a_vb, [&](auto av) {
          rows_loop_tpr<T>(own.g_a, P.a_rp, P.a_ci, av, own.row0, own.row1, [&](int j) { return zv[j]; },
                           [&](int64_t r, int gl, T s1) { dual_row(r, gl, s1, T(0)); });
        });
      }
    }
    subtick(13, tsub);
    T* hxn = W.hx[hb ^ 1];
    T* wxs = W.wx[wb ^ 1];
    const T* wxp = W.wx[wb];
    if (halpern_now && !needE && !check && !avg) {
      // between checks: four coordinates per thread with their loads issued together (same
      // arithmetic; the movement sum takes the same order as the general loop below)
      constexpr int EU = 4;
      const int64_t B = blockDim.x;
      const T* __restrict__ axp = W.ax;
      for (int seg = 0; seg < 6; ++seg) {
        const int64_t a = own.x0[seg], b = own.x1[seg];
        for (int64_t i0 = a + threadIdx.x; i0 < b; i0 += EU * B) {
          T w[EU], h[EU], p[EU], an[EU];
#pragma unroll
          for (int e = 0; e < EU; ++e) {
            const int64_t i = i0 + e * B;
            const bool ok = i < b;
            w[e] = ok ? wxn[i] : T(0);
            h[e] = ok ? hx[i] : T(0);
            p[e] = ok ? wxp[i] : T(0);
            an[e] = ok ? axp[i] : T(0);
          }
#pragma unroll
          for (int e = 0; e < EU; ++e) {
            const int64_t i = i0 + e * B;
            if (i >= b) break;
            const T mv = w[e] - p[e];
            mov_acc += mv * mv;
            wxs[i] = w[e];
            hxn[i] = tc1 * (tr2 * w[e] + tr1 * h[e]) + tc2 * an[e];
          }
        }
      }
    } else
    for (int seg = 0; seg < 6; ++seg) {
      const int64_t a = own.x0[seg], b = own.x1[seg];
      for (int64_t base = a + (threadIdx.x - lane); base < b; base += blockDim.x) {
        const int64_t i = base + lane;
        const bool okc = i < b;
        T hn = T(0);
        if (okc) {
          const T w = wxn[i], h = hx[i];
          const T mv = w - wxp[i];
          mov_acc += mv * mv;
          wxs[i] = w;
          if (needE) { const double d = (double)h - (double)w; v6[1] += d * d; }
          if (check) { const double e = (double)w - (double)W.ax[i]; v6[4] += e * e; }
          if (halpern_now) {
            hn = tc1 * (tr2 * w + tr1 * h) + tc2 * W.ax[i];
            hxn[i] = hn;
          }
          if (avg) {
            hxn[i] = w;
            W.avx[i] = (tkk * W.avx[i] + w) / (tkk + T(1));
          }
        }
      }
    }
    if (halpern_now && k > 0) rx_lmajor(hxn);
    v6[0] = (double)mov_acc;
    __syncthreads();
    subtick(14, tsub);
    if (needE || check) {
      publish<6>(v6, 0, halpern_now && k > 0);
    } else {
      T v6t[6] = {mov_acc, T(0), T(0), T(0), T(0), T(0)};
      publish_t<6>(v6t, 0, halpern_now && k > 0);
    }
    if (!sync_gather(6 + ((halpern_now && k > 0) ? k : 0), 3, 4)) return;
    // ---- control after the dual step
    if (threadIdx.x == 0) {
      State& S = C.s;
      S.ktot = ktot1;
      S.inner_total += C.inner_j;
      S.mov = sqrt(fmax(C.red[0], 0.0));
      if (needE) {
        // E^2 = omega ||dx||^2 + ||dy||^2/omega + 2 eta <A dx, dy> (eq. practical-fixed-point-movement)
        const double E2 = S.omega * C.red[1] + C.red[2] / S.omega + 2.0 * S.eta * C.red[3];
        S.lastE = sqrt(fmax(E2, 0.0));
        if (S.k == 0) { S.E0 = S.lastE; S.Eprev = S.lastE; }
        if (!isfinite(E2)) S.err = kErrNumeric;
      }
      C.pid_dx = sqrt(fmax(C.red[4], 0.0));
      C.pid_dy = sqrt(fmax(C.red[5], 0.0));
      if (halpern_now) {
        for (int l = 0; l < k; ++l) S.t_h[l] = C.red[6 + l];
        S.k += 1;
        S.hb ^= 1;
      }
      if (avg) {
        for (int l = 0; l < k; ++l) S.t_h[l] = C.tcur[l];   // h = w
        S.k += 1;
        S.hb ^= 1;
      }
      S.wb ^= 1;
    }
    __syncthreads();
    if (!check && !(avg && C.s.k >= O.avg_epoch)) continue;
    // ---- check: KKT of the unscaled candidate (the running average for the averaged variant)
    if (check) {
      const bool ok2 = avg ? kkt(W.avx, W.avy, false) : kkt(W.wx[C.s.wb], W.wy, true);
      if (!ok2) return;
      tick(5);
      if (threadIdx.x == 0) {
        State& S = C.s;
        if (S.kkt[3] <= O.tol) S.status = 1;
        else if (S.ktot >= O.max_iter) S.status = 2;
      }
      __syncthreads();
      if (C.s.status != 0 || C.s.err != 0) break;
    }
    if (avg) {
      if (C.s.k >= O.avg_epoch) {
        // restart from the epoch average (Alg. "pdhcq1", averaged branch)
        const int hb2 = C.s.hb;   // after the swap: hx[hb2] holds w; overwrite with the average
        for (int seg = 0; seg < 6; ++seg)
          for (int64_t i = own.x0[seg] + threadIdx.x; i < own.x1[seg]; i += blockDim.x) W.hx[hb2][i] = W.avx[i];
        if (k > 0) rx_lmajor(W.hx[hb2]);
        for (int64_t r = own.row0 + threadIdx.x; r < own.row1; r += blockDim.x) W.hy[hb2][r] = W.avy[r];
        __syncthreads();
        double z1[1] = {0.0};
        publish<1>(z1, 0, k > 0);
        if (!sync_gather(1 + k)) return;
        if (threadIdx.x == 0) {
          for (int l = 0; l < k; ++l) C.s.t_h[l] = C.red[1 + l];
          C.s.k = 0;
          C.s.restarts += 1;
        }
        __syncthreads();
      }
      continue;
    }
    // ---- restart decision (eq. practical-restart-rule)
    if (threadIdx.x == 0) {
      State& S = C.s;
      const double E = S.lastE;
      bool rs = false;
      if (S.k >= 1) {
        if (E <= O.beta_s * S.E0) rs = true;
        else if (E <= O.beta_n * S.E0 && E > S.Eprev) rs = true;
        else if ((double)S.k >= O.beta_a * (double)S.ktot) rs = true;
      }
      S.Eprev = E;
      C.alpha = rs ? 1.0 : 0.0;
    }
    __syncthreads();
    const bool restart = C.alpha != 0.0;
    const int hbn = hb ^ 1;
    const T* wx = W.wx[C.s.wb];
    if (restart) {
      // restart from the final stored candidate (eq. restart-output): a = h = w
      for (int seg = 0; seg < 6; ++seg)
        for (int64_t i = own.x0[seg] + threadIdx.x; i < own.x1[seg]; i += blockDim.x) {
          const T w = wx[i];
          W.ax[i] = w;
          W.hx[hbn][i] = w;
        }
      for (int64_t r = own.row0 + threadIdx.x; r < own.row1; r += blockDim.x) {
        const T w = W.wy[r];
        W.ay[r] = w;
        W.hy[hbn][r] = w;
      }
      if (!team.sync()) return;
      if (threadIdx.x == 0) {
        State& S = C.s;
        // PID primal weight (eqs. pid-error, pid-weight); reading: skipped when a movement is <= 1e-10
        const double dxn = C.pid_dx, dyn = C.pid_dy;
        if (O.pid && dxn > 1e-10 && dyn > 1e-10) {
          const double e = log(dyn / (S.omega * dxn));
          S.pid_int = O.beta_I * S.pid_int + e;
          const double lw = log(S.omega) + O.K_P * e + O.K_I * S.pid_int + O.K_D * (e - S.err_prev);
          S.err_prev = e;
          S.omega = exp(lw);
          S.tau = S.eta / S.omega;
          S.sigma = S.eta * S.omega;
        }
        for (int l = 0; l < k; ++l) S.t_h[l] = C.tcur[l];   // R h_x = R w_x
        S.k = 0;
        S.restarts += 1;
        S.hb = hbn;
      }
      __syncthreads();
      tick(6);
    } else {
      // deferred reflected-Halpern step of a check iteration
      for (int seg = 0; seg < 6; ++seg)
        for (int64_t i = own.x0[seg] + threadIdx.x; i < own.x1[seg]; i += blockDim.x)
          W.hx[hbn][i] = T(c1) * (T(r2) * wx[i] + T(r1) * hx[i]) + T(c2) * W.ax[i];
      if (k > 0) rx_lmajor(W.hx[hbn]);
      for (int64_t r = own.row0 + threadIdx.x; r < own.row1; r += blockDim.x)
        W.hy[hbn][r] = T(c1) * (T(r2) * W.wy[r] + T(r1) * hy[r]) + T(c2) * W.ay[r];
      __syncthreads();
      double z1[1] = {0.0};
      publish<1>(z1, 0, k > 0);
      if (!sync_gather(1 + k)) return;
      if (threadIdx.x == 0) {
        for (int l = 0; l < k; ++l) C.s.t_h[l] = C.red[1 + l];
        C.s.k += 1;
        C.s.hb = hbn;
      }
      __syncthreads();
      tick(6);
    }
  }
  if (O.profile && team.bid() == 0 && threadIdx.x == 0) C.s.prof[7] += (double)(now_ns() - t_begin);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <typename T>
struct KernelArgs {
  Prob<T> P;
  Work<T> W;
  Opts O;
  State* S;
  GridBarrier bar;
  long long budget;
};

__device__ __forceinline__ void load_state(Ctl& C, const State* S) {
  if (threadIdx.x == 0) C.s = *S;
  __syncthreads();
}

// Shared-memory layout of a solver block: Ctl, block_sum scratch, per-warp R
// accumulators, per-warp cone staging.
template <typename T>
__host__ __device__ constexpr size_t solver_smem_bytes(int threads) {
  return sizeof(Ctl) + sizeof(double) * (size_t)kMaxSlots * (threads / 32) + sizeof(double) * (size_t)(threads / 32) * kMaxRank +
         sizeof(T) * (size_t)(threads / 32) * 2 * 128 + 64;
}

template <typename T, class Team, bool GEN>
__device__ __forceinline__ void solver_entry(const KernelArgs<T>& a, Team& team, char* smem) {
  Ctl& C = *reinterpret_cast<Ctl*>(smem);
  const int nw = blockDim.x >> 5;
  double* scratch = reinterpret_cast<double*>(smem + sizeof(Ctl));
  double* wacc = scratch + (size_t)kMaxSlots * nw;
  T* cbuf = reinterpret_cast<T*>(wacc + (size_t)nw * kMaxRank);
  load_state(C, a.S);
  Solver<T, Team, GEN> s(a.P, a.W, a.O, team, C, scratch, wacc, cbuf);
  s.run(a.budget);
  __syncthreads();
  if (team.bid() == 0 && threadIdx.x == 0) {
    if (team.failed) C.s.err = kErrBarrier;
    *a.S = C.s;
  }
  team.finish();
}

template <typename T, bool GEN>
__global__ void __launch_bounds__(512, 1) pdhg_grid_kernel(KernelArgs<T> a) {
  extern __shared__ __align__(16) char smem[];
  GridTeam team;
  team.init(a.bar, a.W.part);
  solver_entry<T, GridTeam, GEN>(a, team, smem);
}

template <typename T, bool GEN>
__global__ void __launch_bounds__(512, 1) pdhg_cta_kernel(KernelArgs<T> a) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double part[kMaxSlots];
  CtaTeam team;
  team.init(part);
  solver_entry<T, CtaTeam, GEN>(a, team, smem);
}

// one thread-block cluster (the whole grid) for problems too small to spread over the
// GPU: cluster barriers and distributed-shared-memory reductions instead of global ones
template <typename T, bool GEN>
__global__ void __launch_bounds__(512, 1) pdhg_cluster_kernel(KernelArgs<T> a) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double part[2 * kMaxSlots];
  ClusterTeam team;
  team.init(part);
  solver_entry<T, ClusterTeam, GEN>(a, team, smem);
}

// Launch of the cluster kernel: `blocks` CTAs forming one cluster (sizes above 8 need the
// non-portable cluster attribute).
template <typename K>
cudaError_t launch_cluster(K kernel, void** args, int blocks, int threads, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (blocks > 8) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = blocks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, (const void*)kernel, args);
}

// Largest cluster (16, 8, 4 or 2 CTAs) of the solver kernel that the device can place with
// the given block size and shared memory; 0 if none.
template <typename K>
int cluster_size_for(K kernel, int threads, size_t smem) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int c = 16; c >= 2; c /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, (const void*)kernel, &cfg) == cudaSuccess && nc >= 1) return c;
    cudaGetLastError();
  }
  return 0;
}

}  // namespace cqp
