// The restarted PDHG iteration as one persistent kernel.
//
// Paper: Alg. "pdhcq1" (reflected-Halpern branch) and Sec. 4: primal prox
// (eq. prox-subproblem) by Jacobi projected BB (eqs. bb-inner-gradient,
// jacobi-bb-step) or, for diagonal Q, one metric projection (eqs.
// diagonal-q-metric, diagonal-q-metric-projection); dual step and
// reflected-Halpern update (eqs. stored-pdhg-candidate, rh-update); restart to
// the last candidate (eq. restart-output); adaptive restart (eqs.
// practical-fixed-point-movement, practical-restart-rule); PID primal weight
// (eqs. pid-error, pid-weight); adaptive inner tolerance (eq.
// monotone-primal-inner-tol, stop rule jacobi-stop-unscale); termination on
// the unscaled candidate.  The Cesaro-averaged variant (compiled Alg.
// "pdhcq1") restarts from the epoch average every avg_epoch iterations.
//
// Execution: every block of the team owns an equal share of each coordinate
// segment (free, nonnegative, SOC blocks, RSOC blocks, exponential cones,
// power cones) and an nnz-balanced range of rows of A.  A phase works on the
// owned data, publishes FP64 block partials, and ends with a team barrier;
// every block then sums the partials in the same order, so all blocks take the
// same control decisions without further communication.  Cone blocks never
// straddle two owners, so projections are block-local and need no barrier.
//
// Inner projected BB in one pass per iteration: the prox objective H is
// quadratic, so g^{j+1} - g^j = (Q + I/tau) s_{j+1} exactly and
//   <s, dg> = sum_i (q_i + 1/tau) s_i^2 + (R s)' D (R s)   (Q = diag(q) + R'DR),
// where R s = R u^{j+1} - R u^j comes out of the same reduction that carries
// ||s||^2 and <s, J s>.  The BB step size alpha_{j+1} is thus known right after
// the pass that produced u^{j+1}, and the gradient at u^{j+1} is formed on the
// fly inside the next pass.  A sparse P part needs P u^{j+1} first, so that mode
// uses two passes per iteration.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "common.cuh"
#include "cones.cuh"

namespace cqp {

enum QMode : int { kQDiag = 0, kQLowRank = 1, kQSparse = 2 };

template <typename T>
struct Prob {
  int64_t n, m;
  const int* a_rp; const int* a_ci; const T* a_v;     // scaled A (m rows)
  const int* t_rp; const int* t_ci; const T* t_v;     // scaled A' (n rows)
  const T* qd;                                        // explicit diagonal part of scaled Q (n)
  const T* jd;                                        // full diagonal of scaled Q (n)
  int k; const T* R; const double* D;                 // scaled low-rank factor (k x n), D (k x k)
  int kpad;                                            // rows of R as stored: k rounded up to 8, rows >= k zero
  double d_scale;                                     // D = d_scale * I when > 0 (else general D)
  const int* p_rp; const int* p_ci; const T* p_v;     // scaled sparse P (n rows) or null
  // BF16-stored matrix values (FP32 iterates only): when set, the products read these in place of
  // a_v, t_v, p_v, cb_v (the same scaled values, exactly representable in BF16)
  const __nv_bfloat16* a_vb; const __nv_bfloat16* t_vb; const __nv_bfloat16* p_vb; const __nv_bfloat16* cb_vb;
  const T* c; const T* b;                             // scaled c, b (general form: b holds the row lower bounds)
  const double* col; const double* row;               // x = beta_b x~/col, y = beta_c y~/row
  double beta_b, beta_c, norm_b, norm_c;              // ||b||, ||c|| of the unscaled data
  int64_t n_free, n_nonneg;                           // [0,n_free) free, then nonneg
  int64_t n_soc; const int64_t* soc_off;              // SOC blocks: coordinates [soc_off[j], soc_off[j+1])
  int64_t n_rsoc; const int64_t* rsoc_off;
  int64_t n_exp, exp_base;                            // exp cones at exp_base + 3 j
  int64_t n_pow, pow_base; const double* pow_alpha;
  // slices (CQP_CONE_EXP1 / POW1): per exp / pow block the fixed middle coordinate in scaled
  // variables, f~ = col / beta_b, or 0 for a full cone (null: no slices in the problem)
  const double* exp_fix; const double* pow_fix;
  // column blocks of A for the dual step's product between checks (cb_n <= 1: not used):
  // block b's rows are rows of the CSR with row pointers cb_rp + b m (into cb_ci, cb_v)
  int cb_n; const int* cb_rp; const int* cb_ci; const T* cb_v;
  // column slices of A' for the A'y pass (tcb_n <= 1: not used): slice b's rows are rows of the
  // CSR with row pointers tcb_rp + b n (into tcb_ci, tcb_v), columns in the b-th range of y
  int tcb_n; const int* tcb_rp; const int* tcb_ci; const T* tcb_v; const __nv_bfloat16* tcb_vb;
  int p_ulen;                                         // > 0: every row of P has exactly p_ulen entries
  int qmode;
  int euclid_cones;                                   // diagonal mode with zero q on cone coordinates
  int tpr_a, tpr_t, tpr_p;                            // threads per row of A, A' and P
  const T* rhi;                                       // general form: scaled row upper bounds (null: A x = b)
  const T* xlo; const T* xhi;                         // general form: scaled bounds of the free segment (null: free)
  const T* csc;                                       // rescaled-cone mode: S_x per coordinate (null: blocks are cones)
};

template <typename T>
struct Work {
  T* hx[2]; T* hy[2];   // reflected-Halpern states (double-buffered)
  T* ax; T* ay;         // anchors
  T* wx[2]; T* wy;      // stored candidates (x double-buffered for the movement)
  T* v;                 // x + tau A'y
  T* z;                 // 2 w_x - h_x, the operand of the dual step's row products
  T* u[2];              // inner iterates
  T* g[2];              // gradients (sparse-P mode)
  T* avx; T* avy;       // running averages (averaged variant)
  T* mbuf;              // metric of cone blocks too large for shared staging
  T* cb_acc;            // partial row sums of the column-blocked product (m)
  T* tcb_acc;           // partial row sums of the column-sliced A'y pass (n)
  float* root;          // last scalar root per cone block (warm starts): SOC, RSOC, exp, pow
  double* sd;           // FP64 dual slack of cone coordinates (KKT)
  double* part;         // block partials [kMaxSlots][nb]
};

struct Opts {
  double rho, eps_min_in, gamma_in, tol;
  double beta_s, beta_n, beta_a, beta_I, K_P, K_I, K_D;
  long long max_iter;
  int check_every, max_inner, jacobi, pid, update, avg_epoch;
  int profile;                     // accumulate per-phase wall time (block 0) into State::prof
  int warm_roots;                  // start cone root-finding from the block's previous root
};

// Control state of one solve (device memory, FP64 scalars).
struct State {
  double tau, sigma, omega, eta;
  double eps_in, E0, Eprev, pid_int, err_prev, mov;
  double t_h[kMaxRank];            // R~ h_x of the current Halpern state
  double kkt[8];                   // eps_p, eps_d, eps_g, rel_kkt, pobj, dobj, ||r_p||, ||r_d||
  double lastE;
  double prof[16];                 // ns per phase: A'y, prox work, prox barriers, dual step, its barrier,
                                   // KKT, restart/Halpern at checks, whole loop; inner-step split:
                                   // elementwise, cone gradient, cone projection, cone bookkeeping;
                                   // dual-step split: z pass, row products, Halpern update of x
  long long k, ktot, restarts, inner_total;
  int hb, wb;                      // current Halpern / candidate buffer
  int status;                      // 0 running, 1 converged, 2 iteration limit
  int err;                         // DevErr
};

// block-shared copy of the control state plus reduction outputs
struct Ctl {
  State s;
  double red[kMaxSlots];           // gathered sums of the last phase
  double w[kMaxRank];              // D~ t for the gradient of the current inner step
  float wf[kMaxRank];              // the same in FP32 (iterate precision of the mixed mode)
  double rblk[kMaxRank];           // this block's R x partials, ready to publish
  double tcur[kMaxRank];           // R~ u^j of the current inner iterate
  double alpha, sJs;
  double pid_dx, pid_dy;           // ||w_x - a_x||, ||w_y - a_y|| of the last check
  long long inner_j;
  unsigned long long t_last;       // profiling clock
};

// ---------------------------------------------------------------------------
// block ownership
// ---------------------------------------------------------------------------
struct Own {
  int64_t x0[6], x1[6];   // owned coordinate ranges: free, nonneg, soc, rsoc, exp, pow
  int64_t f0, f1, nn0, nn1, s0, s1, r0, r1, e0, e1, p0, p1;
  int64_t row0, row1;
  int g_a, g_t, g_p;      // lanes per row of A, A' and P on this block's rows
};

// Batched mode: independent instances of one block-diagonal problem, each solved by
// one thread block (CtaTeam) with its own scaling, step sizes, restarts and stop.
struct BatchArgs {
  int64_t count;
  const int* order;                 // processing order (largest instances first)
  unsigned* queue;                  // next position in `order` (zeroed by the host)
  const Own* own;                   // per instance: its ranges in the permuted layout
  const double* beta_b; const double* beta_c;   // per-instance bound-objective factors
  const double* norm_b; const double* norm_c;   // per-instance ||b||, ||c|| (unscaled)
  const int* rank;                  // per-instance rows of R in use (null: all)
  State* S;                         // per-instance control state
  const int64_t* perm;              // permuted -> original coordinate
  const double* x0; const double* y0;           // unscaled starts, original order (or null)
  double* x_out; double* y_out;     // unscaled final candidates, original order
  long long chunk;                  // outer iterations between time-limit checks
  unsigned long long time_limit_ns; // 0: none
};

// Free and nonnegative coordinates are shared by the work of their A' rows (a coordinate's
// column of A), cone segments by block count; rows of A by nnz (both with kRowWork per row).
template <typename T>
__device__ void make_own(const Prob<T>& P, int b, int nb, Own& o) {
  split_rows_weighted(P.t_rp, 0, P.n_free, b, nb, o.f0, o.f1);
  split_rows_weighted(P.t_rp, P.n_free, P.n_nonneg, b, nb, o.nn0, o.nn1);
  o.nn0 += P.n_free; o.nn1 += P.n_free;
  split_range(P.n_soc, b, nb, o.s0, o.s1);
  split_range(P.n_rsoc, b, nb, o.r0, o.r1);
  split_range(P.n_exp, b, nb, o.e0, o.e1);
  split_range(P.n_pow, b, nb, o.p0, o.p1);
  o.x0[0] = o.f0; o.x1[0] = o.f1;
  o.x0[1] = o.nn0; o.x1[1] = o.nn1;
  o.x0[2] = P.n_soc ? P.soc_off[o.s0] : 0; o.x1[2] = P.n_soc ? P.soc_off[o.s1] : 0;
  o.x0[3] = P.n_rsoc ? P.rsoc_off[o.r0] : 0; o.x1[3] = P.n_rsoc ? P.rsoc_off[o.r1] : 0;
  o.x0[4] = P.exp_base + 3 * o.e0; o.x1[4] = P.exp_base + 3 * o.e1;
  o.x0[5] = P.pow_base + 3 * o.p0; o.x1[5] = P.pow_base + 3 * o.p1;
  split_rows_by_nnz(P.a_rp, P.m, b, nb, o.row0, o.row1);
  o.g_a = block_group_width(P.tpr_a, (int64_t)P.a_rp[o.row1] - P.a_rp[o.row0], o.row1 - o.row0);
  int64_t tn = 0, pn = 0, cnt = 0;
  for (int s = 0; s < 6; ++s) {
    cnt += o.x1[s] - o.x0[s];
    tn += (int64_t)P.t_rp[o.x1[s]] - P.t_rp[o.x0[s]];
    if (P.p_rp) pn += (int64_t)P.p_rp[o.x1[s]] - P.p_rp[o.x0[s]];
  }
  o.g_t = block_group_width(P.tpr_t, tn, cnt);
  o.g_p = P.p_rp ? block_group_width(P.tpr_p, pn, cnt) : P.tpr_p;
}

// ---------------------------------------------------------------------------
// CSR row products by groups of G lanes; every lane of the group gets the sum.
// X(j) returns the operand for column j.
// ---------------------------------------------------------------------------
// Entries of one row handled by lane gl of a G-lane group, kBatch<G> at a time:
// the column indices and values of a batch are loaded first (the last, partial
// batch under a predicate) and the operand gathers of the batch are issued
// together, so each lane keeps several independent loads in flight (the
// persistent kernel runs only 16 warps per SM).  Narrow groups get wider batches.
// ci and v are read-only for the whole kernel, hence the non-coherent loads;
// the gathered operands are written by other phases and use plain loads.
constexpr int kUnroll = 4;
template <int G> struct RowBatch { static constexpr int value = G <= 2 ? 8 : 4; };

// A stored matrix value in the accumulation type (FP32, FP64 or BF16 storage).
template <typename Acc>
__device__ __forceinline__ Acc ld_val(const float* p) { return (Acc)__ldg(p); }
template <typename Acc>
__device__ __forceinline__ Acc ld_val(const double* p) { return (Acc)__ldg(p); }
template <typename Acc>
__device__ __forceinline__ Acc ld_val(const __nv_bfloat16* p) { return (Acc)__bfloat162float(__ldg(p)); }

template <int G, typename Acc, typename T, typename X>
__device__ __forceinline__ Acc seg_dot(const int* __restrict__ ci, const T* __restrict__ v, int beg, int end, int gl,
                                       X xf) {
  constexpr int U = RowBatch<G>::value;
  Acc s = Acc(0);
  for (int k = beg + gl; k < end; k += U * G) {
    int j[U];
    Acc a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int kk = k + u * G;
      const bool ok = kk < end;
      j[u] = ok ? __ldg(ci + kk) : -1;
      a[u] = ok ? ld_val<Acc>(v + kk) : Acc(0);
    }
    Acc g[U];
#pragma unroll
    for (int u = 0; u < U; ++u) g[u] = j[u] >= 0 ? (Acc)xf(j[u]) : Acc(0);
#pragma unroll
    for (int u = 0; u < U; ++u) s += a[u] * g[u];
  }
  return s;
}

template <int G, typename Acc, typename T, typename X>
__device__ __forceinline__ Acc row_dot(const int* rp, const int* ci, const T* v, int64_t row, int gl, X xf) {
  return group_sum<G>(seg_dot<G, Acc>(ci, v, rp[row], rp[row + 1], gl, xf));
}

// Iterate the rows [r0, r1) of a CSR matrix with groups of G lanes; f(row, gl, sum)
// is called by every lane of the group after the reduction.
template <int G, typename Acc, typename T, typename X, typename F>
__device__ __forceinline__ void rows_loop(const int* rp, const int* ci, const T* v, int64_t r0, int64_t r1, X xf, F f) {
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);
  const int64_t gid = threadIdx.x / G, ngr = blockDim.x / G;
  // all lanes of a warp iterate together (group_sum shuffles need full warps)
  const int64_t nrows = r1 - r0;
  const int64_t per_warp_rows = 32 / G;
  const int64_t nwarps = blockDim.x >> 5;
  const int64_t warp = threadIdx.x >> 5;
  for (int64_t base = warp * per_warp_rows; base < nrows; base += nwarps * per_warp_rows) {
    const int64_t r = r0 + base + (lane / G);
    const bool ok = r < r1;
    Acc s = Acc(0);
    if (ok) s = seg_dot<G, Acc>(ci, v, rp[r], rp[r + 1], gl, xf);
    s = group_sum<G>(s);
    if (ok) f(r, gl, s);
  }
  (void)gid;
  (void)ngr;
}

// One lane per row, RB rows per lane at a time: the row pointers of all RB rows are loaded
// first, then kMultiU entries of every row, then their gathers, so a lane keeps 2 RB + 2 RB
// kMultiU independent loads in flight instead of one row's dependent chain (row pointer ->
// entries -> gathered operands).  Short rows (a handful of entries) are otherwise bound by
// that chain's latency.  Each row's entries are still summed in storage order.
constexpr int kMultiRows = 4;
constexpr int kMultiU = 4;
// ulen > 0: every row has exactly ulen entries (rp[r] = ulen r), so the row pointers are not read.
template <int RB, typename Acc, int U = kMultiU, bool PF = false, typename T, typename X, typename F>
__device__ __forceinline__ void rows_loop_multi(const int* rp, const int* ci, const T* v, int64_t r0, int64_t r1, X xf,
                                                F f, int ulen = 0) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const int64_t nrows = r1 - r0;
  const int64_t stride = nwarps * 32 * RB;
  // PF: the row pointers of the lane's next RB rows are loaded while the current rows are summed
  // (measured faster for the column slices of A, slower for those of A')
  int nbeg[RB], nend[RB];
  auto load_ptrs = [&](int64_t bs) {
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const int64_t r = r0 + bs + 32 * q + lane;
      const bool ok = bs < nrows && r < r1;
      if (ulen > 0) {
        nbeg[q] = ok ? (int)(ulen * r) : 0;
        nend[q] = ok ? nbeg[q] + ulen : 0;
      } else {
        nbeg[q] = ok ? rp[r] : 0;
        nend[q] = ok ? rp[r + 1] : 0;
      }
    }
  };
  if (PF) load_ptrs(warp * 32 * RB);
  for (int64_t base = warp * 32 * RB; base < nrows; base += stride) {
    int beg[RB], end[RB];
    Acc s[RB];
    int len = 0;
    if (!PF) load_ptrs(base);
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      beg[q] = nbeg[q];
      end[q] = nend[q];
      s[q] = Acc(0);
    }
    if (PF) load_ptrs(base + stride);
#pragma unroll
    for (int q = 0; q < RB; ++q) len = max(len, end[q] - beg[q]);
    for (int k = 0; k < len; k += U) {
      int j[RB][U];
      Acc a[RB][U];
#pragma unroll
      for (int q = 0; q < RB; ++q)
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int kk = beg[q] + k + u;
          const bool ok = kk < end[q];
          j[q][u] = ok ? __ldg(ci + kk) : -1;
          a[q][u] = ok ? ld_val<Acc>(v + kk) : Acc(0);
        }
      Acc g[RB][U];
#pragma unroll
      for (int q = 0; q < RB; ++q)
#pragma unroll
        for (int u = 0; u < U; ++u) g[q][u] = j[q][u] >= 0 ? (Acc)xf(j[q][u]) : Acc(0);
#pragma unroll
      for (int q = 0; q < RB; ++q)
#pragma unroll
        for (int u = 0; u < U; ++u) s[q] += a[q][u] * g[q][u];
    }
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const int64_t r = r0 + base + 32 * q + lane;
      if (r < r1) f(r, 0, s[q]);
    }
  }
}

// Row widths: tpr = G lanes per row (1..32), or kRowsBatched for one lane per row with
// kMultiRows rows per lane in flight (rows_loop_multi).
constexpr int kRowsBatched = 0;
// The same without the batched variant (it runs as one lane per row), for the rarely run
// passes (KKT checks), so the persistent kernel carries fewer copies of the row loops.
template <typename Acc, typename T, typename X, typename F>
__device__ __forceinline__ void rows_loop_tpr_plain(int tpr, const int* rp, const int* ci, const T* v, int64_t r0,
                                                    int64_t r1, X xf, F f) {
  switch (tpr) {
    case kRowsBatched:
    case 1: rows_loop<1, Acc>(rp, ci, v, r0, r1, xf, f); break;
    case 2: rows_loop<2, Acc>(rp, ci, v, r0, r1, xf, f); break;
    case 4: rows_loop<4, Acc>(rp, ci, v, r0, r1, xf, f); break;
    case 8: rows_loop<8, Acc>(rp, ci, v, r0, r1, xf, f); break;
    case 16: rows_loop<16, Acc>(rp, ci, v, r0, r1, xf, f); break;
    default: rows_loop<32, Acc>(rp, ci, v, r0, r1, xf, f); break;
  }
}

template <typename Acc, typename T, typename X, typename F>
__device__ __forceinline__ void rows_loop_tpr(int tpr, const int* rp, const int* ci, const T* v, int64_t r0, int64_t r1,
                                              X xf, F f, int ulen = 0) {
  switch (tpr) {
    case kRowsBatched: rows_loop_multi<kMultiRows, Acc>(rp, ci, v, r0, r1, xf, f, ulen); break;
    case 1: rows_loop<1, Acc>(rp, ci, v, r0, r1, xf, f); break;
    case 2: rows_loop<2, Acc>(rp, ci, v, r0, r1, xf, f); break;
    case 4: rows_loop<4, Acc>(rp, ci, v, r0, r1, xf, f); break;
    case 8: rows_loop<8, Acc>(rp, ci, v, r0, r1, xf, f); break;
    case 16: rows_loop<16, Acc>(rp, ci, v, r0, r1, xf, f); break;
    default: rows_loop<32, Acc>(rp, ci, v, r0, r1, xf, f); break;
  }
}

// ---------------------------------------------------------------------------
// The solver.  Team is GridTeam (whole GPU) or CtaTeam (one block).
// ---------------------------------------------------------------------------
// GEN: general standard form compiled in (row bounds, box blocks; the pointers are still
// checked at run time).  The equality-form kernels are built with GEN = false.
template <typename T, class Team, bool GEN = false>
struct Solver {
  const Prob<T>& P;
  const Work<T>& W;
  const Opts& O;
  Team& team;
  Ctl& C;
  Own own;
  double* scratch;   // block_sum scratch: kMaxSlots * nwarps doubles (shared)
  double* wacc;      // per-warp R-product accumulators: nwarps * kMaxRank doubles (shared)
  T* cbuf;           // per-warp cone staging: nwarps * 2 * kConeStage (shared)
  static constexpr int kConeStage = 128;

  __device__ Solver(const Prob<T>& p, const Work<T>& w, const Opts& o, Team& t, Ctl& c, double* scr, double* wa,
                    T* cb)
      : P(p), W(w), O(o), team(t), C(c), scratch(scr), wacc(wa), cbuf(cb) {
    make_own(P, team.bid(), team.nb(), own);
  }

  // ---- small helpers -------------------------------------------------------
  __device__ __forceinline__ int nwarps() const { return blockDim.x >> 5; }
  // Runs fn(values) with the BF16 copy of a matrix's values when there is one, else with the
  // iterate-precision copy.  BF16 storage is compiled into the whole-GPU FP32 solver only (the
  // setup runs matrix_bf16 handles on that team).
  static constexpr bool kBf16 = std::is_same<T, float>::value && std::is_same<Team, GridTeam>::value;
  template <typename F>
  __device__ __forceinline__ void vals(const T* v, const __nv_bfloat16* vb, F&& fn) const {
    if constexpr (kBf16) {
      if (vb) {
        fn(vb);
        return;
      }
    }
    fn(v);
  }
  static __device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
  }
  // adds the time since the previous tick to phase `slot` (block 0, thread 0, when profiling)
  __device__ __forceinline__ void tick(int slot) {
    if (O.profile && team.bid() == 0 && threadIdx.x == 0) {
      const unsigned long long t = now_ns();
      C.s.prof[slot] += (double)(t - C.t_last);
      C.t_last = t;
    }
  }
  // sub-phase clock (does not move the main tick clock)
  __device__ __forceinline__ void subtick(int slot, unsigned long long& t0) {
    if (O.profile && team.bid() == 0 && threadIdx.x == 0) {
      const unsigned long long t = now_ns();
      C.s.prof[slot] += (double)(t - t0);
      t0 = t;
    }
  }

  // (R' w)_i with w in shared memory (k entries, iterate precision)
  __device__ __forceinline__ T rtw(int64_t i, const T* w) const {
    T s = T(0);
    for (int l = 0; l < P.k; ++l) s += P.R[(int64_t)l * P.n + i] * w[l];
    return s;
  }
  __device__ __forceinline__ double rtw_d(int64_t i, const double* w) const {
    double s = 0.0;
    for (int l = 0; l < P.k; ++l) s += (double)P.R[(int64_t)l * P.n + i] * w[l];
    return s;
  }

  // publish NS block totals in slots [slot0, slot0+NS) plus, if with_r, the k R sums
  // (block totals in C.rblk, filled by the caller)
  template <int NS>
  __device__ void publish(double (&v)[NS], int slot0, bool with_r) {
    block_sum<NS>(v, scratch, C.red);   // C.red used as temporary block totals
    if (threadIdx.x == 0)
      for (int s = 0; s < NS; ++s) team.publish(slot0 + s, C.red[s]);
    if (with_r)
      for (int l = threadIdx.x; l < P.k; l += blockDim.x) team.publish(slot0 + NS + l, C.rblk[l]);
    __syncthreads();
  }
  // same with per-thread values in T (warp trees in T)
  template <int NS>
  __device__ void publish_t(T (&v)[NS], int slot0, bool with_r) {
    block_sum_r<T, NS>(v, scratch, C.red);
    if (threadIdx.x == 0)
      for (int s = 0; s < NS; ++s) team.publish(slot0 + s, C.red[s]);
    if (with_r)
      for (int l = threadIdx.x; l < P.k; l += blockDim.x) team.publish(slot0 + NS + l, C.rblk[l]);
    __syncthreads();
  }
  // wacc (per-warp R partials) -> C.rblk
  __device__ void rblk_from_wacc() {
    __syncthreads();
    const int nw = nwarps();
    for (int l = threadIdx.x; l < P.k; l += blockDim.x) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += wacc[w * P.k + l];
      C.rblk[l] = t;
    }
    __syncthreads();
  }
  // C.rblk[l] = sum over the owned coordinates of R[l, i] x_i: one warp per l, lanes
  // stream R's row l (contiguous) and x; x must be visible to the block
  __device__ void rx_lmajor(const T* x) {
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = nwarps();
    for (int l = warp; l < P.k; l += nw) {
      const T* Rl = P.R + (int64_t)l * P.n;
      T acc = T(0);
      for (int seg = 0; seg < 6; ++seg)
        for (int64_t i = own.x0[seg] + lane; i < own.x1[seg]; i += 32) acc += Rl[i] * x[i];
      acc = warp_sum(acc);
      if (lane == 0) C.rblk[l] = (double)acc;
    }
    __syncthreads();
  }

  __device__ bool sync_gather(int nslots, int prof_work = -1, int prof_wait = -1) {
    if (prof_work >= 0) tick(prof_work);
    if (!team.sync()) return false;
    team.gather(nslots, C.red);
    if (prof_wait >= 0) tick(prof_wait);
    return true;
  }

  // ---- projections of the owned cone blocks --------------------------------
  // Projects, in place, the owned SOC/RSOC/EXP/POW blocks of x in the metric
  //   kEuclid: M = I;  kJacobi: m_i = diag(Q~)_i + 1/tau (eq. jacobi-inner-metric);
  //   kDiagQ: m_i = 1 + tau q_i (eq. diagonal-q-metric).
  // Rescaled-cone mode (GEN kernels with P.csc): a block is S K, S = diag(csc), and its
  // m-metric projection is S Pi_K^{S m S}(S^-1 x) (eq. scaling-induced-metric).
  // Ends with __syncthreads.
  enum MetricKind : int { kEuclid = 0, kJacobi = 1, kDiagQ = 2 };
  __device__ __forceinline__ T metric(int kind, int64_t i, T tau, T itau) const {
    return kind == kJacobi ? P.jd[i] + itau : (kind == kDiagQ ? T(1) + tau * P.qd[i] : T(1));
  }
  __device__ __noinline__ void project_owned_cones(T* x, int kind, double tau_d) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = nwarps();
    const T* csc = GEN ? P.csc : nullptr;
    const bool euclid = kind == kEuclid && !csc;
    const T tau = T(tau_d), itau = T(1.0 / tau_d);
    T* zs = cbuf + warp * 2 * kConeStage;
    T* ms = zs + kConeStage;
    // SOC and RSOC blocks form one list dealt round-robin to the warps, so a warp
    // takes an RSOC block only after every warp has had a SOC block
    const int64_t nsoc = own.s1 - own.s0, nall = nsoc + (own.r1 - own.r0);
    for (int64_t item = warp; item < nall; item += nw) {
      const int pass = item < nsoc ? 0 : 1;
      const int64_t blk = pass == 0 ? own.s0 + item : own.r0 + (item - nsoc);
      const int64_t* off = pass == 0 ? P.soc_off : P.rsoc_off;
      const int64_t s = off[blk];
      const int d = (int)(off[blk + 1] - s);
      const bool staged = d <= kConeStage;
      T* z = staged ? zs : x + s;
      T* mm = staged ? ms : W.mbuf + s;
      for (int i = lane; i < d; i += 32) {
        if (csc) {
          const T si = csc[s + i];
          const T zi = x[s + i] / si;
          if (staged) zs[i] = zi; else x[s + i] = zi;
          mm[i] = metric(kind, s + i, tau, itau) * si * si;
        } else {
          if (staged) zs[i] = x[s + i];
          if (!euclid) mm[i] = metric(kind, s + i, tau, itau);
        }
      }
      __syncwarp();
      float* gs = O.warm_roots ? W.root + (pass == 0 ? blk : P.n_soc + blk) : nullptr;
      if (pass == 0) {
        if (euclid) warp_soc_euclid<T>(z, d, lane);
        else warp_soc_metric<T>(z, mm, d, lane, gs);
      } else {
        if (euclid) warp_rsoc_euclid<T>(z, d, lane);
        else warp_rsoc_metric<T>(z, mm, d, lane, gs);
      }
      if (staged || csc) {
        for (int i = lane; i < d; i += 32) x[s + i] = (staged ? zs[i] : x[s + i]) * (csc ? csc[s + i] : T(1));
        __syncwarp();
      }
    }
    // exponential and power blocks: one list, one thread per block, so no thread
    // runs an exp and a pow root-finding back to back while others idle
    const int64_t nexp = own.e1 - own.e0, n3 = nexp + (own.p1 - own.p0);
    for (int64_t item = threadIdx.x; item < n3; item += blockDim.x) {
      if (item < nexp) {
        const int64_t e = own.e0 + item;
        const int64_t s = P.exp_base + 3 * e;
        double o[3];
        float* gs = O.warm_roots ? W.root + P.n_soc + P.n_rsoc + e : nullptr;
        const double fx = P.exp_fix ? P.exp_fix[e] : 0.0;
        if (fx > 0.0) {   // slice {(r, f, t): f e^{r/f} <= t} (rejected with csc at setup)
          exp_slice_proj((double)x[s], (double)x[s + 2], fx, (double)metric(kind, s, tau, itau),
                         (double)metric(kind, s + 2, tau, itau), o, gs);
          x[s] = T(o[0]); x[s + 1] = T(o[1]); x[s + 2] = T(o[2]);
          continue;
        }
        if (csc) {
          double sc3[3], z3[3], m3[3];
          for (int q = 0; q < 3; ++q) {
            sc3[q] = (double)csc[s + q];
            z3[q] = (double)x[s + q] / sc3[q];
            m3[q] = (double)metric(kind, s + q, tau, itau) * sc3[q] * sc3[q];
          }
          exp_proj_metric(z3[0], z3[1], z3[2], m3[0], m3[1], m3[2], o);
          for (int q = 0; q < 3; ++q) x[s + q] = T(o[q] * sc3[q]);
          continue;
        }
        if (euclid) exp_proj_euclid((double)x[s], (double)x[s + 1], (double)x[s + 2], o, gs);
        else exp_proj_metric((double)x[s], (double)x[s + 1], (double)x[s + 2], (double)metric(kind, s, tau, itau),
                             (double)metric(kind, s + 1, tau, itau), (double)metric(kind, s + 2, tau, itau), o);
        x[s] = T(o[0]); x[s + 1] = T(o[1]); x[s + 2] = T(o[2]);
        continue;
      }
      const int64_t e = own.p0 + (item - nexp);
      const int64_t s = P.pow_base + 3 * e;
      double o[3];
      const double fx = P.pow_fix ? P.pow_fix[e] : 0.0;
      if (fx > 0.0) {     // slice {(x, f, z): x^a f^{1-a} >= |z|, x >= 0}
        pow_slice_proj((double)x[s], (double)x[s + 2], P.pow_alpha[e], fx, (double)metric(kind, s, tau, itau),
                       (double)metric(kind, s + 2, tau, itau), o,
                       O.warm_roots ? W.root + P.n_soc + P.n_rsoc + P.n_exp + e : nullptr);
        x[s] = T(o[0]); x[s + 1] = T(o[1]); x[s + 2] = T(o[2]);
        continue;
      }
      if (csc) {
        double sc3[3], z3[3], m3[3];
        for (int q = 0; q < 3; ++q) {
          sc3[q] = (double)csc[s + q];
          z3[q] = (double)x[s + q] / sc3[q];
          m3[q] = (double)metric(kind, s + q, tau, itau) * sc3[q] * sc3[q];
        }
        pow_proj(z3[0], z3[1], z3[2], P.pow_alpha[e], m3[0], m3[1], m3[2], o,
                 O.warm_roots ? W.root + P.n_soc + P.n_rsoc + P.n_exp + e : nullptr);
        for (int q = 0; q < 3; ++q) x[s + q] = T(o[q] * sc3[q]);
        continue;
      }
      pow_proj((double)x[s], (double)x[s + 1], (double)x[s + 2], P.pow_alpha[e], (double)metric(kind, s, tau, itau),
               (double)metric(kind, s + 1, tau, itau), (double)metric(kind, s + 2, tau, itau), o,
               O.warm_roots ? W.root + P.n_soc + P.n_rsoc + P.n_exp + e : nullptr);
      x[s] = T(o[0]); x[s + 1] = T(o[1]); x[s + 2] = T(o[2]);
    }
    __syncthreads();
  }

  // Elementwise projection onto the free / nonnegative segments (metric-free, App. A.1)
  __device__ __forceinline__ T proj_elem(int64_t i, T z) const {
    if (i < P.n_free) {
      if (!GEN || !P.xlo) return z;
      const T lo = P.xlo[i], hi = P.xhi[i];   // box bounds (infinite on free coordinates)
      return z < lo ? lo : (z > hi ? hi : z);
    }
    return z > T(0) ? z : T(0);
  }

  // ---- A' products: v = h_x + tau A' h_y on the owned coordinates -----------
  __device__ bool phase_aty(const T* hx, const T* hy, double tau) {
    if (P.tcb_n > 1) {
      // column slices: every block of the team works on the same slice of y (one barrier per
      // slice), so the slice stays in L2 while the entries stream past; a row adds its partial
      // sums in slice order
      T* acc = W.tcb_acc;
      for (int b = 0; b < P.tcb_n; ++b) {
        const bool first = b == 0, last = b == P.tcb_n - 1;
        vals(P.tcb_v, P.tcb_vb, [&](auto tv) {
          for (int seg = 0; seg < 6; ++seg)
            rows_loop_multi<kMultiRows, T>(P.tcb_rp + (int64_t)b * P.n, P.tcb_ci, tv, own.x0[seg], own.x1[seg],
                                           [&](int j) { return hy[j]; }, [&](int64_t i, int gl, T s) {
                                             if (gl != 0) return;
                                             const T t = first ? s : acc[i] + s;
                                             if (last) W.v[i] = hx[i] + T(tau) * t;
                                             else acc[i] = t;
                                           });
        });
        if (!last && !team.sync()) return false;
      }
      __syncthreads();
      return true;
    }
    vals(P.t_v, P.t_vb, [&](auto tv) {
      for (int seg = 0; seg < 6; ++seg) {
        rows_loop_tpr<T>(own.g_t, P.t_rp, P.t_ci, tv, own.x0[seg], own.x1[seg], [&](int j) { return hy[j]; },
                         [&](int64_t i, int gl, T s) {
                           if (gl == 0) W.v[i] = hx[i] + T(tau) * s;
                         });
      }
    });
    __syncthreads();
    return true;
  }

  // ---- one projected (Jacobi-)BB step on the owned coordinates --------------
  // u_next = Pi^J(u_cur - alpha J^{-1} g(u_cur)),   g = Q u + c + (u - v)/tau,
  // with Q u = qd u + R' D t (t = R u_cur, D t in C.w); in sparse-P mode the
  // whole gradient is taken from gs (computed by grad_pass).
  // Accumulates s = u_next - u_cur: v3 = {||s||^2, <s, J s>, sum (qd + 1/tau) s^2,
  // ||u_next||^2} and the block's R u_next in C.rblk.  Per-element work and
  // per-thread partial sums are in the iterate precision T.
  __device__ __forceinline__ const T* wvec() const {
    if constexpr (sizeof(T) == 4) return reinterpret_cast<const T*>(C.wf);
    else return reinterpret_cast<const T*>(C.w);
  }
  __device__ void inner_step(const T* ucur, T* unext, const T* gs, double alpha_d, double tau, T (&v3)[4]) {
    // register width KM = kpad (R is zero-padded to it and D t is zero beyond k)
    if (P.k == 0) inner_step_reg<0>(ucur, unext, gs, alpha_d, tau, v3);
    else if (P.kpad == 8) inner_step_reg<8>(ucur, unext, gs, alpha_d, tau, v3);
    else if (P.kpad == 16) inner_step_reg<16>(ucur, unext, gs, alpha_d, tau, v3);
    else if (P.kpad == 24) inner_step_reg<24>(ucur, unext, gs, alpha_d, tau, v3);
    else if (P.kpad == 32) inner_step_reg<32>(ucur, unext, gs, alpha_d, tau, v3);
    else inner_step_wide(ucur, unext, gs, alpha_d, tau, v3);
  }

  // k <= KM: column i of R is loaded once into registers and serves both the gradient
  // (R' w)_i and the per-thread partials of R u_next (one warp tree per l per pass).
  template <int KM>
  __device__ __noinline__ void inner_step_reg(const T* ucur, T* unext, const T* gs, double alpha_d, double tau,
                                              T (&v3)[4]) {
    const int k = P.k;
    const int64_t n = P.n;
    const T itau = T(1.0 / tau);
    const T alpha = T(alpha_d);
    const bool jac = O.jacobi != 0;
    const T* wr = wvec();            // D t in shared memory (broadcast reads)
    const T* __restrict__ Rm = P.R;
    const T* __restrict__ uc = ucur;
    const T* __restrict__ vv = W.v;
    const T* __restrict__ qd = P.qd;
    const T* __restrict__ cc = P.c;
    const T* __restrict__ jd = P.jd;
    T* __restrict__ un_out = unext;
    T racc[KM > 0 ? KM : 1];
#pragma unroll
    for (int l = 0; l < (KM > 0 ? KM : 1); ++l) racc[l] = T(0);
    auto jm = [&](int64_t i) -> T { return jac ? jd[i] + itau : T(1); };
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    unsigned long long tsub = (O.profile && team.bid() == 0 && threadIdx.x == 0) ? now_ns() : 0ull;
    // elementwise segments (free, nonneg).  Without a low-rank part four elements per thread are
    // loaded together (a streaming pass over n-vectors is otherwise bound by the few loads each
    // of the 16 warps has in flight); the partial sums take the same order as the loop below.
    if constexpr (KM == 0 && sizeof(T) == 4) {
      // FP32: 16-byte loads of four consecutive coordinates, two such chunks in flight per
      // thread (the pass streams five n-vectors; scalar loads leave too few bytes in flight
      // per SM to cover the HBM latency).  Head and tail of a segment off the 4-element grid
      // take the scalar path.
      constexpr int CU = 2;
      const int64_t B = blockDim.x;
      auto elem = [&](int64_t i, T u, T qi, T gv, T cv, T vi, T J) {
        const T g = gs ? gv : qi * u + cv + (u - vi) * itau;
        const T un = proj_elem(i, u - alpha * g / J);
        const T sd = un - u;
        a0 += sd * sd;
        a1 += J * sd * sd;
        a2 += (qi + itau) * sd * sd;
        a3 += un * un;
        return un;
      };
      auto scalar = [&](int64_t i) {
        un_out[i] = elem(i, uc[i], qd[i], gs ? gs[i] : T(0), gs ? T(0) : cc[i], gs ? T(0) : vv[i], jm(i));
      };
      for (int seg = 0; seg < 2; ++seg) {
        const int64_t a = own.x0[seg], b = own.x1[seg];
        const int64_t ah = ((a + 3) & ~int64_t(3)) < b ? ((a + 3) & ~int64_t(3)) : b;
        const int64_t c0 = ah >> 2, c1 = b >> 2 > c0 ? b >> 2 : c0;
        for (int64_t i = a + threadIdx.x; i < ah; i += B) scalar(i);
        for (int64_t i = (c1 << 2) > ah ? (c1 << 2) + threadIdx.x : ah + threadIdx.x; i < b; i += B) scalar(i);
        const float4* __restrict__ u4 = reinterpret_cast<const float4*>(uc);
        const float4* __restrict__ q4 = reinterpret_cast<const float4*>(qd);
        const float4* __restrict__ g4 = reinterpret_cast<const float4*>(gs);
        const float4* __restrict__ c4 = reinterpret_cast<const float4*>(cc);
        const float4* __restrict__ v4 = reinterpret_cast<const float4*>(vv);
        const float4* __restrict__ j4 = reinterpret_cast<const float4*>(jd);
        float4* __restrict__ o4 = reinterpret_cast<float4*>(un_out);
        for (int64_t cq = c0 + threadIdx.x; cq < c1; cq += CU * B) {
          float4 uu[CU], qq[CU], gg[CU], ca[CU], va[CU], jj[CU];
          const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int e = 0; e < CU; ++e) {
            const int64_t c = cq + e * B;
            const bool ok = c < c1;
            uu[e] = ok ? u4[c] : z4;
            qq[e] = ok ? q4[c] : z4;
            gg[e] = (ok && gs) ? g4[c] : z4;
            ca[e] = (ok && !gs) ? c4[c] : z4;
            va[e] = (ok && !gs) ? v4[c] : z4;
            jj[e] = (ok && jac) ? j4[c] : z4;
          }
#pragma unroll
          for (int e = 0; e < CU; ++e) {
            const int64_t c = cq + e * B;
            if (c >= c1) break;
            const T J0 = jac ? jj[e].x + itau : T(1), J1 = jac ? jj[e].y + itau : T(1);
            const T J2 = jac ? jj[e].z + itau : T(1), J3 = jac ? jj[e].w + itau : T(1);
            float4 o;
            o.x = elem(4 * c, uu[e].x, qq[e].x, gg[e].x, ca[e].x, va[e].x, J0);
            o.y = elem(4 * c + 1, uu[e].y, qq[e].y, gg[e].y, ca[e].y, va[e].y, J1);
            o.z = elem(4 * c + 2, uu[e].z, qq[e].z, gg[e].z, ca[e].z, va[e].z, J2);
            o.w = elem(4 * c + 3, uu[e].w, qq[e].w, gg[e].w, ca[e].w, va[e].w, J3);
            o4[c] = o;
          }
        }
      }
    } else if (KM == 0) {
      constexpr int EU = 4;
      const int64_t B = blockDim.x;
      for (int seg = 0; seg < 2; ++seg)
        for (int64_t i0 = own.x0[seg] + threadIdx.x; i0 < own.x1[seg]; i0 += EU * B) {
          T uu[EU], qq[EU], gg[EU], jj[EU], ca[EU], va[EU];
#pragma unroll
          for (int e = 0; e < EU; ++e) {
            const int64_t i = i0 + e * B;
            const bool ok = i < own.x1[seg];
            uu[e] = ok ? uc[i] : T(0);
            qq[e] = ok ? qd[i] : T(0);
            gg[e] = (ok && gs) ? gs[i] : T(0);
            ca[e] = (ok && !gs) ? cc[i] : T(0);
            va[e] = (ok && !gs) ? vv[i] : T(0);
            jj[e] = ok ? jm(i) : T(1);
          }
#pragma unroll
          for (int e = 0; e < EU; ++e) {
            const int64_t i = i0 + e * B;
            if (i >= own.x1[seg]) break;
            const T u = uu[e], qi = qq[e];
            const T g = gs ? gg[e] : qi * u + ca[e] + (u - va[e]) * itau;
            const T J = jj[e];
            const T un = proj_elem(i, u - alpha * g / J);
            un_out[i] = un;
            const T sd = un - u;
            a0 += sd * sd;
            a1 += J * sd * sd;
            a2 += (qi + itau) * sd * sd;
            a3 += un * un;
          }
        }
    } else
    for (int seg = 0; seg < 2; ++seg)
      for (int64_t i = own.x0[seg] + threadIdx.x; i < own.x1[seg]; i += blockDim.x) {
        T rr[KM > 0 ? KM : 1];
        T rw = T(0);
#pragma unroll
        for (int l = 0; l < KM; ++l) {
          rr[l] = __ldg(Rm + (int64_t)l * n + i);
          rw += rr[l] * wr[l];
        }
        const T u = uc[i];
        const T qi = qd[i];
        const T g = gs ? gs[i] : qi * u + cc[i] + (u - vv[i]) * itau + rw;
        const T J = jm(i);
        const T un = proj_elem(i, u - alpha * g / J);
        un_out[i] = un;
        const T sd = un - u;
        a0 += sd * sd;
        a1 += J * sd * sd;
        a2 += (qi + itau) * sd * sd;
        a3 += un * un;
#pragma unroll
        for (int l = 0; l < KM; ++l) racc[l] += rr[l] * un;
      }
    __syncthreads();
    subtick(8, tsub);
    // cone segments: gradient step into unext, then block-local metric projection
    for (int seg = 2; seg < 6; ++seg)
      for (int64_t i = own.x0[seg] + threadIdx.x; i < own.x1[seg]; i += blockDim.x) {
        T rw = T(0);
#pragma unroll
        for (int l = 0; l < KM; ++l) rw += __ldg(Rm + (int64_t)l * n + i) * wr[l];
        const T u = ucur[i];
        const T g = gs ? gs[i] : P.qd[i] * u + P.c[i] + (u - W.v[i]) * itau + rw;
        unext[i] = u - alpha * g / jm(i);
      }
    __syncthreads();
    subtick(9, tsub);
    project_owned_cones(unext, jac ? kJacobi : kEuclid, tau);
    subtick(10, tsub);
    for (int seg = 2; seg < 6; ++seg)
      for (int64_t i = own.x0[seg] + threadIdx.x; i < own.x1[seg]; i += blockDim.x) {
        const T un = unext[i];
        const T sd = un - ucur[i];
        a0 += sd * sd;
        a1 += jm(i) * sd * sd;
        a2 += (P.qd[i] + itau) * sd * sd;
        a3 += un * un;
#pragma unroll
        for (int l = 0; l < KM; ++l) racc[l] += __ldg(Rm + (int64_t)l * n + i) * un;
      }
    if (KM > 0) {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
      for (int l = 0; l < KM; ++l) {
        if (l < k) {
          const T t = warp_sum(racc[l]);
          if (lane == 0) wacc[warp * k + l] = (double)t;
        }
      }
      rblk_from_wacc();
    }
    v3[0] = a0;
    v3[1] = a1;
    v3[2] = a2;
    v3[3] = a3;
    __syncthreads();
    subtick(11, tsub);
  }

  // k > 32: gradient from R row by row, R u_next by the l-major block pass
  __device__ void inner_step_wide(const T* ucur, T* unext, const T* gs, double alpha_d, double tau, T (&v3)[4]) {
    const T itau = T(1.0 / tau);
    const T alpha = T(alpha_d);
    const bool jac = O.jacobi != 0;
    const T* w = wvec();
    auto grad = [&](int64_t i, T u) -> T {
      if (gs) return gs[i];
      return P.qd[i] * u + P.c[i] + (u - W.v[i]) * itau + rtw(i, w);
    };
    auto jm = [&](int64_t i) -> T { return jac ? P.jd[i] + itau : T(1); };
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    for (int seg = 0; seg < 2; ++seg)
      for (int64_t i = own.x0[seg] + threadIdx.x; i < own.x1[seg]; i += blockDim.x) {
        const T u = ucur[i];
        const T J = jm(i);
        const T un = proj_elem(i, u - alpha * grad(i, u) / J);
        unext[i] = un;
        const T sd = un - u;
        a0 += sd * sd;
        a1 += J * sd * sd;
        a2 += (P.qd[i] + itau) * sd * sd;
        a3 += un * un;
      }
    for (int seg = 2; seg < 6; ++seg)
      for (int64_t i = own.x0[seg] + threadIdx.x; i < own.x1[seg]; i += blockDim.x) {
        const T u = ucur[i];
        unext[i] = u - alpha * grad(i, u) / jm(i);
      }
    __syncthreads();
    project_owned_cones(unext, jac ? kJacobi : kEuclid, tau);
    for (int seg = 2; seg < 6; ++seg)
      for (int64_t i = own.x0[seg] + threadIdx.x; i < own.x1[seg]; i += blockDim.x) {
        const T un = unext[i];
        const T sd = un - ucur[i];
        a0 += sd * sd;
        a1 += jm(i) * sd * sd;
        a2 += (P.qd[i] + itau) * sd * sd;
        a3 += un * un;
      }
    rx_lmajor(unext);
    v3[0] = a0;
    v3[1] = a1;
    v3[2] = a2;
    v3[3] = a3;
  }

  // ---- sparse-P mode: gradient at u (P u by the owned rows of P), dots -------
  // writes g(u) to gout; v2 = {<s, dg>} with s = u - uprev, dg = g(u) - gprev
  // The same gradient over rows [r0, r1) with one lane per row and kMultiRows rows in flight
  // (no low-rank part): each row's vector operands are loaded with its entries, ahead of the
  // gathers, instead of after the row sum and behind the previous row's store.  Same
  // arithmetic in the same order as the generic loop.
  template <typename V>
  __device__ T grad_rows_batched(const V* __restrict__ pv, const T* u, const T* uprev, const T* gprev, T* gout, T itau,
                                 bool first, int64_t r0, int64_t r1) {
    constexpr int RB = kMultiRows, U = kMultiU;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5;
    const int ulen = P.p_ulen;
    const int* __restrict__ rp = P.p_rp;
    const int* __restrict__ ci = P.p_ci;
    T acc = T(0);
    for (int64_t base = warp * 32 * RB; base < r1 - r0; base += nwarps * 32 * RB) {
      int beg[RB], end[RB];
      T uu[RB], qq[RB], cc[RB], vv[RB], up[RB], gp[RB], s[RB];
      int len = 0;
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int64_t r = r0 + base + 32 * q + lane;
        const bool ok = r < r1;
        if (ulen > 0) {
          beg[q] = ok ? (int)(ulen * r) : 0;
          end[q] = ok ? beg[q] + ulen : 0;
        } else {
          beg[q] = ok ? rp[r] : 0;
          end[q] = ok ? rp[r + 1] : 0;
        }
        uu[q] = ok ? u[r] : T(0);
        qq[q] = ok ? __ldg(P.qd + r) : T(0);
        cc[q] = ok ? __ldg(P.c + r) : T(0);
        vv[q] = ok ? W.v[r] : T(0);
        up[q] = (ok && !first) ? uprev[r] : T(0);
        gp[q] = (ok && !first) ? gprev[r] : T(0);
        s[q] = T(0);
      }
#pragma unroll
      for (int q = 0; q < RB; ++q) len = max(len, end[q] - beg[q]);
      for (int k = 0; k < len; k += U) {
        int j[RB][U];
        T a[RB][U];
#pragma unroll
        for (int q = 0; q < RB; ++q)
#pragma unroll
          for (int t = 0; t < U; ++t) {
            const int kk = beg[q] + k + t;
            const bool ok = kk < end[q];
            j[q][t] = ok ? __ldg(ci + kk) : -1;
            a[q][t] = ok ? ld_val<T>(pv + kk) : T(0);
          }
        T gth[RB][U];
#pragma unroll
        for (int q = 0; q < RB; ++q)
#pragma unroll
          for (int t = 0; t < U; ++t) gth[q][t] = j[q][t] >= 0 ? u[j[q][t]] : T(0);
#pragma unroll
        for (int q = 0; q < RB; ++q)
#pragma unroll
          for (int t = 0; t < U; ++t) s[q] += a[q][t] * gth[q][t];
      }
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int64_t r = r0 + base + 32 * q + lane;
        if (r < r1) {
          const T g = s[q] + qq[q] * uu[q] + cc[q] + (uu[q] - vv[q]) * itau;
          gout[r] = g;
          if (!first) acc += (uu[q] - up[q]) * (g - gp[q]);
        }
      }
    }
    return acc;
  }

  // The same for FP32 iterates and rows of exactly ulen entries, four consecutive rows per thread:
  // 16-byte loads of the row vectors and of the rows' entries (ulen = 2: eight entries, two int4
  // and two float4 or one uint4 of BF16), the gathers and the store of g likewise four at a time.
  // Rows off the 4-row grid at either end of the range take grad_rows_batched.  Each row's sum is
  // in storage order, as there.
  template <typename V>
  __device__ T grad_rows_vec4(const V* __restrict__ pv, const T* u, const T* uprev, const T* gprev, T* gout, T itau,
                              bool first, int64_t r0, int64_t r1) {
    const int ulen = P.p_ulen;
    const int64_t rh = ((r0 + 3) & ~int64_t(3)) < r1 ? ((r0 + 3) & ~int64_t(3)) : r1;
    const int64_t c0 = rh >> 2, c1 = (r1 >> 2) > c0 ? (r1 >> 2) : c0;
    T acc = grad_rows_batched(pv, u, uprev, gprev, gout, itau, first, r0, rh);
    acc += grad_rows_batched(pv, u, uprev, gprev, gout, itau, first, (c1 << 2) > rh ? (c1 << 2) : rh, r1);
    const int* __restrict__ ci = P.p_ci;
    const float4* __restrict__ u4 = reinterpret_cast<const float4*>(u);
    const float4* __restrict__ q4 = reinterpret_cast<const float4*>(P.qd);
    const float4* __restrict__ cc4 = reinterpret_cast<const float4*>(P.c);
    const float4* __restrict__ v4 = reinterpret_cast<const float4*>(W.v);
    const float4* __restrict__ up4 = reinterpret_cast<const float4*>(uprev);
    const float4* __restrict__ gp4 = reinterpret_cast<const float4*>(gprev);
    float4* __restrict__ g4 = reinterpret_cast<float4*>(gout);
    for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
      const float4 uu = u4[c], qq = q4[c], cv = cc4[c], vv = v4[c];
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 up = first ? z4 : up4[c], gp = first ? z4 : gp4[c];
      const int64_t base = (int64_t)ulen * 4 * c;
      float sr[4] = {0.f, 0.f, 0.f, 0.f};
      if (ulen == 2) {
        const int4 ja = reinterpret_cast<const int4*>(ci + base)[0], jb = reinterpret_cast<const int4*>(ci + base)[1];
        float a[8];
        if constexpr (std::is_same<V, __nv_bfloat16>::value) {
          const uint4 w = *reinterpret_cast<const uint4*>(pv + base);
          const unsigned ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            a[2 * t] = __uint_as_float(ws[t] << 16);
            a[2 * t + 1] = __uint_as_float(ws[t] & 0xFFFF0000u);
          }
        } else {
          const float4 pa = reinterpret_cast<const float4*>(pv + base)[0], pb = reinterpret_cast<const float4*>(pv + base)[1];
          a[0] = pa.x; a[1] = pa.y; a[2] = pa.z; a[3] = pa.w; a[4] = pb.x; a[5] = pb.y; a[6] = pb.z; a[7] = pb.w;
        }
        const int j[8] = {ja.x, ja.y, ja.z, ja.w, jb.x, jb.y, jb.z, jb.w};
        float gv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) gv[t] = u[j[t]];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          sr[q] += a[2 * q] * gv[2 * q];
          sr[q] += a[2 * q + 1] * gv[2 * q + 1];
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          for (int t = 0; t < ulen; ++t) {
            const int64_t e = base + (int64_t)q * ulen + t;
            sr[q] += ld_val<float>(pv + e) * u[__ldg(ci + e)];
          }
      }
      const float uq[4] = {uu.x, uu.y, uu.z, uu.w}, qv[4] = {qq.x, qq.y, qq.z, qq.w}, cq[4] = {cv.x, cv.y, cv.z, cv.w};
      const float vq[4] = {vv.x, vv.y, vv.z, vv.w}, pq[4] = {up.x, up.y, up.z, up.w}, gq[4] = {gp.x, gp.y, gp.z, gp.w};
      float go[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        go[q] = sr[q] + qv[q] * uq[q] + cq[q] + (uq[q] - vq[q]) * itau;
        if (!first) acc += (uq[q] - pq[q]) * (go[q] - gq[q]);
      }
      g4[c] = make_float4(go[0], go[1], go[2], go[3]);
    }
    return acc;
  }

  __device__ void grad_pass(const T* u, const T* uprev, const T* gprev, T* gout, double tau, double (&v2)[2],
                            bool first) {
    const T itau = T(1.0 / tau);
    const T* w = wvec();
    T acc = T(0);
    if (own.g_p == kRowsBatched && P.k == 0) {
      vals(P.p_v, P.p_vb, [&](auto pv) {
        for (int seg = 0; seg < 6; ++seg) {
          if constexpr (sizeof(T) == 4) {
            if (P.p_ulen > 0) {
              acc += grad_rows_vec4(pv, u, uprev, gprev, gout, itau, first, own.x0[seg], own.x1[seg]);
              continue;
            }
          }
          acc += grad_rows_batched(pv, u, uprev, gprev, gout, itau, first, own.x0[seg], own.x1[seg]);
        }
      });
      v2[0] = (double)acc;
      v2[1] = 0.0;
      __syncthreads();
      return;
    }
    for (int seg = 0; seg < 6; ++seg) {
      vals(P.p_v, P.p_vb, [&](auto pv) {
        rows_loop_tpr<T>(own.g_p, P.p_rp, P.p_ci, pv, own.x0[seg], own.x1[seg], [&](int j) { return u[j]; },
                         [&](int64_t i, int gl, T pu) {
                           if (gl == 0) {
                             T g = pu + P.qd[i] * u[i] + P.c[i] + (u[i] - W.v[i]) * itau;
                             if (P.k > 0) g += rtw(i, w);
                             gout[i] = g;
                             if (!first) acc += (u[i] - uprev[i]) * (g - gprev[i]);
                           }
                         },
                         P.p_ulen);
      });
    }
    v2[0] = (double)acc;
    v2[1] = 0.0;
    __syncthreads();
  }

  // ---- the main loop ---------------------------------------------------------
  __device__ void run(long long budget);
  __device__ bool prox_bb(const T* hx, int& ubuf);
  __device__ bool prox_diag(const T* hx);
  __device__ bool kkt(const T* x, const T* y, bool have_rx);
  __device__ void ctl_pid_restart(double dxn, double dyn);
};

}  // namespace cqp
