/*
 * Plain FP64 CPU oracle for restarted reflected-Halpern / averaged PDHG on
 *     min 1/2 x'Qx + c'x   s.t.  A x = b,  x in K.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load or call this library.  It shares no
 * code, header or table with the CUDA library; the two meet only through the
 * seeded instances of the `instances` package.
 *
 * Everything here is written for clarity, not speed: single thread, FP64,
 * straightforward loops, bisection for every scalar root.
 *
 * Pins (tests/test_oracle_*.py): products against dense / exact integer
 * results, every projection against its KKT certificate, brute force and
 * closed forms, the PDHG step against the resolvent identity and Fejer /
 * Halpern bounds, whole solves against closed-form optima, and the control
 * rules of orc_solve (adaptive restart, PID primal weight, adaptive inner
 * tolerance) against hand-computed cases of their printed formulas with the
 * constants of Table practical-defaults (orc_restart_rule, orc_pid_update,
 * orc_inner_tol are the functions orc_solve calls).
 */
#ifndef CQP_ORACLE_H
#define CQP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Cone block types (a block is a contiguous slice of x). */
enum { ORC_FREE = 0, ORC_NONNEG = 1, ORC_SOC = 2, ORC_RSOC = 3, ORC_EXP = 4, ORC_POW = 5, ORC_BOX = 6,
       /* slices with the middle coordinate fixed (Sec. 5.4, eq. fisher-conic and the coordinate
        * count after it: each buyer's (z_i, 1, t_i) is one stored 3-D block with the middle entry
        * held at one and no affine row for it):
        * EXP1 = {(r, f, t): f exp(r/f) <= t}, POW1 = {(x, f, z): x^a f^(1-a) >= |z|, x >= 0},
        * f = blk_fix of the block (1 when blk_fix is NULL); convex sets, not cones */
       ORC_EXP1 = 7, ORC_POW1 = 8 };

typedef struct {
  int64_t m, n;
  /* A in CSR (m rows) */
  const int64_t* a_rowptr; const int64_t* a_colind; const double* a_val;
  /* Q = diag(q_diag) + P + R' D R; any part may be NULL / zero-sized */
  const double* q_diag;                                   /* n or NULL */
  const int64_t* p_rowptr; const int64_t* p_colind; const double* p_val;  /* n x n or NULL */
  int64_t q_rank; const double* q_R; const double* q_D;   /* R: rank x n row-major, D: rank x rank */
  const double* c; const double* b;
  int64_t nblocks;
  const int32_t* blk_type; const int64_t* blk_start; const int64_t* blk_dim; const double* blk_alpha;
  /* general form (solver-input of Sec. 4): row_lo <= A x <= row_hi (NULL: A x = b) and,
   * on ORC_BOX blocks, x_lo <= x <= x_hi (n entries, read on box coordinates only);
   * infinite entries mean no bound */
  const double* row_lo; const double* row_hi; const double* x_lo; const double* x_hi;
  /* per block: the fixed middle coordinate f of ORC_EXP1 / ORC_POW1 blocks (NULL: f = 1) */
  const double* blk_fix;
} orc_problem;

typedef struct {
  int ruiz_iters;        /* 10 */
  double pc_alpha;       /* 1.0; < 0 disables Pock-Chambolle */
  int bound_obj;         /* 1 */
  double eps0_in, gamma_in, eps_min_in;   /* 1e-3, 5e-4, 1e-9 */
  int jacobi;            /* 1: Jacobi-metric BB, 0: Euclidean BB */
  double rho;            /* reflection coefficient, 1.0 */
  double beta_s, beta_n, beta_a;          /* 0.2, 0.8, 0.36 */
  double beta_I, K_P, K_I, K_D;           /* 0.3, 0.99, 0.01, 0.0 */
  int check_every;       /* 64 */
  int64_t max_iter;      /* outer iteration cap */
  int max_inner;         /* 1000 */
  double tol;            /* 1e-4 relative KKT */
  int update;            /* 0 reflected Halpern, 1 Cesaro averaged */
  int avg_epoch;         /* epoch length T of the averaged variant */
  int power_iters;       /* 200 */
  double power_tol;      /* 1e-6 */
  double step_factor;    /* 0.998 */
  int force_inner;       /* 1: always use the BB inner solver even for diagonal Q */
  int pid;               /* 1: primal-weight PID at restarts */
  int hist_cap;          /* capacity of the history arrays in orc_info */
  int rescaled_cones;    /* 0: cone-preserving block scaling (eq. cone-preserving-scaling);
                            1: rescaled-cone mode, coordinatewise factors on cone blocks and
                            projections onto S_j K_j (eq. scaling-induced-metric) */
} orc_options;

typedef struct {
  double eps_p, eps_d, eps_g, rel_kkt;
  double pobj, dobj;
  double norm_res_p, norm_res_d;
} orc_kkt_report;

typedef struct {
  int status;            /* 0 converged, 1 iteration limit */
  int64_t iters, restarts, inner_total;
  double eta, norm_A, omega;
  double beta_b, beta_c;
  orc_kkt_report kkt;
  /* history, one entry per KKT check (caller-owned arrays of hist_cap or NULL) */
  int hist_len;
  int64_t* hist_iter; double* hist_kkt; double* hist_gap; double* hist_E; int32_t* hist_restart;
} orc_info;

void orc_default_options(orc_options* o);

/* threads of the OpenMP build (liboracle_omp.so; no effect in the single-threaded build) and the
 * number a parallel loop will use (1 in the single-threaded build) */
void orc_set_threads(int t);
int orc_max_threads(void);

/* sparse products */
void orc_spmv(int64_t m, const int64_t* rowptr, const int64_t* colind, const double* val,
              const double* x, double* y);
void orc_spmv_t(int64_t m, int64_t n, const int64_t* rowptr, const int64_t* colind, const double* val,
                const double* y, double* out);
void orc_q_apply(const orc_problem* p, const double* x, double* out);

/* projections: metric m (diagonal, same length as the block) may be NULL for Euclidean */
int orc_proj_block(int type, int64_t dim, double alpha, const double* r, const double* m, double* out);
void orc_proj_product(const orc_problem* p, const double* r, const double* m, double* out);
/* projection onto the rescaled cone S K, S = diag(sc) > 0, in the diagonal metric m
 * (NULL: Euclidean): S Pi_K^{S m S}(S^-1 r) (eq. scaling-induced-metric) */
int orc_proj_block_scaled(int type, int64_t dim, double alpha, const double* sc, const double* r, const double* m,
                          double* out);
/* projection onto the slice ORC_EXP1 / ORC_POW1 with middle coordinate f > 0 in the diagonal
 * metric m (NULL: Euclidean); out[1] = f.  Returns -1 for a bad type, dim, alpha or f. */
int orc_proj_slice(int type, double alpha, double f, const double* r, const double* m, double* out);
/* 1 if r lies in the block's cone (tol absolute slack), for tests; slices use f = 1 */
int orc_in_cone(int type, int64_t dim, double alpha, const double* r, double tol);
int orc_in_dual_cone(int type, int64_t dim, double alpha, const double* r, double tol);

/* KKT report of (x, y) on the problem as given */
void orc_kkt(const orc_problem* p, const double* x, const double* y, orc_kkt_report* rep);

/* setup stages, exposed for parity: scaled copies are written into the out arrays
 * (A values in CSR order of the input, c, b, q_diag, R) plus the scaling vectors. */
void orc_rescale(const orc_problem* p, const orc_options* o,
                 double* col_scale, double* row_scale, double* beta_bc,
                 double* a_val_out, double* c_out, double* b_out);
/* largest eigenvalue of the symmetric tridiagonal matrix with diagonal a[0..k) and
 * off-diagonal b[0..k-1) (the Lanczos step of orc_norm_est), by Sturm bisection */
double orc_tridiag_max_eig(const double* a, const double* b, int k);
/* the unnormalised start vector of orc_norm_est: entry j = 1/2 + (top 53 bits of SplitMix64
 * output j+1 from state 0) / 2^53 */
void orc_power_start(int64_t n, double* out);
double orc_norm_est(int64_t m, int64_t n, const int64_t* rowptr, const int64_t* colind, const double* val,
                    int iters, double tol, int* iters_used);

/* one primal-first PDHG operator evaluation on the problem as given (no scaling):
 * x+ = prox_{tau F}(x + tau A'y) solved to tolerance eps_in, y+ = y + sigma (b - A(2x+ - x)).
 * Returns inner iterations used. */
int orc_pdhg_operator(const orc_problem* p, double tau, double sigma, const double* x, const double* y,
                      double eps_in, int max_inner, int jacobi, int force_inner,
                      double* x_out, double* y_out);
/* one prox evaluation p = argmin_{u in K} 1/2 u'Qu + c'u + ||u - v||^2/(2 tau), from u0 */
int orc_prox(const orc_problem* p, double tau, const double* v, const double* u0, double eps_in,
             int max_inner, int jacobi, int force_inner, double* u_out);

/* Control rules of orc_solve, exposed so that they can be pinned on hand-computed cases.
 * orc_restart_rule: 1 if eq. practical-restart-rule restarts at epoch step k >= 1 with fixed-point
 *   errors E = E_{n,k}, E0 = E_{n,0}, Eprev = E at the previous check of the epoch (E0 at its first),
 *   k the epoch's iteration count and ktot the cumulative count; 0 at k = 0.
 * orc_pid_update: eqs. pid-error / pid-weight at a restart with movements dx = ||w_x - x^{n,0}||,
 *   dy = ||w_y - y^{n,0}||; state[0] = I_{n-1}, state[1] = e_{n-1} are updated in place; returns
 *   omega_{n+1}.  Reading: omega is kept (and the state untouched) when o->pid is 0 or a movement
 *   is <= 1e-10.
 * orc_inner_tol: eq. monotone-primal-inner-tol, the tolerance of step k >= 1 from the previous one,
 *   the movement mov = ||x^{n,k} - x^{n,k-1}|| and tau. */
int orc_restart_rule(double E, double E0, double Eprev, int64_t k, int64_t ktot, const orc_options* o);
double orc_pid_update(double omega, double dx, double dy, const orc_options* o, double* state);
double orc_inner_tol(double eps_prev, double mov, double tau, const orc_options* o);

/* full solve; x_out (n), y_out (m) receive the unscaled final candidate.  Returns 0 (converged),
 * 1 (iteration limit) or -1 (invalid problem: a slice block with a non-positive blk_fix) */
int orc_solve(const orc_problem* p, const orc_options* o, const double* x0, const double* y0,
              double* x_out, double* y_out, orc_info* info);

#ifdef __cplusplus
}
#endif
#endif
