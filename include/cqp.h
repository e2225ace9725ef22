/*
 * cqp.h — C ABI of the GB300 conic-QP PDHG library (libcqp_gb300.so).
 *
 * Problem (paper, Sec. 1, eq. "cqp"):
 *     min_x  1/2 x'Qx + c'x   s.t.  A x = b,  x in K = K_1 x ... x K_J,
 * solved by restarted reflected-Halpern PDHG (Alg. "pdhcq1", uncompiled branch,
 * and Sec. 4.2.1 eq. "rh-update") or restarted Cesaro-averaged PDHG (Alg.
 * "pdhcq1", compiled branch), with the practical components of Sec. 4
 * (rescaling Sec. 4.2.2, adaptive inner accuracy Sec. 4.2.3, Jacobi projected
 * BB Sec. 4.2.4 / eq. "jacobi-bb-step", diagonal-Q metric projection eq.
 * "diagonal-q-metric", step sizes eq. "practical-stepsizes", PID primal weight
 * eqs. "pid-error"/"pid-weight", adaptive restart eq. "practical-restart-rule",
 * defaults Table "practical-defaults").  K is a product of free, nonnegative,
 * second-order, rotated second-order, exponential and 3-D power cones
 * (Sec. 4 standard form, eq. "solver-input", equality rows only).
 *
 * Conventions shared by every entry point:
 *  - All functions return an int status: 0 = success, > 0 = solver outcome
 *    (iteration or time limit), < 0 = error (see CQP_ERR_*).  No C++ exception
 *    crosses this boundary and nothing aborts the process.
 *  - Input arrays are borrowed for the duration of the call and never retained;
 *    the library copies what it keeps.  Output arrays are caller-owned.
 *  - "device" pointers are CUDA global-memory pointers of the current device;
 *    "host" pointers are ordinary (preferably pinned) host memory.  Each entry
 *    point states which it expects.
 *  - A stream argument (cudaStream_t passed as void*) may be NULL for the
 *    default stream.  Entry points that return results to the host
 *    synchronise that stream before returning.  A handle allocates and frees
 *    its device memory in order on its stream (opt->stream), so that stream
 *    must outlive the handle.
 *  - Device memory comes from a memory pool the library keeps per device;
 *    memory freed by the library stays reserved for its later allocations
 *    until the process exits (repeated set-ups then cost no driver calls).
 *  - The library needs a GB300 (sm_103a); on any CUDA error the call returns
 *    CQP_ERR_CUDA and cqp_last_error() describes it.
 */
#ifndef CQP_GB300_H
#define CQP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define CQP_OK 0
#define CQP_ITER_LIMIT 1          /* max_iter reached before rel-KKT <= tol */
#define CQP_TIME_LIMIT 2          /* time_limit_s reached */
#define CQP_ERR_INVALID (-1)      /* bad sizes, partition, cone parameters, non-finite data */
#define CQP_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define CQP_ERR_OOM (-3)          /* device allocation failed */
#define CQP_ERR_NUMERICAL (-4)    /* NaN/Inf detected in the FP64 reductions */
#define CQP_ERR_WAIT (-5)         /* a bounded device-side wait expired (grid barrier) */
#define CQP_ERR_UNSUPPORTED (-6)  /* option combination not implemented */

/* ---- cone types (Sec. 4, after eq. "solver-input") ------------------ */
#define CQP_CONE_FREE 0    /* R^d (box with infinite bounds) */
#define CQP_CONE_NONNEG 1  /* R^d_+ */
#define CQP_CONE_SOC 2     /* {(v, t): ||v||_2 <= t}, t is the LAST coordinate, d >= 2 */
#define CQP_CONE_RSOC 3    /* {(v, s, t): ||v||^2 <= 2 s t, s, t >= 0}, s, t last, d >= 3 */
#define CQP_CONE_EXP 4     /* cl{(r, s, t): s > 0, s exp(r/s) <= t}, d = 3 */
#define CQP_CONE_POW 5     /* {(r, s, t): r, s >= 0, r^a s^(1-a) >= |t|}, d = 3, 0 < a < 1 */
#define CQP_CONE_BOX 6     /* {x: x_lo <= x <= x_hi} coordinatewise (cqp_setup_general only), d >= 1 */
/* Slices with the middle coordinate fixed at one (Sec. 5.4, eq. "fisher-conic" and the
 * coordinate count after it: each buyer's (z, 1, t) is a stored 3-D block with no affine
 * row for the one).  Convex sets, not cones; d = 3; the middle entry of x is always 1.
 * Not available in batched mode or with rescaled_cones = 1 (CQP_ERR_UNSUPPORTED).  The KKT
 * report adds inf over the slice of s'x to the dual objective and counts the part of the
 * slack s outside that term's domain as dual residual (exp: s_r <= 0 <= s_t; pow: s_r >= 0). */
#define CQP_CONE_EXP1 7    /* {(r, 1, t): exp(r) <= t} */
#define CQP_CONE_POW1 8    /* {(r, 1, t): r >= 0, r^a >= |t|}, 0 < a < 1 */

/* CSR matrix.  rowptr has nrows+1 entries (int64, rowptr[0] = 0), colind and
 * val have nnz entries; colind in [0, ncols).  nnz must be < 2^31. */
typedef struct {
  int64_t nrows, ncols, nnz;
  const int64_t* rowptr;
  const int32_t* colind;
  const double* val;
} cqp_csr;

/* Structured Q = diag(q) + P + R' D R (Sec. 4.1, "Products with a structured
 * operator"), never formed.  Any part may be absent: diag = NULL, P.rowptr =
 * NULL, rank = 0.  P is n x n symmetric; R is rank x n row-major; D is
 * rank x rank row-major symmetric.  rank <= 64.  Q must be positive
 * semidefinite (not checked). */
typedef struct {
  const double* diag;
  cqp_csr P;
  int64_t rank;
  const double* R;
  const double* D;
} cqp_qop;

/* Cone blocks: nblocks contiguous slices (start, dim) that partition 0..n-1
 * in increasing order; alpha is used by CQP_CONE_POW and CQP_CONE_POW1 only. */
typedef struct {
  int64_t nblocks;
  const int32_t* type;
  const int64_t* start;
  const int64_t* dim;
  const double* alpha;
} cqp_cones;

typedef struct {
  /* arithmetic */
  int32_t precision;        /* 0: FP32 iterates, matrices and SOC roots; FP64 reductions and RSOC/exp/pow roots; 1: all FP64 */
  int32_t update;           /* 0: reflected Halpern (eq. "rh-update"); 1: Cesaro averaged (Alg. "pdhcq1") */
  double rho;               /* reflection coefficient, default 1.0 */
  /* rescaling (Table "practical-defaults") */
  int32_t ruiz_iters;       /* 10 */
  double pc_alpha;          /* 1.0; < 0 disables Pock-Chambolle */
  int32_t bound_obj;        /* 1 */
  int32_t rescaled_cones;   /* 0: cone-preserving block scaling (eq. "cone-preserving-scaling", default);
                               1: rescaled-cone mode, coordinatewise factors on cone blocks, each block
                               projected onto S_j K_j (eq. "scaling-induced-metric"); not in batched mode */
  /* inner solver */
  double eps0_in, gamma_in, eps_min_in;   /* 1e-3, 5e-4, 1e-9 */
  int32_t jacobi;           /* 1 */
  int32_t max_inner;        /* 1000 */
  int32_t force_inner;      /* 1: projected BB even for diagonal Q */
  /* restart / primal weight */
  double beta_s, beta_n, beta_a;          /* 0.2, 0.8, 0.36 */
  double beta_I, K_P, K_I, K_D;           /* 0.3, 0.99, 0.01, 0.0 */
  int32_t pid;              /* 1 */
  int32_t avg_epoch;        /* epoch length of the averaged variant, 64 */
  /* termination */
  double tol;               /* 1e-4 relative KKT */
  int64_t max_iter;         /* outer iterations, 100000 */
  int32_t check_every;      /* KKT / restart check cadence, 64 */
  double time_limit_s;      /* <= 0: none */
  /* step size */
  int32_t power_iters;      /* 200: cap on the Lanczos steps of the ||A~||_2 estimate (at most 256 on the GPU) */
  double power_tol;         /* 1e-6 */
  double step_factor;       /* 0.998 */
  /* execution */
  int32_t input_on_device;  /* 1: every input pointer of cqp_setup is a device pointer */
  int32_t team;             /* 0 auto (n + m > 4096: 1, else 3 where a cluster fits, else 2), 1 whole-GPU
                               cooperative kernel, 2 one thread block, 3 one thread-block cluster of up to
                               16 CTAs (cluster barriers, distributed-shared-memory reductions) */
  int32_t threads;          /* threads per block, 0 = auto */
  int32_t blocks_per_sm;    /* 0 = auto (cooperative team only) */
  int32_t tpr_a, tpr_at, tpr_p; /* threads per CSR row for A, A' and the sparse part P of Q (1..32), -1 = one
                               lane per row with four rows in flight (P: with 16-byte loads of four rows
                               when its rows all have the same length), 0 = autotuned among these (timed
                               per matrix shape, cached) */
  int32_t launch_iters;     /* outer iterations per kernel launch, 0 = auto */
  int32_t profile;          /* 1: record per-phase device time in cqp_result.phase_ms */
  int32_t warm_roots;       /* 1: start each cone block's root-finding from its previous root (default 1) */
  int32_t col_blocks;       /* sparse products over column slices whose slice of the gathered vector stays
                               in L2: the dual step's A z (0 auto: 8 slices when z exceeds 64 MB) and the
                               A'y pass (0 auto: slices of at most 100 MB of y when y exceeds 64 MB);
                               1 off; K >= 2 forces K slices for both (<= 64) */
  int32_t matrix_bf16;      /* 1: BF16-stored values of A and A'; 2: of A, A' and the sparse part P of Q.
                               FP32 accumulation; precision 0, single problems, whole-GPU team only.  The
                               stored values are rounded to BF16 at setup (to FP32, then to BF16,
                               nearest-even each): the problem solved and reported by cqp_kkt is the one
                               with those rounded values.  With 2 the caller must know the rounded P is
                               still positive semidefinite: it is when P is diagonal or a weighted graph
                               Laplacian (both signs of a weight round alike), not in general (entrywise
                               rounding of a matrix with small eigenvalues can make it indefinite).  The
                               cumulative Ruiz and Pock-Chambolle factors and the bound-objective factors
                               are rounded to powers of two, so the scaled values stay exactly
                               representable.  0 (default): values
                               in the iterate precision */
  void* stream;             /* cudaStream_t, NULL = default stream */
} cqp_options;

typedef struct {
  double eps_p, eps_d, eps_g, rel_kkt;    /* relative primal, dual, gap residuals and their max */
  double pobj, dobj;                      /* primal and dual objective values */
  double norm_res_p, norm_res_d;          /* ||Ax - b||_2, ||Pi_K(-s)||_2 with s = Qx + c - A'y */
} cqp_kkt_report;

typedef struct {
  int32_t status;
  int64_t iters, restarts, inner_total, kernel_launches;
  cqp_kkt_report kkt;
  double eta, norm_A, omega;
  double setup_ms, solve_ms;
  /* with opt.profile: device time (block 0) per phase of the iteration: A'y product,
   * prox work, prox barriers, dual step, its barrier, KKT checks, restart/Halpern at
   * checks, whole loop; then the inner BB step split into its elementwise part, cone
   * gradient, cone projection and cone bookkeeping; then the dual step split into the
   * z = 2 w_x - h_x pass (with its barrier), the row products (with the barriers between
   * column slices) and the Halpern update of x; the last entry is unused */
  double phase_ms[16];
  double kernel_ms;                /* CUDA-event time of the solver kernel launches of this solve */
  int64_t setup_launches;          /* kernels launched by cqp_setup for this handle */
} cqp_result;

typedef struct cqp_handle cqp_handle;

/* Fills *opt with the defaults listed above.  Returns CQP_OK. */
int cqp_default_options(cqp_options* opt);

/* Builds the device-resident, rescaled problem (Sec. 4.2.2 rescaling and
 * eq. "practical-stepsizes": Ruiz, Pock-Chambolle and bound-objective scaling,
 * Lanczos estimate of ||A||_2, eta = step_factor/||A||_2).
 *   A: m x n equality matrix; Q: objective operator (NULL = 0); c: n; b: m;
 *   K: cone partition of 0..n-1; opt: NULL = defaults.
 * Pointers are host pointers unless opt->input_on_device = 1.  On success
 * *out owns all device memory of the problem until cqp_free.
 * Errors: CQP_ERR_INVALID (sizes, partition not contiguous/covering, SOC dim
 * < 2, RSOC dim < 3, EXP/POW dim != 3, alpha outside (0,1), rank > 64, nnz >=
 * 2^31, non-finite values), CQP_ERR_OOM, CQP_ERR_CUDA; *out is NULL then. */
int cqp_setup(const cqp_csr* A, const cqp_qop* Q, const double* c, const double* b, const cqp_cones* K,
              const cqp_options* opt, cqp_handle** out);

/* General standard form (Sec. 4, eq. "solver-input"):
 *     min 1/2 x'Qx + c'x   s.t.  row_lo <= A x <= row_hi,  x in K,
 * where K may also hold CQP_CONE_BOX blocks x_lo <= x <= x_hi.  Infinite entries mean
 * no bound; equal finite entries make an equality row.  Arrays follow
 * opt->input_on_device like the other inputs; row_lo, row_hi have m entries (required
 * when m > 0); x_lo, x_hi have n entries, read on box coordinates only (required when
 * a box block exists).  Not available in batched mode. */
typedef struct {
  const double* row_lo;
  const double* row_hi;
  const double* x_lo;
  const double* x_hi;
} cqp_bounds;

/* As cqp_setup for the general form.  The dual step becomes the prox of the support
 * function of [row_lo, row_hi] (y+ = y - sigma v + sigma Pi_[lo,hi](v - y/sigma),
 * v = A(2x+ - x)), box coordinates are clipped in every projection, and the KKT report
 * measures the distance of Ax to [row_lo, row_hi], adds the support terms to the dual
 * objective and their sign conditions to the dual residual.  Errors as cqp_setup, plus
 * CQP_ERR_INVALID for NaN bounds or lo > hi. */
int cqp_setup_general(const cqp_csr* A, const cqp_qop* Q, const double* c, const cqp_bounds* bounds,
                      const cqp_cones* K, const cqp_options* opt, cqp_handle** out);

/* Runs the restarted PDHG loop on the GPU until rel-KKT <= tol (checked on the
 * unscaled candidate every check_every iterations, Sec. 4.2.2 last paragraph),
 * max_iter, or time_limit_s.
 *   x0 (n), y0 (m): optional warm start (NULL = zeros), unscaled.
 *   x_out (n), y_out (m): caller-owned, receive the unscaled final candidate
 *   (may be NULL).  All four are host pointers, or device pointers when
 *   on_device = 1.  res: optional, filled on return.
 * Returns CQP_OK, CQP_ITER_LIMIT, CQP_TIME_LIMIT or an error code. */
int cqp_solve(cqp_handle* h, const double* x0, const double* y0, double* x_out, double* y_out, int32_t on_device,
              cqp_result* res);

/* FP64 KKT report (eq. "kkt-cqp" measured relative to ||b||, ||c||) of the
 * unscaled point (x, y) on the handle's problem, computed on the GPU.
 * x (n), y (m): host pointers, or device pointers when on_device = 1. */
int cqp_kkt(cqp_handle* h, const double* x, const double* y, int32_t on_device, cqp_kkt_report* rep);

/* Releases every resource of h (NULL is allowed). */
void cqp_free(cqp_handle* h);

/* Text for a status code; the last CUDA or validation error of this thread. */
const char* cqp_status_string(int status);
const char* cqp_last_error(void);

/* Number of kernels this library has launched from the calling thread so far
 * (setup, solver, KKT and kernel-level entry points). */
long long cqp_kernel_launches(void);

/* ---- batched solve of many independent problems (one persistent launch) ----
 * Thousands of small, uneven problems are passed as ONE block-diagonal problem:
 * instance i owns the coordinates [x_off[i], x_off[i+1]) and the rows
 * [row_off[i], row_off[i+1]).  Every entry of A and of P must join a row and a
 * column of the same instance, and every cone block must lie inside one
 * instance's coordinates (checked; CQP_ERR_INVALID otherwise).  The low-rank part
 * R'DR acts per instance: instance i's R u sums only over its own columns, so R
 * holds the instances' factors side by side (rows beyond an instance's rank are
 * zero on its columns) and D is shared.
 * Each instance is rescaled, gets its own ||A_i||_2, step sizes, primal weight,
 * restarts, inner tolerance and stop test (rel-KKT of the instance, normalised
 * by its own ||b_i||, ||c_i||), i.e. it follows the method of cqp_solve as if it
 * were solved alone (Alg. pdhcq1, Sec. 4).  The solve is one launch: one thread
 * block per SM takes instances from a work queue, largest first, and solves each
 * with block-level barriers only. */
typedef struct {
  int64_t count;             /* number of instances (>= 1) */
  const int64_t* x_off;      /* host array, count+1 entries, x_off[0] = 0, x_off[count] = n, increasing */
  const int64_t* row_off;    /* host array, count+1 entries, row_off[0] = 0, row_off[count] = m, non-decreasing */
} cqp_batch;

typedef struct {
  int32_t status;            /* CQP_OK, CQP_ITER_LIMIT, CQP_TIME_LIMIT or CQP_ERR_NUMERICAL */
  int64_t iters, restarts, inner_total;
  cqp_kkt_report kkt;        /* of the instance's returned point, relative to its own ||b_i||, ||c_i|| */
} cqp_instance_result;

/* As cqp_setup, for a batch.  opt->team, blocks_per_sm and launch_iters are
 * ignored (the batch always runs one block per instance at a time). */
int cqp_setup_batch(const cqp_csr* A, const cqp_qop* Q, const double* c, const double* b, const cqp_cones* K,
                    const cqp_batch* B, const cqp_options* opt, cqp_handle** out);

/* Solves every instance of a handle made by cqp_setup_batch.  x0, y0, x_out,
 * y_out as in cqp_solve (whole block-diagonal vectors).  per_instance: optional
 * caller-owned array of B->count results.  res: optional summary (status = the
 * worst instance status, iters = max over instances, restarts and inner_total =
 * sums, kkt = the instance with the largest rel_kkt, kernel_ms of the launch).
 * time_limit_s bounds the whole launch: instances still running when it expires
 * stop with CQP_TIME_LIMIT. */
int cqp_solve_batch(cqp_handle* h, const double* x0, const double* y0, double* x_out, double* y_out,
                    int32_t on_device, cqp_instance_result* per_instance, cqp_result* res);

/* ---- kernel-level entry points (device pointers, used for parity and
 * bandwidth measurements).  `precision` selects FP32 (0) or FP64 (1) data:
 * val/x/y are float* or double* accordingly.  rowptr/colind are int32. ---- */

/* y = A x with the CSR kernel of the solver (threads_per_row: 1, 2, 4, 8, 16 or 32 lanes per
 * row; 0 = chosen from the mean row length; -1 = one lane per row with four rows in flight
 * per lane, the solver's variant for short rows whose latency chains would otherwise bind).
 * precision 2: val holds BF16 values (uint16 bit patterns), x and y are float*, sums in FP32
 * (the product of the matrix_bf16 mode).  Returns CQP_ERR_INVALID for bad sizes. */
int cqp_spmv(int32_t precision, int64_t nrows, int64_t ncols, const int32_t* rowptr, const int32_t* colind,
             const void* val, const void* x, void* y, int32_t threads_per_row, void* stream);

/* The same product with two other layouts (kernel-level; device pointers; precision 0, 1 or
 * 2 as in cqp_spmv; well-formed CSR: rowptr non-decreasing from 0 to nnz, columns in range).
 * cqp_spmv_merge: merge-based row splitting (Merrill and Garland, SC 2016): every thread takes
 * an equal share of the m + nnz items of the merge of row ends and entries, so rows of any
 * length are balanced; carries of rows split between threads are added in thread order by a
 * second kernel (deterministic).  Allocates and frees its carry buffers (stream-ordered) and
 * synchronises the stream.  Errors: CQP_ERR_INVALID, CQP_ERR_CUDA. */
int cqp_spmv_merge(int32_t precision, int64_t nrows, int64_t ncols, const int32_t* rowptr, const int32_t* colind,
                   const void* val, const void* x, void* y, void* stream);

/* Sliced ELL with slices of 32 rows: each slice padded to its longest row and stored
 * column-major inside the slice (coalesced 32-row steps; padded slots skipped).  cqp_sell_build
 * copies a device CSR matrix into that layout (the handle owns the copy; synchronises the
 * stream); cqp_sell_stored reports the stored entries (nnz plus padding); cqp_spmv_sell
 * computes y = A x asynchronously on `stream`; cqp_sell_free releases the handle. */
typedef struct cqp_sell cqp_sell;
int cqp_sell_build(int32_t precision, int64_t nrows, int64_t ncols, const int32_t* rowptr, const int32_t* colind,
                   const void* val, void* stream, cqp_sell** out);
int cqp_sell_stored(const cqp_sell* A, int64_t* stored);
int cqp_spmv_sell(const cqp_sell* A, const void* x, void* y, void* stream);
void cqp_sell_free(cqp_sell* A);

/* out = Pi^M_K(r) blockwise (App. "cone-projections"): Euclidean when m is NULL,
 * otherwise the projection in the diagonal metric M = diag(m).  Cone blocks as
 * in cqp_setup but as device arrays (CQP_CONE_EXP1 / POW1 slices included; box
 * blocks are not).  r, m, out have n entries. */
int cqp_project(int32_t precision, int64_t n, const cqp_cones* K_device, const void* r, const void* m, void* out,
                void* stream);

/* ---- allocation-free KKT check (the paper has no counterpart: this is a
 * library convenience) ----
 * Same report as cqp_kkt, but from the caller's own unscaled problem data and
 * without a handle, and without allocating any device memory: it is meant for
 * callers that must not call cudaMalloc, such as code running inside a
 * framework that already owns the device memory pool, or code that has to
 * keep a fixed device footprint.  Its working memory is a static device array
 * of the library, sized for n <= CQP_KKT_STATIC_MAX_N (about 4.1 MiB, held on
 * every GPU that loads the library until the process exits).
 *   A, Q, K: as in cqp_setup, but every array they point to is a device
 *   array (A->rowptr int64, A->colind int32, A->val double).  c (n), b (m),
 *   x (n), y (m): device arrays.  rep: host struct, filled on success.
 *   stream: cudaStream_t or NULL; the call synchronises it before returning.
 * Cone blocks may include the slices CQP_CONE_EXP1 / POW1 (support terms as in
 * cqp_kkt); box blocks are not accepted.
 * Errors: CQP_ERR_INVALID for NULL arguments, n < 1, n > CQP_KKT_STATIC_MAX_N,
 * rank > 64, or malformed A, P or cone blocks (column indices, row pointers --
 * rowptr[0] = 0, non-decreasing, at most nnz -- and the block layout are checked
 * on the device; a bad row is skipped, so nothing is read out of bounds);
 * CQP_ERR_UNSUPPORTED when its stream is being captured (the report is read back
 * to the host); CQP_ERR_CUDA; CQP_ERR_NUMERICAL for a non-finite report.
 * The first call on each device looks up the array's device address, so make
 * it before any stream capture.  All calls on one device share the array:
 * calls that overlap on the GPU (two streams, two threads) race, so serialise
 * them.  Ax - b, A'y, Qx and the cone projections are recomputed every call;
 * A'y is accumulated with atomics, so the last bits may differ between calls. */
#define CQP_KKT_STATIC_MAX_N 524288
int cqp_kkt_static(const cqp_csr* A_device, const cqp_qop* Q_device, const double* c, const double* b,
                   const cqp_cones* K_device, const double* x, const double* y, cqp_kkt_report* rep, void* stream);

#ifdef __cplusplus
}
#endif
#endif
