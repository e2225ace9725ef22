/*
 * cqp_mlp.h: learned warm start for batches of portfolio QPs (libcqp_gb300.so).
 *
 * The paper has no learned component.  This subsystem proposes a start (x0, y0)
 * for cqp_solve_batch on the portfolio family of a batch (per instance: weights x
 * (n_i, nonnegative), then the second-order cone block (w_F (k_i), w_D (n_i), t);
 * rows 1'x = 1, F'x - w_F = 0, D^(1/2) x - w_D = 0, t = sigma_bar).  A 3-layer MLP
 * (features -> 512 -> 512 -> 1 score per asset, ReLU, BF16 weights and activations,
 * FP32 accumulation) scores the assets; x0 is the softmax of the scores within each
 * instance; a dual head on the mean of the last hidden layer gives the budget-row and
 * risk-row duals, and the remaining duals follow as lambda (w_F, w_D) with
 * lambda = y_t / sigma_bar.  The solver itself is unchanged; a cold start remains
 * the fallback, and the solve's own KKT test decides whether the start is good.
 *
 * Conventions as in cqp.h: int status, device pointers, caller-owned buffers,
 * stream NULL = default stream, nothing synchronises unless stated.  BF16 arrays are
 * passed as uint16_t (bit pattern of __nv_bfloat16).  Row-major storage throughout.
 * "Instance" arrays follow the batch layout of cqp_setup_batch; asset_off (count+1)
 * numbers the assets of all instances consecutively (rows of the feature matrix).
 */
#ifndef CQP_GB300_MLP_H
#define CQP_GB300_MLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CQP_WS_HIDDEN 512   /* hidden width */
#define CQP_WS_FEATURES 16  /* feature columns (8 used, zero padded) */

/* Per-asset features X (rows = asset_off[count], CQP_WS_FEATURES BF16 columns) from the
 * batch data: mu = -c, D = q (diagonal of Q), the factor loadings R[0..rank_i-1, x]
 * (R row-major with leading dimension ldr), sigma_bar = last entry of b of each instance.
 * Features: 20 mu, 20 D, 100 |F_j|^2, 0.1 rr with rr = mu/(D + |F_j|^2), 50 (mu - mean mu),
 * log(n_i)/8, k_i/50, 10 sigma_bar, (mu - mean mu)/std mu, D/mean D, |F_j|^2/mean |F|^2,
 * rr/max rr (means, std and max over the instance's assets). */
int cqp_ws_features(int64_t count, const int64_t* x_off, const int64_t* n_assets, const int64_t* asset_off,
                    const int64_t* row_off, const int32_t* rank, const double* c, const double* q, const double* R,
                    int64_t ldr, const double* b, uint16_t* X, void* stream);

/* C = op(A) op(B) on the tensor cores: op(A) is M x K (A itself, row-major with lda,
 * or the transpose of A stored K x M when trans_a), op(B) is K x N likewise.  BF16
 * inputs, FP32 accumulation.  epilogue: 0 C = result (FP32), 1 C = result + bias
 * (FP32, bias has N entries), 2 C = ReLU(result + bias) (BF16), 3 C += result (FP32,
 * atomic; split_k slices of K run in parallel; C must be initialised), 4 C = result
 * (BF16).  The product A B' (trans_a = 0, trans_b = 1) with N a multiple of 256, K a
 * multiple of 64, lda >= K, ldb >= K, ldc >= N all multiples of 8, 16-byte aligned A,
 * B, C (and bias, for epilogues 1 and 2) and epilogue 0, 1, 2 or 4 runs on the
 * fifth-generation tensor cores: a persistent kernel, tcgen05.mma into two accumulators
 * in tensor memory, operands loaded and C stored by tiled tensor copies.  The other forms
 * run on the warp-level tensor-core kernel.  Errors: CQP_ERR_INVALID for bad sizes, or
 * (warp-level kernel) more than 65535 row tiles; asynchronous on `stream` (see
 * cqp_gemm_check). */
int cqp_gemm_bf16(int32_t trans_a, int32_t trans_b, int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda,
                  const uint16_t* B, int64_t ldb, void* C, int64_t ldc, const float* bias, int32_t epilogue,
                  int32_t split_k, void* stream);

/* CQP_ERR_WAIT if a bounded wait (one second) inside one of the tensor-core GEMMs issued so far
 * on the current device expired (that GEMM's output is then incomplete: the blocks stop at the
 * failed wait); CQP_OK otherwise.  Synchronises stream and clears the record. */
int cqp_gemm_check(void* stream);

/* out (cols x rows, BF16, row-major) = in' (in: rows x cols, BF16, row-major). */
int cqp_transpose_bf16(int64_t rows, int64_t cols, const uint16_t* in, uint16_t* out, void* stream);

/* Encoders of the tensor-core GEMM's descriptors, exposed for host tests (PTX ISA tcgen05
 * shared-memory descriptor: start address, leading / stride byte offsets, version bits 46-48 =
 * 0b001, swizzle mode in bits 61-63; instruction descriptor of kind::f16 with BF16 A and B, FP32
 * accumulator, K-major operands, M x N). */
uint64_t cqp_umma_smem_desc(uint32_t smem_addr, uint32_t lbo_bytes, uint32_t sbo_bytes, int32_t swizzle);
uint32_t cqp_umma_instr_desc_bf16(int32_t m, int32_t n);

/* Number of tensor-memory GEMM kernels launched by this process so far (the forms of
 * cqp_gemm_bf16 that take the tcgen05 path); lets callers confirm which kernel ran. */
long long cqp_gemm_tc_launches(void);

/* Head forward: score_j = H2_j . w3 + b3 (FP32), x0 = softmax of the scores within each
 * instance, pooled_i = mean of H2 over the instance's assets (count x 512), ydual_i =
 * pooled_i Wd + bd (count x 2; Wd is 512 x 2 row-major). */
int cqp_ws_head_forward(int64_t count, const int64_t* asset_off, const uint16_t* H2, const float* w3, const float* b3,
                        const float* Wd, const float* bd, float* score, float* x0, float* pooled, float* ydual,
                        void* stream);

/* Training loss sum_i [ n_i sum_j (x0_j - xstar_j)^2 + lam sum_d (ydual_id - ystar_id)^2 ],
 * added to *loss (FP64, caller zeroes it), and the gradients (times `scale`) with
 * respect to the scores (through the softmax) and the dual outputs. */
int cqp_ws_loss(int64_t count, const int64_t* asset_off, const float* x0, const float* xstar, const float* ydual,
                const float* ystar, float lam, float scale, float* dscore, float* dydual, double* loss, void* stream);

/* Head backward: dZ2 = (dscore w3' + dydual Wd' / n_i) masked by [H2 > 0] (BF16,
 * rows x 512); adds the gradients of w3, b3, Wd, bd into gw3, gb3, gWd, gbd (FP32). */
int cqp_ws_head_backward(int64_t count, const int64_t* asset_off, const uint16_t* H2, const float* w3, const float* Wd,
                         const float* dscore, const float* dydual, const float* pooled, uint16_t* dZ2, float* gw3,
                         float* gb3, float* gWd, float* gbd, void* stream);

/* dH := dH * [H > 0] (BF16, rows x cols, in place); if gbias, adds the column sums of
 * the masked dH to gbias (FP32, cols). */
int cqp_relu_backward_bf16(int64_t rows, int64_t cols, const uint16_t* H, uint16_t* dH, float* gbias, void* stream);

/* One Adam step on n FP32 parameters (bias-corrected with `step` >= 1); w_bf16, if
 * given, receives the updated weights in BF16. */
int cqp_adam_step(int64_t n, float* w, const float* g, float* m, float* v, float lr, float beta1, float beta2, float eps,
                  int64_t step, uint16_t* w_bf16, void* stream);

/* The batch start from the head outputs: x = xw (softmax weights), w_F = F'x, w_D =
 * D^(1/2) x, t = sigma_bar; y = (ydual_0 / yb_scale, lambda w_F, lambda w_D, ydual_1)
 * with lambda = ydual_1 / sigma_bar.  dual_mode 0 keeps y0 = 0 (primal start only), 1 sets
 * the budget and risk rows only, 2 the whole dual above.  x0 (n) and y0 (m) in the batch
 * layout (FP64, y0 fully written). */
int cqp_ws_start(int64_t count, const int64_t* x_off, const int64_t* row_off, const int64_t* n_assets,
                 const int64_t* asset_off, const int32_t* rank, const double* q, const double* R, int64_t ldr,
                 const double* b, const float* xw, const float* ydual, float yb_scale, int32_t dual_mode, double* x0,
                 double* y0, void* stream);

#ifdef __cplusplus
}
#endif
#endif
