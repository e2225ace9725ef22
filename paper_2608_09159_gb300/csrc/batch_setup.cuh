// Setup kernels of the batched mode: a batch is one block-diagonal problem whose
// instances get their own norms, bound-objective scaling and step sizes, as if each
// were set up alone (Sec. 4.2.2 rescaling, eq. practical-stepsizes).  Ruiz and
// Pock-Chambolle factors are per row and per column, so the shared passes over the
// whole matrix already give every instance its own factors; only the steps that
// take a norm over the problem are done here, one thread block per instance.
// An instance's coordinates in the permuted layout are the six ranges of its Own.
#pragma once

#include <cstdint>

#include "common.cuh"
#include "setup.cuh"
#include "solver.cuh"

namespace cqp {

constexpr int kBatchSetupThreads = 512;

// every entry of A (or P) must join a row and a column of the same instance
__global__ void k_check_blockdiag(int64_t rows, const int64_t* rp, const int32_t* ci, const int32_t* inst_row,
                                  const int32_t* inst_col, int* bad) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t ir = inst_row[r];
    for (int64_t e = rp[r]; e < rp[r + 1]; ++e)
      if (inst_col[ci[e]] != ir) {
        atomicOr(bad, 16);
        break;
      }
  }
}

// ||b_i||, ||c_i|| of the unscaled data (KKT normalisation), original order
__global__ void __launch_bounds__(kBatchSetupThreads) k_inst_norms(int64_t count, const int64_t* x_off,
                                                                   const int64_t* row_off, const double* c,
                                                                   const double* b, double* norm_b, double* norm_c) {
  __shared__ double red[2 * (kBatchSetupThreads / 32)];
  __shared__ double tot[2];
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    double v[2] = {0.0, 0.0};
    for (int64_t j = x_off[i] + threadIdx.x; j < x_off[i + 1]; j += blockDim.x) v[0] += c[j] * c[j];
    for (int64_t r = row_off[i] + threadIdx.x; r < row_off[i + 1]; r += blockDim.x) v[1] += b[r] * b[r];
    block_sum<2>(v, red, tot);
    if (threadIdx.x == 0) {
      norm_c[i] = sqrt(tot[0]);
      norm_b[i] = sqrt(tot[1]);
    }
    __syncthreads();
  }
}

// bound-objective scaling per instance (reading of Sec. 4.2.2: b~ /= ||b~||+1,
// (c~, Q~) /= ||c~||+1, x measured in units of ||b~||+1 so Q~ is multiplied by
// beta_b / beta_c).  The low-rank part is scaled through the instance's columns of
// R (by sqrt(beta_b / beta_c)) because D is shared by all instances.
__global__ void __launch_bounds__(kBatchSetupThreads) k_inst_bound_obj(
    int64_t count, const Own* own, int64_t n, int enable, double* cv, double* bv, double* qv, int64_t k, double* Rv,
    const int32_t* p_rp, double* pv, double* beta_b, double* beta_c) {
  __shared__ double red[2 * (kBatchSetupThreads / 32)];
  __shared__ double tot[2];
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const Own o = own[i];
    double v[2] = {0.0, 0.0};
    for (int seg = 0; seg < 6; ++seg)
      for (int64_t j = o.x0[seg] + threadIdx.x; j < o.x1[seg]; j += blockDim.x) v[0] += cv[j] * cv[j];
    for (int64_t r = o.row0 + threadIdx.x; r < o.row1; r += blockDim.x) v[1] += bv[r] * bv[r];
    block_sum<2>(v, red, tot);
    const double bb = enable ? sqrt(tot[1]) + 1.0 : 1.0;
    const double bc = enable ? sqrt(tot[0]) + 1.0 : 1.0;
    const double qs = bb / bc, rs = sqrt(qs);
    for (int seg = 0; seg < 6; ++seg)
      for (int64_t j = o.x0[seg] + threadIdx.x; j < o.x1[seg]; j += blockDim.x) {
        cv[j] /= bc;
        qv[j] *= qs;
        for (int64_t l = 0; l < k; ++l) Rv[l * n + j] *= rs;
        if (p_rp)
          for (int e = p_rp[j]; e < p_rp[j + 1]; ++e) pv[e] *= qs;
      }
    for (int64_t r = o.row0 + threadIdx.x; r < o.row1; r += blockDim.x) bv[r] /= bb;
    if (threadIdx.x == 0) {
      beta_b[i] = bb;
      beta_c[i] = bc;
    }
    __syncthreads();
  }
}

// ||A~_i||_2 by the Lanczos process on the instance's block (same reading as k_power:
// SplitMix64 start keyed by the instance-local coordinate index perm[j] - x_off_old[i],
// stop at `tol` relative change of sigma, at beta = 0 or after `iters` steps),
// eta_i = step / ||A~_i||, omega0_i = ||c~_i|| / ||b~_i||.
template <typename T>
__global__ void __launch_bounds__(kBatchSetupThreads) k_inst_power(
    int64_t count, const Own* own, const int32_t* __restrict__ a_rp, const int32_t* __restrict__ a_ci,
    const T* __restrict__ a_v, const int32_t* __restrict__ t_rp, const int32_t* __restrict__ t_ci,
    const T* __restrict__ t_v, const double* cv, const double* bv, double* z, double* zp, double* w, int iters,
    double tol, double step, double* eta, double* omega0, double* norm_a, const int64_t* perm,
    const int64_t* x_off_old) {
  __shared__ double red[2 * (kBatchSetupThreads / 32)];
  __shared__ double tot[2];
  __shared__ double al[kMaxLanczos], be[kMaxLanczos];
  __shared__ double theta;
  const int nit = iters < kMaxLanczos ? iters : kMaxLanczos;
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const Own o = own[i];
    double z2[1] = {0.0};
    for (int seg = 0; seg < 6; ++seg)
      for (int64_t j = o.x0[seg] + threadIdx.x; j < o.x1[seg]; j += blockDim.x) {
        const double u = power_start_value((uint64_t)(perm[j] - x_off_old[i]) + 1);
        z[j] = u;
        zp[j] = 0.0;
        z2[0] += u * u;
      }
    block_sum<1>(z2, red, tot);
    const double zinv = tot[0] > 0.0 ? 1.0 / sqrt(tot[0]) : 0.0;
    for (int seg = 0; seg < 6; ++seg)
      for (int64_t j = o.x0[seg] + threadIdx.x; j < o.x1[seg]; j += blockDim.x) z[j] *= zinv;
    __syncthreads();
    double sig = 0.0, zscale = 1.0, beta_prev = 0.0;
    for (int it = 0; it < nit && o.row1 > o.row0; ++it) {
      double acc[1] = {0.0};
      for (int64_t r = o.row0 + threadIdx.x; r < o.row1; r += blockDim.x) {
        double s = 0.0;
        for (int e = a_rp[r]; e < a_rp[r + 1]; ++e) s += (double)a_v[e] * z[a_ci[e]];
        s *= zscale;
        w[r] = s;
        acc[0] += s * s;
      }
      block_sum<1>(acc, red, tot);
      const double alpha = tot[0];
      acc[0] = 0.0;
      for (int seg = 0; seg < 6; ++seg)
        for (int64_t j = o.x0[seg] + threadIdx.x; j < o.x1[seg]; j += blockDim.x) {
          double s = 0.0;
          for (int e = t_rp[j]; e < t_rp[j + 1]; ++e) s += (double)t_v[e] * w[t_ci[e]];
          const double vj = z[j] * zscale, vp = zp[j];
          s -= alpha * vj + beta_prev * vp;
          zp[j] = vj;
          z[j] = s;
          acc[0] += s * s;
        }
      block_sum<1>(acc, red, tot);
      const double beta = sqrt(tot[0]);
      if (threadIdx.x == 0) al[it] = alpha;
      __syncthreads();
      if (threadIdx.x < 32) {
        const double th = tridiag_max_eig_warp(al, be, it + 1, threadIdx.x);
        if (threadIdx.x == 0) theta = th;
      }
      __syncthreads();
      const double s_new = sqrt(fmax(theta, 0.0));
      const bool done = (it > 0 && fabs(s_new - sig) <= tol * s_new) || beta == 0.0;
      sig = s_new;
      if (done) break;
      if (threadIdx.x == 0) be[it] = beta;
      zscale = 1.0 / beta;
      beta_prev = beta;
      __syncthreads();
    }
    double v[2] = {0.0, 0.0};
    for (int seg = 0; seg < 6; ++seg)
      for (int64_t j = o.x0[seg] + threadIdx.x; j < o.x1[seg]; j += blockDim.x) v[0] += cv[j] * cv[j];
    for (int64_t r = o.row0 + threadIdx.x; r < o.row1; r += blockDim.x) v[1] += bv[r] * bv[r];
    block_sum<2>(v, red, tot);
    if (threadIdx.x == 0) {
      const double cn = sqrt(tot[0]), bn = sqrt(tot[1]);
      eta[i] = step / (sig > 0.0 ? sig : 1.0);
      omega0[i] = (cn > 1e-10 && bn > 1e-10) ? cn / bn : 1.0;
      norm_a[i] = sig;
    }
    __syncthreads();
  }
}

// rows of R that are nonzero on the instance's columns: its rank (R rows are
// stored instance by instance side by side, zero beyond each instance's rank)
__global__ void __launch_bounds__(kBatchSetupThreads) k_inst_rank(int64_t count, const Own* own, int64_t n, int64_t k,
                                                                  const double* Rv, int* rank) {
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const Own o = own[i];
    int r = 0;
    for (int64_t l = k - 1; l >= 0; --l) {
      int nz = 0;
      for (int seg = 0; seg < 6 && !nz; ++seg)
        for (int64_t j = o.x0[seg] + threadIdx.x; j < o.x1[seg]; j += blockDim.x)
          if (Rv[l * n + j] != 0.0) { nz = 1; break; }
      if (__syncthreads_or(nz)) { r = (int)l + 1; break; }
    }
    if (threadIdx.x == 0) rank[i] = r;
    __syncthreads();
  }
}

}  // namespace cqp
