// Batched persistent solve: one launch, one thread block per SM, each block
// repeatedly takes the next instance from a work queue (largest first) and runs
// the whole restarted PDHG solve of that instance with block-level barriers only
// (CtaTeam).  Every instance keeps its own scaling factors, step sizes, primal
// weight, restarts, inner tolerance and termination (Alg. pdhcq1, Sec. 4), as if
// solved alone; the data of all instances share the device arrays of one
// block-diagonal problem and are addressed through the instance's ranges.
#pragma once

#include "solver_impl.cuh"

namespace cqp {

template <typename T>
__global__ void __launch_bounds__(512, 1) pdhg_batch_kernel(KernelArgs<T> a, BatchArgs b) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double part[kMaxSlots];
  __shared__ Prob<T> Pi;
  __shared__ long long cur;
  __shared__ unsigned long long t_begin;
  __shared__ double tot[1];
  __shared__ int stop;
  CtaTeam team;
  team.init(part);
  Ctl& C = *reinterpret_cast<Ctl*>(smem);
  const int nw = blockDim.x >> 5;
  double* scratch = reinterpret_cast<double*>(smem + sizeof(Ctl));
  double* wacc = scratch + (size_t)kMaxSlots * nw;
  T* cbuf = reinterpret_cast<T*>(wacc + (size_t)nw * kMaxRank);
  if (threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_begin));
  const Work<T>& W = a.W;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned q = atomicAdd(b.queue, 1u);
      cur = (int64_t)q < b.count ? (long long)b.order[q] : -1;
    }
    __syncthreads();
    const long long i = cur;
    if (i < 0) break;
    if (threadIdx.x == 0) {
      Pi = a.P;
      Pi.beta_b = b.beta_b[i];
      Pi.beta_c = b.beta_c[i];
      Pi.norm_b = b.norm_b[i];
      Pi.norm_c = b.norm_c[i];
      if (b.rank) {   // rows of R beyond the instance's rank are zero on its columns
        Pi.k = b.rank[i];
        Pi.kpad = (Pi.k + 7) / 8 * 8;
      }
    }
    load_state(C, b.S + i);
    Solver<T, CtaTeam> s(Pi, W, a.O, team, C, scratch, wacc, cbuf);
    s.own = b.own[i];
    s.own.g_a = Pi.tpr_a; s.own.g_t = Pi.tpr_t; s.own.g_p = Pi.tpr_p;
    const Own& o = s.own;
    // scaled start x~ = col x0 / beta_b (permuted), y~ = row y0 / beta_c; anchors and
    // candidates start there, averages at zero
    for (int seg = 0; seg < 6; ++seg)
      for (int64_t j = o.x0[seg] + threadIdx.x; j < o.x1[seg]; j += blockDim.x) {
        const double xv = b.x0 ? b.x0[b.perm[j]] : 0.0;
        const T h = T(xv * Pi.col[j] / Pi.beta_b);
        W.hx[0][j] = h;
        W.ax[j] = h;
        W.wx[0][j] = h;
        if (W.avx) W.avx[j] = T(0);
      }
    for (int64_t r = o.row0 + threadIdx.x; r < o.row1; r += blockDim.x) {
      const double yv = b.y0 ? b.y0[r] : 0.0;
      const T h = T(yv * Pi.row[r] / Pi.beta_c);
      W.hy[0][r] = h;
      W.ay[r] = h;
      W.wy[r] = h;
      if (W.avy) W.avy[r] = T(0);
    }
    __syncthreads();
    // R~ h_x of the start over the instance's own columns
    for (int l = 0; l < Pi.k; ++l) {
      double v[1] = {0.0};
      if (b.x0)
        for (int seg = 0; seg < 6; ++seg)
          for (int64_t j = o.x0[seg] + threadIdx.x; j < o.x1[seg]; j += blockDim.x)
            v[0] += (double)Pi.R[(int64_t)l * Pi.n + j] * (double)W.hx[0][j];
      block_sum<1>(v, scratch, tot);
      if (threadIdx.x == 0) C.s.t_h[l] = tot[0];
    }
    __syncthreads();
    for (;;) {
      s.run(b.chunk);
      __syncthreads();
      if (C.s.status != 0 || C.s.err != 0 || C.s.ktot >= a.O.max_iter) break;
      // the time-limit decision is taken by one thread and shared, so the block leaves together
      if (threadIdx.x == 0) {
        unsigned long long now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        stop = (b.time_limit_ns && now - t_begin > b.time_limit_ns) ? 1 : 0;
        if (stop) C.s.status = 3;
      }
      __syncthreads();
      if (stop) break;
    }
    __syncthreads();
    // unscaled, un-permuted final candidate (average for the averaged variant)
    const T* fx = a.O.update == 1 ? W.avx : W.wx[C.s.wb];
    const T* fy = a.O.update == 1 ? W.avy : W.wy;
    for (int seg = 0; seg < 6; ++seg)
      for (int64_t j = o.x0[seg] + threadIdx.x; j < o.x1[seg]; j += blockDim.x)
        b.x_out[b.perm[j]] = Pi.beta_b * (double)fx[j] / Pi.col[j];
    for (int64_t r = o.row0 + threadIdx.x; r < o.row1; r += blockDim.x)
      b.y_out[r] = Pi.beta_c * (double)fy[r] / Pi.row[r];
    if (threadIdx.x == 0) b.S[i] = C.s;
  }
}

template <typename T>
cudaError_t launch_pdhg_batch(const KernelArgs<T>& a, const BatchArgs& b, int blocks, int threads, cudaStream_t st) {
  using CQP_TT = T;
  const size_t smem = solver_smem_bytes<CQP_TT>(threads);
  cudaError_t e = cudaFuncSetAttribute(pdhg_batch_kernel<CQP_TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  pdhg_batch_kernel<CQP_TT><<<blocks, threads, smem, st>>>(a, b);
  return cudaGetLastError();
}

}  // namespace cqp
