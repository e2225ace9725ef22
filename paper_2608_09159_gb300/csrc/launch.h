// Launchers for the solver kernels, instantiated per precision in
// solver_f32.cu / solver_f64.cu.
#pragma once

#include <cuda_runtime.h>

#include "solver.cuh"

namespace cqp {

template <typename T>
struct KernelArgs;

// How the blocks of a solve cooperate: one block, the whole GPU (cooperative launch, one
// block per SM) or one thread-block cluster.
enum TeamKind : int { kTeamCta = 0, kTeamGrid = 1, kTeamCluster = 2 };

template <typename T>
cudaError_t launch_pdhg(const KernelArgs<T>& a, int team, int blocks, int threads, cudaStream_t st);

// KKT report of the scaled point (x, y) with the handle's data; out receives 8 doubles.
template <typename T>
cudaError_t launch_kkt(const KernelArgs<T>& a, const T* x, const T* y, double* out, int team, int blocks, int threads,
                       cudaStream_t st);

// General-form variant of launch_pdhg (row bounds, box blocks), built in its own
// translation unit; launch_pdhg forwards to it when P.rhi or P.xlo is set.
template <typename T>
cudaError_t launch_pdhg_general(const KernelArgs<T>& a, int team, int blocks, int threads, cudaStream_t st);
template <typename T>
int pdhg_general_blocks_per_sm(int threads);
template <typename T>
int pdhg_general_cluster_size(int threads);

// Largest cluster (16, 8, 4 or 2 CTAs of `threads` threads) every solver kernel variant of
// this precision can be launched with; 0 if none.
template <typename T>
int pdhg_cluster_size(int threads);

// The whole-GPU team's kernels, compiled in their own translation units (CQP_GRID_PART):
// the equality-form solver and KKT kernels and the general-form solver kernel.
template <typename T>
cudaError_t launch_pdhg_grid(const KernelArgs<T>& a, int blocks, int threads, cudaStream_t st);
template <typename T>
cudaError_t launch_kkt_grid(const KernelArgs<T>& a, const T* x, const T* y, double* out, int blocks, int threads,
                            cudaStream_t st);
template <typename T>
int pdhg_grid_blocks_per_sm(int threads);
template <typename T>
cudaError_t launch_pdhg_general_grid(const KernelArgs<T>& a, int blocks, int threads, cudaStream_t st);

// Batched persistent solve (one block per instance at a time, work queue).
template <typename T>
cudaError_t launch_pdhg_batch(const KernelArgs<T>& a, const BatchArgs& b, int blocks, int threads, cudaStream_t st);

// Blocks per SM that can be co-resident for the cooperative solver kernel.
template <typename T>
int pdhg_blocks_per_sm(int threads);

template <typename T>
size_t pdhg_smem(int threads);

// Kernel-level entry points used by the C ABI.
// blocks <= 0: four 512-thread blocks per SM; the threads-per-row autotuner passes the
// solver's own grid (one block per SM) so it times the concurrency the solver runs at.
template <typename T>
cudaError_t launch_spmv(int64_t nrows, const int* rp, const int* ci, const T* v, const T* x, T* y, int tpr,
                        cudaStream_t st, int blocks = 0);
template <typename T>
cudaError_t launch_spmv_bf16(int64_t nrows, const int* rp, const int* ci, const __nv_bfloat16* v, const T* x, T* y,
                             int tpr, cudaStream_t st, int blocks = 0);
template <typename T>
cudaError_t launch_project(int64_t nblocks, const int32_t* type, const int64_t* start, const int64_t* dim,
                           const double* alpha, const T* r, const T* m, T* out, int64_t n, cudaStream_t st);

}  // namespace cqp
