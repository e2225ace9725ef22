// Device-side building blocks shared by the kernels of the library:
// warp/block reductions, the bounded-spin grid barrier and the "team" that a
// solver phase runs on (the whole GPU as one cooperative grid, or one CTA).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cqp {

constexpr int kWarp = 32;
constexpr int kMaxRank = 64;        // largest low-rank factor R supported (rank x n)
constexpr int kMaxSlots = 96;       // FP64 reduction slots per phase

// device-side error codes written to SolverState::err
enum DevErr : int { kErrNone = 0, kErrBarrier = 1, kErrNumeric = 2 };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// sum over aligned groups of G lanes (G a power of two <= 32); every lane of a group gets the group sum
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Sum NS per-thread values over the block; results land in out[0..NS) (shared),
// visible to all threads after the call.  scratch: NS * (blockDim/32) doubles.
template <int NS>
__device__ __forceinline__ void block_sum(double (&v)[NS], double* scratch, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double t = warp_sum(v[s]);
    if (lane == 0) scratch[s * nw + warp] = t;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NS; s += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += scratch[s * nw + w];
    out[s] = t;
  }
  __syncthreads();
}

// Same as block_sum but the per-thread values and the warp trees are in R (the
// iterate precision for per-iteration sums); warp totals are combined in FP64.
template <typename R, int NS>
__device__ __forceinline__ void block_sum_r(R (&v)[NS], double* scratch, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    R t = v[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) scratch[s * nw + warp] = (double)t;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NS; s += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += scratch[s * nw + w];
    out[s] = t;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Teams.  A solver phase is written once against this interface:
//   nb(), bid()            number of blocks in the team and this block's rank
//   sync()                 team-wide barrier (returns false if a bounded wait expired)
//   publish(slot, v)       block total v of reduction slot `slot` (thread 0 only)
//   gather(nslots, out)    after sync(): out[s] = sum over blocks of slot s, in a fixed
//                          order, identical on every block (shared-memory `out`)
//   finish()               before the kernel returns (the cluster team waits for every
//                          block, whose shared memory the others may still read)
// Every block runs the same publish / sync / gather sequence.  The partials alternate
// between two buffers, one per gather: a block that has gathered and runs ahead writes
// its next partials into the other buffer, and it cannot come back to this one before
// the next barrier, which every block reaches only after its own gather.
// ---------------------------------------------------------------------------

struct GridBarrier {
  unsigned* count;   // zeroed by the host before every launch
  int* err;          // device error word
};

// Whole-GPU team: the kernel is launched cooperatively so all blocks are
// co-resident; the barrier spins with an iteration limit and reports expiry
// through *err instead of hanging.
struct GridTeam {
  GridBarrier bar;
  double* part;      // [2][kMaxSlots][gridDim.x] block partials in global memory
  unsigned target;
  int failed;
  int buf;           // buffer of the current publish / gather round

  __device__ void init(GridBarrier b, double* p) {
    bar = b;
    part = p;
    target = 0;
    failed = 0;
    buf = 0;
  }
  __device__ __forceinline__ int nb() const { return gridDim.x; }
  __device__ __forceinline__ int bid() const { return blockIdx.x; }
  __device__ bool sync() {
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(bar.count, 1u);
      long long spins = 0;
      while ((int)(ld_acquire_u32(bar.count) - target) < 0) {
        if (++spins > (1ll << 24) || *(volatile int*)bar.err != 0) {
          atomicCAS(bar.err, 0, (int)kErrBarrier);
          break;
        }
      }
      __threadfence();
    }
    __syncthreads();
    failed = *(volatile int*)bar.err != 0;
    return !failed;
  }
  __device__ __forceinline__ void publish(int slot, double v) {
    part[(buf * kMaxSlots + slot) * gridDim.x + blockIdx.x] = v;
  }
  // one warp per slot, lanes stride over blocks, then a fixed-order shuffle tree
  __device__ void gather(int nslots, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double* pb = part + (size_t)buf * kMaxSlots * gridDim.x;
    for (int s = warp; s < nslots; s += nw) {
      double t = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(&pb[s * gridDim.x + b]);
      t = warp_sum(t);
      if (lane == 0) out[s] = t;
    }
    buf ^= 1;
    __syncthreads();
  }
  __device__ __forceinline__ void finish() {}
};

// Thread-block-cluster team: the blocks of one cluster (launched as the whole grid),
// synchronised by the hardware cluster barrier; every block keeps its partials in its
// own shared memory and reads the others' through distributed shared memory, in rank
// order.  Every block takes the same decisions from the same gathered sums, so all of
// them pass the same barriers and none can wait for a block that has left.
__device__ __forceinline__ double ld_cluster_f64(const double* local, unsigned rank) {
  const unsigned addr = (unsigned)__cvta_generic_to_shared(local);
  unsigned remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(addr), "r"(rank));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(remote) : "memory");
  return v;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct ClusterTeam {
  double* part;      // shared memory of this block, [2][kMaxSlots]
  int failed;
  int buf;
  __device__ void init(double* p) {
    part = p;
    failed = 0;
    buf = 0;
  }
  __device__ __forceinline__ int nb() const { return gridDim.x; }
  __device__ __forceinline__ int bid() const { return blockIdx.x; }
  __device__ __forceinline__ bool sync() {
    __syncthreads();
    cluster_barrier();
    return true;
  }
  __device__ __forceinline__ void publish(int slot, double v) { part[buf * kMaxSlots + slot] = v; }
  __device__ void gather(int nslots, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = warp; s < nslots; s += nw) {
      double t = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) t += ld_cluster_f64(part + buf * kMaxSlots + s, (unsigned)b);
      t = warp_sum(t);
      if (lane == 0) out[s] = t;
    }
    buf ^= 1;
    __syncthreads();
  }
  __device__ __forceinline__ void finish() { cluster_barrier(); }
};

// One-CTA team: barriers are __syncthreads and block totals are final.
struct CtaTeam {
  double* part;      // shared memory, kMaxSlots
  int failed;
  __device__ void init(double* p) {
    part = p;
    failed = 0;
  }
  __device__ __forceinline__ int nb() const { return 1; }
  __device__ __forceinline__ int bid() const { return 0; }
  __device__ __forceinline__ bool sync() {
    __syncthreads();
    return true;
  }
  __device__ __forceinline__ void publish(int slot, double v) { part[slot] = v; }
  __device__ void gather(int nslots, double* out) {
    __syncthreads();
    for (int s = threadIdx.x; s < nslots; s += blockDim.x) out[s] = part[s];
    __syncthreads();
  }
  __device__ __forceinline__ void finish() {}
};

// [lo, hi) share of `count` items for block b of nb
__device__ __forceinline__ void split_range(int64_t count, int b, int nb, int64_t& lo, int64_t& hi) {
  lo = (count * b) / nb;
  hi = (count * (b + 1)) / nb;
}

// first row r with rowptr[r] >= target (rowptr non-decreasing, nrows+1 entries)
__device__ __forceinline__ int64_t lower_bound_rows(const int* rowptr, int64_t nrows, int64_t target) {
  int64_t lo = 0, hi = nrows;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if ((int64_t)rowptr[mid] < target) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Work of a CSR row for the block splits: its entries plus kRowWork for the row itself
// (row pointers, the result, and the per-coordinate vector work of the phases that walk
// the same range), so a range of very short rows is not handed to one block.
constexpr int64_t kRowWork = 8;

// [lo, hi) share for block b of nb of the rows [base, base + count) of a CSR matrix,
// balancing nnz + kRowWork per row (offsets relative to base)
__device__ __forceinline__ void split_rows_weighted(const int* rowptr, int64_t base, int64_t count, int b, int nb,
                                                    int64_t& lo, int64_t& hi) {
  const int64_t r0 = rowptr[base];
  const int64_t work = (int64_t)rowptr[base + count] - r0 + kRowWork * count;
  auto find = [&](int64_t target) {
    int64_t l = 0, h = count;
    while (l < h) {
      const int64_t mid = (l + h) >> 1;
      if ((int64_t)rowptr[base + mid] - r0 + kRowWork * mid < target) l = mid + 1; else h = mid;
    }
    return l;
  };
  lo = b == 0 ? 0 : find((work * b) / nb);
  hi = b == nb - 1 ? count : find((work * (b + 1)) / nb);
}

// rows of a CSR matrix shared among nb blocks with (almost) equal nnz + kRowWork * rows
__device__ __forceinline__ void split_rows_by_nnz(const int* rowptr, int64_t nrows, int b, int nb, int64_t& lo,
                                                  int64_t& hi) {
  split_rows_weighted(rowptr, 0, nrows, b, nb, lo, hi);
}

// Lanes per row for one block's rows: the tuned width, unless the block's rows average
// less than a quarter of it, then the largest power of two not above their mean length
// (short rows under a wide group leave most lanes idle and serialise the block).
__device__ __forceinline__ int block_group_width(int tuned, int64_t nnz, int64_t rows) {
  if (tuned <= 1 || rows <= 0 || 4 * nnz >= (int64_t)tuned * rows) return tuned;   // 0: batched one-lane rows
  int g = 1;
  while (2 * g * rows <= nnz) g *= 2;
  return g;
}

}  // namespace cqp
