// Two more layouts of the sparse product y = A x, next to the solver's CSR row loops:
//
//  * merge-based CSR (Merrill and Garland, "Merge-based parallel sparse matrix-vector
//    multiplication", SC 2016): the merge of the row-end offsets rowptr[1..m] with the entry
//    indices 0..nnz-1 has m + nnz items; every thread takes an equal share of them, so a row of
//    any length is split over as many threads as it needs and no thread waits on another's
//    long row.  A block first finds its share's two ends on the merge path (binary search on
//    the diagonal), stages its entries (column indices, values) and row ends in shared memory
//    with coalesced loads, then each thread walks its items: an entry adds v x[col] to the
//    running sum, a row end stores the sum and starts the next row.  The partial sum of the
//    row a thread stops inside is its carry; a second kernel adds the carries of each row in
//    thread order (one thread per run of equal rows: deterministic, no atomics).
//
//  * sliced ELL with slices of 32 rows (one warp): each slice is padded to its longest row and
//    stored column-major inside the slice, so step j of a warp loads entry j of its 32 rows as
//    one 128-byte (FP32) transaction; padded slots hold column -1 and are skipped.
//
// Both take FP32 or FP64 values with vectors of the same precision, or BF16 values with FP32
// vectors (the product of the matrix_bf16 mode); sums in the vector precision.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "cqp.h"

namespace cqp {
void record_error(const std::string& msg);
void record_launches(long long k);
}  // namespace cqp

namespace {

constexpr int kMergeThreads = 256;
constexpr int kMergeIpt = 7;                               // merge items per thread
constexpr int kMergeTile = kMergeThreads * kMergeIpt;      // items per block

template <typename T>
__device__ __forceinline__ T ldv(const T* p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// rows consumed before diagonal d of the merge path: the smallest i in [max(0, d - nnz),
// min(d, m)] whose row end (item rowptr[i + 1] + i) is not before d
__device__ __forceinline__ int64_t merge_search(const int* rp, int64_t m, int64_t nnz, int64_t d) {
  int64_t lo = d - nnz > 0 ? d - nnz : 0, hi = d < m ? d : m;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)rp[mid + 1] + mid < d) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <typename T, typename V>
__global__ void __launch_bounds__(kMergeThreads) k_spmv_merge(int64_t m, int64_t nnz, const int* __restrict__ rp,
                                                              const int* __restrict__ ci, const V* __restrict__ v,
                                                              const T* __restrict__ x, T* __restrict__ y,
                                                              int64_t* __restrict__ carry_row, T* __restrict__ carry_val) {
  __shared__ int s_ci[kMergeTile];
  __shared__ T s_v[kMergeTile];
  __shared__ int s_end[kMergeTile + 1];   // row ends rowptr[r + 1] of the block's rows
  __shared__ int64_t s_bounds[4];         // row0, k0, row1, k1
  const int64_t total = m + nnz;
  const int64_t d0 = min64((int64_t)blockIdx.x * kMergeTile, total);
  const int64_t d1 = min64(d0 + kMergeTile, total);
  if (threadIdx.x == 0) {
    const int64_t r0 = merge_search(rp, m, nnz, d0), r1 = merge_search(rp, m, nnz, d1);
    s_bounds[0] = r0;
    s_bounds[1] = d0 - r0;
    s_bounds[2] = r1;
    s_bounds[3] = d1 - r1;
  }
  __syncthreads();
  const int64_t row0 = s_bounds[0], k0 = s_bounds[1], row1 = s_bounds[2], k1 = s_bounds[3];
  // the block's entries [k0, k1) and the ends of rows [row0, min(row1 + 1, m)) (row1's end may
  // lie beyond this block; it is needed only to know the row continues)
  const int ne = (int)(k1 - k0);
  const int nr = (int)(min64(row1 + 1, m) - row0);
  for (int i = threadIdx.x; i < ne; i += kMergeThreads) {
    s_ci[i] = __ldg(ci + k0 + i);
    s_v[i] = (T)ldv(v + k0 + i);
  }
  for (int i = threadIdx.x; i < nr; i += kMergeThreads) s_end[i] = __ldg(rp + row0 + i + 1);
  __syncthreads();
  // this thread's share of the block's items, found on the block's part of the merge path
  const int64_t td0 = min64(d0 + (int64_t)threadIdx.x * kMergeIpt, d1);
  const int64_t td1 = min64(td0 + kMergeIpt, d1);
  int64_t lo = max64(row0, td0 - k1), hi = min64(row1, td0 - k0);
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)s_end[mid - row0] + mid < td0) lo = mid + 1;
    else hi = mid;
  }
  int64_t row = lo, k = td0 - lo;
  T sum = T(0);
  for (int64_t it = td0; it < td1; ++it) {
    if (row < m && k < (int64_t)s_end[row - row0]) {
      const int e = (int)(k - k0);
      sum += s_v[e] * x[s_ci[e]];
      ++k;
    } else {
      if (row < m) y[row] = sum;
      sum = T(0);
      ++row;
    }
  }
  const int64_t t = (int64_t)blockIdx.x * kMergeThreads + threadIdx.x;
  carry_row[t] = row;
  carry_val[t] = sum;
}

// y[r] += the carries of row r, in thread order, by the first thread of each run of equal rows
template <typename T>
__global__ void k_spmv_merge_fixup(int64_t nthreads, int64_t m, const int64_t* __restrict__ carry_row,
                                   const T* __restrict__ carry_val, T* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nthreads) return;
  const int64_t r = carry_row[t];
  if (r >= m || (t > 0 && carry_row[t - 1] == r)) return;
  T acc = T(0);
  for (int64_t u = t; u < nthreads && carry_row[u] == r; ++u) acc += carry_val[u];
  y[r] += acc;
}

// ---- sliced ELL (slice height 32) ---------------------------------------------------------
struct SellData {
  int32_t precision;
  int64_t nrows, ncols, nslices, stored;
  int64_t* slice_ptr;   // nslices + 1 offsets into col / val (multiples of 32)
  int* col;             // stored entries, column-major within a slice, -1 in padded slots
  void* val;
};

// width of each slice: the longest of its 32 rows
__global__ void k_sell_widths(int64_t nrows, int64_t nslices, const int* __restrict__ rp, int64_t* __restrict__ w) {
  const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= nslices) return;
  const int64_t r = s * 32 + lane;
  int len = r < nrows ? rp[r + 1] - rp[r] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
  if (lane == 0) w[s] = len;
}

// exclusive scan of 32 w[s] into slice_ptr (one block; sizes are modest for a kernel-level entry)
__global__ void k_sell_scan(int64_t nslices, const int64_t* __restrict__ w, int64_t* __restrict__ ptr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t acc = 0;
  for (int64_t s = 0; s < nslices; ++s) {
    ptr[s] = acc;
    acc += 32 * w[s];
  }
  ptr[nslices] = acc;
}

template <typename V>
__global__ void k_sell_fill(int64_t nrows, int64_t nslices, const int* __restrict__ rp, const int* __restrict__ ci,
                            const V* __restrict__ v, const int64_t* __restrict__ ptr, int* __restrict__ col,
                            V* __restrict__ val) {
  const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= nslices) return;
  const int64_t r = s * 32 + lane;
  const int64_t base = ptr[s], width = (ptr[s + 1] - ptr[s]) / 32;
  const int beg = r < nrows ? rp[r] : 0, len = r < nrows ? rp[r + 1] - rp[r] : 0;
  for (int64_t j = 0; j < width; ++j) {
    const int64_t at = base + j * 32 + lane;
    if (j < len) {
      col[at] = ci[beg + j];
      val[at] = v[beg + j];
    } else {
      col[at] = -1;
      val[at] = V(0.0f);
    }
  }
}

template <typename T, typename V>
__global__ void __launch_bounds__(256) k_spmv_sell(int64_t nrows, int64_t nslices, const int64_t* __restrict__ ptr,
                                                   const int* __restrict__ col, const V* __restrict__ val,
                                                   const T* __restrict__ x, T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nslices; s += nwarps) {
    const int64_t base = ptr[s], width = (ptr[s + 1] - ptr[s]) >> 5;
    T sum = T(0);
    int64_t j = 0;
    for (; j + 4 <= width; j += 4) {   // four slots in flight per lane
      int c[4];
      T a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        c[u] = __ldg(col + base + (j + u) * 32 + lane);
        a[u] = (T)ldv(val + base + (j + u) * 32 + lane);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c[u] >= 0) sum += a[u] * x[c[u]];
    }
    for (; j < width; ++j) {
      const int c = __ldg(col + base + j * 32 + lane);
      if (c >= 0) sum += (T)ldv(val + base + j * 32 + lane) * x[c];
    }
    const int64_t r = s * 32 + lane;
    if (r < nrows) y[r] = sum;
  }
}

int fail_code(int code, const std::string& msg) {
  cqp::record_error(msg);
  return code;
}

#define SV_CK(x)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (x);                                                                           \
    if (e_ != cudaSuccess) return fail_code(CQP_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T, typename V>
int merge_run(int64_t m, const int32_t* rp, const int32_t* ci, const V* v, const T* x, T* y, cudaStream_t st) {
  int32_t nnz32 = 0;
  SV_CK(cudaMemcpyAsync(&nnz32, rp + m, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SV_CK(cudaStreamSynchronize(st));
  const int64_t nnz = nnz32, total = m + nnz;
  const int64_t blocks = (total + kMergeTile - 1) / kMergeTile;
  if (blocks > 2147483647) return fail_code(CQP_ERR_INVALID, "cqp_spmv_merge: too many entries");
  const int64_t nthreads = blocks * kMergeThreads;
  int64_t* crow = nullptr;
  T* cval = nullptr;
  SV_CK(cudaMallocAsync(&crow, nthreads * sizeof(int64_t), st));
  SV_CK(cudaMallocAsync(&cval, nthreads * sizeof(T), st));
  k_spmv_merge<T, V><<<(unsigned)blocks, kMergeThreads, 0, st>>>(m, nnz, rp, ci, v, x, y, crow, cval);
  k_spmv_merge_fixup<T><<<(unsigned)((nthreads + 255) / 256), 256, 0, st>>>(nthreads, m, crow, cval, y);
  cqp::record_launches(2);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(crow, st);
  cudaFreeAsync(cval, st);
  SV_CK(e);
  SV_CK(cudaStreamSynchronize(st));
  return CQP_OK;
}

}  // namespace

struct cqp_sell {
  SellData d;
};

extern "C" {

int cqp_spmv_merge(int32_t precision, int64_t nrows, int64_t ncols, const int32_t* rowptr, const int32_t* colind,
                   const void* val, const void* x, void* y, void* stream) {
  if (nrows < 0 || ncols < 0 || !rowptr || (nrows > 0 && (!colind || !val || !x || !y)) || precision < 0 ||
      precision > 2)
    return fail_code(CQP_ERR_INVALID, "cqp_spmv_merge: bad arguments");
  if (nrows == 0) return CQP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == 1)
    return merge_run<double, double>(nrows, rowptr, colind, (const double*)val, (const double*)x, (double*)y, st);
  if (precision == 2)
    return merge_run<float, __nv_bfloat16>(nrows, rowptr, colind, (const __nv_bfloat16*)val, (const float*)x,
                                           (float*)y, st);
  return merge_run<float, float>(nrows, rowptr, colind, (const float*)val, (const float*)x, (float*)y, st);
}

int cqp_sell_build(int32_t precision, int64_t nrows, int64_t ncols, const int32_t* rowptr, const int32_t* colind,
                   const void* val, void* stream, cqp_sell** out) {
  if (!out) return fail_code(CQP_ERR_INVALID, "cqp_sell_build: out is NULL");
  *out = nullptr;
  if (nrows < 0 || ncols < 0 || !rowptr || (nrows > 0 && (!colind || !val)) || precision < 0 || precision > 2)
    return fail_code(CQP_ERR_INVALID, "cqp_sell_build: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  SellData d{};
  d.precision = precision;
  d.nrows = nrows;
  d.ncols = ncols;
  d.nslices = (nrows + 31) / 32;
  const size_t vsz = precision == 1 ? 8 : (precision == 2 ? 2 : 4);
  int64_t* w = nullptr;
  SV_CK(cudaMallocAsync(&d.slice_ptr, (d.nslices + 1) * sizeof(int64_t), st));
  SV_CK(cudaMallocAsync(&w, std::max<int64_t>(d.nslices, 1) * sizeof(int64_t), st));
  const unsigned wb = (unsigned)std::max<int64_t>(1, (d.nslices + 7) / 8);
  if (d.nslices > 0) k_sell_widths<<<wb, 256, 0, st>>>(nrows, d.nslices, rowptr, w);
  k_sell_scan<<<1, 32, 0, st>>>(d.nslices, w, d.slice_ptr);
  SV_CK(cudaMemcpyAsync(&d.stored, d.slice_ptr + d.nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SV_CK(cudaStreamSynchronize(st));
  cudaFreeAsync(w, st);
  SV_CK(cudaMallocAsync(&d.col, std::max<int64_t>(d.stored, 1) * sizeof(int), st));
  SV_CK(cudaMallocAsync(&d.val, std::max<int64_t>(d.stored, 1) * vsz, st));
  if (d.nslices > 0) {
    if (precision == 1)
      k_sell_fill<double><<<wb, 256, 0, st>>>(nrows, d.nslices, rowptr, colind, (const double*)val, d.slice_ptr,
                                              d.col, (double*)d.val);
    else if (precision == 2)
      k_sell_fill<__nv_bfloat16><<<wb, 256, 0, st>>>(nrows, d.nslices, rowptr, colind, (const __nv_bfloat16*)val,
                                                     d.slice_ptr, d.col, (__nv_bfloat16*)d.val);
    else
      k_sell_fill<float><<<wb, 256, 0, st>>>(nrows, d.nslices, rowptr, colind, (const float*)val, d.slice_ptr, d.col,
                                             (float*)d.val);
  }
  cqp::record_launches(d.nslices > 0 ? 3 : 1);
  SV_CK(cudaGetLastError());
  SV_CK(cudaStreamSynchronize(st));
  *out = new cqp_sell{d};
  return CQP_OK;
}

int cqp_sell_stored(const cqp_sell* A, int64_t* stored) {
  if (!A || !stored) return fail_code(CQP_ERR_INVALID, "cqp_sell_stored: bad arguments");
  *stored = A->d.stored;
  return CQP_OK;
}

int cqp_spmv_sell(const cqp_sell* A, const void* x, void* y, void* stream) {
  if (!A || (A->d.nrows > 0 && (!x || !y))) return fail_code(CQP_ERR_INVALID, "cqp_spmv_sell: bad arguments");
  const SellData& d = A->d;
  if (d.nslices == 0) return CQP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 1;
  SV_CK(cudaGetDevice(&dev));
  SV_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const unsigned blocks = (unsigned)std::min<int64_t>((d.nslices + 7) / 8, (int64_t)nsm * 8);
  if (d.precision == 1)
    k_spmv_sell<double, double><<<blocks, 256, 0, st>>>(d.nrows, d.nslices, d.slice_ptr, d.col, (const double*)d.val,
                                                        (const double*)x, (double*)y);
  else if (d.precision == 2)
    k_spmv_sell<float, __nv_bfloat16><<<blocks, 256, 0, st>>>(d.nrows, d.nslices, d.slice_ptr, d.col,
                                                              (const __nv_bfloat16*)d.val, (const float*)x, (float*)y);
  else
    k_spmv_sell<float, float><<<blocks, 256, 0, st>>>(d.nrows, d.nslices, d.slice_ptr, d.col, (const float*)d.val,
                                                      (const float*)x, (float*)y);
  cqp::record_launches(1);
  SV_CK(cudaGetLastError());
  return CQP_OK;
}

void cqp_sell_free(cqp_sell* A) {
  if (!A) return;
  cudaFree(A->d.slice_ptr);
  cudaFree(A->d.col);
  cudaFree(A->d.val);
  delete A;
}

}  // extern "C"
