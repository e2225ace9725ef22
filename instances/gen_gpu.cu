// Device-side generator of the large sparse QP of instances.large_qp (inputs only: no
// solver arithmetic).  Every draw is Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011)
// at counter (index, 0, 0, 0) under key (seed, stream), mapped to U[0,1) with 53 bits
// (words 0, 1) and to N(0,1) by Box-Muller (words 0,1 and 2,3), exactly as the numpy
// definition in instances/__init__.py; products and sums are rounded one operation at a
// time so the arrays match the CPU generator.
#include <cstdint>

namespace {

__device__ __forceinline__ void philox(uint32_t seed, uint32_t stream, uint64_t idx, uint32_t out[4]) {
  uint32_t c0 = (uint32_t)idx, c1 = (uint32_t)(idx >> 32), c2 = 0u, c3 = 0u;
  uint32_t k0 = seed, k1 = stream;
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
  const uint64_t m = ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
  return (double)m * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double uniform_at(uint32_t seed, uint32_t stream, uint64_t idx) {
  uint32_t w[4];
  philox(seed, stream, idx, w);
  return u53(w[0], w[1]);
}

__device__ __forceinline__ double normal_at(uint32_t seed, uint32_t stream, uint64_t idx) {
  uint32_t w[4];
  philox(seed, stream, idx, w);
  const double u1 = u53(w[0], w[1]), u2 = u53(w[2], w[3]);
  const double two_pi = 6.283185307179586;   // 2 * pi rounded to double, as numpy forms it
  const double r = sqrt(__dmul_rn(-2.0, log1p(-u1)));
  return __dmul_rn(r, cos(__dmul_rn(two_pi, u2)));
}

constexpr int kPerRow = 20;

// rows of A (20 stored entries each, sorted by column, repeats merged into the first
// entry) and b = A x0 with x0_j = |N(0,1)| summed in stored order
__global__ void k_rows(uint32_t seed, int64_t n, int64_t m, int64_t* rowptr, int32_t* colind, double* val, double* b) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    int64_t col[kPerRow];
    double v[kPerRow];
    for (int e = 0; e < kPerRow; ++e) {
      const uint64_t idx = (uint64_t)r * kPerRow + e;
      int64_t cj = (int64_t)__dmul_rn(uniform_at(seed, 1, idx), (double)n);
      col[e] = cj < n - 1 ? cj : n - 1;
      v[e] = normal_at(seed, 2, idx);
    }
    // stable insertion sort by column
    for (int e = 1; e < kPerRow; ++e) {
      const int64_t ck = col[e];
      const double vk = v[e];
      int f = e - 1;
      while (f >= 0 && col[f] > ck) {
        col[f + 1] = col[f];
        v[f + 1] = v[f];
        --f;
      }
      col[f + 1] = ck;
      v[f + 1] = vk;
    }
    int first = 0;
    for (int e = 1; e < kPerRow; ++e) {
      if (col[e] == col[first]) {
        v[first] = __dadd_rn(v[first], v[e]);
        v[e] = 0.0;
      } else {
        first = e;
      }
    }
    double s = 0.0;
    for (int e = 0; e < kPerRow; ++e) {
      const double x0 = fabs(normal_at(seed, 4, (uint64_t)col[e]));
      s = __dadd_rn(s, __dmul_rn(v[e], x0));
      colind[r * kPerRow + e] = (int32_t)col[e];
      val[r * kPerRow + e] = v[e];
    }
    b[r] = s;
    rowptr[r] = r * kPerRow;
    if (r == m - 1) rowptr[m] = m * kPerRow;
  }
}

// c ~ N(0,1), q ~ U[0,1), and P: rows {j: w, partner: -w} of the matching Laplacian
__global__ void k_cols(uint32_t seed, int64_t n, int64_t d, double* c, double* q, int64_t* p_rowptr, int32_t* p_colind,
                       double* p_val) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    c[j] = normal_at(seed, 3, (uint64_t)j);
    q[j] = uniform_at(seed, 5, (uint64_t)j);
    const bool even = (j % 2) == 0;
    const int64_t partner = even ? (j + d) % n : ((j - d) % n + n) % n;
    const int64_t anchor = even ? j : partner;
    const double w = fabs(normal_at(seed, 6, (uint64_t)anchor));
    const bool lo = j < partner;
    p_colind[2 * j] = (int32_t)(lo ? j : partner);
    p_colind[2 * j + 1] = (int32_t)(lo ? partner : j);
    p_val[2 * j] = lo ? w : -w;
    p_val[2 * j + 1] = lo ? -w : w;
    p_rowptr[j] = 2 * j;
    if (j == n - 1) p_rowptr[n] = 2 * n;
  }
}

}  // namespace

extern "C" int igen_large_qp(uint32_t seed, int64_t n, int64_t m, int64_t d, int64_t* a_rowptr, int32_t* a_colind,
                             double* a_val, double* b, double* c, double* q, int64_t* p_rowptr, int32_t* p_colind,
                             double* p_val, void* stream) {
  if (n < 2 || (n % 2) != 0 || m < 1 || d < 1 || (d % 2) == 0 || m * kPerRow >= (int64_t(1) << 31) ||
      2 * n >= (int64_t(1) << 31))
    return -1;
  cudaStream_t st = (cudaStream_t)stream;
  k_rows<<<152 * 16, 256, 0, st>>>(seed, n, m, a_rowptr, a_colind, a_val, b);
  k_cols<<<152 * 16, 256, 0, st>>>(seed, n, d, c, q, p_rowptr, p_colind, p_val);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
