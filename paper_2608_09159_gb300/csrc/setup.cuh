// Setup kernels: layout permutation, transpose, rescaling (Sec. 4.2.2), norm
// estimate (eq. practical-stepsizes).  All arithmetic on the problem data is
// FP64; the scaled matrices are converted to the iterate precision at the end.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

#include "common.cuh"

namespace cqp {

constexpr int kSetupThreads = 256;

inline int grid_for(int64_t n, int threads = kSetupThreads, int cap = 152 * 32) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

#define CQP_GRID_LOOP(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ---- validation: row pointers, colind in range, values finite -------------------
// nnz is the caller's entry count (the length of colind and val), so a malformed
// rowptr cannot make the check itself read past those arrays
__global__ void k_validate_csr(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t* rowptr, const int32_t* colind,
                               const double* val, int* bad) {
  CQP_GRID_LOOP(r, nrows + 1) {
    const int64_t p = rowptr[r];
    if (p < 0 || p > nnz || (r < nrows && p > rowptr[r + 1])) atomicOr(bad, 1);
    if ((r == 0 && p != 0) || (r == nrows && p != nnz)) atomicOr(bad, 1);
  }
  CQP_GRID_LOOP(k, nnz) {
    const int c = colind[k];
    if (c < 0 || c >= ncols) atomicOr(bad, 2);
    if (!isfinite(val[k])) atomicOr(bad, 4);
  }
}
__global__ void k_validate_vec(int64_t n, const double* v, int* bad) {
  CQP_GRID_LOOP(i, n) if (!isfinite(v[i])) atomicOr(bad, 8);
}

// ---- permutation of coordinates into [free | nonneg | soc | rsoc | exp | pow] ----
__global__ void k_gather(int64_t n, const int64_t* perm, const double* in, double* out, double fill) {
  CQP_GRID_LOOP(i, n) out[i] = in ? in[perm[i]] : fill;
}
__global__ void k_remap_cols(int64_t nnz, const int64_t* iperm, const int32_t* in, int32_t* out) {
  CQP_GRID_LOOP(k, nnz) out[k] = (int32_t)iperm[in[k]];
}
__global__ void k_copy_rowptr32(int64_t n1, const int64_t* in, int32_t* out) {
  CQP_GRID_LOOP(i, n1) out[i] = (int32_t)in[i];
}
// R (k x n) columns permuted
__global__ void k_gather_cols(int64_t k, int64_t n, const int64_t* perm, const double* in, double* out) {
  CQP_GRID_LOOP(t, k * n) {
    const int64_t l = t / n, j = t % n;
    out[t] = in[l * n + perm[j]];
  }
}
// permuted sparse P: new row i = old row perm[i], columns remapped
__global__ void k_row_lengths_perm(int64_t n, const int64_t* perm, const int64_t* rp, int32_t* len) {
  CQP_GRID_LOOP(i, n) len[i] = (int32_t)(rp[perm[i] + 1] - rp[perm[i]]);
}
__global__ void k_copy_rows_perm(int64_t n, const int64_t* perm, const int64_t* iperm, const int64_t* rp,
                                 const int32_t* ci, const double* v, const int32_t* nrp, int32_t* nci, double* nv) {
  CQP_GRID_LOOP(i, n) {
    const int64_t o = perm[i];
    int64_t dst = nrp[i];
    for (int64_t t = rp[o]; t < rp[o + 1]; ++t, ++dst) {
      nci[dst] = (int32_t)iperm[ci[t]];
      nv[dst] = v[t];
    }
  }
}

// ---- exclusive scan of int32 counts into int32 offsets (n entries -> n+1) ----------
// three passes: per-block totals, serial scan of the totals, per-block scan + offset
__global__ void k_scan_block_totals(int64_t n, const int32_t* in, int64_t per_block, int64_t* tot) {
  const int64_t b0 = blockIdx.x * per_block, b1 = min(n, b0 + per_block);
  int64_t s = 0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += in[i];
  __shared__ int64_t red[kSetupThreads];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = red[0];
}
__global__ void k_scan_totals(int nb, int64_t* tot) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t s = 0;
    for (int b = 0; b < nb; ++b) { const int64_t t = tot[b]; tot[b] = s; s += t; }
    tot[nb] = s;
  }
}
__global__ void k_scan_apply(int64_t n, const int32_t* in, int64_t per_block, const int64_t* tot, int32_t* out) {
  // serial chunks per thread, then a block scan of the chunk sums
  __shared__ int64_t sums[kSetupThreads];
  const int64_t b0 = blockIdx.x * per_block, b1 = min(n, b0 + per_block);
  const int64_t len = b1 - b0;
  const int64_t chunk = (len + blockDim.x - 1) / blockDim.x;
  const int64_t c0 = b0 + threadIdx.x * chunk, c1 = min(b1, c0 + chunk);
  int64_t s = 0;
  for (int64_t i = c0; i < c1; ++i) s += in[i];
  sums[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = tot[blockIdx.x];
    for (int t = 0; t < (int)blockDim.x; ++t) { const int64_t v = sums[t]; sums[t] = acc; acc += v; }
  }
  __syncthreads();
  int64_t acc = sums[threadIdx.x];
  for (int64_t i = c0; i < c1; ++i) { out[i] = (int32_t)acc; acc += in[i]; }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (int32_t)tot[gridDim.x];
}

// ---- transpose ----------------------------------------------------------------
__global__ void k_count_cols(int64_t nnz, const int32_t* ci, int32_t* cnt) {
  CQP_GRID_LOOP(k, nnz) atomicAdd(&cnt[ci[k]], 1);
}
__global__ void k_scatter_transpose(int64_t m, const int32_t* rp, const int32_t* ci, int32_t* cursor, int32_t* tci,
                                    int32_t* tmap) {
  CQP_GRID_LOOP(r, m) {
    for (int k = rp[r]; k < rp[r + 1]; ++k) {
      const int pos = atomicAdd(&cursor[ci[k]], 1);
      tci[pos] = (int32_t)r;
      tmap[pos] = k;
    }
  }
}
// Order every transposed row by (original row, position in A): a deterministic layout.
// Rows of at most kShortSeg entries are insertion-sorted by one thread (stable, and two
// entries of one row of A arrive in their CSR order from the same scattering thread); longer
// ones are listed for k_sort_long_segments (one block, bitonic sort in shared memory) and,
// beyond kSegSortCap entries, k_sort_huge_segments.
constexpr int kShortSeg = 32;
constexpr int kSegSortCap = 4096;
constexpr int kSegSortThreads = 512;
__global__ void k_sort_segments(int64_t n, const int32_t* trp, int32_t* tci, int32_t* tmap, int32_t* long_list,
                                unsigned* long_count, unsigned* long_max) {
  CQP_GRID_LOOP(j, n) {
    const int b = trp[j], e = trp[j + 1];
    if (e - b > kShortSeg) {
      long_list[atomicAdd(long_count, 1u)] = (int32_t)j;
      atomicMax(long_max, (unsigned)(e - b));
      continue;
    }
    for (int a = b + 1; a < e; ++a) {
      const int key = tci[a], val = tmap[a];
      int t = a - 1;
      while (t >= b && tci[t] > key) { tci[t + 1] = tci[t]; tmap[t + 1] = tmap[t]; --t; }
      tci[t + 1] = key;
      tmap[t + 1] = val;
    }
  }
}

// (row, position) packed so that unsigned order is the layout order
__device__ __forceinline__ unsigned long long seg_key(const int32_t* tci, const int32_t* tmap, int i) {
  return ((unsigned long long)(uint32_t)tci[i] << 32) | (uint32_t)tmap[i];
}
// sorts entries [b, b + len) of tci/tmap (len <= kSegSortCap) with the calling block: bitonic
// sort of the packed keys in shared memory, padded to a power of two with the largest key
__device__ void block_sort_run(int32_t* tci, int32_t* tmap, int b, int len, unsigned long long* s) {
  int P = 1;
  while (P < len) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < len ? seg_key(tci, tmap, b + i) : ~0ull;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = s[i], c = s[ixj];
          if ((a > c) == ((i & k) == 0)) {
            s[i] = c;
            s[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    tci[b + i] = (int32_t)(s[i] >> 32);
    tmap[b + i] = (int32_t)(s[i] & 0xffffffffull);
  }
  __syncthreads();
}
__global__ void __launch_bounds__(kSegSortThreads) k_sort_long_segments(const int32_t* trp, int32_t* tci,
                                                                        int32_t* tmap, const int32_t* list,
                                                                        const unsigned* count) {
  __shared__ unsigned long long s[kSegSortCap];
  const unsigned cnt = *count;
  for (unsigned i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int j = list[i];
    const int b = trp[j], len = trp[j + 1] - b;
    if (len <= kSegSortCap) block_sort_run(tci, tmap, b, len, s);
  }
}
// rows longer than kSegSortCap (one block): kSegSortCap-entry runs sorted in shared memory,
// then merged bottom-up by thread 0 through buf (as many entries as the longest row)
__global__ void __launch_bounds__(kSegSortThreads) k_sort_huge_segments(const int32_t* trp, int32_t* tci,
                                                                        int32_t* tmap, const int32_t* list,
                                                                        const unsigned* count, unsigned long long* buf) {
  __shared__ unsigned long long s[kSegSortCap];
  const unsigned cnt = *count;
  for (unsigned i = 0; i < cnt; ++i) {
    const int j = list[i];
    const int b = trp[j], L = trp[j + 1] - b;
    if (L <= kSegSortCap) continue;
    for (int r = 0; r < L; r += kSegSortCap) block_sort_run(tci, tmap, b + r, min(kSegSortCap, L - r), s);
    if (threadIdx.x == 0) {
      for (int w = kSegSortCap; w < L; w <<= 1) {
        for (int lo = 0; lo < L; lo += 2 * w) {
          const int mid = min(lo + w, L), hi = min(lo + 2 * w, L);
          int p = lo, q = mid, o = lo;
          while (p < mid && q < hi) {
            const unsigned long long kp = seg_key(tci, tmap, b + p), kq = seg_key(tci, tmap, b + q);
            if (kp <= kq) { buf[o++] = kp; ++p; } else { buf[o++] = kq; ++q; }
          }
          while (p < mid) { buf[o++] = seg_key(tci, tmap, b + p); ++p; }
          while (q < hi) { buf[o++] = seg_key(tci, tmap, b + q); ++q; }
        }
        for (int t = 0; t < L; ++t) {
          tci[b + t] = (int32_t)(buf[t] >> 32);
          tmap[b + t] = (int32_t)(buf[t] & 0xffffffffull);
        }
      }
    }
    __syncthreads();
  }
}

// ---- rescaling (Ruiz l_inf, Pock-Chambolle, cone-preserving aggregation) -------------
// row statistic: max |a| (mode 0) or sum |a|^p (mode 1) over each row of A
__global__ void k_row_stat(int64_t m, const int32_t* rp, const double* v, int mode, double p, double* out) {
  CQP_GRID_LOOP(r, m) {
    double s = 0.0;
    for (int k = rp[r]; k < rp[r + 1]; ++k) {
      const double a = fabs(v[k]);
      s = mode == 0 ? fmax(s, a) : s + pow(a, p);
    }
    out[r] = s;
  }
}
// column statistic through the transpose structure (tmap indexes A's values)
__global__ void k_col_stat(int64_t n, const int32_t* trp, const int32_t* tmap, const double* v, int mode, double p,
                           double* out) {
  CQP_GRID_LOOP(j, n) {
    double s = 0.0;
    for (int k = trp[j]; k < trp[j + 1]; ++k) {
      const double a = fabs(v[tmap[k]]);
      s = mode == 0 ? fmax(s, a) : s + pow(a, p);
    }
    out[j] = s;
  }
}
// f = sqrt(stat) (1 where the statistic vanishes)
__global__ void k_sqrt_or_one(int64_t n, double* f) {
  CQP_GRID_LOOP(i, n) f[i] = f[i] > 0.0 ? sqrt(f[i]) : 1.0;
}
// cone blocks of the permuted layout: [b0, b1) coordinate ranges given by offsets
// (SOC, RSOC) or by a base and width 3 (EXP, POW); max (mode 0) or RMS (mode 1)
// ---- column blocks of A for the dual step's product (entry (r, c) is in block c / width) ----
// cnt[b * rows + r] = number of entries of row r in block b
__global__ void k_cb_count(int64_t rows, const int* rp, const int* ci, int64_t width, int nb, int* cnt) {
  CQP_GRID_LOOP(r, rows) {
    const int e0 = rp[r], e1 = rp[r + 1];
    for (int b = 0; b < nb; ++b) {
      int c = 0;
      for (int e = e0; e < e1; ++e) c += (int64_t)ci[e] / width == b;
      cnt[(int64_t)b * rows + r] = c;
    }
  }
}
// entries of row r in block b, in row order, to out[bp[b * rows + r] ...]
template <typename T>
__global__ void k_cb_scatter(int64_t rows, const int* rp, const int* ci, const T* v, int64_t width, int nb,
                             const int* bp, int* oci, T* ov) {
  CQP_GRID_LOOP(r, rows) {
    const int e0 = rp[r], e1 = rp[r + 1];
    for (int b = 0; b < nb; ++b) {
      int pos = bp[(int64_t)b * rows + r];
      for (int e = e0; e < e1; ++e)
        if ((int64_t)ci[e] / width == b) {
          oci[pos] = ci[e];
          ov[pos] = v[e];
          ++pos;
        }
    }
  }
}

// *bad = 1 unless rp[r] = L r for every r <= rows (rows of exactly L entries)
__global__ void k_check_uniform(int64_t rows, const int* rp, int L, int* bad) {
  CQP_GRID_LOOP(r, rows + 1) if ((int64_t)rp[r] != (int64_t)L * r) *bad = 1;
}

// BF16 matrix storage: v <- BF16(FP32(v)), rounding to nearest even at each step
__global__ void k_round_bf16(int64_t n, double* v) {
  CQP_GRID_LOOP(i, n) v[i] = (double)__bfloat162float(__float2bfloat16_rn((float)v[i]));
}

// f <- 2^round(log2 f) for positive finite f (the power of two nearest in ratio: a mantissa
// m in [1/2, 1) rounds up at m >= 1/sqrt 2); scaling by such factors keeps BF16 values exact
__host__ __device__ inline double pow2_round(double f) {
  if (!(f > 0.0) || !isfinite(f)) return f;
  int e = 0;
  const double m = frexp(f, &e);
  return ldexp(1.0, m >= 0.70710678118654752440 ? e : e - 1);
}
// c <- its power of two (pow2_round), f <- the ratio new / old that brings a scaled matrix along
__global__ void k_pow2_ratio(int64_t n, double* c, double* f) {
  CQP_GRID_LOOP(i, n) {
    const double p = pow2_round(c[i]);
    f[i] = p / c[i];
    c[i] = p;
  }
}

// out[i] = BF16(in[map[i]]) (map null: in[i]); the values are exactly representable here
__global__ void k_to_bf16(int64_t n, const int32_t* map, const double* in, __nv_bfloat16* out) {
  CQP_GRID_LOOP(i, n) out[i] = __float2bfloat16_rn((float)in[map ? map[i] : i]);
}

// slice blocks: fix[e] = flag[e] * col[base + 3 e + 1] / beta_b (flag 1 for a slice, 0 for a cone)
__global__ void k_slice_fix(int64_t nblk, int64_t base, const double* col, double beta_b, double* fix) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nblk && fix[e] != 0.0) fix[e] = col[base + 3 * e + 1] / beta_b;
}

__global__ void k_aggregate_blocks(int64_t nblk, const int64_t* off, int64_t base, int width, int mode, double* f) {
  CQP_GRID_LOOP(b, nblk) {
    const int64_t s = off ? off[b] : base + width * b;
    const int64_t e = off ? off[b + 1] : s + width;
    double a = 0.0;
    for (int64_t i = s; i < e; ++i) a = mode == 0 ? fmax(a, f[i]) : a + f[i] * f[i];
    if (mode == 1) a = sqrt(a / (double)(e - s));
    for (int64_t i = s; i < e; ++i) f[i] = a;
  }
}
// A <- diag(1/rowf) A diag(1/colf); col *= colf; row *= rowf
__global__ void k_scale_matrix(int64_t m, const int32_t* rp, const int32_t* ci, double* v, const double* rowf,
                               const double* colf) {
  CQP_GRID_LOOP(r, m) {
    const double fr = rowf[r];
    for (int k = rp[r]; k < rp[r + 1]; ++k) v[k] /= fr * colf[ci[k]];
  }
}
__global__ void k_mul(int64_t n, double* a, const double* f) { CQP_GRID_LOOP(i, n) a[i] *= f[i]; }
__global__ void k_div(int64_t n, double* a, const double* f) { CQP_GRID_LOOP(i, n) a[i] /= f[i]; }
__global__ void k_div2(int64_t n, double* a, const double* f) { CQP_GRID_LOOP(i, n) a[i] /= f[i] * f[i]; }
__global__ void k_fill(int64_t n, double* a, double v) { CQP_GRID_LOOP(i, n) a[i] = v; }
__global__ void k_scal(int64_t n, double* a, double s) { CQP_GRID_LOOP(i, n) a[i] *= s; }
// P~_ij = P_ij / (col_i col_j)
__global__ void k_scale_sym(int64_t n, const int32_t* rp, const int32_t* ci, double* v, const double* col) {
  CQP_GRID_LOOP(r, n) {
    for (int k = rp[r]; k < rp[r + 1]; ++k) v[k] /= col[r] * col[ci[k]];
  }
}
// R~ = R diag(1/col)
__global__ void k_scale_cols(int64_t k, int64_t n, double* R, const double* col) {
  CQP_GRID_LOOP(t, k * n) R[t] /= col[t % n];
}
// full diagonal of Q~ = diag(qd) + P + R' D R
__global__ void k_full_diag(int64_t n, const double* qd, const int32_t* prp, const int32_t* pci, const double* pv,
                            int64_t k, const double* R, const double* D, double* jd) {
  CQP_GRID_LOOP(i, n) {
    double q = qd[i];
    if (prp)
      for (int t = prp[i]; t < prp[i + 1]; ++t)
        if (pci[t] == i) q += pv[t];
    for (int64_t l = 0; l < k; ++l) {
      const double rl = R[l * n + i];
      if (rl == 0.0) continue;
      double s = 0.0;
      for (int64_t l2 = 0; l2 < k; ++l2) s += D[l * k + l2] * R[l2 * n + i];
      q += rl * s;
    }
    jd[i] = q;
  }
}
template <typename T>
__global__ void k_convert(int64_t n, const double* in, T* out) {
  CQP_GRID_LOOP(i, n) out[i] = T(in[i]);
}
template <typename T>
__global__ void k_gather_convert(int64_t n, const int32_t* idx, const double* in, T* out) {
  CQP_GRID_LOOP(i, n) out[i] = T(in[idx[i]]);
}

// ---- reductions (FP64, two-level, deterministic) ----------------------------------
__global__ void k_dot_partial(int64_t n, const double* a, const double* b, double* part) {
  double s = 0.0;
  CQP_GRID_LOOP(i, n) s += a[i] * (b ? b[i] : a[i]);
  __shared__ double red[kSetupThreads];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_sum_partials(int nb, const double* part, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    *out = s;
  }
}

// ---- norm-estimate pieces: y = A x (FP64 accumulation over T values) ----------------
template <typename T>
__global__ void k_spmv_simple(int64_t m, const int32_t* rp, const int32_t* ci, const T* v, const double* x, double* y) {
  CQP_GRID_LOOP(r, m) {
    double s = 0.0;
    for (int k = rp[r]; k < rp[r + 1]; ++k) s += (double)v[k] * x[ci[k]];
    y[r] = s;
  }
}

// ---- general form (rows lo <= Ax <= hi, box blocks) ---------------------------------
// no NaN and lo <= hi (on masked coordinates when mask is given)
__global__ void k_validate_bounds(int64_t n, const double* lo, const double* hi, const uint8_t* mask, int* bad) {
  CQP_GRID_LOOP(i, n) {
    if (mask && !mask[i]) continue;
    const double l = lo[i], h = hi[i];
    if (l != l || h != h || l > h || l == INFINITY || h == -INFINITY) atomicOr(bad, 32);
  }
}
// per-row magnitude of the right-hand side: the largest finite bound magnitude
__global__ void k_bound_mag(int64_t m, const double* lo, const double* hi, double* mag) {
  CQP_GRID_LOOP(i, m) {
    double a = 0.0;
    if (isfinite(lo[i])) a = fmax(a, fabs(lo[i]));
    if (isfinite(hi[i])) a = fmax(a, fabs(hi[i]));
    mag[i] = a;
  }
}
// scaled box bounds of the free segment: x~ = col x / beta_b; free coordinates unbounded
template <typename T>
__global__ void k_box_bounds(int64_t nf, const int64_t* perm, const uint8_t* mask, const double* lo, const double* hi,
                             const double* col, double beta_b, T* olo, T* ohi) {
  CQP_GRID_LOOP(i, nf) {
    const int64_t o = perm[i];
    if (mask[o]) {
      olo[i] = T(lo[o] * col[i] / beta_b);
      ohi[i] = T(hi[o] * col[i] / beta_b);
    } else {
      olo[i] = T(-INFINITY);
      ohi[i] = T(INFINITY);
    }
  }
}

// ---- start vector of the norm estimate (reading): entry j is 1/2 + U_j, U_j in [0, 1) the
// top 53 bits of output j+1 of the SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014)
// started from state 0.  Entries are keyed by the caller's coordinate index, so the start
// does not depend on the solver's permutation.  An all-ones start can be exactly orthogonal
// to the top singular subspace (e.g. the Lasso reformulation with A = I), and the estimate
// then stalls at a smaller singular value; the positive perturbation keeps all-ones'
// overlap with the leading direction of rescaled matrices (same iteration count there).
__device__ __forceinline__ double power_start_value(uint64_t idx) {
  uint64_t z = idx * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return 0.5 + (double)(z >> 11) * (1.0 / 9007199254740992.0);
}
// z[i] = start value of the caller's coordinate perm[i] (unnormalised)
__global__ void k_power_start(int64_t n, const int64_t* perm, double* z) {
  CQP_GRID_LOOP(i, n) z[i] = power_start_value((uint64_t)perm[i] + 1);
}

// ---- largest eigenvalue of a symmetric tridiagonal matrix (diagonal a[0..k), off-diagonal
// b[0..k-1)) by one warp: 32-point multisection of the Gershgorin bracket on the Sturm count
// (Golub and Van Loan, Sec. 8.4.1).  Lane l evaluates the count at the (l+1)-th of 32 interior
// points through the division-free recurrence of the leading principal minors
// p_i = (a_i - x) p_{i-1} - b_{i-1}^2 p_{i-2} (a sign change = an eigenvalue below x; an exact
// zero counts as a change), rescaled by 2^-+500 to stay in range; the bracket shrinks 33-fold
// per step.  Every lane returns the same value.
__device__ __forceinline__ int sturm_below(const double* a, const double* b, int k, double x) {
  double pm = 1.0, p = a[0] - x;
  int below = p <= 0.0 ? 1 : 0;
  for (int i = 1; i < k; ++i) {
    const double q = (a[i] - x) * p - b[i - 1] * b[i - 1] * pm;
    pm = p;
    p = q;
    const double ap = fabs(p);
    if (ap > 0x1p500) { p *= 0x1p-500; pm *= 0x1p-500; }
    else if (ap < 0x1p-500 && ap > 0.0) { p *= 0x1p500; pm *= 0x1p500; }
    if (p == 0.0 || (p < 0.0) != (pm < 0.0)) ++below;
  }
  return below;
}
__device__ double tridiag_max_eig_warp(const double* a, const double* b, int k, int lane) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int step = 0; step < 40 && hi - lo > 1e-15 * fabs(hi); ++step) {
    const double h = (hi - lo) / 33.0;
    const double x = lo + h * (double)(lane + 1);
    const unsigned above = __ballot_sync(0xffffffffu, sturm_below(a, b, k, x) == k);
    if (above == 0u) {
      lo = lo + h * 32.0;
    } else {
      const int l0 = __ffs((int)above) - 1;
      const double nhi = lo + h * (double)(l0 + 1);
      lo = l0 > 0 ? lo + h * (double)l0 : lo;
      hi = nhi;
    }
  }
  return hi;
}

// ---- ||A~||_2 by the Lanczos process on A~'A~, all steps in one cooperative launch
// (eq. practical-stepsizes; reading: SplitMix64 start, no reorthogonalisation, stop at `tol`
// relative change of sigma = sqrt(theta_max(T_j)), at beta_j = 0, or after `iters` steps,
// at most kMaxLanczos).  The current vector is v = zscale z, the previous one zp.  Each step:
// w = A v (slot 0: alpha = ||w||^2 = v'A'A v), then z = A'w - alpha v - beta_prev zp with
// zp = v (slot 1: beta^2 = ||z||^2), two grid barriers and no host round trip.  Every block
// combines the partials in the same fixed order and runs the same tridiagonal eigenvalue
// search (warp 0), so all blocks take the same stop decision.  out[0] = ||A~||_2 estimate,
// out[1] = steps.
constexpr int kPowerThreads = 512;
constexpr int kMaxLanczos = 256;

// one CSR row product in FP64, eight entries at a time (indices and values first, then
// the gathers together) so each thread keeps several loads in flight
template <typename T>
__device__ __forceinline__ double power_row(int beg, int end, const int32_t* __restrict__ ci,
                                            const T* __restrict__ v, const double* x) {
  double s = 0.0;
  for (int k = beg; k < end; k += 8) {
    int j[8];
    double a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool ok = k + u < end;
      j[u] = ok ? __ldg(ci + k + u) : -1;
      a[u] = ok ? (double)__ldg(v + k + u) : 0.0;
    }
    double g[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) g[u] = j[u] >= 0 ? x[j[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += a[u] * g[u];
  }
  return s;
}

template <typename T>
__global__ void __launch_bounds__(kPowerThreads, 1)
    k_power(int64_t m, int64_t n, const int32_t* __restrict__ a_rp, const int32_t* __restrict__ a_ci,
            const T* __restrict__ a_v, const int32_t* __restrict__ t_rp, const int32_t* __restrict__ t_ci,
            const T* __restrict__ t_v, double* z, double* zp, double* w, double* part, GridBarrier bar, int iters,
            double tol, double* out) {
  GridTeam team;
  team.init(bar, part);
  __shared__ double red[kPowerThreads / 32];
  __shared__ double tot[2];
  __shared__ double al[kMaxLanczos], be[kMaxLanczos];
  __shared__ double theta;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  if (iters > kMaxLanczos) iters = kMaxLanczos;
  double sig = 0.0, zscale = 1.0, beta_prev = 0.0;
  int it = 0;
  for (; it < iters; ++it) {
    double acc[1] = {0.0};
    for (int64_t r = tid; r < m; r += nt) {
      const double s = power_row(a_rp[r], a_rp[r + 1], a_ci, a_v, z) * zscale;
      w[r] = s;
      acc[0] += s * s;
    }
    block_sum<1>(acc, red, tot);
    if (threadIdx.x == 0) team.publish(0, tot[0]);
    if (!team.sync()) break;
    team.gather(1, tot);
    const double alpha = tot[0];
    acc[0] = 0.0;
    for (int64_t j = tid; j < n; j += nt) {
      const double vj = z[j] * zscale, vp = zp[j];
      const double s = power_row(t_rp[j], t_rp[j + 1], t_ci, t_v, w) - alpha * vj - beta_prev * vp;
      zp[j] = vj;
      z[j] = s;
      acc[0] += s * s;
    }
    block_sum<1>(acc, red, tot);
    if (threadIdx.x == 0) team.publish(1, tot[0]);
    if (!team.sync()) break;
    team.gather(2, tot);
    const double beta = sqrt(tot[1]);
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
    if (done) {
      ++it;
      break;
    }
    if (threadIdx.x == 0) be[it] = beta;
    zscale = 1.0 / beta;
    beta_prev = beta;
    __syncthreads();
  }
  if (tid == 0) {
    out[0] = sig;
    out[1] = (double)it;
  }
}

}  // namespace cqp
