// Learned warm start for batches of portfolio QPs: a 3-layer BF16 MLP on per-asset
// features proposes the primal start x0 (softmax of the asset scores within each
// instance, so 1'x0 = 1 and x0 >= 0) and two scalar duals per instance (budget row
// and risk row), from which the whole dual start follows (at an optimum the duals
// of the factor and idiosyncratic rows are lambda * (w_F, w_D) with lambda = y_t / t).
// The paper has no learned component; the solver it feeds is unchanged and a cold
// start stays the fallback.
//
// Kernels: features, a tiled BF16 tensor-core GEMM (FP32 accumulation) with fused
// bias/ReLU or split-K epilogues, the score/softmax/dual head forward and backward,
// the training loss gradient, Adam, and the assembly of (x0, y0) for the batch.
#include <cuda_bf16.h>
#include <mma.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <type_traits>

#include "cqp.h"
#include "cqp_mlp.h"
#include "common.cuh"

namespace cqp {
void record_error(const std::string& msg);
void record_launches(long long k);
int gemm_tc_try(int32_t trans_a, int32_t trans_b, int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda,
                const uint16_t* B, int64_t ldb, void* C, int64_t ldc, const float* bias, int32_t epilogue,
                cudaStream_t st, int* rc);
int gemm_tc_status(cudaStream_t st);
}  // namespace cqp

namespace {

using bf16 = __nv_bfloat16;
using namespace nvcuda;

constexpr int kHid = CQP_WS_HIDDEN;
constexpr int kFeat = CQP_WS_FEATURES;

int fail_with(int code, const std::string& msg) {
  cqp::record_error(msg);
  return code;
}

#define MLP_CK(x)                                                                                          \
  do {                                                                                                     \
    cudaError_t e_ = (x);                                                                                  \
    if (e_ != cudaSuccess) return fail_with(CQP_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------------------
// features of asset j of instance i (portfolio batch layout: x_off, n_assets;
// mu = -c, D = q, F_j = column of R, sigma_bar = last entry of b of the instance)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ws_features(int64_t count, const int64_t* x_off, const int64_t* n_assets,
                                                      const int64_t* asset_off, const int64_t* row_off,
                                                      const int32_t* rank, const double* c, const double* q,
                                                      const double* R, int64_t ldr, const double* b, bf16* X) {
  // per-instance statistics: mean and second moment of mu, mean of D, mean of |F_j|^2,
  // max of the return-to-risk ratio mu / (D + |F_j|^2)
  __shared__ double red[8][5];
  __shared__ double st[5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int64_t x0 = x_off[i], na = n_assets[i], a0 = asset_off[i];
    const int k = rank[i];
    double v[5] = {0.0, 0.0, 0.0, 0.0, -1e300};
    for (int64_t j = threadIdx.x; j < na; j += blockDim.x) {
      const double mu = -c[x0 + j], d = q[x0 + j];
      double f2 = 0.0;
      for (int l = 0; l < k; ++l) {
        const double r = R[(int64_t)l * ldr + x0 + j];
        f2 += r * r;
      }
      v[0] += mu;
      v[1] += mu * mu;
      v[2] += d;
      v[3] += f2;
      v[4] = fmax(v[4], mu / (d + f2));
    }
    for (int t = 0; t < 4; ++t) v[t] = cqp::warp_sum(v[t]);
    for (int o = 16; o; o >>= 1) v[4] = fmax(v[4], __shfl_xor_sync(0xffffffffu, v[4], o));
    if (lane == 0)
      for (int t = 0; t < 5; ++t) red[warp][t] = v[t];
    __syncthreads();
    if (threadIdx.x == 0) {
      double a[5] = {0.0, 0.0, 0.0, 0.0, -1e300};
      for (int w = 0; w < nw; ++w) {
        for (int t = 0; t < 4; ++t) a[t] += red[w][t];
        a[4] = fmax(a[4], red[w][4]);
      }
      const double inv = na > 0 ? 1.0 / (double)na : 0.0;
      st[0] = a[0] * inv;
      st[1] = sqrt(fmax(a[1] * inv - st[0] * st[0], 0.0)) + 1e-12;
      st[2] = a[2] * inv + 1e-300;
      st[3] = a[3] * inv + 1e-300;
      st[4] = a[4];
    }
    __syncthreads();
    const double sig = b[row_off[i + 1] - 1];
    for (int64_t j = threadIdx.x; j < na; j += blockDim.x) {
      const double mu = -c[x0 + j], d = q[x0 + j];
      double f2 = 0.0;
      for (int l = 0; l < k; ++l) {
        const double r = R[(int64_t)l * ldr + x0 + j];
        f2 += r * r;
      }
      const double rr = mu / (d + f2);
      float f[kFeat];
      f[0] = (float)(20.0 * mu);
      f[1] = (float)(20.0 * d);
      f[2] = (float)(100.0 * f2);
      f[3] = (float)(0.1 * rr);
      f[4] = (float)(50.0 * (mu - st[0]));
      f[5] = (float)(log((double)na) / 8.0);
      f[6] = (float)(k / 50.0);
      f[7] = (float)(10.0 * sig);
      f[8] = (float)((mu - st[0]) / st[1]);
      f[9] = (float)(d / st[2]);
      f[10] = (float)(f2 / st[3]);
      f[11] = (float)(st[4] > 0.0 ? rr / st[4] : 0.0);
      for (int t = 12; t < kFeat; ++t) f[t] = 0.f;
      bf16* xr = X + (a0 + j) * kFeat;
      for (int t = 0; t < kFeat; ++t) xr[t] = __float2bfloat16(f[t]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// C (M x N) = op(A) (M x K) * op(B) (K x N) on the tensor cores (BF16 in, FP32
// accumulate).  op(A) = A (row-major, lda) or A' (A stored K x M row-major);
// op(B) likewise.  Block tile 128 x 128 x 32, 8 warps of 32 x 64.  Epilogues:
// 0 store FP32, 1 store FP32 + bias, 2 store BF16 with bias and ReLU,
// 3 atomically add FP32 (split-K over gridDim.z), 4 store BF16.
// ---------------------------------------------------------------------------
constexpr int TM = 128, TN = 128, TK = 32;
constexpr int APAD = 8, BPAD = 8;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_bf16(int64_t M, int64_t N, int64_t K, const bf16* __restrict__ A,
                                                   int64_t lda, const bf16* __restrict__ B, int64_t ldb, void* C,
                                                   int64_t ldc, const float* __restrict__ bias, int epi,
                                                   int64_t k_chunk) {
  __shared__ __align__(32) bf16 As[TM][TK + APAD];
  __shared__ __align__(32) bf16 Bs[TK][TN + BPAD];
  __shared__ __align__(32) float Cs[8][16 * 16];
  const int64_t m0 = blockIdx.y * (int64_t)TM, n0 = blockIdx.x * (int64_t)TN;
  const int64_t kb = blockIdx.z * k_chunk, ke = min(K, kb + k_chunk);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp >> 1, wn = warp & 1;   // 4 x 2 warps, each 32 x 64
  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) wmma::fill_fragment(acc[i][j], 0.0f);
  for (int64_t k0 = kb; k0 < ke; k0 += TK) {
    // stage op(A) tile (TM x TK) and op(B) tile (TK x TN), zero outside the matrices
    for (int e = threadIdx.x; e < TM * TK; e += blockDim.x) {
      int mm, kk;
      if (TA) { kk = e / TM; mm = e % TM; } else { mm = e / TK; kk = e % TK; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      bf16 v = __float2bfloat16(0.f);
      if (gm < M && gk < ke) v = TA ? A[gk * lda + gm] : A[gm * lda + gk];
      As[mm][kk] = v;
    }
    for (int e = threadIdx.x; e < TK * TN; e += blockDim.x) {
      int kk, nn;
      if (TB) { kk = e % TK; nn = e / TK; } else { kk = e / TN; nn = e % TN; }
      const int64_t gk = k0 + kk, gn = n0 + nn;
      bf16 v = __float2bfloat16(0.f);
      if (gn < N && gk < ke) v = TB ? B[gn * ldb + gk] : B[gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; kk += 16) {
      wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> fa[2];
      wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> fb[4];
#pragma unroll
      for (int i = 0; i < 2; ++i) wmma::load_matrix_sync(fa[i], &As[wm * 32 + i * 16][kk], TK + APAD);
#pragma unroll
      for (int j = 0; j < 4; ++j) wmma::load_matrix_sync(fb[j], &Bs[kk][wn * 64 + j * 16], TN + BPAD);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) wmma::mma_sync(acc[i][j], fa[i], fb[j], acc[i][j]);
    }
    __syncthreads();
  }
  // epilogue through a per-warp 16 x 16 staging tile
  float* cs = Cs[warp];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      wmma::store_matrix_sync(cs, acc[i][j], 16, wmma::mem_row_major);
      __syncwarp();
      for (int e = lane; e < 256; e += 32) {
        const int r = e >> 4, cc = e & 15;
        const int64_t gm = m0 + wm * 32 + i * 16 + r, gn = n0 + wn * 64 + j * 16 + cc;
        if (gm < M && gn < N) {
          float v = cs[e];
          if (epi == 3) {
            atomicAdd(reinterpret_cast<float*>(C) + gm * ldc + gn, v);
          } else {
            if (bias && (epi == 1 || epi == 2)) v += bias[gn];
            if (epi == 2) reinterpret_cast<bf16*>(C)[gm * ldc + gn] = __float2bfloat16(v > 0.f ? v : 0.f);
            else if (epi == 4) reinterpret_cast<bf16*>(C)[gm * ldc + gn] = __float2bfloat16(v);
            else reinterpret_cast<float*>(C)[gm * ldc + gn] = v;
          }
        }
      }
      __syncwarp();
    }
}

// Vectorised variant for 16-byte aligned operands (leading dimensions multiples of 8):
// each operand tile is staged in its stored layout with 16-byte loads (a transposed
// operand is read by column-major fragments, so nothing is transposed through shared
// memory), and the next K tile is loaded into registers while the current one is
// multiplied.  Same tiles, epilogues and results as k_gemm_bf16.
union Pack8 {
  uint4 v;
  bf16 h[8];
};

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_bf16_v(int64_t M, int64_t N, int64_t K, const bf16* __restrict__ A,
                                                     int64_t lda, const bf16* __restrict__ B, int64_t ldb, void* C,
                                                     int64_t ldc, const float* __restrict__ bias, int epi,
                                                     int64_t k_chunk) {
  // A tile: [TM][TK + APAD] (row-major op(A)) or [TK][TM + APAD] (stored A' layout)
  // B tile: [TK][TN + BPAD] (row-major op(B)) or [TN][TK + BPAD] (stored B' layout)
  constexpr int A_ROWS = TA ? TK : TM, A_COLS = (TA ? TM : TK) + APAD;
  constexpr int B_ROWS = TB ? TN : TK, B_COLS = (TB ? TK : TN) + BPAD;
  __shared__ __align__(128) bf16 As[A_ROWS][A_COLS];
  __shared__ __align__(128) bf16 Bs[B_ROWS][B_COLS];
  __shared__ __align__(32) float Cs[8][16 * 16];
  using LA = typename std::conditional<TA, wmma::col_major, wmma::row_major>::type;
  using LB = typename std::conditional<TB, wmma::col_major, wmma::row_major>::type;
  const int64_t m0 = blockIdx.y * (int64_t)TM, n0 = blockIdx.x * (int64_t)TN;
  const int64_t kb = blockIdx.z * k_chunk, ke = min(K, kb + k_chunk);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp >> 1, wn = warp & 1;
  // each thread moves two 8-element vectors of each tile: vector e covers stored row
  // e / (cols/8), columns 8 * (e % (cols/8)) .. +7
  constexpr int AV = (TA ? TM : TK) / 8, BV = (TB ? TK : TN) / 8;
  Pack8 ra[2], rb[2];
  auto load_a = [&](int64_t k0) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int e = threadIdx.x + t * 256;
      const int r = e / AV, c = (e % AV) * 8;
      // stored element (row, col): !TA: (m, k) = A[m * lda + k]; TA: (k, m) = A[k * lda + m]
      const int64_t grow = TA ? k0 + r : m0 + r, gcol = TA ? m0 + c : k0 + c;
      const int64_t rlim = TA ? ke : M, clim = TA ? M : ke;
      const bf16* src = A + grow * lda + gcol;
      if (grow < rlim && gcol + 7 < clim) {
        ra[t].v = __ldg(reinterpret_cast<const uint4*>(src));
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) ra[t].h[u] = (grow < rlim && gcol + u < clim) ? src[u] : __float2bfloat16(0.f);
      }
    }
  };
  auto load_b = [&](int64_t k0) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int e = threadIdx.x + t * 256;
      const int r = e / BV, c = (e % BV) * 8;
      // stored element: !TB: (k, n) = B[k * ldb + n]; TB: (n, k) = B[n * ldb + k]
      const int64_t grow = TB ? n0 + r : k0 + r, gcol = TB ? k0 + c : n0 + c;
      const int64_t rlim = TB ? N : ke, clim = TB ? ke : N;
      const bf16* src = B + grow * ldb + gcol;
      if (grow < rlim && gcol + 7 < clim) {
        rb[t].v = __ldg(reinterpret_cast<const uint4*>(src));
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) rb[t].h[u] = (grow < rlim && gcol + u < clim) ? src[u] : __float2bfloat16(0.f);
      }
    }
  };
  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) wmma::fill_fragment(acc[i][j], 0.0f);
  if (kb < ke) {
    load_a(kb);
    load_b(kb);
  }
  for (int64_t k0 = kb; k0 < ke; k0 += TK) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int ea = threadIdx.x + t * 256, eb = threadIdx.x + t * 256;
      *reinterpret_cast<uint4*>(&As[ea / AV][(ea % AV) * 8]) = ra[t].v;
      *reinterpret_cast<uint4*>(&Bs[eb / BV][(eb % BV) * 8]) = rb[t].v;
    }
    __syncthreads();
    if (k0 + TK < ke) {   // next tile in flight during the multiply
      load_a(k0 + TK);
      load_b(k0 + TK);
    }
#pragma unroll
    for (int kk = 0; kk < TK; kk += 16) {
      wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, LA> fa[2];
      wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, LB> fb[4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const bf16* pa = TA ? &As[kk][wm * 32 + i * 16] : &As[wm * 32 + i * 16][kk];
        wmma::load_matrix_sync(fa[i], pa, A_COLS);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bf16* pb = TB ? &Bs[wn * 64 + j * 16][kk] : &Bs[kk][wn * 64 + j * 16];
        wmma::load_matrix_sync(fb[j], pb, B_COLS);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) wmma::mma_sync(acc[i][j], fa[i], fb[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* cs = Cs[warp];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      wmma::store_matrix_sync(cs, acc[i][j], 16, wmma::mem_row_major);
      __syncwarp();
      for (int e = lane; e < 256; e += 32) {
        const int r = e >> 4, cc = e & 15;
        const int64_t gm = m0 + wm * 32 + i * 16 + r, gn = n0 + wn * 64 + j * 16 + cc;
        if (gm < M && gn < N) {
          float v = cs[e];
          if (epi == 3) {
            atomicAdd(reinterpret_cast<float*>(C) + gm * ldc + gn, v);
          } else {
            if (bias && (epi == 1 || epi == 2)) v += bias[gn];
            if (epi == 2) reinterpret_cast<bf16*>(C)[gm * ldc + gn] = __float2bfloat16(v > 0.f ? v : 0.f);
            else if (epi == 4) reinterpret_cast<bf16*>(C)[gm * ldc + gn] = __float2bfloat16(v);
            else reinterpret_cast<float*>(C)[gm * ldc + gn] = v;
          }
        }
      }
      __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// head: score_j = H2_j . w3 + b3; x0 = softmax of the scores within the instance;
// pooled_i = mean_j H2_j; ydual_i = pooled_i Wd + bd (2 values)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ws_head_fwd(int64_t count, const int64_t* asset_off, const bf16* H2,
                                                     const float* w3, const float* b3, const float* Wd,
                                                     const float* bd, float* score, float* x0, float* pooled,
                                                     float* ydual) {
  __shared__ float ws[kHid];
  __shared__ float pool[kHid];
  __shared__ float red[8];
  __shared__ float bc[2];
  for (int t = threadIdx.x; t < kHid; t += blockDim.x) ws[t] = w3[t];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int64_t a0 = asset_off[i], a1 = asset_off[i + 1];
    for (int t = threadIdx.x; t < kHid; t += blockDim.x) pool[t] = 0.f;
    __syncthreads();
    float mx = -INFINITY;
    for (int64_t r = a0 + warp; r < a1; r += nw) {
      const bf16* h = H2 + r * kHid;
      float s = 0.f;
      for (int t = lane; t < kHid; t += 32) {
        const float hv = __bfloat162float(h[t]);
        s += hv * ws[t];
        atomicAdd(&pool[t], hv);
      }
      s = cqp::warp_sum(s) + b3[0];
      if (lane == 0) score[r] = s;
      mx = fmaxf(mx, s);
    }
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      float m = -INFINITY;
      for (int w = 0; w < nw; ++w) m = fmaxf(m, red[w]);
      bc[0] = m;
    }
    __syncthreads();
    float se = 0.f;
    for (int64_t r = a0 + threadIdx.x; r < a1; r += blockDim.x) {
      const float e = __expf(score[r] - bc[0]);
      x0[r] = e;
      se += e;
    }
    se = cqp::warp_sum(se);
    if (lane == 0) red[warp] = se;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < nw; ++w) t += red[w];
      bc[1] = t;
    }
    __syncthreads();
    const float inv = 1.f / bc[1];
    for (int64_t r = a0 + threadIdx.x; r < a1; r += blockDim.x) x0[r] *= inv;
    const float invn = a1 > a0 ? 1.f / (float)(a1 - a0) : 0.f;
    for (int t = threadIdx.x; t < kHid; t += blockDim.x) pooled[i * kHid + t] = pool[t] * invn;
    __syncthreads();
    if (warp < 2) {
      float s = 0.f;
      for (int t = lane; t < kHid; t += 32) s += pooled[i * kHid + t] * Wd[t * 2 + warp];
      s = cqp::warp_sum(s);
      if (lane == 0) ydual[i * 2 + warp] = s + bd[warp];
    }
    __syncthreads();
  }
}

// loss_i = n_i sum_j (x0_j - x*_j)^2 + lam sum_d (ydual_id - y*_id)^2; gradients with
// respect to the scores (through the softmax) and the two dual outputs
__global__ void __launch_bounds__(256) k_ws_loss(int64_t count, const int64_t* asset_off, const float* x0,
                                                 const float* xstar, const float* ydual, const float* ystar,
                                                 float lam, float scale, float* dscore, float* dydual,
                                                 double* loss) {
  __shared__ float red[8];
  __shared__ float dot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int64_t a0 = asset_off[i], a1 = asset_off[i + 1];
    const float n = (float)(a1 - a0);
    float l = 0.f, d = 0.f;
    for (int64_t r = a0 + threadIdx.x; r < a1; r += blockDim.x) {
      const float e = x0[r] - xstar[r];
      l += n * e * e;
      d += x0[r] * (2.f * n * e);
    }
    l = cqp::warp_sum(l);
    d = cqp::warp_sum(d);
    if (lane == 0) red[warp] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < nw; ++w) t += red[w];
      dot = t;
    }
    __syncthreads();
    for (int64_t r = a0 + threadIdx.x; r < a1; r += blockDim.x) {
      const float g = 2.f * n * (x0[r] - xstar[r]);
      dscore[r] = scale * x0[r] * (g - dot);
    }
    if (lane == 0) atomicAdd(loss, (double)l);
    if (threadIdx.x < 2) {
      const float e = ydual[i * 2 + threadIdx.x] - ystar[i * 2 + threadIdx.x];
      dydual[i * 2 + threadIdx.x] = scale * 2.f * lam * e;
      atomicAdd(loss, (double)(lam * e * e));
    }
    __syncthreads();
  }
}

// head backward: dZ2 = (dscore w3' + dpool) * [H2 > 0] with dpool_i = dydual_i Wd' / n_i;
// gradients of w3, b3, Wd, bd accumulated into FP32 buffers
__global__ void __launch_bounds__(256) k_ws_head_bwd(int64_t count, const int64_t* asset_off, const bf16* H2,
                                                     const float* w3, const float* Wd, const float* dscore,
                                                     const float* dydual, const float* pooled, bf16* dZ2,
                                                     float* gw3, float* gb3, float* gWd, float* gbd) {
  __shared__ float ws[kHid];
  __shared__ float dp[kHid];
  __shared__ float gacc[kHid];
  for (int t = threadIdx.x; t < kHid; t += blockDim.x) ws[t] = w3[t];
  __syncthreads();
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int64_t a0 = asset_off[i], a1 = asset_off[i + 1];
    const float invn = a1 > a0 ? 1.f / (float)(a1 - a0) : 0.f;
    const float d0 = dydual[i * 2], d1 = dydual[i * 2 + 1];
    for (int t = threadIdx.x; t < kHid; t += blockDim.x) {
      dp[t] = (d0 * Wd[t * 2] + d1 * Wd[t * 2 + 1]) * invn;
      gacc[t] = 0.f;
      const float pv = pooled[i * kHid + t];
      atomicAdd(&gWd[t * 2], pv * d0);
      atomicAdd(&gWd[t * 2 + 1], pv * d1);
    }
    if (threadIdx.x < 2) atomicAdd(&gbd[threadIdx.x], threadIdx.x == 0 ? d0 : d1);
    __syncthreads();
    float sb = 0.f;
    for (int64_t r = a0; r < a1; ++r) {
      const float ds = dscore[r];
      if (threadIdx.x == 0) sb += ds;
      for (int t = threadIdx.x; t < kHid; t += blockDim.x) {
        const float hv = __bfloat162float(H2[r * kHid + t]);
        gacc[t] += hv * ds;
        const float g = hv > 0.f ? ds * ws[t] + dp[t] : 0.f;
        dZ2[r * kHid + t] = __float2bfloat16(g);
      }
    }
    for (int t = threadIdx.x; t < kHid; t += blockDim.x) atomicAdd(&gw3[t], gacc[t]);
    if (threadIdx.x == 0) atomicAdd(gb3, sb);
    __syncthreads();
  }
}

// dZ = dH * [H > 0] (BF16, in place)
__global__ void k_relu_bwd(int64_t n, const bf16* H, bf16* dH) {
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += nt)
    if (!(__bfloat162float(H[e]) > 0.f)) dH[e] = __float2bfloat16(0.f);
}

// column sums of a BF16 matrix (rows x cols) into FP32 (atomics per block)
__global__ void __launch_bounds__(256) k_colsum(int64_t rows, int64_t cols, const bf16* Z, float* out) {
  for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) {
    float s = 0.f;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) s += __bfloat162float(Z[r * cols + c]);
    atomicAdd(&out[c], s);
  }
}

// Adam (FP32 master weights), with a BF16 copy for the GEMMs
__global__ void k_adam(int64_t n, float* w, const float* g, float* m, float* v, float lr, float b1, float b2,
                       float eps, float c1, float c2, bf16* wb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
  }
}

// (x0, y0) of the batch from the head outputs: x = softmax weights, w_F = F'x,
// w_D = D^(1/2) x, t = sigma_bar; y = (y_b, lambda w_F, lambda w_D, y_t) with
// lambda = y_t / sigma_bar.  Coordinates and rows in the portfolio batch layout.
__global__ void __launch_bounds__(256) k_ws_start(int64_t count, const int64_t* x_off, const int64_t* row_off,
                                                  const int64_t* n_assets, const int64_t* asset_off,
                                                  const int32_t* rank, const double* q, const double* R, int64_t ldr,
                                                  const double* b, const float* xw, const float* ydual,
                                                  float yb_scale, int dual_mode, double* x0, double* y0) {
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int64_t xo = x_off[i], ro = row_off[i], na = n_assets[i], a0 = asset_off[i];
    const int k = rank[i];
    const double sig = b[row_off[i + 1] - 1];
    const double yb = dual_mode >= 1 ? (double)ydual[i * 2] / yb_scale : 0.0;
    const double yt = dual_mode >= 1 ? (double)ydual[i * 2 + 1] : 0.0;
    const double lam = (dual_mode >= 2 && sig > 0.0) ? yt / sig : 0.0;
    for (int64_t j = threadIdx.x; j < na; j += blockDim.x) {
      const double xv = (double)xw[a0 + j];
      x0[xo + j] = xv;
      const double wd = sqrt(q[xo + j]) * xv;
      x0[xo + na + k + j] = wd;
      y0[ro + 1 + k + j] = lam * wd;
    }
    for (int l = threadIdx.x >> 5; l < k; l += blockDim.x >> 5) {
      double s = 0.0;
      for (int64_t j = threadIdx.x & 31; j < na; j += 32) s += R[(int64_t)l * ldr + xo + j] * (double)xw[a0 + j];
      s = cqp::warp_sum(s);
      if ((threadIdx.x & 31) == 0) {
        x0[xo + na + l] = s;
        y0[ro + 1 + l] = lam * s;
      }
    }
    if (threadIdx.x == 0) {
      x0[xo + 2 * na + k] = sig;
      y0[ro] = yb;
      y0[row_off[i + 1] - 1] = yt;
    }
    __syncthreads();
  }
}

int grid_rows(int64_t work, int threads = 256, int cap = 152 * 16) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

extern "C" {

int cqp_ws_features(int64_t count, const int64_t* x_off, const int64_t* n_assets, const int64_t* asset_off,
                    const int64_t* row_off, const int32_t* rank, const double* c, const double* q, const double* R,
                    int64_t ldr, const double* b, uint16_t* X, void* stream) {
  if (count < 1 || !x_off || !n_assets || !asset_off || !row_off || !rank || !c || !q || !b || !X || (ldr > 0 && !R))
    return fail_with(CQP_ERR_INVALID, "cqp_ws_features: bad arguments");
  k_ws_features<<<(int)std::min<int64_t>(count, 152 * 8), 256, 0, (cudaStream_t)stream>>>(
      count, x_off, n_assets, asset_off, row_off, rank, c, q, R, ldr, b, reinterpret_cast<bf16*>(X));
  cqp::record_launches(1);
  MLP_CK(cudaGetLastError());
  return CQP_OK;
}

int cqp_gemm_bf16(int32_t trans_a, int32_t trans_b, int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda,
                  const uint16_t* B, int64_t ldb, void* C, int64_t ldc, const float* bias, int32_t epilogue,
                  int32_t split_k, void* stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C || epilogue < 0 || epilogue > 4)
    return fail_with(CQP_ERR_INVALID, "cqp_gemm_bf16: bad arguments");
  if (M == 0 || N == 0) return CQP_OK;
  {
    int rc = CQP_OK;
    if (cqp::gemm_tc_try(trans_a, trans_b, M, N, K, A, lda, B, ldb, C, ldc, bias, epilogue, (cudaStream_t)stream, &rc))
      return rc;
  }
  const int splits = epilogue == 3 ? std::max(1, split_k) : 1;
  int64_t kc = (K + splits - 1) / splits;
  kc = (kc + TK - 1) / TK * TK;
  dim3 grid((unsigned)((N + TN - 1) / TN), (unsigned)((M + TM - 1) / TM), (unsigned)std::max<int64_t>(1, (K + kc - 1) / std::max<int64_t>(kc, 1)));
  if (grid.y > 65535 || grid.z > 65535) return fail_with(CQP_ERR_INVALID, "cqp_gemm_bf16: too many tiles");
  cudaStream_t st = (cudaStream_t)stream;
  const bf16* a = reinterpret_cast<const bf16*>(A);
  const bf16* bb = reinterpret_cast<const bf16*>(B);
  const bool vec = lda % 8 == 0 && ldb % 8 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(B) & 15) == 0;
  if (vec) {
    if (!trans_a && !trans_b) k_gemm_bf16_v<false, false><<<grid, 256, 0, st>>>(M, N, K, a, lda, bb, ldb, C, ldc, bias, epilogue, kc);
    else if (!trans_a && trans_b) k_gemm_bf16_v<false, true><<<grid, 256, 0, st>>>(M, N, K, a, lda, bb, ldb, C, ldc, bias, epilogue, kc);
    else if (trans_a && !trans_b) k_gemm_bf16_v<true, false><<<grid, 256, 0, st>>>(M, N, K, a, lda, bb, ldb, C, ldc, bias, epilogue, kc);
    else k_gemm_bf16_v<true, true><<<grid, 256, 0, st>>>(M, N, K, a, lda, bb, ldb, C, ldc, bias, epilogue, kc);
  } else {
    if (!trans_a && !trans_b) k_gemm_bf16<false, false><<<grid, 256, 0, st>>>(M, N, K, a, lda, bb, ldb, C, ldc, bias, epilogue, kc);
    else if (!trans_a && trans_b) k_gemm_bf16<false, true><<<grid, 256, 0, st>>>(M, N, K, a, lda, bb, ldb, C, ldc, bias, epilogue, kc);
    else if (trans_a && !trans_b) k_gemm_bf16<true, false><<<grid, 256, 0, st>>>(M, N, K, a, lda, bb, ldb, C, ldc, bias, epilogue, kc);
    else k_gemm_bf16<true, true><<<grid, 256, 0, st>>>(M, N, K, a, lda, bb, ldb, C, ldc, bias, epilogue, kc);
  }
  cqp::record_launches(1);
  MLP_CK(cudaGetLastError());
  return CQP_OK;
}

int cqp_ws_head_forward(int64_t count, const int64_t* asset_off, const uint16_t* H2, const float* w3, const float* b3,
                        const float* Wd, const float* bd, float* score, float* x0, float* pooled, float* ydual,
                        void* stream) {
  if (count < 1 || !asset_off || !H2 || !w3 || !b3 || !Wd || !bd || !score || !x0 || !pooled || !ydual)
    return fail_with(CQP_ERR_INVALID, "cqp_ws_head_forward: bad arguments");
  k_ws_head_fwd<<<(int)std::min<int64_t>(count, 152 * 8), 256, 0, (cudaStream_t)stream>>>(
      count, asset_off, reinterpret_cast<const bf16*>(H2), w3, b3, Wd, bd, score, x0, pooled, ydual);
  cqp::record_launches(1);
  MLP_CK(cudaGetLastError());
  return CQP_OK;
}

int cqp_ws_loss(int64_t count, const int64_t* asset_off, const float* x0, const float* xstar, const float* ydual,
                const float* ystar, float lam, float scale, float* dscore, float* dydual, double* loss, void* stream) {
  if (count < 1 || !asset_off || !x0 || !xstar || !ydual || !ystar || !dscore || !dydual || !loss)
    return fail_with(CQP_ERR_INVALID, "cqp_ws_loss: bad arguments");
  k_ws_loss<<<(int)std::min<int64_t>(count, 152 * 8), 256, 0, (cudaStream_t)stream>>>(
      count, asset_off, x0, xstar, ydual, ystar, lam, scale, dscore, dydual, loss);
  cqp::record_launches(1);
  MLP_CK(cudaGetLastError());
  return CQP_OK;
}

int cqp_ws_head_backward(int64_t count, const int64_t* asset_off, const uint16_t* H2, const float* w3, const float* Wd,
                         const float* dscore, const float* dydual, const float* pooled, uint16_t* dZ2, float* gw3,
                         float* gb3, float* gWd, float* gbd, void* stream) {
  if (count < 1 || !asset_off || !H2 || !w3 || !Wd || !dscore || !dydual || !pooled || !dZ2 || !gw3 || !gb3 ||
      !gWd || !gbd)
    return fail_with(CQP_ERR_INVALID, "cqp_ws_head_backward: bad arguments");
  k_ws_head_bwd<<<(int)std::min<int64_t>(count, 152 * 8), 256, 0, (cudaStream_t)stream>>>(
      count, asset_off, reinterpret_cast<const bf16*>(H2), w3, Wd, dscore, dydual, pooled,
      reinterpret_cast<bf16*>(dZ2), gw3, gb3, gWd, gbd);
  cqp::record_launches(1);
  MLP_CK(cudaGetLastError());
  return CQP_OK;
}

int cqp_relu_backward_bf16(int64_t rows, int64_t cols, const uint16_t* H, uint16_t* dH, float* gbias, void* stream) {
  if (rows < 0 || cols < 0 || !H || !dH) return fail_with(CQP_ERR_INVALID, "cqp_relu_backward_bf16: bad arguments");
  if (rows == 0 || cols == 0) return CQP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  k_relu_bwd<<<grid_rows(rows * cols), 256, 0, st>>>(rows * cols, reinterpret_cast<const bf16*>(H),
                                                    reinterpret_cast<bf16*>(dH));
  int launches = 1;
  if (gbias) {
    k_colsum<<<(int)std::min<int64_t>(rows, 152 * 8), 256, 0, st>>>(rows, cols, reinterpret_cast<const bf16*>(dH), gbias);
    ++launches;
  }
  cqp::record_launches(launches);
  MLP_CK(cudaGetLastError());
  return CQP_OK;
}

int cqp_adam_step(int64_t n, float* w, const float* g, float* m, float* v, float lr, float beta1, float beta2, float eps,
                  int64_t step, uint16_t* w_bf16, void* stream) {
  if (n < 0 || !w || !g || !m || !v || step < 1) return fail_with(CQP_ERR_INVALID, "cqp_adam_step: bad arguments");
  if (n == 0) return CQP_OK;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<grid_rows(n), 256, 0, (cudaStream_t)stream>>>(n, w, g, m, v, lr, beta1, beta2, eps, c1, c2,
                                                         reinterpret_cast<bf16*>(w_bf16));
  cqp::record_launches(1);
  MLP_CK(cudaGetLastError());
  return CQP_OK;
}

int cqp_ws_start(int64_t count, const int64_t* x_off, const int64_t* row_off, const int64_t* n_assets,
                 const int64_t* asset_off, const int32_t* rank, const double* q, const double* R, int64_t ldr,
                 const double* b, const float* xw, const float* ydual, float yb_scale, int32_t dual_mode, double* x0,
                 double* y0, void* stream) {
  if (count < 1 || !x_off || !row_off || !n_assets || !asset_off || !rank || !q || !b || !xw || !ydual || !x0 || !y0 ||
      (ldr > 0 && !R) || !(yb_scale > 0.f) || dual_mode < 0 || dual_mode > 2)
    return fail_with(CQP_ERR_INVALID, "cqp_ws_start: bad arguments");
  k_ws_start<<<(int)std::min<int64_t>(count, 152 * 8), 256, 0, (cudaStream_t)stream>>>(
      count, x_off, row_off, n_assets, asset_off, rank, q, R, ldr, b, xw, ydual, yb_scale, dual_mode, x0, y0);
  cqp::record_launches(1);
  MLP_CK(cudaGetLastError());
  return CQP_OK;
}

}  // extern "C"

int cqp_gemm_check(void* stream) { return cqp::gemm_tc_status((cudaStream_t)stream); }

namespace {
// 32 x 32 tiles through shared memory (padded against bank conflicts)
__global__ void __launch_bounds__(256) k_transpose_bf16(int64_t rows, int64_t cols, const bf16* in, bf16* out) {
  __shared__ bf16 t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = in[r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[c * rows + r] = t[threadIdx.x][i];
  }
}
}  // namespace

int cqp_transpose_bf16(int64_t rows, int64_t cols, const uint16_t* in, uint16_t* out, void* stream) {
  if (rows < 0 || cols < 0 || (rows > 0 && cols > 0 && (!in || !out)))
    return fail_with(CQP_ERR_INVALID, "cqp_transpose_bf16: bad arguments");
  if (rows == 0 || cols == 0) return CQP_OK;
  if ((cols + 31) / 32 > 2147483647 || (rows + 31) / 32 > 65535)
    return fail_with(CQP_ERR_INVALID, "cqp_transpose_bf16: too many tiles");
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32)), block(32, 8);
  k_transpose_bf16<<<grid, block, 0, (cudaStream_t)stream>>>(rows, cols, reinterpret_cast<const bf16*>(in),
                                                             reinterpret_cast<bf16*>(out));
  cqp::record_launches(1);
  MLP_CK(cudaGetLastError());
  return CQP_OK;
}
