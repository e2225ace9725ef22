// cqp_kkt_static: the FP64 KKT report of cqp_kkt, computed from caller-held
// device arrays with no device allocation at all.
//
// Why it exists: cqp_kkt needs a handle, and building a handle allocates the
// rescaled problem and the solver's work buffers with cudaMalloc.  Some
// callers cannot allocate at the moment they want a residual check: code that
// runs under a framework which owns the whole device memory pool (its caching
// allocator has already reserved HBM, and a raw cudaMalloc there either fails
// or fragments the pool behind the framework's back), code that must keep a
// fixed memory footprint for its whole lifetime, and code on latency-critical
// paths where an allocation's implicit device synchronisation is not
// acceptable.  This entry point gives them the same report while using only
// the file-scope scratch array below.
//
// The scratch: g_kkt_scratch holds the dual-slack vector (CQP_KKT_STATIC_MAX_N
// doubles), the rank-k product R x (64 doubles), per-block partial sums and the
// result.  Every GPU that loads this library keeps the array (about 4.1 MiB)
// until the process exits.  All calls on one device share it and it keeps the
// previous call's contents, so each call first clears the parts that are
// accumulated into (the dual slack, R x and the error flag); the partial sums
// and the result are fully overwritten.  Calls that overlap on the GPU (from
// two streams, or two host threads) race on the array and give wrong results:
// serialise them.
//
// In host code the name g_kkt_scratch is only a host-side shadow of the device
// array, not a device address: a kernel handed it would fault, or on a system
// where the GPU can read host memory it would quietly use the wrong memory.
// The device address is therefore looked up once per device, with that device
// current, by cudaGetSymbolAddress, and the result is cached.  That lookup
// happens inside the first call on each device, so the first call on a device
// should be made before any stream capture begins.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "cqp.h"
#include "common.cuh"
#include "cones.cuh"

namespace cqp {
void record_error(const std::string& msg);
void record_launches(long long k);
}  // namespace cqp

namespace {

constexpr int kThreads = 256;
constexpr int kMaxGrid = 1024;
constexpr int kRows = 3;   // ||Ax-b||^2, ||b||^2, b'y
constexpr int kCols = 4;   // x'Qx, c'x, ||c||^2, ||Pi_K(-s)||^2 over free/nonneg coordinates
constexpr int kCones = 2;  // ||Pi_K(-s)||^2 over SOC/RSOC/EXP/POW blocks (and slice residuals), slice support terms
constexpr int64_t kMaxN = CQP_KKT_STATIC_MAX_N;
constexpr int kMaxRank = 64;
constexpr int64_t kOffRx = kMaxN;
constexpr int64_t kOffPart = kOffRx + kMaxRank;
constexpr int64_t kOffOut = kOffPart + (int64_t)(kRows + kCols + kCones) * kMaxGrid;
constexpr int64_t kScratchDoubles = kOffOut + 16;  // out[0..8) report, out[8] error flag

static __device__ __align__(256) double g_kkt_scratch[kScratchDoubles];

__global__ void ks_clear(int64_t n, int k, double* __restrict__ s, double* __restrict__ rx, double* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = t; i < n; i += nt) s[i] = 0.0;
  if (t < k) rx[t] = 0.0;
  if (t == 0) out[8] = 0.0;
}

// One warp per row of A: (Ax - b)_i, and A' y scattered into s by atomics.  A row whose
// pointers are out of order or outside [0, nnz] (or rowptr[0] != 0) is flagged and skipped,
// so nothing past the caller's nnz entries is read.
__global__ void __launch_bounds__(kThreads) ks_rows(int64_t m, int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                                                    const int32_t* __restrict__ ci, const double* __restrict__ av,
                                                    const double* __restrict__ x, const double* __restrict__ y,
                                                    const double* __restrict__ b, double* __restrict__ s,
                                                    double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[kRows * (kThreads / 32)];
  __shared__ double tot[kRows];
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double v[kRows] = {0.0, 0.0, 0.0};
  for (int64_t i = w0; i < m; i += nw) {
    const int64_t e0 = rp[i], e1 = rp[i + 1];
    if (e0 < 0 || e1 < e0 || e1 > nnz || (i == 0 && e0 != 0)) {
      if (lane == 0) out[8] = 1.0;
      continue;
    }
    const double yi = y[i];
    double acc = 0.0;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      const int32_t j = ci[e];
      if (j < 0 || j >= n) {
        out[8] = 1.0;
        continue;
      }
      const double a = av[e];
      acc += a * x[j];
      atomicAdd(s + j, a * yi);
    }
    acc = cqp::warp_sum(acc);
    if (lane == 0) {
      const double bi = b[i], r = acc - bi;
      v[0] += r * r;
      v[1] += bi * bi;
      v[2] += bi * yi;
    }
  }
  cqp::block_sum<kRows>(v, red, tot);
  if (threadIdx.x < kRows) part[threadIdx.x * kMaxGrid + blockIdx.x] = tot[threadIdx.x];
}

// rx[l] = sum_j R[l, j] x_j; blockIdx.y = l.
__global__ void __launch_bounds__(kThreads) ks_rx(int64_t n, const double* __restrict__ R,
                                                  const double* __restrict__ x, double* __restrict__ rx) {
  __shared__ double red[kThreads / 32];
  __shared__ double tot[1];
  const int l = blockIdx.y;
  const double* Rl = R + (int64_t)l * n;
  double v[1] = {0.0};
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    v[0] += Rl[j] * x[j];
  cqp::block_sum<1>(v, red, tot);
  if (threadIdx.x == 0) atomicAdd(rx + l, tot[0]);
}

// Index of the cone block holding coordinate j: the last b with start[b] <= j
// (clamped into [0, nblocks) so a malformed partition still reads in bounds;
// ks_cones reports it).
__device__ __forceinline__ int64_t block_of(int64_t j, int64_t nblocks, const int64_t* __restrict__ start) {
  int64_t lo = 0, hi = nblocks - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (start[mid] <= j) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Per coordinate: (Qx)_j, s_j = (Qx)_j + c_j - (A'y)_j, objective sums, and the
// dual residual of free / nonnegative coordinates.  Leaves -s in s.  Rows of P are checked
// like those of A (pointers within [0, pnnz], rowptr[0] = 0).
__global__ void __launch_bounds__(kThreads) ks_cols(int64_t n, int64_t pnnz, const double* __restrict__ qd,
                                                    const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                                                    const double* __restrict__ pv, int k, const double* __restrict__ R,
                                                    const double* __restrict__ D, const double* __restrict__ rx,
                                                    const double* __restrict__ c, const double* __restrict__ x,
                                                    int64_t nblocks, const int32_t* __restrict__ type,
                                                    const int64_t* __restrict__ start, double* __restrict__ s,
                                                    double* __restrict__ part, double* __restrict__ out) {
  __shared__ double w[kMaxRank];
  __shared__ double red[kCols * (kThreads / 32)];
  __shared__ double tot[kCols];
  for (int l = threadIdx.x; l < k; l += blockDim.x) {
    double t = 0.0;
    for (int i = 0; i < k; ++i) t += D[(int64_t)l * k + i] * rx[i];
    w[l] = t;
  }
  __syncthreads();
  double v[kCols] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double xj = x[j], cj = c[j];
    double qx = qd ? qd[j] * xj : 0.0;
    if (prp) {
      const int64_t e0 = prp[j], e1 = prp[j + 1];
      if (e0 < 0 || e1 < e0 || e1 > pnnz || (j == 0 && e0 != 0)) out[8] = 1.0;
      else
        for (int64_t e = e0; e < e1; ++e) {
          const int32_t i = pci[e];
          if (i < 0 || i >= n) { out[8] = 1.0; continue; }
          qx += pv[e] * x[i];
        }
    }
    for (int l = 0; l < k; ++l) qx += R[(int64_t)l * n + j] * w[l];
    const double sj = qx + cj - s[j];
    v[0] += xj * qx;
    v[1] += cj * xj;
    v[2] += cj * cj;
    const int32_t t = type[block_of(j, nblocks, start)];
    if (t == CQP_CONE_FREE) v[3] += sj * sj;
    else if (t == CQP_CONE_NONNEG) { const double u = sj < 0.0 ? -sj : 0.0; v[3] += u * u; }
    s[j] = -sj;
  }
  cqp::block_sum<kCols>(v, red, tot);
  if (threadIdx.x < kCols) part[threadIdx.x * kMaxGrid + blockIdx.x] = tot[threadIdx.x];
}

// One warp per cone block: check the block, project -s onto SOC / RSOC / EXP /
// POW blocks in place (Euclidean projections of the cone library) and sum the
// squared projection.  Slice blocks (EXP1 / POW1) add their support term to the dual
// objective and the part of the slack outside its domain to the dual residual.
__global__ void __launch_bounds__(kThreads) ks_cones(int64_t n, int64_t nblocks, const int32_t* __restrict__ type,
                                                     const int64_t* __restrict__ start, const int64_t* __restrict__ dim,
                                                     const double* __restrict__ alpha, double* __restrict__ s,
                                                     double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[kCones * (kThreads / 32)];
  __shared__ double tot[kCones];
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double v[kCones] = {0.0, 0.0};
  for (int64_t bk = w0; bk < nblocks; bk += nw) {
    const int32_t t = type[bk];
    const int64_t st = start[bk], d = dim[bk];
    const int64_t expect = bk == 0 ? 0 : start[bk - 1] + dim[bk - 1];
    const bool slice = t == CQP_CONE_EXP1 || t == CQP_CONE_POW1;
    bool ok = st == expect && d >= 1 && st + d <= n && ((t >= CQP_CONE_FREE && t <= CQP_CONE_POW) || slice);
    if (bk == nblocks - 1) ok = ok && st + d == n;
    if (t == CQP_CONE_SOC) ok = ok && d >= 2;
    if (t == CQP_CONE_RSOC) ok = ok && d >= 3;
    if (t == CQP_CONE_EXP || t == CQP_CONE_POW || slice) ok = ok && d == 3;
    if (t == CQP_CONE_POW || t == CQP_CONE_POW1) ok = ok && alpha != nullptr && alpha[bk] > 0.0 && alpha[bk] < 1.0;
    if (!ok) {
      if (lane == 0) out[8] = 1.0;
      continue;
    }
    if (t == CQP_CONE_FREE || t == CQP_CONE_NONNEG) continue;  // done coordinate-wise in ks_cols
    double* z = s + st;
    if (slice) {
      if (lane == 0) {
        const double sl[3] = {-z[0], -z[1], -z[2]};
        double o[3];
        v[1] += cqp::slice_support(t == CQP_CONE_POW1, t == CQP_CONE_POW1 ? alpha[bk] : 0.0, sl, o);
        z[0] = o[0]; z[1] = o[1]; z[2] = o[2];
      }
    } else if (t == CQP_CONE_SOC) {
      cqp::warp_soc_euclid<double>(z, (int)d, lane);
    } else if (t == CQP_CONE_RSOC) {
      cqp::warp_rsoc_euclid<double>(z, (int)d, lane);
    } else if (lane == 0) {
      double o[3];
      if (t == CQP_CONE_EXP) cqp::exp_proj_euclid(z[0], z[1], z[2], o);
      else cqp::pow_proj(z[0], z[1], z[2], alpha[bk], 1.0, 1.0, 1.0, o);
      z[0] = o[0]; z[1] = o[1]; z[2] = o[2];
    }
    __syncwarp();
    for (int64_t i = lane; i < d; i += 32) v[0] += z[i] * z[i];
    __syncwarp();
  }
  cqp::block_sum<kCones>(v, red, tot);
  if (threadIdx.x < kCones) part[threadIdx.x * kMaxGrid + blockIdx.x] = tot[threadIdx.x];
}

// Fixed-order sums of the partials and the report (same definitions as cqp_kkt).
__global__ void ks_final(int g_rows, int g_cols, int g_cones, const double* __restrict__ part,
                         double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double r[kRows] = {0.0, 0.0, 0.0}, q[kCols] = {0.0, 0.0, 0.0, 0.0}, dc = 0.0;
  for (int i = 0; i < kRows; ++i)
    for (int g = 0; g < g_rows; ++g) r[i] += part[i * kMaxGrid + g];
  const double* pc = part + kRows * kMaxGrid;
  for (int i = 0; i < kCols; ++i)
    for (int g = 0; g < g_cols; ++g) q[i] += pc[i * kMaxGrid + g];
  const double* pk = pc + kCols * kMaxGrid;
  double sup = 0.0;
  for (int g = 0; g < g_cones; ++g) dc += pk[g];
  for (int g = 0; g < g_cones; ++g) sup += pk[kMaxGrid + g];
  const double xqx = q[0], cx = q[1];
  const double pobj = 0.5 * xqx + cx, dobj = r[2] - 0.5 * xqx + sup;
  const double nrp = sqrt(r[0]), nrd = sqrt(q[3] + dc);
  out[0] = nrp / (1.0 + sqrt(r[1]));
  out[1] = nrd / (1.0 + sqrt(q[2]));
  // an infinite slice support term (dual objective -inf) is the limit eps_g -> 1
  out[2] = isfinite(dobj) ? fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj)) : 1.0;
  out[3] = fmax(out[0], fmax(out[1], out[2]));
  out[4] = pobj;
  out[5] = dobj;
  out[6] = nrp;
  out[7] = nrd;
}

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};
int g_scratch_sms[kMaxDevices] = {};

int grid_for(int64_t work, int sms) {
  const int64_t want = (work + kThreads - 1) / kThreads;
  const int64_t cap = std::min<int64_t>(kMaxGrid, 4LL * sms);
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

int fail_with(int code, const std::string& msg) {
  cqp::record_error(msg);
  return code;
}

#define KS_CK(x)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (x);                                                                        \
    if (e_ != cudaSuccess) return fail_with(CQP_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" int cqp_kkt_static(const cqp_csr* A, const cqp_qop* Q, const double* c, const double* b,
                              const cqp_cones* K, const double* x, const double* y, cqp_kkt_report* rep,
                              void* stream) {
  if (!A || !K || !c || !x || !rep) return fail_with(CQP_ERR_INVALID, "cqp_kkt_static: NULL argument");
  const int64_t m = A->nrows, n = A->ncols;
  if (n < 1 || m < 0) return fail_with(CQP_ERR_INVALID, "cqp_kkt_static: need n >= 1 and m >= 0");
  if (n > kMaxN)
    return fail_with(CQP_ERR_INVALID, "cqp_kkt_static: n = " + std::to_string(n) + " exceeds the static scratch limit " +
                                          std::to_string(kMaxN) + "; use cqp_kkt on a handle instead");
  if (m > 0 && (!A->rowptr || !A->colind || !A->val || !b || !y))
    return fail_with(CQP_ERR_INVALID, "cqp_kkt_static: A, b or y missing");
  if (A->nnz < 0 || A->nnz >= (1LL << 31)) return fail_with(CQP_ERR_INVALID, "cqp_kkt_static: nnz out of range");
  if (K->nblocks < 1 || K->nblocks > n || !K->type || !K->start || !K->dim)
    return fail_with(CQP_ERR_INVALID, "cqp_kkt_static: bad cone partition");
  const double* qd = Q ? Q->diag : nullptr;
  const bool has_p = Q && Q->P.rowptr;
  const int k = Q ? (int)Q->rank : 0;
  if (Q && (Q->rank < 0 || Q->rank > kMaxRank))
    return fail_with(CQP_ERR_INVALID, "cqp_kkt_static: rank must be in [0, 64]");
  if (k > 0 && (!Q->R || !Q->D)) return fail_with(CQP_ERR_INVALID, "cqp_kkt_static: R or D missing");
  if (has_p && (!Q->P.colind || !Q->P.val || Q->P.nrows != n || Q->P.ncols != n || Q->P.nnz < 0 ||
                Q->P.nnz >= (1LL << 31)))
    return fail_with(CQP_ERR_INVALID, "cqp_kkt_static: P must be n x n with 0 <= nnz < 2^31");

  int dev = 0;
  KS_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail_with(CQP_ERR_UNSUPPORTED, "cqp_kkt_static: device ordinal >= 64");
  double* base = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      KS_CK(cudaGetSymbolAddress(&p, g_kkt_scratch));
      int cnt = 0;
      KS_CK(cudaDeviceGetAttribute(&cnt, cudaDevAttrMultiProcessorCount, dev));
      g_scratch_sms[dev] = cnt;
      g_scratch_addr[dev] = (double*)p;
    }
    base = g_scratch_addr[dev];
    sms = g_scratch_sms[dev];
  }
  double* s = base;
  double* rx = base + kOffRx;
  double* part = base + kOffPart;
  double* out = base + kOffOut;
  cudaStream_t st = (cudaStream_t)stream;
  {
    // the report is read back to the host and the stream synchronised, which a stream
    // capture does not allow
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    KS_CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail_with(CQP_ERR_UNSUPPORTED, "cqp_kkt_static: called on a stream that is being captured");
  }

  long long launches = 0;
  const int g_clear = grid_for(n, sms);
  ks_clear<<<g_clear, kThreads, 0, st>>>(n, k, s, rx, out);
  ++launches;
  const int g_rows = m > 0 ? grid_for(m * 32, sms) : 0;
  if (g_rows > 0) {
    ks_rows<<<g_rows, kThreads, 0, st>>>(m, n, A->nnz, A->rowptr, A->colind, A->val, x, y, b, s, part, out);
    ++launches;
  }
  if (k > 0) {
    ks_rx<<<dim3(grid_for(n, sms) / 8 + 1, k), kThreads, 0, st>>>(n, Q->R, x, rx);
    ++launches;
  }
  const int g_cols = grid_for(n, sms);
  ks_cols<<<g_cols, kThreads, 0, st>>>(n, has_p ? Q->P.nnz : 0, qd, has_p ? Q->P.rowptr : nullptr, has_p ? Q->P.colind : nullptr,
                                       has_p ? Q->P.val : nullptr, k, k > 0 ? Q->R : nullptr, k > 0 ? Q->D : nullptr,
                                       rx, c, x, K->nblocks, K->type, K->start, s, part + kRows * kMaxGrid, out);
  const int g_cones = grid_for(K->nblocks * 32, sms);
  ks_cones<<<g_cones, kThreads, 0, st>>>(n, K->nblocks, K->type, K->start, K->dim, K->alpha, s,
                                         part + (kRows + kCols) * kMaxGrid, out);
  ks_final<<<1, 32, 0, st>>>(g_rows, g_cols, g_cones, part, out);
  launches += 3;
  cqp::record_launches(launches);
  KS_CK(cudaGetLastError());
  double h[9];
  KS_CK(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, st));
  KS_CK(cudaStreamSynchronize(st));
  if (h[8] != 0.0)
    return fail_with(CQP_ERR_INVALID, "cqp_kkt_static: malformed A, P or cone partition (index, pointer or block check failed on the device)");
  rep->eps_p = h[0]; rep->eps_d = h[1]; rep->eps_g = h[2]; rep->rel_kkt = h[3];
  rep->pobj = h[4]; rep->dobj = h[5]; rep->norm_res_p = h[6]; rep->norm_res_d = h[7];
  if (!std::isfinite(h[3])) return fail_with(CQP_ERR_NUMERICAL, "cqp_kkt_static: non-finite report");
  return CQP_OK;
}
