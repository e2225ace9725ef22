// C ABI of the library (declarations and contracts in include/cqp.h).
//
// Host orchestration only: validation, layout permutation, transpose,
// rescaling (Sec. 4.2.2), norm estimate (eq. practical-stepsizes), the launch
// loop of the persistent solver kernel, unscaling.  Every step on the data
// runs in the kernels of setup.cuh / solver_impl.cuh.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <stdexcept>
#include <string>
#include <vector>

#include "cqp.h"
#include "launch.h"
#include "setup.cuh"
#include "solver_impl.cuh"
#include "batch_setup.cuh"

namespace {

thread_local std::string g_last_error;
// kernels launched by this library in the calling thread (setup, solve, KKT, entry points)
thread_local long long g_launches = 0;
inline void count_launch() { ++g_launches; }

struct Fail {
  int code;
};

void fail(int code, const std::string& msg) {
  g_last_error = msg;
  throw Fail{code};
}

#define CK(x)                                                                                                 \
  do {                                                                                                        \
    cudaError_t e_ = (x);                                                                                     \
    if (e_ != cudaSuccess) {                                                                                  \
      fail(e_ == cudaErrorMemoryAllocation ? CQP_ERR_OOM : CQP_ERR_CUDA,                                      \
           std::string(#x) + ": " + cudaGetErrorString(e_));                                                 \
    }                                                                                                         \
  } while (0)

// The library's device memory comes from its own stream-ordered pool, one per device,
// which keeps freed blocks for reuse (release threshold at its maximum): repeated set-ups
// and solves then allocate without driver calls or device-wide synchronisation.  Memory
// freed by the library stays reserved for it until the process exits.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

cudaMemPool_t lib_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) fail(CQP_ERR_CUDA, "no current device");
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) fail(CQP_ERR_CUDA, "cudaMemPoolCreate failed");
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pool[dev] = p;
  }
  return g_pool[dev];
}

// device allocations owned by a handle (stream-ordered on the handle's stream, which
// must outlive the handle)
struct Arena {
  std::vector<void*> ptrs;
  cudaStream_t st = nullptr;
  template <typename U>
  U* alloc(int64_t n) {
    void* p = nullptr;
    const size_t bytes = (size_t)std::max<int64_t>(n, 1) * sizeof(U);
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, lib_pool(), st);
    if (e != cudaSuccess) fail(e == cudaErrorMemoryAllocation ? CQP_ERR_OOM : CQP_ERR_CUDA, "device allocation failed");
    ptrs.push_back(p);
    return (U*)p;
  }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    ptrs.clear();
  }
  ~Arena() { release(); }
};

// scoped temporary allocations (set-up, solve and KKT helpers)
struct Temp {
  Arena a;
  explicit Temp(cudaStream_t s) { a.st = s; }
  template <typename U>
  U* alloc(int64_t n) { return a.alloc<U>(n); }
};

double dev_dot(const double* a, const double* b, int64_t n, double* part, double* out, cudaStream_t st) {
  const int nb = cqp::grid_for(n, cqp::kSetupThreads, 1024);
  count_launch(); cqp::k_dot_partial<<<nb, cqp::kSetupThreads, 0, st>>>(n, a, b, part);
  count_launch(); cqp::k_sum_partials<<<1, 32, 0, st>>>(nb, part, out);
  double h = 0.0;
  CK(cudaMemcpyAsync(&h, out, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return h;
}

// exclusive scan of n int32 counts into n+1 int32 offsets
void dev_scan(const int32_t* in, int32_t* out, int64_t n, Temp& tmp, cudaStream_t st) {
  const int64_t per = 1 << 16;
  const int nb = (int)std::max<int64_t>(1, (n + per - 1) / per);
  int64_t* tot = tmp.alloc<int64_t>(nb + 1);
  count_launch(); cqp::k_scan_block_totals<<<nb, cqp::kSetupThreads, 0, st>>>(n, in, per, tot);
  count_launch(); cqp::k_scan_totals<<<1, 32, 0, st>>>(nb, tot);
  count_launch(); cqp::k_scan_apply<<<nb, cqp::kSetupThreads, 0, st>>>(n, in, per, tot, out);
  CK(cudaGetLastError());
}

struct HandleBase {
  virtual ~HandleBase() {}
  virtual int solve(const double* x0, const double* y0, double* xo, double* yo, int on_dev, cqp_result* res) = 0;
  virtual int kkt(const double* x, const double* y, int on_dev, cqp_kkt_report* rep) = 0;
  virtual int solve_batch(const double* x0, const double* y0, double* xo, double* yo, int on_dev,
                          cqp_instance_result* per, cqp_result* res) = 0;
};

// unscale + un-permute: out[perm[i]] = scale * v[i] / f[i]
template <typename T>
__global__ void k_unscale_unperm(int64_t n, const int64_t* perm, const T* v, const double* f, double scale, double* out) {
  CQP_GRID_LOOP(i, n) out[perm ? perm[i] : i] = scale * (double)v[i] / f[i];
}
// permute + scale: v[i] = in[perm[i]] * f[i] / scale
template <typename T>
__global__ void k_perm_scale(int64_t n, const int64_t* perm, const double* in, const double* f, double scale, T* v) {
  CQP_GRID_LOOP(i, n) v[i] = in ? T(in[perm ? perm[i] : i] * f[i] / scale) : T(0);
}
template <typename T>
__global__ void k_copy_vec(int64_t n, const T* a, T* b) {
  CQP_GRID_LOOP(i, n) b[i] = a[i];
}
template <typename T>
__global__ void k_zero(int64_t n, T* a) {
  CQP_GRID_LOOP(i, n) a[i] = T(0);
}
// new coordinate -> old coordinate through the segment table (new_start sorted)
__global__ void k_build_perm(int64_t n, int64_t nseg, const int64_t* seg_new, const int64_t* seg_old, int64_t* perm,
                             int64_t* iperm) {
  CQP_GRID_LOOP(i, n) {
    int64_t lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (seg_new[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int64_t o = seg_old[lo] + (i - seg_new[lo]);
    perm[i] = o;
    iperm[o] = i;
  }
}
// sum of q^2 over [a, b) (cone coordinates: zero q means Euclidean projections)
__global__ void k_sumsq_range(int64_t a, int64_t b, const double* q, double* out) {
  double s = 0.0;
  for (int64_t i = a + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b; i += (int64_t)gridDim.x * blockDim.x)
    s += q[i] * q[i];
  s = cqp::warp_sum(s);
  if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out, s);
}
template <typename T>
__global__ void k_rx_partial(int64_t k, int64_t n, const T* R, const T* x, double* out) {
  // out[l] += sum_i R[l, i] x_i (deterministic enough for a one-off start value)
  for (int64_t l = blockIdx.y; l < k; l += gridDim.y) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      s += (double)R[l * n + i] * (double)x[i];
    s = cqp::warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(&out[l], s);
  }
}
__global__ void k_state_set_th(cqp::State* S, const double* t, int k) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    for (int l = 0; l < k; ++l) S->t_h[l] = t[l];
}

// threads-per-row decisions of the timing autotuner, per device and matrix shape
// (rows, nonzeros, value size), so later set-ups of same-shaped problems skip the sweep
std::mutex g_tune_mu;
std::map<std::tuple<int, int64_t, int64_t, int>, int> g_tune_cache;

int pow2_tpr(double mean) {
  int t = 1;
  while (t < 32 && t < mean) t <<= 1;
  return t;
}

template <typename T>
struct Handle : HandleBase {
  cqp_options opt;
  cudaStream_t st = nullptr;
  int nsm = 152;
  int64_t n = 0, m = 0, nnz = 0, k = 0, pnnz = 0;
  Arena mem;
  int64_t* perm = nullptr;
  int64_t* iperm = nullptr;
  cqp::Prob<T> P{};
  cqp::Work<T> W{};
  cqp::Opts O{};
  cqp::State* S = nullptr;
  unsigned* bar_count = nullptr;
  int* dev_err = nullptr;
  double* kkt_out = nullptr;
  T* tmp_x = nullptr;
  T* tmp_y = nullptr;
  double eta = 0, normA = 0, omega0 = 1, setup_ms = 0;
  int power_its = 0;                 // Lanczos steps of the norm estimate taken by setup
  long long setup_launches = 0;
  int64_t n_roots = 0;
  int team = cqp::kTeamCta;          // how the solver's blocks cooperate (launch.h TeamKind)
  int blocks = 1, threads = 512;
  // batched mode (cqp_setup_batch): per-instance ranges, factors and step sizes
  bool batched = false;
  int64_t bcount = 0;
  cqp::Own* d_own = nullptr;
  double *d_bb = nullptr, *d_bc = nullptr, *d_nb = nullptr, *d_nc = nullptr;
  int* d_order = nullptr;
  int* d_rank = nullptr;
  unsigned* d_queue = nullptr;
  std::vector<double> h_eta, h_om;

  ~Handle() override { mem.release(); }

  cqp::KernelArgs<T> args(long long budget) {
    cqp::KernelArgs<T> a;
    a.P = P;
    a.W = W;
    a.O = O;
    a.S = S;
    a.bar.count = bar_count;
    a.bar.err = dev_err;
    a.budget = budget;
    return a;
  }

  void setup(const cqp_csr* A, const cqp_qop* Q, const double* c_in, const double* b_in, const cqp_cones* K,
             const cqp_options& o, const cqp_batch* B = nullptr, const cqp_bounds* G = nullptr) {
    auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = g_launches;
    opt = o;
    st = (cudaStream_t)o.stream;
    mem.st = st;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    m = A->nrows;
    n = A->ncols;
    nnz = A->nnz;
    const bool on_dev = o.input_on_device != 0;
    Temp tmp(st);
    auto upload = [&](const void* src, size_t bytes) -> const void* {
      if (!src) return nullptr;
      if (on_dev) return src;
      void* d = tmp.alloc<char>((int64_t)bytes);
      CK(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st));
      return d;
    };
    auto fetch = [&](const void* src, size_t bytes, void* dst) {
      if (on_dev) CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
      else memcpy(dst, src, bytes);
    };
    // ---- cone partition (host; nblocks entries) --------------------------------
    const int64_t nb = K->nblocks;
    std::vector<int32_t> bt(nb);
    std::vector<int64_t> bs(nb), bd(nb);
    std::vector<double> ba(nb, 0.0);
    if (nb > 0) {
      fetch(K->type, nb * sizeof(int32_t), bt.data());
      fetch(K->start, nb * sizeof(int64_t), bs.data());
      fetch(K->dim, nb * sizeof(int64_t), bd.data());
      if (K->alpha) fetch(K->alpha, nb * sizeof(double), ba.data());
      CK(cudaStreamSynchronize(st));
    }
    int64_t pos = 0;
    for (int64_t j = 0; j < nb; ++j) {
      if (bs[j] != pos || bd[j] < 1) fail(CQP_ERR_INVALID, "cone blocks must partition 0..n-1 contiguously in order");
      const int t = bt[j];
      if (t < 0 || t > 8) fail(CQP_ERR_INVALID, "unknown cone type");
      const bool slice = t == CQP_CONE_EXP1 || t == CQP_CONE_POW1;
      if (slice && B) fail(CQP_ERR_UNSUPPORTED, "slice blocks (EXP1/POW1) in a batch");
      if (slice && o.rescaled_cones) fail(CQP_ERR_UNSUPPORTED, "slice blocks (EXP1/POW1) with rescaled_cones");
      if (slice && bd[j] != 3) fail(CQP_ERR_INVALID, "EXP1/POW1 block dimension != 3");
      if (t == CQP_CONE_POW1 && !(ba[j] > 0.0 && ba[j] < 1.0)) fail(CQP_ERR_INVALID, "power slice alpha outside (0,1)");
      if (t == CQP_CONE_BOX && (!G || !G->x_lo || !G->x_hi)) fail(CQP_ERR_INVALID, "box blocks need x_lo and x_hi");
      if (t == CQP_CONE_BOX && B) fail(CQP_ERR_UNSUPPORTED, "box blocks in a batch");
      if (t == CQP_CONE_SOC && bd[j] < 2) fail(CQP_ERR_INVALID, "SOC block dimension < 2");
      if (t == CQP_CONE_RSOC && bd[j] < 3) fail(CQP_ERR_INVALID, "RSOC block dimension < 3");
      if ((t == CQP_CONE_EXP || t == CQP_CONE_POW) && bd[j] != 3) fail(CQP_ERR_INVALID, "EXP/POW block dimension != 3");
      if (t == CQP_CONE_POW && !(ba[j] > 0.0 && ba[j] < 1.0)) fail(CQP_ERR_INVALID, "power cone alpha outside (0,1)");
      pos += bd[j];
    }
    if (pos != n) fail(CQP_ERR_INVALID, "cone blocks do not cover 0..n-1");
    // segment table in the new order: free, nonneg, soc, rsoc, exp, pow (stable within a type)
    std::vector<int64_t> seg_new, seg_old;
    if (B && o.rescaled_cones) fail(CQP_ERR_UNSUPPORTED, "rescaled-cone mode in a batch");
    if (o.matrix_bf16 < 0 || o.matrix_bf16 > 2) fail(CQP_ERR_INVALID, "matrix_bf16 must be 0, 1 or 2");
    const bool bf = o.matrix_bf16 != 0;      // A and A' values in BF16
    const bool bfp = o.matrix_bf16 == 2;     // and the sparse part P of Q
    if (bf && (B || !std::is_same<T, float>::value))
      fail(CQP_ERR_UNSUPPORTED, "matrix_bf16 needs FP32 iterates (precision 0) and a single problem");
    std::vector<int64_t> soc_off{0}, rsoc_off{0};
    std::vector<double> pow_al;
    std::vector<double> exp_sl, pow_sl;   // 1 for a slice block, 0 for a cone, in segment order
    bool any_slice = false;
    int64_t cnt[6] = {0, 0, 0, 0, 0, 0};
    // box blocks live in the free segment (their bounds are applied coordinatewise); slices
    // share the exponential / power segments with the cones and are told apart per block
    std::vector<int32_t> seg_of(nb);
    for (int64_t j = 0; j < nb; ++j) {
      const int t = bt[j];
      seg_of[j] = t == CQP_CONE_BOX ? 0 : (t == CQP_CONE_EXP1 ? 4 : (t == CQP_CONE_POW1 ? 5 : t));
      if (t == CQP_CONE_EXP1 || t == CQP_CONE_POW1) any_slice = true;
    }
    for (int64_t j = 0; j < nb; ++j) cnt[seg_of[j]] += bd[j];
    int64_t base[6];
    base[0] = 0;
    for (int t = 1; t < 6; ++t) base[t] = base[t - 1] + cnt[t - 1];
    int64_t fill[6];
    for (int t = 0; t < 6; ++t) fill[t] = base[t];
    for (int t = 0; t < 6; ++t)
      for (int64_t j = 0; j < nb; ++j) {
        if (seg_of[j] != t) continue;
        seg_new.push_back(fill[t]);
        seg_old.push_back(bs[j]);
        if (t == CQP_CONE_SOC) soc_off.push_back(fill[t] + bd[j]);
        if (t == CQP_CONE_RSOC) rsoc_off.push_back(fill[t] + bd[j]);
        if (t == CQP_CONE_POW) pow_al.push_back(ba[j]);
        if (t == CQP_CONE_EXP) exp_sl.push_back(bt[j] == CQP_CONE_EXP1 ? 1.0 : 0.0);
        if (t == CQP_CONE_POW) pow_sl.push_back(bt[j] == CQP_CONE_POW1 ? 1.0 : 0.0);
        fill[t] += bd[j];
      }
    soc_off[0] = base[2];
    rsoc_off[0] = base[3];
    // ---- batched mode: instance of every block and each instance's permuted ranges -----
    std::vector<cqp::Own> hown;
    std::vector<int32_t> inst_col, inst_row;
    if (B) {
      batched = true;
      bcount = B->count;
      if (bcount < 1 || !B->x_off || !B->row_off) fail(CQP_ERR_INVALID, "batch: count >= 1 and offsets required");
      const int64_t* xo = B->x_off;
      const int64_t* ro = B->row_off;
      if (xo[0] != 0 || xo[bcount] != n || ro[0] != 0 || ro[bcount] != m)
        fail(CQP_ERR_INVALID, "batch: offsets must start at 0 and end at n (x_off) and m (row_off)");
      for (int64_t i = 0; i < bcount; ++i)
        if (xo[i + 1] <= xo[i] || ro[i + 1] < ro[i]) fail(CQP_ERR_INVALID, "batch: offsets must increase");
      std::vector<int64_t> ib(nb);
      int64_t cur = 0;
      for (int64_t j = 0; j < nb; ++j) {
        while (bs[j] >= xo[cur + 1]) ++cur;
        if (bs[j] + bd[j] > xo[cur + 1]) fail(CQP_ERR_INVALID, "batch: a cone block straddles two instances");
        ib[j] = cur;
      }
      hown.assign(bcount, cqp::Own{});
      std::vector<int64_t> bidx0(6 * bcount, -1), bidx1(6 * bcount, -1);
      for (auto& ow : hown)
        for (int t = 0; t < 6; ++t) { ow.x0[t] = -1; ow.x1[t] = -1; }
      int64_t f2[6];
      for (int t = 0; t < 6; ++t) f2[t] = base[t];
      int64_t tidx[6] = {0, 0, 0, 0, 0, 0};
      for (int t = 0; t < 6; ++t)
        for (int64_t j = 0; j < nb; ++j) {
          if (bt[j] != t) continue;
          cqp::Own& ow = hown[ib[j]];
          if (ow.x0[t] < 0) { ow.x0[t] = f2[t]; bidx0[6 * ib[j] + t] = tidx[t]; }
          f2[t] += bd[j];
          ow.x1[t] = f2[t];
          ++tidx[t];
          bidx1[6 * ib[j] + t] = tidx[t];
        }
      for (int64_t i = 0; i < bcount; ++i) {
        cqp::Own& ow = hown[i];
        for (int t = 0; t < 6; ++t)
          if (ow.x0[t] < 0) { ow.x0[t] = ow.x1[t] = base[t]; bidx0[6 * i + t] = bidx1[6 * i + t] = 0; }
        ow.f0 = ow.x0[0]; ow.f1 = ow.x1[0];
        ow.nn0 = ow.x0[1]; ow.nn1 = ow.x1[1];
        ow.s0 = bidx0[6 * i + 2]; ow.s1 = bidx1[6 * i + 2];
        ow.r0 = bidx0[6 * i + 3]; ow.r1 = bidx1[6 * i + 3];
        // exp / pow blocks are indexed by their position in the segment (3 coordinates each)
        ow.e0 = (ow.x0[4] - base[4]) / 3; ow.e1 = (ow.x1[4] - base[4]) / 3;
        ow.p0 = (ow.x0[5] - base[5]) / 3; ow.p1 = (ow.x1[5] - base[5]) / 3;
        ow.row0 = ro[i]; ow.row1 = ro[i + 1];
      }
      inst_col.resize(n);
      inst_row.resize(std::max<int64_t>(m, 1));
      for (int64_t i = 0; i < bcount; ++i) {
        for (int64_t j = xo[i]; j < xo[i + 1]; ++j) inst_col[j] = (int32_t)i;
        for (int64_t r = ro[i]; r < ro[i + 1]; ++r) inst_row[r] = (int32_t)i;
      }
    }
    // ---- sizes and options --------------------------------------------------------
    if (m < 0 || n < 1 || nnz < 0 || nnz >= (int64_t(1) << 31)) fail(CQP_ERR_INVALID, "bad matrix sizes");
    k = Q ? Q->rank : 0;
    if (k < 0 || k > cqp::kMaxRank) fail(CQP_ERR_INVALID, "rank of R must be <= 64");
    const bool has_p = Q && Q->P.rowptr;
    pnnz = has_p ? Q->P.nnz : 0;
    if (has_p && (Q->P.nrows != n || Q->P.ncols != n || pnnz >= (int64_t(1) << 31)))
      fail(CQP_ERR_INVALID, "P must be n x n");
    if (k > 0 && (!Q->R || !Q->D)) fail(CQP_ERR_INVALID, "rank > 0 needs R and D");
    // ---- upload inputs (FP64) and validate ------------------------------------------
    // host row pointers are checked before upload (rowptr[0] = 0, non-decreasing, last = nnz);
    // device ones by k_validate_csr below, which reads only the caller's nnz entries
    auto check_rowptr = [&](const int64_t* rp, int64_t rows, int64_t nz, const char* what) {
      if (on_dev || !rp) return;
      bool ok = rp[0] == 0 && rp[rows] == nz;
      for (int64_t r = 0; r < rows && ok; ++r) ok = rp[r] <= rp[r + 1];
      if (!ok) fail(CQP_ERR_INVALID, std::string(what) + ".rowptr must start at 0, not decrease and end at nnz");
    };
    if (!A->rowptr) fail(CQP_ERR_INVALID, "A.rowptr is required (nrows + 1 entries)");
    check_rowptr(A->rowptr, m, nnz, "A");
    if (has_p) check_rowptr(Q->P.rowptr, n, pnnz, "P");
    const int64_t* a_rp64 = (const int64_t*)upload(A->rowptr, (m + 1) * sizeof(int64_t));
    const int32_t* a_ci_in = (const int32_t*)upload(A->colind, nnz * sizeof(int32_t));
    const double* a_v_in = (const double*)upload(A->val, nnz * sizeof(double));
    const double* c_d = (const double*)upload(c_in, n * sizeof(double));
    const bool general = G != nullptr;
    int64_t* d_xoff_old = nullptr;   // batch: instance x offsets in the caller's coordinates
    if (general && m > 0 && (!G->row_lo || !G->row_hi)) fail(CQP_ERR_INVALID, "row_lo and row_hi are required");
    const double* b_d = (const double*)upload(general ? G->row_lo : b_in, m * sizeof(double));
    const double* bhi_d = general ? (const double*)upload(G->row_hi, m * sizeof(double)) : nullptr;
    const double* xlo_d = general && G->x_lo ? (const double*)upload(G->x_lo, n * sizeof(double)) : nullptr;
    const double* xhi_d = general && G->x_hi ? (const double*)upload(G->x_hi, n * sizeof(double)) : nullptr;
    const double* qd_in = Q ? (const double*)upload(Q->diag, n * sizeof(double)) : nullptr;
    const double* R_in = k > 0 ? (const double*)upload(Q->R, k * n * sizeof(double)) : nullptr;
    const double* D_in = k > 0 ? (const double*)upload(Q->D, k * k * sizeof(double)) : nullptr;
    const int64_t* p_rp64 = has_p ? (const int64_t*)upload(Q->P.rowptr, (n + 1) * sizeof(int64_t)) : nullptr;
    const int32_t* p_ci_in = has_p ? (const int32_t*)upload(Q->P.colind, pnnz * sizeof(int32_t)) : nullptr;
    const double* p_v_in = has_p ? (const double*)upload(Q->P.val, pnnz * sizeof(double)) : nullptr;
    if (!c_d || (m > 0 && !b_d)) fail(CQP_ERR_INVALID, "c and b are required");
    int* bad = tmp.alloc<int>(1);
    CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
    count_launch(); cqp::k_validate_csr<<<cqp::grid_for(nnz + m), cqp::kSetupThreads, 0, st>>>(m, n, nnz, a_rp64, a_ci_in, a_v_in, bad);
    count_launch(); cqp::k_validate_vec<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, c_d, bad);
    if (m > 0 && !general) { count_launch(); cqp::k_validate_vec<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, b_d, bad); }
    if (m > 0 && general) { count_launch(); cqp::k_validate_bounds<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, b_d, bhi_d, nullptr, bad); }
    uint8_t* boxmask = nullptr;
    if (xlo_d) {
      std::vector<uint8_t> hm(n, 0);
      for (int64_t j = 0; j < nb; ++j)
        if (bt[j] == CQP_CONE_BOX) memset(hm.data() + bs[j], 1, (size_t)bd[j]);
      boxmask = tmp.alloc<uint8_t>(n);
      CK(cudaMemcpyAsync(boxmask, hm.data(), n, cudaMemcpyHostToDevice, st));
      count_launch(); cqp::k_validate_bounds<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, xlo_d, xhi_d, boxmask, bad);
    }
    if (qd_in) { count_launch(); cqp::k_validate_vec<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, qd_in, bad); }
    if (R_in) { count_launch(); cqp::k_validate_vec<<<cqp::grid_for(k * n), cqp::kSetupThreads, 0, st>>>(k * n, R_in, bad); }
    if (has_p) { count_launch(); cqp::k_validate_csr<<<cqp::grid_for(pnnz + n), cqp::kSetupThreads, 0, st>>>(n, n, pnnz, p_rp64, p_ci_in, p_v_in, bad); }
    int hbad = 0;
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    int64_t last_rp = 0;
    CK(cudaMemcpyAsync(&last_rp, a_rp64 + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hbad) fail(CQP_ERR_INVALID, "invalid or non-finite input data (flags " + std::to_string(hbad) + ")");
    if (last_rp != nnz) fail(CQP_ERR_INVALID, "A.rowptr[m] != nnz");
    double* part = tmp.alloc<double>(1024);
    double* one = tmp.alloc<double>(1);
    // size of the right-hand side (reading: per row the largest finite bound magnitude)
    auto bound_norm = [&](const double* lo, const double* hi) {
      if (m == 0) return 0.0;
      if (!hi) return std::sqrt(dev_dot(lo, nullptr, m, part, one, st));
      double* mag = tmp.alloc<double>(m);
      count_launch(); cqp::k_bound_mag<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, lo, hi, mag);
      return std::sqrt(dev_dot(mag, nullptr, m, part, one, st));
    };
    P.norm_b = bound_norm(b_d, bhi_d);
    P.norm_c = std::sqrt(dev_dot(c_d, nullptr, n, part, one, st));
    if (batched) {
      d_own = mem.alloc<cqp::Own>(bcount);
      CK(cudaMemcpyAsync(d_own, hown.data(), bcount * sizeof(cqp::Own), cudaMemcpyHostToDevice, st));
      int32_t* d_ic = tmp.alloc<int32_t>(n);
      int32_t* d_ir = tmp.alloc<int32_t>(std::max<int64_t>(m, 1));
      CK(cudaMemcpyAsync(d_ic, inst_col.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(d_ir, inst_row.data(), inst_row.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
      CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
      if (m > 0) { count_launch(); cqp::k_check_blockdiag<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, a_rp64, a_ci_in, d_ir, d_ic, bad); }
      if (has_p) { count_launch(); cqp::k_check_blockdiag<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, p_rp64, p_ci_in, d_ic, d_ic, bad); }
      int64_t* d_xo = tmp.alloc<int64_t>(bcount + 1);
      d_xoff_old = d_xo;
      int64_t* d_ro = tmp.alloc<int64_t>(bcount + 1);
      CK(cudaMemcpyAsync(d_xo, B->x_off, (bcount + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(d_ro, B->row_off, (bcount + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
      d_nb = mem.alloc<double>(bcount);
      d_nc = mem.alloc<double>(bcount);
      count_launch(); cqp::k_inst_norms<<<(int)std::min<int64_t>(bcount, 8 * nsm), cqp::kBatchSetupThreads, 0, st>>>(bcount, d_xo, d_ro, c_d, b_d, d_nb, d_nc);
      CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (hbad) fail(CQP_ERR_INVALID, "batch: an entry of A or P joins two instances");
    }
    // ---- permutation ------------------------------------------------------------------
    perm = mem.alloc<int64_t>(n);
    iperm = mem.alloc<int64_t>(n);
    {
      int64_t* sn = tmp.alloc<int64_t>(seg_new.size());
      int64_t* so = tmp.alloc<int64_t>(seg_old.size());
      CK(cudaMemcpyAsync(sn, seg_new.data(), seg_new.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(so, seg_old.data(), seg_old.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
      count_launch(); k_build_perm<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, (int64_t)seg_new.size(), sn, so, perm, iperm);
    }
    // A with remapped columns, FP64 working values
    int32_t* a_rp = mem.alloc<int32_t>(m + 1);
    int32_t* a_ci = mem.alloc<int32_t>(nnz);
    double* av = tmp.alloc<double>(nnz);
    count_launch(); cqp::k_copy_rowptr32<<<cqp::grid_for(m + 1), cqp::kSetupThreads, 0, st>>>(m + 1, a_rp64, a_rp);
    count_launch(); cqp::k_remap_cols<<<cqp::grid_for(nnz), cqp::kSetupThreads, 0, st>>>(nnz, iperm, a_ci_in, a_ci);
    CK(cudaMemcpyAsync(av, a_v_in, nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (bf && nnz > 0) { count_launch(); cqp::k_round_bf16<<<cqp::grid_for(nnz), cqp::kSetupThreads, 0, st>>>(nnz, av); }
    double* cv = tmp.alloc<double>(n);
    double* qv = tmp.alloc<double>(n);
    double* bv = tmp.alloc<double>(std::max<int64_t>(m, 1));
    count_launch(); cqp::k_gather<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, perm, c_d, cv, 0.0);
    count_launch(); cqp::k_gather<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, perm, qd_in, qv, 0.0);
    if (m > 0) CK(cudaMemcpyAsync(bv, b_d, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    double* bhv = nullptr;   // general form: scaled row upper bounds (FP64 working copy)
    if (bhi_d && m > 0) {
      bhv = tmp.alloc<double>(m);
      CK(cudaMemcpyAsync(bhv, bhi_d, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    double* Rv = nullptr;
    double* Dv = nullptr;
    if (k > 0) {
      Rv = tmp.alloc<double>(k * n);
      count_launch(); cqp::k_gather_cols<<<cqp::grid_for(k * n), cqp::kSetupThreads, 0, st>>>(k, n, perm, R_in, Rv);
      Dv = mem.alloc<double>(k * k);
      CK(cudaMemcpyAsync(Dv, D_in, k * k * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    int32_t* p_rp = nullptr;
    int32_t* p_ci = nullptr;
    double* pv = nullptr;
    if (has_p) {
      int32_t* len = tmp.alloc<int32_t>(n);
      p_rp = mem.alloc<int32_t>(n + 1);
      p_ci = mem.alloc<int32_t>(pnnz);
      pv = tmp.alloc<double>(pnnz);
      count_launch(); cqp::k_row_lengths_perm<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, perm, p_rp64, len);
      dev_scan(len, p_rp, n, tmp, st);
      count_launch(); cqp::k_copy_rows_perm<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, perm, iperm, p_rp64, p_ci_in, p_v_in,
                                                                                p_rp, p_ci, pv);
      if (bfp && pnnz > 0) { count_launch(); cqp::k_round_bf16<<<cqp::grid_for(pnnz), cqp::kSetupThreads, 0, st>>>(pnnz, pv); }
    }
    // ---- transpose of A (deterministic: every row of A' sorted by row of A) ------------
    int32_t* t_rp = mem.alloc<int32_t>(n + 1);
    int32_t* t_ci = mem.alloc<int32_t>(nnz);
    int32_t* tmap = tmp.alloc<int32_t>(nnz);
    {
      int32_t* cntc = tmp.alloc<int32_t>(n);
      CK(cudaMemsetAsync(cntc, 0, n * sizeof(int32_t), st));
      count_launch(); cqp::k_count_cols<<<cqp::grid_for(nnz), cqp::kSetupThreads, 0, st>>>(nnz, a_ci, cntc);
      dev_scan(cntc, t_rp, n, tmp, st);
      int32_t* cursor = tmp.alloc<int32_t>(n);
      CK(cudaMemcpyAsync(cursor, t_rp, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
      count_launch(); cqp::k_scatter_transpose<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, a_rp, a_ci, cursor, t_ci, tmap);
      int32_t* long_list = tmp.alloc<int32_t>(n);
      unsigned* long_cm = tmp.alloc<unsigned>(2);   // count, longest
      CK(cudaMemsetAsync(long_cm, 0, 2 * sizeof(unsigned), st));
      count_launch(); cqp::k_sort_segments<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, t_rp, t_ci, tmap, long_list, long_cm, long_cm + 1);
      count_launch(); cqp::k_sort_long_segments<<<2 * nsm, cqp::kSegSortThreads, 0, st>>>(t_rp, t_ci, tmap, long_list, long_cm);
      unsigned hcm[2] = {0u, 0u};
      CK(cudaMemcpyAsync(hcm, long_cm, sizeof(hcm), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (hcm[1] > (unsigned)cqp::kSegSortCap) {
        unsigned long long* sbuf = tmp.alloc<unsigned long long>(hcm[1]);
        count_launch(); cqp::k_sort_huge_segments<<<1, cqp::kSegSortThreads, 0, st>>>(t_rp, t_ci, tmap, long_list, long_cm, sbuf);
      }
    }
    // ---- rescaling (Table practical-defaults: Ruiz x10, Pock-Chambolle alpha = 1,
    // cone-preserving aggregation, bound-objective) -------------------------------------
    double* col = mem.alloc<double>(n);
    double* row = mem.alloc<double>(std::max<int64_t>(m, 1));
    double* colf = tmp.alloc<double>(n);
    double* rowf = tmp.alloc<double>(std::max<int64_t>(m, 1));
    count_launch(); cqp::k_fill<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, col, 1.0);
    if (m > 0) { count_launch(); cqp::k_fill<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, row, 1.0); }
    int64_t* d_soc = mem.alloc<int64_t>(soc_off.size());
    int64_t* d_rsoc = mem.alloc<int64_t>(rsoc_off.size());
    CK(cudaMemcpyAsync(d_soc, soc_off.data(), soc_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_rsoc, rsoc_off.data(), rsoc_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    const int64_t n_soc = (int64_t)soc_off.size() - 1, n_rsoc = (int64_t)rsoc_off.size() - 1;
    const int64_t n_exp = cnt[4] / 3, n_pow = cnt[5] / 3;
    auto aggregate = [&](int mode) {
      if (n_soc) { count_launch(); cqp::k_aggregate_blocks<<<cqp::grid_for(n_soc), cqp::kSetupThreads, 0, st>>>(n_soc, d_soc, 0, 0, mode, colf); }
      if (n_rsoc) { count_launch(); cqp::k_aggregate_blocks<<<cqp::grid_for(n_rsoc), cqp::kSetupThreads, 0, st>>>(n_rsoc, d_rsoc, 0, 0, mode, colf); }
      if (n_exp) { count_launch(); cqp::k_aggregate_blocks<<<cqp::grid_for(n_exp), cqp::kSetupThreads, 0, st>>>(n_exp, nullptr, base[4], 3, mode, colf); }
      if (n_pow) { count_launch(); cqp::k_aggregate_blocks<<<cqp::grid_for(n_pow), cqp::kSetupThreads, 0, st>>>(n_pow, nullptr, base[5], 3, mode, colf); }
    };
    auto scale_step = [&]() {
      count_launch(); cqp::k_scale_matrix<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, a_rp, a_ci, av, rowf, colf);
      count_launch(); cqp::k_mul<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, col, colf);
      if (m > 0) { count_launch(); cqp::k_mul<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, row, rowf); }
    };
    for (int it = 0; it < o.ruiz_iters; ++it) {
      count_launch(); cqp::k_col_stat<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, t_rp, tmap, av, 0, 0.0, colf);
      if (m > 0) { count_launch(); cqp::k_row_stat<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, a_rp, av, 0, 0.0, rowf); }
      count_launch(); cqp::k_sqrt_or_one<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, colf);
      if (m > 0) { count_launch(); cqp::k_sqrt_or_one<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, rowf); }
      if (!o.rescaled_cones) aggregate(0);
      scale_step();
    }
    if (o.pc_alpha >= 0.0) {
      const double al = o.pc_alpha;
      count_launch(); cqp::k_col_stat<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, t_rp, tmap, av, 1, 2.0 - al, colf);
      if (m > 0) { count_launch(); cqp::k_row_stat<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, a_rp, av, 1, al, rowf); }
      count_launch(); cqp::k_sqrt_or_one<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, colf);
      if (m > 0) { count_launch(); cqp::k_sqrt_or_one<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, rowf); }
      if (!o.rescaled_cones) aggregate(1);
      scale_step();
    }
    if (bf) {
      // power-of-two factors keep the BF16 values of A and P exact: the cumulative Ruiz and
      // Pock-Chambolle factors are rounded once, and A is brought to the rounded factors
      count_launch(); cqp::k_pow2_ratio<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, col, colf);
      if (m > 0) { count_launch(); cqp::k_pow2_ratio<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, row, rowf); }
      if (m > 0) { count_launch(); cqp::k_scale_matrix<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, a_rp, a_ci, av, rowf, colf); }
    }
    count_launch(); cqp::k_div<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, cv, col);
    if (m > 0) { count_launch(); cqp::k_div<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, bv, row); }
    if (bhv) { count_launch(); cqp::k_div<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, bhv, row); }
    count_launch(); cqp::k_div2<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, qv, col);
    if (has_p) { count_launch(); cqp::k_scale_sym<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, p_rp, p_ci, pv, col); }
    if (k > 0) { count_launch(); cqp::k_scale_cols<<<cqp::grid_for(k * n), cqp::kSetupThreads, 0, st>>>(k, n, Rv, col); }
    double beta_b = 1.0, beta_c = 1.0;
    if (batched) {
      d_bb = mem.alloc<double>(bcount);
      d_bc = mem.alloc<double>(bcount);
      count_launch();
      cqp::k_inst_bound_obj<<<(int)std::min<int64_t>(bcount, 8 * nsm), cqp::kBatchSetupThreads, 0, st>>>(
          bcount, d_own, n, o.bound_obj, cv, bv, qv, k, Rv, p_rp, pv, d_bb, d_bc);
      if (k > 0) {
        d_rank = mem.alloc<int>(bcount);
        count_launch();
        cqp::k_inst_rank<<<(int)std::min<int64_t>(bcount, 8 * nsm), cqp::kBatchSetupThreads, 0, st>>>(bcount, d_own, n, k, Rv, d_rank);
      }
    } else if (o.bound_obj) {
      beta_b = bound_norm(bv, bhv) + 1.0;
      beta_c = std::sqrt(dev_dot(cv, nullptr, n, part, one, st)) + 1.0;
      if (bf) {
        beta_b = cqp::pow2_round(beta_b);
        beta_c = cqp::pow2_round(beta_c);
      }
      if (m > 0) { count_launch(); cqp::k_scal<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, bv, 1.0 / beta_b); }
      if (bhv) { count_launch(); cqp::k_scal<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, bhv, 1.0 / beta_b); }
      count_launch(); cqp::k_scal<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, cv, 1.0 / beta_c);
      const double qs = beta_b / beta_c;
      count_launch(); cqp::k_scal<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, qv, qs);
      if (has_p) { count_launch(); cqp::k_scal<<<cqp::grid_for(pnnz), cqp::kSetupThreads, 0, st>>>(pnnz, pv, qs); }
      if (k > 0) { count_launch(); cqp::k_scal<<<1, 64, 0, st>>>(k * k, Dv, qs); }
    }
    // full diagonal of Q~ (Jacobi metric) and conversion to the iterate precision
    double* jdv = tmp.alloc<double>(n);
    count_launch(); cqp::k_full_diag<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, qv, p_rp, p_ci, pv, k, Rv, Dv, jdv);
    // in the BF16 mode the iterate-precision copies serve only the norm estimate and the
    // autotuner during setup; the handle keeps the BF16 ones
    T* a_v = bf ? tmp.alloc<T>(nnz) : mem.alloc<T>(nnz);
    T* t_v = bf ? tmp.alloc<T>(nnz) : mem.alloc<T>(nnz);
    count_launch(); cqp::k_convert<T><<<cqp::grid_for(nnz), cqp::kSetupThreads, 0, st>>>(nnz, av, a_v);
    count_launch(); cqp::k_gather_convert<T><<<cqp::grid_for(nnz), cqp::kSetupThreads, 0, st>>>(nnz, tmap, av, t_v);
    __nv_bfloat16* a_vb = nullptr;
    __nv_bfloat16* t_vb = nullptr;
    if (bf && nnz > 0) {
      a_vb = mem.alloc<__nv_bfloat16>(nnz);
      t_vb = mem.alloc<__nv_bfloat16>(nnz);
      count_launch(); cqp::k_to_bf16<<<cqp::grid_for(nnz), cqp::kSetupThreads, 0, st>>>(nnz, nullptr, av, a_vb);
      count_launch(); cqp::k_to_bf16<<<cqp::grid_for(nnz), cqp::kSetupThreads, 0, st>>>(nnz, tmap, av, t_vb);
    }
    T* cT = mem.alloc<T>(n);
    T* bT = mem.alloc<T>(std::max<int64_t>(m, 1));
    T* qT = mem.alloc<T>(n);
    T* jT = mem.alloc<T>(n);
    count_launch(); cqp::k_convert<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, cv, cT);
    if (m > 0) { count_launch(); cqp::k_convert<T><<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, bv, bT); }
    T* rhiT = nullptr;
    if (bhv) {
      rhiT = mem.alloc<T>(m);
      count_launch(); cqp::k_convert<T><<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, bhv, rhiT);
    }
    // box bounds of the free segment, x~ = col x / beta_b (infinite on free coordinates)
    T* xloT = nullptr;
    T* xhiT = nullptr;
    if (xlo_d && cnt[0] > 0) {
      xloT = mem.alloc<T>(cnt[0]);
      xhiT = mem.alloc<T>(cnt[0]);
      count_launch(); cqp::k_box_bounds<T><<<cqp::grid_for(cnt[0]), cqp::kSetupThreads, 0, st>>>(cnt[0], perm, boxmask, xlo_d, xhi_d, col, beta_b, xloT, xhiT);
    }
    count_launch(); cqp::k_convert<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, qv, qT);
    count_launch(); cqp::k_convert<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, jdv, jT);
    // rescaled-cone mode: a cone block of the scaled variable x~ = col x / beta_b is S K with
    // S = diag(col) on the block (the scalar beta_b drops out of a cone)
    T* cscT = nullptr;
    if (o.rescaled_cones && n > base[2]) {
      cscT = mem.alloc<T>(n);
      count_launch(); cqp::k_convert<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, col, cscT);
    }
    // R is stored with its row count padded to a multiple of 8 (zero rows), so the
    // inner step's register loop over a fixed width needs no per-row predicate
    T* RT = nullptr;
    const int64_t kpad = k > 0 ? (k + 7) / 8 * 8 : 0;
    if (k > 0) {
      RT = mem.alloc<T>(kpad * n);
      if (kpad > k) CK(cudaMemsetAsync(RT + k * n, 0, (size_t)(kpad - k) * n * sizeof(T), st));
      count_launch(); cqp::k_convert<T><<<cqp::grid_for(k * n), cqp::kSetupThreads, 0, st>>>(k * n, Rv, RT);
    }
    T* pT = nullptr;
    __nv_bfloat16* pTb = nullptr;
    if (has_p) {
      pT = bfp ? tmp.alloc<T>(pnnz) : mem.alloc<T>(pnnz);
      count_launch(); cqp::k_convert<T><<<cqp::grid_for(pnnz), cqp::kSetupThreads, 0, st>>>(pnnz, pv, pT);
      if (bfp && pnnz > 0) {
        pTb = mem.alloc<__nv_bfloat16>(pnnz);
        count_launch(); cqp::k_to_bf16<<<cqp::grid_for(pnnz), cqp::kSetupThreads, 0, st>>>(pnnz, nullptr, pv, pTb);
      }
    }
    double* palpha = nullptr;
    if (!pow_al.empty()) {
      palpha = mem.alloc<double>(pow_al.size());
      CK(cudaMemcpyAsync(palpha, pow_al.data(), pow_al.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    // slices: the fixed middle coordinate 1 of the caller's variables is col / beta_b in the
    // scaled variable x~ = col x / beta_b (one factor per block: cone-preserving aggregation)
    double* d_exp_fix = nullptr;
    double* d_pow_fix = nullptr;
    if (any_slice) {
      if (n_exp > 0) {
        d_exp_fix = mem.alloc<double>(n_exp);
        CK(cudaMemcpyAsync(d_exp_fix, exp_sl.data(), n_exp * sizeof(double), cudaMemcpyHostToDevice, st));
        count_launch(); cqp::k_slice_fix<<<cqp::grid_for(n_exp), cqp::kSetupThreads, 0, st>>>(n_exp, base[4], col, beta_b, d_exp_fix);
      }
      if (n_pow > 0) {
        d_pow_fix = mem.alloc<double>(n_pow);
        CK(cudaMemcpyAsync(d_pow_fix, pow_sl.data(), n_pow * sizeof(double), cudaMemcpyHostToDevice, st));
        count_launch(); cqp::k_slice_fix<<<cqp::grid_for(n_pow), cqp::kSetupThreads, 0, st>>>(n_pow, base[5], col, beta_b, d_pow_fix);
      }
    }
    // column blocks of A for the dual step: the gathered vector z = 2 w_x - h_x (n entries) is read
    // at random columns; when it is larger than a good part of L2, the product runs over blocks of
    // columns whose slice of z stays in L2 (reading: 8 slices above 64 MB)
    int cb_n = 0;
    int* cb_rp = nullptr;
    int* cb_ci = nullptr;
    T* cb_v = nullptr;
    __nv_bfloat16* cb_vb = nullptr;
    {
      const double zbytes = (double)n * sizeof(T);
      if (o.col_blocks >= 2) cb_n = std::min(o.col_blocks, 64);
      else if (o.col_blocks == 0 && zbytes > 64.0 * 1024 * 1024) cb_n = 8;
      if (batched || m == 0 || nnz == 0) cb_n = 0;
      if ((int64_t)cb_n * m >= (int64_t(1) << 31)) cb_n = 0;
      if (cb_n > 1) {
        const int64_t width = (n + cb_n - 1) / cb_n;
        int* cnt = tmp.alloc<int>((int64_t)cb_n * m);
        cb_rp = mem.alloc<int>((int64_t)cb_n * m + 1);
        cb_ci = mem.alloc<int>(nnz);
        count_launch(); cqp::k_cb_count<<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, a_rp, a_ci, width, cb_n, cnt);
        dev_scan(cnt, cb_rp, (int64_t)cb_n * m, tmp, st);
        if (a_vb) {
          cb_vb = mem.alloc<__nv_bfloat16>(nnz);
          count_launch(); cqp::k_cb_scatter<__nv_bfloat16><<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, a_rp, a_ci, a_vb, width, cb_n, cb_rp, cb_ci, cb_vb);
        } else {
          cb_v = mem.alloc<T>(nnz);
          count_launch(); cqp::k_cb_scatter<T><<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, a_rp, a_ci, a_v, width, cb_n, cb_rp, cb_ci, cb_v);
        }
      }
    }
    // column slices of A' for the A'y pass: its gathered vector y (m entries) is read at random
    // columns; above 64 MB the pass runs over slices of at most 100 MB of y (reading), or over the
    // forced count of col_blocks
    int tcb_n = 0;
    int* tcb_rp = nullptr;
    int* tcb_ci = nullptr;
    T* tcb_v = nullptr;
    __nv_bfloat16* tcb_vb = nullptr;
    {
      const double ybytes = (double)m * sizeof(T);
      if (o.col_blocks >= 2) tcb_n = std::min(o.col_blocks, 64);
      else if (o.col_blocks == 0 && ybytes > 64.0 * 1024 * 1024) tcb_n = (int)std::ceil(ybytes / (100.0 * 1024 * 1024));
      if (tcb_n < 2 || batched || m == 0 || nnz == 0) tcb_n = 0;
      if ((int64_t)tcb_n * n >= (int64_t(1) << 31)) tcb_n = 0;
      if (tcb_n > 1) {
        const int64_t width = (m + tcb_n - 1) / tcb_n;
        int* cnt = tmp.alloc<int>((int64_t)tcb_n * n);
        tcb_rp = mem.alloc<int>((int64_t)tcb_n * n + 1);
        tcb_ci = mem.alloc<int>(nnz);
        count_launch(); cqp::k_cb_count<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, t_rp, t_ci, width, tcb_n, cnt);
        dev_scan(cnt, tcb_rp, (int64_t)tcb_n * n, tmp, st);
        if (t_vb) {
          tcb_vb = mem.alloc<__nv_bfloat16>(nnz);
          count_launch(); cqp::k_cb_scatter<__nv_bfloat16><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, t_rp, t_ci, t_vb, width, tcb_n, tcb_rp, tcb_ci, tcb_vb);
        } else {
          tcb_v = mem.alloc<T>(nnz);
          count_launch(); cqp::k_cb_scatter<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, t_rp, t_ci, t_v, width, tcb_n, tcb_rp, tcb_ci, tcb_v);
        }
      }
    }
    // Euclidean projections suffice when the diagonal Q vanishes on every cone coordinate
    double qcone = 0.0;
    {
      double* acc = tmp.alloc<double>(1);
      CK(cudaMemsetAsync(acc, 0, sizeof(double), st));
      count_launch(); k_sumsq_range<<<cqp::grid_for(n - base[2]), cqp::kSetupThreads, 0, st>>>(base[2], n, qv, acc);
      CK(cudaMemcpyAsync(&qcone, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    // ---- ||A~||_2 by the Lanczos process on A~'A~ (reading: SplitMix64 start keyed by the
    // caller's coordinate index, Rayleigh quotient, stop at power_tol relative change or
    // power_iters) --------------------------------------------------------------------------
    {
      double* z = tmp.alloc<double>(n);
      double* zp = tmp.alloc<double>(n);   // previous Lanczos vector (zero at the start)
      CK(cudaMemsetAsync(zp, 0, n * sizeof(double), st));
      double* w = tmp.alloc<double>(std::max<int64_t>(m, 1));
      double* ppart = tmp.alloc<double>(2 * (int64_t)cqp::kMaxSlots * nsm);   // the grid team's two buffers
      unsigned* pcount = tmp.alloc<unsigned>(1);
      int* perr = tmp.alloc<int>(1);
      double* pout = tmp.alloc<double>(2);
      CK(cudaMemsetAsync(pcount, 0, sizeof(unsigned), st));
      CK(cudaMemsetAsync(perr, 0, sizeof(int), st));
      CK(cudaMemsetAsync(pout, 0, 2 * sizeof(double), st));
      if (!batched) {
        count_launch(); cqp::k_power_start<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, perm, z);
        const double zn = std::sqrt(dev_dot(z, nullptr, n, part, one, st));
        count_launch(); cqp::k_scal<<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, z, zn > 0.0 ? 1.0 / zn : 0.0);
      }
      double sig = 0.0;
      if (batched) {
        double* d_eta = tmp.alloc<double>(bcount);
        double* d_om = tmp.alloc<double>(bcount);
        double* d_na = tmp.alloc<double>(bcount);
        count_launch();
        cqp::k_inst_power<T><<<(int)std::min<int64_t>(bcount, 8 * nsm), cqp::kBatchSetupThreads, 0, st>>>(
            bcount, d_own, a_rp, a_ci, a_v, t_rp, t_ci, t_v, cv, bv, z, zp, w, o.power_iters, o.power_tol,
            o.step_factor, d_eta, d_om, d_na, perm, d_xoff_old);
        h_eta.resize(bcount);
        h_om.resize(bcount);
        std::vector<double> h_na(bcount);
        CK(cudaMemcpyAsync(h_eta.data(), d_eta, bcount * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(h_om.data(), d_om, bcount * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(h_na.data(), d_na, bcount * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (double v : h_na) sig = std::max(sig, v);
      } else if (m > 0) {
        cqp::GridBarrier pbar{pcount, perr};
        int iters = o.power_iters;
        double ptol = o.power_tol;
        const int32_t* arp = a_rp; const int32_t* aci = a_ci; const T* av = a_v;
        const int32_t* trp = t_rp; const int32_t* tci = t_ci; const T* tv = t_v;
        int64_t mm = m, nn = n;
        void* pargs[] = {&mm, &nn, &arp, &aci, &av, &trp, &tci, &tv, &z, &zp, &w, &ppart, &pbar, &iters, &ptol, &pout};
        count_launch();
        CK(cudaLaunchCooperativeKernel((void*)cqp::k_power<T>, dim3(nsm), dim3(cqp::kPowerThreads), pargs, 0, st));
        double hp[2];
        int herr = 0;
        CK(cudaMemcpyAsync(hp, pout, sizeof(hp), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&herr, perr, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (herr != 0) fail(CQP_ERR_WAIT, "norm estimate: grid barrier wait expired");
        sig = hp[0];
        power_its = (int)hp[1];
      }
      normA = sig;
      if (batched) {
        eta = h_eta[0];
        omega0 = h_om[0];
      } else {
        eta = o.step_factor / (sig > 0.0 ? sig : 1.0);
        const double cn = std::sqrt(dev_dot(cv, nullptr, n, part, one, st));
        const double bn = bound_norm(bv, bhv);
        omega0 = (cn > 1e-10 && bn > 1e-10) ? cn / bn : 1.0;   // reading: ||c~||/||b~||
      }
    }
    // ---- problem descriptor ----------------------------------------------------------------
    P.n = n; P.m = m;
    P.a_rp = a_rp; P.a_ci = a_ci; P.a_v = bf ? nullptr : a_v;
    P.t_rp = t_rp; P.t_ci = t_ci; P.t_v = bf ? nullptr : t_v;
    P.a_vb = a_vb; P.t_vb = t_vb; P.p_vb = pTb; P.cb_vb = cb_vb;
    P.tcb_n = tcb_n; P.tcb_rp = tcb_rp; P.tcb_ci = tcb_ci; P.tcb_v = tcb_v; P.tcb_vb = tcb_vb;
    P.qd = qT; P.jd = jT; P.k = (int)k; P.kpad = (int)kpad; P.R = RT; P.D = Dv;
    // D = d I (the common case) lets the kernel skip the k x k products
    P.d_scale = 0.0;
    if (k > 0) {
      std::vector<double> hD(k * k);
      CK(cudaMemcpyAsync(hD.data(), Dv, k * k * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      bool ident = hD[0] > 0.0;
      for (int64_t a = 0; a < k && ident; ++a)
        for (int64_t b2 = 0; b2 < k && ident; ++b2)
          if ((a == b2 && hD[a * k + b2] != hD[0]) || (a != b2 && hD[a * k + b2] != 0.0)) ident = false;
      if (ident) P.d_scale = hD[0];
    }
    P.p_rp = p_rp; P.p_ci = p_ci; P.p_v = bfp ? nullptr : pT;
    P.c = cT; P.b = bT; P.col = col; P.row = row; P.beta_b = beta_b; P.beta_c = beta_c;
    P.rhi = rhiT; P.xlo = xloT; P.xhi = xhiT; P.csc = cscT;
    P.n_free = cnt[0]; P.n_nonneg = cnt[1];
    P.n_soc = n_soc; P.soc_off = d_soc; P.n_rsoc = n_rsoc; P.rsoc_off = d_rsoc;
    P.n_exp = n_exp; P.exp_base = base[4]; P.n_pow = n_pow; P.pow_base = base[5]; P.pow_alpha = palpha;
    P.exp_fix = d_exp_fix; P.pow_fix = d_pow_fix;
    P.cb_n = cb_n; P.cb_rp = cb_rp; P.cb_ci = cb_ci; P.cb_v = cb_v;
    // rows of P of one common length (a matching Laplacian has two per row): their entries are
    // addressed without reading the row pointers
    P.p_ulen = 0;
    if (has_p && n > 0 && pnnz % n == 0 && pnnz / n > 0 && pnnz / n <= 64) {
      int* ubad = tmp.alloc<int>(1);
      CK(cudaMemsetAsync(ubad, 0, sizeof(int), st));
      count_launch(); cqp::k_check_uniform<<<cqp::grid_for(n + 1), cqp::kSetupThreads, 0, st>>>(n, p_rp, (int)(pnnz / n), ubad);
      int hb = 1;
      CK(cudaMemcpyAsync(&hb, ubad, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (!hb) P.p_ulen = (int)(pnnz / n);
    }
    if (has_p) P.qmode = cqp::kQSparse;
    else if (k > 0 || o.force_inner) P.qmode = cqp::kQLowRank;
    else P.qmode = cqp::kQDiag;
    P.euclid_cones = (P.qmode == cqp::kQDiag && qcone == 0.0) ? 1 : 0;
    // threads per CSR row: user choice, else the fastest of 1..16 lanes measured on this
    // matrix shape with the solver's row kernel (CUDA events, best of 2 after one warm-up),
    // remembered per device and shape for the rest of the process
    {
      T* xs = tmp.alloc<T>(n);
      T* ys = tmp.alloc<T>(std::max<int64_t>(std::max(m, n), 1));
      count_launch(); cqp::k_convert<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, jdv, xs);
      // ncols: length of the gathered operand; one lane with four rows in flight is only a
      // candidate when that operand does not fit in a good part of L2 (there the gathers' DRAM
      // latency binds; inside L2 the plain loop measured faster in the solver)
      auto tune = [&](int64_t rows, int64_t ncols, int64_t nz, const int32_t* rp, const int32_t* ci, const T* v) {
        if (rows == 0) return 1;
        int dev = 0;
        CK(cudaGetDevice(&dev));
        const auto key = std::make_tuple(dev, rows, nz, (int)sizeof(T));
        {
          std::lock_guard<std::mutex> lock(g_tune_mu);
          auto it = g_tune_cache.find(key);
          if (it != g_tune_cache.end()) return it->second;
        }
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        // timed on the solver's grid (one 512-thread block per SM), so the choice reflects the
        // loads in flight the persistent kernel has; 32 lanes per row never won.  The narrowest
        // width within 5% of the fastest is taken: inside the solver narrow groups measured
        // better than the standalone timing shows (Lasso model: 1 lane 230 ms, tuned 2 lanes
        // 294 ms of kernel time; SOCP mix: 1 lane within 0.4% of the best)
        // candidate widths in order of preference: one lane per row, one lane with four rows in
        // flight (cqp::kRowsBatched), then 2..16 lanes
        const int cand[6] = {1, cqp::kRowsBatched, 2, 4, 8, 16};
        const bool batched_ok = (double)ncols * sizeof(T) > 32.0 * 1024 * 1024;
        float ms_of[6];
        for (int ti = 0; ti < 6; ++ti) {
          const int t = cand[ti];
          if (t == cqp::kRowsBatched && !batched_ok) { ms_of[ti] = 1e30f; continue; }
          count_launch();
          CK(cqp::launch_spmv<T>(rows, rp, ci, v, xs, ys, t, st, nsm));
          float tot = 1e30f;
          for (int r = 0; r < 2; ++r) {
            CK(cudaEventRecord(e0, st));
            count_launch();
            CK(cqp::launch_spmv<T>(rows, rp, ci, v, xs, ys, t, st, nsm));
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            tot = std::min(tot, ms);
          }
          ms_of[ti] = tot;
        }
        float best_ms = 1e30f;
        for (int ti = 0; ti < 6; ++ti) best_ms = std::min(best_ms, ms_of[ti]);
        int best = 16;
        for (int ti = 5; ti >= 0; --ti)
          if (ms_of[ti] <= 1.05f * best_ms) best = cand[ti];
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
        return best;
      };
      P.tpr_a = o.tpr_a > 0 ? o.tpr_a : (o.tpr_a == -1 ? cqp::kRowsBatched : tune(m, n, nnz, a_rp, a_ci, a_v));
      P.tpr_t = o.tpr_at > 0 ? o.tpr_at : (o.tpr_at == -1 ? cqp::kRowsBatched : tune(n, m, nnz, t_rp, t_ci, t_v));
      P.tpr_p = !has_p ? 1 : (o.tpr_p > 0 ? o.tpr_p : (o.tpr_p == -1 ? cqp::kRowsBatched : tune(n, n, pnnz, p_rp, p_ci, pT)));
    }
    // ---- work buffers and state -------------------------------------------------------------
    const int64_t mm = std::max<int64_t>(m, 1);
    for (int i = 0; i < 2; ++i) {
      W.hx[i] = mem.alloc<T>(n); W.hy[i] = mem.alloc<T>(mm); W.wx[i] = mem.alloc<T>(n);
      W.u[i] = mem.alloc<T>(n);
      W.g[i] = P.qmode == cqp::kQSparse ? mem.alloc<T>(n) : nullptr;
    }
    W.ax = mem.alloc<T>(n); W.ay = mem.alloc<T>(mm); W.wy = mem.alloc<T>(mm); W.v = mem.alloc<T>(n); W.z = mem.alloc<T>(n);
    W.avx = o.update == 1 ? mem.alloc<T>(n) : nullptr;
    W.avy = o.update == 1 ? mem.alloc<T>(mm) : nullptr;
    W.mbuf = mem.alloc<T>(n);
    W.cb_acc = cb_n > 1 ? mem.alloc<T>(m) : nullptr;
    W.tcb_acc = P.tcb_n > 1 ? mem.alloc<T>(n) : nullptr;
    W.sd = mem.alloc<double>(n);
    n_roots = n_soc + n_rsoc + n_exp + n_pow;
    W.root = mem.alloc<float>(std::max<int64_t>(n_roots, 1));
    // team
    // batched instances are small: 64 threads per instance lets eight instances share an SM,
    // which hides more latency than one wide block per instance (measured on GB300:
    // 4,096 portfolio QPs 3.70 s at 512 threads, 2.34 s at 128, 2.22 s at 64)
    threads = o.threads > 0 ? o.threads : (batched ? 64 : 512);
    // problems with more than 4096 coordinates and rows spread over the whole GPU; smaller
    // ones run on one thread-block cluster (up to 16 SMs, cluster barriers and
    // distributed-shared-memory reductions), or on one block where no cluster fits
    const int64_t size = n + m;
    if (!batched) {
      if (bf && o.team != 0 && o.team != 1)
        fail(CQP_ERR_UNSUPPORTED, "matrix_bf16 runs on the whole-GPU team (team 0 or 1)");
      if (o.team == 1 || (o.team == 0 && (size > 4096 || bf))) team = cqp::kTeamGrid;
      else if (o.team == 2) team = cqp::kTeamCta;
      else team = cqp::kTeamCluster;
    }
    if (batched) {
      const int per = cqp::pdhg_blocks_per_sm<T>(threads);
      if (per < 1) fail(CQP_ERR_UNSUPPORTED, "solver kernel does not fit on an SM with this block size");
      blocks = (int)std::min<int64_t>((int64_t)nsm * per, bcount);
    } else if (team == cqp::kTeamGrid) {
      const int per = cqp::pdhg_blocks_per_sm<T>(threads);
      if (per < 1) fail(CQP_ERR_UNSUPPORTED, "solver kernel does not fit on an SM with this block size");
      const int want = o.blocks_per_sm > 0 ? std::min(o.blocks_per_sm, per) : 1;
      blocks = nsm * want;
    } else if (team == cqp::kTeamCluster) {
      blocks = cqp::pdhg_cluster_size<T>(threads);
      if (blocks < 2) {
        if (o.team == 3) fail(CQP_ERR_UNSUPPORTED, "no thread-block cluster of the solver kernel fits this device");
        team = cqp::kTeamCta;
        blocks = 1;
      }
    } else {
      blocks = 1;
    }
    // two buffers of block partials (the grid team alternates between them)
    W.part = mem.alloc<double>(2 * (int64_t)cqp::kMaxSlots * blocks);
    S = mem.alloc<cqp::State>(batched ? bcount : 1);
    if (batched) {
      // largest instances first (coordinates + rows), so the tail of the queue is short
      std::vector<int> ord(bcount);
      for (int64_t i = 0; i < bcount; ++i) ord[i] = (int)i;
      const int64_t* xo = B->x_off;
      const int64_t* ro = B->row_off;
      std::stable_sort(ord.begin(), ord.end(), [&](int a2, int b3) {
        return (xo[a2 + 1] - xo[a2]) + (ro[a2 + 1] - ro[a2]) > (xo[b3 + 1] - xo[b3]) + (ro[b3 + 1] - ro[b3]);
      });
      d_order = mem.alloc<int>(bcount);
      CK(cudaMemcpyAsync(d_order, ord.data(), bcount * sizeof(int), cudaMemcpyHostToDevice, st));
      d_queue = mem.alloc<unsigned>(1);
    }
    bar_count = mem.alloc<unsigned>(1);
    dev_err = mem.alloc<int>(1);
    kkt_out = mem.alloc<double>(8);
    tmp_x = mem.alloc<T>(n);
    tmp_y = mem.alloc<T>(mm);
    O.rho = o.rho; O.eps_min_in = o.eps_min_in; O.gamma_in = o.gamma_in; O.tol = o.tol;
    O.beta_s = o.beta_s; O.beta_n = o.beta_n; O.beta_a = o.beta_a;
    O.beta_I = o.beta_I; O.K_P = o.K_P; O.K_I = o.K_I; O.K_D = o.K_D;
    O.max_iter = o.max_iter; O.check_every = std::max(1, o.check_every); O.max_inner = std::max(1, o.max_inner);
    O.jacobi = o.jacobi; O.pid = o.pid; O.update = o.update; O.avg_epoch = std::max(1, o.avg_epoch);
    O.profile = o.profile;
    O.warm_roots = o.warm_roots;
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    setup_launches = g_launches - launches0;
  }

  int solve(const double* x0, const double* y0, double* xo, double* yo, int on_dev, cqp_result* res) override {
    if (batched) fail(CQP_ERR_UNSUPPORTED, "handle was made by cqp_setup_batch: use cqp_solve_batch");
    auto t0 = std::chrono::steady_clock::now();
    const int64_t mm = std::max<int64_t>(m, 1);
    Temp tmp(st);
    const double* dx0 = x0;
    const double* dy0 = y0;
    if (!on_dev) {
      if (x0) { double* d = tmp.alloc<double>(n); CK(cudaMemcpyAsync(d, x0, n * 8, cudaMemcpyHostToDevice, st)); dx0 = d; }
      if (y0 && m > 0) { double* d = tmp.alloc<double>(m); CK(cudaMemcpyAsync(d, y0, m * 8, cudaMemcpyHostToDevice, st)); dy0 = d; }
    }
    // scaled start: x~ = col x / beta_b (permuted), y~ = row y / beta_c
    count_launch(); k_perm_scale<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, perm, dx0, P.col, P.beta_b, W.hx[0]);
    if (m > 0) { count_launch(); k_perm_scale<T><<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, nullptr, dy0, P.row, P.beta_c, W.hy[0]); }
    count_launch(); k_copy_vec<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, W.hx[0], W.ax);
    count_launch(); k_copy_vec<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, W.hx[0], W.wx[0]);
    count_launch(); k_copy_vec<T><<<cqp::grid_for(mm), cqp::kSetupThreads, 0, st>>>(mm, W.hy[0], W.ay);
    count_launch(); k_copy_vec<T><<<cqp::grid_for(mm), cqp::kSetupThreads, 0, st>>>(mm, W.hy[0], W.wy);
    // no warm start for the cone roots of a new solve (NaN = none)
    CK(cudaMemsetAsync(W.root, 0xff, std::max<int64_t>(n_roots, 1) * sizeof(float), st));
    if (W.avx) {
      count_launch(); k_zero<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, W.avx);
      count_launch(); k_zero<T><<<cqp::grid_for(mm), cqp::kSetupThreads, 0, st>>>(mm, W.avy);
    }
    cqp::State hs;
    memset(&hs, 0, sizeof(hs));
    hs.omega = omega0;
    hs.eta = eta;
    hs.tau = eta / omega0;
    hs.sigma = eta * omega0;
    hs.eps_in = opt.eps0_in;
    CK(cudaMemcpyAsync(S, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
    if (k > 0 && x0) {
      double* t = tmp.alloc<double>(k);
      CK(cudaMemsetAsync(t, 0, k * sizeof(double), st));
      count_launch(); k_rx_partial<T><<<dim3(cqp::grid_for(n, 256, 256), (unsigned)k), 256, 0, st>>>(k, n, P.R, W.hx[0], t);
      count_launch(); k_state_set_th<<<1, 32, 0, st>>>(S, t, (int)k);
    }
    CK(cudaMemsetAsync(dev_err, 0, sizeof(int), st));
    long long per_launch = opt.launch_iters > 0 ? opt.launch_iters : (long long)O.check_every * (team == cqp::kTeamGrid ? 4 : 16);
    int launches = 0;
    int status = CQP_ITER_LIMIT;
    double kernel_ms = 0.0;
    cudaEvent_t ev0, ev1;
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
    cqp::State back;
    for (;;) {
      CK(cudaMemsetAsync(bar_count, 0, sizeof(unsigned), st));
      CK(cudaEventRecord(ev0, st));
      count_launch();
      CK(cqp::launch_pdhg<T>(args(per_launch), team, blocks, threads, st));
      CK(cudaEventRecord(ev1, st));
      ++launches;
      CK(cudaMemcpyAsync(&back, S, sizeof(back), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ev0, ev1));
        kernel_ms += ms;
      }
      if (back.err == cqp::kErrBarrier) { status = CQP_ERR_WAIT; break; }
      if (back.err == cqp::kErrNumeric) { status = CQP_ERR_NUMERICAL; break; }
      if (back.status == 1) { status = CQP_OK; break; }
      if (back.status == 2 || back.ktot >= O.max_iter) { status = CQP_ITER_LIMIT; break; }
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (opt.time_limit_s > 0 && el > opt.time_limit_s) { status = CQP_TIME_LIMIT; break; }
    }
    // final candidate (average for the averaged variant), unscaled and un-permuted
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    const T* fx = opt.update == 1 ? W.avx : W.wx[back.wb];
    const T* fy = opt.update == 1 ? W.avy : W.wy;
    double* ox = tmp.alloc<double>(n);
    double* oy = tmp.alloc<double>(mm);
    count_launch(); k_unscale_unperm<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, perm, fx, P.col, P.beta_b, ox);
    if (m > 0) { count_launch(); k_unscale_unperm<T><<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, nullptr, fy, P.row, P.beta_c, oy); }
    if (xo) CK(cudaMemcpyAsync(xo, ox, n * 8, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (yo && m > 0) CK(cudaMemcpyAsync(yo, oy, m * 8, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (res) {
      memset(res, 0, sizeof(*res));
      res->status = status;
      res->iters = back.ktot;
      res->restarts = back.restarts;
      res->inner_total = back.inner_total;
      res->kernel_launches = launches;
      res->kkt.eps_p = back.kkt[0]; res->kkt.eps_d = back.kkt[1]; res->kkt.eps_g = back.kkt[2];
      res->kkt.rel_kkt = back.kkt[3]; res->kkt.pobj = back.kkt[4]; res->kkt.dobj = back.kkt[5];
      res->kkt.norm_res_p = back.kkt[6]; res->kkt.norm_res_d = back.kkt[7];
      res->eta = eta;
      res->norm_A = normA;
      res->omega = back.omega;
      res->setup_ms = setup_ms;
      res->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      for (int i = 0; i < 16; ++i) res->phase_ms[i] = back.prof[i] * 1e-6;
      res->kernel_ms = kernel_ms;
      res->setup_launches = setup_launches;
    }
    return status;
  }

  int solve_batch(const double* x0, const double* y0, double* xo, double* yo, int on_dev, cqp_instance_result* per,
                  cqp_result* res) override {
    if (!batched) fail(CQP_ERR_UNSUPPORTED, "handle was made by cqp_setup: use cqp_solve");
    auto t0 = std::chrono::steady_clock::now();
    const int64_t mm = std::max<int64_t>(m, 1);
    Temp tmp(st);
    const double* dx0 = x0;
    const double* dy0 = y0;
    if (!on_dev) {
      if (x0) { double* d = tmp.alloc<double>(n); CK(cudaMemcpyAsync(d, x0, n * 8, cudaMemcpyHostToDevice, st)); dx0 = d; }
      if (y0 && m > 0) { double* d = tmp.alloc<double>(m); CK(cudaMemcpyAsync(d, y0, m * 8, cudaMemcpyHostToDevice, st)); dy0 = d; }
    }
    if (m == 0) dy0 = nullptr;
    double* ox = tmp.alloc<double>(n);
    double* oy = tmp.alloc<double>(mm);
    CK(cudaMemsetAsync(W.root, 0xff, std::max<int64_t>(n_roots, 1) * sizeof(float), st));
    CK(cudaMemsetAsync(d_queue, 0, sizeof(unsigned), st));
    std::vector<cqp::State> hs(bcount);
    for (int64_t i = 0; i < bcount; ++i) {
      cqp::State& z = hs[i];
      memset(&z, 0, sizeof(z));
      z.omega = h_om[i];
      z.eta = h_eta[i];
      z.tau = h_eta[i] / h_om[i];
      z.sigma = h_eta[i] * h_om[i];
      z.eps_in = opt.eps0_in;
    }
    CK(cudaMemcpyAsync(S, hs.data(), bcount * sizeof(cqp::State), cudaMemcpyHostToDevice, st));
    cqp::BatchArgs ba{};
    ba.count = bcount;
    ba.order = d_order;
    ba.queue = d_queue;
    ba.own = d_own;
    ba.beta_b = d_bb; ba.beta_c = d_bc; ba.norm_b = d_nb; ba.norm_c = d_nc;
    ba.rank = P.d_scale > 0.0 ? d_rank : nullptr;   // per-instance width needs D = d I (D's stride is the full rank)
    ba.S = S;
    ba.perm = perm;
    ba.x0 = dx0; ba.y0 = dy0;
    ba.x_out = ox; ba.y_out = oy;
    ba.chunk = (long long)O.check_every * 16;
    ba.time_limit_ns = opt.time_limit_s > 0 ? (unsigned long long)(opt.time_limit_s * 1e9) : 0ull;
    cudaEvent_t ev0, ev1;
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
    CK(cudaEventRecord(ev0, st));
    count_launch();
    CK(cqp::launch_pdhg_batch<T>(args(O.max_iter), ba, blocks, threads, st));
    CK(cudaEventRecord(ev1, st));
    std::vector<cqp::State> back(bcount);
    CK(cudaMemcpyAsync(back.data(), S, bcount * sizeof(cqp::State), cudaMemcpyDeviceToHost, st));
    if (xo) CK(cudaMemcpyAsync(xo, ox, n * 8, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (yo && m > 0) CK(cudaMemcpyAsync(yo, oy, m * 8, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev0, ev1));
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    auto rank = [](int stt) { return stt == CQP_OK ? 0 : stt == CQP_ITER_LIMIT ? 1 : stt == CQP_TIME_LIMIT ? 2 : 3; };
    int worst = CQP_OK;
    int64_t max_it = 0, rs = 0, inn = 0, worst_i = 0;
    for (int64_t i = 0; i < bcount; ++i) {
      const cqp::State& b2 = back[i];
      int stt = CQP_ITER_LIMIT;
      if (b2.err == cqp::kErrNumeric) stt = CQP_ERR_NUMERICAL;
      else if (b2.status == 1) stt = CQP_OK;
      else if (b2.status == 3) stt = CQP_TIME_LIMIT;
      if (rank(stt) > rank(worst)) worst = stt;
      max_it = std::max<int64_t>(max_it, b2.ktot);
      rs += b2.restarts;
      inn += b2.inner_total;
      if (b2.kkt[3] > back[worst_i].kkt[3]) worst_i = i;
      if (per) {
        cqp_instance_result& r = per[i];
        r.status = stt;
        r.iters = b2.ktot;
        r.restarts = b2.restarts;
        r.inner_total = b2.inner_total;
        r.kkt.eps_p = b2.kkt[0]; r.kkt.eps_d = b2.kkt[1]; r.kkt.eps_g = b2.kkt[2]; r.kkt.rel_kkt = b2.kkt[3];
        r.kkt.pobj = b2.kkt[4]; r.kkt.dobj = b2.kkt[5]; r.kkt.norm_res_p = b2.kkt[6]; r.kkt.norm_res_d = b2.kkt[7];
      }
    }
    if (res) {
      memset(res, 0, sizeof(*res));
      const cqp::State& b2 = back[worst_i];
      res->status = worst;
      res->iters = max_it;
      res->restarts = rs;
      res->inner_total = inn;
      res->kernel_launches = 1;
      res->kkt.eps_p = b2.kkt[0]; res->kkt.eps_d = b2.kkt[1]; res->kkt.eps_g = b2.kkt[2]; res->kkt.rel_kkt = b2.kkt[3];
      res->kkt.pobj = b2.kkt[4]; res->kkt.dobj = b2.kkt[5]; res->kkt.norm_res_p = b2.kkt[6]; res->kkt.norm_res_d = b2.kkt[7];
      res->eta = eta;
      res->norm_A = normA;
      res->omega = b2.omega;
      res->setup_ms = setup_ms;
      res->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      res->kernel_ms = ms;
      res->setup_launches = setup_launches;
    }
    return worst;
  }

  int kkt(const double* x, const double* y, int on_dev, cqp_kkt_report* rep) override {
    if (batched) fail(CQP_ERR_UNSUPPORTED, "cqp_kkt on a batch handle: each instance reports its KKT in cqp_solve_batch");
    const int64_t mm = std::max<int64_t>(m, 1);
    Temp tmp(st);
    const double* dx = x;
    const double* dy = y;
    if (!on_dev) {
      double* d = tmp.alloc<double>(n);
      CK(cudaMemcpyAsync(d, x, n * 8, cudaMemcpyHostToDevice, st));
      dx = d;
      double* e = tmp.alloc<double>(mm);
      if (m > 0) CK(cudaMemcpyAsync(e, y, m * 8, cudaMemcpyHostToDevice, st));
      dy = e;
    }
    count_launch(); k_perm_scale<T><<<cqp::grid_for(n), cqp::kSetupThreads, 0, st>>>(n, perm, dx, P.col, P.beta_b, tmp_x);
    if (m > 0) { count_launch(); k_perm_scale<T><<<cqp::grid_for(m), cqp::kSetupThreads, 0, st>>>(m, nullptr, dy, P.row, P.beta_c, tmp_y); }
    CK(cudaMemsetAsync(bar_count, 0, sizeof(unsigned), st));
    CK(cudaMemsetAsync(dev_err, 0, sizeof(int), st));
    count_launch();
    CK(cqp::launch_kkt<T>(args(0), tmp_x, tmp_y, kkt_out, team, blocks, threads, st));
    double h[8];
    CK(cudaMemcpyAsync(h, kkt_out, sizeof(h), cudaMemcpyDeviceToHost, st));
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr) return CQP_ERR_WAIT;
    rep->eps_p = h[0]; rep->eps_d = h[1]; rep->eps_g = h[2]; rep->rel_kkt = h[3];
    rep->pobj = h[4]; rep->dobj = h[5]; rep->norm_res_p = h[6]; rep->norm_res_d = h[7];
    return std::isfinite(h[3]) ? CQP_OK : CQP_ERR_NUMERICAL;
  }
};

template <typename F>
int guarded(F f) {
  try {
    return f();
  } catch (const Fail& e) {
    return e.code;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return CQP_ERR_CUDA;
  } catch (...) {
    g_last_error = "unknown error";
    return CQP_ERR_CUDA;
  }
}

}  // namespace

namespace cqp {
// error text and launch count for entry points defined in other translation
// units of this library (they share this thread's cqp_last_error and counter)
void record_error(const std::string& msg) { g_last_error = msg; }
void record_launches(long long k) { g_launches += k; }
}  // namespace cqp

struct cqp_handle {
  HandleBase* impl;
};

extern "C" {

int cqp_default_options(cqp_options* o) {
  if (!o) return CQP_ERR_INVALID;
  memset(o, 0, sizeof(*o));
  o->precision = 0;
  o->update = 0;
  o->rho = 1.0;
  o->ruiz_iters = 10;
  o->pc_alpha = 1.0;
  o->bound_obj = 1;
  o->eps0_in = 1e-3;
  o->gamma_in = 5e-4;
  o->eps_min_in = 1e-9;
  o->jacobi = 1;
  o->max_inner = 1000;
  o->force_inner = 0;
  o->beta_s = 0.2;
  o->beta_n = 0.8;
  o->beta_a = 0.36;
  o->beta_I = 0.3;
  o->K_P = 0.99;
  o->K_I = 0.01;
  o->K_D = 0.0;
  o->pid = 1;
  o->avg_epoch = 64;
  o->tol = 1e-4;
  o->max_iter = 100000;
  o->check_every = 64;
  o->time_limit_s = 0.0;
  o->power_iters = 200;
  o->power_tol = 1e-6;
  o->step_factor = 0.998;
  o->warm_roots = 1;
  o->col_blocks = 0;
  o->matrix_bf16 = 0;
  return CQP_OK;
}

int cqp_setup(const cqp_csr* A, const cqp_qop* Q, const double* c, const double* b, const cqp_cones* K,
              const cqp_options* opt, cqp_handle** out) {
  if (!out) return CQP_ERR_INVALID;
  *out = nullptr;
  if (!A || !K || !c) return CQP_ERR_INVALID;
  cqp_options o;
  if (opt) o = *opt; else cqp_default_options(&o);
  return guarded([&]() {
    HandleBase* h = nullptr;
    if (o.precision == 1) {
      auto* hh = new Handle<double>();
      try { hh->setup(A, Q, c, b, K, o); } catch (...) { delete hh; throw; }
      h = hh;
    } else {
      auto* hh = new Handle<float>();
      try { hh->setup(A, Q, c, b, K, o); } catch (...) { delete hh; throw; }
      h = hh;
    }
    *out = new cqp_handle{h};
    return CQP_OK;
  });
}

int cqp_setup_general(const cqp_csr* A, const cqp_qop* Q, const double* c, const cqp_bounds* bounds,
                      const cqp_cones* K, const cqp_options* opt, cqp_handle** out) {
  if (!out) return CQP_ERR_INVALID;
  *out = nullptr;
  if (!A || !K || !c || !bounds) return CQP_ERR_INVALID;
  cqp_options o;
  if (opt) o = *opt; else cqp_default_options(&o);
  return guarded([&]() {
    HandleBase* h = nullptr;
    if (o.precision == 1) {
      auto* hh = new Handle<double>();
      try { hh->setup(A, Q, c, nullptr, K, o, nullptr, bounds); } catch (...) { delete hh; throw; }
      h = hh;
    } else {
      auto* hh = new Handle<float>();
      try { hh->setup(A, Q, c, nullptr, K, o, nullptr, bounds); } catch (...) { delete hh; throw; }
      h = hh;
    }
    *out = new cqp_handle{h};
    return CQP_OK;
  });
}

int cqp_setup_batch(const cqp_csr* A, const cqp_qop* Q, const double* c, const double* b, const cqp_cones* K,
                    const cqp_batch* B, const cqp_options* opt, cqp_handle** out) {
  if (!out) return CQP_ERR_INVALID;
  *out = nullptr;
  if (!A || !K || !c || !B) return CQP_ERR_INVALID;
  cqp_options o;
  if (opt) o = *opt; else cqp_default_options(&o);
  return guarded([&]() {
    HandleBase* h = nullptr;
    if (o.precision == 1) {
      auto* hh = new Handle<double>();
      try { hh->setup(A, Q, c, b, K, o, B); } catch (...) { delete hh; throw; }
      h = hh;
    } else {
      auto* hh = new Handle<float>();
      try { hh->setup(A, Q, c, b, K, o, B); } catch (...) { delete hh; throw; }
      h = hh;
    }
    *out = new cqp_handle{h};
    return CQP_OK;
  });
}

int cqp_solve_batch(cqp_handle* h, const double* x0, const double* y0, double* x_out, double* y_out, int32_t on_device,
                    cqp_instance_result* per_instance, cqp_result* res) {
  if (!h || !h->impl) return CQP_ERR_INVALID;
  return guarded([&]() { return h->impl->solve_batch(x0, y0, x_out, y_out, on_device, per_instance, res); });
}

int cqp_solve(cqp_handle* h, const double* x0, const double* y0, double* x_out, double* y_out, int32_t on_device,
              cqp_result* res) {
  if (!h || !h->impl) return CQP_ERR_INVALID;
  return guarded([&]() { return h->impl->solve(x0, y0, x_out, y_out, on_device, res); });
}

int cqp_kkt(cqp_handle* h, const double* x, const double* y, int32_t on_device, cqp_kkt_report* rep) {
  if (!h || !h->impl || !x || !rep) return CQP_ERR_INVALID;
  return guarded([&]() { return h->impl->kkt(x, y, on_device, rep); });
}

void cqp_free(cqp_handle* h) {
  if (!h) return;
  delete h->impl;
  delete h;
}

const char* cqp_status_string(int s) {
  switch (s) {
    case CQP_OK: return "converged";
    case CQP_ITER_LIMIT: return "iteration limit";
    case CQP_TIME_LIMIT: return "time limit";
    case CQP_ERR_INVALID: return "invalid input";
    case CQP_ERR_CUDA: return "CUDA error";
    case CQP_ERR_OOM: return "out of device memory";
    case CQP_ERR_NUMERICAL: return "non-finite value in a reduction";
    case CQP_ERR_WAIT: return "a bounded device-side wait expired";
    case CQP_ERR_UNSUPPORTED: return "unsupported option combination";
    default: return "unknown status";
  }
}

const char* cqp_last_error(void) { return g_last_error.c_str(); }

long long cqp_kernel_launches(void) { return g_launches; }

int cqp_spmv(int32_t precision, int64_t nrows, int64_t ncols, const int32_t* rowptr, const int32_t* colind,
             const void* val, const void* x, void* y, int32_t threads_per_row, void* stream) {
  if (nrows < 0 || ncols < 0 || !rowptr || (nrows > 0 && (!colind || !val || !x || !y))) return CQP_ERR_INVALID;
  int tpr = threads_per_row;
  if (tpr != -1 && tpr != 0 && tpr != 1 && tpr != 2 && tpr != 4 && tpr != 8 && tpr != 16 && tpr != 32)
    return CQP_ERR_INVALID;
  const bool batched_rows = tpr == -1;
  return guarded([&]() {
    if (batched_rows) {
      tpr = cqp::kRowsBatched;
    } else if (tpr == 0) {
      int32_t last = 0;
      CK(cudaMemcpy(&last, rowptr + nrows, sizeof(int32_t), cudaMemcpyDeviceToHost));
      tpr = pow2_tpr(nrows > 0 ? (double)last / (double)nrows : 1.0);
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (nrows == 0) return CQP_OK;
    count_launch();
    if (precision == 1)
      CK(cqp::launch_spmv<double>(nrows, rowptr, colind, (const double*)val, (const double*)x, (double*)y, tpr, st));
    else if (precision == 2)
      CK(cqp::launch_spmv_bf16<float>(nrows, rowptr, colind, (const __nv_bfloat16*)val, (const float*)x, (float*)y, tpr,
                                      st));
    else
      CK(cqp::launch_spmv<float>(nrows, rowptr, colind, (const float*)val, (const float*)x, (float*)y, tpr, st));
    CK(cudaStreamSynchronize(st));
    return CQP_OK;
  });
}

int cqp_project(int32_t precision, int64_t n, const cqp_cones* K, const void* r, const void* m, void* out, void* stream) {
  if (!K || !r || !out || n < 0) return CQP_ERR_INVALID;
  return guarded([&]() {
    cudaStream_t st = (cudaStream_t)stream;
    if (K->nblocks == 0) return CQP_OK;
    count_launch();
    if (precision == 1)
      CK(cqp::launch_project<double>(K->nblocks, K->type, K->start, K->dim, K->alpha, (const double*)r,
                                     (const double*)m, (double*)out, n, st));
    else
      CK(cqp::launch_project<float>(K->nblocks, K->type, K->start, K->dim, K->alpha, (const float*)r,
                                    (const float*)m, (float*)out, n, st));
    CK(cudaStreamSynchronize(st));
    return CQP_OK;
  });
}

}  // extern "C"
