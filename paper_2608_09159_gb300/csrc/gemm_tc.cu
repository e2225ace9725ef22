// Warm-start GEMM on the fifth-generation tensor cores of sm_103a:
//     C = A B'    A: M x K row-major, B: N x K row-major (both K-contiguous), BF16,
// FP32 accumulation in tensor memory, with the epilogues of cqp_gemm_bf16 (0: FP32, 1: FP32 plus
// bias, 2: BF16 ReLU(result + bias), 4: BF16).  Output tiles are 128 x 256; a persistent grid of
// one 192-thread block per SM walks them (tile t = blockIdx.x, + gridDim.x, ...):
//   - warp 0 streams 64-wide K slices of A (128 x 64) and B (256 x 64) into shared memory with
//     tiled tensor copies (cp.async.bulk.tensor, 128-byte swizzle, four stages), each stage's
//     arrival counted in bytes on its "full" mbarrier;
//   - warp 1 issues tcgen05.mma (M 128, N 256, K 16 per instruction, four per stage) into one of two
//     128 x 256 FP32 accumulators in tensor memory (512 columns), commits every stage to its "empty"
//     mbarrier, which hands the stage back to warp 0, and each finished tile to "acc_full";
//   - warps 2-5 drain the other accumulator meanwhile (tcgen05.ld), apply the epilogue and write C
//     by tiled tensor stores from swizzled staging buffers.
// Every wait on an mbarrier is bounded (one second): on expiry the kernel records an error and the
// block skips to its exit, where it waits for its copies in flight and frees the tensor memory.
//
// Operand descriptors follow the tcgen05 shared-memory descriptor of the PTX ISA (start address,
// leading and stride byte offsets in 16-byte units, the fixed version bits 46-48 = 0b001, the
// swizzle mode in bits 61-63) and its instruction descriptor for kind::f16 (accumulator format in
// bits 4-5, A and B formats in bits 7-9 and 10-12, K-major bits 15 and 16, N / 8 in bits 17-22,
// M / 16 in bits 24-28).  A 128-byte-swizzled K-major tile stores each row's 64 BF16 values
// (128 bytes) in place, rows 128 bytes apart, groups of 8 rows (the swizzle atom, 1024 bytes)
// 1024 bytes apart: stride byte offset 1024; the K step of 16 values inside the atom advances the
// start address by 32 bytes.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "cqp.h"
#include "cqp_mlp.h"

namespace cqp {
void record_error(const std::string& msg);
void record_launches(long long k);
}  // namespace cqp

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr uint32_t kStageA = BM * BK * 2;                     // 16 KB
constexpr uint32_t kStageB = BN * BK * 2;                     // 32 KB
constexpr uint32_t kTiles = STAGES * (kStageA + kStageB);     // 192 KB
constexpr unsigned long long kWaitNs = 1000000000ull;         // bounded mbarrier waits: one second


// ---- descriptors (host and device, so the host tests can check the encodings) -------------
__host__ __device__ inline uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(layout & 7u) << 61;
  return d;
}
__host__ __device__ inline uint32_t instr_desc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
constexpr uint32_t kSwizzle128B = 2;

// ---- PTX helpers ---------------------------------------------------------------------------
__device__ inline uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ inline void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// true once the phase with the given parity has completed; false if it has not within kWaitNs
__device__ inline bool mbar_wait(uint64_t* b, uint32_t parity) {
  const uint32_t a = su32(b);
  const unsigned long long t0 = global_ns();
  for (long long i = 0; i < (1ll << 30); ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 63) == 63 && global_ns() - t0 > kWaitNs) break;
  }
  return false;
}
__device__ inline void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ inline void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          su32(dst)),
      "l"(map), "r"(su32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ inline void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ inline void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's accumulator lane
__device__ inline void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- the kernel -----------------------------------------------------------------------------
// Warp 0 (lane 0) streams K slices of every tile the CTA owns through the ring; warp 1 (lane 0)
// issues the MMAs of tile j into accumulator j % 2 (tensor-memory columns 256 (j % 2) ..) once the
// epilogue has drained tile j - 2 from it; warps 2-5 drain accumulator j % 2 of tile j (warp w reads
// lanes 32 (w % 4) ..) while the MMAs of tile j + 1 run.  Barriers: full / empty per stage as above,
// acc_full[2] (committed by the MMA thread), acc_empty[2] (one arrival per epilogue warp), done
// (the MMA thread's last commit, awaited before the tensor memory is freed).
//
// The epilogue writes C through shared memory: each warp converts 128 bytes of each of its 32 rows
// (64 BF16 or 32 FP32 columns) into one of its two 4 KB staging buffers, laid out as the tiled
// tensor copy's 128-byte swizzle expects (16-byte chunk c of row r at chunk c ^ (r mod 8), which
// also spreads the warp's 16-byte writes over all banks), and lane 0 stores the 32-row box with
// one tiled tensor store (rows at or beyond M are clipped by the copy).  A buffer is refilled only
// after the store issued from it two steps earlier has read it.
constexpr int PTHREADS = 192;
constexpr uint32_t kPTmemCols = 512;
constexpr uint32_t kOutBuf = 4096;                              // 32 rows x 128 bytes
constexpr uint32_t kOutStage = 4 * 2 * kOutBuf;                 // 4 epilogue warps, 2 buffers each
constexpr uint32_t kPSmem = kTiles + kOutStage + 1024 + 256;   // + alignment of the tiles + barriers
static_assert(kPSmem + 64 <= 232448, "shared memory of the persistent GEMM");

__device__ inline void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map),
               "r"(su32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ inline void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ inline void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ inline void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 64 consecutive FP32 columns of this thread's accumulator lane
__device__ inline void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool kBf16Out>
__global__ void __launch_bounds__(PTHREADS, 1)
    k_gemm_tc_persistent(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                         const __grid_constant__ CUtensorMap tmC, int64_t M, int64_t N, int64_t K,
                         const float* __restrict__ bias, int epilogue, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* tiles = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* out_stage = tiles + kTiles;
  uint64_t* full = (uint64_t*)(out_stage + kOutStage);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  __shared__ volatile int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntn = N / BN, ntiles = ((M + BM - 1) / BM) * ntn;
  const int KT = (int)(K / BK);

  if (threadIdx.x == 0) {
    failed = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(acc_full + a, 1);
      mbar_init(acc_empty + a, 4);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(kPTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int64_t issued = 0;   // K slices whose copies lane 0 of warp 0 has started
  if (warp == 0) {
    if (lane == 0) {
      int64_t it = 0;
      for (int64_t t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
        const int m0 = (int)((t / ntn) * BM), n0 = (int)((t % ntn) * BN);
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int s = (int)(it % STAGES);
          if (it >= STAGES && !mbar_wait(empty + s, (uint32_t)((it / STAGES) - 1) & 1)) {
            failed = 1;
            break;
          }
          mbar_expect_tx(full + s, kStageA + kStageB);
          tma_load_2d(tiles + s * kStageA, &tmA, full + s, kt * BK, m0);
          tma_load_2d(tiles + STAGES * kStageA + s * kStageB, &tmB, full + s, kt * BK, n0);
          issued = it + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc_bf16(BM, BN);
      int64_t it = 0, j = 0;
      for (int64_t t = blockIdx.x; t < ntiles && !failed; t += gridDim.x, ++j) {
        const uint32_t a = (uint32_t)(j & 1);
        if (j >= 2 && !mbar_wait(acc_empty + a, (uint32_t)((j / 2) - 1) & 1)) {
          failed = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + a * BN;
        bool ok = true;
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int s = (int)(it % STAGES);
          if (!mbar_wait(full + s, (uint32_t)(it / STAGES) & 1)) {
            failed = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = su32(tiles + s * kStageA);
          const uint32_t b_base = su32(tiles + STAGES * kStageA + s * kStageB);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t ad = smem_desc(a_base + kk * 32, 16, 1024, kSwizzle128B);
            const uint64_t bd = smem_desc(b_base + kk * 32, 16, 1024, kSwizzle128B);
            umma_bf16(d, ad, bd, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
          }
          umma_commit(empty + s);
        }
        if (!ok) break;
        umma_commit(acc_full + a);
      }
      umma_commit(done);
    }
  } else {
    constexpr int CPS = kBf16Out ? 64 : 32;   // columns per 128-byte row segment
    const int q = warp & 3;                    // the lane quarter of tensor memory this warp may read
    unsigned char* bufs = out_stage + (uint32_t)(warp - 2) * 2 * kOutBuf;
    int sb = 0;
    int64_t j = 0;
    for (int64_t t = blockIdx.x; t < ntiles && !failed; t += gridDim.x, ++j) {
      const uint32_t a = (uint32_t)(j & 1);
      const bool ready = mbar_wait(acc_full + a, (uint32_t)(j / 2) & 1);
      tc_fence_after();
      if (!ready) {
        failed = 1;
        break;
      }
      const int m0 = (int)((t / ntn) * BM), n0 = (int)((t % ntn) * BN);
      const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16) + a * BN;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += CPS) {
        float v[CPS];
        if constexpr (kBf16Out) {
          tmem_ld64(lane_addr + (uint32_t)c0, v);
        } else {
          tmem_ld32(lane_addr + (uint32_t)c0, v);
        }
        if (c0 + CPS == BN) {   // the accumulator is read: hand it back to the MMA thread
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acc_empty + a);
        }
        if (epilogue == 1 || epilogue == 2) {
          const float4* b4 = (const float4*)(bias + n0 + c0);
#pragma unroll
          for (int i = 0; i < CPS / 4; ++i) {
            const float4 bb = __ldg(b4 + i);
            v[4 * i] += bb.x;
            v[4 * i + 1] += bb.y;
            v[4 * i + 2] += bb.z;
            v[4 * i + 3] += bb.w;
          }
        }
        if (epilogue == 2) {
#pragma unroll
          for (int i = 0; i < CPS; ++i) v[i] = fmaxf(v[i], 0.0f);
        }
        unsigned char* buf = bufs + sb * kOutBuf;
        if (lane == 0) bulk_wait_read1();   // the store issued from this buffer two steps ago has read it
        __syncwarp();
        unsigned char* row = buf + lane * 128;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          uint4 w;
          if constexpr (kBf16Out) {
            __align__(16) __nv_bfloat162 h[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[8 * c + 2 * i], v[8 * c + 2 * i + 1]);
            w = *(const uint4*)h;
          } else {
            w = make_uint4(__float_as_uint(v[4 * c]), __float_as_uint(v[4 * c + 1]), __float_as_uint(v[4 * c + 2]),
                           __float_as_uint(v[4 * c + 3]));
          }
          *(uint4*)(row + ((c ^ (lane & 7)) << 4)) = w;
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          tma_store_2d(&tmC, buf, n0 + c0, m0 + q * 32);
          bulk_commit();
        }
        sb ^= 1;
      }
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0 && failed) {
    for (int64_t it = issued - 1; it >= 0 && it >= issued - STAGES; --it)
      mbar_wait(full + it % STAGES, (uint32_t)(it / STAGES) & 1);
  }
  if (warp == 1) {
    // every MMA issued has completed before the accumulators are freed
    mbar_wait(done, 0);
    tc_fence_after();
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPTmemCols) : "memory");
  }
  if (threadIdx.x == 0 && failed) atomicExch(err, 1);
}

// ---- host side -------------------------------------------------------------------------------
// cuTensorMapEncodeTiled, taken from the driver at run time (no link-time dependence on libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
std::once_flag g_encode_once;
int* g_err[64] = {};
std::mutex g_err_mu;
std::atomic<long long> g_tc_launches{0};

bool encode_2d(CUtensorMap* map, const void* base, CUtensorMapDataType type, uint64_t inner, uint64_t outer,
               uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return g_encode(map, type, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

namespace cqp {

// 1 if the tensor-core path takes this GEMM (then *rc holds its status), 0 if the caller should use
// its general kernel.  The path needs op(A) = A (row-major M x K), op(B) = B' with B row-major N x K,
// N a multiple of 256, K a multiple of 64, 16-byte aligned rows and pointers, epilogue 0, 1, 2 or 4.
int gemm_tc_try(int32_t trans_a, int32_t trans_b, int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda,
                const uint16_t* B, int64_t ldb, void* C, int64_t ldc, const float* bias, int32_t epilogue,
                cudaStream_t st, int* rc) {
  if (trans_a || !trans_b || epilogue == 3 || M <= 0 || N % BN != 0 || K % BK != 0 || K == 0) return 0;
  if (lda < K || ldb < K || ldc < N) return 0;
  if (lda % 8 || ldb % 8 || ldc % 8 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((uintptr_t)C & 15)) return 0;
  if ((epilogue == 1 || epilogue == 2) && (!bias || ((uintptr_t)bias & 15))) return 0;
  if (M > (int64_t)INT32_MAX || N > (int64_t)INT32_MAX || K > (int64_t)INT32_MAX) return 0;
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (EncodeTiledFn)fn;
  });
  if (!g_encode) return 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  int* err = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_err_mu);
    if (!g_err[dev]) {
      if (cudaMalloc(&g_err[dev], sizeof(int)) != cudaSuccess) return 0;
      cudaMemset(g_err[dev], 0, sizeof(int));
    }
    err = g_err[dev];
  }
  CUtensorMap ta, tb;
  const CUtensorMapDataType bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (!encode_2d(&ta, A, bf, (uint64_t)K, (uint64_t)M, (uint64_t)lda * 2, BK, BM)) return 0;
  if (!encode_2d(&tb, B, bf, (uint64_t)K, (uint64_t)N, (uint64_t)ldb * 2, BK, BN)) return 0;
  const bool bf_out = epilogue == 2 || epilogue == 4;
  static std::once_flag attr_once;
  static int nsm[64] = {};
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(k_gemm_tc_persistent<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPSmem);
    cudaFuncSetAttribute(k_gemm_tc_persistent<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPSmem);
  });
  if (!nsm[dev] && cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const int64_t ntiles = (N / BN) * ((M + BM - 1) / BM);
  // C through tiled tensor stores: 128-byte row segments (64 BF16 or 32 FP32 columns) x 32 rows
  CUtensorMap tc;
  if (!encode_2d(&tc, C, bf_out ? bf : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (uint64_t)N, (uint64_t)M,
                 (uint64_t)ldc * (bf_out ? 2 : 4), bf_out ? 64 : 32, 32))
    return 0;
  const unsigned blocks = (unsigned)std::min<int64_t>(ntiles, nsm[dev]);
  if (bf_out)
    k_gemm_tc_persistent<true><<<blocks, PTHREADS, kPSmem, st>>>(ta, tb, tc, M, N, K, bias, epilogue, err);
  else
    k_gemm_tc_persistent<false><<<blocks, PTHREADS, kPSmem, st>>>(ta, tb, tc, M, N, K, bias, epilogue, err);
  record_launches(1);
  g_tc_launches.fetch_add(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    record_error(std::string("k_gemm_tc_persistent: ") + cudaGetErrorString(e));
    *rc = CQP_ERR_CUDA;
    return 1;
  }
  *rc = CQP_OK;
  return 1;
}

// status of the tensor-core GEMMs issued so far on the current device: CQP_ERR_WAIT if one of
// their bounded waits expired (the flag is cleared by the read)
int gemm_tc_status(cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || !g_err[dev]) return CQP_OK;
  int h = 0;
  if (cudaMemcpyAsync(&h, g_err[dev], sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CQP_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CQP_ERR_CUDA;
  if (h) {
    cudaMemsetAsync(g_err[dev], 0, sizeof(int), st);
    return CQP_ERR_WAIT;
  }
  return CQP_OK;
}

}  // namespace cqp

extern "C" uint64_t cqp_umma_smem_desc(uint32_t smem_addr, uint32_t lbo_bytes, uint32_t sbo_bytes, int32_t swizzle) {
  return smem_desc(smem_addr, lbo_bytes, sbo_bytes, (uint32_t)swizzle);
}

extern "C" uint32_t cqp_umma_instr_desc_bf16(int32_t m, int32_t n) { return instr_desc_bf16(m, n); }

extern "C" long long cqp_gemm_tc_launches(void) { return g_tc_launches.load(); }
