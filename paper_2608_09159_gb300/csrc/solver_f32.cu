// FP32 instantiation of the solver, KKT and kernel-level entry points.
#define CQP_T float
#include "kernels.inc"

namespace cqp {
template cudaError_t launch_spmv_bf16<float>(int64_t, const int*, const int*, const __nv_bfloat16*, const float*, float*,
                                            int, cudaStream_t, int);
}  // namespace cqp
