// FP32 instantiation of the solver, KKT and kernel-level entry points.
#define CQP_T float
#include "kernels.inc"
