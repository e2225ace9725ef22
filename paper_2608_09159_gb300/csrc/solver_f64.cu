// FP64 instantiation of the solver, KKT and kernel-level entry points.
#define CQP_T double
#include "kernels.inc"
