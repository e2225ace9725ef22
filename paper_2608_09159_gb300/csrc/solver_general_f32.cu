// FP32 instantiation of the general-form solver kernels.
#define CQP_T float
#include "general.inc"
