// FP64 instantiation of the general-form solver kernels.
#define CQP_T double
#include "general.inc"
