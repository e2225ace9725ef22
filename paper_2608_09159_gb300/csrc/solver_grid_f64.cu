// FP64 instantiation of the whole-GPU solver and KKT kernels (equality form).
#define CQP_T double
#define CQP_GRID_PART
#include "kernels.inc"
