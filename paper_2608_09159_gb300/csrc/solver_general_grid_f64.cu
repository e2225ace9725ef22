// FP64 instantiation of the whole-GPU general-form solver kernel.
#define CQP_T double
#define CQP_GRID_PART
#include "general.inc"
