// Specialised GLM kernels, FP64 degree 2 (see dg_fast_impl.cuh).
#define DG_FAST_T double
#define DG_FAST_DEG 2
#define DG_FAST_CONST 1
#include "dg_fast_impl.cuh"
