// Specialised GLM kernels, FP32 degree 3 (see dg_fast_impl.cuh).
#define DG_FAST_T float
#define DG_FAST_DEG 3
#define DG_FAST_CONST 1
#include "dg_fast_impl.cuh"
