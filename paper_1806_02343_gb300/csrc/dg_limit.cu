// Limiters of Sec. 4.2 (TVB-characteristic, LDF slope fix) and Sec. 4.3 (positivity).
#include "dg_limit.cuh"

namespace dgmhd {

int run_limiter(Ctx& c, void* w, double* wmean, uint8_t* troubled, cudaStream_t st) {
  (void)c; (void)w; (void)wmean; (void)troubled; (void)st;
  return DG_E_UNSUPPORTED;
}

}  // namespace dgmhd
