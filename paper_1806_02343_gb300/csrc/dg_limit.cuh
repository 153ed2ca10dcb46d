// Limiters of Sec. 4.2 (TVB-characteristic, LDF slope fix) and Sec. 4.3 (positivity).
#pragma once
#include "dg_ctx.h"

namespace dgmhd {

// Builds the limiter's basis tables (kernel parameters) into c.lim.
int upload_limiter_tables(Ctx& c);

// Applies the enabled limiters in place; troubled (nullable) receives per-cell flags.
int run_limiter(Ctx& c, void* w, double* wmean, uint8_t* troubled, cudaStream_t st);

}  // namespace dgmhd
