// FP32 positivity screen (Sec. 4.3), shared by the screen kernel of the
// limiter and the staged learned indicator, which holds every row of its cells
// in shared memory already.
#pragma once
#include "dg_ctx.h"

namespace dgmhd {

// row of the k-th mean (Legendre mode 0 of rho, m, E, psi; degree-0 LDF rows
// for B in the Powell form; the B_z mode 0 row in 2D)
__host__ __device__ __forceinline__ int screen_mean_row(const Geom& g, int k) {
  if (g.glm || k < 5) return k * g.n;
  if (g.D == 3) return g.ldf0 + (k - 5);
  return k < 7 ? g.ldf0 + (k - 5) : g.bz2d;
}

// Rigorous screen in FP32 from the float mirror of the means: |P_l| <= 1 and
// |phi_j,c| <= maxabs on the cell bound |u_v(x) - mean_v| by dev_v at every
// point; a relative margin 1e-4 covers the rounding of the bound itself. True:
// rho and p clear twice their floors everywhere and the cell needs no work.
// row(r) returns the cell's coefficient of row r.
template <typename Row>
__device__ __forceinline__ bool pos_screen_rows(const Geom& g, const PosScreen& ps, Row row) {
  float mt[8];
#pragma unroll
  for (int k = 0; k < 5; ++k) mt[k] = row(screen_mean_row(g, k));
  if (g.glm) {
#pragma unroll
    for (int k = 5; k < 8; ++k) mt[k] = row(screen_mean_row(g, k));
  } else {
    mt[5] = mt[6] = mt[7] = 0.f;
    for (int j = 0; j < g.D; ++j)
      for (int cc = 0; cc < g.D; ++cc) mt[5 + cc] += row(g.ldf0 + j) * ps.ldf_mean0[j * 3 + cc];
    if (g.bz2d >= 0) mt[7] = row(g.bz2d);
  }
  float dv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int nlg = g.glm ? 8 : 5;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    if (v >= nlg) continue;
    for (int l = 1; l < g.n; ++l) dv[v] += fabsf(row(v * g.n + l));
  }
  if (!g.glm) {
    for (int j = g.D; j < g.ndiv; ++j) {
      const float aj = fabsf(row(g.ldf0 + j));
#pragma unroll
      for (int cc = 0; cc < 3; ++cc)
        if (cc < g.D) dv[5 + cc] += aj * ps.ldf_maxabs[j * 3 + cc];
    }
    if (g.bz2d >= 0)
      for (int l = 1; l < g.n; ++l) dv[7] += fabsf(row(g.bz2d + l));
  }
  const float mg = 1e-4f;
#pragma unroll
  for (int v = 0; v < 8; ++v) dv[v] = dv[v] * (1.f + mg) + mg * fabsf(mt[v]);
  const float rlo = mt[0] - dv[0];
  if (rlo > ps.eps_rho * 2.f) {
    float kin = 0.f, mag = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float mu = fabsf(mt[1 + i]) + dv[1 + i];
      const float bu = fabsf(mt[5 + i]) + dv[5 + i];
      kin += mu * mu;
      mag += bu * bu;
    }
    const float plo = ps.gm1 * (mt[4] - dv[4] - 0.5f * kin / rlo - 0.5f * mag);
    if (plo > ps.eps_p * 2.f + mg * fabsf(mt[4])) return true;
  }
  return false;
}

// ballot compaction of a warp's cells into list[0 .. *count)
__device__ __forceinline__ void append_cells(bool mine, int64_t c, int32_t* __restrict__ list, unsigned* count) {
  const int lane = threadIdx.x & 31;
  const unsigned bal = __ballot_sync(0xffffffffu, mine);
  unsigned at = 0;
  if (lane == 0 && bal) at = atomicAdd(count, (unsigned)__popc(bal));
  at = __shfl_sync(0xffffffffu, at, 0);
  if (mine) list[at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)c;
}

}  // namespace dgmhd
