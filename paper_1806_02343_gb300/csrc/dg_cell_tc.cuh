// Cell update of the GLM scheme (3D uniform mesh, degree 2, FP32 form) with
// the DG contractions of Sec. 3.5 eq. wdot on the fifth-generation tensor core.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "dg_ctx.h"
#include "dg_fast.cuh"

namespace dgmhd {

// Operand tables of the three contractions, as FP32 values split into a TF32
// part and a remainder (hi + lo), each stored as a K-major [N][K] operand of
// tcgen05.mma in 8-row x 16-byte core matrices (tc_kidx):
//   P   [32 points][16 modes]            P_l(xi_q), q < 27, l < 10
//   G_j [16 modes][32 = 3 axes x 9]      w_q d_a P_l(xi_q), q = 9 j + i (k = 9 a + i)
//   S_a [16 modes][24 = 2 sides x 9]     -+ w_p P_l(face (a, s), p): side 0 (the
//                                        cell's -a face) +, side 1 (+a face) -;
//                                        mode 0 is zero (the mean row is summed
//                                        on the CUDA cores, exactly antisymmetric)
// Order in memory: P hi, P lo, G hi [3], G lo [3], S hi [3], S lo [3].
struct TcLayout {
  static constexpr int P = 32 * 16;
  static constexpr int G = 16 * 32;
  static constexpr int S = 16 * 24;
  static constexpr int OFF_PH = 0, OFF_PL = P;
  static constexpr int OFF_GH = 2 * P, OFF_GL = 2 * P + 3 * G;
  static constexpr int OFF_SH = 2 * P + 6 * G, OFF_SL = 2 * P + 6 * G + 3 * S;
  static constexpr int TOTAL = 2 * P + 6 * G + 6 * S;  // floats (25,600 bytes)
};

// element (n, k) of a K-major [N][K] FP32/TF32 operand: core matrices of
// 8 rows x 4 elements (16 bytes), K / 4 of them per 8-row group
__host__ __device__ __forceinline__ int tc_kidx(int n, int k, int K) {
  return (((n >> 3) * (K >> 2) + (k >> 2)) << 5) + ((n & 7) << 2) + (k & 3);
}

// Host: builds the tables (TcLayout::TOTAL floats) from the double-precision
// reference-element tables Pv[l*27+q], dPv[(a*10+l)*27+q], Pf[(f*10+l)*9+p],
// wv[q], wf[p] (f = 2 axis + side).
void build_tc_tables(const std::vector<double>& Pv, const std::vector<double>& dPv, const std::vector<double>& Pf,
                     const std::vector<double>& wv, const std::vector<double>& wf, std::vector<float>& out);

// Launches the cell update (same contract as launch_cell_glm<float, 2>);
// tabs: device copy of the tables. Returns 0, or -3 on a launch error.
int launch_cell_tc(const float* tabs, const FastAll<float, 2>& ft, const FastGeom& g, const float* w, const float* F,
                   float* out, const float* w0, double ca, double cb, int combine, const DevScalars* sc,
                   const double* wmean, const double* w0mean, double* outmean, int nsm, cudaStream_t st);

}  // namespace dgmhd
