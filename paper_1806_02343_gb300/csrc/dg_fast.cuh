// Specialised GLM kernels for uniform 3D meshes: compile-time sizes and the
// basis tables they take as kernel parameters.
#pragma once
#include "dg_ctx.h"

namespace dgmhd {

template <int DEG>
struct FastDims {
  static constexpr int NQ = DEG + 1;
  static constexpr int N = (DEG + 1) * (DEG + 2) * (DEG + 3) / 6;
  static constexpr int QV = NQ * NQ * NQ;
  static constexpr int QF = NQ * NQ;
  static constexpr int QC = QV > 32 ? 16 : QV;  // volume points per shared-memory pass
};

// traces: PL = values on the +axis face (the left cell's side), PR = on the -axis face
template <typename T, int DEG>
struct FaceTabs {
  T PL[FastDims<DEG>::N][FastDims<DEG>::QF];
  T PR[FastDims<DEG>::N][FastDims<DEG>::QF];
};

// P = values at volume points; dPw = weighted gradients w_q d_a P_l(q);
// Pfw = weighted face values w_p P_l(face f, p); minv = 1/M_l
template <typename T, int DEG>
struct CellTabs {
  T P[FastDims<DEG>::N][FastDims<DEG>::QV];
  T dPw[3][FastDims<DEG>::N][FastDims<DEG>::QV];
  T Pfw[6][FastDims<DEG>::N][FastDims<DEG>::QF];
  T minv[FastDims<DEG>::N];
};

template <typename T, int DEG>
struct FastAll {
  FaceTabs<T, DEG> face[3];
  CellTabs<T, DEG> cell;
};

struct FastGeom {
  int nx, ny, nz;
  int64_t ncell, stride;
  double dx, gamma;
  double metric;  // 2 / dx
};

template <typename T, int DEG>
void launch_face_glm(const FastAll<T, DEG>& tabs, const FastGeom& g, const T* w, T* F, const DevScalars* sc,
                     double eps, cudaStream_t st);
template <typename T, int DEG>
void launch_cell_glm(const FastAll<T, DEG>& tabs, const FastGeom& g, const T* w, const T* F, T* out, const T* w0,
                     double ca, double cb, int combine, const DevScalars* sc, const double* wmean,
                     const double* w0mean, double* outmean, cudaStream_t st);

}  // namespace dgmhd
