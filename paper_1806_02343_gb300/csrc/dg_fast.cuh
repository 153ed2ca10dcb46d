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

// Exponents (k1, k2, k3) of the Legendre modes in the basis order (total
// degree, then k1 descending, then k2 descending), and per axis the modes
// whose derivative along it is not identically zero (k_a >= 1): the volume
// integral skips the others at compile time.
template <int DEG>
struct ModeTab {
  static constexpr int N = FastDims<DEG>::N;
  int k[N][3];
  int nz[3][N];
  int cnt[3];
  constexpr ModeTab() : k{}, nz{}, cnt{} {
    int i = 0;
    for (int deg = 0; deg <= DEG; ++deg)
      for (int a = deg; a >= 0; --a)
        for (int b = deg - a; b >= 0; --b) {
          k[i][0] = a;
          k[i][1] = b;
          k[i][2] = deg - a - b;
          ++i;
        }
    for (int ax = 0; ax < 3; ++ax) {
      cnt[ax] = 0;
      for (int l = 0; l < N; ++l)
        if (k[l][ax] > 0) nz[ax][cnt[ax]++] = l;
    }
  }
};

template <int DEG>
constexpr ModeTab<DEG> kModes{};

// Table layouts put the two operands of every packed FMA in one aligned
// 64-bit word (rows padded to an even length, pairs stored side by side).
// traces: PL = values on the +axis face (the left cell's side), PR = on the -axis face
template <typename T, int DEG>
struct FaceTabs {
  static constexpr int QFP = FastDims<DEG>::QF + (FastDims<DEG>::QF & 1);
  alignas(16) T PL[FastDims<DEG>::N][QFP];
  alignas(16) T PR[FastDims<DEG>::N][QFP];
};

// P = values at volume points (rows padded); dP2[a][i][q] = weighted
// gradients w_q d_a P_l(q) of the i-th pair of modes with k_a >= 1 (an odd
// count is padded with mode 0 and zero weight); Pfw[f][p][l] = weighted face
// values w_p P_l(face f, p), modes fastest; minv = 1/M_l
template <int DEG>
struct CellDims {
  static constexpr int QVP = FastDims<DEG>::QV + (FastDims<DEG>::QV & 1);
  static constexpr int MAXPAIR = (FastDims<DEG>::N + 1) / 2;
};
template <typename T, int DEG>
struct CellTabs {
  alignas(16) T P[FastDims<DEG>::N][CellDims<DEG>::QVP];
  alignas(16) T dP2[3][CellDims<DEG>::MAXPAIR][FastDims<DEG>::QV][2];
  alignas(16) T Pfw[6][FastDims<DEG>::QF][FastDims<DEG>::N];
  alignas(16) T minv[FastDims<DEG>::N];
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
  double metric;   // 2 / dx
  double kmean;    // metric / M_0: the mean row's factor (M_0 = 2^3)
  float gamma32, metric32;
};

// copies the tables to the constant bank where this (T, DEG) keeps them there
// (synchronous; returns 0 or -3)
template <typename T, int DEG>
int fast_to_constant(const FastAll<T, DEG>& tabs);
template <typename T, int DEG>
void launch_face_glm(const FastAll<T, DEG>& tabs, const FastGeom& g, const T* w, T* F, const DevScalars* sc,
                     double eps, cudaStream_t st);
template <typename T, int DEG>
void launch_cell_glm(const FastAll<T, DEG>& tabs, const FastGeom& g, const T* w, const T* F, T* out, const T* w0,
                     double ca, double cb, int combine, const DevScalars* sc, const double* wmean,
                     const double* w0mean, double* outmean, cudaStream_t st);

}  // namespace dgmhd
