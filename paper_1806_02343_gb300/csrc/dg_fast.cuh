// Specialised GLM kernels for uniform 3D meshes: compile-time sizes and the
// basis tables they take as kernel parameters.
#pragma once
#include <type_traits>

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

// Powell scheme (Sec. 3.3): the magnetic field's locally divergence-free
// (LDF) coefficients c_j and the Legendre coefficients of its components,
// b[cc][l] = sum_j A[j][cc][l] c_j (every LDF function's components are
// polynomials of total degree <= d, so A is exact). The kernels evaluate and
// integrate B in that Legendre form, then map the residuals back to LDF rows
// with the same matrix: R_j = sum_{cc,l} A[j][cc][l] R[cc][l].
// The first three LDF functions are constant vectors (the cell means of B);
// the others have zero mean.
template <int DEG>
struct PowDims {
  static constexpr int NDIV = DEG == 1 ? 11 : DEG == 2 ? 26 : 50;  // Table A1, D = 3
  static constexpr int NP = (NDIV - 3 + 1) / 2;                   // pairs of non-mean LDF rows
};
template <typename T, int DEG>
struct PowTabs {
  alignas(16) T Af[3][PowDims<DEG>::NDIV][FastDims<DEG>::N];      // forward: [cc][j][l]
  alignas(16) T Ab[PowDims<DEG>::NP][3][FastDims<DEG>::N][2];     // back: rows 3+2k, 4+2k
  alignas(16) T minvL[PowDims<DEG>::NDIV + 1];                    // 1 / LDF mass
  // normal component (axis a) of LDF function j at point p of face 2a + s
  alignas(16) T Ln[3][2][PowDims<DEG>::NDIV][FaceTabs<T, DEG>::QFP];
  alignas(16) T wf[FaceTabs<T, DEG>::QFP];                        // face weights
  double kL[3];   // mean of component cc: minvL[jm] A[jm][cc][0] (times 2/dx in the kernel)
  int jm[3];      // the constant LDF row whose vector is along component cc
  int ok;         // the basis has the structure above (else Powell runs the generic kernels)
};

// (degree 3 runs the Powell scheme on the generic kernels: its tables would
// not fit in the constant bank next to the GLM ones)
struct NoPowTabs {
  int ok;  // 0 (value-initialised with the tables)
};
template <typename T, int DEG>
struct FastAll {
  FaceTabs<T, DEG> face[3];
  CellTabs<T, DEG> cell;
  std::conditional_t<(DEG <= 2), PowTabs<T, DEG>, NoPowTabs> pow;
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
// Powell / LDF kernels (face buffer: 10 slots per face point, see dg_fast_impl.cuh)
template <typename T, int DEG>
void launch_face_pow(const FastAll<T, DEG>& tabs, const FastGeom& g, const T* w, T* F, double eps, cudaStream_t st);
template <typename T, int DEG>
void launch_cell_pow(const FastAll<T, DEG>& tabs, const FastGeom& g, const T* w, const T* F, T* out, const T* w0,
                     double ca, double cb, int combine, const DevScalars* sc, const double* wmean,
                     const double* w0mean, double* outmean, cudaStream_t st);
// Octree meshes (Powell / LDF): the face list of the generic octree kernels
// plus the face blocks of the specialised pass -- bface lists the faces
// grouped by type (axis a, same level / left coarse / right coarse, sub-face),
// block b takes bface[bstart[b] ..] with btype[b] = type | count << 8 (count
// <= 32, type = 9 a + (0 | 1 + sub | 5 + sub)); ftab[type][side][N][QFP] the
// trace tables of the two sides (side 0: the left cell) and
// ctab[30][QF][N] the own-side weighted face tables of the cell pass (0..5:
// the faces, 6 + 4 f + sub: sub-face sub of face f of a coarse cell, weights
// w_p / 4).
template <typename T>
struct OctPow {
  const int32_t* fL;
  const int32_t* fR;
  const int32_t* fmeta;
  const int32_t* cstart;
  const int32_t* centry;
  const double* dxc;
  const int32_t* bface;
  const int32_t* bstart;
  const int32_t* btype;
  const T* ftab;
  const T* ctab;
  const T* ntab;  // [type][side][NDIV][QFP]: normal component of each LDF function on the side's (sub-)face
  int64_t ncell, stride;
  int64_t nblk;
};
template <typename T, int DEG>
void launch_divb_list_pow(const OctPow<T>& o, const T* w, T* jbuf, cudaStream_t st);
template <typename T, int DEG>
void launch_face_list_pow(const OctPow<T>& o, double gamma, const T* w, T* F, double eps, cudaStream_t st);
template <typename T, int DEG>
void launch_cell_list_pow(const OctPow<T>& o, double gamma, const T* w, const T* F, T* out, const T* w0, double ca,
                          double cb, int combine, const DevScalars* sc, const double* wmean, const double* w0mean,
                          double* outmean, cudaStream_t st);

// Powell timestep's face jumps (eq. powell_dt): per face point w_p |B^n_F - B^n_L|
// and w_p |B^n_F - B^n_R|, laid out as the generic k_divb_face writes them
template <typename T, int DEG>
void launch_divb_face_pow(const FastGeom& g, const T* w, T* jbuf, cudaStream_t st);
template <typename T, int DEG>
void launch_cell_glm(const FastAll<T, DEG>& tabs, const FastGeom& g, const T* w, const T* F, T* out, const T* w0,
                     double ca, double cb, int combine, const DevScalars* sc, const double* wmean,
                     const double* w0mean, double* outmean, cudaStream_t st);

}  // namespace dgmhd
