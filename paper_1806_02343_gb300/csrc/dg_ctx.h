// Internal context of the DG-MHD library: mesh, device tables, scratch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/dg_mhd.h"
#include "dg_basis.h"
#include "dg_plan.h"

namespace dgmhd {

constexpr int MAXV = 9;       // conserved variables incl. psi
constexpr int MAXD = 3;       // supported polynomial degree
constexpr int MAXQV = 64;     // (MAXD+1)^3 volume points
constexpr int MAXQF = 16;     // (MAXD+1)^2 points per face
constexpr int MAXROWS = 180;  // 9 * n(3)

// Device-resident basis tables for one (D, d, scheme). T = double or float.
// Layouts (q: volume point, p: face point, f = 2*axis + side, side 1 = +face):
//   Pv[l*Qv+q]            Legendre values at volume points
//   dPv[(a*n+l)*Qv+q]     d/dxi_a of Legendre
//   Pf[(f*n+l)*Qf+p]      Legendre values at face points
//   Lv[(j*DB+c)*Qv+q]     LDF component c at volume points
//   dLv[((a*nd+j)*DB+c)*Qv+q]
//   Lf[((f*nd+j)*DB+c)*Qf+p]
//   wv[q], wf[p], minv[r] = 1/M_r, L0[j*DB+c] = cell mean of LDF component
//   Pp[l*npos + pt], Lp[(j*DB+c)*npos + pt]: values at all volume points and then
//   all face points (npos = Qv + 2D*Qf), for the positivity limiter
template <typename T>
struct Tables {
  T *Pv = nullptr, *dPv = nullptr, *Pf = nullptr;
  T *Lv = nullptr, *dLv = nullptr, *Lf = nullptr, *L0 = nullptr;
  T *wv = nullptr, *wf = nullptr, *minv = nullptr;
  T *Pp = nullptr, *Lp = nullptr;
  // the same tables with the point index padded to a multiple of 4 (zeros),
  // for 16-byte vector loads: dPv4[(a*n+l)*QVP+q], dLv4[((a*nd+j)*DB+c)*QVP+q],
  // Pf4[(f*n+l)*QFP+p], Lf4[((f*nd+j)*DB+c)*QFP+p]; null where not built
  T *dPv4 = nullptr, *dLv4 = nullptr, *Pf4 = nullptr, *Lf4 = nullptr;
};

// point counts padded to a multiple of 4
__host__ __device__ constexpr int pad4(int n) { return (n + 3) & ~3; }

// Kernel-facing description of the discretisation (passed by value).
struct Geom {
  int D, d, n, ndiv, DB;  // DB: LDF components (= D)
  int Qv, Qf, nq1;        // volume pts, face pts, pts per dim
  int V;                  // variables (8 Powell, 9 GLM)
  int nrows;              // DoF rows per cell
  int ldf0;               // first LDF row (5n) or -1
  int bz2d;               // first B_z Legendre row in 2D Powell, or -1
  int glm;                // 1: GLM, 0: Powell
  int nx, ny, nz;         // cells per axis (nz = 1 in 2D)
  int64_t ncell, stride;  // cells and row stride
  double dx, gamma;
  // cells that count in the timestep minimum (a partition's owned cells; NULL: all)
  const uint8_t* owned = nullptr;
  // points per face in the Powell jump buffer of the timestep: Qf (0), or 1
  // where the specialised kernels store each face's two sums
  int jq = 0;
};

// Sizes fixed at compile time (3D, degree DEG >= 0, GLM or Powell): the
// kernel's copy of the Geom gets constant fields, so every loop over modes,
// points and rows has a constant trip count and unrolls. DEG < 0: the sizes
// stay those of the run-time Geom.
template <int DEG, int GLMF>
__device__ __forceinline__ Geom pin_geom(const Geom& gin) {
  Geom g = gin;
  if constexpr (DEG >= 0) {
    constexpr int N = (DEG + 1) * (DEG + 2) * (DEG + 3) / 6;
    constexpr int NDIV = DEG == 0 ? 3 : DEG == 1 ? 11 : DEG == 2 ? 26 : 50;  // Table A1, D = 3
    g.D = 3;
    g.d = DEG;
    g.n = N;
    g.DB = 3;
    g.nq1 = DEG + 1;
    g.Qv = (DEG + 1) * (DEG + 1) * (DEG + 1);
    g.Qf = (DEG + 1) * (DEG + 1);
    g.glm = GLMF;
    g.V = GLMF ? 9 : 8;
    g.ndiv = GLMF ? 0 : NDIV;
    g.ldf0 = GLMF ? -1 : 5 * N;
    g.nrows = GLMF ? 9 * N : 5 * N + NDIV;
    g.bz2d = -1;
  }
  return g;
}

// the run-time Geom agrees with pin_geom<g.d, g.glm> (3D, degree 1 or 2)
inline bool pinned_sizes_ok(const Geom& g) {
  if (g.D != 3 || (g.d != 1 && g.d != 2)) return false;
  const int nm = g.d == 1 ? 4 : 10, nd = g.d == 1 ? 11 : 26;
  return g.n == nm && g.DB == 3 && g.bz2d < 0 && g.nq1 == g.d + 1 && g.Qv == (g.d + 1) * (g.d + 1) * (g.d + 1) &&
         g.Qf == (g.d + 1) * (g.d + 1) && g.V == (g.glm ? 9 : 8) &&
         (g.glm ? (g.ndiv == 0 && g.nrows == 9 * nm && g.ldf0 == -1)
                : (g.ndiv == nd && g.nrows == 5 * nm + nd && g.ldf0 == 5 * nm));
}

// Scalars kept on the device so that a step never waits for the host.
struct DevScalars {
  double dt;       // current timestep
  double ch;       // GLM c_h
  double kappa;    // GLM damping rate c_h^2 / c_p^2
  double dtmin_raw;
  unsigned long long dt_bits;  // atomicMin target (positive doubles order as uint64)
  unsigned long long smax_bits;
  int status;      // latched dg_status bits
  int floor_used;
  double inj_mass;    // mass added by the positivity floors (Sec. 4.3)
  double inj_energy;  // energy added by the positivity floors
  unsigned long long pos_cells;  // cells the positivity limiter rescaled (tau < 1)
  unsigned int nflag;            // cells the indicator flagged in the current limiter pass
  unsigned int npos;             // cells the FP32 positivity screen listed in the current pass
  unsigned long long cnt_flagged;  // cells flagged by the indicator, summed over passes
  unsigned long long cnt_limited;  // cells whose slopes the TVB procedure changed, summed over passes
  float dt32, ch32, kappa32;       // FP32 copies of dt, ch, kappa (written with them)
  float pad32;
  double dt_step;                  // the step's dt; dt itself may be a fraction of it for some stages
  unsigned long long dt64_bits;    // FP32 form: FP64 minimum of the screened cells' FP64 bounds
  unsigned long long cnt_poslisted;  // cells listed for the full positivity procedure, summed over passes
};

// a device scalar in the working precision T (FP32 kernels read the float copy)
template <typename T>
__host__ __device__ __forceinline__ T pick_prec(double d, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return d;
}

// Limiter tables (kernel parameters): degree-1 Legendre mode per axis, mode
// degrees, LDF degrees, LDF component means of degree-0 rows, LDF linear slopes
// <phi_jc, xi_a>/<xi_a, xi_a>, and the exact projection of constant / linear
// fields onto the LDF rows: <phi_jc, 1>/M_j and <phi_jc, xi_a>/M_j.
struct LimTabs {
  int deg1[3];
  int mdeg[64];
  int ldf_deg[64];
  double ldf_mean0[64 * 3];
  double ldf_slope[64 * 9];
  double ldf_pc[64 * 3];
  double ldf_pl[64 * 9];
  double ldf_maxabs[64 * 3];  // upper bound of |phi_j,c| on the cell (sum of |monomial coefficients|)
  // FP32 copies for the FP32 form's limiter arithmetic
  float ldf_mean0_f[64 * 3];
  float ldf_slope_f[64 * 9];
  float ldf_pc_f[64 * 3];
  float ldf_pl_f[64 * 9];
};

// Tables and floors of the FP32 positivity screen (kernel parameter).
struct PosScreen {
  float ldf_mean0[9];       // component means of the degree-0 LDF rows j < D, [j*3 + c]
  float ldf_maxabs[64 * 3]; // bound of |phi_j,c| on the cell
  float eps_rho, eps_p, gm1;
};

// Launch accounting: counts every kernel launch; with `on`, records a CUDA
// event pair on the launch stream around each launch of a given kind.
struct Prof {
  static constexpr int KINDS = 7;
  bool on = false;
  int64_t launches[KINDS] = {0, 0, 0, 0, 0, 0, 0};
  double ms[KINDS] = {0, 0, 0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> pool;
  std::vector<int> kind;   // kind of each recorded pair
  size_t used = 0;         // events in use (2 per pair)
  void begin(int k, cudaStream_t st);
  void end(int k, cudaStream_t st);
  int collect();
  void reset();
  void release();
};

// Learned indicator: exact LDF -> per-component Legendre map
// l2l[(j*3 + c)*MLP_MAXN + l] = <phi_j,c, P_l> / M_l.
constexpr int MLP_MAXN = 20;
constexpr int MLP_MAXIN = 192;
struct MlpTabs {
  float l2l[64 * 3 * MLP_MAXN];
  int deg1[3];      // degree-1 Legendre mode along each axis
  float inv_mdx;    // 1 / (M~ dx)
};

// Octree mesh data owned by a context (device arrays; see dg_amr.cuh).
struct AmrHost {
  bool on = false;
  bool partial = false;  // a partition's local mesh (no regridding)
  int64_t nface = 0;
  int maxent = 0, nsub = 0;
  int32_t *fL = nullptr, *fR = nullptr, *fmeta = nullptr, *cstart = nullptr, *centry = nullptr;
  double* dxc = nullptr;
  double *Psub64 = nullptr, *Lsub64 = nullptr;
  float *Psub32 = nullptr, *Lsub32 = nullptr;
  // the same with the point index zero-padded to a multiple of 4
  double *Psub64p = nullptr, *Lsub64p = nullptr;
  float *Psub32p = nullptr, *Lsub32p = nullptr;
  // host copies of the leaves (regridding plans) and, built on first use, the
  // groups of 2^D sibling leaves (octant order; sorted by parent level and
  // coordinates) with the leaf levels on the device
  int D = 0;
  std::vector<int8_t> hlevel;
  std::vector<int32_t> hijk;
  MortonIndex morton;  // the leaves in Morton order (built with the groups)
  int64_t ngroups = -1;
  std::vector<int32_t> hgroups;
  int32_t* groups = nullptr;
  int8_t* lev_dev = nullptr;
  // specialised Powell kernels (3D, degrees 1 and 2): face blocks by type and
  // the trace / own-side tables in the context's precision (OctPow)
  bool fast = false;
  int32_t *bface = nullptr, *bstart = nullptr, *btype = nullptr;
  int64_t nblk = 0;
  void* ftab = nullptr;
  void* ctab = nullptr;
  void* ntab = nullptr;
  // per leaf and side (2 axis + 1 for +axis): the leaves across it, in face-entry
  // order, side_nb[leaf * 24 + side * 4 + k] (-1 past the count), and
  // side_info[leaf * 6 + side] = count | relation << 4 (0 same level, 1 the
  // leaf is the coarser side, 2 the neighbour is coarser)
  int32_t* side_nb = nullptr;
  uint8_t* side_info = nullptr;
  // the last regrid plan (6 ints per new leaf) and a hash of the marks it was made from
  uint64_t plan_hash = 0;
  std::vector<int32_t> plan;
};

struct Ctx {
  AmrHost amr;
  Prof prof;
  LimTabs lim;
  MlpTabs mlp;
  void* mlp_w1 = nullptr;     // bf16 [64][kp]
  void* mlp_w2 = nullptr;     // bf16 [64][64]
  float* mlp_bias = nullptr;  // b1, b2, w3, b3
  int mlp_kp = 0;
  float mlp_thresh = 0.5f;
  Geom g;
  dg_mhd_params p;
  Basis* hb = nullptr;  // host basis (kept for projection tables)
  Tables<double> t64;
  Tables<float> t32;
  DevScalars* sc = nullptr;        // device
  double* face_buf = nullptr;      // FP64 face fluxes
  float* face_buf32 = nullptr;     // FP32 face fluxes
  void* stage_buf[3] = {nullptr, nullptr, nullptr};  // rhs / stage states
  double* stage_mean[3] = {nullptr, nullptr, nullptr};
  double* cellscratch = nullptr;   // per-cell dt contributions
  int proj_npts = 0;
  double* proj_tab = nullptr;      // projection table [r][q][comp]
  double* proj_w = nullptr;
  uint8_t* troubled = nullptr;     // per-cell limiter flags (scratch)
  int32_t* flag_list = nullptr;    // cells flagged by the indicator in the current pass
  int32_t* pos_list = nullptr;     // cells the positivity screen could not clear in the current pass
  PosScreen pscr;                  // FP32 positivity screen tables
  double* rg_tabs = nullptr;       // regridding tables (dg_regrid.cu), built on first use
  void* qdag_buf = nullptr;        // Powell q^dagger per face point (powell_q = 1)
  int64_t lim_passes = 0;          // limiter passes with TVB since the last counter reset
  int64_t lim_plain_cells = 0;     // cells the plain TVB detection examined since the last reset
  int nsm = 152;                   // streaming multiprocessors of the device
  int fast = 0;                    // specialised GLM path: 10*prec + degree, 0 = none
  void* fast_tabs = nullptr;       // host FastAll<T, DEG> (kernel parameters)
  float* tc_tabs = nullptr;        // device operand tables of the tensor-core cell kernel (FP32, degree 2)
  uint8_t* owned = nullptr;        // device copy of the owned-cell mask (dg_mhd_set_owned), or NULL
  bool glm_speeds_set = false;     // GLM: c_h and the damping rate hold a value (from a dt, set_glm or set_dt)
};

}  // namespace dgmhd

struct dg_mhd_ctx {
  dgmhd::Ctx c;
};
