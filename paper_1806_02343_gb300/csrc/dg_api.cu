// C ABI of the DG-MHD library (see include/dg_mhd.h for the contract).
#include <cuda_runtime.h>

#include <climits>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/dg_mhd.h"
#include "dg_amr.cuh"
#include "dg_basis.h"
#include "dg_ctx.h"
#include "dg_cell_tc.cuh"
#include "dg_fast.cuh"
#include "dg_kernels.cuh"
#include "dg_limit.cuh"
#include "dg_mlp.cuh"

using namespace dgmhd;

namespace {

#define CK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) return DG_E_CUDA;   \
  } while (0)

template <typename T>
int upload(T** dst, const std::vector<double>& src) {
  std::vector<T> tmp(src.begin(), src.end());
  if (tmp.empty()) tmp.push_back(T(0));
  CK(cudaMalloc(dst, tmp.size() * sizeof(T)));
  CK(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
  return DG_OK;
}

struct HostTables {
  std::vector<double> Pv, dPv, Pf, Lv, dLv, Lf, L0, wv, wf, minv, Pp, Lp;
  std::vector<double> dPv4, dLv4, Pf4, Lf4;  // point index padded to a multiple of 4
};

// rows of length len copied into rows of length lenp (zero padding)
std::vector<double> pad_rows(const std::vector<double>& src, int len, int lenp) {
  const size_t rows = src.size() / (size_t)len;
  std::vector<double> out(rows * (size_t)lenp, 0.0);
  for (size_t r = 0; r < rows; ++r)
    for (int k = 0; k < len; ++k) out[r * lenp + k] = src[r * len + k];
  return out;
}

// reference coordinates of volume point q (tensor rule, last axis fastest)
void vol_point(int D, const std::vector<double>& x1, int q, double* xi) {
  const int m = (int)x1.size();
  for (int a = D - 1; a >= 0; --a) {
    xi[a] = x1[q % m];
    q /= m;
  }
  for (int a = D; a < 3; ++a) xi[a] = 0.0;
}

// point p of face f = 2*axis + side: tangential axes in increasing order, last fastest
void face_point(int D, const std::vector<double>& x1, int f, int p, double* xi) {
  const int a = f >> 1;
  const int m = (int)x1.size();
  int others[2], no = 0;
  for (int b = 0; b < D; ++b)
    if (b != a) others[no++] = b;
  for (int j = no - 1; j >= 0; --j) {
    xi[others[j]] = x1[p % m];
    p /= m;
  }
  xi[a] = (f & 1) ? 1.0 : -1.0;
  for (int b = D; b < 3; ++b) xi[b] = 0.0;
}

void build_host_tables(const Basis& B, const Geom& g, HostTables& h) {
  std::vector<double> x1, w1;
  gauss_legendre(g.nq1, x1, w1);
  const int D = g.D, n = g.n, nd = g.ndiv, DB = g.DB, Qv = g.Qv, Qf = g.Qf;
  h.wv.assign(Qv, 1.0);
  for (int q = 0; q < Qv; ++q) {
    int qq = q;
    for (int a = 0; a < D; ++a) {
      h.wv[q] *= w1[qq % g.nq1];
      qq /= g.nq1;
    }
  }
  h.wf.assign(Qf, 1.0);
  for (int p = 0; p < Qf; ++p) {
    int pp = p;
    for (int a = 0; a < D - 1; ++a) {
      h.wf[p] *= w1[pp % g.nq1];
      pp /= g.nq1;
    }
  }
  double xi[3];
  h.Pv.assign((size_t)n * Qv, 0.0);
  h.dPv.assign((size_t)D * n * Qv, 0.0);
  for (int l = 0; l < n; ++l)
    for (int q = 0; q < Qv; ++q) {
      vol_point(D, x1, q, xi);
      h.Pv[(size_t)l * Qv + q] = B.eval(B.leg[l], xi);
      for (int a = 0; a < D; ++a) h.dPv[((size_t)a * n + l) * Qv + q] = B.eval_deriv(B.leg[l], a, xi);
    }
  h.Pf.assign((size_t)2 * D * n * Qf, 0.0);
  for (int f = 0; f < 2 * D; ++f)
    for (int l = 0; l < n; ++l)
      for (int p = 0; p < Qf; ++p) {
        face_point(D, x1, f, p, xi);
        h.Pf[((size_t)f * n + l) * Qf + p] = B.eval(B.leg[l], xi);
      }
  h.Lv.assign((size_t)std::max(1, nd * DB * Qv), 0.0);
  h.dLv.assign((size_t)std::max(1, D * nd * DB * Qv), 0.0);
  h.Lf.assign((size_t)std::max(1, 2 * D * nd * DB * Qf), 0.0);
  h.L0.assign((size_t)std::max(1, nd * DB), 0.0);
  for (int j = 0; j < nd; ++j)
    for (int c = 0; c < DB; ++c) {
      for (int q = 0; q < Qv; ++q) {
        vol_point(D, x1, q, xi);
        h.Lv[((size_t)j * DB + c) * Qv + q] = B.eval(B.ldf[j][c], xi);
        for (int a = 0; a < D; ++a)
          h.dLv[(((size_t)a * nd + j) * DB + c) * Qv + q] = B.eval_deriv(B.ldf[j][c], a, xi);
      }
      for (int f = 0; f < 2 * D; ++f)
        for (int p = 0; p < Qf; ++p) {
          face_point(D, x1, f, p, xi);
          h.Lf[(((size_t)f * nd + j) * DB + c) * Qf + p] = B.eval(B.ldf[j][c], xi);
        }
      if (B.ldf_deg[j] == 0) {
        double z[3] = {0.0, 0.0, 0.0};
        h.L0[(size_t)j * DB + c] = B.eval(B.ldf[j][c], z);
      }
    }
  // all volume then all face points, contiguous per mode (positivity limiter)
  const int npos = Qv + 2 * D * Qf;
  h.Pp.assign((size_t)n * npos, 0.0);
  h.Lp.assign((size_t)std::max(1, nd * DB * npos), 0.0);
  for (int pt = 0; pt < npos; ++pt) {
    if (pt < Qv) vol_point(D, x1, pt, xi);
    else face_point(D, x1, (pt - Qv) / Qf, (pt - Qv) % Qf, xi);
    for (int l = 0; l < n; ++l) h.Pp[(size_t)l * npos + pt] = B.eval(B.leg[l], xi);
    for (int j = 0; j < nd; ++j)
      for (int c = 0; c < DB; ++c) h.Lp[((size_t)j * DB + c) * npos + pt] = B.eval(B.ldf[j][c], xi);
  }
  h.dPv4 = pad_rows(h.dPv, Qv, pad4(Qv));
  h.dLv4 = pad_rows(h.dLv, Qv, pad4(Qv));
  h.Pf4 = pad_rows(h.Pf, Qf, pad4(Qf));
  h.Lf4 = pad_rows(h.Lf, Qf, pad4(Qf));
  h.minv.assign(g.nrows, 0.0);
  for (int r = 0; r < g.nrows; ++r) {
    double m;
    if (g.ldf0 >= 0 && r >= g.ldf0 && r < g.ldf0 + nd) m = B.ldf_mass[r - g.ldf0];
    else if (g.bz2d >= 0 && r >= g.bz2d) m = B.leg_mass[r - g.bz2d];
    else m = B.leg_mass[r % n];
    h.minv[r] = 1.0 / m;
  }
}

template <typename T>
int upload_tables(const HostTables& h, Tables<T>& t) {
  int e;
  if ((e = upload(&t.Pv, h.Pv))) return e;
  if ((e = upload(&t.dPv, h.dPv))) return e;
  if ((e = upload(&t.Pf, h.Pf))) return e;
  if ((e = upload(&t.Lv, h.Lv))) return e;
  if ((e = upload(&t.dLv, h.dLv))) return e;
  if ((e = upload(&t.Lf, h.Lf))) return e;
  if ((e = upload(&t.L0, h.L0))) return e;
  if ((e = upload(&t.wv, h.wv))) return e;
  if ((e = upload(&t.wf, h.wf))) return e;
  if ((e = upload(&t.minv, h.minv))) return e;
  if ((e = upload(&t.Pp, h.Pp))) return e;
  if ((e = upload(&t.Lp, h.Lp))) return e;
  if ((e = upload(&t.dPv4, h.dPv4))) return e;
  if ((e = upload(&t.dLv4, h.dLv4))) return e;
  if ((e = upload(&t.Pf4, h.Pf4))) return e;
  if ((e = upload(&t.Lf4, h.Lf4))) return e;
  return DG_OK;
}

template <typename T>
void free_tables(Tables<T>& t) {
  T* ptrs[] = {t.Pv, t.dPv, t.Pf, t.Lv, t.dLv, t.Lf, t.L0, t.wv, t.wf, t.minv, t.Pp, t.Lp,
               t.dPv4, t.dLv4, t.Pf4, t.Lf4};
  for (T* p : ptrs)
    if (p) cudaFree(p);
  t = Tables<T>();
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Powell kernels' tables (dg_fast.cuh PowTabs): the Legendre coefficients of
// the LDF functions' components by quadrature (exact: every component is a
// polynomial of total degree <= d), checked against the functions themselves;
// ok = 0 when the basis lacks the structure the kernels rely on (three
// constant functions, each along one axis, and no other function with a
// non-zero mean). The same for every context of this degree.
// A[(j * 3 + c) * n + l]: the Legendre coefficients of component c of the 3D
// LDF function j of degree <= deg, by quadrature with deg + 1 Gauss points
// per axis (exact: the products are polynomials of degree <= 2 deg per
// axis), entries below 1e-13 set to zero, and the expansion checked against
// the functions at the points (false if it misses by more than 1e-11).
bool ldf_legendre_3d(int deg, std::vector<double>& A, int& ndiv, int& n) {
  Basis L;
  if (!L.build(3, deg, true)) return false;
  ndiv = L.ndiv;
  n = L.n;
  std::vector<double> x1, w1;
  gauss_legendre(deg + 1, x1, w1);
  int Qv = 1;
  for (int k = 0; k < 3; ++k) Qv *= deg + 1;
  A.assign((size_t)ndiv * 3 * n, 0.0);
  double xi[3];
  for (int q = 0; q < Qv; ++q) {
    vol_point(3, x1, q, xi);
    double wq = 1.0;
    for (int k = 0, qq = q; k < 3; ++k, qq /= deg + 1) wq *= w1[qq % (deg + 1)];
    for (int l = 0; l < n; ++l) {
      const double Pl = L.eval(L.leg[l], xi) * wq / L.leg_mass[l];
      for (int j = 0; j < ndiv; ++j)
        for (int cc = 0; cc < 3; ++cc) A[((size_t)j * 3 + cc) * n + l] += L.eval(L.ldf[j][cc], xi) * Pl;
    }
  }
  for (double& x : A)
    if (std::fabs(x) < 1e-13) x = 0.0;
  for (int q = 0; q < Qv; ++q) {
    vol_point(3, x1, q, xi);
    for (int j = 0; j < ndiv; ++j)
      for (int cc = 0; cc < 3; ++cc) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) s += A[((size_t)j * 3 + cc) * n + l] * L.eval(L.leg[l], xi);
        if (std::fabs(s - L.eval(L.ldf[j][cc], xi)) > 1e-11) return false;
      }
  }
  return true;
}

template <typename T, int DEG>
void build_pow_tabs(PowTabs<T, DEG>& pt) {
  using Dm = FastDims<DEG>;
  constexpr int N = Dm::N, NDIV = PowDims<DEG>::NDIV, NP = PowDims<DEG>::NP;
  pt = PowTabs<T, DEG>();
  std::vector<double> A;
  int nd = 0, nm = 0;
  if (!ldf_legendre_3d(DEG, A, nd, nm) || nd != NDIV || nm != N) return;
  Basis L;
  L.build(3, DEG, true);
  std::vector<double> x1, w1;
  gauss_legendre(DEG + 1, x1, w1);
  double xi[3];
  auto a = [&](int j, int cc, int l) -> double& { return A[((size_t)j * 3 + cc) * N + l]; };
  int seen = 0;
  for (int j = 0; j < NDIV; ++j)
    for (int cc = 0; cc < 3; ++cc)
      for (int l = 0; l < N; ++l) {
        if (j < 3 && l > 0 && a(j, cc, l) != 0.0) return;
        if (j >= 3 && l == 0 && a(j, cc, l) != 0.0) return;
      }
  for (int j = 0; j < 3; ++j) {
    int nz = 0, at = -1;
    for (int cc = 0; cc < 3; ++cc)
      if (a(j, cc, 0) != 0.0) ++nz, at = cc;
    if (nz != 1 || (seen >> at) & 1) return;
    seen |= 1 << at;
    pt.jm[at] = j;
  }
  for (int cc = 0; cc < 3; ++cc)
    for (int j = 0; j < NDIV; ++j)
      for (int l = 0; l < N; ++l) pt.Af[cc][j][l] = (T)a(j, cc, l);
  for (int k = 0; k < NP; ++k)
    for (int e = 0; e < 2; ++e) {
      const int j = 3 + 2 * k + e;
      for (int cc = 0; cc < 3; ++cc)
        for (int l = 0; l < N; ++l) pt.Ab[k][cc][l][e] = j < NDIV ? (T)a(j, cc, l) : T(0);
    }
  for (int j = 0; j < NDIV; ++j) pt.minvL[j] = (T)(1.0 / L.ldf_mass[j]);
  for (int a2 = 0; a2 < 3; ++a2)
    for (int sd = 0; sd < 2; ++sd)
      for (int p = 0; p < Dm::QF; ++p) {
        face_point(3, x1, 2 * a2 + sd, p, xi);
        for (int j = 0; j < NDIV; ++j) pt.Ln[a2][sd][j][p] = (T)L.eval(L.ldf[j][a2], xi);
      }
  for (int p = 0; p < Dm::QF; ++p) {
    double wp = 1.0;
    for (int k = 0, pp = p; k < 2; ++k, pp /= DEG + 1) wp *= w1[pp % (DEG + 1)];
    pt.wf[p] = (T)wp;
  }
  for (int cc = 0; cc < 3; ++cc) pt.kL[cc] = a(pt.jm[cc], cc, 0) / L.ldf_mass[pt.jm[cc]];
  pt.ok = 1;
}

template <typename T, int DEG>
void* make_fast_tabs(const HostTables& h, const Geom& g, const Basis& B) {
  using Dm = FastDims<DEG>;
  // the kernels unroll over the mode exponents known at compile time
  constexpr ModeTab<DEG> MT{};
  if ((int)B.modes.size() != Dm::N) return nullptr;
  for (int l = 0; l < Dm::N; ++l)
    for (int a = 0; a < 3; ++a)
      if (B.modes[l][a] != MT.k[l][a]) return nullptr;
  auto* ft = new FastAll<T, DEG>();
  const int n = g.n, Qv = g.Qv, Qf = g.Qf;
  for (int a = 0; a < 3; ++a)
    for (int l = 0; l < n; ++l)
      for (int p = 0; p < Qf; ++p) {
        ft->face[a].PL[l][p] = (T)h.Pf[((size_t)(2 * a + 1) * n + l) * Qf + p];
        ft->face[a].PR[l][p] = (T)h.Pf[((size_t)(2 * a) * n + l) * Qf + p];
      }
  for (int l = 0; l < n; ++l) {
    for (int q = 0; q < Qv; ++q) ft->cell.P[l][q] = (T)h.Pv[(size_t)l * Qv + q];
    for (int f = 0; f < 6; ++f)
      for (int p = 0; p < Qf; ++p) ft->cell.Pfw[f][p][l] = (T)(h.Pf[((size_t)f * n + l) * Qf + p] * h.wf[p]);
    ft->cell.minv[l] = (T)h.minv[l];
  }
  // gradient pairs: modes with k_a >= 1, in pairs (the last one of an odd
  // count is paired with a zero entry)
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < MT.cnt[a]; ++i) {
      const int l = MT.nz[a][i];
      for (int q = 0; q < Qv; ++q) ft->cell.dP2[a][i / 2][q][i % 2] = (T)(h.dPv[((size_t)a * n + l) * Qv + q] * h.wv[q]);
    }
  static_assert(Dm::N > 0, "");
  if constexpr (DEG <= 2) build_pow_tabs<T, DEG>(ft->pow);
  if (fast_to_constant<T, DEG>(*ft)) {
    delete ft;
    return nullptr;
  }
  return ft;
}

void free_fast_tabs(Ctx& c) {
  if (!c.fast_tabs) return;
  switch (c.fast) {
    case 11: delete (FastAll<float, 1>*)c.fast_tabs; break;
    case 12: delete (FastAll<float, 2>*)c.fast_tabs; break;
    case 13: delete (FastAll<float, 3>*)c.fast_tabs; break;
    case 21: delete (FastAll<double, 1>*)c.fast_tabs; break;
    case 22: delete (FastAll<double, 2>*)c.fast_tabs; break;
  }
  c.fast_tabs = nullptr;
  c.fast = 0;
}

// the Powell tables of the context's specialised kernels have the expected structure
bool fast_pow_ok(const Ctx& c) {
  switch (c.fast) {
    case 11: return ((const FastAll<float, 1>*)c.fast_tabs)->pow.ok != 0;
    case 12: return ((const FastAll<float, 2>*)c.fast_tabs)->pow.ok != 0;
    case 13: return false;
    case 21: return ((const FastAll<double, 1>*)c.fast_tabs)->pow.ok != 0;
    case 22: return ((const FastAll<double, 2>*)c.fast_tabs)->pow.ok != 0;
  }
  return false;
}

FastGeom fast_geom(const Geom& g) {
  FastGeom f;
  f.nx = g.nx; f.ny = g.ny; f.nz = g.nz;
  f.ncell = g.ncell; f.stride = g.stride;
  f.dx = g.dx; f.gamma = g.gamma;
  f.metric = 2.0 / g.dx;
  f.kmean = f.metric / 8.0;
  f.gamma32 = (float)g.gamma;
  f.metric32 = (float)f.metric;
  return f;
}

inline bool fp32(const Ctx& c) { return c.p.precision == DG_PREC_FP32MIX; }

// the Powell kernels exist for degrees 1 and 2 (a degree-3 context never
// selects them: its tables are not built)
template <typename T, int DEG>
void face_pow_fast(const FastAll<T, DEG>& ft, const FastGeom& fg, const T* w, T* F, double eps, cudaStream_t st) {
  if constexpr (DEG <= 2) launch_face_pow<T, DEG>(ft, fg, w, F, eps, st);
}
template <typename T, int DEG>
void cell_pow_fast(const FastAll<T, DEG>& ft, const FastGeom& fg, const T* w, const T* F, T* out, const T* w0,
                   double ca, double cb, int combine, const DevScalars* sc, const double* wmean, const double* w0mean,
                   double* outmean, cudaStream_t st) {
  if constexpr (DEG <= 2)
    launch_cell_pow<T, DEG>(ft, fg, w, F, out, w0, ca, cb, combine, sc, wmean, w0mean, outmean, st);
}

// the tensor-core cell update where the context built its tables (FP32 form,
// degree 2); false: the caller launches the CUDA-core one
template <typename T, int DEG>
bool launch_cell_fast(Ctx& c, const FastAll<T, DEG>& ft, const FastGeom& fg, const T* w, const T* F, T* out,
                      const T* w0, double ca, double cb, int combine, const double* wmean, const double* w0mean,
                      double* outmean, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value && DEG == 2) {
    if (c.tc_tabs) {
      launch_cell_tc(c.tc_tabs, ft, fg, w, F, out, w0, ca, cb, combine, c.sc, wmean, w0mean, outmean, c.nsm, st);
      return true;
    }
  }
  return false;
}


}  // namespace

namespace dgmhd {

// Geometry and host basis for a uniform periodic mesh, for callers that keep
// no context (the allocation-free entry point); mirrors the set-up in init.
int make_geom(const dg_mesh_desc* mesh, int degree, int divB_scheme, double gamma, Basis& B, Geom& g) {
  if (mesh->dim != 2 && mesh->dim != 3) return DG_E_MESH;
  if (mesh->level) return DG_E_UNSUPPORTED;  // uniform meshes only
  if (!mesh->periodic) return DG_E_UNSUPPORTED;
  if (degree < 0 || degree > MAXD) return DG_E_UNSUPPORTED;
  if (divB_scheme != DG_DIVB_POWELL && divB_scheme != DG_DIVB_GLM) return DG_E_ARG;
  if (!(gamma > 1.0)) return DG_E_ARG;
  for (int a = 0; a < mesh->dim; ++a)
    if (mesh->n[a] < 1) return DG_E_MESH;
  if (!(mesh->box_len > 0.0)) return DG_E_MESH;
  g = Geom();
  g.D = mesh->dim;
  g.d = degree;
  g.glm = divB_scheme == DG_DIVB_GLM;
  if (!B.build(g.D, degree, !g.glm)) return DG_E_UNSUPPORTED;
  g.n = B.n;
  g.ndiv = B.ndiv;
  g.DB = g.D;
  g.nq1 = degree + 1;
  g.Qv = 1;
  for (int a = 0; a < g.D; ++a) g.Qv *= g.nq1;
  g.Qf = g.Qv / g.nq1;
  g.V = g.glm ? 9 : 8;
  g.ldf0 = g.glm ? -1 : 5 * g.n;
  g.bz2d = -1;
  g.nrows = g.glm ? 9 * g.n : 5 * g.n + g.ndiv;
  if (!g.glm && g.D == 2) {
    g.bz2d = g.nrows;
    g.nrows += g.n;
  }
  g.nx = mesh->n[0];
  g.ny = mesh->n[1];
  g.nz = g.D == 3 ? mesh->n[2] : 1;
  g.ncell = (int64_t)g.nx * g.ny * g.nz;
  g.stride = (g.ncell + 31) / 32 * 32;
  g.dx = mesh->box_len / g.nx;
  g.gamma = gamma;
  return DG_OK;
}

// Host tables in the order Pv dPv Pf Lv dLv Lf L0 wv wf minv.
void host_tables(const Basis& B, const Geom& g, std::vector<double>* out10) {
  HostTables h;
  build_host_tables(B, g, h);
  out10[0] = h.Pv; out10[1] = h.dPv; out10[2] = h.Pf; out10[3] = h.Lv; out10[4] = h.dLv;
  out10[5] = h.Lf; out10[6] = h.L0; out10[7] = h.wv; out10[8] = h.wf; out10[9] = h.minv;
}

void Prof::begin(int k, cudaStream_t st) {
  launches[k] += 1;
  if (!on) return;
  while (pool.size() < used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    pool.push_back(e);
  }
  cudaEventRecord(pool[used], st);
  kind.push_back(k);
}

void Prof::end(int k, cudaStream_t st) {
  (void)k;
  if (!on || pool.size() < used + 2 || kind.size() * 2 != used + 2) return;
  cudaEventRecord(pool[used + 1], st);
  used += 2;
}

int Prof::collect() {
  if (cudaDeviceSynchronize() != cudaSuccess) return DG_E_CUDA;
  for (size_t i = 0; i + 1 < used; i += 2) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pool[i], pool[i + 1]) == cudaSuccess) ms[kind[i / 2]] += t;
  }
  used = 0;
  kind.clear();
  return DG_OK;
}

void Prof::reset() {
  for (int k = 0; k < KINDS; ++k) {
    launches[k] = 0;
    ms[k] = 0.0;
  }
  used = 0;
  kind.clear();
}

void Prof::release() {
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
  reset();
}

}  // namespace dgmhd

extern "C" {

int dg_mhd_profile(dg_mhd_ctx* ctx, int enable) {
  if (!ctx) return DG_E_ARG;
  ctx->c.prof.reset();
  ctx->c.prof.on = enable != 0;
  return DG_OK;
}

int dg_mhd_profile_read(dg_mhd_ctx* ctx, int kind, double* total_ms, int64_t* launches) {
  if (!ctx || kind < 0 || kind >= Prof::KINDS) return DG_E_ARG;
  int e = ctx->c.prof.collect();
  if (e) return e;
  if (total_ms) *total_ms = ctx->c.prof.ms[kind];
  if (launches) *launches = ctx->c.prof.launches[kind];
  return DG_OK;
}

int64_t dg_mhd_launch_count(const dg_mhd_ctx* ctx) {
  if (!ctx) return 0;
  int64_t s = 0;
  for (int k = 0; k < Prof::KINDS; ++k) s += ctx->c.prof.launches[k];
  return s;
}

void dg_mhd_default_params(dg_mhd_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->cfl = 0.3;
  p->cfl_glm = 0.9;
  p->c_r = 0.18;
  p->c_h_fixed = 0.0;
  p->eta_powell = 0.2;
  p->eps_hlld = 1e-8;
  p->Mtilde = 5.0;
  p->beta = 2.0;
  p->tvb_eps = 1e-8;
  p->eps_rho = 1e-12;
  p->eps_p = 1e-12;
  p->precision = DG_PREC_FP64;
  p->limiter = DG_LIMIT_OFF;
  p->positivity = 0;
  p->rk_order = 3;
  p->powell_q = 0;
}

const char* dg_mhd_strerror(int s) {
  switch (s) {
    case DG_OK: return "ok";
    case DG_E_ARG: return "invalid argument";
    case DG_E_MESH: return "invalid mesh";
    case DG_E_CUDA: return "CUDA runtime error";
    case DG_E_NONFINITE: return "non-finite state or timestep";
    case DG_E_CH: return "GLM c_h below the signal speed";
    case DG_E_TIMEOUT: return "bounded device wait timed out";
    case DG_E_UNSUPPORTED: return "unsupported configuration";
    case DG_W_FLOOR: return "positivity floor injected mass or energy";
    default: return "unknown status";
  }
}

void dg_mhd_destroy(dg_mhd_ctx* ctx) {
  if (!ctx) return;
  Ctx& c = ctx->c;
  c.prof.release();
  free_amr(c);
  free_fast_tabs(c);
  free_tables(c.t64);
  free_tables(c.t32);
  void* ptrs[] = {c.sc, c.face_buf, c.face_buf32, c.stage_buf[0], c.stage_buf[1], c.stage_buf[2],
                  c.stage_mean[0], c.stage_mean[1], c.stage_mean[2], c.cellscratch, c.proj_tab, c.proj_w,
                  c.troubled, c.flag_list, c.pos_list, c.mlp_w1, c.mlp_w2, c.mlp_bias, c.rg_tabs, c.qdag_buf,
                  c.tc_tabs, c.owned};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c.hb;
  delete ctx;
}

int dg_mhd_init(const dg_mesh_desc* mesh, int degree, int divB_scheme, double gamma, const dg_mhd_params* p,
                dg_mhd_ctx** out) {
  if (!mesh || !out) return DG_E_ARG;
  *out = nullptr;
  if (mesh->dim != 2 && mesh->dim != 3) return DG_E_MESH;
  if (!mesh->periodic) return DG_E_UNSUPPORTED;
  if (degree < 0 || degree > MAXD) return DG_E_UNSUPPORTED;
  if (divB_scheme != DG_DIVB_POWELL && divB_scheme != DG_DIVB_GLM) return DG_E_ARG;
  if (!(gamma > 1.0)) return DG_E_ARG;
  const bool octree = mesh->level != nullptr;
  if (octree && !mesh->ijk) return DG_E_MESH;
  if (mesh->partial != 0 && (mesh->partial != 1 || !octree)) return DG_E_ARG;
  if (!octree)
    for (int a = 0; a < mesh->dim; ++a)
      if (mesh->n[a] < 1) return DG_E_MESH;
  if (!(mesh->box_len > 0.0)) return DG_E_MESH;
  {
    // cell indices are 32-bit inside the kernels
    const int64_t cells = octree ? mesh->n_leaves
                                 : (int64_t)mesh->n[0] * mesh->n[1] * (mesh->dim == 3 ? mesh->n[2] : 1);
    if (cells < 1 || cells > (int64_t)INT32_MAX - 64) return DG_E_MESH;
  }
  dg_mhd_params prm;
  if (p) prm = *p;
  else dg_mhd_default_params(&prm);
  if (prm.precision != DG_PREC_FP64 && prm.precision != DG_PREC_FP32MIX) return DG_E_ARG;
  if (!(prm.cfl > 0.0) || !(prm.cfl_glm > 0.0)) return DG_E_ARG;
  if (prm.rk_order < 0 || prm.rk_order > 4) return DG_E_ARG;
  if (prm.powell_q != 0 && prm.powell_q != 1) return DG_E_ARG;
  if (!(prm.eps_hlld >= 0.0 && prm.eps_hlld < 1.0)) return DG_E_ARG;
  if (prm.rk_order == 0) prm.rk_order = degree + 1 < 4 ? degree + 1 : 4;
  // octree meshes: a global, time-independent c_h (Sec. 4.1.5)
  if (octree && divB_scheme == DG_DIVB_GLM && !(prm.c_h_fixed > 0.0)) return DG_E_ARG;

  dg_mhd_ctx* ctx = new (std::nothrow) dg_mhd_ctx();
  if (!ctx) return DG_E_ARG;
  Ctx& c = ctx->c;
  c.p = prm;
  Geom& g = c.g;
  g.D = mesh->dim;
  g.d = degree;
  g.glm = divB_scheme == DG_DIVB_GLM;
  c.hb = new Basis();
  if (!c.hb->build(g.D, degree, !g.glm)) {
    dg_mhd_destroy(ctx);
    return DG_E_UNSUPPORTED;
  }
  g.n = c.hb->n;
  g.ndiv = c.hb->ndiv;
  g.DB = g.D;
  g.nq1 = degree + 1;
  g.Qv = 1;
  for (int a = 0; a < g.D; ++a) g.Qv *= g.nq1;
  g.Qf = g.Qv / g.nq1;
  g.V = g.glm ? 9 : 8;
  if (g.glm) {
    g.nrows = 9 * g.n;
    g.ldf0 = -1;
    g.bz2d = -1;
  } else {
    g.ldf0 = 5 * g.n;
    g.nrows = 5 * g.n + g.ndiv;
    g.bz2d = -1;
    if (g.D == 2) {
      g.bz2d = g.nrows;
      g.nrows += g.n;
    }
  }
  g.nx = octree ? 1 : mesh->n[0];
  g.ny = octree ? 1 : mesh->n[1];
  g.nz = octree ? 1 : (g.D == 3 ? mesh->n[2] : 1);
  g.ncell = octree ? mesh->n_leaves : (int64_t)g.nx * g.ny * g.nz;
  g.stride = (g.ncell + 31) / 32 * 32;
  g.dx = octree ? mesh->box_len : mesh->box_len / g.nx;
  g.gamma = gamma;
  if (octree) {
    const int e = build_amr(c, mesh);
    if (e) {
      dg_mhd_destroy(ctx);
      return e;
    }
  }

  HostTables h;
  build_host_tables(*c.hb, g, h);
  int e;
  if ((e = upload_tables(h, c.t64)) || (e = upload_tables(h, c.t32))) {
    dg_mhd_destroy(ctx);
    return e;
  }
  const size_t esz = fp32(c) ? sizeof(float) : sizeof(double);
  const size_t state_bytes = (size_t)g.nrows * g.stride * esz;
  // Powell / LDF specialised kernels: 10 face-buffer slots per face point
  const bool pow_fast = !g.glm && g.D == 3 && (degree == 1 || degree == 2) && prm.generic_kernels != 1 &&
                        prm.powell_q != 1;
  size_t face_pts = (size_t)g.D * g.stride * g.Qf;
  if (c.amr.on) face_pts = std::max(face_pts, (size_t)c.amr.nface * g.Qf);
  const size_t face_elems = face_pts * (pow_fast ? 10 : 9);
  bool ok = cudaMalloc(&c.sc, sizeof(DevScalars)) == cudaSuccess &&
            cudaMemset(c.sc, 0, sizeof(DevScalars)) == cudaSuccess &&
            cudaMalloc(&c.stage_buf[0], state_bytes) == cudaSuccess &&
            cudaMalloc(&c.stage_buf[1], state_bytes) == cudaSuccess &&
            cudaMalloc(&c.troubled, (size_t)g.stride) == cudaSuccess &&
            cudaMalloc(&c.flag_list, (size_t)g.stride * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&c.pos_list, (size_t)g.stride * sizeof(int32_t)) == cudaSuccess;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
      c.nsm = nsm;
  }
  if (ok) {
    if (fp32(c)) {
      ok = cudaMalloc(&c.face_buf32, face_elems * sizeof(float)) == cudaSuccess &&
           cudaMalloc(&c.stage_mean[0], (size_t)9 * g.stride * sizeof(double)) == cudaSuccess &&
           cudaMalloc(&c.stage_mean[1], (size_t)9 * g.stride * sizeof(double)) == cudaSuccess;
    } else {
      ok = cudaMalloc(&c.face_buf, face_elems * sizeof(double)) == cudaSuccess;
    }
    // Powell q^dagger of eq. powellq-interp: 14 values per face point
    if (ok && prm.powell_q == 1 && !g.glm)
      ok = cudaMalloc(&c.qdag_buf, face_pts * 14 * (fp32(c) ? sizeof(float) : sizeof(double))) == cudaSuccess;
  }
  if (!ok) {
    dg_mhd_destroy(ctx);
    return DG_E_CUDA;
  }
  upload_limiter_tables(c);
  mlp_build_tables(c);
  // specialised Powell / LDF kernels for uniform 3D meshes (not the q^dagger variant)
  if (pow_fast) {
    if (fp32(c)) {
      if (degree == 1) c.fast_tabs = make_fast_tabs<float, 1>(h, g, *c.hb);
      if (degree == 2) c.fast_tabs = make_fast_tabs<float, 2>(h, g, *c.hb);
      if (c.fast_tabs) c.fast = 10 + degree;
    } else {
      if (degree == 1) c.fast_tabs = make_fast_tabs<double, 1>(h, g, *c.hb);
      if (degree == 2) c.fast_tabs = make_fast_tabs<double, 2>(h, g, *c.hb);
      if (c.fast_tabs) c.fast = 20 + degree;
    }
    if (c.fast && !fast_pow_ok(c)) free_fast_tabs(c);
  }
  // specialised GLM kernels for uniform 3D meshes
  if (g.glm && g.D == 3 && prm.generic_kernels != 1 && !c.amr.on) {
    if (fp32(c)) {
      if (degree == 1) c.fast_tabs = make_fast_tabs<float, 1>(h, g, *c.hb);
      if (degree == 2) c.fast_tabs = make_fast_tabs<float, 2>(h, g, *c.hb);
      // degree 3: FP32 only (the FP64 tables exceed the constant bank)
      if (degree == 3) c.fast_tabs = make_fast_tabs<float, 3>(h, g, *c.hb);
      if (c.fast_tabs) c.fast = 10 + degree;
      // degree 2, on request: the cell update's contractions on the tensor
      // core (operand tables in device memory, staged into shared memory by
      // each block). Not the default: the contractions are too small for the
      // tensor core's per-instruction cost on this GPU (see dg_cell_tc.cu)
      if (c.fast == 12 && prm.generic_kernels == 2) {
        std::vector<float> tt;
        build_tc_tables(h.Pv, h.dPv, h.Pf, h.wv, h.wf, tt);
        if (cudaMalloc(&c.tc_tabs, tt.size() * sizeof(float)) != cudaSuccess ||
            cudaMemcpy(c.tc_tabs, tt.data(), tt.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
          dg_mhd_destroy(ctx);
          return DG_E_CUDA;
        }
      }
    } else {
      if (degree == 1) c.fast_tabs = make_fast_tabs<double, 1>(h, g, *c.hb);
      if (degree == 2) c.fast_tabs = make_fast_tabs<double, 2>(h, g, *c.hb);
      if (c.fast_tabs) c.fast = 20 + degree;
    }
  }
  // initial GLM speeds: fixed c_h if given (damping from c_r), else set by dt
  if (g.glm && prm.c_h_fixed > 0.0) {
    launch_set_glm(c.sc, prm.c_h_fixed, prm.c_h_fixed / prm.c_r, nullptr);
    c.glm_speeds_set = true;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    dg_mhd_destroy(ctx);
    return DG_E_CUDA;
  }
  *out = ctx;
  return DG_OK;
}

int dg_mhd_state_layout(const dg_mhd_ctx* ctx, int64_t* n_rows, int64_t* n_mean_rows, int64_t* n_cells,
                        int64_t* cell_stride) {
  if (!ctx) return DG_E_ARG;
  const Geom& g = ctx->c.g;
  if (n_rows) *n_rows = g.nrows;
  if (n_mean_rows) *n_mean_rows = g.glm ? 9 : 8;
  if (n_cells) *n_cells = g.ncell;
  if (cell_stride) *cell_stride = g.stride;
  return DG_OK;
}

int dg_mhd_project(dg_mhd_ctx* ctx, const double* nodal, int npts, void* w, double* wmean, void* stream) {
  if (!ctx || !nodal || !w || npts < 1 || npts > 8) return DG_E_ARG;
  Ctx& c = ctx->c;
  const Geom& g = c.g;
  if (fp32(c) && !wmean) return DG_E_ARG;
  if (npts != c.proj_npts) {
    // table[(r*Qp + q)*3 + k] = k-th active component of row r at point q
    std::vector<double> x1, w1;
    gauss_legendre(npts, x1, w1);
    int Qp = 1;
    for (int a = 0; a < g.D; ++a) Qp *= npts;
    std::vector<double> tab((size_t)g.nrows * Qp * 3, 0.0), wq(Qp, 1.0);
    double xi[3];
    for (int q = 0; q < Qp; ++q) {
      int qq = q;
      for (int a = 0; a < g.D; ++a) {
        wq[q] *= w1[qq % npts];
        qq /= npts;
      }
      vol_point(g.D, x1, q, xi);
      for (int r = 0; r < g.nrows; ++r) {
        double* t = &tab[((size_t)r * Qp + q) * 3];
        if (g.ldf0 >= 0 && r >= g.ldf0 && r < g.ldf0 + g.ndiv) {
          for (int k = 0; k < g.DB; ++k) t[k] = c.hb->eval(c.hb->ldf[r - g.ldf0][k], xi);
        } else {
          const int l = (g.bz2d >= 0 && r >= g.bz2d) ? r - g.bz2d : r % g.n;
          t[0] = c.hb->eval(c.hb->leg[l], xi);
        }
      }
    }
    if (c.proj_tab) cudaFree(c.proj_tab);
    if (c.proj_w) cudaFree(c.proj_w);
    c.proj_tab = nullptr;
    c.proj_w = nullptr;
    if (upload(&c.proj_tab, tab) || upload(&c.proj_w, wq)) return DG_E_CUDA;
    c.proj_npts = npts;
  }
  c.prof.launches[4] += 1;
  if (fp32(c))
    launch_project<float>(g, npts, c.proj_tab, c.proj_w, nodal, c.t32.minv, (float*)w, wmean, S(stream));
  else
    launch_project<double>(g, npts, c.proj_tab, c.proj_w, nodal, c.t64.minv, (double*)w, nullptr, S(stream));
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
}

int dg_mhd_set_glm(dg_mhd_ctx* ctx, double c_h, double damping_rate, void* stream) {
  if (!ctx || !(c_h > 0.0) || !(damping_rate >= 0.0)) return DG_E_ARG;
  launch_set_glm(ctx->c.sc, c_h, damping_rate, S(stream));
  ctx->c.glm_speeds_set = true;
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
}

namespace {

// rhs (combine = 0) or SSP stage out = ca*w0 + cb*(w + dt*L(w)) (combine = 1)
int operator_pass(Ctx& c, const void* w, const double* wmean, void* out, double* outmean, const void* w0,
                  const double* w0mean, double ca, double cb, int combine, cudaStream_t st) {
  const Geom& g = c.g;
  if (c.amr.on && c.amr.fast && c.fast) {
    // specialised Powell kernels over the face list: face pass, then cell pass
#define LISTCASE(code, T, DEG, OP, FB, WM, W0M, OM)                                                         \
  case code: {                                                                                              \
    const auto o = OP(c);                                                                                   \
    c.prof.begin(0, st);                                                                                    \
    launch_face_list_pow<T, DEG>(o, g.gamma, (const T*)w, FB, c.p.eps_hlld, st);                           \
    c.prof.end(0, st);                                                                                      \
    c.prof.begin(1, st);                                                                                    \
    launch_cell_list_pow<T, DEG>(o, g.gamma, (const T*)w, FB, (T*)out, (const T*)w0, ca, cb, combine, c.sc, \
                                 WM, W0M, OM, st);                                                          \
    c.prof.end(1, st);                                                                                      \
    break;                                                                                                  \
  }
    switch (c.fast) {
      LISTCASE(11, float, 1, oct_pow32, c.face_buf32, wmean, w0mean, outmean)
      LISTCASE(12, float, 2, oct_pow32, c.face_buf32, wmean, w0mean, outmean)
      LISTCASE(21, double, 1, oct_pow64, c.face_buf, nullptr, nullptr, nullptr)
      LISTCASE(22, double, 2, oct_pow64, c.face_buf, nullptr, nullptr, nullptr)
    }
#undef LISTCASE
    return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
  }
  if (c.amr.on) {
    c.prof.begin(1, st);
    if (fp32(c))
      launch_amr_operator<float>(c, c.t32, (const float*)w, c.face_buf32, (float*)out, (const float*)w0, ca, cb,
                                 combine, c.sc, wmean, w0mean, outmean, c.p.eps_hlld, st, (float*)c.qdag_buf);
    else
      launch_amr_operator<double>(c, c.t64, (const double*)w, c.face_buf, (double*)out, (const double*)w0, ca, cb,
                                  combine, c.sc, nullptr, nullptr, nullptr, c.p.eps_hlld, st, (double*)c.qdag_buf);
    c.prof.end(1, st);
    c.prof.launches[1] += 1;
    return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
  }
  if (c.fast) {
    const FastGeom fg = fast_geom(g);
#define FASTCASE(code, T, DEG, FB)                                                                          \
  case code: {                                                                                              \
    const auto& ft = *(const FastAll<T, DEG>*)c.fast_tabs;                                                \
    c.prof.begin(0, st);                                                                                    \
    if (g.glm) launch_face_glm<T, DEG>(ft, fg, (const T*)w, FB, c.sc, c.p.eps_hlld, st);                    \
    else face_pow_fast<T, DEG>(ft, fg, (const T*)w, FB, c.p.eps_hlld, st);                                  \
    c.prof.end(0, st);                                                                                      \
    c.prof.begin(1, st);                                                                                    \
    if (!g.glm)                                                                                             \
      cell_pow_fast<T, DEG>(ft, fg, (const T*)w, FB, (T*)out, (const T*)w0, ca, cb, combine, c.sc, wmean,   \
                            w0mean, outmean, st);                                                           \
    else if (!launch_cell_fast<T, DEG>(c, ft, fg, (const T*)w, FB, (T*)out, (const T*)w0, ca, cb, combine, \
                                       wmean, w0mean, outmean, st))                                         \
      launch_cell_glm<T, DEG>(ft, fg, (const T*)w, FB, (T*)out, (const T*)w0, ca, cb, combine, c.sc, wmean, \
                              w0mean, outmean, st);                                                         \
    c.prof.end(1, st);                                                                                      \
    break;                                                                                                  \
  }
    switch (c.fast) {
      FASTCASE(11, float, 1, c.face_buf32)
      FASTCASE(12, float, 2, c.face_buf32)
      FASTCASE(13, float, 3, c.face_buf32)
      FASTCASE(21, double, 1, c.face_buf)
      FASTCASE(22, double, 2, c.face_buf)
    }
#undef FASTCASE
    return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
  }
  if (fp32(c)) {
    c.prof.begin(0, st);
    launch_face<float>(g, c.t32, (const float*)w, c.face_buf32, c.sc, c.p.eps_hlld, st, (float*)c.qdag_buf);
    c.prof.end(0, st);
    c.prof.begin(1, st);
    launch_cell<float>(g, c.t32, (const float*)w, c.face_buf32, (float*)out, (const float*)w0, ca, cb, combine,
                       c.sc, wmean, w0mean, outmean, st, (const float*)c.qdag_buf);
    c.prof.end(1, st);
  } else {
    c.prof.begin(0, st);
    launch_face<double>(g, c.t64, (const double*)w, c.face_buf, c.sc, c.p.eps_hlld, st, (double*)c.qdag_buf);
    c.prof.end(0, st);
    c.prof.begin(1, st);
    launch_cell<double>(g, c.t64, (const double*)w, c.face_buf, (double*)out, (const double*)w0, ca, cb,
                        combine, c.sc, nullptr, nullptr, nullptr, st, (const double*)c.qdag_buf);
    c.prof.end(1, st);
  }
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
}

// Powell face jumps of the timestep by the specialised kernel (uniform 3D,
// degrees 1 and 2); false: the caller runs the generic one
bool divb_face_fast(Ctx& c, const void* w, cudaStream_t st) {
  const FastGeom fg = fast_geom(c.g);
  switch (c.fast) {
    case 11: launch_divb_face_pow<float, 1>(fg, (const float*)w, c.face_buf32, st); return true;
    case 12: launch_divb_face_pow<float, 2>(fg, (const float*)w, c.face_buf32, st); return true;
    case 21: launch_divb_face_pow<double, 1>(fg, (const double*)w, c.face_buf, st); return true;
    case 22: launch_divb_face_pow<double, 2>(fg, (const double*)w, c.face_buf, st); return true;
  }
  return false;
}

int dt_pass(Ctx& c, const void* w, const double* wmean, double* dt_out, cudaStream_t st) {
  const Geom& g = c.g;
  if (g.glm) c.glm_speeds_set = true;  // the finalize kernel derives c_h and the damping from dt
  if (c.amr.on) {
    c.prof.begin(2, st);
    launch_dt_init(c.sc, st);
    if (fp32(c)) launch_amr_dt<float>(c, c.t32, (const float*)w, wmean, c.face_buf32, c.p, c.sc, st);
    else launch_amr_dt<double>(c, c.t64, (const double*)w, nullptr, c.face_buf, c.p, c.sc, st);
    launch_dt_finalize(g, c.p, c.sc, dt_out, st);
    c.prof.end(2, st);
    // k_dt_init, the jump kernel (Powell), k_dt_list (FP32 form: k_dt_list32 + its refine), k_dt_finalize
    c.prof.launches[2] += (g.glm ? 2 : 3) + (fp32(c) ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
  }
  c.prof.begin(2, st);
  // the specialised Powell jump kernel stores two sums per face (gj.jq = 1)
  Geom gj = g;
  if (!g.glm && divb_face_fast(c, w, st)) gj.jq = 1;
  if (fp32(c)) {
    if (!g.glm && !gj.jq) launch_divb_face<float>(g, c.t32, (const float*)w, c.face_buf32, st);
    launch_dt<float>(gj, c.t32, (const float*)w, wmean, c.face_buf32, c.p, c.sc, dt_out, st);
  } else {
    if (!g.glm && !gj.jq) launch_divb_face<double>(g, c.t64, (const double*)w, c.face_buf, st);
    launch_dt<double>(gj, c.t64, (const double*)w, nullptr, c.face_buf, c.p, c.sc, dt_out, st);
  }
  c.prof.end(2, st);
  // k_dt_init + k_dt + k_dt_finalize (FP32 form: k_dt32 + k_dt32_refine in place
  // of k_dt), + k_divb_face for Powell: count the launches beyond the first
  c.prof.launches[2] += (g.glm ? 2 : 3) + (fp32(c) ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
}

int limit_pass(Ctx& c, void* w, double* wmean, uint8_t* troubled, cudaStream_t st) {
  if (c.p.limiter == DG_LIMIT_OFF && !c.p.positivity) return DG_OK;
  // octree meshes: TVB with neighbour means across coarse-fine faces; the
  // learned detector reads the same side averages as its neighbour means
  return run_limiter(c, w, wmean, troubled, st);
}

}  // namespace

int dg_mhd_rhs(dg_mhd_ctx* ctx, const void* w, const double* wmean, void* rhs, double* rhs_mean, void* stream) {
  if (!ctx || !w || !rhs) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (fp32(c) && (!wmean || !rhs_mean)) return DG_E_ARG;
  return operator_pass(c, w, wmean, rhs, rhs_mean, nullptr, nullptr, 0.0, 1.0, 0, S(stream));
}

int dg_mhd_stage(dg_mhd_ctx* ctx, const void* w, const double* wmean, const void* u0, const double* u0mean,
                 void* out, double* outmean, double a, double b, void* stream) {
  if (!ctx || !w || !out || !std::isfinite(a) || !std::isfinite(b)) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (!u0) {
    if (a != 0.0) return DG_E_ARG;
    u0 = w;  // read but weighted by zero
    u0mean = wmean;
  }
  if (fp32(c) && (!wmean || !outmean || !u0mean)) return DG_E_ARG;
  return operator_pass(c, w, wmean, out, outmean, u0, u0mean, a, b, 1, S(stream));
}

int dg_mhd_set_dt(dg_mhd_ctx* ctx, const double* dt_dev, void* stream) {
  if (!ctx || !dt_dev) return DG_E_ARG;
  Ctx& c = ctx->c;
  c.prof.launches[2] += 1;
  launch_dt_from_value(c.g, c.p, dt_dev, c.sc, S(stream));
  c.glm_speeds_set = true;
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
}

int dg_mhd_glm_speeds(dg_mhd_ctx* ctx, double* c_h, double* damping_rate) {
  if (!ctx || !c_h || !damping_rate) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (cudaDeviceSynchronize() != cudaSuccess) return DG_E_CUDA;
  if (cudaMemcpy(c_h, &c.sc->ch, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(damping_rate, &c.sc->kappa, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DG_E_CUDA;
  return DG_OK;
}

int dg_mhd_set_owned(dg_mhd_ctx* ctx, const uint8_t* mask, void* stream) {
  if (!ctx) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (!mask) {
    c.g.owned = nullptr;
    return DG_OK;
  }
  if (!c.owned && cudaMalloc(&c.owned, (size_t)c.g.ncell) != cudaSuccess) {
    c.owned = nullptr;
    return DG_E_CUDA;
  }
  if (cudaMemcpyAsync(c.owned, mask, (size_t)c.g.ncell, cudaMemcpyDeviceToDevice, S(stream)) != cudaSuccess)
    return DG_E_CUDA;
  c.g.owned = c.owned;
  return DG_OK;
}

int dg_mhd_limit(dg_mhd_ctx* ctx, void* w, double* wmean, uint8_t* troubled, void* stream) {
  if (!ctx || !w) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (fp32(c) && !wmean) return DG_E_ARG;
  return limit_pass(c, w, wmean, troubled, S(stream));
}

int dg_mhd_dt(dg_mhd_ctx* ctx, const void* w, const double* wmean, double* dt_dev, void* stream) {
  if (!ctx || !w) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (fp32(c) && !wmean) return DG_E_ARG;
  return dt_pass(c, w, wmean, dt_dev, S(stream));
}

const double* dg_mhd_last_dt(const dg_mhd_ctx* ctx) {
  if (!ctx) return nullptr;
  return &ctx->c.sc->dt;
}

int dg_mhd_step(dg_mhd_ctx* ctx, void* w, double* wmean, const double* dt_dev, void* stream) {
  if (!ctx || !w) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (fp32(c) && !wmean) return DG_E_ARG;
  cudaStream_t st = S(stream);
  int e;
  if (dt_dev) {
    // the step's dt (and GLM c_h) first, so the limiter sees this step's c_h
    c.prof.launches[2] += 1;
    launch_dt_from_value(c.g, c.p, dt_dev, c.sc, st);
    c.glm_speeds_set = true;
    if ((e = limit_pass(c, w, wmean, nullptr, st))) return e;
  } else {
    // dt from the limited state; the limiter uses the c_h of the previous
    // step -- on a GLM context's first step, the c_h of the dt of the input
    // state (the characteristic GLM pair needs c_h > 0)
    if (c.g.glm && !c.glm_speeds_set && (c.p.limiter != DG_LIMIT_OFF || c.p.positivity) &&
        (e = dt_pass(c, w, wmean, nullptr, st)))
      return e;
    if ((e = limit_pass(c, w, wmean, nullptr, st))) return e;
    if ((e = dt_pass(c, w, wmean, nullptr, st))) return e;
  }
  void* s1 = c.stage_buf[0];
  void* s2 = c.stage_buf[1];
  double* m1 = c.stage_mean[0];
  double* m2 = c.stage_mean[1];
  const int order = c.p.rk_order;
  auto axpby = [&](double a, const void* x, const double* xm, double b, const void* y, const double* ym, void* o,
                   double* om) {
    c.prof.launches[1] += 1;
    if (fp32(c))
      launch_axpby<float>(c.g, a, (const float*)x, b, (const float*)y, (float*)o, xm, ym, om, st);
    else
      launch_axpby<double>(c.g, a, (const double*)x, b, (const double*)y, (double*)o, nullptr, nullptr, nullptr,
                           st);
  };
  if (order == 1) {
    // u^{n+1} = u + dt L(u), staged through s1
    if ((e = operator_pass(c, w, wmean, s1, m1, w, wmean, 0.0, 1.0, 1, st))) return e;
    axpby(1.0, s1, m1, 0.0, s1, m1, w, wmean);
    return DG_OK;
  }
  if (order == 2) {
    // u1 = u + dt L(u);  u^{n+1} = 1/2 u + 1/2 (u1 + dt L(u1))
    if ((e = operator_pass(c, w, wmean, s1, m1, w, wmean, 0.0, 1.0, 1, st))) return e;
    if ((e = limit_pass(c, s1, m1, nullptr, st))) return e;
    return operator_pass(c, s1, m1, w, wmean, w, wmean, 0.5, 0.5, 1, st);
  }
  if (order == 4) {
    // Ketcheson's SSPRK(10,4), two registers: q1 (ping-pong between w and s1)
    // and q2 (s2); every operator evaluation advances by dt/6.
    c.prof.launches[2] += 1;
    launch_dt_scale(c.sc, 1.0 / 6.0, st);
    axpby(1.0, w, wmean, 0.0, w, wmean, s2, m2);  // q2 = u
    void* q = w;
    double* qm = wmean;
    auto forward = [&](bool limit_first) -> int {
      void* o = q == w ? s1 : w;
      double* om = q == w ? m1 : wmean;
      int r;
      if (limit_first && (r = limit_pass(c, q, qm, nullptr, st))) return r;
      if ((r = operator_pass(c, q, qm, o, om, q, qm, 0.0, 1.0, 1, st))) return r;
      q = o;
      qm = om;
      return DG_OK;
    };
    for (int i = 0; i < 5; ++i)
      if ((e = forward(i > 0))) return e;
    axpby(1.0 / 25.0, s2, m2, 9.0 / 25.0, q, qm, s2, m2);  // q2 = q2/25 + 9 q1/25
    axpby(15.0, s2, m2, -5.0, q, qm, q, qm);              // q1 = 15 q2 - 5 q1
    for (int i = 0; i < 4; ++i)
      if ((e = forward(true))) return e;
    if ((e = limit_pass(c, q, qm, nullptr, st))) return e;
    // u^{n+1} = q2 + 3/5 q1 + dt/10 L(q1) = q2 + 3/5 (q1 + dt/6 L(q1)); q1 is in s1 here
    if ((e = operator_pass(c, q, qm, w, wmean, s2, m2, 1.0, 0.6, 1, st))) return e;
    c.prof.launches[2] += 1;
    launch_dt_scale(c.sc, 1.0, st);
    return DG_OK;
  }
  // u1 = u + dt L(u)
  if ((e = operator_pass(c, w, wmean, s1, m1, w, wmean, 0.0, 1.0, 1, st))) return e;
  if ((e = limit_pass(c, s1, m1, nullptr, st))) return e;
  // u2 = 3/4 u + 1/4 (u1 + dt L(u1))
  if ((e = operator_pass(c, s1, m1, s2, m2, w, wmean, 0.75, 0.25, 1, st))) return e;
  if ((e = limit_pass(c, s2, m2, nullptr, st))) return e;
  // u^{n+1} = 1/3 u + 2/3 (u2 + dt L(u2))
  if ((e = operator_pass(c, s2, m2, w, wmean, w, wmean, 1.0 / 3.0, 2.0 / 3.0, 1, st))) return e;
  return DG_OK;
}

int dg_mhd_mlp_features(dg_mhd_ctx* ctx, const void* w, const double* wmean, float* X, int ldx, void* stream) {
  if (!ctx || !w || !X) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (fp32(c) && !wmean) return DG_E_ARG;
  if (ldx < 8 * c.g.n + 2 * c.g.D) return DG_E_ARG;
  c.prof.launches[3] += 1;
  return mlp_features_launch(c, w, wmean, X, ldx, S(stream));
}

int dg_mhd_mlp_set_weights(dg_mhd_ctx* ctx, const float* theta, int nin, float threshold) {
  if (!ctx || !theta || !(threshold > 0.f && threshold < 1.f)) return DG_E_ARG;
  return mlp_set_weights(ctx->c, theta, nin, threshold);
}

int dg_mhd_mlp_infer(dg_mhd_ctx* ctx, const void* w, const double* wmean, uint8_t* flags, float* prob,
                     void* stream) {
  if (!ctx || !w) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (fp32(c) && !wmean) return DG_E_ARG;
  c.prof.launches[3] += 1;
  return mlp_infer_launch(c, w, wmean, flags, prob, S(stream));
}

int dg_mhd_mlp_loss_grad(const float* X, int ldx, const uint8_t* y, int64_t n, int nin, const float* theta,
                         float pos_weight, float* grad, double* loss, void* stream) {
  if (!X || !y || !theta || !grad || n < 1 || nin < 1 || ldx < nin || n > (int64_t)1 << 30) return DG_E_ARG;
  void* scratch = nullptr;
  if (cudaMalloc(&scratch, mlp_scratch_bytes((int)n)) != cudaSuccess) return DG_E_CUDA;
  cudaStream_t st = S(stream);
  if (loss) cudaMemsetAsync(loss, 0, sizeof(double), st);
  int e = mlp_loss_grad_dev(X, ldx, y, nullptr, 0, (int)n, nin, theta, grad, loss, pos_weight, (float)n, scratch, st);
  cudaStreamSynchronize(st);
  cudaFree(scratch);
  return e;
}

int dg_mhd_mlp_train(const float* X, int ldx, const uint8_t* y, int64_t n, int nin, float* theta, int epochs,
                     int batch, float lr, float pos_weight, uint64_t seed, double* last_loss, void* stream) {
  if (!X || !y || !theta || n < batch || batch < 1 || epochs < 1 || ldx < nin) return DG_E_ARG;
  return mlp_train_dev(X, ldx, y, n, nin, theta, epochs, batch, lr, pos_weight, seed, last_loss, S(stream));
}

int dg_mhd_counters(dg_mhd_ctx* ctx, int64_t* pos_cells, double* inj_mass, double* inj_energy, int reset) {
  if (!ctx) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (cudaDeviceSynchronize() != cudaSuccess) return DG_E_CUDA;
  DevScalars h;
  if (cudaMemcpy(&h, c.sc, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return DG_E_CUDA;
  if (pos_cells) *pos_cells = (int64_t)h.pos_cells;
  if (inj_mass) *inj_mass = h.inj_mass;
  if (inj_energy) *inj_energy = h.inj_energy;
  if (reset) {
    h.pos_cells = 0;
    h.inj_mass = h.inj_energy = 0.0;
    if (cudaMemcpy(c.sc, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) return DG_E_CUDA;
  }
  return DG_OK;
}

int dg_mhd_ldf_legendre(int degree, int64_t cap, double* A, int* n_div, int* n_modes) {
  if (degree < 0 || degree > MAXD) return DG_E_ARG;
  std::vector<double> M;
  int nd = 0, nm = 0;
  if (!ldf_legendre_3d(degree, M, nd, nm)) return DG_E_UNSUPPORTED;
  if (n_div) *n_div = nd;
  if (n_modes) *n_modes = nm;
  if (A) {
    if (cap < (int64_t)M.size()) return DG_E_ARG;
    std::copy(M.begin(), M.end(), A);
  }
  return DG_OK;
}

int dg_mhd_positivity_listed(dg_mhd_ctx* ctx, int64_t* listed, int reset) {
  if (!ctx || !listed) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (cudaDeviceSynchronize() != cudaSuccess) return DG_E_CUDA;
  unsigned long long v = 0;
  if (cudaMemcpy(&v, &c.sc->cnt_poslisted, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return DG_E_CUDA;
  *listed = (int64_t)v;
  if (reset && cudaMemset(&c.sc->cnt_poslisted, 0, sizeof(v)) != cudaSuccess) return DG_E_CUDA;
  return DG_OK;
}

int dg_mhd_divb(dg_mhd_ctx* ctx, const void* w, const double* wmean, double* res, double* per_cell,
                void* stream) {
  if (!ctx || !w || !res) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (fp32(c) && !wmean) return DG_E_ARG;
  if (c.amr.on) return DG_E_UNSUPPORTED;
  c.prof.launches[2] += 2;
  if (fp32(c))
    launch_divb_diag<float>(c.g, c.t32, (const float*)w, wmean, reinterpret_cast<double*>(c.face_buf32), res,
                            per_cell, S(stream));
  else
    launch_divb_diag<double>(c.g, c.t64, (const double*)w, nullptr, c.face_buf, res, per_cell, S(stream));
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
}

int dg_mhd_limiter_counts(dg_mhd_ctx* ctx, int64_t* passes, int64_t* flagged, int64_t* limited, int reset) {
  if (!ctx) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (cudaDeviceSynchronize() != cudaSuccess) return DG_E_CUDA;
  DevScalars h;
  if (cudaMemcpy(&h, c.sc, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return DG_E_CUDA;
  if (passes) *passes = c.lim_passes;
  if (flagged) *flagged = (int64_t)h.cnt_flagged + c.lim_plain_cells;
  if (limited) *limited = (int64_t)h.cnt_limited;
  if (reset) {
    h.cnt_flagged = h.cnt_limited = 0;
    c.lim_passes = c.lim_plain_cells = 0;
    if (cudaMemcpy(c.sc, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) return DG_E_CUDA;
  }
  return DG_OK;
}

int dg_mhd_status(dg_mhd_ctx* ctx, int sync) {
  if (!ctx) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (sync && cudaDeviceSynchronize() != cudaSuccess) return DG_E_CUDA;
  int st = 0, fl = 0;
  if (cudaMemcpy(&st, &c.sc->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DG_E_CUDA;
  if (cudaMemcpy(&fl, &c.sc->floor_used, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DG_E_CUDA;
  if (sync) {
    int z = 0;
    cudaMemcpy(&c.sc->status, &z, sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(&c.sc->floor_used, &z, sizeof(int), cudaMemcpyHostToDevice);
  }
  if (st & 1) return DG_E_NONFINITE;
  if (st & 4) return DG_E_CH;
  if (st & 8) return DG_E_TIMEOUT;
  if (st & 16) return DG_E_ARG;  // a device-side argument check failed (remap sources)
  if (fl) return DG_W_FLOOR;
  return DG_OK;
}

}  // extern "C"
