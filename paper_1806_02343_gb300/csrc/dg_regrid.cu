// Dynamic regridding of octree meshes (Sec. 5, adaptive mesh refinement):
// the smoothness indicator S_a(u) = sum_{k=1..d} 2^(2k-1) int (d^k u/dxi_a^k)^2
// over the reference cell, refinement marks (refine a leaf if S_a(u) > 2 S~ for
// some monitored field u and direction a; coarsen a group of sibling leaves if
// the restriction of the group has S_a(u) < S~/2 for all), the new 2:1-balanced
// leaf list, and the remap of the state by L2 prolongation (parent octant onto
// the child's basis) and restriction (the children onto the parent's basis) --
// per variable for the Legendre rows, under the vector inner product of eq.
// innerp for the LDF rows.
//
// Tables (double, built here from the library's basis): S_a as quadratic forms
// of a field's coefficients, QL[a][l][l'] for a Legendre variable and
// QB[c][a][j][j'] for the B component c of the LDF rows; the prolongation
// blocks PL[o][l][l'], PB[o][j][j'] (child row from parent row) and the
// restriction blocks RL[o][l][l'], RB[o][j][j'] (parent row from child o's
// row). Octant o: bit a set = upper half along axis a; child point xi maps to
// the parent's (xi + s)/2, s_a = +1 or -1. All integrands are polynomials of
// degree <= 2d: the Gauss rule with d+1 points per dimension is exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/dg_mhd.h"
#include "dg_amr.cuh"
#include "dg_basis.h"

namespace dgmhd {

namespace {

// k-th derivative along `axis` of a basis polynomial at x
double deriv_k(const Basis& B, const std::vector<double>& poly, int axis, int k, const double* x) {
  double s = 0.0;
  for (size_t i = 0; i < B.ms.exps.size(); ++i) {
    const double c = poly[i];
    if (c == 0.0) continue;
    const auto& e = B.ms.exps[i];
    if (e[axis] < k) continue;
    double t = c;
    for (int j = 0; j < k; ++j) t *= (double)(e[axis] - j);
    for (int b = 0; b < B.D; ++b) {
      const int p = e[b] - (b == axis ? k : 0);
      for (int j = 0; j < p; ++j) t *= x[b];
    }
    s += t;
  }
  return s;
}

// tensor Gauss rule with d+1 points per dimension (last axis fastest)
void gauss_tensor(int D, int npts, std::vector<std::array<double, 3>>& pts, std::vector<double>& wts) {
  std::vector<double> x, w;
  gauss_legendre(npts, x, w);
  int total = 1;
  for (int a = 0; a < D; ++a) total *= npts;
  pts.assign(total, {0.0, 0.0, 0.0});
  wts.assign(total, 1.0);
  for (int q = 0; q < total; ++q) {
    int r = q;
    for (int a = D - 1; a >= 0; --a) {
      pts[q][a] = x[r % npts];
      wts[q] *= w[r % npts];
      r /= npts;
    }
  }
}

}  // namespace

// Layout of the regridding tables in one device buffer (offsets in doubles).
struct RgLayout {
  int n = 0, nd = 0, D = 3, no = 8;
  size_t QL = 0, QB = 0, PL = 0, PB = 0, RL = 0, RB = 0, total = 0;
  void set(int D_, int n_, int nd_) {
    D = D_, n = n_, nd = nd_, no = 1 << D;
    QL = 0;
    QB = QL + (size_t)D * n * n;
    PL = QB + (size_t)D * D * nd * nd;
    PB = PL + (size_t)no * n * n;
    RL = PB + (size_t)no * nd * nd;
    RB = RL + (size_t)no * n * n;
    total = RB + (size_t)no * nd * nd;
  }
};

// Host tables of the context's basis; true on success.
bool regrid_tables(const Basis& B, std::vector<double>& tab, RgLayout& L) {
  const int D = B.D, d = B.d, n = B.n, nd = B.ndiv;
  L.set(D, n, nd);
  tab.assign(L.total, 0.0);
  std::vector<std::array<double, 3>> pts;
  std::vector<double> wts;
  gauss_tensor(D, d + 1, pts, wts);
  const int Q = (int)wts.size();
  // smoothness forms: sum_k 2^(2k-1) sum_q w_q d^k phi d^k phi'
  for (int a = 0; a < D; ++a) {
    for (int k = 1; k <= d; ++k) {
      const double fk = std::ldexp(1.0, 2 * k - 1);
      std::vector<double> vl((size_t)n * Q), vb((size_t)D * nd * Q);
      for (int q = 0; q < Q; ++q) {
        for (int l = 0; l < n; ++l) vl[(size_t)l * Q + q] = deriv_k(B, B.leg[l], a, k, pts[q].data());
        for (int c = 0; c < D; ++c)
          for (int j = 0; j < nd; ++j) vb[((size_t)c * nd + j) * Q + q] = deriv_k(B, B.ldf[j][c], a, k, pts[q].data());
      }
      for (int l = 0; l < n; ++l)
        for (int m = 0; m < n; ++m) {
          double s = 0.0;
          for (int q = 0; q < Q; ++q) s += wts[q] * vl[(size_t)l * Q + q] * vl[(size_t)m * Q + q];
          tab[L.QL + ((size_t)a * n + l) * n + m] += fk * s;
        }
      for (int c = 0; c < D; ++c)
        for (int j = 0; j < nd; ++j)
          for (int m = 0; m < nd; ++m) {
            double s = 0.0;
            for (int q = 0; q < Q; ++q)
              s += wts[q] * vb[((size_t)c * nd + j) * Q + q] * vb[((size_t)c * nd + m) * Q + q];
            tab[L.QB + (((size_t)c * D + a) * nd + j) * nd + m] += fk * s;
          }
    }
  }
  // prolongation: child row from parent row, <phi_parent((xi+s)/2), phi_child(xi)> / M_child
  for (int o = 0; o < L.no; ++o) {
    double s[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) s[a] = ((o >> a) & 1) ? 1.0 : -1.0;
    for (int q = 0; q < Q; ++q) {
      double xp[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) xp[a] = 0.5 * (pts[q][a] + s[a]);
      // basis values at the child point and at the mapped parent point
      std::vector<double> lc_v(n), lp_v(n), bc_v((size_t)nd * D), bp_v((size_t)nd * D);
      for (int l = 0; l < n; ++l) {
        lc_v[l] = B.eval(B.leg[l], pts[q].data());
        lp_v[l] = B.eval(B.leg[l], xp);
      }
      for (int j = 0; j < nd; ++j)
        for (int c = 0; c < D; ++c) {
          bc_v[(size_t)j * D + c] = B.eval(B.ldf[j][c], pts[q].data());
          bp_v[(size_t)j * D + c] = B.eval(B.ldf[j][c], xp);
        }
      for (int lc = 0; lc < n; ++lc)
        for (int lp = 0; lp < n; ++lp)
          tab[L.PL + ((size_t)o * n + lc) * n + lp] += wts[q] * lc_v[lc] * lp_v[lp] / B.leg_mass[lc];
      for (int jc = 0; jc < nd; ++jc)
        for (int jp = 0; jp < nd; ++jp) {
          double dot = 0.0;
          for (int c = 0; c < D; ++c) dot += bc_v[(size_t)jc * D + c] * bp_v[(size_t)jp * D + c];
          tab[L.PB + ((size_t)o * nd + jc) * nd + jp] += wts[q] * dot / B.ldf_mass[jc];
        }
    }
  }
  // restriction: parent row r from child o's row r' = 2^-D M_r' / M_r x prolongation(o)[r'][r]
  const double inv = 1.0 / (double)L.no;
  for (int o = 0; o < L.no; ++o) {
    for (int lp = 0; lp < n; ++lp)
      for (int lc = 0; lc < n; ++lc)
        tab[L.RL + ((size_t)o * n + lp) * n + lc] =
            inv * B.leg_mass[lc] / B.leg_mass[lp] * tab[L.PL + ((size_t)o * n + lc) * n + lp];
    for (int jp = 0; jp < nd; ++jp)
      for (int jc = 0; jc < nd; ++jc)
        tab[L.RB + ((size_t)o * nd + jp) * nd + jc] =
            inv * B.ldf_mass[jc] / B.ldf_mass[jp] * tab[L.PB + ((size_t)o * nd + jc) * nd + jp];
  }
  return true;
}

namespace {

constexpr int RG_MAXD = 50;  // LDF rows, degree <= 3

struct RgDev {
  const double* tab;
  int n, nd, D, no;
  size_t QL, QB, PL, PB, RL, RB;
};

// FP64 mean index of row r (mean rows: Legendre mode 0, the D degree-0 LDF
// rows, the 2D B_z mode 0), -1 for the other rows
__host__ __device__ __forceinline__ int rg_mean_index(const Geom& g, int r) {
  if (g.glm || r < 5 * g.n) return r % g.n == 0 ? r / g.n : -1;
  if (g.ldf0 >= 0 && r >= g.ldf0 && r < g.ldf0 + g.ndiv) return r - g.ldf0 < g.D ? 5 + (r - g.ldf0) : -1;
  if (g.bz2d >= 0 && r == g.bz2d) return 7;
  return -1;
}

// row r of cell c in FP64 (the FP64 mean where the row is a mean row)
template <typename T>
__device__ __forceinline__ double rg_val(const Geom& g, const T* w, const double* wmean, int r, int64_t c) {
  if (wmean) {
    const int m = rg_mean_index(g, r);
    if (m >= 0) return wmean[(int64_t)m * g.stride + c];
  }
  return (double)w[(int64_t)r * g.stride + c];
}

// field v: Legendre rows base .. base+n-1 (ldf = false) or, in the Powell form,
// B component v-5 of the LDF rows (ldf = true)
__device__ __forceinline__ bool rg_field(const Geom& g, int v, int* base) {
  if (g.glm || v < 5) {
    *base = v * g.n;
    return false;
  }
  if (g.D == 2 && v == 7) {
    *base = g.bz2d;
    return false;
  }
  *base = g.ldf0;
  return true;
}

// max over the directions of S_a for field v from its coefficients coef[]
__device__ double rg_smax(const Geom& g, const RgDev& L, int v, bool ldf, const double* coef) {
  double smax = 0.0;
  if (!ldf) {
    for (int a = 0; a < g.D; ++a) {
      const double* Q = L.tab + L.QL + (size_t)a * L.n * L.n;
      double s = 0.0;
      for (int l = 1; l < L.n; ++l) {  // mode 0 has no derivative
        double t = 0.0;
        for (int m = 1; m < L.n; ++m) t += Q[l * L.n + m] * coef[m];
        s += coef[l] * t;
      }
      smax = fmax(smax, s);
    }
  } else {
    const int cc = v - 5;
    for (int a = 0; a < g.D; ++a) {
      const double* Q = L.tab + L.QB + ((size_t)cc * L.D + a) * L.nd * L.nd;
      double s = 0.0;
      for (int j = g.D; j < L.nd; ++j) {  // the degree-0 rows have no derivative
        double t = 0.0;
        for (int m = g.D; m < L.nd; ++m) t += Q[j * L.nd + m] * coef[m];
        s += coef[j] * t;
      }
      smax = fmax(smax, s);
    }
  }
  return smax;
}

// s_max[c] = max over the monitored fields (bit v of mask) and directions of S_a
template <typename T>
__global__ void k_rg_smooth(Geom g, RgDev L, const T* __restrict__ w, const double* __restrict__ wmean, int mask,
                            double* __restrict__ s_max) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  double coef[RG_MAXD];
  double smax = 0.0;
  for (int v = 0; v < g.V; ++v) {
    if (!((mask >> v) & 1)) continue;
    int base;
    const bool ldf = rg_field(g, v, &base);
    const int cnt = ldf ? L.nd : L.n;
    for (int l = 0; l < cnt; ++l) coef[l] = rg_val(g, w, wmean, base + l, c);
    smax = fmax(smax, rg_smax(g, L, v, ldf, coef));
  }
  s_max[c] = smax;
}

// refinement marks of the leaves
__global__ void k_rg_marks_leaf(int64_t ncell, const int8_t* __restrict__ level, const double* __restrict__ s_max,
                                double s_tilde, int max_level, int8_t* __restrict__ marks) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  marks[c] = (s_max[c] > 2.0 * s_tilde && level[c] < max_level) ? 1 : 0;
}

// coarsening marks of the sibling groups: the restriction of the group must
// have S_a < S~/2 for every monitored field and direction
template <typename T>
__global__ void k_rg_marks_group(Geom g, RgDev L, const T* __restrict__ w, const double* __restrict__ wmean,
                                 int mask, const int32_t* __restrict__ groups, int64_t ngroups,
                                 const int8_t* __restrict__ level, double s_tilde, int min_level,
                                 int8_t* __restrict__ marks) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= ngroups) return;
  const int32_t* mem = groups + gi * L.no;
  if (level[mem[0]] - 1 < min_level) return;
  for (int o = 0; o < L.no; ++o)
    if (marks[mem[o]] == 1) return;
  double coef[RG_MAXD];
  for (int v = 0; v < g.V; ++v) {
    if (!((mask >> v) & 1)) continue;
    int base;
    const bool ldf = rg_field(g, v, &base);
    const int cnt = ldf ? L.nd : L.n;
    const double* R = L.tab + (ldf ? L.RB : L.RL);
    for (int l = 0; l < cnt; ++l) coef[l] = 0.0;
    for (int o = 0; o < L.no; ++o)
      for (int m = 0; m < cnt; ++m) {
        const double x = rg_val(g, w, wmean, base + m, (int64_t)mem[o]);
        if (x == 0.0) continue;
        for (int l = 0; l < cnt; ++l) coef[l] += R[((size_t)o * cnt + l) * cnt + m] * x;
      }
    if (rg_smax(g, L, v, ldf, coef) >= 0.5 * s_tilde) return;
  }
  for (int o = 0; o < L.no; ++o) marks[mem[o]] = -1;
}

// number of row blocks: the Legendre variables, then the LDF rows, then (2D
// Powell) the B_z Legendre rows
__host__ __device__ inline int rg_nblocks(const Geom& g) {
  return (g.glm ? 9 : 5) + (g.ldf0 >= 0 ? 1 : 0) + (g.bz2d >= 0 ? 1 : 0);
}

// new state: the rows of block b (blockIdx.y) of new cell i from its source
// (src[2i]: kind 0 copy, 1 prolongation, 2 restriction in bits 0-3, octant in
// bits 4-7; src[2i+1]: old cell, or old sibling group for a restriction). Each
// thread reads its sources once. Entries out of range are skipped and latch
// status bit 16 (DG_E_ARG).
template <typename T>
__global__ void k_rg_remap(Geom go, Geom gn, RgDev L, const int32_t* __restrict__ src,
                           const int32_t* __restrict__ groups, int64_t ngroups, const T* __restrict__ w,
                           const double* __restrict__ wmean, T* __restrict__ wn, double* __restrict__ wmean_n,
                           DevScalars* sc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= gn.ncell) return;
  const int code = src[2 * i], idx = src[2 * i + 1];
  const int kind = code & 15, o = (code >> 4) & 15;
  if (code < 0 || kind > 2 || o >= L.no || idx < 0 || (kind < 2 && idx >= go.ncell) ||
      (kind == 2 && idx >= ngroups)) {
    if (b == 0) atomicOr(&sc->status, 16);
    return;
  }
  const int nleg = go.glm ? 9 : 5;
  int base = b * go.n, cnt = L.n;
  bool ldf = false;
  if (b == nleg && go.ldf0 >= 0) {
    base = go.ldf0;
    cnt = L.nd;
    ldf = true;
  } else if (b >= nleg) {
    base = go.bz2d;
  }
  double in[RG_MAXD], out[RG_MAXD];
  if (kind == 0) {
    for (int l = 0; l < cnt; ++l) out[l] = rg_val(go, w, wmean, base + l, (int64_t)idx);
  } else if (kind == 1) {
    for (int m = 0; m < cnt; ++m) in[m] = rg_val(go, w, wmean, base + m, (int64_t)idx);
    const double* P = L.tab + (ldf ? L.PB : L.PL) + (size_t)o * cnt * cnt;
    for (int l = 0; l < cnt; ++l) {
      double v = 0.0;
      for (int m = 0; m < cnt; ++m) v += P[l * cnt + m] * in[m];
      out[l] = v;
    }
  } else {
    for (int l = 0; l < cnt; ++l) out[l] = 0.0;
    const double* R = L.tab + (ldf ? L.RB : L.RL);
    for (int oo = 0; oo < L.no; ++oo) {
      const int64_t cc = groups[(int64_t)idx * L.no + oo];
      for (int m = 0; m < cnt; ++m) in[m] = rg_val(go, w, wmean, base + m, cc);
      const double* Ro = R + (size_t)oo * cnt * cnt;
      for (int l = 0; l < cnt; ++l) {
        double v = out[l];
        for (int m = 0; m < cnt; ++m) v += Ro[l * cnt + m] * in[m];
        out[l] = v;
      }
    }
  }
  for (int l = 0; l < cnt; ++l) {
    const int r = base + l;
    wn[(int64_t)r * gn.stride + i] = (T)out[l];
    const int mi = rg_mean_index(gn, r);
    if (mi >= 0 && wmean_n) wmean_n[(int64_t)mi * gn.stride + i] = out[l];
  }
}

}  // namespace

namespace {

// tables of the context (built and uploaded on first use)
int ensure_tables(Ctx& c, RgDev& L) {
  RgLayout lay;
  std::vector<double> tab;
  if (!c.rg_tabs) {
    if (!regrid_tables(*c.hb, tab, lay)) return DG_E_ARG;
    if (cudaMalloc(&c.rg_tabs, std::max<size_t>(1, tab.size()) * sizeof(double)) != cudaSuccess) return DG_E_CUDA;
    if (cudaMemcpy(c.rg_tabs, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      return DG_E_CUDA;
  } else {
    lay.set(c.hb->D, c.hb->n, c.hb->ndiv);
  }
  L = RgDev{c.rg_tabs, lay.n, lay.nd, lay.D, lay.no, lay.QL, lay.QB, lay.PL, lay.PB, lay.RL, lay.RB};
  return DG_OK;
}

// sibling groups of an octree context (host and device), on first use
int ensure_groups(Ctx& c) {
  AmrHost& h = c.amr;
  if (h.ngroups >= 0) return DG_OK;
  const int D = h.D, no = 1 << D;
  const int64_t N = (int64_t)h.hlevel.size();
  if (h.morton.N != N) {  // built with the face lists at init
    const int e = morton_index(D, N, h.hlevel.data(), h.hijk.data(), h.morton);
    if (e) return e;
  }
  sibling_groups(h.morton, h.hijk.data(), h.hgroups);
  if (!h.groups && cudaMalloc(&h.groups, std::max<size_t>(1, h.hgroups.size()) * sizeof(int32_t)) != cudaSuccess)
    return DG_E_CUDA;
  if (!h.lev_dev && cudaMalloc(&h.lev_dev, std::max<size_t>(1, (size_t)N)) != cudaSuccess) return DG_E_CUDA;
  if (!h.hgroups.empty() &&
      cudaMemcpy(h.groups, h.hgroups.data(), h.hgroups.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
    return DG_E_CUDA;
  if (cudaMemcpy(h.lev_dev, h.hlevel.data(), (size_t)N, cudaMemcpyHostToDevice) != cudaSuccess) return DG_E_CUDA;
  h.ngroups = (int64_t)h.hgroups.size() / no;  // set last: a failed call is retried in full
  return DG_OK;
}

bool mask_ok(const Geom& g, int mask) { return mask > 0 && (mask >> g.V) == 0; }

inline cudaStream_t SR(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

}  // namespace dgmhd

using namespace dgmhd;

extern "C" int dg_mhd_smoothness(dg_mhd_ctx* ctx, const void* w, const double* wmean, int field_mask, double* s_max,
                                 void* stream) {
  if (!ctx || !w || !s_max) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (!mask_ok(c.g, field_mask) || c.g.d > 3) return DG_E_ARG;
  RgDev L;
  int e = ensure_tables(c, L);
  if (e) return e;
  const unsigned nb = (unsigned)((c.g.ncell + 127) / 128);
  if (c.p.precision == DG_PREC_FP32MIX)
    k_rg_smooth<float><<<nb, 128, 0, SR(stream)>>>(c.g, L, (const float*)w, wmean, field_mask, s_max);
  else
    k_rg_smooth<double><<<nb, 128, 0, SR(stream)>>>(c.g, L, (const double*)w, wmean, field_mask, s_max);
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
}

extern "C" int dg_mhd_amr_marks(dg_mhd_ctx* ctx, const void* w, const double* wmean, int field_mask, double s_tilde,
                                int min_level, int max_level, int8_t* marks, double* s_max, void* stream) {
  if (!ctx || !w || !marks || !s_max || !(s_tilde > 0.0)) return DG_E_ARG;
  Ctx& c = ctx->c;
  if (!c.amr.on || c.amr.partial) return DG_E_UNSUPPORTED;
  int e = dg_mhd_smoothness(ctx, w, wmean, field_mask, s_max, stream);
  if (e) return e;
  if ((e = ensure_groups(c))) return e;
  RgDev L;
  if ((e = ensure_tables(c, L))) return e;
  const cudaStream_t st = SR(stream);
  k_rg_marks_leaf<<<(unsigned)((c.g.ncell + 127) / 128), 128, 0, st>>>(c.g.ncell, c.amr.lev_dev, s_max, s_tilde,
                                                                       max_level, marks);
  if (c.amr.ngroups > 0) {
    const unsigned nbg = (unsigned)((c.amr.ngroups + 127) / 128);
    if (c.p.precision == DG_PREC_FP32MIX)
      k_rg_marks_group<float><<<nbg, 128, 0, st>>>(c.g, L, (const float*)w, wmean, field_mask, c.amr.groups,
                                                   c.amr.ngroups, c.amr.lev_dev, s_tilde, min_level, marks);
    else
      k_rg_marks_group<double><<<nbg, 128, 0, st>>>(c.g, L, (const double*)w, wmean, field_mask, c.amr.groups,
                                                    c.amr.ngroups, c.amr.lev_dev, s_tilde, min_level, marks);
  }
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
}

extern "C" int dg_mhd_remap(const dg_mhd_ctx* old_ctx, dg_mhd_ctx* new_ctx, const int32_t* src, const void* w_old,
                            const double* wmean_old, void* w_new, double* wmean_new, void* stream) {
  if (!old_ctx || !new_ctx || !src || !w_old || !w_new) return DG_E_ARG;
  Ctx& co = const_cast<Ctx&>(old_ctx->c);
  Ctx& cn = new_ctx->c;
  const Geom &go = co.g, &gn = cn.g;
  if (go.D != gn.D || go.d != gn.d || go.glm != gn.glm || go.nrows != gn.nrows ||
      co.p.precision != cn.p.precision || !co.amr.on || co.amr.partial || cn.amr.partial)
    return DG_E_ARG;
  if ((wmean_old == nullptr) != (wmean_new == nullptr)) return DG_E_ARG;
  int e = ensure_groups(co);
  if (e) return e;
  RgDev L;
  if ((e = ensure_tables(co, L))) return e;
  if (gn.ncell == 0) return DG_OK;
  const dim3 grid((unsigned)((gn.ncell + 127) / 128), (unsigned)rg_nblocks(go));
  if (co.p.precision == DG_PREC_FP32MIX)
    k_rg_remap<float><<<grid, 128, 0, SR(stream)>>>(go, gn, L, src, co.amr.groups, co.amr.ngroups,
                                                    (const float*)w_old, wmean_old, (float*)w_new, wmean_new, cn.sc);
  else
    k_rg_remap<double><<<grid, 128, 0, SR(stream)>>>(go, gn, L, src, co.amr.groups, co.amr.ngroups,
                                                     (const double*)w_old, wmean_old, (double*)w_new, wmean_new, cn.sc);
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
}

// New leaf list from the marks (host): refine the leaves marked +1, then 2:1
// balance by refining every leaf two levels coarser than a face neighbour
// (until none is), then coarsen the sibling groups whose members are all
// marked -1 where the parent keeps the balance (until no further group can).
// Output in Morton order (lower corner at the finest level, then level).
extern "C" int dg_mhd_regrid_plan(const dg_mhd_ctx* ctx, const int8_t* marks, int64_t cap, int8_t* new_level,
                                  int32_t* new_ijk, int32_t* src, int64_t* n_new) {
  if (!ctx || !marks || !n_new) return DG_E_ARG;
  Ctx& c = const_cast<Ctx&>(ctx->c);
  if (!c.amr.on || c.amr.partial) return DG_E_UNSUPPORTED;
  int e = ensure_groups(c);
  if (e) return e;
  AmrHost& h = c.amr;
  const int D = h.D;
  const int64_t N = (int64_t)h.hlevel.size();
  // FNV-1a hash of the marks: a size query followed by the fill call plans once
  uint64_t hash = 1469598103934665603ull;
  for (int64_t i = 0; i < N; ++i) hash = (hash ^ (uint8_t)marks[i]) * 1099511628211ull;
  if (h.plan.empty() || h.plan_hash != hash) {
    plan_mesh(h.morton, h.hijk.data(), h.hgroups, marks, h.plan);
    h.plan_hash = hash;
  }
  const size_t nn = h.plan.size() / 6;
  *n_new = (int64_t)nn;
  if (!new_level || !new_ijk || !src) return DG_OK;  // size query
  if (cap < (int64_t)nn) return DG_E_ARG;
  for (size_t i = 0; i < nn; ++i) {
    const int32_t* q = &h.plan[i * 6];
    new_level[i] = (int8_t)q[0];
    for (int a = 0; a < D; ++a) new_ijk[i * D + a] = q[1 + a];
    src[2 * i] = q[4];
    src[2 * i + 1] = q[5];
  }
  return DG_OK;
}

// The context's regridding tables without a context (host only).
extern "C" int dg_mhd_regrid_tables(int dim, int degree, int divB_scheme, int64_t cap, double* out,
                                    int64_t* sizes) {
  if (!sizes || (dim != 2 && dim != 3) || degree < 0 || degree > 3 ||
      (divB_scheme != DG_DIVB_POWELL && divB_scheme != DG_DIVB_GLM))
    return DG_E_ARG;
  dgmhd::Basis B;
  if (!B.build(dim, degree, divB_scheme == DG_DIVB_POWELL)) return DG_E_ARG;
  std::vector<double> tab;
  dgmhd::RgLayout L;
  if (!dgmhd::regrid_tables(B, tab, L)) return DG_E_ARG;
  const size_t off[7] = {L.QL, L.QB, L.PL, L.PB, L.RL, L.RB, L.total};
  for (int i = 0; i < 6; ++i) sizes[i] = (int64_t)(off[i + 1] - off[i]);
  if (!out) return DG_OK;  // size query
  if (cap < (int64_t)L.total) return DG_E_ARG;
  std::copy(tab.begin(), tab.end(), out);
  return DG_OK;
}
