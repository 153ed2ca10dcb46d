// Limiters of Sec. 4.2 (characteristic TVB + LDF slope fix) and Sec. 4.3
// (positivity), one thread per cell, state rows read and written coalesced.
//
// k_tvb  reads the cell's mean state, its degree-1 slopes (LDF slopes through
//        the exact table <phi_j,c, xi_a>/<xi_a, xi_a>) and the 2D neighbour
//        means; per direction converts slopes and mean differences to
//        primitive variables (dW/dU at the mean), applies the closed-form left
//        eigenvectors of the Roe & Balsara (1996) normalised 7-wave system plus
//        the divergence wave (Powell) or the (B_n, psi) GLM pair, limits every
//        field with the TVB minmod rule (eq. tvb-limiter), and on a trigger
//        writes R sigma back; any trigger zeroes all weights of degree >= 2 and
//        (Powell) rebuilds the LDF rows of degree <= 1 from the fixed slopes.
// k_pos  floors the cell means (recording injected mass and energy), then
//        tau_rho over all volume and face Gauss points and tau_p from the
//        density-limited state (eq. tau_rho, tau_press), w <- tau w + (1-tau) w_mean.
//        Pressures are screened in the working precision and every point whose
//        pressure may be near or below the floor is re-evaluated in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "dg_limit.cuh"
#include "dg_pos.cuh"
#include "dg_mlp.cuh"

namespace dgmhd {

namespace {

// periodic face neighbour on the uniform mesh (32-bit index arithmetic: cell
// counts stay below 2^31)
__device__ __forceinline__ int64_t nb(const Geom& g, int64_t c, int a, int dir) {
  const unsigned cc = (unsigned)c, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
  const unsigned r = cc / nx;
  int ix = (int)(cc - r * nx), iy = (int)(r % ny), iz = (int)(r / ny);
  if (a == 0) { ix += dir; ix = ix < 0 ? ix + g.nx : (ix >= g.nx ? ix - g.nx : ix); }
  else if (a == 1) { iy += dir; iy = iy < 0 ? iy + g.ny : (iy >= g.ny ? iy - g.ny : iy); }
  else { iz += dir; iz = iz < 0 ? iz + g.nz : (iz >= g.nz ? iz - g.nz : iz); }
  return ((int64_t)iz * g.ny + iy) * g.nx + ix;
}

__device__ __forceinline__ int lmean_row(const Geom& g, int m) {
  if (g.glm) return m * g.n;
  if (m < 5) return m * g.n;
  if (g.D == 3) return g.ldf0 + (m - 5);
  return m < 7 ? g.ldf0 + (m - 5) : g.bz2d;
}

// table entry in the working precision R (FP32 copy or the FP64 table)
template <typename R>
__device__ __forceinline__ R ltab(const double* d, const float* f, int i) {
  if constexpr (sizeof(R) == 4) return f[i];
  else return d[i];
}

// cell means of the conserved variables (B from the degree-0 LDF rows) in the
// working precision R of the limiter
template <typename R, typename T>
__device__ __forceinline__ void cell_mean(const Geom& g, const LimTabs& lt, const T* w, const double* wmean,
                                          int64_t c, R* m) {
  const int64_t S = g.stride;
  const int nm = g.glm ? 9 : 8;
  R raw[9];
  for (int k = 0; k < nm; ++k) raw[k] = wmean ? (R)wmean[k * S + c] : (R)w[(int64_t)lmean_row(g, k) * S + c];
  for (int k = 0; k < 9; ++k) m[k] = R(0);
  for (int k = 0; k < 5; ++k) m[k] = raw[k];
  if (g.glm) {
    for (int k = 5; k < 9; ++k) m[k] = raw[k];
  } else {
    for (int j = 0; j < g.D; ++j)
      for (int cc = 0; cc < g.D; ++cc) m[5 + cc] += raw[5 + j] * ltab<R>(lt.ldf_mean0, lt.ldf_mean0_f, j * 3 + cc);
    if (g.D == 2) m[7] = raw[7];
  }
}

template <typename R>
__device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }
template <typename R>
__device__ __forceinline__ R rmin(R a, R b) { return a < b ? a : b; }
__device__ __forceinline__ double rsq(double x) { return sqrt(x); }
__device__ __forceinline__ float rsq(float x) { return sqrtf(x); }

template <typename R>
__device__ __forceinline__ R minmod3(R a, R b, R c) {
  if (a > R(0) && b > R(0) && c > R(0)) return a < b ? (a < c ? a : c) : (b < c ? b : c);
  if (a < R(0) && b < R(0) && c < R(0)) return a > b ? (a > c ? a : c) : (b > c ? b : c);
  return R(0);
}

// Characteristic basis at mean state m along axis a (primitive variables).
template <typename R>
struct Eig {
  R rho, sr, a2, a, cf, cs, af, as, by, bz, S, ch;
  int n, t1, t2;
  bool glm;
};

template <typename R>
__device__ __forceinline__ void eig_setup(const R* m, int axis, R gamma, bool glm, R ch, R rel, Eig<R>& e) {
  e.n = axis; e.t1 = (axis + 1) % 3; e.t2 = (axis + 2) % 3;
  e.glm = glm; e.ch = ch;
  const R rho = m[0];
  const R v[3] = {m[1] / rho, m[2] / rho, m[3] / rho};
  const R B[3] = {m[5], m[6], m[7]};
  const R p = (gamma - R(1.0)) * (m[4] - R(0.5) * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) -
                                    R(0.5) * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]));
  e.rho = rho;
  e.sr = rsq(rho);
  e.a2 = gamma * p / rho;
  e.a = rsq(e.a2);
  const R bn = B[e.n], bt1 = B[e.t1], bt2 = B[e.t2];
  const R bt2sq = bt1 * bt1 + bt2 * bt2;
  const R b2 = (bn * bn + bt2sq) / rho, cax2 = bn * bn / rho;
  const R disc = rsq(rmax((e.a2 + b2) * (e.a2 + b2) - R(4.0) * e.a2 * cax2, R(0.0)));
  const R cf2 = R(0.5) * (e.a2 + b2 + disc);
  const R cs2 = rmax(R(0.5) * (e.a2 + b2 - disc), R(0.0));
  e.cf = rsq(cf2);
  e.cs = rsq(cs2);
  if (cf2 - cs2 > rel * cf2) {
    e.af = rsq(rmax(e.a2 - cs2, R(0.0)) / (cf2 - cs2));
    e.as = rsq(rmax(cf2 - e.a2, R(0.0)) / (cf2 - cs2));
  } else {
    e.af = R(1.0);
    e.as = R(0.0);
  }
  const R bt = rsq(bt2sq);
  if (bt > rel * rsq(rho * cf2)) {
    e.by = bt1 / bt;
    e.bz = bt2 / bt;
  } else {
    e.by = e.bz = R(0.70710678118654752440);
  }
  e.S = bn >= R(0.0) ? R(1.0) : -R(1.0);
}

// conserved increment dU -> characteristic amplitudes c (V values)
template <typename R>
__device__ __forceinline__ void to_char(const Eig<R>& e, const R* m, R gamma, const R* dU, R* c, int V) {
  const R rho = m[0];
  const R v[3] = {m[1] / rho, m[2] / rho, m[3] / rho};
  const R B[3] = {m[5], m[6], m[7]};
  // dW = dW/dU dU
  R dW[9];
  dW[0] = dU[0];
  for (int i = 0; i < 3; ++i) dW[1 + i] = (dU[1 + i] - v[i] * dU[0]) / rho;
  const R g1 = gamma - R(1.0);
  dW[4] = g1 * (R(0.5) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * dU[0] - (v[0] * dU[1] + v[1] * dU[2] + v[2] * dU[3]) +
                dU[4] - (B[0] * dU[5] + B[1] * dU[6] + B[2] * dU[7]));
  for (int i = 5; i < V; ++i) dW[i] = dU[i];
  const R dr = dW[0], du = dW[1 + e.n], dv = dW[1 + e.t1], dw = dW[1 + e.t2], dp = dW[4];
  const R dby = dW[5 + e.t1], dbz = dW[5 + e.t2];
  const R ia2 = R(1.0) / e.a2;
  const R vpar = e.by * dv + e.bz * dw, bpar = e.by * dby + e.bz * dbz;
  const R vperp = -e.bz * dv + e.by * dw, bperp = -e.bz * dby + e.by * dbz;
  const R sra = e.sr * e.a;
  // fast -, alfven -, slow -, entropy, slow +, alfven +, fast +
  c[0] = R(0.5) * ia2 * (-e.af * e.cf * du + e.as * e.cs * e.S * vpar) + R(0.5) * (e.af * dp / (e.rho * e.a2) + e.as * bpar / sra);
  c[6] = R(0.5) * ia2 * (e.af * e.cf * du - e.as * e.cs * e.S * vpar) + R(0.5) * (e.af * dp / (e.rho * e.a2) + e.as * bpar / sra);
  c[2] = R(0.5) * ia2 * (-e.as * e.cs * du - e.af * e.cf * e.S * vpar) + R(0.5) * (e.as * dp / (e.rho * e.a2) - e.af * bpar / sra);
  c[4] = R(0.5) * ia2 * (e.as * e.cs * du + e.af * e.cf * e.S * vpar) + R(0.5) * (e.as * dp / (e.rho * e.a2) - e.af * bpar / sra);
  c[1] = R(0.5) * vperp + R(0.5) * e.S * bperp / e.sr;
  c[5] = R(0.5) * vperp - R(0.5) * e.S * bperp / e.sr;
  c[3] = dr - dp * ia2;
  const R dbn = dW[5 + e.n];
  if (!e.glm) {
    c[7] = dbn;
  } else if (e.ch > R(0.0)) {
    const R dpsi = dW[8];
    c[7] = R(0.5) * (dbn - dpsi / e.ch);
    c[8] = R(0.5) * (dbn + dpsi / e.ch);
  } else {  // no c_h set yet: B_n and psi as separate fields
    c[7] = dbn;
    c[8] = dW[8];
  }
}

// characteristic amplitudes -> conserved increment
template <typename R>
__device__ __forceinline__ void from_char(const Eig<R>& e, const R* m, R gamma, const R* c, R* dU, int V) {
  const R rho = e.rho, sr = e.sr, a2 = e.a2, a = e.a, S = e.S;
  R dW7[7] = {0, 0, 0, 0, 0, 0, 0};  // rho, u, v, w, p, By, Bz (rotated)
  auto add = [&](R amp, R r0, R r1, R r2, R r3, R r4, R r5, R r6) {
    dW7[0] += amp * r0; dW7[1] += amp * r1; dW7[2] += amp * r2; dW7[3] += amp * r3;
    dW7[4] += amp * r4; dW7[5] += amp * r5; dW7[6] += amp * r6;
  };
  add(c[0], rho * e.af, -e.af * e.cf, e.as * e.cs * e.by * S, e.as * e.cs * e.bz * S, rho * e.af * a2,
      e.as * sr * a * e.by, e.as * sr * a * e.bz);
  add(c[1], 0, 0, -e.bz, e.by, 0, -e.bz * S * sr, e.by * S * sr);
  add(c[2], rho * e.as, -e.as * e.cs, -e.af * e.cf * e.by * S, -e.af * e.cf * e.bz * S, rho * e.as * a2,
      -e.af * sr * a * e.by, -e.af * sr * a * e.bz);
  add(c[3], 1, 0, 0, 0, 0, 0, 0);
  add(c[4], rho * e.as, e.as * e.cs, e.af * e.cf * e.by * S, e.af * e.cf * e.bz * S, rho * e.as * a2,
      -e.af * sr * a * e.by, -e.af * sr * a * e.bz);
  add(c[5], 0, 0, -e.bz, e.by, 0, e.bz * S * sr, -e.by * S * sr);
  add(c[6], rho * e.af, e.af * e.cf, -e.as * e.cs * e.by * S, -e.as * e.cs * e.bz * S, rho * e.af * a2,
      e.as * sr * a * e.by, e.as * sr * a * e.bz);
  R dW[9];
  dW[0] = dW7[0];
  dW[1 + e.n] = dW7[1];
  dW[1 + e.t1] = dW7[2];
  dW[1 + e.t2] = dW7[3];
  dW[4] = dW7[4];
  dW[5 + e.t1] = dW7[5];
  dW[5 + e.t2] = dW7[6];
  if (!e.glm) {
    dW[5 + e.n] = c[7];
  } else if (e.ch > R(0.0)) {
    dW[5 + e.n] = c[7] + c[8];
    dW[8] = e.ch * (c[8] - c[7]);
  } else {
    dW[5 + e.n] = c[7];
    dW[8] = c[8];
  }
  // dU = dU/dW dW
  const R v[3] = {m[1] / m[0], m[2] / m[0], m[3] / m[0]};
  const R B[3] = {m[5], m[6], m[7]};
  dU[0] = dW[0];
  for (int i = 0; i < 3; ++i) dU[1 + i] = v[i] * dW[0] + rho * dW[1 + i];
  dU[4] = R(0.5) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * dW[0] + rho * (v[0] * dW[1] + v[1] * dW[2] + v[2] * dW[3]) +
          dW[4] / (gamma - R(1.0)) + B[0] * dW[5] + B[1] * dW[6] + B[2] * dW[7];
  for (int i = 5; i < V; ++i) dU[i] = dW[i];
}

// Octree neighbours for the limiter: face lists (see dg_amr.cuh) and cell sizes.
struct AmrNb {
  const int32_t* fL;
  const int32_t* fR;
  const int32_t* fmeta;
  const int32_t* cstart;
  const int32_t* centry;
  const double* dxc;
  int on;
  const int32_t* side_nb;    // AmrHost::side_nb: the leaves across each side, in face-entry order
  const uint8_t* side_info;  // count | relation << 4 per leaf and side
};

// The TVB procedure on cell c; returns whether any slope changed. All of it
// runs in the working precision of the state (the FP32 form reads the float
// mirror of the means, which the limiter never changes).
template <typename T>
__device__ bool tvb_cell(const Geom& g, const LimTabs& lt, T* w, const double* wmean, const dg_mhd_params& p,
                         const DevScalars* __restrict__ sc, const AmrNb& an, int64_t c) {
  using R = T;
  const int64_t S = g.stride;
  const int V = g.V;
  R m[9];
  cell_mean<R>(g, lt, (const T*)w, wmean, c, m);
  // degree-1 slopes u_xi[a][v]
  R sl[3][9];
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 9; ++k) sl[a][k] = R(0);
  const int nleg = g.glm ? 9 : 5;
  for (int a = 0; a < g.D; ++a) {
    for (int v = 0; v < nleg; ++v) sl[a][v] = (R)w[(int64_t)(v * g.n + lt.deg1[a]) * S + c];
    if (g.bz2d >= 0) sl[a][7] = (R)w[(int64_t)(g.bz2d + lt.deg1[a]) * S + c];
  }
  if (!g.glm) {
    for (int j = 0; j < g.ndiv; ++j) {
      if (lt.ldf_deg[j] == 0) continue;
      const R wj = (R)w[(int64_t)(g.ldf0 + j) * S + c];
      for (int cc = 0; cc < g.D; ++cc)
        for (int a = 0; a < g.D; ++a) sl[a][5 + cc] += wj * ltab<R>(lt.ldf_slope, lt.ldf_slope_f, (j * 3 + cc) * 3 + a);
    }
  }
  // characteristic limiting
  const R thr = (R)(p.Mtilde * (an.on ? an.dxc[c] : g.dx));
  const R ch = g.glm ? (R)sc->ch : R(0);
  const R rel = sizeof(T) == 4 ? R(1e-6) : R(1e-12);
  const R gam = (R)g.gamma, beta = (R)p.beta, teps = (R)p.tvb_eps;
  bool any = false;
  R nsl[3][9];
  for (int a = 0; a < g.D; ++a) {
    R mp[9], mm[9];
    R fp = R(2), fm = R(2);  // centre distance in units of dx_K / 2
    if (!an.on) {
      cell_mean<R>(g, lt, (const T*)w, wmean, nb(g, c, a, +1), mp);
      cell_mean<R>(g, lt, (const T*)w, wmean, nb(g, c, a, -1), mm);
    } else {
      // octree: average of the leaves across each side (listed per side at
      // set-up, in face-entry order); 2 same level, 3 coarser, 1.5 finer
      int np_ = 0, nm_ = 0;
      for (int k = 0; k < 9; ++k) mp[k] = mm[k] = R(0);
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int sidx = 2 * a + sd;  // sd 1: the +a side
        const int inf = an.side_info[c * 6 + sidx];
        const int cnt = inf & 15, rel = inf >> 4;
        const R fac = rel == 0 ? R(2) : (rel == 1 ? R(1.5) : R(3));
        R* acc = sd ? mp : mm;
        for (int k2 = 0; k2 < cnt; ++k2) {
          R mn[9];
          cell_mean<R>(g, lt, (const T*)w, wmean, (int64_t)an.side_nb[c * 24 + sidx * 4 + k2], mn);
          for (int k = 0; k < 9; ++k) acc[k] += mn[k];
        }
        if (cnt > 0) {
          if (sd) {
            np_ = cnt;
            fp = fac;
          } else {
            nm_ = cnt;
            fm = fac;
          }
        }
      }
      // 1 or 2^(D-1) leaves: exact reciprocals
      const R ip = R(1) / (R)(np_ > 0 ? np_ : 1), im = R(1) / (R)(nm_ > 0 ? nm_ : 1);
      for (int k = 0; k < 9; ++k) {
        mp[k] *= ip;
        mm[k] *= im;
      }
    }
    // one reciprocal per side (exact for the distance 2 of equal cells)
    const R ifp = R(1) / fp, ifm = R(1) / fm;
    R dpl[9], dmi[9];
    for (int k = 0; k < 9; ++k) {
      dpl[k] = (mp[k] - m[k]) * ifp;
      dmi[k] = (m[k] - mm[k]) * ifm;
    }
    Eig<R> e;
    eig_setup(m, a, gam, g.glm != 0, ch, rel, e);
    R cx[9], cp[9], cm[9], sg[9];
    to_char(e, m, gam, sl[a], cx, V);
    to_char(e, m, gam, dpl, cp, V);
    to_char(e, m, gam, dmi, cm, V);
    bool trig = false;
    for (int k = 0; k < V; ++k) {
      sg[k] = cx[k];
      const R ax = cx[k] < R(0) ? -cx[k] : cx[k];
      if (ax > thr) sg[k] = minmod3(cx[k], beta * cp[k], beta * cm[k]);
      const R df = sg[k] - cx[k];
      if ((df < R(0) ? -df : df) > teps) trig = true;
    }
    if (trig) {
      R out[9];
      from_char(e, m, gam, sg, out, V);
      for (int k = 0; k < 9; ++k) nsl[a][k] = k < V ? out[k] : R(0);
      any = true;
    } else {
      for (int k = 0; k < 9; ++k) nsl[a][k] = sl[a][k];
    }
  }
  if (!any) return false;
  // Legendre rows: degree-1 slopes, degree >= 2 zeroed
  for (int r = 0; r < g.nrows; ++r) {
    const bool ldf = g.ldf0 >= 0 && r >= g.ldf0 && r < g.ldf0 + g.ndiv;
    if (ldf) continue;
    int v, l;
    if (g.bz2d >= 0 && r >= g.bz2d) { v = 7; l = r - g.bz2d; }
    else { v = r / g.n; l = r % g.n; }
    const int dg = lt.mdeg[l];
    if (dg == 0) continue;
    R val = R(0);
    if (dg == 1) {
      for (int a = 0; a < g.D; ++a)
        if (lt.deg1[a] == l) val = nsl[a][v];
    }
    w[(int64_t)r * S + c] = (T)val;
  }
  if (!g.glm) {
    // LDF slope fix (Sec. 4.2.4) and exact projection onto LDF degree <= 1
    R Bs[3][3];
    for (int cc = 0; cc < g.D; ++cc)
      for (int a = 0; a < g.D; ++a) Bs[cc][a] = nsl[a][5 + cc];
    R dpos = R(0), dneg = R(0), dsum = R(0);
    for (int k = 0; k < g.D; ++k) {
      dsum += Bs[k][k];
      dpos += rmax(Bs[k][k], R(0));
      dneg += rmax(-Bs[k][k], R(0));
    }
    if (dsum > R(0)) {
      const R f = dneg / dpos;
      for (int k = 0; k < g.D; ++k)
        if (Bs[k][k] > R(0)) Bs[k][k] *= f;
    } else if (dsum < R(0)) {
      const R f = dpos / dneg;
      for (int k = 0; k < g.D; ++k)
        if (Bs[k][k] < R(0)) Bs[k][k] *= f;
    }
    for (int j = 0; j < g.ndiv; ++j) {
      const int64_t i = (int64_t)(g.ldf0 + j) * S + c;
      if (lt.ldf_deg[j] == 0) continue;  // means kept
      if (lt.ldf_deg[j] > 1) {
        w[i] = T(0);
        continue;
      }
      R val = R(0);
      for (int cc = 0; cc < g.D; ++cc) {
        val += ltab<R>(lt.ldf_pc, lt.ldf_pc_f, j * 3 + cc) * m[5 + cc];
        for (int a = 0; a < g.D; ++a) val += ltab<R>(lt.ldf_pl, lt.ldf_pl_f, (j * 3 + cc) * 3 + a) * Bs[cc][a];
      }
      w[i] = (T)val;
    }
  }
  return true;
}

// TVB over every cell (list == nullptr: the plain detector) or over the cells
// the learned indicator listed (list[0 .. sc->nflag)); grid-stride, so any
// grid covers the work. Counts the cells whose slopes changed.
template <typename T, bool SCREEN>
__global__ void k_tvb(Geom g, LimTabs lt, T* w, double* wmean, uint8_t* troubled, const int32_t* __restrict__ list,
                      dg_mhd_params p, DevScalars* sc, AmrNb an, int32_t* __restrict__ plist, PosScreen ps) {
  const int64_t total = list ? (int64_t)sc->nflag : g.ncell;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int64_t S = g.stride;
  unsigned limited = 0;
  // warp-uniform trip count (the positivity append below is a warp ballot)
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < total; i0 += step) {
    const int64_t i = i0 + lane;
    bool fail = false;
    if (i < total) {
      const int64_t c = list ? (int64_t)list[i] : i;
      const bool any = tvb_cell(g, lt, w, wmean, p, sc, an, c);
      if (troubled) troubled[c] = any ? 1 : 0;
      limited += any ? 1u : 0u;
      // FP32 form with the learned indicator: the flagged cells take the
      // positivity screen here, on their limited rows
      if constexpr (SCREEN) fail = !pos_screen_rows(g, ps, [&](int r) { return (float)w[(int64_t)r * S + c]; });
    }
    if constexpr (SCREEN) append_cells(fail, i < total ? (list ? (int64_t)list[i] : i) : 0, plist, &sc->npos);
  }
  limited = __reduce_add_sync(0xffffffffu, limited);
  if (lane == 0 && limited) atomicAdd(&sc->cnt_limited, (unsigned long long)limited);
}

// ------------------------------------------------------------------ positivity
template <typename T>
__device__ __forceinline__ void point_state(const Geom& g, const Tables<T>& tb, const T* w, const double* mr,
                                            int64_t c, int pt, double* u, bool dbl) {
  // pt < Qv: volume point; else face point (f, p)
  const T* P;
  const T* Lt;
  int stride, idx;
  if (pt < g.Qv) {
    P = tb.Pv; Lt = tb.Lv; stride = g.Qv; idx = pt;
  } else {
    const int fp = pt - g.Qv, f = fp / g.Qf;
    P = tb.Pf + (size_t)f * g.n * g.Qf;
    Lt = tb.Lf + (size_t)f * g.ndiv * g.DB * g.Qf;
    stride = g.Qf; idx = fp % g.Qf;
  }
  const int64_t S = g.stride;
  for (int k = 0; k < 9; ++k) u[k] = 0.0;
  const int nleg = g.glm ? 9 : 5;
  for (int v = 0; v < nleg; ++v) {
    double s = mr[v];  // mode 0 (P_0 = 1) from the authoritative mean
    if (dbl) {
      for (int l = 1; l < g.n; ++l) s += (double)w[(int64_t)(v * g.n + l) * S + c] * (double)P[l * stride + idx];
    } else {
      T st = T(0);
      for (int l = 1; l < g.n; ++l) st += w[(int64_t)(v * g.n + l) * S + c] * P[l * stride + idx];
      s += (double)st;
    }
    u[v] = s;
  }
  if (!g.glm) {
    for (int j = 0; j < g.ndiv; ++j) {
      const double wj = j < g.D ? mr[5 + j] : (double)w[(int64_t)(g.ldf0 + j) * S + c];
      for (int cc = 0; cc < g.DB; ++cc) u[5 + cc] += wj * (double)Lt[(j * g.DB + cc) * stride + idx];
    }
    if (g.bz2d >= 0) {
      double s = mr[7];
      for (int l = 1; l < g.n; ++l) s += (double)w[(int64_t)(g.bz2d + l) * S + c] * (double)P[l * stride + idx];
      u[7] = s;
    }
  }
}

// FP32 form: screen every cell; the cells that do not clear it are appended to
// list[0 .. sc->npos) (ballot + one atomic per warp) for k_pos.
template <int DEG, int GLMF>
__global__ void k_pos_screen(Geom gin, PosScreen ps, const float* __restrict__ w, DevScalars* sc,
                             int32_t* __restrict__ list) {
  const Geom g = pin_geom<DEG, GLMF>(gin);
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t S = g.stride;
  const bool fail = c < g.ncell && !pos_screen_rows(g, ps, [&](int r) { return w[(int64_t)r * S + c]; });
  append_cells(fail, c, list, &sc->npos);
}

// Whether the pressure of a point must be decided in FP64. uu: the point's
// state in the working precision, m: the cell means, dev: per variable the sum
// of |coefficients| beyond the mean times the basis bound, tt: the density
// factor. scale_v = |m_v| + tt dev_v bounds every partial sum of u_v, so the
// rounding of u_v is a few ulp of scale_v. The pressure is decided in the
// working precision only if the density carries at most two digits of
// cancellation and the pressure clears the floor by screen_t times the scale
// of each of its terms (energy, kinetic, magnetic); screen_t = 0 (FP64): only
// points below the floor.
template <typename T>
__device__ __forceinline__ bool pos_point_open(const T* uu, const double* m, const T* dev, T tt, T gm1, T eps_p,
                                               T screen_t) {
  T sc[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) sc[v] = (T)fabs(m[v]) + tt * dev[v];
  const T kin = T(0.5) * (uu[1] * uu[1] + uu[2] * uu[2] + uu[3] * uu[3]) / uu[0];
  const T mag = T(0.5) * (uu[5] * uu[5] + uu[6] * uu[6] + uu[7] * uu[7]);
  const T pq = gm1 * (uu[4] - kin - mag);
  if (screen_t == T(0)) return pq < eps_p;
  if (uu[0] < T(1e-2) * sc[0]) return true;
  const T kin_s = T(0.5) * (sc[1] * sc[1] + sc[2] * sc[2] + sc[3] * sc[3]) / uu[0];
  const T mag_s = T(0.5) * (sc[5] * sc[5] + sc[6] * sc[6] + sc[7] * sc[7]);
  return pq < eps_p + screen_t * gm1 * (sc[4] + kin_s + mag_s);
}

// The same test from float copies of the cell's mean magnitudes (|m_v| in
// FP32, converted once per cell): bitwise the same decision, since rounding
// to nearest commutes with the absolute value.
__device__ __forceinline__ bool pos_point_open_f(const float* uu, const float* mabs, const float* dev, float tt,
                                                 float gm1, float eps_p, float screen_t) {
  float sc[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) sc[v] = mabs[v] + tt * dev[v];
  const float kin = 0.5f * (uu[1] * uu[1] + uu[2] * uu[2] + uu[3] * uu[3]) / uu[0];
  const float mag = 0.5f * (uu[5] * uu[5] + uu[6] * uu[6] + uu[7] * uu[7]);
  const float pq = gm1 * (uu[4] - kin - mag);
  if (uu[0] < 1e-2f * sc[0]) return true;
  const float kin_s = 0.5f * (sc[1] * sc[1] + sc[2] * sc[2] + sc[3] * sc[3]) / uu[0];
  const float mag_s = 0.5f * (sc[5] * sc[5] + sc[6] * sc[6] + sc[7] * sc[7]);
  return pq < eps_p + screen_t * gm1 * (sc[4] + kin_s + mag_s);
}

// Positivity procedure of one cell (Sec. 4.3).
template <typename T>
__device__ void pos_cell(const Geom& g, const Tables<T>& tb, const LimTabs& lt, T* w, double* wmean,
                         const dg_mhd_params& p, DevScalars* sc, int64_t c) {
  const int64_t S = g.stride;
  const int nm = g.glm ? 9 : 8;
  const bool mix = wmean != nullptr;
  // raw mean rows (Legendre mode 0 / degree-0 LDF weights)
  double mr[9];
  for (int k = 0; k < nm; ++k) mr[k] = mix ? wmean[k * S + c] : (double)w[(int64_t)lmean_row(g, k) * S + c];
  // physical mean state
  double m[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < 5; ++k) m[k] = mr[k];
  if (g.glm) {
    for (int k = 5; k < 9; ++k) m[k] = mr[k];
  } else {
    for (int j = 0; j < g.D; ++j)
      for (int cc = 0; cc < g.DB; ++cc) m[5 + cc] += mr[5 + j] * (double)tb.L0[j * g.DB + cc];
    if (g.bz2d >= 0) m[7] = mr[7];
  }
  const double gm1 = g.gamma - 1.0;
  double vol = 1.0;
  for (int a = 0; a < g.D; ++a) vol *= g.dx;
  bool changed_mean = false;
  if (m[0] < p.eps_rho) {
    atomicAdd(&sc->inj_mass, (p.eps_rho - m[0]) * vol);
    m[0] = mr[0] = p.eps_rho;
    changed_mean = true;
  }
  auto pres = [&](const double* u) {
    return gm1 * (u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0] -
                  0.5 * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]));
  };
  const double pm = pres(m);
  if (pm < p.eps_p) {
    const double dE = (p.eps_p - pm) / gm1;
    atomicAdd(&sc->inj_energy, dE * vol);
    m[4] += dE;
    mr[4] += dE;
    changed_mean = true;
  }
  if (changed_mean) {
    atomicOr(&sc->floor_used, 1);
    for (int k = 0; k < nm; ++k) {
      const int r = lmean_row(g, k);
      if (mix) wmean[k * S + c] = mr[k];
      w[(int64_t)r * S + c] = (T)mr[k];
    }
  }
  const int npt = g.Qv + 2 * g.D * g.Qf;
  const double pmean = pres(m);
  // per variable, sum of |coefficients| beyond the mean (x |basis| bound): with
  // |mean|, the scale of every point value, which bounds its rounding
  T devt[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  {
    // Rigorous screen: |P_l| <= 1 on the cell, |phi_j,c| <= ldf_maxabs, so
    // |u_v(x) - mean_v| <= dev_v everywhere; if the resulting lower bounds of
    // rho and p clear the floors, every point does and tau = 1.
    const int nlg = g.glm ? 8 : 5;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      if (v >= nlg) continue;
      for (int l = 1; l < g.n; ++l) {
        const T x = w[(int64_t)(v * g.n + l) * S + c];
        devt[v] += x < T(0) ? -x : x;
      }
    }
    if (!g.glm) {
      for (int j = g.D; j < g.ndiv; ++j) {
        T aj = w[(int64_t)(g.ldf0 + j) * S + c];
        aj = aj < T(0) ? -aj : aj;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
          if (cc < g.D) devt[5 + cc] += aj * (T)lt.ldf_maxabs[j * 3 + cc];
      }
      if (g.bz2d >= 0)
        for (int l = 1; l < g.n; ++l) {
          const T x = w[(int64_t)(g.bz2d + l) * S + c];
          devt[7] += x < T(0) ? -x : x;
        }
    }
    double dev[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) dev[v] = (double)devt[v];
    // margin for the rounding of the bounds themselves in the working precision
    const double rel = sizeof(T) == 4 ? 1e-5 : 1e-12;
    for (int v = 0; v < 8; ++v) dev[v] = dev[v] * (1.0 + rel) + rel * fabs(m[v]);
    const double rho_lo = m[0] - dev[0];
    if (rho_lo > p.eps_rho) {
      double kin = 0.0, mag = 0.0;
      for (int i = 0; i < 3; ++i) {
        const double mu = fabs(m[1 + i]) + dev[1 + i], bu = fabs(m[5 + i]) + dev[5 + i];
        kin += mu * mu;
        mag += bu * bu;
      }
      const double p_lo = gm1 * (m[4] - dev[4] - 0.5 * kin / rho_lo - 0.5 * mag);
      if (p_lo > p.eps_p) return;
    }
  }
  // basis value of Legendre mode l / LDF row j component cc at point pt
  auto Pval = [&](int l, int pt) -> T { return tb.Pp[l * npt + pt]; };
  auto Lval = [&](int j, int cc, int pt) -> T { return tb.Lp[(j * g.DB + cc) * npt + pt]; };
  constexpr int PC = 8;  // points per pass: each state row is loaded once per pass
  // screening margin of the working precision: points within it of a floor are
  // re-evaluated in FP64, all others decided in the working precision
  const T screen_t = sizeof(T) == 4 ? T(1e-4) : T(0);
  // tau_rho (eq. tau_rho) over all volume and face points
  double tau = 1.0;
  for (int p0 = 0; p0 < npt; p0 += PC) {
    T acc[PC];
#pragma unroll
    for (int k = 0; k < PC; ++k) acc[k] = T(0);
    for (int l = 1; l < g.n; ++l) {
      const T wv = w[(int64_t)l * S + c];
#pragma unroll
      for (int k = 0; k < PC; ++k)
        if (p0 + k < npt) acc[k] += wv * Pval(l, p0 + k);
    }
#pragma unroll
    for (int k = 0; k < PC; ++k) {
      if (p0 + k >= npt) continue;
      const T rq = (T)mr[0] + acc[k];
      if (rq < (T)p.eps_rho + screen_t * ((T)fabs(m[0]) + devt[0])) {
        // near or below the floor: decide in FP64
        double rd = mr[0];
        for (int l = 1; l < g.n; ++l) rd += (double)w[(int64_t)l * S + c] * (double)Pval(l, p0 + k);
        if (rd < p.eps_rho) tau = fmin(tau, (m[0] - p.eps_rho) / (m[0] - rd));
      }
    }
  }
  tau = fmax(tau, 0.0);
  // tau_p (eq. tau_press) from the density-limited state u' = m + tau (u - m)
  double taup = 1.0;
  const int nleg = g.glm ? 8 : 5;
  for (int p0 = 0; p0 < npt; p0 += PC) {
    // register accumulators: every index below is a compile-time constant
    T acc[PC][8];
#pragma unroll
    for (int k = 0; k < PC; ++k)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[k][v] = T(0);
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      if (v >= nleg) continue;
      for (int l = 1; l < g.n; ++l) {
        const T wv = w[(int64_t)(v * g.n + l) * S + c];
#pragma unroll
        for (int k = 0; k < PC; ++k)
          if (p0 + k < npt) acc[k][v] += wv * Pval(l, p0 + k);
      }
    }
    if (!g.glm) {
      for (int j = g.D; j < g.ndiv; ++j) {
        const T wj = w[(int64_t)(g.ldf0 + j) * S + c];
#pragma unroll
        for (int k = 0; k < PC; ++k)
          if (p0 + k < npt) {
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
              if (cc < g.DB) acc[k][5 + cc] += wj * Lval(j, cc, p0 + k);
          }
      }
      if (g.bz2d >= 0)
        for (int l = 1; l < g.n; ++l) {
          const T wv = w[(int64_t)(g.bz2d + l) * S + c];
#pragma unroll
          for (int k = 0; k < PC; ++k)
            if (p0 + k < npt) acc[k][7] += wv * Pval(l, p0 + k);
        }
    }
    const T gm1t = (T)gm1;
#pragma unroll
    for (int k = 0; k < PC; ++k) {
      if (p0 + k >= npt) continue;
      const T tt = (T)tau;
      T uu[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) uu[v] = (T)m[v] + tt * acc[k][v];  // acc holds u - mean
      if (pos_point_open(uu, m, devt, tt, gm1t, (T)p.eps_p, screen_t)) {
        // FP64 recovery of this point's pressure (E - kinetic - magnetic cancels)
        double u[9];
        point_state(g, tb, (const T*)w, mr, c, p0 + k, u, true);
        for (int v = 0; v < 9; ++v) u[v] = m[v] + tau * (u[v] - m[v]);
        const double pq = pres(u);
        if (pq < p.eps_p) taup = fmin(taup, (pmean - p.eps_p) / (pmean - pq));
      }
    }
  }
  taup = fmax(taup, 0.0);
  const double t = tau * taup;
  if (t >= 1.0) return;
  atomicAdd(&sc->pos_cells, 1ull);
  // scale every non-mean row by tau
  for (int r = 0; r < g.nrows; ++r) {
    bool mean = false;
    for (int k = 0; k < nm; ++k)
      if (lmean_row(g, k) == r) mean = true;
    if (mean) continue;
    const int64_t i = (int64_t)r * S + c;
    w[i] = (T)(t * (double)w[i]);
  }
}

// Every cell (list == nullptr) or the listed cells list[0 .. sc->npos); grid-stride.
template <typename T>
__global__ void k_pos(Geom g, Tables<T> tb, LimTabs lt, T* w, double* wmean, dg_mhd_params p, DevScalars* sc,
                      const int32_t* __restrict__ list) {
  const int64_t total = list ? (int64_t)sc->npos : g.ncell;
  if (list && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&sc->cnt_poslisted, (unsigned long long)total);
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step)
    pos_cell(g, tb, lt, w, wmean, p, sc, list ? (int64_t)list[i] : i);
}

// FP32 form, 3D degrees 1-2: the positivity procedure of pos_cell on the
// listed cells. A warp takes 32 list entries: each lane stages its cell's rows
// (coalesced where the listed cells are neighbours), applies the mean floors
// and the rigorous screen; the cells that stay open are then done one at a
// time by the whole warp, lanes over the volume and face points, the limiting
// factors being warp minima. Every point value is accumulated in the same
// order as in pos_cell, so the two agree bit for bit.
template <int DEG, int GLMF>
__global__ void __launch_bounds__(128) k_pos_list(Geom gin, Tables<float> tb, LimTabs lt, float* w, double* wmean,
                                                  dg_mhd_params p, DevScalars* sc, const int32_t* __restrict__ list) {
  const Geom g = pin_geom<DEG, GLMF>(gin);
  constexpr int N = (DEG + 1) * (DEG + 2) * (DEG + 3) / 6;
  constexpr int NR = GLMF ? 9 * N : 5 * N + (DEG == 1 ? 11 : 26);
  __shared__ float rows[4][NR][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float(*R)[32] = rows[warp];
  const int64_t S = g.stride;
  const int nm = g.glm ? 9 : 8;
  const int npt = g.Qv + 2 * g.D * g.Qf;
  const double gm1 = g.gamma - 1.0;
  const float gm1t = (float)gm1;
  const float screen_t = 1e-4f;
  const double vol = g.dx * g.dx * g.dx;
  auto pres = [&](const double* u) {
    return gm1 * (u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0] -
                  0.5 * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]));
  };
  auto wmin = [](double v) {
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
  };
  const int64_t total = (int64_t)sc->npos;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&sc->cnt_poslisted, (unsigned long long)total);
  for (int64_t i0 = ((int64_t)blockIdx.x * 4 + warp) * 32; i0 < total; i0 += (int64_t)gridDim.x * 4 * 32) {
    const bool valid = i0 + lane < total;
    const int64_t c = valid ? (int64_t)list[i0 + lane] : 0;
    __syncwarp();  // the previous group's reads of R are done
    double mr[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, m[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double pmean = 0.0;
    bool open = false;
    // per variable, sum of |coefficients| beyond the mean (x |basis| bound): with
    // |mean|, the scale of every point value, which bounds its FP32 rounding
    float devt[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
#pragma unroll
      for (int r = 0; r < NR; ++r) R[r][lane] = w[(int64_t)r * S + c];
      for (int k = 0; k < nm; ++k) mr[k] = wmean[k * S + c];
      // physical mean state and the mean floors
      for (int k = 0; k < 5; ++k) m[k] = mr[k];
      if (g.glm) {
        for (int k = 5; k < 9; ++k) m[k] = mr[k];
      } else {
        for (int j = 0; j < g.D; ++j)
          for (int cc = 0; cc < g.DB; ++cc) m[5 + cc] += mr[5 + j] * (double)tb.L0[j * g.DB + cc];
      }
      bool changed_mean = false;
      if (m[0] < p.eps_rho) {
        atomicAdd(&sc->inj_mass, (p.eps_rho - m[0]) * vol);
        m[0] = mr[0] = p.eps_rho;
        changed_mean = true;
      }
      const double pm = pres(m);
      if (pm < p.eps_p) {
        const double dE = (p.eps_p - pm) / gm1;
        atomicAdd(&sc->inj_energy, dE * vol);
        m[4] += dE;
        mr[4] += dE;
        changed_mean = true;
      }
      if (changed_mean) {
        atomicOr(&sc->floor_used, 1);
        for (int k = 0; k < nm; ++k) {
          wmean[k * S + c] = mr[k];
          w[(int64_t)lmean_row(g, k) * S + c] = (float)mr[k];
        }
      }
      pmean = pres(m);
      // the rigorous screen of pos_cell
      const int nlg = g.glm ? 8 : 5;
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        if (v >= nlg) continue;
        for (int l = 1; l < g.n; ++l) devt[v] += fabsf(R[v * g.n + l][lane]);
      }
      if (!g.glm)
        for (int j = g.D; j < g.ndiv; ++j) {
          const float aj = fabsf(R[g.ldf0 + j][lane]);
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) devt[5 + cc] += aj * (float)lt.ldf_maxabs[j * 3 + cc];
        }
      double dev[8];
      for (int v = 0; v < 8; ++v) dev[v] = (double)devt[v] * (1.0 + 1e-5) + 1e-5 * fabs(m[v]);
      open = true;
      const double rho_lo = m[0] - dev[0];
      if (rho_lo > p.eps_rho) {
        double kin = 0.0, mag = 0.0;
        for (int k = 0; k < 3; ++k) {
          const double mu = fabs(m[1 + k]) + dev[1 + k], bu = fabs(m[5 + k]) + dev[5 + k];
          kin += mu * mu;
          mag += bu * bu;
        }
        if (gm1 * (m[4] - dev[4] - 0.5 * kin / rho_lo - 0.5 * mag) > p.eps_p) open = false;
      }
    }
    __syncwarp();  // R complete
    unsigned todo = __ballot_sync(0xffffffffu, open);
    while (todo) {
      const int o = __ffs(todo) - 1;
      todo &= todo - 1;
      // the open cell of lane o, done by the whole warp
      const int64_t co = __shfl_sync(0xffffffffu, c, o);
      double mo[9], mro[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        mo[k] = __shfl_sync(0xffffffffu, m[k], o);
        mro[k] = __shfl_sync(0xffffffffu, mr[k], o);
      }
      const double pmo = __shfl_sync(0xffffffffu, pmean, o);
      float dvo[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) dvo[v] = __shfl_sync(0xffffffffu, devt[v], o);
      // float copies of the cell's constants, converted once per cell (an FP64
      // -> FP32 conversion occupies GB300's FP64 pipe; inside the point loops
      // they made this kernel FP64-bound)
      float mof[8], maf[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        mof[v] = (float)mo[v];
        maf[v] = fabsf(mof[v]);
      }
      const float mr0f = (float)mro[0];
      const float rho_thr = (float)p.eps_rho + screen_t * (maf[0] + dvo[0]);
      const float eps_pf = (float)p.eps_p;
      // tau_rho over the volume and face points
      double tau = 1.0;
      for (int pt = lane; pt < npt; pt += 32) {
        float acc = 0.f;
        for (int l = 1; l < g.n; ++l) acc += R[l][o] * tb.Pp[l * npt + pt];
        if (mr0f + acc < rho_thr) {
          double rd = mro[0];
          for (int l = 1; l < g.n; ++l) rd += (double)R[l][o] * (double)tb.Pp[l * npt + pt];
          if (rd < p.eps_rho) tau = fmin(tau, (mo[0] - p.eps_rho) / (mo[0] - rd));
        }
      }
      tau = fmax(wmin(tau), 0.0);
      // tau_p from the density-limited state m + tau (u - m)
      double taup = 1.0;
      const int nleg = g.glm ? 8 : 5;
      const float tt = (float)tau;
      for (int pt = lane; pt < npt; pt += 32) {
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          if (v >= nleg) continue;
          for (int l = 1; l < g.n; ++l) acc[v] += R[v * g.n + l][o] * tb.Pp[l * npt + pt];
        }
        if (!g.glm)
          for (int j = g.D; j < g.ndiv; ++j) {
            const float wj = R[g.ldf0 + j][o];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) acc[5 + cc] += wj * tb.Lp[(j * g.DB + cc) * npt + pt];
          }
        float uu[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) uu[v] = mof[v] + tt * acc[v];
        if (pos_point_open_f(uu, maf, dvo, tt, gm1t, eps_pf, screen_t)) {
          // FP64 recovery of this point's pressure
          double u[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
          const int nps = g.glm ? 9 : 5;
          for (int v = 0; v < nps; ++v) {
            double sv = mro[v];
            for (int l = 1; l < g.n; ++l) sv += (double)R[v * g.n + l][o] * (double)tb.Pp[l * npt + pt];
            u[v] = sv;
          }
          if (!g.glm)
            for (int j = 0; j < g.ndiv; ++j) {
              const double wj = j < g.D ? mro[5 + j] : (double)R[g.ldf0 + j][o];
              for (int cc = 0; cc < g.DB; ++cc) u[5 + cc] += wj * (double)tb.Lp[(j * g.DB + cc) * npt + pt];
            }
          for (int v = 0; v < 9; ++v) u[v] = mo[v] + tau * (u[v] - mo[v]);
          const double pq = pres(u);
          if (pq < p.eps_p) taup = fmin(taup, (pmo - p.eps_p) / (pmo - pq));
        }
      }
      taup = fmax(wmin(taup), 0.0);
      const double t = tau * taup;
      if (t >= 1.0) continue;
      if (lane == 0) atomicAdd(&sc->pos_cells, 1ull);
      // scale every non-mean row by tau
      for (int r = lane; r < NR; r += 32) {
        bool mean = false;
        for (int k = 0; k < nm; ++k)
          if (lmean_row(g, k) == r) mean = true;
        if (!mean) w[(int64_t)r * S + co] = (float)(t * (double)R[r][o]);
      }
    }
  }
}

}  // namespace

int upload_limiter_tables(Ctx& c) {
  const Basis& B = *c.hb;
  const Geom& g = c.g;
  LimTabs lt;
  std::memset(&lt, 0, sizeof(lt));
  for (int a = 0; a < g.D; ++a)
    for (int l = 0; l < g.n; ++l) {
      const auto& k = B.modes[l];
      if (k[0] + k[1] + k[2] == 1 && k[a] == 1) lt.deg1[a] = l;
    }
  for (int l = 0; l < g.n && l < 64; ++l) lt.mdeg[l] = B.modes[l][0] + B.modes[l][1] + B.modes[l][2];
  for (int j = 0; j < g.ndiv && j < 64; ++j) {
    lt.ldf_deg[j] = B.ldf_deg[j];
    // mean of each component (degree 0 rows only are non-zero)
    for (int cc = 0; cc < g.D; ++cc) {
      double z[3] = {0, 0, 0};
      lt.ldf_mean0[j * 3 + cc] = B.ldf_deg[j] == 0 ? B.eval(B.ldf[j][cc], z) : 0.0;
    }
  }
  // slope and projection tables by exact monomial integration
  const auto& ms = B.ms;
  auto integ = [&](const std::vector<double>& poly, int axis) {
    // int poly * xi_axis (axis < 0: int poly) over [-1,1]^D
    double s = 0.0;
    for (size_t i = 0; i < ms.exps.size(); ++i) {
      if (poly[i] == 0.0) continue;
      double t = poly[i];
      for (int ax = 0; ax < g.D; ++ax) {
        const int k = ms.exps[i][ax] + (ax == axis ? 1 : 0);
        t *= (k & 1) ? 0.0 : 2.0 / (k + 1.0);
      }
      s += t;
    }
    return s;
  };
  double xi2 = 1.0;
  for (int ax = 0; ax < g.D; ++ax) xi2 *= ax == 0 ? 2.0 / 3.0 : 2.0;
  for (int j = 0; j < g.ndiv && j < 64; ++j)
    for (int cc = 0; cc < g.D; ++cc) {
      const double Mj = B.ldf_mass[j];
      lt.ldf_pc[j * 3 + cc] = integ(B.ldf[j][cc], -1) / Mj;
      for (int a = 0; a < g.D; ++a) {
        const double ia = integ(B.ldf[j][cc], a);
        lt.ldf_slope[(j * 3 + cc) * 3 + a] = ia / xi2;
        lt.ldf_pl[(j * 3 + cc) * 3 + a] = ia / Mj;
      }
      double mx = 0.0;
      for (double v : B.ldf[j][cc]) mx += std::fabs(v);
      lt.ldf_maxabs[j * 3 + cc] = mx;
    }
  for (int i = 0; i < 64 * 3; ++i) {
    lt.ldf_mean0_f[i] = (float)lt.ldf_mean0[i];
    lt.ldf_pc_f[i] = (float)lt.ldf_pc[i];
  }
  for (int i = 0; i < 64 * 9; ++i) {
    lt.ldf_slope_f[i] = (float)lt.ldf_slope[i];
    lt.ldf_pl_f[i] = (float)lt.ldf_pl[i];
  }
  c.lim = lt;
  PosScreen& ps = c.pscr;
  std::memset(&ps, 0, sizeof(ps));
  for (int i = 0; i < 9; ++i) ps.ldf_mean0[i] = (float)lt.ldf_mean0[i];
  for (int i = 0; i < 64 * 3; ++i) ps.ldf_maxabs[i] = (float)lt.ldf_maxabs[i];
  ps.eps_rho = (float)c.p.eps_rho;
  ps.eps_p = (float)c.p.eps_p;
  ps.gm1 = (float)(g.gamma - 1.0);
  return DG_OK;
}

int run_limiter(Ctx& c, void* w, double* wmean, uint8_t* troubled, cudaStream_t st) {
  const Geom& g = c.g;
  const unsigned nb = (unsigned)((g.ncell + 127) / 128);
  bool screened = false;  // the positivity screen already ran (indicator: unflagged cells, TVB: flagged ones)
  if (c.p.limiter == DG_LIMIT_TVB || c.p.limiter == DG_LIMIT_MLP) {
    const int32_t* list = nullptr;
    unsigned nbt = nb;
    ++c.lim_passes;
    if (c.p.limiter == DG_LIMIT_MLP) {
      if (!c.mlp_w1) return DG_E_ARG;  // no weights set
      // the indicator appends the cells it flags to flag_list; only those go
      // through the TVB procedure (a persistent grid walks the list)
      if (troubled) cudaMemsetAsync(troubled, 0, (size_t)g.ncell, st);
      cudaMemsetAsync(&c.sc->nflag, 0, sizeof(unsigned), st);
      // FP32 form: the indicator's kernel also screens positivity on the rows it stages
      const bool fuse_pos = c.p.positivity && c.p.precision == DG_PREC_FP32MIX;
      if (fuse_pos) cudaMemsetAsync(&c.sc->npos, 0, sizeof(unsigned), st);
      c.prof.begin(6, st);
      const int e =
          mlp_infer_launch(c, w, wmean, nullptr, nullptr, st, c.flag_list, fuse_pos ? c.pos_list : nullptr, &screened);
      c.prof.end(6, st);
      if (e) return e;
      list = c.flag_list;
      nbt = (unsigned)std::min<int64_t>(nb, (int64_t)c.nsm * 16);
    } else {
      c.lim_plain_cells += g.ncell;
    }
    c.prof.begin(3, st);
    // FP32 form: the float mode-0 rows mirror the FP64 means exactly; reading
    // them avoids FP64 conversions (the limiter never changes the means)
    const AmrNb an{c.amr.fL,  c.amr.fR, c.amr.fmeta, c.amr.cstart, c.amr.centry, c.amr.dxc, c.amr.on ? 1 : 0,
                   c.amr.side_nb, c.amr.side_info};
    if (c.p.precision == DG_PREC_FP32MIX)
      screened ? k_tvb<float, true><<<nbt, 128, 0, st>>>(g, c.lim, (float*)w, nullptr, troubled, list, c.p, c.sc,
                                                          an, c.pos_list, c.pscr)
               : k_tvb<float, false><<<nbt, 128, 0, st>>>(g, c.lim, (float*)w, nullptr, troubled, list, c.p, c.sc,
                                                           an, nullptr, c.pscr);
    else
      k_tvb<double, false><<<nbt, 128, 0, st>>>(g, c.lim, (double*)w, nullptr, troubled, list, c.p, c.sc, an,
                                                nullptr, c.pscr);
    c.prof.end(3, st);
  }
  if (c.p.positivity) {
    c.prof.begin(5, st);
    if (c.p.precision == DG_PREC_FP32MIX) {
      // cheap FP32 screen over every cell; the full procedure only on the few
      // cells it lists (so a warp never waits on one lane's FP64 recovery)
      if (!screened) {
        cudaMemsetAsync(&c.sc->npos, 0, sizeof(unsigned), st);
        auto scr = [&](auto k) { k<<<nb, 128, 0, st>>>(g, c.pscr, (const float*)w, c.sc, c.pos_list); };
        if (!pinned_sizes_ok(g)) scr(k_pos_screen<-1, 0>);
        else if (g.d == 2) g.glm ? scr(k_pos_screen<2, 1>) : scr(k_pos_screen<2, 0>);
        else g.glm ? scr(k_pos_screen<1, 1>) : scr(k_pos_screen<1, 0>);
      }
      const unsigned nbl = (unsigned)std::min<int64_t>(nb, (int64_t)c.nsm * 16);
      auto pw = [&](auto k) { k<<<(unsigned)c.nsm * 8, 128, 0, st>>>(g, c.t32, c.lim, (float*)w, wmean, c.p, c.sc,
                                                                    c.pos_list); };
      if (!pinned_sizes_ok(g) || !wmean)
        k_pos<float><<<nbl, 128, 0, st>>>(g, c.t32, c.lim, (float*)w, wmean, c.p, c.sc, c.pos_list);
      else if (g.d == 2) g.glm ? pw(k_pos_list<2, 1>) : pw(k_pos_list<2, 0>);
      else g.glm ? pw(k_pos_list<1, 1>) : pw(k_pos_list<1, 0>);
      if (!screened) c.prof.launches[5] += 1;  // the screen and the list kernel
    } else {
      k_pos<double><<<nb, 128, 0, st>>>(g, c.t64, c.lim, (double*)w, nullptr, c.p, c.sc, nullptr);
    }
    c.prof.end(5, st);
  }
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_E_CUDA;
}

}  // namespace dgmhd
