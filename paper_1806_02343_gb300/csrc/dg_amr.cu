// Static octree meshes (Sec. 4.4): face lists, coarse-fine sub-face tables
// and the face-list kernels of the DG operator (Sec. 3.5 eq. wdot).
//
// Faces: same-level faces once (from the right cell's -a side); coarse-fine
// faces once per fine cell side, integrated at the FINE face's Gauss points.
// The coarse side evaluates its state at the same physical points, i.e. at
// reference coordinates xi_t = (xi_t,fine + (bit ? 1 : -1)) / 2 of its own
// face, and weighs them by w_p / 2^(D-1) (its reference face measure is 2^(D-1)
// times larger). F* is computed once per point and used by both cells, so the
// discretisation stays conservative. Each cell uses its own metric 2/dx_K.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "dg_amr.cuh"
#include "dg_fast.cuh"
#include "dg_phys.cuh"

namespace dgmhd {

namespace {

constexpr int WPB = 4;  // warps (cells) per block

__device__ __forceinline__ int mrow_a(const Geom& g, int m) {
  if (g.glm) return m * g.n;
  if (m < 5) return m * g.n;
  if (g.D == 3) return g.ldf0 + (m - 5);
  return m < 7 ? g.ldf0 + (m - 5) : g.bz2d;
}

__device__ __forceinline__ int mindex_a(const Geom& g, int r) {
  const int nm = g.glm ? 9 : 8;
  for (int m = 0; m < nm; ++m)
    if (mrow_a(g, m) == r) return m;
  return -1;
}

template <typename T, typename F>
__device__ __forceinline__ void eval_pt(const Geom& g, const T* __restrict__ P, const T* __restrict__ L, int npt,
                                        int pt, F coef, T* u) {
  for (int v = 0; v < g.V; ++v) u[v] = T(0);
  const int nleg = g.glm ? 9 : 5;
  for (int v = 0; v < nleg; ++v) {
    T s = T(0);
    for (int l = 0; l < g.n; ++l) s += coef(v * g.n + l) * P[l * npt + pt];
    u[v] = s;
  }
  if (!g.glm) {
    T b[3] = {T(0), T(0), T(0)};
    for (int j = 0; j < g.ndiv; ++j) {
      const T wj = coef(g.ldf0 + j);
      for (int c = 0; c < g.DB; ++c) b[c] += wj * L[(j * g.DB + c) * npt + pt];
    }
    for (int c = 0; c < g.DB; ++c) u[5 + c] = b[c];
    if (g.bz2d >= 0) {
      T s = T(0);
      for (int l = 0; l < g.n; ++l) s += coef(g.bz2d + l) * P[l * npt + pt];
      u[7] = s;
    }
  }
}

// table of side (cell is L: its +a face; R: its -a face), standard or sub-face
template <typename T>
struct SideTab {
  const T* P;
  const T* L;
  const T* P4;  // the same rows with the point index padded to pad4(Qf)
  const T* L4;
  bool coarse;
};

template <typename T>
__device__ __forceinline__ SideTab<T> side_tab(const Geom& g, const Tables<T>& tb, const AmrDev<T>& am, int meta,
                                              int side) {
  const int a = meta & 3, kind = (meta >> 2) & 3, sub = meta >> 4;
  const int f = side == 0 ? 2 * a + 1 : 2 * a;
  const bool coarse = (side == 0 && kind == 1) || (side == 1 && kind == 2);
  SideTab<T> t;
  const int qf4 = pad4(g.Qf);
  if (coarse) {
    t.P = am.Psub + ((size_t)(f * am.nsub + sub) * g.n) * g.Qf;
    t.L = am.Lsub + ((size_t)(f * am.nsub + sub) * g.ndiv * g.DB) * g.Qf;
    t.P4 = am.Psub4 + ((size_t)(f * am.nsub + sub) * g.n) * qf4;
    t.L4 = am.Lsub4 + ((size_t)(f * am.nsub + sub) * g.ndiv * g.DB) * qf4;
  } else {
    t.P = tb.Pf + (size_t)f * g.n * g.Qf;
    t.L = tb.Lf + (size_t)f * g.ndiv * g.DB * g.Qf;
    t.P4 = tb.Pf4 + (size_t)f * g.n * qf4;
    t.L4 = tb.Lf4 + (size_t)f * g.ndiv * g.DB * qf4;
  }
  t.coarse = coarse;
  return t;
}

template <typename T, int DEG, int GLMF>
__global__ void k_face_list(Geom gin, Tables<T> tb, AmrDev<T> am, const T* __restrict__ w, T* __restrict__ fbuf,
                            const DevScalars* __restrict__ sc, T eps, T* __restrict__ qbuf) {
  const Geom g = pin_geom<DEG, GLMF>(gin);
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= am.nface * g.Qf) return;
  const int64_t f = tid / g.Qf;
  const int p = (int)(tid % g.Qf);
  const int meta = am.fmeta[f];
  const int a = meta & 3;
  const int64_t cL = am.fL[f], cR = am.fR[f], S = g.stride;
  const SideTab<T> tl = side_tab(g, tb, am, meta, 0), tr = side_tab(g, tb, am, meta, 1);
  T uL[MAXV], uR[MAXV], F[MAXV];
  eval_pt(g, tl.P, tl.L, g.Qf, p, [&](int r) { return w[r * S + cL]; }, uL);
  eval_pt(g, tr.P, tr.L, g.Qf, p, [&](int r) { return w[r * S + cR]; }, uR);
  const T ch = g.glm ? (T)sc->ch : T(0);
  const T bnF = face_flux(uL, uR, a, (T)g.gamma, g.glm != 0, ch, eps, F, qbuf ? qbuf + tid * 14 : nullptr);
  T* o = fbuf + tid * 9;
  for (int k = 0; k < g.V; ++k) o[k] = F[k];
  if (!g.glm) o[8] = bnF;
}

// Per-warp shared memory of k_cell_list (elements): state rows, weighted
// volume fluxes, face terms and Powell jump terms of up to maxent face
// entries. VEC: point indices padded to a multiple of 4, regions 16-byte aligned.
__host__ __device__ inline int cell_list_warp_elems(const Geom& g, int maxent, bool vec) {
  const int qv = vec ? pad4(g.Qv) : g.Qv, qf = vec ? pad4(g.Qf) : g.Qf;
  const int nr = vec ? pad4(g.nrows) : g.nrows;
  const int e = nr + g.D * g.V * qv + maxent * qf * g.V + maxent * qf;
  return vec ? pad4(e) : e;
}

// VEC (3D, sizes fixed at compile time, padded tables present): the row
// contractions run as 16-byte vector loads.
constexpr int kEntryChunk = 6;  // face entries staged at a time (a leaf has 6 to 24)
constexpr int kRowsPerLane = 6;  // state rows per lane (at most 180 rows)

template <typename T, int DEG, int GLMF, bool VEC>
__global__ void k_cell_list(Geom gin, Tables<T> tb, AmrDev<T> am, const T* __restrict__ w,
                            const T* __restrict__ fbuf, T* out, const T* w0, double ca, double cb, int combine,
                            const DevScalars* __restrict__ sc, const double* __restrict__ wmean, const double* w0mean,
                            double* outmean, const T* __restrict__ qbuf) {
  const Geom g = pin_geom<DEG, GLMF>(gin);
  // out / outmean may alias w0 / w0mean: each element is read, then written, by one lane.
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * WPB + warp;
  const int QVP = VEC ? pad4(g.Qv) : g.Qv, QFP = VEC ? pad4(g.Qf) : g.Qf;
  const int che = am.maxent < kEntryChunk ? am.maxent : kEntryChunk;  // entries per staged chunk
  const int per_warp = cell_list_warp_elems(g, che, VEC);
  T* wc = reinterpret_cast<T*>(smraw) + (size_t)warp * per_warp;
  T* G = wc + (VEC ? pad4(g.nrows) : g.nrows);
  T* FS = G + g.D * g.V * QVP;
  T* PJ = FS + che * QFP * g.V;
  // face term of (chunk entry e, point p, variable v)
  auto fsi = [&](int e, int p, int v) { return VEC ? (e * g.V + v) * QFP + p : (e * g.Qf + p) * g.V + v; };
  if (c >= g.ncell) return;
  const int64_t S = g.stride;
  const bool mix = wmean != nullptr;
  for (int r = lane; r < g.nrows; r += 32) wc[r] = w[r * S + c];
  __syncwarp();
  if (mix && lane < (g.glm ? 9 : 8)) wc[mrow_a(g, lane)] = (T)wmean[lane * S + c];
  __syncwarp();
  const T gamma = (T)g.gamma;
  const T ch = g.glm ? (T)sc->ch : T(0);
  for (int q = lane; q < g.Qv; q += 32) {
    T u[MAXV];
    eval_pt(g, tb.Pv, tb.Lv, g.Qv, q, [&](int r) { return wc[r]; }, u);
    const T wq = tb.wv[q];
    for (int a = 0; a < g.D; ++a) {
      T f[MAXV];
      flux_dir(u, a, gamma, g.glm != 0, ch * ch, f);
      for (int v = 0; v < g.V; ++v) G[(a * g.V + v) * QVP + q] = wq * f[v];
    }
  }
  if (VEC)
    for (int i = lane; i < g.D * g.V * (QVP - g.Qv); i += 32)
      G[(i / (QVP - g.Qv)) * QVP + g.Qv + i % (QVP - g.Qv)] = T(0);
  __syncwarp();
  // Powell q(<u>_K) from the cell mean (zero when q^dagger is folded into the face terms)
  T qv[MAXV];
  if (!g.glm && qbuf) {
    for (int v = 0; v < MAXV; ++v) qv[v] = T(0);
  } else if (!g.glm) {
    const T rho = wc[0];
    const T vx = wc[g.n] / rho, vy = wc[2 * g.n] / rho, vz = wc[3 * g.n] / rho;
    T b[3] = {T(0), T(0), T(0)};
    for (int j = 0; j < g.DB; ++j)
      for (int cc = 0; cc < g.DB; ++cc) b[cc] += wc[g.ldf0 + j] * tb.L0[j * g.DB + cc];
    if (g.bz2d >= 0) b[2] = wc[g.bz2d];
    qv[0] = T(0); qv[1] = b[0]; qv[2] = b[1]; qv[3] = b[2];
    qv[4] = vx * b[0] + vy * b[1] + vz * b[2];
    qv[5] = vx; qv[6] = vy; qv[7] = vz; qv[8] = T(0);
  }
  // FP32 form: rows other than the degree-0 ones accumulate and combine in
  // FP32 (GB300's FP64 rate is 1/64 of FP32); the degree-0 rows keep FP64.
  // Each lane owns rows lane + 32 i; their accumulators live across the chunks.
  double acc[kRowsPerLane];
  T acct[kRowsPerLane];
  auto row_kind = [&](int r, bool& ldf, int& v, int& l) {
    ldf = g.ldf0 >= 0 && r >= g.ldf0 && r < g.ldf0 + g.ndiv;
    v = (g.bz2d >= 0 && r >= g.bz2d) ? 7 : r / g.n;
    l = ldf ? r - g.ldf0 : ((g.bz2d >= 0 && r >= g.bz2d) ? r - g.bz2d : r % g.n);
  };
  // volume terms
#pragma unroll
  for (int i = 0; i < kRowsPerLane; ++i) {
    acc[i] = 0.0;
    acct[i] = T(0);
    const int r = lane + 32 * i;
    if (r >= g.nrows) continue;
    const bool lowp = sizeof(T) == 4 && (mix ? mindex_a(g, r) : -1) < 0;
    bool ldf;
    int v, l;
    row_kind(r, ldf, v, l);
    T s = T(0);
    if (!ldf) {
      if (l != 0)
        for (int a = 0; a < g.D; ++a) {
          const T* Gp = G + (a * g.V + v) * QVP;
          if constexpr (VEC) {
            s += dotp<T, pad4((DEG + 1) * (DEG + 1) * (DEG + 1))>(Gp, tb.dPv4 + ((size_t)a * g.n + l) * QVP);
          } else {
            const T* Dp = tb.dPv + ((size_t)a * g.n + l) * g.Qv;
            for (int q = 0; q < g.Qv; ++q) s += Gp[q] * Dp[q];
          }
        }
    } else {
      for (int a = 0; a < g.D; ++a)
        for (int cc = 0; cc < g.DB; ++cc) {
          const T* Gp = G + (a * g.V + 5 + cc) * QVP;
          if constexpr (VEC) {
            s += dotp<T, pad4((DEG + 1) * (DEG + 1) * (DEG + 1))>(
                Gp, tb.dLv4 + (((size_t)a * g.ndiv + l) * g.DB + cc) * QVP);
          } else {
            const T* Dp = tb.dLv + (((size_t)a * g.ndiv + l) * g.DB + cc) * g.Qv;
            for (int q = 0; q < g.Qv; ++q) s += Gp[q] * Dp[q];
          }
        }
    }
    if (lowp) acct[i] += s; else acc[i] += (double)s;
  }
  // surface terms, the face entries staged kEntryChunk at a time
  const int e0 = am.cstart[c], ne = am.cstart[c + 1] - e0;
  const T subw = T(1) / T(am.nsub);
  for (int k0 = 0; k0 < ne; k0 += che) {
    const int nc = ne - k0 < che ? ne - k0 : che;
    __syncwarp();  // the previous chunk's reads are done
    if (VEC)
      for (int i = lane; i < nc * (g.V + 1) * (QFP - g.Qf); i += 32) {
        // zero padding of the point index (the padded tables are zero there too)
        const int row = i / (QFP - g.Qf), pp = g.Qf + i % (QFP - g.Qf);
        if (row < nc * g.V) FS[row * QFP + pp] = T(0);
        else PJ[(row - nc * g.V) * QFP + pp] = T(0);
      }
    for (int idx = lane; idx < nc * g.Qf; idx += 32) {
      const int e = idx / g.Qf, p = idx % g.Qf;
      const int ent = am.centry[e0 + k0 + e];
      const int64_t f = ent >> 1;
      const int side = ent & 1;
      const int meta = am.fmeta[f];
      const int a = meta & 3;
      const SideTab<T> t = side_tab(g, tb, am, meta, side);
      const T* F = fbuf + (f * g.Qf + p) * 9;
      // outward normal: +e_a for the left cell, -e_a for the right cell
      const T sgn = side == 0 ? T(1) : T(-1);
      const T wp = tb.wf[p] * (t.coarse ? subw : T(1));
      for (int v = 0; v < g.V; ++v) FS[fsi(e, p, v)] = sgn * wp * F[v];
      if (!g.glm) {
        T ba = T(0);
        for (int j = 0; j < g.ndiv; ++j) ba += wc[g.ldf0 + j] * t.L[(j * g.DB + a) * g.Qf + p];
        const T pj = wp * sgn * (F[8] - ba);
        PJ[e * QFP + p] = pj;
        if (qbuf) {
          // q^dagger of eq. powellq-interp at this point, own trace (side 0: left cell)
          const T* q = qbuf + (f * g.Qf + p) * 14 + (side == 0 ? 0 : 7);
          for (int v = 1; v < 8; ++v) FS[fsi(e, p, v)] += pj * q[v - 1];
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < kRowsPerLane; ++i) {
      const int r = lane + 32 * i;
      if (r >= g.nrows) continue;
      const bool lowp = sizeof(T) == 4 && (mix ? mindex_a(g, r) : -1) < 0;
      bool ldf;
      int v, l;
      row_kind(r, ldf, v, l);
      for (int e = 0; e < nc; ++e) {
        const int ent = am.centry[e0 + k0 + e];
        const SideTab<T> t = side_tab(g, tb, am, am.fmeta[ent >> 1], ent & 1);
        T sf = T(0);
        if (!ldf) {
          if constexpr (VEC) {
            constexpr int QF4 = pad4((DEG + 1) * (DEG + 1));
            const T* Pp = t.P4 + (size_t)l * QFP;
            sf = dotp<T, QF4>(FS + (e * g.V + v) * QFP, Pp);
            if (!g.glm) sf += qv[v] * dotp<T, QF4>(PJ + e * QFP, Pp);
          } else {
            const T* Pp = t.P + (size_t)l * g.Qf;
            for (int p = 0; p < g.Qf; ++p) {
              T term = FS[fsi(e, p, v)];
              if (!g.glm) term += PJ[e * QFP + p] * qv[v];
              sf += term * Pp[p];
            }
          }
        } else {
          for (int cc = 0; cc < g.DB; ++cc) {
            if constexpr (VEC) {
              constexpr int QF4 = pad4((DEG + 1) * (DEG + 1));
              const T* Lp = t.L4 + ((size_t)l * g.DB + cc) * QFP;
              sf += dotp<T, QF4>(FS + (e * g.V + 5 + cc) * QFP, Lp) + qv[5 + cc] * dotp<T, QF4>(PJ + e * QFP, Lp);
            } else {
              const T* Lp = t.L + ((size_t)l * g.DB + cc) * g.Qf;
              for (int p = 0; p < g.Qf; ++p)
                sf += (FS[fsi(e, p, 5 + cc)] + PJ[e * QFP + p] * qv[5 + cc]) * Lp[p];
            }
          }
        }
        if (lowp) acct[i] -= sf; else acc[i] -= (double)sf;
      }
    }
  }
  // combination and write
  const double dt = sc->dt;
  const double kappa = g.glm ? sc->kappa : 0.0;
  const double metric = 2.0 / am.dxc[c];
  const T tm = (T)metric, tdt = (T)dt, tca = (T)ca, tcb = (T)cb;
#pragma unroll
  for (int i = 0; i < kRowsPerLane; ++i) {
    const int r = lane + 32 * i;
    if (r >= g.nrows) continue;
    const int m = mix ? mindex_a(g, r) : -1;
    const bool lowp = sizeof(T) == 4 && m < 0;
    if (lowp) {
      T rt = tm * tb.minv[r] * acct[i];
      if (g.glm && r >= 8 * g.n) rt -= (T)kappa * wc[r];
      if (!combine) out[r * S + c] = rt;
      else out[r * S + c] = tca * w0[r * S + c] + tcb * (wc[r] + tdt * rt);
      continue;
    }
    double rhs = metric * (double)tb.minv[r] * acc[i];
    if (g.glm && r >= 8 * g.n) rhs -= kappa * (double)wc[r];
    if (!combine) {
      out[r * S + c] = (T)rhs;
      if (m >= 0) outmean[m * S + c] = rhs;
    } else if (m >= 0) {
      const double o = ca * w0mean[m * S + c] + cb * (wmean[m * S + c] + dt * rhs);
      outmean[m * S + c] = o;
      out[r * S + c] = (T)o;
    } else {
      out[r * S + c] = (T)(ca * (double)w0[r * S + c] + cb * ((double)wc[r] + dt * rhs));
    }
  }
}

// |B^n_F - B^n_K| weighted by w_p at every face point, for both sides
template <typename T>
__global__ void k_divb_list(Geom g, Tables<T> tb, AmrDev<T> am, const T* __restrict__ w, T* __restrict__ jbuf) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= am.nface * g.Qf) return;
  const int64_t f = tid / g.Qf;
  const int p = (int)(tid % g.Qf);
  const int meta = am.fmeta[f];
  const int a = meta & 3;
  const int64_t cL = am.fL[f], cR = am.fR[f], S = g.stride;
  const SideTab<T> tl = side_tab(g, tb, am, meta, 0), tr = side_tab(g, tb, am, meta, 1);
  T rL = T(0), rR = T(0), bL = T(0), bR = T(0);
  for (int l = 0; l < g.n; ++l) {
    rL += w[l * S + cL] * tl.P[l * g.Qf + p];
    rR += w[l * S + cR] * tr.P[l * g.Qf + p];
  }
  for (int j = 0; j < g.ndiv; ++j) {
    bL += w[(g.ldf0 + j) * S + cL] * tl.L[(j * g.DB + a) * g.Qf + p];
    bR += w[(g.ldf0 + j) * S + cR] * tr.L[(j * g.DB + a) * g.Qf + p];
  }
  const T bF = bn_face(rL, rR, bL, bR);
  const T wp = tb.wf[p];
  jbuf[tid * 2 + 0] = wp * (bF > bL ? bF - bL : bL - bF);
  jbuf[tid * 2 + 1] = wp * (bF > bR ? bF - bR : bR - bF);
}

__device__ __forceinline__ unsigned long long dbits_a(double x) { return (unsigned long long)__double_as_longlong(x); }

// FP64 bound of leaf c (eq. cfl, eq. powell_dt from the face jumps of its
// entries); *smax = the leaf's signal speed sum over the axes / D. Sets status
// bit 1 and returns DBL_MAX where the bound is not a positive finite number.
template <typename T>
__device__ double dt_leaf64(const Geom& g, const Tables<T>& tb, const AmrDev<T>& am, const T* __restrict__ w,
                            const double* __restrict__ wmean, const T* __restrict__ jbuf, const dg_mhd_params& p,
                            DevScalars* __restrict__ sc, int64_t c, double* smax) {
  const int64_t S = g.stride;
  auto mean = [&](int m) { return wmean ? wmean[m * S + c] : (double)w[(int64_t)mrow_a(g, m) * S + c]; };
  const double rho = mean(0);
  const double vx = mean(1) / rho, vy = mean(2) / rho, vz = mean(3) / rho;
  const double E = mean(4);
  double b[3];
  if (g.glm) {
    b[0] = mean(5); b[1] = mean(6); b[2] = mean(7);
  } else {
    b[0] = b[1] = b[2] = 0.0;
    for (int j = 0; j < g.DB; ++j)
      for (int cc = 0; cc < g.DB; ++cc) b[cc] += mean(5 + j) * (double)tb.L0[j * g.DB + cc];
    if (g.bz2d >= 0) b[2] = mean(7);
  }
  const double dx = am.dxc[c];
  const double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const double pr = (g.gamma - 1.0) * (E - 0.5 * rho * (vx * vx + vy * vy + vz * vz) - 0.5 * b2);
  const double cs = sqrt(g.gamma * pr / rho + b2 / rho);
  const double av[3] = {fabs(vx), fabs(vy), fabs(vz)};
  double s = 0.0;
  for (int a = 0; a < g.D; ++a) s += (av[a] + cs) / dx;
  double dtc = p.cfl / (2.0 * g.d + 1.0) / s;
  *smax = s * dx / g.D;
  if (!g.glm) {
    double acc = 0.0;
    for (int e = am.cstart[c]; e < am.cstart[c + 1]; ++e) {
      const int ent = am.centry[e];
      const int64_t f = ent >> 1;
      const double dxf = fmin(am.dxc[am.fL[f]], am.dxc[am.fR[f]]);
      double area = 1.0;
      for (int a = 0; a < g.D - 1; ++a) area *= 0.5 * dxf;
      double js = 0.0;
      const int nq = g.jq ? g.jq : g.Qf;
      for (int q = 0; q < nq; ++q) js += (double)jbuf[(f * nq + q) * 2 + (ent & 1)];
      acc += area * js;
    }
    double divb = acc;
    for (int a = 0; a < g.D; ++a) divb /= dx;
    const double rate = divb * fabs(vx * b[0] + vy * b[1] + vz * b[2]) / E;
    if (rate > 0.0) dtc = fmin(dtc, p.eta_powell / rate);
  }
  if (!(dtc > 0.0) || !isfinite(dtc)) {
    atomicOr(&sc->status, 1);
    dtc = DBL_MAX;
  }
  return dtc;
}

// The same bound in FP32 from the float mirror of the means (the screen of
// the FP32 form, as on uniform meshes): FP64 from the means where the FP32
// pressure would keep less than 1e-3 of E; FLT_MAX where not a positive
// finite number (status bit 1).
__device__ float dt_leaf32(const Geom& g, const Tables<float>& tb, const AmrDev<float>& am,
                           const float* __restrict__ w, const double* __restrict__ wmean,
                           const float* __restrict__ jbuf, const dg_mhd_params& p, DevScalars* __restrict__ sc,
                           int64_t c, float* smax) {
  const int64_t S = g.stride;
  auto mean = [&](int m) { return w[(int64_t)mrow_a(g, m) * S + c]; };
  const float gam = (float)g.gamma;
  const float rho = mean(0), ir = 1.f / rho;
  const float vx = mean(1) * ir, vy = mean(2) * ir, vz = mean(3) * ir;
  const float E = mean(4);
  float b[3];
  if (g.glm) {
    b[0] = mean(5); b[1] = mean(6); b[2] = mean(7);
  } else {
    b[0] = b[1] = b[2] = 0.f;
    for (int j = 0; j < g.DB; ++j)
      for (int cc = 0; cc < g.DB; ++cc) b[cc] += mean(5 + j) * tb.L0[j * g.DB + cc];
    if (g.bz2d >= 0) b[2] = mean(7);
  }
  const float b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  float pr = (gam - 1.f) * (E - 0.5f * rho * (vx * vx + vy * vy + vz * vz) - 0.5f * b2);
  if (!(pr > 1e-3f * E)) {
    double smd;
    const double d64 = dt_leaf64<float>(g, tb, am, w, wmean, jbuf, p, sc, c, &smd);
    *smax = (float)smd;
    return d64 < DBL_MAX ? (float)d64 : FLT_MAX;
  }
  const float dx = (float)am.dxc[c];
  const float cs = sqrtf((gam * pr + b2) * ir);
  const float av[3] = {fabsf(vx), fabsf(vy), fabsf(vz)};
  float sum = 0.f;
  for (int a = 0; a < g.D; ++a) sum += av[a] + cs;
  float dtc = (float)(p.cfl / (2.0 * g.d + 1.0)) * dx / sum;
  *smax = sum / (float)g.D;
  if (!g.glm) {
    float acc = 0.f;
    const int nq = g.jq ? g.jq : g.Qf;
    for (int e = am.cstart[c]; e < am.cstart[c + 1]; ++e) {
      const int ent = am.centry[e];
      const int64_t f = ent >> 1;
      const float dxf = (float)fmin(am.dxc[am.fL[f]], am.dxc[am.fR[f]]);
      float area = 1.f;
      for (int a = 0; a < g.D - 1; ++a) area *= 0.5f * dxf;
      float js = 0.f;
      for (int q = 0; q < nq; ++q) js += jbuf[(f * nq + q) * 2 + (ent & 1)];
      acc += area * js;
    }
    float divb = acc;
    for (int a = 0; a < g.D; ++a) divb /= dx;
    const float rate = divb * fabsf(vx * b[0] + vy * b[1] + vz * b[2]) / E;
    if (rate > 0.f) dtc = fminf(dtc, (float)p.eta_powell / rate);
  }
  if (!(dtc > 0.f) || !isfinite(dtc)) {
    atomicOr(&sc->status, 1);
    dtc = FLT_MAX;
  }
  return dtc;
}

// Pass 1 of the FP32 form's octree timestep: every leaf's FP32 bound, the
// minimum into dt_bits and the signal-speed maximum (block reduction).
__global__ void k_dt_list32(Geom g, Tables<float> tb, AmrDev<float> am, const float* __restrict__ w,
                            const double* __restrict__ wmean, const float* __restrict__ jbuf, dg_mhd_params p,
                            DevScalars* __restrict__ sc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float dtc = FLT_MAX, smax = 0.f;
  if (c < g.ncell && (!g.owned || g.owned[c])) dtc = dt_leaf32(g, tb, am, w, wmean, jbuf, p, sc, c, &smax);
  __shared__ float red[256];
  __shared__ float reds[256];
  red[threadIdx.x] = dtc;
  reds[threadIdx.x] = smax;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      red[threadIdx.x] = fminf(red[threadIdx.x], red[threadIdx.x + o]);
      reds[threadIdx.x] = fmaxf(reds[threadIdx.x], reds[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (red[0] < FLT_MAX) atomicMin(&sc->dt_bits, dbits_a((double)red[0]));
    atomicMax(&sc->smax_bits, dbits_a((double)reds[0]));
  }
}

// Pass 2: the FP64 bounds of the leaves whose FP32 bound lies within 1e-3
// (relative) of the FP32 minimum -- the FP32 bound is within 1e-4 of the FP64
// one, so the leaf holding the FP64 minimum is among them -- min-reduced in
// FP64 into dt64_bits, which the finalize step takes.
constexpr float kDtScreenA = 1e-3f;
__global__ void k_dt_list32_refine(Geom g, Tables<float> tb, AmrDev<float> am, const float* __restrict__ w,
                                   const double* __restrict__ wmean, const float* __restrict__ jbuf,
                                   dg_mhd_params p, DevScalars* __restrict__ sc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double dtc = DBL_MAX;
  if (c < g.ncell && (!g.owned || g.owned[c])) {
    const double m32 = __longlong_as_double((long long)sc->dt_bits);
    const float thr = m32 < DBL_MAX ? (float)m32 * (1.f + kDtScreenA) : -1.f;
    float sm32;
    const float d32 = dt_leaf32(g, tb, am, w, wmean, jbuf, p, sc, c, &sm32);
    if (d32 <= thr) {
      double sm64;
      dtc = dt_leaf64<float>(g, tb, am, w, wmean, jbuf, p, sc, c, &sm64);
    }
  }
  for (int o = 16; o > 0; o >>= 1) dtc = fmin(dtc, __shfl_xor_sync(0xffffffffu, dtc, o));
  if ((threadIdx.x & 31) == 0 && dtc < DBL_MAX) atomicMin(&sc->dt64_bits, dbits_a(dtc));
}

template <typename T>
__global__ void k_dt_list(Geom g, Tables<T> tb, AmrDev<T> am, const T* __restrict__ w,
                          const double* __restrict__ wmean, const T* __restrict__ jbuf, dg_mhd_params p,
                          DevScalars* __restrict__ sc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double dtc = DBL_MAX, smax = 0.0;
  if (c < g.ncell && (!g.owned || g.owned[c])) dtc = dt_leaf64<T>(g, tb, am, w, wmean, jbuf, p, sc, c, &smax);
  __shared__ double red[256];
  __shared__ double reds[256];
  red[threadIdx.x] = dtc;
  reds[threadIdx.x] = smax;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + o]);
      reds[threadIdx.x] = fmax(reds[threadIdx.x], reds[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicMin(&sc->dt_bits, dbits_a(red[0]));
    atomicMax(&sc->smax_bits, dbits_a(reds[0]));
  }
}

template <typename T>
int upload_vec(T** dst, const std::vector<T>& v) {
  if (cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(T)) != cudaSuccess) return DG_E_CUDA;
  if (!v.empty() && cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return DG_E_CUDA;
  return DG_OK;
}

}  // namespace

// -------------------------------------------------------------------- host
int build_amr(Ctx& c, const dg_mesh_desc* mesh) {
  Geom& g = c.g;
  const int D = mesh->dim;
  const int64_t N = mesh->n_leaves;
  // validation (a 2:1-balanced tiling of the cube) and the face lists, on the
  // Morton index of the leaves (kept for regridding)
  MortonIndex mi;
  std::vector<int32_t> fL, fR, fmeta, cstart, centry;
  int maxent = 0;
  const int ef =
      octree_faces(D, N, mesh->level, mesh->ijk, mi, fL, fR, fmeta, cstart, centry, maxent, mesh->partial != 0);
  if (ef) return ef;
  c.amr.partial = mesh->partial != 0;
  const int64_t nf = (int64_t)fL.size();
  std::vector<double> dxc(N);
  for (int64_t cidx = 0; cidx < N; ++cidx) dxc[cidx] = mesh->box_len / (double)(1ll << mesh->level[cidx]);
  // sub-face tables (coarse side), for each face f of the coarse cell and sub-face s
  const Basis& B = *c.hb;
  std::vector<double> x1, w1;
  gauss_legendre(g.nq1, x1, w1);
  const int nsub = 1 << (D - 1);
  std::vector<double> Ps((size_t)2 * D * nsub * g.n * g.Qf, 0.0);
  std::vector<double> Ls((size_t)std::max(1, 2 * D * nsub * g.ndiv * g.DB * g.Qf), 0.0);
  for (int f = 0; f < 2 * D; ++f) {
    const int a = f >> 1;
    int others[2], no = 0;
    for (int b = 0; b < D; ++b)
      if (b != a) others[no++] = b;
    for (int sb = 0; sb < nsub; ++sb)
      for (int p = 0; p < g.Qf; ++p) {
        double xi[3] = {0, 0, 0};
        int pp = p;
        for (int j = no - 1; j >= 0; --j) {
          const double xf = x1[pp % g.nq1];
          pp /= g.nq1;
          xi[others[j]] = 0.5 * (xf + (((sb >> j) & 1) ? 1.0 : -1.0));
        }
        xi[a] = (f & 1) ? 1.0 : -1.0;
        for (int l = 0; l < g.n; ++l) Ps[((size_t)(f * nsub + sb) * g.n + l) * g.Qf + p] = B.eval(B.leg[l], xi);
        for (int j = 0; j < g.ndiv; ++j)
          for (int cc = 0; cc < g.DB; ++cc)
            Ls[(((size_t)(f * nsub + sb) * g.ndiv + j) * g.DB + cc) * g.Qf + p] = B.eval(B.ldf[j][cc], xi);
      }
  }
  AmrHost& h = c.amr;
  h.on = true;
  h.D = D;
  h.hlevel.assign(mesh->level, mesh->level + N);
  h.hijk.assign(mesh->ijk, mesh->ijk + N * D);
  h.morton = std::move(mi);
  h.nface = nf;
  h.maxent = maxent;
  h.nsub = nsub;
  int e;
  if ((e = upload_vec(&h.fL, fL)) || (e = upload_vec(&h.fR, fR)) || (e = upload_vec(&h.fmeta, fmeta)) ||
      (e = upload_vec(&h.cstart, cstart)) || (e = upload_vec(&h.centry, centry)) || (e = upload_vec(&h.dxc, dxc)))
    return e;
  std::vector<float> Psf(Ps.begin(), Ps.end()), Lsf(Ls.begin(), Ls.end());
  if ((e = upload_vec(&h.Psub64, Ps)) || (e = upload_vec(&h.Lsub64, Ls)) || (e = upload_vec(&h.Psub32, Psf)) ||
      (e = upload_vec(&h.Lsub32, Lsf)))
    return e;
  // point index padded to a multiple of 4 (zeros), for the vector contractions
  const int qf4 = pad4(g.Qf);
  auto padded = [&](const std::vector<double>& src) {
    std::vector<double> out(src.size() / g.Qf * qf4, 0.0);
    for (size_t r = 0; r < src.size() / g.Qf; ++r)
      for (int k = 0; k < g.Qf; ++k) out[r * qf4 + k] = src[r * g.Qf + k];
    return out;
  };
  const std::vector<double> Ps4 = padded(Ps), Ls4 = padded(Ls);
  std::vector<float> Ps4f(Ps4.begin(), Ps4.end()), Ls4f(Ls4.begin(), Ls4.end());
  if ((e = upload_vec(&h.Psub64p, Ps4)) || (e = upload_vec(&h.Lsub64p, Ls4)) || (e = upload_vec(&h.Psub32p, Ps4f)) ||
      (e = upload_vec(&h.Lsub32p, Ls4f)))
    return e;
  double dmin = DBL_MAX;
  for (double d : dxc) dmin = std::min(dmin, d);
  g.dx = dmin;
  // the leaves across each side of every leaf, for the limiter's neighbour means
  {
    std::vector<int32_t> snb((size_t)N * 24, -1);
    std::vector<uint8_t> sinf((size_t)N * 6, 0);
    for (int64_t cc = 0; cc < N; ++cc)
      for (int e2 = cstart[cc]; e2 < cstart[cc + 1]; ++e2) {
        const int ent = centry[e2];
        const int64_t f = ent >> 1;
        const int side = ent & 1, m = fmeta[f], a = m & 3, kind = (m >> 2) & 3;
        const int sidx = 2 * a + (side == 0 ? 1 : 0);
        const int cnt = sinf[(size_t)cc * 6 + sidx] & 15;
        if (cnt >= 4) return DG_E_MESH;  // more than 2^(D-1) leaves across one side: not 2:1 balanced
        snb[(size_t)cc * 24 + sidx * 4 + cnt] = side == 0 ? fR[f] : fL[f];
        const bool self_coarse = (side == 0 && kind == 1) || (side == 1 && kind == 2);
        const int rel = kind == 0 ? 0 : (self_coarse ? 1 : 2);
        sinf[(size_t)cc * 6 + sidx] = (uint8_t)((cnt + 1) | (rel << 4));
      }
    int e3;
    if ((e3 = upload_vec(&h.side_nb, snb)) || (e3 = upload_vec(&h.side_info, sinf))) return e3;
  }
  // specialised Powell kernels: faces grouped by type in blocks of <= 32, and
  // the tables of each type (the std tables: the full face; coarse sides: the
  // sub-face tables Ps above)
  if (!g.glm && D == 3 && (g.d == 1 || g.d == 2) && c.p.generic_kernels != 1 && c.p.powell_q != 1) {
    const int n = g.n, Qf = g.Qf, QFP = Qf + (Qf & 1);
    std::vector<std::vector<int32_t>> by_type(27);
    for (int64_t f = 0; f < nf; ++f) {
      const int m = fmeta[f], a = m & 3, kind = (m >> 2) & 3, sb = m >> 4;
      by_type[a * 9 + (kind == 0 ? 0 : kind == 1 ? 1 + sb : 5 + sb)].push_back((int32_t)f);
    }
    std::vector<int32_t> bface, bstart, btype;
    bface.reserve(nf);
    for (int ty = 0; ty < 27; ++ty) {
      const auto& L = by_type[ty];
      for (size_t k = 0; k < L.size(); k += 32) {
        bstart.push_back((int32_t)(bface.size() + k));
        btype.push_back(ty | (int32_t)(std::min<size_t>(32, L.size() - k) << 8));
      }
      bface.insert(bface.end(), L.begin(), L.end());
    }
    // Legendre values on the full face f (its tangential axes in increasing
    // order, the last fastest), and face_val: full face (sb < 0) or sub-face sb
    std::vector<double> Pfull((size_t)2 * D * n * Qf);
    for (int f = 0; f < 2 * D; ++f) {
      const int a = f >> 1;
      int others[2], no = 0;
      for (int b = 0; b < D; ++b)
        if (b != a) others[no++] = b;
      for (int p = 0; p < Qf; ++p) {
        double xi[3] = {0, 0, 0};
        int pp = p;
        for (int j = no - 1; j >= 0; --j) {
          xi[others[j]] = x1[pp % g.nq1];
          pp /= g.nq1;
        }
        xi[a] = (f & 1) ? 1.0 : -1.0;
        for (int l = 0; l < n; ++l) Pfull[((size_t)f * n + l) * Qf + p] = B.eval(B.leg[l], xi);
      }
    }
    auto face_val = [&](int f, int sb, int l, int p) {
      return sb < 0 ? Pfull[((size_t)f * n + l) * Qf + p] : Ps[((size_t)(f * nsub + sb) * n + l) * Qf + p];
    };
    std::vector<double> ftab((size_t)27 * 2 * n * QFP, 0.0), ctab((size_t)30 * Qf * n, 0.0);
    for (int ty = 0; ty < 27; ++ty) {
      const int a = ty / 9, k = ty % 9;
      const int sbL = (k >= 1 && k <= 4) ? k - 1 : -1, sbR = k >= 5 ? k - 5 : -1;
      for (int l = 0; l < n; ++l)
        for (int p = 0; p < Qf; ++p) {
          ftab[(((size_t)ty * 2 + 0) * n + l) * QFP + p] = face_val(2 * a + 1, sbL, l, p);
          ftab[(((size_t)ty * 2 + 1) * n + l) * QFP + p] = face_val(2 * a, sbR, l, p);
        }
    }
    // normal component (axis a) of every LDF function on each type's two (sub-)faces
    const int nd = g.ndiv;
    std::vector<double> ntab((size_t)27 * 2 * nd * QFP, 0.0);
    for (int ty = 0; ty < 27; ++ty) {
      const int a = ty / 9, k = ty % 9;
      const int sbL = (k >= 1 && k <= 4) ? k - 1 : -1, sbR = k >= 5 ? k - 5 : -1;
      for (int sd = 0; sd < 2; ++sd) {
        const int f = sd == 0 ? 2 * a + 1 : 2 * a, sb = sd == 0 ? sbL : sbR;
        int others[2], no = 0;
        for (int b = 0; b < D; ++b)
          if (b != a) others[no++] = b;
        for (int p = 0; p < Qf; ++p) {
          double xi[3] = {0, 0, 0};
          int pp = p;
          for (int j = no - 1; j >= 0; --j) {
            const double xf = x1[pp % g.nq1];
            pp /= g.nq1;
            xi[others[j]] = sb < 0 ? xf : 0.5 * (xf + (((sb >> j) & 1) ? 1.0 : -1.0));
          }
          xi[a] = (f & 1) ? 1.0 : -1.0;
          for (int j = 0; j < nd; ++j)
            ntab[(((size_t)ty * 2 + sd) * nd + j) * QFP + p] = B.eval(B.ldf[j][a], xi);
        }
      }
    }
    std::vector<double> wf(Qf, 1.0);
    for (int p = 0; p < Qf; ++p)
      for (int k = 0, pp = p; k < D - 1; ++k, pp /= g.nq1) wf[p] *= w1[pp % g.nq1];
    for (int t = 0; t < 30; ++t) {
      const int f = t < 6 ? t : (t - 6) / 4, sb = t < 6 ? -1 : (t - 6) % 4;
      for (int p = 0; p < Qf; ++p)
        for (int l = 0; l < n; ++l)
          ctab[((size_t)t * Qf + p) * n + l] = face_val(f, sb, l, p) * wf[p] * (sb < 0 ? 1.0 : 1.0 / nsub);
    }
    if ((e = upload_vec(&h.bface, bface)) || (e = upload_vec(&h.bstart, bstart)) || (e = upload_vec(&h.btype, btype)))
      return e;
    if (c.p.precision == DG_PREC_FP32MIX) {
      std::vector<float> a(ftab.begin(), ftab.end()), b(ctab.begin(), ctab.end()), nt(ntab.begin(), ntab.end());
      if ((e = upload_vec((float**)&h.ftab, a)) || (e = upload_vec((float**)&h.ctab, b)) ||
          (e = upload_vec((float**)&h.ntab, nt)))
        return e;
    } else {
      if ((e = upload_vec((double**)&h.ftab, ftab)) || (e = upload_vec((double**)&h.ctab, ctab)) ||
          (e = upload_vec((double**)&h.ntab, ntab)))
        return e;
    }
    h.nblk = (int64_t)btype.size();
    h.fast = true;
  }
  return DG_OK;
}

OctPow<float> oct_pow32(const Ctx& c) {
  const AmrHost& h = c.amr;
  return OctPow<float>{h.fL, h.fR, h.fmeta, h.cstart, h.centry, h.dxc, h.bface, h.bstart, h.btype,
                       (const float*)h.ftab, (const float*)h.ctab, (const float*)h.ntab, c.g.ncell, c.g.stride,
                       h.nblk};
}
OctPow<double> oct_pow64(const Ctx& c) {
  const AmrHost& h = c.amr;
  return OctPow<double>{h.fL, h.fR, h.fmeta, h.cstart, h.centry, h.dxc, h.bface, h.bstart, h.btype,
                        (const double*)h.ftab, (const double*)h.ctab, (const double*)h.ntab, c.g.ncell,
                        c.g.stride, h.nblk};
}

void free_amr(Ctx& c) {
  AmrHost& h = c.amr;
  void* ptrs[] = {h.fL,     h.fR,     h.fmeta,    h.cstart,   h.centry,   h.dxc,    h.Psub64, h.Lsub64,
                  h.Psub32, h.Lsub32, h.Psub64p, h.Lsub64p, h.Psub32p, h.Lsub32p, h.groups, h.lev_dev,
                  h.bface,  h.bstart, h.btype,    h.ftab,     h.ctab,     h.ntab,     h.side_nb, h.side_info};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  h = AmrHost();
}

template <typename T>
AmrDev<T> amr_dev(const Ctx& c);
template <>
AmrDev<double> amr_dev<double>(const Ctx& c) {
  const AmrHost& h = c.amr;
  return AmrDev<double>{h.fL, h.fR, h.fmeta, h.cstart, h.centry, h.dxc, h.Psub64, h.Lsub64, h.Psub64p, h.Lsub64p,
                         h.nface, h.maxent, h.nsub};
}
template <>
AmrDev<float> amr_dev<float>(const Ctx& c) {
  const AmrHost& h = c.amr;
  return AmrDev<float>{h.fL, h.fR, h.fmeta, h.cstart, h.centry, h.dxc, h.Psub32, h.Lsub32, h.Psub32p, h.Lsub32p,
                        h.nface, h.maxent, h.nsub};
}

template <typename T>
void launch_amr_operator(const Ctx& c, const Tables<T>& tb, const T* w, T* fbuf, T* out, const T* w0, double ca,
                         double cb, int combine, const DevScalars* sc, const double* wmean, const double* w0mean,
                         double* outmean, double eps, cudaStream_t st, T* qbuf) {
  const Geom& g = c.g;
  const AmrDev<T> am = amr_dev<T>(c);
  const int64_t np = am.nface * g.Qf;
  // FP32 only: FP64 is bound by its multiply-add rate, which the padding would raise
  const bool vec = sizeof(T) == 4 && pinned_sizes_ok(g) && tb.dPv4 && tb.dLv4 && tb.Pf4 && tb.Lf4 && am.Psub4 &&
                   am.Lsub4;
  const size_t sm = (size_t)cell_list_warp_elems(g, std::min(am.maxent, kEntryChunk), vec) * WPB * sizeof(T);
  auto run = [&](auto face_k, auto cell_k) {
    face_k<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(g, tb, am, w, fbuf, sc, (T)eps, qbuf);
    cudaFuncSetAttribute(cell_k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cell_k<<<(unsigned)((g.ncell + WPB - 1) / WPB), 32 * WPB, sm, st>>>(g, tb, am, w, fbuf, out, w0, ca, cb, combine,
                                                                       sc, wmean, w0mean, outmean, qbuf);
  };
  // compile-time sizes for the 3D degree-1 and degree-2 schemes
  if (!pinned_sizes_ok(g)) run(k_face_list<T, -1, 0>, k_cell_list<T, -1, 0, false>);
  else if (!vec) {
    if (g.d == 2) g.glm ? run(k_face_list<T, 2, 1>, k_cell_list<T, 2, 1, false>)
                        : run(k_face_list<T, 2, 0>, k_cell_list<T, 2, 0, false>);
    else g.glm ? run(k_face_list<T, 1, 1>, k_cell_list<T, 1, 1, false>)
               : run(k_face_list<T, 1, 0>, k_cell_list<T, 1, 0, false>);
  } else if (g.d == 2) {
    g.glm ? run(k_face_list<T, 2, 1>, k_cell_list<T, 2, 1, true>) : run(k_face_list<T, 2, 0>, k_cell_list<T, 2, 0, true>);
  } else {
    g.glm ? run(k_face_list<T, 1, 1>, k_cell_list<T, 1, 1, true>) : run(k_face_list<T, 1, 0>, k_cell_list<T, 1, 0, true>);
  }
}

// the Powell face jumps by the specialised kernel where the context has it
bool divb_list_fast(const Ctx& c, const float* w, float* jbuf, cudaStream_t st) {
  if (!c.amr.fast) return false;
  if (c.fast == 11) launch_divb_list_pow<float, 1>(oct_pow32(c), w, jbuf, st);
  else if (c.fast == 12) launch_divb_list_pow<float, 2>(oct_pow32(c), w, jbuf, st);
  else return false;
  return true;
}
bool divb_list_fast(const Ctx& c, const double* w, double* jbuf, cudaStream_t st) {
  if (!c.amr.fast) return false;
  if (c.fast == 21) launch_divb_list_pow<double, 1>(oct_pow64(c), w, jbuf, st);
  else if (c.fast == 22) launch_divb_list_pow<double, 2>(oct_pow64(c), w, jbuf, st);
  else return false;
  return true;
}

template <typename T>
void launch_amr_dt(const Ctx& c, const Tables<T>& tb, const T* w, const double* wmean, T* jbuf,
                   const dg_mhd_params& p, DevScalars* sc, cudaStream_t st) {
  Geom g = c.g;
  const AmrDev<T> am = amr_dev<T>(c);
  if (!g.glm && divb_list_fast(c, w, jbuf, st)) {
    g.jq = 1;  // two sums per face
  } else if (!g.glm) {
    const int64_t np = am.nface * g.Qf;
    k_divb_list<T><<<(unsigned)((np + 127) / 128), 128, 0, st>>>(g, tb, am, w, jbuf);
  }
  if constexpr (sizeof(T) == 4) {
    if (wmean) {
      // FP32 form: FP32 screen of every leaf, FP64 bounds of the candidates
      k_dt_list32<<<(unsigned)((g.ncell + 255) / 256), 256, 0, st>>>(g, tb, am, w, wmean, jbuf, p, sc);
      k_dt_list32_refine<<<(unsigned)((g.ncell + 255) / 256), 256, 0, st>>>(g, tb, am, w, wmean, jbuf, p, sc);
      return;
    }
  }
  k_dt_list<T><<<(unsigned)((g.ncell + 255) / 256), 256, 0, st>>>(g, tb, am, w, wmean, jbuf, p, sc);
}

template void launch_amr_operator<double>(const Ctx&, const Tables<double>&, const double*, double*, double*,
                                          const double*, double, double, int, const DevScalars*, const double*,
                                          const double*, double*, double, cudaStream_t, double*);
template void launch_amr_operator<float>(const Ctx&, const Tables<float>&, const float*, float*, float*,
                                         const float*, double, double, int, const DevScalars*, const double*,
                                         const double*, double*, double, cudaStream_t, float*);
template void launch_amr_dt<double>(const Ctx&, const Tables<double>&, const double*, const double*, double*,
                                    const dg_mhd_params&, DevScalars*, cudaStream_t);
template void launch_amr_dt<float>(const Ctx&, const Tables<float>&, const float*, const double*, float*,
                                   const dg_mhd_params&, DevScalars*, cudaStream_t);

}  // namespace dgmhd
