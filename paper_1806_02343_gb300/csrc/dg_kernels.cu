// CUDA-core kernels of the DG-MHD operator (Sec. 3.5 eq. wdot, Sec. 4.1).
//
// k_face   one thread per (axis, cell, face point): traces of both cells at the
//          face point (modal -> nodal, Sec. 3.1), B^n_F (eq. bxface-average-alfven),
//          HLLD (Sec. 4.1.2) and, for GLM, the upwinded psi*, B_n* (Sec. 4.1.5).
//          Writes F* and B^n_F per face point to a face buffer.
// k_cell   one warp per cell: volume fluxes at the Gauss points and the volume
//          integral int f_a . d_a phi_l, the surface integral of F*.n phi_l over
//          the cell's 2D faces, the Powell face term of eq. powell-src-face with
//          q(<u>_K) (eq. powellq-average), the GLM damping source, the mass
//          matrix and the 2/dx metric factor; optionally the SSP-RK combination.
// k_dt     eq. cfl per cell from the cell mean, eq. powell_dt from the face
//          jumps of eq. divb-cell; min-reduced with an atomicMin on the bits.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "dg_kernels.cuh"
#include "dg_phys.cuh"

namespace dgmhd {

namespace {

constexpr int WARPS_PER_BLOCK = 4;

__device__ __forceinline__ void cell_coords(const Geom& g, int64_t c, int& ix, int& iy, int& iz) {
  ix = (int)(c % g.nx);
  int64_t r = c / g.nx;
  iy = (int)(r % g.ny);
  iz = (int)(r / g.ny);
}

__device__ __forceinline__ int64_t cell_index(const Geom& g, int ix, int iy, int iz) {
  return ((int64_t)iz * g.ny + iy) * g.nx + ix;
}

__device__ __forceinline__ int64_t neighbour(const Geom& g, int64_t c, int a, int dir) {
  int ix, iy, iz;
  cell_coords(g, c, ix, iy, iz);
  if (a == 0) ix = (ix + dir + g.nx) % g.nx;
  else if (a == 1) iy = (iy + dir + g.ny) % g.ny;
  else iz = (iz + dir + g.nz) % g.nz;
  return cell_index(g, ix, iy, iz);
}

// state variable of a Legendre row (Powell: rows < ldf0 are hydro, rows >= bz2d are B_z)
__device__ __forceinline__ int legendre_var(const Geom& g, int r) {
  if (g.bz2d >= 0 && r >= g.bz2d) return 7;
  return r / g.n;
}

__device__ __forceinline__ bool is_ldf_row(const Geom& g, int r) {
  return g.ldf0 >= 0 && r >= g.ldf0 && r < g.ldf0 + g.ndiv;
}

// mean row m -> DoF row
__device__ __forceinline__ int mean_row(const Geom& g, int m) {
  if (g.glm) return m * g.n;
  if (m < 5) return m * g.n;
  if (g.D == 3) return g.ldf0 + (m - 5);
  return m < 7 ? g.ldf0 + (m - 5) : g.bz2d;
}

__device__ __forceinline__ int n_mean_rows(const Geom& g) { return g.glm ? 9 : 8; }

// DoF row -> mean row index, or -1
__device__ __forceinline__ int mean_index(const Geom& g, int r) {
  for (int m = 0; m < n_mean_rows(g); ++m)
    if (mean_row(g, m) == r) return m;
  return -1;
}

// Evaluate the state at point index `pt` of a point set given by tables
// P (Legendre, [l][npt]) and L (LDF, [j][c][npt]); coefficients read through `coef`.
template <typename T, typename F>
__device__ __forceinline__ void eval_state(const Geom& g, const T* __restrict__ P, const T* __restrict__ L,
                                           int npt, int pt, F coef, T* u) {
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

// ---------------------------------------------------------------- face fluxes
template <typename T, int DEG, int GLMF>
__global__ void k_face(Geom gin, Tables<T> tb, const T* __restrict__ w, T* __restrict__ fbuf,
                       const DevScalars* __restrict__ sc, T eps, T* __restrict__ qbuf) {
  const Geom g = pin_geom<DEG, GLMF>(gin);
  const int64_t total = (int64_t)g.D * g.ncell * g.Qf;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= total) return;
  const int p = (int)(tid % g.Qf);
  const int64_t fc = tid / g.Qf;
  const int64_t c = fc % g.ncell;
  const int a = (int)(fc / g.ncell);
  const int64_t cl = neighbour(g, c, a, -1);
  const int64_t S = g.stride;
  T uL[MAXV], uR[MAXV];
  const int fL = 2 * a + 1, fR = 2 * a;
  eval_state(g, tb.Pf + (size_t)fL * g.n * g.Qf, tb.Lf + (size_t)fL * g.ndiv * g.DB * g.Qf, g.Qf, p,
             [&](int r) { return w[r * S + cl]; }, uL);
  eval_state(g, tb.Pf + (size_t)fR * g.n * g.Qf, tb.Lf + (size_t)fR * g.ndiv * g.DB * g.Qf, g.Qf, p,
             [&](int r) { return w[r * S + c]; }, uR);
  T F[MAXV];
  const T ch = g.glm ? (T)sc->ch : T(0);
  const T bnF = face_flux(uL, uR, a, (T)g.gamma, g.glm != 0, ch, eps, F, qbuf ? qbuf + tid * 14 : nullptr);
  T* o = fbuf + tid * 9;
  for (int k = 0; k < g.V; ++k) o[k] = F[k];
  if (!g.glm) o[8] = bnF;
}

// ---------------------------------------------------------------- cell update
// Per-warp shared memory of k_cell (elements): state rows, weighted volume
// fluxes G, face terms FS and Powell jump terms PJ. VEC: point indices padded
// to a multiple of 4 and every region 16-byte aligned (vector loads).
__host__ __device__ inline int cell_warp_elems(const Geom& g, bool vec) {
  const int qv = vec ? pad4(g.Qv) : g.Qv, qf = vec ? pad4(g.Qf) : g.Qf;
  const int nr = vec ? pad4(g.nrows) : g.nrows;
  const int e = nr + g.D * g.V * qv + 2 * g.D * qf * g.V + 2 * g.D * qf;
  return vec ? pad4(e) : e;
}

// VEC (3D, sizes fixed at compile time, padded tables present): the row
// contractions run as 16-byte vector loads of the fluxes and the tables
// (four multiply-adds per pair of loads instead of one).
template <typename T, int DEG, int GLMF, bool VEC>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK, VEC ? 8 : 1) k_cell(Geom gin, Tables<T> tb, const T* __restrict__ w, const T* __restrict__ fbuf, T* out,
                       const T* w0, double ca, double cb, int combine, const DevScalars* __restrict__ sc,
                       const double* __restrict__ wmean, const double* w0mean, double* outmean,
                       const T* __restrict__ qbuf) {
  const Geom g = pin_geom<DEG, GLMF>(gin);
  // out may alias w0 (in-place final stage): each element is read and then
  // written by the same thread.
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * WARPS_PER_BLOCK + warp;
  const int QVP = VEC ? pad4(g.Qv) : g.Qv, QFP = VEC ? pad4(g.Qf) : g.Qf;
  const int per_warp = cell_warp_elems(g, VEC);
  T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)warp * per_warp;
  T* wc = sm;
  T* G = wc + (VEC ? pad4(g.nrows) : g.nrows);
  T* FS = G + g.D * g.V * QVP;
  T* PJ = FS + 2 * g.D * QFP * g.V;
  // face term of (face f, point p, variable v)
  auto fsi = [&](int f, int p, int v) { return VEC ? (f * g.V + v) * QFP + p : (f * g.Qf + p) * g.V + v; };
  if (c >= g.ncell) return;
  const int64_t S = g.stride;
  const bool mix = (wmean != nullptr);
  for (int r = lane; r < g.nrows; r += 32) wc[r] = w[r * S + c];
  __syncwarp();
  if (mix && lane < n_mean_rows(g)) wc[mean_row(g, lane)] = (T)wmean[lane * S + c];
  __syncwarp();
  const T gamma = (T)g.gamma;
  const T ch = g.glm ? (T)sc->ch : T(0);
  const T ch2 = ch * ch;
  // volume: fluxes at the Gauss points, weighted
  for (int q = lane; q < g.Qv; q += 32) {
    T u[MAXV];
    eval_state(g, tb.Pv, tb.Lv, g.Qv, q, [&](int r) { return wc[r]; }, u);
    const T wq = tb.wv[q];
    for (int a = 0; a < g.D; ++a) {
      T f[MAXV];
      flux_dir(u, a, gamma, g.glm != 0, ch2, f);
      for (int v = 0; v < g.V; ++v) G[(a * g.V + v) * QVP + q] = wq * f[v];
    }
  }
  if (VEC) {
    // zero padding of the point index (the padded tables are zero there too)
    for (int i = lane; i < g.D * g.V * (QVP - g.Qv); i += 32)
      G[(i / (QVP - g.Qv)) * QVP + g.Qv + i % (QVP - g.Qv)] = T(0);
    for (int i = lane; i < 2 * g.D * (g.V + 1) * (QFP - g.Qf); i += 32) {
      const int row = i / (QFP - g.Qf), pp = g.Qf + i % (QFP - g.Qf);
      if (row < 2 * g.D * g.V) FS[row * QFP + pp] = T(0);
      else PJ[(row - 2 * g.D * g.V) * QFP + pp] = T(0);
    }
  }
  // faces: outward-normal flux times weights, Powell jump terms
  for (int idx = lane; idx < 2 * g.D * g.Qf; idx += 32) {
    const int f = idx / g.Qf, p = idx % g.Qf;
    const int a = f >> 1, side = f & 1;
    const int64_t fc = side ? neighbour(g, c, a, +1) : c;
    const T* F = fbuf + (((int64_t)a * g.ncell + fc) * g.Qf + p) * 9;
    const T sgn = side ? T(1) : T(-1);
    const T wp = tb.wf[p];
    for (int v = 0; v < g.V; ++v) FS[fsi(f, p, v)] = sgn * wp * F[v];
    if (!g.glm) {
      // own normal field B_a at this face point (LDF rows)
      T ba = T(0);
      for (int j = 0; j < g.ndiv; ++j)
        ba += wc[g.ldf0 + j] * tb.Lf[(((size_t)f * g.ndiv + j) * g.DB + a) * g.Qf + p];
      const T pj = wp * sgn * (F[8] - ba);
      PJ[f * QFP + p] = pj;
      if (qbuf) {
        // q^dagger of eq. powellq-interp at this point, own trace: the +a face
        // (side 1) has this cell on its left, the -a face on its right
        const T* q = qbuf + (((int64_t)a * g.ncell + fc) * g.Qf + p) * 14 + (side ? 0 : 7);
        for (int v = 1; v < 8; ++v) FS[fsi(f, p, v)] += pj * q[v - 1];
      }
    }
  }
  __syncwarp();
  // Powell q(<u>_K) = (0, B, v.B, v) from the cell mean (zero when q^dagger
  // is folded into the face terms)
  T qv[MAXV];
  if (!g.glm && qbuf) {
    for (int v = 0; v < MAXV; ++v) qv[v] = T(0);
  } else if (!g.glm) {
    const T rho = wc[0];
    const T vx = wc[g.n] / rho, vy = wc[2 * g.n] / rho, vz = wc[3 * g.n] / rho;
    T b[3] = {T(0), T(0), T(0)};
    for (int j = 0; j < g.DB; ++j)  // degree-0 LDF rows come first
      for (int cc = 0; cc < g.DB; ++cc) b[cc] += wc[g.ldf0 + j] * tb.L0[j * g.DB + cc];
    if (g.bz2d >= 0) b[2] = wc[g.bz2d];
    qv[0] = T(0); qv[1] = b[0]; qv[2] = b[1]; qv[3] = b[2];
    qv[4] = vx * b[0] + vy * b[1] + vz * b[2];
    qv[5] = vx; qv[6] = vy; qv[7] = vz; qv[8] = T(0);
  }
  const double dt = sc->dt;
  const double kappa = g.glm ? sc->kappa : 0.0;
  const double metric = 2.0 / g.dx;
  // FP32 form: rows other than the degree-0 ones accumulate and combine in
  // FP32 (GB300's FP64 rate is 1/64 of FP32); the degree-0 rows keep FP64
  const T tm = (T)metric, tdt = (T)dt, tca = (T)ca, tcb = (T)cb;
  for (int r = lane; r < g.nrows; r += 32) {
    const int m = mix ? mean_index(g, r) : -1;
    const bool lowp = sizeof(T) == 4 && m < 0;
    double acc = 0.0;  // double accumulation: exact conservation of the mean rows
    T acct = T(0);
    if (!is_ldf_row(g, r)) {
      const int v = legendre_var(g, r);
      const int l = (g.bz2d >= 0 && r >= g.bz2d) ? r - g.bz2d : r % g.n;
      T s = T(0);
      if (l != 0) {
        for (int a = 0; a < g.D; ++a) {
          const T* Gp = G + (a * g.V + v) * QVP;
          if constexpr (VEC) {
            s += dotp<T, pad4((DEG + 1) * (DEG + 1) * (DEG + 1))>(Gp, tb.dPv4 + ((size_t)a * g.n + l) * QVP);
          } else {
            const T* Dp = tb.dPv + ((size_t)a * g.n + l) * g.Qv;
            for (int q = 0; q < g.Qv; ++q) s += Gp[q] * Dp[q];
          }
        }
      }
      if (lowp) acct += s; else acc += (double)s;
      for (int f = 0; f < 2 * g.D; ++f) {
        T sf = T(0);
        if constexpr (VEC) {
          constexpr int QF4 = pad4((DEG + 1) * (DEG + 1));
          const T* Pp = tb.Pf4 + ((size_t)f * g.n + l) * QFP;
          sf = dotp<T, QF4>(FS + (f * g.V + v) * QFP, Pp);
          if (!g.glm) sf += qv[v] * dotp<T, QF4>(PJ + f * QFP, Pp);
        } else {
          const T* Pp = tb.Pf + ((size_t)f * g.n + l) * g.Qf;
          for (int p = 0; p < g.Qf; ++p) {
            T term = FS[fsi(f, p, v)];
            if (!g.glm) term += PJ[f * QFP + p] * qv[v];
            sf += term * Pp[p];
          }
        }
        if (lowp) acct -= sf; else acc -= (double)sf;
      }
    } else {
      const int j = r - g.ldf0;
      T s = T(0);
      for (int a = 0; a < g.D; ++a)
        for (int cc = 0; cc < g.DB; ++cc) {
          const T* Gp = G + (a * g.V + 5 + cc) * QVP;
          if constexpr (VEC) {
            s += dotp<T, pad4((DEG + 1) * (DEG + 1) * (DEG + 1))>(
                Gp, tb.dLv4 + (((size_t)a * g.ndiv + j) * g.DB + cc) * QVP);
          } else {
            const T* Dp = tb.dLv + (((size_t)a * g.ndiv + j) * g.DB + cc) * g.Qv;
            for (int q = 0; q < g.Qv; ++q) s += Gp[q] * Dp[q];
          }
        }
      if (lowp) acct += s; else acc += (double)s;
      for (int f = 0; f < 2 * g.D; ++f) {
        T sf = T(0);
        for (int cc = 0; cc < g.DB; ++cc) {
          if constexpr (VEC) {
            constexpr int QF4 = pad4((DEG + 1) * (DEG + 1));
            const T* Lp = tb.Lf4 + (((size_t)f * g.ndiv + j) * g.DB + cc) * QFP;
            sf += dotp<T, QF4>(FS + (f * g.V + 5 + cc) * QFP, Lp) + qv[5 + cc] * dotp<T, QF4>(PJ + f * QFP, Lp);
          } else {
            const T* Lp = tb.Lf + (((size_t)f * g.ndiv + j) * g.DB + cc) * g.Qf;
            for (int p = 0; p < g.Qf; ++p)
              sf += (FS[fsi(f, p, 5 + cc)] + PJ[f * QFP + p] * qv[5 + cc]) * Lp[p];
          }
        }
        if (lowp) acct -= sf; else acc -= (double)sf;
      }
    }
    if (lowp) {
      T rt = tm * tb.minv[r] * acct;
      if (g.glm && r >= 8 * g.n) rt -= (T)kappa * wc[r];
      if (!combine) out[r * S + c] = rt;
      else out[r * S + c] = tca * w0[r * S + c] + tcb * (wc[r] + tdt * rt);
      continue;
    }
    double rhs = metric * (double)tb.minv[r] * acc;
    if (g.glm && r >= 8 * g.n) rhs -= kappa * (double)wc[r];
    if (!combine) {
      out[r * S + c] = (T)rhs;
      if (m >= 0) outmean[m * S + c] = rhs;
    } else if (m >= 0) {
      // FP64 update of a degree-0 row; the float entry mirrors it
      const double o = ca * w0mean[m * S + c] + cb * (wmean[m * S + c] + dt * rhs);
      outmean[m * S + c] = o;
      out[r * S + c] = (T)o;
    } else {
      const double ws = (double)wc[r];
      const double wz = (double)w0[r * S + c];
      out[r * S + c] = (T)(ca * wz + cb * (ws + dt * rhs));
    }
  }
}

// ---------------------------------------------------------------- projection
template <typename T>
__global__ void k_project(Geom g, int Qp, const double* __restrict__ tab, const double* __restrict__ wq,
                          const double* __restrict__ nodal, const T* __restrict__ minv, T* __restrict__ w,
                          double* __restrict__ wmean) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * WARPS_PER_BLOCK + warp;
  if (c >= g.ncell) return;
  const int64_t S = g.stride;
  // tab[(r*Qp + q)*3 + k]: value of row r's k-th active component at point q;
  // the variable of component k is given by the row kind
  for (int r = lane; r < g.nrows; r += 32) {
    double acc = 0.0;
    if (!is_ldf_row(g, r)) {
      const int v = legendre_var(g, r);
      for (int q = 0; q < Qp; ++q) acc += wq[q] * nodal[((int64_t)v * Qp + q) * S + c] * tab[((size_t)r * Qp + q) * 3];
    } else {
      for (int q = 0; q < Qp; ++q)
        for (int k = 0; k < g.DB; ++k)
          acc += wq[q] * nodal[((int64_t)(5 + k) * Qp + q) * S + c] * tab[((size_t)r * Qp + q) * 3 + k];
    }
    acc *= (double)minv[r];
    w[r * S + c] = (T)acc;
  }
  if (wmean != nullptr) {
    __syncwarp();
    for (int m = lane; m < n_mean_rows(g); m += 32) {
      const int r = mean_row(g, m);
      double acc = 0.0;
      if (!is_ldf_row(g, r)) {
        const int v = legendre_var(g, r);
        for (int q = 0; q < Qp; ++q)
          acc += wq[q] * nodal[((int64_t)v * Qp + q) * S + c] * tab[((size_t)r * Qp + q) * 3];
      } else {
        for (int q = 0; q < Qp; ++q)
          for (int k = 0; k < g.DB; ++k)
            acc += wq[q] * nodal[((int64_t)(5 + k) * Qp + q) * S + c] * tab[((size_t)r * Qp + q) * 3 + k];
      }
      wmean[m * S + c] = acc * (double)minv[r];
    }
  }
}

// ---------------------------------------------------------------- Powell |div B| face jumps
template <typename T>
__global__ void k_divb_face(Geom g, Tables<T> tb, const T* __restrict__ w, T* __restrict__ jbuf) {
  const int64_t total = (int64_t)g.D * g.ncell * g.Qf;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= total) return;
  const int p = (int)(tid % g.Qf);
  const int64_t fc = tid / g.Qf;
  const int64_t c = fc % g.ncell;
  const int a = (int)(fc / g.ncell);
  const int64_t cl = neighbour(g, c, a, -1);
  const int64_t S = g.stride;
  const int fL = 2 * a + 1, fR = 2 * a;
  T rL = T(0), rR = T(0), bL = T(0), bR = T(0);
  for (int l = 0; l < g.n; ++l) {
    rL += w[l * S + cl] * tb.Pf[((size_t)fL * g.n + l) * g.Qf + p];
    rR += w[l * S + c] * tb.Pf[((size_t)fR * g.n + l) * g.Qf + p];
  }
  for (int j = 0; j < g.ndiv; ++j) {
    bL += w[(g.ldf0 + j) * S + cl] * tb.Lf[(((size_t)fL * g.ndiv + j) * g.DB + a) * g.Qf + p];
    bR += w[(g.ldf0 + j) * S + c] * tb.Lf[(((size_t)fR * g.ndiv + j) * g.DB + a) * g.Qf + p];
  }
  const T bF = bn_face(rL, rR, bL, bR);
  const T wp = tb.wf[p];
  T* o = jbuf + tid * 2;
  o[0] = wp * (bF > bL ? bF - bL : bL - bF);  // contribution to the L cell
  o[1] = wp * (bF > bR ? bF - bR : bR - bF);  // contribution to the R cell
}

// ---------------------------------------------------------------- dt
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double warp_min(double x) {
  for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// ---------------------------------------------------------------- div B diagnostics (App. C)
// normal component a of B on face f of cell c at face point p (GLM: Legendre
// rows of B_a; Powell: the LDF rows)
template <typename T>
__device__ double bn_trace(const Geom& g, const Tables<T>& tb, const T* w, int64_t c, int f, int a, int p) {
  const int64_t S = g.stride;
  double b = 0.0;
  if (g.glm) {
    for (int l = 0; l < g.n; ++l)
      b += (double)w[(int64_t)((5 + a) * g.n + l) * S + c] * (double)tb.Pf[((size_t)f * g.n + l) * g.Qf + p];
  } else {
    for (int j = 0; j < g.ndiv; ++j)
      b += (double)w[(int64_t)(g.ldf0 + j) * S + c] *
           (double)tb.Lf[(((size_t)f * g.ndiv + j) * g.DB + a) * g.Qf + p];
  }
  return b;
}

// per face point of every face (axis a, right cell c, left cell its -a
// neighbour): w_p |B^n_F - B^n_L|, w_p |B^n_F - B^n_R| and w_p B^n_F
template <typename T>
__global__ void k_divb_diag_face(Geom g, Tables<T> tb, const T* __restrict__ w, double* __restrict__ fb) {
  const int64_t total = (int64_t)g.D * g.ncell * g.Qf;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= total) return;
  const int p = (int)(tid % g.Qf);
  const int64_t fc = tid / g.Qf;
  const int64_t c = fc % g.ncell;
  const int a = (int)(fc / g.ncell);
  const int64_t cl = neighbour(g, c, a, -1);
  const int64_t S = g.stride;
  double rL = 0.0, rR = 0.0;
  for (int l = 0; l < g.n; ++l) {
    rL += (double)w[l * S + cl] * (double)tb.Pf[((size_t)(2 * a + 1) * g.n + l) * g.Qf + p];
    rR += (double)w[l * S + c] * (double)tb.Pf[((size_t)(2 * a) * g.n + l) * g.Qf + p];
  }
  const double bL = bn_trace(g, tb, w, cl, 2 * a + 1, a, p);
  const double bR = bn_trace(g, tb, w, c, 2 * a, a, p);
  const double bF = bn_face(rL, rR, bL, bR);
  const double wp = (double)tb.wf[p];
  double* o = fb + tid * 3;
  o[0] = wp * fabs(bF - bL);
  o[1] = wp * fabs(bF - bR);
  o[2] = wp * bF;
}

// per cell: |div B|_K (eq. divb-cell), signed (eq. divb-gauss, 1/V_K) and
// normalised (eq. divb-normalized); block sums / maxima into res:
// res[0] += sum |div B|_K / ncell (eq. divb-total: equal volumes),
// res[1] += sum normalised / ncell, res[2] = max normalised, res[3] = max |signed|
template <typename T>
__global__ void k_divb_diag_cell(Geom g, Tables<T> tb, const T* __restrict__ w, const double* __restrict__ wmean,
                                 const double* __restrict__ fb, double* res, double* per_cell) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double cell = 0.0, nrm = 0.0, sga = 0.0;
  if (c < g.ncell) {
    const int64_t S = g.stride;
    // (1/V_K) int_K |div B| = 2^-D sum_q w_q |div B(q)|, div B = (2/dx) sum_a dB_a/dxi_a
    double vol = 0.0;
    for (int q = 0; q < g.Qv; ++q) {
      double dv = 0.0;
      for (int a = 0; a < g.D; ++a) {
        if (g.glm) {
          for (int l = 0; l < g.n; ++l)
            dv += (double)w[(int64_t)((5 + a) * g.n + l) * S + c] * (double)tb.dPv[((size_t)a * g.n + l) * g.Qv + q];
        } else {
          for (int j = 0; j < g.ndiv; ++j)
            dv += (double)w[(int64_t)(g.ldf0 + j) * S + c] *
                  (double)tb.dLv[(((size_t)a * g.ndiv + j) * g.DB + a) * g.Qv + q];
        }
      }
      vol += (double)tb.wv[q] * fabs(dv);
    }
    vol *= (2.0 / g.dx) / (double)(1 << g.D);
    double face = 0.0, sg = 0.0;
    for (int a = 0; a < g.D; ++a) {
      const int64_t cp = neighbour(g, c, a, +1);
      for (int p = 0; p < g.Qf; ++p) {
        const double* om = fb + (((int64_t)a * g.ncell + c) * g.Qf + p) * 3;   // own -a face: R side
        const double* op = fb + (((int64_t)a * g.ncell + cp) * g.Qf + p) * 3;  // own +a face: L side
        face += om[1] + op[0];
        sg += op[2] - om[2];
      }
    }
    double meas = 1.0;
    for (int a = 0; a < g.D - 1; ++a) meas *= 0.5 * g.dx;
    for (int a = 0; a < g.D; ++a) meas /= g.dx;
    face *= meas;
    sg *= meas;
    cell = vol + face;
    // |mean B|
    double bm[3] = {0.0, 0.0, 0.0};
    if (g.glm) {
      for (int a = 0; a < 3; ++a) bm[a] = wmean ? wmean[(int64_t)(5 + a) * S + c] : (double)w[(int64_t)(5 + a) * g.n * S + c];
    } else {
      for (int j = 0; j < g.D; ++j) {
        const double wj = wmean ? wmean[(int64_t)(5 + j) * S + c] : (double)w[(int64_t)(g.ldf0 + j) * S + c];
        for (int cc = 0; cc < g.DB; ++cc) bm[cc] += wj * (double)tb.L0[j * g.DB + cc];
      }
      if (g.bz2d >= 0) bm[2] = wmean ? wmean[(int64_t)7 * S + c] : (double)w[(int64_t)g.bz2d * S + c];
    }
    const double bmag = sqrt(bm[0] * bm[0] + bm[1] * bm[1] + bm[2] * bm[2]);
    nrm = bmag > 0.0 ? cell * g.dx / bmag : 0.0;
    sga = fabs(sg);
    if (per_cell) {
      per_cell[c] = cell;
      per_cell[S + c] = sg;
      per_cell[2 * S + c] = nrm;
    }
  }
  __shared__ double r0[256], r1[256], r2[256], r3[256];
  r0[threadIdx.x] = cell;
  r1[threadIdx.x] = nrm;
  r2[threadIdx.x] = nrm;
  r3[threadIdx.x] = sga;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      r0[threadIdx.x] += r0[threadIdx.x + o];
      r1[threadIdx.x] += r1[threadIdx.x + o];
      r2[threadIdx.x] = fmax(r2[threadIdx.x], r2[threadIdx.x + o]);
      r3[threadIdx.x] = fmax(r3[threadIdx.x], r3[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(res, r0[0] / (double)g.ncell);
    atomicAdd(res + 1, r1[0] / (double)g.ncell);
    // non-negative doubles order as their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(res + 2), dbits(r2[0]));
    atomicMax(reinterpret_cast<unsigned long long*>(res + 3), dbits(r3[0]));
  }
}

// eq. cfl (and eq. powell_dt for Powell) of cell c in FP64 from its cell means
// (wmean when given, else the degree-0 rows of w); *smax: the cell's mean
// signal speed sum_a (|v_a| + c) / D. Returns DBL_MAX where the bound is not a
// positive finite number (and sets status bit 1).
template <typename T>
__device__ double dt_cell64(const Geom& g, const Tables<T>& tb, const T* __restrict__ w,
                            const double* __restrict__ wmean, const T* __restrict__ jbuf, const dg_mhd_params& p,
                            DevScalars* __restrict__ sc, int64_t c, double* smax) {
  const int64_t S = g.stride;
  auto mean = [&](int m) {
    return wmean ? wmean[m * S + c] : (double)w[(int64_t)mean_row(g, m) * S + c];
  };
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
  const double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const double pr = (g.gamma - 1.0) * (E - 0.5 * rho * (vx * vx + vy * vy + vz * vz) - 0.5 * b2);
  const double cs = sqrt(g.gamma * pr / rho + b2 / rho);
  const double av[3] = {fabs(vx), fabs(vy), fabs(vz)};
  double s = 0.0;
  for (int a = 0; a < g.D; ++a) s += (av[a] + cs) / g.dx;
  double dtc = p.cfl / (2.0 * g.d + 1.0) / s;
  *smax = s * g.dx / g.D;
  if (!g.glm) {
    // (1/V_K) oint |B^n_F - B^n_K| dS: sum this cell's 2D faces in fixed order
    double acc = 0.0;
    const int nq = g.jq ? g.jq : g.Qf;
    for (int a = 0; a < g.D; ++a) {
      const int64_t cp = neighbour(g, c, a, +1);
      for (int q = 0; q < nq; ++q) {
        acc += (double)jbuf[(((int64_t)a * g.ncell + c) * nq + q) * 2 + 1];   // minus face: R side
        acc += (double)jbuf[(((int64_t)a * g.ncell + cp) * nq + q) * 2 + 0];  // plus face: L side
      }
    }
    double meas = 1.0;
    for (int a = 0; a < g.D - 1; ++a) meas *= 0.5 * g.dx;
    double divb = acc * meas;
    for (int a = 0; a < g.D; ++a) divb /= g.dx;
    const double rate = divb * fabs(vx * b[0] + vy * b[1] + vz * b[2]) / E;
    if (rate > 0.0) dtc = fmin(dtc, p.eta_powell / rate);
  }
  if (!(dtc > 0.0) || !isfinite(dtc)) {
    atomicOr(&sc->status, 1);
    dtc = DBL_MAX;
  }
  return dtc;
}

template <typename T>
__global__ void k_dt(Geom g, Tables<T> tb, const T* __restrict__ w, const double* __restrict__ wmean,
                     const T* __restrict__ jbuf, dg_mhd_params p, DevScalars* __restrict__ sc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double dtc = DBL_MAX, smax = 0.0;
  if (c < g.ncell && (!g.owned || g.owned[c])) dtc = dt_cell64(g, tb, w, wmean, jbuf, p, sc, c, &smax);
  // block reduction then one atomic per block
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
    atomicMin(&sc->dt_bits, dbits(red[0]));
    atomicMax(&sc->smax_bits, dbits(reds[0]));
  }
}

// FP32 screen of the FP32 form's timestep (uniform meshes): the same CFL and
// Powell bounds from the float mirror of the cell means, in single precision,
// with the FP64 means used where the FP32 pressure would lose its digits to
// the cancellation E - kinetic - magnetic. *smax as in dt_cell64. Returns
// FLT_MAX where the bound is not a positive finite number (status bit 1).
// Uniform FP32 constants of the screen, computed once on the host (an FP64
// division per thread costs dozens of FP64 instructions on this GPU).
struct Dt32Const {
  float idx;      // 1 / dx
  float cflfac;   // C / (2 d + 1)
  float gam;      // gamma
  float eta;      // eta of eq. powell_dt
  float invD;     // 1 / D
};

__device__ float dt_cell32(const Geom& g, const Tables<float>& tb, const float* __restrict__ w,
                           const double* __restrict__ wmean, const float* __restrict__ jbuf, const Dt32Const& k,
                           DevScalars* __restrict__ sc, int64_t c, float* smax) {
  const int64_t S = g.stride;
  auto mean = [&](int m) { return w[(int64_t)mean_row(g, m) * S + c]; };
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
  const float gam = k.gam;
  const float b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const float kin = 0.5f * rho * (vx * vx + vy * vy + vz * vz);
  float pr = (gam - 1.f) * (E - kin - 0.5f * b2);
  if (!(pr > 1e-3f * E)) {
    // cancellation (or a non-positive mean pressure): FP64 from the means
    auto md = [&](int m) { return wmean[m * S + c]; };
    const double rd = md(0);
    const double mx = md(1), my = md(2), mz = md(3);
    double bd[3];
    if (g.glm) {
      bd[0] = md(5); bd[1] = md(6); bd[2] = md(7);
    } else {
      bd[0] = bd[1] = bd[2] = 0.0;
      for (int j = 0; j < g.DB; ++j)
        for (int cc = 0; cc < g.DB; ++cc) bd[cc] += md(5 + j) * (double)tb.L0[j * g.DB + cc];
      if (g.bz2d >= 0) bd[2] = md(7);
    }
    pr = (float)((g.gamma - 1.0) * (md(4) - 0.5 * (mx * mx + my * my + mz * mz) / rd -
                                    0.5 * (bd[0] * bd[0] + bd[1] * bd[1] + bd[2] * bd[2])));
  }
  const float cs = sqrtf((gam * pr + b2) * ir);
  const float av[3] = {fabsf(vx), fabsf(vy), fabsf(vz)};
  float sum = 0.f;
  for (int a = 0; a < g.D; ++a) sum += av[a] + cs;
  const float idx = k.idx;
  const float s = sum * idx;
  float dtc = k.cflfac / s;
  *smax = sum * k.invD;
  if (!g.glm) {
    // (1/V_K) oint |B^n_F - B^n_K| dS: this cell's 2D faces in fixed order
    float acc = 0.f;
    const int nq = g.jq ? g.jq : g.Qf;
    for (int a = 0; a < g.D; ++a) {
      const int64_t cp = neighbour(g, c, a, +1);
      for (int q = 0; q < nq; ++q) {
        acc += jbuf[(((int64_t)a * g.ncell + c) * nq + q) * 2 + 1];
        acc += jbuf[(((int64_t)a * g.ncell + cp) * nq + q) * 2 + 0];
      }
    }
    // face measure (dx/2)^(D-1) over the volume dx^D: 2^(1-D) / dx
    const float divb = acc * (g.D == 3 ? 0.25f : 0.5f) * idx;
    const float rate = divb * fabsf(vx * b[0] + vy * b[1] + vz * b[2]) / E;
    if (rate > 0.f) dtc = fminf(dtc, k.eta / rate);
  }
  if (!(dtc > 0.f) || !isfinite(dtc)) {
    atomicOr(&sc->status, 1);
    dtc = FLT_MAX;
  }
  return dtc;
}

// block minimum of a and maximum of b (256 threads), written by thread 0
__device__ __forceinline__ void block_minmax256(unsigned& a, unsigned& b) {
  __shared__ unsigned ra[8], rb[8];
  a = __reduce_min_sync(0xffffffffu, a);
  b = __reduce_max_sync(0xffffffffu, b);
  const int wi = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    ra[wi] = a;
    rb[wi] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    a = threadIdx.x < 8 ? ra[threadIdx.x] : 0xffffffffu;
    b = threadIdx.x < 8 ? rb[threadIdx.x] : 0u;
    a = __reduce_min_sync(0xffffffffu, a);
    b = __reduce_max_sync(0xffffffffu, b);
  }
}

// Pass 1 of the FP32 form's timestep: the FP32 bound of every cell, its
// minimum m32 (warp minimum, one atomic per warp) and the signal-speed maximum.
__global__ void k_dt32(Geom g, Tables<float> tb, const float* __restrict__ w, const double* __restrict__ wmean,
                       const float* __restrict__ jbuf, Dt32Const k, DevScalars* __restrict__ sc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float dtc = FLT_MAX, smax = 0.f;
  if (c < g.ncell && (!g.owned || g.owned[c])) dtc = dt_cell32(g, tb, w, wmean, jbuf, k, sc, c, &smax);
  // positive floats order as their bit patterns: block reduction, one atomic per block
  unsigned mn = __float_as_uint(dtc), mxs = __float_as_uint(smax);
  block_minmax256(mn, mxs);
  if (threadIdx.x == 0) {
    const float dm = __uint_as_float(mn);
    if (dm < FLT_MAX) atomicMin(&sc->dt_bits, dbits((double)dm));
    atomicMax(&sc->smax_bits, dbits((double)__uint_as_float(mxs)));
  }
}

// Pass 2: the timestep is the FP64 minimum of the FP64 bounds (the same
// arithmetic as the plain FP64 path, from the FP64 means). Only the cells
// whose FP32 bound lies within kDtScreen (relative) of the FP32 minimum can
// hold it: the FP32 bound's error is below 1e-4 relative (FP32 rounding of a
// few dozen operations, the FP32 pressure used only while it keeps 1e-3 of E),
// so the cell with the smallest FP64 bound is always among them. They are
// recomputed in FP64 and min-reduced into dt64_bits.
constexpr float kDtScreen = 1e-3f;
__global__ void k_dt32_refine(Geom g, Tables<float> tb, const float* __restrict__ w,
                              const double* __restrict__ wmean, const float* __restrict__ jbuf, Dt32Const k,
                              dg_mhd_params p, DevScalars* __restrict__ sc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double dtc = DBL_MAX;
  if (c < g.ncell && (!g.owned || g.owned[c])) {
    // m32 is a float value (the FP32 pass's minimum); the screen compares in FP32
    const double m32 = __longlong_as_double((long long)sc->dt_bits);
    const float thr = m32 < DBL_MAX ? (float)m32 * (1.f + kDtScreen) : -1.f;
    float sm32;
    const float d32 = dt_cell32(g, tb, w, wmean, jbuf, k, sc, c, &sm32);
    if (d32 <= thr) {
      double sm64;
      dtc = dt_cell64<float>(g, tb, w, wmean, jbuf, p, sc, c, &sm64);
    }
  }
  const double m = warp_min(dtc);
  if ((threadIdx.x & 31) == 0 && m < DBL_MAX) atomicMin(&sc->dt64_bits, dbits(m));
}

__global__ void k_dt_init(DevScalars* sc) {
  sc->dt_bits = dbits(DBL_MAX);
  sc->dt64_bits = dbits(DBL_MAX);
  sc->smax_bits = 0ull;
}

__global__ void k_dt_finalize(Geom g, dg_mhd_params p, DevScalars* sc, const double* dt_in, double* dt_out) {
  // the FP32 form's refined FP64 minimum where that pass ran, else the FP64 pass's minimum
  const double dt64 = __longlong_as_double((long long)sc->dt64_bits);
  double dt = dt_in ? *dt_in : (dt64 < DBL_MAX ? dt64 : __longlong_as_double((long long)sc->dt_bits));
  if (!(dt > 0.0) || !isfinite(dt) || dt >= DBL_MAX) {
    atomicOr(&sc->status, 1);
  }
  sc->dt = dt;
  sc->dt_step = dt;
  sc->dt32 = (float)dt;
  if (dt_out) *dt_out = dt;
  if (g.glm) {
    double ch = p.c_h_fixed > 0.0 ? p.c_h_fixed : p.cfl_glm / (2.0 * g.d + 1.0) * g.dx / (g.D * dt);
    sc->ch = ch;
    sc->ch32 = (float)ch;
    const double tau = fmax(p.c_r / ch, 3.0 * dt);
    sc->kappa = 1.0 / tau;
    sc->kappa32 = (float)sc->kappa;
    if (p.c_h_fixed > 0.0 && !dt_in) {
      const double smax = __longlong_as_double((long long)sc->smax_bits);
      if (ch < smax) atomicOr(&sc->status, 4);
    }
  }
}

// stages of a fraction f of the step (the fourth-order scheme's dt/6)
__global__ void k_dt_scale(DevScalars* sc, double f) {
  sc->dt = sc->dt_step * f;
  sc->dt32 = (float)sc->dt;
}

// out = a x + b y on every state row (blockIdx.y = row); FP32 form: the mean
// rows in FP64 from xm, ym (om written, its float mirror in out)
template <typename T>
__global__ void k_axpby(Geom g, double a, const T* __restrict__ x, double b, const T* __restrict__ y, T* out,
                        const double* __restrict__ xm, const double* __restrict__ ym, double* om) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int r = blockIdx.y;
  const int64_t i = (int64_t)r * g.stride + c;
  if (om) {
    const int nm = g.glm ? 9 : 8;
    for (int m = 0; m < nm; ++m)
      if (mean_row(g, m) == r) {
        const int64_t j = (int64_t)m * g.stride + c;
        const double o = a * xm[j] + b * ym[j];
        om[j] = o;
        out[i] = (T)o;
        return;
      }
  }
  out[i] = (T)a * x[i] + (T)b * y[i];
}

__global__ void k_set_glm(DevScalars* sc, double ch, double kappa) {
  sc->ch = ch;
  sc->kappa = kappa;
  sc->ch32 = (float)ch;
  sc->kappa32 = (float)kappa;
}

}  // namespace

// ---------------------------------------------------------------- launchers
static inline unsigned nblocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T>
void launch_face(const Geom& g, const Tables<T>& tb, const T* w, T* fbuf, const DevScalars* sc, double eps,
                 cudaStream_t st, T* qbuf) {
  const int64_t total = (int64_t)g.D * g.ncell * g.Qf;
  // compile-time sizes for the 3D degree-1 and degree-2 schemes
  auto run = [&](auto k) { k<<<nblocks(total, 128), 128, 0, st>>>(g, tb, w, fbuf, sc, (T)eps, qbuf); };
  if (!pinned_sizes_ok(g)) run(k_face<T, -1, 0>);
  else if (g.d == 2) g.glm ? run(k_face<T, 2, 1>) : run(k_face<T, 2, 0>);
  else g.glm ? run(k_face<T, 1, 1>) : run(k_face<T, 1, 0>);
}

template <typename T>
static size_t cell_smem(const Geom& g, bool vec = false) {
  return (size_t)cell_warp_elems(g, vec) * WARPS_PER_BLOCK * sizeof(T);
}

template <typename T>
void launch_cell(const Geom& g, const Tables<T>& tb, const T* w, const T* fbuf, T* out, const T* w0,
                 double ca, double cb, int combine, const DevScalars* sc, const double* wmean,
                 const double* w0mean, double* outmean, cudaStream_t st, const T* qbuf) {
  // FP32 only: FP64 is bound by its multiply-add rate, which the padding would raise
  const bool vec = sizeof(T) == 4 && pinned_sizes_ok(g) && tb.dPv4 && tb.dLv4 && tb.Pf4 && tb.Lf4;
  const size_t sm = cell_smem<T>(g, vec);
  auto run = [&](auto k) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    k<<<nblocks(g.ncell, WARPS_PER_BLOCK), 32 * WARPS_PER_BLOCK, sm, st>>>(g, tb, w, fbuf, out, w0, ca, cb, combine,
                                                                        sc, wmean, w0mean, outmean, qbuf);
  };
  // compile-time sizes for the 3D degree-1 and degree-2 schemes
  if (!pinned_sizes_ok(g)) run(k_cell<T, -1, 0, false>);
  else if (!vec) g.d == 2 ? (g.glm ? run(k_cell<T, 2, 1, false>) : run(k_cell<T, 2, 0, false>))
                          : (g.glm ? run(k_cell<T, 1, 1, false>) : run(k_cell<T, 1, 0, false>));
  else if (g.d == 2) g.glm ? run(k_cell<T, 2, 1, true>) : run(k_cell<T, 2, 0, true>);
  else g.glm ? run(k_cell<T, 1, 1, true>) : run(k_cell<T, 1, 0, true>);
}

template <typename T>
void launch_project(const Geom& g, int npts, const double* tab, const double* wq, const double* nodal,
                    const T* minv, T* w, double* wmean, cudaStream_t st) {
  int Qp = 1;
  for (int a = 0; a < g.D; ++a) Qp *= npts;
  k_project<T><<<nblocks(g.ncell, WARPS_PER_BLOCK), 32 * WARPS_PER_BLOCK, 0, st>>>(g, Qp, tab, wq, nodal, minv,
                                                                                   w, wmean);
}

template <typename T>
void launch_divb_face(const Geom& g, const Tables<T>& tb, const T* w, T* jbuf, cudaStream_t st) {
  const int64_t total = (int64_t)g.D * g.ncell * g.Qf;
  k_divb_face<T><<<nblocks(total, 128), 128, 0, st>>>(g, tb, w, jbuf);
}

template <typename T>
void launch_dt(const Geom& g, const Tables<T>& tb, const T* w, const double* wmean, const T* jbuf,
               const dg_mhd_params& p, DevScalars* sc, double* dt_out, cudaStream_t st) {
  k_dt_init<<<1, 1, 0, st>>>(sc);
  if constexpr (sizeof(T) == 4) {
    if (wmean) {
      Dt32Const k;
      k.idx = (float)(1.0 / g.dx);
      k.cflfac = (float)(p.cfl / (2.0 * g.d + 1.0));
      k.gam = (float)g.gamma;
      k.eta = (float)p.eta_powell;
      k.invD = 1.f / (float)g.D;
      k_dt32<<<nblocks(g.ncell, 256), 256, 0, st>>>(g, tb, w, wmean, jbuf, k, sc);
      k_dt32_refine<<<nblocks(g.ncell, 256), 256, 0, st>>>(g, tb, w, wmean, jbuf, k, p, sc);
      k_dt_finalize<<<1, 1, 0, st>>>(g, p, sc, nullptr, dt_out);
      return;
    }
  }
  k_dt<T><<<nblocks(g.ncell, 256), 256, 0, st>>>(g, tb, w, wmean, jbuf, p, sc);
  k_dt_finalize<<<1, 1, 0, st>>>(g, p, sc, nullptr, dt_out);
}

void launch_dt_from_value(const Geom& g, const dg_mhd_params& p, const double* dt_in, DevScalars* sc,
                          cudaStream_t st) {
  k_dt_finalize<<<1, 1, 0, st>>>(g, p, sc, dt_in, nullptr);
}

void launch_dt_init(DevScalars* sc, cudaStream_t st) { k_dt_init<<<1, 1, 0, st>>>(sc); }

void launch_dt_scale(DevScalars* sc, double f, cudaStream_t st) { k_dt_scale<<<1, 1, 0, st>>>(sc, f); }

template <typename T>
void launch_divb_diag(const Geom& g, const Tables<T>& tb, const T* w, const double* wmean, double* scratch,
                      double* res, double* per_cell, cudaStream_t st) {
  cudaMemsetAsync(res, 0, 4 * sizeof(double), st);
  const int64_t total = (int64_t)g.D * g.ncell * g.Qf;
  k_divb_diag_face<T><<<nblocks(total, 128), 128, 0, st>>>(g, tb, w, scratch);
  k_divb_diag_cell<T><<<nblocks(g.ncell, 256), 256, 0, st>>>(g, tb, w, wmean, scratch, res, per_cell);
}
template void launch_divb_diag<float>(const Geom&, const Tables<float>&, const float*, const double*, double*,
                                      double*, double*, cudaStream_t);
template void launch_divb_diag<double>(const Geom&, const Tables<double>&, const double*, const double*, double*,
                                       double*, double*, cudaStream_t);

template <typename T>
void launch_axpby(const Geom& g, double a, const T* x, double b, const T* y, T* out, const double* xm,
                  const double* ym, double* om, cudaStream_t st) {
  const dim3 grid((unsigned)((g.ncell + 255) / 256), (unsigned)g.nrows);
  k_axpby<T><<<grid, 256, 0, st>>>(g, a, x, b, y, out, xm, ym, om);
}
template void launch_axpby<float>(const Geom&, double, const float*, double, const float*, float*, const double*,
                                  const double*, double*, cudaStream_t);
template void launch_axpby<double>(const Geom&, double, const double*, double, const double*, double*,
                                   const double*, const double*, double*, cudaStream_t);

void launch_dt_finalize(const Geom& g, const dg_mhd_params& p, DevScalars* sc, double* dt_out, cudaStream_t st) {
  k_dt_finalize<<<1, 1, 0, st>>>(g, p, sc, nullptr, dt_out);
}

void launch_set_glm(DevScalars* sc, double ch, double kappa, cudaStream_t st) {
  k_set_glm<<<1, 1, 0, st>>>(sc, ch, kappa);
}

template <typename T>
__global__ void k_mirror_means(Geom g, const double* __restrict__ wmean, T* __restrict__ w) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int nm = g.glm ? 9 : 8;
  for (int m = 0; m < nm; ++m) w[(int64_t)mean_row(g, m) * g.stride + c] = (T)wmean[(int64_t)m * g.stride + c];
}

template <typename T>
void launch_mirror_means(const Geom& g, const double* wmean, T* w, cudaStream_t st) {
  k_mirror_means<T><<<nblocks(g.ncell, 256), 256, 0, st>>>(g, wmean, w);
}

#define INST(T)                                                                                              \
  template void launch_face<T>(const Geom&, const Tables<T>&, const T*, T*, const DevScalars*, double,      \
                               cudaStream_t, T*);                                                            \
  template void launch_cell<T>(const Geom&, const Tables<T>&, const T*, const T*, T*, const T*, double,     \
                               double, int, const DevScalars*, const double*, const double*, double*,      \
                               cudaStream_t, const T*);                                                      \
  template void launch_project<T>(const Geom&, int, const double*, const double*, const double*, const T*, \
                                  T*, double*, cudaStream_t);                                               \
  template void launch_divb_face<T>(const Geom&, const Tables<T>&, const T*, T*, cudaStream_t);            \
  template void launch_dt<T>(const Geom&, const Tables<T>&, const T*, const double*, const T*,             \
                             const dg_mhd_params&, DevScalars*, double*, cudaStream_t);                    \
  template void launch_mirror_means<T>(const Geom&, const double*, T*, cudaStream_t);
INST(double)
INST(float)

}  // namespace dgmhd
