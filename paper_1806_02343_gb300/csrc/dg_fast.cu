// Specialised kernels of the DG operator for the GLM scheme on uniform 3D
// meshes (Sec. 3.5 eq. wdot; Sec. 4.1.2 HLLD; Sec. 4.1.5 GLM).
//
// Same arithmetic as the generic kernels, organised for the hardware:
// * basis tables are kernel parameters (constant bank), indexed with
//   compile-time offsets inside fully unrolled loops, so every contraction
//   step is one FMA with a constant operand; quadrature weights are folded in;
// * one thread owns one (cell, variable) pair: its n(d) modal coefficients and
//   n(d) accumulators stay in registers; each warp holds one variable for 32
//   consecutive cells, so state loads and stores are 128-byte coalesced and
//   every branch on the variable is warp-uniform;
// * the volume flux of variable v is written as f_a = alpha v_a + beta B_a
//   (+ gamma if a is the variable's own axis), with (alpha, beta, gamma) read
//   from per-point shared memory -- one code path for all nine variables;
// * k_face_glm evaluates the traces of the 32 cell pairs of a block with the
//   same per-(side, variable) mapping, then one thread per face point runs
//   HLLD and stores F* in a [axis][point][var][cell] buffer (cell fastest) that
//   k_cell_glm reads coalesced.
#include <cuda_runtime.h>

#include "dg_fast.cuh"
#include "dg_phys.cuh"

namespace dgmhd {

namespace {

constexpr int TC = 32;        // cells (or faces) per block

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
constexpr int NT = 9 * TC;    // threads per block: one per (variable, cell)

// Cell coordinates, computed once per thread in 32-bit arithmetic (cell
// counts stay below 2^31), and periodic neighbours by add-and-wrap.
struct Coord {
  int ix, iy, iz;
};

__device__ __forceinline__ Coord coord_of(const FastGeom& g, int64_t c) {
  const unsigned cc = (unsigned)c, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
  const unsigned r = cc / nx;
  return Coord{(int)(cc - r * nx), (int)(r % ny), (int)(r / ny)};
}

__device__ __forceinline__ int64_t nbr(const FastGeom& g, Coord k, int a, int dir) {
  if (a == 0) {
    k.ix += dir;
    k.ix = k.ix < 0 ? k.ix + g.nx : (k.ix >= g.nx ? k.ix - g.nx : k.ix);
  } else if (a == 1) {
    k.iy += dir;
    k.iy = k.iy < 0 ? k.iy + g.ny : (k.iy >= g.ny ? k.iy - g.ny : k.iy);
  } else {
    k.iz += dir;
    k.iz = k.iz < 0 ? k.iz + g.nz : (k.iz >= g.nz ? k.iz - g.nz : k.iz);
  }
  return ((int64_t)k.iz * g.ny + k.iy) * g.nx + k.ix;
}

// ------------------------------------------------------------------ faces
template <typename T, int DEG, int A>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && DEG <= 2) ? 4 : 3) k_face_glm(const FaceTabs<T, DEG> tb, const FastGeom g,
                                                 const T* __restrict__ w, T* __restrict__ F,
                                                 const DevScalars* __restrict__ sc, T eps) {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF, NR = 9 * N;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* WL = reinterpret_cast<T*>(smraw);       // [NR][TC]
  T* WR = WL + NR * TC;                      // [NR][TC]
  T* TR = WR + NR * TC;                      // [2][QF][9][TC]
  const int t = threadIdx.x;
  const int f = t & (TC - 1);
  const int v = t >> 5;  // warp-uniform
  const int64_t c0 = (int64_t)blockIdx.x * TC;
  const int64_t c = c0 + f;
  const bool live = c < g.ncell;
  const int64_t S = g.stride;
  const int64_t cl = live ? nbr(g, coord_of(g, c), A, -1) : 0;
  // stage both cells' coefficients (coalesced along cells); all loads of a
  // thread are issued before the first shared-memory store
  {
    constexpr int PER = (NR + 8) / 9;
    T a[PER], b[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int r = v + 9 * i;
      a[i] = (live && r < NR) ? w[r * S + c] : T(1);
      b[i] = (live && r < NR) ? w[r * S + cl] : T(1);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int r = v + 9 * i;
      if (r < NR) {
        WR[r * TC + f] = a[i];
        WL[r * TC + f] = b[i];
      }
    }
  }
  __syncthreads();
  // traces: thread (v, f) evaluates variable v of both sides at the QF points
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T* Ws = s ? WR : WL;
    T wl[N];
#pragma unroll
    for (int l = 0; l < N; ++l) wl[l] = Ws[(v * N + l) * TC + f];
#pragma unroll
    for (int p = 0; p < QF; ++p) {
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) acc += wl[l] * (s ? tb.PR[l][p] : tb.PL[l][p]);
      TR[((s * QF + p) * 9 + v) * TC + f] = acc;
    }
  }
  __syncthreads();
  // HLLD per face point
  const T ch = (T)sc->ch;
  const T gamma = (T)g.gamma;
  for (int p = v; p < QF; p += 9) {
    T uL[9], uR[9], Fo[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      uL[k] = TR[((0 * QF + p) * 9 + k) * TC + f];
      uR[k] = TR[((1 * QF + p) * 9 + k) * TC + f];
    }
    face_flux(uL, uR, A, gamma, true, ch, eps, Fo);
    if (live) {
#pragma unroll
      for (int k = 0; k < 9; ++k) F[((int64_t)(A * QF + p) * 9 + k) * S + c] = Fo[k];
    }
  }
}

// ------------------------------------------------------------------ cells
// primitive slots per volume point
enum { SL_RHO = 0, SL_B = 5, SL_PSI = 8, SL_V = 9, SL_PT = 12, SL_VB = 13, SL_EPT = 14, SL_ZERO = 15, NSL = 16 };

template <typename T, int DEG>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && DEG <= 2) ? 4 : 3) k_cell_glm(const CellTabs<T, DEG> tb, const FastGeom g,
                                                 const T* __restrict__ w, const T* __restrict__ F, T* out,
                                                 const T* w0, double ca, double cb, int combine,
                                                 const DevScalars* __restrict__ sc,
                                                 const double* __restrict__ wmean, const double* w0mean,
                                                 double* outmean) {
  // out / outmean may alias w0 / w0mean: each element is read, then written, by one thread.
  constexpr int N = FastDims<DEG>::N, QV = FastDims<DEG>::QV, QF = FastDims<DEG>::QF;
  constexpr int QC = FastDims<DEG>::QC;  // volume points per pass
  extern __shared__ __align__(16) unsigned char smraw[];
  T* PR = reinterpret_cast<T*>(smraw);  // [QC][NSL][TC]
  const int t = threadIdx.x;
  const int f = t & (TC - 1);
  const int v = t >> 5;  // warp-uniform variable
  const int64_t c = (int64_t)blockIdx.x * TC + f;
  const bool live = c < g.ncell;
  const int64_t S = g.stride;
  const bool mix = wmean != nullptr;
  const T gamma = (T)g.gamma;
  const T ch = (T)sc->ch;

  T wl[N];
#pragma unroll
  for (int l = 0; l < N; ++l) wl[l] = live ? w[(int64_t)(v * N + l) * S + c] : (v == 0 && l == 0 ? T(1) : T(0));
  // (FP32 form: wl[0] is the float mirror of the FP64 mean, an exact copy)
  if (!live && v == 4) wl[0] = T(1);  // keep dummy cells physical (rho = 1, E = 1)

  // flux of variable v: f_a = alpha v_a + beta B_a + (a == gax ? gamma_v : 0)
  int aidx, bidx, gidx, gax;
  T bs, bconst;
  if (v == 0) { aidx = SL_RHO; bidx = SL_ZERO; bs = T(0); bconst = T(0); gidx = SL_ZERO; gax = -1; }
  else if (v <= 3) { aidx = v; bidx = SL_B + v - 1; bs = T(-1); bconst = T(0); gidx = SL_PT; gax = v - 1; }
  else if (v == 4) { aidx = SL_EPT; bidx = SL_VB; bs = T(-1); bconst = T(0); gidx = SL_ZERO; gax = -1; }
  else if (v <= 7) { aidx = v; bidx = SL_V + v - 5; bs = T(-1); bconst = T(0); gidx = SL_PSI; gax = v - 5; }
  else { aidx = SL_ZERO; bidx = SL_ZERO; bs = T(0); bconst = ch * ch; gidx = SL_ZERO; gax = -1; }

  T racc[N];
#pragma unroll
  for (int l = 0; l < N; ++l) racc[l] = T(0);

#pragma unroll
  for (int q0 = 0; q0 < QV; q0 += QC) {
    // projection of variable v to the points of this pass
#pragma unroll
    for (int qq = 0; qq < QC; ++qq) {
      T u = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) u += wl[l] * tb.P[l][q0 + qq];
      PR[(qq * NSL + v) * TC + f] = u;
    }
    __syncthreads();
    // primitives per point
    for (int idx = t; idx < QC * TC; idx += NT) {
      const int qq = idx / TC, ff = idx % TC;
      T* pr = PR + qq * NSL * TC + ff;
      const T rho = pr[0], ir = T(1) / rho;
      const T vx = pr[1 * TC] * ir, vy = pr[2 * TC] * ir, vz = pr[3 * TC] * ir;
      const T bx = pr[5 * TC], by = pr[6 * TC], bz = pr[7 * TC];
      const T b2 = bx * bx + by * by + bz * bz;
      const T E = pr[4 * TC];
      const T p = (gamma - T(1)) * (E - T(0.5) * rho * (vx * vx + vy * vy + vz * vz) - T(0.5) * b2);
      const T pT = p + T(0.5) * b2;
      pr[SL_V * TC] = vx;
      pr[(SL_V + 1) * TC] = vy;
      pr[(SL_V + 2) * TC] = vz;
      pr[SL_PT * TC] = pT;
      pr[SL_VB * TC] = vx * bx + vy * by + vz * bz;
      pr[SL_EPT * TC] = E + pT;
      pr[SL_ZERO * TC] = T(0);
    }
    __syncthreads();
    // volume integral: racc_l += sum_a f_a(q) * w_q d_a P_l(q)
#pragma unroll
    for (int qq = 0; qq < QC; ++qq) {
      const T* pr = PR + qq * NSL * TC + f;
      const T al = pr[aidx * TC];
      const T be = bs * pr[bidx * TC] + bconst;
      const T ga = pr[gidx * TC];
      T fa[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) fa[a] = al * pr[(SL_V + a) * TC] + be * pr[(SL_B + a) * TC] + (a == gax ? ga : T(0));
#pragma unroll
      for (int l = 1; l < N; ++l)
        racc[l] += fa[0] * tb.dPw[0][l][q0 + qq] + fa[1] * tb.dPw[1][l][q0 + qq] + fa[2] * tb.dPw[2][l][q0 + qq];
    }
    __syncthreads();
  }
  // surface integral: -oint F* . n P_l over the six faces. The mean row sums
  // each face in the working precision in a fixed order -- the same products
  // and order in both cells of the face, so the two contributions cancel
  // exactly -- and the six face sums are then combined with more precision
  // than one rounding per face (conservation of the cell means).
  T fsum[6];
  const Coord kc = coord_of(g, live ? c : 0);
  if (live) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int64_t fc = s ? nbr(g, kc, a, +1) : c;
        T fs = T(0);
#pragma unroll
        for (int p = 0; p < QF; ++p) {
          const T Fr = F[((int64_t)(a * QF + p) * 9 + v) * S + fc];
          fs = fma_rn(Fr, tb.Pfw[2 * a][0][p], fs);  // P_0 = 1: same weight on both sides
          const T Fv = s ? -Fr : Fr;
#pragma unroll
          for (int l = 1; l < N; ++l) racc[l] += Fv * tb.Pfw[2 * a + s][l][p];
        }
        fsum[2 * a + s] = s ? -fs : fs;
      }
    }
  }
  if (!live) return;
  const double dt = sc->dt;
  const double kappa = sc->kappa;
  const double metric = g.metric;
  // mode 0 (cell mean)
  {
    const int64_t i = (int64_t)(v * N) * S + c;
    if (sizeof(T) == 4 && mix) {
      // FP32 form. The six face sums are added as an unevaluated float pair
      // (Knuth's TwoSum: s + e equals a + b exactly), so the cell's total is
      // accurate to about 2^-48 of the face sums; it enters the FP64 mean
      // through one conversion. GB300's FP64 rate is 1/64 of FP32: the FP64
      // work here is a handful of operations per (cell, variable).
      float hi = (float)fsum[0], lo = 0.f;
#pragma unroll
      for (int k = 1; k < 6; ++k) {
        const float b = (float)fsum[k];
        const float s2 = __fadd_rn(hi, b);
        const float bb = __fsub_rn(s2, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s2, bb)), __fsub_rn(b, bb));
        hi = s2;
        lo = __fadd_rn(lo, e);
      }
      const double tot = (double)hi + (double)lo;
      const double k1 = metric * (double)tb.minv[0];
      const double wz = wmean[(int64_t)v * S + c];
      if (!combine) {
        double rhs = k1 * tot;
        if (v == 8) rhs = fma(-kappa, wz, rhs);
        out[i] = (T)rhs;
        outmean[(int64_t)v * S + c] = rhs;
      } else {
        // o = ca w0 + cb (wz + dt rhs), rhs = k1 tot (- kappa wz for psi)
        const double kd = cb * dt;
        double base = cb * wz;
        if (ca != 0.0) base = fma(ca, w0mean[(int64_t)v * S + c], base);
        if (v == 8) base = fma(-kd * kappa, wz, base);
        const double o = fma(kd * k1, tot, base);
        outmean[(int64_t)v * S + c] = o;
        out[i] = (T)o;
      }
    } else {
      const double mean_acc = ((double)fsum[0] + (double)fsum[1]) + ((double)fsum[2] + (double)fsum[3]) +
                              ((double)fsum[4] + (double)fsum[5]);
      double rhs = metric * (double)tb.minv[0] * mean_acc;
      const double wz = (double)wl[0];
      if (v == 8) rhs -= kappa * wz;
      if (!combine) out[i] = (T)rhs;
      else out[i] = (T)(ca * (double)w0[i] + cb * (wz + dt * rhs));
    }
  }
  const T tm = (T)metric, tdt = (T)dt, tca = (T)ca, tcb = (T)cb, tk = (T)kappa;
#pragma unroll
  for (int l = 1; l < N; ++l) {
    T rhs = tm * tb.minv[l] * racc[l];
    if (v == 8) rhs -= tk * wl[l];
    const int64_t i = (int64_t)(v * N + l) * S + c;
    if (!combine) out[i] = rhs;
    else out[i] = tca * w0[i] + tcb * (wl[l] + tdt * rhs);
  }
}

template <typename T>
void set_smem_attr(const void* fn, size_t bytes) {
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

template <typename T, int DEG>
size_t fast_face_smem() {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF;
  return (size_t)(2 * 9 * N * TC + 2 * QF * 9 * TC) * sizeof(T);
}

template <typename T, int DEG>
size_t fast_cell_smem() {
  return (size_t)FastDims<DEG>::QC * NSL * TC * sizeof(T);
}

template <typename T, int DEG>
void launch_face_glm(const FastAll<T, DEG>& tabs, const FastGeom& g, const T* w, T* F, const DevScalars* sc,
                     double eps, cudaStream_t st) {
  const unsigned nb = (unsigned)((g.ncell + TC - 1) / TC);
  const size_t sm = fast_face_smem<T, DEG>();
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_face_glm<T, DEG, 0>, sm);
    set_smem_attr<T>((const void*)k_face_glm<T, DEG, 1>, sm);
    set_smem_attr<T>((const void*)k_face_glm<T, DEG, 2>, sm);
    attr = true;
  }
  k_face_glm<T, DEG, 0><<<nb, NT, sm, st>>>(tabs.face[0], g, w, F, sc, (T)eps);
  k_face_glm<T, DEG, 1><<<nb, NT, sm, st>>>(tabs.face[1], g, w, F, sc, (T)eps);
  k_face_glm<T, DEG, 2><<<nb, NT, sm, st>>>(tabs.face[2], g, w, F, sc, (T)eps);
}

template <typename T, int DEG>
void launch_cell_glm(const FastAll<T, DEG>& tabs, const FastGeom& g, const T* w, const T* F, T* out, const T* w0,
                     double ca, double cb, int combine, const DevScalars* sc, const double* wmean,
                     const double* w0mean, double* outmean, cudaStream_t st) {
  const unsigned nb = (unsigned)((g.ncell + TC - 1) / TC);
  const size_t sm = fast_cell_smem<T, DEG>();
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_cell_glm<T, DEG>, sm);
    attr = true;
  }
  k_cell_glm<T, DEG><<<nb, NT, sm, st>>>(tabs.cell, g, w, F, out, w0, ca, cb, combine, sc, wmean, w0mean, outmean);
}

#define INSTF(T, DEG)                                                                                         \
  template void launch_face_glm<T, DEG>(const FastAll<T, DEG>&, const FastGeom&, const T*, T*,              \
                                        const DevScalars*, double, cudaStream_t);                          \
  template void launch_cell_glm<T, DEG>(const FastAll<T, DEG>&, const FastGeom&, const T*, const T*, T*,    \
                                        const T*, double, double, int, const DevScalars*, const double*,    \
                                        const double*, double*, cudaStream_t);
INSTF(float, 1)
INSTF(float, 2)
INSTF(float, 3)
INSTF(double, 1)
INSTF(double, 2)

}  // namespace dgmhd
