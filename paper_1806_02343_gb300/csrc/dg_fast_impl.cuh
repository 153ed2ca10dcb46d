// Specialised kernels of the DG operator (included once per precision and
// degree by the dg_fast_*.cu units) for the GLM scheme and for the Powell
// scheme with the LDF basis on uniform 3D meshes (Sec. 3.5 eq. wdot;
// Sec. 4.1.2 HLLD; Sec. 4.1.3 Powell; Sec. 4.1.5 GLM).
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

#include <type_traits>
#include <utility>

#include "dg_fast.cuh"

#if !defined(DG_FAST_T) || !defined(DG_FAST_DEG) || !defined(DG_FAST_CONST)
#error "include from a dg_fast_<precision><degree>.cu unit that defines DG_FAST_T, DG_FAST_DEG, DG_FAST_CONST"
#endif
#include "dg_phys.cuh"

namespace dgmhd {

namespace {

constexpr int TC = 32;        // cells (or faces) per block

// Reference-element tables in the constant bank. They depend only on the
// scheme and the degree (not on the mesh), so one copy serves every context;
// indexed with compile-time offsets, each table value is a constant operand of
// its FMA. Each (precision, degree) is its own translation unit (they compile
// in parallel) with its own copy.
template <typename T, int DEG>
struct FastConst {
  static constexpr bool on = false;
};
#if DG_FAST_CONST
__constant__ FastAll<DG_FAST_T, DG_FAST_DEG> c_fast;
template <>
struct FastConst<DG_FAST_T, DG_FAST_DEG> {
  static constexpr bool on = true;
  __device__ static const FastAll<DG_FAST_T, DG_FAST_DEG>& get() { return c_fast; }
  static cudaError_t upload(const FastAll<DG_FAST_T, DG_FAST_DEG>& t) {
    return cudaMemcpyToSymbol(c_fast, &t, sizeof(t));
  }
};
#endif

template <typename T, int DEG, int A>
__device__ __forceinline__ const FaceTabs<T, DEG>& face_tabs(const FaceTabs<T, DEG>& param) {
  if constexpr (FastConst<T, DEG>::on) return FastConst<T, DEG>::get().face[A];
  else return param;
}

template <typename T, int DEG>
__device__ __forceinline__ const CellTabs<T, DEG>& cell_tabs(const CellTabs<T, DEG>& param) {
  if constexpr (FastConst<T, DEG>::on) return FastConst<T, DEG>::get().cell;
  else return param;
}

// compile-time loop: f(std::integral_constant<int, i>) for i = 0 .. n-1
template <typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int Nn, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, Nn>{});
}

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Two independent fused multiply-adds, x = a p + x and y = b q + y, each
// rounded once. FP32: one packed f32x2 instruction (sm_100 and later), which
// halves the instruction count of the contractions; FP64: two DFMAs.
__device__ __forceinline__ void fma2(float& x, float& y, float a, float b, float p, float q) {
  asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%0, %1};\n\t"
      "fma.rn.f32x2 rc, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rc;\n\t}"
      : "+f"(x), "+f"(y)
      : "f"(a), "f"(b), "f"(p), "f"(q));
}
__device__ __forceinline__ void fma2(double& x, double& y, double a, double b, double p, double q) {
  x = __fma_rn(a, p, x);
  y = __fma_rn(b, q, y);
}

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

// Asynchronous per-thread copies (cp.async, 4 bytes each) of the rows r = v + 9 i
// (r < NR) of the -axis neighbours of the block's cells into X[r][TC]; waited
// for by cp_async_wait_all and a barrier. Absent cells copy cell 0 (their
// results are not stored).
template <typename T, int NR>
__device__ __forceinline__ void stage_left_async(const FastGeom& g, const T* __restrict__ w, int64_t c, bool live,
                                                 int axis, int v, int f, T* X) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const int64_t cl = live ? nbr(g, coord_of(g, c), axis, -1) : 0;
  const int64_t S = g.stride;
  constexpr int PER = (NR + 8) / 9;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int r = v + 9 * i;
    if (r < NR) {
      const unsigned dst = (unsigned)__cvta_generic_to_shared(X + r * TC + f);
      if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(w + (int64_t)r * S + cl) : "memory");
      else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(w + (int64_t)r * S + cl) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ------------------------------------------------------------------ faces
// The faces normal to axis A whose right cells are the block's 32 cells:
// stage the left cells' (and, with own, this block's) coefficients, traces,
// HLLD. WR keeps this block's coefficients between calls. PRE: the left
// cells' rows are already being copied into WL (asynchronous copies issued
// by the previous axis); NEXT >= 0: once this axis's traces are done, issue
// those copies for axis NEXT, so they run while this axis's HLLD does
// (measured: 11.0 -> 10.5 ms per stage at 256^3).
template <typename T, int DEG, int A, bool OWN, bool PRE = false, int NEXT = -1>
__device__ __forceinline__ void face_axis(const FaceTabs<T, DEG>& tbp, const FastGeom& g, const T* __restrict__ w,
                                          T* __restrict__ F, const DevScalars* __restrict__ sc, T eps, T* WL, T* WR,
                                          T* TR) {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF, NR = 9 * N;
  const FaceTabs<T, DEG>& tb = face_tabs<T, DEG, A>(tbp);
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
  if (PRE) {
    cp_async_wait_all();
  } else {
    constexpr int PER = (NR + 8) / 9;
    T a[PER], b[PER];
    const int64_t S9 = 9 * S;
    const T* pa = w + (int64_t)v * S + c;
    const T* pb = w + (int64_t)v * S + cl;
#pragma unroll
    for (int i = 0; i < PER; ++i, pa += S9, pb += S9) {
      const int r = v + 9 * i;
      if (OWN) a[i] = (live && r < NR) ? *pa : T(1);
      b[i] = (live && r < NR) ? *pb : T(1);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int r = v + 9 * i;
      if (r < NR) {
        if (OWN) WR[r * TC + f] = a[i];
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
    const auto& Pt = s ? tb.PR : tb.PL;
    // two face points per packed FMA
#pragma unroll
    for (int p = 0; p + 1 < QF; p += 2) {
      T a0 = T(0), a1 = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) fma2(a0, a1, wl[l], wl[l], Pt[l][p], Pt[l][p + 1]);
      TR[((s * QF + p) * 9 + v) * TC + f] = a0;
      TR[((s * QF + p + 1) * 9 + v) * TC + f] = a1;
    }
    if (QF & 1) {
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) acc = fma_rn(wl[l], Pt[l][QF - 1], acc);
      TR[((s * QF + QF - 1) * 9 + v) * TC + f] = acc;
    }
  }
  __syncthreads();
  if constexpr (NEXT >= 0) stage_left_async<T, NR>(g, w, c, live, NEXT, v, f, WL);
  // HLLD per face point
  const T ch = pick_prec<T>(sc->ch, sc->ch32);
  const T gamma = pick_prec<T>(g.gamma, g.gamma32);
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
      for (int k = 0; k < 9; ++k) F[((int64_t)(A * QF + p) * 9) * S + c + (int64_t)k * S] = Fo[k];
    }
  }
}

template <typename T, int DEG, int A>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && DEG <= 2) ? 4 : 3) k_face_glm(const FaceTabs<T, DEG> tbp, const FastGeom g,
                                                 const T* __restrict__ w, T* __restrict__ F,
                                                 const DevScalars* __restrict__ sc, T eps) {
  constexpr int NR = 9 * FastDims<DEG>::N;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* WL = reinterpret_cast<T*>(smraw);       // [NR][TC]
  T* WR = WL + NR * TC;                      // [NR][TC]
  T* TR = WR + NR * TC;                      // [2][QF][9][TC]
  face_axis<T, DEG, A, true>(tbp, g, w, F, sc, eps, WL, WR, TR);
}

// All three axes in one pass: the block's own coefficients are read once and
// kept in shared memory for the x, y and z faces (one state read fewer per
// face than three separate passes).
template <typename T, int DEG>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && DEG <= 2) ? 4 : 3) k_face_glm3(
    const FaceTabs<T, DEG> tb0, const FaceTabs<T, DEG> tb1, const FaceTabs<T, DEG> tb2, const FastGeom g,
    const T* __restrict__ w, T* __restrict__ F, const DevScalars* __restrict__ sc, T eps) {
  constexpr int NR = 9 * FastDims<DEG>::N;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* WL = reinterpret_cast<T*>(smraw);
  T* WR = WL + NR * TC;
  T* TR = WR + NR * TC;
  face_axis<T, DEG, 0, true, false, 1>(tb0, g, w, F, sc, eps, WL, WR, TR);
  __syncthreads();
  face_axis<T, DEG, 1, false, true, 2>(tb1, g, w, F, sc, eps, WL, WR, TR);
  __syncthreads();
  face_axis<T, DEG, 2, false, true, -1>(tb2, g, w, F, sc, eps, WL, WR, TR);
}

// ------------------------------------------------------------------ cells
// primitive slots per volume point
enum { SL_RHO = 0, SL_B = 5, SL_PSI = 8, SL_V = 9, SL_PT = 12, SL_VB = 13, SL_EPT = 14, SL_ZERO = 15, NSL = 16 };

template <typename T, int DEG>
__global__ void __launch_bounds__(NT, 3) k_cell_glm(const CellTabs<T, DEG> tbp, const FastGeom g,
                                                 const T* __restrict__ w, const T* __restrict__ F, T* out,
                                                 const T* w0, double ca, double cb, float ca32, float cb32,
                                                 int cmode,
                                                 const DevScalars* __restrict__ sc,
                                                 const double* __restrict__ wmean, const double* w0mean,
                                                 double* outmean) {
  // out / outmean may alias w0 / w0mean: each element is read, then written, by one thread.
  constexpr int N = FastDims<DEG>::N, QV = FastDims<DEG>::QV, QF = FastDims<DEG>::QF;
  constexpr int QC = FastDims<DEG>::QC;  // volume points per pass
  const CellTabs<T, DEG>& tb = cell_tabs<T, DEG>(tbp);
  static_assert(N % 2 == 0, "mode pairs");
  extern __shared__ __align__(16) unsigned char smraw[];
  T* PR = reinterpret_cast<T*>(smraw);  // [QC][NSL][TC]
  const int t = threadIdx.x;
  const int f = t & (TC - 1);
  const int v = t >> 5;  // warp-uniform variable
  const int64_t c = (int64_t)blockIdx.x * TC + f;
  const bool live = c < g.ncell;
  const int64_t S = g.stride;
  const bool mix = wmean != nullptr;
  const T gamma = pick_prec<T>(g.gamma, g.gamma32);
  const T ch = pick_prec<T>(sc->ch, sc->ch32);

  T wl[N];
  {
    // pointer steps of one row (S elements) instead of a 64-bit index per load
    const T* pw = w + (int64_t)(v * N) * S + c;
#pragma unroll
    for (int l = 0; l < N; ++l, pw += S) wl[l] = live ? *pw : (v == 0 && l == 0 ? T(1) : T(0));
  }
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
    // two volume points per packed FMA
#pragma unroll
    for (int qq = 0; qq + 1 < QC; qq += 2) {
      T u0 = T(0), u1 = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) fma2(u0, u1, wl[l], wl[l], tb.P[l][q0 + qq], tb.P[l][q0 + qq + 1]);
      PR[(qq * NSL + v) * TC + f] = u0;
      PR[((qq + 1) * NSL + v) * TC + f] = u1;
    }
    if (QC & 1) {
      T u = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) u = fma_rn(wl[l], tb.P[l][q0 + QC - 1], u);
      PR[((QC - 1) * NSL + v) * TC + f] = u;
    }
    __syncthreads();
    // primitives per point
    for (int idx = t; idx < QC * TC; idx += NT) {
      const int qq = idx / TC, ff = idx % TC;
      T* pr = PR + qq * NSL * TC + ff;
      const T rho = pr[0], ir = rcp(rho);
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
      T fa[3] = {gax == 0 ? ga : T(0), gax == 1 ? ga : T(0), gax == 2 ? ga : T(0)};
      fma2(fa[0], fa[1], be, be, pr[SL_B * TC], pr[(SL_B + 1) * TC]);
      fma2(fa[0], fa[1], al, al, pr[SL_V * TC], pr[(SL_V + 1) * TC]);
      fa[2] = fma_rn(al, pr[(SL_V + 2) * TC], fma_rn(be, pr[(SL_B + 2) * TC], fa[2]));
      // only the modes with a non-zero derivative along a, two per packed FMA
      // (mode indices are template constants: racc stays in registers)
      const int q = q0 + qq;
      static_for<3>([&](auto A) {
        constexpr int a = decltype(A)::value;
        constexpr int cnt = kModes<DEG>.cnt[a];
        static_for<(cnt + 1) / 2>([&](auto I) {
          constexpr int i = decltype(I)::value;
          constexpr int l0 = kModes<DEG>.nz[a][2 * i];
          // odd count: the last pair's second slot is mode 0 with a zero
          // weight (racc[0] is not an output: the mean comes from the faces)
          constexpr int l1 = 2 * i + 1 < cnt ? kModes<DEG>.nz[a][2 * i + 1] : 0;
          fma2(racc[l0], racc[l1], fa[a], fa[a], tb.dP2[a][i][q][0], tb.dP2[a][i][q][1]);
        });
      });
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
    const int64_t S9 = 9 * S;  // between the points of one variable's face rows
    // the next face's QF values are loaded while this face is contracted
    // (measured: 14.8 -> 14.3 ms per stage at 256^3)
    T Fq[2][QF];
    auto ld = [&](int k, T* dst) {
      const int a = k >> 1, s = k & 1;
      const int64_t fc = s ? nbr(g, kc, a, +1) : c;
      const T* q = F + (int64_t)v * S + (int64_t)(a * QF) * S9 + fc;
#pragma unroll
      for (int p = 0; p < QF; ++p, q += S9) dst[p] = *q;
    };
    ld(0, Fq[0]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int k = 2 * a + s;
        if (k + 1 < 6) ld(k + 1, Fq[(k + 1) & 1]);
        const T* Fp = Fq[k & 1];
        // fs: this face's mean-row sum. The weights of mode 0 are w_p on both
        // sides (P_0 = 1) and round-to-nearest is symmetric, so the sum of
        // -F w_p here is bitwise the negation of the neighbour's sum of F w_p.
        T fs = T(0);
#pragma unroll
        for (int p = 0; p < QF; ++p) {
          const T Fr = Fp[p];
          const T Fv = s ? -Fr : Fr;
          const T* Pw = tb.Pfw[2 * a + s][p];
          fma2(fs, racc[1], Fv, Fv, Pw[0], Pw[1]);
#pragma unroll
          for (int l = 2; l + 1 < N; l += 2) fma2(racc[l], racc[l + 1], Fv, Fv, Pw[l], Pw[l + 1]);
        }
        fsum[2 * a + s] = fs;
      }
    }
  }
  if (!live) return;
  // mode 0 (cell mean)
  {
    const int64_t i = (int64_t)(v * N) * S + c;
    if (sizeof(T) == 4 && mix) {
      // FP32 form. The six face sums are added as an unevaluated float pair
      // (Knuth's TwoSum: s + e equals a + b exactly), so the cell's total is
      // accurate to about 2^-48 of the face sums; it enters the FP64 mean
      // through one conversion. GB300's FP64 rate is 1/64 of FP32: the FP64
      // work here is a handful of operations per (cell, variable), and no
      // thread converts a uniform FP64 scalar (float copies are passed).
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
      const double wz = wmean[(int64_t)v * S + c];
      if (cmode == 0) {
        double rhs = g.kmean * tot;
        if (v == 8) rhs = fma(-sc->kappa, wz, rhs);
        out[i] = (T)rhs;
        outmean[(int64_t)v * S + c] = rhs;
      } else {
        // o = ca w0 + cb (wz + dt rhs), rhs = kmean tot (- kappa wz for psi)
        const double kd = cb * sc->dt;
        double base = cb * wz;
        if (cmode == 2) base = fma(ca, w0mean[(int64_t)v * S + c], base);
        if (v == 8) base = fma(-kd * sc->kappa, wz, base);
        const double o = fma(kd * g.kmean, tot, base);
        outmean[(int64_t)v * S + c] = o;
        out[i] = (T)o;
      }
    } else {
      const double dt = sc->dt, kappa = sc->kappa;
      const double mean_acc = ((double)fsum[0] + (double)fsum[1]) + ((double)fsum[2] + (double)fsum[3]) +
                              ((double)fsum[4] + (double)fsum[5]);
      double rhs = g.metric * (double)tb.minv[0] * mean_acc;
      const double wz = (double)wl[0];
      if (v == 8) rhs -= kappa * wz;
      if (cmode == 0) out[i] = (T)rhs;
      else out[i] = (T)(ca * (double)w0[i] + cb * (wz + dt * rhs));
    }
  }
  const T tm = pick_prec<T>(g.metric, g.metric32), tdt = pick_prec<T>(sc->dt, sc->dt32);
  const T tca = pick_prec<T>(ca, ca32), tcb = pick_prec<T>(cb, cb32), tk = pick_prec<T>(sc->kappa, sc->kappa32);
  {
    const int64_t i1 = (int64_t)(v * N + 1) * S + c;
    T* po = out + i1;
    const T* p0 = cmode == 0 ? nullptr : w0 + i1;
#pragma unroll
    for (int l = 1; l < N; ++l, po += S) {
      T rhs = tm * tb.minv[l] * racc[l];
      if (v == 8) rhs -= tk * wl[l];
      if (cmode == 0) {
        *po = rhs;
      } else {
        *po = tca * *p0 + tcb * (wl[l] + tdt * rhs);
        p0 += S;
      }
    }
  }
}

// ------------------------------------------------------------------ Powell / LDF
// The same organisation for the Powell scheme with the LDF basis (Sec. 3.3,
// Sec. 4.1.3): eight variables, the magnetic field carried inside the kernels
// in the Legendre form of its three components (PowTabs). Thread (v, cell):
// v < 5 the Legendre variables, v = 5 + cc component cc of B. The face pass
// stores per face point the eight flux components and, for the Powell face
// term, B^n_F minus each side's own normal trace: slot 8 for the left cell,
// slot 9 for the right cell.
constexpr int NFS = 10;       // face-buffer slots per face point (Powell)
constexpr int NTP = 8 * TC;   // cell pass: one thread per (variable, cell)

template <typename T, int DEG>
__device__ __forceinline__ const PowTabs<T, DEG>& pow_tabs() {
  static_assert(FastConst<T, DEG>::on, "the Powell kernels read their tables from the constant bank");
  return FastConst<T, DEG>::get().pow;
}

// b[l] = sum_j Af[CC][j][l] X[j * TC]: Legendre coefficients of component CC
// of B from the LDF coefficients staged at X (two modes per packed FMA)
template <typename T, int DEG, int CC>
__device__ __forceinline__ void ldf_to_legendre(const T* X, T (&b)[FastDims<DEG>::N]) {
  constexpr int N = FastDims<DEG>::N, NDIV = PowDims<DEG>::NDIV;
  const PowTabs<T, DEG>& pt = pow_tabs<T, DEG>();
#pragma unroll
  for (int l = 0; l < N; ++l) b[l] = T(0);
#pragma unroll
  for (int j = 0; j < NDIV; ++j) {
    const T x = X[j * TC];
#pragma unroll
    for (int l = 0; l < N; l += 2) fma2(b[l], b[l + 1], x, x, pt.Af[CC][j][l], pt.Af[CC][j][l + 1]);
  }
}

template <typename T, int DEG>
__device__ __forceinline__ void ldf_to_legendre(int cc, const T* X, T (&b)[FastDims<DEG>::N]) {
  if (cc == 0) ldf_to_legendre<T, DEG, 0>(X, b);
  else if (cc == 1) ldf_to_legendre<T, DEG, 1>(X, b);
  else ldf_to_legendre<T, DEG, 2>(X, b);
}

// traces of one side at the QF points of a face (two points per packed FMA)
template <typename T, int DEG, typename Tab>
__device__ __forceinline__ void face_trace(const T (&wl)[FastDims<DEG>::N], const Tab& Pt, T* out) {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF;
#pragma unroll
  for (int p = 0; p + 1 < QF; p += 2) {
    T a0 = T(0), a1 = T(0);
#pragma unroll
    for (int l = 0; l < N; ++l) fma2(a0, a1, wl[l], wl[l], Pt[l][p], Pt[l][p + 1]);
    out[p * 8 * TC] = a0;
    out[(p + 1) * 8 * TC] = a1;
  }
  if (QF & 1) {
    T acc = T(0);
#pragma unroll
    for (int l = 0; l < N; ++l) acc = fma_rn(wl[l], Pt[l][QF - 1], acc);
    out[(QF - 1) * 8 * TC] = acc;
  }
}

// The faces normal to axis A whose right cells are the block's 32 cells.
// WL / WR: raw state rows of the left / own cells; BR: the own cells' B in
// Legendre form (computed with OWN, kept for the next axes); TR: traces
// [side][point][variable][cell].
template <typename T, int DEG, int A, bool OWN, bool PRE = false, int NEXT = -1>
__device__ __forceinline__ void face_axis_pow(const FastGeom& g, const T* __restrict__ w, T* __restrict__ F, T eps,
                                              T* WL, T* WR, T* BR, T* TR) {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF, NDIV = PowDims<DEG>::NDIV, NRP = 5 * N + NDIV;
  const FaceTabs<T, DEG>& tb = FastConst<T, DEG>::get().face[A];
  const int t = threadIdx.x;
  const int f = t & (TC - 1);
  const int v = t >> 5;  // 0..8, warp-uniform
  const int64_t c = (int64_t)blockIdx.x * TC + f;
  const bool live = c < g.ncell;
  const int64_t S = g.stride;
  const int64_t cl = live ? nbr(g, coord_of(g, c), A, -1) : 0;
  if (PRE) {
    cp_async_wait_all();  // the left cells' rows, copied while the previous axis ran HLLD
  } else {
    constexpr int PER = (NRP + 8) / 9;
    T a[PER], b[PER];
    const int64_t S9 = 9 * S;
    const T* pa = w + (int64_t)v * S + c;
    const T* pb = w + (int64_t)v * S + cl;
#pragma unroll
    for (int i = 0; i < PER; ++i, pa += S9, pb += S9) {
      const int r = v + 9 * i;
      if (OWN) a[i] = (live && r < NRP) ? *pa : T(1);
      b[i] = (live && r < NRP) ? *pb : T(1);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int r = v + 9 * i;
      if (r < NRP) {
        if (OWN) WR[r * TC + f] = a[i];
        WL[r * TC + f] = b[i];
      }
    }
  }
  __syncthreads();
  if (v < 8) {
    T wl[N];
    // left cell
    if (v < 5) {
#pragma unroll
      for (int l = 0; l < N; ++l) wl[l] = WL[(v * N + l) * TC + f];
    } else {
      ldf_to_legendre<T, DEG>(v - 5, WL + 5 * N * TC + f, wl);
    }
    face_trace<T, DEG>(wl, tb.PL, TR + v * TC + f);
    // own cell
    if (v < 5) {
#pragma unroll
      for (int l = 0; l < N; ++l) wl[l] = WR[(v * N + l) * TC + f];
    } else if (OWN) {
      ldf_to_legendre<T, DEG>(v - 5, WR + 5 * N * TC + f, wl);
#pragma unroll
      for (int l = 0; l < N; ++l) BR[((v - 5) * N + l) * TC + f] = wl[l];
    } else {
#pragma unroll
      for (int l = 0; l < N; ++l) wl[l] = BR[((v - 5) * N + l) * TC + f];
    }
    face_trace<T, DEG>(wl, tb.PR, TR + (QF * 8 + v) * TC + f);
  }
  __syncthreads();
  if constexpr (NEXT >= 0) stage_left_async<T, NRP>(g, w, c, live, NEXT, v, f, WL);
  // HLLD per face point (Sec. 4.1.2), B^n_F of eq. bxface-average
  const T gamma = pick_prec<T>(g.gamma, g.gamma32);
  for (int p = v; p < QF; p += 9) {
    T uL[9], uR[9], Fo[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uL[k] = TR[((0 * QF + p) * 8 + k) * TC + f];
      uR[k] = TR[((1 * QF + p) * 8 + k) * TC + f];
    }
    uL[8] = uR[8] = T(0);
    const T bnF = face_flux(uL, uR, A, gamma, false, T(0), eps, Fo);
    if (live) {
      T* o = F + (int64_t)((A * QF + p) * NFS) * S + c;
#pragma unroll
      for (int k = 0; k < 8; ++k) o[(int64_t)k * S] = Fo[k];
      o[(int64_t)8 * S] = bnF - uL[5 + A];
      o[(int64_t)9 * S] = bnF - uR[5 + A];
    }
  }
}

template <typename T, int DEG>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && DEG <= 2) ? 4 : 2) k_face_pow3(const FastGeom g,
                                                                                       const T* __restrict__ w,
                                                                                       T* __restrict__ F, T eps) {
  constexpr int N = FastDims<DEG>::N, NRP = 5 * N + PowDims<DEG>::NDIV;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* WL = reinterpret_cast<T*>(smraw);  // [NRP][TC]
  T* WR = WL + NRP * TC;                // [NRP][TC]
  T* BR = WR + NRP * TC;                // [3 N][TC]
  T* TR = BR + 3 * N * TC;              // [2][QF][8][TC]
  face_axis_pow<T, DEG, 0, true, false, 1>(g, w, F, eps, WL, WR, BR, TR);
  __syncthreads();
  face_axis_pow<T, DEG, 1, false, true, 2>(g, w, F, eps, WL, WR, BR, TR);
  __syncthreads();
  face_axis_pow<T, DEG, 2, false, true, -1>(g, w, F, eps, WL, WR, BR, TR);
}

// Sum of a cell's six face sums of one mean row. FP32: an unevaluated float
// pair (Knuth's TwoSum: s + e equals a + b exactly), accurate to about 2^-48
// of the face sums, rounded once to double; FP64: in pairs.
template <typename T>
__device__ __forceinline__ double face_total(const T (&fs)[6]) {
  if constexpr (sizeof(T) == 4) {
    float hi = fs[0], lo = 0.f;
#pragma unroll
    for (int k = 1; k < 6; ++k) {
      const float b = fs[k];
      const float s2 = __fadd_rn(hi, b);
      const float bb = __fsub_rn(s2, hi);
      const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s2, bb)), __fsub_rn(b, bb));
      hi = s2;
      lo = __fadd_rn(lo, e);
    }
    return (double)hi + (double)lo;
  } else {
    return ((double)fs[0] + (double)fs[1]) + ((double)fs[2] + (double)fs[3]) + ((double)fs[4] + (double)fs[5]);
  }
}

// Pieces of the Powell cell update shared by the uniform and octree kernels
// (thread (v, cell), 8 warps of 32 cells). Shared memory: PR [QC][NSL][TC]
// point values, LS [NDIV][TC] the LDF coefficients, QM [8][TC] cell means.

// loads the state: v < 5 its Legendre row block, v >= 5 the LDF rows (staged
// in LS by the three B warps) turned into the Legendre form of component v - 5;
// QM[v] = the mean of variable v
template <typename T, int DEG>
__device__ __forceinline__ void pow_load(const T* __restrict__ w, int64_t S, int64_t c, bool live, int v, int f,
                                         T* LS, T* QM, T (&wl)[FastDims<DEG>::N]) {
  constexpr int N = FastDims<DEG>::N, NDIV = PowDims<DEG>::NDIV;
  if (v < 5) {
    const T* pw = w + (int64_t)(v * N) * S + c;
#pragma unroll
    for (int l = 0; l < N; ++l, pw += S) wl[l] = live ? *pw : ((l == 0 && (v == 0 || v == 4)) ? T(1) : T(0));
  } else {
    for (int j = v - 5; j < NDIV; j += 3) LS[j * TC + f] = live ? w[(int64_t)(5 * N + j) * S + c] : T(0);
  }
  __syncthreads();
  if (v >= 5) ldf_to_legendre<T, DEG>(v - 5, LS + f, wl);
  QM[v * TC + f] = wl[0];
}

// volume integral of variable v (Sec. 3.5 eq. wdot): racc_l = sum_a sum_q
// f_a(q) w_q d_a P_l(q), the fluxes at the Gauss points from the projected
// state; racc[0] stays zero
template <typename T, int DEG>
__device__ __forceinline__ void pow_volume(const T (&wl)[FastDims<DEG>::N], T* PR, T gamma, int v, int f,
                                           T (&racc)[FastDims<DEG>::N]) {
  constexpr int N = FastDims<DEG>::N, QV = FastDims<DEG>::QV, QC = FastDims<DEG>::QC;
  const CellTabs<T, DEG>& tb = FastConst<T, DEG>::get().cell;
  const int t = threadIdx.x;
  // flux of variable v: f_a = alpha v_a + beta B_a (+ p_T if a is the momentum's axis)
  int aidx, bidx, gidx, gax;
  T bs;
  if (v == 0) { aidx = SL_RHO; bidx = SL_ZERO; bs = T(0); gidx = SL_ZERO; gax = -1; }
  else if (v <= 3) { aidx = v; bidx = SL_B + v - 1; bs = T(-1); gidx = SL_PT; gax = v - 1; }
  else if (v == 4) { aidx = SL_EPT; bidx = SL_VB; bs = T(-1); gidx = SL_ZERO; gax = -1; }
  else { aidx = v; bidx = SL_V + v - 5; bs = T(-1); gidx = SL_ZERO; gax = -1; }
#pragma unroll
  for (int l = 0; l < N; ++l) racc[l] = T(0);
#pragma unroll
  for (int q0 = 0; q0 < QV; q0 += QC) {
#pragma unroll
    for (int qq = 0; qq + 1 < QC; qq += 2) {
      T u0 = T(0), u1 = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) fma2(u0, u1, wl[l], wl[l], tb.P[l][q0 + qq], tb.P[l][q0 + qq + 1]);
      PR[(qq * NSL + v) * TC + f] = u0;
      PR[((qq + 1) * NSL + v) * TC + f] = u1;
    }
    if (QC & 1) {
      T u = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) u = fma_rn(wl[l], tb.P[l][q0 + QC - 1], u);
      PR[((QC - 1) * NSL + v) * TC + f] = u;
    }
    __syncthreads();
    for (int idx = t; idx < QC * TC; idx += NTP) {
      const int qq = idx / TC, ff = idx % TC;
      T* pr = PR + qq * NSL * TC + ff;
      const T rho = pr[0], ir = rcp(rho);
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
#pragma unroll
    for (int qq = 0; qq < QC; ++qq) {
      const T* pr = PR + qq * NSL * TC + f;
      const T al = pr[aidx * TC];
      const T be = bs * pr[bidx * TC];
      const T ga = pr[gidx * TC];
      T fa[3] = {gax == 0 ? ga : T(0), gax == 1 ? ga : T(0), gax == 2 ? ga : T(0)};
      fma2(fa[0], fa[1], be, be, pr[SL_B * TC], pr[(SL_B + 1) * TC]);
      fma2(fa[0], fa[1], al, al, pr[SL_V * TC], pr[(SL_V + 1) * TC]);
      fa[2] = fma_rn(al, pr[(SL_V + 2) * TC], fma_rn(be, pr[(SL_B + 2) * TC], fa[2]));
      const int q = q0 + qq;
      static_for<3>([&](auto AX) {
        constexpr int a = decltype(AX)::value;
        constexpr int cnt = kModes<DEG>.cnt[a];
        static_for<(cnt + 1) / 2>([&](auto I) {
          constexpr int i = decltype(I)::value;
          constexpr int l0 = kModes<DEG>.nz[a][2 * i];
          constexpr int l1 = 2 * i + 1 < cnt ? kModes<DEG>.nz[a][2 * i + 1] : 0;
          fma2(racc[l0], racc[l1], fa[a], fa[a], tb.dP2[a][i][q][0], tb.dP2[a][i][q][1]);
        });
      });
    }
    __syncthreads();
  }
}

// Powell source q(<u>_K) = (0, B, v.B, v) of variable v from the cell means
// (Sec. 4.1.3); it multiplies the face terms (B^n_F - B_n) of the own side
template <typename T>
__device__ __forceinline__ T pow_q(const T* QM, int v, int f) {
  if (v == 0) return T(0);
  const T rho = QM[f];
  if (v <= 3) return QM[(4 + v) * TC + f];
  if (v == 4) {
    const T vx = QM[1 * TC + f] / rho, vy = QM[2 * TC + f] / rho, vz = QM[3 * TC + f] / rho;
    return vx * QM[5 * TC + f] + vy * QM[6 * TC + f] + vz * QM[7 * TC + f];
  }
  return QM[(v - 4) * TC + f] / rho;
}

// The update of the cell's rows from racc (modes >= 1) and tot (the mean row's
// face total): rhs = tm minv racc for the Legendre rows, the LDF rows through
// the back transform (B residuals exchanged in RL = PR), the mean rows in FP64
// with factor km. Ends with a barrier that every thread of the block reaches.
template <typename T, int DEG>
__device__ __forceinline__ void pow_store(const T (&wl)[FastDims<DEG>::N], const T (&racc)[FastDims<DEG>::N],
                                          double tot, bool live, int v, int f, int64_t S, int64_t c, T* PR,
                                          const T* LS, T tm, double km, T* out, const T* w0, double ca, double cb,
                                          float ca32, float cb32, int cmode, const DevScalars* __restrict__ sc,
                                          const double* __restrict__ wmean, const double* w0mean, double* outmean) {
  constexpr int N = FastDims<DEG>::N, NDIV = PowDims<DEG>::NDIV, NP = PowDims<DEG>::NP;
  const CellTabs<T, DEG>& tb = FastConst<T, DEG>::get().cell;
  const PowTabs<T, DEG>& pt = pow_tabs<T, DEG>();
  T* RL = PR;  // [3][N][TC]
  if (v >= 5) {
#pragma unroll
    for (int l = 1; l < N; ++l) RL[((v - 5) * N + l) * TC + f] = racc[l];
  }
  __syncthreads();
  if (!live) return;
  const bool mix = wmean != nullptr;
  const T tdt = pick_prec<T>(sc->dt, sc->dt32);
  const T tca = pick_prec<T>(ca, ca32), tcb = pick_prec<T>(cb, cb32);
  // mean row: Legendre mode 0 of variable v < 5, the constant LDF row jm[cc] of component cc
  {
    const int row = v < 5 ? v * N : 5 * N + pt.jm[v - 5];
    const int m = v < 5 ? v : 5 + pt.jm[v - 5];
    const int64_t i = (int64_t)row * S + c;
    if (sizeof(T) == 4 && mix) {
      const double wz = wmean[(int64_t)m * S + c];
      if (cmode == 0) {
        const double rhs = km * tot;
        out[i] = (T)rhs;
        outmean[(int64_t)m * S + c] = rhs;
      } else {
        const double kd = cb * sc->dt;
        double base = cb * wz;
        if (cmode == 2) base = fma(ca, w0mean[(int64_t)m * S + c], base);
        const double o = fma(kd * km, tot, base);
        outmean[(int64_t)m * S + c] = o;
        out[i] = (T)o;
      }
    } else {
      const double rhs = km * tot;
      const double wz = v < 5 ? (double)wl[0] : (double)LS[pt.jm[v - 5] * TC + f];
      if (cmode == 0) out[i] = (T)rhs;
      else out[i] = (T)(ca * (double)w0[i] + cb * (wz + sc->dt * rhs));
    }
  }
  if (v < 5) {
    const int64_t i1 = (int64_t)(v * N + 1) * S + c;
    T* po = out + i1;
    const T* p0 = cmode == 0 ? nullptr : w0 + i1;
#pragma unroll
    for (int l = 1; l < N; ++l, po += S) {
      const T rhs = tm * tb.minv[l] * racc[l];
      if (cmode == 0) {
        *po = rhs;
      } else {
        *po = tca * *p0 + tcb * (wl[l] + tdt * rhs);
        p0 += S;
      }
    }
  } else {
    // non-mean LDF rows j = 3 + 2k, 4 + 2k, pair k on component thread k mod 3
    const int cc = v - 5;
    static_for<NP>([&](auto K) {
      constexpr int k = decltype(K)::value;
      constexpr int j0 = 3 + 2 * k, j1 = j0 + 1;
      if (k % 3 == cc) {
        T R0 = T(0), R1 = T(0);
        static_for<3>([&](auto CCI) {
          constexpr int c2 = decltype(CCI)::value;
#pragma unroll
          for (int l = 1; l < N; ++l) {
            const T x = RL[(c2 * N + l) * TC + f];
            fma2(R0, R1, x, x, pt.Ab[k][c2][l][0], pt.Ab[k][c2][l][1]);
          }
        });
        auto put = [&](int j, T R) {
          const int64_t i = (int64_t)(5 * N + j) * S + c;
          const T rhs = tm * pt.minvL[j] * R;
          if (cmode == 0) out[i] = rhs;
          else out[i] = tca * w0[i] + tcb * (LS[j * TC + f] + tdt * rhs);
        };
        put(j0, R0);
        if constexpr (j1 < NDIV) put(j1, R1);
      }
    });
  }
}

template <typename T, int DEG>
__global__ void __launch_bounds__(NTP, 3) k_cell_pow(const FastGeom g, const T* __restrict__ w,
                                                     const T* __restrict__ F, T* out, const T* w0, double ca,
                                                     double cb, float ca32, float cb32, int cmode,
                                                     const DevScalars* __restrict__ sc,
                                                     const double* __restrict__ wmean, const double* w0mean,
                                                     double* outmean) {
  // out / outmean may alias w0 / w0mean: each element is read, then written, by one thread.
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF, QC = FastDims<DEG>::QC;
  constexpr int NDIV = PowDims<DEG>::NDIV;
  const CellTabs<T, DEG>& tb = FastConst<T, DEG>::get().cell;
  const PowTabs<T, DEG>& pt = pow_tabs<T, DEG>();
  static_assert(N % 2 == 0, "mode pairs");
  static_assert(3 * N <= QC * NSL, "residual exchange fits in the point buffer");
  extern __shared__ __align__(16) unsigned char smraw[];
  T* PR = reinterpret_cast<T*>(smraw);
  T* LS = PR + QC * NSL * TC;
  T* QM = LS + NDIV * TC;
  const int f = threadIdx.x & (TC - 1);
  const int v = threadIdx.x >> 5;  // warp-uniform variable, 0..7
  const int64_t c = (int64_t)blockIdx.x * TC + f;
  const bool live = c < g.ncell;
  const int64_t S = g.stride;
  T wl[N], racc[N];
  pow_load<T, DEG>(w, S, c, live, v, f, LS, QM, wl);
  pow_volume<T, DEG>(wl, PR, pick_prec<T>(g.gamma, g.gamma32), v, f, racc);
  const T qv = pow_q(QM, v, f);
  // surface integral (mean row per face in a fixed order, as in k_cell_glm)
  T fsum[6];
  const Coord kc = coord_of(g, live ? c : 0);
  if (live) {
    const int64_t SP = (int64_t)NFS * S;  // between the points of one slot
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int64_t fc = s ? nbr(g, kc, a, +1) : c;
        const int64_t base = (int64_t)(a * QF) * SP + fc;
        T Fp[QF];
        {
          const T* q = F + base + (int64_t)v * S;
#pragma unroll
          for (int p = 0; p < QF; ++p, q += SP) Fp[p] = *q;
        }
        if (v > 0) {
          // +a face (s = 1): this cell is the left one, slot 8; -a face: slot 9
          const T* d = F + base + (int64_t)(s ? 8 : 9) * S;
#pragma unroll
          for (int p = 0; p < QF; ++p, d += SP) Fp[p] = fma_rn(qv, *d, Fp[p]);
        }
        T fs = T(0);
#pragma unroll
        for (int p = 0; p < QF; ++p) {
          const T Fv = s ? -Fp[p] : Fp[p];
          const T* Pw = tb.Pfw[2 * a + s][p];
          fma2(fs, racc[1], Fv, Fv, Pw[0], Pw[1]);
#pragma unroll
          for (int l = 2; l + 1 < N; l += 2) fma2(racc[l], racc[l + 1], Fv, Fv, Pw[l], Pw[l + 1]);
        }
        fsum[2 * a + s] = fs;
      }
    }
  }
  const double km = v < 5 ? g.kmean : g.metric * (live ? pt.kL[v - 5] : 0.0);
  pow_store<T, DEG>(wl, racc, live ? face_total<T>(fsum) : 0.0, live, v, f, S, c, PR, LS,
                    pick_prec<T>(g.metric, g.metric32), km, out, w0, ca, cb, ca32, cb32, cmode, sc, wmean, w0mean,
                    outmean);
}

// ------------------------------------------------------------------ Powell on octree face lists
// Faces are processed in blocks of up to 32 faces of one type (axis a; same
// level, or the left or right side coarse with sub-face s), listed by the
// host: each block stages its type's two trace tables. Face-buffer layout:
// [face][point][slot], NFS slots as in the uniform pass.
template <typename T, int DEG>
__device__ __forceinline__ void face_trace_smem(const T (&wl)[FastDims<DEG>::N], const T* Pt, T* out) {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF, QFP = FaceTabs<T, DEG>::QFP;
#pragma unroll
  for (int p = 0; p + 1 < QF; p += 2) {
    T a0 = T(0), a1 = T(0);
#pragma unroll
    for (int l = 0; l < N; ++l) fma2(a0, a1, wl[l], wl[l], Pt[l * QFP + p], Pt[l * QFP + p + 1]);
    out[p * 8 * TC] = a0;
    out[(p + 1) * 8 * TC] = a1;
  }
  if (QF & 1) {
    T acc = T(0);
#pragma unroll
    for (int l = 0; l < N; ++l) acc = fma_rn(wl[l], Pt[l * QFP + QF - 1], acc);
    out[(QF - 1) * 8 * TC] = acc;
  }
}

template <typename T, int DEG, int A>
__device__ __forceinline__ void list_hlld(const T* TRC, int v, int f, bool live, int64_t fid, T gamma, T eps,
                                          T* __restrict__ F) {
  constexpr int QF = FastDims<DEG>::QF;
  for (int p = v; p < QF; p += 9) {
    T uL[9], uR[9], Fo[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uL[k] = TRC[((0 * QF + p) * 8 + k) * TC + f];
      uR[k] = TRC[((1 * QF + p) * 8 + k) * TC + f];
    }
    uL[8] = uR[8] = T(0);
    const T bnF = face_flux(uL, uR, A, gamma, false, T(0), eps, Fo);
    if (live) {
      T* q = F + (fid * QF + p) * NFS;
#pragma unroll
      for (int k = 0; k < 8; ++k) q[k] = Fo[k];
      q[8] = bnF - uL[5 + A];
      q[9] = bnF - uR[5 + A];
    }
  }
}

template <typename T, int DEG>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && DEG <= 2) ? 4 : 2) k_face_list_pow(const OctPow<T> o,
                                                                                          T gamma, T eps,
                                                                                          const T* __restrict__ w,
                                                                                          T* __restrict__ F) {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF, NDIV = PowDims<DEG>::NDIV, NRP = 5 * N + NDIV;
  constexpr int QFP = FaceTabs<T, DEG>::QFP;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* TT = reinterpret_cast<T*>(smraw);  // [2][N][QFP] the type's left / right trace tables
  T* WL = TT + 2 * N * QFP;             // [NRP][TC]
  T* WR = WL + NRP * TC;                // [NRP][TC]
  T* TRC = WR + NRP * TC;               // [2][QF][8][TC]
  const int t = threadIdx.x;
  const int f = t & (TC - 1);
  const int v = t >> 5;
  const int bt = o.btype[blockIdx.x];
  const int type = bt & 255, cnt = bt >> 8;
  const int A = type / 9;
  const bool live = f < cnt;
  const int64_t fid = live ? o.bface[o.bstart[blockIdx.x] + f] : 0;
  const int64_t cL = live ? o.fL[fid] : 0, cR = live ? o.fR[fid] : 0;
  const int64_t S = o.stride;
  for (int i = t; i < 2 * N * QFP; i += NT) TT[i] = o.ftab[(size_t)type * 2 * N * QFP + i];
  {
    constexpr int PER = (NRP + 8) / 9;
    T a[PER], b[PER];
    const int64_t S9 = 9 * S;
    const T* pa = w + (int64_t)v * S + cL;
    const T* pb = w + (int64_t)v * S + cR;
#pragma unroll
    for (int i = 0; i < PER; ++i, pa += S9, pb += S9) {
      const int r = v + 9 * i;
      a[i] = (live && r < NRP) ? *pa : T(1);
      b[i] = (live && r < NRP) ? *pb : T(1);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int r = v + 9 * i;
      if (r < NRP) {
        WL[r * TC + f] = a[i];
        WR[r * TC + f] = b[i];
      }
    }
  }
  __syncthreads();
  if (v < 8) {
    T wl[N];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const T* W = s ? WR : WL;
      if (v < 5) {
#pragma unroll
        for (int l = 0; l < N; ++l) wl[l] = W[(v * N + l) * TC + f];
      } else {
        ldf_to_legendre<T, DEG>(v - 5, W + 5 * N * TC + f, wl);
      }
      face_trace_smem<T, DEG>(wl, TT + s * N * QFP, TRC + (s * QF * 8 + v) * TC + f);
    }
  }
  __syncthreads();
  if (A == 0) list_hlld<T, DEG, 0>(TRC, v, f, live, fid, gamma, eps, F);
  else if (A == 1) list_hlld<T, DEG, 1>(TRC, v, f, live, fid, gamma, eps, F);
  else list_hlld<T, DEG, 2>(TRC, v, f, live, fid, gamma, eps, F);
}

template <typename T, int DEG>
__global__ void __launch_bounds__(NTP, 3) k_cell_list_pow(const OctPow<T> o, T gamma, const T* __restrict__ w,
                                                          const T* __restrict__ F, T* out, const T* w0, double ca,
                                                          double cb, float ca32, float cb32, int cmode,
                                                          const DevScalars* __restrict__ sc,
                                                          const double* __restrict__ wmean, const double* w0mean,
                                                          double* outmean) {
  // out / outmean may alias w0 / w0mean: each element is read, then written, by one thread.
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF, QC = FastDims<DEG>::QC;
  constexpr int NDIV = PowDims<DEG>::NDIV;
  constexpr int NCT = 6 + 6 * 4;  // own-side tables: 6 faces, 6 faces x 4 sub-faces
  const PowTabs<T, DEG>& pt = pow_tabs<T, DEG>();
  extern __shared__ __align__(16) unsigned char smraw[];
  T* PR = reinterpret_cast<T*>(smraw);
  T* LS = PR + QC * NSL * TC;
  T* QM = LS + NDIV * TC;
  T* CT = QM + 8 * TC;  // [NCT][QF][N] weighted own-side tables
  const int t = threadIdx.x;
  const int f = t & (TC - 1);
  const int v = t >> 5;
  const int64_t c = (int64_t)blockIdx.x * TC + f;
  const bool live = c < o.ncell;
  const int64_t S = o.stride;
  for (int i = t; i < NCT * QF * N; i += NTP) CT[i] = o.ctab[i];
  T wl[N], racc[N];
  pow_load<T, DEG>(w, S, c, live, v, f, LS, QM, wl);  // (its barrier covers CT)
  pow_volume<T, DEG>(wl, PR, gamma, v, f, racc);
  const T qv = pow_q(QM, v, f);
  // surface: the cell's face entries (6 to 24), mean-row face sums added as a
  // float pair in entry order (the two sides of a face sum the same products,
  // the coarse side scaled by 1/4, a power of two)
  T hi = T(0), lo = T(0);
  if (live) {
    const int e1 = o.cstart[c + 1];
    for (int e = o.cstart[c]; e < e1; ++e) {
      const int ent = o.centry[e];
      const int64_t fid = ent >> 1;
      const int side = ent & 1;  // 0: this cell is the face's left cell (its +a face)
      const int meta = o.fmeta[fid];
      const int a = meta & 3, kind = (meta >> 2) & 3, sub = meta >> 4;
      const int fo = side == 0 ? 2 * a + 1 : 2 * a;
      const bool coarse = (side == 0 && kind == 1) || (side == 1 && kind == 2);
      const T* Pt = CT + (coarse ? 6 + fo * 4 + sub : fo) * QF * N;
      const T* q = F + fid * QF * NFS;
      T Fp[QF];
#pragma unroll
      for (int p = 0; p < QF; ++p) Fp[p] = q[p * NFS + v];
      if (v > 0) {
#pragma unroll
        for (int p = 0; p < QF; ++p) Fp[p] = fma_rn(qv, q[p * NFS + 8 + side], Fp[p]);
      }
      T fs = T(0);
#pragma unroll
      for (int p = 0; p < QF; ++p) {
        const T Fv = side == 0 ? -Fp[p] : Fp[p];
        const T* Pw = Pt + p * N;
        fma2(fs, racc[1], Fv, Fv, Pw[0], Pw[1]);
#pragma unroll
        for (int l = 2; l + 1 < N; l += 2) fma2(racc[l], racc[l + 1], Fv, Fv, Pw[l], Pw[l + 1]);
      }
      if constexpr (sizeof(T) == 4) {
        const T s2 = __fadd_rn(hi, fs);
        const T bb = __fsub_rn(s2, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s2, bb)), __fsub_rn(fs, bb)));
        hi = s2;
      } else {
        hi += fs;
      }
    }
  }
  const double metric = live ? 2.0 / o.dxc[c] : 0.0;
  const double km = v < 5 ? metric * 0.125 : metric * (live ? pt.kL[v - 5] : 0.0);
  pow_store<T, DEG>(wl, racc, (double)hi + (double)lo, live, v, f, S, c, PR, LS, (T)metric, km, out, w0, ca, cb,
                    ca32, cb32, cmode, sc, wmean, w0mean, outmean);
}

// Stages the density and LDF rows (N + NDIV) of cell cb into XB (with BOTH)
// and of cell ca into XA, thread (v, f) rows v + 9 i; every load is issued
// before the first shared-memory store. Absent faces stage rho = 1, zeros.
template <typename T, int DEG, bool BOTH>
__device__ __forceinline__ void stage_rd(const T* __restrict__ w, int64_t S, int64_t cb, int64_t ca, bool live,
                                         int v, int f, T* XB, T* XA) {
  constexpr int N = FastDims<DEG>::N, NRD = N + PowDims<DEG>::NDIV, PER = (NRD + 8) / 9;
  T a[PER], b[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int r = v + 9 * i;
    const int64_t row = r < N ? r : 5 * N + (r - N);
    const bool ok = live && r < NRD;
    if (BOTH) b[i] = ok ? w[row * S + cb] : (r == 0 ? T(1) : T(0));
    a[i] = ok ? w[row * S + ca] : (r == 0 ? T(1) : T(0));
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int r = v + 9 * i;
    if (r < NRD) {
      if (BOTH) XB[r * TC + f] = b[i];
      XA[r * TC + f] = a[i];
    }
  }
}

// Face jumps of the normal field for the Powell timestep (eq. powell_dt):
// per face normal to each axis (right cell = this block's cell), B^n_F from
// the two traces (eq. bxface-average) at every point and the weighted
// distances to each side's own normal trace, summed over the face's points:
// jbuf[(axis * ncell + cell) * 2 + side] (side 0: the left cell). Block of 32
// cells x 4 warps: warp 0 / 1 the density traces of the left / own cells,
// warp 2 / 3 their normal-field traces (from the LDF rows), every point of
// the face per thread (compile-time table offsets; four code paths per axis).
constexpr int NTD = 4 * TC;

template <typename T, int DEG, int A>
__device__ __forceinline__ void divb_traces(const T* __restrict__ w, int64_t S, int64_t cx, bool live, int role,
                                            int f, T* TD) {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF, NDIV = PowDims<DEG>::NDIV;
  const FaceTabs<T, DEG>& tb = FastConst<T, DEG>::get().face[A];
  const PowTabs<T, DEG>& pt = pow_tabs<T, DEG>();
  T acc[QF];
#pragma unroll
  for (int p = 0; p < QF; ++p) acc[p] = T(0);
  if (role < 2) {
    // density: rows 0..N-1; left cell on its +A face (PL), own cell on its -A face (PR)
    T x[N];
    const T* pw = w + cx;
#pragma unroll
    for (int l = 0; l < N; ++l, pw += S) x[l] = live ? *pw : (l == 0 ? T(1) : T(0));
#pragma unroll
    for (int l = 0; l < N; ++l)
#pragma unroll
      for (int p = 0; p < QF; ++p) acc[p] = fma_rn(x[l], role == 0 ? tb.PL[l][p] : tb.PR[l][p], acc[p]);
  } else {
    // normal field from the LDF rows
    const T* pw = w + (int64_t)(5 * N) * S + cx;
#pragma unroll
    for (int j = 0; j < NDIV; ++j, pw += S) {
      const T x = live ? *pw : T(0);
#pragma unroll
      for (int p = 0; p < QF; ++p) acc[p] = fma_rn(x, role == 2 ? pt.Ln[A][1][j][p] : pt.Ln[A][0][j][p], acc[p]);
    }
  }
#pragma unroll
  for (int p = 0; p < QF; ++p) TD[(role * QF + p) * TC + f] = acc[p];
}

template <typename T, int DEG>
__global__ void __launch_bounds__(NTD) k_divb_face_pow(const FastGeom g, const T* __restrict__ w,
                                                       T* __restrict__ jbuf) {
  constexpr int QF = FastDims<DEG>::QF;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* TD = reinterpret_cast<T*>(smraw);  // [4][QF][TC] traces: rho L, rho R, B_n L, B_n R
  T* JS = TD + 4 * QF * TC;             // [2][QF][TC] weighted jumps per point
  const PowTabs<T, DEG>& pt = pow_tabs<T, DEG>();
  const int t = threadIdx.x;
  const int f = t & (TC - 1);
  const int role = t >> 5;  // warp-uniform
  const int64_t c = (int64_t)blockIdx.x * TC + f;
  const bool live = c < g.ncell;
  const int64_t S = g.stride;
  const Coord kc = coord_of(g, live ? c : 0);
  static_for<3>([&](auto AX) {
    constexpr int A = decltype(AX)::value;
    const int64_t cl = live ? nbr(g, kc, A, -1) : 0;
    const int64_t cx = (role & 1) ? c : cl;
    if (A > 0) __syncthreads();  // the previous axis is done with TD and JS
    if (role == 0) divb_traces<T, DEG, A>(w, S, cx, live, 0, f, TD);
    else if (role == 1) divb_traces<T, DEG, A>(w, S, cx, live, 1, f, TD);
    else if (role == 2) divb_traces<T, DEG, A>(w, S, cx, live, 2, f, TD);
    else divb_traces<T, DEG, A>(w, S, cx, live, 3, f, TD);
    __syncthreads();
    for (int i = t; i < QF * TC; i += NTD) {
      const int p = i / TC, ff = i % TC;
      const T rL = TD[(0 * QF + p) * TC + ff], rR = TD[(1 * QF + p) * TC + ff];
      const T bL = TD[(2 * QF + p) * TC + ff], bR = TD[(3 * QF + p) * TC + ff];
      const T bF = bn_face(rL, rR, bL, bR);
      const T wp = pt.wf[p];
      JS[(0 * QF + p) * TC + ff] = wp * (bF > bL ? bF - bL : bL - bF);
      JS[(1 * QF + p) * TC + ff] = wp * (bF > bR ? bF - bR : bR - bF);
    }
    __syncthreads();
    // the face's two sums over its points, in point order
    if (t < 2 * TC) {
      const int sd = t / TC, ff = t % TC;
      const int64_t cc = (int64_t)blockIdx.x * TC + ff;
      T sum = T(0);
#pragma unroll
      for (int p = 0; p < QF; ++p) sum += JS[(sd * QF + p) * TC + ff];
      if (cc < g.ncell) jbuf[((int64_t)A * g.ncell + cc) * 2 + sd] = sum;
    }
  });
}

// Face jumps of the normal field on an octree (the Powell timestep, eq.
// powell_dt), per face block of one type: the density traces through the
// type's trace tables, the normal field through the LDF functions' normal
// components on the type's (sub-)faces (ntab); each face's two sums over its
// points at jbuf[face * 2 + side].
template <typename T, int DEG>
__global__ void __launch_bounds__(NT) k_divb_list_pow(const OctPow<T> o, const T* __restrict__ w,
                                                      T* __restrict__ jbuf) {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF, NDIV = PowDims<DEG>::NDIV, NRD = N + NDIV;
  constexpr int QFP = FaceTabs<T, DEG>::QFP;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* TT = reinterpret_cast<T*>(smraw);  // [2][N][QFP] density trace tables
  T* TN = TT + 2 * N * QFP;             // [2][NDIV][QFP] normal LDF components
  T* XL = TN + 2 * NDIV * QFP;          // [NRD][TC]
  T* XR = XL + NRD * TC;                // [NRD][TC]
  T* JS = XR + NRD * TC;                // [2][QF][TC] weighted jumps per point
  const PowTabs<T, DEG>& pt = pow_tabs<T, DEG>();
  const int t = threadIdx.x;
  const int f = t & (TC - 1);
  const int v = t >> 5;
  const int bt = o.btype[blockIdx.x];
  const int type = bt & 255, cnt = bt >> 8;
  const bool live = f < cnt;
  const int64_t fid = live ? o.bface[o.bstart[blockIdx.x] + f] : 0;
  const int64_t cL = live ? o.fL[fid] : 0, cR = live ? o.fR[fid] : 0;
  const int64_t S = o.stride;
  for (int i = t; i < 2 * N * QFP; i += NT) TT[i] = o.ftab[(size_t)type * 2 * N * QFP + i];
  for (int i = t; i < 2 * NDIV * QFP; i += NT) TN[i] = o.ntab[(size_t)type * 2 * NDIV * QFP + i];
  stage_rd<T, DEG, true>(w, S, cR, cL, live, v, f, XR, XL);
  __syncthreads();
  for (int p = v; p < QF; p += 9) {
    T rL = T(0), rR = T(0), bL = T(0), bR = T(0);
#pragma unroll
    for (int l = 0; l < N; ++l) {
      rL = fma_rn(XL[l * TC + f], TT[l * QFP + p], rL);
      rR = fma_rn(XR[l * TC + f], TT[(N + l) * QFP + p], rR);
    }
#pragma unroll
    for (int j = 0; j < NDIV; ++j) {
      bL = fma_rn(XL[(N + j) * TC + f], TN[j * QFP + p], bL);
      bR = fma_rn(XR[(N + j) * TC + f], TN[(NDIV + j) * QFP + p], bR);
    }
    const T bF = bn_face(rL, rR, bL, bR);
    const T wp = pt.wf[p];
    JS[(0 * QF + p) * TC + f] = wp * (bF > bL ? bF - bL : bL - bF);
    JS[(1 * QF + p) * TC + f] = wp * (bF > bR ? bF - bR : bR - bF);
  }
  __syncthreads();
  if (t < 2 * TC) {
    const int sd = t / TC, ff = t % TC;
    T sum = T(0);
#pragma unroll
    for (int p = 0; p < QF; ++p) sum += JS[(sd * QF + p) * TC + ff];
    if (ff < cnt) jbuf[(int64_t)o.bface[o.bstart[blockIdx.x] + ff] * 2 + sd] = sum;
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
  static bool attr3 = false;
  if (!attr3) {
    set_smem_attr<T>((const void*)k_face_glm3<T, DEG>, sm);
    attr3 = true;
  }
  k_face_glm3<T, DEG><<<nb, NT, sm, st>>>(tabs.face[0], tabs.face[1], tabs.face[2], g, w, F, sc, (T)eps);
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
  // cmode: 0 plain rhs, 1 SSP combination with ca == 0, 2 with ca != 0
  const int cmode = combine ? (ca != 0.0 ? 2 : 1) : 0;
  k_cell_glm<T, DEG><<<nb, NT, sm, st>>>(tabs.cell, g, w, F, out, w0, ca, cb, (float)ca, (float)cb, cmode, sc,
                                         wmean, w0mean, outmean);
}

template <typename T, int DEG>
size_t pow_face_smem() {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF, NRP = 5 * N + PowDims<DEG>::NDIV;
  return (size_t)(2 * NRP * TC + 3 * N * TC + 2 * QF * 8 * TC) * sizeof(T);
}

template <typename T, int DEG>
size_t pow_cell_smem() {
  return (size_t)(FastDims<DEG>::QC * NSL * TC + PowDims<DEG>::NDIV * TC + 8 * TC) * sizeof(T);
}

template <typename T, int DEG>
void launch_face_pow(const FastAll<T, DEG>&, const FastGeom& g, const T* w, T* F, double eps, cudaStream_t st) {
  const unsigned nb = (unsigned)((g.ncell + TC - 1) / TC);
  const size_t sm = pow_face_smem<T, DEG>();
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_face_pow3<T, DEG>, sm);
    attr = true;
  }
  k_face_pow3<T, DEG><<<nb, NT, sm, st>>>(g, w, F, (T)eps);
}

template <typename T, int DEG>
void launch_cell_pow(const FastAll<T, DEG>&, const FastGeom& g, const T* w, const T* F, T* out, const T* w0,
                     double ca, double cb, int combine, const DevScalars* sc, const double* wmean,
                     const double* w0mean, double* outmean, cudaStream_t st) {
  const unsigned nb = (unsigned)((g.ncell + TC - 1) / TC);
  const size_t sm = pow_cell_smem<T, DEG>();
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_cell_pow<T, DEG>, sm);
    attr = true;
  }
  const int cmode = combine ? (ca != 0.0 ? 2 : 1) : 0;
  k_cell_pow<T, DEG><<<nb, NTP, sm, st>>>(g, w, F, out, w0, ca, cb, (float)ca, (float)cb, cmode, sc, wmean, w0mean,
                                          outmean);
}

template <typename T, int DEG>
void launch_divb_face_pow(const FastGeom& g, const T* w, T* jbuf, cudaStream_t st) {
  const unsigned nb = (unsigned)((g.ncell + TC - 1) / TC);
  const size_t sm = (size_t)6 * FastDims<DEG>::QF * TC * sizeof(T);
  k_divb_face_pow<T, DEG><<<nb, NTD, sm, st>>>(g, w, jbuf);
}

template <typename T, int DEG>
void launch_face_list_pow(const OctPow<T>& o, double gamma, const T* w, T* F, double eps, cudaStream_t st) {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF;
  constexpr int NDIV = PowDims<DEG>::NDIV, NRP = 5 * N + NDIV, QFP = FaceTabs<T, DEG>::QFP;
  const size_t smf = (size_t)(2 * N * QFP + 2 * NRP * TC + 2 * QF * 8 * TC) * sizeof(T);
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_face_list_pow<T, DEG>, smf);
    attr = true;
  }
  if (o.nblk > 0) k_face_list_pow<T, DEG><<<(unsigned)o.nblk, NT, smf, st>>>(o, (T)gamma, (T)eps, w, F);
}

template <typename T, int DEG>
void launch_cell_list_pow(const OctPow<T>& o, double gamma, const T* w, const T* F, T* out, const T* w0, double ca,
                          double cb, int combine, const DevScalars* sc, const double* wmean, const double* w0mean,
                          double* outmean, cudaStream_t st) {
  constexpr int N = FastDims<DEG>::N, QF = FastDims<DEG>::QF, QC = FastDims<DEG>::QC;
  constexpr int NDIV = PowDims<DEG>::NDIV;
  const size_t smc = (size_t)(QC * NSL * TC + NDIV * TC + 8 * TC + 30 * QF * N) * sizeof(T);
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_cell_list_pow<T, DEG>, smc);
    attr = true;
  }
  const int cmode = combine ? (ca != 0.0 ? 2 : 1) : 0;
  const unsigned nb = (unsigned)((o.ncell + TC - 1) / TC);
  k_cell_list_pow<T, DEG><<<nb, NTP, smc, st>>>(o, (T)gamma, w, F, out, w0, ca, cb, (float)ca, (float)cb, cmode, sc,
                                                wmean, w0mean, outmean);
}

template <typename T, int DEG>
void launch_divb_list_pow(const OctPow<T>& o, const T* w, T* jbuf, cudaStream_t st) {
  constexpr int N = FastDims<DEG>::N, NDIV = PowDims<DEG>::NDIV, QFP = FaceTabs<T, DEG>::QFP;
  const size_t sm = (size_t)(2 * N * QFP + 2 * NDIV * QFP + 2 * (N + NDIV) * TC + 2 * FastDims<DEG>::QF * TC) *
                    sizeof(T);
  if (o.nblk > 0) k_divb_list_pow<T, DEG><<<(unsigned)o.nblk, NT, sm, st>>>(o, w, jbuf);
}

template <typename T, int DEG>
int fast_to_constant(const FastAll<T, DEG>& tabs) {
  if constexpr (FastConst<T, DEG>::on) return FastConst<T, DEG>::upload(tabs) == cudaSuccess ? 0 : -3;
  return 0;
}

#define INSTF(T, DEG)                                                                                         \
  template void launch_face_glm<T, DEG>(const FastAll<T, DEG>&, const FastGeom&, const T*, T*,              \
                                        const DevScalars*, double, cudaStream_t);                          \
  template void launch_cell_glm<T, DEG>(const FastAll<T, DEG>&, const FastGeom&, const T*, const T*, T*,    \
                                        const T*, double, double, int, const DevScalars*, const double*,    \
                                        const double*, double*, cudaStream_t);          \
  template int fast_to_constant<T, DEG>(const FastAll<T, DEG>&);
// the Powell kernels for degrees 1 and 2
#define INSTP(T, DEG)                                                                                         \
  template void launch_face_pow<T, DEG>(const FastAll<T, DEG>&, const FastGeom&, const T*, T*, double,        \
                                        cudaStream_t);                                                        \
  template void launch_cell_pow<T, DEG>(const FastAll<T, DEG>&, const FastGeom&, const T*, const T*, T*,    \
                                        const T*, double, double, int, const DevScalars*, const double*,    \
                                        const double*, double*, cudaStream_t);                              \
  template void launch_divb_face_pow<T, DEG>(const FastGeom&, const T*, T*, cudaStream_t);                    \
  template void launch_face_list_pow<T, DEG>(const OctPow<T>&, double, const T*, T*, double, cudaStream_t);   \
  template void launch_cell_list_pow<T, DEG>(const OctPow<T>&, double, const T*, const T*, T*, const T*, double, \
                                             double, int, const DevScalars*, const double*, const double*,      \
                                             double*, cudaStream_t);                                           \
  template void launch_divb_list_pow<T, DEG>(const OctPow<T>&, const T*, T*, cudaStream_t);
INSTF(DG_FAST_T, DG_FAST_DEG)
#if DG_FAST_DEG <= 2
INSTP(DG_FAST_T, DG_FAST_DEG)
#endif

}  // namespace dgmhd
