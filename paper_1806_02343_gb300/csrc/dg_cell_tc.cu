// Cell update of the DG operator (Sec. 3.5 eq. wdot) for the GLM scheme
// (Sec. 4.1.5) on uniform 3D meshes, degree 2, FP32 form: the three
// contractions of the cell -- the projection of the modal weights to the 27
// volume Gauss points (eq. u-exp), the volume integral of f_a d_a phi_l and the
// surface integral of F* phi_l over the six faces -- run on the tensor core as
// 3xTF32 products with FP32 accumulation in tensor memory; the pointwise
// physics (primitives, the volume flux), the cell-mean row and the SSP
// combination stay on the CUDA cores.
//
// Selected with generic_kernels = 2; the default cell update keeps the
// contractions on the CUDA cores (k_cell_glm, packed FP32 FMAs), which is
// faster on GB300: a kind::tf32 MMA with M = 128 occupies the tensor core for
// about 106 cycles (independent accumulators) to 235 cycles (one dependent
// chain) whatever N up to 64 and wherever A lives, i.e. 154 FP32 FMA per cycle
// and SM at N = 16 against 256 for packed FMAs on the CUDA cores -- and the
// 3xTF32 split needs three products. The contractions of a degree-2 cell
// (N = 10 modes or 27 points) cannot amortise that cost (39.7 ms per stage at
// 256^3 here against 14.5 ms). The tensor core's FP32 accumulation also
// loses more than FMA chains: 2.3e-4 of the largest operator value at 256^3
// against 2.6e-5.
//
// Organisation (one persistent block of 288 threads per half SM):
// * thread t = 32 v + c owns variable v of cell c of a 32-cell tile (a warp
//   holds one variable of 32 consecutive cells: coalesced row loads);
// * MMA rows are the (variable, cell) pairs: row 32 v + c lies in M-tile v / 4
//   (three M = 128 tiles, the third holding psi only), tensor-memory lane
//   32 (v % 4) + c -- the lanes warp v may access;
// * per M-tile 80 tensor-memory columns: [0, 16) the accumulator (modes), [16,
//   80) scratch for the A operands (hi and lo parts) written by tcgen05.st and
//   for the projection's output;
// * the tables (TF32 hi/lo, K-major core matrices) are fetched once per block
//   by one bulk asynchronous copy into shared memory;
// * seven MMA batches per tile (projection, three volume chunks of 9 points,
//   three face axes), each issued by one thread and committed to an mbarrier;
//   every wait is bounded (about one second), after which the block records
//   status bit 8 (DG_E_TIMEOUT) and stops.
//
// The F* buffer is the one written by k_face_glm3 ([axis][point][var][cell]).
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <algorithm>
#include <cstring>

#include "dg_cell_tc.cuh"
#include "dg_phys.cuh"
#include "dg_tc.cuh"

namespace dgmhd {

namespace {

constexpr int TC = 32;         // cells per tile
constexpr int NT = 9 * TC;     // threads per block
constexpr int NM = 10;         // modes (degree 2)
constexpr int QV = 27;         // volume points
constexpr int QF = 9;          // points per face
constexpr int ACC = 0;         // accumulator columns of an M-tile
constexpr int SCR = 16;        // first scratch column of an M-tile
constexpr int MTC = 80;        // columns per M-tile
constexpr uint32_t TMEM_COLS = 256;
constexpr long long kWaitCycles = 2000000000ll;  // about one second at GB300 clocks
constexpr int PR_FLOATS = QV * 16 * TC;          // per-point primitive slots
constexpr size_t SMEM_BYTES = (size_t)TcLayout::TOTAL * 4 + (size_t)PR_FLOATS * 4 + 64;

// primitive slots per volume point (as in k_cell_glm)
enum { SL_RHO = 0, SL_B = 5, SL_PSI = 8, SL_V = 9, SL_PT = 12, SL_VB = 13, SL_EPT = 14, SL_ZERO = 15, NSL = 16 };

struct TcScal {
  float minv[NM];  // 1 / M_l
  float wf[QF];    // face weights (mode-0 face values times the weights)
};

struct Coord3 {
  int ix, iy, iz;
};
__device__ __forceinline__ Coord3 coord3(const FastGeom& g, int64_t c) {
  const unsigned cc = (unsigned)c, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
  const unsigned r = cc / nx;
  return Coord3{(int)(cc - r * nx), (int)(r % ny), (int)(r / ny)};
}
// periodic neighbour along +a
__device__ __forceinline__ int64_t nbr_plus(const FastGeom& g, Coord3 k, int a) {
  if (a == 0) k.ix = k.ix + 1 == g.nx ? 0 : k.ix + 1;
  else if (a == 1) k.iy = k.iy + 1 == g.ny ? 0 : k.iy + 1;
  else k.iz = k.iz + 1 == g.nz ? 0 : k.iz + 1;
  return ((int64_t)k.iz * g.ny + k.iy) * g.nx + k.ix;
}

// hi / lo words of the 3xTF32 split of x: hi = tf32(x), lo = tf32(x - hi),
// both rounded to nearest (the tensor core would truncate the low bits of a
// wider lo, a bias that accumulates over the sums), |x - hi - lo| <= 2^-24 |x|
__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo) {
  const float h = tc::tf32_rna(x);
  hi = __float_as_uint(h);
  lo = __float_as_uint(tc::tf32_rna(x - h));
}

__global__ void __launch_bounds__(NT, 2)
    k_cell_tc(const float* __restrict__ tabs, TcScal ts, FastGeom g, const float* __restrict__ w,
              const float* __restrict__ F, float* out, const float* w0, double ca, double cb, float ca32, float cb32,
              int cmode, DevScalars* __restrict__ sc, const double* __restrict__ wmean, const double* w0mean,
              double* outmean) {
  // out / outmean may alias w0 / w0mean: each element is read, then written, by one thread.
  extern __shared__ __align__(128) unsigned char smraw[];
  float* tb = reinterpret_cast<float*>(smraw);          // TcLayout tables
  float* PR = tb + TcLayout::TOTAL;                     // [27][16][32]
  uint64_t* bar = reinterpret_cast<uint64_t*>(PR + PR_FLOATS);  // [0] tables, [1] MMA commits
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);

  const int t = threadIdx.x, v = t >> 5, lane = t & 31;
  if (t == 0) {
    tc::mbar_init(bar, 1);
    tc::mbar_init(bar + 1, 1);
    tc::mbar_fence_init();
  }
  if (v == 0) tc::tmem_alloc(tslot, TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = *tslot;
  if (t == 0) {
    tc::mbar_expect_tx(bar, (unsigned)(TcLayout::TOTAL * 4));
    tc::bulk_g2s(tb, tabs, (unsigned)(TcLayout::TOTAL * 4), bar);
  }
  // every thread waits (bounded); the block agrees on the outcome
  auto wait_all = [&](uint64_t* b, unsigned parity) {
    const bool ok = tc::mbar_wait_bounded(b, parity, kWaitCycles);
    return __syncthreads_and(ok) != 0;
  };
  bool tabs_pending = true;
  int mma_pending = -1;  // parity of a commit not yet observed, else -1
  unsigned mph = 0;      // commits observed on bar[1]
  const int64_t S = g.stride;
  const int mt = v >> 2;
  const uint32_t trow = tm + ((uint32_t)(32 * (v & 3)) << 16) + (uint32_t)(mt * MTC);  // this thread's row
  const float gamma = g.gamma32;
  const float ch = sc->ch32;

  // flux of variable v: f_a = alpha v_a + beta B_a + (a == gax ? gamma_v : 0)
  int aidx, bidx, gidx, gax;
  float bs, bconst;
  if (v == 0) { aidx = SL_RHO; bidx = SL_ZERO; bs = 0.f; bconst = 0.f; gidx = SL_ZERO; gax = -1; }
  else if (v <= 3) { aidx = v; bidx = SL_B + v - 1; bs = -1.f; bconst = 0.f; gidx = SL_PT; gax = v - 1; }
  else if (v == 4) { aidx = SL_EPT; bidx = SL_VB; bs = -1.f; bconst = 0.f; gidx = SL_ZERO; gax = -1; }
  else if (v <= 7) { aidx = v; bidx = SL_V + v - 5; bs = -1.f; bconst = 0.f; gidx = SL_PSI; gax = v - 5; }
  else { aidx = SL_ZERO; bidx = SL_ZERO; bs = 0.f; bconst = ch * ch; gidx = SL_ZERO; gax = -1; }

  const uint32_t IDP = tc::idesc_tf32_f32(128, 32);  // projection: N = 32 points
  const uint32_t IDA = tc::idesc_tf32_f32(128, 16);  // integrals: N = 16 modes
  // one elected thread issues a batch: for each M-tile, per K-step of 8 the
  // three products hi*hi + hi*lo + lo*hi
  auto issue = [&](uint32_t dcol, int ksteps, const float* bh, const float* bl, uint32_t sbo, uint32_t idesc,
                   bool first) {
    tc::fence_after_sync();
#pragma unroll 1
    for (int m = 0; m < 3; ++m) {
      const uint32_t base = tm + (uint32_t)(m * MTC);
#pragma unroll 1
      for (int ks = 0; ks < ksteps; ++ks) {
        const uint64_t dh = tc::smem_desc(tc::smem_u32(bh + ks * 64), 128, sbo);
        const uint64_t dl = tc::smem_desc(tc::smem_u32(bl + ks * 64), 128, sbo);
        const uint32_t ah = base + SCR + 8 * ks, al = base + SCR + 32 + 8 * ks;
        tc::mma_tf32_ts(base + dcol, ah, dh, idesc, !(first && ks == 0));
        tc::mma_tf32_ts(base + dcol, ah, dl, idesc, true);
        tc::mma_tf32_ts(base + dcol, al, dh, idesc, true);
      }
    }
    tc::commit(bar + 1);
  };
  // the previous batch's completion (its A operands may then be overwritten)
  auto wait_mma = [&]() {
    const bool ok = wait_all(bar + 1, mph & 1u);
    if (ok) {
      ++mph;
      mma_pending = -1;
      tc::fence_after_sync();
    }
    return ok;
  };
  // operands written by every thread become visible to the issuing thread
  auto publish = [&]() {
    tc::st_wait();
    tc::fence_before_sync();
    __syncthreads();
  };

  if (!wait_all(bar, 0)) {
    if (t == 0) atomicOr(&sc->status, 8);
  } else {
    tabs_pending = false;
    const int64_t ntile = (g.ncell + TC - 1) / TC;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
      const int64_t c = tile * TC + lane;
      const bool live = c < g.ncell;
      // ---- modal weights of (v, c); dead cells get a physical dummy state
      float wl[NM];
      {
        const float* pw = w + (int64_t)(v * NM) * S + c;
#pragma unroll
        for (int l = 0; l < NM; ++l, pw += S) wl[l] = live ? *pw : ((v == 0 || v == 4) && l == 0 ? 1.f : 0.f);
      }
      {
        uint32_t a[32];
#pragma unroll
        for (int l = 0; l < 16; ++l) {
          if (l < NM) split(wl[l], a[l], a[16 + l]);
          else a[l] = a[16 + l] = 0u;
        }
        tc::st32(trow + SCR, a);  // hi in SCR .. SCR+15, lo in SCR+16 .. SCR+31
      }
      publish();
      // ---- projection to the volume points: D[(v,c)][q] in columns SCR+32 ..
      if (t == 0) {
        // K = 16 modes: the hi part at SCR + 8 ks, the lo part 16 further
        tc::fence_after_sync();
#pragma unroll 1
        for (int m = 0; m < 3; ++m) {
          const uint32_t base = tm + (uint32_t)(m * MTC);
#pragma unroll 1
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t dh = tc::smem_desc(tc::smem_u32(tb + TcLayout::OFF_PH + ks * 64), 128, 512);
            const uint64_t dl = tc::smem_desc(tc::smem_u32(tb + TcLayout::OFF_PL + ks * 64), 128, 512);
            const uint32_t ah = base + SCR + 8 * ks, al = base + SCR + 16 + 8 * ks;
            tc::mma_tf32_ts(base + SCR + 32, ah, dh, IDP, ks > 0);
            tc::mma_tf32_ts(base + SCR + 32, ah, dl, IDP, true);
            tc::mma_tf32_ts(base + SCR + 32, al, dh, IDP, true);
          }
        }
        tc::commit(bar + 1);
      }
      mma_pending = (int)(mph & 1u);
      if (!wait_mma()) break;
      {
        float u[32];
        tc::ld32(trow + SCR + 32, u);
#pragma unroll
        for (int q = 0; q < QV; ++q) PR[(q * NSL + v) * TC + lane] = u[q];
      }
      tc::fence_before_sync();
      __syncthreads();
      // ---- primitives per point
      for (int idx = t; idx < QV * TC; idx += NT) {
        const int q = idx >> 5, ff = idx & 31;
        float* pr = PR + q * NSL * TC + ff;
        const float rho = pr[0], ir = rcp(rho);
        const float vx = pr[1 * TC] * ir, vy = pr[2 * TC] * ir, vz = pr[3 * TC] * ir;
        const float bx = pr[5 * TC], by = pr[6 * TC], bz = pr[7 * TC];
        const float b2 = bx * bx + by * by + bz * bz;
        const float E = pr[4 * TC];
        const float p = (gamma - 1.f) * (E - 0.5f * rho * (vx * vx + vy * vy + vz * vz) - 0.5f * b2);
        const float pT = p + 0.5f * b2;
        pr[SL_V * TC] = vx;
        pr[(SL_V + 1) * TC] = vy;
        pr[(SL_V + 2) * TC] = vz;
        pr[SL_PT * TC] = pT;
        pr[SL_VB * TC] = vx * bx + vy * by + vz * bz;
        pr[SL_EPT * TC] = E + pT;
        pr[SL_ZERO * TC] = 0.f;
      }
      __syncthreads();
      // ---- volume integral: three chunks of 9 points, K = (axis, point) -> 32
      bool ok = true;
#pragma unroll 1
      for (int j = 0; j < 3; ++j) {
        uint32_t a[64];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const float* pr = PR + (9 * j + i) * NSL * TC + lane;
          const float al = pr[aidx * TC];
          const float be = bs * pr[bidx * TC] + bconst;
          const float ga = pr[gidx * TC];
          float fa[3];
#pragma unroll
          for (int ax = 0; ax < 3; ++ax)
            fa[ax] = fmaf(al, pr[(SL_V + ax) * TC], fmaf(be, pr[(SL_B + ax) * TC], gax == ax ? ga : 0.f));
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) split(fa[ax], a[9 * ax + i], a[32 + 9 * ax + i]);
        }
#pragma unroll
        for (int k = 27; k < 32; ++k) a[k] = a[32 + k] = 0u;
        if (j > 0 && !(ok = wait_mma())) break;
        tc::st32(trow + SCR, a);
        tc::st32(trow + SCR + 32, a + 32);
        publish();
        if (t == 0)
          issue(ACC, 4, tb + TcLayout::OFF_GH + j * TcLayout::G, tb + TcLayout::OFF_GL + j * TcLayout::G, 1024, IDA,
                j == 0);
        mma_pending = (int)(mph & 1u);
      }
      if (!ok) break;
      // ---- surface integral, one face axis at a time; the mean row's face
      // sums on the CUDA cores (the same products and order in both cells of a
      // face: the two contributions cancel exactly)
      // the six face sums in the order (x-, x+, y-, y+, z-, z+), added as an
      // unevaluated float pair (Knuth's TwoSum: s + e equals a + b exactly)
      float mhi = 0.f, mlo = 0.f;
      const Coord3 kc = coord3(g, live ? c : 0);
#pragma unroll 1
      for (int ax = 0; ax < 3; ++ax) {
        uint32_t a[64];
        const int64_t S9 = 9 * S;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int64_t fc = s ? nbr_plus(g, kc, ax) : c;
          const float* q = F + (int64_t)v * S + (int64_t)(ax * QF) * S9 + fc;
          float fs = 0.f;
#pragma unroll
          for (int p = 0; p < QF; ++p, q += S9) {
            const float Fr = live ? *q : 0.f;
            const float Fv = s ? -Fr : Fr;
            fs = __fmaf_rn(Fv, ts.wf[p], fs);
            split(Fr, a[9 * s + p], a[32 + 9 * s + p]);  // the table carries the side's sign
          }
          if (ax == 0 && s == 0) {
            mhi = fs;
          } else {
            const float s2 = __fadd_rn(mhi, fs);
            const float bb = __fsub_rn(s2, mhi);
            const float e = __fadd_rn(__fsub_rn(mhi, __fsub_rn(s2, bb)), __fsub_rn(fs, bb));
            mhi = s2;
            mlo = __fadd_rn(mlo, e);
          }
        }
#pragma unroll
        for (int k = 18; k < 32; ++k) a[k] = a[32 + k] = 0u;
        if (!(ok = wait_mma())) break;
        tc::st32(trow + SCR, a);
        tc::st32(trow + SCR + 32, a + 32);
        publish();
        if (t == 0)
          issue(ACC, 3, tb + TcLayout::OFF_SH + ax * TcLayout::S, tb + TcLayout::OFF_SL + ax * TcLayout::S, 768, IDA,
                false);
        mma_pending = (int)(mph & 1u);
      }
      if (!ok) break;
      if (!wait_mma()) break;
      float racc[16];
      tc::ld16(trow + ACC, racc);
      tc::fence_before_sync();
      if (live) {
        // ---- mode 0 (cell mean): the float pair of the face sums enters the
        // FP64 mean through one conversion
        const int64_t i0 = (int64_t)(v * NM) * S + c;
        const double tot = (double)mhi + (double)mlo;
        const double wz = wmean[(int64_t)v * S + c];
        if (cmode == 0) {
          double rhs = g.kmean * tot;
          if (v == 8) rhs = fma(-sc->kappa, wz, rhs);
          out[i0] = (float)rhs;
          outmean[(int64_t)v * S + c] = rhs;
        } else {
          const double kd = cb * sc->dt;
          double base = cb * wz;
          if (cmode == 2) base = fma(ca, w0mean[(int64_t)v * S + c], base);
          if (v == 8) base = fma(-kd * sc->kappa, wz, base);
          const double o = fma(kd * g.kmean, tot, base);
          outmean[(int64_t)v * S + c] = o;
          out[i0] = (float)o;
        }
        // ---- modes 1 .. 9
        const float tmet = g.metric32, tdt = sc->dt32, tk = sc->kappa32;
        float* po = out + i0 + S;
        const float* p0 = cmode == 0 ? nullptr : w0 + i0 + S;
#pragma unroll
        for (int l = 1; l < NM; ++l, po += S) {
          float rhs = tmet * ts.minv[l] * racc[l];
          if (v == 8) rhs -= tk * wl[l];
          if (cmode == 0) {
            *po = rhs;
          } else {
            *po = ca32 * *p0 + cb32 * (wl[l] + tdt * rhs);
            p0 += S;
          }
        }
      }
    }
    if (mma_pending >= 0) {
      // a timed-out batch: record it, wait once more (bounded) before the
      // columns are freed
      if (t == 0) atomicOr(&sc->status, 8);
      tc::mbar_wait_bounded(bar + 1, (unsigned)mma_pending, kWaitCycles);
    }
  }
  if (tabs_pending) tc::mbar_wait_bounded(bar, 0, kWaitCycles);
  tc::fence_before_sync();
  __syncthreads();
  if (v == 0) tc::tmem_dealloc(tm, TMEM_COLS);
}

float tf32_round_host(double x) {
  // nearest TF32 (10 explicit mantissa bits) of the float nearest x
  float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return f;  // inf / nan unchanged
  u = (u + 0x1000u) & 0xffffe000u;
  std::memcpy(&f, &u, 4);
  return f;
}

}  // namespace

void build_tc_tables(const std::vector<double>& Pv, const std::vector<double>& dPv, const std::vector<double>& Pf,
                     const std::vector<double>& wv, const std::vector<double>& wf, std::vector<float>& out) {
  out.assign(TcLayout::TOTAL, 0.f);
  auto put = [&](int off_hi, int off_lo, int n, int k, int K, double val) {
    const float h = tf32_round_host(val);
    out[off_hi + tc_kidx(n, k, K)] = h;
    out[off_lo + tc_kidx(n, k, K)] = tf32_round_host(val - (double)h);
  };
  for (int q = 0; q < QV; ++q)
    for (int l = 0; l < NM; ++l) put(TcLayout::OFF_PH, TcLayout::OFF_PL, q, l, 16, Pv[(size_t)l * QV + q]);
  for (int j = 0; j < 3; ++j)
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < 9; ++i) {
        const int q = 9 * j + i;
        for (int l = 1; l < NM; ++l)
          put(TcLayout::OFF_GH + j * TcLayout::G, TcLayout::OFF_GL + j * TcLayout::G, l, 9 * a + i, 32,
              dPv[((size_t)a * NM + l) * QV + q] * wv[q]);
      }
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s)
      for (int p = 0; p < QF; ++p)
        for (int l = 1; l < NM; ++l)
          put(TcLayout::OFF_SH + a * TcLayout::S, TcLayout::OFF_SL + a * TcLayout::S, l, 9 * s + p, 24,
              (s ? -1.0 : 1.0) * Pf[((size_t)(2 * a + s) * NM + l) * QF + p] * wf[p]);
}

int launch_cell_tc(const float* tabs, const FastAll<float, 2>& ft, const FastGeom& g, const float* w, const float* F,
                   float* out, const float* w0, double ca, double cb, int combine, const DevScalars* sc,
                   const double* wmean, const double* w0mean, double* outmean, int nsm, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_cell_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES) != cudaSuccess)
      return -3;
    attr = true;
  }
  TcScal ts;
  for (int l = 0; l < NM; ++l) ts.minv[l] = ft.cell.minv[l];
  for (int p = 0; p < QF; ++p) ts.wf[p] = ft.cell.Pfw[0][p][0];
  const int64_t ntile = (g.ncell + TC - 1) / TC;
  // two resident blocks per SM: 2 x 256 tensor-memory columns fill the SM's 512
  const unsigned nb = (unsigned)std::min<int64_t>(ntile, (int64_t)2 * nsm);
  const int cmode = combine ? (ca != 0.0 ? 2 : 1) : 0;
  k_cell_tc<<<nb, NT, SMEM_BYTES, st>>>(tabs, ts, g, w, F, out, w0, ca, cb, (float)ca, (float)cb, cmode,
                                        const_cast<DevScalars*>(sc), wmean, w0mean, outmean);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace dgmhd
