// Learned troubled-cell indicator: features, BF16 tensor-core inference fused
// with the feature pass, and FP32 training kernels (forward, backward, Adam).
//
// Detection is its own step of the limiter (Sec. 4.2: first detect troubled
// cells, then limit them); this network replaces the TVB detection and only the
// cells it flags go through the characteristic TVB procedure.
//
// Features of a cell (nin = 8 n(d) + 10 D): Legendre coefficients of the 8 MHD
// variables (LDF B mapped exactly to per-component Legendre coefficients), each
// variable divided by s_v = |mean_v| + max_nb |mean_nb,v - mean_v| + 1e-12,
// then rho_nb / rho - 1 for the neighbours -x, +x, -y, +y (, -z, +z), then the
// degree-1 coefficient of each variable along each direction over M~ dx.
// Network: nin -> 64 -> 64 -> 1, ReLU, sigmoid. Weights (flat FP32):
// W1[64][nin], b1[64], W2[64][64], b2[64], w3[64], b3.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "dg_mlp.cuh"
#include "dg_pos.cuh"
#include "dg_tc.cuh"

namespace dgmhd {

namespace {

constexpr int HID = 64;

// periodic face neighbour on the uniform mesh (cell counts stay below 2^31,
// so the index arithmetic is 32-bit)
__device__ __forceinline__ int64_t nbc(const Geom& g, int64_t c, int a, int dir) {
  const unsigned cc = (unsigned)c, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
  const unsigned r = cc / nx;
  int ix = (int)(cc - r * nx), iy = (int)(r % ny), iz = (int)(r / ny);
  if (a == 0) { ix += dir; ix = ix < 0 ? ix + g.nx : (ix >= g.nx ? ix - g.nx : ix); }
  else if (a == 1) { iy += dir; iy = iy < 0 ? iy + g.ny : (iy >= g.ny ? iy - g.ny : iy); }
  else { iz += dir; iz = iz < 0 ? iz + g.nz : (iz >= g.nz ? iz - g.nz : iz); }
  return ((int64_t)iz * g.ny + iy) * g.nx + ix;
}

__device__ __forceinline__ int mrow(const Geom& g, int m) {
  if (g.glm) return m * g.n;
  if (m < 5) return m * g.n;
  if (g.D == 3) return g.ldf0 + (m - 5);
  return m < 7 ? g.ldf0 + (m - 5) : g.bz2d;
}

// Discretisation sizes seen by the feature code: RtDims reads them from the
// Geom at run time; CtDims<GLM, DEG> fixes them at compile time (3D), so the
// loops over variables and modes unroll and every row index is a constant.
struct RtDims {
  const Geom& g;
  const MlpTabs& mt;
  __device__ int n() const { return g.n; }
  __device__ bool glm() const { return g.glm != 0; }
  __device__ int D() const { return g.D; }
  __device__ int ldf0() const { return g.ldf0; }
  __device__ int ndiv() const { return g.ndiv; }
  __device__ int bz2d() const { return g.bz2d; }
  __device__ int deg1(int a) const { return mt.deg1[a]; }
  __device__ int mrow(int k) const { return dgmhd::mrow(g, k); }
};

template <bool GLM, int DEG>
struct CtDims {
  static constexpr int N = (DEG + 1) * (DEG + 2) * (DEG + 3) / 6;
  // LDF basis size in 3D (Table A1): 3, 11, 26, 50 for degrees 0..3
  static constexpr int NDIV = DEG == 0 ? 3 : DEG == 1 ? 11 : DEG == 2 ? 26 : 50;
  __device__ static constexpr int n() { return N; }
  __device__ static constexpr bool glm() { return GLM; }
  __device__ static constexpr int D() { return 3; }
  __device__ static constexpr int ldf0() { return GLM ? -1 : 5 * N; }
  __device__ static constexpr int ndiv() { return GLM ? 0 : NDIV; }
  __device__ static constexpr int bz2d() { return -1; }
  // degree-1 modes in the basis order: (1,0,0), (0,1,0), (0,0,1)
  __device__ static constexpr int deg1(int a) { return 1 + a; }
  __device__ static constexpr int mrow(int k) { return (GLM || k < 5) ? k * N : 5 * N + (k - 5); }
};

// physical cell means of the 8 MHD variables from the raw mean rows
template <typename Dm>
__device__ __forceinline__ void phys_means(const Dm& dm, const MlpTabs& mt, const float* raw, float* m) {
#pragma unroll
  for (int k = 0; k < 5; ++k) m[k] = raw[k];
  if (dm.glm()) {
#pragma unroll
    for (int k = 5; k < 8; ++k) m[k] = raw[k];
  } else {
    m[5] = m[6] = m[7] = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc)
        if (j < dm.D() && cc < dm.D()) m[5 + cc] += raw[5 + j] * mt.l2l[(j * 3 + cc) * MLP_MAXN + 0];
    if (dm.D() == 2) m[7] = raw[7];
  }
}

// State of one cell and of its face neighbours read straight from the state
// rows (FP32 form: the float mode-0 rows mirror the FP64 means exactly).
template <typename T>
struct GlobalSrc {
  const Geom& g;
  const T* w;
  int64_t c;
  __device__ float row(int r) const { return (float)w[(int64_t)r * g.stride + c]; }
  __device__ void nbraw(int a, int s, float* raw) const {
    const int64_t cn = nbc(g, c, a, s ? 1 : -1);
    for (int k = 0; k < 8; ++k) raw[k] = (float)w[(int64_t)mrow(g, k) * g.stride + cn];
  }
  __device__ float imdx(const MlpTabs& mt) const { return mt.inv_mdx; }
};

// Octree meshes (the per-side leaf lists of the context): the neighbour mean on side
// (a, s) is the average of the leaves across that side (one of the same level
// or coarser, or the 2^(D-1) finer ones), as the octree TVB procedure reads
// it; the slope scale is the leaf's own M~ dx_K. A side without a leaf (the
// edge of a partition's local mesh) reads the cell's own means.
struct AmrFeat {
  const int32_t* side_nb;    // the leaves across each side, in face-entry order (AmrHost::side_nb)
  const uint8_t* side_info;  // count | relation << 4 per leaf and side
  const double* dxc;
  double dxmin;  // the mesh's smallest cell (the one inv_mdx was made with)
  int on;
};

template <typename T>
struct AmrSrc {
  const Geom& g;
  const T* w;
  int64_t c;
  const AmrFeat& af;
  __device__ float row(int r) const { return (float)w[(int64_t)r * g.stride + c]; }
  __device__ void nbraw(int a, int s, float* raw) const {
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int sidx = 2 * a + (s ? 1 : 0);
    const int cnt = af.side_info[c * 6 + sidx] & 15;
    for (int k2 = 0; k2 < cnt; ++k2) {
      const int64_t cn = af.side_nb[c * 24 + sidx * 4 + k2];
      for (int k = 0; k < 8; ++k) acc[k] += (float)w[(int64_t)mrow(g, k) * g.stride + cn];
    }
    if (cnt == 0) {
      for (int k = 0; k < 8; ++k) raw[k] = (float)w[(int64_t)mrow(g, k) * g.stride + c];
      return;
    }
    const float inv = 1.f / (float)cnt;  // 1 or 2^(D-1): exact
    for (int k = 0; k < 8; ++k) raw[k] = acc[k] * inv;
  }
  __device__ float imdx(const MlpTabs& mt) const { return mt.inv_mdx * (float)(af.dxmin / af.dxc[c]); }
};

// features of one cell, written through put(k, value) for k in [0, nin)
// part < 0: every feature; else the work split between nparts (2 or 4)
// threads of the cell: part 0 writes the neighbour-density features; the
// Legendre variables go to the parts in order (GLM: 8 / nparts each; Powell:
// the 5 hydro variables), the LDF-mapped B to the last part (Powell).
template <typename Dm, typename Src, typename Put>
__device__ __forceinline__ void features_of(const Dm& dm, const MlpTabs& mt, const Src& src, Put put,
                                            int part = -1, int nparts = 2) {
  auto owner = [&](int v) {
    if (dm.glm()) return (v * nparts) >> 3;
    return nparts == 2 ? 0 : (v < 2 ? 0 : v < 4 ? 1 : 2);
  };
  const int ldf_part = nparts - 1;
  const int n = dm.n();
  float m[8];
  {
    float raw[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) raw[k] = src.row(dm.mrow(k));
    phys_means(dm, mt, raw, m);
  }
  float dmax[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= dm.D()) break;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      float raw[8], mn[8];
      src.nbraw(a, s, raw);
      phys_means(dm, mt, raw, mn);
#pragma unroll
      for (int k = 0; k < 8; ++k) dmax[k] = fmaxf(dmax[k], fabsf(mn[k] - m[k]));
      if (part <= 0) put(8 * n + 2 * a + s, mn[0] / m[0] - 1.f);
    }
  }
  float inv[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) inv[k] = 1.f / (fabsf(m[k]) + dmax[k] + 1e-12f);
  const float imdx = src.imdx(mt);
  const int nleg = dm.glm() ? 8 : 5;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const bool leg = v < nleg || (!dm.glm() && dm.D() == 2 && v == 7);
    if (!leg) continue;
    if (part >= 0 && owner(v) != part) continue;
    const int r0 = (v == 7 && !dm.glm()) ? dm.bz2d() : v * n;
#pragma unroll
    for (int l = 0; l < n; ++l) {
      const float av = (l == 0) ? m[v] : src.row(r0 + l);
      put(v * n + l, av * inv[v]);
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (a < dm.D() && l == dm.deg1(a)) put(8 * n + 2 * dm.D() + 8 * a + v, av * imdx);
    }
  }
  if (!dm.glm() && (part < 0 || part == ldf_part)) {
    // LDF B -> per-component Legendre coefficients (exact map)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      if (cc >= dm.D()) break;
#pragma unroll
      for (int l = 0; l < n; ++l) {
        float acc = 0.f;
        for (int j = 0; j < dm.ndiv(); ++j) acc += src.row(dm.ldf0() + j) * mt.l2l[(j * 3 + cc) * MLP_MAXN + l];
        put((5 + cc) * n + l, acc * inv[5 + cc]);
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (a < dm.D() && l == dm.deg1(a)) put(8 * n + 2 * dm.D() + 8 * a + 5 + cc, acc * imdx);
      }
    }
  }
}

template <typename T, typename Put>
__device__ __forceinline__ void cell_features(const Geom& g, const MlpTabs& mt, const T* w, const double* /*wmean*/,
                                              int64_t c, const AmrFeat& af, Put put) {
  if (af.on) features_of(RtDims{g, mt}, mt, AmrSrc<T>{g, w, c, af}, put);
  else features_of(RtDims{g, mt}, mt, GlobalSrc<T>{g, w, c}, put);
}

template <typename T>
__global__ void k_features(Geom g, MlpTabs mt, const T* __restrict__ w, const double* __restrict__ wmean,
                           float* __restrict__ X, int ldx, AmrFeat af) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int nin = 8 * g.n + 10 * g.D;
  float* xr = X + c * ldx;
  for (int k = nin; k < ldx; ++k) xr[k] = 0.f;
  cell_features(g, mt, w, wmean, c, af, [&](int k, float v) { xr[k] = v; });
}

// ---------------------------------------------------------------- inference (BF16 mma.sync)
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Network on the 32 cells of one warp: rows Xw[0..32) of bf16 features (row
// stride LD1) -> probabilities; writes the flags of the 32 cells to flw[0..32)
// and, for live cells, flag / prob. base = first cell of the warp.
template <int KP, int NTILE = 2>
__device__ __forceinline__ void infer_warp(const __nv_bfloat16* Xw, const __nv_bfloat16* W1s,
                                           const __nv_bfloat16* W2s, const float* bs, uint8_t* flw, int64_t base,
                                           int64_t ncell, float thresh, uint8_t* __restrict__ flag,
                                           float* __restrict__ prob) {
  constexpr int LD1 = KP + 8, LD2 = HID + 8;
  const int lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3;
  for (int tile = 0; tile < NTILE; ++tile) {
    const __nv_bfloat16* Xt = Xw + tile * 16 * LD1;
    float h1[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      h1[j][0] = bs[8 * j + 2 * tq];
      h1[j][1] = bs[8 * j + 2 * tq + 1];
      h1[j][2] = bs[8 * j + 2 * tq];
      h1[j][3] = bs[8 * j + 2 * tq + 1];
    }
#pragma unroll
    for (int kk = 0; kk < KP / 16; ++kk) {
      uint32_t a[4];
      a[0] = *reinterpret_cast<const uint32_t*>(Xt + gq * LD1 + 16 * kk + 2 * tq);
      a[1] = *reinterpret_cast<const uint32_t*>(Xt + (gq + 8) * LD1 + 16 * kk + 2 * tq);
      a[2] = *reinterpret_cast<const uint32_t*>(Xt + gq * LD1 + 16 * kk + 8 + 2 * tq);
      a[3] = *reinterpret_cast<const uint32_t*>(Xt + (gq + 8) * LD1 + 16 * kk + 8 + 2 * tq);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t b[2];
        b[0] = *reinterpret_cast<const uint32_t*>(W1s + (8 * j + gq) * LD1 + 16 * kk + 2 * tq);
        b[1] = *reinterpret_cast<const uint32_t*>(W1s + (8 * j + gq) * LD1 + 16 * kk + 8 + 2 * tq);
        mma_bf16(h1[j], a, b);
      }
    }
    // ReLU; accumulator tiles 2kk, 2kk+1 form the A fragment of layer 2's k-step kk
    float h2[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      h2[j][0] = bs[HID + 8 * j + 2 * tq];
      h2[j][1] = bs[HID + 8 * j + 2 * tq + 1];
      h2[j][2] = bs[HID + 8 * j + 2 * tq];
      h2[j][3] = bs[HID + 8 * j + 2 * tq + 1];
    }
#pragma unroll
    for (int kk = 0; kk < HID / 16; ++kk) {
      uint32_t a[4];
      a[0] = pack_bf16(fmaxf(h1[2 * kk][0], 0.f), fmaxf(h1[2 * kk][1], 0.f));
      a[1] = pack_bf16(fmaxf(h1[2 * kk][2], 0.f), fmaxf(h1[2 * kk][3], 0.f));
      a[2] = pack_bf16(fmaxf(h1[2 * kk + 1][0], 0.f), fmaxf(h1[2 * kk + 1][1], 0.f));
      a[3] = pack_bf16(fmaxf(h1[2 * kk + 1][2], 0.f), fmaxf(h1[2 * kk + 1][3], 0.f));
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t b[2];
        b[0] = *reinterpret_cast<const uint32_t*>(W2s + (8 * j + gq) * LD2 + 16 * kk + 2 * tq);
        b[1] = *reinterpret_cast<const uint32_t*>(W2s + (8 * j + gq) * LD2 + 16 * kk + 8 + 2 * tq);
        mma_bf16(h2[j], a, b);
      }
    }
    // output layer: rows gq and gq+8 of the tile, reduced over the quad
    float o0 = 0.f, o1 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float w0 = bs[2 * HID + 8 * j + 2 * tq], w1 = bs[2 * HID + 8 * j + 2 * tq + 1];
      o0 += fmaxf(h2[j][0], 0.f) * w0 + fmaxf(h2[j][1], 0.f) * w1;
      o1 += fmaxf(h2[j][2], 0.f) * w0 + fmaxf(h2[j][3], 0.f) * w1;
    }
    o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
    o0 += __shfl_xor_sync(0xffffffffu, o0, 2);
    o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
    o1 += __shfl_xor_sync(0xffffffffu, o1, 2);
    if (tq == 0) {
      const float b3 = bs[3 * HID];
      const int r0 = tile * 16 + gq;
      const int64_t c0 = base + r0;
      const float p0 = 1.f / (1.f + __expf(-(o0 + b3)));
      const float p1 = 1.f / (1.f + __expf(-(o1 + b3)));
      flw[r0] = p0 > thresh ? 1 : 0;
      flw[r0 + 8] = p1 > thresh ? 1 : 0;
      if (c0 < ncell) {
        if (flag) flag[c0] = p0 > thresh ? 1 : 0;
        if (prob) prob[c0] = p0;
      }
      if (c0 + 8 < ncell) {
        if (flag) flag[c0 + 8] = p1 > thresh ? 1 : 0;
        if (prob) prob[c0 + 8] = p1;
      }
    }
  }
}

// appends the warp's flagged live cells to list (ballot + one atomic per warp)
__device__ __forceinline__ void compact_warp(bool mine, int64_t c, int32_t* __restrict__ list,
                                             DevScalars* __restrict__ sc) {
  const int lane = threadIdx.x & 31;
  const unsigned bal = __ballot_sync(0xffffffffu, mine);
  const int cnt = __popc(bal);
  unsigned at = 0;
  if (lane == 0 && cnt) {
    at = atomicAdd(&sc->nflag, (unsigned)cnt);
    atomicAdd(&sc->cnt_flagged, (unsigned long long)cnt);
  }
  at = __shfl_sync(0xffffffffu, at, 0);
  if (mine) list[at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)c;
}

// One warp infers 32 cells (two m16 tiles); KP = padded input width (multiple of 16).
// Shared layout: W1s[64][KP+8] bf16, W2s[64][72] bf16, Xs[warps][32][KP+8] bf16, biases f32,
// flags of the warp's 32 cells. Persistent: the weights are staged once per block and the
// block walks 128-cell tiles with a grid stride. With `list`, each warp appends its flagged
// cells (ballot + one atomic per warp) to list and counts them in sc.
template <typename T, int KP>
__global__ void __launch_bounds__(128) k_mlp_infer(Geom g, MlpTabs mt, const T* __restrict__ w,
                                                   const double* __restrict__ wmean,
                                                   const __nv_bfloat16* __restrict__ W1,
                                                   const __nv_bfloat16* __restrict__ W2,
                                                   const float* __restrict__ bias, float thresh,
                                                   uint8_t* __restrict__ flag, float* __restrict__ prob,
                                                   int32_t* __restrict__ list, DevScalars* __restrict__ sc,
                                                   AmrFeat af) {
  constexpr int LD1 = KP + 8, LD2 = HID + 8;
  extern __shared__ __align__(128) unsigned char smraw[];
  __nv_bfloat16* W1s = reinterpret_cast<__nv_bfloat16*>(smraw);
  __nv_bfloat16* W2s = W1s + HID * LD1;
  __nv_bfloat16* Xs = W2s + HID * LD2;
  float* bs = reinterpret_cast<float*>(Xs + 4 * 32 * LD1);  // b1[64], b2[64], w3[64], b3
  uint8_t* fl = reinterpret_cast<uint8_t*>(bs + 3 * HID + 1);  // [4][32]
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int i = t; i < HID * KP; i += 128) W1s[(i / KP) * LD1 + i % KP] = W1[i];
  for (int i = t; i < HID * HID; i += 128) W2s[(i / HID) * LD2 + i % HID] = W2[i];
  for (int i = t; i < 3 * HID + 1; i += 128) bs[i] = bias[i];
  __syncthreads();
  const int nin = 8 * g.n + 10 * g.D;
  for (int64_t base = (int64_t)blockIdx.x * 128; base < g.ncell; base += (int64_t)gridDim.x * 128) {
    // features of this thread's cell (rows of Xs are private to the warp)
    const int64_t c = base + t;
    const bool live = c < g.ncell;
    {
      __nv_bfloat16* xr = Xs + (warp * 32 + lane) * LD1;
      for (int k = live ? nin : 0; k < KP; ++k) xr[k] = __float2bfloat16_rn(0.f);
      if (live) cell_features(g, mt, w, wmean, c, af, [&](int k, float v) { xr[k] = __float2bfloat16_rn(v); });
    }
    __syncwarp();
    infer_warp<KP>(Xs + warp * 32 * LD1, W1s, W2s, bs, fl + warp * 32, base + warp * 32, g.ncell, thresh, flag,
                   prob);
    __syncwarp();
    if (list) compact_warp(live && fl[warp * 32 + lane] != 0, c, list, sc);
    __syncwarp();
  }
}

// ---------------------------------------------------------------- training (FP32)
// Z[b][o] = sum_k A[idx(b)][k] W[o][k] + bias[o] (A rows gathered through perm if given)
__global__ void k_dense(const float* __restrict__ A, int lda, const int64_t* __restrict__ perm, int64_t off,
                        const float* __restrict__ W, const float* __restrict__ bias, float* __restrict__ Z, int nb,
                        int nin, int nout, int relu_in) {
  const int o = threadIdx.x % nout;
  const int b = blockIdx.x * (blockDim.x / nout) + threadIdx.x / nout;
  if (b >= nb || threadIdx.x >= (blockDim.x / nout) * nout) return;
  const int64_t row = perm ? perm[off + b] : off + b;
  const float* a = A + row * lda;
  float s = bias[o];
  for (int k = 0; k < nin; ++k) {
    float x = a[k];
    if (relu_in) x = fmaxf(x, 0.f);
    s += x * W[o * nin + k];
  }
  Z[(int64_t)b * nout + o] = s;
}

// output layer, loss and delta3 = (p - y) * weight / n
__global__ void k_out(const float* __restrict__ Z2, const float* __restrict__ w3, float b3,
                      const uint8_t* __restrict__ y, const int64_t* __restrict__ perm, int64_t off, int nb,
                      float pos_weight, float inv_n, float* __restrict__ d3, double* __restrict__ loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  float z = b3;
  for (int k = 0; k < HID; ++k) z += fmaxf(Z2[(int64_t)b * HID + k], 0.f) * w3[k];
  const float p = 1.f / (1.f + expf(-z));
  const int64_t row = perm ? perm[off + b] : off + b;
  const float yy = y[row] ? 1.f : 0.f;
  // weighted BCE: -(pw y log p + (1-y) log(1-p)); dL/dz = pw y (p - 1) + (1 - y) p
  d3[b] = (pos_weight * yy * (p - 1.f) + (1.f - yy) * p) * inv_n;
  if (loss) {
    const double l = -(pos_weight * yy * log((double)p + 1e-12) + (1.0 - yy) * log(1.0 - (double)p + 1e-12));
    atomicAdd(loss, l * (double)inv_n);
  }
}

// delta2[b][k] = d3[b] * w3[k] * (Z2 > 0)
__global__ void k_back2(const float* __restrict__ d3, const float* __restrict__ w3, const float* __restrict__ Z2,
                        float* __restrict__ d2, int nb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nb * HID) return;
  const int k = (int)(i % HID);
  const int64_t b = i / HID;
  d2[i] = Z2[i] > 0.f ? d3[b] * w3[k] : 0.f;
}

// delta1[b][k] = sum_o d2[b][o] W2[o][k] * (Z1 > 0)
__global__ void k_back1(const float* __restrict__ d2, const float* __restrict__ W2, const float* __restrict__ Z1,
                        float* __restrict__ d1, int nb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nb * HID) return;
  const int k = (int)(i % HID);
  const int64_t b = i / HID;
  float s = 0.f;
  for (int o = 0; o < HID; ++o) s += d2[b * HID + o] * W2[o * HID + k];
  d1[i] = Z1[i] > 0.f ? s : 0.f;
}

// gW[o][k] = sum_b delta[b][o] act(A[row(b)][k]); gb[o] = sum_b delta[b][o] (fixed order)
__global__ void k_wgrad(const float* __restrict__ delta, int nout, const float* __restrict__ A, int lda,
                        const int64_t* __restrict__ perm, int64_t off, int nin, int relu_in, int nb,
                        float* __restrict__ gW, float* __restrict__ gb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nout * (nin + 1)) return;
  const int o = i / (nin + 1), k = i % (nin + 1);
  float s = 0.f;
  for (int b = 0; b < nb; ++b) {
    const float d = delta[(int64_t)b * nout + o];
    if (k == nin) {
      s += d;
    } else {
      const int64_t row = perm ? perm[off + b] : off + b;
      float x = A[row * lda + k];
      if (relu_in) x = fmaxf(x, 0.f);
      s += d * x;
    }
  }
  if (k == nin) gb[o] = s;
  else gW[o * nin + k] = s;
}

__global__ void k_gout(const float* __restrict__ d3, const float* __restrict__ Z2, int nb, float* __restrict__ gw3,
                       float* __restrict__ gb3) {
  const int k = threadIdx.x;
  if (k > HID) return;
  float s = 0.f;
  for (int b = 0; b < nb; ++b) s += k == HID ? d3[b] : d3[b] * fmaxf(Z2[(int64_t)b * HID + k], 0.f);
  if (k == HID) *gb3 = s;
  else gw3[k] = s;
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ gr, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = gr[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int rows, int cols,
                          int ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * ldd) return;
  const int r = i / ldd, k = i % ldd;
  dst[i] = __float2bfloat16_rn(k < cols ? src[r * cols + k] : 0.f);
}

struct Scratch {
  float *Z1 = nullptr, *Z2 = nullptr, *d1 = nullptr, *d2 = nullptr, *d3 = nullptr;
};

// ---------------------------------------------------------------- staged inference
// FP32 form on uniform 3D meshes whose x-rows hold whole 128-cell tiles: the
// state rows of a tile (128 consecutive cells, 512 B per row) and the mean
// rows of its four y/z neighbour tiles are fetched by bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier) into shared memory; the
// features are then built from shared memory, so each block keeps ~57 KB of
// loads in flight instead of each thread walking 80+ dependent global loads.

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// a cell of the staged tile: own rows st[r][t], y/z neighbour means nbm[q][k][t]
// (q = 2 (axis - 1) + side), x neighbours inside the tile or, at its two ends,
// xe[side][k]
template <typename Dm>
struct StagedSrc {
  Dm dm;
  const float* st;
  const float* nbm;
  const float* xe;
  int t;
  __device__ float row(int r) const { return st[r * 128 + t]; }
  __device__ float imdx(const MlpTabs& mt) const { return mt.inv_mdx; }
  __device__ void nbraw(int a, int s, float* raw) const {
    if (a == 0) {
      const int tt = t + (s ? 1 : -1);
      if (tt < 0 || tt > 127)
        for (int k = 0; k < 8; ++k) raw[k] = xe[s * 8 + k];
      else
        for (int k = 0; k < 8; ++k) raw[k] = st[dm.mrow(k) * 128 + tt];
    } else {
      const int q = 2 * (a - 1) + s;
      for (int k = 0; k < 8; ++k) raw[k] = nbm[(q * 8 + k) * 128 + t];
    }
  }
};

constexpr long long kWaitCycles = 2000000000ll;  // about one second at GB300 clocks

template <int KP, bool GLM, int DEG, int NTH>
__global__ void __launch_bounds__(NTH) k_mlp_staged(Geom g, MlpTabs mt, const float* __restrict__ w,
                                                    const __nv_bfloat16* __restrict__ W1,
                                                    const __nv_bfloat16* __restrict__ W2,
                                                    const float* __restrict__ bias, float thresh,
                                                    uint8_t* __restrict__ flag, float* __restrict__ prob,
                                                    int32_t* __restrict__ list, DevScalars* __restrict__ sc,
                                                    int nrs, int nbuf, int32_t* __restrict__ plist, PosScreen ps) {
  extern __shared__ __align__(128) unsigned char smraw[];
  // nbuf tile buffers, each [nrs][128] own rows then [4][8][128] neighbour means
  float* buf = reinterpret_cast<float*>(smraw);
  const int bufsz = (nrs + 32) * 128;
  float* xe = buf + nbuf * bufsz;                        // [2][8]
  uint64_t* bar = reinterpret_cast<uint64_t*>(xe + 16);  // [0], [1]: tile copies; [2]: MMA completion
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
  // tensor-core operands in the K-major core-matrix layout (dg_tc.cuh)
  __nv_bfloat16* W1s = reinterpret_cast<__nv_bfloat16*>(xe + 32);  // [HID][KP]
  __nv_bfloat16* W2s = W1s + HID * KP;                              // [HID][HID]
  __nv_bfloat16* Xs = W2s + HID * HID;  // [128][KP] features; then layer 1's output [128][HID]
  float* bs = reinterpret_cast<float*>(Xs + 128 * KP);  // b1[64], b2[64], w3[64], b3
  // NP = NTH / 128 threads per cell split the feature work; the NTH / 32 warps
  // split the epilogues: warp w reads tensor-memory lanes 32 (w % 4).. and a
  // group of CW = HID / CG columns, CG = NTH / 128 groups
  constexpr int NP = NTH / 128, CG = NTH / 128, CW = HID / CG;
  static_assert(CW == 32 || CW == 16, "column groups of 32 or 16");
  float* part = bs + 3 * HID + 1;                       // [CG][128] partial sums of the output layer
  uint8_t* fl = reinterpret_cast<uint8_t*>(part + CG * 128);  // [128] flags of the tile
  uint8_t* sfail = fl + 128;                              // [128] positivity screen not cleared
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int cell = t & 127, fpart = t >> 7;
  for (int i = t; i < HID * KP; i += NTH) W1s[tc::kmajor_index(i / KP, i % KP, KP)] = W1[i];
  for (int i = t; i < HID * HID; i += NTH) W2s[tc::kmajor_index(i / HID, i % HID, HID)] = W2[i];
  for (int i = t; i < 3 * HID + 1; i += NTH) bs[i] = bias[i];
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    mbar_init(bar + 2, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // 128 tensor-memory columns: layer 1's accumulator [128 x 64], then layer 2's
  if (warp == 0) tc::tmem_alloc(tslot, 128);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = *tslot;
  constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, HID);
  const int64_t S = g.stride;
  const int nin = 8 * g.n + 10 * g.D;
  const unsigned bytes = (unsigned)(nrs + 32) * 512u;
  const int64_t ntile = g.ncell / 128;
  // thread 0: bulk copies of tile `tl` into buffer b, completion counted on bar[b]
  auto issue = [&](int64_t tl, int b) {
    float* st = buf + b * bufsz;
    float* nbm = st + nrs * 128;
    const int64_t c0 = tl * 128;
    // the buffer's previous reads (generic proxy) are ordered before these writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(bar + b, bytes);
    for (int r = 0; r < nrs; ++r) bulk_g2s(st + r * 128, w + (int64_t)r * S + c0, 512u, bar + b);
    for (int q = 0; q < 4; ++q) {
      const int64_t cn = nbc(g, c0, 1 + (q >> 1), (q & 1) ? 1 : -1);  // the whole tile shifts
      for (int k = 0; k < 8; ++k)
        bulk_g2s(nbm + (q * 8 + k) * 128, w + (int64_t)mrow(g, k) * S + cn, 512u, bar + b);
    }
  };
  // bounded wait of every thread on an mbarrier phase; false on timeout (all threads agree)
  auto wait_all = [&](uint64_t* b, unsigned parity) {
    bool ok = false;
    const long long t0 = clock64();
    while (!(ok = mbar_try_wait(b, parity)))
      if (clock64() - t0 > kWaitCycles) break;
    return __syncthreads_and(ok) != 0;
  };
  // two buffers: the next tile's copies run while this one is computed.
  // Every thread tracks which buffers have copies issued but not yet observed
  // complete (the issue decisions are block-uniform): a block that gives up on
  // a wait drains them before it exits, so no asynchronous write into its
  // shared memory outlives it.
  unsigned pend = 0;  // bit b: copies into buffer b issued, completion not yet observed
  if (nbuf == 2 && blockIdx.x < ntile) {
    if (t == 0) issue(blockIdx.x, 0);
    pend |= 1u;
  }
  unsigned par = 0;  // bit b: phase parity of bar[b]
  int it = 0;
  int mma_pending = -1;  // parity of an MMA commit not yet observed (timeout path), else -1
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x, ++it) {
    const int64_t c0 = tile * 128;
    const int b = nbuf == 2 ? (it & 1) : 0;
    const int64_t next = tile + gridDim.x;
    if (nbuf == 1) {
      if (t == 0) issue(tile, 0);
      pend |= 1u;
    } else if (next < ntile) {
      if (t == 0) issue(next, b ^ 1);  // released by the previous iteration's barrier
      pend |= 1u << (b ^ 1);
    }
    if (t < 16) {
      const int sd = t >> 3, k = t & 7;
      xe[t] = w[(int64_t)mrow(g, k) * S + nbc(g, c0 + (sd ? 127 : 0), 0, sd ? 1 : -1)];
    }
    // bounded wait for the tile's bytes (every thread polls: measured faster
    // than one polling warp and a block barrier)
    if (!wait_all(bar + b, (par >> b) & 1u)) {
      if (t == 0) atomicOr(&sc->status, 8);
      break;
    }
    par ^= 1u << b;
    pend &= ~(1u << b);
    const float* st = buf + b * bufsz;
    {
      using Dm = CtDims<GLM, DEG>;
      if (fpart == NP - 1)
        for (int q = nin; q < KP; ++q) Xs[tc::kmajor_index(cell, q, KP)] = __float2bfloat16_rn(0.f);
      features_of(Dm{}, mt, StagedSrc<Dm>{Dm{}, st, st + nrs * 128, xe, cell},
                  [&](int q, float v) { Xs[tc::kmajor_index(cell, q, KP)] = __float2bfloat16_rn(v); }, fpart,
                  NP);
    }
    tc::fence_proxy_async();  // the features, written by every thread, become tensor-core operands
    __syncthreads();
    // layer 1 on the tensor core: D1[128 x 64] = X[128 x KP] W1^T (FP32 in tensor memory)
    if (t == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < KP / 16; ++kk)
        tc::mma_bf16(tm, tc::smem_desc(tc::smem_u32(Xs + kk * 128), 128, KP * 16),
                     tc::smem_desc(tc::smem_u32(W1s + kk * 128), 128, KP * 16), IDESC, kk > 0);
      tc::commit(bar + 2);
    }
    mma_pending = 0;
    if (plist && t < 128) {
      // FP32 positivity screen on the staged rows (they hold every row the
      // screen reads), while the tensor core runs layer 1; only the cells the
      // indicator does not flag are listed from it (the TVB kernel screens the
      // flagged ones after limiting them)
      Geom gp = g;
      if constexpr (DEG <= 2) gp = pin_geom<DEG, GLM ? 1 : 0>(g);
      sfail[t] = pos_screen_rows(gp, ps, [&](int r) { return st[r * 128 + t]; }) ? 0 : 1;
    }
    if (!wait_all(bar + 2, 0)) {
      if (t == 0) atomicOr(&sc->status, 8);
      break;
    }
    mma_pending = -1;
    tc::fence_after_sync();
    // epilogue 1: warp w reads lanes 32 (w % 4).. of columns CW (w / 4)..; bias,
    // ReLU, BF16 into layer 2's A operand (over the features: layer 1 is done)
    const int quarter = warp & 3, colh = warp >> 2, row = 32 * quarter + lane;
    const uint32_t tlane = (uint32_t)(32 * quarter) << 16;
    {
      float v[CW];
      if constexpr (CW == 32) tc::ld32(tm + tlane + CW * colh, v);
      else tc::ld16(tm + tlane + CW * colh, v);
      // 16-byte stores of eight BF16 values: the 8 rows of a core matrix fill 128 contiguous bytes
#pragma unroll
      for (int j = 0; j < CW / 8; ++j) {
        uint4 pk;
        uint32_t* pw = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = CW * colh + 8 * j + 2 * e;
          pw[e] = pack_bf16(fmaxf(v[8 * j + 2 * e] + bs[k], 0.f), fmaxf(v[8 * j + 2 * e + 1] + bs[k + 1], 0.f));
        }
        *reinterpret_cast<uint4*>(Xs + tc::kmajor_index(row, CW * colh + 8 * j, HID)) = pk;
      }
    }
    tc::fence_before_sync();
    tc::fence_proxy_async();
    __syncthreads();
    // layer 2: D2[128 x 64] = H1[128 x 64] W2^T, in columns 64..127
    if (t == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < HID / 16; ++kk)
        tc::mma_bf16(tm + HID, tc::smem_desc(tc::smem_u32(Xs + kk * 128), 128, HID * 16),
                     tc::smem_desc(tc::smem_u32(W2s + kk * 128), 128, HID * 16), IDESC, kk > 0);
      tc::commit(bar + 2);
    }
    mma_pending = 1;
    if (!wait_all(bar + 2, 1)) {
      if (t == 0) atomicOr(&sc->status, 8);
      break;
    }
    mma_pending = -1;
    tc::fence_after_sync();
    // epilogue 2: bias, ReLU and this warp's share of the output layer's dot product
    {
      float v[CW];
      if constexpr (CW == 32) tc::ld32(tm + tlane + HID + CW * colh, v);
      else tc::ld16(tm + tlane + HID + CW * colh, v);
      float o = 0.f;
#pragma unroll
      for (int j = 0; j < CW; ++j) o += fmaxf(v[j] + bs[HID + CW * colh + j], 0.f) * bs[2 * HID + CW * colh + j];
      part[colh * 128 + row] = o;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (t < 128) {
      float z = bs[3 * HID];
#pragma unroll
      for (int gq = 0; gq < CG; ++gq) z += part[gq * 128 + t];
      const float p = 1.f / (1.f + __expf(-z));
      fl[t] = p > thresh ? 1 : 0;
      const int64_t cc = c0 + t;
      if (cc < g.ncell) {
        if (flag) flag[cc] = p > thresh ? 1 : 0;
        if (prob) prob[cc] = p;
      }
    }
    __syncthreads();  // the flags of the tile are written
    if (list && warp < 8)
      compact_warp(lane < 16 && fl[warp * 16 + (lane & 15)] != 0, c0 + warp * 16 + lane, list, sc);
    if (plist && warp < 8) {
      const int cl = warp * 16 + (lane & 15);
      append_cells(lane < 16 && fl[cl] == 0 && sfail[cl] != 0, c0 + cl, plist, &sc->npos);
    }
    __syncthreads();  // every read of this buffer, of xe and of the flags done before they are refilled
  }
  if (mma_pending >= 0) {
    // a commit not observed in time: wait once more (bounded) before the columns are freed
    const long long t0 = clock64();
    while (!mbar_try_wait(bar + 2, (unsigned)mma_pending))
      if (clock64() - t0 > kWaitCycles) break;
  }
  // timeout path: no new copies were issued after the failed wait; drain those
  // still in flight (bounded) before the block's shared memory is released
  for (int bb = 0; bb < 2; ++bb) {
    if (!((pend >> bb) & 1u)) continue;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar + bb, (par >> bb) & 1u))
      if (clock64() - t0 > kWaitCycles) break;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tm, 128);
}

}  // namespace

// full-batch (or mini-batch) loss and gradient; grad layout = theta layout
int mlp_loss_grad_dev(const float* X, int ldx, const uint8_t* y, const int64_t* perm, int64_t off, int nb, int nin,
                      const float* theta, float* grad, double* loss, float pos_weight, float norm_n, void* scratch,
                      cudaStream_t st) {
  const float* W1 = theta;
  const float* b1 = W1 + HID * nin;
  const float* W2 = b1 + HID;
  const float* b2 = W2 + HID * HID;
  const float* w3 = b2 + HID;
  float* gW1 = grad;
  float* gb1 = gW1 + HID * nin;
  float* gW2 = gb1 + HID;
  float* gb2 = gW2 + HID * HID;
  float* gw3 = gb2 + HID;
  float* gb3 = gw3 + HID;
  float* s = static_cast<float*>(scratch);
  float* Z1 = s;
  float* Z2 = Z1 + (size_t)nb * HID;
  float* d1 = Z2 + (size_t)nb * HID;
  float* d2 = d1 + (size_t)nb * HID;
  float* d3 = d2 + (size_t)nb * HID;
  float b3;
  if (cudaMemcpyAsync(&b3, w3 + HID, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess) return -3;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -3;
  const int per = 256 / HID;
  k_dense<<<(nb + per - 1) / per, per * HID, 0, st>>>(X, ldx, perm, off, W1, b1, Z1, nb, nin, HID, 0);
  k_dense<<<(nb + per - 1) / per, per * HID, 0, st>>>(Z1, HID, nullptr, 0, W2, b2, Z2, nb, HID, HID, 1);
  k_out<<<(nb + 255) / 256, 256, 0, st>>>(Z2, w3, b3, y, perm, off, nb, pos_weight, 1.f / norm_n, d3, loss);
  const int64_t nh = (int64_t)nb * HID;
  k_back2<<<(unsigned)((nh + 255) / 256), 256, 0, st>>>(d3, w3, Z2, d2, nb);
  k_back1<<<(unsigned)((nh + 255) / 256), 256, 0, st>>>(d2, W2, Z1, d1, nb);
  k_gout<<<1, 128, 0, st>>>(d3, Z2, nb, gw3, gb3);
  k_wgrad<<<(HID * (HID + 1) + 127) / 128, 128, 0, st>>>(d2, HID, Z1, HID, nullptr, 0, HID, 1, nb, gW2, gb2);
  k_wgrad<<<(HID * (nin + 1) + 127) / 128, 128, 0, st>>>(d1, HID, X, ldx, perm, off, nin, 0, nb, gW1, gb1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

size_t mlp_scratch_bytes(int nb) { return ((size_t)nb * HID * 4 + nb) * sizeof(float); }

int mlp_train_dev(const float* X, int ldx, const uint8_t* y, int64_t n, int nin, float* theta, int epochs,
                  int batch, float lr, float pos_weight, uint64_t seed, double* last_loss, cudaStream_t st) {
  const int np = mlp_n_params(nin);
  float *grad = nullptr, *m = nullptr, *v = nullptr;
  void* scratch = nullptr;
  int64_t* perm = nullptr;
  double* dloss = nullptr;
  int e = 0;
  if (cudaMalloc(&grad, np * sizeof(float)) || cudaMalloc(&m, np * sizeof(float)) ||
      cudaMalloc(&v, np * sizeof(float)) || cudaMalloc(&scratch, mlp_scratch_bytes(batch)) ||
      cudaMalloc(&perm, n * sizeof(int64_t)) || cudaMalloc(&dloss, sizeof(double)))
    e = -3;
  if (!e) {
    cudaMemsetAsync(m, 0, np * sizeof(float), st);
    cudaMemsetAsync(v, 0, np * sizeof(float), st);
    std::vector<int64_t> hp(n);
    for (int64_t i = 0; i < n; ++i) hp[i] = i;
    std::mt19937_64 rng(seed);
    int t = 0;
    for (int ep = 0; ep < epochs && !e; ++ep) {
      std::shuffle(hp.begin(), hp.end(), rng);
      if (cudaMemcpyAsync(perm, hp.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, st)) e = -3;
      cudaMemsetAsync(dloss, 0, sizeof(double), st);
      for (int64_t off = 0; off + batch <= n && !e; off += batch) {
        ++t;
        e = mlp_loss_grad_dev(X, ldx, y, perm, off, batch, nin, theta, grad, ep == epochs - 1 ? dloss : nullptr,
                              pos_weight, (float)batch, scratch, st);
        const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
        k_adam<<<(np + 255) / 256, 256, 0, st>>>(theta, grad, m, v, np, lr, 0.9f, 0.999f, 1e-8f, c1, c2);
      }
      if (cudaStreamSynchronize(st) != cudaSuccess) e = -3;
    }
    if (!e && last_loss) {
      double l = 0.0;
      cudaMemcpy(&l, dloss, sizeof(double), cudaMemcpyDeviceToHost);
      const int64_t nbat = n / batch;
      *last_loss = nbat ? l / (double)nbat : 0.0;
    }
  }
  cudaFree(grad);
  cudaFree(m);
  cudaFree(v);
  cudaFree(scratch);
  cudaFree(perm);
  cudaFree(dloss);
  return e;
}

static AmrFeat amr_feat(const Ctx& c) {
  return AmrFeat{c.amr.side_nb, c.amr.side_info, c.amr.dxc, c.g.dx, c.amr.on ? 1 : 0};
}

int mlp_build_tables(Ctx& c) {
  const Basis& B = *c.hb;
  const Geom& g = c.g;
  MlpTabs mt;
  std::memset(&mt, 0, sizeof(mt));
  if (g.n > MLP_MAXN || 8 * g.n + 10 * g.D > MLP_MAXIN) return -7;
  for (int a = 0; a < g.D; ++a)
    for (int l = 0; l < g.n; ++l) {
      const auto& k = B.modes[l];
      if (k[0] + k[1] + k[2] == 1 && k[a] == 1) mt.deg1[a] = l;
    }
  mt.inv_mdx = (float)(1.0 / (c.p.Mtilde * g.dx));
  if (!g.glm) {
    // <phi_j,c, P_l> / M_l by exact monomial integration
    const auto& ms = B.ms;
    for (int j = 0; j < g.ndiv && j < 64; ++j)
      for (int cc = 0; cc < g.D; ++cc)
        for (int l = 0; l < g.n; ++l) {
          double s = 0.0;
          for (size_t i = 0; i < ms.exps.size(); ++i) {
            const double a = B.ldf[j][cc][i];
            if (a == 0.0) continue;
            for (size_t k = 0; k < ms.exps.size(); ++k) {
              const double b = B.leg[l][k];
              if (b == 0.0) continue;
              double t = a * b;
              for (int ax = 0; ax < g.D; ++ax) {
                const int e = ms.exps[i][ax] + ms.exps[k][ax];
                t *= (e & 1) ? 0.0 : 2.0 / (e + 1.0);
              }
              s += t;
            }
          }
          mt.l2l[(j * 3 + cc) * MLP_MAXN + l] = (float)(s / B.leg_mass[l]);
        }
  }
  c.mlp = mt;
  return 0;
}

int mlp_features_launch(Ctx& c, const void* w, const double* wmean, float* X, int ldx, cudaStream_t st) {
  const Geom& g = c.g;
  const unsigned nb = (unsigned)((g.ncell + 127) / 128);
  if (c.p.precision == DG_PREC_FP32MIX)
    k_features<float><<<nb, 128, 0, st>>>(g, c.mlp, (const float*)w, nullptr, X, ldx, amr_feat(c));
  else
    k_features<double><<<nb, 128, 0, st>>>(g, c.mlp, (const double*)w, nullptr, X, ldx, amr_feat(c));
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mlp_set_weights(Ctx& c, const float* theta_dev, int nin, float thresh) {
  const Geom& g = c.g;
  if (nin != 8 * g.n + 10 * g.D) return -1;
  const int kp = (nin + 15) / 16 * 16;
  if (kp != 64 && kp != 80 && kp != 112 && kp != 192) return -7;
  if (!c.mlp_w1) {
    if (cudaMalloc(&c.mlp_w1, (size_t)HID * kp * 2) || cudaMalloc(&c.mlp_w2, (size_t)HID * HID * 2) ||
        cudaMalloc(&c.mlp_bias, (3 * HID + 1) * sizeof(float)))
      return -3;
  }
  const float* W1 = theta_dev;
  const float* b1 = W1 + HID * nin;
  const float* W2 = b1 + HID;
  const float* b2 = W2 + HID * HID;
  const float* w3 = b2 + HID;
  k_to_bf16<<<(HID * kp + 255) / 256, 256>>>(W1, (__nv_bfloat16*)c.mlp_w1, HID, nin, kp);
  k_to_bf16<<<(HID * HID + 255) / 256, 256>>>(W2, (__nv_bfloat16*)c.mlp_w2, HID, HID, HID);
  cudaMemcpy(c.mlp_bias, b1, HID * sizeof(float), cudaMemcpyDeviceToDevice);
  cudaMemcpy(c.mlp_bias + HID, b2, HID * sizeof(float), cudaMemcpyDeviceToDevice);
  cudaMemcpy(c.mlp_bias + 2 * HID, w3, (HID + 1) * sizeof(float), cudaMemcpyDeviceToDevice);
  c.mlp_kp = kp;
  c.mlp_thresh = thresh;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -3;
}

// shared memory of k_mlp_staged for nrs staged rows and nbuf tile buffers
template <int KP>
static size_t staged_smem(int nrs, int nbuf) {
  return (size_t)nbuf * (nrs + 32) * 512 + 128 + (size_t)HID * KP * 2 + (size_t)HID * HID * 2 + (size_t)128 * KP * 2 +
         (3 * HID + 1) * sizeof(float) + 512 * sizeof(float) + 256;
}

// threads per block of the staged kernel: two per cell of the 128-cell tile
// (measured at 256^3: four per cell, 512 threads, 3.97 against 3.92 ms per
// stage; two tile buffers at one block per SM 6.8 ms)
constexpr int kStagedThreads = 256;

// the staged kernel applies: FP32 form, uniform 3D mesh, x-rows of whole
// 128-cell tiles, and the shared memory fits. Two tile buffers only where two
// blocks still fit on an SM: measured at degree 2, one double-buffered block
// of 4 warps per SM is twice as slow as two single-buffered ones (the feature
// code needs the warps to hide its latencies).
template <int KP>
static bool staged_ok(const Ctx& c, int* nrs, int* nbuf) {
  const Geom& g = c.g;
  if (c.p.precision != DG_PREC_FP32MIX || c.amr.on || g.D != 3 || g.nx % 128 != 0) return false;
  *nrs = g.glm ? 8 * g.n : g.nrows;
  *nbuf = 2 * (staged_smem<KP>(*nrs, 2) + 1024) <= 228 * 1024 ? 2 : 1;
  return staged_smem<KP>(*nrs, *nbuf) <= 227 * 1024;
}

template <int KP, bool GLM, int DEG>
static void staged_launch(Ctx& c, const void* w, uint8_t* flag, float* prob, cudaStream_t st, int32_t* list,
                          int nrs, int nbuf, int32_t* plist) {
  const Geom& g = c.g;
  const size_t sm = staged_smem<KP>(nrs, nbuf);
  static size_t attr = 0;
  if (attr < sm) {
    cudaFuncSetAttribute(k_mlp_staged<KP, GLM, DEG, kStagedThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
    attr = sm;
  }
  // resident blocks per SM from the SM's shared memory (1 KB reserved per
  // block) and the kernel's registers
  static int per_sm = 0;
  static size_t per_sm_smem = 0;
  if (per_sm_smem != sm) {
    per_sm_smem = sm;
    int dev = 0, smem_sm = 0;
    cudaFuncAttributes fa;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    per_sm = smem_sm / (int)(sm + 1024);
    if (cudaFuncGetAttributes(&fa, k_mlp_staged<KP, GLM, DEG, kStagedThreads>) == cudaSuccess && fa.numRegs > 0)
      per_sm = std::min(per_sm, 65536 / (fa.numRegs * kStagedThreads));
    per_sm = std::max(per_sm, 1);
  }
  // at most four blocks per SM: each holds 128 of the SM's 512 tensor-memory columns
  const unsigned nb = (unsigned)std::min<int64_t>(g.ncell / 128, (int64_t)c.nsm * std::min(per_sm, 4));
  k_mlp_staged<KP, GLM, DEG, kStagedThreads><<<nb, kStagedThreads, sm, st>>>(
      g, c.mlp, (const float*)w, (const __nv_bfloat16*)c.mlp_w1, (const __nv_bfloat16*)c.mlp_w2, c.mlp_bias,
      c.mlp_thresh, flag, prob, list, c.sc, nrs, nbuf, plist, c.pscr);
}

template <typename T, int KP>
static void infer_launch(Ctx& c, const void* w, const double* wmean, uint8_t* flag, float* prob, cudaStream_t st,
                         int32_t* list, int32_t* plist, bool* screened) {
  int nrs = 0, nbuf = 1;
  if constexpr (sizeof(T) == 4) {
    if (staged_ok<KP>(c, &nrs, &nbuf)) {
      // compile-time feature code for the scheme and degree (KP follows the degree)
      constexpr int DEG = KP == 64 ? 1 : KP == 112 ? 2 : KP == 192 ? 3 : 0;
      if constexpr (DEG > 0) {
        if (c.g.d == DEG) {
          if (c.g.glm) staged_launch<KP, true, DEG>(c, w, flag, prob, st, list, nrs, nbuf, plist);
          else staged_launch<KP, false, DEG>(c, w, flag, prob, st, list, nrs, nbuf, plist);
          if (screened) *screened = plist != nullptr;
          return;
        }
      }
    }
  }
  const Geom& g = c.g;
  const size_t sm = (size_t)HID * (KP + 8) * 2 + (size_t)HID * (HID + 8) * 2 + (size_t)4 * 32 * (KP + 8) * 2 +
                    (3 * HID + 1) * sizeof(float) + 128;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_infer<T, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  // persistent grid: a few blocks per SM (the weights are staged once per block)
  const int64_t tiles = (g.ncell + 127) / 128;
  const unsigned nb = (unsigned)std::min<int64_t>(tiles, (int64_t)c.nsm * 4);
  k_mlp_infer<T, KP><<<nb, 128, sm, st>>>(g, c.mlp, (const T*)w, wmean, (const __nv_bfloat16*)c.mlp_w1,
                                           (const __nv_bfloat16*)c.mlp_w2, c.mlp_bias, c.mlp_thresh, flag, prob,
                                           list, c.sc, amr_feat(c));
}

int mlp_infer_launch(Ctx& c, const void* w, const double* wmean, uint8_t* flag, float* prob, cudaStream_t st,
                     int32_t* list, int32_t* pos_list, bool* screened) {
  if (screened) *screened = false;
  if (!c.mlp_w1) return -1;
  const bool f32 = c.p.precision == DG_PREC_FP32MIX;
  // FP32 form: features read the float mirror of the FP64 means (exact copies)
  switch (c.mlp_kp) {
#define KPCASE(K)                                                                 \
  case K:                                                                         \
    if (f32) infer_launch<float, K>(c, w, nullptr, flag, prob, st, list, pos_list, screened); \
    else infer_launch<double, K>(c, w, nullptr, flag, prob, st, list, nullptr, nullptr);      \
    break;
    KPCASE(64)
    KPCASE(80)
    KPCASE(112)
    KPCASE(192)
#undef KPCASE
    default:
      return -7;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace dgmhd
