// Operator evaluation that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host framework that owns every byte of
// device memory through its own pool, code that runs while the device must not
// be synchronised (cudaMalloc/cudaFree may synchronise), or an embedding that
// forbids growing the device footprint after start-up. For them this file keeps
// all device scratch of one right-hand-side evaluation -- the basis tables, the
// device scalars and the face-flux buffer -- in one file-scope __device__ array
// of fixed size. Every GPU that loads the library holds this array until exit.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/dg_mhd.h"
#include "dg_basis.h"
#include "dg_ctx.h"
#include "dg_kernels.cuh"

namespace dgmhd {
// defined in dg_api.cu
int make_geom(const dg_mesh_desc* mesh, int degree, int divB_scheme, double gamma, Basis& B, Geom& g);
void host_tables(const Basis& B, const Geom& g, std::vector<double>* out10);
}  // namespace dgmhd

using namespace dgmhd;

namespace {

constexpr size_t kScratchDoubles = size_t(4) << 20;  // 32 MiB
static __device__ __align__(256) double g_scratch[kScratchDoubles];

inline size_t round256(size_t n_doubles) { return (n_doubles + 31) / 32 * 32; }

// Host copies of the reference-element tables, one set per (dimension, degree,
// scheme), built on first use and kept until the process exits: the
// asynchronous uploads below read them after this function has returned, so
// their storage must outlive every call.
struct HostTabs {
  std::vector<double> t[10];  // Pv dPv Pf Lv dLv Lf L0 wv wf minv
};
std::mutex g_tabs_mu;
std::map<std::tuple<int, int, int>, HostTabs>& tabs_cache() {
  static std::map<std::tuple<int, int, int>, HostTabs> m;  // never destroyed before exit
  return m;
}

const HostTabs& host_tabs_for(const Basis& B, const Geom& g, int divB_scheme) {
  std::lock_guard<std::mutex> lk(g_tabs_mu);
  auto key = std::make_tuple(g.D, g.d, divB_scheme);
  auto& m = tabs_cache();
  auto it = m.find(key);
  if (it == m.end()) {
    HostTabs h;
    host_tables(B, g, h.t);
    it = m.emplace(key, std::move(h)).first;  // std::map nodes never move afterwards
  }
  return it->second;
}

// Sets status bit 1 (non-finite) if any entry of the rhs rows is NaN or infinite.
__global__ void k_noalloc_finite(const double* __restrict__ rhs, int nrows, int64_t ncell, int64_t stride,
                                 DevScalars* sc) {
  bool bad = false;
  const int64_t total = (int64_t)nrows * ncell;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ncell, c = i - r * ncell;
    bad |= !isfinite(rhs[r * stride + c]);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&sc->status, 1);
}

// Copies the status word of the scalars to the caller's device int.
__global__ void k_noalloc_status(const DevScalars* sc, int* status_dev) { *status_dev = sc->status; }

}  // namespace

extern "C" int dg_mhd_rhs_noalloc(const dg_mesh_desc* mesh, int degree, int divB_scheme, double gamma,
                                  const dg_mhd_params* p, double c_h, double damping_rate, const double* w,
                                  double* rhs, int* status_dev, void* stream) {
  if (!mesh || !w || !rhs) return DG_E_ARG;
  Basis B;
  Geom g;
  int e = make_geom(mesh, degree, divB_scheme, gamma, B, g);
  if (e) return e;
  if (g.glm && (!(c_h > 0.0) || !(damping_rate >= 0.0))) return DG_E_ARG;
  dg_mhd_params prm;
  if (p) prm = *p;
  else dg_mhd_default_params(&prm);
  // the HLLD degeneracy tolerance is the only parameter read here
  if (!(prm.eps_hlld >= 0.0 && prm.eps_hlld < 1.0)) return DG_E_ARG;

  const HostTabs& ht = host_tabs_for(B, g, divB_scheme);
  size_t off[10], total = 0;
  for (int i = 0; i < 10; ++i) {
    off[i] = total;
    total += round256(ht.t[i].size());
  }
  const size_t sc_off = total;
  total += round256((sizeof(DevScalars) + sizeof(double) - 1) / sizeof(double));
  const size_t face_off = total;
  const size_t face_elems = (size_t)g.D * (size_t)g.ncell * g.Qf * 9;
  total += round256(face_elems);
  if (total > kScratchDoubles) return DG_E_ARG;  // problem larger than the static scratch

  // The array's device address on the current device, looked up on every call
  // (the lookup allocates nothing). On a device's first call with lazily
  // loaded modules it may load this library's module: that can allocate and
  // synchronise, so such callers make one warm-up call at start-up.
  void* pv = nullptr;
  if (cudaGetSymbolAddress(&pv, g_scratch) != cudaSuccess || pv == nullptr) return DG_E_CUDA;
  double* base = static_cast<double*>(pv);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < 10; ++i)
    if (!ht.t[i].empty() &&
        cudaMemcpyAsync(base + off[i], ht.t[i].data(), ht.t[i].size() * sizeof(double), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return DG_E_CUDA;
  Tables<double> tb;
  double** dst[10] = {&tb.Pv, &tb.dPv, &tb.Pf, &tb.Lv, &tb.dLv, &tb.Lf, &tb.L0, &tb.wv, &tb.wf, &tb.minv};
  for (int i = 0; i < 10; ++i) *dst[i] = base + off[i];
  DevScalars* sc = reinterpret_cast<DevScalars*>(base + sc_off);
  // the scalars start from zero on every call (status word included)
  if (cudaMemsetAsync(sc, 0, sizeof(DevScalars), st) != cudaSuccess) return DG_E_CUDA;
  if (g.glm) launch_set_glm(sc, c_h, damping_rate, st);
  double* fbuf = base + face_off;  // fully written by the face kernel before it is read
  launch_face<double>(g, tb, w, fbuf, sc, prm.eps_hlld, st);
  launch_cell<double>(g, tb, w, fbuf, rhs, nullptr, 0.0, 1.0, 0, sc, nullptr, nullptr, nullptr, st);
  // the call's device status word (bit 1: a non-finite value in rhs), copied
  // out before a later call clears it
  if (status_dev) {
    k_noalloc_finite<<<64, 256, 0, st>>>(rhs, g.nrows, g.ncell, g.stride, sc);
    k_noalloc_status<<<1, 1, 0, st>>>(sc, status_dev);
  }
  if (cudaGetLastError() != cudaSuccess) return DG_E_CUDA;
  return DG_OK;
}
