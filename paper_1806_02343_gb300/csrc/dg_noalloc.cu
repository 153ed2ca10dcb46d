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

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};

inline size_t round256(size_t n_doubles) { return (n_doubles + 31) / 32 * 32; }

// Device address of g_scratch on the current device; resolved once per device.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DG_E_CUDA;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return DG_E_CUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return DG_OK;
}

}  // namespace

extern "C" int dg_mhd_rhs_noalloc(const dg_mesh_desc* mesh, int degree, int divB_scheme, double gamma,
                                  const dg_mhd_params* p, double c_h, double damping_rate, const double* w,
                                  double* rhs, void* stream) {
  if (!mesh || !w || !rhs) return DG_E_ARG;
  Basis B;
  Geom g;
  int e = make_geom(mesh, degree, divB_scheme, gamma, B, g);
  if (e) return e;
  if (g.glm && !(c_h > 0.0)) return DG_E_ARG;
  dg_mhd_params prm;
  if (p) prm = *p;
  else dg_mhd_default_params(&prm);

  std::vector<double> tabs[10];  // Pv dPv Pf Lv dLv Lf L0 wv wf minv
  host_tables(B, g, tabs);
  size_t off[10], total = 0;
  for (int i = 0; i < 10; ++i) {
    off[i] = total;
    total += round256(tabs[i].size());
  }
  const size_t sc_off = total;
  total += round256((sizeof(DevScalars) + sizeof(double) - 1) / sizeof(double));
  const size_t face_off = total;
  const size_t face_elems = (size_t)g.D * (size_t)g.ncell * g.Qf * 9;
  total += round256(face_elems);
  if (total > kScratchDoubles) return DG_E_ARG;  // problem larger than the static scratch

  double* base = nullptr;
  if ((e = scratch_address(&base))) return e;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < 10; ++i)
    if (!tabs[i].empty() &&
        cudaMemcpyAsync(base + off[i], tabs[i].data(), tabs[i].size() * sizeof(double), cudaMemcpyHostToDevice,
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
  if (cudaGetLastError() != cudaSuccess) return DG_E_CUDA;
  // the host vectors above are pageable: the copies were staged before returning
  return DG_OK;
}
