// Static octree meshes: face lists and the face-list operator kernels.
#pragma once
#include "dg_ctx.h"

namespace dgmhd {

// face f: left cell fL, right cell fR, meta = axis | kind << 2 | sub << 4
// (kind 0 same level, 1 left cell coarse, 2 right cell coarse; sub = sub-face
// of the coarse face, bit j for the j-th tangential axis in increasing order).
// cell c: entries centry[cstart[c] .. cstart[c+1]) = (face << 1) | side,
// side 0 if the cell is the face's left cell. Psub/Lsub: coarse-side tables
// [(face * nsub + sub) ...] at the fine face's points mapped into the coarse face.
template <typename T>
struct AmrDev {
  const int32_t* fL;
  const int32_t* fR;
  const int32_t* fmeta;
  const int32_t* cstart;
  const int32_t* centry;
  const double* dxc;
  const T* Psub;
  const T* Lsub;
  const T* Psub4;  // Psub / Lsub with the point index padded to pad4(Qf)
  const T* Lsub4;
  int64_t nface;
  int maxent;
  int nsub;
};

int build_amr(Ctx& c, const dg_mesh_desc* mesh);
// the specialised Powell kernels' view of the octree (AmrHost::fast)
template <typename T>
struct OctPow;
OctPow<float> oct_pow32(const Ctx& c);
OctPow<double> oct_pow64(const Ctx& c);
void free_amr(Ctx& c);

template <typename T>
void launch_amr_operator(const Ctx& c, const Tables<T>& tb, const T* w, T* fbuf, T* out, const T* w0, double ca,
                         double cb, int combine, const DevScalars* sc, const double* wmean, const double* w0mean,
                         double* outmean, double eps, cudaStream_t st, T* qbuf = nullptr);
template <typename T>
void launch_amr_dt(const Ctx& c, const Tables<T>& tb, const T* w, const double* wmean, T* jbuf,
                   const dg_mhd_params& p, DevScalars* sc, cudaStream_t st);

}  // namespace dgmhd
