// Kernels of the CUDA-core DG-MHD path (FP64 plain form and the FP32 form).
#pragma once
#include "dg_ctx.h"

namespace dgmhd {

// launches (all asynchronous on `st`)
// qbuf (Powell, nullable): q^dagger of eq. powellq-interp per face point,
// 14 values (left then right trace), written by launch_face and read by
// launch_cell in place of q(<u>_K)
template <typename T>
void launch_face(const Geom& g, const Tables<T>& tb, const T* w, T* fbuf, const DevScalars* sc, double eps,
                 cudaStream_t st, T* qbuf = nullptr);
template <typename T>
void launch_cell(const Geom& g, const Tables<T>& tb, const T* w, const T* fbuf, T* out, const T* w0,
                 double ca, double cb, int combine, const DevScalars* sc, const double* wmean,
                 const double* w0mean, double* outmean, cudaStream_t st, const T* qbuf = nullptr);
template <typename T>
void launch_project(const Geom& g, int npts, const double* tab, const double* wq, const double* nodal,
                    const T* minv, T* w, double* wmean, cudaStream_t st);
template <typename T>
void launch_divb_face(const Geom& g, const Tables<T>& tb, const T* w, T* jbuf, cudaStream_t st);
template <typename T>
void launch_dt(const Geom& g, const Tables<T>& tb, const T* w, const double* wmean, const T* jbuf,
               const dg_mhd_params& p, DevScalars* sc, double* dt_out, cudaStream_t st);
void launch_dt_from_value(const Geom& g, const dg_mhd_params& p, const double* dt_in, DevScalars* sc,
                          cudaStream_t st);
void launch_set_glm(DevScalars* sc, double ch, double kappa, cudaStream_t st);
void launch_dt_init(DevScalars* sc, cudaStream_t st);
// div B diagnostics of App. C (uniform meshes): res[4] on the device, per_cell
// [3][stride] or null; scratch: 3 doubles per face point
template <typename T>
void launch_divb_diag(const Geom& g, const Tables<T>& tb, const T* w, const double* wmean, double* scratch,
                      double* res, double* per_cell, cudaStream_t st);
// sets the device dt to f times the step's dt (and its FP32 copy)
void launch_dt_scale(DevScalars* sc, double f, cudaStream_t st);
// out = a x + b y over all state rows; FP32 form: FP64 means from xm, ym into om
template <typename T>
void launch_axpby(const Geom& g, double a, const T* x, double b, const T* y, T* out, const double* xm,
                  const double* ym, double* om, cudaStream_t st);
void launch_dt_finalize(const Geom& g, const dg_mhd_params& p, DevScalars* sc, double* dt_out, cudaStream_t st);
template <typename T>
void launch_mirror_means(const Geom& g, const double* wmean, T* w, cudaStream_t st);

}  // namespace dgmhd
