// Learned troubled-cell indicator (see dg_mlp.cu).
#pragma once
#include "dg_ctx.h"

namespace dgmhd {

inline int mlp_n_params(int nin) { return 64 * nin + 64 + 64 * 64 + 64 + 64 + 1; }

int mlp_build_tables(Ctx& c);
int mlp_features_launch(Ctx& c, const void* w, const double* wmean, float* X, int ldx, cudaStream_t st);
int mlp_set_weights(Ctx& c, const float* theta_dev, int nin, float thresh);
// flag / prob / list may be null; with list, the flagged cells are appended to
// list[0 .. c.sc->nflag) (the caller zeroes nflag first). With pos_list (FP32
// form), the staged kernel also runs the FP32 positivity screen on the cells
// it does not flag and appends those that do not clear it to
// pos_list[0 .. c.sc->npos) (the caller zeroes npos first and screens the
// flagged cells after limiting them); *screened tells whether it did.
int mlp_infer_launch(Ctx& c, const void* w, const double* wmean, uint8_t* flag, float* prob, cudaStream_t st,
                     int32_t* list = nullptr, int32_t* pos_list = nullptr, bool* screened = nullptr);
size_t mlp_scratch_bytes(int nb);
int mlp_loss_grad_dev(const float* X, int ldx, const uint8_t* y, const int64_t* perm, int64_t off, int nb, int nin,
                      const float* theta, float* grad, double* loss, float pos_weight, float norm_n, void* scratch,
                      cudaStream_t st);
int mlp_train_dev(const float* X, int ldx, const uint8_t* y, int64_t n, int nin, float* theta, int epochs, int batch,
                  float lr, float pos_weight, uint64_t seed, double* last_loss, cudaStream_t st);

}  // namespace dgmhd
