// The opaque surv_workspace of the C ABI: device buffers that grow on demand
// and are reused across calls, the cached sweep graph of the last fit, and
// the state the differentiable form keeps between its forward and backward
// calls.  Internal to the library.
#pragma once

#include <cstddef>
#include <cstdint>

#include "internal.h"

struct surv_workspace {
  struct Buf {
    void* p = nullptr;
    size_t cap = 0;
  };
  enum Id {
    TIME, STATUS, COLPTR, ROWIDX, VALUES, XD, E, ETA, W2, GEND, DK, CK, GK, GKFF, WK0, WOFF, DTX, BETA, WIDTH, PEN, REC,
    SLOTS, CTRL, BLOCKCNT, SORTWORK, PERM, PF, WT, AGG,
    // differentiable form (cox_nll_forward / cox_nll_backward)
    NLL_Y, NLL_BCAT, NLL_REC, NLL_WT, NLL_DEN, NLL_LAM, NLL_G, NLL_GB, NLL_GEND, NLL_DK, NLL_WK0, NLL_BLK,
    NLL_CTRL, NLL_XP, NLL_ERR, NLL_FIN,
    // cross-validated path (cox_cv_path) and lambda_max
    CV_FOLD, CV_DK, CV_DTX, CV_E, CV_ETA, CV_REC, CV_WT, CV_AGG, CV_PART, CV_GCTL, CV_BETA, CV_WIDTH, CV_PEN,
    CV_OUT, CV_FITS, CV_CTRL, CV_DEN, CV_HELD, CV_MEAN, LM_LAM, LM_R, LM_G,
    // sparse-numerator form
    SN_GRP, SN_DEN, SN_V1, SN_V2, SN_LAM, SN_W, SN_PDEN, SN_LL, SN_PCOL,
    NBUF
  };
  int device = -1;
  Buf bufs[NBUF];
  survgpu::GraphCache graph;  // instantiated sweep graph of the last fit
  // shape of the last cox_nll_forward (what cox_nll_backward continues from)
  int64_t nll_n = -1;
  int32_t nll_p = 0, nll_c = 0, nll_K = 0, nll_G = 0, nll_wpc = 0, nll_wpw = 0;
  const void* nll_x = nullptr;
  const void* nll_xt = nullptr;   // X as the tensor-core kernels read it (padded copy if needed)
  int64_t nll_ld = 0;              // its row pitch in elements
  bool nll_err_init = false;       // the tensor-core kernels' error word has been zeroed
  // CTAs per fit chosen by the cross-validation tuner, and the shape it was
  // tuned for (n, p, fits, layout * 2 + precision, dtype, layout tag)
  int32_t cv_tuned_ctas = 0;
  int32_t cv_tuned_form = 0;     // and the form of the row pass (CcdParams::pass_form)
  int32_t cv_tuned_tile = 0;     // and its tile shape (CcdParams::tile_form)
  int64_t cv_tune_key[6] = {0, 0, 0, 0, 0, 0};
};

namespace survgpu {
// Grow buffer `id` to at least `bytes` (api.cu); SURV_* error code.
int ws_ensure(surv_workspace* ws, int id, size_t bytes, void** out);
// Tensor-core products of the differentiable form (nll_tc.cu).  X: n rows of
// p bfloat16 with row pitch ldx (a multiple of 8, 16-byte aligned base);
// BcatT / Gcat: the bf16 split in 2 Cp columns (hi at c, lo at Cp + c).  A
// bounded device wait that expires sets *err.
cudaError_t nll_xb_tc(const void* X, int64_t n, int p, int64_t ldx, const void* BcatT, int C, int Cp, float* eta,
                      unsigned* err, cudaStream_t s);
size_t nll_xtg_part_floats(int64_t n, int p, int NB, int* nx);
// Whether X B with p covariates and C columns fits the forward kernel (B is
// kept in shared memory beside at least three X stages).
bool nll_tc_fits(int p, int C);
cudaError_t nll_xtg_tc(const void* X, int64_t n, int p, int64_t ldx, const void* Gcat, int C, int Cp, float* part,
                       int nx, float* grad_B, unsigned* err, cudaStream_t s);
}  // namespace survgpu
