// The predictor of a load step (Sec. 2.1, 2.3) as per-voxel coefficients,
// shared by the predictor pass (history.cu) and the double-word constitutive
// pass that applies it on the fly (constitutive_dw.cu).  Every form is
//   F <- F + v1 (A - F) + v2 (B - F) + sh,   then slot dst (0: A, 1: B) <- old F
// with
//   uniform    (no kept state):   v1 = v2 = 0, dst = -1,
//   linear     (A = Fprev):       v1 = -alpha, v2 = 0, dst = 0 (F + alpha (F - Fprev)),
//   quadratic  (A, B the slots):  v1, v2 the weights of the step's start, dst its slot;
// sh[c] = 0 on a stress-controlled component, else the uniform shift that
// makes the average of component c the prescribed F-bar.
#pragma once

#include "launch.h"

// predictor kinds (the context's MF_PRED_*: 0 uniform, 1 linear, 2 quadratic)
struct PredArgs {
  double* A;            // Fprev (linear), slot A (quadratic), else null
  double* B;            // slot B (quadratic), else null
  const HistState* hs;
  int kind;
};

struct PredCoef {
  double v1, v2;
  double sh[9];
  int dst;
};

// The coefficients of the step that k_step_begin prepared; sc->meanF: the
// averages of the current (last converged) F.
__device__ __forceinline__ PredCoef pred_coef(const PredArgs& pa, const Scalars* sc) {
  const HistState* hs = pa.hs;
  PredCoef k;
  k.v1 = 0.0;
  k.v2 = 0.0;
  k.dst = -1;
  if (pa.kind == 2) {
    const bool qx = hs->extrapolated && hs->quad;
    k.v1 = qx ? hs->w[1] : 0.0;
    k.v2 = qx ? hs->w[2] : 0.0;
    k.dst = hs->dst;
    for (int c = 0; c < 9; ++c) k.sh[c] = hs->mask[c] ? 0.0 : hs->target[c] - (qx ? hs->pmean[c] : sc->meanF[c]);
  } else {
    const double a = (pa.kind == 1 && hs->extrapolated) ? hs->alpha : 0.0;
    if (pa.kind == 1) {
      k.v1 = -a;
      k.dst = 0;
    }
    for (int c = 0; c < 9; ++c)
      k.sh[c] = hs->mask[c] ? 0.0 : hs->target[c] - (sc->meanF[c] + a * (sc->meanF[c] - hs->fmean2[c]));
  }
  return k;
}
