// Device-side Newton control of a load history (Sec. 2.3, Eq. linequil2ast
// and eq:mixedeqil; Sec. 4 stopping rules).  With these kernels a whole load
// history of a cell runs as one graph launch: a WHILE node over the load
// steps, inside it a WHILE node over the Newton iterations, inside that the
// WHILE node of the CG iterations.  Every decision the host used to take
// between launches -- the forcing of the inner solve, the null rigid
// rotations, the arithmetic of the projection of a correction, the Newton
// convergence test, the recording of a step's averages -- is taken here by
// one thread, which sets the graph's conditional handles.
#include <math.h>

#include "../../include/mixfft.h"
#include "dw.cuh"
#include "launch.h"
#include "predict.cuh"

namespace {

constexpr int kThreads = 256;
// corrections of at least this size relative to F are projected in the outer
// arithmetic under MF_PROJ_AUTO (their FP32 projection would leave ~1e-10 of F)
constexpr double kProjOuterAbove = 1e-3;


int grid_for(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return (int)g;
}
// grid-stride passes that usually return at once (they act only when a
// rigid rotation is null): four blocks per SM at most
int rare_grid(long long n) {
  const int g = grid_for(n);
  return g < 4 * 152 ? g : 4 * 152;
}

// ------------------------------------------------------------ null rotations
// Cyclic Jacobi eigen-decomposition of a symmetric m x m matrix (m <= 3): on
// return A holds the eigenvalues on its diagonal, V the eigenvectors.
__device__ void jacobi3(int m, double A[3][3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) off += A[p][q] * A[p][q];
    if (off < 1e-300) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        if (A[p][q] == 0.0) continue;
        const double th = 0.5 * (A[q][q] - A[p][p]) / A[p][q];
        const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

__device__ void skew3(const double w[3], double W[9]) {
  W[0] = 0; W[1] = -w[2]; W[2] = w[1];
  W[3] = w[2]; W[4] = 0; W[5] = -w[0];
  W[6] = -w[1]; W[7] = w[0]; W[8] = 0;
}

// tr(Wa^T Wb M) = sum_ij Wa_ij (Wb M)_ij
__device__ double tr_wwm(const double* Wa, const double* Wb, const double* M) {
  double s = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double wm = 0.0;
      for (int k = 0; k < 3; ++k) wm += Wb[3 * i + k] * M[3 * k + j];
      s += Wa[3 * i + j] * wm;
    }
  return s;
}

// Rigid rotations of the cell that the linearised problem cannot see (the
// paper is silent on them; they arise under stress control).  A rotation
// increment W (skew) gives the compatible field n = W F; it is admissible
// when (W <F>)_ij = 0 on every strain-controlled component.  By objectivity
// the curvature n_a . A n_b is tr(W_a^T W_b T), T = sum_v P_v F_v^T, and
// n_a . n_b = tr(W_a^T W_b S), S = sum_v F_v F_v^T.  The admissible
// rotations whose curvature is below tau * kappa are returned with the n_k
// orthonormal.
__device__ void null_rotations_dev(const double* meanF, const unsigned char* mask, const double* T,
                                   const double* S, double kappa, double tau, Defl* d) {
  d->m = 0;
  double Wg[3][9];
  for (int a = 0; a < 3; ++a) {
    double w[3] = {0, 0, 0};
    w[a] = 1.0;
    skew3(w, Wg[a]);
  }
  double CtC[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int c = 0; c < 9; ++c) {
    if (mask[c]) continue;
    const int i = c / 3, j = c % 3;
    double row[3];
    for (int a = 0; a < 3; ++a)
      row[a] = Wg[a][3 * i] * meanF[j] + Wg[a][3 * i + 1] * meanF[3 + j] + Wg[a][3 * i + 2] * meanF[6 + j];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) CtC[a][b] += row[a] * row[b];
  }
  // no admissible rotation when C^T C is clearly nonsingular: its smallest
  // eigenvalue is at least det / tr^2, and a det above 1e-12 tr^3 (far above
  // its rounding) with tr above 1e-6 puts it above the 1e-20 of the test
  // below; the eigen-decomposition, slow in one thread, is skipped then
  // (the common case of mixed control with strain-controlled shear components)
  const double tr = CtC[0][0] + CtC[1][1] + CtC[2][2];
  const double det = CtC[0][0] * (CtC[1][1] * CtC[2][2] - CtC[1][2] * CtC[2][1]) -
                     CtC[0][1] * (CtC[1][0] * CtC[2][2] - CtC[1][2] * CtC[2][0]) +
                     CtC[0][2] * (CtC[1][0] * CtC[2][1] - CtC[1][1] * CtC[2][0]);
  if (tr > 1e-6 && det > 1e-12 * tr * tr * tr) return;
  double V[3][3];
  jacobi3(3, CtC, V);
  double Z[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  int m = 0;
  for (int k = 0; k < 3; ++k)
    if (fabs(CtC[k][k]) <= 1e-20) {
      for (int a = 0; a < 3; ++a) Z[a][m] = V[a][k];
      ++m;
    }
  if (m == 0) return;
  double R[3][3], G[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      R[a][b] = 0.5 * (tr_wwm(Wg[a], Wg[b], T) + tr_wwm(Wg[b], Wg[a], T));
      G[a][b] = tr_wwm(Wg[a], Wg[b], S);
    }
  double Rz[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Gz[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int p = 0; p < m; ++p)
    for (int q = 0; q < m; ++q)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          Rz[p][q] += Z[a][p] * R[a][b] * Z[b][q];
          Gz[p][q] += Z[a][p] * G[a][b] * Z[b][q];
        }
  // G-orthonormal eigenvectors of Rz v = lambda Gz v: Gz = Q g Q^T, then the
  // standard problem for g^-1/2 Q^T Rz Q g^-1/2
  double Qg[3][3];
  jacobi3(m, Gz, Qg);
  double H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int p = 0; p < m; ++p)
    for (int q = 0; q < m; ++q) {
      double s = 0.0;
      for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) s += Qg[a][p] * Rz[a][b] * Qg[b][q];
      H[p][q] = s / sqrt(Gz[p][p] * Gz[q][q]);
    }
  double U[3][3];
  jacobi3(m, H, U);
  for (int k = 0; k < m; ++k) {
    if (fabs(H[k][k]) > tau * kappa) continue;
    double v[3] = {0, 0, 0};
    for (int p = 0; p < m; ++p) {
      double s = 0.0;
      for (int q = 0; q < m; ++q) s += Qg[p][q] * U[q][k] / sqrt(Gz[q][q]);
      v[p] = s;
    }
    double w[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a)
      for (int p = 0; p < m; ++p) w[a] += Z[a][p] * v[p];
    skew3(w, d->W[d->m]);
    ++d->m;
  }
}

__device__ int flags_to_status(int flags) {
  if (flags & MF_FLAG_TIMEOUT) return MF_DEVICE_TIMEOUT;
  if (flags & MF_FLAG_NONPOS_J) return MF_NONPOSITIVE_J;
  if (flags & (MF_FLAG_BREAKDOWN | MF_FLAG_NONFINITE)) return MF_CG_BREAKDOWN;
  return MF_OK;
}

// ------------------------------------------------------------ control kernels
__global__ void k_hist_init(HistState* hs, cudaGraphConditionalHandle h_step, int kernels) {
  hs->k = 0;
  hs->status = MF_OK;
  hs->launches = kernels;
  cudaGraphSetConditional(h_step, hs->nsteps > 0 ? 1u : 0u);
}

// The quadratic predictor's start of a step (MF_PRED_QUADRATIC).  The
// converged state of a hyperelastic law is a function of the load, so F at
// the new target is interpolated from the kept states with this step's
// mask: the last converged one (in F, target t1) and those in slots A and B
// (targets t2, t3).  With A and B usable and the three targets on one line
// at distinct positions: Lagrange weights in the position s along that line
// (s = 0 at t1); with one of them: linear along the line through it; else no
// extrapolation.  A target at a kept one gets that state exactly.  Then the
// last converged state takes a slot: the one holding its own target (a
// repeated load), else the one holding this step's target (the step
// reconverges that state), else the older one; so the slots keep distinct
// loads and a reversal returns to a kept state.  Returns 1 when F is
// extrapolated.
__device__ bool same_target(const double* a, const double* b) {
  double d = 0.0, m = 0.0;
  for (int c = 0; c < 9; ++c) {
    d += (a[c] - b[c]) * (a[c] - b[c]);
    m += a[c] * a[c] + b[c] * b[c];
  }
  return d <= 1e-24 * m;
}

__device__ int quadratic_start(HistState* hs, const StepIn& row) {
  bool okF = hs->nprev >= 1, okA = hs->nprev >= 2, okB = hs->nprev >= 3;
  for (int c = 0; c < 9; ++c) {
    if (row.mask[c] != hs->mprev[c]) okF = false;
    if (row.mask[c] != hs->mprev2[c]) okA = false;
    if (row.mask[c] != hs->mprev3[c]) okB = false;
  }
  okA = okA && okF && !same_target(hs->t2, hs->t1);
  okB = okB && okF && !same_target(hs->t3, hs->t1);
  double w1 = 0.0, w2 = 0.0;
  int ex = 0;
  if (okA || okB) {
    const double* tn = okA ? hs->t2 : hs->t3;
    // (one thread: FP64 divisions are slow here, so each quotient is taken
    // once, after its sum)
    double nd = 0.0;
    for (int c = 0; c < 9; ++c) nd += (tn[c] - hs->t1[c]) * (tn[c] - hs->t1[c]);
    nd = sqrt(nd);
    double st = 0.0;
    for (int c = 0; c < 9; ++c) st += (row.target[c] - hs->t1[c]) * (tn[c] - hs->t1[c]);
    st /= nd;
    if (okA && okB) {
      double sB = 0.0, q3 = 0.0;
      for (int c = 0; c < 9; ++c) sB += (hs->t3[c] - hs->t1[c]) * (hs->t2[c] - hs->t1[c]);
      sB /= nd;
      const double sBn = sB / nd;
      for (int c = 0; c < 9; ++c) {
        const double off = (hs->t3[c] - hs->t1[c]) - sBn * (hs->t2[c] - hs->t1[c]);
        q3 += off * off;
      }
      const double sA = nd;
      const bool on_line = q3 <= 1e-20 * (sB * sB + sA * sA);
      const bool distinct = fabs(sB) > 1e-6 * sA && fabs(sB - sA) > 1e-6 * sA;
      if (on_line && distinct) {
        const double a1 = st * (st - sB) / (sA * (sA - sB));
        const double a2 = st * (st - sA) / (sB * (sB - sA));
        // far outside the three states the weights amplify their rounding
        if (fabs(1.0 - a1 - a2) + fabs(a1) + fabs(a2) <= 20.0) {
          w1 = a1;
          w2 = a2;
          ex = 1;
        }
      }
    }
    if (!ex) {
      // linear along the line through the usable slot
      if (okA) w1 = st / nd;
      else w2 = st / nd;
      ex = 1;
    }
  }
  hs->quad = ex;
  hs->w[1] = w1;
  hs->w[2] = w2;
  hs->w[0] = 1.0 - w1 - w2;
  for (int c = 0; c < 9; ++c)
    hs->pmean[c] = hs->fmean1[c] + w1 * (hs->fmean2[c] - hs->fmean1[c]) + w2 * (hs->fmean3[c] - hs->fmean1[c]);
  // the slot for the last converged state (none before the first one)
  if (hs->nprev >= 1) {
    int dst;
    if (hs->nprev < 2) dst = 0;
    else if (same_target(hs->t1, hs->t2)) dst = 0;
    else if (hs->nprev < 3) dst = 1;
    else if (same_target(hs->t1, hs->t3)) dst = 1;
    else if (same_target(row.target, hs->t2)) dst = 0;   // this step reconverges that state
    else if (same_target(row.target, hs->t3)) dst = 1;
    else dst = hs->age2 <= hs->age3 ? 0 : 1;
    hs->dst = dst;
    double* tt = dst == 0 ? hs->t2 : hs->t3;
    double* fm = dst == 0 ? hs->fmean2 : hs->fmean3;
    unsigned char* mm = dst == 0 ? hs->mprev2 : hs->mprev3;
    for (int c = 0; c < 9; ++c) {
      tt[c] = hs->t1[c];
      fm[c] = hs->fmean1[c];
      mm[c] = hs->mprev[c];
    }
    if (dst == 0) hs->age2 = hs->nseen;
    else hs->age3 = hs->nseen;
  }
  return ex;
}

// The control kernels below run their logic in one thread on a copy of the
// history state in shared memory, read and written back by a whole warp in
// parallel: the logic's many dependent accesses to the state then cost
// shared-memory latency instead of global-memory latency each.
static_assert(sizeof(HistState) % 8 == 0, "HistState is copied in 8-byte words");
template <typename Fn>
__device__ __forceinline__ void on_shared_state(HistState* hs_g, Fn fn) {
  __shared__ __align__(16) unsigned long long raw[sizeof(HistState) / 8];
  unsigned long long* g = reinterpret_cast<unsigned long long*>(hs_g);
  for (int i = threadIdx.x; i < (int)(sizeof(HistState) / 8); i += blockDim.x) raw[i] = g[i];
  __syncthreads();
  if (threadIdx.x == 0) fn(reinterpret_cast<HistState*>(raw));
  __syncthreads();
  for (int i = threadIdx.x; i < (int)(sizeof(HistState) / 8); i += blockDim.x) g[i] = raw[i];
}
constexpr int kCtlThreads = 32;

// Load step k of the table: control mask, targets, P-bar (Sec. 2.3).  With
// the extrapolating predictor and the last two converged steps at hand (same
// mask), the factor alpha of the increment: the projection of this step's
// target increment on the last one, alpha = dT_k . dT_(k-1) / abs(dT_(k-1))^2
// (1 along a ramp, -1 back across a reversal of the load); with the
// quadratic predictor, quadratic_start.  An extrapolated start is close to
// the solution: its first residual runs in the outer arithmetic (FP32
// rounding, relative to abs(P), would no longer be small against it).
__global__ void k_step_begin(HistState* hs_g, HistTables t, cudaGraphConditionalHandle h_first, int set_first) {
  on_shared_state(hs_g, [&](HistState* hs) {
    const StepIn& row = t.in[hs->k];
    if (hs->ident) {
      // the reference state as the last converged one, at this mask's zero
      // load: P-bar = 0 on the stress-controlled components, F-bar = I on the
      // strain-controlled ones (both laws give P(I) = 0)
      for (int c = 0; c < 9; ++c) {
        const double id = (c % 4 == 0) ? 1.0 : 0.0;
        hs->t1[c] = row.mask[c] ? 0.0 : id;
        hs->fmean1[c] = id;
        hs->mprev[c] = row.mask[c];
      }
      hs->ident = 0;
    }
    bool same = hs->nprev >= 2;
    for (int c = 0; c < 9; ++c) {
      const unsigned char m = row.mask[c];
      const double v = row.target[c];
      hs->mask[c] = m;
      hs->target[c] = v;
      hs->pbar[c] = m ? v : 0.0;
      if (m != hs->mprev[c]) same = false;
    }
    double num = 0.0, den = 0.0;
    for (int c = 0; c < 9; ++c) {
      const double d1 = hs->target[c] - hs->t1[c], d0 = hs->t1[c] - hs->t2[c];
      num += d1 * d0;
      den += d0 * d0;
    }
    int ex = (hs->extrap == 1 && same && den > 0.0) ? 1 : 0;
    hs->alpha = ex ? num / den : 0.0;
    hs->quad = 0;
    hs->dst = -1;
    if (hs->extrap == 2) ex = quadratic_start(hs, row);
    hs->extrapolated = ex;
    hs->nn = 0;
    hs->ncg = 0;
    hs->ratio = INFINITY;
    hs->last = 0;
    // the first residual of a step uses FP32 transforms where they exist,
    // unless the start was extrapolated
    hs->res32 = hs->dw_res && !ex;
    if (set_first) cudaGraphSetConditional(h_first, ex ? 1u : 0u);
  });
}

// Predictor of a load step (Sec. 2.1, 2.3), the forms of pred_coef: with
// the extrapolating predictor, F <- F + alpha (F - Fprev) and Fprev <- F,
// the state the next step extrapolates from; with the quadratic one (Fprev2
// given: the slots A = Fprev, B = Fprev2) the weights and the slot of
// quadratic_start; then every strain-controlled component shifted uniformly
// so that its average is the prescribed F-bar.  After an FP32 update
// (after_update) only the shift, to the averages of that update.  (A
// double-word context applies the step's predictor inside its first
// constitutive pass instead.)
__global__ void k_predictor_hist(double* __restrict__ F, PredArgs pa, long long N, const Scalars* sc,
                                 bool after_update) {
  const HistState* hs = pa.hs;
  const long long v0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, dv = (long long)gridDim.x * blockDim.x;
  if (after_update || pa.kind == 0) {
    // the strain-controlled components only
    const PredCoef k = pred_coef(pa, sc);
    for (int c = 0; c < 9; ++c) {
      if (hs->mask[c]) continue;
      const double shift = after_update ? hs->target[c] - sc->meanF_new[c] : k.sh[c];
      for (long long v = v0; v < N; v += dv) F[c * N + v] += shift;
    }
    return;
  }
  // a flat pass over the 9N values, two per step (16-byte accesses where N
  // is even; a pair never spans two components then), the coefficients in
  // shared memory; the form of predict.cuh
  __shared__ double sh[9];
  __shared__ double w12[2];
  __shared__ int dsts;
  if (threadIdx.x == 0) {
    const PredCoef k = pred_coef(pa, sc);
    for (int c = 0; c < 9; ++c) sh[c] = k.sh[c];
    w12[0] = k.v1;
    w12[1] = k.v2;
    dsts = k.dst;
  }
  __syncthreads();
  const double v1 = w12[0], v2 = w12[1];
  const int dst = dsts;
  double* __restrict__ A = pa.A;
  double* __restrict__ B = pa.B;
  auto one = [&](double f, double a, double b, int c) {
    double fn = f;
    if (v1 != 0.0) fn += v1 * (a - f);
    if (v2 != 0.0) fn += v2 * (b - f);
    return fn + sh[c];
  };
  const long long n9 = 9 * N;
  if ((N & 1) == 0) {
    double2* __restrict__ F2 = reinterpret_cast<double2*>(F);
    double2* __restrict__ A2 = reinterpret_cast<double2*>(A);
    double2* __restrict__ B2 = reinterpret_cast<double2*>(B);
    for (long long q = v0; q < n9 / 2; q += dv) {
      const int c = (int)((2 * q) / N);
      const double2 f = F2[q];
      const double2 a = v1 != 0.0 ? A2[q] : make_double2(0.0, 0.0);
      const double2 b = v2 != 0.0 ? B2[q] : make_double2(0.0, 0.0);
      if (dst == 0) A2[q] = f;
      else if (dst == 1) B2[q] = f;
      F2[q] = make_double2(one(f.x, a.x, b.x, c), one(f.y, a.y, b.y, c));
    }
  } else {
    for (long long i = v0; i < n9; i += dv) {
      const int c = (int)(i / N);
      const double f = F[i];
      const double a = v1 != 0.0 ? A[i] : 0.0;
      const double b = v2 != 0.0 ? B[i] : 0.0;
      if (dst == 0) A[i] = f;
      else if (dst == 1) B[i] = f;
      F[i] = one(f, a, b, c);
    }
  }
}

// Before a Newton iteration: failures of the constitutive pass end the
// history; the iteration cap; the null rotations of the FP32 inner solves
// (from T and S of that pass); the forcing of the inner solve: sqrt(cg_rel)
// for the first iteration of a step and for one whose predecessor's
// correction was below sqrt(tol_newton), cg_rel otherwise.
__global__ void k_newton_pre(HistState* hs_g, const Scalars* sc, cudaGraphConditionalHandle h_go,
                             cudaGraphConditionalHandle h_newton, int first) {
  on_shared_state(hs_g, [&](HistState* hs) {
    int st = flags_to_status(sc->flags);
    if (!st && hs->nn >= hs->max_newton) st = MF_NOT_CONVERGED;
    if (st) {
      if (!hs->status) hs->status = st;
      cudaGraphSetConditional(h_go, 0u);
      cudaGraphSetConditional(h_newton, 0u);
      return;
    }
    hs->defl.m = 0;
    if (hs->f32) null_rotations_dev(sc->meanF, hs->mask, sc->T, sc->S, hs->kappa, 1e-6, &hs->defl);
    // the first iteration of an extrapolated step is expected to be followed
    // by one more only: its solve need only leave the next correction below
    // the Newton tolerance.  Its correction is about the larger of the last two
    // steps' first ones (r; two, because the step across a load reversal
    // starts exact and its first correction says nothing about the next), and
    // the next about eta r, so eta = 0.1 tol_newton / r (the choice of
    // forcing terms of inexact Newton methods from the expected convergence),
    // at least cg_rel.  Its upper bound matters when r is below tol_newton and
    // the step ends on this correction: the step leaves an error of about eta
    // times its start's error, and the start carries the kept states' errors
    // with the gain sum abs(w) of the extrapolation (7 for the quadratic one
    // along a ramp: w = 3, -3, 1), so the states' errors evolve as e' = eta
    // (tau + sum abs(w) e), tau the extrapolation's own error.  The bound
    // 0.25 / sum abs(w) holds that gain to 1/4 (errors from earlier steps
    // shrink fourfold per step, and e settles near 1.3 eta tau); it is kept
    // within [sqrt(cg_rel), 0.1], 0.1 keeping the computed correction, whose
    // size the Newton test reads, within about 10 %.
    const bool loose = (first && !hs->extrapolated) || hs->ratio < sqrt(hs->tol_newton);
    double eta = loose ? sqrt(hs->cg_rel) : hs->cg_rel;
    const double r = fmax(hs->first_ratio, hs->first_ratio2);
    hs->eta_hi = 0.0;
    if (first && hs->extrapolated && r > 0.0 && isfinite(r)) {
      const double gain = hs->quad ? fabs(hs->w[0]) + fabs(hs->w[1]) + fabs(hs->w[2])
                                   : 1.0 + 2.0 * fabs(hs->alpha);
      const double hi = fmax(sqrt(hs->cg_rel), fmin(0.1, 0.25 / fmax(gain, 1.0)));
      eta = fmin(hi, fmax(hs->cg_rel, 0.1 * hs->tol_newton / r));
      // refined at the CG start from this step's own first residual (k_fin_cg_init_h)
      hs->eta_hi = hi;
    }
    hs->cg_rel_cur = hs->forcing ? eta : 0.0;
    cudaGraphSetConditional(h_go, 1u);
  });
}

// Projection of the FP32 correction onto the range of G* before the update:
// 0 none (a late correction below 1e-6 of F, after one that small; or the
// first correction of an extrapolated step expected below kProjSkipBelow of
// F: the FP32 rounding outside range(G*), about 1e-5 of a correction, is
// then below 1e-13 of F), 1 FP32 transforms, 2 outer arithmetic
// (MF_PROJ_OUTER, or MF_PROJ_AUTO for a correction expected to be at least
// kProjOuterAbove of F).
constexpr double kProjSkipBelow = 1e-8;
__global__ void k_proj_decide(HistState* hs_g, cudaGraphConditionalHandle h_proj, int first) {
  on_shared_state(hs_g, [&](HistState* hs) {
    const int nn = hs->nn;
    const double ratio = hs->ratio;
    const bool outer =
        hs->proj_arith == MF_PROJ_OUTER ||
        (hs->proj_arith == MF_PROJ_AUTO &&
         (first ? !(hs->first_ratio < kProjOuterAbove) : !(ratio < 10.0 * kProjOuterAbove)));
    const bool tiny_first = first && hs->extrapolated && hs->proj_arith != MF_PROJ_OUTER &&
                            fmax(hs->first_ratio, hs->first_ratio2) < kProjSkipBelow;
    const bool project = !tiny_first && (outer || nn < 2 || !(ratio < 1e-6));
    const int kind = !project ? 0 : (outer ? 2 : 1);
    hs->proj_kind = kind;
    cudaGraphSetConditional(h_proj, (unsigned)kind);
  });
}

// After the update: the outcome of the inner solve (an FP32 inner solve that
// ended on a direction of non-positive curvature after some progress ends
// without failing: its flag is cleared), the iteration counts, the size of
// the correction and the Newton stop test (Sec. 4: max_v abs(dF_v) /
// abs(<F>) < tol_newton; never on a correction from the FP32 residual of a
// step's first iteration).  Then the pass that follows: P alone (the step
// ends), or P with what the next iteration needs and the next residual in
// the outer arithmetic.  (FP32 residuals later in a step were tried: their
// rounding, relative to abs(P), is no longer small against the shrinking
// residual, and the 128^3 polycrystal needed a fourth Newton iteration per
// step.)
__global__ void k_newton_post(HistState* hs_g, Scalars* sc, cudaGraphConditionalHandle h_cons) {
  on_shared_state(hs_g, [&](HistState* hs) {
    int flags = sc->flags;
    if (hs->f32 && (flags & MF_FLAG_BREAKDOWN) && !(flags & ~MF_FLAG_BREAKDOWN) && sc->its > 1) {
      sc->flags = 0;
      flags = 0;
    }
    int st = flags_to_status(flags);
    if (!st && !sc->done) st = MF_NOT_CONVERGED;
    hs->ncg += sc->its;
    double fn = 0.0;
    for (int q = 0; q < 9; ++q) fn += sc->meanF_new[q] * sc->meanF_new[q];
    const double ratio = sqrt(sc->dF2max) / sqrt(fn);
    hs->ratio = ratio;
    hs->nn += 1;
    if (hs->nn == 1) {
      hs->first_ratio2 = hs->first_ratio;
      hs->first_ratio = ratio;
      if (hs->rms0 > 0.0 && isfinite(ratio)) {
        hs->kr2 = hs->kr1;
        hs->kr1 = ratio / hs->rms0;
      }
    }
    if (st && !hs->status) hs->status = st;
    const int last = (ratio < hs->tol_newton && !hs->res32) ? 1 : 0;
    // a step that ends on an FP32 correction applied as computed (no
    // projection, no deflation), with more steps to come in this launch:
    // <P> at the final F from the linearisation, <P(F)> + <K:dF>; the error,
    // of the order of abs(K') abs(dF)^2 with abs(dF) < tol_newton abs(F), is
    // far below the averages' accuracy.  <K:dF> = sum_k alpha_k <K:p_k>, the
    // solve's z-passes having added each iteration's term to sc->lin (the
    // null-frequency coefficient of K:p_k), so no pass over the fields runs
    // (kind 2: no body).  The last step of a launch evaluates P, so the
    // fields a caller reads are exact.
    const bool lin = last && hs->f32 && hs->proj_kind == 0 && hs->defl.m == 0 && hs->k + 1 < hs->nsteps;
    const int kind = last ? (lin ? 2 : 0) : 1;
    if (lin) {
      // the update's averages as they are: the strain-controlled ones differ
      // from F-bar by the rounding of the FP32 correction's average (far below
      // 1e-14 of F for a correction below tol_newton); the next step's
      // predictor, which shifts F by F-bar minus these, removes it
      for (int c = 0; c < 9; ++c) {
        sc->meanP[c] += sc->lin[c];
        sc->meanF[c] = sc->meanF_new[c];
      }
    }
    hs->last = last;
    hs->res32 = 0;
    hs->cons_kind = kind;
    cudaGraphSetConditional(h_cons, (unsigned)kind);
  });
}

// After the constitutive pass that follows an update: its failures, the
// launch count of the iteration, and whether another Newton iteration runs.
__global__ void k_newton_cond(HistState* hs_g, const Scalars* sc, cudaGraphConditionalHandle h_newton,
                              IterCounts cnt) {
  on_shared_state(hs_g, [&](HistState* hs) {
    const int st = flags_to_status(sc->flags);
    if (st && !hs->status) hs->status = st;
    const int its = sc->its;
    hs->launches += cnt.fixed + cnt.proj[hs->proj_kind] + cnt.cons[hs->cons_kind] +
                    (long long)cnt.cg_body * (its == 0 ? 1 : (its + 1) / 2);
    cudaGraphSetConditional(h_newton, (!hs->last && !hs->status) ? 1u : 0u);
  });
}

// End of a load step: record <F>, <P> (Sec. 2.2) and the iteration counts;
// continue with the next step unless the history failed.
__global__ void k_step_end(HistState* hs_g, const Scalars* sc, HistTables t, cudaGraphConditionalHandle h_step,
                           int kernels, int kernels_ex) {
  on_shared_state(hs_g, [&](HistState* hs) {
    hs->launches += hs->extrapolated ? kernels_ex : kernels;
    if (!hs->status) {
      const int k = hs->k;
      // the converged step joins the states the predictor extrapolates from
      // (the quadratic predictor's slots were filled at the step's start)
      for (int c = 0; c < 9; ++c) {
        if (hs->extrap != 2) {
          hs->t2[c] = hs->t1[c];
          hs->fmean2[c] = hs->fmean1[c];
        }
        hs->t1[c] = hs->target[c];
        hs->fmean1[c] = sc->meanF[c];
        hs->mprev[c] = hs->mask[c];
      }
      hs->nprev = hs->nprev < 3 ? hs->nprev + 1 : 3;
      hs->nseen += 1;
      StepOut& row = t.out[k];
      for (int c = 0; c < 9; ++c) {
        row.Fbar[c] = sc->meanF[c];
        row.Pbar[c] = sc->meanP[c];
      }
      row.newton = hs->nn;
      row.cg = hs->ncg;
      hs->k = k + 1;
    }
    cudaGraphSetConditional(h_step, (!hs->status && hs->k < hs->nsteps) ? 1u : 0u);
  });
}

// Start of a CG loop inside a history graph: counters reset and the loop's
// condition set explicitly (skipped at once when the start already met the
// tolerance or a flag is up).
__global__ void k_cg_start_h(Scalars* sc, int max_its, cudaGraphConditionalHandle h_cg) {
  sc->its = 0;
  sc->arrive = 0u;
  sc->max_its = max_its;
  const int stop = (sc->done || sc->flags) ? 1 : 0;
  sc->stop = stop;
  cudaGraphSetConditional(h_cg, stop ? 0u : 1u);
}

// ------------------------------------------------------------ pass variants
// CG start (r = b in the inner type, r.r) with the tolerance and forcing of
// the current iteration: stop at rms(r) <= max(tol_cg, cg_rel_cur * rms(r0)).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_init_h(const double* __restrict__ b, T* __restrict__ r,
                                                        long long n9, double* __restrict__ partials) {
  __shared__ double red[kThreads / 32];
  double acc = 0.0;
  float fs = 0.f, fc = 0.f;
  // r = b rounded to FP32, r.r as a Neumaier-compensated FP32 sum of the
  // exact squares (square and its FMA error)
  auto put = [&](float v) {
    const float pr = v * v;
    const float e = fmaf(v, v, -pr);
    float t = fs + pr;
    fc += (fabsf(fs) >= fabsf(pr)) ? ((fs - t) + pr) : ((pr - t) + fs);
    fs = t;
    t = fs + e;
    fc += (fabsf(fs) >= fabsf(e)) ? ((fs - t) + e) : ((e - t) + fs);
    fs = t;
  };
  auto rnd = [](double x) {
    const dw d = dw_split(x);
    return __fadd_rn(d.hi, d.lo);
  };
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, di = (long long)gridDim.x * blockDim.x;
  long long head = 0;
  if constexpr (sizeof(T) == 4) {
    // four elements per step with 16-byte accesses where the buffers allow
    if ((((uintptr_t)b | (uintptr_t)r) & 15) == 0) {
      head = n9 & ~3LL;
      const double2* b2 = reinterpret_cast<const double2*>(b);
      float4* r4 = reinterpret_cast<float4*>(r);
      for (long long q = i0; q < head / 4; q += di) {
        const double2 u = b2[2 * q], w = b2[2 * q + 1];
        const float4 v = make_float4(rnd(u.x), rnd(u.y), rnd(w.x), rnd(w.y));
        r4[q] = v;
        put(v.x);
        put(v.y);
        put(v.z);
        put(v.w);
      }
    }
  }
  for (long long i = head + i0; i < n9; i += di) {
    if constexpr (sizeof(T) == 4) {
      const float v = rnd(b[i]);
      r[i] = v;
      put(v);
    } else {
      const T v = (T)b[i];
      r[i] = v;
      acc += (double)v * (double)v;
    }
  }
  if constexpr (sizeof(T) == 4) acc = (double)fs + (double)fc;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

// CG start: r.r, the stop threshold rms(r) <= max(tol_cg, eta rms(r0)).  At
// a step's first Newton iteration rms(r0) is recorded; for an extrapolated
// step's first solve eta is refined from it: the first correction relative
// to F has been close to k rms(r0) with the same k from step to step (k
// reflects the operator's stiffness, not the quality of the start), so the
// expected correction is r = 2 max(k of the last two steps) rms(r0) (2 a
// margin) and eta = 0.1 tol_newton / r within the bounds of k_newton_pre.
// This follows a change of the predictor's order (uniform, then linear,
// then quadratic on a history's first steps), which the last steps' first
// corrections alone do not see.  Too loose an eta costs at most one more
// Newton iteration: a step ends only on a correction below tol_newton, and
// the error it leaves is below eta tol_newton.
__global__ void __launch_bounds__(kThreads) k_fin_cg_init_h(const double* __restrict__ partials, int npart,
                                                            long long N, HistState* hs, Scalars* sc) {
  __shared__ double shm[kThreads];
  double s = 0.0;
  for (int b = threadIdx.x; b < npart; b += kThreads) s += partials[b];
  shm[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) shm[threadIdx.x] += shm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double rr = shm[0];
    sc->rr = rr;
    sc->rr0 = rr;
    sc->alpha = 0.0;
    sc->beta = 0.0;
    for (int c = 0; c < 9; ++c) sc->lin[c] = 0.0;
    const double rms = sqrt(rr / (double)N);
    if (hs->nn == 0) hs->rms0 = rms;
    if (hs->eta_hi > 0.0 && hs->cg_rel_cur > 0.0) {
      const double k = fmax(hs->kr1, hs->kr2);
      if (k > 0.0 && isfinite(k) && rms > 0.0) {
        const double r = 2.0 * k * rms;
        hs->cg_rel_cur = fmin(hs->eta_hi, fmax(hs->cg_rel, 0.1 * hs->tol_newton / r));
      }
    }
    double thr = hs->tol_cg;
    if (hs->cg_rel_cur > 0.0) thr = fmax(hs->tol_cg, hs->cg_rel_cur * rms);
    sc->thr2N = thr * thr * (double)N;
    sc->done = (rr <= sc->thr2N) ? 1 : 0;
  }
}

// B = sum_v y_v F_v^T (n_k . y = W_k : B); nothing when no rotation is null.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_defl_reduce_h(const T* __restrict__ y, const double* __restrict__ F,
                                                            long long N, const HistState* hs,
                                                            double* __restrict__ partials) {
  if (hs->defl.m == 0) return;
  __shared__ double red[9][kThreads / 32];
  double acc[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) acc[c] = 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    double f[9], q[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) { f[c] = F[c * N + v]; q[c] = (double)y[c * N + v]; }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        acc[3 * i + j] += q[3 * i] * f[3 * j] + q[3 * i + 1] * f[3 * j + 1] + q[3 * i + 2] * f[3 * j + 2];
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    double s = acc[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = s;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[threadIdx.x][w];
    partials[blockIdx.x * 9 + threadIdx.x] = s;
  }
}

// What = sum_k (n_k . y) W_k (zero when no rotation is null).
__global__ void __launch_bounds__(kThreads) k_defl_fin_h(const double* __restrict__ partials, int nblk,
                                                         const HistState* hs, Scalars* sc) {
  const Defl& d = hs->defl;
  if (d.m == 0) {
    if (threadIdx.x < 9) sc->What[threadIdx.x] = 0.0;
    return;
  }
  __shared__ double shm[kThreads];
  __shared__ double B[9];
  for (int col = 0; col < 9; ++col) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += kThreads) s += partials[(long long)b * 9 + col];
    shm[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) shm[threadIdx.x] += shm[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) B[col] = shm[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double W[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < d.m; ++k) {
      double ck = 0.0;
      for (int t = 0; t < 9; ++t) ck += d.W[k][t] * B[t];
      for (int t = 0; t < 9; ++t) W[t] += ck * d.W[k][t];
    }
    for (int t = 0; t < 9; ++t) sc->What[t] = W[t];
  }
}

template <typename T>
__global__ void k_defl_apply_h(T* __restrict__ y, const double* __restrict__ F, long long N, const HistState* hs,
                               const Scalars* sc) {
  if (hs->defl.m == 0) return;
  double W[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) W[t] = sc->What[t];
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    double f[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) f[c] = F[c * N + v];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double corr = W[3 * i] * f[j] + W[3 * i + 1] * f[3 + j] + W[3 * i + 2] * f[6 + j];
        y[(3 * i + j) * N + v] = (T)((double)y[(3 * i + j) * N + v] - corr);
      }
  }
}

// F += x (minus What F when a rotation is null).  Partials: columns 0-8 the
// sums of the applied correction, column 9 the block max of abs(dF_v)^2.
// An FP32 correction without deflation is widened exactly and summed with
// Neumaier-compensated FP32 sums (no FP64 arithmetic per element).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_newton_update_h(double* __restrict__ F, const T* __restrict__ x,
                                                              long long N, double* __restrict__ partials,
                                                              const HistState* hs, const Scalars* sc) {
  __shared__ double red[11][kThreads / 32];
  const bool defl = hs->defl.m > 0;
  if (sizeof(T) == 4 && !defl) return;   // k_newton_update_f32_h
  double acc[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) acc[c] = 0.0;
  float xs[9], xc[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) { xs[c] = 0.f; xc[c] = 0.f; }
  double mx = 0.0;
  double W[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) W[t] = defl ? sc->What[t] : 0.0;
  if (defl || sizeof(T) == 8) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
      double f[9], d[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) { f[c] = F[c * N + v]; d[c] = (double)x[c * N + v]; }
      if (defl) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            d[3 * i + j] -= W[3 * i] * f[j] + W[3 * i + 1] * f[3 + j] + W[3 * i + 2] * f[6 + j];
      }
      double n2 = 0.0;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        F[c * N + v] = f[c] + d[c];
        acc[c] += d[c];
        n2 += d[c] * d[c];
      }
      mx = fmax(mx, n2);
    }
  } else {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
      float n2 = 0.f;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const float d = (float)x[c * N + v];
        F[c * N + v] = F[c * N + v] + f32_as_f64(d);
        const float tt = xs[c] + d;
        xc[c] += (fabsf(xs[c]) >= fabsf(d)) ? ((xs[c] - tt) + d) : ((d - tt) + xs[c]);
        xs[c] = tt;
        n2 = fmaf(d, d, n2);
      }
      mx = fmax(mx, (double)n2);
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] = (double)xs[c] + (double)xc[c];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    double s = acc[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[c][warp] = s;
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[9][warp] = mx;
  __syncthreads();
  if (threadIdx.x < 9) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[threadIdx.x][w];
    partials[blockIdx.x * 10 + threadIdx.x] = s;
  } else if (threadIdx.x == 9) {
    double m = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) m = fmax(m, red[9][w]);
    partials[blockIdx.x * 10 + 9] = m;
  }
}

// The common case of k_newton_update_h on its own: an FP32 correction
// without deflation (the other kernel returns at once then, and this one
// otherwise).  Few registers, so that enough voxels' loads are in flight for
// a pass bound by HBM; same partials.
// With p0 (the CG directions' buffers) the solve's last lagging update is
// taken here instead of in x: dF = x + alpha p (the arithmetic of
// k_axpy_last), or 0 when no CG iteration ran.
__global__ void __launch_bounds__(kThreads, 3) k_newton_update_f32_h(double* __restrict__ F,
                                                                     const float* __restrict__ x,
                                                                     const float* __restrict__ p0,
                                                                     const float* __restrict__ p1, long long N,
                                                                     double* __restrict__ partials,
                                                                     const HistState* hs, const Scalars* sc) {
  if (hs->defl.m > 0) return;
  const int its = p0 ? sc->its : -1;
  const float* __restrict__ p = (its > 0) ? ((its & 1) ? p1 : p0) : nullptr;
  const float a = p ? (float)sc->alpha : 0.f;
  __shared__ double red[11][kThreads / 32];
  float xs[9], xc[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) { xs[c] = 0.f; xc[c] = 0.f; }
  float mx = 0.f;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    float d[9];
    double f[9];
    if (its == 0) {
#pragma unroll
      for (int c = 0; c < 9; ++c) { d[c] = 0.f; f[c] = F[c * N + v]; }
    } else if (p) {
      float q[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) { d[c] = x[c * N + v]; q[c] = p[c * N + v]; f[c] = F[c * N + v]; }
#pragma unroll
      for (int c = 0; c < 9; ++c) d[c] += a * q[c];
    } else {
#pragma unroll
      for (int c = 0; c < 9; ++c) { d[c] = x[c * N + v]; f[c] = F[c * N + v]; }
    }
    float n2 = 0.f;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      F[c * N + v] = f[c] + f32_as_f64(d[c]);
      const float tt = xs[c] + d[c];
      xc[c] += (fabsf(xs[c]) >= fabsf(d[c])) ? ((xs[c] - tt) + d[c]) : ((d[c] - tt) + xs[c]);
      xs[c] = tt;
      n2 = fmaf(d[c], d[c], n2);
    }
    mx = fmaxf(mx, n2);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    double sv = (double)xs[c] + (double)xc[c];
    for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
    if (lane == 0) red[c][warp] = sv;
  }
  double m = (double)mx;
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) red[9][warp] = m;
  __syncthreads();
  if (threadIdx.x < 9) {
    double sv = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) sv += red[threadIdx.x][w];
    partials[blockIdx.x * 10 + threadIdx.x] = sv;
  } else if (threadIdx.x == 9) {
    double mm = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) mm = fmax(mm, red[9][w]);
    partials[blockIdx.x * 10 + 9] = mm;
  }
}

// The solve's last lagging update x += alpha p (k_axpy_last) for an FP32
// correction that is deflated before the update (k_newton_update_h reads
// x); without deflation k_newton_update_f32_h takes it on the fly.
__global__ void k_axpy_last_defl_h(float* __restrict__ x, const float* __restrict__ p0,
                                   const float* __restrict__ p1, long long n, const HistState* hs,
                                   const Scalars* sc) {
  if (hs->defl.m == 0) return;
  const int its = sc->its;
  const float* p = (its & 1) ? p1 : p0;
  const float a = (float)sc->alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (its == 0) x[i] = 0.f;
    else x[i] += a * p[i];
  }
}

// Columns 0-8: the new averages; column 9: max abs(dF_v)^2 (grid 10).
__global__ void __launch_bounds__(kThreads) k_fin_newton_h(const double* __restrict__ partials, int nblk,
                                                           long long N, Scalars* sc) {
  __shared__ double shm[kThreads];
  const int col = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kThreads) {
    const double v = partials[(long long)b * 10 + col];
    s = (col < 9) ? s + v : fmax(s, v);
  }
  shm[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      shm[threadIdx.x] = (col < 9) ? shm[threadIdx.x] + shm[threadIdx.x + w] : fmax(shm[threadIdx.x], shm[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (col < 9) {
      sc->meanF_new[col] = sc->meanF[col] + shm[0] / (double)N;
    } else {
      sc->dF2max = shm[0];
      if (!isfinite(shm[0])) atomicOr(&sc->flags, MF_FLAG_NONFINITE);
    }
  }
}

}  // namespace

cudaError_t mf_launch_hist_init(HistState* hs, cudaGraphConditionalHandle h_step, int kernels, cudaStream_t st) {
  k_hist_init<<<1, 1, 0, st>>>(hs, h_step, kernels);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_step_begin(HistState* hs, HistTables t, cudaGraphConditionalHandle* h_first, cudaStream_t st) {
  k_step_begin<<<1, kCtlThreads, 0, st>>>(hs, t, h_first ? *h_first : cudaGraphConditionalHandle(), h_first ? 1 : 0);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_predictor_hist(double* F, double* Fprev, double* Fprev2, long long N, const HistState* hs,
                                     const Scalars* sc, bool after_update, cudaStream_t st) {
  const PredArgs pa{Fprev, Fprev2, hs, Fprev2 ? 2 : (Fprev ? 1 : 0)};
  k_predictor_hist<<<grid_for(N), kThreads, 0, st>>>(F, pa, N, sc, after_update);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_newton_pre(HistState* hs, const Scalars* sc, cudaGraphConditionalHandle h_go,
                                 cudaGraphConditionalHandle h_newton, bool first, cudaStream_t st) {
  k_newton_pre<<<1, kCtlThreads, 0, st>>>(hs, sc, h_go, h_newton, first ? 1 : 0);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_proj_decide(HistState* hs, cudaGraphConditionalHandle h_proj, bool first, cudaStream_t st) {
  k_proj_decide<<<1, kCtlThreads, 0, st>>>(hs, h_proj, first ? 1 : 0);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_newton_post(HistState* hs, Scalars* sc, cudaGraphConditionalHandle h_cons, cudaStream_t st) {
  k_newton_post<<<1, kCtlThreads, 0, st>>>(hs, sc, h_cons);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_newton_cond(HistState* hs, const Scalars* sc, cudaGraphConditionalHandle h_newton,
                                  IterCounts cnt, cudaStream_t st) {
  k_newton_cond<<<1, kCtlThreads, 0, st>>>(hs, sc, h_newton, cnt);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_step_end(HistState* hs, const Scalars* sc, HistTables t, cudaGraphConditionalHandle h_step,
                               int kernels, int kernels_ex, cudaStream_t st) {
  k_step_end<<<1, kCtlThreads, 0, st>>>(hs, sc, t, h_step, kernels, kernels_ex);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_cg_init_hist(const double* b, void* r, bool f32, long long n9, double* partials, int nblk,
                                   long long N, HistState* hs, Scalars* sc, cudaStream_t st) {
  if (f32) k_cg_init_h<float><<<nblk, kThreads, 0, st>>>(b, (float*)r, n9, partials);
  else k_cg_init_h<double><<<nblk, kThreads, 0, st>>>(b, (double*)r, n9, partials);
  k_fin_cg_init_h<<<1, kThreads, 0, st>>>(partials, nblk, N, hs, sc);
  g_mf_launches += 2;
  return cudaGetLastError();
}

cudaError_t mf_launch_defl_project_hist(void* y, bool f32, bool apply, const double* F, long long N,
                                        const HistState* hs, double* partials, int nblk, Scalars* sc,
                                        cudaStream_t st) {
  if (f32) k_defl_reduce_h<float><<<nblk, kThreads, 0, st>>>((const float*)y, F, N, hs, partials);
  else k_defl_reduce_h<double><<<nblk, kThreads, 0, st>>>((const double*)y, F, N, hs, partials);
  k_defl_fin_h<<<1, kThreads, 0, st>>>(partials, nblk, hs, sc);
  g_mf_launches += 2;
  if (apply) {
    // a grid of a few blocks per SM: the pass usually returns at once (no
    // null rotation), and launching a full grid of empty blocks costs time
    if (f32) k_defl_apply_h<float><<<rare_grid(N), kThreads, 0, st>>>((float*)y, F, N, hs, sc);
    else k_defl_apply_h<double><<<rare_grid(N), kThreads, 0, st>>>((double*)y, F, N, hs, sc);
    g_mf_launches += 1;
  }
  return cudaGetLastError();
}

cudaError_t mf_launch_newton_update_hist(double* F, const void* x, bool f32, long long N, double* partials,
                                         int nblk, const HistState* hs, Scalars* sc, cudaStream_t st,
                                         const void* p0, const void* p1) {
  // one wave of the update kernels (at most three blocks per SM resident)
  nblk = nblk < 3 * 152 ? nblk : 3 * 152;
  if (f32) {
    k_newton_update_h<float><<<nblk, kThreads, 0, st>>>(F, (const float*)x, N, partials, hs, sc);
    k_newton_update_f32_h<<<nblk, kThreads, 0, st>>>(F, (const float*)x, (const float*)p0, (const float*)p1, N,
                                                    partials, hs, sc);
    g_mf_launches += 1;
  } else {
    k_newton_update_h<double><<<nblk, kThreads, 0, st>>>(F, (const double*)x, N, partials, hs, sc);
  }
  k_fin_newton_h<<<10, kThreads, 0, st>>>(partials, nblk, N, sc);
  g_mf_launches += 2;
  return cudaGetLastError();
}

cudaError_t mf_launch_axpy_last_defl_hist(float* x, const float* p0, const float* p1, long long n,
                                          const HistState* hs, const Scalars* sc, cudaStream_t st) {
  k_axpy_last_defl_h<<<rare_grid(n), kThreads, 0, st>>>(x, p0, p1, n, hs, sc);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_cg_start_hist(Scalars* sc, int max_its, cudaGraphConditionalHandle h_cg, cudaStream_t st) {
  k_cg_start_h<<<1, 1, 0, st>>>(sc, max_its, h_cg);
  g_mf_launches += 1;
  return cudaGetLastError();
}
