// Argument blocks and host-side launchers shared by the library's
// translation units (host code only; no torch types).
#pragma once

#include <utility>

#include "common.cuh"

// Launch k<<<g, b, sm, st>>>(args...), with the programmatic
// stream-serialization attribute when pdl is set (the kernel then calls
// pdl_wait() before it touches anything its predecessor writes).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 g, dim3 b, size_t sm, cudaStream_t st, Args&&... args) {
  if (!pdl) {
    k<<<g, b, sm, st>>>(std::forward<Args>(args)...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

struct XYArgs {
  int v2;          // 1: fixed-size kernels (transform2*.cu), tables of that layout
  int split;       // with v2: separate row (x) and column (y) kernels (transform3.cuh)
  const int* skip; // if non-null and *skip != 0 the kernel returns at once (finished CG)
  int fin;         // fused (v2, not split) inverse pass with the CG update: finish beta in its last block
  int pdl;         // v2 fused kernels: launch with programmatic dependent launch (see launch_k)
  int persist;     // FP32 v2 forward pass as the persistent bulk-copy kernel (k_xyf_p)
  int cluster_f;   // FP32 v2 forward pass (nx = 128) as the two-CTA cluster kernel (k_xyf_c)
  int cluster_i;   // FP32 v2 inverse pass (nx = 128) as the two-CTA cluster kernel (k_xyi_c)
  int* flags;      // device flags word (MF_FLAG_TIMEOUT from bounded waits), or null
  int nx, ny, nz;
  long long N;
  AxisPlan px;     // length nx
  AxisPlan pyh;    // length ny/2 (the y transform after its first radix-2 stage)
  const void* twx; // W_nx^t, t < nx   (complex of the kernel's type)
  const void* twy; // W_ny^t, t < ny
  const int* xpos; // position of x-frequency k after the x DIF, k < nx
};

struct ZArgs {
  int v2;
  const int* skip;
  int pdl;           // v2 kernels: launch with programmatic dependent launch (see launch_k)
  int nx, ny, nz;
  long long N;
  AxisPlan pz;
  const void* twz;   // W_nz^t
  const int* xk;     // slot -> kx
  const int* xe;     // slot -> parity e
  const int* yk;     // row q' -> ky half index
  const int* zk;     // position -> kz
  int S;             // columns per block
  unsigned mask;     // bit c set: component c stress controlled
  double scale;      // multiplies every coefficient (1/N, or -1/N for the residual)
  double add[9];     // added at the null frequency after scaling (residual: P-bar)
  double* mean_out;  // residual: receives the null-frequency coefficient / N
  const double* add_dev;  // if non-null: the values to add, read on the device (replaces add)
  double* lin;            // operator in a CG iteration: lin[c] += *lin_alpha * (null-frequency coefficient / N)
  const double* lin_alpha;
};

// Process-wide count of kernel launches issued by the library.
extern long long g_mf_launches;

// transform2_f32.cu / transform2_f64.cu: fixed-size kernels for square x-y
// planes nx = ny and nx, nz in {16, 32, 48, 64, 96, 128}.  Their spectrum layout:
// per (c, z) ny rows (digit-reversed ky, yk table of ny entries) of nx/2 slots
// (digit-reversed kx, xk table of nx/2 entries), xpos = slot of kx.
bool mf_v2_supported(int nx, int ny, int nz);
// the split row/column x-y kernels exist for these plane sizes (nx = ny)
bool mf_split_supported(int nx);
// the persistent FP32 forward kernel exists for these plane sizes (nx = ny)
bool mf_persist_supported(int nx);
// the two-CTA cluster FP32 x-y kernels exist for these plane sizes (nx = ny)
bool mf_cluster_supported(int nx);
// x-y kernel blocks of one pass, i.e. the block partials the inverse pass
// writes (one per (c, z) plane fused, one per row block split)
int mf_xy_blocks(int ny, int nz, bool split);
cudaError_t mf_v2_xyf_f32(const void* in, void* spec, const XYArgs& a, cudaStream_t st);
cudaError_t mf_v2_xyi_f32(int mode, const void* spec, void* out, double* partials, const XYArgs& a,
                          const Scalars* sc, cudaStream_t st);
cudaError_t mf_v2_zp_f32(int mode, void* spec, const ZArgs& a, cudaStream_t st);
cudaError_t mf_v2_xyf_f64(const void* in, void* spec, const XYArgs& a, cudaStream_t st);
cudaError_t mf_v2_xyi_f64(int mode, const void* spec, void* out, double* partials, const XYArgs& a,
                          const Scalars* sc, cudaStream_t st);
cudaError_t mf_v2_zp_f64(int mode, void* spec, const ZArgs& a, cudaStream_t st);

// transform2_f32.cu: one block waits, at most max_polls polls, on a barrier
// nothing arrives at, and sets MF_FLAG_TIMEOUT in *flags (device int)
cudaError_t mf_launch_wait_selftest(int max_polls, int* flags, cudaStream_t st);

// transform2_dw.cu: the residual transforms in double-word FP32 arithmetic
// (P in, b out in FP64; spectrum and twiddle tables double-word complex)
cudaError_t mf_v2_xyf_dw(const double* in, void* spec, const XYArgs& a, cudaStream_t st);
cudaError_t mf_v2_zp_dw(void* spec, const ZArgs& a, cudaStream_t st);
cudaError_t mf_v2_xyi_dw(const void* spec, double* out, double* partials, const XYArgs& a, cudaStream_t st);

// transform.cu
// b = -G*(P - P-bar) (null frequency per za); dw: double-word transforms
// (fixed-size kernels only; xa, za then point at the double-word tables).
// The generic kernels also leave block partial sums of b.b in partials; the
// fixed-size ones do not (nothing reads them).
cudaError_t mf_launch_residual(const double* P, void* spec, double* b, double* partials,
                               const XYArgs& xa, const ZArgs& za, bool dw, cudaStream_t st);
// The same residual with FP32 transforms (fixed-size kernels; xa, za with the
// FP32 tables): P rounded into Pf (P null: Pf already holds P in FP32), b
// through bf, both 9N floats of scratch.  Accurate to FP32 relative to
// abs(P): for residuals far from convergence.
cudaError_t mf_launch_residual_f32(const double* P, float* Pf, void* spec, float* bf, double* b,
                                   const XYArgs& xa, const ZArgs& za, cudaStream_t st);
// which: 0 x-y forward of t, 1 z-pass, 2 x-y inverse with the CG residual update
cudaError_t mf_launch_project_part(int which, bool f32, const void* t, void* spec, void* r,
                                   double* partials, const XYArgs& xa, const ZArgs& za,
                                   const Scalars* sc, cudaStream_t st);
// y = G*(t): x-y forward of t, z-pass, x-y inverse.  inv_mode 0 stores y in
// out; 3 performs the CG update out -= alpha y (alpha in sc) and writes the
// block partials of out.out.
cudaError_t mf_launch_project(bool f32, const void* t, void* spec, void* out, int inv_mode,
                              double* partials, const XYArgs& xa, const ZArgs& za,
                              const Scalars* sc, cudaStream_t st);

// cg.cu
struct TangentArgs {
  const void* K45;       // packed tangent (TAN 0)
  const float* H;        // F - I in FP32 (matrix-free tangents)
  const int32_t* phase;
  const float* table;    // neo-Hookean (mu, lam) or SVK 6x6 Voigt per phase, FP32
  const float* scale;    // per-voxel scale or null
};
// tan: 0 packed K (FP64 or FP32), 1 neo-Hookean from H, 2 SVK from H (FP32).
// fin_alpha (cg, partials non-null): the pass also finishes alpha (last block).
// pdl: launched with programmatic dependent launch (see launch_k).
cudaError_t mf_launch_tangent(const void* pin, const void* r, void* pout, void* x, bool f32, int tan,
                              bool cg, const TangentArgs& ta, void* t, long long N, double* partials,
                              int nblk, Scalars* sc, cudaStream_t st, bool fin_alpha = false, bool pdl = false);
cudaError_t mf_launch_fin_beta(const double* partials, int n, Scalars* sc, cudaStream_t st);
cudaError_t mf_launch_cg_batch_init(Scalars* sc, int max_its, cudaStream_t st);
cudaError_t mf_launch_cg_cond(const Scalars* sc, cudaGraphConditionalHandle h, cudaStream_t st, bool pdl = false);
cudaError_t mf_launch_axpy_last(void* x, const void* p0, const void* p1, bool f32, long long n,
                                const Scalars* sc, cudaStream_t st);
cudaError_t mf_launch_axpy_alpha(void* x, const void* p, bool f32, long long n, const Scalars* sc,
                                 cudaStream_t st);
cudaError_t mf_launch_make_H(const double* F, float* H, long long N, cudaStream_t st);

// cufft_path.cu (comparison path)
struct MfCufft;
int mf_cufft_plan(MfCufft* p, int nx, int ny, int nz, bool f32, cudaStream_t st, size_t* need);
int mf_cufft_bind(MfCufft* p, void* dev);
int mf_cufft_project(MfCufft* p, bool f32, const void* t, void* y, int nx, int ny, int nz,
                     const uint8_t* mask, cudaStream_t st, int which);
void mf_cufft_destroy(MfCufft* p);
MfCufft* mf_cufft_new();
void mf_cufft_delete(MfCufft* p);

// pointwise.cu
struct MatArgs {
  int model;              // 0 neo-Hookean, 1 St Venant-Kirchhoff (cubic, rotated)
  int nphase;
  const double* table;    // neo-Hookean: (mu, lam) per phase; SVK: 36 Voigt entries per phase
  const int32_t* phase;
  const double* scale;    // per-voxel multiplier of P and K, or null
};
// P (and K if want_K) at F, voxel averages of F and P; with moments (and
// !want_K) also the rotation moments T, S into sc.
cudaError_t mf_launch_constitutive(const double* F, double* P, void* K45, bool k_f32, bool want_K,
                                   bool moments, const MatArgs& m, long long N, double* partials,
                                   int nblk, Scalars* sc, cudaStream_t st);
// column sums of constitutive partials into meanF, meanP (and T, S if ncol 36)
cudaError_t mf_launch_fin_means(const double* partials, int nblk, int ncol, long long N, Scalars* sc,
                                cudaStream_t st);
// constitutive_dw.cu: P (no tangent) in double-word arithmetic, the averages,
// and optionally H = F - I (FP32, H non-null) and the rotation moments;
// table_dw: the material table as double-word values (layout of MatArgs.table)
// Pf (with H, moments and table32, the FP32 copy of the material table):
// P evaluated in FP32 from H and stored to Pf (9N floats) instead of P;
// the averages of F keep double-word accuracy, those of P are FP32's.
// pred (predict.cuh; with H and moments only): the load step's predictor
// applied to F in the same pass, F overwritten by the predicted state.
struct PredArgs;
cudaError_t mf_launch_constitutive_dw(const double* F, double* P, float* H, bool moments, const MatArgs& m,
                                      const void* table_dw, long long N, double* partials, int nblk,
                                      Scalars* sc, cudaStream_t st, float* Pf = nullptr,
                                      const float* table32 = nullptr, const PredArgs* pred = nullptr);
cudaError_t mf_launch_mean_F(const double* F, long long N, double* partials, int nblk, Scalars* sc,
                             cudaStream_t st);
cudaError_t mf_launch_predictor(double* F, long long N, const uint8_t* mask9, const double* target9,
                                const Scalars* sc, bool after_update, cudaStream_t st);
cudaError_t mf_launch_cg_init(const double* b, void* x, void* r, void* p, bool f32, long long n9,
                              double* partials, int nblk, double tol_cg, double cg_rel, long long N,
                              Scalars* sc, cudaStream_t st);
// Null rotations: up to three skew generators W_k (row-major 3x3) with the
// fields n_k = W_k F orthonormal.
struct Defl {
  int m;
  double W[3][9];
};
cudaError_t mf_launch_newton_update(double* F, const void* x, bool f32, bool defl, long long N,
                                    double* partials, int nblk, Scalars* sc, cudaStream_t st);
// Removes from y (9N, double or float) its components along the n_k:
// y -= What F with What = sum_k (n_k . y) W_k; What is kept in sc for reuse.
cudaError_t mf_launch_defl_project(void* y, bool f32, bool apply, const double* F, long long N,
                                   const Defl& d, double* partials, int nblk, Scalars* sc,
                                   cudaStream_t st);

// history.cu: the Newton control of a load history on the device, so that
// a whole history is one graph launch (steps, Newton iterations and CG
// iterations as nested conditional nodes).  Per-step inputs come from a
// device table, per-step outputs go to one.
constexpr int kHistSteps = 1024;   // steps per launch (longer histories: several launches)
struct HistState {
  // parameters, written by the host before a launch
  int nsteps;              // steps in the table for this launch
  int max_newton, max_cg;
  int forcing;             // CG forcing sequence (FP32 inner, or FP64 with inexact Newton)
  int f32;                 // FP32-inner context: null rotations, re-imposed strain control
  int proj_arith;          // MF_PROJ_* of the FP32 corrections
  double tol_newton, tol_cg, cg_rel, kappa;
  double first_ratio;      // size of the last step's first correction (persists across launches)
  double first_ratio2;     // the same of the step before (persists across launches)
  double kr1, kr2;         // first correction / first rms(r0) of the last two steps (persist)
  double rms0;             // rms of the current step's first residual
  double eta_hi;           // upper bound of the current forcing (0: no refinement at the CG start)
  int extrap;              // predictor: 0 uniform, 1 linear from the last two converged
                           // steps, 2 quadratic from the last three (MF_PRED_*)
  // persists across launches (the host keeps it between calls): the last
  // three converged steps behind F, for the extrapolating predictors
  // linear (extrap 1): t1, t2 the last two steps' targets.  Quadratic
  // (extrap 2): t1 the last step's (the state in F), t2 and t3 those of the
  // states kept in the two extra fields (slots A and B, distinct targets;
  // a new state replaces a slot with its target, else the older slot)
  int nprev;               // converged states recorded (0 .. 3)
  double t1[9], t2[9], t3[9];             // their targets
  double fmean1[9], fmean2[9], fmean3[9]; // their <F>
  unsigned char mprev[9], mprev2[9], mprev3[9];   // their control masks
  int nseen;               // converged steps so far (the slots' ages)
  int ident;               // F is the reference state F = I, in equilibrium at zero
                           // load (P(I) = 0): a converged state whose target the
                           // next step's mask gives (P-bar 0, F-bar = I)
  int age2, age3;          // when slots A and B were written
  // state
  int k;                   // step of the table being solved
  int nn, ncg;             // Newton and CG iterations of the step so far
  int status;              // mf_status of the history (first failure)
  int last;                // the constitutive pass after this update ends the step
  int dw_res;              // the context has the FP32 residual kernels (double-word outer level)
  int res32;               // the current iteration's residual came from FP32 transforms
  int cons_kind;           // pass after this update: 0 P alone, 1 P with the next residual
  int proj_kind;           // projection of this correction: 0 none, 1 FP32, 2 outer arithmetic
  double ratio;            // max_v abs(dF_v) / abs(<F>) of the last correction
  double cg_rel_cur;       // forcing of the current CG solve (0: tol_cg alone)
  int extrapolated;        // this step started from an extrapolated F
  double alpha;            // its linear extrapolation factor
  int quad;                // quadratic predictor: the weights below apply
  double w[3];             // F <- F + w1 (A - F) + w2 (B - F); w0 = 1 - w1 - w2
  double pmean[9];         // the predicted <F> (quadratic predictor)
  int dst;                 // slot the last converged F is copied to: 0 A, 1 B, -1 none
  double target[9], pbar[9];
  unsigned char mask[9];
  Defl defl;               // null rotations of the current Newton iteration
  long long launches;      // kernels the graph ran (accumulated by the control kernels)
};
// Kernel counts of the captured pieces of one Newton iteration, for the
// launch counter: fixed part, per projection kind, per final/next pass.
struct IterCounts {
  int fixed, proj[3], cons[3], cg_body;
};
// One row of the step table (in) and of the result table (out).
struct StepIn {
  double target[9];        // P-bar where mask is 1, F-bar where 0
  unsigned char mask[9];
  unsigned char pad[7];
};
struct StepOut {
  double Fbar[9], Pbar[9]; // <F>, <P> of the converged step
  int newton, cg;          // iterations of the step
};
// Device block of a history: the state, then kHistSteps result rows, then
// kHistSteps step rows (state + results come back in one copy).
struct HistTables {
  const StepIn* in;
  StepOut* out;
};
cudaError_t mf_launch_hist_init(HistState* hs, cudaGraphConditionalHandle h_step, int kernels, cudaStream_t st);
// h_first: set to 1 when the step's first residual runs in the outer
// arithmetic (an extrapolated start), 0 for the FP32 one (may be null)
cudaError_t mf_launch_step_begin(HistState* hs, HistTables t, cudaGraphConditionalHandle* h_first, cudaStream_t st);
// Fprev (9N, may be null when the predictor does not extrapolate): the
// converged F before the current one; the step's predictor replaces it by
// the current F and extrapolates F along the last increment
cudaError_t mf_launch_predictor_hist(double* F, double* Fprev, double* Fprev2, long long N, const HistState* hs,
                                     const Scalars* sc, bool after_update, cudaStream_t st);
cudaError_t mf_launch_newton_pre(HistState* hs, const Scalars* sc, cudaGraphConditionalHandle h_go,
                                 cudaGraphConditionalHandle h_newton, bool first, cudaStream_t st);
cudaError_t mf_launch_proj_decide(HistState* hs, cudaGraphConditionalHandle h_proj, bool first, cudaStream_t st);
cudaError_t mf_launch_newton_post(HistState* hs, Scalars* sc, cudaGraphConditionalHandle h_cons, cudaStream_t st);
cudaError_t mf_launch_newton_cond(HistState* hs, const Scalars* sc, cudaGraphConditionalHandle h_newton,
                                  IterCounts cnt, cudaStream_t st);
// kernels, kernels_ex: the step's kernels outside its Newton iterations, for
// a uniform and an extrapolated start (launch counter)
cudaError_t mf_launch_step_end(HistState* hs, const Scalars* sc, HistTables t, cudaGraphConditionalHandle h_step,
                               int kernels, int kernels_ex, cudaStream_t st);
// CG start with the tolerance and forcing of the current Newton iteration read
// from the history state
cudaError_t mf_launch_cg_init_hist(const double* b, void* r, bool f32, long long n9, double* partials, int nblk,
                                   long long N, HistState* hs, Scalars* sc, cudaStream_t st);
// CG counters reset for a loop inside a history graph; sets the loop's
// condition (0 when the start already stopped it)
cudaError_t mf_launch_cg_start_hist(Scalars* sc, int max_its, cudaGraphConditionalHandle h_cg, cudaStream_t st);
// Null-rotation projection with the rotations read from the device (a pass
// with hs->defl.m == 0 returns at once)
cudaError_t mf_launch_defl_project_hist(void* y, bool f32, bool apply, const double* F, long long N,
                                        const HistState* hs, double* partials, int nblk, Scalars* sc,
                                        cudaStream_t st);
// Newton update; the null-rotation correction is subtracted when hs->defl.m > 0.
// p0, p1 (FP32, the CG directions' buffers): x still lacks the solve's last
// lagging update alpha p, which the update adds on the fly when nothing is
// deflated; mf_launch_axpy_last_defl_hist, launched before the deflation,
// applies it to x otherwise.
cudaError_t mf_launch_newton_update_hist(double* F, const void* x, bool f32, long long N, double* partials,
                                         int nblk, const HistState* hs, Scalars* sc, cudaStream_t st,
                                         const void* p0 = nullptr, const void* p1 = nullptr);
cudaError_t mf_launch_axpy_last_defl_hist(float* x, const float* p0, const float* p1, long long n,
                                          const HistState* hs, const Scalars* sc, cudaStream_t st);

// adjoint.cu: adjoint sensitivity at a converged state (neo-Hookean parameters)
struct AdjWeights {
  double wF[9];   // weights of <F> in the response
  double wP[9];   // weights of <P>
};
// q = W_P (uniform field of the inner type)
cudaError_t mf_launch_adj_rhs_fill(void* q, bool f32, long long N, const AdjWeights& w, cudaStream_t st);
// t += W_F (inner type, in place)
cudaError_t mf_launch_adj_rhs_add(void* t, bool f32, long long N, const AdjWeights& w, cudaStream_t st);
// b (FP64) = y (inner type), n entries
cudaError_t mf_launch_to_double(const void* y, double* b, bool f32, long long n, cudaStream_t st);
// out[2p], out[2p+1] = dJ/dmu_p, dJ/dlam_p; dscale (if non-null) = dJ/ds_v.
// partials: nblk * 2 * nphase doubles.
cudaError_t mf_launch_adj_grad(const double* F, const double* P, const void* lam, bool f32, const int32_t* phase,
                               const double* scale, long long N, int nphase, const AdjWeights& w,
                               double* partials, int nblk, double* out, double* dscale, cudaStream_t st);
