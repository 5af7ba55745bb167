/*
 * mixfft.h -- C ABI of the GB300 library for Galerkin FFT homogenization
 * with macroscopic stress and mixed stress/strain control
 * (Lucarini & Segurado, "An algorithm for stress and mixed control in
 * Galerkin based FFT homogenization", arXiv:1901.06531).
 *
 * Problem statement (Sec. 2): a periodic cell of nx*ny*nz unit voxels, a
 * phase id per voxel with per-phase material parameters, and a load history
 * in which each of the nine components of the macroscopic deformation
 * gradient F-bar or of the macroscopic first Piola stress P-bar is
 * prescribed per step (Sec. 2.3, Eq. eq:mixedeqil).  Each step is solved by
 * Newton (Eq. eq:lineariz) with conjugate gradients on the linear system
 *     G*(K : dF) = -G*(P(F) - P-bar)                      (Eq. linequil2ast)
 * where G* is the projection operator whose null frequency carries the
 * per-component control (Eq. eq:Gnewnew).
 *
 * Conventions for every entry point:
 *  - tensor fields are component-major, c = 3*i + j for component ij, each
 *    component a [z][y][x] block with x fastest: field[c*N + (z*ny + y)*nx + x],
 *    N = nx*ny*nz;
 *  - masks are 9 bytes, 1 = stress controlled (P-bar prescribed), 0 = strain
 *    controlled (F-bar prescribed);
 *  - "host" pointers are ordinary CPU memory owned by the caller and only read
 *    or written during the call; "device" pointers are CUDA global memory on
 *    the context's device, owned by the caller;
 *  - every call returns an mf_status; no call throws or aborts.  After
 *    MF_CUDA_ERROR the context should be destroyed.
 *  - a context is not thread safe; calls on one context are serialised on its
 *    CUDA stream.
 */
#ifndef MIXFFT_H
#define MIXFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MF_OK = 0,
  MF_INVALID_ARG = 1,     /* bad size, pointer, model or parameter; nothing launched */
  MF_NOT_CONVERGED = 2,   /* Newton or CG iteration cap reached */
  MF_CG_BREAKDOWN = 3,    /* p.Ap <= 0 or non-finite in CG (indefinite tangent) */
  MF_NONPOSITIVE_J = 4,   /* det F <= 0 in a neo-Hookean voxel */
  MF_CUDA_ERROR = 5,      /* a CUDA runtime call failed */
  MF_DEVICE_TIMEOUT = 6,  /* a bounded device-side wait gave up */
  MF_NO_WORKSPACE = 7,    /* mf_bind_workspace was not called or is too small */
  MF_TOO_LARGE = 8        /* the cell exceeds the static scratch of mf_residual_noalloc */
} mf_status;

typedef enum { MF_FP64 = 0, MF_FP32_INNER = 1 } mf_precision;
typedef enum { MF_NEOHOOKE = 0, MF_SVK_CUBIC = 1 } mf_model;
typedef enum { MF_OUTER_DOUBLE_WORD = 0, MF_OUTER_FP64 = 1 } mf_outer_arith;
typedef enum { MF_PROJ_FP32 = 0, MF_PROJ_OUTER = 1, MF_PROJ_AUTO = 2 } mf_projection_arith;
typedef enum { MF_PRED_UNIFORM = 0, MF_PRED_EXTRAPOLATE = 1, MF_PRED_QUADRATIC = 2 } mf_predictor;

typedef struct mf_ctx mf_ctx;

/* Create a context for one cell of nx*ny*nz voxels on the current CUDA device.
 * nx, ny: even, of the form 2^a 3^b, 4..256; nz: 2^a 3^b, 2..256.  The x-y
 * plane of one component must fit in shared memory (nx*ny <= 16384), except
 * for nx = ny = 256 with nz in {16, 32, 48, 64, 96, 128, 256}, which the
 * separate row and column kernels serve (mf_set_xy_split).
 * precision MF_FP64: every step in FP64.  MF_FP32_INNER: the CG iterations
 * (transforms, projection, tangent apply, vector updates) run in FP32 with
 * FP64-combined dot products, while P, the residual, the null-frequency
 * control and the Newton update keep FP64 accuracy (defect correction; see
 * mf_set_outer_arith).
 * stream: a cudaStream_t (NULL = legacy default stream) used for every launch
 * and copy of this context.  *out is NULL on failure. */
int mf_create(mf_ctx** out, int nx, int ny, int nz, int precision, void* stream);

/* Bytes of device workspace the context needs (fields F, P, K, residual, CG
 * vectors, spectrum, tables, reduction scratch), 256-byte aligned. */
size_t mf_workspace_bytes(const mf_ctx* ctx);

/* Hand the context a device buffer of at least mf_workspace_bytes() bytes,
 * 256-byte aligned, owned by the caller and kept alive until mf_destroy or
 * the next bind.  The library allocates no device memory of its own. */
int mf_bind_workspace(mf_ctx* ctx, void* dev, size_t bytes);

/* Microstructure and phase parameters (Sec. 2.1: the cell is a spatial
 * arrangement of phases; Sec. 3 materials).
 *   phase  host, N int32 in [0, nphase), x fastest;
 *   model  MF_NEOHOOKE: params host (nphase, 2) = (mu, lambda) per phase;
 *          MF_SVK_CUBIC: params host (nphase, 3) = (C11, C12, C44), rot host
 *          (nphase, 3, 3) row-major rotation per phase or NULL (identity);
 *          the stiffness of phase p is C'_ijkl = R_ia R_jb R_kc R_ld C_abcd;
 *   scale  host, N doubles multiplying P and K per voxel, or NULL.
 * Copies are enqueued on the stream; the host arrays may be reused on return.
 * Resets F to the identity. */
int mf_set_material(mf_ctx* ctx, int model, int nphase, const double* params,
                    const double* rot, const int32_t* phase, const double* scale);

/* Set the deformation-gradient field from host memory (9N doubles) or, with
 * F_host NULL, to the identity everywhere. */
int mf_set_F(mf_ctx* ctx, const double* F_host);

/* Run a load history (Sec. 2.3; Sec. 4 stopping rules).
 *   mask    host, nsteps*9 bytes, 1 = P-bar prescribed, 0 = F-bar prescribed;
 *   target  host, nsteps*9 doubles: P-bar where mask is 1, F-bar where 0;
 *   tol_newton: stop when max_v |dF_v| / |<F>| < tol_newton;
 *   tol_cg: CG stops when sqrt(sum_v |r_v|^2 / N) <= tol_cg (MF_FP64), or
 *           <= max(tol_cg, cg_rel * initial value) (MF_FP32_INNER);
 *   cg_rel: relative CG forcing term for MF_FP32_INNER (and for MF_FP64 with
 *           mf_set_inexact_newton); the first Newton iteration of a step
 *           that starts from the uniform predictor uses sqrt(cg_rel), and
 *           its residual (and the P it transforms) is computed in FP32 (it
 *           is always followed by another iteration: a step never ends on
 *           it); a step that starts extrapolated (mf_set_predictor) takes
 *           its first residual in the outer arithmetic and cg_rel; an
 *           iteration whose predecessor's correction was below
 *           sqrt(tol_newton) (expected to be the last) uses sqrt(cg_rel);
 *   Fbar_out, Pbar_out: host, nsteps*9 doubles or NULL: <F>, <P> per step
 *           (FP32-inner contexts: a step other than the launch's last that
 *           ends on a correction applied as computed reports <P> from the
 *           linearisation <P(F)> + <K:dF>, a remainder of order
 *           abs(K') abs(dF)^2, and <F> as updated; the last step of a
 *           launch evaluates P at its final F);
 *   iters_out: host, nsteps*2 int32 or NULL: Newton iterations and total CG
 *              iterations per step.
 * The run continues from the current F (identity after mf_set_material).
 * On a failure the outputs of the completed steps are written and the
 * status of the failing step is returned.
 * Execution: the history runs as one CUDA graph launch per stretch of steps
 * with one control mask (at most 1024 steps per launch): the loops over
 * steps, Newton iterations and CG iterations are conditional nodes of the
 * graph, and every decision between them (forcing, null rotations,
 * projection arithmetic, the Newton test, the recording of each step's
 * averages) is taken on the device; the host waits once, at the end.  The
 * graph is built and instantiated on the first call with a given mask and
 * max_cg and kept by the context. */
int mf_solve(mf_ctx* ctx, int nsteps, const uint8_t* mask, const double* target,
             double tol_newton, double tol_cg, double cg_rel, int max_newton,
             int max_cg, double* Fbar_out, double* Pbar_out, int32_t* iters_out);

/* Run the same load history layout on n independent cells at once (the
 * batched form: many RVEs of different grid sizes and control masks).  Each
 * context must have its own workspace.  When every cell keeps one control
 * mask over the history and nsteps <= 1024, all cells run as ONE graph
 * launch (on the first context's stream): each cell's load history, as
 * described for mf_solve, is an independent chain of that graph, so the
 * cells' device work overlaps and no host round trip happens until all
 * cells are done.  The batched graph is kept for the next call with the same
 * contexts, masks and max_cg.  Otherwise the cells run one after another.
 *   masks, targets: host, n*nsteps*9, cell-major (cell i starts at 9*nsteps*i);
 *   Fbar_out, Pbar_out: host, n*nsteps*9 or NULL; iters_out: n*nsteps*2 or
 *   NULL; status_out: host, n int32 or NULL, each cell's mf_status.
 * Returns MF_OK when every cell succeeded, else the first failing status.
 * A context may appear only once. */
int mf_solve_batch(int n, mf_ctx* const* ctxs, int nsteps, const uint8_t* masks, const double* targets,
                   double tol_newton, double tol_cg, double cg_rel, int max_newton, int max_cg,
                   double* Fbar_out, double* Pbar_out, int32_t* iters_out, int32_t* status_out);

/* Device-to-device copies of the deformation gradient field (9N doubles),
 * ordered on the context's stream (no host synchronisation): mf_save_F copies
 * the context's F to F_dev; mf_load_F replaces it by F_dev (a checkpoint of a
 * converged step, for example) and invalidates the stored tangent.  F_dev:
 * device, 9N doubles, owned by the caller, not inside the workspace. */
int mf_save_F(mf_ctx* ctx, double* F_dev);
int mf_load_F(mf_ctx* ctx, const double* F_dev);

/* Copy the current F and P fields to host memory (9N doubles each; either
 * pointer may be NULL).  P is the stress at the current F. */
int mf_get_fields(mf_ctx* ctx, double* F_host, double* P_host);

/* ---- operator-level entry points (tests, benchmarks, adjoints) ---------- */

/* Evaluate P(F) and K = dP/dF (Eq. eq:lineariz) at the current F.  K is kept
 * in the context (45 packed entries per voxel, FP64 or FP32 by precision). */
int mf_constitutive(mf_ctx* ctx);

/* Evaluate P(F) alone (no tangent) at the current F, with its voxel
 * averages: the constitutive pass of the last Newton step.  MF_FP32_INNER
 * contexts use the outer arithmetic (mf_set_outer_arith), MF_FP64 contexts
 * FP64.  meanP_host: host 9 doubles or NULL, receives <P>. */
int mf_stress(mf_ctx* ctx, double* meanP_host);

/* Copy the tangent to host memory as 45 packed symmetric entries per voxel:
 * K45_host[t*N + v], t = a*9 - a*(a-1)/2 + (b - a) for a <= b, a = 3i+j,
 * b = 3k+l, value K_ijkl (converted to double). */
int mf_get_tangent(mf_ctx* ctx, double* K45_host);

/* Projected tangent product y = G*(K : x) (left side of Eq. linequil2ast,
 * G* of Eq. eq:Gnewnew with the given mask), using the tangent at the F of
 * the last mf_constitutive: the packed FP64 tangent for MF_FP64, the
 * matrix-free FP32 tangent (from F - I and the phase parameters) for
 * MF_FP32_INNER.  x_dev, y_dev: device, 9N values of the context's inner
 * type (double for MF_FP64, float for MF_FP32_INNER); may not alias. */
int mf_matvec(mf_ctx* ctx, const void* x_dev, void* y_dev, const uint8_t* mask);

/* Right-hand side b = -G*(P - P-bar) of Eq. (linequil2ast) in FP64 from the
 * P of the last mf_constitutive.  b_dev: device, 9N doubles.  meanP_host:
 * host, 9 doubles or NULL, receives <P> (Sec. 2.2: the null-frequency
 * coefficient of P). */
int mf_residual(mf_ctx* ctx, const uint8_t* mask, const double* pbar, double* b_dev,
                double* meanP_host);

/* Residual without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc when they need the
 * residual (a host callback, an allocator hook, a runtime that fixed its
 * device memory budget at start-up).  It computes the same
 * b = -G*(P - P-bar) as mf_residual, in FP64, without a context:
 *   nx, ny, nz: as for mf_create, with nx*ny*nz <= 262144 (64^3); a larger
 *               cell returns MF_TOO_LARGE and launches nothing;
 *   P_dev:  device, 9N doubles (caller's), read only;
 *   mask, pbar: host, 9 bytes / 9 doubles, as for mf_residual;
 *   b_dev:  device, 9N doubles (caller's), written; must not alias P_dev;
 *   meanP_host: host, 9 doubles or NULL, receives <P>;
 *   stream: cudaStream_t for every copy and launch (NULL = default stream).
 * All other memory -- the half spectrum, index and twiddle tables, reduction
 * partials -- lives in one file-scope static device array of 18,958,592
 * bytes (18.1 MiB) that every GPU loading the library holds until the
 * process exits.  No cudaMalloc or cudaFree is called.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current) and caches it for the process; make that first call
 * outside any stream capture.  The cached address does not survive a reset
 * of the device (cudaDeviceReset): do not call this entry point after one.
 * stream must belong to the current device (MF_INVALID_ARG otherwise).  All
 * calls share the one array and each call overwrites it, so calls that may
 * overlap on the GPU (different streams, or different host threads) race:
 * serialise them.  The call synchronises its stream before returning. */
int mf_residual_noalloc(int nx, int ny, int nz, const double* P_dev, const uint8_t* mask,
                        const double* pbar, double* b_dev, double* meanP_host, void* stream);

/* Benchmark hook: time the four kernels of one CG iteration separately with
 * CUDA events on the context's stream, each launch preceded by an L2 flush (a
 * memset of the 9N-double residual buffer): [0] the tangent pass (direction
 * and solution updates, K:p, p.Kp), [1] the x-y forward transform, [2] the
 * z-pass with G-hat-star, [3] the x-y inverse transform with the residual
 * update.  Operands are the context's CG vectors; needs the operator of the
 * last mf_constitutive.  graph 0: events around every launch (the time
 * includes the launch's own start-up on the device); graph 1: the reps
 * (flush, launch) pairs run as one CUDA graph, events around the graph, minus
 * the same graph without the launches (the kernels as they run back to back
 * inside the CG graph, plus the write-back of their dirty lines).  ms_out:
 * host, 4 floats, mean milliseconds per launch. */
int mf_time_kernels(mf_ctx* ctx, const uint8_t* mask, int reps, int graph, float* ms_out);

/* Measurement hook: the FMA throughput of the current device in TFLOP/s
 * (2 flops per FMA), FP64 (precision MF_FP64) or FP32 (MF_FP32_INNER), from
 * independent FMA chains on every SM with no memory traffic (CUDA events
 * around three launches after one untimed launch, legacy stream).  The FP64
 * path of this library is bound by this rate, not by HBM: its roofline
 * fraction is taken against it. */
int mf_probe_fma(int precision, double* tflops_out);

/* Bounds checks of the debug build (the library compiled with MF_DEBUG, see
 * the package's build script): the generic and fixed-size transform kernels
 * and the tangent pass check every shared- and global-memory index against
 * its buffer (the split 256^2-plane kernels are not instrumented); an index
 * outside is counted and recorded (source line, index, extent) and the
 * access is redirected to element 0 of that buffer, so nothing faults.  This
 * call synchronises the device, returns the number of failed checks since the
 * last call in *count_out (the first one's line, index and extent in the
 * other outputs, each may be NULL) and clears the records.  A release build
 * sets *count_out to -1. */
int mf_debug_report(long long* count_out, int* line_out, long long* index_out, long long* extent_out);

/* Self-test of those checks (debug build only): one thread checks index 7
 * against a 4-element device array; the failure is recorded (mf_debug_report
 * then returns count 1, index 7, extent 4) and the write goes to element 0.
 * A release build launches nothing and returns MF_INVALID_ARG. */
int mf_debug_selftest(void);

/* Phase timestamps of load histories (the library compiled with MF_TRACE,
 * the package's build script with trace=True, libmixfft_trace.so).  The
 * graph of a history (mf_solve, mf_solve_batch) records, in one-thread
 * kernels between its phases, the device's global timer (ns) and a phase id:
 * MF_TRACE_STEP_START and MF_TRACE_ITER_START where a load step and a Newton
 * iteration begin, every other id where the phase it names ends, so a
 * phase's duration is its mark minus the mark before.  The marks add a
 * launch each (a few us per mark), so traced histories run slower than
 * release ones; they are for the composition of a step, not its time.  This
 * call synchronises the device, copies up to `cap` entries (oldest first)
 * into t_ns and ids, sets *n_out to the number recorded since the last call
 * (the device keeps at most 65536) and clears them.  A release build
 * returns MF_INVALID_ARG. */
typedef enum {
  MF_TRACE_STEP_START = 1,          /* a load step begins */
  MF_TRACE_STEP_BEGIN = 2,          /* the step's control kernel (targets, predictor weights) */
  MF_TRACE_FIRST_CONSTITUTIVE = 3,  /* the predictor and the constitutive pass */
  MF_TRACE_FIRST_RESIDUAL = 4,      /* the step's first residual */
  MF_TRACE_ITER_START = 10,         /* a Newton iteration begins */
  MF_TRACE_NEWTON_PRE = 11,         /* its control kernel and the right-hand side's null rotations */
  MF_TRACE_CG_INIT = 12,            /* the CG start */
  MF_TRACE_CG_LOOP = 13,            /* the CG iterations */
  MF_TRACE_PROJECTION = 14,         /* the projection choice and the projection of the correction */
  MF_TRACE_DEFLATION = 15,          /* the correction's null rotations */
  MF_TRACE_UPDATE = 16,             /* the Newton update */
  MF_TRACE_NEWTON_POST = 17,        /* the Newton test */
  MF_TRACE_FBAR = 18,               /* F-bar re-imposed on the strain-controlled components */
  MF_TRACE_CONSTITUTIVE = 19,       /* the constitutive pass after the update */
  MF_TRACE_RESIDUAL = 20,           /* the next iteration's residual */
  MF_TRACE_CONS_SWITCH = 21,        /* the end of the pass after the update */
  MF_TRACE_NEWTON_LOOP = 30,        /* the step's further Newton iterations */
  MF_TRACE_STEP_END = 31            /* the step's closing control kernel */
} mf_trace_phase;
int mf_trace_read(int cap, unsigned long long* t_ns, int* ids, int* n_out);

/* Number of kernel launches the library has issued in this process (all
 * contexts); differences around a region count its launches. */
long long mf_kernel_launches(void);

/* ---- comparison path: cuFFT transforms (timing and cross-checks only) ----
 * The same projected operator y = G*(K : x) as mf_matvec, with the library's
 * tangent pass but cuFFT's 3D real-to-complex / complex-to-real transforms
 * and a natural-order G-hat-star (Eq. eq:Gnewnew).  The solver never uses
 * it.  mf_cufft_workspace_bytes creates the cuFFT plans (cuFFT keeps its own
 * plan data) and returns the bytes of device buffer the caller must bind
 * with mf_cufft_bind (natural-order spectrum and cuFFT work area), or 0 on
 * failure.  mf_matvec_cufft: as mf_matvec.  mf_time_cufft: mean ms per
 * launch of [0] the forward transform, [1] G-hat-star, [2] the inverse, each
 * after an L2 flush, on the context's CG vectors. */
size_t mf_cufft_workspace_bytes(mf_ctx* ctx);
int mf_cufft_bind(mf_ctx* ctx, void* dev, size_t bytes);
int mf_matvec_cufft(mf_ctx* ctx, const void* x_dev, void* y_dev, const uint8_t* mask);
int mf_time_cufft(mf_ctx* ctx, const uint8_t* mask, int reps, float* ms_out);

/* Wait for the context's stream. */
int mf_sync(mf_ctx* ctx);

/* Failure-detection self-test: one block on the current device waits on a
 * shared-memory barrier that nothing completes, with the bound every
 * barrier wait of the library has (here max_polls polls, 1..2^20).  The
 * wait gives up, the block records a device timeout and exits, and the call
 * returns MF_DEVICE_TIMEOUT (anything else is a failure of the mechanism);
 * the device stays usable.  Synchronous on the legacy stream; allocates
 * nothing (the flag word is a static device variable). */
int mf_selftest_wait_timeout(int max_polls);

/* Autotuner: time the z-pass tile candidates (4, 8, 16 columns per block) of
 * the fixed-size transform kernels for this context's size and precision and
 * keep the fastest (CUDA events on the context's stream, L2 flushed before
 * every launch); also the residual's z-pass tile (4, 8) and, for FP32-inner
 * contexts whose planes have the persistent or the cluster x-y kernels, the
 * schedules of the x-y passes (forward: one block per plane, the persistent
 * bulk-copy kernel or the two-CTA cluster kernel; inverse: one block per
 * plane or the cluster kernel; mf_set_xy_persistent and mf_set_xy_cluster
 * take precedence).  The choices are
 * cached per (nx, ny, nz, precision, outer arithmetic) for the process;
 * mf_solve and mf_solve_batch run the tuner on a context's first solve if
 * nothing is cached.  This call re-times and replaces the cached choices.
 * zs_out: host int32 or NULL, the chosen width; ms_out: host 3 floats or
 * NULL, mean ms per width (-1 when not applicable); xy_out: host int32 or
 * NULL, the context's x-y forward schedule after the call (0 one block per
 * plane, 1 persistent, 2 cluster); xy_ms_out: host 2 floats or NULL, mean ms
 * of the forward pass per plane and persistent (-1 when not timed; all five
 * timings through mf_xy_schedule).
 * Contexts served by the generic kernels keep their fixed tile. */
int mf_autotune(mf_ctx* ctx, int32_t* zs_out, float* ms_out, int32_t* xy_out, float* xy_ms_out);

/* Adjoint sensitivity of the homogenized response at the current F, which
 * must be a converged state of a step solved with control mask `mask` (for
 * example right after mf_solve, or after mf_set_F with a stored converged
 * field).  The response is J = wF . <F> + wP . <P> (9 weights each).  At
 * equilibrium G*(P - P-bar) = 0 (Eq. linequil2ast with dF = 0); differentiating
 * it gives, with the symmetric projected tangent A = G* K G*,
 *     A lambda = G*(W_F + K : W_P),
 *     dJ/dtheta = (1/N) sum_v (W_P - lambda_v) : dP_v/dtheta,
 * one linear solve by the same CG as the Newton iterations (the loop is one
 * graph launch).  Neo-Hookean law only (MF_INVALID_ARG otherwise); nphase at
 * most 2048 and at most 4.5 N.
 *   mask: host 9 bytes; wF, wP: host 9 doubles;
 *   tol_cg, cg_rel: stop when rms(r) <= max(tol_cg, cg_rel * rms(r0)), in
 *     both precisions (cg_rel 0: tol_cg alone);
 *   J_out: host double or NULL;
 *   dJ_dparams: host 2*nphase doubles or NULL: (dJ/dmu_p, dJ/dlam_p) per phase;
 *   dJ_dscale_dev: device N doubles or NULL: dJ/ds_v for the per-voxel scale
 *     s_v of mf_set_material (P_v = s_v P(F_v; mu, lam)); with no scale bound
 *     the derivative is taken at s = 1;
 *   cg_its_out: host int32 or NULL, CG iterations.
 * F is left unchanged; P and the tangent are recomputed at F; the CG vectors
 * are overwritten.  Synchronous. */
int mf_adjoint(mf_ctx* ctx, const uint8_t* mask, const double* wF, const double* wP, double tol_cg,
               double cg_rel, int max_cg, double* J_out, double* dJ_dparams, double* dJ_dscale_dev,
               int32_t* cg_its_out);

/* x-y transform kernels of a context on the fixed-size path: 0 = one kernel
 * per (component, z) plane holding the whole x-y plane in shared memory (the
 * default where the plane fits); 1 = separate row (x) and column (y) kernels
 * through global memory (the default, and the only choice, for nx = ny =
 * 256; available for nx = ny = 32 as well, for testing).  Results agree to
 * rounding.  MF_INVALID_ARG for a choice the context's size does not
 * support. */
int mf_set_xy_split(mf_ctx* ctx, int split);

/* The FP32 x-y forward transform of an FP32-inner context as a persistent
 * kernel (1) or one block per (component, z) plane (0): one block per SM
 * walks the planes, each plane arriving by one bulk copy (the TMA unit) into
 * one of two shared-memory staging buffers while the block transforms the
 * previous one.  Same stages in the same order: results are identical.
 * Without this call the autotuner chooses (mf_autotune); with it the choice
 * is fixed for the context.  Available for nx = ny in {48, 64, 96, 128} on
 * the fused (non-split) kernels; MF_INVALID_ARG otherwise.  Its barrier
 * waits are bounded; a wait that gives up makes the solve return
 * MF_DEVICE_TIMEOUT. */
int mf_set_xy_persistent(mf_ctx* ctx, int on);

/* The FP32 x-y passes of an FP32-inner context with 128 x 128 planes as
 * kernels of two-CTA clusters, one cluster per (component, z) plane: bit 0
 * the forward pass, bit 1 the inverse pass (with the CG update), 0 neither.
 * The y transform's first radix-2 stage (rows j and j + 64, Eq.
 * eql_discrete2's DFT along y) is applied to the real rows before the x
 * transform; each CTA then keeps one 64-row half of the plane's spectrum in
 * its shared memory (32 KB instead of 66 KB) and the two exchange rows
 * through distributed shared memory.  Same spectrum layout as the per-plane
 * kernels; results agree with theirs to FP32 rounding.  The cluster forward
 * pass takes precedence over the persistent one.  Without this call the
 * autotuner chooses (mf_autotune); with it the choice is fixed for the
 * context.  MF_INVALID_ARG for other sizes, precisions, the split kernels, or
 * `which` outside 0..3. */
int mf_set_xy_cluster(mf_ctx* ctx, int which);

/* The x-y schedules of a context: fwd_out (host int32 or NULL) 0 one block
 * per plane, 1 persistent, 2 cluster; inv_out (host int32 or NULL) 0 one
 * block per plane, 2 cluster; ms_out (host 5 floats or NULL) the
 * autotuner's mean ms per launch of the forward pass per plane, persistent
 * and cluster, and of the inverse pass per plane and cluster (-1 when not
 * timed).  No device work. */
int mf_xy_schedule(mf_ctx* ctx, int32_t* fwd_out, int32_t* inv_out, float* ms_out);

/* FP32-inner contexts: arithmetic of the projection x <- G*(x) applied to
 * the FP32 corrections before the Newton update (FP32 rounding leaves in
 * a correction components that G* annihilates: invisible to the FP64
 * residual, they still shift the equilibrium through the nonlinear law, by
 * about the rounding of the projection, a few eps32 times the correction).
 * MF_PROJ_FP32: the FP32 transform kernels, on every correction but the
 * late ones that follow a correction below 1e-6 of F (their out-of-range
 * rounding is ~1e-13 of F); the field error then grows with the sum of the
 * correction sizes (about 4e-8 after a 20 % stretch in 8 steps).
 * MF_PROJ_OUTER: every correction widened to FP64 and projected in the
 * outer arithmetic (double-word transforms, or FP64 with MF_OUTER_FP64):
 * the fields agree with FP64 solves to well below FP32 rounding, at the cost
 * of a residual-sized transform per Newton iteration.  MF_PROJ_AUTO (the
 * default): the outer arithmetic for the corrections of at least 1e-3 of F
 * (max_v abs(dF_v) / abs(<F>); for the first correction of a step, the size
 * of the previous step's first correction decides, and after mf_set_F,
 * mf_set_material or mf_load_F the first step's first correction takes the
 * outer arithmetic), FP32 for the smaller ones, whose rounding stays below
 * about 1e-10 of F each.  MF_INVALID_ARG for an unknown value, or for a
 * value other than MF_PROJ_FP32 on a non-FP32-inner context. */
int mf_set_projection_arith(mf_ctx* ctx, int arith);

/* Start of the Newton iterations of a load step (Sec. 2.1 writes the start
 * as the last converged fluctuation on the new average; the paper fixes
 * nothing more).  MF_PRED_UNIFORM (default): the last converged F with each
 * strain-controlled component shifted uniformly to the prescribed F-bar.
 * MF_PRED_EXTRAPOLATE: when the last two converged steps of the context had
 * the same control mask, F is first extrapolated along the last increment,
 * F + alpha (F - F_prev), alpha the projection of this step's increment of the
 * prescribed values on the last one (1 along a ramp, -1 back across a
 * reversal), then shifted as above; the first residual of such a step runs
 * in the outer arithmetic, and its inner solve is forced to 0.1 tol_newton
 * over the expected size of its first correction (the larger of the last
 * two steps' first corrections relative to F), within [cg_rel,
 * sqrt(cg_rel)].  MF_PRED_QUADRATIC: with three converged steps of the same
 * mask whose prescribed values lie on one line at distinct positions, F is
 * the quadratic through the three states (Lagrange weights in the position
 * along that line; the converged state of a hyperelastic law is a function
 * of the load), else as MF_PRED_EXTRAPOLATE; one more field of 9 N doubles
 * in the workspace holds the third state.  The converged state is the same
 * to the Newton tolerance; the iteration counts drop along smooth load
 * paths.  The converged steps are remembered across mf_solve calls (not
 * across mf_set_F, mf_set_material, mf_load_F or a failed step); after
 * mf_set_F(NULL) (and at creation) F = I counts as the first one, the
 * equilibrium at zero load (P-bar = 0, F-bar = I) under the first step's
 * mask, since both laws give P(I) = 0.
 * MF_INVALID_ARG for another value. */
int mf_set_predictor(mf_ctx* ctx, int kind);

/* Stopping rule of the CG solves of an MF_FP64 context (Sec. 4 gives the
 * CG tolerance only as an absolute bound on the voxel-averaged residual).
 * on = 0 (the default for MF_FP64): every Newton iteration solves to
 * rms(r) <= tol_cg.  on = 1: the inexact-Newton forcing sequence of the
 * FP32-inner mode, rms(r) <= max(tol_cg, f * rms(r0)) with f = sqrt(cg_rel)
 * for the first Newton iteration of a step and for an iteration whose
 * predecessor's correction was below sqrt(tol_newton), f = cg_rel otherwise;
 * the converged state is the same to the Newton tolerance, with fewer CG
 * iterations.  FP32-inner contexts always use the forcing sequence: on = 0
 * is MF_INVALID_ARG for them, as is any other value. */
int mf_set_inexact_newton(mf_ctx* ctx, int on);

/* Arithmetic of the outer (defect-correction) level of MF_FP32_INNER
 * contexts: the stress P(F) of the constitutive pass (Eq. eq:lineariz) and
 * the transforms of the residual b = -G*(P - P-bar) (Eq. linequil2ast, right
 * side).  MF_OUTER_DOUBLE_WORD (the default) evaluates them in double-word
 * FP32 arithmetic (hi + lo pairs, about 48 significant bits; F and P are read
 * and written in FP64): P on every grid, the residual transforms wherever the
 * fixed-size transform kernels serve the grid (nx = ny, nx and nz in
 * {16, 32, 48, 64, 96, 128}), FP64 elsewhere.  MF_OUTER_FP64 evaluates both
 * in FP64.  The averages, the Newton update, the predictor and every
 * reduction stay FP64 in both.  MF_FP64 contexts ignore the setting; the
 * tangent of mf_constitutive is always FP64.  Returns MF_INVALID_ARG for
 * another value. */
int mf_set_outer_arith(mf_ctx* ctx, int arith);

/* Name and description of the CUDA error behind the last MF_CUDA_ERROR
 * returned by any context in this process ("" if none); static storage. */
const char* mf_last_cuda_error(void);

/* Static description of a status code. */
const char* mf_status_string(int status);

void mf_destroy(mf_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MIXFFT_H */
