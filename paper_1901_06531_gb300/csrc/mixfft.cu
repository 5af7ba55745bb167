// C ABI of the library (include/mixfft.h): context, workspace layout, plans
// and tables, and the host side of the Newton-CG loop of Eq. (linequil2ast)
// under the per-component stress/strain control of Eq. (eq:mixedeqil).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/mixfft.h"
#include "dw.cuh"
#include "fft2.cuh"
#include "launch.h"
#include "predict.cuh"

namespace {

// Phase timestamps of a load history (trace build, -DMF_TRACE): a one-thread
// kernel between the graph's phases records the device's global timer and
// the phase id (ids in include/mixfft.h, mf_trace_read); the release build
// launches nothing.
#ifdef MF_TRACE
constexpr int kTraceCap = 65536;
__device__ unsigned long long g_trace_t[kTraceCap];
__device__ int g_trace_id[kTraceCap];
__device__ int g_trace_n;
__global__ void k_trace_mark(int id) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  const int i = atomicAdd(&g_trace_n, 1);
  if (i < kTraceCap) {
    g_trace_t[i] = t;
    g_trace_id[i] = id;
  }
}
void trace_mark(cudaStream_t s, int id) { k_trace_mark<<<1, 1, 0, s>>>(id); }
#else
void trace_mark(cudaStream_t, int) {}
#endif

constexpr int kMaxPhases = 65536;
constexpr int kPointwiseBlocks = 152 * 8;

bool make_plan(int n, AxisPlan* p) {
  p->n = n;
  p->nst = 0;
  int m = n;
  while (m % 4 == 0) { p->rad[p->nst++] = 4; m /= 4; }
  if (m % 2 == 0) { p->rad[p->nst++] = 2; m /= 2; }
  while (m % 3 == 0) {
    if (p->nst >= MF_MAX_STAGES) return false;
    p->rad[p->nst++] = 3;
    m /= 3;
  }
  return m == 1 && p->nst <= MF_MAX_STAGES;
}

// Position of frequency k after the DIF stages of plan p.
int dif_pos(const AxisPlan& p, int k) {
  int pos = 0, L = p.n;
  for (int st = 0; st < p.nst; ++st) {
    const int r = p.rad[st], m = L / r;
    pos += m * (k % r);
    k /= r;
    L = m;
  }
  return pos;
}

bool smooth_size(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Cyclic Jacobi eigen-decomposition of a symmetric m x m matrix (m <= 3):
// on return A holds the eigenvalues on its diagonal, V the eigenvectors (columns).
void jacobi_eig(int m, double A[3][3], double V[3][3]) {
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
        for (int k = 0; k < m; ++k) {   // A <- J^T A J
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

void skew_of(const double w[3], double W[9]) {
  W[0] = 0; W[1] = -w[2]; W[2] = w[1];
  W[3] = w[2]; W[4] = 0; W[5] = -w[0];
  W[6] = -w[1]; W[7] = w[0]; W[8] = 0;
}

// Rigid rotations of the cell that the linearised problem cannot see.
// A rotation increment W (skew) gives the compatible field n = W F; it is
// admissible when (W <F>)_ij = 0 on every strain-controlled component.  By
// objectivity (P(QF) = Q P(F)) the curvature n_a . A n_b equals
// tr(W_a^T W_b T), T = sum_v P_v F_v^T, and n_a . n_b = tr(W_a^T W_b S),
// S = sum_v F_v F_v^T.  Admissible rotations whose curvature is below
// tau * kappa (kappa a stiffness scale) are returned with n_k orthonormal.
Defl null_rotations(const double meanF[9], const uint8_t* mask, const double T[9], const double S[9],
                    double kappa, double tau) {
  Defl d;
  memset(&d, 0, sizeof(d));
  double Wg[3][9];
  for (int a = 0; a < 3; ++a) {
    double w[3] = {0, 0, 0};
    w[a] = 1.0;
    skew_of(w, Wg[a]);
  }
  // admissibility: C^T C over the strain-controlled components
  double CtC[3][3] = {{0}};
  for (int c = 0; c < 9; ++c) {
    if (mask[c]) continue;
    const int i = c / 3, j = c % 3;
    double row[3];
    for (int a = 0; a < 3; ++a)
      row[a] = Wg[a][3 * i] * meanF[j] + Wg[a][3 * i + 1] * meanF[3 + j] + Wg[a][3 * i + 2] * meanF[6 + j];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) CtC[a][b] += row[a] * row[b];
  }
  double V[3][3];
  jacobi_eig(3, CtC, V);
  double Z[3][3];
  int m = 0;
  for (int k = 0; k < 3; ++k)
    if (fabs(CtC[k][k]) <= 1e-20)
      { for (int a = 0; a < 3; ++a) Z[a][m] = V[a][k]; ++m; }
  if (m == 0) return d;
  auto trWW = [&](const double* Wa, const double* Wb, const double* M) {
    // tr(Wa^T Wb M) = sum_ij Wa_ij (Wb M)_ij
    double s = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double wm = 0.0;
        for (int k = 0; k < 3; ++k) wm += Wb[3 * i + k] * M[3 * k + j];
        s += Wa[3 * i + j] * wm;
      }
    return s;
  };
  double R[3][3], G[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      R[a][b] = 0.5 * (trWW(Wg[a], Wg[b], T) + trWW(Wg[b], Wg[a], T));
      G[a][b] = trWW(Wg[a], Wg[b], S);
    }
  double Rz[3][3] = {{0}}, Gz[3][3] = {{0}};
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
  jacobi_eig(m, Gz, Qg);
  double H[3][3] = {{0}};
  for (int p = 0; p < m; ++p)
    for (int q = 0; q < m; ++q) {
      double s = 0.0;
      for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) s += Qg[a][p] * Rz[a][b] * Qg[b][q];
      H[p][q] = s / sqrt(Gz[p][p] * Gz[q][q]);
    }
  double U[3][3];
  jacobi_eig(m, H, U);
  for (int k = 0; k < m; ++k) {
    if (fabs(H[k][k]) > tau * kappa) continue;
    double v[3] = {0, 0, 0};        // coefficients in the Z basis
    for (int p = 0; p < m; ++p) {
      double s = 0.0;
      for (int q = 0; q < m; ++q) s += Qg[p][q] * U[q][k] / sqrt(Gz[q][q]);
      v[p] = s;
    }
    double w[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a)
      for (int p = 0; p < m; ++p) w[a] += Z[a][p] * v[p];
    skew_of(w, d.W[d.m]);
    ++d.m;
  }
  return d;
}

#ifdef MF_DEBUG
// Readers of the per-translation-unit bounds-check records of the debug build.
struct DebugReader {
  void (*read)(MfDebugRecord*);
  void (*clear)();
};
std::vector<DebugReader>& debug_readers() {
  static std::vector<DebugReader> v;
  return v;
}
#endif

// An instantiated load-history graph of a context, per control mask and CG cap.
struct HistGraph {
  unsigned mask;
  int max_cg;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

long long g_ctx_serial = 0;   // identifies contexts in the batched-graph cache

// The history state padded so that the result rows follow it (state and
// results come back to the host in one copy).
constexpr size_t hist_state_bytes() { return (sizeof(HistState) + 15) & ~(size_t)15; }

}  // namespace

#ifdef MF_DEBUG
void mf_debug_register(void (*read)(MfDebugRecord*), void (*clear)()) {
  debug_readers().push_back(DebugReader{read, clear});
}
#endif

struct mf_ctx {
  int nx, ny, nz;
  long long N;
  int prec;
  int v2 = 0;              // fixed-size transform kernels and their table layout
  int xy_split = 0;        // with v2: separate row and column kernels for the x-y transform
  cudaStream_t st;
  AxisPlan px, pyh, pz;
  int zS;                  // z-pass tile of the operator (CG loop)
  int zSr = 8;             // z-pass tile of the residual (fixed-size kernels)
  // workspace
  char* ws = nullptr;
  size_t ws_need = 0;
  // offsets into the workspace
  size_t oF, oP, ob, oK, ox, or_, op, op2, oAp, oH, ospec, ophase, oscale, oscale32, otable,
      otable32, otabledw, opart, osc, ores, oxpos, oxk, oxe, oyk, ozk, otw64, otw32, otwdw;
  // load-history state and tables (history.cu)
  size_t ohist, othout, othin, oFprev, oFprev2;
  int predictor = MF_PRED_UNIFORM;  // mf_set_predictor
  HistState keep;                   // the history fields that persist between calls (nprev, t1, ...)
  char* pin = nullptr;              // pinned staging of the history block (cudaMallocHost)
  std::vector<HistGraph> hist;      // instantiated history graphs
  cudaStream_t caps[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // capture streams, one per nesting level
  long long serial = 0;             // creation number (batched-graph cache key)
  int gen = 0;                      // bumped whenever the captured kernels change
  size_t npart;
  // material
  int model = -1, nphase = 0;
  double kappa = 1.0;      // stiffness scale of the material (null-rotation test)
  bool has_scale = false;
  bool have_K = false;     // packed tangent of the current F is in the workspace
  bool have_H = false;     // FP32 H = F - I of the current F is in the workspace
  MfCufft* cufft = nullptr;   // comparison path, created on demand
  bool cufft_bound = false;
  // CG loop as one graph launch: a WHILE node whose body is two iterations
  cudaGraph_t cg_graph = nullptr;
  int cg_body_kernels = 0;      // kernel launches per pass of the CG graph's body
  int pw_blocks = 1;            // blocks of the grid-stride pointwise passes (one voxel per thread at most)
  int xy_persist = 0;           // FP32 x-y forward pass as the persistent bulk-copy kernel
  int xy_persist_user = 0;      // set by mf_set_xy_persistent: the autotuner keeps it
  int xy_cluster = 0;           // FP32 x-y passes as two-CTA cluster kernels: bit 0 forward, bit 1 inverse
  int xy_cluster_user = 0;      // set by mf_set_xy_cluster: the autotuner keeps it
  int proj_arith = MF_PROJ_AUTO;   // arithmetic of the projection of each FP32 correction
  double first_ratio = INFINITY;   // max_v abs(dF_v)/abs(<F>) of the last step's first correction
  cudaGraphExec_t cg_exec = nullptr;
  unsigned cg_mask = 0xffffffffu;
  cudaStream_t cap_st = nullptr;   // private stream for graph capture (the legacy stream cannot capture)
  bool tuned = false;              // z-pass tile chosen by the autotuner
  int outer_arith = MF_OUTER_DOUBLE_WORD;
  bool forcing64 = false;          // MF_FP64: inexact-Newton forcing of the FP32-inner mode

  template <typename T> T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
  bool f32() const { return prec == MF_FP32_INNER; }
  // outer level in double-word FP32 (FP32-inner mode): P on every grid, the
  // residual transforms where the fixed-size kernels exist
  bool dw_outer() const { return f32() && outer_arith == MF_OUTER_DOUBLE_WORD; }
  bool dw_residual() const { return dw_outer() && v2; }
  size_t inner_size() const { return f32() ? sizeof(float) : sizeof(double); }
};

namespace {

char g_last_cuda_error[256] = "";

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MF_OK;
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return MF_CUDA_ERROR;
}

// Twiddle table of an arithmetic: FP32, FP64 or double-word complex.
size_t tw_offset(const mf_ctx* c, bool f32, bool dw, size_t* esz) {
  *esz = f32 ? sizeof(float2) : sizeof(double2);
  return dw ? c->otwdw : f32 ? c->otw32 : c->otw64;
}

XYArgs xy_args(const mf_ctx* c, bool f32, bool dw = false) {
  XYArgs a{};
  a.v2 = c->v2;
  a.split = c->xy_split;
  a.skip = nullptr;
  a.fin = 0;
  // the fused fixed-size kernels wait for their predecessor themselves
  // (pdl_wait): launch them with programmatic dependent launch everywhere
  a.pdl = (c->v2 && !c->xy_split) ? 1 : 0;
  a.persist = (f32 && !dw && c->xy_persist && c->v2 && !c->xy_split) ? 1 : 0;
  const bool clu = f32 && !dw && c->v2 && !c->xy_split && mf_cluster_supported(c->nx);
  a.cluster_f = (clu && (c->xy_cluster & 1)) ? 1 : 0;
  a.cluster_i = (clu && (c->xy_cluster & 2)) ? 1 : 0;
  a.flags = &c->at<Scalars>(c->osc)->flags;
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz; a.N = c->N;
  a.px = c->px; a.pyh = c->pyh;
  size_t esz;
  const size_t tw = tw_offset(c, f32, dw, &esz);
  a.twx = c->ws + tw;
  a.twy = c->ws + tw + esz * c->nx;
  a.xpos = c->at<int>(c->oxpos);
  return a;
}

ZArgs z_args(const mf_ctx* c, bool f32, const uint8_t* mask, double scale, bool dw = false) {
  ZArgs a{};
  memset(&a, 0, sizeof(a));
  a.v2 = c->v2;
  a.pdl = c->v2;   // the fixed-size z-pass waits for its predecessor itself
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz; a.N = c->N;
  a.pz = c->pz;
  size_t esz;
  const size_t tw = tw_offset(c, f32, dw, &esz);
  a.twz = c->ws + tw + esz * (c->nx + c->ny);
  a.xk = c->at<int>(c->oxk);
  a.xe = c->at<int>(c->oxe);
  a.yk = c->at<int>(c->oyk);
  a.zk = c->at<int>(c->ozk);
  a.S = c->zS;
  a.mask = 0;
  for (int k = 0; k < 9; ++k)
    if (mask[k]) a.mask |= 1u << k;
  a.scale = scale;
  a.mean_out = nullptr;
  a.lin = nullptr;
  a.lin_alpha = nullptr;
  return a;
}

MatArgs mat_args(const mf_ctx* c) {
  MatArgs m;
  m.model = c->model;
  m.nphase = c->nphase;
  m.table = c->at<double>(c->otable);
  m.phase = c->at<int32_t>(c->ophase);
  m.scale = c->has_scale ? c->at<double>(c->oscale) : nullptr;
  return m;
}

int read_scalars(mf_ctx* c, Scalars* h) {
  cudaError_t e = cudaMemcpyAsync(h, c->ws + c->osc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st);
  if (e != cudaSuccess) return MF_CUDA_ERROR;
  return cuda_status(cudaStreamSynchronize(c->st));
}

int flags_status(int flags) {
  if (flags & MF_FLAG_TIMEOUT) return MF_DEVICE_TIMEOUT;
  if (flags & MF_FLAG_NONPOS_J) return MF_NONPOSITIVE_J;
  if (flags & (MF_FLAG_BREAKDOWN | MF_FLAG_NONFINITE)) return MF_CG_BREAKDOWN;
  return MF_OK;
}

// P (and optionally the packed K) at the current F, voxel averages of F and
// P; with want_H the FP32 H = F - I for the matrix-free tangent.  p32 (the
// double-word path, with H and moments): P evaluated in FP32 and left, in
// FP32, in the scratch the FP32 residual transforms read (the t vector), P
// itself untouched.
int run_constitutive(mf_ctx* c, bool want_K, bool want_H, bool moments = false, bool p32 = false,
                     cudaStream_t cap = nullptr, const PredArgs* pred = nullptr) {
  // cap: the stream of a graph capture (the passes become graph nodes; the
  // context's record of what the workspace holds is left alone); pred: the
  // load step's predictor applied in the same pass (double-word pass only)
  cudaStream_t st = cap ? cap : c->st;
  if (pred && (want_K || !c->dw_outer())) return MF_INVALID_ARG;
  if (!want_K && c->dw_outer()) {
    // P, H and the moments in one double-word pass
    const bool f32p = p32 && want_H && moments;
    const cudaError_t e = mf_launch_constitutive_dw(c->at<double>(c->oF), c->at<double>(c->oP),
                                                    want_H ? c->at<float>(c->oH) : nullptr, moments, mat_args(c),
                                                    c->ws + c->otabledw, c->N, c->at<double>(c->opart),
                                                    c->pw_blocks, c->at<Scalars>(c->osc), st,
                                                    f32p ? c->at<float>(c->oAp) : nullptr,
                                                    c->at<float>(c->otable32), pred);
    if (!cap) {
      c->have_K = false;
      c->have_H = want_H && e == cudaSuccess;
    }
    return cuda_status(e);
  }
  cudaError_t e = mf_launch_constitutive(c->at<double>(c->oF), c->at<double>(c->oP), c->ws + c->oK,
                                         c->f32(), want_K, moments, mat_args(c), c->N,
                                         c->at<double>(c->opart), c->pw_blocks,
                                         c->at<Scalars>(c->osc), st);
  if (!cap) c->have_K = want_K && e == cudaSuccess;
  if (e == cudaSuccess && want_H) e = mf_launch_make_H(c->at<double>(c->oF), c->at<float>(c->oH), c->N, st);
  if (!cap) c->have_H = want_H && e == cudaSuccess;
  return cuda_status(e);
}

bool operator_ready(const mf_ctx* c) { return c->f32() ? c->have_H : c->have_K; }

// fp32: the residual with FP32 transforms (double-word outer arithmetic on
// the fixed-size kernels only); its error is FP32 rounding relative to abs(P),
// harmless while the residual is large
int run_residual(mf_ctx* c, const uint8_t* mask, const double* pbar, double* b, double* mean_out,
                 bool fp32 = false, bool p_in_t = false) {
  if (fp32 && c->dw_residual()) {
    // p_in_t: the constitutive pass left P in FP32 in the t vector
    ZArgs za = z_args(c, true, mask, -1.0 / (double)c->N);
    for (int k = 0; k < 9; ++k) za.add[k] = mask[k] ? pbar[k] : 0.0;
    za.mean_out = mean_out;
    return cuda_status(mf_launch_residual_f32(p_in_t ? nullptr : c->at<double>(c->oP), c->at<float>(c->oAp),
                                              c->ws + c->ospec, c->at<float>(c->op2), b, xy_args(c, true), za,
                                              c->st));
  }
  const bool dw = c->dw_residual();
  ZArgs za = z_args(c, false, mask, -1.0 / (double)c->N, dw);
  if (c->v2) za.S = c->zSr;
  for (int k = 0; k < 9; ++k) za.add[k] = mask[k] ? pbar[k] : 0.0;
  za.mean_out = mean_out;
  return cuda_status(mf_launch_residual(c->at<double>(c->oP), c->ws + c->ospec, b,
                                        c->at<double>(c->opart), xy_args(c, false, dw), za, dw, c->st));
}

TangentArgs tangent_args(const mf_ctx* c) {
  TangentArgs ta;
  ta.K45 = c->ws + c->oK;
  ta.H = c->at<float>(c->oH);
  ta.phase = c->at<int32_t>(c->ophase);
  ta.table = c->at<float>(c->otable32);
  ta.scale = c->has_scale ? c->at<float>(c->oscale32) : nullptr;
  return ta;
}

// Tangent flavour of the inner solve: the packed tangent in FP64, the
// matrix-free law in FP32.
int tangent_kind(const mf_ctx* c) {
  if (!c->f32()) return 0;
  return c->model == MF_NEOHOOKE ? 1 : 2;
}

// y = G*(K : x) for a device vector x of the inner type.
int run_matvec(mf_ctx* c, const void* x, void* y, const uint8_t* mask) {
  const ZArgs za = z_args(c, c->f32(), mask, 1.0 / (double)c->N);
  const XYArgs xa = xy_args(c, c->f32());
  cudaError_t e = mf_launch_tangent(x, nullptr, nullptr, nullptr, c->f32(), tangent_kind(c), false,
                                    tangent_args(c), c->ws + c->oAp, c->N, nullptr, c->pw_blocks,
                                    nullptr, c->st, false, true);
  if (e == cudaSuccess)
    e = mf_launch_project(c->f32(), c->ws + c->oAp, c->ws + c->ospec, y, 0, nullptr, xa, za, nullptr,
                          c->st);
  return cuda_status(e);
}

// Drop every captured graph of the context (the CG loop, the load
// histories): called whenever the kernels or tiles they hold change.
void free_cg_graph(mf_ctx* c) {
  if (c->cg_exec) cudaGraphExecDestroy(c->cg_exec);
  if (c->cg_graph) cudaGraphDestroy(c->cg_graph);
  c->cg_exec = nullptr;
  c->cg_graph = nullptr;
  c->cg_mask = 0xffffffffu;
  for (HistGraph& h : c->hist) {
    if (h.exec) cudaGraphExecDestroy(h.exec);
    if (h.graph) cudaGraphDestroy(h.graph);
  }
  c->hist.clear();
  ++c->gen;
}

unsigned mask_bits(const uint8_t* mask) {
  unsigned m = 0;
  for (int k = 0; k < 9; ++k)
    if (mask[k]) m |= 1u << k;
  return m;
}

// Capture the body of the CG iteration loop into `body` on stream cs: two
// iterations (the two directions swap buffers) and a one-thread kernel that
// keeps the loop's condition h set while the device-side stop flag is clear.
// The kernels of an iteration that starts after the stop return at once, so
// the iteration count (kept on the device) is exact.
cudaError_t capture_cg_body(mf_ctx* c, cudaStream_t cs, cudaGraph_t body, const uint8_t* mask,
                            cudaGraphConditionalHandle h) {
  const bool f32 = c->f32();
  void* x = c->ws + c->ox;
  void* r = c->ws + c->or_;
  void* pbuf[2] = {c->ws + c->op, c->ws + c->op2};
  void* t = c->ws + c->oAp;
  Scalars* sc = c->at<Scalars>(c->osc);
  double* part = c->at<double>(c->opart);
  ZArgs za = z_args(c, f32, mask, 1.0 / (double)c->N);
  XYArgs xa = xy_args(c, f32);
  za.skip = &sc->stop;
  xa.skip = &sc->stop;
  // FP32: the z-pass adds alpha_k <t_k> (t_k = K:p_k, its null-frequency
  // coefficient / N) to sc->lin, so that a solve ends with <K:x> at hand
  // (x = sum_k alpha_k p_k; the linearised end-of-step averages)
  if (f32) {
    za.lin = sc->lin;
    za.lin_alpha = &sc->alpha;
  }
  // the fused x-y inverse kernel finishes beta itself; the split and generic
  // kernels leave it to k_fin_beta
  xa.fin = (xa.v2 && !xa.split) ? 1 : 0;
  // programmatic dependent launch along the body (tangent, the fused
  // transform passes, the loop condition): each kernel is scheduled as its
  // predecessor's blocks exit, loads its constant tables, then waits for the
  // predecessor's completion (saves the launch gap: 8 CG-bound 32^3 cells
  // solve in half the time; neutral at 128^3)
  const bool pdl = xa.v2 && !xa.split;
  const TangentArgs ta = tangent_args(c);
  const int tk = tangent_kind(c);
  const int nplanes = mf_xy_blocks(c->ny, c->nz, c->xy_split != 0);
  cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  for (int it = 0; it < 2 && e == cudaSuccess; ++it) {
    e = mf_launch_tangent(pbuf[it], r, pbuf[1 - it], x, f32, tk, true, ta, t, c->N, part, c->pw_blocks, sc,
                          cs, true, pdl);
    if (e == cudaSuccess) e = mf_launch_project(f32, t, c->ws + c->ospec, r, 3, part, xa, za, sc, cs);
    if (e == cudaSuccess && !xa.fin) e = mf_launch_fin_beta(part, nplanes, sc, cs);
  }
  // per iteration: tangent, the transform passes (two more for the split x-y
  // kernels), k_fin_beta unless fused; k_cg_cond once per body
  c->cg_body_kernels = 2 * (1 + ((xa.v2 && xa.split) ? 5 : 3) + (xa.fin ? 0 : 1)) + 1;
  if (e == cudaSuccess) e = mf_launch_cg_cond(sc, h, cs, pdl);
  cudaGraph_t captured = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
  return e != cudaSuccess ? e : e2;
}

// The CG iteration loop of one linear solve as a graph: a WHILE conditional
// node whose body is capture_cg_body's.
int build_cg_graph(mf_ctx* c, const uint8_t* mask) {
  free_cg_graph(c);
  if (!c->cap_st) {
    const cudaError_t ec = cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking);
    if (ec != cudaSuccess) { c->cap_st = nullptr; return cuda_status(ec); }
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cuda_status(e);
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_status(e);
  }
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_status(e);
  }
  const long long l0 = g_mf_launches;
  e = capture_cg_body(c, c->cap_st, np.conditional.phGraph_out[0], mask, h);
  g_mf_launches = l0;   // captured, not launched
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->cg_exec, g, 0);
  if (e != cudaSuccess) {
    cuda_status(e);
    cudaGetLastError();
    cudaGraphDestroy(g);
    c->cg_exec = nullptr;
    return MF_CUDA_ERROR;
  }
  c->cg_graph = g;
  c->cg_mask = mask_bits(mask);
  return MF_OK;
}

// ---------------------------------------------------------------- autotuner
// The z-pass tile (columns per block: 4, 8 or 16 for the fixed-size kernels)
// trades shared memory per block against blocks per SM and DRAM segment
// length; the best choice depends on the z length and the precision.  Each
// candidate is timed with CUDA events on the context's stream (L2 flushed
// before every launch, one untimed launch first) and the fastest kept; the
// choice is cached for the process per (nx, ny, nz, precision).
struct TuneEntry { int nx, ny, nz, prec, dw, S, Sr, xyp, xyc; float ms[3], msr[2], msxy[3], msxi[2]; };
std::vector<TuneEntry> g_tune_cache;
std::mutex g_tune_mutex;

int autotune(mf_ctx* c, int reps) {
  if (!c->v2) { c->tuned = true; return MF_OK; }
  const int dwr = c->dw_residual() ? 1 : 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (const TuneEntry& t : g_tune_cache)
      if (t.nx == c->nx && t.ny == c->ny && t.nz == c->nz && t.prec == c->prec && t.dw == dwr) {
        c->zS = t.S;
        c->zSr = t.Sr;
        if (!c->xy_persist_user && c->xy_persist != t.xyp) {
          c->xy_persist = t.xyp;
          free_cg_graph(c);
        }
        if (!c->xy_cluster_user && c->xy_cluster != t.xyc) {
          c->xy_cluster = t.xyc;
          free_cg_graph(c);
        }
        c->tuned = true;
        return MF_OK;
      }
  }
  const bool f32 = c->f32();
  const int cands[3] = {4, 8, 16};
  const uint8_t mask[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
  ZArgs za = z_args(c, f32, mask, 1.0 / (double)c->N);
  const XYArgs xa = xy_args(c, f32);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MF_CUDA_ERROR;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return MF_CUDA_ERROR; }
  TuneEntry te{c->nx,        c->ny,        c->nz,   c->prec,          dwr,     c->zS, c->zSr, c->xy_persist,
               c->xy_cluster, {0, 0, 0},    {0, 0},  {-1, -1, -1},     {-1, -1}};
  float best = 1e30f;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    za.S = cands[i];
    if ((c->ny * (c->nx / 2)) % za.S) { te.ms[i] = -1; continue; }
    double tot = 0.0;
    for (int r = -1; r < reps && e == cudaSuccess; ++r) {
      e = cudaMemsetAsync(c->ws + c->ob, 0, 9 * c->N * sizeof(double), c->st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, c->st);
      if (e == cudaSuccess)
        e = mf_launch_project_part(1, f32, nullptr, c->ws + c->ospec, nullptr, nullptr, xa, za, nullptr, c->st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (r >= 0) tot += ms;
    }
    te.ms[i] = (float)(tot / reps);
    if (e == cudaSuccess && te.ms[i] < best) { best = te.ms[i]; te.S = cands[i]; }
  }
  // the residual's z-pass (FP64 or double word), tiles 4 and 8
  ZArgs zr = z_args(c, false, mask, -1.0 / (double)c->N, dwr != 0);
  const int rcands[2] = {4, 8};
  float bestr = 1e30f;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    zr.S = rcands[i];
    double tot = 0.0;
    for (int r = -1; r < reps && e == cudaSuccess; ++r) {
      e = cudaMemsetAsync(c->ws + c->ob, 0, 9 * c->N * sizeof(double), c->st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, c->st);
      if (e == cudaSuccess) e = dwr ? mf_v2_zp_dw(c->ws + c->ospec, zr, c->st) : mf_v2_zp_f64(1, c->ws + c->ospec, zr, c->st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (r >= 0) tot += ms;
    }
    te.msr[i] = (float)(tot / reps);
    if (e == cudaSuccess && te.msr[i] < bestr) { bestr = te.msr[i]; te.Sr = rcands[i]; }
  }
  // the schedules of the FP32 x-y passes: forward one block per plane, the
  // persistent bulk-copy kernel or the two-CTA cluster kernel; inverse (with
  // the CG update) one block per plane or the cluster kernel.  Another form
  // than one block per plane is taken only when it is faster by more than 3%
  // (single timed launches: a tie keeps the per-plane default), unless
  // mf_set_xy_persistent / mf_set_xy_cluster chose
  auto time_pass = [&](int which, const XYArgs& xf, float* out) {
    double tot = 0.0;
    for (int r = -1; r < reps && e == cudaSuccess; ++r) {
      e = cudaMemsetAsync(c->ws + c->ob, 0, 9 * c->N * sizeof(double), c->st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, c->st);
      if (e == cudaSuccess)
        e = which == 0 ? mf_launch_project_part(0, f32, c->ws + c->oAp, c->ws + c->ospec, nullptr, nullptr, xf, za,
                                                nullptr, c->st)
                       : mf_launch_project_part(2, f32, nullptr, c->ws + c->ospec, c->ws + c->or_,
                                                c->at<double>(c->opart), xf, za, c->at<Scalars>(c->osc), c->st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (r >= 0) tot += ms;
    }
    *out = (float)(tot / reps);
  };
  const bool xyp_ok = f32 && !c->xy_split && mf_persist_supported(c->nx);
  const bool xyc_ok = f32 && !c->xy_split && mf_cluster_supported(c->nx);
  if (e == cudaSuccess && (xyp_ok || xyc_ok)) {
    XYArgs xf = xa;
    xf.persist = 0;
    xf.cluster_f = 0;
    xf.cluster_i = 0;
    time_pass(0, xf, &te.msxy[0]);
    if (xyp_ok) {
      xf.persist = 1;
      time_pass(0, xf, &te.msxy[1]);
      xf.persist = 0;
    }
    if (xyc_ok) {
      xf.cluster_f = 1;
      time_pass(0, xf, &te.msxy[2]);
      xf.cluster_f = 0;
      time_pass(1, xf, &te.msxi[0]);
      xf.cluster_i = 1;
      time_pass(1, xf, &te.msxi[1]);
    }
    if (e == cudaSuccess) {
      int best_f = 0;
      for (int f = 1; f < 3; ++f)
        if (te.msxy[f] > 0 && te.msxy[f] < 0.97f * te.msxy[0] && te.msxy[f] < te.msxy[best_f]) best_f = f;
      te.xyp = best_f == 1 ? 1 : 0;
      te.xyc = (best_f == 2 ? 1 : 0) | ((te.msxi[1] > 0 && te.msxi[1] < 0.97f * te.msxi[0]) ? 2 : 0);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) { cudaGetLastError(); return cuda_status(e); }
  c->zS = te.S;
  c->zSr = te.Sr;
  if (!c->xy_persist_user) c->xy_persist = te.xyp;
  if (!c->xy_cluster_user) c->xy_cluster = te.xyc;
  c->tuned = true;
  free_cg_graph(c);   // a captured loop holds the old tile
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tune_cache.push_back(te);
  return MF_OK;
}

// Enqueue one linear solve of Eq. (linequil2ast) by CG from dF = 0 (the
// solution is left in the x vector; stop at rms(r) <= max(tol_cg, cg_rel *
// rms(r0))): CG start, the graph with the device-side
// iteration loop, and the last lagging solution update.  Per iteration: the
// tangent pass (direction update, lagging solution update, K:p and p.Kp), the
// three transform passes whose last one updates the residual, and two
// one-block reductions.
int launch_cg(mf_ctx* c, const uint8_t* mask, double tol_cg, double cg_rel, int max_cg) {
  const bool f32 = c->f32();
  const long long n9 = 9 * c->N;
  Scalars* sc = c->at<Scalars>(c->osc);
  double* part = c->at<double>(c->opart);
  if (!c->cg_exec || c->cg_mask != mask_bits(mask)) {
    const int s = build_cg_graph(c, mask);
    if (s) return s;
  }
  cudaError_t e = mf_launch_cg_init(c->at<double>(c->ob), c->ws + c->ox, c->ws + c->or_, c->ws + c->op, f32, n9,
                                    part, c->pw_blocks, tol_cg, cg_rel, c->N, sc, c->st);
  if (e == cudaSuccess) e = mf_launch_cg_batch_init(sc, max_cg, c->st);
  if (e == cudaSuccess) e = cudaGraphLaunch(c->cg_exec, c->st);
  if (e == cudaSuccess)
    e = mf_launch_axpy_last(c->ws + c->ox, c->ws + c->op, c->ws + c->op2, f32, n9, sc, c->st);
  return cuda_status(e);
}

// Outcome of the solve from the scalars read back after it.  *clear is set
// when an FP32 inner solve ended on a direction of non-positive curvature
// after some progress: that ends the inner solve without failing it (the FP64
// outer iteration continues from the current iterate; alpha was 0 for that
// direction) and the caller clears the flag.
int cg_outcome(const mf_ctx* c, const Scalars& h, bool* clear) {
  *clear = false;
  if (c->f32() && (h.flags & MF_FLAG_BREAKDOWN) && !(h.flags & ~MF_FLAG_BREAKDOWN) && h.its > 1) {
    *clear = true;
    return MF_OK;
  }
  const int s = flags_status(h.flags);
  if (s) return s;
  if (!h.done) return MF_NOT_CONVERGED;
  return MF_OK;
}

// ---------------------------------------------------------------- load histories
// A load history of a cell runs as one graph launch (Sec. 2.3; Sec. 4
// stopping rules): a WHILE node over the steps of the history table; in its
// body the predictor, the first constitutive pass, the first Newton
// iteration and a WHILE node over the further Newton iterations; in each
// iteration an IF node (the iteration runs unless a failure or the cap ended
// the step), the residual, the CG start, the WHILE node of the CG
// iterations, a SWITCH node over the projection of an FP32 correction (none,
// FP32, outer arithmetic; each branch ends with the Newton update) and an
// IF/ELSE node over the following constitutive pass (P alone when the
// correction passed the Newton test, else P with the tangent or H and the
// rotation moments).  One-thread kernels (history.cu) take the decisions and
// set the handles.  The graph is built by stream capture; conditional nodes
// are added at the capture point and their bodies captured on further
// streams, one per nesting level.

// A conditional handle on the graph that stream s is capturing into.
cudaError_t cap_handle(cudaStream_t s, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(h, g, 0, 0);
  return e;
}

// A conditional node at the capture point of s (the capture continues after
// it); bodies receives its size body graphs.
cudaError_t cap_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                            unsigned size, cudaGraph_t* bodies) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> dv(deps, deps + nd);
  std::vector<cudaGraphEdgeData> ev(nd);
  for (size_t i = 0; i < nd; ++i) {
    if (edges) ev[i] = edges[i];
    else memset(&ev[i], 0, sizeof(ev[i]));
  }
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = size;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, dv.data(), ev.data(), nd, &np);
  if (e != cudaSuccess) return e;
  for (unsigned i = 0; i < size; ++i) bodies[i] = np.conditional.phGraph_out[i];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

cudaError_t cap_begin(cudaStream_t s, cudaGraph_t g) {
  return cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
}

cudaError_t cap_end(cudaStream_t s, cudaError_t e) {
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(s, &out);
  return e != cudaSuccess ? e : e2;
}

HistTables hist_tables(const mf_ctx* c) {
  HistTables t;
  t.in = c->at<StepIn>(c->othin);
  t.out = c->at<StepOut>(c->othout);
  return t;
}

// The residual b = -G*(P - P-bar) of a Newton iteration, captured on st,
// P-bar of the step read on the device.  res32: FP32 transforms of the P the
// preceding pass left in FP32 in the t vector (double-word outer level);
// otherwise the outer arithmetic (double word where the fixed-size kernels
// exist, else FP64).
cudaError_t capture_residual(mf_ctx* c, const uint8_t* mask, bool res32, cudaStream_t st) {
  const long long N = c->N;
  HistState* hs = c->at<HistState>(c->ohist);
  double* b = c->at<double>(c->ob);
  if (res32) {
    ZArgs za = z_args(c, true, mask, -1.0 / (double)N);
    za.add_dev = hs->pbar;
    za.mean_out = c->at<double>(c->ores);
    return mf_launch_residual_f32(nullptr, c->at<float>(c->oAp), c->ws + c->ospec, c->at<float>(c->op2), b,
                                  xy_args(c, true), za, st);
  }
  const bool dw = c->dw_residual();
  ZArgs za = z_args(c, false, mask, -1.0 / (double)N, dw);
  if (c->v2) za.S = c->zSr;
  za.add_dev = hs->pbar;
  za.mean_out = c->at<double>(c->ores);
  return mf_launch_residual(c->at<double>(c->oP), c->ws + c->ospec, b, c->at<double>(c->opart),
                            xy_args(c, false, dw), za, dw, st);
}

// Capture one Newton iteration (its residual already computed) on caps[lvl]
// (capturing into a step body or the Newton loop's body); caps[lvl + 1] and
// caps[lvl + 2] take the nested bodies.  h_newton: the Newton loop's
// condition, set at the end.  The iteration ends with the pass after the
// update and, unless the step ended, the next iteration's residual.
cudaError_t capture_iteration(mf_ctx* c, cudaStream_t* caps, int lvl, bool first, const uint8_t* mask, int max_cg,
                              cudaGraphConditionalHandle h_newton) {
  const bool f32 = c->f32();
  const bool dwr = c->dw_residual();
  const long long N = c->N;
  HistState* hs = c->at<HistState>(c->ohist);
  Scalars* sc = c->at<Scalars>(c->osc);
  double* part = c->at<double>(c->opart);
  double* F = c->at<double>(c->oF);
  double* b = c->at<double>(c->ob);
  cudaStream_t s = caps[lvl], s1 = caps[lvl + 1], s2 = caps[lvl + 2];
  const long long l0 = g_mf_launches;
  long long in_bodies = 0;
  IterCounts cnt;
  memset(&cnt, 0, sizeof(cnt));
  cudaGraphConditionalHandle h_go;
  cudaError_t e = cap_handle(s, &h_go);
  trace_mark(s, MF_TRACE_ITER_START);
  if (e == cudaSuccess) e = mf_launch_newton_pre(hs, sc, h_go, h_newton, first, s);
  cudaGraph_t go_body = nullptr;
  if (e == cudaSuccess) e = cap_conditional(s, h_go, cudaGraphCondTypeIf, 1, &go_body);
  if (e != cudaSuccess) return e;
  e = cap_begin(s1, go_body);
  if (e != cudaSuccess) return e;
  // FP32 inner solves: the null rotations out of the right-hand side
  if (f32) e = mf_launch_defl_project_hist(b, false, true, F, N, hs, part, c->pw_blocks, sc, s1);
  trace_mark(s1, MF_TRACE_NEWTON_PRE);
  if (e == cudaSuccess)
    e = mf_launch_cg_init_hist(b, c->ws + c->or_, f32, 9 * N, part, c->pw_blocks, N, hs, sc, s1);
  trace_mark(s1, MF_TRACE_CG_INIT);
  cudaGraphConditionalHandle h_cg;
  if (e == cudaSuccess) e = cap_handle(s1, &h_cg);
  if (e == cudaSuccess) e = mf_launch_cg_start_hist(sc, max_cg, h_cg, s1);
  cudaGraph_t cg_body = nullptr;
  if (e == cudaSuccess) e = cap_conditional(s1, h_cg, cudaGraphCondTypeWhile, 1, &cg_body);
  if (e == cudaSuccess) {
    const long long lb = g_mf_launches;
    e = capture_cg_body(c, s2, cg_body, mask, h_cg);
    in_bodies += g_mf_launches - lb;
    cnt.cg_body = c->cg_body_kernels;
  }
  trace_mark(s1, MF_TRACE_CG_LOOP);
  // the solve's last lagging update x += alpha p: FP64 here; FP32 in each
  // branch below (the unprojected correction takes it inside the update)
  if (e == cudaSuccess && !f32)
    e = mf_launch_axpy_last(c->ws + c->ox, c->ws + c->op, c->ws + c->op2, f32, 9 * N, sc, s1);
  if (e == cudaSuccess && f32) {
    // projection of the FP32 correction onto the range of G* (its rounding
    // leaves components the residual cannot see), then the Newton update
    cudaGraphConditionalHandle h_proj;
    e = cap_handle(s1, &h_proj);
    if (e == cudaSuccess) e = mf_launch_proj_decide(hs, h_proj, first, s1);
    cudaGraph_t pb[3] = {nullptr, nullptr, nullptr};
    if (e == cudaSuccess) e = cap_conditional(s1, h_proj, cudaGraphCondTypeSwitch, 3, pb);
    for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
      const long long lb = g_mf_launches;
      e = cap_begin(s2, pb[kind]);
      if (e != cudaSuccess) break;
      void* corr = c->ws + c->ox;
      bool corr32 = true;
      if (kind == 0) e = mf_launch_axpy_last_defl_hist(c->at<float>(c->ox), c->at<float>(c->op), c->at<float>(c->op2),
                                                      9 * N, hs, sc, s2);
      else e = mf_launch_axpy_last(c->ws + c->ox, c->ws + c->op, c->ws + c->op2, true, 9 * N, sc, s2);
      if (e != cudaSuccess) {
      } else if (kind == 1) {
        const ZArgs za = z_args(c, true, mask, 1.0 / (double)N);
        e = mf_launch_project(true, c->ws + c->ox, c->ws + c->ospec, c->ws + c->op2, 0, nullptr, xy_args(c, true), za,
                              nullptr, s2);
        corr = c->ws + c->op2;
      } else if (kind == 2) {
        ZArgs za = z_args(c, false, mask, 1.0 / (double)N, dwr);
        if (c->v2) za.S = c->zSr;
        e = mf_launch_to_double(c->ws + c->ox, b, true, 9 * N, s2);
        if (e == cudaSuccess) {
          if (dwr) {
            const XYArgs xd = xy_args(c, false, true);
            e = mf_v2_xyf_dw(b, c->ws + c->ospec, xd, s2);
            if (e == cudaSuccess) e = mf_v2_zp_dw(c->ws + c->ospec, za, s2);
            if (e == cudaSuccess) e = mf_v2_xyi_dw(c->ws + c->ospec, b, nullptr, xd, s2);
          } else {
            e = mf_launch_project(false, b, c->ws + c->ospec, b, 0, nullptr, xy_args(c, false), za, nullptr, s2);
          }
        }
        corr = b;
        corr32 = false;
      }
      trace_mark(s2, MF_TRACE_PROJECTION);
      if (e == cudaSuccess)
        e = mf_launch_defl_project_hist(corr, corr32, false, F, N, hs, part, c->pw_blocks, sc, s2);
      trace_mark(s2, MF_TRACE_DEFLATION);
      if (e == cudaSuccess)
        e = mf_launch_newton_update_hist(F, corr, corr32, N, part, c->pw_blocks, hs, sc, s2,
                                         kind == 0 ? c->ws + c->op : nullptr, kind == 0 ? c->ws + c->op2 : nullptr);
      trace_mark(s2, MF_TRACE_UPDATE);
      e = cap_end(s2, e);
      cnt.proj[kind] = (int)(g_mf_launches - lb);
      in_bodies += g_mf_launches - lb;
    }
  } else if (e == cudaSuccess) {
    e = mf_launch_newton_update_hist(F, c->ws + c->ox, false, N, part, c->pw_blocks, hs, sc, s1);
  }
  // the Newton test, then the pass after the update: 0 P alone (the step
  // ends), 1 P with the tangent or H and the rotation moments, and the next
  // iteration's residual in the outer arithmetic
  cudaGraphConditionalHandle h_cons;
  if (e == cudaSuccess) e = cap_handle(s1, &h_cons);
  if (e == cudaSuccess) e = mf_launch_newton_post(hs, sc, h_cons, s1);
  trace_mark(s1, MF_TRACE_NEWTON_POST);
  // (FP32 inner) 2: the step ends, its averages from the linearisation,
  // which k_newton_post takes from the sums the solve's z-passes kept (no
  // body: the switch runs none for a value past its last body)
  const int nkind = 2;
  cudaGraph_t cb[2] = {nullptr, nullptr};
  if (e == cudaSuccess) e = cap_conditional(s1, h_cons, cudaGraphCondTypeSwitch, nkind, cb);
  for (int kind = 0; kind < nkind && e == cudaSuccess; ++kind) {
    const long long lb = g_mf_launches;
    e = cap_begin(s2, cb[kind]);
    if (e != cudaSuccess) break;
    const bool more = kind != 0;
    // FP32 corrections carry a rounding-level average on the strain-controlled
    // components; the outer level re-imposes F-bar there before the pass over
    // F (after a kind-2 ending the next step's predictor does, from the
    // averages k_newton_post records)
    int st = 0;
    if (f32 && mf_launch_predictor_hist(F, nullptr, nullptr, N, hs, sc, true, s2) != cudaSuccess) st = MF_CUDA_ERROR;
    trace_mark(s2, MF_TRACE_FBAR);
    if (!st) st = run_constitutive(c, more && !f32, more && f32, more && f32, false, s2);
    trace_mark(s2, MF_TRACE_CONSTITUTIVE);
    if (!st && more && capture_residual(c, mask, false, s2) != cudaSuccess) st = MF_CUDA_ERROR;
    trace_mark(s2, MF_TRACE_RESIDUAL);
    e = cap_end(s2, st ? cudaErrorUnknown : cudaSuccess);
    cnt.cons[kind] = (int)(g_mf_launches - lb);
    in_bodies += g_mf_launches - lb;
  }
  // the kernels outside the bodies, including the condition kernel below
  cnt.fixed = (int)(g_mf_launches - l0 - in_bodies) + 1;
  if (!f32) cnt.proj[1] = cnt.proj[2] = 0;
  trace_mark(s1, MF_TRACE_CONS_SWITCH);
  if (e == cudaSuccess) e = mf_launch_newton_cond(hs, sc, h_newton, cnt, s1);
  return cap_end(s1, e);
}

// Capture a whole load history of the cell into graph G (as a root chain of
// its own: several cells can share one graph).
cudaError_t build_history(mf_ctx* c, cudaGraph_t G, const uint8_t* mask, int max_cg) {
  for (int i = 0; i < 5; ++i)
    if (!c->caps[i]) {
      const cudaError_t ec = cudaStreamCreateWithFlags(&c->caps[i], cudaStreamNonBlocking);
      if (ec != cudaSuccess) { c->caps[i] = nullptr; return ec; }
    }
  const bool f32 = c->f32();
  const long long N = c->N;
  HistState* hs = c->at<HistState>(c->ohist);
  Scalars* sc = c->at<Scalars>(c->osc);
  double* part = c->at<double>(c->opart);
  double* F = c->at<double>(c->oF);
  const HistTables t = hist_tables(c);
  cudaStream_t* caps = c->caps;
  const long long l0 = g_mf_launches;
  cudaError_t e = cap_begin(caps[0], G);
  if (e != cudaSuccess) return e;
  e = mf_launch_mean_F(F, N, part, c->pw_blocks, sc, caps[0]);
  cudaGraphConditionalHandle h_step;
  if (e == cudaSuccess) e = cap_handle(caps[0], &h_step);
  if (e == cudaSuccess) e = mf_launch_hist_init(hs, h_step, 3, caps[0]);
  cudaGraph_t B1 = nullptr;
  if (e == cudaSuccess) e = cap_conditional(caps[0], h_step, cudaGraphCondTypeWhile, 1, &B1);
  if (e == cudaSuccess) {
    // the body of one load step
    e = cap_begin(caps[1], B1);
    if (e == cudaSuccess) {
      const long long ls = g_mf_launches;
      const bool extrap = c->predictor != MF_PRED_UNIFORM;
      double* Fprev2 = c->predictor == MF_PRED_QUADRATIC ? c->at<double>(c->oFprev2) : nullptr;
      const bool dwr = c->dw_residual();
      // with the extrapolating predictor on a double-word context, the first
      // residual's arithmetic follows the start (IF: extrapolated -> outer)
      cudaGraphConditionalHandle h_first;
      const bool choose = extrap && dwr;
      if (choose) e = cap_handle(caps[1], &h_first);
      trace_mark(caps[1], MF_TRACE_STEP_START);
      if (e == cudaSuccess) e = mf_launch_step_begin(hs, t, choose ? &h_first : nullptr, caps[1]);
      trace_mark(caps[1], MF_TRACE_STEP_BEGIN);
      // the predictor: in the double-word constitutive pass that follows
      // (FP32 inner with a double-word outer level), else a pass of its own
      double* Fprev = extrap ? c->at<double>(c->oFprev) : nullptr;
      const PredArgs pred{Fprev, Fprev2, hs, Fprev2 ? 2 : (Fprev ? 1 : 0)};
      const bool fuse_pred = f32 && c->dw_outer();
      if (e == cudaSuccess && !fuse_pred) e = mf_launch_predictor_hist(F, Fprev, Fprev2, N, hs, sc, false, caps[1]);
      // the pass after the predictor: FP64 P and K, or (FP32 inner) H and the
      // rotation moments, with P itself in FP32 for an FP32 first residual;
      // then the first residual
      int step_kernels = 0, step_kernels_ex = 0;
      auto first_pass = [&](bool res32, cudaStream_t st) {
        int r = run_constitutive(c, !f32, f32, f32, res32, st, fuse_pred ? &pred : nullptr);
        trace_mark(st, MF_TRACE_FIRST_CONSTITUTIVE);
        if (!r && capture_residual(c, mask, res32, st) != cudaSuccess) r = MF_CUDA_ERROR;
        trace_mark(st, MF_TRACE_FIRST_RESIDUAL);
        return r ? cudaErrorUnknown : cudaSuccess;
      };
      if (e == cudaSuccess && !choose) {
        e = first_pass(dwr, caps[1]);
        step_kernels = step_kernels_ex = (int)(g_mf_launches - ls) + 1;
      } else if (e == cudaSuccess) {
        const int base = (int)(g_mf_launches - ls) + 1;
        cudaGraph_t fb[2] = {nullptr, nullptr};
        e = cap_conditional(caps[1], h_first, cudaGraphCondTypeIf, 2, fb);
        for (int br = 0; br < 2 && e == cudaSuccess; ++br) {   // body 0: extrapolated start
          const long long lb = g_mf_launches;
          e = cap_begin(caps[2], fb[br]);
          if (e == cudaSuccess) e = cap_end(caps[2], first_pass(br == 1, caps[2]));
          (br == 0 ? step_kernels_ex : step_kernels) = base + (int)(g_mf_launches - lb);
        }
      }
      cudaGraphConditionalHandle h_newton;
      if (e == cudaSuccess) e = cap_handle(caps[1], &h_newton);
      if (e == cudaSuccess) e = capture_iteration(c, caps, 1, true, mask, max_cg, h_newton);
      cudaGraph_t B2 = nullptr;
      if (e == cudaSuccess) e = cap_conditional(caps[1], h_newton, cudaGraphCondTypeWhile, 1, &B2);
      if (e == cudaSuccess) {
        e = cap_begin(caps[2], B2);
        if (e == cudaSuccess) e = cap_end(caps[2], capture_iteration(c, caps, 2, false, mask, max_cg, h_newton));
      }
      trace_mark(caps[1], MF_TRACE_NEWTON_LOOP);
      if (e == cudaSuccess) e = mf_launch_step_end(hs, sc, t, h_step, step_kernels, step_kernels_ex, caps[1]);
      trace_mark(caps[1], MF_TRACE_STEP_END);
      e = cap_end(caps[1], e);
    }
  }
  e = cap_end(caps[0], e);
  g_mf_launches = l0;   // captured, not launched
  return e;
}

// The instantiated history graph of a context for a control mask and CG cap
// (built on first use).
cudaGraphExec_t history_exec(mf_ctx* c, const uint8_t* mask, int max_cg, int* status) {
  const unsigned mb = mask_bits(mask);
  for (const HistGraph& h : c->hist)
    if (h.mask == mb && h.max_cg == max_cg) return h.exec;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = build_history(c, g, mask, max_cg);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    *status = cuda_status(e);
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return nullptr;
  }
  c->hist.push_back(HistGraph{mb, max_cg, g, ex});
  return ex;
}

// Pinned staging of the history block: the state, kHistSteps result rows,
// kHistSteps step rows (host memory; allocated on a context's first solve).
int hist_staging(mf_ctx* c) {
  if (c->pin) return MF_OK;
  const size_t bytes = hist_state_bytes() + (size_t)kHistSteps * (sizeof(StepOut) + sizeof(StepIn));
  if (cudaMallocHost((void**)&c->pin, bytes) != cudaSuccess) {
    c->pin = nullptr;
    return MF_CUDA_ERROR;
  }
  return MF_OK;
}

HistState* pin_state(mf_ctx* c) { return reinterpret_cast<HistState*>(c->pin); }
StepOut* pin_out(mf_ctx* c) { return reinterpret_cast<StepOut*>(c->pin + hist_state_bytes()); }
StepIn* pin_in(mf_ctx* c) {
  return reinterpret_cast<StepIn*>(c->pin + hist_state_bytes() + (size_t)kHistSteps * sizeof(StepOut));
}

// The history parameters and step rows [k0, k1) to the device, on st.
cudaError_t upload_history(mf_ctx* c, const uint8_t* mask, const double* target, int k0, int k1, double tol_newton,
                           double tol_cg, double cg_rel, int max_newton, int max_cg, cudaStream_t st) {
  HistState* hh = pin_state(c);
  memset(hh, 0, sizeof(*hh));
  hh->nsteps = k1 - k0;
  hh->max_newton = max_newton;
  hh->max_cg = max_cg;
  hh->forcing = (c->f32() || c->forcing64) ? 1 : 0;
  hh->f32 = c->f32() ? 1 : 0;
  hh->dw_res = c->dw_residual() ? 1 : 0;
  hh->proj_arith = c->proj_arith;
  hh->tol_newton = tol_newton;
  hh->tol_cg = tol_cg;
  hh->cg_rel = cg_rel;
  hh->kappa = c->kappa;
  hh->first_ratio = c->first_ratio;
  hh->first_ratio2 = c->keep.first_ratio2;
  hh->kr1 = c->keep.kr1;
  hh->kr2 = c->keep.kr2;
  hh->rms0 = 0.0;
  hh->eta_hi = 0.0;
  hh->ratio = INFINITY;
  hh->extrap = c->predictor;
  hh->nprev = c->keep.nprev;
  memcpy(hh->t1, c->keep.t1, sizeof(hh->t1));
  memcpy(hh->t2, c->keep.t2, sizeof(hh->t2));
  memcpy(hh->t3, c->keep.t3, sizeof(hh->t3));
  memcpy(hh->fmean1, c->keep.fmean1, sizeof(hh->fmean1));
  memcpy(hh->fmean2, c->keep.fmean2, sizeof(hh->fmean2));
  memcpy(hh->fmean3, c->keep.fmean3, sizeof(hh->fmean3));
  memcpy(hh->mprev, c->keep.mprev, sizeof(hh->mprev));
  memcpy(hh->mprev2, c->keep.mprev2, sizeof(hh->mprev2));
  memcpy(hh->mprev3, c->keep.mprev3, sizeof(hh->mprev3));
  hh->nseen = c->keep.nseen;
  hh->ident = c->keep.ident;
  hh->age2 = c->keep.age2;
  hh->age3 = c->keep.age3;
  StepIn* in = pin_in(c);
  for (int k = k0; k < k1; ++k) {
    StepIn& r = in[k - k0];
    memset(&r, 0, sizeof(r));
    memcpy(r.target, target + 9 * (size_t)k, 9 * sizeof(double));
    memcpy(r.mask, mask + 9 * (size_t)k, 9);
  }
  cudaError_t e = cudaMemcpyAsync(c->ws + c->ohist, hh, sizeof(HistState), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->ws + c->othin, in, sizeof(StepIn) * (k1 - k0), cudaMemcpyHostToDevice, st);
  return e;
}

// The state and the result rows of n steps back to the staging block, on st.
cudaError_t download_history(mf_ctx* c, int n, cudaStream_t st) {
  return cudaMemcpyAsync(c->pin, c->ws + c->ohist, hist_state_bytes() + sizeof(StepOut) * n,
                         cudaMemcpyDeviceToHost, st);
}

// After the download completed: the completed steps' rows into the caller's
// arrays at [k0, ...); returns the history's status.
int finish_history(mf_ctx* c, int k0, int k1, double* Fbar_out, double* Pbar_out, int32_t* iters_out) {
  const HistState& hs = *pin_state(c);
  const StepOut* out = pin_out(c);
  for (int k = 0; k < hs.k && k0 + k < k1; ++k) {
    if (Fbar_out) memcpy(Fbar_out + 9 * (size_t)(k0 + k), out[k].Fbar, 9 * sizeof(double));
    if (Pbar_out) memcpy(Pbar_out + 9 * (size_t)(k0 + k), out[k].Pbar, 9 * sizeof(double));
    if (iters_out) { iters_out[2 * (k0 + k)] = out[k].newton; iters_out[2 * (k0 + k) + 1] = out[k].cg; }
  }
  c->first_ratio = hs.first_ratio;
  c->keep = hs;
  if (hs.status) {
    c->keep.nprev = 0;
    c->keep.ident = 0;
  }
  c->have_K = false;
  c->have_H = false;
  g_mf_launches += hs.launches;
  return hs.status;
}

bool same_mask(const uint8_t* a, const uint8_t* b) { return memcmp(a, b, 9) == 0; }

// One cell: the history in segments of constant control mask (at most
// kHistSteps steps each), one graph launch per segment.
int solve_cell(mf_ctx* c, int nsteps, const uint8_t* mask, const double* target, double tol_newton, double tol_cg,
               double cg_rel, int max_newton, int max_cg, double* Fbar_out, double* Pbar_out, int32_t* iters_out) {
  int s = hist_staging(c);
  if (s) return s;
  for (int k0 = 0; k0 < nsteps;) {
    int k1 = k0 + 1;
    while (k1 < nsteps && k1 - k0 < kHistSteps && same_mask(mask + 9 * (size_t)k1, mask + 9 * (size_t)k0)) ++k1;
    cudaGraphExec_t ex = history_exec(c, mask + 9 * (size_t)k0, max_cg, &s);
    if (!ex) return s;
    cudaError_t e = upload_history(c, mask, target, k0, k1, tol_newton, tol_cg, cg_rel, max_newton, max_cg, c->st);
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, c->st);
    if (e == cudaSuccess) e = download_history(c, k1 - k0, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_status(e);
    s = finish_history(c, k0, k1, Fbar_out, Pbar_out, iters_out);
    if (s) return s;
    k0 = k1;
  }
  return MF_OK;
}

int check_solve_args(const mf_ctx* c, int nsteps, const uint8_t* mask, const double* target, double tol_newton,
                     double tol_cg, double cg_rel, int max_newton, int max_cg) {
  if (!c || nsteps < 0 || (nsteps > 0 && (!mask || !target)) || !(tol_newton > 0) || !(tol_cg > 0) ||
      max_newton < 1 || max_cg < 1 || !(cg_rel >= 0))
    return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  if (c->model < 0) return MF_INVALID_ARG;
  for (int i = 0; i < 9 * nsteps; ++i)
    if (mask[i] > 1 || !isfinite(target[i])) return MF_INVALID_ARG;
  return MF_OK;
}

}  // namespace

extern "C" {

const char* mf_status_string(int s) {
  switch (s) {
    case MF_OK: return "ok";
    case MF_INVALID_ARG: return "invalid argument";
    case MF_NOT_CONVERGED: return "not converged";
    case MF_CG_BREAKDOWN: return "CG breakdown (p.Ap <= 0 or non-finite)";
    case MF_NONPOSITIVE_J: return "det F <= 0";
    case MF_CUDA_ERROR: return "CUDA error";
    case MF_DEVICE_TIMEOUT: return "device timeout";
    case MF_NO_WORKSPACE: return "no workspace bound";
    case MF_TOO_LARGE: return "cell larger than the static scratch of mf_residual_noalloc (64^3 voxels)";
    default: return "unknown status";
  }
}

int mf_create(mf_ctx** out, int nx, int ny, int nz, int precision, void* stream) {
  if (!out) return MF_INVALID_ARG;
  *out = nullptr;
  if (precision != MF_FP64 && precision != MF_FP32_INNER) return MF_INVALID_ARG;
  if (nx < 4 || ny < 4 || nz < 2 || nx > 256 || ny > 256 || nz > 256) return MF_INVALID_ARG;
  if ((nx & 1) || (ny & 1) || !smooth_size(nx) || !smooth_size(ny) || !smooth_size(nz))
    return MF_INVALID_ARG;
  // one component's x-y plane must fit in shared memory (FP64 residual),
  // unless the split row/column kernels serve the plane
  const bool big_plane = (size_t)(ny / 2) * nx * sizeof(double2) + (size_t)(nx + ny) * 20 > 200 * 1024;
  if (big_plane && !(mf_v2_supported(nx, ny, nz) && mf_split_supported(nx))) return MF_INVALID_ARG;
  mf_ctx* c = new (std::nothrow) mf_ctx();
  if (!c) return MF_INVALID_ARG;
  c->nx = nx; c->ny = ny; c->nz = nz;
  c->N = (long long)nx * ny * nz;
  c->prec = precision;
  c->serial = ++g_ctx_serial;
  memset(&c->keep, 0, sizeof(c->keep));
  c->v2 = mf_v2_supported(nx, ny, nz) ? 1 : 0;
  c->xy_split = big_plane ? 1 : 0;
  c->st = (cudaStream_t)stream;
  if (!make_plan(nx, &c->px) || !make_plan(ny / 2, &c->pyh) || !make_plan(nz, &c->pz)) {
    delete c;
    return MF_INVALID_ARG;
  }
  // z-pass tile: columns per block so that 9 * nz * S complex doubles fit
  int S = 16;
  while (S > 1 && (size_t)9 * nz * S * sizeof(double2) > 150 * 1024) S /= 2;
  c->zS = S;
  // pointwise passes: one voxel per thread for small cells, else 8 blocks per SM
  c->pw_blocks = (int)((c->N + 255) / 256 < kPointwiseBlocks ? (c->N + 255) / 256 : kPointwiseBlocks);

  const long long N = c->N;
  const size_t isz = c->inner_size();
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
  c->oF = take(9 * N * sizeof(double));
  c->oP = take(9 * N * sizeof(double));
  c->ob = take(9 * N * sizeof(double));
  c->oK = take(45 * N * isz);
  c->ox = take(9 * N * isz);
  c->or_ = take(9 * N * isz);
  c->op = take(9 * N * isz);
  c->op2 = take(9 * N * isz);
  c->oAp = take(9 * N * isz);
  c->oH = take(precision == MF_FP32_INNER ? 9 * N * sizeof(float) : 256);
  c->ospec = take(9 * (N / 2) * sizeof(double2));
  c->ophase = take(N * sizeof(int32_t));
  c->oscale = take(N * sizeof(double));
  c->oscale32 = take(N * sizeof(float));
  c->otable = take((size_t)kMaxPhases * 36 * sizeof(double));
  c->otable32 = take((size_t)kMaxPhases * 36 * sizeof(float));
  c->otabledw = take((size_t)kMaxPhases * 36 * sizeof(dw));
  // widest reduction: the constitutive pass with rotation moments, 36 columns per block
  c->npart = (size_t)(kPointwiseBlocks > 9 * nz ? kPointwiseBlocks : 9 * nz) * 36;
  c->opart = take(c->npart * sizeof(double));
  c->osc = take(sizeof(Scalars));
  c->ohist = take(hist_state_bytes() + (size_t)kHistSteps * sizeof(StepOut));
  c->othout = c->ohist + hist_state_bytes();
  c->othin = take((size_t)kHistSteps * sizeof(StepIn));
  c->oFprev = take(9 * N * sizeof(double));
  c->oFprev2 = take(9 * N * sizeof(double));
  c->ores = take(9 * sizeof(double));
  c->oxpos = take(nx * sizeof(int));
  c->oxk = take(nx * sizeof(int));
  c->oxe = take(nx * sizeof(int));
  c->oyk = take(ny * sizeof(int));
  c->ozk = take(nz * sizeof(int));
  c->otw64 = take((nx + ny + nz) * sizeof(double2));
  c->otw32 = take((nx + ny + nz) * sizeof(float2));
  c->otwdw = take((nx + ny + nz) * sizeof(dwc));
  c->ws_need = off;
  *out = c;
  return MF_OK;
}

size_t mf_workspace_bytes(const mf_ctx* c) { return c ? c->ws_need : 0; }

int mf_bind_workspace(mf_ctx* c, void* dev, size_t bytes) {
  if (!c || !dev || bytes < c->ws_need || ((uintptr_t)dev & 255)) return MF_INVALID_ARG;
  c->ws = (char*)dev;
  c->model = -1;
  c->have_K = false;
  free_cg_graph(c);
  // host-built tables: digit-reversal maps and twiddles
  const int nx = c->nx, ny = c->ny, nz = c->nz;
  std::vector<int> xpos(nx, 0), xk(nx, 0), xe(nx, 0), yk(ny, 0), zk(nz, 0);
  if (c->v2) {
    // half-length rows: slot of kx < nx/2; rows hold ky in digit-reversed order
    const int h = nx / 2;
    for (int k = 0; k < h; ++k) xpos[k] = fft2::dif_pos(h, k);
    for (int k = 0; k < h; ++k) xk[xpos[k]] = k;
    for (int k = 0; k < ny; ++k) yk[fft2::dif_pos(ny, k)] = k;
    for (int k = 0; k < nz; ++k) zk[fft2::dif_pos(nz, k)] = k;
  } else {
    for (int k = 0; k < nx; ++k) xpos[k] = dif_pos(c->px, k);
    for (int k = 0; k < nx; ++k) {
      const int s = xpos[k];
      if (k < nx / 2) { xk[s] = k; xe[s] = 0; }
      else if (k == nx / 2) { xk[s] = 0; xe[s] = 1; }
      else { xk[s] = nx - k; xe[s] = 1; }
    }
    for (int k = 0; k < ny / 2; ++k) yk[dif_pos(c->pyh, k)] = k;
    for (int k = 0; k < nz; ++k) zk[dif_pos(c->pz, k)] = k;
  }
  std::vector<double2> tw64(nx + ny + nz);
  std::vector<float2> tw32(nx + ny + nz);
  std::vector<dwc> twdw(nx + ny + nz);
  int o = 0;
  for (int n : {nx, ny, nz}) {
    for (int t = 0; t < n; ++t) {
      const double ang = -2.0 * M_PI * (double)t / (double)n;
      tw64[o + t] = make_double2(cos(ang), sin(ang));
      tw32[o + t] = make_float2((float)tw64[o + t].x, (float)tw64[o + t].y);
      twdw[o + t].x = dw(tw64[o + t].x);
      twdw[o + t].y = dw(tw64[o + t].y);
    }
    o += n;
  }
  cudaError_t e = cudaSuccess;
  auto put = [&](size_t off, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ws + off, src, bytes, cudaMemcpyHostToDevice, c->st);
  };
  put(c->oxpos, xpos.data(), nx * sizeof(int));
  put(c->oxk, xk.data(), nx * sizeof(int));
  put(c->oxe, xe.data(), nx * sizeof(int));
  put(c->oyk, yk.data(), ny * sizeof(int));
  put(c->ozk, zk.data(), nz * sizeof(int));
  put(c->otw64, tw64.data(), tw64.size() * sizeof(double2));
  put(c->otw32, tw32.data(), tw32.size() * sizeof(float2));
  put(c->otwdw, twdw.data(), twdw.size() * sizeof(dwc));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + c->osc, 0, sizeof(Scalars), c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);   // host vectors go out of scope
  return cuda_status(e);
}

int mf_set_material(mf_ctx* c, int model, int nphase, const double* params, const double* rot,
                    const int32_t* phase, const double* scale) {
  if (!c) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  if ((model != MF_NEOHOOKE && model != MF_SVK_CUBIC) || nphase < 1 || nphase > kMaxPhases || !params ||
      !phase)
    return MF_INVALID_ARG;
  for (long long v = 0; v < c->N; ++v)
    if (phase[v] < 0 || phase[v] >= nphase) return MF_INVALID_ARG;
  std::vector<double> table;
  if (model == MF_NEOHOOKE) {
    table.assign(params, params + 2 * nphase);
    for (double x : table)
      if (!isfinite(x)) return MF_INVALID_ARG;
  } else {
    table.assign((size_t)36 * nphase, 0.0);
    for (int p = 0; p < nphase; ++p) {
      const double c11 = params[3 * p], c12 = params[3 * p + 1], c44 = params[3 * p + 2];
      if (!isfinite(c11) || !isfinite(c12) || !isfinite(c44)) return MF_INVALID_ARG;
      // cubic tensor in the crystal frame
      double C[3][3][3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          for (int cc = 0; cc < 3; ++cc)
            for (int d = 0; d < 3; ++d) {
              double v = 0.0;
              if (a == b && cc == d) v += c12;
              if (a == cc && b == d) v += c44;
              if (a == d && b == cc) v += c44;
              if (a == b && b == cc && cc == d) v += c11 - c12 - 2.0 * c44;
              C[a][b][cc][d] = v;
            }
      double R[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
      if (rot)
        for (int i = 0; i < 9; ++i) {
          R[i / 3][i % 3] = rot[9 * p + i];
          if (!isfinite(rot[9 * p + i])) return MF_INVALID_ARG;
        }
      // C'_ijkl = R_ia R_jb R_kc R_ld C_abcd, one index at a time
      double T1[3][3][3][3], T2[3][3][3][3];
      for (int i = 0; i < 3; ++i) for (int b = 0; b < 3; ++b) for (int cc = 0; cc < 3; ++cc)
        for (int d = 0; d < 3; ++d) {
          double s = 0; for (int a = 0; a < 3; ++a) s += R[i][a] * C[a][b][cc][d]; T1[i][b][cc][d] = s;
        }
      for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) for (int cc = 0; cc < 3; ++cc)
        for (int d = 0; d < 3; ++d) {
          double s = 0; for (int b = 0; b < 3; ++b) s += R[j][b] * T1[i][b][cc][d]; T2[i][j][cc][d] = s;
        }
      for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) {
          double s = 0; for (int cc = 0; cc < 3; ++cc) s += R[k][cc] * T2[i][j][cc][d]; T1[i][j][k][d] = s;
        }
      for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          double s = 0; for (int d = 0; d < 3; ++d) s += R[l][d] * T1[i][j][k][d]; T2[i][j][k][l] = s;
        }
      static const int vi[6] = {0, 1, 2, 1, 0, 0}, vj[6] = {0, 1, 2, 2, 2, 1};
      for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) table[36 * p + 6 * I + J] = T2[vi[I]][vj[I]][vi[J]][vj[J]];
    }
  }
  if (scale)
    for (long long v = 0; v < c->N; ++v)
      if (!isfinite(scale[v])) return MF_INVALID_ARG;
  std::vector<float> table32(table.begin(), table.end());
  std::vector<dw> tabledw(table.begin(), table.end());
  cudaError_t e = cudaMemcpyAsync(c->ws + c->otable, table.data(), table.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->ws + c->otable32, table32.data(), table32.size() * sizeof(float),
                        cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->ws + c->otabledw, tabledw.data(), tabledw.size() * sizeof(dw),
                        cudaMemcpyHostToDevice, c->st);
  std::vector<float> scale32;
  if (scale) scale32.assign(scale, scale + c->N);
  if (e == cudaSuccess && scale)
    e = cudaMemcpyAsync(c->ws + c->oscale32, scale32.data(), c->N * sizeof(float), cudaMemcpyHostToDevice,
                        c->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->ws + c->ophase, phase, c->N * sizeof(int32_t), cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess && scale)
    e = cudaMemcpyAsync(c->ws + c->oscale, scale, c->N * sizeof(double), cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return MF_CUDA_ERROR;
  double kap = 0.0;
  for (int p = 0; p < nphase; ++p)
    kap = fmax(kap, model == MF_NEOHOOKE ? fabs(params[2 * p]) : fabs(params[3 * p + 2]));
  double smax = 1.0;
  if (scale) {
    smax = 0.0;
    for (long long v = 0; v < c->N; ++v) smax = fmax(smax, fabs(scale[v]));
  }
  c->kappa = kap * smax > 0 ? kap * smax : 1.0;
  c->model = model;
  c->nphase = nphase;
  c->has_scale = scale != nullptr;
  c->have_K = false;
  return mf_set_F(c, nullptr);
}

int mf_set_F(mf_ctx* c, const double* F_host) {
  if (!c) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  c->first_ratio = INFINITY;
  c->keep.first_ratio2 = INFINITY;
  c->keep.kr1 = c->keep.kr2 = 0.0;
  // the extrapolating predictors start over; F = I is itself a converged
  // state (zero load), the first one they extrapolate from
  c->keep.nprev = F_host ? 0 : 1;
  c->keep.ident = F_host ? 0 : 1;
  const long long N = c->N;
  double* F = c->at<double>(c->oF);
  cudaError_t e;
  if (F_host) {
    e = cudaMemcpyAsync(F, F_host, 9 * N * sizeof(double), cudaMemcpyHostToDevice, c->st);
  } else {
    std::vector<double> ident(9 * N, 0.0);
    for (long long v = 0; v < N; ++v) ident[v] = ident[4 * N + v] = ident[8 * N + v] = 1.0;
    e = cudaMemcpyAsync(F, ident.data(), 9 * N * sizeof(double), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + c->osc, 0, sizeof(Scalars), c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  c->have_K = false;
  c->have_H = false;
  return cuda_status(e);
}

int mf_save_F(mf_ctx* c, double* F_dev) {
  if (!c || !F_dev) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  return cuda_status(cudaMemcpyAsync(F_dev, c->ws + c->oF, 9 * c->N * sizeof(double), cudaMemcpyDeviceToDevice,
                                     c->st));
}

int mf_load_F(mf_ctx* c, const double* F_dev) {
  if (!c || !F_dev) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  c->first_ratio = INFINITY;
  c->keep.first_ratio2 = INFINITY;
  c->keep.kr1 = c->keep.kr2 = 0.0;
  c->keep.nprev = 0;   // the extrapolating predictors start over
  c->keep.ident = 0;
  const char* p = (const char*)F_dev;
  if (p + 9 * c->N * sizeof(double) > c->ws && p < c->ws + c->ws_need) return MF_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(c->ws + c->oF, F_dev, 9 * c->N * sizeof(double), cudaMemcpyDeviceToDevice,
                                  c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + c->osc, 0, sizeof(Scalars), c->st);
  c->have_K = false;
  c->have_H = false;
  return cuda_status(e);
}

int mf_constitutive(mf_ctx* c) {
  if (!c) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  if (c->model < 0) return MF_INVALID_ARG;
  int s = run_constitutive(c, true, c->f32());
  if (s) return s;
  Scalars h;
  s = read_scalars(c, &h);
  if (s) return s;
  return flags_status(h.flags);
}

int mf_stress(mf_ctx* c, double* meanP_host) {
  if (!c) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  if (c->model < 0) return MF_INVALID_ARG;
  int s = run_constitutive(c, false, false);
  if (s) return s;
  Scalars h;
  s = read_scalars(c, &h);
  if (s) return s;
  if (meanP_host) memcpy(meanP_host, h.meanP, sizeof(h.meanP));
  return flags_status(h.flags);
}

int mf_get_tangent(mf_ctx* c, double* K45_host) {
  if (!c || !K45_host) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  if (!c->have_K) return MF_INVALID_ARG;
  const size_t n = 45 * (size_t)c->N;
  if (!c->f32()) {
    cudaError_t e = cudaMemcpyAsync(K45_host, c->ws + c->oK, n * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    return cuda_status(e);
  }
  std::vector<float> tmp(n);
  cudaError_t e = cudaMemcpyAsync(tmp.data(), c->ws + c->oK, n * sizeof(float), cudaMemcpyDeviceToHost,
                                  c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return MF_CUDA_ERROR;
  for (size_t i = 0; i < n; ++i) K45_host[i] = tmp[i];
  return MF_OK;
}

int mf_matvec(mf_ctx* c, const void* x_dev, void* y_dev, const uint8_t* mask) {
  if (!c || !x_dev || !y_dev || !mask || x_dev == y_dev) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  if (!operator_ready(c)) return MF_INVALID_ARG;
  return run_matvec(c, x_dev, y_dev, mask);
}

int mf_residual(mf_ctx* c, const uint8_t* mask, const double* pbar, double* b_dev, double* meanP_host) {
  if (!c || !mask || !pbar || !b_dev) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  if (c->model < 0) return MF_INVALID_ARG;
  double* mean = c->at<double>(c->ores);
  int s = run_residual(c, mask, pbar, b_dev, mean);
  if (s) return s;
  if (meanP_host) {
    cudaError_t e = cudaMemcpyAsync(meanP_host, mean, 9 * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    return cuda_status(e);
  }
  return MF_OK;
}

int mf_solve(mf_ctx* c, int nsteps, const uint8_t* mask, const double* target, double tol_newton,
             double tol_cg, double cg_rel, int max_newton, int max_cg, double* Fbar_out,
             double* Pbar_out, int32_t* iters_out) {
  int s = check_solve_args(c, nsteps, mask, target, tol_newton, tol_cg, cg_rel, max_newton, max_cg);
  if (s) return s;
  if (!c->tuned && (s = autotune(c, 3))) return s;
  return solve_cell(c, nsteps, mask, target, tol_newton, tol_cg, cg_rel, max_newton, max_cg, Fbar_out, Pbar_out,
                    iters_out);
}

}  // extern "C"

namespace {

// The batched graph of the last mf_solve_batch call: every cell's history as
// a root chain of one graph, reused while the same contexts (by creation
// number and graph generation), masks and CG cap come back.
struct BatchGraph {
  std::vector<long long> key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
BatchGraph g_batch;
std::mutex g_batch_mutex;

void drop_batch_graph() {
  if (g_batch.exec) cudaGraphExecDestroy(g_batch.exec);
  if (g_batch.graph) cudaGraphDestroy(g_batch.graph);
  g_batch = BatchGraph();
}

}  // namespace

extern "C" {

int mf_solve_batch(int n, mf_ctx* const* ctxs, int nsteps, const uint8_t* masks, const double* targets,
                   double tol_newton, double tol_cg, double cg_rel, int max_newton, int max_cg,
                   double* Fbar_out, double* Pbar_out, int32_t* iters_out, int32_t* status_out) {
  if (n < 1 || !ctxs) return MF_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const int s = check_solve_args(ctxs[i], nsteps, masks ? masks + (size_t)9 * nsteps * i : nullptr,
                                   targets ? targets + (size_t)9 * nsteps * i : nullptr, tol_newton, tol_cg,
                                   cg_rel, max_newton, max_cg);
    if (s) return s;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return MF_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i) {
    if (ctxs[i]->tuned) continue;
    const int s = autotune(ctxs[i], 3);
    if (s) return s;
  }
  if (nsteps == 0) {
    if (status_out)
      for (int i = 0; i < n; ++i) status_out[i] = MF_OK;
    return MF_OK;
  }
  // one launch for all cells when each cell keeps one control mask over the
  // history and the history fits the step table; otherwise cell by cell
  bool one_launch = nsteps <= kHistSteps;
  for (int i = 0; i < n && one_launch; ++i) {
    const uint8_t* m = masks + (size_t)9 * nsteps * i;
    for (int k = 1; k < nsteps && one_launch; ++k) one_launch = same_mask(m + 9 * (size_t)k, m);
  }
  int first = MF_OK;
  if (!one_launch) {
    for (int i = 0; i < n; ++i) {
      const size_t o9 = (size_t)9 * nsteps * i;
      const int s = solve_cell(ctxs[i], nsteps, masks + o9, targets + o9, tol_newton, tol_cg, cg_rel, max_newton,
                               max_cg, Fbar_out ? Fbar_out + o9 : nullptr, Pbar_out ? Pbar_out + o9 : nullptr,
                               iters_out ? iters_out + (size_t)2 * nsteps * i : nullptr);
      if (status_out) status_out[i] = s;
      if (s && !first) first = s;
    }
    return first;
  }
  std::lock_guard<std::mutex> lk(g_batch_mutex);
  std::vector<long long> key;
  key.push_back(max_cg);
  for (int i = 0; i < n; ++i) {
    key.push_back(ctxs[i]->serial);
    key.push_back(ctxs[i]->gen);
    key.push_back((long long)mask_bits(masks + (size_t)9 * nsteps * i));
  }
  cudaError_t e = cudaSuccess;
  if (key != g_batch.key || !g_batch.exec) {
    drop_batch_graph();
    e = cudaGraphCreate(&g_batch.graph, 0);
    for (int i = 0; i < n && e == cudaSuccess; ++i)
      e = build_history(ctxs[i], g_batch.graph, masks + (size_t)9 * nsteps * i, max_cg);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g_batch.exec, g_batch.graph, 0);
    if (e != cudaSuccess) {
      drop_batch_graph();
      cudaGetLastError();
      return cuda_status(e);
    }
    g_batch.key = key;
  }
  // every cell's inputs on the launch stream, one launch, every cell's outputs
  cudaStream_t st = ctxs[0]->st;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    if (ctxs[i]->st != st) e = cudaStreamSynchronize(ctxs[i]->st);
    if (e == cudaSuccess && hist_staging(ctxs[i])) return MF_CUDA_ERROR;
  }
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const size_t o9 = (size_t)9 * nsteps * i;
    e = upload_history(ctxs[i], masks + o9, targets + o9, 0, nsteps, tol_newton, tol_cg, cg_rel, max_newton, max_cg,
                       st);
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(g_batch.exec, st);
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = download_history(ctxs[i], nsteps, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  for (int i = 0; i < n; ++i) {
    const size_t o9 = (size_t)9 * nsteps * i;
    const int s = finish_history(ctxs[i], 0, nsteps, Fbar_out ? Fbar_out + o9 : nullptr,
                                 Pbar_out ? Pbar_out + o9 : nullptr,
                                 iters_out ? iters_out + (size_t)2 * nsteps * i : nullptr);
    if (status_out) status_out[i] = s;
    if (s && !first) first = s;
  }
  return first;
}

int mf_get_fields(mf_ctx* c, double* F_host, double* P_host) {
  if (!c) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  cudaError_t e = cudaSuccess;
  if (F_host)
    e = cudaMemcpyAsync(F_host, c->ws + c->oF, 9 * c->N * sizeof(double), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess && P_host)
    e = cudaMemcpyAsync(P_host, c->ws + c->oP, 9 * c->N * sizeof(double), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  return cuda_status(e);
}

int mf_time_kernels(mf_ctx* c, const uint8_t* mask, int reps, int graph, float* ms_out) {
  if (!c || !mask || !ms_out || reps < 1 || (graph != 0 && graph != 1)) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  if (!operator_ready(c)) return MF_INVALID_ARG;
  const bool f32 = c->f32();
  const ZArgs za = z_args(c, f32, mask, 1.0 / (double)c->N);
  const XYArgs xa = xy_args(c, f32);
  const TangentArgs ta = tangent_args(c);
  Scalars* sc = c->at<Scalars>(c->osc);
  double* part = c->at<double>(c->opart);
  // operands: a CG state made of the context's vectors (values are not used
  // for anything but timing); alpha = beta = 0 keeps them bounded; its = 1:
  // a later iteration's tangent pass (the first one reads two vectors less)
  static const int kOne = 1;
  cudaError_t e = cudaMemsetAsync(c->ws + c->osc, 0, sizeof(Scalars), c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sc->its, &kOne, sizeof(int), cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess && graph && !c->cap_st) {
    e = cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking);
    if (e != cudaSuccess) c->cap_st = nullptr;
  }
  cudaEvent_t e0, e1;
  if (e != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess) return MF_CUDA_ERROR;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return MF_CUDA_ERROR; }
  auto flush = [&](cudaStream_t s, int r) {   // L2 flush: a memset larger than L2
    return cudaMemsetAsync(c->ws + c->ob, r & 0xff, 9 * c->N * sizeof(double), s);
  };
  auto kernel = [&](cudaStream_t s, int which) {
    if (which == 0)
      return mf_launch_tangent(c->ws + c->op, c->ws + c->or_, c->ws + c->op2, c->ws + c->ox, f32, tangent_kind(c),
                               true, ta, c->ws + c->oAp, c->N, part, c->pw_blocks, sc, s);
    return mf_launch_project_part(which - 1, f32, c->ws + c->oAp, c->ws + c->ospec, c->ws + c->or_, part, xa, za,
                                  sc, s);
  };
  // graph mode: `reps` (flush, kernel) pairs captured as one graph, timed
  // with events around one launch of it, minus the same graph of flushes
  // alone; what is left is the kernels and their share of the gaps between
  // graph nodes (and the write-back of their dirty lines by the next flush)
  auto graph_ms = [&](int which, float* ms) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaError_t ee = cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeRelaxed);
    for (int r = 0; r < reps && ee == cudaSuccess; ++r) {
      ee = flush(c->cap_st, r);
      if (ee == cudaSuccess && which >= 0) ee = kernel(c->cap_st, which);
    }
    const cudaError_t ec = cudaStreamEndCapture(c->cap_st, &g);
    if (ee == cudaSuccess) ee = ec;
    if (ee == cudaSuccess) ee = cudaGraphInstantiate(&ge, g, 0);
    if (ee == cudaSuccess) ee = cudaGraphLaunch(ge, c->st);   // untimed: first touches
    if (ee == cudaSuccess) ee = cudaEventRecord(e0, c->st);
    if (ee == cudaSuccess) ee = cudaGraphLaunch(ge, c->st);
    if (ee == cudaSuccess) ee = cudaEventRecord(e1, c->st);
    if (ee == cudaSuccess) ee = cudaEventSynchronize(e1);
    if (ee == cudaSuccess) ee = cudaEventElapsedTime(ms, e0, e1);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    return ee;
  };
  float base = 0.f;
  if (graph) e = graph_ms(-1, &base);
  for (int which = 0; which < 4 && e == cudaSuccess; ++which) {
    if (graph) {
      float ms = 0.f;
      e = graph_ms(which, &ms);
      ms_out[which] = (ms - base) / (float)reps;
      continue;
    }
    double tot = 0.0;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
      e = flush(c->st, r);
      if (e == cudaSuccess) e = cudaEventRecord(e0, c->st);
      if (e == cudaSuccess) e = kernel(c->st, which);
      if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      tot += ms;
    }
    ms_out[which] = (float)(tot / reps);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) cudaGetLastError();
  return cuda_status(e);
}

int mf_adjoint(mf_ctx* c, const uint8_t* mask, const double* wF, const double* wP, double tol_cg, double cg_rel,
               int max_cg, double* J_out, double* dJ_dparams, double* dJ_dscale_dev, int32_t* cg_its_out) {
  if (!c || !mask || !wF || !wP || !(tol_cg > 0) || !(cg_rel >= 0) || max_cg < 1) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  if (c->model != MF_NEOHOOKE || c->nphase > 2048 || 2LL * c->nphase > 9 * c->N) return MF_INVALID_ARG;
  for (int k = 0; k < 9; ++k)
    if (mask[k] > 1 || !isfinite(wF[k]) || !isfinite(wP[k])) return MF_INVALID_ARG;
  int s = MF_OK;
  if (!c->tuned && (s = autotune(c, 3))) return s;
  const bool f32 = c->f32();
  const long long N = c->N;
  AdjWeights w;
  memcpy(w.wF, wF, sizeof(w.wF));
  memcpy(w.wP, wP, sizeof(w.wP));
  Scalars* sc = c->at<Scalars>(c->osc);
  double* part = c->at<double>(c->opart);
  double* F = c->at<double>(c->oF);
  double* b = c->at<double>(c->ob);
  // P and the tangent at F (FP32: H and the rotation moments)
  s = run_constitutive(c, !f32, f32, f32);
  Scalars h;
  if (!s) s = read_scalars(c, &h);
  if (!s) s = flags_status(h.flags);
  if (s) return s;
  // right-hand side G*(W_F + K : W_P)
  const XYArgs xa = xy_args(c, f32);
  const ZArgs za = z_args(c, f32, mask, 1.0 / (double)N);
  cudaError_t e = mf_launch_adj_rhs_fill(c->ws + c->op, f32, N, w, c->st);
  if (e == cudaSuccess)
    e = mf_launch_tangent(c->ws + c->op, nullptr, nullptr, nullptr, f32, tangent_kind(c), false, tangent_args(c),
                          c->ws + c->oAp, N, nullptr, c->pw_blocks, nullptr, c->st);
  if (e == cudaSuccess) e = mf_launch_adj_rhs_add(c->ws + c->oAp, f32, N, w, c->st);
  if (e == cudaSuccess)
    e = mf_launch_project(f32, c->ws + c->oAp, c->ws + c->ospec, c->ws + c->op2, 0, nullptr, xa, za, nullptr,
                          c->st);
  if (e == cudaSuccess) e = mf_launch_to_double(c->ws + c->op2, b, f32, 9 * N, c->st);
  // FP32: the same null-rotation deflation as the Newton iterations
  Defl defl;
  defl.m = 0;
  if (e == cudaSuccess && f32) {
    defl = null_rotations(h.meanF, mask, h.T, h.S, c->kappa, 1e-6);
    if (defl.m > 0) e = mf_launch_defl_project(b, false, true, F, N, defl, part, c->pw_blocks, sc, c->st);
  }
  if (e != cudaSuccess) return cuda_status(e);
  s = launch_cg(c, mask, tol_cg, cg_rel, max_cg);
  Scalars hc;
  if (!s) s = read_scalars(c, &hc);
  if (s) return s;
  g_mf_launches += (long long)c->cg_body_kernels * (hc.its == 0 ? 1 : (hc.its + 1) / 2);
  bool clear = false;
  s = cg_outcome(c, hc, &clear);
  if (s) return s;
  if (clear) e = cudaMemsetAsync(&sc->flags, 0, sizeof(int), c->st);
  if (e == cudaSuccess && defl.m > 0)
    e = mf_launch_defl_project(c->ws + c->ox, true, true, F, N, defl, part, c->pw_blocks, sc, c->st);
  // parameter derivatives; the per-phase sums land in b (free after the CG start)
  const int per = 2 * c->nphase;
  int nblk = (int)(c->npart / per);
  if (nblk > c->pw_blocks) nblk = c->pw_blocks;
  if (e == cudaSuccess)
    e = mf_launch_adj_grad(F, c->at<double>(c->oP), c->ws + c->ox, f32, c->at<int32_t>(c->ophase),
                           c->has_scale ? c->at<double>(c->oscale) : nullptr, N, c->nphase, w, part, nblk, b,
                           dJ_dscale_dev, c->st);
  if (e == cudaSuccess && dJ_dparams)
    e = cudaMemcpyAsync(dJ_dparams, b, per * sizeof(double), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_status(e);
  if (J_out) {
    double J = 0.0;
    for (int k = 0; k < 9; ++k) J += wF[k] * h.meanF[k] + wP[k] * h.meanP[k];
    *J_out = J;
  }
  if (cg_its_out) *cg_its_out = hc.its;
  return MF_OK;
}

int mf_set_xy_split(mf_ctx* c, int split) {
  if (!c || (split != 0 && split != 1)) return MF_INVALID_ARG;
  if (split && !(c->v2 && mf_split_supported(c->nx))) return MF_INVALID_ARG;
  const bool big_plane = (size_t)(c->ny / 2) * c->nx * sizeof(double2) + (size_t)(c->nx + c->ny) * 20 > 200 * 1024;
  if (!split && big_plane) return MF_INVALID_ARG;
  if (c->xy_split != split) free_cg_graph(c);   // the captured loop holds the old kernels
  c->xy_split = split;
  return MF_OK;
}

int mf_set_xy_persistent(mf_ctx* c, int on) {
  if (!c || (on != 0 && on != 1)) return MF_INVALID_ARG;
  if (on && !(c->prec == MF_FP32_INNER && c->v2 && !c->xy_split && mf_persist_supported(c->nx)))
    return MF_INVALID_ARG;
  if (c->xy_persist != on) free_cg_graph(c);   // the captured loop holds the old kernels
  c->xy_persist = on;
  c->xy_persist_user = 1;
  return MF_OK;
}

int mf_set_xy_cluster(mf_ctx* c, int which) {
  if (!c || which < 0 || which > 3) return MF_INVALID_ARG;
  if (which && !(c->prec == MF_FP32_INNER && c->v2 && !c->xy_split && mf_cluster_supported(c->nx)))
    return MF_INVALID_ARG;
  if (c->xy_cluster != which) free_cg_graph(c);   // the captured loop holds the old kernels
  c->xy_cluster = which;
  c->xy_cluster_user = 1;
  return MF_OK;
}

int mf_xy_schedule(mf_ctx* c, int32_t* fwd_out, int32_t* inv_out, float* ms_out) {
  if (!c) return MF_INVALID_ARG;
  const bool clu = c->prec == MF_FP32_INNER && c->v2 && !c->xy_split && mf_cluster_supported(c->nx);
  if (fwd_out) *fwd_out = (clu && (c->xy_cluster & 1)) ? 2 : c->xy_persist;
  if (inv_out) *inv_out = (clu && (c->xy_cluster & 2)) ? 2 : 0;
  if (ms_out) {
    for (int i = 0; i < 5; ++i) ms_out[i] = -1.f;
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (const TuneEntry& t : g_tune_cache)
      if (t.nx == c->nx && t.ny == c->ny && t.nz == c->nz && t.prec == c->prec &&
          t.dw == (c->dw_residual() ? 1 : 0)) {
        for (int i = 0; i < 3; ++i) ms_out[i] = t.msxy[i];
        for (int i = 0; i < 2; ++i) ms_out[3 + i] = t.msxi[i];
      }
  }
  return MF_OK;
}

int mf_set_projection_arith(mf_ctx* c, int arith) {
  if (!c || (arith != MF_PROJ_FP32 && arith != MF_PROJ_OUTER && arith != MF_PROJ_AUTO)) return MF_INVALID_ARG;
  if (arith != MF_PROJ_FP32 && c->prec != MF_FP32_INNER) return MF_INVALID_ARG;
  c->proj_arith = arith;
  return MF_OK;
}

int mf_set_predictor(mf_ctx* c, int kind) {
  if (!c || (kind != MF_PRED_UNIFORM && kind != MF_PRED_EXTRAPOLATE && kind != MF_PRED_QUADRATIC))
    return MF_INVALID_ARG;
  if (c->predictor != kind) free_cg_graph(c);   // the captured histories hold the predictor's passes
  c->predictor = kind;
  return MF_OK;
}

int mf_set_inexact_newton(mf_ctx* c, int on) {
  if (!c || (on != 0 && on != 1)) return MF_INVALID_ARG;
  if (c->f32() && !on) return MF_INVALID_ARG;
  c->forcing64 = on != 0;
  return MF_OK;
}

int mf_set_outer_arith(mf_ctx* c, int arith) {
  if (!c || (arith != MF_OUTER_DOUBLE_WORD && arith != MF_OUTER_FP64)) return MF_INVALID_ARG;
  if (c->outer_arith != arith) {
    c->tuned = false;    // the residual tile is tuned per arithmetic
    free_cg_graph(c);    // the captured histories hold the outer level's kernels
  }
  c->outer_arith = arith;
  return MF_OK;
}

long long mf_kernel_launches(void) { return g_mf_launches; }

int mf_trace_read(int cap, unsigned long long* t_ns, int* ids, int* n_out) {
#ifdef MF_TRACE
  if (cap < 0 || !n_out || (cap > 0 && (!t_ns || !ids))) return MF_INVALID_ARG;
  int n = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return MF_CUDA_ERROR;
  if (cudaMemcpyFromSymbol(&n, g_trace_n, sizeof(int)) != cudaSuccess) return MF_CUDA_ERROR;
  const int k = n < kTraceCap ? (n < cap ? n : cap) : (kTraceCap < cap ? kTraceCap : cap);
  if (k > 0 && (cudaMemcpyFromSymbol(t_ns, g_trace_t, sizeof(unsigned long long) * k) != cudaSuccess ||
                cudaMemcpyFromSymbol(ids, g_trace_id, sizeof(int) * k) != cudaSuccess))
    return MF_CUDA_ERROR;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_trace_n, &zero, sizeof(int)) != cudaSuccess) return MF_CUDA_ERROR;
  *n_out = n;
  return MF_OK;
#else
  (void)cap; (void)t_ns; (void)ids;
  if (n_out) *n_out = 0;
  return MF_INVALID_ARG;
#endif
}

int mf_debug_report(long long* count_out, int* line_out, long long* index_out, long long* extent_out) {
  if (!count_out) return MF_INVALID_ARG;
#ifdef MF_DEBUG
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e);
  long long total = 0;
  bool have = false;
  for (const DebugReader& r : debug_readers()) {
    MfDebugRecord rec;
    memset(&rec, 0, sizeof(rec));
    r.read(&rec);
    total += (long long)rec.count;
    if (rec.count && !have) {
      have = true;
      if (line_out) *line_out = rec.line;
      if (index_out) *index_out = rec.index;
      if (extent_out) *extent_out = rec.extent;
    }
    r.clear();
  }
  *count_out = total;
  return cuda_status(cudaGetLastError());
#else
  (void)line_out;
  (void)index_out;
  (void)extent_out;
  *count_out = -1;
  return MF_OK;
#endif
}

int mf_sync(mf_ctx* c) {
  if (!c) return MF_INVALID_ARG;
  return cuda_status(cudaStreamSynchronize(c->st));
}

namespace {
__device__ int g_selftest_flags;   // the self-test's flag word (no allocation)
}

int mf_selftest_wait_timeout(int max_polls) {
  if (max_polls < 1 || max_polls > (1 << 20)) return MF_INVALID_ARG;
  int* flags = nullptr;
  const int zero = 0;
  int got = 0;
  cudaError_t e = cudaGetSymbolAddress((void**)&flags, g_selftest_flags);
  if (e == cudaSuccess) e = cudaMemcpy(flags, &zero, sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = mf_launch_wait_selftest(max_polls, flags, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(&got, flags, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  return flags_status(got);
}

const char* mf_last_cuda_error(void) { return g_last_cuda_error; }

int mf_autotune(mf_ctx* c, int32_t* zs_out, float* ms_out, int32_t* xy_out, float* xy_ms_out) {
  if (!c) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  c->tuned = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (size_t i = 0; i < g_tune_cache.size(); ++i) {
      const TuneEntry& t = g_tune_cache[i];
      if (t.nx == c->nx && t.ny == c->ny && t.nz == c->nz && t.prec == c->prec &&
          t.dw == (c->dw_residual() ? 1 : 0)) {
        g_tune_cache.erase(g_tune_cache.begin() + i);
        break;
      }
    }
  }
  const int s = autotune(c, 5);
  if (s) return s;
  if (zs_out) *zs_out = c->zS;
  if (ms_out) {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (const TuneEntry& t : g_tune_cache)
      if (t.nx == c->nx && t.ny == c->ny && t.nz == c->nz && t.prec == c->prec &&
          t.dw == (c->dw_residual() ? 1 : 0))
        for (int i = 0; i < 3; ++i) ms_out[i] = t.ms[i];
  }
  if (xy_out) *xy_out = (c->xy_cluster & 1) && mf_cluster_supported(c->nx) ? 2 : c->xy_persist;
  if (xy_ms_out) {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (const TuneEntry& t : g_tune_cache)
      if (t.nx == c->nx && t.ny == c->ny && t.nz == c->nz && t.prec == c->prec &&
          t.dw == (c->dw_residual() ? 1 : 0))
        for (int i = 0; i < 2; ++i) xy_ms_out[i] = t.msxy[i];
  }
  return MF_OK;
}

void mf_destroy(mf_ctx* c) {
  if (!c) return;
  free_cg_graph(c);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  for (cudaStream_t s : c->caps)
    if (s) cudaStreamDestroy(s);
  if (c->pin) cudaFreeHost(c->pin);
  mf_cufft_delete(c->cufft);
  delete c;
}

size_t mf_cufft_workspace_bytes(mf_ctx* c) {
  if (!c) return 0;
  if (!c->cufft) c->cufft = mf_cufft_new();
  size_t need = 0;
  if (mf_cufft_plan(c->cufft, c->nx, c->ny, c->nz, c->f32(), c->st, &need) != MF_OK) return 0;
  return need;
}

int mf_cufft_bind(mf_ctx* c, void* dev, size_t bytes) {
  if (!c || !dev || ((uintptr_t)dev & 255)) return MF_INVALID_ARG;
  const size_t need = mf_cufft_workspace_bytes(c);
  if (need == 0) return MF_CUDA_ERROR;
  if (bytes < need) return MF_INVALID_ARG;
  const int s = mf_cufft_bind(c->cufft, dev);
  c->cufft_bound = (s == MF_OK);
  return s;
}

int mf_matvec_cufft(mf_ctx* c, const void* x_dev, void* y_dev, const uint8_t* mask) {
  if (!c || !x_dev || !y_dev || !mask || x_dev == y_dev) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  if (!c->cufft_bound || !operator_ready(c)) return MF_INVALID_ARG;
  cudaError_t e = mf_launch_tangent(x_dev, nullptr, nullptr, nullptr, c->f32(), tangent_kind(c), false,
                                    tangent_args(c), c->ws + c->oAp, c->N, nullptr, c->pw_blocks,
                                    nullptr, c->st);
  if (e != cudaSuccess) return MF_CUDA_ERROR;
  return mf_cufft_project(c->cufft, c->f32(), c->ws + c->oAp, y_dev, c->nx, c->ny, c->nz, mask, c->st, -1);
}

int mf_time_cufft(mf_ctx* c, const uint8_t* mask, int reps, float* ms_out) {
  if (!c || !mask || !ms_out || reps < 1) return MF_INVALID_ARG;
  if (!c->ws) return MF_NO_WORKSPACE;
  if (!c->cufft_bound) return MF_INVALID_ARG;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MF_CUDA_ERROR;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return MF_CUDA_ERROR; }
  int s = MF_OK;
  for (int which = 0; which < 3 && s == MF_OK; ++which) {
    double tot = 0.0;
    for (int r = 0; r < reps && s == MF_OK; ++r) {
      cudaError_t e = cudaMemsetAsync(c->ws + c->ob, r & 0xff, 9 * c->N * sizeof(double), c->st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, c->st);
      if (e != cudaSuccess) { s = MF_CUDA_ERROR; break; }
      s = mf_cufft_project(c->cufft, c->f32(), c->ws + c->oAp, c->ws + c->or_, c->nx, c->ny, c->nz, mask,
                           c->st, which);
      if (s) break;
      e = cudaEventRecord(e1, c->st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) { s = MF_CUDA_ERROR; break; }
      tot += ms;
    }
    ms_out[which] = (float)(tot / reps);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

}  // extern "C"
