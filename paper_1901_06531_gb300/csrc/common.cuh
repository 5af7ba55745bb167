// Shared device machinery: complex helpers, per-axis FFT plans and the
// in-place shared-memory FFT stages used by every transform kernel.
//
// Transforms are computed in place with mixed-radix (2, 3, 4) stages.  The
// forward transform is decimation in frequency (natural order in, digit-
// reversed order out), the inverse is its exact adjoint, decimation in time
// (digit-reversed in, natural out).  The spectrum therefore never needs a
// reordering pass: the projection is applied in digit-reversed order, with
// each position's frequency read from a small table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define MF_MAX_STAGES 10

// Bounds checks of the debug build (compiled with -DMF_DEBUG; release builds
// compile them away).  MF_AT(i, n) is i when 0 <= i < n; otherwise the
// failure is counted, the first one (source line, index, extent) recorded,
// and element 0 -- in bounds -- is used instead, so that the kernel runs to
// its end and the host reads the record (mf_debug_report) rather than the
// GPU faulting.  Every translation unit has its own record and registers a
// reader and a reset for it with the library at load time.
#ifdef MF_DEBUG
struct MfDebugRecord {
  unsigned long long count;
  long long index, extent;
  int line, pad;
};
void mf_debug_register(void (*read)(MfDebugRecord*), void (*clear)());
static __device__ MfDebugRecord g_mf_debug;
static void mf_debug_read_tu(MfDebugRecord* r) { cudaMemcpyFromSymbol(r, g_mf_debug, sizeof(*r)); }
static void mf_debug_clear_tu() {
  MfDebugRecord z = {0ull, 0, 0, 0, 0};
  cudaMemcpyToSymbol(g_mf_debug, &z, sizeof(z));
}
static const bool g_mf_debug_registered = (mf_debug_register(mf_debug_read_tu, mf_debug_clear_tu), true);
__device__ __forceinline__ long long mf_dbg_check(long long i, long long n, int line) {
  if (i >= 0 && i < n) return i;
  if (atomicAdd(&g_mf_debug.count, 1ull) == 0ull) {
    g_mf_debug.index = i;
    g_mf_debug.extent = n;
    g_mf_debug.line = line;
  }
  return 0;
}
#define MF_AT(i, n) mf_dbg_check((long long)(i), (long long)(n), __LINE__)
#else
#define MF_AT(i, n) (i)
#endif

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may be scheduled as soon as the blocks of
// its predecessor in the stream have exited, before that grid's completion
// (its memory flush) and the launch that would normally follow it; pdl_wait()
// returns once the predecessor grid has completed and its memory operations
// are visible.  For a kernel launched without the attribute it returns at
// once.  (No kernel here signals its dependents early: measured on the 128^3
// cell, dependents resident during the predecessor's last wave slowed it.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Grid of a grid-stride elementwise pass over n items with `threads` per
// block: one item per thread for small passes, at most 8 blocks per SM (152
// SMs) otherwise.
inline int stride_grid(long long n, int threads = 256) {
  const long long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b < 152 * 8 ? b : 152 * 8));
}

struct AxisPlan {
  int n;                     // transform length
  int nst;                   // number of stages
  int rad[MF_MAX_STAGES];    // radix of each stage in DIF order
};

template <typename T> struct CT;
template <> struct CT<double> { typedef double2 t; };
template <> struct CT<float> { typedef float2 t; };

__device__ __forceinline__ double2 cmake(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 cmake(float a, float b) { return make_float2(a, b); }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
#ifndef MF_NO_F32X2
// FP32 complex add and subtract as one packed two-lane instruction (sm_100
// and later: add.f32x2, sub.f32x2), each lane rounded to nearest like the
// scalar pair; the butterflies of the FP32 transforms are mostly these.
__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
#endif
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
// multiply by -i (FWD) or +i (INV)
template <typename C, bool INV> __device__ __forceinline__ C rot90(C a) {
  C r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

// Small DFT of length R on registers: y_k = sum_j x_j w^(jk), w = exp(-+2 pi i/R).
template <int R, bool INV, typename C> struct Radix;

template <bool INV, typename C> struct Radix<2, INV, C> {
  static __device__ __forceinline__ void run(C* v) {
    C a = v[0], b = v[1]; v[0] = cadd(a, b); v[1] = csub(a, b);
  }
};

template <bool INV, typename C> struct Radix<4, INV, C> {
  static __device__ __forceinline__ void run(C* v) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = rot90<C, INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
  }
};

template <bool INV, typename C> struct Radix<3, INV, C> {
  static __device__ __forceinline__ void run(C* v) {
    typedef decltype(v[0].x) T;
    const T h = (T)0.5;
    const T s3 = (T)0.86602540378443864676372317075294;   // sin(2 pi / 3)
    C a = v[0];
    C t1 = cadd(v[1], v[2]);
    C d = csub(v[1], v[2]);
    C t2; t2.x = a.x - h * t1.x; t2.y = a.y - h * t1.y;
    // forward: y1 = t2 - i s3 d, y2 = t2 + i s3 d; inverse: signs of i swap
    C t3; t3.x = s3 * d.x; t3.y = s3 * d.y;
    C it3 = rot90<C, INV>(t3);     // -i*t3 forward, +i*t3 inverse
    v[0] = cadd(a, t1);
    v[1] = cadd(t2, it3);
    v[2] = csub(t2, it3);
  }
};

// One in-place radix-R stage over `nseq` sequences of length n in shared
// memory.  Element j of sequence s is at buf[(s / nlo) * hs + (s % nlo) * ls + j * es].
// L is the current sub-transform length (n at the first DIF stage); the
// twiddle table holds W_ntab^t = exp(-2 pi i t / ntab) with n | ntab.
// SEQ_FAST chooses the thread order: consecutive threads walk sequences
// (strided transforms) or butterflies (contiguous transforms).
template <typename C, int R, bool INV, bool SEQ_FAST>
__device__ __forceinline__ void fft_stage(C* buf, int n, int L, int nseq, int nlo, int hs,
                                          int ls, int es, const C* tw, int ntab, int ext) {
  const int m = L / R;
  const int nb = n / R;
  const int total = nb * nseq;
  const int tstep = ntab / L;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int s, b;
    if (SEQ_FAST) { s = t % nseq; b = t / nseq; } else { b = t % nb; s = t / nb; }
    const int blk = b / m;
    const int j0 = b - blk * m;
    const int base = (s / nlo) * hs + (s % nlo) * ls + (blk * L + j0) * es;
    const int step = m * es;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = buf[MF_AT(base + r * step, ext)];
    if (!INV) {
      Radix<R, false, C>::run(v);
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul(v[k], tw[MF_AT(j0 * k * tstep, ntab)]);
    } else {
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], tw[MF_AT(j0 * k * tstep, ntab)]);
      Radix<R, true, C>::run(v);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) buf[MF_AT(base + r * step, ext)] = v[r];
  }
}

template <typename C, bool INV, bool SEQ_FAST>
__device__ __forceinline__ void fft_stage_dispatch(int R, C* buf, int n, int L, int nseq, int nlo,
                                                   int hs, int ls, int es, const C* tw, int ntab, int ext) {
  if (R == 4) fft_stage<C, 4, INV, SEQ_FAST>(buf, n, L, nseq, nlo, hs, ls, es, tw, ntab, ext);
  else if (R == 2) fft_stage<C, 2, INV, SEQ_FAST>(buf, n, L, nseq, nlo, hs, ls, es, tw, ntab, ext);
  else fft_stage<C, 3, INV, SEQ_FAST>(buf, n, L, nseq, nlo, hs, ls, es, tw, ntab, ext);
}

// Full transform of every sequence: DIF forward (INV = false) or its adjoint
// DIT inverse (INV = true, unnormalised).  Ends with __syncthreads(); the
// caller synchronises before the first stage.  ext: elements of buf (the
// debug build checks every index against it).
template <typename C, bool INV, bool SEQ_FAST>
__device__ __forceinline__ void fft_run(C* buf, const AxisPlan& pl, int nseq, int nlo, int hs,
                                        int ls, int es, const C* tw, int ntab, int ext) {
  if (!INV) {
    int L = pl.n;
    for (int st = 0; st < pl.nst; ++st) {
      const int R = pl.rad[st];
      fft_stage_dispatch<C, false, SEQ_FAST>(R, buf, pl.n, L, nseq, nlo, hs, ls, es, tw, ntab, ext);
      L /= R;
      __syncthreads();
    }
  } else {
    int Ls[MF_MAX_STAGES];
    int L = pl.n;
    for (int st = 0; st < pl.nst; ++st) { Ls[st] = L; L /= pl.rad[st]; }
    for (int st = pl.nst - 1; st >= 0; --st) {
      fft_stage_dispatch<C, true, SEQ_FAST>(pl.rad[st], buf, pl.n, Ls[st], nseq, nlo, hs, ls, es,
                                            tw, ntab, ext);
      __syncthreads();
    }
  }
}

// Index of the packed symmetric 9x9 tangent entry (a, b), a, b in [0, 9).
__host__ __device__ __forceinline__ int sym45(int a, int b) {
  if (a > b) { int t = a; a = b; b = t; }
  return a * 9 - (a * (a - 1)) / 2 + (b - a);
}

// Device-side scalar block shared by the Newton/CG kernels (FP64).
struct Scalars {
  double rr;          // current r.r
  double rr0;         // r.r at CG start
  double pAp;
  double alpha;
  double beta;
  double thr2N;       // CG stop: rr <= thr2N
  double meanF[9];
  double meanP[9];
  double dF2max;      // max_v |dF_v|^2 of the last Newton update
  double meanF_new[9];
  double T[9];        // sum_v P_v F_v^T   (rotation moments, row-major)
  double S[9];        // sum_v F_v F_v^T
  double What[9];     // skew matrix of the last null-rotation projection
  double lin[9];      // FP32 inner solve: sum over its iterations of alpha_k <t_k> (= <K:x>, x = sum alpha_k p_k)
  int flags;          // bit 0: breakdown, bit 1: nonpositive J, bit 2: non-finite
  int done;           // CG converged
  int its;            // CG iterations completed
  int stop;           // CG finished (converged, failed or capped): iteration kernels return at once
  int max_its;
  unsigned arrive;    // blocks of the current pass that have stored their partial sum
};

// Grid-wide sum finished by the last block to arrive: every block has stored
// its partial sum in partials[blockIdx.x] (thread 0 wrote it); thread 0
// publishes it and counts the block in *arrive.  The block that arrives last
// adds all partials in a fixed order, leaves the total in *total (read by
// every thread), resets the counter and returns true; the others return
// false.  No block waits on another.
__device__ __forceinline__ bool last_block_total(const double* partials, unsigned* arrive, double* total) {
  __shared__ unsigned s_last;
  __shared__ double s_red[32];
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(arrive, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double s = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += __ldcg(partials + b);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < (blockDim.x >> 5)) ? s_red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) { s_red[0] = t; *arrive = 0u; }
  }
  __syncthreads();
  *total = s_red[0];
  return true;
}

#define MF_FLAG_BREAKDOWN 1
#define MF_FLAG_NONPOS_J 2
#define MF_FLAG_NONFINITE 4
#define MF_FLAG_TIMEOUT 8     // a bounded device-side wait gave up

// CG scalar updates after the curvature p.Ap and after the new r.r (shared by
// the one-block finishing kernels and the last blocks of fused passes).
__device__ __forceinline__ void cg_finish_alpha(double pAp, Scalars* sc) {
  sc->pAp = pAp;
  if (!(pAp > 0.0) || !isfinite(pAp)) {
    sc->flags |= MF_FLAG_BREAKDOWN;
    sc->alpha = 0.0;
    sc->stop = 1;
  } else {
    sc->alpha = sc->rr / pAp;
  }
}

__device__ __forceinline__ void cg_finish_beta(double rr, Scalars* sc) {
  if (!isfinite(rr)) sc->flags |= MF_FLAG_NONFINITE;
  sc->beta = rr / sc->rr;
  sc->rr = rr;
  sc->done = (rr <= sc->thr2N) ? 1 : 0;
  sc->its += 1;
  sc->stop = (sc->done || sc->flags || sc->its >= sc->max_its) ? 1 : 0;
}
