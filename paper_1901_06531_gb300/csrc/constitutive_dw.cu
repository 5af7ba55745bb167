// Constitutive update P(F) (Eq. eq:lineariz's P; no tangent) in double-word
// FP32 arithmetic for the FP32-inner mode, with the voxel averages of F and
// P, optionally the FP32 H = F - I of the matrix-free tangent and the
// rotation moments, in one pass over F.  A variant evaluates P in plain
// FP32 and stores it in FP32 (the first Newton iteration of a step).
//
// Both laws are evaluated from H = F - I, so that no large term cancels:
//   St Venant-Kirchhoff  E = (H + H^T + H^T H)/2, S = C : E, P = S + H S;
//   neo-Hookean          J - 1 = tr H + (tr^2 H - tr H^2)/2 + det H,
//                        P = mu F + (lam ln J - mu) F^-T, F^-T = cof(F)/J,
// every product and sum in double-word arithmetic (about 48 bits), ln J
// from FP64 log1p of J - 1.  F is read and P written in FP64.
#include "dw.cuh"
#include "launch.h"
#include "predict.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ dw half(dw a) { return dw(0.5f * a.hi, 0.5f * a.lo); }   // exact
__device__ __forceinline__ dw twice(dw a) { return dw(2.0f * a.hi, 2.0f * a.lo); }  // exact
__device__ __forceinline__ constexpr int vgt(int i, int j) {
  return i == j ? i : (i + j == 3 ? 3 : (i + j == 2 ? 4 : 5));
}

// Every sum of products below is one compensated accumulation (DwAcc).
__device__ __forceinline__ void svk_dw(const dw (&h)[9], const dw* __restrict__ cv, dw (&P)[9]) {
  dw e6[6];
  auto E = [&](int a, int b) {
    DwAcc s(h[3 * a + b]);
    s.add(h[3 * b + a]);
#pragma unroll
    for (int k = 0; k < 3; ++k) s.fma(h[3 * k + a], h[3 * k + b]);
    return half(s.value());
  };
  e6[0] = E(0, 0); e6[1] = E(1, 1); e6[2] = E(2, 2);
  e6[3] = twice(E(1, 2)); e6[4] = twice(E(0, 2)); e6[5] = twice(E(0, 1));
  dw sv[6];
#pragma unroll
  for (int I = 0; I < 6; ++I) {
    DwAcc acc(cv[6 * I] * e6[0]);
#pragma unroll
    for (int J = 1; J < 6; ++J) acc.fma(cv[6 * I + J], e6[J]);
    sv[I] = acc.value();
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      DwAcc acc(sv[vgt(i, j)]);
#pragma unroll
      for (int k = 0; k < 3; ++k) acc.fma(h[3 * i + k], sv[vgt(k, j)]);
      P[3 * i + j] = acc.value();
    }
}

// Returns false when J <= 0 (P is then zero).
__device__ __forceinline__ bool neohooke_dw(const dw (&h)[9], const dw (&f)[9], dw mu, dw lam, dw (&P)[9]) {
  const dw one(1.0f, 0.0f);
  // a b - c d
  auto det2 = [](dw a, dw b, dw c, dw d) {
    DwAcc s;
    s.fma(a, b);
    s.fma(-c, d);
    return s.value();
  };
  DwAcc tr(h[0]);
  tr.add(h[4]);
  tr.add(h[8]);
  const dw trH = tr.value();
  DwAcc t2;   // tr(H H) = sum_i h_ii^2 + 2 sum_(i<j) h_ij h_ji
  t2.fma(h[0], h[0]);
  t2.fma(h[4], h[4]);
  t2.fma(h[8], h[8]);
  t2.fma(twice(h[1]), h[3]);
  t2.fma(twice(h[2]), h[6]);
  t2.fma(twice(h[5]), h[7]);
  const dw trH2 = t2.value();
  DwAcc dh;   // det H by the first row
  dh.fma(h[0], det2(h[4], h[8], h[5], h[7]));
  dh.fma(-h[1], det2(h[3], h[8], h[5], h[6]));
  dh.fma(h[2], det2(h[3], h[7], h[4], h[6]));
  DwAcc q;    // (tr^2 H - tr H^2) / 2
  q.fma(trH, trH);
  q.add(-trH2);
  DwAcc jm(trH);
  jm.add(half(q.value()));
  jm.add(dh.value());
  const dw Jm1 = jm.value();
  const dw J = Jm1 + one;
  if (!(J.hi > 0.0f)) {
#pragma unroll
    for (int c = 0; c < 9; ++c) P[c] = dw(0.0f, 0.0f);
    return false;
  }
  const dw iJ = one / J;
  dw G[9];   // F^-T = cof(F) / J
  G[0] = det2(f[4], f[8], f[5], f[7]) * iJ;
  G[1] = det2(f[5], f[6], f[3], f[8]) * iJ;
  G[2] = det2(f[3], f[7], f[4], f[6]) * iJ;
  G[3] = det2(f[2], f[7], f[1], f[8]) * iJ;
  G[4] = det2(f[0], f[8], f[2], f[6]) * iJ;
  G[5] = det2(f[1], f[6], f[0], f[7]) * iJ;
  G[6] = det2(f[1], f[5], f[2], f[4]) * iJ;
  G[7] = det2(f[2], f[3], f[0], f[5]) * iJ;
  G[8] = det2(f[0], f[4], f[1], f[3]) * iJ;
  const dw lnJ = dw_split(log1p(dw_join(Jm1)));
  const dw cg = lam * lnJ - mu;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    DwAcc pc;
    pc.fma(mu, f[c]);
    pc.fma(cg, G[c]);
    P[c] = pc.value();
  }
  return true;
}

// The same laws in plain FP32 from H (the first Newton iteration of a load
// step, whose residual is taken with FP32 transforms anyway).
__device__ __forceinline__ void svk_f32(const float (&h)[9], const float* __restrict__ cv, float (&P)[9]) {
  auto E = [&](int a, int b) {
    return 0.5f * (h[3 * a + b] + h[3 * b + a] + h[a] * h[b] + h[3 + a] * h[3 + b] + h[6 + a] * h[6 + b]);
  };
  const float e6[6] = {E(0, 0), E(1, 1), E(2, 2), 2.f * E(1, 2), 2.f * E(0, 2), 2.f * E(0, 1)};
  float sv[6];
#pragma unroll
  for (int I = 0; I < 6; ++I) {
    float acc = 0.f;
#pragma unroll
    for (int J = 0; J < 6; ++J) acc = fmaf(cv[6 * I + J], e6[J], acc);
    sv[I] = acc;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float acc = sv[vgt(i, j)];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = fmaf(h[3 * i + k], sv[vgt(k, j)], acc);
      P[3 * i + j] = acc;
    }
}

// Returns false when J <= 0 (P is then zero).
__device__ __forceinline__ bool neohooke_f32(const float (&h)[9], float mu, float lam, float (&P)[9]) {
  float f[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) f[c] = (c == 0 || c == 4 || c == 8) ? 1.f + h[c] : h[c];
  const float trH = h[0] + h[4] + h[8];
  const float trH2 = h[0] * h[0] + h[4] * h[4] + h[8] * h[8] + 2.f * (h[1] * h[3] + h[2] * h[6] + h[5] * h[7]);
  const float detH = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                     h[2] * (h[3] * h[7] - h[4] * h[6]);
  const float Jm1 = trH + 0.5f * (trH * trH - trH2) + detH;
  const float J = 1.f + Jm1;
  if (!(J > 0.f)) {
#pragma unroll
    for (int c = 0; c < 9; ++c) P[c] = 0.f;
    return false;
  }
  const float iJ = 1.f / J;
  float G[9];   // F^-T = cof(F) / J
  G[0] = (f[4] * f[8] - f[5] * f[7]) * iJ;
  G[1] = (f[5] * f[6] - f[3] * f[8]) * iJ;
  G[2] = (f[3] * f[7] - f[4] * f[6]) * iJ;
  G[3] = (f[2] * f[7] - f[1] * f[8]) * iJ;
  G[4] = (f[0] * f[8] - f[2] * f[6]) * iJ;
  G[5] = (f[1] * f[6] - f[0] * f[7]) * iJ;
  G[6] = (f[1] * f[5] - f[2] * f[4]) * iJ;
  G[7] = (f[2] * f[3] - f[0] * f[5]) * iJ;
  G[8] = (f[0] * f[4] - f[1] * f[3]) * iJ;
  const float cg = lam * log1pf(Jm1) - mu;
#pragma unroll
  for (int c = 0; c < 9; ++c) P[c] = mu * f[c] + cg * G[c];
  return true;
}

template <int NC>
__device__ __forceinline__ void block_sum_dw(double (&v)[NC], double* out) {
  __shared__ double red[NC][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double s = v[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[c][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < NC) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Columns of the block partials: F 0-8, P 9-17, and with MOM T = sum P F^T
// 18-26, S = sum F F^T 27-35 (FP32 products of the high parts: only used to
// detect null rotations).  P32: P evaluated in FP32 from H and written, in
// FP32, to Pf instead of P (the averages of F stay double word).  PRED: the
// load step's predictor (pred_coef) applied to F first, the predicted F
// stored and evaluated (the pass is compute bound, so the predictor's loads
// and stores cost little here against a pass of their own).
template <int MODEL, bool WH, bool MOM, bool P32, bool PRED>
__global__ void __launch_bounds__(kThreads, 2) k_constitutive_dw(double* __restrict__ F, double* __restrict__ P,
                                                              float* __restrict__ Pf, float* __restrict__ H,
                                                              MatArgs m, const dw* __restrict__ table,
                                                              const float* __restrict__ table32, long long N,
                                                              double* __restrict__ partials, Scalars* sc,
                                                              PredArgs pa) {
  constexpr int NC = MOM ? 36 : 18;
  __shared__ double tot[NC];
  DwAcc acc[18];   // per-thread sums of F and P, normalised once at the end
  float mom[18];
#pragma unroll
  for (int c = 0; c < 18; ++c) mom[c] = 0.f;
  bool bad = false;
  __shared__ PredCoef pk_s;   // the predictor's coefficients (PRED), read from shared memory at each use
  if constexpr (PRED) {
    if (threadIdx.x == 0) pk_s = pred_coef(pa, sc);
    __syncthreads();
  }
  volatile PredCoef& pk = pk_s;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    double fd[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) fd[c] = F[c * N + v];
    if constexpr (PRED) {
      // every load of the voxel issued before any store (the slots and F
      // are distinct fields)
      double* __restrict__ A = pa.A;
      double* __restrict__ B = pa.B;
      const double v1 = pk.v1, v2 = pk.v2;
      const int dst = pk.dst;
      double fa[9], fb[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        fa[c] = v1 != 0.0 ? A[c * N + v] : 0.0;
        fb[c] = v2 != 0.0 ? B[c * N + v] : 0.0;
      }
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const double f = fd[c];
        double fn = f;
        if (v1 != 0.0) fn += v1 * (fa[c] - f);
        if (v2 != 0.0) fn += v2 * (fb[c] - f);
        if (dst == 0) A[c * N + v] = f;
        else if (dst == 1) B[c * N + v] = f;
        fd[c] = fn + pk.sh[c];
        F[c * N + v] = fd[c];
      }
    }
    const int ph = m.phase[v];
    dw h[9], f[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      f[c] = dw_split(fd[c]);
      // diagonal: hi - 1 is exact for hi in [1/2, 2] (Sterbenz)
      h[c] = (c == 0 || c == 4 || c == 8) ? dw(f[c].hi - 1.0f, 0.0f) + dw(f[c].lo, 0.0f) : f[c];
    }
    dw p[9];
    if constexpr (P32) {
      float hf[9], pf[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) hf[c] = h[c].hi;
      if constexpr (MODEL == 0) {
        if (!neohooke_f32(hf, table32[2 * ph], table32[2 * ph + 1], pf)) bad = true;
      } else {
        svk_f32(hf, table32 + 36 * ph, pf);
      }
      const float s = m.scale ? (float)m.scale[v] : 1.f;
#pragma unroll
      for (int c = 0; c < 9; ++c) p[c] = dw(s * pf[c], 0.0f);
    } else {
      if constexpr (MODEL == 0) {
        if (!neohooke_dw(h, f, table[2 * ph], table[2 * ph + 1], p)) bad = true;
      } else {
        svk_dw(h, table + 36 * ph, p);
      }
      if (m.scale) {
        const dw s = dw_split(m.scale[v]);
#pragma unroll
        for (int c = 0; c < 9; ++c) p[c] = s * p[c];
      }
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      if constexpr (P32) Pf[c * N + v] = p[c].hi;
      else P[c * N + v] = dw_join(p[c]);
      if (WH) H[c * N + v] = h[c].hi;
      acc[c].add(f[c]);
      acc[9 + c].add(p[c]);
    }
    if (MOM) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          mom[3 * i + j] += p[3 * i].hi * f[3 * j].hi + p[3 * i + 1].hi * f[3 * j + 1].hi +
                            p[3 * i + 2].hi * f[3 * j + 2].hi;
          mom[9 + 3 * i + j] += f[3 * i].hi * f[3 * j].hi + f[3 * i + 1].hi * f[3 * j + 1].hi +
                                f[3 * i + 2].hi * f[3 * j + 2].hi;
        }
    }
  }
  if (bad) atomicOr(&sc->flags, MF_FLAG_NONPOS_J);
  double a[NC];
#pragma unroll
  for (int c = 0; c < 18; ++c) a[c] = dw_join(acc[c].value());
  if constexpr (MOM) {
#pragma unroll
    for (int c = 0; c < 18; ++c) a[18 + c] = (double)mom[c];
  }
  block_sum_dw<NC>(a, tot);
  if (threadIdx.x < NC) partials[blockIdx.x * NC + threadIdx.x] = tot[threadIdx.x];
}

template <int MODEL>
cudaError_t launch_model(double* F, double* P, float* Pf, float* H, bool moments, const MatArgs& m, const dw* table,
                         const float* table32, long long N, double* partials, int nblk, Scalars* sc,
                         const PredArgs* pred, cudaStream_t st) {
  const PredArgs pa = pred ? *pred : PredArgs{nullptr, nullptr, nullptr, 0};
#define MF_CDW(WH, MOM, P32, PR)                                                                               \
  k_constitutive_dw<MODEL, WH, MOM, P32, PR><<<nblk, kThreads, 0, st>>>(F, P, Pf, H, m, table, table32, N, \
                                                                        partials, sc, pa)
  if (pred && Pf && H && moments) MF_CDW(true, true, true, true);
  else if (pred && H && moments && !Pf) MF_CDW(true, true, false, true);
  else if (pred) return cudaErrorInvalidValue;   // the predictor rides on the full passes only
  else if (Pf && H && moments) MF_CDW(true, true, true, false);
  else if (H && moments) MF_CDW(true, true, false, false);
  else if (H) MF_CDW(true, false, false, false);
  else if (moments) MF_CDW(false, true, false, false);
  else MF_CDW(false, false, false, false);
#undef MF_CDW
  return cudaGetLastError();
}

}  // namespace

cudaError_t mf_launch_constitutive_dw(const double* F, double* P, float* H, bool moments, const MatArgs& m,
                                      const void* table_dw, long long N, double* partials, int nblk,
                                      Scalars* sc, cudaStream_t st, float* Pf, const float* table32,
                                      const PredArgs* pred) {
  const dw* table = (const dw*)table_dw;
  if (Pf && !(H && moments && table32)) return cudaErrorInvalidValue;   // the FP32-P pass is the full one
  // F is written only by the predictor (pred non-null)
  double* Fw = const_cast<double*>(F);
  cudaError_t e = m.model == 0
                      ? launch_model<0>(Fw, P, Pf, H, moments, m, table, table32, N, partials, nblk, sc, pred, st)
                      : launch_model<1>(Fw, P, Pf, H, moments, m, table, table32, N, partials, nblk, sc, pred, st);
  g_mf_launches += 1;
  if (e != cudaSuccess) return e;
  return mf_launch_fin_means(partials, nblk, moments ? 36 : 18, N, sc, st);
}
