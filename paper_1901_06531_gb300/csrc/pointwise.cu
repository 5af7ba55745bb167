// Voxel-wise kernels of the Newton-CG loop: constitutive update (P and K,
// Eq. eq:lineariz), voxel averages (Sec. 2.2), the strain-control predictor
// (Sec. 2.1/2.3), the CG recurrences with FP64 dot products, and the Newton
// update with its max |dF| test (Sec. 4).  Every reduction writes one
// partial per block and is finished by a single block in a fixed order, so
// results are bitwise reproducible run to run.
#include <string.h>

#include "dw.cuh"
#include "launch.h"

namespace {

constexpr int kRedThreads = 256;

// Sum NC columns over the block; thread 0..NC-1 of warp 0 end up holding the
// totals in out[col] (a shared array).
template <int NC>
__device__ __forceinline__ void block_sum(double (&v)[NC], double* out) {
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
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) s += red[threadIdx.x][w];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Deterministic column sums of partials[nblk][ncol] by one block.
__device__ __forceinline__ double column_sum(const double* partials, int nblk, int ncol, int col,
                                             double* shm) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partials[(long long)b * ncol + col];
  shm[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) shm[threadIdx.x] += shm[threadIdx.x + w];
    __syncthreads();
  }
  const double r = shm[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double column_max(const double* partials, int nblk, int ncol, int col,
                                             double* shm) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s = fmax(s, partials[(long long)b * ncol + col]);
  shm[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) shm[threadIdx.x] = fmax(shm[threadIdx.x], shm[threadIdx.x + w]);
    __syncthreads();
  }
  const double r = shm[0];
  __syncthreads();
  return r;
}

__host__ __device__ constexpr int voigt(int i, int j) {
  return i == j ? i : (i + j == 3 ? 3 : (i + j == 2 ? 4 : 5));
}

template <typename TK>
__device__ __forceinline__ void store_K(void* K45, long long N, long long v, int t, double val) {
  reinterpret_cast<TK*>(K45)[(long long)t * N + v] = (TK)val;
}

// Neo-Hookean: W = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2,
// P = mu F + (lam ln J - mu) F^-T,
// K_ijkl = mu d_ik d_jl + lam G_ij G_kl + (mu - lam ln J) G_il G_kj, G = F^-T.
template <typename TK>
__device__ __forceinline__ bool neohooke(const double (&f)[9], double mu, double lam, double s,
                                         double (&P)[9], void* K45, long long N, long long v,
                                         bool want_K) {
  const double c00 = f[4] * f[8] - f[5] * f[7];
  const double c01 = f[5] * f[6] - f[3] * f[8];
  const double c02 = f[3] * f[7] - f[4] * f[6];
  const double J = f[0] * c00 + f[1] * c01 + f[2] * c02;
  if (!(J > 0.0)) {
#pragma unroll
    for (int c = 0; c < 9; ++c) P[c] = 0.0;
    if (want_K)
      for (int t = 0; t < 45; ++t) store_K<TK>(K45, N, v, t, 0.0);
    return false;
  }
  const double iJ = 1.0 / J;
  // G = F^-T = cofactor(F) / J
  double G[9];
  G[0] = c00 * iJ; G[1] = c01 * iJ; G[2] = c02 * iJ;
  G[3] = (f[2] * f[7] - f[1] * f[8]) * iJ;
  G[4] = (f[0] * f[8] - f[2] * f[6]) * iJ;
  G[5] = (f[1] * f[6] - f[0] * f[7]) * iJ;
  G[6] = (f[1] * f[5] - f[2] * f[4]) * iJ;
  G[7] = (f[2] * f[3] - f[0] * f[5]) * iJ;
  G[8] = (f[0] * f[4] - f[1] * f[3]) * iJ;
  const double lnJ = log(J);
  const double cg = lam * lnJ - mu;
#pragma unroll
  for (int c = 0; c < 9; ++c) P[c] = s * (mu * f[c] + cg * G[c]);
  if (want_K) {
    const double c3 = mu - lam * lnJ;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
#pragma unroll
      for (int b = a; b < 9; ++b) {
        const int i = a / 3, j = a % 3, k = b / 3, l = b % 3;
        double val = lam * G[a] * G[b] + c3 * G[3 * i + l] * G[3 * k + j];
        if (i == k && j == l) val += mu;
        store_K<TK>(K45, N, v, sym45(a, b), s * val);
      }
    }
  }
  return true;
}

// St Venant-Kirchhoff: E = (F^T F - I)/2, S = C : E, P = F S,
// K_ijkl = d_ik S_lj + F_ia F_kc C_ajcl; C given as a 6x6 Voigt matrix.
template <typename TK>
__device__ __forceinline__ void svk(const double (&f)[9], const double* __restrict__ cv, double s,
                                    double (&P)[9], void* K45, long long N, long long v,
                                    bool want_K) {
  double E[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      E[a][b] = 0.5 * (f[a] * f[b] + f[3 + a] * f[3 + b] + f[6 + a] * f[6 + b] - (a == b ? 1.0 : 0.0));
  const double e6[6] = {E[0][0], E[1][1], E[2][2], 2.0 * E[1][2], 2.0 * E[0][2], 2.0 * E[0][1]};
  double C[36];
#pragma unroll
  for (int t = 0; t < 36; ++t) C[t] = cv[t];
  double sv[6];
#pragma unroll
  for (int I = 0; I < 6; ++I) {
    double acc = 0.0;
#pragma unroll
    for (int J = 0; J < 6; ++J) acc += C[6 * I + J] * e6[J];
    sv[I] = acc;
  }
  double S[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) S[a][b] = sv[voigt(a, b)];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      P[3 * i + j] = s * (f[3 * i] * S[0][j] + f[3 * i + 1] * S[1][j] + f[3 * i + 2] * S[2][j]);
  if (!want_K) return;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const int k = b / 3, l = b % 3;
    double D[3][3];   // D_aj = sum_c C_ajcl F_kc
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) acc += C[6 * voigt(a, j) + voigt(c, l)] * f[3 * k + c];
        D[a][j] = acc;
      }
#pragma unroll
    for (int a2 = 0; a2 <= b; ++a2) {
      const int i = a2 / 3, j = a2 % 3;
      double val = f[3 * i] * D[0][j] + f[3 * i + 1] * D[1][j] + f[3 * i + 2] * D[2][j];
      if (i == k) val += S[l][j];
      store_K<TK>(K45, N, v, sym45(a2, b), s * val);
    }
  }
}

// P (and with WK the packed K) per voxel, and block partial sums of F and P;
// with MOM also the rotation moments T = sum P F^T and S = sum F F^T (FP32
// products, used only to detect null rotations).  Columns: F 0-8, P 9-17,
// T 18-26, S 27-35.
template <typename TK, bool WK, bool MOM>
__global__ void __launch_bounds__(kRedThreads) k_constitutive(const double* __restrict__ F,
                                                              double* __restrict__ P, void* K45,
                                                              MatArgs m, long long N,
                                                              double* __restrict__ partials,
                                                              Scalars* sc) {
  constexpr int NC = MOM ? 36 : 18;
  __shared__ double tot[NC];
  double acc[NC];
#pragma unroll
  for (int c = 0; c < 18; ++c) acc[c] = 0.0;
  float mom[18];
#pragma unroll
  for (int c = 0; c < 18; ++c) mom[c] = 0.f;
  bool bad = false;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    double f[9], p[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) f[c] = F[c * N + v];
    const int ph = m.phase[v];
    const double s = m.scale ? m.scale[v] : 1.0;
    if (m.model == 0) {
      if (!neohooke<TK>(f, m.table[2 * ph], m.table[2 * ph + 1], s, p, K45, N, v, WK)) bad = true;
    } else {
      svk<TK>(f, m.table + 36 * ph, s, p, K45, N, v, WK);
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      P[c * N + v] = p[c];
      acc[c] += f[c];
      acc[9 + c] += p[c];
    }
    if (MOM) {
      float ff[9], pf[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) { ff[c] = (float)f[c]; pf[c] = (float)p[c]; }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          mom[3 * i + j] += pf[3 * i] * ff[3 * j] + pf[3 * i + 1] * ff[3 * j + 1] + pf[3 * i + 2] * ff[3 * j + 2];
          mom[9 + 3 * i + j] += ff[3 * i] * ff[3 * j] + ff[3 * i + 1] * ff[3 * j + 1] + ff[3 * i + 2] * ff[3 * j + 2];
        }
    }
  }
  if (bad) atomicOr(&sc->flags, MF_FLAG_NONPOS_J);
  if constexpr (MOM) {
#pragma unroll
    for (int c = 0; c < 18; ++c) acc[18 + c] = (double)mom[c];
  }
  block_sum<NC>(acc, tot);
  if (threadIdx.x < NC) partials[blockIdx.x * NC + threadIdx.x] = tot[threadIdx.x];
}

// One block per column (grid ncol): the column sums of the block partials in
// a fixed order.
__global__ void __launch_bounds__(kRedThreads) k_fin_means(const double* __restrict__ partials, int nblk,
                                                           int ncol, long long N, Scalars* sc) {
  __shared__ double shm[kRedThreads];
  const int col = blockIdx.x;
  const double s = column_sum(partials, nblk, ncol, col, shm);
  if (threadIdx.x == 0) {
    if (col < 9) sc->meanF[col] = s / (double)N;
    else if (col < 18) sc->meanP[col - 9] = s / (double)N;
    else if (col < 27) sc->T[col - 18] = s;
    else sc->S[col - 27] = s;
  }
}

__global__ void __launch_bounds__(kRedThreads) k_mean_F(const double* __restrict__ F, long long N,
                                                        double* __restrict__ partials) {
  __shared__ double tot[9];
  double acc[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) acc[c] = 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] += F[c * N + v];
  }
  block_sum<9>(acc, tot);
  if (threadIdx.x < 9) partials[blockIdx.x * 9 + threadIdx.x] = tot[threadIdx.x];
}

struct Load9 {
  double target[9];
  unsigned char mask[9];
};

// Predictor of a load step: every strain-controlled component is shifted
// uniformly so that its voxel average equals the prescribed F-bar.  With
// after_update the averages measured by the last Newton update are used (the
// FP32 inner solves re-impose the strain control in FP64 after each update).
__global__ void k_predictor(double* __restrict__ F, long long N, Load9 ld, const Scalars* sc,
                            bool after_update) {
  const double* mean = after_update ? sc->meanF_new : sc->meanF;
  for (int c = 0; c < 9; ++c) {
    if (ld.mask[c]) continue;
    const double d = ld.target[c] - mean[c];
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x)
      F[c * N + v] += d;
  }
}

// r = b rounded to the inner type and the block partials of r.r (x and the
// previous direction are not touched: the first tangent pass, its = 0, takes
// p = r and writes x = 0 without reading either).  FP32: b is rounded
// through its double-word split (no FP64 instruction, the FP64 pipe being
// slow on this part) and r.r is summed from exact FP32 products with
// Neumaier compensation, thread totals in FP64.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_cg_init(const double* __restrict__ b, T* __restrict__ r,
                                                         long long n9, double* __restrict__ partials) {
  __shared__ double tot[1];
  double acc[1] = {0.0};
  float fs = 0.f, fc = 0.f;
  auto fadd = [&](float v) {
    const float t = fs + v;
    fc += (fabsf(fs) >= fabsf(v)) ? ((fs - t) + v) : ((v - t) + fs);
    fs = t;
  };
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n9;
       i += (long long)gridDim.x * blockDim.x) {
    if constexpr (sizeof(T) == 4) {
      const dw d = dw_split(b[i]);
      const float v = __fadd_rn(d.hi, d.lo);
      r[i] = v;
      const float pr = v * v;
      fadd(pr);
      fadd(fmaf(v, v, -pr));
    } else {
      const T v = (T)b[i];
      r[i] = v;
      acc[0] += (double)v * (double)v;
    }
  }
  if constexpr (sizeof(T) == 4) acc[0] = (double)fs + (double)fc;
  block_sum<1>(acc, tot);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot[0];
}

__global__ void __launch_bounds__(kRedThreads) k_fin_cg_init(const double* __restrict__ partials, int npart,
                                                             double tol_cg, double cg_rel, long long N,
                                                             Scalars* sc) {
  __shared__ double shm[kRedThreads];
  const double rr = column_sum(partials, npart, 1, 0, shm);
  if (threadIdx.x == 0) {
    sc->rr = rr;
    sc->rr0 = rr;
    sc->alpha = 0.0;
    sc->beta = 0.0;
    double thr = tol_cg;
    if (cg_rel > 0.0) thr = fmax(tol_cg, cg_rel * sqrt(rr / (double)N));
    sc->thr2N = thr * thr * (double)N;
    sc->done = (rr <= sc->thr2N) ? 1 : 0;
  }
}

// F += x, or with DEFL F += x - What F (What from the projection of x).
// Partials: columns 0-8 the sums of the correction (the new averages are the
// old ones plus its mean), column 9 the block max of abs(dF_v)^2.
template <typename T, bool DEFL>
__global__ void __launch_bounds__(kRedThreads) k_newton_update(double* __restrict__ F,
                                                               const T* __restrict__ x, long long N,
                                                               double* __restrict__ partials,
                                                               const Scalars* sc) {
  __shared__ double tot[10];
  double acc[10];
#pragma unroll
  for (int c = 0; c < 10; ++c) acc[c] = 0.0;
  float xs[9], xc[9];          // compensated FP32 sums of an FP32 correction
#pragma unroll
  for (int c = 0; c < 9; ++c) { xs[c] = 0.f; xc[c] = 0.f; }
  double mx = 0.0;
  double W[9];
  if (DEFL) {
#pragma unroll
    for (int t = 0; t < 9; ++t) W[t] = sc->What[t];
  }
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    double f[9];
    T xv[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) { f[c] = F[c * N + v]; xv[c] = x[c * N + v]; }
    if (DEFL || sizeof(T) == 8) {
      double d[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) d[c] = (double)xv[c];
      if (DEFL) {
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
    } else {
      float n2 = 0.f;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const float d = (float)xv[c];
        F[c * N + v] = f[c] + f32_as_f64(d);
        const float tt = xs[c] + d;
        xc[c] += (fabsf(xs[c]) >= fabsf(d)) ? ((xs[c] - tt) + d) : ((d - tt) + xs[c]);
        xs[c] = tt;
        n2 = fmaf(d, d, n2);
      }
      mx = fmax(mx, (double)n2);
    }
  }
  if (!(DEFL || sizeof(T) == 8)) {
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] = (double)xs[c] + (double)xc[c];
  }
  block_sum<10>(acc, tot);   // column 9 unused by the sum
  // block max of |dF_v|^2
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
    partials[blockIdx.x * 10 + 9] = mm;
  }
  if (threadIdx.x < 9) partials[blockIdx.x * 10 + threadIdx.x] = tot[threadIdx.x];
}

// B = sum_v y_v F_v^T, the moments that give n_k . y = W_k : B.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_defl_reduce(const T* __restrict__ y,
                                                             const double* __restrict__ F, long long N,
                                                             double* __restrict__ partials) {
  __shared__ double tot[9];
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
  block_sum<9>(acc, tot);
  if (threadIdx.x < 9) partials[blockIdx.x * 9 + threadIdx.x] = tot[threadIdx.x];
}

__global__ void __launch_bounds__(kRedThreads) k_defl_fin(const double* __restrict__ partials, int nblk,
                                                          Defl d, Scalars* sc) {
  __shared__ double shm[kRedThreads];
  __shared__ double B[9];
  for (int col = 0; col < 9; ++col) {
    const double s = column_sum(partials, nblk, 9, col, shm);
    if (threadIdx.x == 0) B[col] = s;
  }
  __syncthreads();
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
__global__ void k_defl_apply(T* __restrict__ y, const double* __restrict__ F, long long N,
                             const Scalars* sc) {
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

// One block per column (grid 10): columns 0-8 the new averages, column 9
// the max of abs(dF_v)^2.
__global__ void __launch_bounds__(kRedThreads) k_fin_newton(const double* __restrict__ partials, int nblk,
                                                            long long N, Scalars* sc) {
  __shared__ double shm[kRedThreads];
  const int col = blockIdx.x;
  if (col < 9) {
    const double s = column_sum(partials, nblk, 10, col, shm);
    if (threadIdx.x == 0) sc->meanF_new[col] = sc->meanF[col] + s / (double)N;
  } else {
    const double m = column_max(partials, nblk, 10, 9, shm);
    if (threadIdx.x == 0) {
      sc->dF2max = m;
      if (!isfinite(m)) atomicOr(&sc->flags, MF_FLAG_NONFINITE);
    }
  }
}

int grid_for(long long n) {
  long long g = (n + kRedThreads - 1) / kRedThreads;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t mf_launch_fin_means(const double* partials, int nblk, int ncol, long long N, Scalars* sc,
                                cudaStream_t st) {
  k_fin_means<<<ncol, kRedThreads, 0, st>>>(partials, nblk, ncol, N, sc);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_constitutive(const double* F, double* P, void* K45, bool k_f32, bool want_K,
                                   bool moments, const MatArgs& m, long long N, double* partials,
                                   int nblk, Scalars* sc, cudaStream_t st) {
  if (want_K) {
    if (k_f32) k_constitutive<float, true, false><<<nblk, kRedThreads, 0, st>>>(F, P, K45, m, N, partials, sc);
    else k_constitutive<double, true, false><<<nblk, kRedThreads, 0, st>>>(F, P, K45, m, N, partials, sc);
  } else if (moments) {
    k_constitutive<double, false, true><<<nblk, kRedThreads, 0, st>>>(F, P, K45, m, N, partials, sc);
  } else {
    k_constitutive<double, false, false><<<nblk, kRedThreads, 0, st>>>(F, P, K45, m, N, partials, sc);
  }
  {
    const int ncol = (moments && !want_K) ? 36 : 18;
    k_fin_means<<<ncol, kRedThreads, 0, st>>>(partials, nblk, ncol, N, sc);
  }
  g_mf_launches += 2;
  return cudaGetLastError();
}

cudaError_t mf_launch_mean_F(const double* F, long long N, double* partials, int nblk, Scalars* sc,
                             cudaStream_t st) {
  k_mean_F<<<nblk, kRedThreads, 0, st>>>(F, N, partials);
  // columns 0..8 of a 9-column table
  k_fin_means<<<9, kRedThreads, 0, st>>>(partials, nblk, 9, N, sc);
  g_mf_launches += 2;
  return cudaGetLastError();
}

cudaError_t mf_launch_predictor(double* F, long long N, const uint8_t* mask9, const double* target9,
                                const Scalars* sc, bool after_update, cudaStream_t st) {
  Load9 ld;
  for (int c = 0; c < 9; ++c) { ld.mask[c] = mask9[c]; ld.target[c] = target9[c]; }
  k_predictor<<<grid_for(9 * N) > 4096 ? 4096 : grid_for(9 * N), kRedThreads, 0, st>>>(F, N, ld, sc, after_update);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_cg_init(const double* b, void* x, void* r, void* p, bool f32, long long n9,
                              double* partials, int nblk, double tol_cg, double cg_rel, long long N,
                              Scalars* sc, cudaStream_t st) {
  (void)x;
  (void)p;
  if (f32) k_cg_init<float><<<nblk, kRedThreads, 0, st>>>(b, (float*)r, n9, partials);
  else k_cg_init<double><<<nblk, kRedThreads, 0, st>>>(b, (double*)r, n9, partials);
  k_fin_cg_init<<<1, kRedThreads, 0, st>>>(partials, nblk, tol_cg, cg_rel, N, sc);
  g_mf_launches += 2;
  return cudaGetLastError();
}

cudaError_t mf_launch_newton_update(double* F, const void* x, bool f32, bool defl, long long N,
                                    double* partials, int nblk, Scalars* sc, cudaStream_t st) {
  const float* xf = (const float*)x;
  const double* xd = (const double*)x;
  if (f32 && defl) k_newton_update<float, true><<<nblk, kRedThreads, 0, st>>>(F, xf, N, partials, sc);
  else if (f32) k_newton_update<float, false><<<nblk, kRedThreads, 0, st>>>(F, xf, N, partials, sc);
  else if (defl) k_newton_update<double, true><<<nblk, kRedThreads, 0, st>>>(F, xd, N, partials, sc);
  else k_newton_update<double, false><<<nblk, kRedThreads, 0, st>>>(F, xd, N, partials, sc);
  k_fin_newton<<<10, kRedThreads, 0, st>>>(partials, nblk, N, sc);
  g_mf_launches += 2;
  return cudaGetLastError();
}

cudaError_t mf_launch_defl_project(void* y, bool f32, bool apply, const double* F, long long N,
                                   const Defl& d, double* partials, int nblk, Scalars* sc,
                                   cudaStream_t st) {
  if (f32) k_defl_reduce<float><<<nblk, kRedThreads, 0, st>>>((const float*)y, F, N, partials);
  else k_defl_reduce<double><<<nblk, kRedThreads, 0, st>>>((const double*)y, F, N, partials);
  k_defl_fin<<<1, kRedThreads, 0, st>>>(partials, nblk, d, sc);
  g_mf_launches += 2;
  if (apply) {
    const int g = grid_for(N) > 4096 ? 4096 : grid_for(N);
    if (f32) k_defl_apply<float><<<g, kRedThreads, 0, st>>>((float*)y, F, N, sc);
    else k_defl_apply<double><<<g, kRedThreads, 0, st>>>((double*)y, F, N, sc);
    g_mf_launches += 1;
  }
  return cudaGetLastError();
}
