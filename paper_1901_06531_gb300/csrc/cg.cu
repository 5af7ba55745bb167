// Conjugate-gradient iteration on the projected tangent operator of
// Eq. (linequil2ast), restructured so that every vector update rides on a
// pass that streams the same data anyway:
//
//   tangent pass : p = r + beta p', x += alpha' p' (alpha', p' of the previous
//                  iteration), t = K : p, partial sums of p . t
//   transforms   : y = G*(t) (x-y forward, z-pass with G-hat-star, x-y inverse)
//   inverse pass : r -= alpha y, partial sums of r . r
//
// p . A p = p . G*(K:p) = p . (K:p) because every CG direction lies in the
// range of the orthogonal projection G* (b does, and A maps into it), so the
// curvature is available before the transforms run.
//
// The tangent K = dP/dF (Eq. eq:lineariz) is either read packed (45 entries
// per voxel) or, in FP32, applied without being stored, from H = F - I and
// the phase's parameters:
//   neo-Hookean   K:q = mu q + lam (G:q) G + (mu - lam ln J) G q^T G, G = F^-T
//   St V.-K.      K:q = q S + F (C : sym(F^T q)),  S = C : E,  E = (H + H^T + H^T H)/2
#include <type_traits>

#include "launch.h"

namespace {

constexpr int kThreads = 256;

template <int NC>
__device__ __forceinline__ void block_sum_cg(double (&v)[NC], double* out) {
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

// Per-thread dot-product accumulator: exact FP32 products (two-product by FMA)
// summed with Neumaier compensation in FP32; the thread totals are then
// combined in FP64.  FP64 arithmetic per element would cost as much as the
// whole pass on a part whose FP64 rate is 1/57 of its FP32 rate.
struct Dot32 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_term(float v) {
    const float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    add_term(p);
    add_term(fmaf(a, b, -p));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ constexpr int vgt(int i, int j) {
  return i == j ? i : (i + j == 3 ? 3 : (i + j == 2 ? 4 : 5));
}

// t = K : q for St Venant-Kirchhoff from H = F - I and a 6x6 Voigt stiffness.
__device__ __forceinline__ void svk_apply(const float (&h)[9], const float* __restrict__ C,
                                          const float (&q)[9], float (&t)[9]) {
  float e6[6], d6[6];
  // E = (H + H^T + H^T H)/2 in Voigt form with engineering shears
  float E[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      E[a][b] = 0.5f * (h[3 * a + b] + h[3 * b + a] + h[a] * h[b] + h[3 + a] * h[3 + b] + h[6 + a] * h[6 + b]);
  e6[0] = E[0][0]; e6[1] = E[1][1]; e6[2] = E[2][2];
  e6[3] = 2.f * E[1][2]; e6[4] = 2.f * E[0][2]; e6[5] = 2.f * E[0][1];
  // dE = sym(F^T q), F = I + H
  float D[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      D[a][b] = q[3 * a + b] + h[a] * q[b] + h[3 + a] * q[3 + b] + h[6 + a] * q[6 + b];  // (F^T q)_ab
  d6[0] = D[0][0]; d6[1] = D[1][1]; d6[2] = D[2][2];
  d6[3] = D[1][2] + D[2][1]; d6[4] = D[0][2] + D[2][0]; d6[5] = D[0][1] + D[1][0];
  float sv[6], dv[6];
#pragma unroll
  for (int I = 0; I < 6; ++I) {
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int J = 0; J < 6; ++J) { a += C[6 * I + J] * e6[J]; b += C[6 * I + J] * d6[J]; }
    sv[I] = a; dv[I] = b;
  }
  // t = q S + F dS
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float acc = dv[vgt(i, j)];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc += q[3 * i + k] * sv[vgt(k, j)] + h[3 * i + k] * dv[vgt(k, j)];
      t[3 * i + j] = acc;
    }
}

// t = K : q for the neo-Hookean law from H = F - I.
__device__ __forceinline__ void neohooke_apply(const float (&h)[9], float mu, float lam,
                                               const float (&q)[9], float (&t)[9]) {
  const float f0 = 1.f + h[0], f4 = 1.f + h[4], f8 = 1.f + h[8];
  const float c00 = f4 * f8 - h[5] * h[7];
  const float c01 = h[5] * h[6] - h[3] * f8;
  const float c02 = h[3] * h[7] - f4 * h[6];
  // J - 1 without cancellation: tr H + (tr^2 H - tr H^2)/2 + det H
  const float trH = h[0] + h[4] + h[8];
  const float tr2 = h[0] * h[0] + h[4] * h[4] + h[8] * h[8] +
                    2.f * (h[1] * h[3] + h[2] * h[6] + h[5] * h[7]);
  const float detH = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                     h[2] * (h[3] * h[7] - h[4] * h[6]);
  const float Jm1 = trH + 0.5f * (trH * trH - tr2) + detH;
  const float J = 1.f + Jm1;
  const float iJ = 1.f / J;
  float G[9];
  G[0] = c00 * iJ; G[1] = c01 * iJ; G[2] = c02 * iJ;
  G[3] = (h[2] * h[7] - h[1] * f8) * iJ;
  G[4] = (f0 * f8 - h[2] * h[6]) * iJ;
  G[5] = (h[1] * h[6] - f0 * h[7]) * iJ;
  G[6] = (h[1] * h[5] - h[2] * f4) * iJ;
  G[7] = (h[2] * h[3] - f0 * h[5]) * iJ;
  G[8] = (f0 * f4 - h[1] * h[3]) * iJ;
  const float lnJ = log1pf(Jm1);
  const float c3 = mu - lam * lnJ;
  float gq = 0.f;
#pragma unroll
  for (int c = 0; c < 9; ++c) gq += G[c] * q[c];
  // (G q^T G)_ij = sum_kl G_il q_kl G_kj
  float M[3][3];   // M_lj = sum_k q_kl G_kj = (q^T G)_lj
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[l][j] = q[l] * G[j] + q[3 + l] * G[3 + j] + q[6 + l] * G[6 + j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float gqg = G[3 * i] * M[0][j] + G[3 * i + 1] * M[1][j] + G[3 * i + 2] * M[2][j];
      t[3 * i + j] = mu * q[3 * i + j] + lam * gq * G[3 * i + j] + c3 * gqg;
    }
}

// TAN 0: packed tangent K45 of type T; 1: neo-Hookean from H; 2: SVK from H.
// CG true: p = r + beta p', x += alpha' p' first (p' = pin); false: p = pin.
// FIN (with CG): the last block to finish sums the partials of p.t and sets
// alpha (no separate finishing launch).
template <typename T, int TAN, bool CG, bool FIN>
__global__ void __launch_bounds__(kThreads) k_tangent(const T* __restrict__ pin, const T* __restrict__ r,
                                                      T* __restrict__ pout, T* __restrict__ x,
                                                      TangentArgs ta, T* __restrict__ t, long long N,
                                                      double* __restrict__ partials, Scalars* sc) {
  static_assert(!FIN || CG, "the fused finish belongs to the CG pass");
  __shared__ double tot[1];
  T beta = (T)0, alpha = (T)0;
  pdl_wait();
  bool first = false;   // first CG iteration: p = r, x = 0 (neither previous vector is read)
  if (CG) {
    if (*(volatile const int*)&sc->stop) return;
    beta = (T)sc->beta;
    alpha = (T)sc->alpha;
    first = sc->its == 0;
  }
  double acc64 = 0.0;
  Dot32 acc32;
  // one voxel; FIRST: p = r, x = 0 without loading the previous vectors
  // (the loop is instantiated once per case, so that in each every load of
  // the voxel is issued before any arithmetic)
  auto voxel = [&](long long v, auto first_tag) {
    constexpr bool FIRST = decltype(first_tag)::value;
    v = MF_AT(v, N);   // every access below is c * N + v (c < 9) or t * N + v (t < 45)
    T po[9], rv[9], xv[9];
    float h[9];
    int ph = 0;
    if constexpr (FIRST) {
#pragma unroll
      for (int c = 0; c < 9; ++c) { rv[c] = r[c * N + v]; po[c] = (T)0; xv[c] = (T)0; }
    } else {
#pragma unroll
      for (int c = 0; c < 9; ++c) po[c] = pin[c * N + v];
      if (CG) {
#pragma unroll
        for (int c = 0; c < 9; ++c) { rv[c] = r[c * N + v]; xv[c] = x[c * N + v]; }
      }
    }
    if (TAN != 0) {
#pragma unroll
      for (int c = 0; c < 9; ++c) h[c] = ta.H[c * N + v];
      ph = ta.phase[v];
    }
    T q[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      if (CG) {
        q[c] = rv[c] + beta * po[c];
        x[c * N + v] = xv[c] + alpha * po[c];
        pout[c * N + v] = q[c];
      } else {
        q[c] = po[c];
      }
    }
    T o[9];
    if (TAN == 0) {
      const T* K = reinterpret_cast<const T*>(ta.K45);
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        T s = (T)0;
#pragma unroll
        for (int b = 0; b < 9; ++b) s += K[(long long)sym45(a, b) * N + v] * q[b];
        o[a] = s;
      }
    } else {
      float qf[9], tf[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) qf[c] = (float)q[c];
      if (TAN == 1) neohooke_apply(h, ta.table[2 * ph], ta.table[2 * ph + 1], qf, tf);
      else svk_apply(h, ta.table + 36 * ph, qf, tf);
      const float s = ta.scale ? ta.scale[v] : 1.f;
#pragma unroll
      for (int c = 0; c < 9; ++c) o[c] = (T)(s * tf[c]);
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      t[c * N + v] = o[c];
      if (sizeof(T) == 4) acc32.add_prod((float)q[c], (float)o[c]);
      else acc64 += (double)q[c] * (double)o[c];
    }
  };
  const long long v0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long dv = (long long)gridDim.x * blockDim.x;
  if (CG && first) {
    for (long long v = v0; v < N; v += dv) voxel(v, std::true_type{});
  } else {
    for (long long v = v0; v < N; v += dv) voxel(v, std::false_type{});
  }
  if (partials) {
    double acc[1] = {sizeof(T) == 4 ? acc32.value() : acc64};
    block_sum_cg<1>(acc, tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot[0];
    if constexpr (FIN) {
      double pAp;
      if (last_block_total(partials, &sc->arrive, &pAp) && threadIdx.x == 0) cg_finish_alpha(pAp, sc);
    }
  }
}

__device__ __forceinline__ double col_sum(const double* partials, int n, double* shm) {
  double s = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) s += partials[b];
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

__global__ void __launch_bounds__(kThreads) k_fin_beta(const double* __restrict__ partials, int n,
                                                       Scalars* sc) {
  __shared__ double shm[kThreads];
  if (*(volatile const int*)&sc->stop) return;
  const double rr = col_sum(partials, n, shm);
  if (threadIdx.x == 0) cg_finish_beta(rr, sc);
}

template <typename T>
__global__ void k_axpy_alpha(T* __restrict__ x, const T* __restrict__ p, long long n, const Scalars* sc) {
  const T a = (T)sc->alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] += a * p[i];
}

// End of a CG body in a graph: keep looping while the solve has not stopped.
__global__ void k_cg_cond(const Scalars* sc, cudaGraphConditionalHandle h) {
  pdl_wait();
  cudaGraphSetConditional(h, *(volatile const int*)&sc->stop ? 0u : 1u);
}

// Final lagging update x += alpha p, with p the direction of the last
// completed iteration (iteration j writes pbuf[(j+1) % 2]).
template <typename T>
__global__ void k_axpy_last(T* __restrict__ x, const T* __restrict__ p0, const T* __restrict__ p1, long long n,
                            const Scalars* sc) {
  const int its = sc->its;
  if (its == 0) {   // no iteration ran (converged at the start, or stopped in the first): x = 0
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
      x[i] = (T)0;
    return;
  }
  const T* p = (its & 1) ? p1 : p0;
  const T a = (T)sc->alpha;
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, di = (long long)gridDim.x * blockDim.x;
  long long head = 0;
  if constexpr (sizeof(T) == 4) {
    // 16-byte accesses where both vectors allow them (the same arithmetic)
    if ((((uintptr_t)x | (uintptr_t)p) & 15) == 0) {
      head = n & ~3LL;
      float4* x4 = reinterpret_cast<float4*>(x);
      const float4* p4 = reinterpret_cast<const float4*>(p);
      for (long long i = i0; i < head / 4; i += di) {
        float4 xv = x4[i];
        const float4 pv = p4[i];
        xv.x += a * pv.x;
        xv.y += a * pv.y;
        xv.z += a * pv.z;
        xv.w += a * pv.w;
        x4[i] = xv;
      }
    }
  }
  for (long long i = head + i0; i < n; i += di) x[i] += a * p[i];
}

// H = F - I in FP32 (the state the matrix-free tangent needs).
__global__ void k_make_H(const double* __restrict__ F, float* __restrict__ H, long long N) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const double d = (c == 0 || c == 4 || c == 8) ? 1.0 : 0.0;
      H[c * N + v] = (float)(F[c * N + v] - d);
    }
  }
}

}  // namespace

cudaError_t mf_launch_tangent(const void* pin, const void* r, void* pout, void* x, bool f32, int tan,
                              bool cg, const TangentArgs& ta, void* t, long long N, double* partials,
                              int nblk, Scalars* sc, cudaStream_t st, bool fin_alpha, bool pdl) {
  cudaError_t e = cudaSuccess;
#define MF_TAN(T, K, CGV, FV)                                                                                 \
  e = launch_k(pdl, k_tangent<T, K, CGV, FV>, dim3(nblk), dim3(kThreads), 0, st, (const T*)pin, (const T*)r, \
               (T*)pout, (T*)x, ta, (T*)t, N, partials, sc)
#define MF_TAN_CG(T, K)                                       \
  do {                                                        \
    if (!cg) MF_TAN(T, K, false, false);                      \
    else if (fin_alpha && partials) MF_TAN(T, K, true, true); \
    else MF_TAN(T, K, true, false);                           \
  } while (0)
  if (f32) {
    if (tan == 0) MF_TAN_CG(float, 0);
    else if (tan == 1) MF_TAN_CG(float, 1);
    else MF_TAN_CG(float, 2);
  } else {
    MF_TAN_CG(double, 0);
  }
#undef MF_TAN_CG
#undef MF_TAN
  g_mf_launches += 1;
  return e;
}

__global__ void k_cg_batch_init(Scalars* sc, int max_its) {
  sc->its = 0;
  sc->arrive = 0u;
  sc->max_its = max_its;
  sc->stop = (sc->done || sc->flags) ? 1 : 0;
}

cudaError_t mf_launch_cg_batch_init(Scalars* sc, int max_its, cudaStream_t st) {
  k_cg_batch_init<<<1, 1, 0, st>>>(sc, max_its);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_fin_beta(const double* partials, int n, Scalars* sc, cudaStream_t st) {
  k_fin_beta<<<1, kThreads, 0, st>>>(partials, n, sc);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_axpy_alpha(void* x, const void* p, bool f32, long long n, const Scalars* sc,
                                 cudaStream_t st) {
  const int g = stride_grid(n, kThreads);
  if (f32) k_axpy_alpha<float><<<g, kThreads, 0, st>>>((float*)x, (const float*)p, n, sc);
  else k_axpy_alpha<double><<<g, kThreads, 0, st>>>((double*)x, (const double*)p, n, sc);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_make_H(const double* F, float* H, long long N, cudaStream_t st) {
  k_make_H<<<stride_grid(N, kThreads), kThreads, 0, st>>>(F, H, N);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_cg_cond(const Scalars* sc, cudaGraphConditionalHandle h, cudaStream_t st, bool pdl) {
  g_mf_launches += 1;
  return launch_k(pdl, k_cg_cond, dim3(1), dim3(1), 0, st, sc, h);
}

cudaError_t mf_launch_axpy_last(void* x, const void* p0, const void* p1, bool f32, long long n,
                                const Scalars* sc, cudaStream_t st) {
  const int g = stride_grid(n, kThreads);
  if (f32) k_axpy_last<float><<<g, kThreads, 0, st>>>((float*)x, (const float*)p0, (const float*)p1, n, sc);
  else k_axpy_last<double><<<g, kThreads, 0, st>>>((double*)x, (const double*)p0, (const double*)p1, n, sc);
  g_mf_launches += 1;
  return cudaGetLastError();
}
