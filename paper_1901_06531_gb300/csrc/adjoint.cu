// Adjoint sensitivity of the homogenized response at a converged load step.
//
// At convergence G*(P(F, theta) - P-bar) = 0 (Eq. linequil2ast at dF = 0).
// For J = wF . <F> + wP . <P> the derivative with respect to any material
// parameter theta is
//     dJ/dtheta = (1/N) sum_v (W_P - lambda_v) : dP_v/dtheta,
//     A lambda = G*(W_F + K : W_P),   A = G* K G*,
// with W_F, W_P the uniform fields of the weights: one CG solve with the
// same symmetric projected tangent as the Newton iterations.  For the
// neo-Hookean law dP/dmu = s (F - F^-T), dP/dlam = s ln J F^-T (on the voxels
// of the phase) and dP_v/ds_v = P_v / s_v.
#include "launch.h"

namespace {

constexpr int kThreads = 256;

template <typename T>
__global__ void k_fill_uniform(T* __restrict__ q, long long N, AdjWeights w) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 9; ++c) q[c * N + v] = (T)w.wP[c];
  }
}

// t += W_F (in place, the inner type)
template <typename T>
__global__ void k_add_uniform(T* __restrict__ t, long long N, AdjWeights w) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 9; ++c) t[c * N + v] += (T)w.wF[c];
  }
}

template <typename T>
__global__ void k_to_double(const T* __restrict__ y, double* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)y[i];
}

// Per-voxel contraction (W_P - lambda) : dP/dtheta; block partials of the
// per-phase sums (columns 2p: mu_p, 2p+1: lam_p) and the per-voxel scale
// derivative.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_adj_grad(const double* __restrict__ F, const double* __restrict__ P,
                                                       const T* __restrict__ lam, const int32_t* __restrict__ phase,
                                                       const double* __restrict__ scale, long long N, int nphase,
                                                       AdjWeights w, double* __restrict__ partials,
                                                       double* __restrict__ dscale) {
  extern __shared__ double sacc[];   // [2 * nphase]
  for (int i = threadIdx.x; i < 2 * nphase; i += blockDim.x) sacc[i] = 0.0;
  __syncthreads();
  const double invN = 1.0 / (double)N;
  // every lane of a warp runs the same number of iterations (blockDim is a
  // multiple of 32), so the warp-wide shuffles below see all 32 lanes
  for (long long base = blockIdx.x * (long long)blockDim.x; base < N; base += (long long)gridDim.x * blockDim.x) {
    const long long v = base + threadIdx.x;
    const bool valid = v < N;
    double a = 0.0, b = 0.0;
    int ph = -1;
    if (valid) {
      double f[9], d[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        f[c] = F[c * N + v];
        d[c] = w.wP[c] - (double)lam[c * N + v];
      }
      const double c00 = f[4] * f[8] - f[5] * f[7];
      const double c01 = f[5] * f[6] - f[3] * f[8];
      const double c02 = f[3] * f[7] - f[4] * f[6];
      const double J = f[0] * c00 + f[1] * c01 + f[2] * c02;
      const double iJ = 1.0 / J;
      double G[9];   // F^-T
      G[0] = c00 * iJ; G[1] = c01 * iJ; G[2] = c02 * iJ;
      G[3] = (f[2] * f[7] - f[1] * f[8]) * iJ;
      G[4] = (f[0] * f[8] - f[2] * f[6]) * iJ;
      G[5] = (f[1] * f[6] - f[0] * f[7]) * iJ;
      G[6] = (f[1] * f[5] - f[2] * f[4]) * iJ;
      G[7] = (f[2] * f[3] - f[0] * f[5]) * iJ;
      G[8] = (f[0] * f[4] - f[1] * f[3]) * iJ;
      const double lnJ = log(J);
      const double s = scale ? scale[v] : 1.0;
      double dmu = 0.0, dlam = 0.0, dP = 0.0;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        dmu += d[c] * (f[c] - G[c]);
        dlam += d[c] * G[c];
        dP += d[c] * P[c * N + v];
      }
      ph = phase[v];
      a = s * dmu * invN;
      b = s * lnJ * dlam * invN;
      if (dscale) dscale[v] = dP / s * invN;
    }
    // lanes of one phase (the common case inside a grain) reduce by shuffles
    // and add once; mixed warps add per lane
    const int ph0 = __shfl_sync(0xffffffffu, ph, 0);
    if (__all_sync(0xffffffffu, ph == ph0 || ph < 0)) {
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      if ((threadIdx.x & 31) == 0 && ph0 >= 0) {
        atomicAdd(&sacc[2 * ph0], a);
        atomicAdd(&sacc[2 * ph0 + 1], b);
      }
    } else if (ph >= 0) {
      atomicAdd(&sacc[2 * ph], a);
      atomicAdd(&sacc[2 * ph + 1], b);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * nphase; i += blockDim.x) partials[(long long)blockIdx.x * 2 * nphase + i] = sacc[i];
}

__global__ void __launch_bounds__(kThreads) k_adj_fin(const double* __restrict__ partials, int nblk, int ncol,
                                                      double* __restrict__ out) {
  __shared__ double shm[kThreads];
  for (int col = 0; col < ncol; ++col) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partials[(long long)b * ncol + col];
    shm[threadIdx.x] = s;
    __syncthreads();
    for (int wdt = blockDim.x / 2; wdt > 0; wdt >>= 1) {
      if (threadIdx.x < wdt) shm[threadIdx.x] += shm[threadIdx.x + wdt];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[col] = shm[0];
    __syncthreads();
  }
}

}  // namespace

cudaError_t mf_launch_adj_rhs_fill(void* q, bool f32, long long N, const AdjWeights& w, cudaStream_t st) {
  if (f32) k_fill_uniform<float><<<stride_grid(N), kThreads, 0, st>>>((float*)q, N, w);
  else k_fill_uniform<double><<<stride_grid(N), kThreads, 0, st>>>((double*)q, N, w);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_adj_rhs_add(void* t, bool f32, long long N, const AdjWeights& w, cudaStream_t st) {
  if (f32) k_add_uniform<float><<<stride_grid(N), kThreads, 0, st>>>((float*)t, N, w);
  else k_add_uniform<double><<<stride_grid(N), kThreads, 0, st>>>((double*)t, N, w);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_to_double(const void* y, double* b, bool f32, long long n, cudaStream_t st) {
  if (f32) k_to_double<float><<<stride_grid(n), kThreads, 0, st>>>((const float*)y, b, n);
  else k_to_double<double><<<stride_grid(n), kThreads, 0, st>>>((const double*)y, b, n);
  g_mf_launches += 1;
  return cudaGetLastError();
}

cudaError_t mf_launch_adj_grad(const double* F, const double* P, const void* lam, bool f32, const int32_t* phase,
                               const double* scale, long long N, int nphase, const AdjWeights& w,
                               double* partials, int nblk, double* out, double* dscale, cudaStream_t st) {
  const size_t sm = (size_t)2 * nphase * sizeof(double);
  if (f32)
    k_adj_grad<float><<<nblk, kThreads, sm, st>>>(F, P, (const float*)lam, phase, scale, N, nphase, w, partials,
                                                  dscale);
  else
    k_adj_grad<double><<<nblk, kThreads, sm, st>>>(F, P, (const double*)lam, phase, scale, N, nphase, w,
                                                   partials, dscale);
  k_adj_fin<<<1, kThreads, 0, st>>>(partials, nblk, 2 * nphase, out);
  g_mf_launches += 2;
  return cudaGetLastError();
}
