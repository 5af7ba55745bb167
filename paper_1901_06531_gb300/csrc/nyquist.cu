// Nyquist content of an FP32 Newton correction.
//
// In exact arithmetic every correction lies in the range of G*, which holds
// no Nyquist frequency (G-hat-star is zero wherever an axis index is n_a/2,
// Eq. eq:G), so F - F-bar never acquires any.  An FP32 correction does: its
// rounding errors have components along the Nyquist modes, G* cannot see them
// in the residual, and through the heterogeneous, nonlinear law they shift
// the non-Nyquist equilibrium as well.  The FP32-inner Newton update
// therefore adds x - Pi x, Pi the orthogonal projection onto the modes with
// at least one axis at its Nyquist index:
//   Pi = Px + Py + Pz - PxPy - PxPz - PyPz + PxPyPz,
//   (Px v)(x, y, z) = (-1)^x / nx * sum_x' (-1)^x' v(x', y, z)   (nx even; 0 for odd nx),
// grouped as (Pi v) = (-1)^x Rx(z, y) + (-1)^y Ry(z, x) + (-1)^z Rz(y, x).
// The alternating sums are accumulated in double-word FP32 arithmetic (the
// FP64 pipe of this part is slow) and the projection is applied in FP64 by
// the Newton update kernel.
#include "dw.cuh"
#include "launch.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ dw dw_add_f(dw a, float v) { return a + dw(v, 0.0f); }

__device__ __forceinline__ dw warp_sum(dw a) {
  for (int o = 16; o > 0; o >>= 1) {
    const dw b(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
    a = a + b;
  }
  return a;
}

// One block per (component, z plane): Sx(y) = sum_x (-1)^x v, Sy(x) =
// sum_y (-1)^y v, Sxy = sum_y (-1)^y Sx(y).
__global__ void __launch_bounds__(kThreads) k_nyq_plane(const float* __restrict__ v, NyqArgs a, long long N) {
  __shared__ dw rows[256];
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int c = blockIdx.x / nz, z = blockIdx.x - (blockIdx.x / nz) * nz;
  const float* pl = v + (long long)c * N + (long long)z * ny * nx;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int y = warp; y < ny; y += nw) {
    dw acc(0.0f, 0.0f);
    for (int x = lane; x < nx; x += 32) {
      const float t = pl[(long long)y * nx + x];
      acc = dw_add_f(acc, (x & 1) ? -t : t);
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      rows[y] = acc;
      a.Sx[((long long)c * nz + z) * ny + y] = dw_join(acc);
    }
  }
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    dw acc(0.0f, 0.0f);
    for (int y = 0; y < ny; ++y) {
      const float t = pl[(long long)y * nx + x];
      acc = dw_add_f(acc, (y & 1) ? -t : t);
    }
    a.Sy[((long long)c * nz + z) * nx + x] = dw_join(acc);
  }
  __syncthreads();
  if (warp == 0) {
    dw acc(0.0f, 0.0f);
    for (int y = lane; y < ny; y += 32) acc = acc + ((y & 1) ? -rows[y] : rows[y]);
    acc = warp_sum(acc);
    if (lane == 0) a.Sxy[(long long)c * nz + z] = dw_join(acc);
  }
}

// Sz(y, x) = sum_z (-1)^z v, one thread per (component, y, x).
__global__ void __launch_bounds__(kThreads) k_nyq_z(const float* __restrict__ v, NyqArgs a, long long N) {
  const long long plane = (long long)a.ny * a.nx;
  const long long total = 9 * plane;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / plane);
    const long long yx = i - c * plane;
    const float* col = v + (long long)c * N + yx;
    dw acc(0.0f, 0.0f);
    for (int z = 0; z < a.nz; ++z) {
      const float t = col[(long long)z * plane];
      acc = dw_add_f(acc, (z & 1) ? -t : t);
    }
    a.Sz[i] = dw_join(acc);
  }
}

// Mixed sums and the three grouped terms; one block per component.
__global__ void __launch_bounds__(kThreads) k_nyq_terms(NyqArgs a) {
  const int c = blockIdx.x;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const bool ex = !(nx & 1), ey = !(ny & 1), ez = !(nz & 1);
  __shared__ double sxyz;
  const double* Sxy = a.Sxy + (long long)c * nz;
  const double* Sz = a.Sz + (long long)c * ny * nx;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += (z & 1) ? -Sxy[z] : Sxy[z];
    sxyz = s;
  }
  __syncthreads();
  // Rz(y, x) = Sz / nz
  for (int i = threadIdx.x; i < ny * nx; i += blockDim.x)
    a.Rz[(long long)c * ny * nx + i] = ez ? (float)(Sz[i] / nz) : 0.0f;
  // Ry(z, x) = Sy / ny - (-1)^z Syz(x) / (ny nz),  Syz(x) = sum_y (-1)^y Sz(y, x)
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    double syz = 0.0;
    for (int y = 0; y < ny; ++y) syz += (y & 1) ? -Sz[(long long)y * nx + x] : Sz[(long long)y * nx + x];
    for (int z = 0; z < nz; ++z) {
      double r = 0.0;
      if (ey) {
        r = a.Sy[((long long)c * nz + z) * nx + x] / ny;
        if (ez) r -= ((z & 1) ? -syz : syz) / ((double)ny * nz);
      }
      a.Ry[((long long)c * nz + z) * nx + x] = (float)r;
    }
  }
  // Rx(z, y) = Sx/nx - (-1)^y Sxy(z)/(nx ny) - (-1)^z Sxz(y)/(nx nz)
  //            + (-1)^(y+z) Sxyz/(nx ny nz),  Sxz(y) = sum_x (-1)^x Sz(y, x)
  for (int y = threadIdx.x; y < ny; y += blockDim.x) {
    double sxz = 0.0;
    for (int x = 0; x < nx; ++x) sxz += (x & 1) ? -Sz[(long long)y * nx + x] : Sz[(long long)y * nx + x];
    for (int z = 0; z < nz; ++z) {
      double r = 0.0;
      if (ex) {
        r = a.Sx[((long long)c * nz + z) * ny + y] / nx;
        const double sy = (y & 1) ? -1.0 : 1.0, sz = (z & 1) ? -1.0 : 1.0;
        if (ey) r -= sy * Sxy[z] / ((double)nx * ny);
        if (ez) r -= sz * sxz / ((double)nx * nz);
        if (ey && ez) r += sy * sz * sxyz / ((double)nx * ny * nz);
      }
      a.Rx[((long long)c * nz + z) * ny + y] = (float)r;
    }
  }
}

}  // namespace

cudaError_t mf_launch_nyquist_terms(const float* x, const NyqArgs& a, long long N, cudaStream_t st) {
  k_nyq_plane<<<9 * a.nz, kThreads, 0, st>>>(x, a, N);
  const long long total = 9LL * a.ny * a.nx;
  long long g = (total + kThreads - 1) / kThreads;
  if (g > 4096) g = 4096;
  k_nyq_z<<<(int)g, kThreads, 0, st>>>(x, a, N);
  k_nyq_terms<<<9, kThreads, 0, st>>>(a);
  g_mf_launches += 3;
  return cudaGetLastError();
}

size_t mf_nyquist_scratch_bytes(int nx, int ny, int nz) {
  const size_t d = (size_t)9 * ((size_t)nz * ny + (size_t)nz * nx + nz + (size_t)ny * nx);
  const size_t f = (size_t)9 * ((size_t)nz * ny + (size_t)nz * nx + (size_t)ny * nx);
  return d * sizeof(double) + f * sizeof(float) + 64;
}

NyqArgs mf_nyquist_args(void* scratch, int nx, int ny, int nz) {
  NyqArgs a;
  a.nx = nx; a.ny = ny; a.nz = nz;
  double* d = (double*)scratch;
  a.Sx = d; d += (size_t)9 * nz * ny;
  a.Sy = d; d += (size_t)9 * nz * nx;
  a.Sxy = d; d += (size_t)9 * nz;
  a.Sz = d; d += (size_t)9 * ny * nx;
  float* f = (float*)d;
  a.Rx = f; f += (size_t)9 * nz * ny;
  a.Ry = f; f += (size_t)9 * nz * nx;
  a.Rz = f;
  return a;
}
