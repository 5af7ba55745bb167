// The projected-operator passes: y = F^-1{ G-hat-star : F{ K : x } }
// (Eq. linequil2ast) and the residual b = -F^-1{ G-hat-star : F{ P - P-bar } }.
//
// Three kernels per application, each one pass over HBM:
//   xy_forward : per (z-plane, component c): (K:x)_c or P_c for the plane,
//                real-to-complex transform along x (two rows packed as one
//                complex row), then the complex transform along y; the plane
//                stays in shared memory throughout.
//   zpass      : per tile of (ky, kx) columns, all nine components: forward
//                transform along z, G-hat-star (Eq. eq:Gnewnew) with the
//                per-component null-frequency control, inverse along z.
//   xy_inverse : per (z-plane, component): inverse along y, complex-to-real
//                along x, optional dot product with a second field.
//
// Spectrum layout (per component c and plane z, one contiguous block of
// ny/2 x nx complex values, row q', slot s):
//   slot s holds x-frequency kx(s) in [0, nx/2) of parity e(s) -- the x-Nyquist
//   coefficient is never stored because G-hat-star is zero there;
//   row q' holds y-frequency ky = 2 * yk(q') + e(s);
//   plane position p holds z-frequency kz = zk(p) during the z-pass.
// The 1/N of the forward transform is applied once, in the z-pass.
#include "common.cuh"
#include "dw.cuh"

#include "launch.h"

// ---------------------------------------------------------------- xy forward
// MODE 1: the input is the field itself, component c (the tangent has been
// applied by the streaming pass).
template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_xy_forward(const T* __restrict__ in, const T* __restrict__ K45,
                                                    typename CT<T>::t* __restrict__ spec, XYArgs a) {
  typedef typename CT<T>::t C;
  if (a.skip && *(volatile const int*)a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = a.nx, ny = a.ny, hy = ny / 2;
  const int P = hy * nx;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* twx = buf + P;
  C* twy = twx + nx;
  int* xpos = reinterpret_cast<int*>(twy + ny);
  const C* gtwx = reinterpret_cast<const C*>(a.twx);
  const C* gtwy = reinterpret_cast<const C*>(a.twy);
  for (int i = threadIdx.x; i < nx; i += blockDim.x) { twx[i] = gtwx[i]; xpos[i] = a.xpos[i]; }
  for (int i = threadIdx.x; i < ny; i += blockDim.x) twy[i] = gtwy[i];

  const int c = blockIdx.x % 9;
  const int z = blockIdx.x / 9;
  const long long N = a.N;
  const long long plane = (long long)z * ny * nx;

  for (int idx = threadIdx.x; idx < P; idx += blockDim.x) {
    const int q = idx / nx, j = idx - (idx / nx) * nx;
    const long long v0 = plane + (long long)q * nx + j;
    const long long v1 = v0 + (long long)hy * nx;
    buf[MF_AT(idx, P)] = cmake(in[MF_AT(c * N + v0, 9 * N)], in[MF_AT(c * N + v1, 9 * N)]);
  }
  __syncthreads();

  // x transform of the hy packed rows (contiguous sequences)
  fft_run<C, false, false>(buf, a.px, hy, 1, nx, 0, 1, twx, nx, P);

  // split the packed rows into the spectra of rows q and q+hy, and apply the
  // first (radix-2) stage of the y transform, which combines exactly those two
  const int hx = nx / 2;
  for (int idx = threadIdx.x; idx < hy * hx; idx += blockDim.x) {
    const int q = idx / hx, k = idx - (idx / hx) * hx;
    const int sa = xpos[MF_AT(k, nx)];
    const int sb = xpos[MF_AT(k == 0 ? hx : nx - k, nx)];
    const C za = buf[MF_AT(q * nx + sa, P)], zb = buf[MF_AT(q * nx + sb, P)];
    C xa, xb;
    if (k == 0) {
      xa = cmake(za.x, (T)0);
      xb = cmake(za.y, (T)0);
    } else {
      xa = cmake((T)0.5 * (za.x + zb.x), (T)0.5 * (za.y - zb.y));
      xb = cmake((T)0.5 * (za.y + zb.y), (T)-0.5 * (za.x - zb.x));
    }
    buf[MF_AT(q * nx + sa, P)] = cadd(xa, xb);
    buf[MF_AT(q * nx + sb, P)] = cmul(csub(xa, xb), twy[MF_AT(q, ny)]);
  }
  __syncthreads();

  // remaining y stages: nx column sequences of length hy, stride nx
  fft_run<C, false, true>(buf, a.pyh, nx, nx, 0, 1, nx, twy, ny, P);

  const long long o = ((long long)c * a.nz + z) * P;
  for (int idx = threadIdx.x; idx < P; idx += blockDim.x) spec[MF_AT(o + idx, 9LL * a.nz * P)] = buf[idx];
}

// ---------------------------------------------------------------- xy inverse
// y = oscale * (inverse transform of the plane).  DOT 0: out[c] = y.
// DOT 1: out[c] = y and the block's partial of sum y * w[c] (FP64) goes to
// partials[blockIdx.x].  DOT 2: out[c] = y and the partial of sum y^2.
// DOT 3 (CG residual update): out[c] -= alpha * y with alpha from sc, and the
// partial of sum out[c]^2 after the update; y itself is not stored.
template <typename T, int DOT>
__global__ void __launch_bounds__(512) k_xy_inverse(const typename CT<T>::t* __restrict__ spec,
                                                    T* __restrict__ out, const T* __restrict__ w,
                                                    double* __restrict__ partials, T oscale,
                                                    XYArgs a, const Scalars* sc) {
  typedef typename CT<T>::t C;
  if (a.skip && *(volatile const int*)a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int nx = a.nx, ny = a.ny, hy = ny / 2;
  const int P = hy * nx;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* twx = buf + P;
  C* twy = twx + nx;
  int* xpos = reinterpret_cast<int*>(twy + ny);
  const C* gtwx = reinterpret_cast<const C*>(a.twx);
  const C* gtwy = reinterpret_cast<const C*>(a.twy);
  for (int i = threadIdx.x; i < nx; i += blockDim.x) { twx[i] = gtwx[i]; xpos[i] = a.xpos[i]; }
  for (int i = threadIdx.x; i < ny; i += blockDim.x) twy[i] = gtwy[i];

  const int c = blockIdx.x % 9;
  const int z = blockIdx.x / 9;
  const long long N = a.N;
  const long long o = ((long long)c * a.nz + z) * P;
  for (int idx = threadIdx.x; idx < P; idx += blockDim.x) buf[MF_AT(idx, P)] = spec[MF_AT(o + idx, 9LL * a.nz * P)];
  __syncthreads();

  fft_run<C, true, true>(buf, a.pyh, nx, nx, 0, 1, nx, twy, ny, P);

  const int hx = nx / 2;
  for (int idx = threadIdx.x; idx < hy * hx; idx += blockDim.x) {
    const int q = idx / hx, k = idx - (idx / hx) * hx;
    const int sa = xpos[MF_AT(k, nx)];
    const int sb = xpos[MF_AT(k == 0 ? hx : nx - k, nx)];
    const C y0 = buf[MF_AT(q * nx + sa, P)];
    const C t = cmulc(buf[MF_AT(q * nx + sb, P)], twy[MF_AT(q, ny)]);
    const C xa = cadd(y0, t), xb = csub(y0, t);
    if (k == 0) {
      buf[MF_AT(q * nx + sa, P)] = cmake(xa.x, xb.x);
      buf[MF_AT(q * nx + sb, P)] = cmake((T)0, (T)0);
    } else {
      buf[MF_AT(q * nx + sa, P)] = cmake(xa.x - xb.y, xa.y + xb.x);
      buf[MF_AT(q * nx + sb, P)] = cmake(xa.x + xb.y, xb.x - xa.y);
    }
  }
  __syncthreads();

  fft_run<C, true, false>(buf, a.px, hy, 1, nx, 0, 1, twx, nx, P);

  const long long plane = (long long)z * ny * nx;
  double acc = 0.0;
  T alpha = (T)0;
  if (DOT == 3) alpha = (T)sc->alpha;
  for (int idx = threadIdx.x; idx < P; idx += blockDim.x) {
    const int q = idx / nx, j = idx - (idx / nx) * nx;
    const long long v0 = plane + (long long)q * nx + j;
    const long long v1 = v0 + (long long)hy * nx;
    const C v = buf[MF_AT(idx, P)];
    const T o0 = v.x * oscale, o1 = v.y * oscale;
    const long long i0 = MF_AT(c * N + v0, 9 * N), i1 = MF_AT(c * N + v1, 9 * N);
    if (DOT == 3) {
      const T r0 = out[i0] - alpha * o0;
      const T r1 = out[i1] - alpha * o1;
      out[i0] = r0;
      out[i1] = r1;
      acc += (double)r0 * (double)r0 + (double)r1 * (double)r1;
    } else {
      out[i0] = o0;
      out[i1] = o1;
    }
    if (DOT == 1) acc += (double)o0 * (double)w[i0] + (double)o1 * (double)w[i1];
    if (DOT == 2) acc += (double)o0 * (double)o0 + (double)o1 * (double)o1;
  }
  if (DOT) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) partials[blockIdx.x] = s;
    }
  }
}

// ---------------------------------------------------------------- z pass
// MODE 0: projected operator (with a.lin, the null-frequency coefficient / N
// times *a.lin_alpha added to a.lin).  MODE 1: residual (adds a.add at the
// null frequency and records the null-frequency coefficient / N in a.mean_out).
template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_zpass(typename CT<T>::t* __restrict__ spec, ZArgs a) {
  typedef typename CT<T>::t C;
  if (a.skip && *(volatile const int*)a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = a.nx, ny = a.ny, nz = a.nz, S = a.S;
  const int ncol = (ny / 2) * nx;
  C* buf = reinterpret_cast<C*>(smem_raw);        // [9][nz][S]
  C* twz = buf + 9 * nz * S;
  int* zk = reinterpret_cast<int*>(twz + nz);
  const C* gtwz = reinterpret_cast<const C*>(a.twz);
  for (int i = threadIdx.x; i < nz; i += blockDim.x) { twz[i] = gtwz[i]; zk[i] = a.zk[i]; }

  const int col0 = blockIdx.x * S;
  const int tot = 9 * nz * S;
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int s = idx % S;
    const int cz = idx / S;          // c * nz + z
    const int col = col0 + s;
    buf[MF_AT(idx, tot)] =
        (col < ncol) ? spec[MF_AT((long long)cz * ncol + col, 9LL * nz * ncol)] : cmake((T)0, (T)0);
  }
  __syncthreads();

  fft_run<C, false, true>(buf, a.pz, 9 * S, S, nz * S, 1, S, twz, nz, tot);

  const T scale = (T)a.scale;
  const int zstride = nz * S;
  for (int idx = threadIdx.x; idx < nz * S; idx += blockDim.x) {
    const int s = idx % S, p = idx / S;
    const int col = col0 + s;
    if (col >= ncol) continue;
    const int qr = col / nx, slot = col - (col / nx) * nx;
    const int kx = a.xk[MF_AT(slot, nx)];
    const int ky = 2 * a.yk[MF_AT(qr, ny / 2)] + a.xe[MF_AT(slot, nx)];
    const int kz = zk[MF_AT(p, nz)];
    C* e = buf + MF_AT(idx, tot - 8 * zstride);   // e[c * zstride], c < 9
    const bool nyq = (2 * ky == ny) || ((nz % 2 == 0) && (2 * kz == nz));
    if (nyq) {
#pragma unroll
      for (int c = 0; c < 9; ++c) e[c * zstride] = cmake((T)0, (T)0);
    } else if (kx == 0 && ky == 0 && kz == 0) {
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const C X = e[c * zstride];
        if (MODE == 1 && a.mean_out) a.mean_out[c] = (double)X.x / (double)a.N;
        if (MODE == 0 && a.lin) a.lin[c] += *a.lin_alpha * ((double)X.x / (double)a.N);
        if (a.mask & (1u << c)) {
          T add = (MODE == 1) ? (T)(a.add_dev ? a.add_dev[c] : a.add[c]) : (T)0;
          e[c * zstride] = cmake(scale * X.x + add, scale * X.y);
        } else {
          e[c * zstride] = cmake((T)0, (T)0);
        }
      }
    } else {
      const int kys = (ky < ny / 2) ? ky : ky - ny;
      const int kzs = (2 * kz < nz) ? kz : kz - nz;
      const T xi0 = (T)kx / (T)nx, xi1 = (T)kys / (T)ny, xi2 = (T)kzs / (T)nz;
      const T inv = scale / (xi0 * xi0 + xi1 * xi1 + xi2 * xi2);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const C A0 = e[(3 * i + 0) * zstride];
        const C A1 = e[(3 * i + 1) * zstride];
        const C A2 = e[(3 * i + 2) * zstride];
        C q;
        q.x = (A0.x * xi0 + A1.x * xi1 + A2.x * xi2) * inv;
        q.y = (A0.y * xi0 + A1.y * xi1 + A2.y * xi2) * inv;
        e[(3 * i + 0) * zstride] = cmake(q.x * xi0, q.y * xi0);
        e[(3 * i + 1) * zstride] = cmake(q.x * xi1, q.y * xi1);
        e[(3 * i + 2) * zstride] = cmake(q.x * xi2, q.y * xi2);
      }
    }
  }
  __syncthreads();

  fft_run<C, true, true>(buf, a.pz, 9 * S, S, nz * S, 1, S, twz, nz, tot);

  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int s = idx % S;
    const int cz = idx / S;
    const int col = col0 + s;
    if (col < ncol) spec[MF_AT((long long)cz * ncol + col, 9LL * nz * ncol)] = buf[MF_AT(idx, tot)];
  }
}

// ---------------------------------------------------------------- launchers
long long g_mf_launches = 0;


template <typename T>
static size_t xy_smem(const XYArgs& a) {
  typedef typename CT<T>::t C;
  return (size_t)(a.ny / 2) * a.nx * sizeof(C) + (size_t)(a.nx + a.ny) * sizeof(C) +
         (size_t)a.nx * sizeof(int);
}

template <typename T>
static size_t z_smem(const ZArgs& a) {
  typedef typename CT<T>::t C;
  return (size_t)9 * a.nz * a.S * sizeof(C) + (size_t)a.nz * sizeof(C) + (size_t)a.nz * sizeof(int);
}

template <typename T, int MODE>
static cudaError_t launch_xy_forward(const T* in, const T* K45, void* spec, const XYArgs& a,
                                     cudaStream_t st) {
  const size_t sm = xy_smem<T>(a);
  cudaError_t e = cudaFuncSetAttribute(k_xy_forward<T, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_xy_forward<T, MODE><<<9 * a.nz, 512, sm, st>>>(in, K45, (typename CT<T>::t*)spec, a);
  ++g_mf_launches;
  return cudaGetLastError();
}

template <typename T, int DOT>
static cudaError_t launch_xy_inverse(const void* spec, T* out, const T* w, double* partials,
                                     T oscale, const XYArgs& a, cudaStream_t st,
                                     const Scalars* sc = nullptr) {
  const size_t sm = xy_smem<T>(a);
  cudaError_t e = cudaFuncSetAttribute(k_xy_inverse<T, DOT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_xy_inverse<T, DOT><<<9 * a.nz, 512, sm, st>>>((const typename CT<T>::t*)spec, out, w,
                                                  partials, oscale, a, sc);
  ++g_mf_launches;
  return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t launch_zpass(void* spec, const ZArgs& a, cudaStream_t st) {
  const size_t sm = z_smem<T>(a);
  cudaError_t e = cudaFuncSetAttribute(k_zpass<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  const int ncol = (a.ny / 2) * a.nx;
  const int nblk = (ncol + a.S - 1) / a.S;
  k_zpass<T, MODE><<<nblk, 512, sm, st>>>((typename CT<T>::t*)spec, a);
  ++g_mf_launches;
  return cudaGetLastError();
}

cudaError_t mf_launch_residual(const double* P, void* spec, double* b, double* partials,
                               const XYArgs& xa, const ZArgs& za, bool dw, cudaStream_t st) {
  if (xa.v2 && dw) {
    cudaError_t e = mf_v2_xyf_dw(P, spec, xa, st);
    if (e == cudaSuccess) e = mf_v2_zp_dw(spec, za, st);
    if (e == cudaSuccess) e = mf_v2_xyi_dw(spec, b, partials, xa, st);
    return e;
  }
  if (xa.v2) {
    cudaError_t e = mf_v2_xyf_f64(P, spec, xa, st);
    if (e == cudaSuccess) e = mf_v2_zp_f64(1, spec, za, st);
    if (e == cudaSuccess) e = mf_v2_xyi_f64(0, spec, b, partials, xa, nullptr, st);
    return e;
  }
  cudaError_t e = launch_xy_forward<double, 1>(P, nullptr, spec, xa, st);
  if (e != cudaSuccess) return e;
  e = launch_zpass<double, 1>(spec, za, st);
  if (e != cudaSuccess) return e;
  return launch_xy_inverse<double, 2>(spec, b, nullptr, partials, 1.0, xa, st);
}

namespace {

// FP64 -> FP32 rounded through the double-word split (no FP64 instruction)
__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const dw d = dw_split(a[i]);
    b[i] = __fadd_rn(d.hi, d.lo);
  }
}

__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = f32_as_f64(a[i]);
}

}  // namespace

cudaError_t mf_launch_residual_f32(const double* P, float* Pf, void* spec, float* bf, double* b,
                                   const XYArgs& xa, const ZArgs& za, cudaStream_t st) {
  if (!xa.v2) return cudaErrorInvalidValue;
  const long long n9 = 9 * xa.N;
  cudaError_t e = cudaSuccess;
  if (P) {
    k_d2f<<<stride_grid(n9), 256, 0, st>>>(P, Pf, n9);
    e = cudaGetLastError();
    g_mf_launches += 1;
  }
  if (e == cudaSuccess) e = mf_v2_xyf_f32(Pf, spec, xa, st);
  if (e == cudaSuccess) e = mf_v2_zp_f32(1, spec, za, st);
  if (e == cudaSuccess) e = mf_v2_xyi_f32(0, spec, bf, nullptr, xa, nullptr, st);
  if (e == cudaSuccess) {
    k_f2d<<<stride_grid(n9), 256, 0, st>>>(bf, b, n9);
    e = cudaGetLastError();
  }
  g_mf_launches += 1;
  return e;
}

cudaError_t mf_launch_project(bool f32, const void* t, void* spec, void* out, int inv_mode,
                              double* partials, const XYArgs& xa, const ZArgs& za,
                              const Scalars* sc, cudaStream_t st) {
  cudaError_t e;
  if (xa.v2) {
    e = f32 ? mf_v2_xyf_f32(t, spec, xa, st) : mf_v2_xyf_f64(t, spec, xa, st);
    if (e == cudaSuccess) e = f32 ? mf_v2_zp_f32(0, spec, za, st) : mf_v2_zp_f64(0, spec, za, st);
    if (e == cudaSuccess)
      e = f32 ? mf_v2_xyi_f32(inv_mode, spec, out, partials, xa, sc, st)
              : mf_v2_xyi_f64(inv_mode, spec, out, partials, xa, sc, st);
    return e;
  }
  if (f32) {
    e = launch_xy_forward<float, 1>((const float*)t, nullptr, spec, xa, st);
    if (e == cudaSuccess) e = launch_zpass<float, 0>(spec, za, st);
    if (e != cudaSuccess) return e;
    if (inv_mode == 3) return launch_xy_inverse<float, 3>(spec, (float*)out, nullptr, partials, 1.0f, xa, st, sc);
    return launch_xy_inverse<float, 0>(spec, (float*)out, nullptr, nullptr, 1.0f, xa, st);
  }
  e = launch_xy_forward<double, 1>((const double*)t, nullptr, spec, xa, st);
  if (e == cudaSuccess) e = launch_zpass<double, 0>(spec, za, st);
  if (e != cudaSuccess) return e;
  if (inv_mode == 3) return launch_xy_inverse<double, 3>(spec, (double*)out, nullptr, partials, 1.0, xa, st, sc);
  return launch_xy_inverse<double, 0>(spec, (double*)out, nullptr, nullptr, 1.0, xa, st);
}

cudaError_t mf_launch_project_part(int which, bool f32, const void* t, void* spec, void* r,
                                   double* partials, const XYArgs& xa, const ZArgs& za,
                                   const Scalars* sc, cudaStream_t st) {
  if (xa.v2) {
    if (which == 0) return f32 ? mf_v2_xyf_f32(t, spec, xa, st) : mf_v2_xyf_f64(t, spec, xa, st);
    if (which == 1) return f32 ? mf_v2_zp_f32(0, spec, za, st) : mf_v2_zp_f64(0, spec, za, st);
    return f32 ? mf_v2_xyi_f32(3, spec, r, partials, xa, sc, st) : mf_v2_xyi_f64(3, spec, r, partials, xa, sc, st);
  }
  if (f32) {
    if (which == 0) return launch_xy_forward<float, 1>((const float*)t, nullptr, spec, xa, st);
    if (which == 1) return launch_zpass<float, 0>(spec, za, st);
    return launch_xy_inverse<float, 3>(spec, (float*)r, nullptr, partials, 1.0f, xa, st, sc);
  }
  if (which == 0) return launch_xy_forward<double, 1>((const double*)t, nullptr, spec, xa, st);
  if (which == 1) return launch_zpass<double, 0>(spec, za, st);
  return launch_xy_inverse<double, 3>(spec, (double*)r, nullptr, partials, 1.0, xa, st, sc);
}

bool mf_v2_supported(int nx, int ny, int nz) {
  auto ok = [](int n) { return n == 16 || n == 32 || n == 48 || n == 64 || n == 96 || n == 128 || n == 256; };
  return nx == ny && ok(nx) && ok(nz);
}

bool mf_split_supported(int nx) { return nx == 32 || nx == 256; }
bool mf_persist_supported(int nx) { return nx == 48 || nx == 64 || nx == 96 || nx == 128; }
bool mf_cluster_supported(int nx) { return nx == 128; }

int mf_xy_blocks(int ny, int nz, bool split) { return split ? 9 * nz * (ny / 16) : 9 * nz; }
