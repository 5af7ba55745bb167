// Split x and y transforms for x-y planes too large for one block's shared
// memory (nx = ny = 256; one 256 x 128 complex plane is 256 KB in FP32).
// A row kernel takes kRows rows of one (component, z) plane (x transform of
// the half-length rows and the split into the real-row spectrum; inverse:
// the merge, the inverse x transform and the output), a column kernel takes
// kCols slots of one plane (the y transform, in place).  The spectrum layout
// is the one of the fused kernels (transform2.cuh): per (c, z) ny rows in
// digit-reversed ky order of nx/2 slots in digit-reversed kx order; between
// the row and the column kernels the rows are in natural y order.
#pragma once

#include "transform2.cuh"

namespace tr3 {

constexpr int kRows = 16;     // rows per row-kernel block
constexpr int kCols = 16;     // slots per column-kernel block
constexpr int kThreads = 256;

template <typename T, int NX>
struct RowShape {
  typedef typename CT<T>::t C;
  static constexpr int H = NX / 2;
  static constexpr int PX = H + 1;
  static constexpr size_t smem() {
    return (size_t)kRows * PX * sizeof(C) + (size_t)NX * sizeof(C) + (size_t)H * sizeof(int);
  }
};

template <typename T, int NY>
struct ColShape {
  typedef typename CT<T>::t C;
  static constexpr size_t smem() { return (size_t)NY * kCols * sizeof(C) + (size_t)NY * sizeof(C); }
};

// Forward rows: real rows (the IO type) -> row spectra (natural y).
// Grid: 9 * nz * (NY / kRows).
template <typename T, int NX>
__global__ void __launch_bounds__(kThreads) k_xrow(const typename tr2::IOT<T>::t* __restrict__ in,
                                                   typename CT<T>::t* __restrict__ spec, int nz, long long N,
                                                   const typename CT<T>::t* __restrict__ gtw,
                                                   const int* __restrict__ gpos, const int* skip) {
  typedef RowShape<T, NX> Sh;
  typedef typename CT<T>::t C;
  typedef typename CT<typename tr2::IOT<T>::t>::t CI;
  static_assert(sizeof(C) == sizeof(CI), "in-place conversion needs equal element sizes");
  if (skip && *(volatile const int*)skip) return;
  constexpr int H = Sh::H, PX = Sh::PX, NY = NX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* twx = buf + kRows * PX;
  int* posx = reinterpret_cast<int*>(twx + NX);
  for (int i = threadIdx.x; i < NX; i += kThreads) twx[i] = gtw[i];
  for (int i = threadIdx.x; i < H; i += kThreads) posx[i] = gpos[i];
  constexpr int nrb = NY / kRows;
  const int rb = blockIdx.x % nrb, cz = blockIdx.x / nrb;   // cz = c * nz + z
  const int c = cz / nz, z = cz - c * nz;
  const CI* src = reinterpret_cast<const CI*>(in + c * N + ((long long)z * NY + rb * kRows) * NX);
  for (int idx = threadIdx.x; idx < kRows * H; idx += kThreads) {
    const int y = idx / H, j = idx - y * H;
    tr2::cp_async_elem(reinterpret_cast<CI*>(buf + y * PX + j), src + idx);
  }
  tr2::cp_async_wait_all();
  if constexpr (!std::is_same<C, CI>::value) {
    for (int idx = threadIdx.x; idx < kRows * H; idx += kThreads) {   // each thread converts its own copies
      const int y = idx / H, j = idx - y * H;
      const CI v = *reinterpret_cast<const CI*>(buf + y * PX + j);
      tr2::io_in(buf[y * PX + j], v);
    }
  }
  __syncthreads();
  fft2::forward<C, H, NX, kRows, 1, PX, 0, 1>(buf, twx);
  constexpr int NP = H / 2 + 1;
  for (int idx = threadIdx.x; idx < kRows * NP; idx += kThreads) {
    const int y = idx % kRows, k = idx / kRows;
    const int km = (H - k) % H;
    C* row = buf + y * PX;
    const int pa = posx[k], pb = posx[km];
    const C za = row[pa], zb = row[pb];
    if (km != k) row[pb] = tr2::split_one<T>(zb, za, twx[km]);
    row[pa] = tr2::split_one<T>(za, zb, twx[k]);
  }
  __syncthreads();
  C* dst = spec + ((long long)cz * NY + rb * kRows) * H;
  for (int idx = threadIdx.x; idx < kRows * H; idx += kThreads) {
    const int y = idx / H, j = idx - y * H;
    dst[idx] = buf[y * PX + j];
  }
}

// y transform of kCols slots of one plane, in place: forward (natural rows in,
// digit-reversed out) or inverse.  Grid: 9 * nz * (H / kCols).
template <typename T, int NY, bool INV>
__global__ void __launch_bounds__(kThreads) k_ycol(typename CT<T>::t* __restrict__ spec, int H,
                                                   const typename CT<T>::t* __restrict__ gtwy,
                                                   const int* skip) {
  typedef typename CT<T>::t C;
  if (skip && *(volatile const int*)skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);   // [NY][kCols]
  C* twy = buf + NY * kCols;
  for (int i = threadIdx.x; i < NY; i += kThreads) twy[i] = gtwy[i];
  const int ncb = H / kCols;
  const int cb = blockIdx.x % ncb, cz = blockIdx.x / ncb;
  C* pl = spec + (long long)cz * NY * H + cb * kCols;
  for (int idx = threadIdx.x; idx < NY * kCols; idx += kThreads) {
    const int y = idx / kCols, s = idx - y * kCols;
    tr2::cp_async_elem(buf + idx, pl + (long long)y * H + s);
  }
  tr2::cp_async_wait_all();
  __syncthreads();
  if (INV) fft2::inverse<C, NY, NY, kCols, 1, 1, 0, kCols>(buf, twy);
  else fft2::forward<C, NY, NY, kCols, 1, 1, 0, kCols>(buf, twy);
  for (int idx = threadIdx.x; idx < NY * kCols; idx += kThreads) {
    const int y = idx / kCols, s = idx - y * kCols;
    pl[(long long)y * H + s] = buf[idx];
  }
}

// Inverse rows: row spectra (natural y) -> real rows, with the output modes
// of tr2::k_xyi (0: store; 2: store and partial sums of y.y; 3: r -= alpha y
// and partial sums of r.r, one partial per block).  Grid: 9 * nz * (NY / kRows).
template <typename T, int NX, int MODE>
__global__ void __launch_bounds__(kThreads) k_xrowi(const typename CT<T>::t* __restrict__ spec,
                                                    typename tr2::IOT<T>::t* __restrict__ out,
                                                    double* __restrict__ partials, int nz, long long N,
                                                    const typename CT<T>::t* __restrict__ gtw,
                                                    const int* __restrict__ gpos, const Scalars* sc,
                                                    const int* skip) {
  typedef RowShape<T, NX> Sh;
  typedef typename CT<T>::t C;
  typedef typename tr2::IOT<T>::t TI;
  typedef typename CT<TI>::t CI;
  static_assert(MODE != 3 || std::is_same<C, CI>::value, "the CG update runs in the compute type");
  if (skip && *(volatile const int*)skip) return;
  constexpr int H = Sh::H, PX = Sh::PX, NY = NX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* twx = buf + kRows * PX;
  int* posx = reinterpret_cast<int*>(twx + NX);
  for (int i = threadIdx.x; i < NX; i += kThreads) twx[i] = gtw[i];
  for (int i = threadIdx.x; i < H; i += kThreads) posx[i] = gpos[i];
  constexpr int nrb = NY / kRows;
  const int rb = blockIdx.x % nrb, cz = blockIdx.x / nrb;
  const int c = cz / nz, z = cz - c * nz;
  const C* src = spec + ((long long)cz * NY + rb * kRows) * H;
  for (int idx = threadIdx.x; idx < kRows * H; idx += kThreads) {
    const int y = idx / H, j = idx - y * H;
    tr2::cp_async_elem(buf + y * PX + j, src + idx);
  }
  tr2::cp_async_wait_all();
  __syncthreads();
  constexpr int NP = H / 2 + 1;
  for (int idx = threadIdx.x; idx < kRows * NP; idx += kThreads) {
    const int y = idx % kRows, k = idx / kRows;
    const int km = (H - k) % H;
    C* row = buf + y * PX;
    const int pa = posx[k], pb = posx[km];
    const C xa = row[pa], xb = row[pb];
    if (k == 0) {   // X_0 real, X_H = 0: Z_0 = x0 + i x0
      C z0;
      z0.x = xa.x; z0.y = xa.x;
      row[pa] = z0;
      continue;
    }
    if (km != k) row[pb] = tr2::merge_one<T>(xb, xa, twx[km]);
    row[pa] = tr2::merge_one<T>(xa, xb, twx[k]);
  }
  __syncthreads();
  fft2::inverse<C, H, NX, kRows, 1, PX, 0, 1>(buf, twx);
  CI* dst = reinterpret_cast<CI*>(out + c * N + ((long long)z * NY + rb * kRows) * NX);
  double acc = 0.0;
  float fs = 0.f, fc = 0.f;
  auto fadd = [&](float v) {
    const float tt = fs + v;
    fc += (fabsf(fs) >= fabsf(v)) ? ((fs - tt) + v) : ((v - tt) + fs);
    fs = tt;
  };
  auto fsq = [&](float v) {
    const float p = v * v;
    fadd(p);
    fadd(fmaf(v, v, -p));
  };
  T alpha = (T)0;
  if (MODE == 3) alpha = (T)sc->alpha;
  for (int idx = threadIdx.x; idx < kRows * H; idx += kThreads) {
    const int y = idx / H, j = idx - y * H;
    const C v = buf[y * PX + j];
    if constexpr (MODE == 3) {
      C r = dst[idx];
      r.x -= alpha * v.x;
      r.y -= alpha * v.y;
      dst[idx] = r;
      if (sizeof(T) == 4) { fsq((float)r.x); fsq((float)r.y); }
      else acc += (double)r.x * (double)r.x + (double)r.y * (double)r.y;
    } else {
      const CI w = tr2::io_out(v);
      dst[idx] = w;
      if (MODE == 2) {
        if (sizeof(TI) == 4) { fsq((float)w.x); fsq((float)w.y); }
        else acc += (double)w.x * (double)w.x + (double)w.y * (double)w.y;
      }
    }
  }
  if (sizeof(TI) == 4) acc = (double)fs + (double)fc;
  if (MODE >= 2) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double s = (threadIdx.x < (kThreads >> 5)) ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) partials[blockIdx.x] = s;
    }
  }
}

// ---------------------------------------------------------------- launchers
template <typename K>
cudaError_t set_smem(K kernel, size_t sm) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <typename T, int NX>
cudaError_t xyf(const void* in, void* spec, const XYArgs& a, cudaStream_t st) {
  typedef typename CT<T>::t C;
  typedef typename tr2::IOT<T>::t TI;
  const size_t sr = RowShape<T, NX>::smem(), sc = ColShape<T, NX>::smem();
  cudaError_t e = set_smem(k_xrow<T, NX>, sr);
  if (e == cudaSuccess) e = set_smem(k_ycol<T, NX, false>, sc);
  if (e != cudaSuccess) return e;
  k_xrow<T, NX><<<9 * a.nz * (NX / kRows), kThreads, sr, st>>>((const TI*)in, (C*)spec, a.nz, a.N,
                                                                  (const C*)a.twx, a.xpos, a.skip);
  k_ycol<T, NX, false><<<9 * a.nz * (NX / 2 / kCols), kThreads, sc, st>>>((C*)spec, NX / 2, (const C*)a.twy,
                                                                           a.skip);
  g_mf_launches += 2;
  return cudaGetLastError();
}

template <typename T, int NX, int MODE>
cudaError_t xyi(const void* spec, void* out, double* partials, const XYArgs& a, const Scalars* sc,
                cudaStream_t st) {
  typedef typename CT<T>::t C;
  typedef typename tr2::IOT<T>::t TI;
  const size_t sr = RowShape<T, NX>::smem(), scl = ColShape<T, NX>::smem();
  cudaError_t e = set_smem(k_xrowi<T, NX, MODE>, sr);
  if (e == cudaSuccess) e = set_smem(k_ycol<T, NX, true>, scl);
  if (e != cudaSuccess) return e;
  k_ycol<T, NX, true><<<9 * a.nz * (NX / 2 / kCols), kThreads, scl, st>>>((C*)spec, NX / 2, (const C*)a.twy,
                                                                          a.skip);
  k_xrowi<T, NX, MODE><<<9 * a.nz * (NX / kRows), kThreads, sr, st>>>((const C*)spec, (TI*)out, partials, a.nz,
                                                                      a.N, (const C*)a.twx, a.xpos, sc, a.skip);
  g_mf_launches += 2;
  return cudaGetLastError();
}

}  // namespace tr3
