// Launchers of the fixed-size transform kernels for one precision T; included
// by transform2_f32.cu and transform2_f64.cu (one translation unit each).
#pragma once

#include "transform2.cuh"
#include "transform2c.cuh"
#include "transform3.cuh"

namespace tr2 {

// The shared-memory opt-in of a fixed-size kernel: its size is a constant of
// the instantiation, so it is set once per process (on the device current at
// the first launch; one process drives one device) instead of at every
// launch, which for small cells costs as much host time as the launch.
template <auto K>
cudaError_t smem_once(size_t sm) {
  static const cudaError_t e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  return e;
}

inline int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      return 1;
  }
  return n;
}

template <int NX>
cudaError_t launch_xyf_p(const float* in, void* spec, const XYArgs& a, cudaStream_t st) {
  const size_t sm = PersistShape<NX>::smem();
  cudaError_t e = smem_once<k_xyf_p<NX>>(sm);
  if (e != cudaSuccess) return e;
  const int nplanes = 9 * a.nz;
  const int grid = nplanes < num_sms() ? nplanes : num_sms();
  ++g_mf_launches;
  return launch_k(a.pdl != 0, k_xyf_p<NX>, dim3(grid), dim3(kPersistThreads), sm, st, in, (float2*)spec, a.nz,
                  a.N, (const float2*)a.twx, a.xpos, a.skip, a.flags);
}

// the two-CTA cluster kernels (FP32, 128 x 128 planes): grid of 2 x 9 nz
// CTAs, consecutive pairs forming a cluster
inline cudaError_t launch_xyf_c(const float* in, void* spec, const XYArgs& a, cudaStream_t st) {
  const size_t sm = clu::smem();
  cudaError_t e = smem_once<k_xyf_c<clu::NX>>(sm);
  if (e != cudaSuccess) return e;
  ++g_mf_launches;
  return launch_k(a.pdl != 0, k_xyf_c<clu::NX>, dim3(18 * a.nz), dim3(clu::kCThreads), sm, st, in, (float2*)spec, a.nz, a.N,
                  (const float2*)a.twx, a.skip);
}

template <int MODE>
cudaError_t launch_xyi_c(const void* spec, float* out, double* partials, const XYArgs& a, const Scalars* sc,
                         cudaStream_t st) {
  const size_t sm = clu::smem();
  cudaError_t e = smem_once<k_xyi_c<MODE>>(sm);
  if (e != cudaSuccess) return e;
  ++g_mf_launches;
  return launch_k(a.pdl != 0, k_xyi_c<MODE>, dim3(18 * a.nz), dim3(clu::kCThreads), sm, st, (const float2*)spec,
                  out, partials, a.nz, a.N, (const float2*)a.twx, const_cast<Scalars*>(sc), a.skip,
                  MODE == 3 ? a.fin : 0);
}

template <typename T, int NX>
cudaError_t launch_xyf(const typename IOT<T>::t* in, void* spec, const XYArgs& a, cudaStream_t st) {
  typedef typename CT<T>::t C;
  if constexpr (std::is_same<T, float>::value && NX == clu::NX) {
    if (a.cluster_f) return launch_xyf_c(in, spec, a, st);
  }
  if constexpr (std::is_same<T, float>::value && RowPlan<NX / 2>::NST == 2) {
    if (a.persist) return launch_xyf_p<NX>(in, spec, a, st);
  }
  const size_t sm = XYShape<T, NX>::smem();
  cudaError_t e = smem_once<k_xyf<T, NX>>(sm);
  if (e != cudaSuccess) return e;
  ++g_mf_launches;
  return launch_k(a.pdl != 0, k_xyf<T, NX>, dim3(9 * a.nz), dim3(xy_threads<T, NX>()), sm, st, in, (C*)spec, a.nz, a.N,
                  (const C*)a.twx, a.xpos, a.skip);
}

template <typename T, int NX, int MODE>
cudaError_t launch_xyi(const void* spec, typename IOT<T>::t* out, double* partials, const XYArgs& a,
                       const Scalars* sc, cudaStream_t st) {
  typedef typename CT<T>::t C;
  if constexpr (std::is_same<T, float>::value && NX == clu::NX) {
    if (a.cluster_i) return launch_xyi_c<MODE>(spec, out, partials, a, sc, st);
  }
  const size_t sm = XYShape<T, NX>::smem();
  cudaError_t e = smem_once<k_xyi<T, NX, MODE>>(sm);
  if (e != cudaSuccess) return e;
  // the scalar block is written only by the fused finish (a.fin, MODE 3)
  ++g_mf_launches;
  return launch_k(a.pdl != 0, k_xyi<T, NX, MODE>, dim3(9 * a.nz), dim3(xy_threads<T, NX>()), sm, st, (const C*)spec,
                  out, partials, a.nz, a.N, (const C*)a.twx, a.xpos, const_cast<Scalars*>(sc), a.skip,
                  MODE == 3 ? a.fin : 0);
}

template <typename T, int NZ, int MODE, int S>
cudaError_t launch_zp_s(void* spec, const ZArgs& a, cudaStream_t st) {
  typedef typename CT<T>::t C;
  typedef ZShape<T, NZ, S> Sh;
  const size_t sm = Sh::smem();
  cudaError_t e = smem_once<k_zp<T, NZ, MODE, S>>(sm);
  if (e != cudaSuccess) return e;
  const int ncol = a.ny * (a.nx / 2);
  if (ncol % S) return cudaErrorInvalidValue;
  ++g_mf_launches;
  return launch_k(a.pdl != 0, k_zp<T, NZ, MODE, S>, dim3(3 * (ncol / S)), dim3(z_threads(S)), sm, st, (C*)spec, a);
}

// The tile the autotuner chose: a.S in {4, 8, 16} for the operator (MODE 0,
// inside the CG loop), {4, 8} for the residual (MODE 1); else the default.
template <typename T, int NZ, int MODE>
cudaError_t launch_zp(void* spec, const ZArgs& a, cudaStream_t st) {
  if (a.S == 4) return launch_zp_s<T, NZ, MODE, 4>(spec, a, st);
  if constexpr (MODE == 0) {
    if (a.S == 16) return launch_zp_s<T, NZ, MODE, 16>(spec, a, st);
  }
  return launch_zp_s<T, NZ, MODE, 8>(spec, a, st);
}

template <typename T>
cudaError_t xyf(const void* in, void* spec, const XYArgs& a, cudaStream_t st) {
  const typename IOT<T>::t* p = (const typename IOT<T>::t*)in;
  if (a.split) {
    switch (a.nx) {
      case 32: return tr3::xyf<T, 32>(in, spec, a, st);
      case 256: return tr3::xyf<T, 256>(in, spec, a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.nx) {
    case 16: return launch_xyf<T, 16>(p, spec, a, st);
    case 32: return launch_xyf<T, 32>(p, spec, a, st);
    case 48: return launch_xyf<T, 48>(p, spec, a, st);
    case 64: return launch_xyf<T, 64>(p, spec, a, st);
    case 96: return launch_xyf<T, 96>(p, spec, a, st);
    case 128: return launch_xyf<T, 128>(p, spec, a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int MODE>
cudaError_t xyi_m(const void* spec, void* out, double* partials, const XYArgs& a, const Scalars* sc,
                  cudaStream_t st) {
  typename IOT<T>::t* o = (typename IOT<T>::t*)out;
  if (a.split) {
    switch (a.nx) {
      case 32: return tr3::xyi<T, 32, MODE>(spec, out, partials, a, sc, st);
      case 256: return tr3::xyi<T, 256, MODE>(spec, out, partials, a, sc, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.nx) {
    case 16: return launch_xyi<T, 16, MODE>(spec, o, partials, a, sc, st);
    case 32: return launch_xyi<T, 32, MODE>(spec, o, partials, a, sc, st);
    case 48: return launch_xyi<T, 48, MODE>(spec, o, partials, a, sc, st);
    case 64: return launch_xyi<T, 64, MODE>(spec, o, partials, a, sc, st);
    case 96: return launch_xyi<T, 96, MODE>(spec, o, partials, a, sc, st);
    case 128: return launch_xyi<T, 128, MODE>(spec, o, partials, a, sc, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t xyi(int mode, const void* spec, void* out, double* partials, const XYArgs& a, const Scalars* sc,
                cudaStream_t st) {
  if (mode == 0) return xyi_m<T, 0>(spec, out, partials, a, sc, st);
  if (mode == 2) return xyi_m<T, 2>(spec, out, partials, a, sc, st);
  if (mode == 3) return xyi_m<T, 3>(spec, out, partials, a, sc, st);
  return cudaErrorInvalidValue;
}

template <typename T, int MODE>
cudaError_t zp_m(void* spec, const ZArgs& a, cudaStream_t st) {
  switch (a.nz) {
    case 16: return launch_zp<T, 16, MODE>(spec, a, st);
    case 32: return launch_zp<T, 32, MODE>(spec, a, st);
    case 48: return launch_zp<T, 48, MODE>(spec, a, st);
    case 64: return launch_zp<T, 64, MODE>(spec, a, st);
    case 96: return launch_zp<T, 96, MODE>(spec, a, st);
    case 128: return launch_zp<T, 128, MODE>(spec, a, st);
    case 256: return launch_zp<T, 256, MODE>(spec, a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t zp(int mode, void* spec, const ZArgs& a, cudaStream_t st) {
  return mode == 1 ? zp_m<T, 1>(spec, a, st) : zp_m<T, 0>(spec, a, st);
}

}  // namespace tr2
