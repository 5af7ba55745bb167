// FP64 instances of the fixed-size transform kernels.
#include "transform2_impl.cuh"

cudaError_t mf_v2_xyf_f64(const void* in, void* spec, const XYArgs& a, cudaStream_t st) {
  return tr2::xyf<double>(in, spec, a, st);
}
cudaError_t mf_v2_xyi_f64(int mode, const void* spec, void* out, double* partials, const XYArgs& a,
                          const Scalars* sc, cudaStream_t st) {
  return tr2::xyi<double>(mode, spec, out, partials, a, sc, st);
}
cudaError_t mf_v2_zp_f64(int mode, void* spec, const ZArgs& a, cudaStream_t st) {
  return tr2::zp<double>(mode, spec, a, st);
}
