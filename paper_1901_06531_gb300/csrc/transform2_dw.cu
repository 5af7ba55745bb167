// Double-word instances of the fixed-size transform kernels: the FP64
// residual b = -G*(P - P-bar) of the FP32-inner mode, computed with
// double-word FP32 arithmetic (P read and b written in FP64).
#include "transform2_impl.cuh"

cudaError_t mf_v2_xyf_dw(const double* in, void* spec, const XYArgs& a, cudaStream_t st) {
  return tr2::xyf<dw>(in, spec, a, st);
}
cudaError_t mf_v2_zp_dw(void* spec, const ZArgs& a, cudaStream_t st) {
  return tr2::zp_m<dw, 1>(spec, a, st);
}
cudaError_t mf_v2_xyi_dw(const void* spec, double* out, double* partials, const XYArgs& a, cudaStream_t st) {
  return tr2::xyi_m<dw, 0>(spec, out, partials, a, nullptr, st);
}
