// FP32 instances of the fixed-size transform kernels.
#include "transform2_impl.cuh"

cudaError_t mf_v2_xyf_f32(const void* in, void* spec, const XYArgs& a, cudaStream_t st) {
  return tr2::xyf<float>(in, spec, a, st);
}
cudaError_t mf_v2_xyi_f32(int mode, const void* spec, void* out, double* partials, const XYArgs& a,
                          const Scalars* sc, cudaStream_t st) {
  return tr2::xyi<float>(mode, spec, out, partials, a, sc, st);
}
cudaError_t mf_v2_zp_f32(int mode, void* spec, const ZArgs& a, cudaStream_t st) {
  return tr2::zp<float>(mode, spec, a, st);
}

// Self-test of the bounded barrier wait the bulk-copy kernels use: one block
// waits on a barrier that nothing arrives at; after max_polls polls the wait
// gives up and the block records MF_FLAG_TIMEOUT in *flags, as a bulk-copy
// kernel whose copy never landed would.
namespace {
__global__ void k_wait_selftest(int max_polls, int* flags) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    bulk::init(&bar, 1);
    bulk::fence_init();
  }
  __syncthreads();
  const bool ok = bulk::wait(&bar, 0u, max_polls);   // phase 0 never completes
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(flags, MF_FLAG_TIMEOUT);
}
}  // namespace

cudaError_t mf_launch_wait_selftest(int max_polls, int* flags, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(max_polls, flags);
  ++g_mf_launches;
  return cudaGetLastError();
}
