// Comparison path: the projected operator y = G*(K : x) with cuFFT doing the
// transforms (3D real-to-complex over the nine components, G-hat-star in
// natural frequency order, 3D complex-to-real).  Used only to time and to
// cross-check the library's own transform kernels; the solver never uses it.
//
// Memory: the caller binds one buffer (mf_cufft_workspace_bytes) holding the
// natural-order half spectrum (9 x nz x ny x (nx/2+1) complex) and cuFFT's
// work area.  cuFFT keeps its own plan data.
#include <cufft.h>
#include <string.h>

#include "../../include/mixfft.h"
#include "launch.h"

namespace {

// G-hat-star (Eq. eq:Gnewnew) on the natural-order half spectrum, times scale.
template <typename C, typename T>
__global__ void k_gstar_natural(C* __restrict__ spec, int nx, int ny, int nz, unsigned mask, T scale) {
  const int hx = nx / 2 + 1;
  const long long nf = (long long)nz * ny * hx;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf;
       f += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(f % hx);
    const int ky = (int)((f / hx) % ny);
    const int kz = (int)(f / ((long long)hx * ny));
    C* e = spec + f;
    const bool nyq = (2 * kx == nx) || (2 * ky == ny) || ((nz % 2 == 0) && (2 * kz == nz));
    if (nyq) {
      for (int c = 0; c < 9; ++c) { e[c * nf].x = (T)0; e[c * nf].y = (T)0; }
    } else if (kx == 0 && ky == 0 && kz == 0) {
      for (int c = 0; c < 9; ++c) {
        if (mask & (1u << c)) { e[c * nf].x *= scale; e[c * nf].y *= scale; }
        else { e[c * nf].x = (T)0; e[c * nf].y = (T)0; }
      }
    } else {
      const int kys = (2 * ky < ny) ? ky : ky - ny;
      const int kzs = (2 * kz < nz) ? kz : kz - nz;
      const T xi0 = (T)kx / (T)nx, xi1 = (T)kys / (T)ny, xi2 = (T)kzs / (T)nz;
      const T inv = scale / (xi0 * xi0 + xi1 * xi1 + xi2 * xi2);
      for (int i = 0; i < 3; ++i) {
        const C A0 = e[(3 * i) * nf], A1 = e[(3 * i + 1) * nf], A2 = e[(3 * i + 2) * nf];
        const T qx = (A0.x * xi0 + A1.x * xi1 + A2.x * xi2) * inv;
        const T qy = (A0.y * xi0 + A1.y * xi1 + A2.y * xi2) * inv;
        e[(3 * i) * nf].x = qx * xi0; e[(3 * i) * nf].y = qy * xi0;
        e[(3 * i + 1) * nf].x = qx * xi1; e[(3 * i + 1) * nf].y = qy * xi1;
        e[(3 * i + 2) * nf].x = qx * xi2; e[(3 * i + 2) * nf].y = qy * xi2;
      }
    }
  }
}

}  // namespace

struct MfCufft {
  cufftHandle fwd = 0, inv = 0;
  bool made = false;
  void* spec = nullptr;
  void* work = nullptr;
  size_t spec_bytes = 0, work_bytes = 0;
};

// Plans for one context (batch of nine 3D transforms); returns bytes needed.
int mf_cufft_plan(MfCufft* p, int nx, int ny, int nz, bool f32, cudaStream_t st, size_t* need) {
  if (!p->made) {
    int n[3] = {nz, ny, nx};
    const long long N = (long long)nx * ny * nz;
    const long long nf = (long long)nz * ny * (nx / 2 + 1);
    if (cufftCreate(&p->fwd) != CUFFT_SUCCESS || cufftCreate(&p->inv) != CUFFT_SUCCESS) return MF_CUDA_ERROR;
    cufftSetAutoAllocation(p->fwd, 0);
    cufftSetAutoAllocation(p->inv, 0);
    size_t wf = 0, wi = 0;
    const cufftType tf = f32 ? CUFFT_R2C : CUFFT_D2Z, ti = f32 ? CUFFT_C2R : CUFFT_Z2D;
    if (cufftMakePlanMany(p->fwd, 3, n, nullptr, 1, (int)N, nullptr, 1, (int)nf, tf, 9, &wf) != CUFFT_SUCCESS)
      return MF_CUDA_ERROR;
    if (cufftMakePlanMany(p->inv, 3, n, nullptr, 1, (int)nf, nullptr, 1, (int)N, ti, 9, &wi) != CUFFT_SUCCESS)
      return MF_CUDA_ERROR;
    cufftSetStream(p->fwd, st);
    cufftSetStream(p->inv, st);
    p->spec_bytes = ((size_t)9 * nf * (f32 ? sizeof(float2) : sizeof(double2)) + 255) & ~(size_t)255;
    p->work_bytes = ((wf > wi ? wf : wi) + 255) & ~(size_t)255;
    p->made = true;
  }
  *need = p->spec_bytes + p->work_bytes;
  return MF_OK;
}

int mf_cufft_bind(MfCufft* p, void* dev) {
  if (!p->made) return MF_INVALID_ARG;
  p->spec = dev;
  p->work = (char*)dev + p->spec_bytes;
  if (cufftSetWorkArea(p->fwd, p->work) != CUFFT_SUCCESS || cufftSetWorkArea(p->inv, p->work) != CUFFT_SUCCESS)
    return MF_CUDA_ERROR;
  return MF_OK;
}

// which: -1 all three parts; 0 forward transform, 1 G-hat-star, 2 inverse.
int mf_cufft_project(MfCufft* p, bool f32, const void* t, void* y, int nx, int ny, int nz, const uint8_t* mask,
                     cudaStream_t st, int which) {
  unsigned m = 0;
  for (int c = 0; c < 9; ++c)
    if (mask[c]) m |= 1u << c;
  const long long N = (long long)nx * ny * nz;
  const long long nf = (long long)nz * ny * (nx / 2 + 1);
  cufftResult r = CUFFT_SUCCESS;
  if (which < 0 || which == 0) {
    r = f32 ? cufftExecR2C(p->fwd, (cufftReal*)t, (cufftComplex*)p->spec)
            : cufftExecD2Z(p->fwd, (cufftDoubleReal*)t, (cufftDoubleComplex*)p->spec);
    if (r != CUFFT_SUCCESS) return MF_CUDA_ERROR;
  }
  if (which < 0 || which == 1) {
    const int blocks = 152 * 4;
    if (f32) k_gstar_natural<float2, float><<<blocks, 256, 0, st>>>((float2*)p->spec, nx, ny, nz, m, 1.0f / (float)N);
    else k_gstar_natural<double2, double><<<blocks, 256, 0, st>>>((double2*)p->spec, nx, ny, nz, m, 1.0 / (double)N);
    ++g_mf_launches;
    if (cudaGetLastError() != cudaSuccess) return MF_CUDA_ERROR;
  }
  if (which < 0 || which == 2) {
    r = f32 ? cufftExecC2R(p->inv, (cufftComplex*)p->spec, (cufftReal*)y)
            : cufftExecZ2D(p->inv, (cufftDoubleComplex*)p->spec, (cufftDoubleReal*)y);
    if (r != CUFFT_SUCCESS) return MF_CUDA_ERROR;
  }
  (void)nf;
  return MF_OK;
}

MfCufft* mf_cufft_new() { return new MfCufft(); }
void mf_cufft_delete(MfCufft* p) {
  if (p) { mf_cufft_destroy(p); delete p; }
}

void mf_cufft_destroy(MfCufft* p) {
  if (p->made) {
    cufftDestroy(p->fwd);
    cufftDestroy(p->inv);
  }
  p->made = false;
}
