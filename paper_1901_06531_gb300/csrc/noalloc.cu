// Residual entry point that allocates nothing (mf_residual_noalloc).
//
// Some callers cannot allocate device memory at the point where they need the
// residual: code running inside a host callback or a custom allocator hook,
// a caller that has pinned its whole device memory budget up front, or an
// embedding runtime that forbids cudaMalloc after start-up.  This variant
// takes the stress field and the output field from the caller and keeps the
// only other memory the transforms need -- the half spectrum, the index and
// twiddle tables and the reduction partials -- in one file-scope static
// device array of fixed size.  Every GPU that loads the library holds that
// array (kNoallocScratchBytes) until the process exits.
#include <math.h>
#include <string.h>

#include <vector>

#include "../../include/mixfft.h"
#include "launch.h"

namespace {

constexpr long long kNoallocMaxVoxels = 64LL * 64 * 64;
constexpr size_t kSpecBytes = (size_t)9 * (kNoallocMaxVoxels / 2) * sizeof(double2);
constexpr size_t kTableBytes = 64 * 1024;
constexpr size_t kPartialBytes = (size_t)9 * 256 * sizeof(double);
constexpr size_t kMeanBytes = 256;
constexpr size_t kNoallocScratchBytes = kSpecBytes + kTableBytes + kPartialBytes + kMeanBytes;

}  // namespace

// The scratch array.  Host code must not use this name as an address: the
// device address comes from cudaGetSymbolAddress, on every call.
static __device__ __align__(256) unsigned char g_mf_noalloc_scratch[kNoallocScratchBytes];

namespace {

bool na_plan(int n, AxisPlan* p) {
  p->n = n;
  p->nst = 0;
  int m = n;
  while (m % 4 == 0) { p->rad[p->nst++] = 4; m /= 4; }
  if (m % 2 == 0) { p->rad[p->nst++] = 2; m /= 2; }
  while (m % 3 == 0) {
    if (p->nst >= MF_MAX_STAGES) return false;
    p->rad[p->nst++] = 3;
    m /= 3;
  }
  return m == 1 && p->nst <= MF_MAX_STAGES;
}

int na_pos(const AxisPlan& p, int k) {
  int pos = 0, L = p.n;
  for (int st = 0; st < p.nst; ++st) {
    const int r = p.rad[st], m = L / r;
    pos += m * (k % r);
    k /= r;
    L = m;
  }
  return pos;
}

bool na_smooth(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

}  // namespace

extern "C" int mf_residual_noalloc(int nx, int ny, int nz, const double* P_dev, const uint8_t* mask,
                                   const double* pbar, double* b_dev, double* meanP_host,
                                   void* stream) {
  if (!P_dev || !mask || !pbar || !b_dev || P_dev == (const double*)b_dev) return MF_INVALID_ARG;
  if (nx < 4 || ny < 4 || nz < 2 || nx > 256 || ny > 256 || nz > 256) return MF_INVALID_ARG;
  if ((nx & 1) || (ny & 1) || !na_smooth(nx) || !na_smooth(ny) || !na_smooth(nz)) return MF_INVALID_ARG;
  if ((size_t)(ny / 2) * nx * sizeof(double2) + (size_t)(nx + ny) * 20 > 200 * 1024) return MF_INVALID_ARG;
  const long long N = (long long)nx * ny * nz;
  if (N > kNoallocMaxVoxels) return MF_TOO_LARGE;
  for (int c = 0; c < 9; ++c)
    if (mask[c] > 1 || !isfinite(pbar[c])) return MF_INVALID_ARG;
  AxisPlan px, pyh, pz;
  if (!na_plan(nx, &px) || !na_plan(ny / 2, &pyh) || !na_plan(nz, &pz)) return MF_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;

  // the device address of the scratch array, looked up on every call (a
  // device or primary-context reset may reload the module elsewhere) with
  // the current device, so the stream must belong to it
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MF_CUDA_ERROR;
  if (st) {
    int sdev = -1;
    if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) return MF_CUDA_ERROR;
    if (sdev != dev) return MF_INVALID_ARG;
  }
  void* sym = nullptr;
  if (cudaGetSymbolAddress(&sym, g_mf_noalloc_scratch) != cudaSuccess || !sym) return MF_CUDA_ERROR;
  unsigned char* base = (unsigned char*)sym;
  void* spec = base;
  unsigned char* tab = base + kSpecBytes;
  double* partials = (double*)(base + kSpecBytes + kTableBytes);
  double* mean = (double*)(base + kSpecBytes + kTableBytes + kPartialBytes);

  // index maps and twiddles, rewritten every call (sizes may differ)
  std::vector<int> xpos(nx), xk(nx), xe(nx), yk(ny / 2), zk(nz);
  for (int k = 0; k < nx; ++k) xpos[k] = na_pos(px, k);
  for (int k = 0; k < nx; ++k) {
    const int s = xpos[k];
    if (k < nx / 2) { xk[s] = k; xe[s] = 0; }
    else if (k == nx / 2) { xk[s] = 0; xe[s] = 1; }
    else { xk[s] = nx - k; xe[s] = 1; }
  }
  for (int k = 0; k < ny / 2; ++k) yk[na_pos(pyh, k)] = k;
  for (int k = 0; k < nz; ++k) zk[na_pos(pz, k)] = k;
  std::vector<double2> tw(nx + ny + nz);
  int o = 0;
  for (int n : {nx, ny, nz}) {
    for (int t = 0; t < n; ++t) {
      const double ang = -2.0 * M_PI * (double)t / (double)n;
      tw[o + t] = make_double2(cos(ang), sin(ang));
    }
    o += n;
  }
  size_t off = 0;
  auto place = [&](size_t bytes) { size_t r = off; off += (bytes + 255) & ~(size_t)255; return r; };
  const size_t o_tw = place(tw.size() * sizeof(double2));
  const size_t o_xpos = place(nx * sizeof(int)), o_xk = place(nx * sizeof(int)),
               o_xe = place(nx * sizeof(int)), o_yk = place((ny / 2) * sizeof(int)),
               o_zk = place(nz * sizeof(int));
  if (off > kTableBytes) return MF_TOO_LARGE;
  cudaError_t e = cudaMemcpyAsync(tab + o_tw, tw.data(), tw.size() * sizeof(double2),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tab + o_xpos, xpos.data(), nx * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tab + o_xk, xk.data(), nx * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tab + o_xe, xe.data(), nx * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tab + o_yk, yk.data(), (ny / 2) * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tab + o_zk, zk.data(), nz * sizeof(int), cudaMemcpyHostToDevice, st);
  // nothing in the pipeline reads scratch before writing it; the mean slot is
  // cleared so that a failed launch cannot hand back the previous call's mean
  if (e == cudaSuccess) e = cudaMemsetAsync(mean, 0, kMeanBytes, st);
  if (e != cudaSuccess) return MF_CUDA_ERROR;

  XYArgs xa;
  memset(&xa, 0, sizeof(xa));   // persist, flags and the rest unused by the generic kernels: zero
  xa.v2 = 0;
  xa.split = 0;
  xa.skip = nullptr;
  xa.fin = 0;
  xa.pdl = 0;
  xa.nx = nx; xa.ny = ny; xa.nz = nz; xa.N = N;
  xa.px = px; xa.pyh = pyh;
  xa.twx = tab + o_tw;
  xa.twy = tab + o_tw + sizeof(double2) * nx;
  xa.xpos = (const int*)(tab + o_xpos);
  ZArgs za;
  memset(&za, 0, sizeof(za));
  za.nx = nx; za.ny = ny; za.nz = nz; za.N = N;
  za.pz = pz;
  za.twz = tab + o_tw + sizeof(double2) * (nx + ny);
  za.xk = (const int*)(tab + o_xk);
  za.xe = (const int*)(tab + o_xe);
  za.yk = (const int*)(tab + o_yk);
  za.zk = (const int*)(tab + o_zk);
  int S = 16;
  while (S > 1 && (size_t)9 * nz * S * sizeof(double2) > 150 * 1024) S /= 2;
  za.S = S;
  za.mask = 0;
  for (int c = 0; c < 9; ++c) {
    if (mask[c]) za.mask |= 1u << c;
    za.add[c] = mask[c] ? pbar[c] : 0.0;
  }
  za.scale = -1.0 / (double)N;
  za.mean_out = mean;
  e = mf_launch_residual(P_dev, spec, b_dev, partials, xa, za, false, st);
  if (e == cudaSuccess && meanP_host)
    e = cudaMemcpyAsync(meanP_host, mean, 9 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? MF_OK : MF_CUDA_ERROR;
}
