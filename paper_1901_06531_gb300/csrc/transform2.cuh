// Fixed-size transform kernels (square x-y planes NX = NY, z length NZ, both
// compile-time) for the projected operator and the residual.
//
// Real-to-complex along x by the half-length method: a real row of NX values
// is read as H = NX/2 complex samples z_j = t_2j + i t_2j+1, transformed at
// length H, and split into the NX-point spectrum by
//     X_k = E_k + W_NX^k O_k,  E_k = (Z_k + conj Z_(H-k)) / 2,
//     O_k = (Z_k - conj Z_(H-k)) / 2i,            k = 0 .. H-1
// (the x-Nyquist coefficient is not kept: G-hat-star is zero there).  Rows
// therefore load and store contiguously.  The complex y transform follows on
// the H columns; the z-pass transforms along z, applies G-hat-star and
// transforms back.  Spectrum per (c, z): NY rows (digit-reversed ky) of H
// slots (digit-reversed kx), dense.
#pragma once

#include <type_traits>

#include "bulk.cuh"
#include "dw.cuh"
#include "fft2.cuh"
#include "launch.h"

namespace tr2 {

// Type of the real fields a kernel reads or writes in global memory: the
// compute type itself, except for the double-word kernels, which read P and
// write the residual in FP64 and hold the spectrum as double-word complex
// (16 bytes, the size of an FP64 complex).
template <typename T> struct IOT { typedef T t; };
template <> struct IOT<dw> { typedef double t; };

__device__ __forceinline__ void io_in(float2& d, float2 s) { d = s; }
__device__ __forceinline__ void io_in(double2& d, double2 s) { d = s; }
__device__ __forceinline__ void io_in(dwc& d, double2 s) { d = to_dwc(s); }
__device__ __forceinline__ float2 io_out(float2 v) { return v; }
__device__ __forceinline__ double2 io_out(double2 v) { return v; }
__device__ __forceinline__ double2 io_out(dwc v) { return to_double2(v); }

constexpr int kThreads = 256;
// x-y kernels: 16-byte elements (FP64, double word) hold one 128 x 128 plane
// in 133 KB of shared memory, one block per SM, so they run twice the
// threads; FP32 128 x 128 planes (66 KB) run two blocks of 512 threads per
// SM at 64 registers a thread (about 1% faster than three blocks of 256 on
// the GB300), other FP32 planes blocks of 256
constexpr int kXY128Threads = 512;
template <typename T, int NX> __host__ __device__ constexpr int xy_threads() {
  return sizeof(typename CT<T>::t) == 16 ? 512 : (NX == 128 ? kXY128Threads : 256);
}
// resident blocks per SM the register allocation of an FP32 128 x 128 x-y
// kernel is held to when it runs 512 threads: two (64 registers a thread)
template <typename T, int NX> __host__ __device__ constexpr int xy_min_blocks() {
  return (sizeof(typename CT<T>::t) == 8 && NX == 128 && kXY128Threads == 512) ? 2 : 1;
}
// z-pass threads per block for a tile of S columns of one row group (three
// components): 24 S, one butterfly per thread in a radix-16 stage of the
// 128-point transform and two in its radix-8 stage (3 x S x 128/R)
__host__ __device__ constexpr int z_threads(int S) { return 24 * S; }
// resident z-pass blocks per SM the register allocation is held to: five
// blocks of 192 threads for the FP32 operator pass (S = 8, MODE 0), else what
// the compiler chooses
template <typename T> __host__ __device__ constexpr int z_min_blocks(int S, int mode) {
  return (sizeof(typename CT<T>::t) == 8 && S == 8 && mode == 0) ? 5 : 1;
}

// Asynchronous global -> shared copies of one complex element (8 or 16
// bytes); many in flight per thread without holding registers.
template <typename C>
__device__ __forceinline__ void cp_async_elem(C* smem, const C* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(C) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T, int NX>
struct XYShape {
  typedef typename CT<T>::t C;
  static constexpr int H = NX / 2;
  static constexpr int PX = H + 1;            // odd pitch: rows fall in different banks
  static constexpr int NY = NX;
  // tables after the plane: twx (NX), twy (NY), tw0 (64, see x_stage0_128), posx (H ints)
  static constexpr size_t smem() {
    return (size_t)NY * PX * sizeof(C) + (size_t)(NX + NY + 64) * sizeof(C) + (size_t)H * sizeof(int);
  }
};

template <typename C>
__device__ __forceinline__ void load_tables(C* twx, C* twy, int* posx, const C* gtw, const int* gpos,
                                            int nx, int ny, int h, C* tw0 = nullptr) {
  for (int i = threadIdx.x; i < nx; i += blockDim.x) twx[i] = gtw[i];
  for (int i = threadIdx.x; i < ny; i += blockDim.x) twy[i] = gtw[nx + i];
  for (int i = threadIdx.x; i < h; i += blockDim.x) posx[i] = gpos[i];
  if (tw0)   // tw0[8k + b] = W_64^(b k) = W_128^(2 b k) (nx = 128)
    for (int i = threadIdx.x; i < 64; i += blockDim.x) tw0[i] = gtw[2 * (i & 7) * (i >> 3)];
}

// First x stage of an FP32 128 x 128 plane (half-length transform of 64
// points: radix 8, M = 8, eight butterflies per row; forward DIF, or with
// INV its adjoint as the last inverse stage), TPB threads (a multiple of
// 256).  Lanes are (row, butterfly b) with the four rows of a warp 8 apart
// (row (w mod 8) + 8i + 32 (w / 8) + pass offset): with the row pitch PX =
// 65 (1 mod 16) rows 8 apart start 8 elements apart modulo the 16
// eight-byte bank pairs, so each half-warp's 16 accesses of positions b + 8k
// (two rows of 8 consecutive) hit distinct banks; the twiddles W_64^(bk) come
// from the [k][b] table tw0 for the same reason.  ld(row, pos) gives an
// input, st(row, pos, value) takes an output.
template <bool INV, int TPB, typename LD, typename ST>
__device__ __forceinline__ void x_stage0_128(const float2* tw0, LD ld, ST st) {
  typedef float2 C;
  static_assert(TPB % 256 == 0 && TPB <= 1024, "whole groups of eight warps");
  constexpr int kRowsPerPass = TPB / 8;   // eight lanes per row
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, b = l & 7, i = l >> 3;
  const int row0 = (w & 7) + 8 * i + 32 * (w >> 3);
#pragma unroll 1
  for (int P = 0; P < 128 / kRowsPerPass; ++P) {
    const int row = kRowsPerPass * P + row0;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = ld(row, b + 8 * r);
    if (!INV) {
      fft2::Dft<8, false, C>::run(v);
#pragma unroll
      for (int k = 1; k < 8; ++k) v[k] = cmul(v[k], tw0[8 * k + b]);
    } else {
#pragma unroll
      for (int k = 1; k < 8; ++k) v[k] = cmulc(v[k], tw0[8 * k + b]);
      fft2::Dft<8, true, C>::run(v);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) st(row, b + 8 * k, v[k]);
  }
}

// ------------------------------------------------------------- row spectra
// The half-length x transform (H = NX/2 points) has one or two stages.  Its
// last stage (radix RB, no twiddles: its M is 1) has RA = H/RB butterflies
// per row; butterfly b holds the positions b*RB + r, i.e. the frequencies
// k = b + RA r.  The partner H - k of (b, r) is (RA - b, RB - 1 - r) for
// b != 0 and (0, (RB - r) % RB) for b = 0.  A task takes butterflies b and
// RA - b of one row, so both members of every pair of the split (forward) or
// merge (inverse) are in its registers, and that step is fused with the last
// forward (first inverse) stage.
template <int H> struct RowPlan {
  static constexpr int NST = fft2::nst(H);
  static constexpr int RB = fft2::rad(H, NST - 1);
  static constexpr int RA = H / RB;
  static constexpr int NT = RA / 2 + 1;   // tasks per row
};

// X_k = E_k + W_NX^k O_k, E_k = (Z_k + conj Z_(H-k)) / 2, O_k = (Z_k - conj Z_(H-k)) / 2i
template <typename T, typename C>
__device__ __forceinline__ C split_one(C za, C zb, C w) {
  C e, o;
  e.x = (T)0.5 * (za.x + zb.x); e.y = (T)0.5 * (za.y - zb.y);
  o.x = (T)0.5 * (za.y + zb.y); o.y = (T)-0.5 * (za.x - zb.x);
  return cadd(e, cmul(o, w));
}

// Z_k = E_k + i O_k, E_k = X_k + conj X_(H-k), O_k = (X_k - conj X_(H-k)) conj(W_NX^k)
// (the adjoint of the split, times 2)
template <typename T, typename C>
__device__ __forceinline__ C merge_one(C xa, C xb, C w) {
  C e, d;
  e.x = xa.x + xb.x; e.y = xa.y - xb.y;
  d.x = xa.x - xb.x; d.y = xa.y + xb.y;
  const C o = cmulc(d, w);
  C z;
  z.x = e.x - o.y; z.y = e.y + o.x;
  return z;
}

// Last x stage + split.  ld(y, pos): input at position pos of row y; the
// outputs go to buf (row pitch PX).
template <typename T, int NX, int TPB, typename LD>
__device__ __forceinline__ void x_last_split(typename CT<T>::t* buf, const typename CT<T>::t* twx, LD ld) {
  typedef typename CT<T>::t C;
  typedef RowPlan<NX / 2> RP;
  constexpr int RA = RP::RA, RB = RP::RB, PX = NX / 2 + 1, NY = NX;
  for (int task = threadIdx.x; task < NY * RP::NT; task += TPB) {
    const int y = task % NY, t = task / NY;
    const int b0 = t, b1 = (t == 0) ? 0 : RA - t;
    C u[RB], w[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) u[r] = ld(y, b0 * RB + r);
    fft2::Dft<RB, false, C>::run(u);
    C* row = buf + y * PX;
    if (b1 != b0) {
#pragma unroll
      for (int r = 0; r < RB; ++r) w[r] = ld(y, b1 * RB + r);
      fft2::Dft<RB, false, C>::run(w);
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int rp = RB - 1 - r;
        const int k = b0 + RA * r, km = b1 + RA * rp;
        row[MF_AT(b0 * RB + r, NX / 2)] = split_one<T>(u[r], w[rp], twx[k]);
        row[MF_AT(b1 * RB + rp, NX / 2)] = split_one<T>(w[rp], u[r], twx[km]);
      }
    } else {
      // b0 = b1 (b0 = 0 or RA/2): the pairs lie within u; the partner index
      // is a compile-time function of r in each case, so u stays in registers
      auto pair = [&](int r, int rp) {
        const int k = b0 + RA * r, km = b0 + RA * rp;
        const C za = u[r], zb = u[rp];
        row[b0 * RB + r] = split_one<T>(za, zb, twx[k]);
        if (rp != r) row[b0 * RB + rp] = split_one<T>(zb, za, twx[km]);
      };
      if (b0 == 0) {
#pragma unroll
        for (int r = 0; r < RB; ++r)
          if ((RB - r) % RB >= r) pair(r, (RB - r) % RB);
      } else {
#pragma unroll
        for (int r = 0; r < RB; ++r)
          if (RB - 1 - r >= r) pair(r, RB - 1 - r);
      }
    }
  }
}

// Merge + first inverse x stage (in place in buf).  The x-constant
// coefficient keeps only its real part and X_H (Nyquist) is zero, so
// Z_0 = x0 + i x0 with x0 = Re X_0.
template <typename T, int NX, int TPB>
__device__ __forceinline__ void x_merge_first(typename CT<T>::t* buf, const typename CT<T>::t* twx) {
  typedef typename CT<T>::t C;
  typedef RowPlan<NX / 2> RP;
  constexpr int RA = RP::RA, RB = RP::RB, PX = NX / 2 + 1, NY = NX;
  for (int task = threadIdx.x; task < NY * RP::NT; task += TPB) {
    const int y = task % NY, t = task / NY;
    const int b0 = t, b1 = (t == 0) ? 0 : RA - t;
    C* row = buf + y * PX;
    C u[RB], w[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) u[r] = row[b0 * RB + r];
    if (b1 != b0) {
#pragma unroll
      for (int r = 0; r < RB; ++r) w[r] = row[b1 * RB + r];
      C zu[RB], zw[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int rp = RB - 1 - r;
        const int k = b0 + RA * r, km = b1 + RA * rp;
        zu[r] = merge_one<T>(u[r], w[rp], twx[k]);
        zw[rp] = merge_one<T>(w[rp], u[r], twx[km]);
      }
      fft2::Dft<RB, true, C>::run(zu);
      fft2::Dft<RB, true, C>::run(zw);
#pragma unroll
      for (int r = 0; r < RB; ++r) { row[b0 * RB + r] = zu[r]; row[b1 * RB + r] = zw[r]; }
    } else {
      // b0 = b1 (b0 = 0 or RA/2): partner indices fixed at compile time per case
      C zu[RB];
      if (b0 == 0) {
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          if (r == 0) {
            const T x0 = u[0].x;
            zu[0].x = x0; zu[0].y = x0;
          } else {
            zu[r] = merge_one<T>(u[r], u[(RB - r) % RB], twx[RA * r]);
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < RB; ++r) zu[r] = merge_one<T>(u[r], u[RB - 1 - r], twx[b0 + RA * r]);
      }
      fft2::Dft<RB, true, C>::run(zu);
#pragma unroll
      for (int r = 0; r < RB; ++r) row[b0 * RB + r] = zu[r];
    }
  }
}

// ------------------------------------------------------------------ forward
template <typename T, int NX>
__global__ void __launch_bounds__(xy_threads<T, NX>(), xy_min_blocks<T, NX>()) k_xyf(const typename IOT<T>::t* __restrict__ in,
                                                  typename CT<T>::t* __restrict__ spec, int nz, long long N,
                                                  const typename CT<T>::t* __restrict__ gtw,
                                                  const int* __restrict__ gpos, const int* skip) {
  typedef XYShape<T, NX> Sh;
  constexpr int TPB = xy_threads<T, NX>();
  typedef typename CT<T>::t C;
  typedef typename CT<typename IOT<T>::t>::t CI;
  constexpr int H = Sh::H, PX = Sh::PX, NY = Sh::NY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* twx = buf + NY * PX;
  C* twy = twx + NX;
  C* tw0 = twy + NY;
  int* posx = reinterpret_cast<int*>(tw0 + 64);
  // constant: loaded before the wait for the predecessor
  load_tables(twx, twy, posx, gtw, gpos, NX, NY, H, (sizeof(C) == 8 && NX == 128) ? tw0 : nullptr);
  pdl_wait();
  if (skip && *(volatile const int*)skip) return;
  const int c = blockIdx.x % 9, z = blockIdx.x / 9;
  const CI* src = reinterpret_cast<const CI*>(in + c * N + (long long)z * NY * NX);
  // row y, sample j (the real values 2j, 2j+1 as one complex sample)
  auto gload = [&](int y, int j) {
    C v;
    io_in(v, src[MF_AT((long long)y * H + j, NY * H)]);
    return v;
  };
  if constexpr (sizeof(C) == 8) {
    // FP32: the x transform touches shared memory twice per sample
    __syncthreads();   // tables
    if constexpr (RowPlan<H>::NST == 2) {
      // first x stage straight from global memory (consecutive threads take
      // consecutive butterflies of a row: 64-byte row segments per warp access)
      if constexpr (NX == 128)
        x_stage0_128<false, TPB>(tw0, gload, [&](int q, int e, C v) { buf[MF_AT(q * PX + e, NY * PX)] = v; });
      else
        fft2::stage_io<C, H, NX, 0, false, NY, 1, PX, 0, 1, false>(
            twx, [&](int q, int, int e) { return gload(q, e); },
            [&](int, int i, int, C v) { buf[MF_AT(i, NY * PX)] = v; });
      __syncthreads();
      x_last_split<T, NX, TPB>(buf, twx, [&](int y, int pos) { return buf[MF_AT(y * PX + pos, NY * PX)]; });
    } else {
      x_last_split<T, NX, TPB>(buf, twx, gload);
    }
  } else {
    // 16-byte types (FP64, double word) are arithmetic bound: the plane is
    // copied in asynchronously (and converted in place), then the stages and
    // the split run over shared memory
    for (int idx = threadIdx.x; idx < NY * H; idx += TPB) {
      const int y = idx / H, j = idx - (idx / H) * H;
      cp_async_elem(reinterpret_cast<CI*>(buf + y * PX + j), src + idx);
    }
    cp_async_wait_all();
    if constexpr (!std::is_same<C, CI>::value) {
      for (int idx = threadIdx.x; idx < NY * H; idx += TPB) {   // each thread converts its own copies
        const int y = idx / H, j = idx - (idx / H) * H;
        const CI v = *reinterpret_cast<const CI*>(buf + y * PX + j);
        io_in(buf[y * PX + j], v);
      }
    }
    __syncthreads();
    fft2::forward<C, H, NX, NY, 1, PX, 0, 1>(buf, twx);
    constexpr int NP = H / 2 + 1;
    for (int idx = threadIdx.x; idx < NY * NP; idx += TPB) {
      const int y = idx % NY, k = idx / NY;
      const int km = (H - k) % H;
      C* row = buf + y * PX;
      const int pa = posx[k], pb = posx[km];
      const C za = row[pa], zb = row[pb];
      if (km != k) row[pb] = split_one<T>(zb, za, twx[km]);
      row[pa] = split_one<T>(za, zb, twx[k]);
    }
  }
  __syncthreads();
  // y: H columns of NY samples, stride PX; the last stage stores the
  // spectrum rows (consecutive threads take consecutive columns)
  C* dst = spec + ((long long)c * nz + z) * NY * H;
  fft2::forward_out<C, NY, NY, H, 1, 1, 0, PX>(buf, twy, [&](int q, int e, C v) { dst[MF_AT(e * H + q, NY * H)] = v; });
}

// ------------------------------------------------------- persistent forward
// The same x-y forward pass (FP32, planes whose half-length x transform has
// two stages: NX in {48, 64, 96, 128}) as a persistent kernel: one block of
// kPersistThreads per SM walks the (c, z) planes; each plane (NY x NX
// contiguous reals) arrives by one bulk copy in one of two staging buffers,
// so the copy of the block's plane i + 2 runs while plane i is transformed.
// Results are identical to k_xyf's (same stages, same order).
constexpr int kPersistThreads = 512;
constexpr int kMaxPolls = 1 << 22;   // bound of every barrier wait

template <int NX> struct PersistShape {
  typedef XYShape<float, NX> Sh;
  static constexpr int PLANE = Sh::NY * Sh::H;   // complex samples of one plane
  static constexpr size_t smem() { return (size_t)2 * PLANE * sizeof(float2) + Sh::smem(); }
};

template <int NX>
__global__ void __launch_bounds__(kPersistThreads, 1)
    k_xyf_p(const float* __restrict__ in, float2* __restrict__ spec, int nz, long long N,
            const float2* __restrict__ gtw, const int* __restrict__ gpos, const int* skip, int* flags) {
  typedef float2 C;
  typedef XYShape<float, NX> Sh;
  constexpr int H = Sh::H, PX = Sh::PX, NY = Sh::NY, TPB = kPersistThreads;
  constexpr int PLANE = PersistShape<NX>::PLANE;
  constexpr unsigned PBYTES = PLANE * sizeof(C);
  static_assert(RowPlan<H>::NST == 2, "first x stage reads the staging buffer");
  static_assert(PBYTES % 128 == 0, "staging buffers stay 128-byte aligned");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* stg = reinterpret_cast<C*>(smem_raw);   // [2][PLANE]
  C* buf = stg + 2 * PLANE;
  C* twx = buf + NY * PX;
  C* twy = twx + NX;
  int* posx = reinterpret_cast<int*>(twy + NY + 64);
  __shared__ __align__(8) uint64_t bar[2];
  const int nplanes = 9 * nz;
  if (threadIdx.x == 0) {
    bulk::init(&bar[0], 1);
    bulk::init(&bar[1], 1);
    bulk::fence_init();
  }
  load_tables(twx, twy, posx, gtw, gpos, NX, NY, H);   // constant: loaded before the wait for the predecessor
  pdl_wait();
  __syncthreads();
  if (skip && *(volatile const int*)skip) return;
  auto plane = [&](int p) { return in + (p % 9) * N + (long long)(p / 9) * NY * NX; };
  if (threadIdx.x == 0) {
    for (int k = 0; k < 2; ++k) {
      const int p = blockIdx.x + k * gridDim.x;
      if (p < nplanes) {
        bulk::expect_tx(&bar[k], PBYTES);
        bulk::g2s(stg + k * PLANE, plane(p), PBYTES, &bar[k]);
      }
    }
  }
  int i = 0;
  for (int p = blockIdx.x; p < nplanes; p += gridDim.x, ++i) {
    const int s = i & 1;
    const bool ok = bulk::wait(&bar[s], (unsigned)(i >> 1) & 1u, kMaxPolls);
    if (__syncthreads_or(!ok)) {
      // give up: record the timeout, let the copies in flight land, exit
      if (threadIdx.x == 0) {
        if (flags) atomicOr(flags, MF_FLAG_TIMEOUT);
        bulk::wait(&bar[s], (unsigned)(i >> 1) & 1u, kMaxPolls);
        if (p + gridDim.x < nplanes) bulk::wait(&bar[s ^ 1], (unsigned)((i + 1) >> 1) & 1u, kMaxPolls);
      }
      return;
    }
    const C* st = stg + s * PLANE;
    // first x stage: staging -> working buffer (consecutive threads take
    // consecutive butterflies of a row)
    fft2::stage_io<C, H, NX, 0, false, NY, 1, PX, 0, 1, false>(
        twx, [&](int q, int, int e) { return st[q * H + e]; }, [&](int, int i2, int, C v) { buf[i2] = v; });
    __syncthreads();
    if (threadIdx.x == 0) {   // refill the staging buffer just read with the plane after next
      const int pn = p + 2 * gridDim.x;
      if (pn < nplanes) {
        bulk::fence_proxy_async();
        bulk::expect_tx(&bar[s], PBYTES);
        bulk::g2s(stg + s * PLANE, plane(pn), PBYTES, &bar[s]);
      }
    }
    x_last_split<float, NX, TPB>(buf, twx, [&](int y, int pos) { return buf[y * PX + pos]; });
    __syncthreads();
    C* dst = spec + ((long long)(p % 9) * nz + p / 9) * NY * H;
    fft2::forward_out<C, NY, NY, H, 1, 1, 0, PX>(buf, twy, [&](int q, int e, C v) { dst[e * H + q] = v; });
    __syncthreads();   // the working buffer is refilled by the next plane
  }
}

// ------------------------------------------------------------------ inverse
// MODE 0: out[c] = y.  MODE 2: out[c] = y, partial sum y^2.  MODE 3: out[c] -=
// alpha y (alpha from sc), partial sum out^2; with fin the last block to
// finish also sums the partials and updates beta, r.r and the stop flag (the
// work of k_fin_beta, without its launch).
template <typename T, int NX, int MODE>
__global__ void __launch_bounds__(xy_threads<T, NX>(), xy_min_blocks<T, NX>()) k_xyi(const typename CT<T>::t* __restrict__ spec,
                                                  typename IOT<T>::t* __restrict__ out,
                                                  double* __restrict__ partials, int nz, long long N,
                                                  const typename CT<T>::t* __restrict__ gtw,
                                                  const int* __restrict__ gpos, Scalars* sc,
                                                  const int* skip, int fin) {
  typedef XYShape<T, NX> Sh;
  constexpr int TPB = xy_threads<T, NX>();
  typedef typename CT<T>::t C;
  typedef typename IOT<T>::t TI;
  typedef typename CT<TI>::t CI;
  static_assert(MODE != 3 || std::is_same<C, CI>::value, "the CG update runs in the compute type");
  constexpr int H = Sh::H, PX = Sh::PX, NY = Sh::NY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* twx = buf + NY * PX;
  C* twy = twx + NX;
  C* tw0 = twy + NY;
  int* posx = reinterpret_cast<int*>(tw0 + 64);
  // constant: loaded before the wait for the predecessor
  load_tables(twx, twy, posx, gtw, gpos, NX, NY, H, (sizeof(C) == 8 && NX == 128) ? tw0 : nullptr);
  pdl_wait();
  if (skip && *(volatile const int*)skip) return;
  const int c = blockIdx.x % 9, z = blockIdx.x / 9;
  if (MODE == 3) {
    // the residual plane is read only at the end: start pulling it into L2 now
    const char* rp = reinterpret_cast<const char*>(out + c * N + (long long)z * NY * NX);
    constexpr int kLines = (NY * NX * (int)sizeof(T)) / 128;
    for (int i = threadIdx.x; i < kLines; i += TPB)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(rp + 128 * i));
  }
  const C* src = spec + ((long long)c * nz + z) * NY * H;
  __syncthreads();   // tables
  // y: the first inverse stage reads the spectrum rows from global memory
  fft2::inverse_in<C, NY, NY, H, 1, 1, 0, PX>(buf, twy, [&](int q, int e) { return src[MF_AT(e * H + q, NY * H)]; });
  if constexpr (sizeof(C) == 8) {
    // merge of each row's spectrum, fused with the first inverse x stage
    x_merge_first<T, NX, TPB>(buf, twx);
  } else {
    constexpr int NP = H / 2 + 1;
    for (int idx = threadIdx.x; idx < NY * NP; idx += TPB) {
      const int y = idx % NY, k = idx / NY;
      const int km = (H - k) % H;
      C* row = buf + y * PX;
      const int pa = posx[k], pb = posx[km];
      const C xa = row[pa], xb = row[pb];
      if (k == 0) {
        const T x0 = xa.x;
        C z0; z0.x = x0; z0.y = x0;
        row[pa] = z0;
        continue;
      }
      if (km != k) row[pb] = merge_one<T>(xb, xa, twx[km]);
      row[pa] = merge_one<T>(xa, xb, twx[k]);
    }
    __syncthreads();
    fft2::inverse<C, H, NX, NY, 1, PX, 0, 1>(buf, twx);
  }
  __syncthreads();
  CI* dst = reinterpret_cast<CI*>(out + c * N + (long long)z * NY * NX);
  // per-thread sums: FP64 for FP64 data; for FP32 data exact FP32 products
  // with Neumaier-compensated FP32 accumulation, combined in FP64 below
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
  // the output of sample (row y, j): y = G*(.) stored, or r -= alpha y
  auto emit = [&](long long idx, C v) {
    idx = MF_AT(idx, NY * H);
    if constexpr (MODE == 3) {
      C r = dst[idx];
      r.x -= alpha * v.x;
      r.y -= alpha * v.y;
      dst[idx] = r;
      if (sizeof(T) == 4) { fsq((float)r.x); fsq((float)r.y); }
      else acc += (double)r.x * (double)r.x + (double)r.y * (double)r.y;
    } else {
      const CI w = io_out(v);
      dst[idx] = w;
      if (MODE == 2) {
        if (sizeof(TI) == 4) { fsq((float)w.x); fsq((float)w.y); }
        else acc += (double)w.x * (double)w.x + (double)w.y * (double)w.y;
      }
    }
  };
  // The last inverse x stage writes global memory directly when the outputs
  // one butterfly step r covers (e = j0 + M0 r, M0 consecutive elements of a
  // row per step) fill whole 32-byte sectors.  Otherwise (H = 24, 48: M0 = 3)
  // the read-modify-write of r (MODE 3) would load sectors that the previous
  // step has just stored, and every load would wait for those stores; the
  // stage then runs in shared memory and a coalesced loop does the update.
  constexpr int M0 = H / fft2::rad(H, 0);
  constexpr bool kDirect = sizeof(C) == 8 && RowPlan<H>::NST == 2 && (MODE != 3 || (M0 * 8) % 32 == 0);
  if constexpr (kDirect && NX == 128) {
    x_stage0_128<true, TPB>(tw0, [&](int q, int e) { return buf[MF_AT(q * PX + e, NY * PX)]; },
                       [&](int q, int e, C v) { emit((long long)q * H + e, v); });
  } else if constexpr (kDirect) {
    // consecutive threads take consecutive butterflies of a row
    fft2::stage_io<C, H, NX, 0, true, NY, 1, PX, 0, 1, false>(
        twx, [&](int, int i, int) { return buf[MF_AT(i, NY * PX)]; },
        [&](int q, int, int e, C v) { emit((long long)q * H + e, v); });
  } else {
    if constexpr (sizeof(C) == 8 && RowPlan<H>::NST == 2) {
      fft2::stage<C, H, NX, 0, true, NY, 1, PX, 0, 1, false>(buf, twx);
      __syncthreads();
    }
#pragma unroll 8
    for (int idx = threadIdx.x; idx < NY * H; idx += TPB) {
      const int y = idx / H, j = idx - (idx / H) * H;
      emit(idx, buf[MF_AT(y * PX + j, NY * PX)]);
    }
  }
  if (sizeof(TI) == 4) acc = (double)fs + (double)fc;
  if (MODE >= 2) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double s = (threadIdx.x < (TPB >> 5)) ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) partials[blockIdx.x] = s;
    }
    if (MODE == 3 && fin) {
      double rr;
      if (last_block_total(partials, &sc->arrive, &rr) && threadIdx.x == 0) cg_finish_beta(rr, sc);
    }
  }
}

// ------------------------------------------------------------------ z-pass
// G-hat-star (Eq. eq:Gnewnew) mixes only the three components of one row i of
// the tensor (out_ij = (sum_l A_il xi_l / abs(xi)^2) xi_j), so a block takes
// one row group (components 3i, 3i+1, 3i+2) of S consecutive (ky, kx)
// columns.  The transform along z passes through shared memory only between
// stages: the first forward stage reads the spectrum from global memory, the
// last forward stage, G-hat-star and the first inverse stage run together in
// registers (a thread holds the three components of R positions of one
// column; the last DIF stage and the first DIT stage have no twiddles), and
// the last inverse stage writes global memory.  Element (component cl,
// position z, column s) lives at cl*CP + z*ZS + s; the paddings of ZS and CP
// were chosen with a wavefront model of these access patterns.
template <typename T, int NZ>
constexpr int z_default_S() { return 8; }

template <typename T, int NZ, int S_ = z_default_S<T, NZ>()>
struct ZShape {
  typedef typename CT<T>::t C;
  static constexpr int S = S_;
  static constexpr bool E8 = sizeof(C) == 8;
  static constexpr int ZS = S + ((E8 && S < 16) ? 1 : 0);
  static constexpr int CP = NZ * ZS + (E8 ? (S == 8 ? 1 : 0) : (S == 4 ? 4 : 0));
  // after the three components: twz (NZ), zk (NZ ints), xiz (NZ reals)
  static constexpr size_t smem() {
    return (size_t)3 * CP * sizeof(C) + (size_t)NZ * sizeof(C) + (size_t)NZ * sizeof(int) +
           (size_t)NZ * sizeof(typename std::conditional<sizeof(C) == 8, float, double>::type);
  }
};

// MODE 0: operator (scale, mask; with a.lin, the null-frequency coefficient
// / N times *a.lin_alpha added to a.lin, read before the transform).  MODE 1: residual (adds a.add at the
// null frequency, records the null-frequency coefficient / N in a.mean_out).
// Grid: 3 row groups x (ncol / S) column tiles.
template <typename T, int NZ, int MODE, int S_>
__global__ void __launch_bounds__(z_threads(S_), z_min_blocks<T>(S_, MODE)) k_zp(typename CT<T>::t* __restrict__ spec, ZArgs a) {
  typedef ZShape<T, NZ, S_> Sh;
  constexpr int kZThreads = z_threads(S_);
  typedef typename CT<T>::t C;
  constexpr int S = Sh::S, CP = Sh::CP, ZS = Sh::ZS;
  constexpr int NST = fft2::nst(NZ);
  constexpr int RL = fft2::rad(NZ, NST - 1);   // radix of the last DIF stage (its M is 1)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);   // [3][CP]
  C* twz = buf + 3 * CP;
  int* zk = reinterpret_cast<int*>(twz + NZ);
  // xi_z of each position (k_z / NZ, signed), NaN at the z-Nyquist frequency
  typedef typename std::conditional<sizeof(C) == 8, float, double>::type TX;
  TX* xiz = reinterpret_cast<TX*>(zk + NZ);
  const C* gtwz = reinterpret_cast<const C*>(a.twz);
  // constant tables: loaded before the wait for the predecessor
  for (int i = threadIdx.x; i < NZ; i += kZThreads) {
    twz[i] = gtwz[i];
    const int kz = a.zk[i];
    zk[i] = kz;
    const int kzs = (2 * kz < NZ) ? kz : kz - NZ;
    xiz[i] = ((NZ % 2 == 0) && (2 * kz == NZ)) ? (TX)NAN : (TX)kzs * ((TX)1 / (TX)NZ);
  }
  pdl_wait();
  if (a.skip && *(volatile const int*)a.skip) return;
  const int H = a.nx / 2;
  const int ncol = a.ny * H;
  const int ntile = ncol / S;
  const int g = blockIdx.x / ntile;                 // row group: components 3g .. 3g+2
  const int col0 = (blockIdx.x - g * ntile) * S;
  C* gsp = spec + (long long)(3 * g) * NZ * ncol + col0;
  // global element of (sequence q = cl*S + s, position z), relative to gsp
  // (the debug build checks it against the spectrum's 9 NZ ncol elements)
  const long long goff = (long long)(3 * g) * NZ * ncol + col0;
  auto gidx = [&](int q, int z) {
    return MF_AT(goff + ((long long)(q / S) * NZ + z) * ncol + (q % S), 9LL * NZ * ncol) - goff;
  };
  if (MODE == 0 && a.lin) {
    // the null-frequency coefficient of each component of the row group is
    // the sum over z of its planes' (kx, ky) = (0, 0) coefficients: read
    // here, before the transform overwrites them, by the block holding that
    // column (one warp per component, summed in FP64)
    int sdc = -1;
    for (int s = 0; s < S; ++s) {
      const int col = col0 + s, row = col / H, slot = col - row * H;
      if (a.xk[slot] == 0 && a.yk[row] == 0) sdc = s;
    }
    if (sdc >= 0 && threadIdx.x < 96) {
      const int cl = threadIdx.x >> 5, lane = threadIdx.x & 31;
      double sum = 0.0;
      for (int z = lane; z < NZ; z += 32) sum += (double)gsp[gidx(cl * S + sdc, z)].x;
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) a.lin[3 * g + cl] += *a.lin_alpha * (sum / (double)a.N);
    }
  }
  __syncthreads();
  if constexpr (NST > 1) {
    // first forward stage: global -> registers -> shared
    fft2::stage_io<C, NZ, NZ, 0, false, 3 * S, S, CP, 1, ZS, true>(
        twz, [&](int q, int, int z) { return gsp[gidx(q, z)]; }, [&](int, int i, int, C v) { buf[MF_AT(i, 3 * CP)] = v; });
    __syncthreads();
    if constexpr (NST > 2) {
      fft2::stage<C, NZ, NZ, 1, false, 3 * S, S, CP, 1, ZS, true>(buf, twz);
      __syncthreads();
    }
  }
  const T scale = (T)a.scale;
  // xi_a = k_a / n_a through reciprocals taken once (exact for powers of two,
  // within one rounding otherwise); 1 / abs(xi)^2 as a correctly rounded FP32
  // reciprocal in FP32, a division in the 16-byte types
  const T rnx = (T)1 / (T)a.nx, rny = (T)1 / (T)a.ny, rnz = (T)1 / (T)NZ;
  // G-hat-star on the three components (v0, v1, v2) at column s, position z
  auto gstar = [&](int s, int z, C& v0, C& v1, C& v2) {
    const int col = col0 + s;
    const int row = col / H, slot = col - (col / H) * H;
    const int kx = a.xk[slot];
    const int ky = a.yk[row];
    const int kz = zk[z];
    C* v[3] = {&v0, &v1, &v2};
    if ((2 * ky == a.ny) || ((NZ % 2 == 0) && (2 * kz == NZ))) {
#pragma unroll
      for (int cl = 0; cl < 3; ++cl) *v[cl] = cmake((T)0, (T)0);
    } else if (kx == 0 && ky == 0 && kz == 0) {
#pragma unroll
      for (int cl = 0; cl < 3; ++cl) {
        const int cc = 3 * g + cl;
        const C X = *v[cl];
        if (MODE == 1 && a.mean_out) a.mean_out[cc] = (double)X.x / (double)a.N;
        if (a.mask & (1u << cc)) {
          const T add = (MODE == 1) ? (T)(a.add_dev ? a.add_dev[cc] : a.add[cc]) : (T)0;
          *v[cl] = cmake(scale * X.x + add, scale * X.y);
        } else {
          *v[cl] = cmake((T)0, (T)0);
        }
      }
    } else {
      const int kys = (2 * ky < a.ny) ? ky : ky - a.ny;
      const int kzs = (2 * kz < NZ) ? kz : kz - NZ;
      const T xi0 = (T)kx * rnx, xi1 = (T)kys * rny, xi2 = (T)kzs * rnz;
      const T den = xi0 * xi0 + xi1 * xi1 + xi2 * xi2;
      T inv;
      if constexpr (sizeof(T) == 4) inv = scale * __frcp_rn(den);
      else inv = scale / den;
      C q;
      q.x = (v0.x * xi0 + v1.x * xi1 + v2.x * xi2) * inv;
      q.y = (v0.y * xi0 + v1.y * xi1 + v2.y * xi2) * inv;
      v0 = cmake(q.x * xi0, q.y * xi0);
      v1 = cmake(q.x * xi1, q.y * xi1);
      v2 = cmake(q.x * xi2, q.y * xi2);
    }
  };
  if constexpr (sizeof(C) == 8) {
    // FP32: last forward stage, G-hat-star and first inverse stage in
    // registers (three components of RL positions of one column per thread)
    constexpr int NB = NZ / RL;
    for (int t = threadIdx.x; t < S * NB; t += kZThreads) {
      const int s = t % S, blk = t / S;
      C v[3][RL];
#pragma unroll
      for (int cl = 0; cl < 3; ++cl)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int z = blk * RL + r;
          v[cl][r] = (NST > 1) ? buf[MF_AT(cl * CP + z * ZS + s, 3 * CP)] : gsp[gidx(cl * S + s, z)];
        }
#pragma unroll
      for (int cl = 0; cl < 3; ++cl) fft2::Dft<RL, false, C>::run(v[cl]);
#pragma unroll
      for (int r = 0; r < RL; ++r) gstar(s, blk * RL + r, v[0][r], v[1][r], v[2][r]);
#pragma unroll
      for (int cl = 0; cl < 3; ++cl) fft2::Dft<RL, true, C>::run(v[cl]);
#pragma unroll
      for (int cl = 0; cl < 3; ++cl)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int z = blk * RL + r;
          if (NST > 1) buf[MF_AT(cl * CP + z * ZS + s, 3 * CP)] = v[cl][r];
          else gsp[gidx(cl * S + s, z)] = v[cl][r];
        }
    }
  } else {
    // 16-byte types (FP64, double word): registers are scarcer, so the last
    // forward stage, G-hat-star and the first inverse stage are separate
    // passes over shared memory
    if constexpr (NST == 1) {
      for (int idx = threadIdx.x; idx < 3 * NZ * S; idx += kZThreads) {
        const int s2 = idx % S, cz = idx / S, cl = cz / NZ, z = cz - cl * NZ;
        buf[cl * CP + z * ZS + s2] = gsp[gidx(cl * S + s2, z)];
      }
      __syncthreads();
    }
    fft2::stage<C, NZ, NZ, NST - 1, false, 3 * S, S, CP, 1, ZS, true>(buf, twz);
    __syncthreads();
    for (int idx = threadIdx.x; idx < NZ * S; idx += kZThreads) {
      const int s2 = idx % S, z = idx / S;
      C* e = buf + z * ZS + s2;
      gstar(s2, z, e[0], e[CP], e[2 * CP]);
    }
    __syncthreads();
    fft2::stage<C, NZ, NZ, NST - 1, true, 3 * S, S, CP, 1, ZS, true>(buf, twz);
    if constexpr (NST == 1) {
      __syncthreads();
      for (int idx = threadIdx.x; idx < 3 * NZ * S; idx += kZThreads) {
        const int s2 = idx % S, cz = idx / S, cl = cz / NZ, z = cz - cl * NZ;
        gsp[gidx(cl * S + s2, z)] = buf[cl * CP + z * ZS + s2];
      }
    }
  }
  if constexpr (NST > 1) {
    __syncthreads();
    if constexpr (NST > 2) {
      fft2::stage<C, NZ, NZ, 1, true, 3 * S, S, CP, 1, ZS, true>(buf, twz);
      __syncthreads();
    }
    // last inverse stage: shared -> registers -> global
    fft2::stage_io<C, NZ, NZ, 0, true, 3 * S, S, CP, 1, ZS, true>(
        twz, [&](int, int i, int) { return buf[MF_AT(i, 3 * CP)]; }, [&](int q, int, int z, C v) { gsp[gidx(q, z)] = v; });
  }
}

}  // namespace tr2
