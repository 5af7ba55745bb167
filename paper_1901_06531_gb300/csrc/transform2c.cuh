// Cluster x-y kernels: FP32, 128 x 128 planes, one plane per cluster of two
// CTAs that exchange half of their rows through distributed shared memory.
//
// The y transform (length 128) starts with a radix-2 DIF stage: rows j and
// j + 64 become s_j = t_j + t_(j+64) and W_128^j d_j, d_j = t_j - t_(j+64),
// followed by one 64-point transform over the s rows and one over the d
// rows.  That stage only adds and subtracts whole rows and scales a row by a
// constant, so it commutes with the x transform and is applied to the real
// input rows: CTA h (h = 0, 1) reads the row pairs j in [32h, 32h + 32),
// transforms s_j and d_j along x (the half-length method of transform2.cuh)
// and stores row j of the s spectra in CTA 0, row j of the W_128^j d spectra
// in CTA 1.  After one cluster barrier each CTA holds a 64-point
// sub-transform (64 rows x 64 slots, 32 KB instead of the 66 KB of a whole
// plane) and finishes it with two radix-8 stages.  The inverse runs the same
// steps backwards (the adjoint): radix-8 stages on each CTA's sub-transform,
// a cluster barrier, and per row pair the inverse x transforms of s-row j
// and of conj(W_128^j) times d-row j (one of the two rows read from the
// other CTA), added and subtracted into rows j and j + 64.
//
// The 64-point x transforms run per warp, four row pairs per warp and eight
// lanes per row (lane b takes the radix-8 butterfly b of the first stage and
// the block of positions 8b .. 8b+7 of the second), with no block barrier:
// a warp passes its rows through its own 4-row shared scratch between the
// two stages, and the split of the half-length spectrum into the x spectrum
// pairs lane b with lane 8 - b of the same row through shuffles.  Shared
// rows are XOR-swizzled (swz) so that the three access patterns -- lanes
// over (row, butterfly), over (row, block) and over consecutive slots of one
// row -- are free of bank conflicts.
//
// The spectrum in global memory is the one the per-plane kernels write (y
// frequencies in the digit order of the 16 x 8 DIF): the y frequency k =
// h + 2 k_B + 16 k_C that this factorisation (2 x 8 x 8) leaves at
// sub-transform h, block k_B, position k_C is stored in row 8 (h + 2 k_B)
// + k_C.  The z-pass and the tables are therefore shared with the other
// x-y kernels; results agree with theirs to rounding (other twiddle
// products, other summation order).
#pragma once

#include "transform2.cuh"

namespace tr2 {
namespace clu {

constexpr int NX = 128, H = 64, HALF = 64;   // plane width, slots per row, rows per sub-transform
constexpr int kCThreads = 256;
constexpr int kWarps = kCThreads / 32;
constexpr int kScratchRows = 4;              // per warp
constexpr int kMain = HALF * H;              // elements of the sub-transform buffer
constexpr int kScratch = kWarps * kScratchRows * H;

__host__ __device__ constexpr size_t smem() {
  return (size_t)(kMain + kScratch + NX + 64) * sizeof(float2);
}

// shared index of (row y, slot p) in a swizzled buffer of 64-slot rows:
// bits 0-2 of the slot are XORed with bits 3-5, bit 3 with the row parity
__device__ __forceinline__ int swz(int y, int p) { return y * H + (p ^ ((p >> 3) & 7) ^ ((y & 1) << 3)); }

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// all threads of both CTAs: arrive (release: this thread's earlier memory
// accesses are performed first), then wait (acquire) for every arrival
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }
// the address in CTA `rank`'s shared memory of the variable at local address a
__device__ __forceinline__ unsigned map_rank(const void* a, unsigned rank) {
  unsigned d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"((unsigned)__cvta_generic_to_shared(a)), "r"(rank));
  return d;
}
__device__ __forceinline__ void st_remote(unsigned addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ float2 ld_remote(unsigned addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}

// twiddles: twx[t] = W_128^t from the context table; tw0[8k + b] = W_64^(b k)
// (the first x stage's, laid out so that lanes b hit distinct banks)
__device__ __forceinline__ void load_tables(float2* twx, float2* tw0, const float2* gtw) {
  for (int i = threadIdx.x; i < NX; i += kCThreads) twx[i] = gtw[i];
  for (int i = threadIdx.x; i < 64; i += kCThreads) tw0[i] = gtw[(2 * (i & 7) * (i >> 3)) & (NX - 1)];
}

// the partner's value for the split/merge of X_k, k = b + 8r, with X_(64-k):
// lane b' = (8 - b) % 8 holds it at index 7 - r, or (8 - r) % 8 when b = 0
// (then b' = 0 too); each lane sends what its partner needs
template <int R>
__device__ __forceinline__ float2 partner(const float2* u, int b, int pl) {
  const float2 snd = (b == 0) ? u[(8 - R) & 7] : u[7 - R];
  float2 w;
  w.x = __shfl_sync(0xffffffffu, snd.x, pl);
  w.y = __shfl_sync(0xffffffffu, snd.y, pl);
  return w;
}

}  // namespace clu

// ------------------------------------------------------------------ forward
// (a template only so that each translation unit that includes this header
// instantiates it where it is launched)
template <int NXC>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(clu::kCThreads, 4)
    k_xyf_c(const float* __restrict__ in, float2* __restrict__ spec, int nz, long long N,
            const float2* __restrict__ gtw, const int* skip) {
  using namespace clu;
  static_assert(NXC == NX, "128 x 128 planes");
  typedef float2 C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* mainb = reinterpret_cast<C*>(smem_raw);   // [64][64] this CTA's sub-transform
  C* scr = mainb + kMain;                      // [warp][4][64]
  C* twx = scr + kScratch;
  C* tw0 = twx + NX;
  load_tables(twx, tw0, gtw);   // constant: loaded before the wait for the predecessor
  pdl_wait();
  const bool sk = skip && *(volatile const int*)skip;   // the same flag, read by both CTAs
  // both CTAs have started (their shared memory may be written) and the
  // tables are visible to the block
  cluster_arrive();
  cluster_wait();
  if (sk) return;
  const unsigned h = cluster_rank();
  const int plane = blockIdx.x >> 1;
  const int c = plane % 9, z = plane / 9;
  const C* src = reinterpret_cast<const C*>(in + c * N + (long long)z * NX * NX);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = lane >> 3, b = lane & 7;
  const int j = 32 * (int)h + 4 * warp + p;   // row pair (j, j + 64)
  const int pl = (lane & ~7) | ((8 - b) & 7);
  C* ws = scr + warp * kScratchRows * H;
  const unsigned peer_main = map_rank(mainb, h ^ 1u);

  // first x stage (radix 8, M = 8) of s_j and d_j, read from the real rows
  C s[8], d[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const C a = src[MF_AT(j * H + b + 8 * r, NX * H)];
    const C e = src[MF_AT((j + 64) * H + b + 8 * r, NX * H)];
    s[r] = make_float2(a.x + e.x, a.y + e.y);
    d[r] = make_float2(a.x - e.x, a.y - e.y);
  }
  fft2::Dft<8, false, C>::run(s);
  fft2::Dft<8, false, C>::run(d);
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    const C w = tw0[k * 8 + b];
    s[k] = cmul(s[k], w);
    d[k] = cmul(d[k], w);
  }
  // second x stage (radix 8 over positions 8b .. 8b+7) and the split; the
  // row goes to sub-transform `dr` (0: s rows, 1: d rows times W_128^j)
  auto finish_row = [&](const C* v, unsigned dr) {
#pragma unroll
    for (int k = 0; k < 8; ++k) ws[MF_AT(swz(p, b + 8 * k), kScratchRows * H)] = v[k];
    __syncwarp();
    C u[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) u[r] = ws[MF_AT(swz(p, 8 * b + r), kScratchRows * H)];
    __syncwarp();   // the scratch rows are free again
    fft2::Dft<8, false, C>::run(u);   // Z_k, k = b + 8r
    const C wj = twx[j];
    C X[8];
    X[0] = split_one<float>(u[0], partner<0>(u, b, pl), twx[b]);
    X[1] = split_one<float>(u[1], partner<1>(u, b, pl), twx[b + 8]);
    X[2] = split_one<float>(u[2], partner<2>(u, b, pl), twx[b + 16]);
    X[3] = split_one<float>(u[3], partner<3>(u, b, pl), twx[b + 24]);
    X[4] = split_one<float>(u[4], partner<4>(u, b, pl), twx[b + 32]);
    X[5] = split_one<float>(u[5], partner<5>(u, b, pl), twx[b + 40]);
    X[6] = split_one<float>(u[6], partner<6>(u, b, pl), twx[b + 48]);
    X[7] = split_one<float>(u[7], partner<7>(u, b, pl), twx[b + 56]);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const C xv = dr ? cmul(X[r], wj) : X[r];
      const int i = MF_AT(swz(j, 8 * b + r), kMain);
      if (dr == h) mainb[i] = xv;
      else st_remote(peer_main + 8u * (unsigned)i, xv);
    }
  };
  finish_row(s, 0u);
  finish_row(d, 1u);
  // every row of both sub-transforms is in place
  cluster_arrive();
  cluster_wait();

  // y: radix-8 stage (M = 8) of the 64-point sub-transform, then the last
  // radix-8 stage, which stores the spectrum rows
  for (int t = threadIdx.x; t < 8 * H; t += kCThreads) {
    const int q = t & (H - 1), j0 = t >> 6;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = mainb[MF_AT(swz(j0 + 8 * r, q), kMain)];
    fft2::Dft<8, false, C>::run(v);
#pragma unroll
    for (int k = 1; k < 8; ++k) v[k] = cmul(v[k], twx[2 * j0 * k]);
#pragma unroll
    for (int k = 0; k < 8; ++k) mainb[MF_AT(swz(j0 + 8 * k, q), kMain)] = v[k];
  }
  __syncthreads();
  C* dst = spec + ((long long)c * nz + z) * NX * H;
  for (int t = threadIdx.x; t < 8 * H; t += kCThreads) {
    const int q = t & (H - 1), blk = t >> 6;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = mainb[MF_AT(swz(8 * blk + r, q), kMain)];
    fft2::Dft<8, false, C>::run(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) dst[MF_AT((8 * (int)h + 16 * blk + r) * H + q, NX * H)] = v[r];
  }
}

// ------------------------------------------------------------------ inverse
// MODE as k_xyi: 0 out = y; 2 out = y and partial sums of y^2; 3 out -=
// alpha y and partial sums of out^2, with fin the last block finishing beta.
template <int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(clu::kCThreads, 4)
    k_xyi_c(const float2* __restrict__ spec, float* __restrict__ out, double* __restrict__ partials, int nz,
            long long N, const float2* __restrict__ gtw, Scalars* sc, const int* skip, int fin) {
  using namespace clu;
  typedef float2 C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  C* mainb = reinterpret_cast<C*>(smem_raw);
  C* scr = mainb + kMain;
  C* twx = scr + kScratch;
  C* tw0 = twx + NX;
  load_tables(twx, tw0, gtw);   // constant: loaded before the wait for the predecessor
  pdl_wait();
  // the same flag, read by both CTAs: both return before any cluster barrier
  if (skip && *(volatile const int*)skip) return;
  const unsigned h = cluster_rank();
  const int plane = blockIdx.x >> 1;
  const int c = plane % 9, z = plane / 9;
  C* dst = reinterpret_cast<C*>(out + c * N + (long long)z * NX * NX);
  if (MODE == 3) {
    // the residual rows this CTA updates (j and j + 64, j in [32h, 32h + 32))
    // are read only at the end: start pulling them into L2 now
    const char* r0 = reinterpret_cast<const char*>(dst + 32 * h * H);
    const char* r1 = reinterpret_cast<const char*>(dst + (32 * h + 64) * H);
    constexpr int kLines = 32 * H * (int)sizeof(C) / 128;
    for (int i = threadIdx.x; i < kLines; i += kCThreads) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(r0 + 128 * i));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(r1 + 128 * i));
    }
  }
  __syncthreads();   // tables
  const C* src = spec + ((long long)c * nz + z) * NX * H;
  // y: the last forward stage inverted (reads the spectrum rows), then the
  // radix-8 stage with M = 8
  for (int t = threadIdx.x; t < 8 * H; t += kCThreads) {
    const int q = t & (H - 1), blk = t >> 6;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = src[MF_AT((8 * (int)h + 16 * blk + r) * H + q, NX * H)];
    fft2::Dft<8, true, C>::run(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) mainb[MF_AT(swz(8 * blk + r, q), kMain)] = v[r];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 8 * H; t += kCThreads) {
    const int q = t & (H - 1), j0 = t >> 6;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = mainb[MF_AT(swz(j0 + 8 * r, q), kMain)];
#pragma unroll
    for (int k = 1; k < 8; ++k) v[k] = cmulc(v[k], twx[2 * j0 * k]);
    fft2::Dft<8, true, C>::run(v);
#pragma unroll
    for (int k = 0; k < 8; ++k) mainb[MF_AT(swz(j0 + 8 * k, q), kMain)] = v[k];
  }
  // both sub-transforms are complete
  cluster_arrive();
  cluster_wait();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = lane >> 3, b = lane & 7;
  const int j = 32 * (int)h + 4 * warp + p;
  const int pl = (lane & ~7) | ((8 - b) & 7);
  C* ws = scr + warp * kScratchRows * H;
  const unsigned peer_main = map_rank(mainb, h ^ 1u);
  // inverse x transform of row j of sub-transform sr (1: times conj W_128^j):
  // merge with block 8 - b and the first inverse x stage (radix 8 over
  // positions 8b .. 8b+7), then the last one (radix 8, M = 8); res[k] is
  // the sample at position b + 8k
  auto x_row = [&](unsigned sr, C* res) {
    C u[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = MF_AT(swz(j, 8 * b + r), kMain);
      u[r] = (sr == h) ? mainb[i] : ld_remote(peer_main + 8u * (unsigned)i);
    }
    if (sr) {
      const C wj = twx[j];
#pragma unroll
      for (int r = 0; r < 8; ++r) u[r] = cmulc(u[r], wj);
    }
    C zu[8];
    zu[0] = merge_one<float>(u[0], partner<0>(u, b, pl), twx[b]);
    zu[1] = merge_one<float>(u[1], partner<1>(u, b, pl), twx[b + 8]);
    zu[2] = merge_one<float>(u[2], partner<2>(u, b, pl), twx[b + 16]);
    zu[3] = merge_one<float>(u[3], partner<3>(u, b, pl), twx[b + 24]);
    zu[4] = merge_one<float>(u[4], partner<4>(u, b, pl), twx[b + 32]);
    zu[5] = merge_one<float>(u[5], partner<5>(u, b, pl), twx[b + 40]);
    zu[6] = merge_one<float>(u[6], partner<6>(u, b, pl), twx[b + 48]);
    zu[7] = merge_one<float>(u[7], partner<7>(u, b, pl), twx[b + 56]);
    // the x-constant coefficient keeps only its real part (X_64 is zero)
    if (b == 0) zu[0] = make_float2(u[0].x, u[0].x);
    fft2::Dft<8, true, C>::run(zu);
#pragma unroll
    for (int r = 0; r < 8; ++r) ws[MF_AT(swz(p, 8 * b + r), kScratchRows * H)] = zu[r];
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 8; ++k) res[k] = ws[MF_AT(swz(p, b + 8 * k), kScratchRows * H)];
    __syncwarp();
#pragma unroll
    for (int k = 1; k < 8; ++k) res[k] = cmulc(res[k], tw0[k * 8 + b]);
    fft2::Dft<8, true, C>::run(res);
  };
  C sv[8], dv[8];
  x_row(0u, sv);
  x_row(1u, dv);
  // this CTA's reads of the other's shared memory are done
  cluster_arrive();

  double acc = 0.0;
  float fs = 0.f, fc = 0.f;
  auto fadd = [&](float v) {
    const float tt = fs + v;
    fc += (fabsf(fs) >= fabsf(v)) ? ((fs - tt) + v) : ((v - tt) + fs);
    fs = tt;
  };
  auto fsq = [&](float v) {
    const float pr = v * v;
    fadd(pr);
    fadd(fmaf(v, v, -pr));
  };
  float alpha = 0.f;
  if (MODE == 3) alpha = (float)sc->alpha;
  auto emit = [&](int idx, C v) {
    idx = MF_AT(idx, NX * H);
    if constexpr (MODE == 3) {
      C r = dst[idx];
      r.x -= alpha * v.x;
      r.y -= alpha * v.y;
      dst[idx] = r;
      fsq(r.x);
      fsq(r.y);
    } else {
      dst[idx] = v;
      if (MODE == 2) { fsq(v.x); fsq(v.y); }
    }
  };
  // rows j and j + 64: s + d and s - d
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    emit(j * H + b + 8 * k, make_float2(sv[k].x + dv[k].x, sv[k].y + dv[k].y));
    emit((j + 64) * H + b + 8 * k, make_float2(sv[k].x - dv[k].x, sv[k].y - dv[k].y));
  }
  // the other CTA no longer reads this one's shared memory
  cluster_wait();
  if (MODE >= 2) {
    acc = (double)fs + (double)fc;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double s2 = (threadIdx.x < kWarps) ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (threadIdx.x == 0) partials[blockIdx.x] = s2;
    }
    if (MODE == 3 && fin) {
      double rr;
      if (last_block_total(partials, &sc->arrive, &rr) && threadIdx.x == 0) cg_finish_beta(rr, sc);
    }
  }
}

}  // namespace tr2
