// Compile-time FFT machinery for the fixed-size transform kernels.
//
// A transform of length N runs as a few in-place stages over shared memory.
// Each thread loads one radix-R butterfly (R up to 16) into registers, does
// the R-point DFT there, applies the stage twiddles and stores it back, so a
// length-128 transform takes two shared-memory passes (16 x 8) instead of
// four.  Every size, stride and index is a template constant, so the
// address arithmetic folds to shifts and multiplies.  As in common.cuh the
// forward transform is decimation in frequency (digit-reversed output) and
// the inverse is its adjoint (digit-reversed input).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace fft2 {

// Stage radices per length (DIF order).
__host__ __device__ constexpr int nst(int n) {
  return n == 2 || n == 3 || n == 4 || n == 8 || n == 16 ? 1
       : n == 6 || n == 12 || n == 24 || n == 32 || n == 48 || n == 64 || n == 128 || n == 256 ? 2
       : n == 96 || n == 192 ? 3 : 0;
}
__host__ __device__ constexpr int rad(int n, int s) {
  return n == 2 ? 2 : n == 3 ? 3 : n == 4 ? 4 : n == 8 ? 8 : n == 16 ? 16
       : n == 6 ? (s == 0 ? 2 : 3)
       : n == 12 ? (s == 0 ? 4 : 3)
       : n == 24 ? (s == 0 ? 8 : 3)
       : n == 32 ? (s == 0 ? 8 : 4)
       : n == 48 ? (s == 0 ? 16 : 3)
       : n == 64 ? 8
       : n == 96 ? (s == 0 ? 8 : s == 1 ? 4 : 3)
       : n == 128 ? (s == 0 ? 16 : 8)
       : n == 192 ? (s == 0 ? 16 : s == 1 ? 4 : 3)
       : n == 256 ? 16 : 0;
}
// Sub-transform length at stage s.
__host__ __device__ constexpr int len(int n, int s) { return s == 0 ? n : len(n, s - 1) / rad(n, s - 1); }

// Position of frequency k after the DIF stages of length n.
__host__ __device__ constexpr int dif_pos(int n, int k) {
  int pos = 0, L = n;
  for (int s = 0; s < nst(n); ++s) {
    const int r = rad(n, s), m = L / r;
    pos += m * (k % r);
    k /= r;
    L = m;
  }
  return pos;
}

// cos and sin of 2 pi e / 16, e = 0..15
__host__ __device__ constexpr double c16(int e) {
  constexpr double t[16] = {1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
                            0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613,
                            -1.0, -0.92387953251128675613, -0.70710678118654752440, -0.38268343236508977173,
                            0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613};
  return t[e & 15];
}
__host__ __device__ constexpr double s16(int e) { return c16(e + 12); }   // sin(x) = cos(x - pi/2)

// v * W_R^e (forward, W = exp(-2 pi i / R)) or v * conj(W_R^e) (inverse); R | 16
template <int R, int E, bool INV, typename C>
__device__ __forceinline__ C twc(C v) {
  constexpr int e16 = ((E % R) * (16 / R)) & 15;
  if constexpr (e16 == 0) return v;
  else if constexpr (e16 == 8) { v.x = -v.x; v.y = -v.y; return v; }
  else if constexpr (e16 == 4) return rot90<C, INV>(v);           // * -i (fwd), * +i (inv)
  else if constexpr (e16 == 12) return rot90<C, !INV>(v);
  else {
    typedef decltype(v.x) T;
    const T c = (T)c16(e16);
    const T s = INV ? (T)s16(e16) : (T)-s16(e16);       // W^e = cos - i sin
    if constexpr (!std::is_floating_point<T>::value) {
      // double word: the fused complex product (its TwoProd errors gathered
      // before one TwoSum per part) instead of four products and two sums
      C w;
      w.x = c;
      w.y = s;
      return cmul(v, w);
    } else {
      C r;
      r.x = v.x * c - v.y * s;
      r.y = v.x * s + v.y * c;
      return r;
    }
  }
}

// In-register DFT of length R on v[0..R-1] (natural in, natural out).
template <int R, bool INV, typename C> struct Dft;

template <bool INV, typename C> struct Dft<2, INV, C> {
  static __device__ __forceinline__ void run(C* v) {
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  }
};
template <bool INV, typename C> struct Dft<3, INV, C> {
  static __device__ __forceinline__ void run(C* v) { Radix<3, INV, C>::run(v); }
};
template <bool INV, typename C> struct Dft<4, INV, C> {
  static __device__ __forceinline__ void run(C* v) { Radix<4, INV, C>::run(v); }
};

// R = R1 * R2 with n = R2 n1 + n2 and k = k1 + R1 k2.
template <int R1, int R2, bool INV, typename C>
__device__ __forceinline__ void dft_composite(C* v) {
  constexpr int R = R1 * R2;
  C a[R];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    C t[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) t[n1] = v[R2 * n1 + n2];
    Dft<R1, INV, C>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) a[n2 * R1 + k1] = t[k1];
  }
  // twiddles W_R^(n2 k1)
#pragma unroll
  for (int n2 = 1; n2 < R2; ++n2) {
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
      const int e = n2 * k1;
      C& x = a[n2 * R1 + k1];
      switch (e) {   // resolved at compile time after unrolling
        case 1: x = twc<R, 1, INV>(x); break;
        case 2: x = twc<R, 2, INV>(x); break;
        case 3: x = twc<R, 3, INV>(x); break;
        case 4: x = twc<R, 4, INV>(x); break;
        case 6: x = twc<R, 6, INV>(x); break;
        case 9: x = twc<R, 9, INV>(x); break;
        default: break;
      }
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    C t[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) t[n2] = a[n2 * R1 + k1];
    Dft<R2, INV, C>::run(t);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[k2];
  }
}

template <bool INV, typename C> struct Dft<8, INV, C> {
  static __device__ __forceinline__ void run(C* v) { dft_composite<4, 2, INV, C>(v); }
};
template <bool INV, typename C> struct Dft<16, INV, C> {
  static __device__ __forceinline__ void run(C* v) { dft_composite<4, 4, INV, C>(v); }
};

// One stage over NSEQ sequences of length N in shared memory.  Element j of
// sequence q lives at buf[(q / SQ) * SQSTR + (q % SQ) * SSTR + j * ESTR]
// (SQ = 1 gives buf[q * SQSTR + j * ESTR]).  The twiddle table holds
// W_NTAB^t, N | NTAB.  SEQFAST: consecutive threads take consecutive
// sequences (else consecutive butterflies of one sequence).
//
// stage_io takes the butterfly inputs from ld(q, i, e) and hands its outputs
// to st(q, i, e, value), where i is the shared-memory index and e the
// position along the sequence; stage() is stage_io on shared memory.  The
// first or last stage of a transform can so read from or write to global
// memory directly.
template <typename C, int N, int NTAB, int S, bool INV, int NSEQ, int SQ, int SQSTR, int SSTR,
          int ESTR, bool SEQFAST, typename LD, typename ST>
__device__ __forceinline__ void stage_io(const C* __restrict__ tw, LD ld, ST st) {
  constexpr int R = rad(N, S);
  constexpr int L = len(N, S);
  constexpr int M = L / R;
  constexpr int NB = N / R;
  constexpr int TOTAL = NSEQ * NB;
  constexpr int TSTEP = NTAB / L;
  for (int t = threadIdx.x; t < TOTAL; t += blockDim.x) {
    int q, b;
    if (SEQFAST) { q = t % NSEQ; b = t / NSEQ; } else { b = t % NB; q = t / NB; }
    const int blk = b / M;
    const int j0 = b - blk * M;
    const int base = (q / SQ) * SQSTR + (q % SQ) * SSTR + (blk * L + j0) * ESTR;
    const int e0 = blk * L + j0;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld(q, base + r * M * ESTR, e0 + r * M);
    if (!INV) {
      Dft<R, false, C>::run(v);
      if (M > 1) {
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = cmul(v[k], tw[MF_AT(j0 * k * TSTEP, NTAB)]);
      }
    } else {
      if (M > 1) {
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], tw[MF_AT(j0 * k * TSTEP, NTAB)]);
      }
      Dft<R, true, C>::run(v);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) st(q, base + r * M * ESTR, e0 + r * M, v[r]);
  }
}

// Largest shared-memory index a stage over this layout touches, plus one:
// the extent the debug build checks stage() accesses against.
template <int N, int NSEQ, int SQ, int SQSTR, int SSTR, int ESTR>
__host__ __device__ constexpr int layout_extent() {
  return ((NSEQ - 1) / SQ) * SQSTR + ((NSEQ - 1) % SQ) * SSTR + (N - 1) * ESTR + 1;
}

template <typename C, int N, int NTAB, int S, bool INV, int NSEQ, int SQ, int SQSTR, int SSTR,
          int ESTR, bool SEQFAST>
__device__ __forceinline__ void stage(C* __restrict__ buf, const C* __restrict__ tw) {
  constexpr int EXT = layout_extent<N, NSEQ, SQ, SQSTR, SSTR, ESTR>();
  stage_io<C, N, NTAB, S, INV, NSEQ, SQ, SQSTR, SSTR, ESTR, SEQFAST>(
      tw, [&](int, int i, int) { return buf[MF_AT(i, EXT)]; }, [&](int, int i, int, C v) { buf[MF_AT(i, EXT)] = v; });
}

// Whole transform (all stages), with a barrier after each stage.  SEQFAST is
// chosen per stage: consecutive threads take consecutive butterflies while the
// butterfly spacing M * ESTR is at least 16 elements, else consecutive
// sequences (the caller pads SQSTR so that those fall in different banks).
template <typename C, int N, int NTAB, bool INV, int NSEQ, int SQ, int SQSTR, int SSTR, int ESTR,
          int S = 0>
__device__ __forceinline__ void run_stages_fwd(C* buf, const C* tw) {
  if constexpr (S < nst(N)) {
    constexpr int M = len(N, S) / rad(N, S);
    constexpr bool SF = !(ESTR == 1 && M >= 16);
    stage<C, N, NTAB, S, false, NSEQ, SQ, SQSTR, SSTR, ESTR, SF>(buf, tw);
    __syncthreads();
    run_stages_fwd<C, N, NTAB, INV, NSEQ, SQ, SQSTR, SSTR, ESTR, S + 1>(buf, tw);
  }
}
template <typename C, int N, int NTAB, int NSEQ, int SQ, int SQSTR, int SSTR, int ESTR, int S = nst(N) - 1>
__device__ __forceinline__ void run_stages_inv(C* buf, const C* tw) {
  if constexpr (S >= 0) {
    constexpr int M = len(N, S) / rad(N, S);
    constexpr bool SF = !(ESTR == 1 && M >= 16);
    stage<C, N, NTAB, S, true, NSEQ, SQ, SQSTR, SSTR, ESTR, SF>(buf, tw);
    __syncthreads();
    run_stages_inv<C, N, NTAB, NSEQ, SQ, SQSTR, SSTR, ESTR, S - 1>(buf, tw);
  }
}

template <typename C, int N, int NTAB, int NSEQ, int SQ, int SQSTR, int SSTR, int ESTR>
__device__ __forceinline__ void forward(C* buf, const C* tw) {
  run_stages_fwd<C, N, NTAB, false, NSEQ, SQ, SQSTR, SSTR, ESTR>(buf, tw);
}

// Forward transform whose last stage sends its outputs to st(q, e, value)
// (sequence q, digit-reversed position e) instead of shared memory; no
// barrier after it.
template <typename C, int N, int NTAB, int NSEQ, int SQ, int SQSTR, int SSTR, int ESTR, int S = 0,
          typename ST>
__device__ __forceinline__ void forward_out(C* buf, const C* tw, ST st) {
  constexpr int M = len(N, S) / rad(N, S);
  constexpr bool SF = !(ESTR == 1 && M >= 16);
  if constexpr (S + 1 < nst(N)) {
    stage<C, N, NTAB, S, false, NSEQ, SQ, SQSTR, SSTR, ESTR, SF>(buf, tw);
    __syncthreads();
    forward_out<C, N, NTAB, NSEQ, SQ, SQSTR, SSTR, ESTR, S + 1>(buf, tw, st);
  } else {
    constexpr int EXT = layout_extent<N, NSEQ, SQ, SQSTR, SSTR, ESTR>();
    stage_io<C, N, NTAB, S, false, NSEQ, SQ, SQSTR, SSTR, ESTR, SF>(
        tw, [&](int, int i, int) { return buf[MF_AT(i, EXT)]; }, [&](int q, int, int e, C v) { st(q, e, v); });
  }
}

// Inverse transform whose first stage reads its inputs from ld(q, e) instead
// of shared memory; ends with a barrier like inverse().
template <typename C, int N, int NTAB, int NSEQ, int SQ, int SQSTR, int SSTR, int ESTR, typename LD>
__device__ __forceinline__ void inverse_in(C* buf, const C* tw, LD ld) {
  constexpr int S = nst(N) - 1;
  constexpr int M = len(N, S) / rad(N, S);
  constexpr bool SF = !(ESTR == 1 && M >= 16);
  constexpr int EXT = layout_extent<N, NSEQ, SQ, SQSTR, SSTR, ESTR>();
  stage_io<C, N, NTAB, S, true, NSEQ, SQ, SQSTR, SSTR, ESTR, SF>(
      tw, [&](int q, int, int e) { return ld(q, e); }, [&](int, int i, int, C v) { buf[MF_AT(i, EXT)] = v; });
  __syncthreads();
  if constexpr (S > 0) run_stages_inv<C, N, NTAB, NSEQ, SQ, SQSTR, SSTR, ESTR, S - 1>(buf, tw);
}
template <typename C, int N, int NTAB, int NSEQ, int SQ, int SQSTR, int SSTR, int ESTR>
__device__ __forceinline__ void inverse(C* buf, const C* tw) {
  run_stages_inv<C, N, NTAB, NSEQ, SQ, SQSTR, SSTR, ESTR>(buf, tw);
}

}  // namespace fft2
