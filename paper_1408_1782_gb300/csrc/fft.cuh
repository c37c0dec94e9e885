// Block-level FFT building blocks for the spectral collision operator.
//
// A length-n DFT (n = A*B) is done in two in-place stages on a line of
// double2 values (Cooley-Tukey "four-step" split, no reordering pass):
//   t = B*t1 + t2,  k = k1 + A*k2
//   forward: X[k1 + A k2] = sum_t2 e^{-2pi i t2 k2/B} [ e^{-2pi i t2 k1/n} sum_t1 e^{-2pi i t1 k1/A} x[B t1 + t2] ]
// Stage 1 reads positions B*t1 + t2 and writes back to the same positions
// (holding index k1 at B*k1 + t2); stage 2 reads the B contiguous values at
// B*k1 + (0..B-1) and writes them back in place.  The spectrum therefore sits
// in the "permuted" order pos(k) = B*(k mod A) + (k div A).  The inverse runs
// the two stages backwards and takes permuted input to natural output.  All
// spectral-space tables of the library are stored in this permuted order.
//
// Sign convention: forward = sum x e^{-2 pi i ...}, inverse = sum X e^{+2 pi i ...},
// both unnormalised.
#pragma once

#include <cuda_runtime.h>

namespace qbe {

template <int n> struct Split;
template <> struct Split<16>  { static constexpr int A = 4,  B = 4;  };
template <> struct Split<32>  { static constexpr int A = 4,  B = 8;  };
template <> struct Split<64>  { static constexpr int A = 8,  B = 8;  };
template <> struct Split<128> { static constexpr int A = 8,  B = 16; };
template <> struct Split<256> { static constexpr int A = 16, B = 16; };
template <> struct Split<96>  { static constexpr int A = 12, B = 8;  };
template <> struct Split<192> { static constexpr int A = 12, B = 16; };

// Frequency index (0..n-1, standard wrap) stored at permuted position pos.
template <int n>
__host__ __device__ __forceinline__ int freq_of_pos(int pos) {
  constexpr int A = Split<n>::A, B = Split<n>::B;
  return pos / B + A * (pos % B);
}
// Permuted position of frequency index k.
template <int n>
__host__ __device__ __forceinline__ int pos_of_freq(int k) {
  constexpr int A = Split<n>::A, B = Split<n>::B;
  return B * (k % A) + k / A;
}

// Real type of a complex vector type, and fused multiply-add per precision.
template <class C2> struct RealOf;
template <> struct RealOf<double2> { using type = double; };
template <> struct RealOf<float2> { using type = float; };
template <class T> struct Vec2Of;
template <> struct Vec2Of<double> { using type = double2; };
template <> struct Vec2Of<float> { using type = float2; };
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double2 mk2(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mk2(float x, float y) { return make_float2(x, y); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaT(a.x, b.x, -a.y * b.y), fmaT(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaT(a.x, b.x, a.y * b.y), fmaT(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fmaT(a.x, b.x, -a.y * b.y), fmaT(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a * conj(b)
  return make_double2(fmaT(a.x, b.x, a.y * b.y), fmaT(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// cos(2 pi k / 16) for integer k (mathematical constants cos(pi/8), sin(pi/8), sqrt(1/2)).
__host__ __device__ constexpr double cos16(int k) {
  constexpr double c1 = 0.92387953251128675613;   // cos(pi/8)
  constexpr double s1 = 0.38268343236508977173;   // sin(pi/8)
  constexpr double r2 = 0.70710678118654752440;   // sqrt(1/2)
  k &= 15;
  return k == 0 ? 1.0 : k == 1 ? c1 : k == 2 ? r2 : k == 3 ? s1 : k == 4 ? 0.0 : k == 5 ? -s1
       : k == 6 ? -r2 : k == 7 ? -c1 : k == 8 ? -1.0 : k == 9 ? -c1 : k == 10 ? -r2 : k == 11 ? -s1
       : k == 12 ? 0.0 : k == 13 ? s1 : k == 14 ? r2 : c1;
}
__host__ __device__ constexpr double sin16(int k) { return cos16(k - 4); }

// x * exp(SIGN * 2 pi i k / R) for R <= 16, k a compile-time constant after unrolling.
template <int R, int SIGN, class C2>
__device__ __forceinline__ C2 twid(int k, C2 x) {
  using T = typename RealOf<C2>::type;
  const int k16 = (k * (16 / R)) & 15;
  if (k16 == 0) return x;
  if (k16 == 8) return mk2(-x.x, -x.y);
  if (k16 == 4) return SIGN > 0 ? mk2(-x.y, x.x) : mk2(x.y, -x.x);
  if (k16 == 12) return SIGN > 0 ? mk2(x.y, -x.x) : mk2(-x.y, x.x);
  const T c = (T)cos16(k16), s = (T)(SIGN * sin16(k16));
  return mk2(fmaT(x.x, c, -x.y * s), fmaT(x.x, s, x.y * c));
}

__host__ __device__ constexpr int ilog2c(int r) { return r <= 1 ? 0 : 1 + ilog2c(r / 2); }
// Bit reversal of i within `bits` <= 4 bits (closed form so that it folds after unrolling).
__host__ __device__ constexpr int bitrev(int i, int bits) {
  return (((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3)) >> (4 - bits);
}

// One radix-2 decimation-in-time stage of butterfly span S on R registers.
// Butterflies with a non-trivial twiddle w = c + i s use the cosine-factored
// form (u +- w x) = u +- c (x + (s/c) i x): six FMAs instead of two products,
// two FMAs and four additions (|s/c| <= tan(3 pi/8) for R <= 16).
template <int R, int SIGN, int S, class C2>
struct DftStage {
  __device__ __forceinline__ static void run(C2 (&b)[R]) {
    using T = typename RealOf<C2>::type;
#pragma unroll
    for (int g = 0; g < R; g += S) {
#pragma unroll
      for (int k = 0; k < S / 2; ++k) {
        const int k16 = (k * (16 / S)) & 15;
        const C2 u = b[g + k];
        const C2 x = b[g + k + S / 2];
        if ((k16 & 3) == 0) {
          const C2 t = twid<16, SIGN>(k16, x);
          b[g + k] = cadd(u, t);
          b[g + k + S / 2] = csub(u, t);
        } else {
          const T c = (T)cos16(k16);
          const T r = (T)((SIGN * sin16(k16)) / cos16(k16));
          const T qx = fmaT(-r, x.y, x.x);
          const T qy = fmaT(r, x.x, x.y);
          b[g + k] = mk2(fmaT(c, qx, u.x), fmaT(c, qy, u.y));
          b[g + k + S / 2] = mk2(fmaT(-c, qx, u.x), fmaT(-c, qy, u.y));
        }
      }
    }
    DftStage<R, SIGN, 2 * S, C2>::run(b);
  }
};
template <int R, int SIGN, class C2>
struct DftStage<R, SIGN, 2 * R, C2> {
  __device__ __forceinline__ static void run(C2 (&)[R]) {}
};

// cos(2 pi k / 12) for integer k.
__host__ __device__ constexpr double cos12(int k) {
  constexpr double h3 = 0.86602540378443864676;   // sqrt(3)/2
  k = ((k % 12) + 12) % 12;
  return k == 0 ? 1.0 : k == 1 ? h3 : k == 2 ? 0.5 : k == 3 ? 0.0 : k == 4 ? -0.5 : k == 5 ? -h3
       : k == 6 ? -1.0 : k == 7 ? -h3 : k == 8 ? -0.5 : k == 9 ? 0.0 : k == 10 ? 0.5 : h3;
}
__host__ __device__ constexpr double sin12(int k) { return cos12(k - 3); }

// In-register DFT of length R (natural order in and out): R a power of two <= 16
// (radix-2 decimation in time), or R = 3 * 2^q <= 12 (one radix-3 decimation-in-time
// step on top of power-of-two sub-DFTs).
template <int R, int SIGN, class C2, bool POW2 = ((R & (R - 1)) == 0)>
struct Dft;

template <int R, int SIGN, class C2>
struct Dft<R, SIGN, C2, true> {
  __device__ __forceinline__ static void run(C2 (&a)[R]) {
    constexpr int L2 = ilog2c(R);
    C2 b[R];
#pragma unroll
    for (int i = 0; i < R; ++i) b[i] = a[bitrev(i, L2)];
    DftStage<R, SIGN, 2, C2>::run(b);
#pragma unroll
    for (int i = 0; i < R; ++i) a[i] = b[i];
  }
};

template <int R, int SIGN, class C2>
struct Dft<R, SIGN, C2, false> {
  static_assert(R % 3 == 0 && R <= 12, "mixed-radix DFT supports 3, 6, 12");
  __device__ __forceinline__ static void run(C2 (&a)[R]) {
    using T = typename RealOf<C2>::type;
    constexpr int Q = R / 3;
    C2 s0[Q], s1[Q], s2[Q];
#pragma unroll
    for (int t = 0; t < Q; ++t) { s0[t] = a[3 * t]; s1[t] = a[3 * t + 1]; s2[t] = a[3 * t + 2]; }
    Dft<Q, SIGN, C2>::run(s0);
    Dft<Q, SIGN, C2>::run(s1);
    Dft<Q, SIGN, C2>::run(s2);
    const T h3 = (T)(SIGN * 0.86602540378443864676);   // SIGN * sqrt(3)/2
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      // twiddles exp(SIGN 2 pi i r k / R), r = 1, 2 (angles in twelfths: (12/R) r k)
      const int e1 = (12 / R) * k, e2 = 2 * (12 / R) * k;
      const C2 x0 = s0[k];
      C2 x1 = s1[k], x2 = s2[k];
      if (e1 % 12 != 0) {
        const T c = (T)cos12(e1), sn = (T)(SIGN * sin12(e1));
        x1 = mk2(fmaT(x1.x, c, -x1.y * sn), fmaT(x1.x, sn, x1.y * c));
      }
      if (e2 % 12 != 0) {
        const T c = (T)cos12(e2), sn = (T)(SIGN * sin12(e2));
        x2 = mk2(fmaT(x2.x, c, -x2.y * sn), fmaT(x2.x, sn, x2.y * c));
      }
      // radix-3 butterfly with w = exp(SIGN 2 pi i / 3)
      const C2 t1 = cadd(x1, x2);
      const C2 t2 = mk2(fmaT((T)-0.5, t1.x, x0.x), fmaT((T)-0.5, t1.y, x0.y));
      const C2 d = csub(x1, x2);
      const C2 t3 = mk2(-h3 * d.y, h3 * d.x);   // i * SIGN * sqrt(3)/2 * (x1 - x2)
      a[k] = cadd(x0, t1);
      a[k + Q] = cadd(t2, t3);
      a[k + 2 * Q] = csub(t2, t3);
    }
  }
};

template <int R, int SIGN, class C2>
__device__ __forceinline__ void dft(C2 (&a)[R]) {
  Dft<R, SIGN, C2>::run(a);
}

// DFT of length R (a power of two) of the inputs a[i] multiplied by real scales sc[i], the scaling
// fused into the first radix-2 stage: u su +- x sx as t = x sx (one multiplication per component)
// and two FMAs, instead of two multiplications and two additions per component.
template <int R, int SIGN, class C2>
__device__ __forceinline__ void dft_scaled(C2 (&a)[R], const typename RealOf<C2>::type (&sc)[R]) {
  static_assert((R & (R - 1)) == 0 && R >= 2, "power-of-two length");
  constexpr int L2 = ilog2c(R);
  C2 b[R];
#pragma unroll
  for (int g = 0; g < R; g += 2) {
    const int iu = bitrev(g, L2), ix = bitrev(g + 1, L2);
    const C2 u = a[iu], x = a[ix];
    const C2 t = mk2(x.x * sc[ix], x.y * sc[ix]);
    b[g] = mk2(fmaT(u.x, sc[iu], t.x), fmaT(u.y, sc[iu], t.y));
    b[g + 1] = mk2(fmaT(u.x, sc[iu], -t.x), fmaT(u.y, sc[iu], -t.y));
  }
  DftStage<R, SIGN, 4, C2>::run(b);
#pragma unroll
  for (int i = 0; i < R; ++i) a[i] = b[i];
}

// DFT of length 16 whose inputs a[4..11] are zero -- a stage-B line of the 128-point padded grid
// holding only band-limited (Xi) frequencies -- with the first radix-2 stage reduced to copies: its
// butterflies pair a[r] with a[r + 8], r < 8, and one of the two is zero.
template <int SIGN, class C2>
__device__ __forceinline__ void dft16_xi(C2 (&a)[16]) {
  C2 b[16];
#pragma unroll
  for (int g = 0; g < 16; g += 2) {
    const int r = bitrev(g, 4);   // 0..7; bitrev(g + 1, 4) = r + 8
    if (r < 4) {
      b[g] = a[r];
      b[g + 1] = a[r];
    } else {
      b[g] = a[r + 8];
      b[g + 1] = mk2(-a[r + 8].x, -a[r + 8].y);
    }
  }
  DftStage<16, SIGN, 4, C2>::run(b);
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = b[i];
}

// Padded grids whose stage-B lines (B = 16) hold the band-limited frequencies |k| < n/4 (Xi) at
// t = 0..3, 12..15 only: n = A B with n / 4 = 4 A.
template <int n>
__host__ __device__ constexpr bool xi_prunable() {
  return Split<n>::B == 16;
}

// FFT of nl lines of length n held in shared (or global) memory:
// element e of line l at buf[l*ls + e*es].  tw[t2*A + k1] = exp(-2 pi i t2 k1 / n).
// SIGN < 0: forward, natural -> permuted.  SIGN > 0: inverse, permuted -> natural.
// XI (inverse only): the input is zero outside Xi, so where xi_prunable<n>() the first stage reads
// the Xi values of each line only and runs dft16_xi.
// Must be called by every thread of the block; ends with __syncthreads().
template <int n, int SIGN, bool XI = false, class C2>
__device__ __forceinline__ void fft_lines(C2* buf, int nl, int ls, int es, const C2* __restrict__ tw) {
  constexpr int A = Split<n>::A, B = Split<n>::B;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (SIGN < 0) {
    for (int task = tid; task < nl * B; task += nt) {
      const int l = task % nl, t2 = task / nl;
      C2* base = buf + l * ls + t2 * es;
      C2 a[A];
#pragma unroll
      for (int t1 = 0; t1 < A; ++t1) a[t1] = base[B * t1 * es];
      dft<A, -1>(a);
#pragma unroll
      for (int k1 = 1; k1 < A; ++k1) a[k1] = cmul(a[k1], tw[t2 * A + k1]);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) base[B * k1 * es] = a[k1];
    }
    __syncthreads();
    for (int task = tid; task < nl * A; task += nt) {
      const int l = task % nl, k1 = task / nl;
      C2* base = buf + l * ls + B * k1 * es;
      C2 b[B];
#pragma unroll
      for (int t2 = 0; t2 < B; ++t2) b[t2] = base[t2 * es];
      dft<B, -1>(b);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) base[k2 * es] = b[k2];
    }
    __syncthreads();
  } else {
    for (int task = tid; task < nl * A; task += nt) {
      const int l = task % nl, k1 = task / nl;
      C2* base = buf + l * ls + B * k1 * es;
      C2 b[B];
      if constexpr (XI && xi_prunable<n>()) {
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) b[k2] = (k2 < 4 || k2 >= 12) ? base[k2 * es] : mk2((typename RealOf<C2>::type)0, (typename RealOf<C2>::type)0);
        dft16_xi<1>(b);
      } else {
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) b[k2] = base[k2 * es];
        dft<B, 1>(b);
      }
#pragma unroll
      for (int t2 = 0; t2 < B; ++t2) base[t2 * es] = b[t2];
    }
    __syncthreads();
    for (int task = tid; task < nl * B; task += nt) {
      const int l = task % nl, t2 = task / nl;
      C2* base = buf + l * ls + t2 * es;
      C2 a[A];
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) a[k1] = base[B * k1 * es];
#pragma unroll
      for (int k1 = 1; k1 < A; ++k1) a[k1] = cmulc(a[k1], tw[t2 * A + k1]);
      dft<A, 1>(a);
#pragma unroll
      for (int t1 = 0; t1 < A; ++t1) base[B * t1 * es] = a[t1];
    }
    __syncthreads();
  }
}

// Circular convolution along lines: forward FFT, multiplication of each
// spectral value by mul(line, pos) (pos = permuted position), inverse FFT.  The
// second forward stage, the multiplication and the first inverse stage act on
// the same B contiguous values, so they are fused in registers.
template <int n, class C2, class MUL>
__device__ __forceinline__ void fft_conv_lines(C2* buf, int nl, int ls, int es, const C2* __restrict__ tw, MUL mul) {
  constexpr int A = Split<n>::A, B = Split<n>::B;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int task = tid; task < nl * B; task += nt) {
    const int l = task % nl, t2 = task / nl;
    C2* base = buf + l * ls + t2 * es;
    C2 a[A];
#pragma unroll
    for (int t1 = 0; t1 < A; ++t1) a[t1] = base[B * t1 * es];
    dft<A, -1>(a);
#pragma unroll
    for (int k1 = 1; k1 < A; ++k1) a[k1] = cmul(a[k1], tw[t2 * A + k1]);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) base[B * k1 * es] = a[k1];
  }
  __syncthreads();
  for (int task = tid; task < nl * A; task += nt) {
    const int l = task % nl, k1 = task / nl;
    C2* base = buf + l * ls + B * k1 * es;
    C2 b[B];
#pragma unroll
    for (int t2 = 0; t2 < B; ++t2) b[t2] = base[t2 * es];
    dft<B, -1>(b);
    typename RealOf<C2>::type sc[B];
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) sc[k2] = (typename RealOf<C2>::type)mul(l, B * k1 + k2);
    dft_scaled<B, 1>(b, sc);
#pragma unroll
    for (int t2 = 0; t2 < B; ++t2) base[t2 * es] = b[t2];
  }
  __syncthreads();
  for (int task = tid; task < nl * B; task += nt) {
    const int l = task % nl, t2 = task / nl;
    C2* base = buf + l * ls + t2 * es;
    C2 a[A];
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) a[k1] = base[B * k1 * es];
#pragma unroll
    for (int k1 = 1; k1 < A; ++k1) a[k1] = cmulc(a[k1], tw[t2 * A + k1]);
    dft<A, 1>(a);
#pragma unroll
    for (int t1 = 0; t1 < A; ++t1) base[B * t1 * es] = a[t1];
  }
  __syncthreads();
}

// Chunk sizes (rows per row-pass chunk, columns per column-pass chunk) so that a
// chunk of complex doubles occupies about 64 KB of shared memory (three blocks
// per SM fit) and the radix-B stage has at least one task per thread.
__host__ __device__ constexpr int largest_divisor_le(int n, int cap) {
  return cap >= n ? n : (n % cap == 0 ? cap : largest_divisor_le(n, cap - 1));
}

template <int n, int ELEM = 16, int CB = 65536> struct Chunk {
  static constexpr int RC0 = CB / (n * ELEM);
  static constexpr int RC = largest_divisor_le(n, RC0);
  static constexpr int CC = RC;
  static constexpr int LS = n + 1;                 // padded row stride (odd => no bank conflicts)
  static constexpr int SMEM_ELEMS = (RC * LS > CC * n ? RC * LS : CC * n);
};

// Row pass over an n x n field (rows = fixed ix, transform along iy):
// for each chunk: sm[r][iy] = ld(ix, iy); [FFT DIR1]; [sm = mid(ix, iy, sm)]; [FFT DIR2]; st(ix, iy, sm).
// DIR = 0 skips that transform; HAS_MID selects the pointwise middle step.
template <int n, int DIR1, bool HAS_MID, int DIR2, int CB = 65536, bool XI = false, class C2, class LD, class MID,
          class ST>
__device__ __forceinline__ void row_pass(C2* sm, const C2* tw, LD ld, MID mid, ST st) {
  constexpr int RC = Chunk<n, sizeof(C2), CB>::RC, LS = Chunk<n, sizeof(C2), CB>::LS;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int r0 = 0; r0 < n; r0 += RC) {
#pragma unroll 4
    for (int idx = tid; idx < RC * n; idx += nt) {
      const int r = idx / n, iy = idx % n;
      sm[r * LS + iy] = ld(r0 + r, iy);
    }
    __syncthreads();
    if (DIR1 != 0) fft_lines<n, (DIR1 < 0 ? -1 : 1), XI>(sm, RC, LS, 1, tw);
    if (HAS_MID) {
  #pragma unroll 4
    for (int idx = tid; idx < RC * n; idx += nt) {
        const int r = idx / n, iy = idx % n;
        sm[r * LS + iy] = mid(r0 + r, iy, sm[r * LS + iy]);
      }
      __syncthreads();
    }
    if (DIR2 != 0) fft_lines<n, (DIR2 < 0 ? -1 : 1)>(sm, RC, LS, 1, tw);
#pragma unroll 4
    for (int idx = tid; idx < RC * n; idx += nt) {
      const int r = idx / n, iy = idx % n;
      st(r0 + r, iy, sm[r * LS + iy]);
    }
    __syncthreads();
  }
}

// Column pass (transform along ix) over chunks of CC columns held as sm[ix][c].
template <int n, int DIR1, bool HAS_MID, int DIR2, int CB = 65536, class C2, class LD, class MID, class ST>
__device__ __forceinline__ void col_pass(C2* sm, const C2* tw, LD ld, MID mid, ST st) {
  constexpr int CC = Chunk<n, sizeof(C2), CB>::CC;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int c0 = 0; c0 < n; c0 += CC) {
#pragma unroll 4
    for (int idx = tid; idx < CC * n; idx += nt) {
      const int ix = idx / CC, c = idx % CC;
      sm[ix * CC + c] = ld(ix, c0 + c);
    }
    __syncthreads();
    if (DIR1 != 0) fft_lines<n, (DIR1 < 0 ? -1 : 1)>(sm, CC, 1, CC, tw);
    if (HAS_MID) {
  #pragma unroll 4
    for (int idx = tid; idx < CC * n; idx += nt) {
        const int ix = idx / CC, c = idx % CC;
        sm[ix * CC + c] = mid(ix, c0 + c, sm[ix * CC + c]);
      }
      __syncthreads();
    }
    if (DIR2 != 0) fft_lines<n, (DIR2 < 0 ? -1 : 1)>(sm, CC, 1, CC, tw);
#pragma unroll 4
    for (int idx = tid; idx < CC * n; idx += nt) {
      const int ix = idx / CC, c = idx % CC;
      st(ix, c0 + c, sm[ix * CC + c]);
    }
    __syncthreads();
  }
}

// Column pass doing a circular convolution along ix for each column iy:
// sm[ix][c] = ld(ix, iy); forward FFT; times mul(pos_x, iy); inverse FFT; st(ix, iy, value).
template <int n, int CB = 65536, class C2, class LD, class MUL, class ST>
__device__ __forceinline__ void col_conv_pass(C2* sm, const C2* tw, LD ld, MUL mul, ST st) {
  constexpr int CC = Chunk<n, sizeof(C2), CB>::CC;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int c0 = 0; c0 < n; c0 += CC) {
#pragma unroll 4
    for (int idx = tid; idx < CC * n; idx += nt) {
      const int ix = idx / CC, c = idx % CC;
      sm[ix * CC + c] = ld(ix, c0 + c);
    }
    __syncthreads();
    fft_conv_lines<n>(sm, CC, 1, CC, tw, [&](int l, int pos) { return mul(pos, c0 + l); });
#pragma unroll 4
    for (int idx = tid; idx < CC * n; idx += nt) {
      const int ix = idx / CC, c = idx % CC;
      st(ix, c0 + c, sm[ix * CC + c]);
    }
    __syncthreads();
  }
}

// Column pass over a subset of columns cols[0..ncols) (chunks of CC columns).
template <int n, int DIR1, bool HAS_MID, int DIR2, int CB = 65536, bool XI = false, class C2, class LD, class MID,
          class ST>
__device__ __forceinline__ void col_pass_list(C2* sm, const C2* tw, const int* cols, int ncols, LD ld, MID mid,
                                              ST st) {
  constexpr int CC = Chunk<n, sizeof(C2), CB>::CC;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int c0 = 0; c0 < ncols; c0 += CC) {
    const int nc = (ncols - c0) < CC ? (ncols - c0) : CC;
#pragma unroll 4
    for (int idx = tid; idx < nc * n; idx += nt) {
      const int ix = idx / nc, c = idx % nc;
      sm[ix * CC + c] = ld(ix, cols[c0 + c]);
    }
    __syncthreads();
    if (DIR1 != 0) fft_lines<n, (DIR1 < 0 ? -1 : 1), XI>(sm, nc, 1, CC, tw);
    if (HAS_MID) {
  #pragma unroll 4
    for (int idx = tid; idx < nc * n; idx += nt) {
        const int ix = idx / nc, c = idx % nc;
        sm[ix * CC + c] = mid(ix, cols[c0 + c], sm[ix * CC + c]);
      }
      __syncthreads();
    }
    if (DIR2 != 0) fft_lines<n, (DIR2 < 0 ? -1 : 1)>(sm, nc, 1, CC, tw);
#pragma unroll 4
    for (int idx = tid; idx < nc * n; idx += nt) {
      const int ix = idx / nc, c = idx % nc;
      st(ix, cols[c0 + c], sm[ix * CC + c]);
    }
    __syncthreads();
  }
}

struct NoMid {
  template <class C2>
  __device__ C2 operator()(int, int, C2 v) const { return v; }
};

// Load the n-point twiddle table into shared memory.
template <int n, class C2>
__device__ __forceinline__ void load_twiddles(C2* sm_tw, const C2* __restrict__ g_tw) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) sm_tw[i] = g_tw[i];
  __syncthreads();
}

}  // namespace qbe
