// Fast Fourier spectral collision operator C[W] = C_c[W] + C_d[W] of
// Lu & Mendl, Sec. 3.2, for 2x2 Hermitian Wigner matrices in Pauli form.
//
// Fine ("doubly padded") grid: n = 2N points per dimension, v' = -L + (L/N) i',
// fine frequencies sigma in [-N, N-1] (standard wrap).  A field on Xi is
// zero-padded to the fine grid; products of at most three Xi-limited fields
// are then free of aliasing on Xi (Sec. 1 and Sec. 3.2, "double zero padding").
// Real fields travel two at a time as the real and imaginary parts of one
// complex field; every kernel multiplier (phi, psi, psi', K) is real and has
// definite parity, so the pairing is exact.
//
// Terms (w = Pauli components, eta = diag(1,-1,-1,-1)):
//   C_c  = -2 (D x w).sigma,  D(v) = int int P(1/(u.u')) (2w0(v+u)-1) w_vec(v+u+u')   (I1, eq. CcPauliCarleman)
//   C_d  = 2 pi K2 (1 - W) - 2 pi K3.sigma + pi {W, K4.sigma}                         (I2, I3, I4, eq. CdPauli)
//   K2   = sum_a eta_a int int delta(u.u') w_a(v+u) w_a(v+u')
//   K3_b = sum_a eta_a int int delta(u.u') w_a(v+u) w_a(v+u') (eta w)_b(v+u+u')
//   K4_b = int int delta(u.u') (2 w0(v+u) - 1) (eta w)_b(v+u+u')
// with G_J (eq. approxG), H_J (eq. approxH-J) and the Hu-Ying form H_JM
// (eq. approxH-JM) for K3.  Algebraic regroupings relative to the printed
// algorithm (exact up to rounding):
//   * I1: K_j'(sigma) = sum_j omega_G[j][j'] phi_j(sigma) is tabulated, so the
//     J^2 outer convolutions become J (the j-sum is linear and acts after the
//     first convolution);
//   * psi'_j = psi_{j + J/2} (theta_j^perp = theta_{j+J/2} up to sign, psi even),
//     so the I2 and I4 inverse transforms are shared;
//   * I3: the weight (pi/J) w_m is split as sqrt((pi/J) w_m) into both shifted
//     factors; each accumulated K3 term carries it exactly once.
//
// Precision: every kernel is a template on the real type T of its transforms,
// products and per-unit accumulations (double: the plain FP64 form; float: the
// FP32-split form).  The state W comes in and C[W] goes out in FP64, and the
// reduction of the per-unit K3 partial sums is done in FP64 in both forms.
#pragma once

#include <cmath>
#include <cstdio>
#include <type_traits>

#include "fft.cuh"
#include "internal.h"

namespace qbe {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Fine frequency index k (0..n-1) lies in Xi without its -N/2 line.
template <int n>
__device__ __forceinline__ bool in_xi(int k) {
  constexpr int N = n / 2;
  return (k < N / 2) || (k > n - N / 2);
}

template <class C2>
__device__ __forceinline__ void zero_fields(C2* p, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) p[i] = mk2((typename RealOf<C2>::type)0, (typename RealOf<C2>::type)0);
  __syncthreads();
}

template <class T>
__device__ __forceinline__ typename Vec2Of<T>::type zero2() {
  return mk2((T)0, (T)0);
}

// Job of a global I3 unit: the last job whose first unit is <= gunit (uniform across the block).
template <class T>
__device__ __forceinline__ int i3_job_of(const I3Jobs<T>& jobs, int gunit) {
  int k = 0;
  while (k + 1 < jobs.njobs && gunit >= jobs.job[k + 1].unit_begin) ++k;
  return k;
}

// --------------------------------------------------------------------------
// Prep: Xi coefficients of the four Pauli components (paired) and the
// fine-grid interpolants.  One block per cell.
//   what[c][0] = w0^ + i w1^, [1] = w2^ + i w3^, [2] = w1^ + i w2^, [3] = w3^
//   wfine[c][0] = w0 + i w1, [1] = w2 + i w3  on the fine grid.
// The coarse DFT is the fine forward FFT of the zero-interleaved samples
// (its spectrum repeats with period N), scaled by 1/N^2 and cut to Xi.
// --------------------------------------------------------------------------
template <int n, class T>
__global__ void __launch_bounds__(kThreads) k_prep(const double* __restrict__ w, typename Vec2Of<T>::type* what,
                                                   typename Vec2Of<T>::type* wfine, typename Vec2Of<T>::type* ws,
                                                   const typename Vec2Of<T>::type* __restrict__ gtw) {
  using C2 = typename Vec2Of<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* sm = tw + n;
  load_twiddles<n>(tw, gtw);
  constexpr int N = n / 2, P = n * n;
  const int c = blockIdx.x;
  const double* wc = w + (size_t)c * 4 * N * N;
  C2* G = ws + (size_t)blockIdx.x * P;
  const T invN2 = (T)(1.0 / ((double)N * N));
  for (int q = 0; q < 4; ++q) {
    const int a = (q == 0) ? 0 : (q == 1) ? 2 : (q == 2) ? 1 : 3;
    const int b = (q == 0) ? 1 : (q == 1) ? 3 : (q == 2) ? 2 : -1;
    row_pass<n, -1, false, 0>(
        sm, tw,
        [&](int ix, int iy) {
          if ((ix | iy) & 1) return zero2<T>();
          const int i = ix >> 1, j = iy >> 1;
          return mk2((T)wc[(a * N + i) * N + j], b >= 0 ? (T)wc[(b * N + i) * N + j] : (T)0);
        },
        NoMid(), [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
    C2* out = what + ((size_t)c * 4 + q) * P;
    col_pass<n, -1, false, 0>(
        sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) {
          const bool keep = in_xi<n>(freq_of_pos<n>(ix)) && in_xi<n>(freq_of_pos<n>(iy));
          out[ix * n + iy] = keep ? cscale(v, invN2) : zero2<T>();
        });
  }
  for (int p = 0; p < 2; ++p) {
    const C2* in = what + ((size_t)c * 4 + p) * P;
    C2* out = wfine + ((size_t)c * 2 + p) * P;
    col_pass<n, 1, false, 0>(
        sm, tw, [&](int ix, int iy) { return in[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
    row_pass<n, 1, false, 0>(
        sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) { out[ix * n + iy] = v; });
  }
}

// --------------------------------------------------------------------------
// I1 (conservative part): D^_b(sigma) = sum_j' K_j'(sigma) FFT[(2w0-1) IFFT(phi'_j' w_b^)].
// One block per cell; pairs (w1 + i w2) and (w3).
// --------------------------------------------------------------------------
template <int n, class T>
__global__ void __launch_bounds__(kThreads) k_i1(const typename Vec2Of<T>::type* what,
                                                 const typename Vec2Of<T>::type* wfine, typename Vec2Of<T>::type* Dacc,
                                                 typename Vec2Of<T>::type* ws,
                                                 const typename Vec2Of<T>::type* __restrict__ gtw,
                                                 const T* __restrict__ phip, const T* __restrict__ Ktab, int J,
                                                 int nch) {
  using C2 = typename Vec2Of<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* sm = tw + n;
  load_twiddles<n>(tw, gtw);
  constexpr int P = n * n;
  // block (cell c, angle chunk ch): angles j' in [J ch / nch, J (ch + 1) / nch); D partial [c][ch]
  const int c = blockIdx.x / nch, ch = blockIdx.x % nch;
  C2* G = ws + (size_t)blockIdx.x * P;
  C2* D = Dacc + (size_t)blockIdx.x * 2 * P;
  zero_fields(D, 2 * P);
  const C2* wf0 = wfine + (size_t)c * 2 * P;
  for (int jp = J * ch / nch; jp < J * (ch + 1) / nch; ++jp) {
    const T* ph = phip + (size_t)jp * P;
    const T* K = Ktab + (size_t)jp * P;
    for (int p = 0; p < 2; ++p) {
      const C2* in = what + ((size_t)c * 4 + 2 + p) * P;
      C2* Dp = D + (size_t)p * P;
      col_pass<n, 1, false, 0>(
          sm, tw, [&](int ix, int iy) { return cscale(in[ix * n + iy], ph[ix * n + iy]); }, NoMid(),
          [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
      row_pass<n, 1, true, -1>(
          sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; },
          [&](int ix, int iy, C2 v) { return cscale(v, (T)2 * wf0[ix * n + iy].x - (T)1); },
          [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
      col_pass<n, -1, false, 0>(
          sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
          [&](int ix, int iy, C2 v) {
            const T k = K[ix * n + iy];
            const C2 d = Dp[ix * n + iy];
            Dp[ix * n + iy] = mk2(fmaT(k, v.x, d.x), fmaT(k, v.y, d.y));
          });
    }
  }
}

// --------------------------------------------------------------------------
// I2 and I4: one block per cell, loop over angle pairs (j, j + J/2).
//   F_{a,j} = IFFT(psi_j w_a^) (real), pairs (0,1), (2,3)
//   K2  += 2 (pi/J) sum_a eta_a F_{a,j} F_{a,j+J/2}
//   K4^ += (pi/J) [psi_j FFT((2w0-1) F_{.,j+J/2}) + psi_{j+J/2} FFT((2w0-1) F_{.,j})] / n^2
// --------------------------------------------------------------------------
template <int n, class T>
__global__ void __launch_bounds__(kThreads) k_i24(const typename Vec2Of<T>::type* what,
                                                  const typename Vec2Of<T>::type* wfine, T* K2acc,
                                                  typename Vec2Of<T>::type* K4acc, typename Vec2Of<T>::type* ws,
                                                  const typename Vec2Of<T>::type* __restrict__ gtw,
                                                  const T* __restrict__ psi, int J, int nch) {
  using C2 = typename Vec2Of<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* sm = tw + n;
  load_twiddles<n>(tw, gtw);
  constexpr int P = n * n;
  // block (cell c, chunk ch) of the J/2 angle pairs; K2, K4 partials [c][ch]
  const int c = blockIdx.x / nch, ch = blockIdx.x % nch;
  C2* slot = ws + (size_t)blockIdx.x * 5 * P;
  C2* FA = slot;            // [2][P]
  C2* FB = slot + 2 * P;    // [2][P]
  C2* G = slot + 4 * P;
  T* K2 = K2acc + (size_t)blockIdx.x * P;
  C2* K4 = K4acc + (size_t)blockIdx.x * 2 * P;
  for (int i = threadIdx.x; i < P; i += blockDim.x) K2[i] = (T)0;
  zero_fields(K4, 2 * P);
  const C2* wf0 = wfine + (size_t)c * 2 * P;
  const T wj = (T)(kPi / J);
  const T scale = (T)(kPi / J / (double)P);
  const int H = J / 2;
  for (int j = H * ch / nch; j < H * (ch + 1) / nch; ++j) {
    const int jp = j + J / 2;
    for (int p = 0; p < 2; ++p) {
      const C2* in = what + ((size_t)c * 4 + p) * P;
      for (int h = 0; h < 2; ++h) {
        const T* ps = psi + (size_t)(h == 0 ? j : jp) * P;
        C2* F = (h == 0 ? FA : FB) + (size_t)p * P;
        col_pass<n, 1, false, 0>(
            sm, tw, [&](int ix, int iy) { return cscale(in[ix * n + iy], ps[ix * n + iy]); }, NoMid(),
            [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
        row_pass<n, 1, false, 0>(
            sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
            [&](int ix, int iy, C2 v) { F[ix * n + iy] = v; });
      }
    }
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      const C2 a0 = FA[i], a1 = FA[P + i], b0 = FB[i], b1 = FB[P + i];
      const T s = a0.x * b0.x - a0.y * b0.y - a1.x * b1.x - a1.y * b1.y;
      K2[i] = fmaT((T)2 * wj, s, K2[i]);
    }
    __syncthreads();
    for (int p = 0; p < 2; ++p) {
      C2* K4p = K4 + (size_t)p * P;
      for (int h = 0; h < 2; ++h) {
        const C2* F = (h == 0 ? FB : FA) + (size_t)p * P;   // psi_j pairs with F_{j+J/2}
        const T* ps = psi + (size_t)(h == 0 ? j : jp) * P;
        row_pass<n, -1, false, 0>(
            sm, tw, [&](int ix, int iy) { return cscale(F[ix * n + iy], (T)2 * wf0[ix * n + iy].x - (T)1); },
            NoMid(), [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
        col_pass<n, -1, false, 0>(
            sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
            [&](int ix, int iy, C2 v) {
              const T k = scale * ps[ix * n + iy];
              const C2 d = K4p[ix * n + iy];
              K4p[ix * n + iy] = mk2(fmaT(k, v.x, d.x), fmaT(k, v.y, d.y));
            });
      }
    }
  }
}

// Sum of the per-chunk partials of k_i1 (D, 2 complex fields) and k_i24 (K2 real, K4 2 complex)
// of each cell, in chunk order: part[c][ch][...] -> acc[c][...].
template <class T>
__global__ void __launch_bounds__(kThreads) k_reduce_chunks(const T* __restrict__ Dpart, const T* __restrict__ K2part,
                                                            const T* __restrict__ K4part, T* Dacc, T* K2acc, T* K4acc,
                                                            int nch, int ncells, size_t P) {
  const size_t per_c = 4 * P, per_r = P;   // reals per cell: D and K4 (2 complex fields each), K2
  const size_t total = (size_t)ncells * (2 * per_c + per_r);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const T* src;
    T* dst;
    size_t c, e, stride;
    if (i < (size_t)ncells * per_c) {
      c = i / per_c; e = i % per_c; src = Dpart; dst = Dacc; stride = per_c;
    } else if (i < (size_t)ncells * 2 * per_c) {
      const size_t k = i - (size_t)ncells * per_c;
      c = k / per_c; e = k % per_c; src = K4part; dst = K4acc; stride = per_c;
    } else {
      const size_t k = i - (size_t)ncells * 2 * per_c;
      c = k / per_r; e = k % per_r; src = K2part; dst = K2acc; stride = per_r;
    }
    const T* p = src + (c * nch) * stride + e;
    T sum = p[0];
    for (int ch = 1; ch < nch; ++ch) sum += p[(size_t)ch * stride];
    dst[c * stride + e] = sum;
  }
}

// --------------------------------------------------------------------------
// I3 (dominant, Hu-Ying form eq. approxH-JM).  Persistent blocks over units
// (cell, j, m-chunk).  For each m:
//   Sigma_p = IFFT(e^{i alpha_jm.sigma} sqrt(c_jm) w^_pair p)   (shifted fields S_a = w_a(v + rho_m theta_j))
//   for a, p:  T = IFFT(psi'_j FFT(w_a Sigma_p)) / n^2;  acc_p += eta_a S_a T
// The unit's partial sum acc[2][n*n] (pairs (0,1), (2,3), real space) is
// written to its own slot of K3part and reduced in fixed order later.
// --------------------------------------------------------------------------
// The staged kernel's launch shape (threads per block, shared-memory chunk bytes of its row and
// column passes, blocks per SM) is a template parameter: the autotuner chooses among the
// instantiated shapes (i3_variant below).
template <int n, class T, int NTH = 256, int CB = 65536, int MINB = 3>
__global__ void __launch_bounds__(NTH, MINB)
    k_i3(const I3Jobs<T> jobs, typename Vec2Of<T>::type* ws, const typename Vec2Of<T>::type* __restrict__ gtw) {
  using C2 = typename Vec2Of<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* sm = tw + n;
  __shared__ int xcols[n];          // permuted positions whose frequency lies in Xi (incl. its -N/2 line)
  __shared__ unsigned char xmask[n];
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int pos = 0; pos < n; ++pos) {
      const int k = freq_of_pos<n>(pos);
      const bool in = (k < n / 4) || (k >= n - n / 4);
      xmask[pos] = in ? 1 : 0;
      if (in) xcols[cnt++] = pos;
    }
  }
  load_twiddles<n>(tw, gtw);
  constexpr int P = n * n;
  C2* slot = ws + (size_t)blockIdx.x * 3 * P;
  C2* Sig = slot;           // [2][P]
  C2* G = slot + 2 * P;
  for (int gunit = blockIdx.x; gunit < jobs.total; gunit += gridDim.x) {
    const I3Job<T>& jb = jobs.job[i3_job_of(jobs, gunit)];
    const int unit = gunit - jb.unit_begin;
    const int J = jb.J, M = jb.M, nmc = jb.nmc, mch = jb.mch;
    const C2* what = jb.what;
    const T* __restrict__ psip_s = jb.psip_s;
    const C2* __restrict__ phase = jb.phase;
    const int c = unit / (J * nmc);
    const int j = (unit / nmc) % J;
    const int mc = unit % nmc;
    C2* acc = jb.K3part + (size_t)unit * 2 * P;
    zero_fields(acc, 2 * P);
    const T* psp = psip_s + (size_t)j * P;
    const C2* wf = jb.wfine + (size_t)c * 2 * P;
    const int m0 = mc * mch, m1 = min(M, m0 + mch);
    for (int m = m0; m < m1; ++m) {
      const C2* px = phase + ((size_t)j * M + m) * 2 * n;
      const C2* py = px + n;
      for (int p = 0; p < 2; ++p) {
        const C2* in = what + ((size_t)c * 4 + p) * P;
        C2* S = Sig + (size_t)p * P;
        // only the n/2 columns (y frequencies) of Xi are non-zero: transform those
        col_pass_list<n, 1, false, 0, CB, true>(
            sm, tw, xcols, n / 2,
            [&](int ix, int iy) { return xmask[ix] ? cmul(in[ix * n + iy], cmul(px[ix], py[iy])) : zero2<T>(); },
            NoMid(), [&](int ix, int iy, C2 v) { S[ix * n + iy] = v; });
        row_pass<n, 1, false, 0, CB, true>(
            sm, tw, [&](int ix, int iy) { return xmask[iy] ? S[ix * n + iy] : zero2<T>(); }, NoMid(),
            [&](int ix, int iy, C2 v) { S[ix * n + iy] = v; });
      }
      for (int a = 0; a < 4; ++a) {
        const C2* wa = wf + (size_t)(a >> 1) * P;
        const C2* Sa = Sig + (size_t)(a >> 1) * P;
        const bool im = (a & 1) != 0;
        const bool pos_eta = (a == 0);
        for (int p = 0; p < 2; ++p) {
          const C2* Sp = Sig + (size_t)p * P;
          C2* accp = acc + (size_t)p * P;
          row_pass<n, -1, false, 0, CB>(
              sm, tw,
              [&](int ix, int iy) {
                const C2 z = wa[ix * n + iy];
                return cscale(Sp[ix * n + iy], im ? z.y : z.x);
              },
              NoMid(), [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
          col_conv_pass<n, CB>(
              sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; },
              [&](int ix, int iy) { return psp[ix * n + iy]; },
              [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
          row_pass<n, 1, false, 0, CB>(
              sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
              [&](int ix, int iy, C2 v) {
                // eta_a = +1 for a = 0, -1 otherwise: the sign goes into the FMAs
                const C2 s = Sa[ix * n + iy];
                const T f = im ? s.y : s.x;
                const C2 d = accp[ix * n + iy];
                accp[ix * n + iy] = pos_eta ? mk2(fmaT(f, v.x, d.x), fmaT(f, v.y, d.y))
                                            : mk2(fmaT(-f, v.x, d.x), fmaT(-f, v.y, d.y));
              });
        }
      }
    }
  }
}

// --------------------------------------------------------------------------
// I3 with the transform field resident in shared memory (FP32, n <= 128: an
// n x (n+1) complex float field is at most 129 KB).  Same units, arithmetic
// and accumulation order as k_i3 (the line transforms are the same code, so
// results are bitwise identical); each convolution (row FFT, column psi'
// convolution, row IFFT) runs entirely on chip, global memory holds only the
// two shifted fields per block and the partial sums.
// --------------------------------------------------------------------------
constexpr int kThreadsI3Smem = 1024;

template <int n>
__global__ void __launch_bounds__(kThreadsI3Smem, 1) k_i3_smem(const I3Jobs<float> jobs, float2* ws,
                                                             const float2* __restrict__ gtw) {
  using C2 = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* G = tw + n;                       // [n][LS]
  float* psm = reinterpret_cast<float*>(G + n * (n + 1));   // psi'_j of the current unit, [n][n]
  constexpr int LS = n + 1, P = n * n;
  constexpr int kIter = (P + kThreadsI3Smem - 1) / kThreadsI3Smem;
  __shared__ unsigned char xmask[n];
  for (int pos = threadIdx.x; pos < n; pos += blockDim.x) {
    const int k = freq_of_pos<n>(pos);
    xmask[pos] = ((k < n / 4) || (k >= n - n / 4)) ? 1 : 0;
  }
  load_twiddles<n>(tw, gtw);
  C2* Sig = ws + (size_t)blockIdx.x * 3 * P;   // [2][P]
  for (int gunit = blockIdx.x; gunit < jobs.total; gunit += gridDim.x) {
    const I3Job<float>& jb = jobs.job[i3_job_of(jobs, gunit)];
    const int unit = gunit - jb.unit_begin;
    const int J = jb.J, M = jb.M, nmc = jb.nmc, mch = jb.mch;
    const C2* what = jb.what;
    const float* __restrict__ psip_s = jb.psip_s;
    const C2* __restrict__ phase = jb.phase;
    const int c = unit / (J * nmc);
    const int j = (unit / nmc) % J;
    const int mc = unit % nmc;
    C2* acc = jb.K3part + (size_t)unit * 2 * P;
    zero_fields(acc, 2 * P);
    {
      const float4* src = reinterpret_cast<const float4*>(psip_s + (size_t)j * P);
      float4* dst = reinterpret_cast<float4*>(psm);
      for (int i4 = threadIdx.x; i4 < P / 4; i4 += blockDim.x) dst[i4] = src[i4];
      __syncthreads();
    }
    const C2* wf = jb.wfine + (size_t)c * 2 * P;
    const int m0 = mc * mch, m1 = min(M, m0 + mch);
    for (int m = m0; m < m1; ++m) {
      const C2* px = phase + ((size_t)j * M + m) * 2 * n;
      const C2* py = px + n;
      for (int p = 0; p < 2; ++p) {
        const C2* in = what + ((size_t)c * 4 + p) * P;
        for (int idx = threadIdx.x; idx < P; idx += blockDim.x) {
          const int ix = idx / n, iy = idx % n;
          G[ix * LS + iy] = (xmask[ix] && xmask[iy]) ? cmul(in[idx], cmul(px[ix], py[iy])) : zero2<float>();
        }
        __syncthreads();
        fft_lines<n, 1, true>(G, n, 1, LS, tw);     // columns (along ix), input zero outside Xi
        fft_lines<n, 1, true>(G, n, LS, 1, tw);     // rows (along iy), zero outside the Xi columns
        C2* S = Sig + (size_t)p * P;
        for (int idx = threadIdx.x; idx < P; idx += blockDim.x) S[idx] = G[(idx / n) * LS + idx % n];
        __syncthreads();
      }
      for (int a = 0; a < 4; ++a) {
        const C2* wa = wf + (size_t)(a >> 1) * P;
        const C2* Sa = Sig + (size_t)(a >> 1) * P;
        const bool im = (a & 1) != 0;
        const float eta = (a == 0) ? 1.f : -1.f;
        for (int p = 0; p < 2; ++p) {
          const C2* __restrict__ Sp = Sig + (size_t)p * P;
          const C2* __restrict__ wv = wa;
          const C2* __restrict__ sa = Sa;
          C2* __restrict__ accp = acc + (size_t)p * P;
          // element loops with a compile-time trip count, unrolled so each thread keeps several
          // L2 loads in flight (one block per SM leaves few warps to hide their latency)
#pragma unroll 8
          for (int k = 0; k < kIter; ++k) {
            const int idx = threadIdx.x + k * kThreadsI3Smem;
            if (kIter * kThreadsI3Smem == P || idx < P) {
              const C2 z = wv[idx];
              G[(idx / n) * LS + idx % n] = cscale(Sp[idx], im ? z.y : z.x);
            }
          }
          __syncthreads();
          fft_lines<n, -1>(G, n, LS, 1, tw);                                           // rows forward
          fft_conv_lines<n>(G, n, 1, LS, tw, [&](int l, int pos) { return psm[pos * n + l]; });   // columns
          fft_lines<n, 1>(G, n, LS, 1, tw);                                            // rows inverse
#pragma unroll 8
          for (int k = 0; k < kIter; ++k) {
            const int idx = threadIdx.x + k * kThreadsI3Smem;
            if (kIter * kThreadsI3Smem == P || idx < P) {
              const C2 v = G[(idx / n) * LS + idx % n];
              const C2 s2 = sa[idx];
              const float f = eta * (im ? s2.y : s2.x);
              const C2 d = accp[idx];
              accp[idx] = mk2(fmaT(f, v.x, d.x), fmaT(f, v.y, d.y));
            }
          }
          __syncthreads();
        }
      }
    }
  }
}

template <int n>
constexpr bool use_i3_smem() {
  return n <= 128;
}

template <int n>
constexpr size_t i3_smem_bytes() {   // twiddles, the field (padded rows), psi'_j
  return (size_t)(n + n * (n + 1)) * sizeof(float2) + (size_t)n * n * sizeof(float);
}

#include "i3_fused.cuh"
#include "i3_staged_fused.cuh"

// Padded sizes with the fused shared-memory FP32 kernel (whole row tasks per thread for its shapes).
template <int n>
__host__ __device__ constexpr bool use_i3_fused() {
  return n == 64 || n == 96 || n == 128;
}
// Its launch shapes per size: (threads, blocks per SM, accumulation mode of k_i3_fused), and the
// default variant (I3 launch of 128 cells, J = M = 32, on a GB300: N = 32 28.6 ms for shape 0,
// 32.5 and 35.4 for shapes 1 and 2, 31.0 for k_i3_smem; N = 48 74.7 ms for k_i3_smem, 77.5, 81.7,
// 108.6 for the fused shapes; N = 64 100.9 ms for shape 0, 116.3, 112.1, 124.0 for k_i3_smem).
template <int n> struct FusedShapes;
template <> struct FusedShapes<64> {
  static constexpr int T0 = 512, B0 = 2, M0 = 1, T1 = 512, B1 = 2, M1 = 2, T2 = 256, B2 = 4, M2 = 2, DEFAULT = 0;
};
template <> struct FusedShapes<96> {
  static constexpr int T0 = 768, B0 = 1, M0 = 0, T1 = 768, B1 = 1, M1 = 2, T2 = 384, B2 = 2, M2 = 2, DEFAULT = 3;
};
template <> struct FusedShapes<128> {   // variant 4: k_i3_wl, 88.8 ms (shape 0: 101.1 ms)
  static constexpr int T0 = 512, B0 = 1, M0 = 1, T1 = 1024, B1 = 1, M1 = 2, T2 = 1024, B2 = 1, M2 = 0, DEFAULT = 4;
};

// --------------------------------------------------------------------------
// I3 on padded grids above 128 points in FP32 (n = 192, 256: one field is 288 or 512 KB, more
// than one block's shared memory).  A cluster of kI3Cluster CTAs works on one unit at a time:
// CTA r holds rows [r R, r R + R) of the transform field (R = n / kI3Cluster) for the row
// transforms and columns [r R, r R + R) for the column psi' convolution, with the angle's psi'
// columns in shared memory.  The transposes between the two go through the cluster's field in
// global memory, stored transposed (G'[ky][x]) so that the line stages load and store it directly,
// coalesced, ordered by cluster barriers; per cluster that field and the two shifted fields
// (3 n^2 complex values) stay L2-resident, where 152 independent units of the staged kernel
// (about 2.5 MB each) would not.  Same units and line transforms as k_i3.  Every CTA of a cluster
// runs the same loop trip counts, so every barrier is reached by all of them (hardware barriers,
// no spin waits).
// --------------------------------------------------------------------------
// Measured at N = 128 (32 cells, C[W] I3 launch), element passes through shared memory around
// every global access: 4 CTAs x 1024 threads 239.9 ms; 8 CTAs x 512 threads (two CTAs of
// different clusters per SM) 255.4 ms; the staged k_i3 294.5 ms.  With the line stages reading
// and writing the transposed field directly: 219.1 ms (1024 threads, mode 0 below), 192.4 ms
// (512 threads, mode 1).
constexpr int kI3Cluster = 4;             // CTAs per cluster
constexpr int kThreadsI3Cluster = 1024;   // threads per CTA of mode 0

template <int n>
__host__ __device__ constexpr bool use_i3_cluster() {
  return n > 128;
}

template <int n>
__host__ __device__ constexpr int i3_cluster_slab() {   // complex elements of the row / column slab
  constexpr int R = n / kI3Cluster;
  return R * (n + 1) > n * R ? R * (n + 1) : n * R;
}

template <int n>
constexpr size_t i3_cluster_smem_bytes() {   // twiddles (two orders), the slab, psi' columns
  return (size_t)(2 * n + i3_cluster_slab<n>()) * sizeof(float2) + (size_t)n * (n / kI3Cluster) * sizeof(float);
}

__device__ __forceinline__ int cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}
__device__ __forceinline__ int cluster_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return (int)r;
}
__device__ __forceinline__ int cluster_count() {
  unsigned r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return (int)r;
}
// All threads of all CTAs of the cluster.  The arrive has release and the wait acquire semantics at
// cluster scope, so global writes made before it by any thread of the cluster are visible after it
// to every thread of the cluster; reads of another CTA's writes use ld.global.cg (L2, the point of
// coherence) so that no stale L1 line can serve them.
__device__ __forceinline__ void cluster_sync_global() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The cluster kernel's launch shapes: NT threads per CTA and the accumulation mode.  MODE 0: loop a
// (outer), p (inner), each convolution's last stage adds eta_a S_a T into the unit's partial sum in
// global memory (read-modify-write per convolution).  MODE 1: loop p (outer), a (inner), the last
// stage accumulates over a in registers (each thread owns the same points in every convolution) and
// the partial sum is written once per (m, p); NT = R B / 2, so that every thread owns two row tasks.
template <int n>
constexpr int i3_cluster_threads(int mode) {
  return mode == 0 ? kThreadsI3Cluster : (n / kI3Cluster) * Split<n>::B / 2;
}

template <int n, int NT, int MODE>
__global__ void __cluster_dims__(kI3Cluster, 1, 1) __launch_bounds__(NT, 1)
    k_i3_cluster(const I3Jobs<float> jobs, float2* ws, const float2* __restrict__ gtw) {
  static_assert(n / kI3Cluster * n >= NT, "at least one element per thread in every phase");
  using C2 = float2;
  constexpr int R = n / kI3Cluster, LS = n + 1, P = n * n;
  constexpr int XC = (n / 2) / kI3Cluster;           // Xi columns per CTA in the shift transforms
  constexpr int A = Split<n>::A, B = Split<n>::B;
  constexpr int TA = (R * B + NT - 1) / NT;          // row tasks (r, t2) per thread in an A stage
  constexpr int TB = (R * A + NT - 1) / NT;          // tasks (r, k1) per thread in a B stage
  static_assert(MODE == 0 || R * B == 2 * NT, "register accumulation: two row tasks per thread");
  static_assert(n % kI3Cluster == 0 && (n / 2) % kI3Cluster == 0, "cluster split");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* twT = tw + n;                                  // twT[k1 B + t2] = tw[t2 A + k1] (t2-fastest lanes)
  C2* F = twT + n;                                   // [R][LS] row or line slab, [n][XC] shift column slab
  float* psl = reinterpret_cast<float*>(F + i3_cluster_slab<n>());   // psi'_j of this CTA's lines, [n][R]
  __shared__ int xcols[n];
  __shared__ unsigned char xmask[n];
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int pos = 0; pos < n; ++pos) {
      const int k = freq_of_pos<n>(pos);
      const bool in = (k < n / 4) || (k >= n - n / 4);
      xmask[pos] = in ? 1 : 0;
      if (in) xcols[cnt++] = pos;
    }
  }
  for (int pos = threadIdx.x; pos < n; pos += NT) twT[(pos % A) * B + pos / A] = gtw[pos];
  load_twiddles<n>(tw, gtw);
  const int tid = threadIdx.x;
  const int rank = cluster_rank();
  const int r0 = rank * R;                           // this CTA's first row / column
  C2* Gs = ws + (size_t)cluster_index() * 3 * P;     // the cluster's transform field
  C2* Sig = Gs + P;                                  // the two shifted pairs
  // One Psi'_j convolution of the field load(idx) (idx = r n + y, r a row of this CTA), with the
  // last stage's results handed to epi(i, t1, idx, v) (i: the thread's row task, t1: its element).
  // Between the passes the cluster's field is stored transposed, Gs'[ky][x] (ky in the row
  // transform's permuted order): the row passes reach it from stage B (lanes = consecutive rows of
  // this CTA) and the line pass from stage A (contiguous in x), so every global access is inside a
  // line stage and coalesced.
  auto convolve = [&](auto load, auto epi) {
#pragma unroll
    for (int i = 0; i < TA; ++i) {                   // forward rows: stage A loads the product
      const int task = tid + i * NT;
      if (TA * NT == R * B || task < R * B) {
        const int r = task / B, t2 = task % B;
        C2 v[A];
#pragma unroll
        for (int t1 = 0; t1 < A; ++t1) v[t1] = load(r * n + B * t1 + t2);
        dft<A, -1>(v);
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], twT[k1 * B + t2]);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) F[r * LS + B * k1 + t2] = v[k1];
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TB; ++i) {
      const int task = tid + i * NT;
      if (TB * NT == R * A || task < R * A) {
        const int r = task % R, k1 = task / R;
        C2 b[B];
#pragma unroll
        for (int t = 0; t < B; ++t) b[t] = F[r * LS + B * k1 + t];
        dft<B, -1>(b);
#pragma unroll
        for (int t = 0; t < B; ++t) Gs[(size_t)(B * k1 + t) * n + r0 + r] = b[t];
      }
    }
    cluster_sync_global();                           // all rows transformed
    // psi' convolution along x on this CTA's lines ky in [r0, r0 + R)
#pragma unroll
    for (int i = 0; i < TA; ++i) {
      const int task = tid + i * NT;
      if (TA * NT == R * B || task < R * B) {
        const int cc = task / B, t2 = task % B;
        C2 v[A];
#pragma unroll
        for (int t1 = 0; t1 < A; ++t1) v[t1] = __ldcg(&Gs[(size_t)(r0 + cc) * n + B * t1 + t2]);
        dft<A, -1>(v);
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], twT[k1 * B + t2]);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) F[cc * LS + B * k1 + t2] = v[k1];
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TB; ++i) {
      const int task = tid + i * NT;
      if (TB * NT == R * A || task < R * A) {
        const int cc = task % R, k1 = task / R;
        C2 b[B];
#pragma unroll
        for (int t = 0; t < B; ++t) b[t] = F[cc * LS + B * k1 + t];
        dft<B, -1>(b);
        float sc[B];
#pragma unroll
        for (int t = 0; t < B; ++t) sc[t] = psl[(B * k1 + t) * R + cc];
        dft_scaled<B, 1>(b, sc);
#pragma unroll
        for (int t = 0; t < B; ++t) F[cc * LS + B * k1 + t] = b[t];
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TA; ++i) {
      const int task = tid + i * NT;
      if (TA * NT == R * B || task < R * B) {
        const int cc = task / B, t2 = task % B;
        C2 v[A];
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) v[k1] = F[cc * LS + B * k1 + t2];
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1) v[k1] = cmulc(v[k1], twT[k1 * B + t2]);
        dft<A, 1>(v);
#pragma unroll
        for (int t1 = 0; t1 < A; ++t1) Gs[(size_t)(r0 + cc) * n + B * t1 + t2] = v[t1];
      }
    }
    cluster_sync_global();                           // all lines convolved
    // inverse rows on this CTA's rows: stage B loads, stage A hands its results to the epilogue
#pragma unroll
    for (int i = 0; i < TB; ++i) {
      const int task = tid + i * NT;
      if (TB * NT == R * A || task < R * A) {
        const int r = task % R, k1 = task / R;
        C2 b[B];
#pragma unroll
        for (int t = 0; t < B; ++t) b[t] = __ldcg(&Gs[(size_t)(B * k1 + t) * n + r0 + r]);
        dft<B, 1>(b);
#pragma unroll
        for (int t = 0; t < B; ++t) F[r * LS + B * k1 + t] = b[t];
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TA; ++i) {
      const int task = tid + i * NT;
      if (TA * NT == R * B || task < R * B) {
        const int r = task / B, t2 = task % B;
        C2 v[A];
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) v[k1] = F[r * LS + B * k1 + t2];
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1) v[k1] = cmulc(v[k1], twT[k1 * B + t2]);
        dft<A, 1>(v);
#pragma unroll
        for (int t1 = 0; t1 < A; ++t1) epi(i, t1, r * n + B * t1 + t2, v[t1]);
      }
    }
    __syncthreads();
  };
  for (int gunit = cluster_index(); gunit < jobs.total; gunit += cluster_count()) {
    const I3Job<float>& jb = jobs.job[i3_job_of(jobs, gunit)];
    const int unit = gunit - jb.unit_begin;
    const int J = jb.J, M = jb.M, nmc = jb.nmc, mch = jb.mch;
    const C2* what = jb.what;
    const C2* __restrict__ phase = jb.phase;
    const int c = unit / (J * nmc);
    const int j = (unit / nmc) % J;
    const int mc = unit % nmc;
    C2* acc = jb.K3part + (size_t)unit * 2 * P;
    if (MODE == 0) {
      #pragma unroll 1
      for (int idx = tid; idx < R * n; idx += NT) {
        acc[(size_t)r0 * n + idx] = zero2<float>();
        acc[P + (size_t)r0 * n + idx] = zero2<float>();
      }
    }
    const float* __restrict__ psp = jb.psip_s + (size_t)j * P;
    #pragma unroll 1
    for (int idx = tid; idx < n * R; idx += NT) psl[idx] = psp[(idx / R) * n + r0 + idx % R];
    __syncthreads();
    const C2* wf = jb.wfine + (size_t)c * 2 * P;
    const int m0 = mc * mch, m1 = min(M, m0 + mch);
    for (int m = m0; m < m1; ++m) {
      const C2* px = phase + ((size_t)j * M + m) * 2 * n;
      const C2* py = px + n;
      cluster_sync_global();                         // the previous m's (or unit's) Sig and Gs are read
      // shifted fields, column transforms over this CTA's share of the Xi columns
      for (int p = 0; p < 2; ++p) {
        const C2* in = what + ((size_t)c * 4 + p) * P;
        C2* S = Sig + (size_t)p * P;
        #pragma unroll 1
        for (int idx = tid; idx < n * XC; idx += NT) {
          const int ix = idx / XC, cc = idx % XC, iy = xcols[rank * XC + cc];
          F[idx] = xmask[ix] ? cmul(in[ix * n + iy], cmul(px[ix], py[iy])) : zero2<float>();
        }
        __syncthreads();
        fft_lines<n, 1, true>(F, XC, 1, XC, tw);
        #pragma unroll 1
        for (int idx = tid; idx < n * XC; idx += NT) {
          const int ix = idx / XC, cc = idx % XC;
          S[ix * n + xcols[rank * XC + cc]] = F[idx];
        }
        __syncthreads();
      }
      cluster_sync_global();                         // the Xi columns of both shifted fields are complete
      // row transforms over this CTA's rows (columns outside Xi are zero)
      for (int p = 0; p < 2; ++p) {
        C2* S = Sig + (size_t)p * P + (size_t)r0 * n;
        #pragma unroll 1
        #pragma unroll 1
      for (int idx = tid; idx < R * n; idx += NT) {
          const int r = idx / n, iy = idx % n;
          F[r * LS + iy] = xmask[iy] ? __ldcg(&S[idx]) : zero2<float>();
        }
        __syncthreads();
        fft_lines<n, 1, true>(F, R, LS, 1, tw);
        #pragma unroll 1
        for (int idx = tid; idx < R * n; idx += NT) S[idx] = F[(idx / n) * LS + idx % n];
        __syncthreads();
      }
      // from here on this CTA reads only its own rows of the shifted fields
      if constexpr (MODE == 0) {
        for (int a = 0; a < 4; ++a) {
          // component im of the fine pair and of the shifted pair, loaded as single floats
          const int im = a & 1;
          const float* wa = reinterpret_cast<const float*>(wf + (size_t)(a >> 1) * P + (size_t)r0 * n) + im;
          const float* Sa = reinterpret_cast<const float*>(Sig + (size_t)(a >> 1) * P + (size_t)r0 * n) + im;
          const float eta = (a == 0) ? 1.f : -1.f;
          for (int p = 0; p < 2; ++p) {
            const C2* Sp = Sig + (size_t)p * P + (size_t)r0 * n;
            C2* accp = acc + (size_t)p * P + (size_t)r0 * n;
            convolve([&](int idx) { return cscale(Sp[idx], wa[2 * idx]); },
                     [&](int, int, int idx, C2 v) {
                       const float f = eta * Sa[2 * idx];
                       const C2 d = accp[idx];
                       accp[idx] = mk2(fmaT(f, v.x, d.x), fmaT(f, v.y, d.y));
                     });
          }
        }
      } else {
        const bool first_m = (m == m0);
        for (int p = 0; p < 2; ++p) {
          const C2* Sp = Sig + (size_t)p * P + (size_t)r0 * n;
          C2* accp = acc + (size_t)p * P + (size_t)r0 * n;
          C2 racc[TA][A];
          for (int a = 0; a < 4; ++a) {
            const C2* wa = wf + (size_t)(a >> 1) * P + (size_t)r0 * n;
            const C2* Sa = Sig + (size_t)(a >> 1) * P + (size_t)r0 * n;
            const bool im = (a & 1) != 0;
            const float eta = (a == 0) ? 1.f : -1.f;
            convolve(
                [&](int idx) {
                  const C2 z = wa[idx];
                  return cscale(Sp[idx], im ? z.y : z.x);
                },
                [&](int i, int t1, int idx, C2 v) {
                  const C2 sv = Sa[idx];
                  const float f = eta * (im ? sv.y : sv.x);
                  if (a == 0) racc[i][t1] = mk2(f * v.x, f * v.y);
                  else racc[i][t1] = mk2(fmaT(f, v.x, racc[i][t1].x), fmaT(f, v.y, racc[i][t1].y));
                });
          }
#pragma unroll
          for (int i = 0; i < TA; ++i) {
            const int task = tid + i * NT, r = task / B, t2 = task % B;
#pragma unroll
            for (int t1 = 0; t1 < A; ++t1) {
              const int idx = r * n + B * t1 + t2;
              accp[idx] = first_m ? racc[i][t1] : cadd(accp[idx], racc[i][t1]);
            }
          }
        }
      }
    }
  }
}

// --------------------------------------------------------------------------
// Assemble C on the fine grid from D, K2, K3, K4 (Pauli formulas of Sec. 3.1),
// then FFT, cut to Xi (without the -N/2 line), inverse FFT and sample the
// coarse nodes.  One block per cell.  The K3 partial sums are added in FP64.
// --------------------------------------------------------------------------
template <int n, class T>
__global__ void __launch_bounds__(kThreads) k_assemble(const typename Vec2Of<T>::type* wfine,
                                                       const typename Vec2Of<T>::type* Dacc, const T* K2acc,
                                                       const typename Vec2Of<T>::type* K4acc,
                                                       const typename Vec2Of<T>::type* K3part, int nparts,
                                                       typename Vec2Of<T>::type* ws,
                                                       const typename Vec2Of<T>::type* __restrict__ gtw,
                                                       double* cout) {
  using C2 = typename Vec2Of<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* sm = tw + n;
  load_twiddles<n>(tw, gtw);
  constexpr int N = n / 2, P = n * n;
  const int c = blockIdx.x;
  C2* slot = ws + (size_t)blockIdx.x * 6 * P;
  C2* B0 = slot;
  // D pairs -> slot[0], slot[1]; K4 pairs -> slot[2], slot[3] (inverse 2-D transforms)
  for (int f = 0; f < 4; ++f) {
    const C2* in = (f < 2) ? (Dacc + ((size_t)c * 2 + f) * P) : (K4acc + ((size_t)c * 2 + (f - 2)) * P);
    C2* out = slot + (size_t)f * P;
    col_pass<n, 1, false, 0>(
        sm, tw, [&](int ix, int iy) { return in[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) { out[ix * n + iy] = v; });
    row_pass<n, 1, false, 0>(
        sm, tw, [&](int ix, int iy) { return out[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) { out[ix * n + iy] = v; });
  }
  const C2* parts = K3part + (size_t)c * nparts * 2 * P;
  const C2* wf0 = wfine + (size_t)c * 2 * P;
  const C2* wf1 = wf0 + P;
  const T* K2 = K2acc + (size_t)c * P;
  const double tp = 2.0 * kPi;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    double k3ax = 0, k3ay = 0, k3bx = 0, k3by = 0;
    for (int u = 0; u < nparts; ++u) {
      const C2 x = parts[(size_t)u * 2 * P + i];
      const C2 y = parts[(size_t)u * 2 * P + P + i];
      k3ax += (double)x.x; k3ay += (double)x.y; k3bx += (double)y.x; k3by += (double)y.y;
    }
    const double w0 = wf0[i].x, w1 = wf0[i].y, w2 = wf1[i].x, w3 = wf1[i].y;
    const double D1 = slot[i].x, D2 = slot[i].y, D3 = slot[P + i].x;
    const double K40 = slot[2 * P + i].x, K41 = -(double)slot[2 * P + i].y;   // eta_b applied
    const double K42 = -(double)slot[3 * P + i].x, K43 = -(double)slot[3 * P + i].y;
    const double K30 = k3ax, K31 = -k3ay, K32 = -k3bx, K33 = -k3by;
    const double k2 = K2[i];
    const double C0 = tp * (k2 * (1.0 - w0) - K30 + w0 * K40 + w1 * K41 + w2 * K42 + w3 * K43);
    const double C1 = -2.0 * (D2 * w3 - D3 * w2) + tp * (-k2 * w1 - K31 + w0 * K41 + K40 * w1);
    const double C2v = -2.0 * (D3 * w1 - D1 * w3) + tp * (-k2 * w2 - K32 + w0 * K42 + K40 * w2);
    const double C3 = -2.0 * (D1 * w2 - D2 * w1) + tp * (-k2 * w3 - K33 + w0 * K43 + K40 * w3);
    B0[i] = mk2((T)C0, (T)C1);
    B0[P + i] = mk2((T)C2v, (T)C3);
  }
  __syncthreads();
  const T invP = (T)(1.0 / (double)P);
  double* co = cout + (size_t)c * 4 * N * N;
  C2* H = slot + 2 * P;
  for (int p = 0; p < 2; ++p) {
    const C2* F = B0 + (size_t)p * P;
    row_pass<n, -1, false, 0>(
        sm, tw, [&](int ix, int iy) { return F[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) { H[ix * n + iy] = v; });
    col_pass<n, -1, true, 1>(
        sm, tw, [&](int ix, int iy) { return H[ix * n + iy]; },
        [&](int ix, int iy, C2 v) {
          const bool keep = in_xi<n>(freq_of_pos<n>(ix)) && in_xi<n>(freq_of_pos<n>(iy));
          return keep ? cscale(v, invP) : zero2<T>();
        },
        [&](int ix, int iy, C2 v) { H[ix * n + iy] = v; });
    row_pass<n, 1, false, 0>(
        sm, tw, [&](int ix, int iy) { return H[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) {
          if (((ix | iy) & 1) == 0) {
            const int i = ix >> 1, j = iy >> 1;
            co[((2 * p) * N + i) * N + j] = (double)v.x;
            co[((2 * p + 1) * N + i) * N + j] = (double)v.y;
          }
        });
  }
}

}  // namespace

template <int n, class T>
size_t smem_bytes() {
  using C2 = typename Vec2Of<T>::type;
  return (size_t)(n + Chunk<n, sizeof(C2)>::SMEM_ELEMS) * sizeof(C2);
}

template <int n, class T, int CB>
size_t i3_staged_smem_bytes() {
  using C2 = typename Vec2Of<T>::type;
  return (size_t)(n + Chunk<n, sizeof(C2), CB>::SMEM_ELEMS) * sizeof(C2);
}

// Launch variants of the I3 kernel for padded size n and transform type T: the shapes the
// autotuner chooses among (i3_default_variant gives the one a new handle starts with).
//   FP64 (every size): the staged kernel as (threads, chunk bytes, blocks per SM)
//     0: (256, 64 KB, 3)   1: (128, 32 KB, 6);  k_i3_sf 2: (256, 64 KB, 3)   3: (128, 32 KB, 6)
//   FP32, n = 64, 96, 128: 0, 1, 2: the fused shared-memory kernel in the FusedShapes<n> shapes,
//     3: k_i3_smem (1024 threads, element passes through shared memory)
//   FP32, n <= 32: k_i3_smem;  FP32, n > 128: the cluster kernel, 0: 1024 threads per CTA with a
//     partial-sum update per convolution, 1: two row tasks per thread with register accumulation.
struct I3Launch {
  const void* fn = nullptr;
  int threads = 0;
  size_t smem = 0;
  bool cluster = false;
  const char* name = "";
};

template <int n, class T>
constexpr int i3_nvariants() {
  if constexpr (std::is_same<T, float>::value) {
    if constexpr (use_i3_cluster<n>()) return 2;
    else if constexpr (use_i3_fused<n>()) return n == kWlN ? 5 : 4;   // 128 points: + k_i3_wl
    else return 1;
  } else {
    return 4;
  }
}

template <int n, class T>
I3Launch i3_variant(int v) {
  I3Launch l;
  if constexpr (std::is_same<T, float>::value && use_i3_cluster<n>()) {
    constexpr int NT1 = i3_cluster_threads<n>(1);
    if (v == 1)
      l = {(const void*)k_i3_cluster<n, NT1, 1>, NT1, i3_cluster_smem_bytes<n>(), true,
           n == 256 ? "cluster of 4 CTAs x 512 threads, register accumulation"
                    : "cluster of 4 CTAs x 384 threads, register accumulation"};
    else
      l = {(const void*)k_i3_cluster<n, kThreadsI3Cluster, 0>, kThreadsI3Cluster, i3_cluster_smem_bytes<n>(), true,
           "cluster of 4 CTAs x 1024 threads"};
  } else if constexpr (std::is_same<T, float>::value && use_i3_fused<n>()) {
    using S = FusedShapes<n>;
    constexpr const char* names[3] = {"fused, per-convolution partial sums", "fused, register accumulation",
                                      "fused, paired w with register accumulation"};
    if (v == 0)
      l = {(const void*)k_i3_fused<n, S::T0, S::B0, S::M0>, S::T0, i3_fused_smem_bytes<n>(), false, names[S::M0]};
    else if (v == 1)
      l = {(const void*)k_i3_fused<n, S::T1, S::B1, S::M1>, S::T1, i3_fused_smem_bytes<n>(), false, names[S::M1]};
    else if (v == 2)
      l = {(const void*)k_i3_fused<n, S::T2, S::B2, S::M2>, S::T2, i3_fused_smem_bytes<n>(), false, names[S::M2]};
    else if (v == 4 && n == kWlN)
      l = {(const void*)k_i3_wl, kWlThreads, i3_wl_smem_bytes(), false,
           "fused, warp-local passes, register accumulation"};
    else
      l = {(const void*)k_i3_smem<n>, kThreadsI3Smem, i3_smem_bytes<n>(), false, "shared-memory, 1024 threads"};
  } else if constexpr (std::is_same<T, float>::value) {
    l = {(const void*)k_i3_smem<n>, kThreadsI3Smem, i3_smem_bytes<n>(), false, "shared-memory, 1024 threads"};
  } else {
    if (v == 1)
      l = {(const void*)k_i3<n, T, 128, 32768, 6>, 128, i3_staged_smem_bytes<n, T, 32768>(), false,
           "staged, 128 threads, 32 KB chunks"};
    else if (v == 2)
      l = {(const void*)k_i3_sf<n, T, 256, 65536, 3>, 256, i3_sf_smem_bytes<n, T, 65536>(), false,
           "staged with fused loads and stores, 256 threads, 64 KB chunks"};
    else if (v == 3)
      l = {(const void*)k_i3_sf<n, T, 128, 32768, 6>, 128, i3_sf_smem_bytes<n, T, 32768>(), false,
           "staged with fused loads and stores, 128 threads, 32 KB chunks"};
    else
      l = {(const void*)k_i3<n, T, 256, 65536, 3>, 256, i3_staged_smem_bytes<n, T, 65536>(), false,
           "staged, 256 threads, 64 KB chunks"};
  }
  return l;
}

template <int n, class T>
void set_smem_attributes() {
  static unsigned long long done = 0;
  if (!first_on_device(done)) return;
  const int sm = (int)smem_bytes<n, T>();
  cudaFuncSetAttribute(k_prep<n, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_i1<n, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_i24<n, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_assemble<n, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  for (int v = 0; v < i3_nvariants<n, T>(); ++v) {
    const I3Launch l = i3_variant<n, T>(v);
    cudaFuncSetAttribute(l.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.smem);
  }
}

// Clusters of the cluster variant v of k_i3_cluster<n> that can be resident at once on the current
// device (cached per device and variant).
template <int n>
int i3_max_clusters(int v) {
  static int cached[64][2] = {};
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  v = (v == 1) ? 1 : 0;
  if (cached[dev & 63][v] > 0) return cached[dev & 63][v];
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const I3Launch l = i3_variant<n, float>(v);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kI3Cluster * (nsm > 0 ? nsm : 1));
  cfg.blockDim = dim3(l.threads);
  cfg.dynamicSmemBytes = l.smem;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, l.fn, &cfg) != cudaSuccess || ncl < 1) {
    cudaGetLastError();
    ncl = (nsm > 0 ? nsm : 1) / kI3Cluster;
  }
  cached[dev & 63][v] = ncl < 1 ? 1 : ncl;
  return cached[dev & 63][v];
}

// Resident blocks per SM of an I3 variant (at least 1).
template <int n, class T>
int i3_blocks_per_sm(int v) {
  set_smem_attributes<n, T>();
  if (v < 0 || v >= i3_nvariants<n, T>()) v = 0;
  const I3Launch l = i3_variant<n, T>(v);
  int b = 0;
  if constexpr (std::is_same<T, float>::value && use_i3_cluster<n>()) {
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    b = (i3_max_clusters<n>(v) * kI3Cluster + nsm - 1) / (nsm > 0 ? nsm : 1);
  } else if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, l.fn, l.threads, l.smem) != cudaSuccess) {
    cudaGetLastError();
    b = 1;
  }
  return b < 1 ? 1 : b;
}

template <int n, class T>
int i3_variant_count() {
  return i3_nvariants<n, T>();
}

// The variant a new handle starts with (the fastest measured on a GB300 for this size).  FP64, I3
// launch in ms for variants 0..3 (J = M = 32): N = 16, 128 cells 136.8 136.2 132.9 129.4;
// N = 32, 128 cells 652.2 640.5 625.3 630.4; N = 48, 64 cells 868.4 886.2 860.3 879.5; N = 64,
// 32 cells 752.1 760.2 732.5 742.2; N = 128, 8 cells 897.0 902.9 885.5 901.9.
// FP32 cluster kernel (I3 launch, J = M = 32): N = 128, 32 cells 219.1 ms (variant 0), 192.4 ms
// (variant 1); N = 96, 64 cells 217.6 and 208.9 ms.
template <int n, class T>
int i3_default_variant() {
  if constexpr (std::is_same<T, float>::value && use_i3_fused<n>()) return FusedShapes<n>::DEFAULT;
  else if constexpr (std::is_same<T, float>::value && use_i3_cluster<n>()) return 1;
  else if constexpr (std::is_same<T, double>::value) return 2;
  else return 0;
}

// Work units (or, for the cluster form, clusters) a launch of variant v with `grid` blocks and
// `total` units processes at once: the persistent grid the launcher uses (see i3_group_n).  Unit u
// goes to block (cluster) u mod this number.
template <int n, class T>
int i3_variant_concurrency(int v, int grid, int total) {
  if (v < 0 || v >= i3_nvariants<n, T>()) v = 0;
  int g = total < grid ? total : grid;
  if constexpr (std::is_same<T, float>::value && use_i3_cluster<n>()) {
    int ncl = grid / kI3Cluster;
    const int cmax = i3_max_clusters<n>(v);
    if (ncl > cmax) ncl = cmax;
    if (ncl > total) ncl = total;
    g = ncl < 1 ? 1 : ncl;
  } else {
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int gmax = nsm * i3_blocks_per_sm<n, T>(v);
    if (g > gmax) g = gmax;
  }
  return g < 1 ? 1 : g;
}

template <int n, class T>
const char* i3_variant_name(int v) {
  if (v < 0 || v >= i3_nvariants<n, T>()) return nullptr;
  return i3_variant<n, T>(v).name;
}

// I1 and I2/I4 of ncells cells over (cell, angle chunk) blocks (cw.nch chunks per cell), then the
// chunk partials summed into Dacc, K2acc, K4acc (skipped with one chunk: the kernels write there).
template <int n, class T>
cudaError_t per_cell_terms(const Tables& t, CollisionWork& cw, typename Vec2Of<T>::type* ws, int ncells,
                           cudaStream_t s, long long& launches, KernelTimer* tm) {
  using C2 = typename Vec2Of<T>::type;
  const TabPtrs<T> tb = tab_ptrs<T>(t);
  const C2* what = (const C2*)cw.what;
  const C2* wfine = (const C2*)cw.wfine;
  const size_t sm = smem_bytes<n, T>();
  const int nch = cw.nch < 1 ? 1 : cw.nch;
  C2* D = (C2*)(nch > 1 ? cw.Dpart : cw.Dacc);
  T* K2 = (T*)(nch > 1 ? cw.K2part : cw.K2acc);
  C2* K4 = (C2*)(nch > 1 ? cw.K4part : cw.K4acc);
  if (tm) tm->begin(KG_I1, s);
  k_i1<n, T><<<ncells * nch, kThreads, sm, s>>>(what, wfine, D, ws, tb.tw, tb.phip, tb.Ktab, t.J, nch);
  if (tm) tm->end(s);
  if (tm) tm->begin(KG_I24, s);
  k_i24<n, T><<<ncells * nch, kThreads, sm, s>>>(what, wfine, K2, K4, ws, tb.tw, tb.psi, t.J, nch);
  if (nch > 1) {
    k_reduce_chunks<T><<<(ncells * 5 * n * n + kThreads * 8 - 1) / (kThreads * 8), kThreads, 0, s>>>(
        (const T*)cw.Dpart, (const T*)cw.K2part, (const T*)cw.K4part, (T*)cw.Dacc, (T*)cw.K2acc, (T*)cw.K4acc, nch,
        ncells, (size_t)n * n);
    ++launches;
  }
  if (tm) tm->end(s);
  launches += 2;
  return cudaGetLastError();
}

// The collision operator in three parts: the per-cell terms before I3 (prep, I1, I2/I4), the I3
// launch (a work queue over the units of one or several simulations of the same padded size), and
// the per-cell assembly.  collide_batch_n runs all three for one simulation.
template <int n, class T>
cudaError_t collide_pre_n(const Tables& t, CollisionWork& cw, const double* w, int ncells, cudaStream_t s,
                          long long& launches, KernelTimer* tm) {
  using C2 = typename Vec2Of<T>::type;
  set_smem_attributes<n, T>();
  const TabPtrs<T> tb = tab_ptrs<T>(t);
  C2* what = (C2*)cw.what;
  C2* wfine = (C2*)cw.wfine;
  C2* ws = (C2*)cw.ws;
  const size_t sm = smem_bytes<n, T>();
  auto begin = [&](int g) { if (tm) tm->begin(g, s); };
  auto end = [&]() { if (tm) tm->end(s); };
  begin(KG_PREP);
  k_prep<n, T><<<ncells, kThreads, sm, s>>>(w, what, wfine, ws, tb.tw);
  end();
  cudaError_t e = per_cell_terms<n, T>(t, cw, ws, ncells, s, launches, tm);
  if (e != cudaSuccess) return e;
  ++launches;
  return cudaGetLastError();
}

template <int n, class T>
I3Job<T> i3_job(const Tables& t, const CollisionWork& cw, int ncells, int unit_begin) {
  using C2 = typename Vec2Of<T>::type;
  const TabPtrs<T> tb = tab_ptrs<T>(t);
  I3Job<T> jb;
  jb.what = (const C2*)cw.what;
  jb.wfine = (const C2*)cw.wfine;
  jb.K3part = (C2*)cw.K3part;
  jb.psip_s = tb.psip_s;
  jb.phase = tb.phase;
  jb.J = t.J;
  jb.M = t.M;
  jb.nmc = cw.nmc;
  jb.mch = cw.mch;
  jb.unit_begin = unit_begin;
  jb.nunits = ncells * t.J * cw.nmc;
  return jb;
}

// I3 over the units of njobs simulations (same n and precision, njobs <= kMaxI3Jobs); ws must hold
// 3 (2N)^2 complex values for each of `grid` blocks (the cluster form uses one such slot per cluster
// of kI3Cluster blocks).
template <int n, class T>
cudaError_t i3_group_n(const Tables* const* tabs, const CollisionWork* const* cws, const int* ncells, int njobs,
                       void* ws, int grid, cudaStream_t s, long long& launches, int max_units) {
  using C2 = typename Vec2Of<T>::type;
  if (njobs < 1 || njobs > kMaxI3Jobs) return cudaErrorInvalidValue;
  set_smem_attributes<n, T>();
  I3Jobs<T> jobs;
  jobs.njobs = njobs;
  int total = 0;
  for (int k = 0; k < njobs; ++k) {
    jobs.job[k] = i3_job<n, T>(*tabs[k], *cws[k], ncells[k], total);
    total += jobs.job[k].nunits;
  }
  jobs.total = (max_units > 0 && max_units < total) ? max_units : total;   // a prefix (autotuner samples)
  total = jobs.total;
  if (total == 0) return cudaSuccess;
  const TabPtrs<T> tb = tab_ptrs<T>(*tabs[0]);
  int v = cws[0]->i3_variant;
  if (v < 0 || v >= i3_nvariants<n, T>()) v = 0;
  const I3Launch l = i3_variant<n, T>(v);
  int g = total < grid ? total : grid;
  if constexpr (std::is_same<T, float>::value && use_i3_cluster<n>()) {
    int ncl = grid / kI3Cluster;
    const int cmax = i3_max_clusters<n>(v);
    if (ncl > cmax) ncl = cmax;
    if (ncl > total) ncl = total;
    if (ncl < 1) ncl = 1;
    g = ncl * kI3Cluster;
  } else {
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int gmax = nsm * i3_blocks_per_sm<n, T>(v);      // persistent: never more than fit at once
    if (g > gmax) g = gmax;
  }
  C2* wsp = (C2*)ws;
  const C2* twp = tb.tw;
  void* args[] = {(void*)&jobs, (void*)&wsp, (void*)&twp};
  cudaError_t e = cudaLaunchKernel(l.fn, dim3(g), dim3(l.threads), args, l.smem, s);
  ++launches;
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int n, class T>
cudaError_t collide_post_n(const Tables& t, CollisionWork& cw, double* c, int ncells, cudaStream_t s,
                           long long& launches, KernelTimer* tm) {
  using C2 = typename Vec2Of<T>::type;
  set_smem_attributes<n, T>();
  const TabPtrs<T> tb = tab_ptrs<T>(t);
  if (tm) tm->begin(KG_ASSEMBLE, s);
  k_assemble<n, T><<<ncells, kThreads, smem_bytes<n, T>(), s>>>((C2*)cw.wfine, (C2*)cw.Dacc, (T*)cw.K2acc,
                                                                (C2*)cw.K4acc, (C2*)cw.K3part, t.J * cw.nmc,
                                                                (C2*)cw.ws, tb.tw, c);
  if (tm) tm->end(s);
  ++launches;
  return cudaGetLastError();
}

template <int n, class T>
cudaError_t collide_batch_n(const Tables& t, CollisionWork& cw, const double* w, double* c, int ncells,
                            cudaStream_t s, long long& launches, KernelTimer* tm) {
  cudaError_t e = collide_pre_n<n, T>(t, cw, w, ncells, s, launches, tm);
  if (e != cudaSuccess) return e;
  const Tables* tp = &t;
  const CollisionWork* cp = &cw;
  if (tm) tm->begin(KG_I3, s);
  e = i3_group_n<n, T>(&tp, &cp, &ncells, 1, cw.ws, cw.grid_i3, s, launches, 0);
  if (tm) tm->end(s);
  if (e != cudaSuccess) return e;
  return collide_post_n<n, T>(t, cw, c, ncells, s, launches, tm);
}

}  // namespace qbe
