// Vector-Jacobian product of the discrete collision operator: given a
// cotangent lambda of C[W] on the velocity grid, the gradient of <lambda, C[W]>
// with respect to W.  Used by the adjoint of the split time step.
//
// Every dependence of C on W goes through the fine-grid interpolant w^fine
// = I(W) (band-limited to Xi), so the kernels accumulate a fine-grid cotangent
// nu_a of each Pauli component and finish with I^T nu = 4 E P nu (band-limit
// to Xi, sample the coarse nodes; E samples the even fine nodes).  The
// transposes used, all exact for the discrete operators:
//   * a Fourier multiplier m(sigma) transposes to m(-sigma): even real
//     multipliers (psi, psi') are self-adjoint; odd ones are handled as the
//     real operators "multiply by i phi'" and "multiply by i K", which are
//     antisymmetric;
//   * the Hu-Ying shift S (multiplier e^{i alpha.sigma}) transposes to the
//     shift back (conjugate phase);
//   * the projection of C_fine to Xi is self-adjoint; sampling transposes to
//     zero interleaving.
// With lambda band-limited by that projection, the only frequency at which
// these statements need care (the unpaired -N line of the padded grid) never
// reaches Xi.  Terms (as in the forward kernels, raw accumulators):
//   D_b = -K'(f A_{j'} w_b),   K2 = 2 (pi/J) sum eta_a F_{a,j} F_{a,j+J/2},
//   K4raw_b = (pi/J) sum_j Psi_j(f F_{b,j+J/2}),
//   K3raw_b = sum_{j,m,a} eta_a S(w_a) Psi'_j(w_a S(w_b)),   f = 2 w0 - 1.
#pragma once

#include "collision_kernels.cuh"

namespace qbe {

namespace {

template <class C2>
__device__ __forceinline__ C2 mul_i(C2 v, typename RealOf<C2>::type s) {   // v * (i s)
  return mk2(-s * v.y, s * v.x);
}

// --------------------------------------------------------------------------
// Seed: mu = P(E^T lambda) on the fine grid, the forward D and K4 fields, and
// the transpose of the pointwise Pauli assembly.  One block per cell.
// Outputs: nu[c][2] (direct cotangent of the w pairs), nuf[c] (cotangent of
// f = 2 w0 - 1), muD[c][2] (pairs (D1,D2),(D3,-)), muK2[c], mu4[c][2] (raw K4
// pairs), mu3[c][2] (raw K3 pairs).
// --------------------------------------------------------------------------
template <int n, class T>
__global__ void __launch_bounds__(kThreads) k_vjp_seed(
    const double* __restrict__ lam, const typename Vec2Of<T>::type* wfine, const typename Vec2Of<T>::type* Dacc,
    const T* K2acc, const typename Vec2Of<T>::type* K4acc, typename Vec2Of<T>::type* nu, T* nuf,
    typename Vec2Of<T>::type* muD, T* muK2, typename Vec2Of<T>::type* mu4, typename Vec2Of<T>::type* mu3,
    typename Vec2Of<T>::type* ws, const typename Vec2Of<T>::type* __restrict__ gtw) {
  using C2 = typename Vec2Of<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* sm = tw + n;
  load_twiddles<n>(tw, gtw);
  constexpr int N = n / 2, P = n * n;
  const int c = blockIdx.x;
  C2* slot = ws + (size_t)blockIdx.x * 6 * P;
  C2* MU = slot;             // [2] cotangent of C_fine pairs (0,1), (2,3)
  C2* DK = slot + 2 * P;     // [4] D pairs, K4 pairs in real space
  const double* lc = lam + (size_t)c * 4 * N * N;
  const T invP = (T)(1.0 / (double)P);
  for (int p = 0; p < 2; ++p) {
    C2* M = MU + (size_t)p * P;
    row_pass<n, -1, false, 0>(
        sm, tw,
        [&](int ix, int iy) {
          if ((ix | iy) & 1) return zero2<T>();
          const int i = ix >> 1, j = iy >> 1;
          return mk2((T)lc[((2 * p) * N + i) * N + j], (T)lc[((2 * p + 1) * N + i) * N + j]);
        },
        NoMid(), [&](int ix, int iy, C2 v) { M[ix * n + iy] = v; });
    col_pass<n, -1, true, 1>(
        sm, tw, [&](int ix, int iy) { return M[ix * n + iy]; },
        [&](int ix, int iy, C2 v) {
          const bool keep = in_xi<n>(freq_of_pos<n>(ix)) && in_xi<n>(freq_of_pos<n>(iy));
          return keep ? cscale(v, invP) : zero2<T>();
        },
        [&](int ix, int iy, C2 v) { M[ix * n + iy] = v; });
    row_pass<n, 1, false, 0>(
        sm, tw, [&](int ix, int iy) { return M[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) { M[ix * n + iy] = v; });
  }
  for (int f = 0; f < 4; ++f) {
    const C2* in = (f < 2) ? (Dacc + ((size_t)c * 2 + f) * P) : (K4acc + ((size_t)c * 2 + (f - 2)) * P);
    C2* out = DK + (size_t)f * P;
    col_pass<n, 1, false, 0>(
        sm, tw, [&](int ix, int iy) { return in[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) { out[ix * n + iy] = v; });
    row_pass<n, 1, false, 0>(
        sm, tw, [&](int ix, int iy) { return out[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) { out[ix * n + iy] = v; });
  }
  const C2* wf0 = wfine + (size_t)c * 2 * P;
  const C2* wf1 = wf0 + P;
  const T* K2 = K2acc + (size_t)c * P;
  C2* nuc = nu + (size_t)c * 2 * P;
  T* nufc = nuf + (size_t)c * P;
  C2* muDc = muD + (size_t)c * 2 * P;
  T* muK2c = muK2 + (size_t)c * P;
  C2* mu4c = mu4 + (size_t)c * 2 * P;
  C2* mu3c = mu3 + (size_t)c * 2 * P;
  const double tp = 2.0 * kPi;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const double m0 = MU[i].x, m1 = MU[i].y, m2 = MU[P + i].x, m3 = MU[P + i].y;
    const double w0 = wf0[i].x, w1 = wf0[i].y, w2 = wf1[i].x, w3 = wf1[i].y;
    const double D1 = DK[i].x, D2 = DK[i].y, D3 = DK[P + i].x;
    const double K40 = DK[2 * P + i].x, K41 = -(double)DK[2 * P + i].y;
    const double K42 = -(double)DK[3 * P + i].x, K43 = -(double)DK[3 * P + i].y;
    const double k2 = K2[i];
    // C0 = 2pi[K2(1-w0) - K3_0 + w0 K4_0 + w.K4];  C_c = -2 (D x w)_c + 2pi[-K2 w_c - K3_c + w0 K4_c + K4_0 w_c]
    const double g0 = tp * (m0 * (K40 - k2) + m1 * K41 + m2 * K42 + m3 * K43);
    // -2 (mu x D)_c + 2 pi (m0 K4_c + m_c (K4_0 - K2))
    const double g1 = -2.0 * (m2 * D3 - m3 * D2) + tp * (m0 * K41 + m1 * (K40 - k2));
    const double g2 = -2.0 * (m3 * D1 - m1 * D3) + tp * (m0 * K42 + m2 * (K40 - k2));
    const double g3 = -2.0 * (m1 * D2 - m2 * D1) + tp * (m0 * K43 + m3 * (K40 - k2));
    nuc[i] = mk2((T)g0, (T)g1);
    nuc[P + i] = mk2((T)g2, (T)g3);
    nufc[i] = (T)0;
    // muD = -2 (w x mu)
    const double dd1 = -2.0 * (w2 * m3 - w3 * m2), dd2 = -2.0 * (w3 * m1 - w1 * m3), dd3 = -2.0 * (w1 * m2 - w2 * m1);
    muDc[i] = mk2((T)dd1, (T)dd2);
    muDc[P + i] = mk2((T)dd3, (T)0);
    muK2c[i] = (T)(tp * (m0 * (1.0 - w0) - m1 * w1 - m2 * w2 - m3 * w3));
    // K4_b = eta_b raw_b
    const double q0 = tp * (m0 * w0 + m1 * w1 + m2 * w2 + m3 * w3);
    const double q1 = -tp * (m0 * w1 + m1 * w0), q2 = -tp * (m0 * w2 + m2 * w0), q3 = -tp * (m0 * w3 + m3 * w0);
    mu4c[i] = mk2((T)q0, (T)q1);
    mu4c[P + i] = mk2((T)q2, (T)q3);
    // K3_b = eta_b raw_b, C_b has -2 pi K3_b
    mu3c[i] = mk2((T)(-tp * m0), (T)(tp * m1));
    mu3c[P + i] = mk2((T)(tp * m2), (T)(tp * m3));
  }
}

// --------------------------------------------------------------------------
// I1 transpose.  D_b = -K'(f A w_b) with A = "multiply by i phi'_j'", K' = "by i K_j'":
//   nu_f += sum_j' (K' mu_b)(A w_b),   nu_b += -A(f K' mu_b).  One block per cell.
// --------------------------------------------------------------------------
template <int n, class T>
__global__ void __launch_bounds__(kThreads) k_i1_vjp(
    const typename Vec2Of<T>::type* what, const typename Vec2Of<T>::type* wfine,
    const typename Vec2Of<T>::type* muD, typename Vec2Of<T>::type* nu, T* nuf, typename Vec2Of<T>::type* ws,
    const typename Vec2Of<T>::type* __restrict__ gtw, const T* __restrict__ phip, const T* __restrict__ Ktab,
    int J, int nch) {
  using C2 = typename Vec2Of<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* sm = tw + n;
  load_twiddles<n>(tw, gtw);
  constexpr int P = n * n;
  // block (cell c, angle chunk ch); with nch > 1, nu and nuf are per-(cell, chunk) partials (zeroed
  // here, completed by k_i24_vjp, summed by k_add_chunks), with nch = 1 the cell's own accumulators
  const int c = blockIdx.x / nch, ch = blockIdx.x % nch;
  C2* slot = ws + (size_t)blockIdx.x * 3 * P;
  C2* Aw = slot;          // A w_pair
  C2* Bm = slot + P;      // K' mu_pair
  C2* G = slot + 2 * P;
  const C2* wf0 = wfine + (size_t)c * 2 * P;
  C2* nuc = nu + (size_t)blockIdx.x * 2 * P;
  T* nufc = nuf + (size_t)blockIdx.x * P;
  if (nch > 1) {
    zero_fields(nuc, 2 * P);
    for (int i = threadIdx.x; i < P; i += blockDim.x) nufc[i] = (T)0;
    __syncthreads();
  }
  const T invP = (T)(1.0 / (double)P);
  for (int jp = J * ch / nch; jp < J * (ch + 1) / nch; ++jp) {
    const T* ph = phip + (size_t)jp * P;
    const T* K = Ktab + (size_t)jp * P;
    for (int p = 0; p < 2; ++p) {
      const C2* in = what + ((size_t)c * 4 + 2 + p) * P;
      const C2* mu = muD + ((size_t)c * 2 + p) * P;
      // Aw = IFFT(i phi' w^)
      col_pass<n, 1, false, 0>(
          sm, tw, [&](int ix, int iy) { return mul_i(in[ix * n + iy], ph[ix * n + iy]); }, NoMid(),
          [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
      row_pass<n, 1, false, 0>(
          sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
          [&](int ix, int iy, C2 v) { Aw[ix * n + iy] = v; });
      // Bm = IFFT(i K FFT(mu))   (K already carries 1/n^2)
      row_pass<n, -1, false, 0>(
          sm, tw, [&](int ix, int iy) { return mu[ix * n + iy]; }, NoMid(),
          [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
      col_pass<n, -1, true, 1>(
          sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; },
          [&](int ix, int iy, C2 v) { return mul_i(v, K[ix * n + iy]); },
          [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
      row_pass<n, 1, false, 0>(
          sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
          [&](int ix, int iy, C2 v) { Bm[ix * n + iy] = v; });
      // nu_f += Re.Re + Im.Im ;  then -A(f Bm) into nu (pair layout of this p)
      row_pass<n, -1, false, 0>(
          sm, tw,
          [&](int ix, int iy) {
            const int i = ix * n + iy;
            const C2 a = Aw[i], b = Bm[i];
            nufc[i] += a.x * b.x + a.y * b.y;
            return cscale(b, (T)2 * wf0[i].x - (T)1);
          },
          NoMid(), [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
      col_pass<n, -1, true, 1>(
          sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; },
          [&](int ix, int iy, C2 v) { return mul_i(v, -ph[ix * n + iy] * invP); },
          [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
      row_pass<n, 1, false, 0>(
          sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
          [&](int ix, int iy, C2 v) {
            const int i = ix * n + iy;
            // pair p = 0 carries components (1, 2) -> nu pair 0 .y and nu pair 1 .x; p = 1 carries (3, -)
            if (p == 0) {
              nuc[i].y += v.x;
              nuc[P + i].x += v.y;
            } else {
              nuc[P + i].y += v.x;
            }
          });
    }
  }
}

// --------------------------------------------------------------------------
// I2/I4 transpose.  F_{a,j} = Psi_j w_a (even multipliers: self-adjoint).
//   K2 = 2 (pi/J) sum_{j<J/2} sum_a eta_a F_{a,j} F_{a,j'} ,  j' = j + J/2
//   K4raw_b = (pi/J) sum_{j<J/2} [Psi_j(f F_{b,j'}) + Psi_j'(f F_{b,j})]
// One block per cell.
// --------------------------------------------------------------------------
template <int n, class T>
__global__ void __launch_bounds__(kThreads) k_i24_vjp(
    const typename Vec2Of<T>::type* what, const typename Vec2Of<T>::type* wfine, const T* muK2,
    const typename Vec2Of<T>::type* mu4, typename Vec2Of<T>::type* nu, T* nuf, typename Vec2Of<T>::type* ws,
    const typename Vec2Of<T>::type* __restrict__ gtw, const T* __restrict__ psi, int J, int nch) {
  using C2 = typename Vec2Of<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* sm = tw + n;
  load_twiddles<n>(tw, gtw);
  constexpr int P = n * n;
  // block (cell c, chunk ch of the J/2 angle pairs); nu, nuf as in k_i1_vjp
  const int c = blockIdx.x / nch, ch = blockIdx.x % nch;
  C2* slot = ws + (size_t)blockIdx.x * 7 * P;
  C2* FA = slot;             // [2] F_{.,j}
  C2* FB = slot + 2 * P;     // [2] F_{.,j'}
  C2* PM = slot + 4 * P;     // [2] Psi(mu4) for the current direction
  C2* G = slot + 6 * P;
  const C2* wf0 = wfine + (size_t)c * 2 * P;
  const T* mk2c = muK2 + (size_t)c * P;
  const C2* m4 = mu4 + (size_t)c * 2 * P;
  C2* nuc = nu + (size_t)blockIdx.x * 2 * P;
  T* nufc = nuf + (size_t)blockIdx.x * P;
  const T wj = (T)(kPi / J);
  const T invP = (T)(1.0 / (double)P);
  const int H = J / 2;
  for (int j = H * ch / nch; j < H * (ch + 1) / nch; ++j) {
    const int jq = j + J / 2;
    for (int p = 0; p < 2; ++p) {
      const C2* in = what + ((size_t)c * 4 + p) * P;
      for (int h = 0; h < 2; ++h) {
        const T* ps = psi + (size_t)(h == 0 ? j : jq) * P;
        C2* F = (h == 0 ? FA : FB) + (size_t)p * P;
        col_pass<n, 1, false, 0>(
            sm, tw, [&](int ix, int iy) { return cscale(in[ix * n + iy], ps[ix * n + iy]); }, NoMid(),
            [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
        row_pass<n, 1, false, 0>(
            sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
            [&](int ix, int iy, C2 v) { F[ix * n + iy] = v; });
      }
    }
    for (int h = 0; h < 2; ++h) {
      const T* ps = psi + (size_t)(h == 0 ? j : jq) * P;       // Psi_j pairs with F_{j'}, Psi_j' with F_j
      const T* pq = psi + (size_t)(h == 0 ? jq : j) * P;
      const C2* Fo = (h == 0 ? FB : FA);                          // the other direction's F
      for (int p = 0; p < 2; ++p) {
        const C2* F = Fo + (size_t)p * P;
        const C2* mup = m4 + (size_t)p * P;
        C2* PMp = PM + (size_t)p * P;
        const T eta0 = (p == 0) ? (T)1 : (T)-1;
        // K2 part: nu_a += 2 (pi/J) eta_a Psi_{dir}(muK2 * F_other)
        // K4 part: PMp = Psi_{dir}(mu4_pair)
        for (int part = 0; part < 2; ++part) {
          row_pass<n, -1, false, 0>(
              sm, tw,
              [&](int ix, int iy) {
                const int i = ix * n + iy;
                return part == 0 ? cscale(F[i], mk2c[i]) : mup[i];
              },
              NoMid(), [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
          col_pass<n, -1, true, 1>(
              sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; },
              [&](int ix, int iy, C2 v) { return cscale(v, ps[ix * n + iy] * invP); },
              [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
          row_pass<n, 1, false, 0>(
              sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
              [&](int ix, int iy, C2 v) {
                const int i = ix * n + iy;
                if (part == 0) {
                  C2 o = nuc[(size_t)p * P + i];
                  o.x += (T)2 * wj * eta0 * v.x;     // eta of component 2p
                  o.y += (T)2 * wj * (T)(-1) * v.y;  // eta of component 2p+1 (always -1)
                  nuc[(size_t)p * P + i] = o;
                } else {
                  PMp[i] = v;
                }
              });
        }
        // nu_f += (pi/J) PM . F_other ; nu_b += (pi/J) Psi_other(f PM)
        row_pass<n, -1, false, 0>(
            sm, tw,
            [&](int ix, int iy) {
              const int i = ix * n + iy;
              const C2 pmv = PMp[i], fv = F[i];
              nufc[i] += wj * (pmv.x * fv.x + pmv.y * fv.y);
              return cscale(pmv, (T)2 * wf0[i].x - (T)1);
            },
            NoMid(), [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
        col_pass<n, -1, true, 1>(
            sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; },
            [&](int ix, int iy, C2 v) { return cscale(v, pq[ix * n + iy] * invP); },
            [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
        row_pass<n, 1, false, 0>(
            sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
            [&](int ix, int iy, C2 v) {
              const int i = ix * n + iy;
              C2 o = nuc[(size_t)p * P + i];
              o.x += wj * v.x;
              o.y += wj * v.y;
              nuc[(size_t)p * P + i] = o;
            });
      }
    }
  }
}

// nu[c] += sum_ch nupart[c][ch] (2 complex fields) and nuf[c] += sum_ch nufpart[c][ch] (1 real
// field), in chunk order: the per-(cell, chunk) partials of k_i1_vjp + k_i24_vjp.
template <class T>
__global__ void __launch_bounds__(kThreads) k_add_chunks(const T* __restrict__ nupart, const T* __restrict__ nufpart,
                                                         T* nu, T* nuf, int nch, int ncells, size_t P) {
  const size_t per_c = 4 * P;
  const size_t total = (size_t)ncells * (per_c + P);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const T* src;
    T* dst;
    size_t c, e, stride;
    if (i < (size_t)ncells * per_c) {
      c = i / per_c; e = i % per_c; src = nupart; dst = nu; stride = per_c;
    } else {
      const size_t k = i - (size_t)ncells * per_c;
      c = k / P; e = k % P; src = nufpart; dst = nuf; stride = P;
    }
    const T* p = src + (c * nch) * stride + e;
    T sum = p[0];
    for (int ch = 1; ch < nch; ++ch) sum += p[(size_t)ch * stride];
    dst[c * stride + e] += sum;
  }
}

// The Fourier-space partials of the I3 transpose are kept only on the frequencies the final
// projection keeps (in_xi in both coordinates, n/2 - 1 per coordinate): slot[pos] is the compact
// index of permuted position pos, or -1.  Every kernel that reads or writes the compact partials
// builds the table with this same ascending loop.
template <int n>
__host__ __device__ constexpr int xi_kept() {
  return n / 2 - 1;
}
template <int n>
__device__ __forceinline__ void build_xi_slots(int* slot, int* kept_pos) {
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int pos = 0; pos < n; ++pos) {
      const bool keep = in_xi<n>(freq_of_pos<n>(pos));
      slot[pos] = keep ? cnt : -1;
      if (keep) kept_pos[cnt++] = pos;
    }
  }
  __syncthreads();
}

// dst = Psi'_j(x) for the field x(i) = ld(i), i = ix * n + iy: row FFT, column convolution with the
// angle's psi' table, row IFFT (the forward's convolution); G is the staging field.
template <int n, class C2, class T, class LD>
__device__ __forceinline__ void psi_conv(C2* sm, const C2* tw, const T* __restrict__ psp, C2* G, LD ld, C2* dst) {
  row_pass<n, -1, false, 0>(
      sm, tw, [&](int ix, int iy) { return ld(ix * n + iy); }, NoMid(),
      [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
  col_conv_pass<n>(
      sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, [&](int ix, int iy) { return psp[ix * n + iy]; },
      [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
  row_pass<n, 1, false, 0>(
      sm, tw, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
      [&](int ix, int iy, C2 v) { dst[ix * n + iy] = v; });
}

// --------------------------------------------------------------------------
// I3 transpose (Hu-Ying term).  K3raw_b = sum_{j,m} sum_a eta_a S(w_a) T_ab,
// T_ab = Psi'(w_a S(w_b)), with cotangents mu_b of K3raw_b:
//   (i)   nu_a += S^T(eta_a sum_b mu_b T_ab)
//   (ii)  nu_a += eta_a sum_b Q_ab S(w_b),        Q_ab = Psi'(mu_b S(w_a))
//   (iii) nu_b += S^T(sum_a eta_a w_a Q_ab)
// (i) and (iii) are summed before one forward FFT and accumulated in Fourier
// space with the conjugate phase; (ii) is accumulated in real space.
// Persistent blocks over units (cell, j, m-chunk); per unit outputs a real
// partial [2][P] and a spectral partial [2][Q] on the kept frequencies
// (Q = (n/2 - 1)^2, see build_xi_slots).
// Several cotangents (K of them, mu3 / part_r / part_s of cotangent k at
// offsets k * mu_stride, k * part_stride and k * spart_stride) share the shifted fields and the
// T transforms, which depend on the state only: per (j, m) 8 + 8 K
// convolutions instead of 16 K.
// --------------------------------------------------------------------------
template <int n, class T>
__global__ void __launch_bounds__(kThreads, 2) k_i3_vjp(
    const typename Vec2Of<T>::type* what, const typename Vec2Of<T>::type* wfine,
    const typename Vec2Of<T>::type* mu3, typename Vec2Of<T>::type* part_r, typename Vec2Of<T>::type* part_s,
    typename Vec2Of<T>::type* ws, const typename Vec2Of<T>::type* __restrict__ gtw,
    const T* __restrict__ psip_s, const typename Vec2Of<T>::type* __restrict__ phase, int J, int M, int nmc, int mch,
    int nunits, int K, size_t mu_stride, size_t part_stride, size_t spart_stride) {
  using C2 = typename Vec2Of<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* sm = tw + n;
  __shared__ int xcols[n];
  __shared__ unsigned char xmask[n];
  __shared__ int kslot[n];
  __shared__ int kcols[n];
  constexpr int NQ = xi_kept<n>(), Q = NQ * NQ;
  build_xi_slots<n>(kslot, kcols);
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
  C2* slot = ws + (size_t)blockIdx.x * (7 + 2 * K) * P;
  C2* Sig = slot;            // [2] shifted pairs
  C2* Tp = slot + 2 * P;     // [2] T_{a, pair}
  C2* Qp = slot + 4 * P;     // [2] Q_{a, pair}
  C2* G = slot + 6 * P;
  C2* XZall = slot + 7 * P;  // [K][2] (i)+(iii) real-space terms, pairs by component
  for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
    const int c = unit / (J * nmc);
    const int j = (unit / nmc) % J;
    const int mc = unit % nmc;
    for (int k = 0; k < K; ++k) {
      zero_fields(part_r + k * part_stride + (size_t)unit * 2 * P, 2 * P);
      zero_fields(part_s + k * spart_stride + (size_t)unit * 2 * Q, 2 * Q);
    }
    const T* psp = psip_s + (size_t)j * P;
    const C2* wf = wfine + (size_t)c * 2 * P;
    const int m0 = mc * mch, m1 = min(M, m0 + mch);
    for (int m = m0; m < m1; ++m) {
      const C2* px = phase + ((size_t)j * M + m) * 2 * n;
      const C2* py = px + n;
      for (int p = 0; p < 2; ++p) {
        const C2* in = what + ((size_t)c * 4 + p) * P;
        C2* S = Sig + (size_t)p * P;
        col_pass_list<n, 1, false, 0, 65536, true>(
            sm, tw, xcols, n / 2,
            [&](int ix, int iy) { return xmask[ix] ? cmul(in[ix * n + iy], cmul(px[ix], py[iy])) : zero2<T>(); },
            NoMid(), [&](int ix, int iy, C2 v) { S[ix * n + iy] = v; });
        row_pass<n, 1, false, 0, 65536, true>(
            sm, tw, [&](int ix, int iy) { return xmask[iy] ? S[ix * n + iy] : zero2<T>(); }, NoMid(),
            [&](int ix, int iy, C2 v) { S[ix * n + iy] = v; });
      }
      zero_fields(XZall, 2 * K * P);
      for (int a = 0; a < 4; ++a) {
        const C2* wa = wf + (size_t)(a >> 1) * P;
        const C2* Sa = Sig + (size_t)(a >> 1) * P;
        const bool im = (a & 1) != 0;
        const T eta_a = (a == 0) ? (T)1 : (T)-1;
        // T_{a, pair} = Psi'(w_a S_pair): the state's, shared by every cotangent
        for (int p = 0; p < 2; ++p) {
          const C2* Sp = Sig + (size_t)p * P;
          psi_conv<n>(sm, tw, psp, G,
                      [&](int i) {
                        const C2 z = wa[i];
                        return cscale(Sp[i], im ? z.y : z.x);
                      },
                      Tp + (size_t)p * P);
        }
        for (int k = 0; k < K; ++k) {
          const C2* mu = mu3 + k * mu_stride + (size_t)c * 2 * P;
          C2* XZ = XZall + (size_t)k * 2 * P;
          // Q_{a, pair} = Psi'(S_a mu_pair)
          for (int p = 0; p < 2; ++p) {
            const C2* mup = mu + (size_t)p * P;
            psi_conv<n>(sm, tw, psp, G,
                        [&](int i) {
                          const C2 sv = Sa[i];
                          return cscale(mup[i], im ? sv.y : sv.x);
                        },
                        Qp + (size_t)p * P);
          }
          // pointwise: (i) X_a = eta_a sum_b mu_b T_ab ; (ii) Y_a = eta_a sum_b Q_ab S_b ; (iii) Z_b += eta_a w_a Q_ab
          C2* accr_a = part_r + k * part_stride + (size_t)unit * 2 * P + (size_t)(a >> 1) * P;
          C2* XZ_a = XZ + (size_t)(a >> 1) * P;
          for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const C2 t0 = Tp[i], t1 = Tp[P + i], q0 = Qp[i], q1 = Qp[P + i];
            const C2 m0v = mu[i], m1v = mu[P + i];
            const C2 s0 = Sig[i], s1 = Sig[P + i];
            const C2 wz = wa[i];
            const T wv = im ? wz.y : wz.x;
            const T X = eta_a * (m0v.x * t0.x + m0v.y * t0.y + m1v.x * t1.x + m1v.y * t1.y);
            const T Y = eta_a * (q0.x * s0.x + q0.y * s0.y + q1.x * s1.x + q1.y * s1.y);
            if (im) {
              accr_a[i].y += Y;
              XZ_a[i].y += X;
            } else {
              accr_a[i].x += Y;
              XZ_a[i].x += X;
            }
            const T e = eta_a * wv;
            XZ[i].x += e * q0.x;
            XZ[i].y += e * q0.y;
            XZ[P + i].x += e * q1.x;
            XZ[P + i].y += e * q1.y;
          }
          __syncthreads();
        }
      }
      // S^T: forward FFT of the XZ pairs, times the conjugate phase, accumulated in Fourier space on
      // the kept frequencies only (column transforms of the kept columns only)
      for (int k = 0; k < K; ++k) {
        for (int p = 0; p < 2; ++p) {
          const C2* src = XZall + (size_t)(2 * k + p) * P;
          C2* dst = part_s + k * spart_stride + (size_t)unit * 2 * Q + (size_t)p * Q;
          row_pass<n, -1, false, 0>(
              sm, tw, [&](int ix, int iy) { return src[ix * n + iy]; }, NoMid(),
              [&](int ix, int iy, C2 v) { G[ix * n + iy] = v; });
          col_pass_list<n, -1, false, 0>(
              sm, tw, kcols, NQ, [&](int ix, int iy) { return G[ix * n + iy]; }, NoMid(),
              [&](int ix, int iy, C2 v) {
                const int sx = kslot[ix];
                if (sx < 0) return;
                const C2 ph = cmul(px[ix], py[iy]);
                const C2 z = cmulc(v, ph);
                C2* o = dst + sx * NQ + kslot[iy];
                C2 d = *o;
                d.x += z.x;
                d.y += z.y;
                *o = d;
              });
        }
      }
    }
  }
}

// --------------------------------------------------------------------------
// I3 transpose with the transform field resident in shared memory (FP32,
// n <= 128), the counterpart of k_i3_smem.  Each convolution's epilogue adds
// its terms straight into the accumulators, so T_ab and Q_ab are never stored:
//   after T_ap = Psi'(w_a S_p):  XZ_a += eta_a mu_p . T_ap           (i)
//   after Q_ap = Psi'(S_a mu_p): part_r_a += eta_a Q_ap . S_p         (ii)
//                                XZ_p += eta_a w_a Q_ap               (iii)
// then S^T of XZ in Fourier space as in k_i3_vjp.
// --------------------------------------------------------------------------
template <int n>
__global__ void __launch_bounds__(kThreadsI3Smem, 1) k_i3_vjp_smem(
    const float2* what, const float2* wfine, const float2* mu3, float2* part_r, float2* part_s, float2* ws,
    const float2* __restrict__ gtw, const float* __restrict__ psip_s, const float2* __restrict__ phase, int J, int M,
    int nmc, int mch, int nunits, int K, size_t mu_stride, size_t part_stride, size_t spart_stride) {
  using C2 = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* G = tw + n;                       // [n][LS]
  float* psm = reinterpret_cast<float*>(G + n * (n + 1));   // psi'_j of the current unit, [n][n]
  constexpr int LS = n + 1, P = n * n;
  constexpr int kIter = (P + kThreadsI3Smem - 1) / kThreadsI3Smem;
  __shared__ unsigned char xmask[n];
  __shared__ int kslot[n];
  __shared__ int kcols[n];
  constexpr int NQ = xi_kept<n>(), Q = NQ * NQ;
  for (int pos = threadIdx.x; pos < n; pos += blockDim.x) {
    const int k = freq_of_pos<n>(pos);
    xmask[pos] = ((k < n / 4) || (k >= n - n / 4)) ? 1 : 0;
  }
  build_xi_slots<n>(kslot, kcols);
  load_twiddles<n>(tw, gtw);
  C2* slot = ws + (size_t)blockIdx.x * (2 + 2 * K) * P;
  C2* Sig = slot;            // [2]
  C2* XZall = slot + 2 * P;  // [K][2]
  for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
    const int c = unit / (J * nmc);
    const int j = (unit / nmc) % J;
    const int mc = unit % nmc;
    for (int k = 0; k < K; ++k) {
      zero_fields(part_r + k * part_stride + (size_t)unit * 2 * P, 2 * P);
      zero_fields(part_s + k * spart_stride + (size_t)unit * 2 * Q, 2 * Q);
    }
    {
      const float4* src = reinterpret_cast<const float4*>(psip_s + (size_t)j * P);
      float4* dst = reinterpret_cast<float4*>(psm);
      for (int i4 = threadIdx.x; i4 < P / 4; i4 += blockDim.x) dst[i4] = src[i4];
      __syncthreads();
    }
    const C2* wf = wfine + (size_t)c * 2 * P;
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
        fft_lines<n, 1, true>(G, n, 1, LS, tw);   // shifts: input zero outside Xi x Xi
        fft_lines<n, 1, true>(G, n, LS, 1, tw);
        C2* S = Sig + (size_t)p * P;
        for (int idx = threadIdx.x; idx < P; idx += blockDim.x) S[idx] = G[(idx / n) * LS + idx % n];
        __syncthreads();
      }
      zero_fields(XZall, 2 * K * P);
      for (int a = 0; a < 4; ++a) {
        const C2* wa = wf + (size_t)(a >> 1) * P;
        const C2* Sa = Sig + (size_t)(a >> 1) * P;
        const bool im = (a & 1) != 0;
        const float eta_a = (a == 0) ? 1.f : -1.f;
        for (int p = 0; p < 2; ++p) {
          const C2* Sp = Sig + (size_t)p * P;
          // which 0: T = Psi'(w_a S_pair), the state's, shared by every cotangent;
          // which 1: Q = Psi'(S_a mu_pair), once per cotangent
          for (int which = 0; which < 1 + K; ++which) {
            const int kq = which - 1;                          // cotangent of a Q transform
            const C2* __restrict__ src = which == 0 ? Sp : mu3 + kq * mu_stride + (size_t)c * 2 * P + (size_t)p * P;
            const C2* __restrict__ scl = which == 0 ? wa : Sa;
#pragma unroll 8
            for (int k = 0; k < kIter; ++k) {
              const int idx = threadIdx.x + k * kThreadsI3Smem;
              if (kIter * kThreadsI3Smem == P || idx < P) {
                const C2 z = scl[idx];
                G[(idx / n) * LS + idx % n] = cscale(src[idx], im ? z.y : z.x);
              }
            }
            __syncthreads();
            fft_lines<n, -1>(G, n, LS, 1, tw);
            fft_conv_lines<n>(G, n, 1, LS, tw, [&](int l, int pos) { return psm[pos * n + l]; });
            fft_lines<n, 1>(G, n, LS, 1, tw);
            if (which == 0) {
              // (i): X_a += eta_a mu_pair . T for every cotangent
              for (int kc = 0; kc < K; ++kc) {
                const C2* __restrict__ mv_ = mu3 + kc * mu_stride + (size_t)c * 2 * P + (size_t)p * P;
                float* __restrict__ xz =
                    reinterpret_cast<float*>(XZall + (size_t)(2 * kc + (a >> 1)) * P) + (im ? 1 : 0);
#pragma unroll 8
                for (int k = 0; k < kIter; ++k) {
                  const int idx = threadIdx.x + k * kThreadsI3Smem;
                  if (kIter * kThreadsI3Smem == P || idx < P) {
                    const C2 g = G[(idx / n) * LS + idx % n];
                    const C2 mv = mv_[idx];
                    xz[2 * idx] += eta_a * (mv.x * g.x + mv.y * g.y);
                  }
                }
              }
            } else {
              // (ii) into the real-space partial, (iii) into Z_pair
              const C2* __restrict__ sp_ = Sp;
              const C2* __restrict__ wa_ = wa;
              float* __restrict__ ar = reinterpret_cast<float*>(part_r + kq * part_stride + (size_t)unit * 2 * P +
                                                                (size_t)(a >> 1) * P) + (im ? 1 : 0);
              C2* __restrict__ xzp = XZall + (size_t)(2 * kq + p) * P;
#pragma unroll 4
              for (int k = 0; k < kIter; ++k) {
                const int idx = threadIdx.x + k * kThreadsI3Smem;
                if (kIter * kThreadsI3Smem == P || idx < P) {
                  const C2 g = G[(idx / n) * LS + idx % n];
                  const C2 sp = sp_[idx];
                  const C2 z = wa_[idx];
                  ar[2 * idx] += eta_a * (g.x * sp.x + g.y * sp.y);
                  const float e = eta_a * (im ? z.y : z.x);
                  C2 o = xzp[idx];
                  o.x += e * g.x;
                  o.y += e * g.y;
                  xzp[idx] = o;
                }
              }
            }
            __syncthreads();
          }
        }
      }
      for (int kc = 0; kc < K; ++kc) {
        for (int p = 0; p < 2; ++p) {
          const C2* src = XZall + (size_t)(2 * kc + p) * P;
          C2* dst = part_s + kc * spart_stride + (size_t)unit * 2 * Q + (size_t)p * Q;
          for (int idx = threadIdx.x; idx < P; idx += blockDim.x) G[(idx / n) * LS + idx % n] = src[idx];
          __syncthreads();
          fft_lines<n, -1>(G, n, LS, 1, tw);    // rows
          fft_lines<n, -1>(G, n, 1, LS, tw);    // columns
          // accumulated on the kept frequencies only
          for (int q = threadIdx.x; q < Q; q += blockDim.x) {
            const int ix = kcols[q / NQ], iy = kcols[q % NQ];
            const C2 z = cmulc(G[ix * LS + iy], cmul(px[ix], py[iy]));
            C2 d = dst[q];
            d.x += z.x;
            d.y += z.y;
            dst[q] = d;
          }
          __syncthreads();
        }
      }
    }
  }
}

#include "i3_vjp_wl.cuh"

// --------------------------------------------------------------------------
// Final: nu = direct + I1 + I2/I4 + 2 nu_f (into w0) + sum of the I3 real
// partials; gradient = 4 E P (nu + IFFT(H) / n^2) with H the sum of the I3
// spectral partials.  P keeps the kept frequencies only and FFT(IFFT(H)) =
// n^2 H, so H (stored on those frequencies) is added to FFT(nu) there.
// One block per cell; writes grad[c][4][N][N] (FP64).
// --------------------------------------------------------------------------
template <int n, class T>
__global__ void __launch_bounds__(kThreads) k_vjp_final(
    const typename Vec2Of<T>::type* nu, const T* nuf, const typename Vec2Of<T>::type* part_r,
    const typename Vec2Of<T>::type* part_s, int nparts, typename Vec2Of<T>::type* ws,
    const typename Vec2Of<T>::type* __restrict__ gtw, double* grad, int accumulate) {
  using C2 = typename Vec2Of<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);
  C2* sm = tw + n;
  __shared__ int kslot[n];
  __shared__ int kcols[n];
  build_xi_slots<n>(kslot, kcols);
  load_twiddles<n>(tw, gtw);
  constexpr int N = n / 2, P = n * n;
  constexpr int NQ = xi_kept<n>(), Q = NQ * NQ;
  const int c = blockIdx.x;
  C2* slot = ws + (size_t)blockIdx.x * 5 * P;
  C2* V = slot;            // [2] total real-space cotangent pairs
  C2* F = slot + 2 * P;    // [2] their transforms
  C2* H = slot + 4 * P;    // [2][Q] spectral sum on the kept frequencies
  const C2* pr = part_r + (size_t)c * nparts * 2 * P;
  const C2* ps = part_s + (size_t)c * nparts * 2 * Q;
  for (int i = threadIdx.x; i < 2 * P; i += blockDim.x) {
    double sx = 0, sy = 0;
    for (int u = 0; u < nparts; ++u) {
      const C2 a = pr[(size_t)u * 2 * P + i];
      sx += (double)a.x; sy += (double)a.y;
    }
    const C2 d = nu[(size_t)c * 2 * P + i];
    double vx = (double)d.x + sx, vy = (double)d.y + sy;
    if (i < P) vx += 2.0 * (double)nuf[(size_t)c * P + i];
    V[i] = mk2((T)vx, (T)vy);
  }
  for (int i = threadIdx.x; i < 2 * Q; i += blockDim.x) {
    double hx = 0, hy = 0;
    for (int u = 0; u < nparts; ++u) {
      const C2 b = ps[(size_t)u * 2 * Q + i];
      hx += (double)b.x; hy += (double)b.y;
    }
    H[i] = mk2((T)hx, (T)hy);
  }
  __syncthreads();
  const T invP = (T)(1.0 / (double)P);
  for (int p = 0; p < 2; ++p) {
    C2* Vp = V + (size_t)p * P;
    C2* Fp = F + (size_t)p * P;
    const C2* Hp = H + (size_t)p * Q;
    // 4 E P (V + IFFT(H) / n^2)
    row_pass<n, -1, false, 0>(
        sm, tw, [&](int ix, int iy) { return Vp[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) { Fp[ix * n + iy] = v; });
    col_pass<n, -1, true, 1>(
        sm, tw, [&](int ix, int iy) { return Fp[ix * n + iy]; },
        [&](int ix, int iy, C2 v) {
          const int sx = kslot[ix], sy = kslot[iy];
          if (sx < 0 || sy < 0) return zero2<T>();
          const C2 h = Hp[sx * NQ + sy];
          return cscale(cadd(v, h), invP);
        },
        [&](int ix, int iy, C2 v) { Fp[ix * n + iy] = v; });
    double* g = grad + (size_t)c * 4 * N * N;
    row_pass<n, 1, false, 0>(
        sm, tw, [&](int ix, int iy) { return Fp[ix * n + iy]; }, NoMid(),
        [&](int ix, int iy, C2 v) {
          if (((ix | iy) & 1) == 0) {
            const int i = ix >> 1, j = iy >> 1;
            double* g0 = g + ((2 * p) * N + i) * N + j;
            double* g1 = g + ((2 * p + 1) * N + i) * N + j;
            *g0 = (accumulate ? *g0 : 0.0) + 4.0 * (double)v.x;
            *g1 = (accumulate ? *g1 : 0.0) + 4.0 * (double)v.y;
          }
        });
  }
}

}  // namespace

template <int n, class T>
void set_vjp_smem_attributes() {
  static unsigned long long done = 0;
  if (!first_on_device(done)) return;
  const int sm = (int)smem_bytes<n, T>();
  cudaFuncSetAttribute(k_vjp_seed<n, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_i1_vjp<n, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_i24_vjp<n, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_i3_vjp<n, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_vjp_final<n, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if constexpr (std::is_same<T, float>::value && use_i3_smem<n>())
    cudaFuncSetAttribute(k_i3_vjp_smem<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)i3_smem_bytes<n>());
  if constexpr (std::is_same<T, float>::value && n == kWlN)
    cudaFuncSetAttribute(k_i3_vjp_wl<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)i3_vjp_wl_smem_bytes());
}

// I3 transpose kernels per (n, T): the warp-local kernel (FP32, 128 points, one cotangent) is variant
// 0 where it exists, the element-pass shared-memory kernel variant 1; other sizes have one.
template <int n, class T>
constexpr int i3_vjp_variant_count() {
  return (std::is_same<T, float>::value && n == kWlN) ? 2 : 1;
}

// Forward prep/I1/I2+I4 once (the VJP needs wfine, D^, K2, K4^), then per cotangent the seed and the
// I1 and I2/I4 transposes, one I3 transpose launch for all K cotangents, and per cotangent the final
// assembly.  Cotangent k uses copy k of every cotangent buffer of vw.
template <int n, class T>
cudaError_t collide_vjp_n(const Tables& t, CollisionWork& cw, VjpWork& vw, const double* w, const double* const* lam,
                          double* const* grad, int K, int ncells, int accumulate, cudaStream_t s, long long& launches,
                          KernelTimer* tm) {
  using C2 = typename Vec2Of<T>::type;
  set_smem_attributes<n, T>();
  set_vjp_smem_attributes<n, T>();
  const TabPtrs<T> tb = tab_ptrs<T>(t);
  C2* what = (C2*)cw.what;
  C2* wfine = (C2*)cw.wfine;
  C2* Dacc = (C2*)cw.Dacc;
  T* K2acc = (T*)cw.K2acc;
  C2* K4acc = (C2*)cw.K4acc;
  C2* ws = (C2*)vw.ws;
  const size_t sm = smem_bytes<n, T>();
  constexpr size_t P = (size_t)n * n;
  const size_t c_stride = (size_t)vw.nb * 2 * P;           // complex cotangent buffers, per cotangent
  const size_t r_stride = (size_t)vw.nb * P;               // real cotangent buffers, per cotangent
  const size_t nparts = (size_t)vw.nb * t.J * vw.nmc;
  const size_t part_stride = nparts * 2 * P;
  const size_t spart_stride = nparts * 2 * (size_t)xi_kept<n>() * xi_kept<n>();
  auto begin = [&](int g) { if (tm) tm->begin(g, s); };
  auto end = [&]() { if (tm) tm->end(s); };
  begin(KG_VJP);
  k_prep<n, T><<<ncells, kThreads, sm, s>>>(w, what, wfine, ws, tb.tw);
  ++launches;
  {
    const cudaError_t e = per_cell_terms<n, T>(t, cw, ws, ncells, s, launches, nullptr);
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; k < K; ++k) {
    C2* nu = (C2*)vw.nu + k * c_stride;
    T* nuf = (T*)vw.nuf + k * r_stride;
    C2* muD = (C2*)vw.muD + k * c_stride;
    T* muK2 = (T*)vw.muK2 + k * r_stride;
    C2* mu4 = (C2*)vw.mu4 + k * c_stride;
    C2* mu3 = (C2*)vw.mu3 + k * c_stride;
    k_vjp_seed<n, T><<<ncells, kThreads, sm, s>>>(lam[k], wfine, Dacc, K2acc, K4acc, nu, nuf, muD, muK2, mu4, mu3,
                                                  ws, tb.tw);
    // I1 and I2/I4 transposes over (cell, angle chunk) blocks; their per-chunk cotangents go to the
    // forward's chunk-partial buffers (free once per_cell_terms has reduced them) and are summed in
    // chunk order into nu and nuf
    const int nch = cw.nch < 1 ? 1 : cw.nch;
    C2* nup = nch > 1 ? (C2*)cw.Dpart : nu;
    T* nufp = nch > 1 ? (T*)cw.K2part : nuf;
    k_i1_vjp<n, T><<<ncells * nch, kThreads, sm, s>>>(what, wfine, muD, nup, nufp, ws, tb.tw, tb.phip, tb.Ktab, t.J,
                                                      nch);
    k_i24_vjp<n, T><<<ncells * nch, kThreads, sm, s>>>(what, wfine, muK2, mu4, nup, nufp, ws, tb.tw, tb.psi, t.J,
                                                       nch);
    launches += 3;
    if (nch > 1) {
      k_add_chunks<T><<<(ncells * 5 * n * n + kThreads * 8 - 1) / (kThreads * 8), kThreads, 0, s>>>(
          (const T*)nup, (const T*)nufp, (T*)nu, nuf, nch, ncells, (size_t)n * n);
      ++launches;
    }
  }
  end();
  const int nunits = ncells * t.J * vw.nmc;
  const int grid = nunits < vw.grid ? nunits : vw.grid;
  begin(KG_VJP_I3);
  if constexpr (std::is_same<T, float>::value && use_i3_smem<n>()) {
    bool wl = false;
    if constexpr (n == kWlN) {
      wl = (K == 1 && vw.i3v == 0);
      if (wl)
        k_i3_vjp_wl<n><<<grid, kWlThreads, i3_vjp_wl_smem_bytes(), s>>>(
            what, wfine, (C2*)vw.mu3, (C2*)vw.part_r, (C2*)vw.part_s, ws, tb.tw, tb.psip_s, tb.phase, t.J, t.M,
            vw.nmc, vw.mch, nunits);
    }
    if (!wl)
      k_i3_vjp_smem<n><<<grid, kThreadsI3Smem, i3_smem_bytes<n>(), s>>>(
          what, wfine, (C2*)vw.mu3, (C2*)vw.part_r, (C2*)vw.part_s, ws, tb.tw, tb.psip_s, tb.phase, t.J, t.M,
          vw.nmc, vw.mch, nunits, K, c_stride, part_stride, spart_stride);
  } else
    k_i3_vjp<n, T><<<grid, kThreads, sm, s>>>(what, wfine, (C2*)vw.mu3, (C2*)vw.part_r, (C2*)vw.part_s, ws, tb.tw,
                                              tb.psip_s, tb.phase, t.J, t.M, vw.nmc, vw.mch, nunits, K, c_stride,
                                              part_stride, spart_stride);
  end();
  ++launches;
  begin(KG_VJP);
  for (int k = 0; k < K; ++k) {
    k_vjp_final<n, T><<<ncells, kThreads, sm, s>>>((C2*)vw.nu + k * c_stride, (T*)vw.nuf + k * r_stride,
                                                   (C2*)vw.part_r + k * part_stride, (C2*)vw.part_s + k * spart_stride,
                                                   t.J * vw.nmc, ws, tb.tw, grad[k], accumulate);
    ++launches;
  }
  end();
  return cudaGetLastError();
}

template <int n, class T>
int i3_vjp_blocks_per_sm() {
  set_vjp_smem_attributes<n, T>();
  int b = 0;
  if constexpr (std::is_same<T, float>::value && n == kWlN) {
    int b2 = 0;   // the grid serves both variants: the smaller residency of the two
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_i3_vjp_smem<n>, kThreadsI3Smem, i3_smem_bytes<n>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_i3_vjp_wl<n>, kWlThreads, i3_vjp_wl_smem_bytes());
    if (b2 < b) b = b2;
  } else if constexpr (std::is_same<T, float>::value && use_i3_smem<n>())
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_i3_vjp_smem<n>, kThreadsI3Smem, i3_smem_bytes<n>());
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_i3_vjp<n, T>, kThreads, smem_bytes<n, T>());
  return b < 1 ? 1 : b;
}

}  // namespace qbe
