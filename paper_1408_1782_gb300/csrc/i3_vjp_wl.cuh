// Transpose of the I3 (Hu-Ying, eq. approxH-JM) term's derivative on the padded grid of 128 points in
// FP32, one cotangent per product, with the warp-local passes of k_i3_wl.  Included by
// collision_vjp.cuh inside its anonymous namespace.
//
// Per (cell, j, m), with T_ap = Psi'_j(w_a S_p) and Q_ap = Psi'_j(S_a mu_p), a = 2 q + im (w_a, S_a:
// component im of the fine pair q and of the shifted pair q), the transpose adds
//   (i)   eta_a mu_p . T_ap      into component im of XZ_q,
//   (iii) eta_a w_a Q_ap         into XZ_p,
//   (ii)  eta_a Q_ap . S_p       into component im of the unit's real-space partial of pair q,
// and then S^T of XZ_0 and XZ_1 (forward transform, times the conjugate phase, kept frequencies) into
// the unit's Fourier-space partials.  The sixteen convolutions are ordered by the field they feed:
// for x = 0, 1, the four T_{2x+im,p} and the four Q_{a,x} all reach XZ_x, which is accumulated in
// registers (every convolution's last stage gives each thread the same 32 points), and the S^T of
// XZ_x starts from those registers, so XZ is never stored.  The partials are read and written only
// at the thread's own points; the shifted fields are complete for every thread after the block
// barrier that ends their transform.
#pragma once

// One Psi'_j convolution of the field load(idx) (idx = x * n + y) on the warp-local passes; epi(k, t1,
// idx, v) receives the result at the thread's points (row task k, element t1).
template <class LOAD, class EPI>
__device__ __forceinline__ void wl_convolve(float2* G, const float2* tw, const float2* twT, const float* psm,
                                            int w, int lane, int g, int tt, LOAD load, EPI epi) {
  using C2 = float2;
  constexpr int n = kWlN, A = Split<n>::A, B = Split<n>::B, TPT = n * B / kWlThreads;
  const int t2r = lane & 15;
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    const int x = 8 * w + (lane >> 4) + 2 * k;
    C2 v[A];
#pragma unroll
    for (int t1 = 0; t1 < A; ++t1) v[t1] = load(x * n + B * t1 + t2r);
    dft<A, -1>(v);
#pragma unroll
    for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], twT[k1 * B + t2r]);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) G[wl_addr(x, B * k1 + t2r)] = v[k1];
  }
  __syncwarp();
  wl_rows_stage_b<-1>(G, w, lane);
  __syncthreads();
  wl_cols_stage_a<-1>(G, tw, g, tt);
  wl_pair_sync(g);
  {
    const int y = 16 * g + (tt & 15);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int k1 = (tt >> 4) + 4 * i;
      C2 b[B];
#pragma unroll
      for (int t = 0; t < B; ++t) b[t] = G[wl_addr(B * k1 + t, y)];
      dft<B, -1>(b);
      float sc[B];
#pragma unroll
      for (int t = 0; t < B; ++t) sc[t] = psm[(B * k1 + t) * kWlPsiPitch + y];
      dft_scaled<B, 1>(b, sc);
#pragma unroll
      for (int t = 0; t < B; ++t) G[wl_addr(B * k1 + t, y)] = b[t];
    }
  }
  wl_pair_sync(g);
  wl_cols_stage_a<1>(G, tw, g, tt);
  __syncthreads();
  wl_rows_stage_b<1>(G, w, lane);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    const int x = 8 * w + (lane >> 4) + 2 * k;
    C2 v[A];
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) v[k1] = G[wl_addr(x, B * k1 + t2r)];
#pragma unroll
    for (int k1 = 1; k1 < A; ++k1) v[k1] = cmulc(v[k1], twT[k1 * B + t2r]);
    dft<A, 1>(v);
#pragma unroll
    for (int t1 = 0; t1 < A; ++t1) epi(k, t1, x * n + B * t1 + t2r, v[t1]);
  }
  __syncwarp();   // this warp's rows of G are rewritten by the next convolution's first stage
}

template <int n>
__global__ void __launch_bounds__(kWlThreads, 1) k_i3_vjp_wl(
    const float2* what, const float2* wfine, const float2* mu3, float2* part_r, float2* part_s, float2* ws,
    const float2* __restrict__ gtw, const float* __restrict__ psip_s, const float2* __restrict__ phase, int J, int M,
    int nmc, int mch, int nunits) {
  static_assert(n == kWlN, "warp-local passes: 128-point grid");
  using C2 = float2;
  constexpr int A = Split<n>::A, B = Split<n>::B, P = n * n, NT = kWlThreads;
  constexpr int TPT = n * B / NT;   // 4 row tasks (row, t2) per thread in the first and last stages
  constexpr int NQ = xi_kept<n>(), Q = NQ * NQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);                   // tw[t2 A + k1]
  C2* twT = tw + n;                                           // twT[k1 B + t2]
  C2* G = twT + n;                                            // skewed field
  float* psm = reinterpret_cast<float*>(G + n * kWlPitch);    // psi'_j of the current unit, [n][kWlPsiPitch]
  __shared__ int kslot[n];
  __shared__ int kcols[n];
  for (int pos = threadIdx.x; pos < n; pos += blockDim.x) twT[(pos % A) * B + pos / A] = gtw[pos];
  load_twiddles<n>(tw, gtw);
  build_xi_slots<n>(kslot, kcols);
  C2* Sig = ws + (size_t)blockIdx.x * 2 * P;   // [2][P], the shifted pairs of the current m
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, g = w >> 1, tt = tid & 63;
  const int t2r = lane & 15;
  auto row_of = [&](int k) { return 8 * w + (lane >> 4) + 2 * k; };
  for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
    const int c = unit / (J * nmc);
    const int j = (unit / nmc) % J;
    const int mc = unit % nmc;
    C2* pr = part_r + (size_t)unit * 2 * P;
    C2* ps = part_s + (size_t)unit * 2 * Q;
    {
      const float4* src = reinterpret_cast<const float4*>(psip_s + (size_t)j * P);
      for (int i4 = tid; i4 < P / 4; i4 += NT) {
        const float4 q4 = src[i4];
        float* d = psm + (4 * i4 / n) * kWlPsiPitch + (4 * i4) % n;
        d[0] = q4.x; d[1] = q4.y; d[2] = q4.z; d[3] = q4.w;
      }
      __syncthreads();
    }
    const C2* __restrict__ wf = wfine + (size_t)c * 2 * P;
    const C2* __restrict__ mu = mu3 + (size_t)c * 2 * P;
    const int m0 = mc * mch, m1 = min(M, m0 + mch);
    for (int m = m0; m < m1; ++m) {
      const C2* px = phase + ((size_t)j * M + m) * 2 * n;
      const C2* py = px + n;
      const bool first_m = (m == m0);
      // shifted pairs S_p (as in k_i3_wl; S complete for every thread when wl_shift returns)
      for (int p = 0; p < 2; ++p)
        wl_shift(G, tw, twT, what + ((size_t)c * 4 + p) * P, px, py, Sig + (size_t)p * P, w, lane, g, tt);
      for (int x = 0; x < 2; ++x) {
        C2 racc[TPT][A];   // XZ_x at the thread's points
#pragma unroll
        for (int k = 0; k < TPT; ++k)
#pragma unroll
          for (int t1 = 0; t1 < A; ++t1) racc[k][t1] = zero2<float>();
        // (i): T_ap = Psi'(w_a S_p), a = 2 x + im, into component im of XZ_x
        const C2* __restrict__ wx = wf + (size_t)x * P;
        for (int p = 0; p < 2; ++p) {
          const C2* Sp = Sig + (size_t)p * P;     // rewritten every m: plain (coherent) loads
          const C2* __restrict__ mp = mu + (size_t)p * P;
          for (int im = 0; im < 2; ++im) {
            const float eta = (x == 0 && im == 0) ? 1.f : -1.f;
            const float cx = im ? 0.f : eta, cy = im ? eta : 0.f;
            wl_convolve(
                G, tw, twT, psm, w, lane, g, tt,
                [&](int idx) {
                  const C2 z = wx[idx];
                  return cscale(Sp[idx], im ? z.y : z.x);
                },
                [&](int k, int t1, int idx, C2 v) {
                  const C2 mv = mp[idx];
                  const float d = fmaf(mv.x, v.x, mv.y * v.y);
                  racc[k][t1].x = fmaf(cx, d, racc[k][t1].x);
                  racc[k][t1].y = fmaf(cy, d, racc[k][t1].y);
                });
          }
        }
        // (iii) and (ii): Q_ax = Psi'(S_a mu_x) for every a
        const C2* Sx = Sig + (size_t)x * P;
        const C2* __restrict__ mx = mu + (size_t)x * P;
        for (int a = 0; a < 4; ++a) {
          const int q = a >> 1;
          const bool im = (a & 1) != 0;
          const float eta = (a == 0) ? 1.f : -1.f;
          const C2* Sa = Sig + (size_t)q * P;
          const C2* __restrict__ wa = wf + (size_t)q * P;
          float* prq = reinterpret_cast<float*>(pr + (size_t)q * P) + (im ? 1 : 0);
          const bool first = first_m && x == 0;   // the unit's first contribution to this component
          wl_convolve(
              G, tw, twT, psm, w, lane, g, tt,
              [&](int idx) {
                const C2 s = Sa[idx];
                return cscale(mx[idx], im ? s.y : s.x);
              },
              [&](int k, int t1, int idx, C2 v) {
                const C2 z = wa[idx];
                const float e = eta * (im ? z.y : z.x);
                racc[k][t1].x = fmaf(e, v.x, racc[k][t1].x);
                racc[k][t1].y = fmaf(e, v.y, racc[k][t1].y);
                const C2 s = Sx[idx];
                const float d = eta * fmaf(v.x, s.x, v.y * s.y);
                prq[2 * idx] = first ? d : prq[2 * idx] + d;
              });
        }
        // S^T of XZ_x: forward rows from the registers, forward columns, and on the kept frequencies
        // times the conjugate phase into the unit's Fourier-space partial of pair x
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
          const int xr = row_of(k);
          C2 v[A];
#pragma unroll
          for (int t1 = 0; t1 < A; ++t1) v[t1] = racc[k][t1];
          dft<A, -1>(v);
#pragma unroll
          for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], twT[k1 * B + t2r]);
#pragma unroll
          for (int k1 = 0; k1 < A; ++k1) G[wl_addr(xr, B * k1 + t2r)] = v[k1];
        }
        __syncwarp();
        wl_rows_stage_b<-1>(G, w, lane);
        __syncthreads();
        wl_cols_stage_a<-1>(G, tw, g, tt);
        wl_pair_sync(g);
        {
          const int y = 16 * g + (tt & 15);
          const int sy = kslot[y];
          C2* dst = ps + (size_t)x * Q;
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const int k1 = (tt >> 4) + 4 * i;
            C2 b[B];
#pragma unroll
            for (int t = 0; t < B; ++t) b[t] = G[wl_addr(B * k1 + t, y)];
            dft<B, -1>(b);
            if (sy >= 0) {
#pragma unroll
              for (int t = 0; t < B; ++t) {
                const int xp = B * k1 + t;
                const int sx = kslot[xp];
                if (sx >= 0) {
                  const C2 z = cmulc(b[t], cmul(px[xp], py[y]));
                  C2* o = dst + sx * NQ + sy;
                  *o = first_m ? z : cadd(*o, z);
                }
              }
            }
          }
        }
        __syncthreads();   // G's rows are rewritten by the next convolution's first stage
      }
    }
    __syncthreads();       // psm is reloaded by the next unit
  }
}

constexpr size_t i3_vjp_wl_smem_bytes() { return i3_wl_smem_bytes(); }
