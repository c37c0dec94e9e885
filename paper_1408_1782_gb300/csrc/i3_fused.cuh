// I3 (Hu-Ying term, eq. approxH-JM) in FP32 with the transform field resident in shared memory
// and the global traffic of every convolution fused into its first and last line stages.
// Included by collision_kernels.cuh inside its anonymous namespace.
//
// Units and arithmetic are those of k_i3 / k_i3_smem: for each (cell, j, m-chunk) unit and each m,
//   Sigma_p = IFFT2(e^{i alpha_jm.sigma} sqrt(c_jm) w^_pair p)             (p = 0, 1)
//   acc_p  += sum_a eta_a S_a IFFT2(psi'_j FFT2(w_a Sigma_p)) / n^2       (a = 0..3)
// The field G (n x (n+1) complex, padded rows) holds one transform at a time.  A length-n line
// transform is two register stages, radix A over elements B t1 + t2 ("stage A") and radix B over
// B contiguous elements ("stage B"), with one shared-memory round trip between them
// (fft.cuh).  Compared with k_i3_smem:
//   * the product w_a Sigma_p is formed while loading the forward row transform's stage A, whose
//     tasks (row, t2) run t2-fastest across a warp, so the global loads are coalesced and go
//     straight into registers (no element pass through shared memory);
//   * the inverse row transform's stage A multiplies by eta_a S_a in registers and accumulates
//     the four a of one (m, p) in per-thread registers (each thread owns the same elements in
//     every a); the unit's partial sum in global memory is read and written once per (m, p)
//     instead of once per convolution, and written without a read at the chunk's first m;
//   * the shift transforms load the phase-multiplied Xi coefficients inside the first column
//     stage and store the shifted field from the last row stage.
// Each convolution therefore moves its field through the L1/shared-memory path 14.5 times
// (128 KB per pass at n = 128) instead of 21 times.
#pragma once

template <int n>
struct FusedShape {
  static constexpr int A = Split<n>::A, B = Split<n>::B, LS = n + 1, P = n * n;
};

// Stage B of the n row transforms (radix B on B contiguous elements; tasks row-fastest, so the
// 32 lanes of a warp hit 32 rows whose padded stride n + 1 spreads them over all banks).
template <int n, int SIGN>
__device__ __forceinline__ void rows_stage_b(float2* G) {
  constexpr int A = FusedShape<n>::A, B = FusedShape<n>::B, LS = FusedShape<n>::LS;
  for (int task = threadIdx.x; task < n * A; task += blockDim.x) {
    const int l = task % n, k1 = task / n;
    float2* base = G + l * LS + B * k1;
    float2 b[B];
#pragma unroll
    for (int t = 0; t < B; ++t) b[t] = base[t];
    dft<B, SIGN>(b);
#pragma unroll
    for (int t = 0; t < B; ++t) base[t] = b[t];
  }
  __syncthreads();
}

// Stage A of the n column transforms, tasks column-fastest.  Forward: natural input, twiddled
// output in place; inverse: conjugate twiddles, then the DFT.
template <int n, int SIGN>
__device__ __forceinline__ void cols_stage_a(float2* G, const float2* tw) {
  constexpr int A = FusedShape<n>::A, B = FusedShape<n>::B, LS = FusedShape<n>::LS;
  for (int task = threadIdx.x; task < n * B; task += blockDim.x) {
    const int l = task % n, t2 = task / n;
    float2* base = G + l + t2 * LS;
    float2 a[A];
#pragma unroll
    for (int k = 0; k < A; ++k) a[k] = base[B * k * LS];
    if (SIGN < 0) {
      dft<A, -1>(a);
#pragma unroll
      for (int k = 1; k < A; ++k) a[k] = cmul(a[k], tw[t2 * A + k]);
    } else {
#pragma unroll
      for (int k = 1; k < A; ++k) a[k] = cmulc(a[k], tw[t2 * A + k]);
      dft<A, 1>(a);
    }
#pragma unroll
    for (int k = 0; k < A; ++k) base[B * k * LS] = a[k];
  }
  __syncthreads();
}

// Stage B of the n column transforms (contiguous in the permuted frequency order along x);
// ld(x, y) supplies the input when LOAD is set (the first stage of the shift transforms).
template <int n, int SIGN, bool LOAD, class LD>
__device__ __forceinline__ void cols_stage_b(float2* G, LD ld) {
  constexpr int A = FusedShape<n>::A, B = FusedShape<n>::B, LS = FusedShape<n>::LS;
  for (int task = threadIdx.x; task < n * A; task += blockDim.x) {
    const int l = task % n, k1 = task / n;
    float2* base = G + l + B * k1 * LS;
    float2 b[B];
#pragma unroll
    for (int t = 0; t < B; ++t) b[t] = LOAD ? ld(B * k1 + t, l) : base[t * LS];
    dft<B, SIGN>(b);
#pragma unroll
    for (int t = 0; t < B; ++t) base[t * LS] = b[t];
  }
  __syncthreads();
}

template <int n>
constexpr size_t i3_fused_smem_bytes() {   // twiddles (two orders), the field (padded rows), psi'_j
  return (size_t)(2 * n + n * (n + 1)) * sizeof(float2) + (size_t)n * n * sizeof(float);
}

// Accumulation modes of k_i3_fused:
//   0  pairs p of shifted fields (Sigma_p = S_2p + i S_2p+1) against one real w_a; the last stage
//      reads and writes the unit's partial sum for every a;
//   1  as 0, with the four a of one (m, p) accumulated in per-thread complex registers and the
//      partial sum updated once per (m, p);
//   2  pairs of w (w_2q + i w_2q+1, the fine-grid field as stored) against one real shifted field
//      S_b: Psi' maps real fields to real fields, so Re and Im of the result carry a = 2q and
//      2q + 1, and K3_b = sum_q [eta_2q S_2q Re + eta_2q+1 S_2q+1 Im] accumulates in one real
//      register per element over the two q of one (m, b); the partial sum's b component is
//      updated once per (m, b).  Half the accumulator registers of mode 1, so 1024 threads fit.
template <int n, int NT, int MINB, int MODE>
__global__ void __launch_bounds__(NT, MINB) k_i3_fused(const I3Jobs<float> jobs, float2* ws,
                                                    const float2* __restrict__ gtw) {
  using C2 = float2;
  constexpr int A = FusedShape<n>::A, B = FusedShape<n>::B, LS = FusedShape<n>::LS, P = FusedShape<n>::P;
  constexpr int TPT = n * B / NT;   // row tasks (row, t2) per thread in the fused row stages
  static_assert(TPT >= 1 && TPT * NT == n * B, "whole row tasks per thread");
  static_assert(MODE >= 0 && MODE <= 2, "accumulation mode");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);                   // tw[t2 A + k1] (stage-order lanes)
  C2* twT = tw + n;                                           // twT[k1 B + t2] = tw[t2 A + k1]
  C2* G = twT + n;                                            // [n][LS]
  float* psm = reinterpret_cast<float*>(G + n * LS);          // psi'_j of the current unit, [n][n]
  __shared__ unsigned char xmask[n];
  for (int pos = threadIdx.x; pos < n; pos += blockDim.x) {
    const int k = freq_of_pos<n>(pos);
    xmask[pos] = ((k < n / 4) || (k >= n - n / 4)) ? 1 : 0;
    twT[(pos % A) * B + pos / A] = gtw[pos];
  }
  load_twiddles<n>(tw, gtw);
  C2* Sig = ws + (size_t)blockIdx.x * 3 * P;   // modes 0, 1: [2][P] complex pairs; mode 2: [4][P] real
  float* Sgr = reinterpret_cast<float*>(Sig);
  const int tid = threadIdx.x;
  // row tasks of this thread in the fused stages: (l, t2) with t2 = tid mod B fixed (NT is a multiple
  // of B), l = (tid + k NT) / B
  const int t2 = tid % B;
  for (int gunit = blockIdx.x; gunit < jobs.total; gunit += gridDim.x) {
    const I3Job<float>& jb = jobs.job[i3_job_of(jobs, gunit)];
    const int unit = gunit - jb.unit_begin;
    const int J = jb.J, M = jb.M, nmc = jb.nmc, mch = jb.mch;
    const C2* what = jb.what;
    const C2* __restrict__ phase = jb.phase;
    const int c = unit / (J * nmc);
    const int j = (unit / nmc) % J;
    const int mc = unit % nmc;
    C2* acc = jb.K3part + (size_t)unit * 2 * P;
    {
      const float4* src = reinterpret_cast<const float4*>(jb.psip_s + (size_t)j * P);
      float4* dst = reinterpret_cast<float4*>(psm);
      for (int i4 = tid; i4 < P / 4; i4 += NT) dst[i4] = src[i4];
      __syncthreads();
    }
    const C2* wf = jb.wfine + (size_t)c * 2 * P;
    const int m0 = mc * mch, m1 = min(M, m0 + mch);
    for (int m = m0; m < m1; ++m) {
      const C2* px = phase + ((size_t)j * M + m) * 2 * n;
      const C2* py = px + n;
      const bool first_m = (m == m0);
      // shifted pairs: inverse column transforms (the phase-multiplied Xi coefficients are loaded
      // in the first stage), inverse row transforms (the last stage stores to global memory)
      for (int p = 0; p < 2; ++p) {
        const C2* in = what + ((size_t)c * 4 + p) * P;
        cols_stage_b<n, 1, true>(G, [&](int ix, int iy) {
          return (xmask[ix] && xmask[iy]) ? cmul(in[ix * n + iy], cmul(px[ix], py[iy])) : zero2<float>();
        });
        cols_stage_a<n, 1>(G, tw);
        rows_stage_b<n, 1>(G);
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
          const int l = (tid + k * NT) / B;
          C2 v[A];
#pragma unroll
          for (int k1 = 0; k1 < A; ++k1) v[k1] = G[l * LS + B * k1 + t2];
#pragma unroll
          for (int k1 = 1; k1 < A; ++k1) v[k1] = cmulc(v[k1], twT[k1 * B + t2]);
          dft<A, 1>(v);
#pragma unroll
          for (int t1 = 0; t1 < A; ++t1) {
            const int idx = l * n + B * t1 + t2;
            if constexpr (MODE == 2) {
              Sgr[(size_t)(2 * p) * P + idx] = v[t1].x;
              Sgr[(size_t)(2 * p + 1) * P + idx] = v[t1].y;
            } else {
              Sig[(size_t)p * P + idx] = v[t1];
            }
          }
        }
        __syncthreads();
      }
      // convolutions: 4 (outer) x 2 (inner) per m
      for (int o = 0; o < 4 / (MODE == 2 ? 1 : 2); ++o) {
        C2* accp = acc + (size_t)(MODE == 2 ? (o >> 1) : o) * P;
        constexpr int NI = MODE == 2 ? 2 : 4;
        C2 racc[MODE == 1 ? TPT : 1][A];
        float racr[MODE == 2 ? TPT : 1][A];
        for (int i = 0; i < NI; ++i) {
          // MODE 0/1: o = p (shifted pair), i = a;  MODE 2: o = b (real shifted field), i = q (w pair)
          const int a = MODE == 2 ? -1 : i;
          // forward row transforms of the product: stage A with the product formed on load
#pragma unroll
          for (int k = 0; k < TPT; ++k) {
            const int l = (tid + k * NT) / B;
            C2 v[A];
#pragma unroll
            for (int t1 = 0; t1 < A; ++t1) {
              const int idx = l * n + B * t1 + t2;
              if constexpr (MODE == 2) {
                v[t1] = cscale(wf[(size_t)i * P + idx], Sgr[(size_t)o * P + idx]);
              } else {
                const C2 z = wf[(size_t)(a >> 1) * P + idx];
                v[t1] = cscale(Sig[(size_t)o * P + idx], (a & 1) ? z.y : z.x);
              }
            }
            dft<A, -1>(v);
#pragma unroll
            for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], twT[k1 * B + t2]);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) G[l * LS + B * k1 + t2] = v[k1];
          }
          __syncthreads();
          rows_stage_b<n, -1>(G);
          fft_conv_lines<n>(G, n, 1, LS, tw, [&](int l, int pos) { return psm[pos * n + l]; });   // columns
          rows_stage_b<n, 1>(G);
          // inverse row stage A, multiplied and accumulated
#pragma unroll
          for (int k = 0; k < TPT; ++k) {
            const int l = (tid + k * NT) / B;
            C2 v[A];
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) v[k1] = G[l * LS + B * k1 + t2];
#pragma unroll
            for (int k1 = 1; k1 < A; ++k1) v[k1] = cmulc(v[k1], twT[k1 * B + t2]);
            dft<A, 1>(v);
#pragma unroll
            for (int t1 = 0; t1 < A; ++t1) {
              const int idx = l * n + B * t1 + t2;
              if constexpr (MODE == 2) {
                // eta = (1, -1, -1, -1): S_2q carries +1 only for q = 0
                const float s0 = Sgr[(size_t)(2 * i) * P + idx], s1 = Sgr[(size_t)(2 * i + 1) * P + idx];
                const float t = fmaT(i == 0 ? s0 : -s0, v[t1].x, -s1 * v[t1].y);
                racr[k][t1] = (i == 0) ? t : racr[k][t1] + t;
              } else {
                const C2 sv = Sig[(size_t)(a >> 1) * P + idx];
                const float f = (a == 0 ? 1.f : -1.f) * ((a & 1) ? sv.y : sv.x);
                if constexpr (MODE == 1) {
                  if (a == 0) racc[k][t1] = mk2(f * v[t1].x, f * v[t1].y);
                  else racc[k][t1] = mk2(fmaT(f, v[t1].x, racc[k][t1].x), fmaT(f, v[t1].y, racc[k][t1].y));
                } else {
                  const C2 d = (first_m && a == 0) ? zero2<float>() : accp[idx];
                  accp[idx] = mk2(fmaT(f, v[t1].x, d.x), fmaT(f, v[t1].y, d.y));
                }
              }
            }
          }
          __syncthreads();
        }
        // the unit's partial sum: written at the chunk's first m, accumulated afterwards
        if constexpr (MODE == 1) {
#pragma unroll
          for (int k = 0; k < TPT; ++k) {
            const int l = (tid + k * NT) / B;
#pragma unroll
            for (int t1 = 0; t1 < A; ++t1) {
              const int idx = l * n + B * t1 + t2;
              accp[idx] = first_m ? racc[k][t1] : cadd(accp[idx], racc[k][t1]);
            }
          }
        } else if constexpr (MODE == 2) {
          float* accr = reinterpret_cast<float*>(accp) + (o & 1);    // component b of pair b >> 1
#pragma unroll
          for (int k = 0; k < TPT; ++k) {
            const int l = (tid + k * NT) / B;
#pragma unroll
            for (int t1 = 0; t1 < A; ++t1) {
              const int idx = 2 * (l * n + B * t1 + t2);
              accr[idx] = first_m ? racr[k][t1] : accr[idx] + racr[k][t1];
            }
          }
        }
      }
    }
    __syncthreads();   // psm is reloaded by the next unit
  }
}

// --------------------------------------------------------------------------
// The fused FP32 I3 kernel with warp-local passes (padded grid of 128 points, 512 threads, the
// accumulation of mode 1).  In the row passes warp w owns rows [8 w, 8 w + 8), in the column passes
// warp pair g owns columns [16 g, 16 g + 16): their stages synchronise with __syncwarp or a named
// barrier of the pair, and the block synchronises only where the passes change ownership (rows ->
// columns, columns -> rows), twice per convolution instead of seven times, so warps in different
// stages overlap their shared-memory, global and arithmetic latencies.  Field layout: element
// (x, y) at x * WL_PITCH + y + y / 16 (one pad word per 16 elements, row pitch 146 = 2 mod 16),
// which keeps every stage's accesses free of bank conflicts under the lane mappings below.
// --------------------------------------------------------------------------
constexpr int kWlN = 128, kWlThreads = 512, kWlPitch = 146;

__device__ __forceinline__ int wl_addr(int x, int y) { return x * kWlPitch + y + (y >> 4); }

__device__ __forceinline__ void wl_pair_sync(int g) {   // the two warps of pair g (ids 1..8)
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(64) : "memory");
}

constexpr int kWlPsiPitch = kWlN + 1;   // psi'_j rows padded: the two half-warps of a column stage
                                         // read rows 16 apart, which would share banks at pitch 128
constexpr size_t i3_wl_smem_bytes() {    // twiddles (two orders), the skewed field, psi'_j
  return (size_t)(2 * kWlN + kWlN * kWlPitch) * sizeof(float2) + (size_t)kWlN * kWlPsiPitch * sizeof(float);
}

// Column pass stages of warp pair g on its 16 columns (tt = thread index within the pair).
// Stage A: tasks (column c = tt mod 16, t2 = tt / 16 + 4 i); stage B: (c, k1 = tt / 16 + 4 i).
template <int SIGN>
__device__ __forceinline__ void wl_cols_stage_a(float2* G, const float2* tw, int g, int tt) {
  constexpr int A = Split<kWlN>::A, B = Split<kWlN>::B;
  const int y = 16 * g + (tt & 15);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int t2 = (tt >> 4) + 4 * i;
    float2 v[A];
#pragma unroll
    for (int k = 0; k < A; ++k) v[k] = G[wl_addr(B * k + t2, y)];
    if (SIGN < 0) {
      dft<A, -1>(v);
#pragma unroll
      for (int k = 1; k < A; ++k) v[k] = cmul(v[k], tw[t2 * A + k]);
    } else {
#pragma unroll
      for (int k = 1; k < A; ++k) v[k] = cmulc(v[k], tw[t2 * A + k]);
      dft<A, 1>(v);
    }
#pragma unroll
    for (int k = 0; k < A; ++k) G[wl_addr(B * k + t2, y)] = v[k];
  }
}

// Row pass stage B of warp w on its 8 rows: tasks (row 8 w + (lane mod 8), k1 = lane / 8 + 4 i).
template <int SIGN>
__device__ __forceinline__ void wl_rows_stage_b(float2* G, int w, int lane) {
  constexpr int B = Split<kWlN>::B;
  const int x = 8 * w + (lane & 7);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int k1 = (lane >> 3) + 4 * i;
    float2 b[B];
#pragma unroll
    for (int t = 0; t < B; ++t) b[t] = G[wl_addr(x, B * k1 + t)];
    dft<B, SIGN>(b);
#pragma unroll
    for (int t = 0; t < B; ++t) G[wl_addr(x, B * k1 + t)] = b[t];
  }
}

// The shifted pair S = S_jm(w_p) (eq. approxH-JM's spectral shift: the phase-multiplied Xi
// coefficients of `in`, inverse 2-D transform) into S[x n + y] (natural order) on the warp-local
// passes.  The coefficients are zero outside Xi x Xi, a quarter of the padded grid: in the permuted
// order a stage-B line of 16 holds Xi frequencies at t = 0..3, 12..15 only, so the rows are
// transformed first and only the four Xi rows of each warp (stage B with its first radix-2 stage
// reduced, stage A), then every column from those rows alone (stage B reduced in the same way, stage
// A storing S, coalesced along y).  The other rows of G are not touched.  Ends with a block barrier:
// S is complete for every thread and G is free.
__device__ __forceinline__ void wl_shift(float2* G, const float2* tw, const float2* twT, const float2* in,
                                         const float2* px, const float2* py, float2* S, int w, int lane, int g,
                                         int tt) {
  using C2 = float2;
  constexpr int n = kWlN, A = Split<n>::A, B = Split<n>::B;
  static_assert(A == 8 && B == 16, "Xi pattern of the 8 x 16 split");
  const int xr0 = 8 * w + 4 * (w & 1);   // this warp's Xi rows: x mod 16 in 0..3 or 12..15
  {
    const int x = xr0 + (lane & 3), k1 = lane >> 2;
    const C2 pxx = px[x];
    C2 b[B];
#pragma unroll
    for (int t = 0; t < B; ++t) {
      if (t < 4 || t >= 12) {
        const int y = B * k1 + t;
        b[t] = cmul(in[x * n + y], cmul(pxx, py[y]));
      } else {
        b[t] = zero2<float>();
      }
    }
    dft16_xi<1>(b);
#pragma unroll
    for (int t = 0; t < B; ++t) G[wl_addr(x, B * k1 + t)] = b[t];
  }
  __syncwarp();
  const int t2r = lane & 15;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int x = xr0 + (lane >> 4) + 2 * i;
    C2 v[A];
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) v[k1] = G[wl_addr(x, B * k1 + t2r)];
#pragma unroll
    for (int k1 = 1; k1 < A; ++k1) v[k1] = cmulc(v[k1], twT[k1 * B + t2r]);
    dft<A, 1>(v);
#pragma unroll
    for (int t1 = 0; t1 < A; ++t1) G[wl_addr(x, B * t1 + t2r)] = v[t1];
  }
  __syncthreads();
  const int y = 16 * g + (tt & 15);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int k1 = (tt >> 4) + 4 * i;
    C2 b[B];
#pragma unroll
    for (int t = 0; t < B; ++t) b[t] = (t < 4 || t >= 12) ? G[wl_addr(B * k1 + t, y)] : zero2<float>();
    dft16_xi<1>(b);
#pragma unroll
    for (int t = 0; t < B; ++t) G[wl_addr(B * k1 + t, y)] = b[t];
  }
  wl_pair_sync(g);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int t2 = (tt >> 4) + 4 * i;
    C2 v[A];
#pragma unroll
    for (int k = 0; k < A; ++k) v[k] = G[wl_addr(B * k + t2, y)];
#pragma unroll
    for (int k = 1; k < A; ++k) v[k] = cmulc(v[k], tw[t2 * A + k]);
    dft<A, 1>(v);
#pragma unroll
    for (int k = 0; k < A; ++k) S[(B * k + t2) * n + y] = v[k];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kWlThreads, 1) k_i3_wl(const I3Jobs<float> jobs, float2* ws,
                                                        const float2* __restrict__ gtw) {
  using C2 = float2;
  constexpr int n = kWlN, A = Split<n>::A, B = Split<n>::B, P = n * n, NT = kWlThreads;
  constexpr int TPT = n * B / NT;   // 4 row tasks (row, t2) per thread in the fused row stages
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);                   // tw[t2 A + k1]
  C2* twT = tw + n;                                           // twT[k1 B + t2]
  C2* G = twT + n;                                            // skewed field
  float* psm = reinterpret_cast<float*>(G + n * kWlPitch);    // psi'_j of the current unit, [n][kWlPsiPitch]
  for (int pos = threadIdx.x; pos < n; pos += blockDim.x) twT[(pos % A) * B + pos / A] = gtw[pos];
  load_twiddles<n>(tw, gtw);
  C2* Sig = ws + (size_t)blockIdx.x * 3 * P;   // [2][P]
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, g = w >> 1, tt = tid & 63;
  const int t2r = lane & 15;                   // t2 of this thread's row tasks
  // row task k of this thread: row 8 w + lane / 16 + 2 k, t2 = lane mod 16
  auto row_of = [&](int k) { return 8 * w + (lane >> 4) + 2 * k; };
  for (int gunit = blockIdx.x; gunit < jobs.total; gunit += gridDim.x) {
    const I3Job<float>& jb = jobs.job[i3_job_of(jobs, gunit)];
    const int unit = gunit - jb.unit_begin;
    const int J = jb.J, M = jb.M, nmc = jb.nmc, mch = jb.mch;
    const C2* what = jb.what;
    const C2* __restrict__ phase = jb.phase;
    const int c = unit / (J * nmc);
    const int j = (unit / nmc) % J;
    const int mc = unit % nmc;
    C2* acc = jb.K3part + (size_t)unit * 2 * P;
    {
      const float4* src = reinterpret_cast<const float4*>(jb.psip_s + (size_t)j * P);
      for (int i4 = tid; i4 < P / 4; i4 += NT) {
        const float4 q = src[i4];
        float* d = psm + (4 * i4 / n) * kWlPsiPitch + (4 * i4) % n;
        d[0] = q.x; d[1] = q.y; d[2] = q.z; d[3] = q.w;
      }
      __syncthreads();
    }
    const C2* wf = jb.wfine + (size_t)c * 2 * P;
    const int m0 = mc * mch, m1 = min(M, m0 + mch);
    for (int m = m0; m < m1; ++m) {
      const C2* px = phase + ((size_t)j * M + m) * 2 * n;
      const C2* py = px + n;
      const bool first_m = (m == m0);
      // shifted pairs (S complete for every thread when wl_shift returns)
      for (int p = 0; p < 2; ++p)
        wl_shift(G, tw, twT, what + ((size_t)c * 4 + p) * P, px, py, Sig + (size_t)p * P, w, lane, g, tt);
      for (int p = 0; p < 2; ++p) {
        const C2* Sp = Sig + (size_t)p * P;      // rewritten every m: plain (coherent) loads
        C2* accp = acc + (size_t)p * P;
        C2 racc[TPT][A];
        for (int a = 0; a < 4; ++a) {
          // component im of the fine pair and of the shifted pair, loaded as single floats
          const int im = a & 1;
          const float* __restrict__ wa = reinterpret_cast<const float*>(wf + (size_t)(a >> 1) * P) + im;
          const float* Sa = reinterpret_cast<const float*>(Sig + (size_t)(a >> 1) * P) + im;
          // forward rows of w_a Sigma_p (warp-local): stage A loads the product, stage B
#pragma unroll
          for (int k = 0; k < TPT; ++k) {
            const int x = row_of(k);
            C2 v[A];
#pragma unroll
            for (int t1 = 0; t1 < A; ++t1) {
              const int idx = x * n + B * t1 + t2r;
              v[t1] = cscale(Sp[idx], wa[2 * idx]);
            }
            dft<A, -1>(v);
#pragma unroll
            for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], twT[k1 * B + t2r]);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) G[wl_addr(x, B * k1 + t2r)] = v[k1];
          }
          __syncwarp();
          wl_rows_stage_b<-1>(G, w, lane);
          __syncthreads();
          // columns (pair-local): forward stage A, stage B with psi'_j, inverse stage A
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
          // inverse rows (warp-local): stage B, stage A times eta_a S_a, accumulated over a
          wl_rows_stage_b<1>(G, w, lane);
          __syncwarp();
          const float eta = (a == 0) ? 1.f : -1.f;
#pragma unroll
          for (int k = 0; k < TPT; ++k) {
            const int x = row_of(k);
            float f[A];
#pragma unroll
            for (int t1 = 0; t1 < A; ++t1) f[t1] = eta * Sa[2 * (x * n + B * t1 + t2r)];
            C2 v[A];
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) v[k1] = G[wl_addr(x, B * k1 + t2r)];
#pragma unroll
            for (int k1 = 1; k1 < A; ++k1) v[k1] = cmulc(v[k1], twT[k1 * B + t2r]);
            dft<A, 1>(v);
#pragma unroll
            for (int t1 = 0; t1 < A; ++t1) {
              if (a == 0) racc[k][t1] = mk2(f[t1] * v[t1].x, f[t1] * v[t1].y);
              else racc[k][t1] = mk2(fmaT(f[t1], v[t1].x, racc[k][t1].x), fmaT(f[t1], v[t1].y, racc[k][t1].y));
            }
          }
          __syncwarp();   // this warp's rows of G are rewritten by the next a's forward stage A
        }
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
          const int x = row_of(k);
#pragma unroll
          for (int t1 = 0; t1 < A; ++t1) {
            const int idx = x * n + B * t1 + t2r;
            accp[idx] = first_m ? racc[k][t1] : cadd(accp[idx], racc[k][t1]);
          }
        }
      }
      __syncthreads();   // G and Sig are rewritten by the next m's shift transforms
    }
    __syncthreads();     // psm is reloaded by the next unit
  }
}
