// I3 (Hu-Ying term, eq. approxH-JM) for fields larger than one block's shared memory (the FP64 form):
// staged row and column passes over chunks of RC rows / CC lines, with every global load and store
// of a convolution fused into a line stage.  Included by collision_kernels.cuh inside its anonymous
// namespace.
//
// The block's scratch field between the passes is stored transposed, G'[ky][x] (ky in the row
// transform's permuted order), so that each pass reads and writes it with coalesced accesses
// straight from its line stages:
//   row pass, forward:  stage A loads w_a Sigma_p (tasks (row, t2), t2-fastest), stage B stores its
//                       B spectral values of a row into B lines of G' (lanes = consecutive rows);
//   line pass (x):      stage A loads a line of G' (contiguous in x), stage B with the psi'_j
//                       multiplier between forward and inverse, stage A stores the line back;
//   row pass, inverse:  stage B loads B lines of G' at its row (lanes = consecutive rows), stage A
//                       multiplies by eta_a S_a and accumulates into the unit's partial sum.
// Shared memory holds one chunk at a time; no pass copies a chunk through it without transforming.
#pragma once

template <int n, class T, int NTH, int CB, int MINB>
__global__ void __launch_bounds__(NTH, MINB)
    k_i3_sf(const I3Jobs<T> jobs, typename Vec2Of<T>::type* ws, const typename Vec2Of<T>::type* __restrict__ gtw) {
  using C2 = typename Vec2Of<T>::type;
  constexpr int A = Split<n>::A, B = Split<n>::B, P = n * n;
  constexpr int RC = Chunk<n, sizeof(C2), CB>::RC, CC = Chunk<n, sizeof(C2), CB>::CC, LS = Chunk<n, sizeof(C2), CB>::LS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* tw = reinterpret_cast<C2*>(smem_raw);   // tw[t2 A + k1]
  C2* twT = tw + n;                           // twT[k1 B + t2] = tw[t2 A + k1] (t2-fastest lanes)
  C2* sm = twT + n;                           // one chunk: [RC][LS] rows, or [CC][LS] lines of G'
  static_assert(RC == CC, "row and line chunks share the buffer");
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
  for (int pos = threadIdx.x; pos < n; pos += NTH) twT[(pos % A) * B + pos / A] = gtw[pos];
  load_twiddles<n>(tw, gtw);
  const int tid = threadIdx.x;
  C2* slot = ws + (size_t)blockIdx.x * 3 * P;
  C2* Sig = slot;           // [2][P]
  C2* G = slot + 2 * P;     // G'[ky][x] between the passes
  for (int gunit = blockIdx.x; gunit < jobs.total; gunit += gridDim.x) {
    const I3Job<T>& jb = jobs.job[i3_job_of(jobs, gunit)];
    const int unit = gunit - jb.unit_begin;
    const int J = jb.J, M = jb.M, nmc = jb.nmc, mch = jb.mch;
    const C2* what = jb.what;
    const C2* __restrict__ phase = jb.phase;
    const int c = unit / (J * nmc);
    const int j = (unit / nmc) % J;
    const int mc = unit % nmc;
    C2* acc = jb.K3part + (size_t)unit * 2 * P;
    zero_fields(acc, 2 * P);
    const T* __restrict__ psp = jb.psip_s + (size_t)j * P;
    const C2* wf = jb.wfine + (size_t)c * 2 * P;
    const int m0 = mc * mch, m1 = min(M, m0 + mch);
    for (int m = m0; m < m1; ++m) {
      const C2* px = phase + ((size_t)j * M + m) * 2 * n;
      const C2* py = px + n;
      // shifted pairs, as in k_i3 (only the Xi columns are transformed along x)
      for (int p = 0; p < 2; ++p) {
        const C2* in = what + ((size_t)c * 4 + p) * P;
        C2* S = Sig + (size_t)p * P;
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
        const bool pos_eta = (a == 0);   // eta_a = +1 for a = 0, -1 otherwise
        for (int p = 0; p < 2; ++p) {
          const C2* Sp = Sig + (size_t)p * P;
          C2* accp = acc + (size_t)p * P;
          // ---- row pass, forward: rows r0..r0+RC into lines of G' ----
          for (int r0 = 0; r0 < n; r0 += RC) {
            for (int task = tid; task < RC * B; task += NTH) {
              const int r = task / B, t2 = task % B, row = r0 + r;
              C2 v[A];
#pragma unroll
              for (int t1 = 0; t1 < A; ++t1) {
                const int idx = row * n + B * t1 + t2;
                const C2 z = wa[idx];
                v[t1] = cscale(Sp[idx], im ? z.y : z.x);
              }
              dft<A, -1>(v);
#pragma unroll
              for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], twT[k1 * B + t2]);
#pragma unroll
              for (int k1 = 0; k1 < A; ++k1) sm[r * LS + B * k1 + t2] = v[k1];
            }
            __syncthreads();
            for (int task = tid; task < RC * A; task += NTH) {
              const int r = task % RC, k1 = task / RC;
              const C2* base = sm + r * LS + B * k1;
              C2 b[B];
#pragma unroll
              for (int t = 0; t < B; ++t) b[t] = base[t];
              dft<B, -1>(b);
#pragma unroll
              for (int t = 0; t < B; ++t) G[(B * k1 + t) * n + r0 + r] = b[t];
            }
            __syncthreads();
          }
          // ---- line pass along x: forward, psi'_j, inverse on lines c0..c0+CC of G' ----
          for (int c0 = 0; c0 < n; c0 += CC) {
            for (int task = tid; task < CC * B; task += NTH) {
              const int cc = task / B, t2 = task % B;
              C2 v[A];
#pragma unroll
              for (int t1 = 0; t1 < A; ++t1) v[t1] = G[(c0 + cc) * n + B * t1 + t2];
              dft<A, -1>(v);
#pragma unroll
              for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], twT[k1 * B + t2]);
#pragma unroll
              for (int k1 = 0; k1 < A; ++k1) sm[cc * LS + B * k1 + t2] = v[k1];
            }
            __syncthreads();
            for (int task = tid; task < CC * A; task += NTH) {
              const int cc = task % CC, k1 = task / CC;
              C2* base = sm + cc * LS + B * k1;
              C2 b[B];
#pragma unroll
              for (int t = 0; t < B; ++t) b[t] = base[t];
              dft<B, -1>(b);
              T sc[B];
#pragma unroll
              for (int t = 0; t < B; ++t) sc[t] = psp[(B * k1 + t) * n + c0 + cc];
              dft_scaled<B, 1>(b, sc);
#pragma unroll
              for (int t = 0; t < B; ++t) base[t] = b[t];
            }
            __syncthreads();
            for (int task = tid; task < CC * B; task += NTH) {
              const int cc = task / B, t2 = task % B;
              C2 v[A];
#pragma unroll
              for (int k1 = 0; k1 < A; ++k1) v[k1] = sm[cc * LS + B * k1 + t2];
#pragma unroll
              for (int k1 = 1; k1 < A; ++k1) v[k1] = cmulc(v[k1], twT[k1 * B + t2]);
              dft<A, 1>(v);
#pragma unroll
              for (int t1 = 0; t1 < A; ++t1) G[(c0 + cc) * n + B * t1 + t2] = v[t1];
            }
            __syncthreads();
          }
          // ---- row pass, inverse, accumulated with eta_a S_a ----
          for (int r0 = 0; r0 < n; r0 += RC) {
            for (int task = tid; task < RC * A; task += NTH) {
              const int r = task % RC, k1 = task / RC;
              C2* base = sm + r * LS + B * k1;
              C2 b[B];
#pragma unroll
              for (int t = 0; t < B; ++t) b[t] = G[(B * k1 + t) * n + r0 + r];
              dft<B, 1>(b);
#pragma unroll
              for (int t = 0; t < B; ++t) base[t] = b[t];
            }
            __syncthreads();
            for (int task = tid; task < RC * B; task += NTH) {
              const int r = task / B, t2 = task % B, row = r0 + r;
              C2 v[A];
#pragma unroll
              for (int k1 = 0; k1 < A; ++k1) v[k1] = sm[r * LS + B * k1 + t2];
#pragma unroll
              for (int k1 = 1; k1 < A; ++k1) v[k1] = cmulc(v[k1], twT[k1 * B + t2]);
              dft<A, 1>(v);
#pragma unroll
              for (int t1 = 0; t1 < A; ++t1) {
                const int idx = row * n + B * t1 + t2;
                const C2 s = Sa[idx];
                const T f = im ? s.y : s.x;
                const C2 d = accp[idx];
                accp[idx] = pos_eta ? mk2(fmaT(f, v[t1].x, d.x), fmaT(f, v[t1].y, d.y))
                                    : mk2(fmaT(-f, v[t1].x, d.x), fmaT(-f, v[t1].y, d.y));
              }
            }
            __syncthreads();
          }
        }
      }
    }
  }
}

template <int n, class T, int CB>
constexpr size_t i3_sf_smem_bytes() {   // twiddles (two orders) and one chunk of RC padded lines
  using C2 = typename Vec2Of<T>::type;
  return (size_t)(2 * n + Chunk<n, sizeof(C2), CB>::RC * Chunk<n, sizeof(C2), CB>::LS) * sizeof(C2);
}
