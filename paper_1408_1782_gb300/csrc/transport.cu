// Transport (Sec. 4, eq. slopeLimiterStep with eq. minmod), boundary ghost
// cells (Sec. 2: periodic, Dirichlet, Maxwell), the precession term
// -i[B.sigma, W] = 2 (B x w).sigma inside Heun's RK2, and the moments
// (eqs. density, velocity, internal_energy).  All kernels stream the state
// [cell][4][ix][iy] once; consecutive threads take consecutive velocities so
// every access is coalesced.
#include "internal.h"

#include <cstdlib>

namespace qbe {

namespace {

// eq. minmod: a if |a| <= |b| and ab > 0; b if |b| < |a| and ab > 0; 0 otherwise.  Signs and
// magnitudes are compared on the IEEE bit patterns (integer pipe) instead of FP64 products and
// compares: for finite a, b the value is the same (a zero operand yields zero either way) except
// where the FP64 product a*b would underflow to zero (|a b| < 5e-324), where this returns the
// smaller operand instead of zero.
__device__ __forceinline__ double minmod(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  if ((ia ^ ib) < 0) return 0.0;                                   // opposite signs
  const long long ma = ia & 0x7fffffffffffffffLL, mb = ib & 0x7fffffffffffffffLL;
  return ma <= mb ? a : b;
}

// Outgoing number flux of the boundary cells (Maxwell walls):
//   fbar[0] = dv^2 sum_{v_x < 0} 2 w0(x=0 cell) |v_x|,  fbar[1] = dv^2 sum_{v_x > 0} 2 w0(last cell) |v_x|
__global__ void __launch_bounds__(256) k_wall_flux(const double* __restrict__ W, int Nx, int N, double L,
                                                   double* fbar) {
  __shared__ double red[256];
  const int side = blockIdx.x;
  const int NN = N * N;
  const double dv = 2.0 * L / N;
  const double* w0 = W + (size_t)(side == 0 ? 0 : Nx - 1) * 4 * NN;
  double acc = 0.0;
  for (int i = threadIdx.x; i < NN; i += blockDim.x) {
    const int ix = i / N;
    const double vx = dv * (ix - N / 2);
    const bool out = side == 0 ? (vx < 0.0) : (vx > 0.0);
    if (out) acc += 2.0 * w0[i] * fabs(vx);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) fbar[side] = red[0] * dv * dv;
}

struct Ghost {
  int kind;
  double alpha, ZL, ZR;
  const double* phiL;
  const double* phiR;
  const double* fbar;
};

// Value of component c at velocity (ix, iy) in cell jj (may be a ghost cell).
// The sign of v_x = dv (ix - N/2) is that of ix - N/2.
__device__ __forceinline__ double cell_value(const double* __restrict__ W, int jj, int c, int ix, int iy, int Nx,
                                             int N, const Ghost& g) {
  const size_t NN = (size_t)N * N;
  const size_t off = (size_t)c * NN + (size_t)ix * N + iy;
  if (jj >= 0 && jj < Nx) return W[(size_t)jj * 4 * NN + off];
  if (g.kind == QBE_PERIODIC) {
    const int w = (jj % Nx + Nx) % Nx;
    return W[(size_t)w * 4 * NN + off];
  }
  const bool left = jj < 0;
  const int b = left ? 0 : Nx - 1;
  const bool incoming = left ? (ix > N / 2) : (ix < N / 2);
  if (!incoming) return W[(size_t)b * 4 * NN + off];          // outgoing or v_x = 0: copy of the boundary cell
  const double* phi = left ? g.phiL : g.phiR;
  if (g.kind == QBE_DIRICHLET) return phi[off];
  // Maxwell: (1 - alpha) W_b(-v_x, v_y) + alpha W_FD(v) Fbar / Z
  const int mx = N - ix;                                        // index of -k_x
  const double spec = (mx < N) ? W[(size_t)b * 4 * NN + (size_t)c * NN + (size_t)mx * N + iy] : 0.0;
  const double fb = left ? g.fbar[0] : g.fbar[1];
  const double Z = left ? g.ZL : g.ZR;
  return (1.0 - g.alpha) * spec + g.alpha * phi[off] * (fb / Z);
}

// Coefficients of eq. slopeLimiterStep in the upwind frame for a velocity with |v_x| = av:
// c_g = 2 k |v_x| and c_l = k (1 - |nu|) |v_x|, k = tau / (2 dx), |nu| = tau |v_x| / dx, kt = tau / dx.
__host__ __device__ __forceinline__ void advect_coefs(double av, double kt, double& cg, double& cl) {
  cg = kt * av;
  cl = 0.5 * kt * (1.0 - kt * av) * av;
}

// The table of both coefficients per velocity row, built on the host for each sub-step and passed
// by value (__grid_constant__: read from the constant bank, one broadcast per warp for N >= 32).
// The device does no FP64 division and no per-block table set-up: on this part FP64 arithmetic
// issues at about two lanes per clock per SM, so it is the bound of the transport kernels.
struct AdvectCoefs {
  double cg[128], cl[128];     // N <= 128
};

AdvectCoefs make_advect_coefs(int N, double dv, double kt) {
  AdvectCoefs t{};
  for (int ix = 0; ix < N; ++ix) advect_coefs(dv * std::abs(ix - N / 2), kt, t.cg[ix], t.cl[ix]);
  return t;
}

// One grid row per (cell j, component c) (blockIdx.y = 4 j + c); threads over the N*N velocities,
// so the stencil cells and their ghost rules are uniform over a block and a warp shares v_x
// (N >= 32).  With s = sgn v_x and the upwind-ordered stencil q_d = W(j + s (d - 2)), d = 0..3,
// eq. slopeLimiterStep reduces to
//   W_out = q2 - c_g (q2 - q1) + c_l (minmod(q2 - q1, q1 - q0) - minmod(q3 - q2, q2 - q1)),
// c_g = 2 k |v_x|, c_l = k (1 - |nu|) |v_x|, k = tau / (2 dx), nu = tau v_x / dx: the Godunov term
// and the limiter term (sgn nu - nu)/2 of the downwind slope vanish.  (v_x = 0 leaves W unchanged.)
// The two coefficients per velocity row are computed once per block; what remains per output is
// three differences, one subtraction and two FMAs in FP64, the limiter on the integer pipe.
__global__ void __launch_bounds__(256) k_advect(const double* __restrict__ W, double* __restrict__ Wout, int Nx,
                                                int N, const __grid_constant__ AdvectCoefs cf, Ghost g) {
  const int NN = N * N;
  const int j = blockIdx.y >> 2, c = blockIdx.y & 3;
  double* out = Wout + (size_t)blockIdx.y * NN;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < NN; v += gridDim.x * blockDim.x) {
    const int ix = v / N, iy = v - ix * N;
    const int sgn = ix < N / 2 ? -1 : 1;
    const double q0 = cell_value(W, j - 2 * sgn, c, ix, iy, Nx, N, g);
    const double q1 = cell_value(W, j - sgn, c, ix, iy, Nx, N, g);
    const double q2 = cell_value(W, j, c, ix, iy, Nx, N, g);
    const double q3 = cell_value(W, j + sgn, c, ix, iy, Nx, N, g);
    const double b = q2 - q1;
    const double su = minmod(b, q1 - q0);
    const double s0 = minmod(q3 - q2, b);
    double r = fma(-cf.cg[ix], b, q2);
    r = fma(cf.cl[ix], su - s0, r);
    out[v] = r;
  }
}

__device__ __forceinline__ void prec(const double* b, double w1, double w2, double w3, double& p1, double& p2,
                                     double& p3) {
  p1 = 2.0 * (b[1] * w3 - b[2] * w2);
  p2 = 2.0 * (b[2] * w1 - b[0] * w3);
  p3 = 2.0 * (b[0] * w2 - b[1] * w1);
}

// F0 = C + 2 (B x w).sigma;  W1 = W + dt F0
// blockIdx.y = cell, threads over the velocities.
__global__ void __launch_bounds__(256) k_rk1(const double* __restrict__ W, const double* __restrict__ C,
                                             const double* __restrict__ B, double dt, double* __restrict__ F0,
                                             double* __restrict__ W1, int Nx, int N) {
  const int NN = N * N;
  const int cell = blockIdx.y;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < NN; v += gridDim.x * blockDim.x) {
    const size_t base = (size_t)cell * 4 * NN + v;
    const double w0 = W[base], w1 = W[base + NN], w2 = W[base + 2 * NN], w3 = W[base + 3 * NN];
    double p1, p2, p3;
    prec(B + 3 * cell, w1, w2, w3, p1, p2, p3);
    const double f0 = C[base], f1 = C[base + NN] + p1, f2 = C[base + 2 * NN] + p2, f3 = C[base + 3 * NN] + p3;
    F0[base] = f0; F0[base + NN] = f1; F0[base + 2 * NN] = f2; F0[base + 3 * NN] = f3;
    W1[base] = w0 + dt * f0; W1[base + NN] = w1 + dt * f1;
    W1[base + 2 * NN] = w2 + dt * f2; W1[base + 3 * NN] = w3 + dt * f3;
  }
}

// Wout = W + dt/2 (F0 + C1 + 2 (B x w1).sigma)   (Heun)
__global__ void __launch_bounds__(256) k_rk2(const double* W, const double* __restrict__ F0,
                                             const double* __restrict__ C1, const double* __restrict__ W1,
                                             const double* __restrict__ B, double dt, double* Wout, int Nx, int N) {
  const int NN = N * N;
  const int cell = blockIdx.y;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < NN; v += gridDim.x * blockDim.x) {
    const size_t base = (size_t)cell * 4 * NN + v;
    double p1, p2, p3;
    prec(B + 3 * cell, W1[base + NN], W1[base + 2 * NN], W1[base + 3 * NN], p1, p2, p3);
    const double g[4] = {C1[base], C1[base + NN] + p1, C1[base + 2 * NN] + p2, C1[base + 3 * NN] + p3};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const size_t o = base + c * NN;
      Wout[o] = W[o] + 0.5 * dt * (F0[o] + g[c]);
    }
  }
}

// Per cell: rho (4), momentum (2), energy (1), all times dv^2.
__global__ void __launch_bounds__(256) k_moments(const double* __restrict__ W, int N, double L, double* out7) {
  __shared__ double red[7][256];
  const int cell = blockIdx.x;
  const size_t NN = (size_t)N * N;
  const double dv = 2.0 * L / N;
  const double* w = W + (size_t)cell * 4 * NN;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (size_t i = threadIdx.x; i < NN; i += blockDim.x) {
    const int ix = (int)(i / N), iy = (int)(i % N);
    const double vx = dv * (ix - N / 2), vy = dv * (iy - N / 2);
    const double a0 = w[i];
    acc[0] += a0; acc[1] += w[NN + i]; acc[2] += w[2 * NN + i]; acc[3] += w[3 * NN + i];
    const double tr = 2.0 * a0;
    acc[4] += vx * tr; acc[5] += vy * tr; acc[6] += 0.5 * (vx * vx + vy * vy) * tr;
  }
  for (int k = 0; k < 7; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 7; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 7) out7[(size_t)cell * 7 + threadIdx.x] = red[threadIdx.x][0] * dv * dv;
}

// ---------------------------------------------------------------------------
// Adjoint of the transport substep.  In the upwind frame of k_advect (s = sgn v_x, cell index
// m -> W(j + s m)) the update of output cell jo is
//   W_out(jo) = (1 - c_g) W(jo) + c_g W(jo - s) + c_l (sig(jo - s) - sig(jo)),
//   sig(m)    = minmod(W(m + s) - W(m), W(m) - W(m - s)),
// so with the minmod branches frozen at the forward state it is linear in W, and the cotangent
// of any cell i (interior or ghost) is
//   lam_in(i) = (1 - c_g) lam(i) + c_g lam(i + s) + sum_{m in {i - s, i, i + s}} mu(m) dsig(m)/dW(i),
//   mu(m)     = c_l (lam(m + s) - lam(m))        (lam = 0 outside the domain),
// which reads five W and four lam values.  The branch convention is eq. minmod's in the x
// order: zero unless ab > 0; a tie |a| = |b| takes the x-forward difference W(m + 1) - W(m),
// i.e. the first argument for s > 0 and the second for s < 0.  The ghost cells' cotangents
// reach the interior through the ghost rules (Sec. 2): periodic wrap, the copied boundary cell
// (outgoing velocities), the specular image (1 - alpha) W_b(-v_x, v_y) and the diffusive part
// alpha W_FD(v) Fbar / Z with Fbar a linear functional of the boundary cell's w0.
// ---------------------------------------------------------------------------

// Frozen branch of sig: 0 zero, 1 the first argument a, 2 the second b.  Signs and magnitudes
// on the bit patterns; a zero operand gives the zero branch (as ab > 0 fails for it).
__device__ __forceinline__ int minmod_branch(double a, double b, bool tie_a) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const long long ma = ia & 0x7fffffffffffffffLL, mb = ib & 0x7fffffffffffffffLL;
  if ((ia ^ ib) < 0 || ma == 0 || mb == 0) return 0;
  return (ma < mb || (tie_a && ma == mb)) ? 1 : 2;
}

__device__ __forceinline__ double lam_at(const double* __restrict__ lam, int jj, int Nx, size_t off, size_t NN4,
                                         int kind) {
  if (kind == QBE_PERIODIC) jj = (jj % Nx + Nx) % Nx;
  else if (jj < 0 || jj >= Nx) return 0.0;
  return lam[(size_t)jj * NN4 + off];
}

// Cotangent of cell i (any index, ghosts included) at (c, ix, iy), before the ghost rules.
__device__ __forceinline__ double cell_cotangent(const double* __restrict__ W, const double* __restrict__ lam,
                                                 int i, int c, int ix, int iy, int Nx, int N, double cg, double cl,
                                                 const Ghost& g) {
  const int s = ix < N / 2 ? -1 : 1;
  const size_t NN = (size_t)N * N;
  const size_t off = (size_t)c * NN + (size_t)ix * N + iy;
  double w[5], l[4];          // w[e + 2] = W(i + s e), e = -2..2;  l[e + 1] = lam(i + s e), e = -1..2
#pragma unroll
  for (int e = 0; e < 5; ++e) w[e] = cell_value(W, i + s * (e - 2), c, ix, iy, Nx, N, g);
#pragma unroll
  for (int e = 0; e < 4; ++e) l[e] = lam_at(lam, i + s * (e - 1), Nx, off, 4 * NN, g.kind);
  const bool tie_a = s > 0;
  double acc = fma(cg, l[2] - l[1], l[1]);
  // sig(i - s): i is its W(m + s) (branch a: +mu)
  if (minmod_branch(w[2] - w[1], w[1] - w[0], tie_a) == 1) acc = fma(cl, l[1] - l[0], acc);
  // sig(i): i is its W(m) (branch a: -mu, branch b: +mu)
  const int b0 = minmod_branch(w[3] - w[2], w[2] - w[1], tie_a);
  if (b0 != 0) acc = fma(b0 == 1 ? -cl : cl, l[2] - l[1], acc);
  // sig(i + s): i is its W(m - s) (branch b: -mu)
  if (minmod_branch(w[4] - w[3], w[3] - w[2], tie_a) == 2) acc = fma(-cl, l[3] - l[2], acc);
  return acc;
}

// Maxwell walls: gsum[side] = sum over incoming velocities and components of the two ghost
// cells' cotangents times W_FD (the diffusive part's dependence on Fbar).
__global__ void __launch_bounds__(256) k_wall_adj(const double* __restrict__ W, const double* __restrict__ lam,
                                                  int Nx, int N, const __grid_constant__ AdvectCoefs cf, Ghost g,
                                                  double* gsum) {
  __shared__ double red[256];
  const int side = blockIdx.x;
  const int NN = N * N;
  const double* phi = side == 0 ? g.phiL : g.phiR;
  double acc = 0.0;
  for (int t = threadIdx.x; t < 4 * NN; t += blockDim.x) {
    const int c = t / NN, ix = (t % NN) / N, iy = t % N;
    const bool incoming = side == 0 ? (ix > N / 2) : (ix < N / 2);
    if (!incoming) continue;
    const double cg = cf.cg[ix], cl = cf.cl[ix];
    const int g0 = side == 0 ? -2 : Nx, g1 = side == 0 ? -1 : Nx + 1;
    const double lg = cell_cotangent(W, lam, g0, c, ix, iy, Nx, N, cg, cl, g) +
                      cell_cotangent(W, lam, g1, c, ix, iy, Nx, N, cg, cl, g);
    acc += lg * phi[t];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) gsum[side] = red[0];
}

// Grid as k_advect: blockIdx.y = 4 j + c, threads over the velocities.
__global__ void __launch_bounds__(256) k_advect_vjp(const double* __restrict__ W, const double* __restrict__ lam,
                                                    double* __restrict__ lam_in, int Nx, int N, double dv,
                                                    const __grid_constant__ AdvectCoefs cf, Ghost g,
                                                    const double* __restrict__ gsum) {
  const int NN = N * N;
  const int j = blockIdx.y >> 2, c = blockIdx.y & 3;
  double* out = lam_in + (size_t)blockIdx.y * NN;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < NN; v += gridDim.x * blockDim.x) {
    const int ix = v / N, iy = v - ix * N;
    const double cg = cf.cg[ix], cl = cf.cl[ix];
    double acc = cell_cotangent(W, lam, j, c, ix, iy, Nx, N, cg, cl, g);
    if (g.kind != QBE_PERIODIC) {
      for (int side = 0; side < 2; ++side) {
        if (j != (side == 0 ? 0 : Nx - 1)) continue;
        const int g0 = side == 0 ? -2 : Nx, g1 = side == 0 ? -1 : Nx + 1;
        const bool incoming = side == 0 ? (ix > N / 2) : (ix < N / 2);
        if (!incoming)   // both ghosts copy this boundary value
          acc += cell_cotangent(W, lam, g0, c, ix, iy, Nx, N, cg, cl, g) +
                 cell_cotangent(W, lam, g1, c, ix, iy, Nx, N, cg, cl, g);
        if (g.kind == QBE_MAXWELL) {
          // specular image: this value feeds the ghosts at velocity index N - ix (v_x -> -v_x) when those are
          // incoming (|v_x| and so c_g, c_l are the same there)
          const int mx = N - ix;
          const bool m_in = side == 0 ? (mx > N / 2) : (mx < N / 2);
          if (mx < N && m_in)
            acc += (1.0 - g.alpha) * (cell_cotangent(W, lam, g0, c, mx, iy, Nx, N, cg, cl, g) +
                                      cell_cotangent(W, lam, g1, c, mx, iy, Nx, N, cg, cl, g));
          // diffusive part through Fbar = dv^2 sum_{outgoing} 2 w0 |v_x|
          const bool outg = side == 0 ? (ix < N / 2) : (ix > N / 2);
          if (c == 0 && outg) {
            const double Z = side == 0 ? g.ZL : g.ZR;
            acc += g.alpha / Z * dv * dv * 2.0 * (dv * abs(ix - N / 2)) * gsum[side];
          }
        }
      }
    }
    out[v] = acc;
  }
}

// Adjoint of Heun's method for dW/dt = C[W] + 2 (B x w).sigma (k_rk1, k_rk2).
// Forward: F0 = C(U) + P_B U, W1 = U + dt F0, Z = U + dt/2 (F0 + C(W1) + P_B W1).
// Given lam = dZ-cotangent and G1 = C'(W1)^T lam (one collision VJP):
//   lW1 = dt/2 G1 + P_B^T (dt/2 lam),  lF0 = dt/2 lam + dt lW1,
//   lU  = lam + lW1 + P_B^T lF0 + C'(U)^T lF0   (the last term by a second VJP),
// with P_B^T mu = -2 B x mu; the B-gradient per cell is
//   sum_v [2 W1 x (dt/2 lam) + 2 U x lF0].
// One block per cell (the B reduction is per cell); writes lF0 and the
// partial lU, accumulates gB[cell].
__global__ void __launch_bounds__(256) k_rk_vjp(const double* __restrict__ U, const double* __restrict__ W1,
                                                const double* __restrict__ lam, const double* __restrict__ G1,
                                                const double* __restrict__ B, double dt, double* __restrict__ lF0,
                                                double* __restrict__ lU, double* gB, int N) {
  __shared__ double red[3][256];
  const size_t NN = (size_t)N * N;
  const int cell = blockIdx.x;
  const double* b = B + 3 * cell;
  const size_t cb = (size_t)cell * 4 * NN;
  double gb[3] = {0, 0, 0};
  for (size_t v = threadIdx.x; v < NN; v += blockDim.x) {
    const size_t base = cb + v;
    double l[4], g1[4], lw1[4], lf[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      l[c] = lam[base + c * NN];
      g1[c] = G1[base + c * NN];
    }
    const double h = 0.5 * dt;
    // P_B^T (h lam) = -2 B x (h lam)
    lw1[0] = h * g1[0];
    lw1[1] = h * g1[1] - 2.0 * h * (b[1] * l[3] - b[2] * l[2]);
    lw1[2] = h * g1[2] - 2.0 * h * (b[2] * l[1] - b[0] * l[3]);
    lw1[3] = h * g1[3] - 2.0 * h * (b[0] * l[2] - b[1] * l[1]);
#pragma unroll
    for (int c = 0; c < 4; ++c) lf[c] = h * l[c] + dt * lw1[c];
    double pu[4];
    pu[0] = 0.0;
    pu[1] = -2.0 * (b[1] * lf[3] - b[2] * lf[2]);
    pu[2] = -2.0 * (b[2] * lf[1] - b[0] * lf[3]);
    pu[3] = -2.0 * (b[0] * lf[2] - b[1] * lf[1]);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      lF0[base + c * NN] = lf[c];
      lU[base + c * NN] = l[c] + lw1[c] + pu[c];
    }
    const double x1 = W1[base + NN], x2 = W1[base + 2 * NN], x3 = W1[base + 3 * NN];
    const double u1 = U[base + NN], u2 = U[base + 2 * NN], u3 = U[base + 3 * NN];
    // 2 x x (h lam) + 2 u x lF0
    gb[0] += 2.0 * h * (x2 * l[3] - x3 * l[2]) + 2.0 * (u2 * lf[3] - u3 * lf[2]);
    gb[1] += 2.0 * h * (x3 * l[1] - x1 * l[3]) + 2.0 * (u3 * lf[1] - u1 * lf[3]);
    gb[2] += 2.0 * h * (x1 * l[2] - x2 * l[1]) + 2.0 * (u1 * lf[2] - u2 * lf[1]);
  }
  for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = gb[k];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 3) gB[(size_t)cell * 3 + threadIdx.x] += red[threadIdx.x][0];
}

// Final-time observables per cell: [0] = dv^2 sum 2 w3 (spin polarisation
// along z), [1] = dv^2 sum v_x |v|^2/2 2 w0 (energy flux); times dx after the
// fixed-order sum over cells in k_observables_sum.
__global__ void __launch_bounds__(256) k_observables(const double* __restrict__ W, int N, double L, double* part) {
  __shared__ double red[2][256];
  const int cell = blockIdx.x;
  const size_t NN = (size_t)N * N;
  const double dv = 2.0 * L / N;
  const double* w = W + (size_t)cell * 4 * NN;
  double a = 0.0, e = 0.0;
  for (size_t i = threadIdx.x; i < NN; i += blockDim.x) {
    const int ix = (int)(i / N), iy = (int)(i % N);
    const double vx = dv * (ix - N / 2), vy = dv * (iy - N / 2);
    a += 2.0 * w[3 * NN + i];
    e += vx * 0.5 * (vx * vx + vy * vy) * 2.0 * w[i];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = e;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) part[(size_t)cell * 2 + threadIdx.x] = red[threadIdx.x][0] * dv * dv;
}

__global__ void k_observables_sum(const double* __restrict__ part, int Nx, double* out) {
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int j = 0; j < Nx; ++j) s += part[(size_t)j * 2 + threadIdx.x];
    out[threadIdx.x] = s / Nx;
  }
}

// lam = gbar[0] dP_z/dW + gbar[1] dPhi_E/dW
__global__ void __launch_bounds__(256) k_observables_vjp(const double* __restrict__ gbar, int Nx, int N, double L,
                                                         double* __restrict__ lam) {
  const size_t NN = (size_t)N * N;
  const size_t total = (size_t)Nx * 4 * NN;
  const double dv = 2.0 * L / N;
  const double s = dv * dv / Nx;
  const double g0 = gbar[0], g1 = gbar[1];
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)((t / NN) % 4);
    const int ix = (int)((t % NN) / N), iy = (int)(t % N);
    const double vx = dv * (ix - N / 2), vy = dv * (iy - N / 2);
    double v = 0.0;
    if (c == 3) v = 2.0 * s * g0;
    if (c == 0) v = s * g1 * vx * (vx * vx + vy * vy);
    lam[t] = v;
  }
}

// Grid over (velocity blocks) x (rows): rows = cells (x4 components for per-component kernels).
dim3 grid_rows(int NN, int rows) {
  const int bx = (NN + 255) / 256;
  return dim3(bx < 1 ? 1 : bx, rows);
}

int grid_for(size_t total) {
  size_t g = (total + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t advect_substep(const double* Win, double* Wout, int Nx, int N, double L, double tau,
                           const BoundaryDev& bc, cudaStream_t s, long long& launches, KernelTimer* tm) {
  if (tm) tm->begin(KG_TRANSPORT, s);
  if (bc.kind == QBE_MAXWELL) {
    k_wall_flux<<<2, 256, 0, s>>>(Win, Nx, N, L, bc.fbar);
    ++launches;
  }
  Ghost g{bc.kind, bc.alpha, bc.ZL, bc.ZR, bc.phiL, bc.phiR, bc.fbar};
  const AdvectCoefs cf = make_advect_coefs(N, 2.0 * L / N, tau / (1.0 / Nx));
  k_advect<<<grid_rows(N * N, Nx * 4), 256, 0, s>>>(Win, Wout, Nx, N, cf, g);
  if (tm) tm->end(s);
  ++launches;
  return cudaGetLastError();
}

cudaError_t rk_stage1(const double* W, const double* C, const double* B, double dt, double* F0, double* W1,
                      int Nx, int N, cudaStream_t s, long long& launches, KernelTimer* tm) {
  if (tm) tm->begin(KG_RK, s);
  k_rk1<<<grid_rows(N * N, Nx), 256, 0, s>>>(W, C, B, dt, F0, W1, Nx, N);
  if (tm) tm->end(s);
  ++launches;
  return cudaGetLastError();
}

cudaError_t rk_stage2(const double* W, const double* F0, const double* C1, const double* W1, const double* B,
                      double dt, double* Wout, int Nx, int N, cudaStream_t s, long long& launches, KernelTimer* tm) {
  if (tm) tm->begin(KG_RK, s);
  k_rk2<<<grid_rows(N * N, Nx), 256, 0, s>>>(W, F0, C1, W1, B, dt, Wout, Nx, N);
  if (tm) tm->end(s);
  ++launches;
  return cudaGetLastError();
}

cudaError_t moments_launch(const double* W, int Nx, int N, double L, double* out7, cudaStream_t s,
                           long long& launches) {
  k_moments<<<Nx, 256, 0, s>>>(W, N, L, out7);
  ++launches;
  return cudaGetLastError();
}

cudaError_t advect_substep_vjp(const double* Win, const double* lam_out, double* lam_in, int Nx, int N, double L,
                               double tau, const BoundaryDev& bc, double* gsum, cudaStream_t s,
                               long long& launches, KernelTimer* tm) {
  if (tm) tm->begin(KG_ADJ_TRANSPORT, s);
  if (bc.kind == QBE_MAXWELL) {
    k_wall_flux<<<2, 256, 0, s>>>(Win, Nx, N, L, bc.fbar);
    ++launches;
  }
  Ghost g{bc.kind, bc.alpha, bc.ZL, bc.ZR, bc.phiL, bc.phiR, bc.fbar};
  const double dv = 2.0 * L / N;
  const AdvectCoefs cf = make_advect_coefs(N, dv, tau / (1.0 / Nx));
  if (bc.kind == QBE_MAXWELL) {
    k_wall_adj<<<2, 256, 0, s>>>(Win, lam_out, Nx, N, cf, g, gsum);
    ++launches;
  }
  k_advect_vjp<<<grid_rows(N * N, Nx * 4), 256, 0, s>>>(Win, lam_out, lam_in, Nx, N, dv, cf, g, gsum);
  if (tm) tm->end(s);
  ++launches;
  return cudaGetLastError();
}

cudaError_t rk_vjp_launch(const double* U, const double* W1, const double* lam, const double* G1, const double* B,
                          double dt, double* lF0, double* lU, double* gB, int Nx, int N, cudaStream_t s,
                          long long& launches, KernelTimer* tm) {
  if (tm) tm->begin(KG_ADJ_TRANSPORT, s);
  k_rk_vjp<<<Nx, 256, 0, s>>>(U, W1, lam, G1, B, dt, lF0, lU, gB, N);
  if (tm) tm->end(s);
  ++launches;
  return cudaGetLastError();
}

cudaError_t observables_launch(const double* W, int Nx, int N, double L, double* part, double* out2,
                               cudaStream_t s, long long& launches) {
  k_observables<<<Nx, 256, 0, s>>>(W, N, L, part);
  k_observables_sum<<<1, 32, 0, s>>>(part, Nx, out2);
  launches += 2;
  return cudaGetLastError();
}

cudaError_t observables_vjp_launch(const double* gbar, int Nx, int N, double L, double* lam, cudaStream_t s,
                                   long long& launches) {
  k_observables_vjp<<<grid_for((size_t)Nx * 4 * N * N), 256, 0, s>>>(gbar, Nx, N, L, lam);
  ++launches;
  return cudaGetLastError();
}

}  // namespace qbe
