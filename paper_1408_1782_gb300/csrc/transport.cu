// Transport (Sec. 4, eq. slopeLimiterStep with eq. minmod), boundary ghost
// cells (Sec. 2: periodic, Dirichlet, Maxwell), the precession term
// -i[B.sigma, W] = 2 (B x w).sigma inside Heun's RK2, and the moments
// (eqs. density, velocity, internal_energy).  All kernels stream the state
// [cell][4][ix][iy] once; consecutive threads take consecutive velocities so
// every access is coalesced.
#include "internal.h"

namespace qbe {

namespace {

__device__ __forceinline__ double minmod(double a, double b) {
  // a if |a| <= |b| and ab > 0; b if |b| < |a| and ab > 0; 0 otherwise
  return (a * b > 0.0) ? (fabs(a) <= fabs(b) ? a : b) : 0.0;
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
__device__ __forceinline__ double cell_value(const double* __restrict__ W, int jj, int c, int ix, int iy, int Nx,
                                             int N, double vx, const Ghost& g) {
  const size_t NN = (size_t)N * N;
  const size_t off = (size_t)c * NN + (size_t)ix * N + iy;
  if (jj >= 0 && jj < Nx) return W[(size_t)jj * 4 * NN + off];
  if (g.kind == QBE_PERIODIC) {
    const int w = (jj % Nx + Nx) % Nx;
    return W[(size_t)w * 4 * NN + off];
  }
  const bool left = jj < 0;
  const int b = left ? 0 : Nx - 1;
  const bool incoming = left ? (vx > 0.0) : (vx < 0.0);
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

__global__ void __launch_bounds__(256) k_advect(const double* __restrict__ W, double* __restrict__ Wout, int Nx,
                                                int N, double L, double tau, Ghost g) {
  const size_t NN = (size_t)N * N;
  const size_t total = (size_t)Nx * 4 * NN;
  const double dv = 2.0 * L / N;
  const double dx = 1.0 / Nx;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / (4 * NN));
    const int c = (int)((t / NN) % 4);
    const int ix = (int)((t % NN) / N);
    const int iy = (int)(t % N);
    const double vx = dv * (ix - N / 2);
    double Wv[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) Wv[d] = cell_value(W, j - 2 + d, c, ix, iy, Nx, N, vx, g);
    const double Sm1 = minmod(Wv[2] - Wv[1], Wv[1] - Wv[0]);
    const double S0 = minmod(Wv[3] - Wv[2], Wv[2] - Wv[1]);
    const double Sp1 = minmod(Wv[4] - Wv[3], Wv[3] - Wv[2]);
    const double nu = tau * vx / dx;
    const double sg = (nu > 0.0) ? 1.0 : (nu < 0.0 ? -1.0 : 0.0);
    const double lim = 0.5 * (sg - nu);
    const double godunov = -vx * (Wv[3] - Wv[1]) + fabs(vx) * (Wv[3] - 2.0 * Wv[2] + Wv[1]);
    const double limiter = lim * (-vx * (Sp1 - Sm1) + fabs(vx) * (Sp1 - 2.0 * S0 + Sm1));
    Wout[t] = Wv[2] + (tau / (2.0 * dx)) * (godunov + limiter);
  }
}

__device__ __forceinline__ void prec(const double* b, double w1, double w2, double w3, double& p1, double& p2,
                                     double& p3) {
  p1 = 2.0 * (b[1] * w3 - b[2] * w2);
  p2 = 2.0 * (b[2] * w1 - b[0] * w3);
  p3 = 2.0 * (b[0] * w2 - b[1] * w1);
}

// F0 = C + 2 (B x w).sigma;  W1 = W + dt F0
__global__ void __launch_bounds__(256) k_rk1(const double* __restrict__ W, const double* __restrict__ C,
                                             const double* __restrict__ B, double dt, double* __restrict__ F0,
                                             double* __restrict__ W1, int Nx, int N) {
  const size_t NN = (size_t)N * N;
  const size_t total = (size_t)Nx * NN;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const size_t cell = t / NN, v = t % NN;
    const size_t base = cell * 4 * NN + v;
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
  const size_t NN = (size_t)N * N;
  const size_t total = (size_t)Nx * NN;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const size_t cell = t / NN, v = t % NN;
    const size_t base = cell * 4 * NN + v;
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
  const size_t total = (size_t)Nx * 4 * N * N;
  k_advect<<<grid_for(total), 256, 0, s>>>(Win, Wout, Nx, N, L, tau, g);
  if (tm) tm->end(s);
  ++launches;
  return cudaGetLastError();
}

cudaError_t rk_stage1(const double* W, const double* C, const double* B, double dt, double* F0, double* W1,
                      int Nx, int N, cudaStream_t s, long long& launches, KernelTimer* tm) {
  if (tm) tm->begin(KG_RK, s);
  k_rk1<<<grid_for((size_t)Nx * N * N), 256, 0, s>>>(W, C, B, dt, F0, W1, Nx, N);
  if (tm) tm->end(s);
  ++launches;
  return cudaGetLastError();
}

cudaError_t rk_stage2(const double* W, const double* F0, const double* C1, const double* W1, const double* B,
                      double dt, double* Wout, int Nx, int N, cudaStream_t s, long long& launches, KernelTimer* tm) {
  if (tm) tm->begin(KG_RK, s);
  k_rk2<<<grid_for((size_t)Nx * N * N), 256, 0, s>>>(W, F0, C1, W1, B, dt, Wout, Nx, N);
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

}  // namespace qbe
