// Diagnostics of the solver state (Sec. 2 and Sec. 5): local entropy
// (eq. entropy_def), the Fermi-Dirac state with the moments of a cell or of
// the whole domain (eq. W_FermiDirac, eq. momentsFermiDirac), the quantum
// relative entropy (eqs. relentropy_hom, relentropy_inhom, relentropy_local)
// and the trace-norm L1 distance to a Fermi-Dirac state.
//
// A 2x2 Hermitian W = w0 1 + w.sigma has eigenvalues w0 +- |w|; a
// Fermi-Dirac state F = n_up |up><up| + n_dn |dn><dn| with |up><up| =
// (1 + r.sigma)/2 (r the unit Bloch vector of the up state) has Pauli form
// ((n_up + n_dn)/2, (n_up - n_dn)/2 r), and tr[X log F] = <up|X|up> log n_up +
// <dn|X|dn> log n_dn with <up|X|up> = x0 + x.r, <dn|X|dn> = x0 - x.r.
#include <cmath>
#include <vector>

#include "internal.h"

namespace qbe {

namespace {

__device__ __forceinline__ double xlogx(double x) { return x > 0.0 ? x * log(x) : 0.0; }

// Per cell: dv^2 sum_v -[lam log lam + (1 - lam) log(1 - lam)] over both eigenvalues.
__global__ void __launch_bounds__(256) k_entropy(const double* __restrict__ W, int N, double L, double* out) {
  __shared__ double red[256];
  const int cell = blockIdx.x;
  const size_t NN = (size_t)N * N;
  const double dv = 2.0 * L / N;
  const double* w = W + (size_t)cell * 4 * NN;
  double acc = 0.0;
  for (size_t i = threadIdx.x; i < NN; i += blockDim.x) {
    const double r = sqrt(w[NN + i] * w[NN + i] + w[2 * NN + i] * w[2 * NN + i] + w[3 * NN + i] * w[3 * NN + i]);
    const double lp = w[i] + r, lm = w[i] - r;
    acc -= xlogx(lp) + xlogx(1.0 - lp) + xlogx(lm) + xlogx(1.0 - lm);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[cell] = red[0] * dv * dv;
}

// Per cell: relative entropy to, and trace-norm distance from, the Fermi-Dirac
// state fd[cell] (or fd[0] for every cell when nfd == 1).
__global__ void __launch_bounds__(256) k_relative_entropy(const double* __restrict__ W, int N, double L,
                                                          const FdDev* __restrict__ fd, int nfd, double* rel,
                                                          double* l1) {
  __shared__ double red[2][256];
  const int cell = blockIdx.x;
  const FdDev f = fd[nfd == 1 ? 0 : cell];
  const size_t NN = (size_t)N * N;
  const double dv = 2.0 * L / N;
  const double* w = W + (size_t)cell * 4 * NN;
  double a_rel = 0.0, a_l1 = 0.0;
  for (size_t i = threadIdx.x; i < NN; i += blockDim.x) {
    const int ix = (int)(i / N), iy = (int)(i % N);
    const double vx = dv * (ix - N / 2) - f.u[0], vy = dv * (iy - N / 2) - f.u[1];
    const double e = 0.5 * (vx * vx + vy * vy);
    const double xu = (e - f.mu_up) / f.T, xd = (e - f.mu_dn) / f.T;
    // n = 1/(e^x + 1), log n = -log(1 + e^x), log(1 - n) = -log(1 + e^-x), stable for either sign of x
    const double ln_nu = -(fmax(xu, 0.0) + log1p(exp(-fabs(xu))));
    const double ln_nd = -(fmax(xd, 0.0) + log1p(exp(-fabs(xd))));
    const double ln_mu = -(fmax(-xu, 0.0) + log1p(exp(-fabs(xu))));
    const double ln_md = -(fmax(-xd, 0.0) + log1p(exp(-fabs(xd))));
    const double nu = exp(ln_nu), nd = exp(ln_nd);
    const double w0 = w[i], w1 = w[NN + i], w2 = w[2 * NN + i], w3 = w[3 * NN + i];
    const double r = sqrt(w1 * w1 + w2 * w2 + w3 * w3);
    const double lp = w0 + r, lm = w0 - r;
    const double wr = w1 * f.bloch[0] + w2 * f.bloch[1] + w3 * f.bloch[2];
    const double pu = w0 + wr, pd = w0 - wr;          // <up|W|up>, <dn|W|dn>
    a_rel += xlogx(lp) + xlogx(lm) + xlogx(1.0 - lp) + xlogx(1.0 - lm) - pu * ln_nu - pd * ln_nd -
             (1.0 - pu) * ln_mu - (1.0 - pd) * ln_md;
    const double f0 = 0.5 * (nu + nd), fh = 0.5 * (nu - nd);
    const double d0 = w0 - f0, d1 = w1 - fh * f.bloch[0], d2 = w2 - fh * f.bloch[1], d3 = w3 - fh * f.bloch[2];
    const double dr = sqrt(d1 * d1 + d2 * d2 + d3 * d3);
    a_l1 += fabs(d0 + dr) + fabs(d0 - dr);
  }
  red[0][threadIdx.x] = a_rel;
  red[1][threadIdx.x] = a_l1;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    rel[cell] = red[0][0] * dv * dv;
    if (l1) l1[cell] = red[1][0] * dv * dv;
  }
}

// ---------------------------------------------------------------------------
// Host: dilogarithm and the Fermi-Dirac fit.
// ---------------------------------------------------------------------------
constexpr double kPiH = 3.14159265358979323846;

// Bernoulli numbers B_0..B_{2K} from sum_{k<=m} C(m+1, k) B_k = 0.
const std::vector<long double>& bernoulli() {
  static std::vector<long double> B;
  if (B.empty()) {
    const int n = 40;
    B.assign(n + 1, 0.0L);
    B[0] = 1.0L;
    for (int m = 1; m <= n; ++m) {
      long double s = 0.0L, c = 1.0L;          // c = C(m+1, k)
      for (int k = 0; k < m; ++k) {
        s += c * B[k];
        c = c * (long double)(m + 1 - k) / (long double)(k + 1);
      }
      B[m] = -s / (long double)(m + 1);
    }
  }
  return B;
}

// Li2(x) for x in [-1, 0]: Li2(x) = sum_{n>=0} B_n u^{n+1}/(n+1)!, u = -log(1 - x), |u| <= log 2
// (the series of 't Hooft and Veltman, convergent for |u| < 2 pi).
double li2_m1_0(double x) {
  const auto& B = bernoulli();
  const long double u = -log1pl(-(long double)x);
  long double term = u, sum = 0.0L;                 // term = u^{n+1}/(n+1)!
  for (size_t n = 0; n + 1 < B.size(); ++n) {
    sum += B[n] * term;
    term *= u / (long double)(n + 2);
  }
  return (double)sum;
}

// -Li2(-e^t): for t > 0 by the inversion Li2(-z) + Li2(-1/z) = -pi^2/6 - log(z)^2/2.
double neg_li2_neg_exp(double t) {
  if (t <= 0.0) return -li2_m1_0(-std::exp(t));
  return kPiH * kPiH / 6.0 + 0.5 * t * t + li2_m1_0(-std::exp(-t));
}

double softplus(double t) { return t > 0.0 ? t + std::log1p(std::exp(-t)) : std::log1p(std::exp(t)); }

// log(e^a - 1) for a > 0
double log_expm1(double a) { return a < 30.0 ? std::log(std::expm1(a)) : a + std::log(-std::expm1(-a)); }

}  // namespace

cudaError_t entropy_launch(const double* W, int Nx, int N, double L, double* out, cudaStream_t s,
                           long long& launches) {
  k_entropy<<<Nx, 256, 0, s>>>(W, N, L, out);
  ++launches;
  return cudaGetLastError();
}

cudaError_t relative_entropy_launch(const double* W, int Nx, int N, double L, const FdDev* fd, int nfd, double* rel,
                                    double* l1, cudaStream_t s, long long& launches) {
  k_relative_entropy<<<Nx, 256, 0, s>>>(W, N, L, fd, nfd, rel, l1);
  ++launches;
  return cudaGetLastError();
}

double dilog(double x) {
  if (x >= -1.0 && x <= 0.0) return li2_m1_0(x);
  if (x < -1.0) return -kPiH * kPiH / 6.0 - 0.5 * std::log(-x) * std::log(-x) - li2_m1_0(1.0 / x);
  return std::nan("");
}

// Fit (Sec. 5.2): eigenbasis of rho; T, mu_s from rho_s = 2 pi T log(1 + e^{mu_s/T}) and
// eps = T sum_s(-Li2(-e^{mu_s/T})) / sum_s log(1 + e^{mu_s/T}), eps the internal energy per particle.
void fd_fit_from_moments(const double rho4[4], const double mom[2], double energy, qbe_fermi_dirac& out) {
  out = qbe_fermi_dirac{};
  const double r = std::sqrt(rho4[1] * rho4[1] + rho4[2] * rho4[2] + rho4[3] * rho4[3]);
  const double r_up = rho4[0] + r, r_dn = rho4[0] - r;          // eigenvalues of rho = rho0 1 + rho.sigma
  double b[3] = {0.0, 0.0, 1.0};
  if (r > 0.0) {
    b[0] = rho4[1] / r;
    b[1] = rho4[2] / r;
    b[2] = rho4[3] / r;
  }
  for (int k = 0; k < 3; ++k) out.bloch[k] = b[k];
  // |up> = (cos(theta/2), e^{i phi} sin(theta/2)), |dn> = (-e^{-i phi} sin(theta/2), cos(theta/2))
  const double ct = std::sqrt(std::fmax(0.0, 0.5 * (1.0 + b[2]))), st = std::sqrt(std::fmax(0.0, 0.5 * (1.0 - b[2])));
  const double rho_xy = std::hypot(b[0], b[1]);
  const double cph = rho_xy > 0.0 ? b[0] / rho_xy : 1.0, sph = rho_xy > 0.0 ? b[1] / rho_xy : 0.0;
  out.U_re[0][0] = ct;         out.U_im[0][0] = 0.0;
  out.U_re[1][0] = cph * st;   out.U_im[1][0] = sph * st;
  out.U_re[0][1] = -cph * st;  out.U_im[0][1] = sph * st;
  out.U_re[1][1] = ct;         out.U_im[1][1] = 0.0;
  const double tr = r_up + r_dn;                                  // = 2 rho0 = int tr W
  if (!(tr > 0.0)) return;
  out.u[0] = mom[0] / tr;
  out.u[1] = mom[1] / tr;
  const double eps = energy / tr - 0.5 * (out.u[0] * out.u[0] + out.u[1] * out.u[1]);
  if (!(r_dn > 0.0) || !(eps > 0.0)) return;
  const double eps0 = (r_up * r_up + r_dn * r_dn) / (4.0 * kPiH * tr);   // T -> 0 limit
  if (!(eps > eps0)) return;
  auto mus = [&](double T, double& mu_up, double& mu_dn) {
    mu_up = T * log_expm1(r_up / (2.0 * kPiH * T));
    mu_dn = T * log_expm1(r_dn / (2.0 * kPiH * T));
  };
  auto f = [&](double lt) {
    const double T = std::exp(lt);
    double mu_up, mu_dn;
    mus(T, mu_up, mu_dn);
    const double num = neg_li2_neg_exp(mu_up / T) + neg_li2_neg_exp(mu_dn / T);
    const double den = softplus(mu_up / T) + softplus(mu_dn / T);
    return T * num / den - eps;
  };
  // eps(T) rises monotonically from eps0 (T -> 0) to ~T (T -> infinity): bracket, then bisect in log T
  double lo = std::log(eps), hi = lo + 1.0;
  for (int i = 0; i < 200 && f(lo) > 0.0; ++i) lo -= 2.0;
  for (int i = 0; i < 200 && f(hi) < 0.0; ++i) hi += 2.0;
  if (!(f(lo) <= 0.0 && f(hi) >= 0.0)) return;
  for (int i = 0; i < 200 && hi - lo > 1e-16 * std::fmax(1.0, std::fabs(lo)); ++i) {
    const double mid = 0.5 * (lo + hi);
    if (f(mid) < 0.0) lo = mid; else hi = mid;
  }
  out.T = std::exp(0.5 * (lo + hi));
  mus(out.T, out.mu_up, out.mu_dn);
  out.ok = 1;
}

}  // namespace qbe
