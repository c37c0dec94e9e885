// Host-side construction of the quadrature tables of Sec. 3.2 and of the wall
// Fermi-Dirac states of Sec. 2, uploaded once per solver.
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace qbe {

namespace {

constexpr double kPi = 3.14159265358979323846;

void split_of(int n, int& A, int& B) {
  switch (n) {
    case 16: A = 4; B = 4; break;
    case 32: A = 4; B = 8; break;
    case 64: A = 8; B = 8; break;
    case 128: A = 8; B = 16; break;
    case 256: A = 16; B = 16; break;
    case 96: A = 12; B = 8; break;
    case 192: A = 12; B = 16; break;
    default: A = B = 0;
  }
}

// phi_R(s) = int_0^R sin(pi s r / L) dr = (2L/(pi s)) sin^2(pi s R / (2L))   (Sec. 3.2)
double phi_R(double s, double L, double R) {
  if (s == 0.0) return 0.0;
  const double t = std::sin(kPi * s * R / (2.0 * L));
  return (2.0 * L / (kPi * s)) * t * t;
}

// psi_R(s) = int_{-R}^{R} exp(i pi s r / L) dr = (2L/(pi s)) sin(pi R s / L)  (eq. approxH-J)
double psi_R(double s, double L, double R) {
  if (s == 0.0) return 2.0 * R;
  return (2.0 * L / (kPi * s)) * std::sin(kPi * R * s / L);
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_M.
void gauss_legendre(int M, std::vector<double>& x, std::vector<double>& w) {
  x.assign(M, 0.0);
  w.assign(M, 0.0);
  for (int i = 0; i < (M + 1) / 2; ++i) {
    long double z = std::cos(kPi * (i + 0.75) / (M + 0.5));
    long double pp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = 0;
      for (int k = 1; k <= M; ++k) {
        const long double p2 = p1;
        p1 = p0;
        p0 = ((2.0L * k - 1) * z * p1 - (k - 1.0L) * p2) / k;
      }
      pp = M * (z * p0 - p1) / (z * z - 1.0L);
      const long double dz = p0 / pp;
      z -= dz;
      if (std::fabs((double)dz) < 1e-19) break;
    }
    {
      long double p0 = 1, p1 = 0;
      for (int k = 1; k <= M; ++k) {
        const long double p2 = p1;
        p1 = p0;
        p0 = ((2.0L * k - 1) * z * p1 - (k - 1.0L) * p2) / k;
      }
      pp = M * (z * p0 - p1) / (z * z - 1.0L);
    }
    x[i] = -(double)z;
    x[M - 1 - i] = (double)z;
    const double wi = (double)(2.0L / ((1.0L - z * z) * pp * pp));
    w[i] = wi;
    w[M - 1 - i] = wi;
  }
  if (M % 2 == 1) x[M / 2] = 0.0;
}

template <class T>
bool upload(T*& dst, const std::vector<T>& src, std::string& err) {
  if (cudaMalloc((void**)&dst, src.size() * sizeof(T)) != cudaSuccess) {
    err = "cudaMalloc failed for kernel tables";
    return false;
  }
  if (cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    err = "cudaMemcpy failed for kernel tables";
    return false;
  }
  return true;
}

}  // namespace

template <class D, class S>
std::vector<D> to_f32(const std::vector<S>& v);
template <>
std::vector<float> to_f32<float, double>(const std::vector<double>& v) {
  std::vector<float> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
  return o;
}
template <>
std::vector<float2> to_f32<float2, double2>(const std::vector<double2>& v) {
  std::vector<float2> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].x, (float)v[i].y);
  return o;
}

bool build_tables(int N, int J, int M, double L, double R, Tables& t, std::string& err, bool with_f32) {
  const int n = 2 * N;
  int A = 0, B = 0;
  split_of(n, A, B);
  if (A == 0) {
    err = "unsupported N (supported: 8, 16, 32, 48, 64, 96, 128)";
    return false;
  }
  t.N = N; t.n = n; t.J = J; t.M = M; t.L = L; t.R = R;
  const size_t P = (size_t)n * n;

  // twiddles exp(-2 pi i t2 k1 / n), index t2*A + k1
  std::vector<double2> tw(n);
  for (int t2 = 0; t2 < B; ++t2)
    for (int k1 = 0; k1 < A; ++k1) {
      const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)(t2 * k1) / n;
      tw[t2 * A + k1] = make_double2((double)std::cos(ang), (double)std::sin(ang));
    }

  // signed fine frequency of each permuted position
  std::vector<int> sig(n);
  for (int pos = 0; pos < n; ++pos) {
    const int k = pos / B + A * (pos % B);
    sig[pos] = k < N ? k : k - n;
  }
  std::vector<double> th_c(J), th_s(J), thp_c(J), thp_s(J);
  for (int j = 0; j < J; ++j) {
    th_c[j] = std::cos(j * kPi / J);                      // theta_j, eq. theta_grid
    th_s[j] = std::sin(j * kPi / J);
    thp_c[j] = std::cos((j + 0.5) * kPi / J);             // theta'_j
    thp_s[j] = std::sin((j + 0.5) * kPi / J);
  }
  std::vector<double> phip(J * P), Ktab(J * P, 0.0), psi(J * P), psip(J * P);
  std::vector<double> phi_j(J);
  const double invP = 1.0 / (double)P;
  for (int px = 0; px < n; ++px)
    for (int py = 0; py < n; ++py) {
      const double sx = sig[px], sy = sig[py];
      const size_t o = (size_t)px * n + py;
      for (int j = 0; j < J; ++j) {
        phi_j[j] = phi_R(sx * th_c[j] + sy * th_s[j], L, R);
        phip[j * P + o] = phi_R(sx * thp_c[j] + sy * thp_s[j], L, R);
        psi[j * P + o] = psi_R(sx * th_c[j] + sy * th_s[j], L, R);
        psip[j * P + o] = psi_R(-sx * th_s[j] + sy * th_c[j], L, R) * invP;   // theta^perp = (-sin, cos)
      }
      for (int jp = 0; jp < J; ++jp) {
        double acc = 0.0;
        for (int j = 0; j < J; ++j) {
          // omega_G[j][j'] = -(2 pi / J)^2 / (theta_j . theta'_j')   (eq. approxG)
          const double dot = th_c[j] * thp_c[jp] + th_s[j] * thp_s[jp];
          acc += -(2.0 * kPi / J) * (2.0 * kPi / J) / dot * phi_j[j];
        }
        Ktab[jp * P + o] = acc * invP;
      }
    }

  // Hu-Ying phases: alpha_{j,m} = pi rho_m theta_j / L on Gauss-Legendre nodes of [-R, R]
  std::vector<double> gx, gw;
  gauss_legendre(M, gx, gw);
  std::vector<double2> phase((size_t)J * M * 2 * n);
  for (int j = 0; j < J; ++j)
    for (int m = 0; m < M; ++m) {
      const double rho = R * gx[m], wm = R * gw[m];
      const double ax = kPi * rho * th_c[j] / L, ay = kPi * rho * th_s[j] / L;
      const double sq = std::sqrt(kPi / J * wm);
      double2* row = &phase[((size_t)j * M + m) * 2 * n];
      for (int pos = 0; pos < n; ++pos) {
        const double a = ax * sig[pos], b = ay * sig[pos];
        row[pos] = make_double2(sq * std::cos(a), sq * std::sin(a));
        row[n + pos] = make_double2(std::cos(b), std::sin(b));
      }
    }

  bool ok = upload(t.tw, tw, err) && upload(t.phip, phip, err) && upload(t.Ktab, Ktab, err) &&
            upload(t.psi, psi, err) && upload(t.psip_s, psip, err) && upload(t.phase, phase, err);
  if (ok && with_f32) {
    ok = upload(t.tw_f, to_f32<float2>(tw), err) && upload(t.phip_f, to_f32<float>(phip), err) &&
         upload(t.Ktab_f, to_f32<float>(Ktab), err) && upload(t.psi_f, to_f32<float>(psi), err) &&
         upload(t.psip_s_f, to_f32<float>(psip), err) && upload(t.phase_f, to_f32<float2>(phase), err);
  }
  return ok;
}

void free_tables(Tables& t) {
  cudaFree(t.tw); cudaFree(t.phip); cudaFree(t.Ktab); cudaFree(t.psi); cudaFree(t.psip_s); cudaFree(t.phase);
  cudaFree(t.tw_f); cudaFree(t.phip_f); cudaFree(t.Ktab_f); cudaFree(t.psi_f); cudaFree(t.psip_s_f);
  cudaFree(t.phase_f);
  t = Tables();
}

void fermi_dirac_pauli(const qbe_fd& fd, int N, double L, std::vector<double>& out) {
  out.assign((size_t)4 * N * N, 0.0);
  const double dv = 2.0 * L / N;
  for (int ix = 0; ix < N; ++ix)
    for (int iy = 0; iy < N; ++iy) {
      const double vx = dv * (ix - N / 2), vy = dv * (iy - N / 2);
      const double e = 0.5 * (vx * vx + vy * vy);
      double occ[2];
      const double mu[2] = {fd.mu_up, fd.mu_dn};
      for (int s = 0; s < 2; ++s) {
        const double x = fd.beta * (e - mu[s]);
        occ[s] = x > 0 ? std::exp(-x) / (1.0 + std::exp(-x)) : 1.0 / (1.0 + std::exp(x));
      }
      double w[4] = {0, 0, 0, 0};
      for (int s = 0; s < 2; ++s) {
        const std::complex<double> a(fd.U_re[0][s], fd.U_im[0][s]);
        const std::complex<double> b(fd.U_re[1][s], fd.U_im[1][s]);
        const std::complex<double> ab = std::conj(a) * b;
        w[0] += 0.5 * occ[s] * (std::norm(a) + std::norm(b));
        w[1] += 0.5 * occ[s] * 2.0 * ab.real();
        w[2] += 0.5 * occ[s] * 2.0 * ab.imag();
        w[3] += 0.5 * occ[s] * (std::norm(a) - std::norm(b));
      }
      for (int c = 0; c < 4; ++c) out[((size_t)c * N + ix) * N + iy] = w[c];
    }
}

}  // namespace qbe
