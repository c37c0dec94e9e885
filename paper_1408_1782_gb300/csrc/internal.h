// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <type_traits>
#include <vector>

#include "../../include/qbe.h"

namespace qbe {

// Device-side kernel tables for one grid (all spectral tables in the permuted
// order of the line FFT, see fft.cuh).
struct Tables {
  int N = 0, n = 0, J = 0, M = 0;
  double L = 0, R = 0;
  double2* tw = nullptr;        // [n]      exp(-2 pi i t2 k1 / n), index t2*A + k1
  double* phip = nullptr;       // [J][n*n] phi_R(sigma . theta'_j)                       (eq. approxG)
  double* Ktab = nullptr;       // [J][n*n] sum_j omega_G[j][j'] phi_R(sigma.theta_j) / n^2 (eq. approxG)
  double* psi = nullptr;        // [J][n*n] psi_R(sigma . theta_j)                        (eq. approxH-J)
  double* psip_s = nullptr;     // [J][n*n] psi_R(sigma . theta_j^perp) / n^2              (eq. approxH-J)
  double2* phase = nullptr;     // [J*M][2][n] sqrt(pi w_m / J) e^{i alpha_x sigma_x}, e^{i alpha_y sigma_y} (eq. approxH-JM)
  // FP32 copies of the same tables (FP32-split form only; null otherwise)
  float2* tw_f = nullptr;
  float* phip_f = nullptr;
  float* Ktab_f = nullptr;
  float* psi_f = nullptr;
  float* psip_s_f = nullptr;
  float2* phase_f = nullptr;
};

// Typed view of the tables for the transform precision T.
template <class T> struct TabPtrs;
template <> struct TabPtrs<double> {
  const double2* tw; const double* phip; const double* Ktab; const double* psi; const double* psip_s;
  const double2* phase;
};
template <> struct TabPtrs<float> {
  const float2* tw; const float* phip; const float* Ktab; const float* psi; const float* psip_s;
  const float2* phase;
};
template <class T> TabPtrs<T> tab_ptrs(const Tables& t);
template <> inline TabPtrs<double> tab_ptrs<double>(const Tables& t) {
  return {t.tw, t.phip, t.Ktab, t.psi, t.psip_s, t.phase};
}
template <> inline TabPtrs<float> tab_ptrs<float>(const Tables& t) {
  return {t.tw_f, t.phip_f, t.Ktab_f, t.psi_f, t.psip_s_f, t.phase_f};
}

// One simulation's share of an I3 launch: the Hu-Ying kernels run a work queue over
// the (cell, j, m-chunk) units of up to kMaxI3Jobs simulations of the same padded size
// (passed by value as a kernel parameter).
constexpr int kMaxI3Jobs = 64;
template <class T>
struct I3Job {
  const typename std::conditional<sizeof(T) == 8, double2, float2>::type* what;
  const typename std::conditional<sizeof(T) == 8, double2, float2>::type* wfine;
  typename std::conditional<sizeof(T) == 8, double2, float2>::type* K3part;
  const T* psip_s;
  const typename std::conditional<sizeof(T) == 8, double2, float2>::type* phase;
  int J, M, nmc, mch;
  int unit_begin;   // first global unit of this simulation
  int nunits;
};
template <class T>
struct I3Jobs {
  I3Job<T> job[kMaxI3Jobs];
  int njobs;
  int total;
};

// Per-evaluation buffers of the collision operator for a batch of nb cells.
struct CollisionWork {
  int prec = 0;        // 0: FP64 transforms, 1: FP32 transforms (FP32-split form)
  int nb = 0;          // cells per batch
  int nmc = 1;         // m-chunks per (cell, j) unit of the I3 kernel
  int mch = 1;         // m values per chunk
  int grid_i3 = 0;     // persistent grid of the I3 kernel
  int grid_max = 0;    // its occupancy limit (SMs x resident blocks, the largest over the variants)
  int i3_variant = 0;  // launch variant of the I3 kernel (i3_variants)
  size_t nparts_cap = 0;  // (cell, j, m-chunk) units the partial-sum buffer K3part holds
  // buffers of the transform precision (complex = double2 or float2)
  void* what = nullptr;      // [nb][4][n*n] spectral pairs (w0+iw1, w2+iw3, w1+iw2, w3)
  void* wfine = nullptr;     // [nb][2][n*n] fine-grid fields (w0+iw1, w2+iw3)
  void* Dacc = nullptr;      // [nb][2][n*n] spectral D (pairs (1,2), (3,-))
  void* K2acc = nullptr;     // [nb][n*n] (real)
  void* K4acc = nullptr;     // [nb][2][n*n] spectral K4 pairs (0,1), (2,3)
  int nch = 1;               // angle chunks per cell of the I1 and I2/I4 kernels
  void* Dpart = nullptr;     // their per-chunk partials [nb][nch][...] (nch > 1 only)
  void* K2part = nullptr;
  void* K4part = nullptr;
  void* K3part = nullptr;    // [nb*J*nmc][2][n*n] fine-grid K3 pair partial sums
  void* ws = nullptr;        // per-CTA scratch
  size_t ws_fields = 0;      // complex n*n fields of scratch per CTA slot
  int ws_slots = 0;          // number of CTA slots in ws
  double* cbuf = nullptr;    // [nb][4][N][N] staging for collide in/out
  double* wbuf = nullptr;
};

// Extra buffers of the collision operator's vector-Jacobian product
// (collision_vjp.cuh) for a batch of nb cells and up to kcap cotangents at once;
// the forward intermediates (what, wfine, D, K2, K4) are recomputed into the
// CollisionWork of the same batch.  Every cotangent buffer below holds kcap
// copies of the shape given, one per cotangent.
constexpr int kMaxCotangents = 4;
struct VjpWork {
  int prec = 0;
  int nb = 0;
  int kcap = 1;          // cotangents one product can carry
  int nmc = 1;           // m-chunks per (cell, j) unit of the I3 transpose kernel
  int mch = 1;
  int grid = 0;          // persistent grid of the I3 transpose kernel
  int i3v = 0;           // I3 transpose kernel variant (vjp_i3_variants)
  void* nu = nullptr;    // [nb][2][n*n] fine-grid cotangent pairs (0,1), (2,3)
  void* nuf = nullptr;   // [nb][n*n] (real) cotangent of f = 2 w0 - 1
  void* muD = nullptr;   // [nb][2][n*n] cotangent of D pairs (1,2), (3,-)
  void* muK2 = nullptr;  // [nb][n*n] (real)
  void* mu4 = nullptr;   // [nb][2][n*n] cotangent of the raw K4 pairs
  void* mu3 = nullptr;   // [nb][2][n*n] cotangent of the raw K3 pairs
  void* part_r = nullptr;  // [nb*J*nmc][2][n*n] I3 transpose partials, real space
  void* part_s = nullptr;  // [nb*J*nmc][2][(n/2-1)^2] I3 transpose partials, Fourier space, kept frequencies
  void* ws = nullptr;
};

// Launch configuration helpers.
constexpr int kThreads = 256;

// Per-device once-flags (function attributes are set per device): true the first time for the
// current device.
inline bool first_on_device(unsigned long long& done_mask) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (done_mask & bit) return false;
  done_mask |= bit;
  return true;
}

// Kernel groups for the per-kernel device-time accounting (qbe_kernel_time).
enum KernelGroup { KG_PREP = 0, KG_I1 = 1, KG_I24 = 2, KG_I3 = 3, KG_ASSEMBLE = 4, KG_TRANSPORT = 5, KG_RK = 6,
                   KG_VJP = 7, KG_VJP_I3 = 8, KG_ADJ_TRANSPORT = 9, KG_COUNT = 10 };

// Brackets launches with CUDA events on their stream when enabled; the events
// are resolved (and the stream synchronised) only in collect().
struct KernelTimer {
  bool on = false;
  struct Pending {
    int which;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  double total_ms[KG_COUNT] = {};
  long long count[KG_COUNT] = {};
  void begin(int which, cudaStream_t s) {
    if (!on) return;
    Pending p{which, nullptr, nullptr};
    cudaEventCreate(&p.a);
    cudaEventCreate(&p.b);
    cudaEventRecord(p.a, s);
    pending.push_back(p);
  }
  void end(cudaStream_t s) {
    if (!on || pending.empty()) return;
    cudaEventRecord(pending.back().b, s);
  }
  cudaError_t collect() {
    cudaError_t err = cudaSuccess;
    for (auto& p : pending) {
      float ms = 0.f;
      cudaError_t e = cudaEventSynchronize(p.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
      if (e == cudaSuccess) {
        total_ms[p.which] += ms;
        count[p.which] += 1;
      } else {
        err = e;
      }
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    pending.clear();
    return err;
  }
  void reset() {
    collect();
    for (int i = 0; i < KG_COUNT; ++i) { total_ms[i] = 0; count[i] = 0; }
  }
};

// Host-side table construction (tables.cpp); with_f32 also uploads FP32 copies.
bool build_tables(int N, int J, int M, double L, double R, Tables& t, std::string& err, bool with_f32 = false);
void free_tables(Tables& t);

// Wall Fermi-Dirac state in Pauli form on the coarse grid [4][N][N] (eq. W_FermiDirac).
void fermi_dirac_pauli(const qbe_fd& fd, int N, double L, std::vector<double>& out);

// Collision operator on a batch (collision.cu).  w, c: device [nb][4][N][N].
cudaError_t collide_batch(const Tables& t, CollisionWork& cw, const double* w, double* c, int ncells,
                          cudaStream_t s, long long& launches, KernelTimer* tm);
cudaError_t alloc_collision_work(const Tables& t, int nb, CollisionWork& cw, int prec = 0);
template <int n, class T>
cudaError_t collide_batch_n(const Tables& t, CollisionWork& cw, const double* w, double* c, int ncells, cudaStream_t s,
                            long long& launches, KernelTimer* tm);
template <int n, class T>
int i3_blocks_per_sm(int variant);
template <int n, class T>
int i3_variant_count();
template <int n, class T>
int i3_default_variant();
template <int n, class T>
int i3_variant_concurrency(int variant, int grid, int total);
template <int n, class T>
const char* i3_variant_name(int variant);
// Launch variants of the I3 kernel ("tile shapes" the autotuner chooses among) for a grid and
// precision: their number, resident blocks per SM, and a description.
int i3_variants(int n, int prec);
int i3_default(int n, int prec);
int i3_variant_bps(int n, int prec, int variant);
int i3_concurrency(int n, int prec, int variant, int grid, int total);
const char* i3_variant_desc(int n, int prec, int variant);
// The collision operator in parts (collision_kernels.cuh): the per-cell terms before I3, the I3
// work queue over one or several simulations of the same padded size, the per-cell assembly.
cudaError_t collide_pre(const Tables& t, CollisionWork& cw, const double* w, int ncells, cudaStream_t s,
                        long long& launches);
cudaError_t collide_post(const Tables& t, CollisionWork& cw, double* c, int ncells, cudaStream_t s,
                         long long& launches);
cudaError_t i3_group(const Tables* const* tabs, const CollisionWork* const* cws, const int* ncells, int njobs,
                     void* ws, int grid, cudaStream_t s, long long& launches, int max_units = 0);
template <int n, class T>
cudaError_t collide_pre_n(const Tables& t, CollisionWork& cw, const double* w, int ncells, cudaStream_t s,
                          long long& launches, KernelTimer* tm);
template <int n, class T>
cudaError_t collide_post_n(const Tables& t, CollisionWork& cw, double* c, int ncells, cudaStream_t s,
                           long long& launches, KernelTimer* tm);
template <int n, class T>
cudaError_t i3_group_n(const Tables* const* tabs, const CollisionWork* const* cws, const int* ncells, int njobs,
                       void* ws, int grid, cudaStream_t s, long long& launches, int max_units);
void free_collision_work(CollisionWork& cw);

// Vector-Jacobian products of the collision operator (collision_vjp.cuh) at
// one state for K <= vw.kcap cotangents: grad[k] (+)= (dC/dW)^T lam[k] for w,
// lam[k], grad[k] device [ncells][4][N][N]; accumulate selects += instead of =.
// The state's forward transforms are shared by the K products.  Uses cw's
// forward buffers as scratch.
cudaError_t collide_vjp(const Tables& t, CollisionWork& cw, VjpWork& vw, const double* w, const double* const* lam,
                        double* const* grad, int K, int ncells, int accumulate, cudaStream_t s, long long& launches,
                        KernelTimer* tm);
cudaError_t alloc_vjp_work(const Tables& t, int nb, VjpWork& vw, int prec = 0, int kcap = 1);
// How many cotangents one product should carry for this grid and precision form (1 .. kMaxCotangents).
int vjp_cotangent_group(const Tables& t, int prec);
// I3 transpose kernel variants for a padded grid and precision (0: the default, the fastest measured).
int vjp_i3_variants(int n, int prec);
void free_vjp_work(VjpWork& vw);
template <int n, class T>
cudaError_t collide_vjp_n(const Tables& t, CollisionWork& cw, VjpWork& vw, const double* w, const double* const* lam,
                          double* const* grad, int K, int ncells, int accumulate, cudaStream_t s, long long& launches,
                          KernelTimer* tm);
template <int n, class T>
int i3_vjp_blocks_per_sm();

// Transport, precession/RK and moments (transport.cu).
struct BoundaryDev {
  int kind = QBE_PERIODIC;
  double alpha = 0.0;
  double* phiL = nullptr;   // [4][N][N] wall state at x = 0
  double* phiR = nullptr;   // [4][N][N] wall state at x = 1
  double ZL = 1.0, ZR = 1.0;
  double* fbar = nullptr;   // [2] outgoing number fluxes (device scratch)
};

cudaError_t advect_substep(const double* Win, double* Wout, int Nx, int N, double L, double tau,
                           const BoundaryDev& bc, cudaStream_t s, long long& launches, KernelTimer* tm);
cudaError_t rk_stage1(const double* W, const double* C, const double* B, double dt, double* F0, double* W1,
                      int Nx, int N, cudaStream_t s, long long& launches, KernelTimer* tm);
cudaError_t rk_stage2(const double* W, const double* F0, const double* C1, const double* W1, const double* B,
                      double dt, double* Wout, int Nx, int N, cudaStream_t s, long long& launches, KernelTimer* tm);
// Adjoints (transport.cu): the transpose of one transport substep at the
// forward input Win (gsum: device scratch [2]); of Heun's RK2 with the
// precession term given G1 = C'(W1)^T lam (writes lF0 and the partial lU,
// accumulates gB); the final-time observables and their gradient.
cudaError_t advect_substep_vjp(const double* Win, const double* lam_out, double* lam_in, int Nx, int N, double L,
                               double tau, const BoundaryDev& bc, double* gsum, cudaStream_t s, long long& launches,
                               KernelTimer* tm);
cudaError_t rk_vjp_launch(const double* U, const double* W1, const double* lam, const double* G1, const double* B,
                          double dt, double* lF0, double* lU, double* gB, int Nx, int N, cudaStream_t s,
                          long long& launches, KernelTimer* tm);
cudaError_t observables_launch(const double* W, int Nx, int N, double L, double* part, double* out2,
                               cudaStream_t s, long long& launches);
cudaError_t observables_vjp_launch(const double* gbar, int Nx, int N, double L, double* lam, cudaStream_t s,
                                   long long& launches);
// Diagnostics (diagnostics.cu).  FdDev: one Fermi-Dirac state W_FD(v - u) with
// the unit Bloch vector of its up state.
struct FdDev {
  double T, mu_up, mu_dn;
  double bloch[3];
  double u[2];
};
cudaError_t entropy_launch(const double* W, int Nx, int N, double L, double* out, cudaStream_t s,
                           long long& launches);
cudaError_t relative_entropy_launch(const double* W, int Nx, int N, double L, const FdDev* fd, int nfd, double* rel,
                                    double* l1, cudaStream_t s, long long& launches);
void fd_fit_from_moments(const double rho4[4], const double mom[2], double energy, qbe_fermi_dirac& out);
double dilog(double x);

cudaError_t moments_launch(const double* W, int Nx, int N, double L, double* out7, cudaStream_t s,
                           long long& launches);

}  // namespace qbe
