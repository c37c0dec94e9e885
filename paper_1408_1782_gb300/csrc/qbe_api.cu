// C ABI (include/qbe.h): solver handle, argument checks, host/device copies
// and the split time step of Sec. 4.
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace qbe;

namespace {

// Device buffer that only grows.
struct DevBuf {
  double* p = nullptr;
  size_t n = 0;   // doubles
  cudaError_t ensure(size_t want) {
    if (want <= n) return cudaSuccess;
    cudaFree(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMalloc((void**)&p, want * sizeof(double));
    if (e == cudaSuccess) n = want;
    return e;
  }
  void release() {
    cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

}  // namespace

struct qbe_handle {
  qbe_grid g{};
  cudaStream_t stream = nullptr;
  std::string err;
  Tables tab;
  CollisionWork cw;
  double* W = nullptr;     // state [Nx][4][N][N]
  double* Wa = nullptr;    // second state buffer (transport ping-pong, RK stage)
  double* F0 = nullptr;    // RK first slope
  double* Cb = nullptr;    // collision output
  double* B = nullptr;     // [Nx][3]
  double* mom = nullptr;   // [Nx][7]
  double* fbar = nullptr;  // [2]
  double* phiL = nullptr;  // [4][N][N]
  double* phiR = nullptr;
  BoundaryDev bc;
  bool has_state = false;
  long long launches = 0;
  KernelTimer timer;
  // adjoint: collision VJP buffers (allocated on first use), the tape of the
  // last qbe_step_checkpointed call and the reverse sweep's scratch
  VjpWork vw;
  bool vw_ready = false;
  double* lbuf = nullptr;      // [nb][4][N][N] host-path staging of the cotangent
  bool tape_valid = false;
  double tape_dt = 0.0;
  int tape_nsteps = 0, tape_every = 1;
  bool tape_full = false;
  int vjp_i3v = 0;             // I3 transpose kernel variant (qbe_set_vjp_i3_variant)      // snaps holds every step's intermediate states (qbe_step_taped)
  DevBuf ckpt;                 // [ceil(nsteps/every)] states
  DevBuf snaps;                // [every][2 sA + 2] states of one segment, or [nsteps][2 sA + 2]
  DevBuf adj;                  // [5] states: two cotangent buffers, G1, lF0, final state
  DevBuf small;                // gsum[2], gbar[2], obs_out[2], gB[Nx][3], obs_part[Nx][2]
  DevBuf gradb;                // [ncot][Nx][3] field gradients of a reverse sweep
};

namespace {

int tune_group(const std::vector<qbe_handle*>& hs, cudaStream_t s, double* best_ms, std::string& err);

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int fail(qbe_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(qbe_handle* h, cudaError_t e, const char* where) {
  return fail(h, QBE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t state_elems(const qbe_handle* h) { return (size_t)h->g.Nx * 4 * h->g.N * h->g.N; }

int transport_substeps(double tau, double dx, double L) {
  const double nu = std::fabs(tau) * L / dx;
  int s = (int)std::ceil(nu / 1.0 - 1e-12);
  return s < 1 ? 1 : s;
}

// snaps (optional): receives the input state of every substep, in order.
int do_advect(qbe_handle* h, double tau, double* snaps = nullptr) {
  const int Nx = h->g.Nx, N = h->g.N;
  const int s = transport_substeps(tau, 1.0 / Nx, h->g.L);
  const size_t S = state_elems(h);
  for (int k = 0; k < s; ++k) {
    if (snaps) {
      cudaError_t e = cudaMemcpyAsync(snaps + (size_t)k * S, h->W, S * sizeof(double), cudaMemcpyDeviceToDevice,
                                      h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "advect snapshot");
    }
    cudaError_t e = advect_substep(h->W, h->Wa, Nx, N, h->g.L, tau / s, h->bc, h->stream, h->launches, &h->timer);
    if (e != cudaSuccess) return cuda_fail(h, e, "advect");
    std::swap(h->W, h->Wa);
  }
  return QBE_OK;
}

int do_collide_dev(qbe_handle* h, const double* w, double* c, int ncells) {
  const size_t per = (size_t)4 * h->g.N * h->g.N;
  for (int c0 = 0; c0 < ncells; c0 += h->cw.nb) {
    const int nc = (ncells - c0) < h->cw.nb ? (ncells - c0) : h->cw.nb;
    cudaError_t e = collide_batch(h->tab, h->cw, w + (size_t)c0 * per, c + (size_t)c0 * per, nc, h->stream,
                                  h->launches, &h->timer);
    if (e != cudaSuccess) return cuda_fail(h, e, "collide");
  }
  return QBE_OK;
}

// snaps (optional): receives the stage inputs U (= W) and W1.
int do_rk2(qbe_handle* h, double dt, double* snaps = nullptr) {
  const int Nx = h->g.Nx, N = h->g.N;
  const size_t S = state_elems(h);
  if (snaps) {
    cudaError_t e = cudaMemcpyAsync(snaps, h->W, S * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "rk snapshot");
  }
  int r = do_collide_dev(h, h->W, h->Cb, Nx);
  if (r) return r;
  cudaError_t e = rk_stage1(h->W, h->Cb, h->B, dt, h->F0, h->Wa, Nx, N, h->stream, h->launches, &h->timer);
  if (e != cudaSuccess) return cuda_fail(h, e, "rk stage 1");
  if (snaps) {
    e = cudaMemcpyAsync(snaps + S, h->Wa, S * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "rk snapshot");
  }
  r = do_collide_dev(h, h->Wa, h->Cb, Nx);
  if (r) return r;
  e = rk_stage2(h->W, h->F0, h->Cb, h->Wa, h->B, dt, h->W, Nx, N, h->stream, h->launches, &h->timer);
  if (e != cudaSuccess) return cuda_fail(h, e, "rk stage 2");
  return QBE_OK;
}

// Substeps of each transport half step (the same count do_advect uses).
int half_substeps(const qbe_handle* h, double dt) { return transport_substeps(0.5 * dt, 1.0 / h->g.Nx, h->g.L); }

// snaps (optional): the 2 sA + 2 intermediate states of the step, in order
// (inputs of the first half's substeps, U, W1, inputs of the second half's substeps).
int do_step(qbe_handle* h, double dt, double* snaps = nullptr) {
  const int sA = half_substeps(h, dt);
  const size_t S = state_elems(h);
  int r = do_advect(h, 0.5 * dt, snaps);
  if (!r) r = do_rk2(h, dt, snaps ? snaps + (size_t)sA * S : nullptr);
  if (!r) r = do_advect(h, 0.5 * dt, snaps ? snaps + (size_t)(sA + 2) * S : nullptr);
  return r;
}

// Adjoint workspace for products carrying up to kneed cotangents at once (grown on demand).
int ensure_vjp(qbe_handle* h, int kneed = 1) {
  if (h->vw_ready && h->vw.kcap >= kneed) return QBE_OK;
  if (h->vw_ready) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint workspace resize");
    free_vjp_work(h->vw);
    cudaFree(h->lbuf);
    h->lbuf = nullptr;
    h->vw_ready = false;
  }
  cudaError_t e = alloc_vjp_work(h->tab, h->cw.nb, h->vw, h->g.precision, kneed);
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&h->lbuf, (size_t)h->cw.nb * 4 * h->g.N * h->g.N * sizeof(double));
  if (e != cudaSuccess) {
    free_vjp_work(h->vw);
    cudaFree(h->lbuf);
    h->lbuf = nullptr;
    return fail(h, QBE_ERR_ALLOC, std::string("adjoint workspace: ") + cudaGetErrorString(e));
  }
  h->vw.i3v = h->vjp_i3v;
  h->vw_ready = true;
  return QBE_OK;
}

// grad[k] (+)= (dC/dW)^T lam[k] at the state w for K <= kMaxCotangents cotangents (device
// [ncells][4][N][N] each), in batches of cw.nb cells; the K products share the state's transforms.
int do_collide_vjp_dev(qbe_handle* h, const double* w, const double* const* lam, double* const* grad, int K,
                       int ncells, int accumulate) {
  int r = ensure_vjp(h, K);
  if (r) return r;
  const size_t per = (size_t)4 * h->g.N * h->g.N;
  const double* lk[kMaxCotangents];
  double* gk[kMaxCotangents];
  for (int c0 = 0; c0 < ncells; c0 += h->cw.nb) {
    const int nc = (ncells - c0) < h->cw.nb ? (ncells - c0) : h->cw.nb;
    for (int k = 0; k < K; ++k) {
      lk[k] = lam[k] + (size_t)c0 * per;
      gk[k] = grad[k] + (size_t)c0 * per;
    }
    cudaError_t e = collide_vjp(h->tab, h->cw, h->vw, w + (size_t)c0 * per, lk, gk, K, nc, accumulate, h->stream,
                                h->launches, &h->timer);
    if (e != cudaSuccess) return cuda_fail(h, e, "collide vjp");
  }
  return QBE_OK;
}

int do_collide_vjp_dev(qbe_handle* h, const double* w, const double* lam, double* grad, int ncells, int accumulate) {
  return do_collide_vjp_dev(h, w, &lam, &grad, 1, ncells, accumulate);
}

// Reverse of one recorded step for K <= kMaxCotangents cotangents at once: *lam[k] (cotangent of
// the step's output) becomes the cotangent of its input; gB[k] accumulates the field gradient.
// *lam[k] and *tmp[k] are swapped as the sweep ping-pongs between them; G1[k], lF0[k] are scratch.
// The two collision products of the step (at W1 and at U) each serve all K cotangents.
int step_vjp_group(qbe_handle* h, double dt, const double* snaps, double** lam, double** tmp, double* const* G1,
                   double* const* lF0, double* const* gB, int K, double* gsum) {
  const int Nx = h->g.Nx, N = h->g.N;
  const int sA = half_substeps(h, dt);
  const double tau = 0.5 * dt / sA;
  const size_t S = state_elems(h);
  for (int q = 0; q < K; ++q)
    for (int k = sA - 1; k >= 0; --k) {
      cudaError_t e = advect_substep_vjp(snaps + (size_t)(sA + 2 + k) * S, lam[q], tmp[q], Nx, N, h->g.L, tau,
                                         h->bc, gsum, h->stream, h->launches, &h->timer);
      if (e != cudaSuccess) return cuda_fail(h, e, "advect vjp");
      std::swap(lam[q], tmp[q]);
    }
  const double* U = snaps + (size_t)sA * S;
  const double* W1 = snaps + (size_t)(sA + 1) * S;
  int r = do_collide_vjp_dev(h, W1, lam, G1, K, Nx, 0);
  if (r) return r;
  for (int q = 0; q < K; ++q) {
    cudaError_t e = rk_vjp_launch(U, W1, lam[q], G1[q], h->B, dt, lF0[q], tmp[q], gB[q], Nx, N, h->stream,
                                  h->launches, &h->timer);
    if (e != cudaSuccess) return cuda_fail(h, e, "rk vjp");
  }
  r = do_collide_vjp_dev(h, U, lF0, tmp, K, Nx, 1);
  if (r) return r;
  for (int q = 0; q < K; ++q) {
    std::swap(lam[q], tmp[q]);
    for (int k = sA - 1; k >= 0; --k) {
      cudaError_t e = advect_substep_vjp(snaps + (size_t)k * S, lam[q], tmp[q], Nx, N, h->g.L, tau, h->bc, gsum,
                                         h->stream, h->launches, &h->timer);
      if (e != cudaSuccess) return cuda_fail(h, e, "advect vjp");
      std::swap(lam[q], tmp[q]);
    }
  }
  return QBE_OK;
}

size_t small_elems(const qbe_handle* h) { return 6 + (size_t)h->g.Nx * 5; }

bool valid_fd(const qbe_fd* f) {
  return f && std::isfinite(f->beta) && f->beta > 0 && std::isfinite(f->mu_up) && std::isfinite(f->mu_dn);
}

}  // namespace

extern "C" {

int qbe_create(const qbe_grid* g, qbe_handle** out) {
  if (!out) return QBE_ERR_ARG;
  *out = nullptr;
  if (!g) return QBE_ERR_ARG;
  const bool n_ok = g->N == 8 || g->N == 16 || g->N == 32 || g->N == 48 || g->N == 64 || g->N == 96 || g->N == 128;
  if (!n_ok || g->Nx < 1 || g->J < 2 || g->J > 64 || (g->J % 2) != 0 || g->M < 1 || g->M > 64 ||
      !(g->L > 0) || !(g->R > 0) || !std::isfinite(g->L) || !std::isfinite(g->R))
    return QBE_ERR_ARG;
  if (g->precision != 0 && g->precision != 1) return QBE_ERR_UNSUPPORTED;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || g->device < 0 || g->device >= ndev) return QBE_ERR_CUDA;
  qbe_handle* h = new (std::nothrow) qbe_handle();
  if (!h) return QBE_ERR_ALLOC;
  h->g = *g;
  DeviceGuard dg(g->device);
  std::string err;
  if (!build_tables(g->N, g->J, g->M, g->L, g->R, h->tab, err, g->precision == 1)) {
    qbe_destroy(h);
    return QBE_ERR_ALLOC;
  }
  // collision batch: all cells of the state (one evaluation per RK stage)
  if (alloc_collision_work(h->tab, g->Nx, h->cw, g->precision) != cudaSuccess) {
    qbe_destroy(h);
    return QBE_ERR_ALLOC;
  }
  const size_t se = state_elems(h) * sizeof(double);
  const size_t wall = (size_t)4 * g->N * g->N * sizeof(double);
  if (cudaMalloc(&h->W, se) != cudaSuccess || cudaMalloc(&h->Wa, se) != cudaSuccess ||
      cudaMalloc(&h->F0, se) != cudaSuccess || cudaMalloc(&h->Cb, se) != cudaSuccess ||
      cudaMalloc(&h->B, (size_t)g->Nx * 3 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->mom, (size_t)g->Nx * 7 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->fbar, 2 * sizeof(double)) != cudaSuccess || cudaMalloc(&h->phiL, wall) != cudaSuccess ||
      cudaMalloc(&h->phiR, wall) != cudaSuccess) {
    qbe_destroy(h);
    return QBE_ERR_ALLOC;
  }
  if (cudaMemset(h->B, 0, (size_t)g->Nx * 3 * sizeof(double)) != cudaSuccess ||
      cudaMemset(h->W, 0, se) != cudaSuccess || cudaMemset(h->fbar, 0, 2 * sizeof(double)) != cudaSuccess) {
    qbe_destroy(h);
    return QBE_ERR_CUDA;
  }
  h->bc.kind = QBE_PERIODIC;
  h->bc.phiL = h->phiL;
  h->bc.phiR = h->phiR;
  h->bc.fbar = h->fbar;
  *out = h;
  return QBE_OK;
}

void qbe_destroy(qbe_handle* h) {
  if (!h) return;
  DeviceGuard dg(h->g.device);
  h->timer.collect();
  free_tables(h->tab);
  free_collision_work(h->cw);
  cudaFree(h->W); cudaFree(h->Wa); cudaFree(h->F0); cudaFree(h->Cb); cudaFree(h->B);
  cudaFree(h->mom); cudaFree(h->fbar); cudaFree(h->phiL); cudaFree(h->phiR);
  free_vjp_work(h->vw);
  cudaFree(h->lbuf);
  h->ckpt.release(); h->snaps.release(); h->adj.release(); h->small.release(); h->gradb.release();
  delete h;
}

const char* qbe_last_error(const qbe_handle* h) { return h ? h->err.c_str() : "null handle"; }

long long qbe_launch_count(const qbe_handle* h) { return h ? h->launches : 0; }

int qbe_enable_timing(qbe_handle* h, int enable) {
  if (!h) return QBE_ERR_ARG;
  DeviceGuard dg(h->g.device);
  h->timer.reset();
  h->timer.on = enable != 0;
  return QBE_OK;
}

int qbe_kernel_time(qbe_handle* h, int which, double* total_ms, long long* launches) {
  if (!h) return QBE_ERR_ARG;
  if (which < 0 || which >= KG_COUNT) return fail(h, QBE_ERR_ARG, "unknown kernel group");
  DeviceGuard dg(h->g.device);
  cudaError_t e = h->timer.collect();
  if (e != cudaSuccess) return cuda_fail(h, e, "kernel timing");
  if (total_ms) *total_ms = h->timer.total_ms[which];
  if (launches) *launches = h->timer.count[which];
  return QBE_OK;
}

int qbe_i3_shape(const qbe_handle* h, int* variant, int* nvariants, int* grid, int* m_chunks) {
  if (!h) return QBE_ERR_ARG;
  if (variant) *variant = h->cw.i3_variant;
  if (nvariants) *nvariants = i3_variants(h->tab.n, h->cw.prec);
  if (grid) *grid = h->cw.grid_i3;
  if (m_chunks) *m_chunks = h->cw.nmc;
  return QBE_OK;
}

const char* qbe_i3_variant_name(const qbe_handle* h, int variant) {
  if (!h) return nullptr;
  return i3_variant_desc(h->tab.n, h->cw.prec, variant);
}

int qbe_set_i3_shape(qbe_handle* h, int variant, int grid, int m_chunks) {
  if (!h) return QBE_ERR_ARG;
  if (variant < -1 || variant >= i3_variants(h->tab.n, h->cw.prec) || grid < 0 || m_chunks < 0)
    return fail(h, QBE_ERR_ARG, "set_i3_shape: variant, grid or m-chunks out of range");
  const int cap_nmc = (int)(h->cw.nparts_cap / ((size_t)h->cw.nb * h->tab.J));
  if (m_chunks > cap_nmc) return fail(h, QBE_ERR_ARG, "set_i3_shape: more m-chunks than the partial sums hold");
  if (variant >= 0) h->cw.i3_variant = variant;
  if (grid > 0) {
    const int cap = (int)(h->cw.ws_fields / 3);
    h->cw.grid_i3 = grid < cap ? grid : cap;
  }
  if (m_chunks > 0) {
    h->cw.mch = (h->tab.M + m_chunks - 1) / m_chunks;
    h->cw.nmc = (h->tab.M + h->cw.mch - 1) / h->cw.mch;
  }
  return QBE_OK;
}

int qbe_vjp_i3_variant(const qbe_handle* h, int* variant, int* nvariants) {
  if (!h) return QBE_ERR_ARG;
  if (variant) *variant = h->vjp_i3v;
  if (nvariants) *nvariants = vjp_i3_variants(h->tab.n, h->g.precision);
  return QBE_OK;
}

int qbe_set_vjp_i3_variant(qbe_handle* h, int variant) {
  if (!h) return QBE_ERR_ARG;
  const int nv = vjp_i3_variants(h->tab.n, h->g.precision);
  if (variant < -1 || variant >= nv) return fail(h, QBE_ERR_ARG, "set_vjp_i3_variant: variant out of range");
  h->vjp_i3v = variant < 0 ? 0 : variant;
  h->vw.i3v = h->vjp_i3v;
  return QBE_OK;
}

int qbe_autotune(qbe_handle* h, double* best_ms) {
  if (!h) return QBE_ERR_ARG;
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "autotune: no state");
  DeviceGuard dg(h->g.device);
  std::string err;
  const int rc = tune_group({h}, h->stream, best_ms, err);
  return rc == QBE_OK ? rc : fail(h, rc, err);
}

int qbe_set_stream(qbe_handle* h, void* stream) {
  if (!h) return QBE_ERR_ARG;
  h->stream = (cudaStream_t)stream;
  return QBE_OK;
}

int qbe_set_boundary(qbe_handle* h, int bc, const qbe_fd* left, const qbe_fd* right, double alpha) {
  if (!h) return QBE_ERR_ARG;
  if (bc != QBE_PERIODIC && bc != QBE_DIRICHLET && bc != QBE_MAXWELL)
    return fail(h, QBE_ERR_ARG, "unknown boundary kind");
  DeviceGuard dg(h->g.device);
  h->tape_valid = false;
  if (bc == QBE_PERIODIC) {
    h->bc.kind = bc;
    return QBE_OK;
  }
  if (!valid_fd(left) || !valid_fd(right)) return fail(h, QBE_ERR_ARG, "invalid wall Fermi-Dirac state");
  if (bc == QBE_MAXWELL && !(alpha >= 0.0 && alpha <= 1.0)) return fail(h, QBE_ERR_ARG, "alpha outside [0,1]");
  const int N = h->g.N;
  std::vector<double> pl, pr;
  fermi_dirac_pauli(*left, N, h->g.L, pl);
  fermi_dirac_pauli(*right, N, h->g.L, pr);
  // Z = dv^2 sum_{incoming v} tr W_FD |v_x|   (Sec. 2, diffusive reflection)
  const double dv = 2.0 * h->g.L / N;
  double ZL = 0, ZR = 0;
  for (int ix = 0; ix < N; ++ix)
    for (int iy = 0; iy < N; ++iy) {
      const double vx = dv * (ix - N / 2);
      if (vx > 0) ZL += 2.0 * pl[(size_t)ix * N + iy] * vx;
      if (vx < 0) ZR += 2.0 * pr[(size_t)ix * N + iy] * (-vx);
    }
  ZL *= dv * dv;
  ZR *= dv * dv;
  if (bc == QBE_MAXWELL && alpha > 0 && (!(ZL > 0) || !(ZR > 0)))
    return fail(h, QBE_ERR_ARG, "diffusive wall state has zero incoming flux");
  cudaError_t e = cudaMemcpyAsync(h->phiL, pl.data(), pl.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->phiR, pr.data(), pr.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_boundary");
  h->bc.kind = bc;
  h->bc.alpha = bc == QBE_MAXWELL ? alpha : 0.0;
  h->bc.ZL = ZL > 0 ? ZL : 1.0;
  h->bc.ZR = ZR > 0 ? ZR : 1.0;
  return QBE_OK;
}

int qbe_set_bfield(qbe_handle* h, const double* B, int on_device) {
  if (!h || !B) return h ? fail(h, QBE_ERR_ARG, "null B") : QBE_ERR_ARG;
  DeviceGuard dg(h->g.device);
  const size_t bytes = (size_t)h->g.Nx * 3 * sizeof(double);
  h->tape_valid = false;
  cudaError_t e = cudaMemcpyAsync(h->B, B, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? QBE_OK : cuda_fail(h, e, "set_bfield");
}

int qbe_set_state(qbe_handle* h, const double* w, int on_device) {
  if (!h || !w) return h ? fail(h, QBE_ERR_ARG, "null state") : QBE_ERR_ARG;
  DeviceGuard dg(h->g.device);
  h->tape_valid = false;
  cudaError_t e = cudaMemcpyAsync(h->W, w, state_elems(h) * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
  h->has_state = true;
  return QBE_OK;
}

int qbe_get_state(qbe_handle* h, double* w, int on_device) {
  if (!h || !w) return h ? fail(h, QBE_ERR_ARG, "null state") : QBE_ERR_ARG;
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  DeviceGuard dg(h->g.device);
  cudaError_t e = cudaMemcpyAsync(w, h->W, state_elems(h) * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? QBE_OK : cuda_fail(h, e, "get_state");
}

int qbe_collide(qbe_handle* h, const double* w, double* c, int ncells, int on_device) {
  if (!h) return QBE_ERR_ARG;
  if (!w || !c || ncells < 1) return fail(h, QBE_ERR_ARG, "collide: null pointer or ncells < 1");
  DeviceGuard dg(h->g.device);
  if (on_device) return do_collide_dev(h, w, c, ncells);
  const size_t per = (size_t)4 * h->g.N * h->g.N;
  for (int c0 = 0; c0 < ncells; c0 += h->cw.nb) {
    const int nc = (ncells - c0) < h->cw.nb ? (ncells - c0) : h->cw.nb;
    cudaError_t e = cudaMemcpyAsync(h->cw.wbuf, w + (size_t)c0 * per, (size_t)nc * per * sizeof(double),
                                    cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "collide H2D");
    int r = do_collide_dev(h, h->cw.wbuf, h->cw.cbuf, nc);
    if (r) return r;
    e = cudaMemcpyAsync(c + (size_t)c0 * per, h->cw.cbuf, (size_t)nc * per * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "collide D2H");
  }
  return QBE_OK;
}

int qbe_advect(qbe_handle* h, double tau) {
  if (!h) return QBE_ERR_ARG;
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  if (!std::isfinite(tau)) return fail(h, QBE_ERR_ARG, "tau not finite");
  DeviceGuard dg(h->g.device);
  h->tape_valid = false;
  return do_advect(h, tau);
}

int qbe_collide_rk2(qbe_handle* h, double dt) {
  if (!h) return QBE_ERR_ARG;
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  if (!std::isfinite(dt)) return fail(h, QBE_ERR_ARG, "dt not finite");
  DeviceGuard dg(h->g.device);
  h->tape_valid = false;
  return do_rk2(h, dt);
}

int qbe_step(qbe_handle* h, double dt, int nsteps) {
  if (!h) return QBE_ERR_ARG;
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  if (!std::isfinite(dt) || nsteps < 0) return fail(h, QBE_ERR_ARG, "bad dt or nsteps");
  DeviceGuard dg(h->g.device);
  h->tape_valid = false;
  for (int s = 0; s < nsteps; ++s) {
    const int r = do_step(h, dt);
    if (r) return r;
  }
  return QBE_OK;
}

int qbe_moments(qbe_handle* h, double* rho, double* mom, double* energy, int on_device) {
  if (!h) return QBE_ERR_ARG;
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  DeviceGuard dg(h->g.device);
  const int Nx = h->g.Nx;
  cudaError_t e = moments_launch(h->W, Nx, h->g.N, h->g.L, h->mom, h->stream, h->launches);
  if (e != cudaSuccess) return cuda_fail(h, e, "moments");
  std::vector<double> m((size_t)Nx * 7);
  e = cudaMemcpyAsync(m.data(), h->mom, m.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "moments D2H");
  std::vector<double> r4((size_t)Nx * 4), m2((size_t)Nx * 2), en((size_t)Nx);
  for (int c = 0; c < Nx; ++c) {
    for (int k = 0; k < 4; ++k) r4[(size_t)c * 4 + k] = m[(size_t)c * 7 + k];
    m2[(size_t)c * 2] = m[(size_t)c * 7 + 4];
    m2[(size_t)c * 2 + 1] = m[(size_t)c * 7 + 5];
    en[c] = m[(size_t)c * 7 + 6];
  }
  const cudaMemcpyKind k = on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  if (rho) e = cudaMemcpy(rho, r4.data(), r4.size() * sizeof(double), k);
  if (e == cudaSuccess && mom) e = cudaMemcpy(mom, m2.data(), m2.size() * sizeof(double), k);
  if (e == cudaSuccess && energy) e = cudaMemcpy(energy, en.data(), en.size() * sizeof(double), k);
  return e == cudaSuccess ? QBE_OK : cuda_fail(h, e, "moments copy");
}

int qbe_collide_vjp(qbe_handle* h, const double* w, const double* lam, double* grad, int ncells, int on_device) {
  if (!h) return QBE_ERR_ARG;
  if (!w || !lam || !grad || ncells < 1) return fail(h, QBE_ERR_ARG, "collide_vjp: null pointer or ncells < 1");
  DeviceGuard dg(h->g.device);
  if (on_device) return do_collide_vjp_dev(h, w, lam, grad, ncells, 0);
  int r = ensure_vjp(h);
  if (r) return r;
  const size_t per = (size_t)4 * h->g.N * h->g.N;
  for (int c0 = 0; c0 < ncells; c0 += h->cw.nb) {
    const int nc = (ncells - c0) < h->cw.nb ? (ncells - c0) : h->cw.nb;
    const size_t bytes = (size_t)nc * per * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(h->cw.wbuf, w + (size_t)c0 * per, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->lbuf, lam + (size_t)c0 * per, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "collide_vjp H2D");
    r = do_collide_vjp_dev(h, h->cw.wbuf, h->lbuf, h->cw.cbuf, nc, 0);
    if (r) return r;
    e = cudaMemcpyAsync(grad + (size_t)c0 * per, h->cw.cbuf, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "collide_vjp D2H");
  }
  return QBE_OK;
}

int qbe_collide_vjp_n(qbe_handle* h, int ncot, const double* w, const double* lam, double* grad, int ncells,
                      int on_device) {
  if (!h) return QBE_ERR_ARG;
  if (!w || !lam || !grad || ncells < 1 || ncot < 1)
    return fail(h, QBE_ERR_ARG, "collide_vjp_n: null pointer, ncells < 1 or ncot < 1");
  if (on_device != 1) return fail(h, QBE_ERR_ARG, "collide_vjp_n: device memory only");
  DeviceGuard dg(h->g.device);
  const size_t per = (size_t)ncells * 4 * h->g.N * h->g.N;
  const double* lk[kMaxCotangents];
  double* gk[kMaxCotangents];
  const int kg = vjp_cotangent_group(h->tab, h->g.precision);
  for (int k0 = 0; k0 < ncot; k0 += kg) {
    const int K = (ncot - k0) < kg ? (ncot - k0) : kg;
    for (int k = 0; k < K; ++k) {
      lk[k] = lam + (size_t)(k0 + k) * per;
      gk[k] = grad + (size_t)(k0 + k) * per;
    }
    const int r = do_collide_vjp_dev(h, w, lk, gk, K, ncells, 0);
    if (r) return r;
  }
  return QBE_OK;
}

int qbe_step_checkpointed(qbe_handle* h, double dt, int nsteps, int checkpoint_every) {
  if (!h) return QBE_ERR_ARG;
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  if (!std::isfinite(dt) || nsteps < 1 || checkpoint_every < 1)
    return fail(h, QBE_ERR_ARG, "bad dt, nsteps or checkpoint_every");
  DeviceGuard dg(h->g.device);
  h->tape_valid = false;
  if (h->tape_full) h->snaps.release();   // a full tape's storage; the reverse sweep takes one segment's
  h->tape_full = false;
  const size_t S = state_elems(h);
  const int every = checkpoint_every < nsteps ? checkpoint_every : nsteps;
  const size_t nck = (size_t)(nsteps + every - 1) / every;
  cudaError_t e = h->ckpt.ensure(nck * S);
  if (e != cudaSuccess) return fail(h, QBE_ERR_ALLOC, "checkpoint storage");
  for (int s = 0; s < nsteps; ++s) {
    if (s % every == 0) {
      e = cudaMemcpyAsync(h->ckpt.p + (size_t)(s / every) * S, h->W, S * sizeof(double), cudaMemcpyDeviceToDevice,
                          h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint");
    }
    const int r = do_step(h, dt);
    if (r) return r;
  }
  h->tape_valid = true;
  h->tape_full = false;
  h->tape_dt = dt;
  h->tape_nsteps = nsteps;
  h->tape_every = every;
  return QBE_OK;
}

int qbe_step_taped(qbe_handle* h, double dt, int nsteps) {
  if (!h) return QBE_ERR_ARG;
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  if (!std::isfinite(dt) || nsteps < 1) return fail(h, QBE_ERR_ARG, "bad dt or nsteps");
  DeviceGuard dg(h->g.device);
  h->tape_valid = false;
  const size_t per_step = (size_t)(2 * half_substeps(h, dt) + 2) * state_elems(h);
  if ((size_t)nsteps > SIZE_MAX / sizeof(double) / per_step) return fail(h, QBE_ERR_ALLOC, "tape size overflows");
  cudaError_t e = h->snaps.ensure((size_t)nsteps * per_step);
  if (e != cudaSuccess) {
    cudaGetLastError();   // an out-of-memory cudaMalloc leaves no sticky error; clear the last-error slot
    return fail(h, QBE_ERR_ALLOC, std::string("tape storage: ") + cudaGetErrorString(e));
  }
  for (int s = 0; s < nsteps; ++s) {
    const int r = do_step(h, dt, h->snaps.p + (size_t)s * per_step);
    if (r) return r;
  }
  h->tape_valid = true;
  h->tape_full = true;
  h->tape_dt = dt;
  h->tape_nsteps = nsteps;
  h->tape_every = nsteps;
  return QBE_OK;
}

int qbe_step_vjp_n(qbe_handle* h, int ncot, const double* lam_final, double* lam_init, double* grad_B,
                   int on_device) {
  if (!h) return QBE_ERR_ARG;
  if (ncot < 1 || !lam_final || !lam_init) return fail(h, QBE_ERR_ARG, "step_vjp: ncot < 1 or null cotangent");
  if (!h->tape_valid) return fail(h, QBE_ERR_STATE, "no valid tape (call qbe_step_checkpointed first)");
  DeviceGuard dg(h->g.device);
  const int Nx = h->g.Nx;
  const double dt = h->tape_dt;
  const int nsteps = h->tape_nsteps, every = h->tape_every;
  const size_t S = state_elems(h);
  const size_t nb3 = (size_t)Nx * 3;
  const int sA = half_substeps(h, dt);
  const size_t per_step = (size_t)(2 * sA + 2) * S;
  // cotangents travel through the sweep in groups (vjp_cotangent_group: up to four, or one for the
  // FP32 shared-memory transpose)
  const int kmax = vjp_cotangent_group(h->tab, h->g.precision);
  const int kg = ncot < kmax ? ncot : kmax;
  int r = ensure_vjp(h, kg);
  if (r) return r;
  if ((!h->tape_full && h->snaps.ensure((size_t)every * per_step) != cudaSuccess) ||
      h->adj.ensure((2 * (size_t)ncot + 2 * (size_t)kg + 1) * S) != cudaSuccess ||
      h->small.ensure(small_elems(h)) != cudaSuccess || h->gradb.ensure((size_t)ncot * nb3) != cudaSuccess)
    return fail(h, QBE_ERR_ALLOC, "adjoint sweep storage");
  // per cotangent k: lam[k], tmp[k] (ping-pong); per group slot q: G1[q], lF0[q]; the final state
  std::vector<double*> lam(ncot), tmp(ncot), gBk(ncot);
  for (int k = 0; k < ncot; ++k) {
    lam[k] = h->adj.p + (size_t)(2 * k) * S;
    tmp[k] = h->adj.p + (size_t)(2 * k + 1) * S;
    gBk[k] = h->gradb.p + (size_t)k * nb3;
  }
  double* G1[kMaxCotangents];
  double* lF0[kMaxCotangents];
  for (int q = 0; q < kg; ++q) {
    G1[q] = h->adj.p + (size_t)(2 * ncot + 2 * q) * S;
    lF0[q] = G1[q] + S;
  }
  double* Wfin = h->adj.p + (size_t)(2 * ncot + 2 * kg) * S;
  double* gsum = h->small.p;
  const size_t sb = S * sizeof(double);
  const cudaMemcpyKind in_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind out_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaMemsetAsync(h->gradb.p, 0, (size_t)ncot * nb3 * sizeof(double), h->stream);
  for (int k = 0; k < ncot && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(lam[k], lam_final + (size_t)k * S, sb, in_kind, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Wfin, h->W, sb, cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "step_vjp setup");
  const int nseg = (nsteps + every - 1) / every;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int s0 = seg * every;
    const int len = (nsteps - s0) < every ? (nsteps - s0) : every;
    // recompute the segment from its checkpoint once, recording every step's intermediate states
    // (a full tape already holds them: one segment of nsteps steps)
    if (!h->tape_full) {
      e = cudaMemcpyAsync(h->W, h->ckpt.p + (size_t)seg * S, sb, cudaMemcpyDeviceToDevice, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "restore checkpoint");
      for (int i = 0; i < len; ++i) {
        r = do_step(h, dt, h->snaps.p + (size_t)i * per_step);
        if (r) return r;
      }
    }
    for (int i = len - 1; i >= 0; --i)
      for (int k0 = 0; k0 < ncot; k0 += kg) {
        const int K = (ncot - k0) < kg ? (ncot - k0) : kg;
        r = step_vjp_group(h, dt, h->snaps.p + (size_t)i * per_step, &lam[k0], &tmp[k0], G1, lF0, &gBk[k0], K,
                           gsum);
        if (r) return r;
      }
  }
  e = cudaMemcpyAsync(h->W, Wfin, sb, cudaMemcpyDeviceToDevice, h->stream);
  for (int k = 0; k < ncot && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(lam_init + (size_t)k * S, lam[k], sb, out_kind, h->stream);
  if (e == cudaSuccess && grad_B)
    e = cudaMemcpyAsync(grad_B, h->gradb.p, (size_t)ncot * nb3 * sizeof(double), out_kind, h->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? QBE_OK : cuda_fail(h, e, "step_vjp output");
}

int qbe_step_vjp(qbe_handle* h, const double* lam_final, double* lam_init, double* grad_B, int on_device) {
  return qbe_step_vjp_n(h, 1, lam_final, lam_init, grad_B, on_device);
}

int qbe_observables(qbe_handle* h, const double* w, double* out, int on_device) {
  if (!h) return QBE_ERR_ARG;
  if (!out) return fail(h, QBE_ERR_ARG, "observables: null output");
  if (!w && !h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  DeviceGuard dg(h->g.device);
  if (h->small.ensure(small_elems(h)) != cudaSuccess || h->adj.ensure(5 * state_elems(h)) != cudaSuccess)
    return fail(h, QBE_ERR_ALLOC, "observables scratch");
  double* o2 = h->small.p + 4;
  double* part = h->small.p + 6 + (size_t)h->g.Nx * 3;
  const double* src = w ? w : h->W;
  cudaError_t e = cudaSuccess;
  if (w && !on_device) {
    e = cudaMemcpyAsync(h->adj.p, w, state_elems(h) * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    src = h->adj.p;
  }
  if (e == cudaSuccess) e = observables_launch(src, h->g.Nx, h->g.N, h->g.L, part, o2, h->stream, h->launches);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, o2, 2 * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? QBE_OK : cuda_fail(h, e, "observables");
}

int qbe_observables_vjp(qbe_handle* h, const double* gbar, double* lam, int on_device) {
  if (!h) return QBE_ERR_ARG;
  if (!gbar || !lam) return fail(h, QBE_ERR_ARG, "observables_vjp: null pointer");
  DeviceGuard dg(h->g.device);
  if (h->small.ensure(small_elems(h)) != cudaSuccess || h->adj.ensure(5 * state_elems(h)) != cudaSuccess)
    return fail(h, QBE_ERR_ALLOC, "observables scratch");
  double* g2 = h->small.p + 2;
  cudaError_t e = cudaMemcpyAsync(g2, gbar, 2 * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
  double* dst = on_device ? lam : h->adj.p;
  if (e == cudaSuccess) e = observables_vjp_launch(g2, h->g.Nx, h->g.N, h->g.L, dst, h->stream, h->launches);
  if (e == cudaSuccess && !on_device)
    e = cudaMemcpyAsync(lam, dst, state_elems(h) * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? QBE_OK : cuda_fail(h, e, "observables_vjp");
}

int qbe_entropy(qbe_handle* h, double* S, int on_device) {
  if (!h) return QBE_ERR_ARG;
  if (!S) return fail(h, QBE_ERR_ARG, "entropy: null output");
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  DeviceGuard dg(h->g.device);
  if (h->small.ensure(small_elems(h)) != cudaSuccess) return fail(h, QBE_ERR_ALLOC, "diagnostics scratch");
  double* dst = on_device ? S : h->small.p + 6;
  cudaError_t e = entropy_launch(h->W, h->g.Nx, h->g.N, h->g.L, dst, h->stream, h->launches);
  if (e == cudaSuccess && !on_device)
    e = cudaMemcpyAsync(S, dst, (size_t)h->g.Nx * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? QBE_OK : cuda_fail(h, e, "entropy");
}

int qbe_fd_fit_moments(const double* rho4, const double* mom, double energy, qbe_fermi_dirac* out) {
  if (!rho4 || !mom || !out || !std::isfinite(energy)) return QBE_ERR_ARG;
  fd_fit_from_moments(rho4, mom, energy, *out);
  return QBE_OK;
}

double qbe_dilog(double x) { return dilog(x); }

int qbe_fd_fit(qbe_handle* h, int global, qbe_fermi_dirac* out) {
  if (!h) return QBE_ERR_ARG;
  if (!out) return fail(h, QBE_ERR_ARG, "fd_fit: null output");
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  DeviceGuard dg(h->g.device);
  const int Nx = h->g.Nx;
  cudaError_t e = moments_launch(h->W, Nx, h->g.N, h->g.L, h->mom, h->stream, h->launches);
  std::vector<double> m((size_t)Nx * 7);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m.data(), h->mom, m.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "fd_fit moments");
  if (global) {
    double avg[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int j = 0; j < Nx; ++j)
      for (int k = 0; k < 7; ++k) avg[k] += m[(size_t)j * 7 + k];
    for (int k = 0; k < 7; ++k) avg[k] /= Nx;
    fd_fit_from_moments(avg, avg + 4, avg[6], out[0]);
    return QBE_OK;
  }
  for (int j = 0; j < Nx; ++j) fd_fit_from_moments(&m[(size_t)j * 7], &m[(size_t)j * 7 + 4], m[(size_t)j * 7 + 6], out[j]);
  return QBE_OK;
}

int qbe_relative_entropy(qbe_handle* h, const qbe_fermi_dirac* ref, int nref, double* rel, double* l1, int on_device) {
  if (!h) return QBE_ERR_ARG;
  const int Nx = h->g.Nx;
  if (!ref || !rel || (nref != 1 && nref != Nx)) return fail(h, QBE_ERR_ARG, "relative_entropy: bad arguments");
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  std::vector<FdDev> fd((size_t)nref);
  for (int k = 0; k < nref; ++k) {
    if (!ref[k].ok || !(ref[k].T > 0.0)) return fail(h, QBE_ERR_ARG, "relative_entropy: reference not fitted");
    fd[k].T = ref[k].T;
    fd[k].mu_up = ref[k].mu_up;
    fd[k].mu_dn = ref[k].mu_dn;
    for (int c = 0; c < 3; ++c) fd[k].bloch[c] = ref[k].bloch[c];
    fd[k].u[0] = ref[k].u[0];
    fd[k].u[1] = ref[k].u[1];
  }
  DeviceGuard dg(h->g.device);
  const size_t fd_doubles = (size_t)nref * sizeof(FdDev) / sizeof(double);
  if (h->adj.ensure(5 * state_elems(h)) != cudaSuccess || h->small.ensure(small_elems(h)) != cudaSuccess)
    return fail(h, QBE_ERR_ALLOC, "diagnostics scratch");
  // reference states and (host path) outputs staged in the adjoint scratch, which is idle here
  FdDev* dfd = reinterpret_cast<FdDev*>(h->adj.p);
  double* drel = on_device ? rel : h->adj.p + fd_doubles;
  double* dl1 = l1 ? (on_device ? l1 : h->adj.p + fd_doubles + Nx) : nullptr;
  cudaError_t e = cudaMemcpyAsync(dfd, fd.data(), fd.size() * sizeof(FdDev), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = relative_entropy_launch(h->W, Nx, h->g.N, h->g.L, dfd, nref, drel, dl1, h->stream, h->launches);
  if (e == cudaSuccess && !on_device)
    e = cudaMemcpyAsync(rel, drel, (size_t)Nx * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && !on_device && l1)
    e = cudaMemcpyAsync(l1, dl1, (size_t)Nx * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? QBE_OK : cuda_fail(h, e, "relative_entropy");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent simulations: one CUDA graph launch per split step.
// ---------------------------------------------------------------------------

struct qbe_batch {
  std::vector<qbe_handle*> sims;
  int device = 0;
  cudaStream_t stream = nullptr;          // launch stream (caller's)
  std::vector<cudaStream_t> side;         // one capture branch per simulation
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double graph_dt = 0.0;
  std::vector<double> tuned_ms;
  std::string err;
};

namespace {

// The I3 launch shape of a group of simulations of one padded size and precision (a single
// simulation is a group of one): for every launch variant, persistent grid (blocks per SM) and
// m-chunking, two waves of the group's work queue are timed on the simulations' current state
// (the per-cell terms are computed first, so the I3 inputs are those of the state).  The launch
// assigns unit u to block (cluster) u mod G, so its time is that of the busiest block: the sample's
// time divided by its busiest block's m-evaluations gives the cost of one m, and the candidate's
// time is that cost times the busiest block's m-evaluations over the whole queue (units of
// different members carry different numbers of m).  The fastest shape is set on every member;
// returns its predicted launch time in ms.
int tune_group(const std::vector<qbe_handle*>& hs, cudaStream_t s, double* best_ms, std::string& err) {
  if (hs.empty()) return QBE_ERR_ARG;
  qbe_handle* h0 = hs[0];
  const int n = h0->tab.n, prec = h0->cw.prec;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h0->g.device);
  std::vector<int> nc(hs.size()), nmc_max(hs.size());
  std::vector<const Tables*> tabs;
  std::vector<const CollisionWork*> cws;
  long long scratch = 0;
  for (size_t i = 0; i < hs.size(); ++i) {
    qbe_handle* h = hs[i];
    if (!h->has_state) { err = "autotune: a simulation has no state"; return QBE_ERR_STATE; }
    nc[i] = h->g.Nx < h->cw.nb ? h->g.Nx : h->cw.nb;
    if (collide_pre(h->tab, h->cw, h->W, nc[i], s, scratch) != cudaSuccess) {
      err = "autotune: per-cell terms failed";
      return QBE_ERR_CUDA;
    }
    // the largest m-chunking the partial-sum buffers hold (set at allocation, or by an earlier tuning)
    nmc_max[i] = (int)(h->cw.nparts_cap / ((size_t)h->cw.nb * h->tab.J));
    if (nmc_max[i] < 1) nmc_max[i] = 1;
    tabs.push_back(&h->tab);
    cws.push_back(&h->cw);
  }
  int nmc_top = 1;
  for (int v : nmc_max) nmc_top = v > nmc_top ? v : nmc_top;
  const int ws_blocks = (int)(h0->cw.ws_fields / 3);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    err = "autotune: event creation failed";
    return QBE_ERR_CUDA;
  }
  auto apply = [&](int v, int nmc) {
    for (size_t i = 0; i < hs.size(); ++i) {
      CollisionWork& cw = hs[i]->cw;
      const int M = hs[i]->tab.M;
      const int want = nmc < nmc_max[i] ? nmc : nmc_max[i];
      cw.i3_variant = v;
      cw.mch = (M + want - 1) / want;
      cw.nmc = (M + cw.mch - 1) / cw.mch;
    }
  };
  double best = 1e300;
  int bv = 0, bgrid = h0->cw.grid_i3, bnmc = h0->cw.nmc;
  int rc = QBE_OK;
  const int nv = i3_variants(n, prec);
  for (int v = 0; v < nv && rc == QBE_OK; ++v) {
    const int bpsv = i3_variant_bps(n, prec, v);
    for (int bps = 1; bps <= bpsv && rc == QBE_OK; ++bps) {
      int grid = bps * nsm;
      if (grid > ws_blocks) grid = ws_blocks;
      if (grid < 1) grid = 1;
      for (int nmc = nmc_top; nmc >= 1 && rc == QBE_OK; nmc = (nmc == 1 ? 0 : (nmc + 1) / 2)) {
        apply(v, nmc);
        // the queue's units in launch order, each with its number of m evaluations
        std::vector<int> mwork;
        for (size_t i = 0; i < hs.size(); ++i) {
          const CollisionWork& cw = hs[i]->cw;
          const int M = hs[i]->tab.M;
          for (long long u = 0; u < (long long)nc[i] * hs[i]->tab.J * cw.nmc; ++u) {
            const int mc = (int)(u % cw.nmc), m0 = mc * cw.mch;
            mwork.push_back((M - m0) < cw.mch ? (M - m0) : cw.mch);
          }
        }
        const long long total = (long long)mwork.size();
        const int conc_full = i3_concurrency(n, prec, v, grid, (int)(total < INT_MAX ? total : INT_MAX));
        const int sample = (int)(total < 2LL * conc_full ? total : 2LL * conc_full);
        const int conc_sample = i3_concurrency(n, prec, v, grid, sample);
        auto busiest = [&](long long units, int conc) {   // m evaluations of the busiest block
          std::vector<long long> load(conc, 0);
          for (long long u = 0; u < units; ++u) load[u % conc] += mwork[u];
          long long mx = 0;
          for (long long x : load) mx = x > mx ? x : mx;
          return mx;
        };
        long long lc = 0;
        cudaError_t e = i3_group(tabs.data(), cws.data(), nc.data(), (int)hs.size(), h0->cw.ws, grid, s, lc, sample);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess)
          e = i3_group(tabs.data(), cws.data(), nc.data(), (int)hs.size(), h0->cw.ws, grid, s, lc, sample);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
          err = std::string("autotune: timing run failed: ") + cudaGetErrorString(e);
          rc = QBE_ERR_CUDA;
          break;
        }
        const double per_m = ms / (double)busiest(sample, conc_sample);
        const double pred = per_m * (double)busiest(total, conc_full);
        if (pred < best) { best = pred; bv = v; bgrid = grid; bnmc = nmc; }
        if (nmc == 1) break;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != QBE_OK) return rc;
  apply(bv, bnmc);
  for (auto h : hs) h->cw.grid_i3 = bgrid;
  if (best_ms) *best_ms = best;
  return QBE_OK;
}

int bfail(qbe_batch* b, int code, const std::string& msg) {
  b->err = msg;
  return code;
}

void drop_graph(qbe_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// One split step of every simulation, captured in phases: per-simulation branches run the
// transport and the per-cell collision terms; between them, one I3 launch per padded-grid size and
// precision runs a work queue over the (simulation, cell, j, m-chunk) units of all simulations of
// that size (Sec. 3.2; the simulations are independent).  Per simulation the arithmetic is that of
// do_step: the same kernels on the same units.
// Groups of simulations sharing the I3 kernel (padded size and precision), at most kMaxI3Jobs each.
std::vector<std::vector<size_t>> i3_groups(const qbe_batch* b) {
  std::vector<std::vector<size_t>> groups;
  for (size_t i = 0; i < b->sims.size(); ++i) {
    const qbe_handle* h = b->sims[i];
    bool placed = false;
    for (auto& g : groups) {
      const qbe_handle* h0 = b->sims[g[0]];
      if (h0->tab.n == h->tab.n && h0->cw.prec == h->cw.prec && (int)g.size() < kMaxI3Jobs) {
        g.push_back(i);
        placed = true;
        break;
      }
    }
    if (!placed) groups.push_back({i});
  }
  return groups;
}

int batch_capture_step(qbe_batch* b, double dt, cudaStream_t origin) {
  const size_t ns = b->sims.size();
  auto branch = [&](size_t i) { return origin == b->side[i] ? origin : b->side[i]; };
  auto fork = [&]() {
    cudaEventRecord(b->fork, origin);
    for (size_t i = 0; i < ns; ++i)
      if (branch(i) != origin) cudaStreamWaitEvent(branch(i), b->fork, 0);
  };
  auto join = [&]() {
    for (size_t i = 0; i < ns; ++i)
      if (branch(i) != origin) {
        cudaEventRecord(b->join[i], branch(i));
        cudaStreamWaitEvent(origin, b->join[i], 0);
      }
  };
  const std::vector<std::vector<size_t>> groups = i3_groups(b);
  auto i3_all = [&](long long& launches) {
    for (auto& g : groups) {
      std::vector<const Tables*> tabs;
      std::vector<const CollisionWork*> cws;
      std::vector<int> nc;
      for (size_t i : g) {
        tabs.push_back(&b->sims[i]->tab);
        cws.push_back(&b->sims[i]->cw);
        nc.push_back(b->sims[i]->g.Nx);
      }
      const CollisionWork& c0 = b->sims[g[0]]->cw;
      const int cap = (int)(c0.ws_fields / 3);            // blocks the first simulation's scratch can hold
      const int grid = c0.grid_i3 < cap ? c0.grid_i3 : cap;   // the group's (tuned) persistent grid
      cudaError_t e = i3_group(tabs.data(), cws.data(), nc.data(), (int)g.size(), c0.ws, grid, origin, launches);
      if (e != cudaSuccess) return QBE_ERR_CUDA;
    }
    return QBE_OK;
  };
  std::vector<cudaStream_t> saved(ns);
  std::vector<bool> was_on(ns);
  for (size_t i = 0; i < ns; ++i) {
    qbe_handle* h = b->sims[i];
    saved[i] = h->stream;
    was_on[i] = h->timer.on;
    h->timer.on = false;
    h->stream = branch(i);
  }
  int r = QBE_OK;
  long long& launches = b->sims[0]->launches;
  // transport half step, first collision's per-cell terms
  fork();
  for (size_t i = 0; i < ns && !r; ++i) {
    qbe_handle* h = b->sims[i];
    r = do_advect(h, 0.5 * dt);
    if (!r && collide_pre(h->tab, h->cw, h->W, h->g.Nx, h->stream, h->launches) != cudaSuccess) r = QBE_ERR_CUDA;
  }
  join();
  if (!r) r = i3_all(launches);
  // first collision's assembly, RK stage 1, second collision's per-cell terms
  fork();
  for (size_t i = 0; i < ns && !r; ++i) {
    qbe_handle* h = b->sims[i];
    const int Nx = h->g.Nx, N = h->g.N;
    if (collide_post(h->tab, h->cw, h->Cb, Nx, h->stream, h->launches) != cudaSuccess ||
        rk_stage1(h->W, h->Cb, h->B, dt, h->F0, h->Wa, Nx, N, h->stream, h->launches, nullptr) != cudaSuccess ||
        collide_pre(h->tab, h->cw, h->Wa, Nx, h->stream, h->launches) != cudaSuccess)
      r = QBE_ERR_CUDA;
  }
  join();
  if (!r) r = i3_all(launches);
  // second collision's assembly, RK stage 2, transport half step
  fork();
  for (size_t i = 0; i < ns && !r; ++i) {
    qbe_handle* h = b->sims[i];
    const int Nx = h->g.Nx, N = h->g.N;
    if (collide_post(h->tab, h->cw, h->Cb, Nx, h->stream, h->launches) != cudaSuccess ||
        rk_stage2(h->W, h->F0, h->Cb, h->Wa, h->B, dt, h->W, Nx, N, h->stream, h->launches, nullptr) !=
            cudaSuccess)
      r = QBE_ERR_CUDA;
    if (!r) r = do_advect(h, 0.5 * dt);   // even number of state-buffer swaps over the step: ends in h->W
  }
  join();
  for (size_t i = 0; i < ns; ++i) {
    b->sims[i]->stream = saved[i];
    b->sims[i]->timer.on = was_on[i];
  }
  return r;
}

}  // namespace

extern "C" {

int qbe_batch_create(qbe_handle* const* sims, int nsims, qbe_batch** out) {
  if (!out) return QBE_ERR_ARG;
  *out = nullptr;
  if (!sims || nsims < 1) return QBE_ERR_ARG;
  for (int i = 0; i < nsims; ++i)
    if (!sims[i] || sims[i]->g.device != sims[0]->g.device) return QBE_ERR_ARG;
  for (int i = 0; i < nsims; ++i)
    for (int k = 0; k < i; ++k)
      if (sims[i] == sims[k]) return QBE_ERR_ARG;                  // each simulation once
  qbe_batch* b = new (std::nothrow) qbe_batch();
  if (!b) return QBE_ERR_ALLOC;
  b->sims.assign(sims, sims + nsims);
  b->device = sims[0]->g.device;
  b->tuned_ms.assign(nsims, 0.0);
  DeviceGuard dg(b->device);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < nsims; ++i) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    b->side.push_back(st);
    b->join.push_back(ev);
  }
  if (!ok) {
    qbe_batch_destroy(b);
    return QBE_ERR_CUDA;
  }
  *out = b;
  return QBE_OK;
}

void qbe_batch_destroy(qbe_batch* b) {
  if (!b) return;
  DeviceGuard dg(b->device);
  drop_graph(b);
  for (auto st : b->side) if (st) cudaStreamDestroy(st);
  for (auto ev : b->join) if (ev) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

const char* qbe_batch_last_error(const qbe_batch* b) { return b ? b->err.c_str() : "null batch"; }

int qbe_batch_set_stream(qbe_batch* b, void* stream) {
  if (!b) return QBE_ERR_ARG;
  b->stream = (cudaStream_t)stream;
  return QBE_OK;
}

int qbe_batch_autotune(qbe_batch* b) {
  if (!b) return QBE_ERR_ARG;
  DeviceGuard dg(b->device);
  drop_graph(b);                                       // launch shapes are baked into the graph
  cudaStream_t s = b->stream ? b->stream : b->side[0];
  std::vector<std::vector<size_t>> groups = i3_groups(b);
  for (auto& g : groups) {
    std::vector<qbe_handle*> hs;
    for (size_t i : g) hs.push_back(b->sims[i]);
    double ms = 0.0;
    std::string err;
    const int rc = tune_group(hs, s, &ms, err);
    if (rc != QBE_OK) return bfail(b, rc, err);
    for (size_t i : g) b->tuned_ms[i] = ms;
  }
  return QBE_OK;
}

int qbe_batch_tuned_shape(const qbe_batch* b, int sim, int* i3_grid, int* m_chunks, double* ms) {
  if (!b || sim < 0 || sim >= (int)b->sims.size()) return QBE_ERR_ARG;
  if (i3_grid) *i3_grid = b->sims[sim]->cw.grid_i3;
  if (m_chunks) *m_chunks = b->sims[sim]->cw.nmc;
  if (ms) *ms = b->tuned_ms[sim];
  return QBE_OK;
}

int qbe_batch_step(qbe_batch* b, double dt, int nsteps) {
  if (!b) return QBE_ERR_ARG;
  if (!std::isfinite(dt) || nsteps < 0) return bfail(b, QBE_ERR_ARG, "bad dt or nsteps");
  for (auto h : b->sims)
    if (!h->has_state) return bfail(b, QBE_ERR_STATE, "a simulation has no state");
  for (auto h : b->sims) h->tape_valid = false;
  DeviceGuard dg(b->device);
  if (!b->exec || b->graph_dt != dt) {
    drop_graph(b);
    cudaError_t e = cudaStreamBeginCapture(b->stream ? b->stream : b->side[0], cudaStreamCaptureModeThreadLocal);
    // the legacy default stream cannot be captured: capture on the first branch stream instead
    cudaStream_t origin = b->stream ? b->stream : b->side[0];
    if (e != cudaSuccess) return bfail(b, QBE_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    int r = batch_capture_step(b, dt, origin);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(origin, &g);
    if (r != QBE_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bfail(b, r != QBE_OK ? r : QBE_ERR_CUDA, "capture of the batched step failed");
    }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
      drop_graph(b);
      return bfail(b, QBE_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    }
    b->graph_dt = dt;
  }
  cudaStream_t launch = b->stream ? b->stream : b->side[0];
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = cudaGraphLaunch(b->exec, launch);
    if (e != cudaSuccess) return bfail(b, QBE_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  }
  if (!b->stream) {
    cudaError_t e = cudaStreamSynchronize(launch);
    if (e != cudaSuccess) return bfail(b, QBE_ERR_CUDA, std::string("batch step: ") + cudaGetErrorString(e));
  }
  return QBE_OK;
}

}  // extern "C"
