// C ABI (include/qbe.h): solver handle, argument checks, host/device copies
// and the split time step of Sec. 4.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace qbe;

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
};

namespace {

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

int do_advect(qbe_handle* h, double tau) {
  const int Nx = h->g.Nx, N = h->g.N;
  const int s = transport_substeps(tau, 1.0 / Nx, h->g.L);
  for (int k = 0; k < s; ++k) {
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

int do_rk2(qbe_handle* h, double dt) {
  const int Nx = h->g.Nx, N = h->g.N;
  int r = do_collide_dev(h, h->W, h->Cb, Nx);
  if (r) return r;
  cudaError_t e = rk_stage1(h->W, h->Cb, h->B, dt, h->F0, h->Wa, Nx, N, h->stream, h->launches, &h->timer);
  if (e != cudaSuccess) return cuda_fail(h, e, "rk stage 1");
  r = do_collide_dev(h, h->Wa, h->Cb, Nx);
  if (r) return r;
  e = rk_stage2(h->W, h->F0, h->Cb, h->Wa, h->B, dt, h->W, Nx, N, h->stream, h->launches, &h->timer);
  if (e != cudaSuccess) return cuda_fail(h, e, "rk stage 2");
  return QBE_OK;
}

bool valid_fd(const qbe_fd* f) {
  return f && std::isfinite(f->beta) && f->beta > 0 && std::isfinite(f->mu_up) && std::isfinite(f->mu_dn);
}

}  // namespace

extern "C" {

int qbe_create(const qbe_grid* g, qbe_handle** out) {
  if (!out) return QBE_ERR_ARG;
  *out = nullptr;
  if (!g) return QBE_ERR_ARG;
  const bool n_ok = g->N == 8 || g->N == 16 || g->N == 32 || g->N == 64 || g->N == 128;
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
  cudaError_t e = cudaMemcpyAsync(h->B, B, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? QBE_OK : cuda_fail(h, e, "set_bfield");
}

int qbe_set_state(qbe_handle* h, const double* w, int on_device) {
  if (!h || !w) return h ? fail(h, QBE_ERR_ARG, "null state") : QBE_ERR_ARG;
  DeviceGuard dg(h->g.device);
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
  return do_advect(h, tau);
}

int qbe_collide_rk2(qbe_handle* h, double dt) {
  if (!h) return QBE_ERR_ARG;
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  if (!std::isfinite(dt)) return fail(h, QBE_ERR_ARG, "dt not finite");
  DeviceGuard dg(h->g.device);
  return do_rk2(h, dt);
}

int qbe_step(qbe_handle* h, double dt, int nsteps) {
  if (!h) return QBE_ERR_ARG;
  if (!h->has_state) return fail(h, QBE_ERR_STATE, "no state set");
  if (!std::isfinite(dt) || nsteps < 0) return fail(h, QBE_ERR_ARG, "bad dt or nsteps");
  DeviceGuard dg(h->g.device);
  for (int s = 0; s < nsteps; ++s) {
    int r = do_advect(h, 0.5 * dt);
    if (!r) r = do_rk2(h, dt);
    if (!r) r = do_advect(h, 0.5 * dt);
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

}  // extern "C"
