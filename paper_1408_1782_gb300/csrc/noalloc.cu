// qbe_collide_noalloc: the collision operator C[W] without any memory allocation.
//
// Some callers cannot allocate device memory when they call into a library:
// code hosted by a framework that owns the GPU's memory budget and forbids
// allocations, latency-critical paths where cudaMalloc's implicit device
// synchronisation is not acceptable, or deployments that must reserve every
// byte when the library is loaded.  For them this entry point keeps its kernel
// tables and all of its collision scratch in one statically sized device array
// (below), which every GPU that loads the library holds until the process
// exits.  The caller passes only the input and output device buffers.
//
// The work itself is the same as qbe_collide: the same kernels, launched with
// their tables and scratch pointing into the static array.
#include <cmath>

#include "fft.cuh"
#include "internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;   // 64 MiB, see QBE_NOALLOC_SCRATCH_BYTES in qbe.h
constexpr int kMaxDevices = 64;

// The scratch: quadrature tables followed by the collision workspace.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceSlot {
  unsigned char* base = nullptr;  // the array's device address on this device, as last resolved
  // grid whose tables the array currently holds (as far as the host can know)
  bool tables = false;
  // a call was recorded into a stream capture: the array's contents then depend on when that
  // graph is replayed, so every later call rebuilds the tables
  bool captured = false;
  int N = 0, J = 0, M = 0;
  double L = 0, R = 0;
};
static DeviceSlot g_slots[kMaxDevices];

constexpr double kPi = 3.14159265358979323846;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t tw, phip, Ktab, psi, psip, phase, gl, tables_end;
};

Layout layout_for(int n, int J, int M) {
  const size_t P = (size_t)n * n;
  Layout l{};
  size_t o = 0;
  l.tw = o;    o = align256(o + (size_t)n * sizeof(double2));
  l.phip = o;  o = align256(o + (size_t)J * P * sizeof(double));
  l.Ktab = o;  o = align256(o + (size_t)J * P * sizeof(double));
  l.psi = o;   o = align256(o + (size_t)J * P * sizeof(double));
  l.psip = o;  o = align256(o + (size_t)J * P * sizeof(double));
  l.phase = o; o = align256(o + (size_t)J * M * 2 * n * sizeof(double2));
  l.gl = o;    o = align256(o + (size_t)2 * M * sizeof(double));
  l.tables_end = o;
  return l;
}

template <int n> struct SplitOf { static constexpr int A = qbe::Split<n>::A, B = qbe::Split<n>::B; };

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the Legendre recurrence), one thread per node.
__global__ void k_noalloc_gauss(double* gl, int M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double z = cos(kPi * (i + 0.75) / (M + 0.5));
  double dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = 0.0;
    for (int k = 1; k <= M; ++k) {
      const double p2 = p1;
      p1 = p0;
      p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
    }
    dp = M * (z * p0 - p1) / (z * z - 1.0);
    const double dz = p0 / dp;
    z -= dz;
    if (fabs(dz) < 1e-16) break;
  }
  double p0 = 1.0, p1 = 0.0;
  for (int k = 1; k <= M; ++k) {
    const double p2 = p1;
    p1 = p0;
    p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
  }
  dp = M * (z * p0 - p1) / (z * z - 1.0);
  gl[i] = -z;                                   // ascending nodes
  gl[M + i] = 2.0 / ((1.0 - z * z) * dp * dp);
}

__device__ double phi_R(double s, double L, double R) {
  if (s == 0.0) return 0.0;
  const double t = sin(kPi * s * R / (2.0 * L));
  return (2.0 * L / (kPi * s)) * t * t;
}
__device__ double psi_R(double s, double L, double R) {
  if (s == 0.0) return 2.0 * R;
  return (2.0 * L / (kPi * s)) * sin(kPi * R * s / L);
}

// Tables of Sec. 3.2 in the permuted spectral order (same content as the
// host-built tables of qbe_create), written straight into the static array.
template <int n>
__global__ void k_noalloc_tables(unsigned char* base, Layout lay, int J, int M, double L, double R) {
  constexpr int A = SplitOf<n>::A, B = SplitOf<n>::B, N = n / 2;
  const size_t P = (size_t)n * n;
  double2* tw = (double2*)(base + lay.tw);
  double* phip = (double*)(base + lay.phip);
  double* Ktab = (double*)(base + lay.Ktab);
  double* psi = (double*)(base + lay.psi);
  double* psip = (double*)(base + lay.psip);
  double2* phase = (double2*)(base + lay.phase);
  const double* gl = (const double*)(base + lay.gl);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  auto sig = [&](int pos) {
    const int k = pos / B + A * (pos % B);
    return (double)(k < N ? k : k - n);
  };
  for (size_t i = t0; i < (size_t)n; i += stride) {
    const int t2 = (int)i / A, k1 = (int)i % A;
    double s, c;
    sincospi(-2.0 * (double)(t2 * k1) / n, &s, &c);
    tw[i] = make_double2(c, s);
  }
  for (size_t i = t0; i < (size_t)J * P; i += stride) {
    const int j = (int)(i / P);
    const size_t o = i % P;
    const double sx = sig((int)(o / n)), sy = sig((int)(o % n));
    double sj, cj, sp, cp;
    sincospi((double)j / J, &sj, &cj);
    sincospi((j + 0.5) / J, &sp, &cp);
    phip[i] = phi_R(sx * cp + sy * sp, L, R);
    psi[i] = psi_R(sx * cj + sy * sj, L, R);
    psip[i] = psi_R(-sx * sj + sy * cj, L, R) / (double)P;
    double acc = 0.0;                                     // K_j'(sigma) with j' = j
    for (int jj = 0; jj < J; ++jj) {
      double s2, c2;
      sincospi((double)jj / J, &s2, &c2);
      const double dot = c2 * cp + s2 * sp;
      acc += -(2.0 * kPi / J) * (2.0 * kPi / J) / dot * phi_R(sx * c2 + sy * s2, L, R);
    }
    Ktab[i] = acc / (double)P;
  }
  for (size_t i = t0; i < (size_t)J * M * 2 * n; i += stride) {
    const int pos = (int)(i % n);
    const int axis = (int)((i / n) % 2);
    const int jm = (int)(i / (2 * n));
    const int j = jm / M, m = jm % M;
    const double rho = R * gl[m], wm = R * gl[M + m];
    double sj, cj;
    sincospi((double)j / J, &sj, &cj);
    const double a = kPi * rho * (axis == 0 ? cj : sj) / L * sig(pos);
    double sa, ca;
    sincos(a, &sa, &ca);
    const double sq = axis == 0 ? sqrt(kPi / J * wm) : 1.0;
    phase[i] = make_double2(sq * ca, sq * sa);
  }
}

template <int n>
cudaError_t build_tables_dev(unsigned char* base, const Layout& lay, int J, int M, double L, double R,
                             cudaStream_t s) {
  k_noalloc_gauss<<<(M + 63) / 64, 64, 0, s>>>((double*)(base + lay.gl), M);
  k_noalloc_tables<n><<<152 * 4, 256, 0, s>>>(base, lay, J, M, L, R);
  return cudaGetLastError();
}

}  // namespace

extern "C" int qbe_collide_noalloc(const qbe_grid* g, const double* w, double* c, int ncells, void* stream) {
  if (!g || !w || !c || ncells < 1) return QBE_ERR_ARG;
  const bool n_ok = g->N == 8 || g->N == 16 || g->N == 32 || g->N == 64;
  if (!n_ok || g->J < 2 || g->J > 64 || (g->J % 2) != 0 || g->M < 1 || g->M > 64 || !(g->L > 0) ||
      !(g->R > 0) || !std::isfinite(g->L) || !std::isfinite(g->R))
    return QBE_ERR_ARG;
  if (g->precision != 0) return QBE_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QBE_ERR_CUDA;
  if (g->device != dev) return QBE_ERR_ARG;          // runs on the caller's current device
  const int n = 2 * g->N;
  const Layout lay = layout_for(n, g->J, g->M);
  // I3 persistent grid: at most one block per SM, and per-block scratch of three fields
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QBE_ERR_CUDA;
  const size_t P = (size_t)n * n;
  auto need = [&](int nb, int grid) {     // mirrors the carving of the workspace below
    size_t wsf = 6 * (size_t)nb;
    if (3 * (size_t)grid > wsf) wsf = 3 * (size_t)grid;
    return lay.tables_end + align256((size_t)nb * 4 * P * sizeof(double2)) +
           2 * align256((size_t)nb * 2 * P * sizeof(double2)) + align256((size_t)nb * P * sizeof(double)) +
           align256((size_t)nb * 2 * P * sizeof(double2)) + align256((size_t)nb * g->J * 2 * P * sizeof(double2)) +
           align256(wsf * P * sizeof(double2));
  };
  // largest batch (<= ncells) and I3 grid that fit
  int nb = ncells < (1 << 20) ? ncells : (1 << 20), grid = 0;
  for (;;) {
    grid = (long long)nb * g->J < nsm ? nb * g->J : nsm;
    if (need(nb, grid) <= kScratchBytes || nb == 1) break;
    nb = nb / 2 > 0 ? nb / 2 : 1;
  }
  while (need(nb, grid) > kScratchBytes && grid > 1) grid /= 2;
  if (need(nb, grid) > kScratchBytes) return QBE_ERR_ARG;   // grid too large for the static scratch

  DeviceSlot& slot = g_slots[dev];
  // Resolved on every call (it allocates nothing): a new context may place the array elsewhere.
  void* sym = nullptr;
  if (cudaGetSymbolAddress(&sym, g_noalloc_scratch) != cudaSuccess || !sym) return QBE_ERR_CUDA;
  if ((unsigned char*)sym != slot.base) {
    slot.base = (unsigned char*)sym;
    slot.tables = false;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return QBE_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) slot.captured = true;
  unsigned char* base = slot.base;
  if (slot.captured || !slot.tables || slot.N != g->N || slot.J != g->J || slot.M != g->M || slot.L != g->L ||
      slot.R != g->R) {
    slot.tables = false;          // the build below overwrites the table area
    cudaError_t e;
    switch (n) {
      case 16: e = build_tables_dev<16>(base, lay, g->J, g->M, g->L, g->R, s); break;
      case 32: e = build_tables_dev<32>(base, lay, g->J, g->M, g->L, g->R, s); break;
      case 64: e = build_tables_dev<64>(base, lay, g->J, g->M, g->L, g->R, s); break;
      default: e = build_tables_dev<128>(base, lay, g->J, g->M, g->L, g->R, s); break;
    }
    if (e != cudaSuccess) return QBE_ERR_CUDA;
    slot.tables = true;
    slot.N = g->N; slot.J = g->J; slot.M = g->M; slot.L = g->L; slot.R = g->R;
  }
  qbe::Tables t;
  t.N = g->N; t.n = n; t.J = g->J; t.M = g->M; t.L = g->L; t.R = g->R;
  t.tw = (double2*)(base + lay.tw);
  t.phip = (double*)(base + lay.phip);
  t.Ktab = (double*)(base + lay.Ktab);
  t.psi = (double*)(base + lay.psi);
  t.psip_s = (double*)(base + lay.psip);
  t.phase = (double2*)(base + lay.phase);
  qbe::CollisionWork cw;
  cw.nb = nb; cw.nmc = 1; cw.mch = g->M; cw.grid_i3 = grid; cw.nparts_cap = (size_t)nb * g->J;
  unsigned char* wp = base + lay.tables_end;
  auto take = [&](size_t bytes) { unsigned char* r = wp; wp += align256(bytes); return r; };
  cw.what = (double2*)take((size_t)nb * 4 * P * sizeof(double2));
  cw.wfine = (double2*)take((size_t)nb * 2 * P * sizeof(double2));
  cw.Dacc = (double2*)take((size_t)nb * 2 * P * sizeof(double2));
  cw.K2acc = (double*)take((size_t)nb * P * sizeof(double));
  cw.K4acc = (double2*)take((size_t)nb * 2 * P * sizeof(double2));
  cw.K3part = (double2*)take((size_t)nb * g->J * 2 * P * sizeof(double2));
  size_t wsf = 6 * (size_t)nb;
  if (3 * (size_t)grid > wsf) wsf = 3 * (size_t)grid;
  cw.ws = (double2*)take(wsf * P * sizeof(double2));
  cw.ws_fields = wsf;
  cw.ws_slots = nb > grid ? nb : grid;
  long long launches = 0;
  const size_t per = (size_t)4 * g->N * g->N;
  for (int c0 = 0; c0 < ncells; c0 += nb) {
    const int nc = (ncells - c0) < nb ? (ncells - c0) : nb;
    cudaError_t e = qbe::collide_batch(t, cw, w + (size_t)c0 * per, c + (size_t)c0 * per, nc, s, launches, nullptr);
    if (e != cudaSuccess) return QBE_ERR_CUDA;
  }
  return QBE_OK;
}
