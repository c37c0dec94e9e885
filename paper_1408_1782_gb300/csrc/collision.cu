// Size dispatch and workspace allocation of the collision operator; the
// kernels are instantiated per fine-grid size in collision_n*.cu.
#include "internal.h"

namespace qbe {

cudaError_t collide_batch(const Tables& t, CollisionWork& cw, const double* w, double* c, int ncells,
                          cudaStream_t s, long long& launches, KernelTimer* tm) {
  if (cw.prec == 1) {
    switch (t.n) {
      case 16: return collide_batch_n<16, float>(t, cw, w, c, ncells, s, launches, tm);
      case 32: return collide_batch_n<32, float>(t, cw, w, c, ncells, s, launches, tm);
      case 64: return collide_batch_n<64, float>(t, cw, w, c, ncells, s, launches, tm);
      case 128: return collide_batch_n<128, float>(t, cw, w, c, ncells, s, launches, tm);
      case 256: return collide_batch_n<256, float>(t, cw, w, c, ncells, s, launches, tm);
    case 96: return collide_batch_n<96, float>(t, cw, w, c, ncells, s, launches, tm);
    case 192: return collide_batch_n<192, float>(t, cw, w, c, ncells, s, launches, tm);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (t.n) {
    case 16: return collide_batch_n<16, double>(t, cw, w, c, ncells, s, launches, tm);
    case 32: return collide_batch_n<32, double>(t, cw, w, c, ncells, s, launches, tm);
    case 64: return collide_batch_n<64, double>(t, cw, w, c, ncells, s, launches, tm);
    case 128: return collide_batch_n<128, double>(t, cw, w, c, ncells, s, launches, tm);
    case 256: return collide_batch_n<256, double>(t, cw, w, c, ncells, s, launches, tm);
    case 96: return collide_batch_n<96, double>(t, cw, w, c, ncells, s, launches, tm);
    case 192: return collide_batch_n<192, double>(t, cw, w, c, ncells, s, launches, tm);
    default: return cudaErrorInvalidValue;
  }
}


#define QBE_SIZE_SWITCH(CALL, FAIL)                                   \
  if (prec == 1) {                                                    \
    switch (n) {                                                      \
      case 16: return CALL(16, float); case 32: return CALL(32, float); \
      case 64: return CALL(64, float); case 128: return CALL(128, float); \
      case 256: return CALL(256, float); case 96: return CALL(96, float); \
      case 192: return CALL(192, float); default: return FAIL;          \
    }                                                                 \
  }                                                                   \
  switch (n) {                                                        \
    case 16: return CALL(16, double); case 32: return CALL(32, double); \
    case 64: return CALL(64, double); case 128: return CALL(128, double); \
    case 256: return CALL(256, double); case 96: return CALL(96, double); \
    case 192: return CALL(192, double); default: return FAIL;           \
  }

int i3_variants(int n, int prec) {
#define QBE_CALL(nn, T) i3_variant_count<nn, T>()
  QBE_SIZE_SWITCH(QBE_CALL, 0)
#undef QBE_CALL
}

int i3_default(int n, int prec) {
#define QBE_CALL(nn, T) i3_default_variant<nn, T>()
  QBE_SIZE_SWITCH(QBE_CALL, 0)
#undef QBE_CALL
}

int i3_variant_bps(int n, int prec, int variant) {
#define QBE_CALL(nn, T) i3_blocks_per_sm<nn, T>(variant)
  QBE_SIZE_SWITCH(QBE_CALL, 1)
#undef QBE_CALL
}

int i3_concurrency(int n, int prec, int variant, int grid, int total) {
#define QBE_CALL(nn, T) i3_variant_concurrency<nn, T>(variant, grid, total)
  QBE_SIZE_SWITCH(QBE_CALL, 1)
#undef QBE_CALL
}

const char* i3_variant_desc(int n, int prec, int variant) {
#define QBE_CALL(nn, T) i3_variant_name<nn, T>(variant)
  QBE_SIZE_SWITCH(QBE_CALL, nullptr)
#undef QBE_CALL
}

// Angle chunks per cell of the I1 and I2/I4 kernels: enough (cell, chunk) blocks to fill about one
// wave of the device (3 resident 256-thread blocks per SM), at most J/2 (the I2/I4 angle pairs).
int per_cell_chunks(int nb, int J) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int cap = 3 * (nsm > 0 ? nsm : 1);
  int nch = (cap + nb / 2) / (nb > 0 ? nb : 1);
  if (nch > J / 2) nch = J / 2;
  return nch < 1 ? 1 : nch;
}

cudaError_t alloc_collision_work(const Tables& t, int nb, CollisionWork& cw, int prec) {
  const size_t P = (size_t)t.n * t.n;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int nv = i3_variants(t.n, prec);
  if (nv < 1) return cudaErrorInvalidValue;
  const int v0 = i3_default(t.n, prec);
  const int bps = i3_variant_bps(t.n, prec, v0);
  int bps_max = bps;
  for (int v = 0; v < nv; ++v) {
    const int b = i3_variant_bps(t.n, prec, v);
    if (b > bps_max) bps_max = b;
  }
  cw.prec = prec;
  cw.nb = nb;
  cw.i3_variant = v0;
  cw.grid_i3 = nsm * bps;
  cw.grid_max = nsm * bps_max;
  // enough (cell, j, m-chunk) units for about 8 waves of the persistent grid
  int nmc = (8 * cw.grid_i3 + nb * t.J - 1) / (nb * t.J);
  if (nmc < 1) nmc = 1;
  if (nmc > t.M) nmc = t.M;
  cw.mch = (t.M + nmc - 1) / nmc;
  cw.nmc = (t.M + cw.mch - 1) / cw.mch;
  const size_t nparts = (size_t)nb * t.J * cw.nmc;
  cw.nparts_cap = nparts;
  cw.ws_slots = nb > cw.grid_i3 ? nb : cw.grid_i3;
  cw.nch = per_cell_chunks(nb, t.J);
  size_t ws_fields = 6 * (size_t)nb;
  if (5 * (size_t)nb * cw.nch > ws_fields) ws_fields = 5 * (size_t)nb * cw.nch;   // k_i24: 5 fields per block
  if (3 * (size_t)cw.grid_max > ws_fields) ws_fields = 3 * (size_t)cw.grid_max;
  cw.ws_fields = ws_fields;
  const size_t N = t.N;
  const size_t cz = prec == 1 ? sizeof(float2) : sizeof(double2);   // complex element
  const size_t rz = cz / 2;                                           // real element
  cudaError_t e;
#define QBE_ALLOC(ptr, bytes) \
  if ((e = cudaMalloc((void**)&(ptr), (bytes))) != cudaSuccess) { free_collision_work(cw); return e; }
  QBE_ALLOC(cw.what, (size_t)nb * 4 * P * cz);
  QBE_ALLOC(cw.wfine, (size_t)nb * 2 * P * cz);
  QBE_ALLOC(cw.Dacc, (size_t)nb * 2 * P * cz);
  QBE_ALLOC(cw.K2acc, (size_t)nb * P * rz);
  QBE_ALLOC(cw.K4acc, (size_t)nb * 2 * P * cz);
  if (cw.nch > 1) {
    QBE_ALLOC(cw.Dpart, (size_t)nb * cw.nch * 2 * P * cz);
    QBE_ALLOC(cw.K2part, (size_t)nb * cw.nch * P * rz);
    QBE_ALLOC(cw.K4part, (size_t)nb * cw.nch * 2 * P * cz);
  }
  QBE_ALLOC(cw.K3part, nparts * 2 * P * cz);
  QBE_ALLOC(cw.ws, ws_fields * P * cz);
  QBE_ALLOC(cw.cbuf, (size_t)nb * 4 * N * N * sizeof(double));
  QBE_ALLOC(cw.wbuf, (size_t)nb * 4 * N * N * sizeof(double));
#undef QBE_ALLOC
  return cudaSuccess;
}

void free_collision_work(CollisionWork& cw) {
  cudaFree(cw.what); cudaFree(cw.wfine); cudaFree(cw.Dacc); cudaFree(cw.K2acc); cudaFree(cw.K4acc);
  cudaFree(cw.Dpart); cudaFree(cw.K2part); cudaFree(cw.K4part);
  cudaFree(cw.K3part); cudaFree(cw.ws); cudaFree(cw.cbuf); cudaFree(cw.wbuf);
  cw = CollisionWork();
}


#define QBE_VJP_SWITCH(T, CALL)                       \
  switch (t.n) {                                      \
    case 16: return CALL(16, T);                      \
    case 32: return CALL(32, T);                      \
    case 64: return CALL(64, T);                      \
    case 128: return CALL(128, T);                    \
    case 256: return CALL(256, T);                    \
    case 96: return CALL(96, T);                      \
    case 192: return CALL(192, T);                    \
    default: break;                                   \
  }

namespace {
int vjp_bps(const Tables& t, int prec) {
#define QBE_BPS(n, T) i3_vjp_blocks_per_sm<n, T>()
  if (prec == 1) {
    QBE_VJP_SWITCH(float, QBE_BPS)
  } else {
    QBE_VJP_SWITCH(double, QBE_BPS)
  }
#undef QBE_BPS
  return 0;
}
}  // namespace

cudaError_t collide_pre(const Tables& t, CollisionWork& cw, const double* w, int ncells, cudaStream_t s,
                        long long& launches) {
#define QBE_PRE_CALL(n, T) collide_pre_n<n, T>(t, cw, w, ncells, s, launches, nullptr)
  if (cw.prec == 1) {
    QBE_VJP_SWITCH(float, QBE_PRE_CALL)
  } else {
    QBE_VJP_SWITCH(double, QBE_PRE_CALL)
  }
#undef QBE_PRE_CALL
  return cudaErrorInvalidValue;
}

cudaError_t collide_post(const Tables& t, CollisionWork& cw, double* c, int ncells, cudaStream_t s,
                         long long& launches) {
#define QBE_POST_CALL(n, T) collide_post_n<n, T>(t, cw, c, ncells, s, launches, nullptr)
  if (cw.prec == 1) {
    QBE_VJP_SWITCH(float, QBE_POST_CALL)
  } else {
    QBE_VJP_SWITCH(double, QBE_POST_CALL)
  }
#undef QBE_POST_CALL
  return cudaErrorInvalidValue;
}

cudaError_t i3_group(const Tables* const* tabs, const CollisionWork* const* cws, const int* ncells, int njobs,
                     void* ws, int grid, cudaStream_t s, long long& launches, int max_units) {
  if (njobs < 1) return cudaErrorInvalidValue;
  const Tables& t = *tabs[0];
  for (int k = 1; k < njobs; ++k)
    if (tabs[k]->n != t.n || cws[k]->prec != cws[0]->prec) return cudaErrorInvalidValue;
#define QBE_GROUP_CALL(n, T) i3_group_n<n, T>(tabs, cws, ncells, njobs, ws, grid, s, launches, max_units)
  if (cws[0]->prec == 1) {
    QBE_VJP_SWITCH(float, QBE_GROUP_CALL)
  } else {
    QBE_VJP_SWITCH(double, QBE_GROUP_CALL)
  }
#undef QBE_GROUP_CALL
  return cudaErrorInvalidValue;
}

cudaError_t collide_vjp(const Tables& t, CollisionWork& cw, VjpWork& vw, const double* w, const double* const* lam,
                        double* const* grad, int K, int ncells, int accumulate, cudaStream_t s, long long& launches,
                        KernelTimer* tm) {
  if (ncells > cw.nb || ncells > vw.nb || cw.prec != vw.prec || K < 1 || K > vw.kcap) return cudaErrorInvalidValue;
#define QBE_VJP_CALL(n, T) collide_vjp_n<n, T>(t, cw, vw, w, lam, grad, K, ncells, accumulate, s, launches, tm)
  if (vw.prec == 1) {
    QBE_VJP_SWITCH(float, QBE_VJP_CALL)
  } else {
    QBE_VJP_SWITCH(double, QBE_VJP_CALL)
  }
#undef QBE_VJP_CALL
  return cudaErrorInvalidValue;
}

// Cotangents one collision product should carry.  The staged transpose kernels (FP64, and FP32 on
// grids above 128 points) are bound by their transforms, so sharing the state's Psi' convolutions saves
// about a quarter of the work per product at two cotangents (measured: FP64, N = 64, 16 cells, 847 ms
// per single launch against 1297 ms for two).  The FP32 shared-memory kernels run their transforms on
// chip: the element-pass kernel is bound by its global accumulators, and every further cotangent adds
// three fields of them per block, which pushes the working set out of L2 (two cotangents: 685 ms
// against 2 x 333 ms, L2 hit rate 85 % -> 68 %); the warp-local kernel (128 points) holds one
// cotangent's shifted-back sums in registers, which leave no room for a second.  Both take one
// cotangent at a time.
int vjp_cotangent_group(const Tables& t, int prec) { return (prec == 1 && t.n <= 128) ? 1 : kMaxCotangents; }

int vjp_i3_variants(int n, int prec) { return (prec == 1 && n == 128) ? 2 : 1; }

cudaError_t alloc_vjp_work(const Tables& t, int nb, VjpWork& vw, int prec, int kcap) {
  const size_t P = (size_t)t.n * t.n;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int bps = vjp_bps(t, prec);
  if (bps < 1) return cudaErrorInvalidValue;
  if (kcap < 1 || kcap > kMaxCotangents) return cudaErrorInvalidValue;
  vw.prec = prec;
  vw.nb = nb;
  vw.kcap = kcap;
  vw.grid = nsm * bps;
  // about 4 waves of (cell, j, m-chunk) units
  int nmc = (4 * vw.grid + nb * t.J - 1) / (nb * t.J);
  if (nmc < 1) nmc = 1;
  if (nmc > t.M) nmc = t.M;
  vw.mch = (t.M + nmc - 1) / nmc;
  vw.nmc = (t.M + vw.mch - 1) / vw.mch;
  const size_t nparts = (size_t)nb * t.J * vw.nmc;
  // per-cell kernels: 7 fields per cell; I3 transpose: 7 + 2 K fields per block (staged form)
  size_t ws_fields = 7 * (size_t)nb;
  if ((7 + 2 * (size_t)kcap) * vw.grid > ws_fields) ws_fields = (7 + 2 * (size_t)kcap) * vw.grid;
  // per (cell, angle chunk) block: the recomputed forward's I2/I4 kernel 5 fields, the I2/I4
  // transpose 7
  const size_t nch = (size_t)per_cell_chunks(nb, t.J);
  if (7 * (size_t)nb * nch > ws_fields) ws_fields = 7 * (size_t)nb * nch;
  const size_t kc = (size_t)kcap;
  const size_t cz = prec == 1 ? sizeof(float2) : sizeof(double2);
  const size_t rz = cz / 2;
  cudaError_t e;
#define QBE_ALLOC(ptr, bytes) \
  if ((e = cudaMalloc((void**)&(ptr), (bytes))) != cudaSuccess) { free_vjp_work(vw); return e; }
  QBE_ALLOC(vw.nu, kc * nb * 2 * P * cz);
  QBE_ALLOC(vw.nuf, kc * nb * P * rz);
  QBE_ALLOC(vw.muD, kc * nb * 2 * P * cz);
  QBE_ALLOC(vw.muK2, kc * nb * P * rz);
  QBE_ALLOC(vw.mu4, kc * nb * 2 * P * cz);
  QBE_ALLOC(vw.mu3, kc * nb * 2 * P * cz);
  QBE_ALLOC(vw.part_r, kc * nparts * 2 * P * cz);
  const size_t Q = (size_t)(t.n / 2 - 1) * (t.n / 2 - 1);   // kept frequencies (Fourier-space partials)
  QBE_ALLOC(vw.part_s, kc * nparts * 2 * Q * cz);
  QBE_ALLOC(vw.ws, ws_fields * P * cz);
#undef QBE_ALLOC
  return cudaSuccess;
}

void free_vjp_work(VjpWork& vw) {
  cudaFree(vw.nu); cudaFree(vw.nuf); cudaFree(vw.muD); cudaFree(vw.muK2); cudaFree(vw.mu4); cudaFree(vw.mu3);
  cudaFree(vw.part_r); cudaFree(vw.part_s); cudaFree(vw.ws);
  vw = VjpWork();
}

}  // namespace qbe
