/*
 * qbe.h -- C ABI of the GB300 (sm_103a) library for the spatially
 * inhomogeneous matrix-valued quantum Boltzmann equation of Lu & Mendl,
 * "Numerical scheme for a spatially inhomogeneous matrix-valued quantum
 * Boltzmann equation" (arXiv:1408.1782):
 *
 *     d_t W + v_x d_x W = C[W] - i [B . sigma, W]                 (eq. boltzmann)
 *
 * on Omega = (0,1) (one space dimension, two velocity dimensions, Sec. 2).
 *
 * Data conventions (all entry points):
 *  - A state is a set of 2x2 Hermitian Wigner matrices stored as real Pauli
 *    components w = (w0, w1, w2, w3), W = w0*1 + w1*s1 + w2*s2 + w3*s3
 *    (Sec. 3.1, eq. spin_repr).
 *  - Layout: double w[cell][4][ix][iy], row-major, iy fastest, with velocity
 *    v = (2L/N) * (ix - N/2, iy - N/2), i.e. v in (2L/N) Xi with
 *    Xi = {-N/2..N/2-1}^2 (Sec. 3.2 eq. fourier_grid, Sec. 5.1).
 *  - Cell centres x_j = (j + 1/2)/Nx.
 *  - Arithmetic is IEEE FP64 throughout, except the collision transforms of
 *    the FP32-split form (qbe_grid.precision = 1).
 *  - Pointers: "on_device" = 1 means the pointer is device memory of the
 *    handle's GPU; 0 means host memory.  The caller owns every pointer it
 *    passes; the library copies host inputs before returning and never keeps
 *    a caller pointer.  The library owns its own device buffers.
 *  - Calls are ordered on the handle's stream (qbe_set_stream; default: the
 *    legacy default stream).  Calls that take or return host memory
 *    synchronise that stream before returning; device-pointer calls are
 *    asynchronous.
 *  - Every entry point returns QBE_OK (0) or a negative QBE_ERR_* code; the
 *    message of the last failure is available from qbe_last_error().  No entry
 *    point aborts the process.
 */
#ifndef QBE_H
#define QBE_H

#ifdef __cplusplus
extern "C" {
#endif

#define QBE_OK 0
#define QBE_ERR_ARG (-1)          /* invalid argument (size, pointer, range)        */
#define QBE_ERR_CUDA (-2)         /* a CUDA runtime call or kernel launch failed     */
#define QBE_ERR_ALLOC (-3)        /* device or host allocation failed                */
#define QBE_ERR_STATE (-4)        /* call out of order (e.g. step before set_state)  */
#define QBE_ERR_UNSUPPORTED (-5)  /* valid in the paper, not supported by this library */

/* Discretisation (Sec. 3.2, Sec. 5): N velocity points per dimension (Fourier
 * cut-off, N in {8, 16, 32, 48, 64, 96, 128}); Nx finite volumes; J angular points on
 * the half circle (eq. theta_grid; even, 2..64); M Gauss-Legendre radial nodes
 * (eq. approxH-JM; 1..64); L half-width of the periodised velocity box
 * [-L, L]^2; R truncation radius of the collision integrals (B_R).
 * precision: 0 = plain FP64; 1 = FP32-split form (the collision operator's
 * transforms, products and per-unit accumulations in FP32; its input, output
 * and the reduction of its per-unit partial sums, the transport with its
 * boundary projections, the RK2 accumulation and the moments in FP64).  The
 * paper's values are L = 12, R = 7.5, J = M = 32. */
typedef struct qbe_grid {
  int N;
  int Nx;
  int J;
  int M;
  double L;
  double R;
  int precision;
  int device;
} qbe_grid;

/* Boundary conditions on the incoming boundary Sigma_- (Sec. 2). */
typedef enum qbe_bc { QBE_PERIODIC = 0, QBE_DIRICHLET = 1, QBE_MAXWELL = 2 } qbe_bc;

/* A Fermi-Dirac state (eq. W_FermiDirac): W_FD(v) = sum_s n_s(v) |s><s| with
 * n_s = 1/(exp(beta (|v|^2/2 - mu_s)) + 1), |up>, |down> the columns of the
 * unitary U (U[row][col] = U_re + i U_im), beta = 1/(k_B T) > 0. */
typedef struct qbe_fd {
  double beta;
  double mu_up;
  double mu_dn;
  double U_re[2][2];
  double U_im[2][2];
} qbe_fd;

typedef struct qbe_handle qbe_handle;

/* Create a solver for grid g on device g->device.  Allocates the state, the
 * kernel tables (G and H quadratures of eqs. approxG, approxH-J, approxH-JM)
 * and the collision workspace.  *out receives the handle (NULL on failure).
 * Errors: QBE_ERR_ARG (bad sizes, odd J, N unsupported), QBE_ERR_ALLOC,
 * QBE_ERR_CUDA. */
int qbe_create(const qbe_grid* g, qbe_handle** out);

/* Release all device and host memory of h (NULL is ignored). */
void qbe_destroy(qbe_handle* h);

/* Message of the last failing call on h ("" if none); owned by h. */
const char* qbe_last_error(const qbe_handle* h);

/* Order all later work of h on the CUDA stream `stream` (a cudaStream_t, may
 * be NULL for the legacy default stream). */
int qbe_set_stream(qbe_handle* h, void* stream);

/* Boundary condition (Sec. 2): QBE_PERIODIC (left/right ignored), QBE_DIRICHLET
 * (incoming values are the Fermi-Dirac states *left at x = 0, *right at x = 1),
 * QBE_MAXWELL (R = (1 - alpha) L + alpha D with diffusive states *left, *right,
 * accommodation alpha in [0, 1]).  Default after create: periodic.
 * Errors: QBE_ERR_ARG (bad kind, NULL state for D/M, beta <= 0, alpha out of
 * [0,1]). */
int qbe_set_boundary(qbe_handle* h, int bc, const qbe_fd* left, const qbe_fd* right, double alpha);

/* External magnetic field B[cell][3] at the cell centres (eq. boltzmann).
 * Default after create: zero. */
int qbe_set_bfield(qbe_handle* h, const double* B, int on_device);

/* Copy a state w[Nx][4][N][N] into the solver / out of the solver. */
int qbe_set_state(qbe_handle* h, const double* w, int on_device);
int qbe_get_state(qbe_handle* h, double* w, int on_device);

/* Collision operator C[W] = C_c[W] + C_d[W] (eqs. Cc, Cd in the Pauli form
 * eq. CcPauli, eq. CdPauli) by the fast Fourier spectral method of Sec. 3.2
 * (Carleman representation, quadratures G_J, H_J, H_JM, double zero padding),
 * for ncells independent cells: w[ncells][4][N][N] -> c[ncells][4][N][N].
 * Does not touch the solver state.  The -N/2 Fourier line (no +N/2 partner in
 * Xi) is excluded from input and output so that every field is real.
 * Errors: QBE_ERR_ARG (ncells < 1, NULL pointers). */
int qbe_collide(qbe_handle* h, const double* w, double* c, int ncells, int on_device);

/* Transport operator A(tau) on the solver state: the minmod slope-limiter
 * finite-volume update of eq. slopeLimiterStep applied per velocity and per
 * Pauli component (eq. minmod), with two ghost cells per side filled from the
 * boundary condition, sub-cycled so that |v_x| tau_sub / dx <= 1 (Sec. 4).
 * Errors: QBE_ERR_STATE (no state set). */
int qbe_advect(qbe_handle* h, double tau);

/* Collision + precession substep of length dt on the solver state: Heun's
 * second-order Runge-Kutta method for dW/dt = C[W] + 2 (B x w).sigma
 * (eq. boltzmann; -i[B.sigma, W] in Pauli form, Sec. 3.1). */
int qbe_collide_rk2(qbe_handle* h, double dt);

/* nsteps split time steps A(dt/2) o RK2[C + B](dt) o A(dt/2) (Sec. 4). */
int qbe_step(qbe_handle* h, double dt, int nsteps);

/* Moments of the solver state per cell (eqs. density, velocity,
 * internal_energy): rho[Nx][4] = Pauli components of int W dv,
 * mom[Nx][2] = int v tr W dv, energy[Nx] = int |v|^2/2 tr W dv, all as grid
 * sums times (2L/N)^2.  Any output pointer may be NULL. */
int qbe_moments(qbe_handle* h, double* rho, double* mom, double* energy, int on_device);

/* ---- Differentiation -------------------------------------------------
 * The paper computes no derivatives: these entry points are exact
 * vector-Jacobian products (transposed derivatives) of the discrete maps
 * above, for gradients of a final-time observable with respect to the
 * initial state and the field B.  C[W] is a cubic polynomial in W (eq.
 * CcPauli, eq. CdPauli), so its derivative is the same family of FFT
 * convolutions with reflected multipliers; the transport update (eq.
 * slopeLimiterStep) is differentiated at the minmod branches (eq. minmod) the
 * forward call takes (a tie |a| = |b| takes a's branch), the Maxwell wall's
 * outgoing flux (Sec. 2) as the linear functional it is, and the precession
 * term -i[B.sigma, W] = 2 (B x w).sigma as the bilinear map it is.  Each
 * product is computed in the handle's precision form. */

/* grad = (dC/dW at w)^T lam for ncells independent cells: w, lam, grad
 * [ncells][4][N][N] (grad may alias lam).  Does not touch the solver state.
 * The first call allocates the product's workspace (about twice the
 * collision workspace).  Errors: QBE_ERR_ARG, QBE_ERR_ALLOC, QBE_ERR_CUDA. */
int qbe_collide_vjp(qbe_handle* h, const double* w, const double* lam, double* grad, int ncells, int on_device);

/* ncot products at the same state at once: grad[k] = (dC/dW at w)^T lam[k],
 * k < ncot, with lam, grad [ncot][ncells][4][N][N] and w [ncells][4][N][N],
 * all DEVICE memory (on_device must be 1).  The products are evaluated in
 * groups that share the state's transforms (for the I3 term, the Psi'
 * convolutions of the state: 8 of the 16 per (j, m) and product); groups
 * are as in qbe_step_vjp_n;
 * each result equals qbe_collide_vjp's bit for bit.  Grows the workspace to
 * the group size on first use.  Errors: QBE_ERR_ARG (ncot < 1, ncells < 1,
 * null pointers, on_device != 1), QBE_ERR_ALLOC, QBE_ERR_CUDA. */
int qbe_collide_vjp_n(qbe_handle* h, int ncot, const double* w, const double* lam, double* grad, int ncells,
                      int on_device);

/* qbe_step(h, dt, nsteps) that also records a tape for qbe_step_vjp: the
 * state before every checkpoint_every-th step (ceil(nsteps/checkpoint_every)
 * states of device memory, kept by h and reused).  Any later call that
 * changes the state, the field or the boundary invalidates the tape.
 * Errors: QBE_ERR_ARG (nsteps < 1, checkpoint_every < 1), QBE_ERR_STATE. */
int qbe_step_checkpointed(qbe_handle* h, double dt, int nsteps, int checkpoint_every);

/* qbe_step(h, dt, nsteps) that records a full tape: every intermediate state
 * of every step (nsteps (2 s + 2) states of device memory, s the transport
 * substeps of a half step: the inputs of the transport substeps, U and W1 of
 * the Heun step), so that qbe_step_vjp(_n) recomputes nothing and its
 * reverse sweep does only the transposed work.  The storage is kept by h
 * until it is destroyed or a later qbe_step_checkpointed releases it.  The
 * tape is invalidated as qbe_step_checkpointed's is.  Errors: QBE_ERR_ARG
 * (nsteps < 1, dt not finite), QBE_ERR_STATE, QBE_ERR_ALLOC (the tape does
 * not fit: nothing was stepped, the state is unchanged and no tape is
 * valid), QBE_ERR_CUDA. */
int qbe_step_taped(qbe_handle* h, double dt, int nsteps);

/* Reverse sweep over the tape of the last qbe_step_checkpointed(h, dt,
 * nsteps, k) or qbe_step_taped(h, dt, nsteps) call, which mapped W_0 to W_n:
 * lam_init = (dW_n/dW_0)^T lam_final ([Nx][4][N][N]) and, if grad_B is not
 * NULL, grad_B = (dW_n/dB)^T lam_final ([Nx][3]).  With checkpoints, each
 * segment of k steps is recomputed from its checkpoint with every
 * intermediate state kept (k (2 s + 2) states, s the transport substeps of a
 * half step), then swept backwards; a full tape is swept as it is.  Both
 * tapes give the same result bit for bit.  The state
 * is W_n again on return.  Errors: QBE_ERR_STATE (no valid tape),
 * QBE_ERR_ARG, QBE_ERR_ALLOC, QBE_ERR_CUDA. */
int qbe_step_vjp(qbe_handle* h, const double* lam_final, double* lam_init, double* grad_B, int on_device);

/* The same reverse sweep for ncot cotangents at once (e.g. the gradients of
 * several observables): each segment is recomputed once and the cotangents
 * are swept over its intermediate states in groups; within a group each
 * collision product (dC/dW)^T is evaluated for all members at once, sharing
 * the state's transforms (the I3 term's Psi' convolutions of the state, half
 * of the transpose's work).  Groups hold up to four cotangents, one in the
 * FP32-split form on padded grids up to 128 points, whose transpose keeps its
 * transforms in shared memory and is bound by its per-cotangent global
 * accumulators instead.  lam_final, lam_init [ncot][Nx][4][N][N],
 * grad_B [ncot][Nx][3] (may be NULL).  Results equal ncot calls of
 * qbe_step_vjp bit for bit.  Extra memory: two states per cotangent, and the
 * collision product's cotangent buffers once per group member. */
int qbe_step_vjp_n(qbe_handle* h, int ncot, const double* lam_final, double* lam_init, double* grad_B,
                   int on_device);

/* Final-time observables of a state w[Nx][4][N][N] (NULL: the solver
 * state): out[0] = P_z = dx dv^2 sum 2 w3 (total spin polarisation along z,
 * tr(sigma_3 W) = 2 w3), out[1] = Phi_E = dx dv^2 sum v_x |v|^2/2 2 w0
 * (energy flux, tr W = 2 w0), sums over all cells and velocities, dx = 1/Nx,
 * dv = 2L/N (eqs. density, internal_energy).  w and out are both host or
 * both device memory. */
int qbe_observables(qbe_handle* h, const double* w, double* out, int on_device);

/* lam = gbar[0] dP_z/dW + gbar[1] dPhi_E/dW ([Nx][4][N][N]); gbar[2]. */
int qbe_observables_vjp(qbe_handle* h, const double* gbar, double* lam, int on_device);

/* ---- Diagnostics (Sec. 2, Sec. 5) --------------------------------------
 * A Fermi-Dirac state with mean velocity u (eq. W_FermiDirac; the average
 * velocity shifts W_FD(v) -> W_FD(v - u), Sec. 5.2):
 *   W_FD(v) = sum_s (exp((|v - u|^2/2 - mu_s)/T) + 1)^-1 |s><s|,
 * T = k_B T, |up> = column 0 of U, |up><up| = (1 + bloch.sigma)/2. */
typedef struct qbe_fermi_dirac {
  double T;            /* k_B T; 0 when ok == 0 */
  double mu_up;
  double mu_dn;
  double bloch[3];     /* unit Bloch vector of |up> */
  double U_re[2][2];   /* U[row][col] = U_re + i U_im; columns |up>, |down> */
  double U_im[2][2];
  double u[2];         /* mean velocity */
  int ok;              /* 1: fitted; 0: no Fermi-Dirac state has these moments */
} qbe_fermi_dirac;

/* Local entropy per cell S[W](x_j) = -int tr[W log W + (1 - W) log(1 - W)] dv
 * (eq. entropy_def) as dv^2 sum_v over the eigenvalues w0 +- |w| (0 log 0 =
 * 0): S[Nx]. */
int qbe_entropy(qbe_handle* h, double* S, int on_device);

/* Fermi-Dirac state with the moments (grid sums, eqs. density, velocity,
 * internal_energy) of each cell (global = 0: out[Nx]) or of the whole domain
 * (global = 1: x-averaged moments, out[1]).  The eigenbasis is that of the spin
 * density rho (up = larger eigenvalue); T, mu_up, mu_dn solve eq.
 * momentsFermiDirac for the eigenvalues of rho and the internal energy per
 * particle (Sec. 5.2).  out is host memory.  A state whose internal energy
 * is at or below the T -> 0 limit sum_s rho_s^2 / (4 pi tr rho), or with a
 * non-positive eigenvalue of rho, gets ok = 0. */
int qbe_fd_fit(qbe_handle* h, int global, qbe_fermi_dirac* out);

/* The same fit for given moments (host only, no GPU): rho4 = Pauli components
 * of int W dv, mom = int v tr W dv, energy = int |v|^2/2 tr W dv. */
int qbe_fd_fit_moments(const double* rho4, const double* mom, double energy, qbe_fermi_dirac* out);

/* Dilogarithm Li2(x) for real x <= 0 (host; the fit's special function):
 * 't Hooft-Veltman Bernoulli series in -log(1 - x) on [-1, 0], inversion
 * below -1.  NaN for x > 0. */
double qbe_dilog(double x);

/* Per cell: quantum relative entropy S(W(x_j) || F_j) = int tr[W (log W -
 * log F) + (1 - W)(log(1 - W) - log(1 - F))] dv (eq. relentropy_hom) and, if
 * l1 is not NULL, the distance int ||W - F||_1 dv (trace norm), with F_j =
 * ref[j] (nref = Nx, local: eq. relentropy_local) or ref[0] (nref = 1, global:
 * eq. relentropy_inhom); the x-integrals are the means over cells.  ref is host
 * memory; rel[Nx], l1[Nx] host or device.  Errors: QBE_ERR_ARG (nref not 1 or
 * Nx, a reference with ok == 0). */
int qbe_relative_entropy(qbe_handle* h, const qbe_fermi_dirac* ref, int nref, double* rel, double* l1, int on_device);

/* Number of kernel launches issued by the library since create (for
 * benchmarking bookkeeping). */
long long qbe_launch_count(const qbe_handle* h);

/* Device-time accounting per kernel group (diagnostics; not part of the
 * method).  qbe_enable_timing(h, 1) clears the counters and brackets every
 * later launch of the library with CUDA events on h's stream;
 * qbe_kernel_time() synchronises the stream and returns the accumulated
 * device time (ms) and launch count of one group since enabling.  Groups:
 * 0 coefficients/prep, 1 I1 (C_c), 2 I2+I4, 3 I3 (Hu-Ying term),
 * 4 assembly/projection, 5 transport, 6 RK/precession update, 7-9 the
 * adjoint's kernels (below). */
#define QBE_KG_PREP 0
#define QBE_KG_I1 1
#define QBE_KG_I24 2
#define QBE_KG_I3 3
#define QBE_KG_ASSEMBLE 4
#define QBE_KG_TRANSPORT 5
#define QBE_KG_RK 6
#define QBE_KG_VJP 7           /* collision product: recomputed forward terms, seed, I1/I2/I4 transposes, final */
#define QBE_KG_VJP_I3 8        /* collision product: transpose of the I3 (Hu-Ying) term */
#define QBE_KG_ADJ_TRANSPORT 9 /* transposes of the transport substeps and of the RK2 + precession update */
int qbe_enable_timing(qbe_handle* h, int enable);
int qbe_kernel_time(qbe_handle* h, int which, double* total_ms, long long* launches);

/* Arithmetic issue rates of the device (measurement behind the "alu"
 * rooflines; not part of the method).  Runs, on `stream` (a cudaStream_t;
 * NULL: the default stream) of device `device`, kernels of 8 blocks of 256
 * threads per SM whose threads each advance eight independent chains of one
 * operation, one warm-up and one timed launch each, and writes
 * rates[0..3] = FP64 fma, FP64 add, FP64 mul and FP32 fma lane-operations
 * per second.  Synchronises the stream; allocates and frees about 2.5 MB of
 * device memory.  Errors: QBE_ERR_ARG (rates NULL, device < 0),
 * QBE_ERR_CUDA. */
int qbe_arith_issue_rates(int device, void* stream, double* rates);

/* Launch shape of the I3 (Hu-Ying term, eq. approxH-JM) kernel -- the dominant
 * part of C[W] (Sec. 3.2) -- and its autotuner.  A shape is
 *   - a launch variant: one of the kernel forms instantiated for this padded
 *     grid size 2N and precision.  FP64: the staged kernel with 256 threads and
 *     64 KB shared-memory chunks (3 blocks per SM) or 128 threads and 32 KB
 *     chunks (6 per SM), or the staged kernel with its global loads and
 *     stores fused into the line stages (256 threads, 64 KB).  FP32-split form, 2N = 64, 96, 128: the fused
 *     shared-memory kernel in three thread/accumulation shapes, or the kernel
 *     whose element passes go through shared memory, and at 2N = 128 also the
 *     kernel with warp-local passes; 2N <= 32: the element-pass kernel
 *     only; 2N = 192, 256: the cluster kernel with 1024 threads per CTA, or
 *     with two row tasks per thread and register accumulation;
 *   - the persistent grid (blocks; at most the variant's residency);
 *   - the number of m-chunks per (cell, angle) work unit.
 * qbe_i3_shape reports the current shape and the number of variants
 * (any pointer may be NULL).  qbe_i3_variant_name describes a variant (NULL
 * when out of range; static storage).  qbe_set_i3_shape sets a shape: variant
 * -1 keeps the variant, grid 0 and m_chunks 0 keep theirs; m_chunks may not
 * exceed the value set when the handle was created (QBE_ERR_ARG).
 * qbe_autotune times every variant x grid x m-chunking candidate on the
 * current state -- two waves of the I3 work queue each, after the per-cell
 * terms of that state, scaled from the sample's busiest block to the busiest
 * block of the whole queue -- and keeps the fastest; best_ms (may be NULL) receives its predicted I3 launch time.  It
 * needs a state (QBE_ERR_STATE), synchronises the stream, and leaves the state
 * unchanged.  The variants compute the same sums in different orders:
 * results of different shapes agree to rounding (FP64: ~1e-15 relative; the
 * FP32-split form: within its stated tolerance). */
int qbe_i3_shape(const qbe_handle* h, int* variant, int* nvariants, int* grid, int* m_chunks);
const char* qbe_i3_variant_name(const qbe_handle* h, int variant);
int qbe_set_i3_shape(qbe_handle* h, int variant, int grid, int m_chunks);
int qbe_autotune(qbe_handle* h, double* best_ms);

/* Kernel variant of the transpose of the I3 term in the collision product
 * (qbe_collide_vjp, and the reverse sweeps of qbe_step_vjp).  FP32-split form
 * at 2N = 128: variant 0 (the default) runs the convolutions on warp-local
 * passes with the sums into XZ held in registers (one cotangent per product),
 * variant 1 the kernel whose element passes go through shared memory; every
 * other grid and precision has one variant.  The variants agree to rounding.
 * qbe_vjp_i3_variant reports the current variant and the count (either
 * pointer may be NULL); qbe_set_vjp_i3_variant sets it (-1: the default;
 * QBE_ERR_ARG when out of range). */
int qbe_vjp_i3_variant(const qbe_handle* h, int* variant, int* nvariants);
int qbe_set_vjp_i3_variant(qbe_handle* h, int variant);

/* ------------------------------------------------------------------------
 * Batches of independent simulations: several solver handles -- any mix of
 * N, Nx, J, M, precision, boundary conditions and B fields, all on one
 * device -- stepped together (the simulations are independent, Sec. 3.2).
 * The first qbe_batch_step with a given dt captures one split step (Sec. 4)
 * of every simulation into a CUDA graph; every step is then one graph launch.
 * The graph runs, per simulation on its own branch, the transport and the
 * per-cell collision terms, and between them one I3 (Hu-Ying term) launch per
 * padded-grid size and precision whose work queue covers the (simulation,
 * cell, angle, m-chunk) units of every simulation of that size.  Results
 * equal those of qbe_step on each handle (the same kernels on the same units).
 * qbe_batch_autotune chooses, per padded-grid size and precision, the I3
 * launch shape (variant, persistent grid, m-chunks; see qbe_autotune) of the
 * group's shared work-queue launch by timing two waves of it per candidate on
 * the simulations' current states, sets it on every member (qbe_i3_shape
 * reports it) and drops any captured graph; another shape sums the I3 terms
 * in another order (results then differ from untuned steps by rounding).
 * The handles stay owned by the caller and must outlive the batch; each may
 * appear once.  With a stream set (qbe_batch_set_stream) the steps are
 * asynchronous on it; without one, qbe_batch_step synchronises before it
 * returns.
 * ------------------------------------------------------------------------ */
typedef struct qbe_batch qbe_batch;
int qbe_batch_create(qbe_handle* const* sims, int nsims, qbe_batch** out);
void qbe_batch_destroy(qbe_batch* b);
const char* qbe_batch_last_error(const qbe_batch* b);
int qbe_batch_set_stream(qbe_batch* b, void* stream);
int qbe_batch_autotune(qbe_batch* b);
/* Tuned I3 launch shape of simulation `sim` (persistent grid, m-chunks) and
 * the predicted time of its group's I3 launch with it (ms, 0 before
 * autotuning); the variant is reported by qbe_i3_shape on the handle. */
int qbe_batch_tuned_shape(const qbe_batch* b, int sim, int* i3_grid, int* m_chunks, double* ms);
int qbe_batch_step(qbe_batch* b, double dt, int nsteps);

/* Collision operator without any memory allocation (the paper has no
 * counterpart: this is a deployment variant of qbe_collide).
 *
 * For callers that cannot allocate device memory at call time -- code hosted
 * by a framework that owns the GPU's memory budget and forbids allocations,
 * latency-critical paths where cudaMalloc's implicit device synchronisation is
 * not acceptable, or deployments that must reserve all memory when the
 * library is loaded.  It computes the same C[W] as qbe_collide for
 * w[ncells][4][N][N] -> c[ncells][4][N][N], both DEVICE pointers of the
 * calling thread's current device (g->device must equal it), on `stream`
 * (a cudaStream_t, NULL = legacy default stream), asynchronously.
 *
 * Memory: no cudaMalloc, no cudaFree, no host heap.  Kernel tables and every
 * piece of scratch live in one statically sized device array of
 * QBE_NOALLOC_SCRATCH_BYTES that every GPU which loads the library holds until
 * the process exits.  Every call resolves that array's address
 * (cudaGetSymbolAddress, which allocates nothing) and a call whose grid
 * (N, J, M, L, R) differs from the previous call's rebuilds the tables in the
 * array with two extra kernel launches; make the first call on a device before
 * any stream capture.  A call issued while its stream is being captured always
 * records the rebuild, and every later call on that device rebuilds too (the
 * host can no longer tell which grid the array holds).  Cells are
 * processed in batches that fit the array.  Every call shares the array and
 * leaves its contents behind; the kernels initialise everything they read, so
 * no clearing is needed between calls, but calls that overlap on the GPU (on
 * different streams, or from several host threads) race and must be ordered
 * by the caller.
 *
 * Limits: N in {8, 16, 32, 64}; J even in 2..64; M in 1..64; precision 0.
 * The grid must fit: tables (4 J (2N)^2 doubles + 2 J M (2N) complex) plus,
 * for one cell, (10 + 2 J) (2N)^2 complex + (2N)^2 doubles of workspace plus
 * scratch of the I3 blocks, within QBE_NOALLOC_SCRATCH_BYTES (e.g. N = 64 with
 * J = M = 32 fits, one cell per batch).  Larger grids return QBE_ERR_ARG.
 * Errors: QBE_ERR_ARG (bad sizes, NULL pointers, grid too large, device
 * mismatch), QBE_ERR_UNSUPPORTED (precision != 0), QBE_ERR_CUDA. */
#define QBE_NOALLOC_SCRATCH_BYTES (64ull << 20)
int qbe_collide_noalloc(const qbe_grid* g, const double* w, double* c, int ncells, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QBE_H */
