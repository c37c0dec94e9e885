"""Seeded synthetic inputs for the matrix-valued quantum Boltzmann solver.

This module only *creates* input states; it contains none of the solver's
arithmetic (no collision operator, transport, boundary projection, time step
or moment).  Both the CPU oracle (through the tests and the benchmark) and the
CUDA library receive the arrays produced here, so it is the one piece of code
the two sides share.

State layout everywhere: Pauli components ``w[cell][c][ix][iy]`` (float64),
c = 0..3 for (identity, sigma_1, sigma_2, sigma_3), velocity
``v = (2L/N) * (ix - N/2, iy - N/2)`` (Sec. 3.2, eq. fourier_grid: v in (2L/N) Xi),
``iy`` fastest.  A Hermitian 2x2 matrix W is ``w0*1 + w1*s1 + w2*s2 + w3*s3``
(eq. spin_repr), so ``w_c = tr(W sigma_c)/2``.

Recipes:
* ``synthetic_w``: W(x,v) = exp(-iX) U0 diag(n_up, n_dn) U0^+ exp(iX), the
  v-dependent basis rotation pattern of the homogeneous example (Sec. 5.2,
  eq. W0homogeneous) with x-dependent temperature, chemical potentials, drift
  and basis, optionally plus a small smooth random Hermitian perturbation whose
  eigenvalues are then clipped to [0, 1].
* ``validation_w``: the fixed test state of Sec. 5.1 (eq. validationW).
* ``homogeneous_w0``: the initial state of Sec. 5.2 (eq. W0homogeneous).
* ``rotating_b``: the external field of Sec. 5.3 (eq. Bext_rot).
* ``bandlimited_w``: random real Pauli fields whose Fourier coefficients on
  the grid Xi vanish outside |xi_x|, |xi_y| <= band (used where a test needs the
  spectral interpolant to be exact).
"""
from __future__ import annotations

import numpy as np

SIGMA = np.array(
    [
        [[1, 0], [0, 1]],
        [[0, 1], [1, 0]],
        [[0, -1j], [1j, 0]],
        [[1, 0], [0, -1]],
    ],
    dtype=np.complex128,
)


def velocity_axis(N: int, L: float) -> np.ndarray:
    """1-D velocity nodes (2L/N) k, k = -N/2 .. N/2-1."""
    return (2.0 * L / N) * np.arange(-N // 2, N // 2, dtype=np.float64)


def velocity_mesh(N: int, L: float):
    a = velocity_axis(N, L)
    return np.meshgrid(a, a, indexing="ij")


def cell_centres(Nx: int) -> np.ndarray:
    """Finite-volume centres x_j = (j + 1/2)/Nx on Omega = (0, 1)."""
    return (np.arange(Nx, dtype=np.float64) + 0.5) / Nx


def matrix_to_pauli(Wm: np.ndarray) -> np.ndarray:
    """[..., 2, 2] Hermitian -> [..., 4] real Pauli components (tr(W s_c)/2)."""
    out = np.einsum("...ij,cji->...c", Wm, SIGMA) * 0.5
    return out.real.copy()


def pauli_to_matrix(w: np.ndarray) -> np.ndarray:
    """[..., 4] -> [..., 2, 2]."""
    return np.einsum("...c,cij->...ij", w.astype(np.complex128), SIGMA)


def _su2_exp(vec: np.ndarray) -> np.ndarray:
    """exp(i vec.sigma) for real 3-vectors [..., 3] (closed form)."""
    n = np.linalg.norm(vec, axis=-1)
    safe = np.where(n > 0, n, 1.0)
    unit = vec / safe[..., None]
    c = np.cos(n)[..., None, None]
    s = np.sin(n)[..., None, None]
    us = np.einsum("...a,aij->...ij", unit.astype(np.complex128), SIGMA[1:])
    eye = np.eye(2, dtype=np.complex128)
    return c * eye + 1j * s * us


def _fd_occupation(beta, energy, mu):
    x = beta * (energy - mu)
    return 0.5 * (1.0 - np.tanh(0.5 * x))  # 1/(e^x+1), overflow free


def synthetic_w(N: int, Nx: int, L: float = 12.0, seed: int = 0, perturb: float = 0.0) -> np.ndarray:
    """Fermi-Dirac-like state with x- and v-dependent spin basis; [Nx, 4, N, N]."""
    rng = np.random.default_rng(seed)
    x = cell_centres(Nx)
    vx, vy = velocity_mesh(N, L)
    ph_beta, ph_mu = rng.uniform(0, 2 * np.pi, 2)
    beta = 1.25 + 0.75 * np.sin(2 * np.pi * x + ph_beta)          # in [0.5, 2]
    mu = np.cos(2 * np.pi * x + ph_mu)                              # in [-1, 1]
    mu_up, mu_dn = mu + 0.5, mu - 0.5
    v0x, v0y = 0.3 * np.cos(2 * np.pi * x), 0.3 * np.sin(2 * np.pi * x)
    # U0(x) = exp(i sum_q c_q.sigma sin(2 pi q x + phi_q))
    cq = rng.uniform(-0.6, 0.6, (2, 3))
    phq = rng.uniform(0, 2 * np.pi, 2)
    u0vec = sum(cq[q][None, :] * np.sin(2 * np.pi * (q + 1) * x + phq[q])[:, None] for q in range(2))
    U0 = _su2_exp(u0vec)                                            # [Nx,2,2]
    # X(x,v) = sum_a sigma_a p_a(x) g_a(v)
    env = np.exp(-(vx**2 + vy**2) / 18.0)
    g = np.stack([(vx - 1.0) * env, 2.0 / (vx**2 + vy**2 + 1.0), np.cos(vx + 0.5 * vy) * env])  # [3,N,N]
    pa = rng.uniform(0.5, 1.0, 3)
    pb = rng.uniform(0.2, 0.5, 3)
    pph = rng.uniform(0, 2 * np.pi, 3)
    p = pa[None, :] + pb[None, :] * np.sin(2 * np.pi * x[:, None] + pph[None, :])   # [Nx,3]
    Xvec = np.einsum("ja,axy->jxya", p, g)                           # [Nx,N,N,3]
    E = _su2_exp(-Xvec)                                               # exp(-iX)
    e_up = 0.5 * ((vx[None] - v0x[:, None, None]) ** 2 + (vy[None] - v0y[:, None, None]) ** 2)
    n_up = _fd_occupation(beta[:, None, None], e_up, mu_up[:, None, None])
    n_dn = _fd_occupation(beta[:, None, None], e_up, mu_dn[:, None, None])
    D = np.zeros((Nx, N, N, 2, 2), dtype=np.complex128)
    D[..., 0, 0] = n_up
    D[..., 1, 1] = n_dn
    U = U0[:, None, None]
    Wm = E @ U @ D @ np.conj(np.swapaxes(U, -1, -2)) @ np.conj(np.swapaxes(E, -1, -2))
    if perturb > 0.0:
        Wm = Wm + perturb * _smooth_hermitian(N, Nx, L, rng)
        lam, V = np.linalg.eigh(Wm)
        lam = np.clip(lam, 0.0, 1.0)
        Wm = V @ (lam[..., None] * np.conj(np.swapaxes(V, -1, -2)))
    w = matrix_to_pauli(Wm)                                           # [Nx,N,N,4]
    return np.ascontiguousarray(np.moveaxis(w, -1, 1))


def _smooth_hermitian(N, Nx, L, rng):
    """Low-mode random Hermitian field x Gaussian envelope, smooth in x; [Nx,N,N,2,2]."""
    x = cell_centres(Nx)
    vx, vy = velocity_mesh(N, L)
    env = np.exp(-(vx**2 + vy**2) / 8.0)
    comps = []
    for _c in range(4):
        f = np.zeros((Nx, N, N))
        for _m in range(3):
            kx, ky = rng.uniform(-0.8, 0.8, 2)
            ph, phx, amp = rng.uniform(0, 2 * np.pi), rng.uniform(0, 2 * np.pi), rng.uniform(0.3, 1.0)
            f += amp * np.cos(kx * vx + ky * vy + ph)[None] * np.cos(2 * np.pi * x + phx)[:, None, None]
        comps.append(f * env[None])
    w = np.stack(comps, axis=-1)
    return pauli_to_matrix(w)


def validation_w(N: int, L: float = 12.0) -> np.ndarray:
    """The fixed Wigner state of Sec. 5.1 (eq. validationW); [4, N, N]."""
    vx, vy = velocity_mesh(N, L)
    w0 = (1.0 / (3 * np.pi)) * (1 + vx) * np.exp(-0.5 * (vx - 0.5) ** 2 - 0.5 * (vy + vx) ** 2)
    w1 = (3 * np.sqrt(6.0 / 5.0) / (55 * np.pi)) * (1 - vx - vy / 6.0) ** 2 * np.exp(
        -(2 * vx + vy) ** 2 / 12.0 - vy**2 / 10.0)
    w2 = (1.0 / (4 * np.pi * np.sqrt(2.0))) * np.exp(-(vx - 1) ** 2 / 8.0 - vy**2 / 4.0)
    w3 = (9.0 / (56 * np.pi)) * (1.0 / 3.0 + vx) ** 2 * np.exp(-(vx - vy) ** 2 / 8.0 - (vx + 2 * vy) ** 2 / 8.0)
    return np.stack([w0, w1, w2, w3])


def homogeneous_w0(N: int, L: float = 12.0, vy_smoothing: float = 0.0, rotation: float = 1.0) -> np.ndarray:
    """Initial state of Sec. 5.2 (eq. W0homogeneous): kT=5/4, mu=(1, 3/2), v0=(0.4,-0.1); [4,N,N].

    Variants for convergence studies (defaults give the paper's state): ``vy_smoothing`` = e > 0
    replaces |v_y| in X(v) by sqrt(v_y^2 + e^2) (no kink at v_y = 0); ``rotation`` scales the
    sigma part of X(v) (0: the Fermi-Dirac state U0 diag(n) U0^+ without v-dependent rotation)."""
    vx, vy = velocity_mesh(N, L)
    c, s = np.cos(np.pi / 5), np.sin(np.pi / 5)
    U0 = np.array([[c, -1j * s], [s, 1j * c]], dtype=np.complex128)
    kT, mus, v0 = 1.25, (1.0, 1.5), (0.4, -0.1)
    e = 0.5 * ((vx - v0[0]) ** 2 + (vy - v0[1]) ** 2)
    D = np.zeros((N, N, 2, 2), dtype=np.complex128)
    D[..., 0, 0] = _fd_occupation(1.0 / kT, e, mus[0])
    D[..., 1, 1] = _fd_occupation(1.0 / kT, e, mus[1])
    # X(v) = sin(vy^2) 1 + (vx-1) s1 + 2/(vx^2+|vy|+1) s2 + cos(vx + vy/2) s3
    ay = np.abs(vy) if vy_smoothing <= 0.0 else np.sqrt(vy**2 + vy_smoothing**2)
    xvec = rotation * np.stack([vx - 1.0, 2.0 / (vx**2 + ay + 1.0), np.cos(vx + 0.5 * vy)], axis=-1)
    E = _su2_exp(-xvec) * np.exp(-1j * np.sin(vy**2))[..., None, None]
    Wm = E @ U0 @ D @ np.conj(U0.T) @ np.conj(np.swapaxes(E, -1, -2))
    return np.ascontiguousarray(np.moveaxis(matrix_to_pauli(Wm), -1, 0))


def rotating_b(Nx: int) -> np.ndarray:
    """B(x) = (0, cos 2 pi x, sin 2 pi x) at the cell centres (eq. Bext_rot); [Nx, 3]."""
    x = cell_centres(Nx)
    return np.stack([np.zeros_like(x), np.cos(2 * np.pi * x), np.sin(2 * np.pi * x)], axis=-1)


def uniform_b(Nx: int, b) -> np.ndarray:
    return np.tile(np.asarray(b, dtype=np.float64)[None, :], (Nx, 1))


def bandlimited_w(N: int, band: int, ncells: int = 1, seed: int = 0, scale: float = 0.2) -> np.ndarray:
    """Random real Pauli fields with Fourier support |xi_x|,|xi_y| <= band on Xi; [ncells,4,N,N]."""
    assert 2 * band < N // 2, "band too wide for the grid"
    rng = np.random.default_rng(seed)
    k = np.arange(-N // 2, N // 2)
    out = np.zeros((ncells, 4, N, N))
    modes = [(a, b) for a in range(-band, band + 1) for b in range(-band, band + 1)]
    for cidx in range(ncells):
        for comp in range(4):
            f = np.zeros((N, N))
            for (a, b) in modes:
                amp = rng.normal() * scale / (1 + a * a + b * b)
                ph = rng.uniform(0, 2 * np.pi)
                f += amp * np.cos(2 * np.pi * (a * k[:, None] + b * k[None, :]) / N + ph)
            if comp == 0:
                f += 0.3
            out[cidx, comp] = f
    return out


# Named workloads.  Sizes follow the paper's parameters (L=12, R=7.5, J=M=32,
# Sec. 5) and the benchmark configurations.
WORKLOADS = {
    "plain_fp64_n16": dict(N=16, Nx=16, L=12.0, R=7.5, J=32, M=32, bc="periodic",
                           B=(0.0, 0.0, 0.0), dt=0.01, steps=10, perturb=0.0, precision=0),
    "plain_fp64_n64": dict(N=64, Nx=128, L=12.0, R=7.5, J=32, M=32, bc="dirichlet",
                           wall=dict(beta=1.0, mu_up=0.0, mu_dn=0.0),
                           B=(0.0, 0.0, 0.5), dt=0.005, steps=1000, perturb=0.05, precision=0),
    "precision_n128": dict(N=128, Nx=256, L=12.0, R=7.5, J=32, M=32, bc="maxwell", alpha=0.5,
                           wall=dict(beta=1.0, mu_up=0.0, mu_dn=0.0),
                           B=(0.3, 0.0, 0.4), dt=0.002, steps=200, perturb=0.05, precision=1),
    # gradient of the final-time spin polarisation and energy flux w.r.t. the initial W and B
    "adjoint_n64": dict(N=64, Nx=128, L=12.0, R=7.5, J=32, M=32, bc="periodic",
                        B=(0.3, 0.0, 0.4), dt=0.005, steps=200, checkpoint_every=20, perturb=0.05, precision=1),
}


def minmod_tie_w(N: int, Nx: int, L: float = 12.0, seed: int = 0) -> np.ndarray:
    """A state whose x-differences are exactly 0 or 1/64: one cell of synthetic_w rounded to
    multiples of 1/64 and repeated over x, plus a ramp of 1/64 per cell on w0 where |v| < 4.
    Every limiter argument pair with ab > 0 is then an exact tie |a| = |b| (away from walls)."""
    W = np.repeat(np.round(synthetic_w(N, 1, L=L, seed=seed) * 64.0) / 64.0, Nx, axis=0)
    vx, vy = velocity_mesh(N, L)
    W[:, 0] += (np.arange(Nx)[:, None, None] / 64.0) * ((vx**2 + vy**2) < 16.0)
    return W


def random_field(shape, seed: int = 0, scale: float = 1.0) -> np.ndarray:
    """Seeded standard-normal field of the given shape (tangent directions and cotangents)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(scale * rng.standard_normal(shape))


def fermi_dirac_w(N: int, Nx: int, beta: float, mu_up: float, mu_dn: float, U=None, L: float = 12.0) -> np.ndarray:
    """Uniform Fermi-Dirac state (eq. W_FermiDirac) in every cell; U's columns are the spin basis; [Nx,4,N,N]."""
    vx, vy = velocity_mesh(N, L)
    e = 0.5 * (vx**2 + vy**2)
    U = np.eye(2, dtype=np.complex128) if U is None else np.asarray(U, dtype=np.complex128)
    D = np.zeros((N, N, 2, 2), dtype=np.complex128)
    D[..., 0, 0] = _fd_occupation(beta, e, mu_up)
    D[..., 1, 1] = _fd_occupation(beta, e, mu_dn)
    Wm = U[None, None] @ D @ np.conj(U.T)[None, None]
    w = np.moveaxis(matrix_to_pauli(Wm), -1, 0)
    return np.ascontiguousarray(np.repeat(w[None], Nx, axis=0))
