"""Plain FP64 CPU oracle for Lu & Mendl, "Numerical scheme for a spatially
inhomogeneous matrix-valued quantum Boltzmann equation" (arXiv:1408.1782).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this module.  It shares no code with the CUDA library and
imports nothing from it; it is slow on purpose and follows the paper's steps
in the paper's order and notation so that it can be read against the text.
The discrete FFT on the padded grid is used only as the transform primitive
(numpy.fft); ``to_fine``/``from_fine`` are pinned against the explicit
exponential sums in the tests.

Conventions (all FP64):
* velocity nodes v_k = (2L/N) k, k in Xi = {-N/2..N/2-1}^2 (Sec. 3.2,
  eq. fourier_grid and Sec. 5.1); arrays [..., ix, iy] with k = (ix-N/2, iy-N/2);
* averaged Fourier coefficients on Xi, fhat(xi) = N^-2 sum_k f(v_k) e^{-i pi xi.v_k/L}
  (Sec. 3.2, the "slashed" average integral);
* "double zero padding" (Sec. 1 and Sec. 3.2): products of trigonometric
  polynomials are formed on the 2N x 2N grid v' = (L/N) k', k' in [-N, N-1]^2,
  coefficients sigma in [-N, N-1]^2 (array index s = sigma + N);
* Pauli components w = (w0, w1, w2, w3), W = w . (1, sigma) (eq. spin_repr);
  eta = diag(1,-1,-1,-1).

Readings of the paper taken here (each also listed in the design notes):
* phi_R(s) = (2L/(pi s)) sin^2(pi s R/(2L)) (the printed bracket has the
  opposite sign; G uses phi_R twice so G is unaffected);
* psi'_{R,j}(chi) = (2L/(pi chi.theta_j^perp)) sin(pi R chi.theta_j^perp / L)
  (the printed denominator reads xi.theta_j);
* the I2 formula uses omega_{H,j} and psi' (the printed omega_{G,j} and tilde-psi);
* J must be even (for odd J some theta_j . theta'_j' vanish);
* nyquist="zero" (canonical): the xi = -N/2 row and column of Xi, which has no
  +N/2 partner, is set to zero on input and output so every field is real;
  nyquist="keep" evaluates the literal Xi in complex arithmetic and returns the
  real part of C;
* time integrator of the collision + precession substep: Heun's RK2;
* splitting A(dt/2) o [collide + B](dt) o A(dt/2) (Sec. 4);
* transport sub-cycling so that |nu| = |v_x| tau / dx <= 1;
* minmod per real Pauli component; ghost cells two per side (periodic wrap;
  Dirichlet: Phi for incoming v, copy of the boundary cell otherwise;
  Maxwell: (1-alpha) W_b(-v_x, v_y) + alpha W_FD Fbar/Z for incoming v, the
  unpaired column k_x = -N/2 at x = 1 receiving only the diffusive part).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

ETA = np.array([1.0, -1.0, -1.0, -1.0])
SIGMA = np.array(
    [[[1, 0], [0, 1]], [[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]],
    dtype=np.complex128,
)
LEVI_CIVITA = [(1, 2, 3, 1.0), (1, 3, 2, -1.0), (2, 3, 1, 1.0), (2, 1, 3, -1.0), (3, 1, 2, 1.0), (3, 2, 1, -1.0)]


@dataclass(frozen=True)
class Params:
    """Discretisation parameters (Sec. 3.2 and Sec. 5: L=12, R=7.5, J=M=32)."""

    N: int
    L: float = 12.0
    R: float = 7.5
    J: int = 32
    M: int = 32
    nyquist: str = "zero"

    def __post_init__(self):
        if self.N % 2 or self.N < 4:
            raise ValueError("N must be even and >= 4")
        if self.J % 2 or self.J < 2:
            raise ValueError("J must be even (staggered grid theta'_j never orthogonal to theta_j)")
        if self.nyquist not in ("zero", "keep"):
            raise ValueError("nyquist must be 'zero' or 'keep'")


# ----------------------------------------------------------------------------
# Grids (Sec. 3.2, eq. fourier_grid; Sec. 5.1: v in (2L/N) Xi)
# ----------------------------------------------------------------------------

def xi_axis(p: Params) -> np.ndarray:
    return np.arange(-p.N // 2, p.N // 2)


def velocity_nodes(p: Params):
    a = (2.0 * p.L / p.N) * xi_axis(p)
    return np.meshgrid(a, a, indexing="ij")


def delta_v(p: Params) -> float:
    return 2.0 * p.L / p.N


def sigma_mesh(p: Params):
    """Frequencies sigma in [-N, N-1]^2 of the padded grid, index s = sigma + N."""
    s = np.arange(-p.N, p.N)
    return np.meshgrid(s, s, indexing="ij")


# ----------------------------------------------------------------------------
# Fourier coefficients on Xi and the padded grid (Sec. 3.2)
# ----------------------------------------------------------------------------

def coarse_to_xi(f: np.ndarray, p: Params) -> np.ndarray:
    """fhat(xi) = N^-2 sum_k f(v_k) exp(-i pi xi.v_k/L), written as the explicit sum."""
    k = xi_axis(p)
    E = np.exp(-2j * np.pi * np.outer(k, k) / p.N)       # E[xi, k] = e^{-i pi xi (2L/N) k / L}
    fh = np.einsum("ak,...kl,bl->...ab", E, f, E) / p.N**2
    if p.nyquist == "zero":
        fh = fh.copy()
        fh[..., 0, :] = 0.0
        fh[..., :, 0] = 0.0
    return fh


def xi_to_coarse(fh: np.ndarray, p: Params) -> np.ndarray:
    """f(v_k) = sum_{xi in Xi} fhat(xi) exp(i pi xi.v_k/L) (explicit sum)."""
    k = xi_axis(p)
    E = np.exp(2j * np.pi * np.outer(k, k) / p.N)        # E[k, xi]
    return np.einsum("ka,...ab,lb->...kl", E, fh, E)


def embed(fh: np.ndarray, p: Params) -> np.ndarray:
    """Place coefficients on Xi into the padded frequency array [..., 2N, 2N] (zero padding)."""
    N = p.N
    out = np.zeros(fh.shape[:-2] + (2 * N, 2 * N), dtype=np.complex128)
    out[..., N // 2: 3 * N // 2, N // 2: 3 * N // 2] = fh
    return out


def restrict(c: np.ndarray, p: Params) -> np.ndarray:
    """Keep the coefficients with sigma in Xi (truncation to the Fourier grid)."""
    N = p.N
    return c[..., N // 2: 3 * N // 2, N // 2: 3 * N // 2]


def to_fine(c: np.ndarray, p: Params) -> np.ndarray:
    """Evaluate sum_sigma c(sigma) exp(i pi sigma.v'/L) at v' = (L/N) k', k' in [-N,N-1]^2."""
    M2 = 2 * p.N
    ax = (-2, -1)
    return (M2 * M2) * np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(c, axes=ax), axes=ax), axes=ax)


def from_fine(f: np.ndarray, p: Params) -> np.ndarray:
    """Averaged coefficients c(sigma) = (2N)^-2 sum_k' f(v'_k') exp(-i pi sigma.v'/L)."""
    M2 = 2 * p.N
    ax = (-2, -1)
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(f, axes=ax), axes=ax), axes=ax) / (M2 * M2)


def conv(a: np.ndarray, b: np.ndarray, p: Params) -> np.ndarray:
    """(a * b)(sigma) = sum_{chi + eta = sigma} a(chi) b(eta), via the padded grid."""
    return from_fine(to_fine(a, p) * to_fine(b, p), p)


# ----------------------------------------------------------------------------
# Kernel quadratures (Sec. 3.2)
# ----------------------------------------------------------------------------

def theta(p: Params) -> np.ndarray:
    """theta_j = exp(i (j-1) pi / J), j = 1..J, as unit vectors [J, 2] (eq. theta_grid)."""
    t = np.arange(p.J) * np.pi / p.J
    return np.stack([np.cos(t), np.sin(t)], axis=-1)


def theta_prime(p: Params) -> np.ndarray:
    """theta'_j = exp(i (j-1/2) pi / J) (eq. theta_grid)."""
    t = (np.arange(p.J) + 0.5) * np.pi / p.J
    return np.stack([np.cos(t), np.sin(t)], axis=-1)


def perp(th: np.ndarray) -> np.ndarray:
    """Rotation by pi/2."""
    return np.stack([-th[..., 1], th[..., 0]], axis=-1)


def phi_R(s: np.ndarray, p: Params) -> np.ndarray:
    """phi_R(s) = int_0^R sin(pi s r/L) dr = (2L/(pi s)) sin^2(pi s R/(2L)); phi_R(0) = 0."""
    s = np.asarray(s, dtype=np.float64)
    safe = np.where(s == 0.0, 1.0, s)
    val = (2.0 * p.L / (np.pi * safe)) * np.sin(np.pi * safe * p.R / (2.0 * p.L)) ** 2
    return np.where(s == 0.0, 0.0, val)


def psi_R(s: np.ndarray, p: Params) -> np.ndarray:
    """psi_R(s) = int_{-R}^{R} exp(i pi s r/L) dr = (2L/(pi s)) sin(pi R s/L); psi_R(0) = 2R."""
    s = np.asarray(s, dtype=np.float64)
    safe = np.where(s == 0.0, 1.0, s)
    val = (2.0 * p.L / (np.pi * safe)) * np.sin(np.pi * p.R * safe / p.L)
    return np.where(s == 0.0, 2.0 * p.R, val)


def omega_G(p: Params) -> np.ndarray:
    """omega_{G,j,j'} = -(2 pi/J)^2 / (theta_j . theta'_j') (eq. approxG)."""
    return -((2.0 * np.pi / p.J) ** 2) / (theta(p) @ theta_prime(p).T)


def gauss_legendre(p: Params):
    """Gauss-Legendre nodes rho_{R,m} and weights w_{R,m} on [-R, R] (eq. approxH-JM)."""
    x, w = np.polynomial.legendre.leggauss(p.M)
    return p.R * x, p.R * w


def phi_tables(p: Params):
    """phi_{R,j}(sigma) and phi'_{R,j'}(sigma) on the padded frequency grid."""
    SX, SY = sigma_mesh(p)
    th, thp = theta(p), theta_prime(p)
    phi = np.stack([phi_R(SX * t[0] + SY * t[1], p) for t in th])
    phip = np.stack([phi_R(SX * t[0] + SY * t[1], p) for t in thp])
    return phi, phip


def psi_tables(p: Params):
    """psi_{R,j}(sigma) = psi_R(sigma.theta_j), psi'_{R,j}(sigma) = psi_R(sigma.theta_j^perp) (eq. approxH-J)."""
    SX, SY = sigma_mesh(p)
    th = theta(p)
    tp = perp(th)
    psi = np.stack([psi_R(SX * t[0] + SY * t[1], p) for t in th])
    psip = np.stack([psi_R(SX * t[0] + SY * t[1], p) for t in tp])
    return psi, psip


# ----------------------------------------------------------------------------
# The four integral types in Fourier form (Sec. 3.2).  Arguments are embedded
# coefficient arrays (zero outside Xi); results are embedded, zero outside Xi.
# ----------------------------------------------------------------------------

def _keep_xi(c: np.ndarray, p: Params) -> np.ndarray:
    return embed(restrict(c, p), p)


def I1(fh, gh, hh, p: Params):
    """I1(v) = int int P(1/(u.u')) f(v+u) g(v+u+u') h(v) du du' with G from eq. approxG.

    hat I1(xi) = sum_{j,j'} omega_G[j,j'] sum_zeta [ sum_eta fhat(xi-zeta-eta) phi'_j'(eta) ghat(eta) ]
                 phi_j(xi - zeta) hhat(zeta); for each (j, j') two convolutions.
    """
    phi, phip = phi_tables(p)
    wG = omega_G(p)
    out = 0.0
    for jp in range(p.J):
        A = conv(fh, phip[jp] * gh, p)
        for j in range(p.J):
            out = out + conv(wG[j, jp] * phi[j] * A, hh, p)
    return _keep_xi(out, p)


def I2(fh, gh, hh, p: Params):
    """I2(v) = int int delta(u.u') f(v+u) g(v+u') h(v), H from eq. approxH-J (omega_H = pi/J).

    hat I2(xi) = sum_j omega_H sum_zeta sum_{chi+eta=xi-zeta} (psi_j fhat)(chi) (psi'_j ghat)(eta) hhat(zeta).
    """
    psi, psip = psi_tables(p)
    out = 0.0
    for j in range(p.J):
        A = conv(psi[j] * fh, psip[j] * gh, p)
        out = out + (np.pi / p.J) * conv(A, hh, p)
    return _keep_xi(out, p)


def I4(fh, gh, hh, p: Params):
    """I4(v) = int int delta(u.u') f(v+u) g(v+u+u') h(v): kernel H(chi+eta, eta) (like I1, with H_J)."""
    psi, psip = psi_tables(p)
    out = 0.0
    for j in range(p.J):
        A = conv(fh, psip[j] * gh, p)
        out = out + conv((np.pi / p.J) * psi[j] * A, hh, p)
    return _keep_xi(out, p)


def I3(fh, gh, hh, p: Params):
    """I3(v) = int int delta(u.u') f(v+u) g(v+u') h(v+u+u') via the Hu-Ying form eq. approxH-JM.

    hat I3(xi) = sum_{j,m} tilde omega_{H,j,m} sum_chi (e^{i alpha_jm.chi} fhat(chi)) psi'_j(xi-chi)
                 sum_{eta+zeta=xi-chi} ghat(eta) (e^{i alpha_jm.zeta} hhat(zeta)),
    tilde omega_{H,j,m} = (pi/J) w_{R,m},  alpha_{j,m} = pi rho_{R,m} theta_j / L.
    The m-loop is evaluated as one array axis.
    """
    SX, SY = sigma_mesh(p)
    th = theta(p)
    _, psip = psi_tables(p)
    rho, wR = gauss_legendre(p)
    batch = fh.ndim - 2
    out = 0.0
    for j in range(p.J):
        ax_ = np.pi * rho * th[j, 0] / p.L
        ay_ = np.pi * rho * th[j, 1] / p.L
        phase = np.exp(1j * (ax_[:, None, None] * SX[None] + ay_[:, None, None] * SY[None]))  # [M,2N,2N]
        phase = phase.reshape((p.M,) + (1,) * batch + phase.shape[1:])
        inner = conv(gh[None], phase * hh[None], p)                 # sum_{eta+zeta} g(eta) e^{i a.zeta} h(zeta)
        term = conv(phase * fh[None], psip[j] * inner, p)           # sum_chi (e^{i a.chi} f)(chi) psi'(xi-chi) inner
        wt = ((np.pi / p.J) * wR).reshape((p.M,) + (1,) * (batch + 2))
        out = out + np.sum(wt * term, axis=0)
    return _keep_xi(out, p)


# ----------------------------------------------------------------------------
# Collision operator in Pauli form after the Carleman change of variables
# (eq. CcPauliCarleman and the Carleman form of eq. CdPauli, Sec. 3.1-3.2)
# ----------------------------------------------------------------------------

def collision_terms(wh: np.ndarray, p: Params):
    """The Pauli-form collision operator as a list of integral terms.

    Each entry (part, component, coefficient, kind, f, g, h) contributes
    coefficient * I_kind[f, g, h] to component `component` of C_c (part "c") or
    C_d (part "d"); wh [..., 4, 2N, 2N] are embedded Pauli coefficients.
    """
    N = p.N
    one = np.zeros(wh.shape[:-3] + (2 * N, 2 * N), dtype=np.complex128)
    one[..., N, N] = 1.0                                       # the constant function 1
    w = [wh[..., a, :, :] for a in range(4)]
    ew = [ETA[a] * w[a] for a in range(4)]                      # (eta w)_a
    f = 2.0 * w[0] - one                                       # 2 w0 - 1
    terms = []
    # Conservative part: i (2w0(v+u) - 1) [W(v+u+u'), W(v)] with -i[W2, W1] = 2 (w2 x w1).sigma
    for (c, d, e, s) in LEVI_CIVITA:
        terms.append(("c", c, -2.0 * s, "I1", f, w[d], w[e]))
    # Dissipative part, first term: 2 pi <w(v+u), w(v+u')>_eta (1 - W(v))
    for c in range(4):
        h = (one if c == 0 else 0.0 * one) - w[c]
        for a in range(4):
            terms.append(("d", c, 2.0 * np.pi * ETA[a], "I2", w[a], w[a], h))
    # second term: -2 pi <w(v+u), w(v+u')>_eta (eta w(v+u+u')).sigma
    for c in range(4):
        for a in range(4):
            terms.append(("d", c, -2.0 * np.pi * ETA[a], "I3", w[a], w[a], ew[c]))
    # third term: pi (2 w0(v+u) - 1) {W(v), (eta w(v+u+u')).sigma}, with
    # {W1, W2} = 2((w1_0 w2 + w2_0 w1).sigma - <w1, w2>_eta 1)
    terms.append(("d", 0, 4.0 * np.pi, "I4", f, ew[0], w[0]))
    for a in range(4):
        terms.append(("d", 0, -2.0 * np.pi * ETA[a], "I4", f, ew[a], w[a]))
    for c in range(1, 4):
        terms.append(("d", c, 2.0 * np.pi, "I4", f, ew[c], w[0]))
        terms.append(("d", c, 2.0 * np.pi, "I4", f, ew[0], w[c]))
    return terms


_INTEGRALS = {"I1": I1, "I2": I2, "I3": I3, "I4": I4}


def evaluate_term(args):
    """Evaluate one (kind, f, g, h, params) integral term (usable with any map)."""
    kind, f, g, h, p = args
    return _INTEGRALS[kind](f, g, h, p)


def collision_xi(wh: np.ndarray, p: Params, mapper=map):
    """C[W] on Xi from embedded Pauli coefficients wh [..., 4, 2N, 2N]; returns (Cc_hat, Cd_hat).

    The terms are independent; `mapper` (default: the builtin map) may evaluate
    them concurrently.  They are summed in list order.
    """
    terms = collision_terms(wh, p)
    values = list(mapper(evaluate_term, [(t[3], t[4], t[5], t[6], p) for t in terms]))
    Cc = np.zeros_like(wh)
    Cd = np.zeros_like(wh)
    for (part, c, coef, _kind, _f, _g, _h), v in zip(terms, values):
        tgt = Cc if part == "c" else Cd
        tgt[..., c, :, :] += coef * v
    return Cc, Cd


def collision_parts(w: np.ndarray, p: Params, mapper=map):
    """(C_c, C_d) on the velocity grid for Pauli states w [..., 4, N, N] (real)."""
    wh = embed(coarse_to_xi(w.astype(np.complex128), p), p)
    Cc_h, Cd_h = collision_xi(wh, p, mapper)
    out = []
    for Ch in (Cc_h, Cd_h):
        cx = restrict(Ch, p).copy()
        if p.nyquist == "zero":
            cx[..., 0, :] = 0.0
            cx[..., :, 0] = 0.0
        out.append(xi_to_coarse(cx, p))
    return out[0], out[1]


def collision(w: np.ndarray, p: Params, return_imag: bool = False, mapper=map):
    """C[W] = C_c + C_d on the grid (real part; imaginary residue optionally returned)."""
    Cc, Cd = collision_parts(w, p, mapper)
    C = Cc + Cd
    if return_imag:
        return C.real.copy(), C.imag.copy()
    return C.real.copy()


# ----------------------------------------------------------------------------
# Precession -i[B.sigma, W] = 2 (B x w).sigma (eq. boltzmann, Pauli commutator of Sec. 3.1)
# ----------------------------------------------------------------------------

def precession(w: np.ndarray, B: np.ndarray) -> np.ndarray:
    """w [Nx,4,N,N], B [Nx,3] -> 2 (B x w_vec) in components 1..3, 0 in component 0."""
    out = np.zeros_like(w)
    b = B[:, :, None, None]
    out[:, 1] = 2.0 * (b[:, 1] * w[:, 3] - b[:, 2] * w[:, 2])
    out[:, 2] = 2.0 * (b[:, 2] * w[:, 1] - b[:, 0] * w[:, 3])
    out[:, 3] = 2.0 * (b[:, 0] * w[:, 2] - b[:, 1] * w[:, 1])
    return out


# ----------------------------------------------------------------------------
# Fermi-Dirac states (eq. W_FermiDirac) and moments (eq. density, velocity, energy)
# ----------------------------------------------------------------------------

def fermi_dirac_pauli(beta, mu_up, mu_dn, U, p: Params) -> np.ndarray:
    """W_FD(v) = sum_s (e^{beta(|v|^2/2 - mu_s)} + 1)^{-1} |s><s|, |s> the columns of U; [4,N,N]."""
    vx, vy = velocity_nodes(p)
    e = 0.5 * (vx**2 + vy**2)
    n = [1.0 / (np.exp(beta * (e - mu)) + 1.0) for mu in (mu_up, mu_dn)]
    U = np.asarray(U, dtype=np.complex128)
    Wm = np.zeros(vx.shape + (2, 2), dtype=np.complex128)
    for s in range(2):
        u = U[:, s]
        Wm += n[s][..., None, None] * np.outer(u, np.conj(u))[None, None]
    w = 0.5 * np.einsum("xyij,cji->cxy", Wm, SIGMA)
    return w.real.copy()


def moments(w: np.ndarray, p: Params):
    """Per cell: rho (4 Pauli comps of int W dv), momentum int v tr W dv (2), energy int |v|^2/2 tr W dv."""
    vx, vy = velocity_nodes(p)
    dv2 = delta_v(p) ** 2
    rho = dv2 * w.sum(axis=(-2, -1))
    trW = 2.0 * w[..., 0, :, :]
    mom = dv2 * np.stack([(vx * trW).sum(axis=(-2, -1)), (vy * trW).sum(axis=(-2, -1))], axis=-1)
    en = dv2 * (0.5 * (vx**2 + vy**2) * trW).sum(axis=(-2, -1))
    return rho, mom, en


# ----------------------------------------------------------------------------
# Transport: minmod slope-limiter finite volumes (Sec. 4, eq. slopeLimiterStep, eq. minmod)
# with boundary ghost cells from Sec. 2 (periodic, Dirichlet, Maxwell)
# ----------------------------------------------------------------------------

@dataclass
class Boundary:
    kind: str = "periodic"          # "periodic" | "dirichlet" | "maxwell"
    left: tuple | None = None       # (beta, mu_up, mu_dn, U) of the wall Fermi-Dirac state
    right: tuple | None = None
    alpha: float = 0.0              # Maxwell accommodation coefficient


def minmod(a, b):
    """eq. minmod: a if |a|<=|b| and ab>0; b if |b|<|a| and ab>0; 0 if ab<=0."""
    return np.where(a * b > 0.0, np.where(np.abs(a) <= np.abs(b), a, b), 0.0)


def _ghosts(W, p: Params, bc: Boundary):
    """Two ghost cells on each side; returns the extended array [Nx+4, 4, N, N]."""
    vx, vy = velocity_nodes(p)
    Nx = W.shape[0]
    ext = np.empty((Nx + 4,) + W.shape[1:])
    ext[2:Nx + 2] = W
    if bc.kind == "periodic":
        ext[0:2] = W[Nx - 2:Nx]
        ext[Nx + 2:] = W[0:2]
        return ext
    # outgoing (and v_x = 0): copy of the boundary cell
    ext[0:2] = W[0]
    ext[Nx + 2:] = W[Nx - 1]
    inL = vx > 0.0                 # incoming at x = 0 (n = -1)
    inR = vx < 0.0                 # incoming at x = 1 (n = +1)
    if bc.kind == "dirichlet":
        PhiL = fermi_dirac_pauli(*bc.left, p)
        PhiR = fermi_dirac_pauli(*bc.right, p)
        for g in (0, 1):
            ext[g][:, inL] = PhiL[:, inL]
            ext[Nx + 2 + g][:, inR] = PhiR[:, inR]
        return ext
    if bc.kind == "maxwell":
        dv2 = delta_v(p) ** 2
        a = bc.alpha
        N = p.N
        for side in ("L", "R"):
            Wb = W[0] if side == "L" else W[Nx - 1]
            fd = fermi_dirac_pauli(*(bc.left if side == "L" else bc.right), p)
            n = -1.0 if side == "L" else 1.0
            out_mask = (vx * n) > 0.0
            in_mask = (vx * n) < 0.0
            Fbar = dv2 * np.sum(2.0 * Wb[0][out_mask] * np.abs(vx[out_mask]))   # outgoing number flux
            Z = dv2 * np.sum(2.0 * fd[0][in_mask] * np.abs(vx[in_mask]))         # normalisation
            refl = np.zeros_like(Wb)            # L_x F (v_x, v_y) = F(-v_x, v_y); k_x -> -k_x
            for ix in range(N):
                mx = N - ix                     # index of -k_x: k = ix - N/2 -> -k -> N/2 - k + ... = N - ix
                if 0 <= mx < N:
                    refl[:, ix, :] = Wb[:, mx, :]
            ghost = (1.0 - a) * refl + a * fd * (Fbar / Z)
            for g in (0, 1):
                tgt = ext[g] if side == "L" else ext[Nx + 2 + g]
                tgt[:, in_mask] = ghost[:, in_mask]
        return ext
    raise ValueError(bc.kind)


def limiter_update(ext, tau, dx, p: Params):
    """eq. slopeLimiterStep (Delta t -> tau) on the interior of ext [n+4, 4, N, N] (two ghosts per side)."""
    vx, _ = velocity_nodes(p)
    n = ext.shape[0] - 4
    # S_j for j = -1 .. n (ext indices 1 .. n+2)
    S = np.zeros_like(ext)
    S[1:n + 3] = minmod(ext[2:n + 4] - ext[1:n + 3], ext[1:n + 3] - ext[0:n + 2])
    nu = tau * vx / dx
    lim = 0.5 * (np.sign(nu) - nu)
    Wm1, W0, Wp1 = ext[1:n + 1], ext[2:n + 2], ext[3:n + 3]
    Sm1, S0, Sp1 = S[1:n + 1], S[2:n + 2], S[3:n + 3]
    godunov = -vx * (Wp1 - Wm1) + np.abs(vx) * (Wp1 - 2.0 * W0 + Wm1)
    limiter = lim * (-vx * (Sp1 - Sm1) + np.abs(vx) * (Sp1 - 2.0 * S0 + Sm1))
    return W0 + (tau / (2.0 * dx)) * (godunov + limiter)


def advect_substep(W, tau, dx, p: Params, bc: Boundary):
    """One application of eq. slopeLimiterStep with time step tau (Delta t -> tau)."""
    return limiter_update(_ghosts(W, p, bc), tau, dx, p)


def transport_substeps(tau, dx, p: Params, nu_max: float = 1.0) -> int:
    """Sub-steps so that max |v_x| tau_sub / dx <= nu_max (max |v_x| on the grid is L)."""
    nu = abs(tau) * p.L / dx
    return max(1, int(np.ceil(nu / nu_max - 1e-12)))


def advect(W, tau, p: Params, bc: Boundary):
    """Transport operator A(tau) (sub-cycled)."""
    Nx = W.shape[0]
    dx = 1.0 / Nx
    s = transport_substeps(tau, dx, p)
    for _ in range(s):
        W = advect_substep(W, tau / s, dx, p, bc)
    return W


# ----------------------------------------------------------------------------
# Collision + precession substep (Heun's RK2) and the split time step (Sec. 4)
# ----------------------------------------------------------------------------

def rhs(W, B, p: Params):
    return collision(W, p) + precession(W, B)


def collide_rk2(W, B, dt, p: Params):
    F0 = rhs(W, B, p)
    W1 = W + dt * F0
    F1 = rhs(W1, B, p)
    return W + 0.5 * dt * (F0 + F1)


def step(W, B, dt, p: Params, bc: Boundary):
    """A(dt/2) o RK2[C + B](dt) o A(dt/2)."""
    W = advect(W, 0.5 * dt, p, bc)
    W = collide_rk2(W, B, dt, p)
    W = advect(W, 0.5 * dt, p, bc)
    return W
