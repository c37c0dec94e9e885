"""Diagnostics of a Wigner state: entropy, Fermi-Dirac fit, quantum relative
entropy and L1 distance (Lu & Mendl, Sec. 2 and Sec. 5).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests, the smoke
check and the benchmark's CPU baseline may import it.  Plain definitions in
FP64 with library primitives as steps (numpy's eigh for 2x2 Hermitian
eigenpairs, scipy's spence for the dilogarithm, scipy's brentq for the
scalar fit).

* Entropy (eq. entropy_def): S[W](x) = -int tr[W log W + W~ log W~] dv,
  W~ = 1 - W, on the grid as dv^2 sum_v (0 log 0 = 0).
* Fermi-Dirac state (eq. W_FermiDirac) with a mean velocity u (Sec. 5.2: the
  average velocity shifts W_FD(v) -> W_FD(v - u)):
  W_FD(v) = sum_s (exp((|v - u|^2/2 - mu_s)/T) + 1)^-1 |s><s|.
* Fit (Sec. 5.2): the eigenbasis of W_FD is that of the spin density rho
  (eq. density); T, mu_up, mu_dn match the eigenvalues of rho and the
  internal energy through the closed forms eq. momentsFermiDirac,
  rho_s = 2 pi T log(1 + e^{mu_s/T}), eps = T (-sum_s Li2(-e^{mu_s/T})) /
  sum_s log(1 + e^{mu_s/T}), eps = (int |v - u|^2/2 tr W dv) / tr rho
  (eq. internal_energy), u = (int v tr W dv) / tr rho (eq. velocity).
  Readings: the up state takes the larger eigenvalue of rho; the moments are
  the grid sums (dv^2 sum_v); the global fit uses the x-averaged moments.
* Quantum relative entropy (eq. relentropy_hom):
  S(W || W_FD) = int tr[W (log W - log W_FD) + W~ (log W~ - log W~_FD)] dv,
  and over x (eqs. relentropy_inhom, relentropy_local) the average over cells
  (dx = 1/Nx, the x-domain has length 1).
* L1 distance (Fig. 4c): int ||W(v) - W_FD(v)||_1 dv with the trace norm
  (sum of absolute eigenvalues) of the 2x2 difference (reading: the paper does
  not name the matrix norm).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.optimize import brentq
from scipy.special import spence

from . import qbe_oracle as O


def pauli_to_matrix(w):
    """[..., 4] Pauli components -> [..., 2, 2] complex matrices (eq. spin_repr)."""
    return np.einsum("...a,aij->...ij", w.astype(np.complex128), O.SIGMA)


def _xlogx(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    pos = x > 0.0
    out[pos] = x[pos] * np.log(x[pos])
    return out


def entropy(W, p: O.Params):
    """Local entropy per cell, [Nx]."""
    Wm = pauli_to_matrix(np.moveaxis(W, 1, -1))          # [Nx, N, N, 2, 2]
    lam = np.linalg.eigvalsh(Wm)
    dens = -(_xlogx(lam) + _xlogx(1.0 - lam)).sum(axis=-1)
    return O.delta_v(p) ** 2 * dens.sum(axis=(-2, -1))


def li2(z):
    """Dilogarithm Li2(z) for real z <= 1 (scipy's spence: Li2(z) = spence(1 - z))."""
    return spence(1.0 - z)


def fd_density(T, mu):
    """rho_s = 2 pi T log(1 + e^{mu/T}) (eq. momentsFermiDirac, per spin state)."""
    return 2.0 * np.pi * T * np.logaddexp(0.0, mu / T)


def neg_li2_neg_exp(t):
    """-Li2(-e^t) for real t; for t > 0 by the inversion Li2(-z) + Li2(-1/z) = -pi^2/6 - log(z)^2/2."""
    if t <= 0.0:
        return -li2(-np.exp(t))
    return np.pi**2 / 6.0 + 0.5 * t * t + li2(-np.exp(-t))


def fd_energy(T, mus):
    """eps = T (-sum_s Li2(-e^{mu_s/T})) / sum_s log(1 + e^{mu_s/T}) (eq. momentsFermiDirac)."""
    num = sum(neg_li2_neg_exp(m / T) for m in mus)
    den = sum(np.logaddexp(0.0, m / T) for m in mus)
    return T * num / den


def _log_expm1(a):
    """log(e^a - 1) for a > 0 without overflow."""
    return np.log(np.expm1(a)) if a < 30.0 else a + np.log(-np.expm1(-a))


@dataclass
class FDFit:
    T: float
    mu_up: float
    mu_dn: float
    U: np.ndarray          # columns |up>, |down>
    u: np.ndarray          # mean velocity (2)
    ok: bool = True


def moments_of(W, p: O.Params):
    """(rho as 2x2, momentum (2), energy) of one cell's state [4, N, N] as grid sums."""
    rho4, mom, en = O.moments(W[None], p)
    return pauli_to_matrix(rho4[0]), mom[0], en[0]


def fit_from_moments(rho, mom, energy) -> FDFit:
    """Fermi-Dirac state with the same spin density, momentum and energy (Sec. 5.2)."""
    lam, vec = np.linalg.eigh(rho)                    # ascending
    r_up, r_dn = lam[1], lam[0]
    U = vec[:, ::-1]                                  # up = larger eigenvalue
    tr = r_up + r_dn
    u = np.asarray(mom) / tr
    eps = energy / tr - 0.5 * float(u @ u)
    if not (r_dn > 0.0 and eps > 0.0):
        return FDFit(np.nan, np.nan, np.nan, U, u, ok=False)

    def mus(T):
        # rho_s = 2 pi T log(1 + e^{mu_s/T})  =>  mu_s = T log(e^{rho_s/(2 pi T)} - 1)
        return [T * _log_expm1(r / (2.0 * np.pi * T)) for r in (r_up, r_dn)]

    f = lambda lt: fd_energy(np.exp(lt), mus(np.exp(lt))) - eps
    eps0 = (r_up**2 + r_dn**2) / (4.0 * np.pi * tr)   # T -> 0 limit (both states filled to their Fermi level)
    if eps <= eps0:
        return FDFit(0.0, np.nan, np.nan, U, u, ok=False)
    lo, hi = np.log(eps), np.log(eps) + 1.0
    while f(lo) > 0.0:
        lo -= 2.0
    while f(hi) < 0.0:
        hi += 2.0
    T = float(np.exp(brentq(f, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)))
    mu_up, mu_dn = mus(T)
    return FDFit(T, float(mu_up), float(mu_dn), U, u)


def fit_local(W, p: O.Params):
    return [fit_from_moments(*moments_of(W[j], p)) for j in range(W.shape[0])]


def fit_global(W, p: O.Params) -> FDFit:
    """One Fermi-Dirac state for the x-averaged moments (dx = 1/Nx)."""
    rho4, mom, en = O.moments(W, p)
    return fit_from_moments(pauli_to_matrix(rho4.mean(axis=0)), mom.mean(axis=0), en.mean(axis=0))


def fd_occupations(fit: FDFit, p: O.Params):
    """n_up(v), n_dn(v) of W_FD(v - u), [2, N, N]."""
    vx, vy = O.velocity_nodes(p)
    e = 0.5 * ((vx - fit.u[0]) ** 2 + (vy - fit.u[1]) ** 2)
    return np.stack([1.0 / (np.exp((e - m) / fit.T) + 1.0) for m in (fit.mu_up, fit.mu_dn)])


def fd_state(fit: FDFit, p: O.Params):
    """W_FD(v - u) as 2x2 matrices [N, N, 2, 2]."""
    n = fd_occupations(fit, p)
    out = np.zeros(n.shape[1:] + (2, 2), dtype=np.complex128)
    for s in range(2):
        out += n[s][..., None, None] * np.outer(fit.U[:, s], np.conj(fit.U[:, s]))[None, None]
    return out


def relative_entropy_cell(Wc, fit: FDFit, p: O.Params):
    """S(W || W_FD) of one cell's state [4, N, N] (eq. relentropy_hom).

    tr[X log X] from the eigenvalues of X; tr[X log F] = sum_s <s|X|s> log n_s from the spectral form
    of F = W_FD (its eigenvalues n_s(v) are known exactly, down to the 1e-39 of the tails)."""
    Wm = pauli_to_matrix(np.moveaxis(Wc, 0, -1))           # [N, N, 2, 2]
    n = fd_occupations(fit, p)
    I = np.eye(2)
    total = 0.0
    for X, occ in ((Wm, n), (I - Wm, 1.0 - n)):
        lam = np.linalg.eigvalsh(X)
        total += float(_xlogx(lam).sum())
        for s in range(2):
            u = fit.U[:, s]
            diag = np.einsum("i,xyij,j->xy", np.conj(u), X, u).real
            total -= float(np.sum(diag * np.log(occ[s])))
    return O.delta_v(p) ** 2 * total


def l1_distance_cell(Wc, fit: FDFit, p: O.Params):
    Wm = pauli_to_matrix(np.moveaxis(Wc, 0, -1))
    D = Wm - fd_state(fit, p)
    return O.delta_v(p) ** 2 * float(np.abs(np.linalg.eigvalsh(D)).sum())


def relative_entropy(W, fits, p: O.Params):
    """Per cell S(W(x) || fits[x]) (one fit: the same state for every cell)."""
    fits = fits if isinstance(fits, (list, tuple)) else [fits] * W.shape[0]
    return np.array([relative_entropy_cell(W[j], fits[j], p) for j in range(W.shape[0])])


def l1_distance(W, fits, p: O.Params):
    fits = fits if isinstance(fits, (list, tuple)) else [fits] * W.shape[0]
    return np.array([l1_distance_cell(W[j], fits[j], p) for j in range(W.shape[0])])
