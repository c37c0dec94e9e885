"""Pins of the oracle's diagnostics (oracle/diagnostics.py) on closed forms and
exact identities of the paper (Sec. 2, Sec. 5).  CPU only."""
import numpy as np
import pytest

from oracle import diagnostics as D
from oracle import qbe_oracle as O
from paper_1408_1782_gb300 import inputs


def rotation(theta, phi):
    """A 2x2 unitary whose first column is the spin state along (theta, phi)."""
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -s * np.exp(-1j * phi)], [s * np.exp(1j * phi), c]], dtype=np.complex128)


def fd_cell(fit, p):
    """Pauli components [4, N, N] of W_FD(v - u)."""
    Fm = D.fd_state(fit, p)
    return np.moveaxis(0.5 * np.einsum("xyij,aji->xya", Fm, O.SIGMA).real, -1, 0).copy()


def test_dilogarithm_special_values():
    assert abs(D.li2(-1.0) + np.pi**2 / 12) < 1e-15
    assert abs(D.li2(1.0) - np.pi**2 / 6) < 1e-15
    assert abs(D.li2(0.5) - (np.pi**2 / 12 - 0.5 * np.log(2) ** 2)) < 1e-15


def test_entropy_of_fermi_dirac_state_matches_thermodynamics():
    """In 2-D with omega = |v|^2/2 the grand potential is -E, so S = sum_s (2 E_s - mu_s N_s)/T with
    N_s = 2 pi T log(1 + z_s), E_s = 2 pi T^2 (-Li2(-z_s)), z_s = e^{mu_s/T} (eq. momentsFermiDirac).
    The grid sum is a trapezoidal rule: its error is ~exp(-2 pi d / dv) with d the distance of the
    Fermi function's nearest complex singularity (|v|^2 = 2 mu + 2 pi i T) from the real axis, here
    d ~ 1.4, dv = 0.375: ~1e-10."""
    p = O.Params(N=64, L=12.0)
    fit = D.FDFit(T=0.8, mu_up=0.7, mu_dn=-0.4, U=rotation(0.9, 0.3), u=np.zeros(2))
    W = fd_cell(fit, p)[None]
    S = D.entropy(W, p)[0]
    ref = 0.0
    for mu in (fit.mu_up, fit.mu_dn):
        z = np.exp(mu / fit.T)
        Ns = 2 * np.pi * fit.T * np.log1p(z)
        Es = 2 * np.pi * fit.T**2 * (-D.li2(-z))
        ref += (2 * Es - mu * Ns) / fit.T
    assert abs(S - ref) < 1e-9 * ref


@pytest.mark.parametrize("N,T,mu_up,mu_dn,u", [(64, 0.8, 0.7, -0.4, (0.0, 0.0)), (64, 1.6, -0.5, 1.2, (0.3, -0.2)),
                                                (128, 0.4, 1.5, 1.0, (-0.1, 0.25))])
def test_fit_recovers_a_fermi_dirac_state(N, T, mu_up, mu_dn, u):
    """The fit matches continuum moments (eq. momentsFermiDirac) to the grid moments, whose quadrature
    error exp(-2 pi d/dv) (d ~ 0.7 sqrt(T)-ish distance of the Fermi function's complex singularity) is
    below 1e-9 on these grids; T = 0.4 needs N = 128 (at N = 64 it is 1e-5)."""
    p = O.Params(N=N, L=12.0)
    fit = D.FDFit(T=T, mu_up=mu_up, mu_dn=mu_dn, U=rotation(1.1, -0.7), u=np.array(u))
    W = fd_cell(fit, p)
    got = D.fit_from_moments(*D.moments_of(W, p))
    assert got.ok
    assert abs(got.T - T) < 1e-9 * T
    hi, lo = (mu_up, mu_dn) if mu_up > mu_dn else (mu_dn, mu_up)
    assert abs(got.mu_up - hi) < 1e-8 and abs(got.mu_dn - lo) < 1e-8
    assert np.abs(got.u - np.array(u)).max() < 1e-10
    # same spin projectors
    U = fit.U if mu_up > mu_dn else fit.U[:, ::-1]
    for s in range(2):
        P1 = np.outer(U[:, s], U[:, s].conj())
        P2 = np.outer(got.U[:, s], got.U[:, s].conj())
        assert np.abs(P1 - P2).max() < 1e-10


def test_relative_entropy_of_a_state_to_itself_is_zero_and_l1_too():
    p = O.Params(N=16)
    fit = D.FDFit(T=1.0, mu_up=0.3, mu_dn=-0.2, U=rotation(0.4, 1.0), u=np.array([0.1, 0.0]))
    W = fd_cell(fit, p)[None]
    assert abs(D.relative_entropy(W, fit, p)[0]) < 1e-12
    assert D.l1_distance(W, fit, p)[0] < 1e-14


def test_relative_entropy_is_nonnegative_and_fd_maximises_entropy():
    """Klein's inequality; the Fermi-Dirac state with the moments of W has the larger entropy (Sec. 2)."""
    p = O.Params(N=32)
    W = inputs.synthetic_w(32, 3, seed=5, perturb=0.05)
    fits = D.fit_local(W, p)
    rel = D.relative_entropy(W, fits, p)
    assert np.all(rel > 0)
    S = D.entropy(W, p)
    S_fd = D.entropy(np.stack([fd_cell(f, p) for f in fits]), p)
    assert np.all(S_fd > S)


def test_pythagorean_identity_of_global_and_local_relative_entropy():
    """S(W || W_FD) = S(W || W_FD,loc) + S(W_FD,loc || W_FD) when W_FD,loc has the moments of W
    (Sec. 5.3): log(W_FD/(1 - W_FD)) is affine in (1, v, |v|^2) times spin projectors.  The fit matches the
    continuum moments; the grid moments of the fitted state differ from them by the grid's quadrature error
    (~1e-9 at N = 32, L = 12), which bounds the gap."""
    p = O.Params(N=32)
    W = inputs.synthetic_w(32, 3, seed=7, perturb=0.05)
    glob = D.fit_global(W, p)
    loc = D.fit_local(W, p)
    lhs = D.relative_entropy(W, glob, p)
    F_loc = np.stack([fd_cell(f, p) for f in loc])
    rhs = D.relative_entropy(W, loc, p) + D.relative_entropy(F_loc, glob, p)
    assert np.abs(lhs - rhs).max() < 1e-7 * np.abs(lhs).max()


def test_l1_distance_of_a_diagonal_difference():
    p = O.Params(N=8)
    fit = D.FDFit(T=1.0, mu_up=0.0, mu_dn=0.0, U=np.eye(2, dtype=complex), u=np.zeros(2))
    F = fd_cell(fit, p)
    W = F.copy()
    W[3] += 0.01          # +-0.01 on the two eigenvalues
    assert abs(D.l1_distance(W[None], fit, p)[0] - O.delta_v(p) ** 2 * 0.02 * 64) < 1e-14
