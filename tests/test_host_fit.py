"""Host-side parts of the library's diagnostics (no GPU): its dilogarithm and its
Fermi-Dirac fit (eq. momentsFermiDirac), against the definitions and the oracle."""
import numpy as np
import pytest

from oracle import diagnostics as D
from oracle import qbe_oracle as O


@pytest.fixture(scope="module")
def qbe():
    import __graft_entry__ as g

    g.build()
    from paper_1408_1782_gb300 import qbe as q

    return q


def li2_series(x, terms=80):
    """Li2(x) = sum_k x^k / k^2 (|x| <= 1/2 here)."""
    return sum(x**k / k**2 for k in range(1, terms))


def test_dilog_against_its_power_series_and_special_values(qbe):
    for x in (-1e-12, -1e-8, -0.01, -0.2, -0.5):
        assert abs(qbe.dilog(x) - li2_series(x)) <= 2e-16 * abs(li2_series(x))
    assert abs(qbe.dilog(-1.0) + np.pi**2 / 12) < 2e-16
    assert qbe.dilog(0.0) == 0.0


def test_dilog_inversion_and_reflection_consistency(qbe):
    """Li2(-z) + Li2(-1/z) = -pi^2/6 - log(z)^2/2 across the [-1, 0] boundary, and agreement with scipy's
    spence away from 0 (where spence(1 - x) loses relative digits)."""
    for z in (1.5, 3.0, 17.0, 1e3, 1e8):
        lhs = qbe.dilog(-z) + qbe.dilog(-1.0 / z)
        assert abs(lhs + np.pi**2 / 6 + 0.5 * np.log(z) ** 2) < 1e-14 * (1 + 0.5 * np.log(z) ** 2)
    for x in (-0.3, -0.9, -1.5, -40.0):
        assert abs(qbe.dilog(x) - D.li2(x)) < 1e-14 * abs(D.li2(x))


def rotation(theta, phi):
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -s * np.exp(-1j * phi)], [s * np.exp(1j * phi), c]], dtype=np.complex128)


@pytest.mark.parametrize("T,mu_up,mu_dn,u", [(0.8, 0.7, -0.4, (0.0, 0.0)), (1.6, -0.5, 1.2, (0.3, -0.2)),
                                              (2.5, -2.0, -1.0, (0.05, 0.1))])
def test_fd_fit_matches_the_oracle_fit(qbe, T, mu_up, mu_dn, u):
    """Both fits solve eq. momentsFermiDirac for the same grid moments (different root finders)."""
    p = O.Params(N=64, L=12.0)
    fit = D.FDFit(T=T, mu_up=mu_up, mu_dn=mu_dn, U=rotation(1.1, -0.7), u=np.array(u))
    Fm = D.fd_state(fit, p)
    W = np.moveaxis(0.5 * np.einsum("xyij,aji->xya", Fm, O.SIGMA).real, -1, 0)[None].copy()
    rho4, mom, en = O.moments(W, p)
    ref = D.fit_from_moments(D.pauli_to_matrix(rho4[0]), mom[0], en[0])
    got = qbe.fd_fit_moments(rho4[0], mom[0], en[0])
    assert got.ok == 1 and ref.ok
    assert abs(got.T - ref.T) < 1e-12 * ref.T
    assert abs(got.mu_up - ref.mu_up) < 1e-11 and abs(got.mu_dn - ref.mu_dn) < 1e-11
    assert np.abs(np.array(got.u[:]) - ref.u).max() < 1e-15
    for s in range(2):
        a = got.U()[:, s]
        b = ref.U[:, s]
        assert np.abs(np.outer(a, a.conj()) - np.outer(b, b.conj())).max() < 1e-12
    bl = np.array(got.bloch[:])
    up = got.U()[:, 0]
    assert np.abs(bl - np.array([2 * (up[0].conj() * up[1]).real, 2 * (up[0].conj() * up[1]).imag,
                                 abs(up[0]) ** 2 - abs(up[1]) ** 2])).max() < 1e-14


def test_fd_fit_rejects_states_below_the_zero_temperature_energy(qbe):
    # rho = diag(1, 1) (Pauli 1, 0, 0, 0) with internal energy below sum rho_s^2 / (4 pi tr rho)
    eps0 = 2.0 / (4 * np.pi * 2.0)
    out = qbe.fd_fit_moments([1.0, 0.0, 0.0, 0.0], [0.0, 0.0], 0.5 * eps0 * 2.0)
    assert out.ok == 0
    out = qbe.fd_fit_moments([1.0, 0.0, 0.0, 1.0], [0.0, 0.0], 5.0)     # an eigenvalue 0
    assert out.ok == 0
