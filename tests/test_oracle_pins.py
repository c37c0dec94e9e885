"""Pins of the FP64 oracle against things other than itself: explicit sums,
closed forms, brute-force triple sums, the paper's matrix-form integrand,
invariants and textbook special cases.  CPU only."""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import direct as D
from oracle import qbe_oracle as O
from paper_1408_1782_gb300 import inputs

SIGMA = O.SIGMA


# --------------------------------------------------------------------------
# Transforms: padded-grid FFT helpers against the explicit exponential sums
# --------------------------------------------------------------------------

def test_to_fine_from_fine_match_explicit_sums():
    p = O.Params(N=6)
    rng = np.random.default_rng(0)
    c = rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12))
    s = np.arange(-6, 6)
    kp = np.arange(-6, 6)
    v = (p.L / p.N) * kp
    # f(v') = sum_sigma c(sigma) exp(i pi sigma.v'/L)
    E = np.exp(1j * np.pi * np.outer(v, s) / p.L)               # [k', sigma]
    f_explicit = E @ c @ E.T
    assert np.abs(O.to_fine(c, p) - f_explicit).max() < 1e-12 * np.abs(f_explicit).max()
    Einv = np.exp(-1j * np.pi * np.outer(s, v) / p.L) / 12.0
    c_back = Einv @ f_explicit @ Einv.T
    assert np.abs(O.from_fine(f_explicit, p) - c_back).max() < 1e-13 * np.abs(c).max()
    assert np.abs(c_back - c).max() < 1e-13 * np.abs(c).max()


def test_coarse_transform_roundtrip_and_fine_interpolant():
    p = O.Params(N=8, nyquist="keep")
    rng = np.random.default_rng(1)
    f = rng.normal(size=(8, 8))
    fh = O.coarse_to_xi(f, p)
    assert np.abs(O.xi_to_coarse(fh, p) - f).max() < 1e-13
    # the zero-padded interpolant on the 2N grid passes through the coarse samples at even k'
    fine = O.to_fine(O.embed(fh, p), p)
    assert np.abs(fine[::2, ::2] - f).max() < 1e-12
    # conv of two Xi-supported spectra equals the product of the interpolants' coefficients
    g = rng.normal(size=(8, 8))
    gh = O.coarse_to_xi(g, p)
    prod = O.conv(O.embed(fh, p), O.embed(gh, p), p)
    direct = np.zeros((16, 16), dtype=complex)
    k = O.xi_axis(p)
    for a in range(8):
        for b in range(8):
            for c_ in range(8):
                for d in range(8):
                    direct[k[a] + k[c_] + 8, k[b] + k[d] + 8] += fh[a, b] * gh[c_, d]
    assert np.abs(prod - direct).max() < 1e-13 * np.abs(direct).max()


# --------------------------------------------------------------------------
# Kernel functions and quadratures (eq. theta_grid, approxG, approxH-J, approxH-JM)
# --------------------------------------------------------------------------

def test_phi_and_psi_are_their_defining_integrals():
    p = O.Params(N=16)
    for s in (0.0, 1e-9, 0.37, 1.0, 5.5, 13.0, -7.25):
        ref_phi = integrate.quad(lambda r: np.sin(np.pi * s * r / p.L), 0, p.R, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
        ref_psi = integrate.quad(lambda r: np.cos(np.pi * s * r / p.L), -p.R, p.R, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
        assert abs(O.phi_R(np.array(s), p) - ref_phi) < 1e-12
        assert abs(O.psi_R(np.array(s), p) - ref_psi) < 1e-12


@pytest.mark.parametrize("M", [1, 4, 7, 32])
def test_gauss_legendre_exact_on_polynomials(M):
    p = O.Params(N=8, M=M)
    rho, w = O.gauss_legendre(p)
    for k in range(2 * M):
        exact = 0.0 if k % 2 else 2 * p.R ** (k + 1) / (k + 1)
        assert abs(np.sum(w * rho**k) - exact) <= 1e-12 * max(1.0, p.R ** (k + 1))
    assert np.all(w > 0)


def test_H_at_origin_is_4_pi_R_squared():
    """int int delta(u.u') over B_R x B_R = 4 pi R^2; both quadratures reproduce it exactly."""
    for J, M in ((2, 1), (8, 5), (32, 32)):
        p = O.Params(N=8, J=J, M=M)
        z = np.zeros((1, 2))
        assert abs(D.kernel_HJ(z, z, p)[0] - 4 * np.pi * p.R**2) < 1e-11
        assert abs(D.kernel_HJM(z, z, p)[0] - 4 * np.pi * p.R**2) < 1e-11
    # and the oracle's tables agree at sigma = 0
    p = O.Params(N=8, J=8, M=6)
    psi, psip = O.psi_tables(p)
    assert abs((np.pi / p.J) * np.sum(psi[:, 8, 8] * psip[:, 8, 8]) - 4 * np.pi * p.R**2) < 1e-11


def test_H_J_converges_to_the_angular_integral():
    """H(xi,chi) = int_0^pi psi(xi.theta) psi(chi.theta^perp) dtheta (delta(u.u') in polar form)."""
    p64 = O.Params(N=8, J=64)
    for xi, chi in (((1.0, 2.0), (-3.0, 1.0)), ((4.0, 0.0), (0.0, 3.0)), ((2.0, -5.0), (1.0, 1.0))):
        xi_, chi_ = np.array(xi), np.array(chi)

        def f(t):
            th = np.array([np.cos(t), np.sin(t)])
            tp = np.array([-np.sin(t), np.cos(t)])
            return float(O.psi_R(np.array(xi_ @ th), p64) * O.psi_R(np.array(chi_ @ tp), p64))
        ref = integrate.quad(f, 0, np.pi, epsabs=1e-13, epsrel=1e-13, limit=400)[0]
        got = D.kernel_HJ(xi_[None], chi_[None], p64)[0]
        assert abs(got - ref) < 1e-9 * max(1.0, abs(ref))


def test_G_J_converges_exponentially_in_J():
    """Staggered trapezoidal rule for the principal value (Sec. 3.2); error decays fast with J."""
    xi = np.array([[2.0, -1.0], [0.0, 3.0], [5.0, 4.0]])
    chi = np.array([[1.0, 1.0], [-2.0, 0.0], [3.0, -6.0]])
    ref = D.kernel_G(xi, chi, O.Params(N=8, J=96))
    errs = [np.abs(D.kernel_G(xi, chi, O.Params(N=8, J=J)) - ref).max() / np.abs(ref).max() for J in (8, 16, 32)]
    assert errs[2] < 1e-8 and errs[1] < errs[0] and errs[2] < errs[1]


def test_odd_J_rejected():
    with pytest.raises(ValueError):
        O.Params(N=8, J=5)


# --------------------------------------------------------------------------
# Pauli algebra (Sec. 3.1) against explicit 2x2 complex matrix products
# --------------------------------------------------------------------------

def _m(w):
    return np.einsum("c,cij->ij", w.astype(complex), SIGMA)


def test_pauli_identities_against_matrix_form():
    rng = np.random.default_rng(7)
    I = np.eye(2)
    tr = np.trace
    ip = lambda a, b: a @ (O.ETA * b)
    for _ in range(20):
        w1, w2, w3, w4 = (rng.normal(size=4) for _ in range(4))
        W1, W2, W3, W4 = map(_m, (w1, w2, w3, w4))
        # anticommutator and commutator
        assert np.abs(W1 @ W2 + W2 @ W1 - 2 * (_m(w1[0] * w2 + w2[0] * w1) - ip(w1, w2) * I)).max() < 1e-13
        cross = np.cross(w2[1:], w1[1:])
        assert np.abs(-1j * (W2 @ W1 - W1 @ W2) - _m(np.r_[0.0, 2 * cross])).max() < 1e-13

        def A(W1, W2, W3, W4):
            W2t, W4t = I - W2, I - W4
            return (-W4 @ W2t @ W3 + W4 * tr(W2t @ W3)
                    - (W4t @ W3 - W4t @ W2 - W2t @ W3 + W4t * tr(W2) - W4t * tr(W3) + tr(W3 @ W2t) * I) @ W1)

        def AA(*x):
            a = A(*x)
            return a + a.conj().T

        sym = 0.5 * (AA(W1, W2, W3, W4) + AA(W1, W2, W4, W3))
        # eq. CdPauli integrand
        X = _m(O.ETA * w2)
        pauli = 2 * ip(w3, w4) * (I - W1 - X) + (w3[0] + w4[0] - 1) * (W1 @ X + X @ W1)
        assert np.abs(sym - pauli).max() < 1e-12
        # eq. AW_Hubbard representation
        W1t, W2t, W3t, W4t = I - W1, I - W2, I - W3, I - W4

        def Aq(W1, W2, W3, W4):
            W1t, W2t, W3t, W4t = I - W1, I - W2, I - W3, I - W4
            return (-W1t @ W3 @ W2t @ W4 - W4 @ W2t @ W3 @ W1t + W1 @ W3t @ W2 @ W4t + W4t @ W2 @ W3t @ W1
                    + (W1t @ W3 + W3 @ W1t) * tr(W2t @ W4) - (W1 @ W3t + W3t @ W1) * tr(W2 @ W4t))
        assert np.abs(0.5 * (Aq(W1, W2, W3, W4) + Aq(W1, W2, W4, W3)) - sym).max() < 1e-12
        # eq. Heff integrand -> Pauli form
        He = lambda W2, W3, W4: W3 @ W4 - W2 @ W3 - W3 @ W2 - tr(W4) * W3 + tr(W2) * W3 + W2
        hs = 0.5 * (He(W2, W3, W4) + He(W2, W4, W3))
        hp = (ip(w2, w2) - ip(w3 - w2, w4 - w2)) * I - (w3[0] + w4[0] - 1) * W2
        assert np.abs(hs - hp).max() < 1e-12


# --------------------------------------------------------------------------
# The four Fourier integrals against literal triple sums
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nyq", ["zero", "keep"])
@pytest.mark.parametrize("N", [4, 6])
def test_integrals_match_bruteforce_triple_sums(nyq, N):
    p = O.Params(N=N, J=4, M=3, nyquist=nyq)
    rng = np.random.default_rng(N)
    f, g, h = (rng.normal(size=(N, N)) for _ in range(3))
    fh, gh, hh = (O.coarse_to_xi(x.astype(complex), p) for x in (f, g, h))
    for kind, fn in (("I1", O.I1), ("I2", O.I2), ("I3", O.I3), ("I4", O.I4)):
        bf = D.integral_bruteforce(kind, fh, gh, hh, p)
        orc = O.restrict(fn(O.embed(fh, p), O.embed(gh, p), O.embed(hh, p), p), p)
        assert np.abs(bf - orc).max() < 1e-13 * np.abs(bf).max(), kind


# --------------------------------------------------------------------------
# Whole C[W] against the paper's matrix-form integrand (eq. Cc/Heff, eq. Cd)
# --------------------------------------------------------------------------

def test_collision_matches_matrix_form_quadrature():
    """Band-limited W: the spectral method is exact up to the angular rule; J >= 12 removes the
    asymmetry of the staggered rule under u <-> u' below round-off, M = 24 makes Hu-Ying exact."""
    p = O.Params(N=12, J=12, M=24)
    w = inputs.bandlimited_w(12, 1, 1, seed=3)[0]
    Cc, Cd = O.collision_parts(w[None], p)
    pts = [(2, 3), (5, 5), (7, 1), (10, 9)]
    dc, dd = D.collision_direct(w, p, n_radial=24, points=pts)
    for i, (a, b) in enumerate(pts):
        assert np.abs(Cc[0, :, a, b] - dc[:, i]).max() < 1e-12 * np.abs(Cc).max()
        assert np.abs(Cd[0, :, a, b] - dd[:, i]).max() < 1e-12 * np.abs(Cd).max()


def test_scalar_reduction_to_uehling_uhlenbeck():
    """W = n 1: C_c = 0, no spin part, and C_d = 2 pi int int delta(u.u') [n3 n4 (1-n1)(1-n2) - n1 n2 (1-n3)(1-n4)]."""
    p = O.Params(N=12, J=8, M=24)
    rng = np.random.default_rng(4)
    n = inputs.bandlimited_w(12, 1, 1, seed=11)[0, 0]
    w = np.zeros((1, 4, 12, 12))
    w[0, 0] = n
    Cc, Cd = O.collision_parts(w, p)
    assert np.abs(Cc).max() < 1e-13
    assert np.abs(Cd[0, 1:]).max() < 1e-13 * np.abs(Cd).max()
    nh = O.coarse_to_xi(n.astype(complex), O.Params(12, nyquist="keep"))
    vx, vy = O.velocity_nodes(p)
    r, wr = np.polynomial.legendre.leggauss(24)
    r, wr = p.R * r, p.R * wr
    for (ix, iy) in ((3, 4), (6, 6), (9, 2)):
        v = np.array([vx[ix, iy], vy[ix, iy]])
        tot = 0.0
        for t in np.arange(p.J) * np.pi / p.J:
            th, tp = np.array([np.cos(t), np.sin(t)]), np.array([-np.sin(t), np.cos(t)])
            P3 = v + r[:, None, None] * th
            P4 = v + r[None, :, None] * tp
            P2 = v + r[:, None, None] * th + r[None, :, None] * tp
            ev = lambda P: D.trig_eval(nh, p, P.reshape(-1, 2)).real
            n1 = n[ix, iy]
            n3 = ev(np.broadcast_to(P3, P2.shape)).reshape(24, 24)
            n4 = ev(np.broadcast_to(P4, P2.shape)).reshape(24, 24)
            n2 = ev(P2).reshape(24, 24)
            integrand = n3 * n4 * (1 - n1) * (1 - n2) - n1 * n2 * (1 - n3) * (1 - n4)
            tot += (np.pi / p.J) * np.einsum("a,b,ab->", wr, wr, integrand)
        ref = 2 * np.pi * tot
        assert abs(Cd[0, 0, ix, iy].real - ref) < 1e-11 * np.abs(Cd).max()


def test_commuting_states_have_no_conservative_part():
    """All W(v) diagonal in one fixed basis: [W(v+u+u'), W(v)] = 0 so C_c = 0 (eq. Cc)."""
    p = O.Params(N=8, J=6, M=4)
    rng = np.random.default_rng(5)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    a = inputs.synthetic_w(8, 1, seed=2)[0]
    w = np.zeros((1, 4, 8, 8))
    w[0, 0] = a[0]
    w[0, 1:] = axis[:, None, None] * a[3][None]
    Cc, Cd = O.collision_parts(w, p)
    assert np.abs(Cc).max() < 1e-13
    # the dissipative spin part stays along the same axis
    perp_part = Cd[0, 1:].real - axis[:, None, None] * np.einsum("c,cxy->xy", axis, Cd[0, 1:].real)[None]
    assert np.abs(perp_part).max() < 1e-12 * np.abs(Cd).max()


def test_density_conservation_at_paper_quadrature():
    """sum_v C(v) = 0 up to the quadrature error; at N=16, J=M=32 that error is below 1e-13."""
    p = O.Params(N=16, J=32, M=32)
    w = inputs.synthetic_w(16, 1, seed=0)
    Cc, Cd = O.collision_parts(w, p)
    for C in (Cc.real, Cd.real):
        rho, _, _ = O.moments(C, p)
        scale = O.delta_v(p) ** 2 * np.abs(C).sum()
        assert np.abs(rho).max() < 1e-13 * scale


def test_fermi_dirac_equilibrium_residual_decays_with_N():
    """C[W_FD] vanishes in the continuum (Sec. 2); on the grid (J = M = 32) it decreases
    spectrally with N: about 38% of a perturbed state's |C| at N=16, 7% at N=24."""
    res = {}
    for N in (16, 24):
        p = O.Params(N=N, J=32, M=32)
        wfd = O.fermi_dirac_pauli(1.0, 0.5, -0.5, np.eye(2), p)[None]
        res[N] = np.abs(O.collision(wfd, p)).max()
    p = O.Params(N=24, J=32, M=32)
    pert = np.abs(O.collision(inputs.synthetic_w(24, 1, seed=1), p)).max()
    assert res[24] < 0.3 * res[16]
    assert res[24] < 0.1 * pert


def test_nyquist_readings():
    """Canonical reading (Nyquist line zeroed): every field is real, C has no imaginary residue.
    Literal Xi: complex fields; the two readings differ by an amount that shrinks with N."""
    gaps = []
    for N in (16, 32):
        p0 = O.Params(N=N, J=4, M=4)
        p1 = O.Params(N=N, J=4, M=4, nyquist="keep")
        w = inputs.synthetic_w(N, 1, seed=4)
        C0, im0 = O.collision(w, p0, return_imag=True)
        C1, im1 = O.collision(w, p1, return_imag=True)
        assert np.abs(im0).max() < 1e-13 * np.abs(C0).max()
        gaps.append(np.abs(C0 - C1).max() / np.abs(C0).max())
    assert gaps[1] < 0.5 * gaps[0]


# --------------------------------------------------------------------------
# Fermi-Dirac moments (eq. momentsFermiDirac)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("beta,mu_up,mu_dn", [(1.0, 1.0, 1.5), (0.8, 1.5, -1.5), (2.0, -0.4, 0.3)])
def test_fermi_dirac_moments_closed_form(beta, mu_up, mu_dn):
    """Grid sums converge exponentially (trapezoidal rule on a smooth decaying integrand); the
    coldest state (T = 1/2) needs N = 128 for round-off agreement with the analytic moments."""
    p = O.Params(N=128)
    c, s = np.cos(0.3), np.sin(0.3)
    U = np.array([[c, -s], [s, c]])
    w = O.fermi_dirac_pauli(beta, mu_up, mu_dn, U, p)
    rho, mom, en = O.moments(w[None], p)
    T = 1.0 / beta
    z = np.exp(np.array([mu_up, mu_dn]) / T)
    rho_fd = 2 * np.pi * T * np.sum(np.log1p(z))                   # = tr rho
    li2 = special.spence(1.0 + z)                                   # Li2(-z) = spence(1 + z)
    eps_fd = T * (-np.sum(li2)) / np.sum(np.log1p(z))
    assert abs(2 * rho[0, 0] - rho_fd) < 1e-13 * rho_fd
    assert abs(en[0] / (2 * rho[0, 0]) - eps_fd) < 1e-13 * eps_fd
    assert np.abs(mom).max() < 1e-10 * rho_fd


# --------------------------------------------------------------------------
# Transport (Sec. 4, eq. slopeLimiterStep) and boundaries (Sec. 2)
# --------------------------------------------------------------------------

def _flux_form_limiter_step(u, nu):
    """LeVeque's slope-limited upwind method in flux form (minmod slopes), periodic, one component."""
    up1, um1 = np.roll(u, -1), np.roll(u, 1)
    s = np.where((up1 - u) * (u - um1) > 0, np.where(np.abs(up1 - u) <= np.abs(u - um1), up1 - u, u - um1), 0.0)
    if nu >= 0:
        F = nu * u + 0.5 * nu * (1 - nu) * s                # flux through the right face of cell j
        return u - (F - np.roll(F, 1))
    F = nu * up1 - 0.5 * nu * (1 + nu) * np.roll(s, -1)
    return u - (F - np.roll(F, 1))


def test_minmod_step_equals_flux_form_slope_limiter():
    p = O.Params(N=4)
    rng = np.random.default_rng(9)
    Nx = 11
    W = rng.normal(size=(Nx, 4, 4, 4))
    dx = 1.0 / Nx
    tau = 0.7 * dx / p.L
    out = O.advect_substep(W, tau, dx, p, O.Boundary("periodic"))
    vx, _ = O.velocity_nodes(p)
    for ix in range(4):
        for c in range(4):
            nu = tau * vx[ix, 0] / dx
            ref = _flux_form_limiter_step(W[:, c, ix, 1], nu)
            assert np.abs(out[:, c, ix, 1] - ref).max() < 1e-13


def test_transport_periodic_invariants():
    p = O.Params(N=8)
    Nx = 16
    dx = 1.0 / Nx
    rng = np.random.default_rng(3)
    W = rng.uniform(0, 1, size=(Nx, 4, 8, 8))
    bc = O.Boundary("periodic")
    # constant state preserved
    C = np.ones((Nx, 4, 8, 8)) * 0.3
    assert np.abs(O.advect(C, 0.013, p, bc) - C).max() < 1e-15
    # conservation of sum_j W_j (flux form)
    out = O.advect(W, 0.02, p, bc)
    assert np.abs(out.sum(0) - W.sum(0)).max() < 1e-12
    # total variation does not increase (TVD)
    tv = lambda X: np.abs(np.diff(np.concatenate([X, X[:1]]), axis=0)).sum(0)
    assert np.all(tv(out) <= tv(W) + 1e-12)
    # |nu| = 1: exact shift by one cell in the upwind direction
    vx, _ = O.velocity_nodes(p)
    ix = 0                                        # v_x = -L
    tau = dx / p.L
    out1 = O.advect_substep(W, tau, dx, p, bc)
    assert np.abs(out1[:, :, ix, :] - np.roll(W, -1, axis=0)[:, :, ix, :]).max() < 1e-14


def test_transport_subcycling_count():
    p = O.Params(N=16)
    assert O.transport_substeps(0.005, 1 / 16, p) == 1    # nu = 0.96
    assert O.transport_substeps(0.0025, 1 / 128, p) == 4  # nu = 3.84


def test_dirichlet_keeps_matching_equilibrium_at_rest():
    """Dirichlet walls equal to a spatially uniform state: transport leaves it unchanged."""
    p = O.Params(N=8)
    fd = (1.0, 0.5, -0.5, np.eye(2))
    w = O.fermi_dirac_pauli(*fd, p)
    W = np.broadcast_to(w, (6, 4, 8, 8)).copy()
    out = O.advect(W, 0.01, p, O.Boundary("dirichlet", fd, fd))
    assert np.abs(out - W).max() < 1e-15


def test_maxwell_diffuse_wall_balances_number_flux():
    """alpha = 1: the ghost's incoming number flux equals the outgoing flux Fbar (definition of Z)."""
    p = O.Params(N=8)
    rng = np.random.default_rng(2)
    W = rng.uniform(0, 0.4, size=(5, 4, 8, 8))
    fdL = (1.0, 0.3, -0.2, np.eye(2))
    fdR = (0.7, 0.1, 0.1, np.eye(2))
    bc = O.Boundary("maxwell", fdL, fdR, alpha=1.0)
    ext = O._ghosts(W, p, bc)
    vx, _ = O.velocity_nodes(p)
    dv2 = O.delta_v(p) ** 2
    out_flux_L = dv2 * np.sum((2 * W[0, 0] * np.abs(vx))[vx < 0])
    in_flux_L = dv2 * np.sum((2 * ext[1, 0] * np.abs(vx))[vx > 0])
    assert abs(out_flux_L - in_flux_L) < 1e-12 * out_flux_L
    out_flux_R = dv2 * np.sum((2 * W[-1, 0] * np.abs(vx))[vx > 0])
    in_flux_R = dv2 * np.sum((2 * ext[-2, 0] * np.abs(vx))[vx < 0])
    assert abs(out_flux_R - in_flux_R) < 1e-12 * out_flux_R
    # alpha = 0: pure specular reflection of the boundary cell
    ext0 = O._ghosts(W, p, O.Boundary("maxwell", fdL, fdR, alpha=0.0))
    for ix in range(1, 8):
        mx = 8 - ix
        if vx[ix, 0] > 0:
            assert np.abs(ext0[0][:, ix] - W[0][:, mx]).max() == 0.0


# --------------------------------------------------------------------------
# Precession and the RK2 substep
# --------------------------------------------------------------------------

def test_precession_is_the_commutator_and_rotates_spin():
    rng = np.random.default_rng(8)
    w = rng.normal(size=(3, 4, 2, 2))
    B = rng.normal(size=(3, 3))
    P = O.precession(w, B)
    for c in range(3):
        Bm = np.einsum("a,aij->ij", B[c].astype(complex), SIGMA[1:])
        Wm = _m(w[c, :, 0, 1])
        ref = -1j * (Bm @ Wm - Wm @ Bm)
        assert np.abs(_m(P[c, :, 0, 1]) - ref).max() < 1e-13


def test_rk2_substep_second_order_on_pure_precession():
    """W = 1/2 + a.sigma, constant in v: every collision term cancels (2w0-1 = 0 and
    1 - W - (eta w).sigma = 0), so the substep is pure precession w' = 2 B x w, whose exact
    solution rotates a about B by the angle 2|B|t.  Heun's global error must be O(dt^2).
    A small truncation radius R keeps the linearised collision operator (eigenvalues of order
    2 pi * 4 pi R^2) from amplifying round-off at these step sizes."""
    p = O.Params(N=4, R=0.05, J=2, M=1)
    B = np.array([[0.3, -0.2, 0.5], [0.0, 0.7, 0.1]])
    a = np.array([[0.2, 0.1, -0.15], [0.0, -0.25, 0.1]])
    w0 = np.zeros((2, 4, 4, 4))
    w0[:, 0] = 0.5
    w0[:, 1:] = a[:, :, None, None]
    assert np.abs(O.collision(w0, p)).max() < 1e-12
    T = 0.4
    exact = []
    for c in range(2):
        b = np.linalg.norm(B[c])
        n = B[c] / b
        th = 2 * b * T
        v = a[c]
        exact.append(v * np.cos(th) + np.cross(n, v) * np.sin(th) + n * (n @ v) * (1 - np.cos(th)))
    exact = np.array(exact)
    errs = []
    for nsteps in (8, 16, 32):
        W = w0.copy()
        for _ in range(nsteps):
            W = O.collide_rk2(W, B, T / nsteps, p)
        errs.append(np.abs(W[:, 1:, 1, 2] - exact).max())
        assert np.abs(W[:, 0] - 0.5).max() < 1e-13
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


# --------------------------------------------------------------------------
# Sub-cycled transport A(tau) and the split step (Sec. 4, eq. slopeLimiterStep)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("s", [2, 3])
def test_advect_subcycles_in_equal_unit_courant_steps(s):
    """A(tau) with tau = s dx/L takes s sub-steps of tau/s: on the row v_x = -L each has
    |nu| = 1, where eq. slopeLimiterStep is an exact shift by one cell (Godunov moves the
    whole cell, the limiter factor (sgn nu - nu)/2 vanishes).  A(tau) is then a shift by s
    cells; sub-steps of length tau (|nu| = s) or a wrong count give something else."""
    p = O.Params(N=8)
    Nx = 10
    dx = 1.0 / Nx
    W = np.random.default_rng(20 + s).uniform(0, 1, size=(Nx, 4, 8, 8))
    out = O.advect(W, s * dx / p.L, p, O.Boundary("periodic"))
    assert np.abs(out[:, :, 0, :] - np.roll(W, -s, axis=0)[:, :, 0, :]).max() < 1e-14


def test_advect_subcycles_match_textbook_flux_form():
    """A(tau) with tau = 1.5 dx/L: two sub-steps of Courant number -0.75 (max |v_x| = L) on
    the row v_x = -L, and two of -0.75 |v_x|/L on the others; each is LeVeque's flux-form
    minmod step (written out independently in this file)."""
    p = O.Params(N=8)
    Nx = 12
    dx = 1.0 / Nx
    W = np.random.default_rng(31).normal(size=(Nx, 4, 8, 8))
    out = O.advect(W, 1.5 * dx / p.L, p, O.Boundary("periodic"))
    vx, _ = O.velocity_nodes(p)
    for ix in range(8):
        nu = 0.75 * vx[ix, 0] / p.L
        for c in (0, 3):
            u = W[:, c, ix, 5]
            ref = _flux_form_limiter_step(_flux_form_limiter_step(u, nu), nu)
            assert np.abs(out[:, c, ix, 5] - ref).max() < 1e-13


def _heun_linear(A, dt):
    """Heun's method on w' = A w is exactly w -> (1 + dt A + dt^2 A^2 / 2) w."""
    return np.eye(A.shape[0]) + dt * A + 0.5 * dt * dt * A @ A


def test_step_is_half_transport_collision_half_transport():
    """step = A(dt/2) o RK2(dt) o A(dt/2) (Sec. 4).  With dt/2 = dx/L every half step shifts
    the row v_x = -L by exactly one cell.  w0 = 1/2 makes C_c and the I4 term vanish and a
    truncation radius R = 1e-6 makes the rest O(R^2), so the substep is Heun on the
    precession w' = 2 B(x) x w, a linear map per cell.  Along the row the step must give
    out_i = H(B_{i+1}) W_{i+2}: collision placed first or last would use B_{i+2} or B_i,
    full-length transport steps would shift by four cells."""
    p = O.Params(N=4, R=1e-6, J=2, M=1)
    Nx = 8
    dx = 1.0 / Nx
    dt = 2.0 * dx / p.L
    rng = np.random.default_rng(44)
    x = (np.arange(Nx) + 0.5) / Nx
    W = np.zeros((Nx, 4, 4, 4))
    W[:, 0] = 0.5
    W[:, 1:] = 0.3 * np.stack([np.cos(2 * np.pi * x), np.sin(4 * np.pi * x), np.cos(6 * np.pi * x + 1)], -1)[:, :, None, None]
    W += 0.05 * rng.normal(size=W.shape) * np.array([0, 1, 1, 1])[None, :, None, None]
    bc = O.Boundary("periodic")
    out0 = O.step(W, np.zeros((Nx, 3)), dt, p, bc)
    assert np.abs(out0[:, :, 0, :] - np.roll(W, -2, axis=0)[:, :, 0, :]).max() < 1e-10
    B = np.stack([1.5 * np.sin(2 * np.pi * x), 0.8 + np.cos(2 * np.pi * x), -np.cos(4 * np.pi * x)], -1)
    out = O.step(W, B, dt, p, bc)
    for i in range(Nx):
        b = B[(i + 1) % Nx]
        A = 2.0 * np.array([[0, -b[2], b[1]], [b[2], 0, -b[0]], [-b[1], b[0], 0]])   # w -> 2 b x w
        ref = _heun_linear(A, dt) @ W[(i + 2) % Nx, 1:, 0, :]
        assert np.abs(out[i, 1:, 0, :] - ref).max() < 1e-10
        assert np.abs(out[i, 0, 0, :] - 0.5).max() < 1e-12
        wrong = _heun_linear(A, dt) @ W[(i + 2) % Nx, 1:, 0, :] - _heun_linear(
            2.0 * np.array([[0, -B[i][2], B[i][1]], [B[i][2], 0, -B[i][0]], [-B[i][1], B[i][0], 0]]), dt
        ) @ W[(i + 2) % Nx, 1:, 0, :]
        assert np.abs(wrong).max() > 1e-4          # the placements are distinguishable
