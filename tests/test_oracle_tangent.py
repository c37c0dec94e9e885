"""Pins of the oracle's forward-mode derivatives (oracle/tangent.py) against
finite differences of the oracle's own maps and against closed forms.  CPU only.

Finite differences here are central, relative step 1e-6 of the state's scale:
their truncation error is O(h^2) and rounding O(eps/h), about 1e-9 relative.
The limiter is piecewise linear, so a difference whose two points fall on
different minmod branches is meaningless; directions through the transport
are therefore relative (dW = r W, r random): where W is tiny (the Fermi-Dirac
tails) its slopes are tiny too, and an absolute perturbation would flip their
branches.
"""
import numpy as np
import pytest

from oracle import qbe_oracle as O
from oracle import tangent as T
from paper_1408_1782_gb300 import inputs

FD_TOL = 1e-7


def central(f, x, dx, h):
    return (f(x + h * dx) - f(x - h * dx)) / (2.0 * h)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def small():
    p = O.Params(N=8, J=4, M=2)
    w = inputs.synthetic_w(8, 3, seed=5, perturb=0.05)
    dw = inputs.random_field(w.shape, seed=6, scale=0.05)
    return p, w, dw


def test_collision_jvp_is_exact_for_any_step(small):
    """C is cubic along a line: the five-point difference does not depend on h."""
    p, w, dw = small
    a = T.collision_jvp(w, dw, p)
    b = T.collision_jvp(w, 0.37 * dw, p) / 0.37
    assert rel(b, a) < 1e-12


def test_collision_jvp_against_central_differences(small):
    p, w, dw = small
    a = T.collision_jvp(w, dw, p)
    fd = central(lambda x: O.collision(x, p), w, dw, 1e-6 * np.abs(w).max() / np.abs(dw).max())
    assert rel(a, fd) < FD_TOL


def test_collision_jvp_second_order_taylor_remainder(small):
    """C(w + e dw) - C(w) - e JVP = O(e^2): halving e quarters the remainder."""
    p, w, dw = small
    a = T.collision_jvp(w, dw, p)
    c0 = O.collision(w, p)
    r = [np.abs(O.collision(w + e * dw, p) - c0 - e * a).max() for e in (0.2, 0.1)]
    assert 3.0 < r[0] / r[1] < 5.0


def test_collision_vjp_brute_force_is_the_transpose(small):
    """<lam, J dw> = <J^T lam, dw> with J^T lam assembled from unit directions (one cell, N = 8)."""
    p, w, dw = small
    w1, dw1 = w[:1], dw[:1]
    lam = inputs.random_field(w1.shape, seed=7)
    g = T.collision_vjp_brute(w1, lam, p)
    lhs = np.sum(lam * T.collision_jvp(w1, dw1, p))
    assert abs(lhs - np.sum(g * dw1)) < 1e-11 * np.abs(lam).max() * np.abs(g).max() * dw1.size


@pytest.mark.parametrize("kind", ["periodic", "dirichlet", "maxwell"])
def test_advect_tangent_against_central_differences(kind):
    p = O.Params(N=8, J=4, M=2)
    Nx = 7
    W = inputs.synthetic_w(8, Nx, seed=11, perturb=0.05)
    dW = inputs.random_field(W.shape, seed=12) * W
    fd = (1.0, 0.2, -0.3, np.eye(2))
    bc = O.Boundary(kind, fd, (0.8, 0.0, 0.1, np.eye(2)), alpha=0.6)
    tau = 0.03
    _, t = T.advect_jvp(W, dW, tau, p, bc)
    ref = central(lambda x: O.advect(x, tau, p, bc), W, dW, 1e-6)
    assert rel(t, ref) < FD_TOL


def test_ghost_tangent_is_linear_part_of_the_affine_ghost_map():
    """Dirichlet ghosts hold the constant wall state: its derivative is zero there."""
    p = O.Params(N=8, J=4, M=2)
    fd = (1.0, 0.2, -0.3, np.eye(2))
    bc = O.Boundary("dirichlet", fd, fd)
    dW = inputs.random_field((4, 4, 8, 8), seed=3)
    g = T.ghosts_tangent(dW, p, bc)
    vx, _ = O.velocity_nodes(p)
    assert np.all(g[0][:, vx > 0] == 0.0) and np.all(g[-1][:, vx < 0] == 0.0)
    assert np.array_equal(g[2:-2], dW)


@pytest.mark.parametrize("kind", ["periodic", "maxwell"])
def test_step_tangent_against_central_differences(kind):
    """Derivative of one split step in W and in B together."""
    p = O.Params(N=8, J=4, M=2)
    Nx = 5
    W = inputs.synthetic_w(8, Nx, seed=21, perturb=0.05)
    B = inputs.uniform_b(Nx, (0.3, -0.2, 0.5))
    dW = inputs.random_field(W.shape, seed=22) * W
    dB = inputs.random_field(B.shape, seed=23, scale=0.5)
    fd = (1.0, 0.0, 0.0, np.eye(2))
    bc = O.Boundary(kind, fd, fd, alpha=0.5)
    dt = 0.01
    _, t = T.step_jvp(W, B, dt, p, bc, dW, dB)
    h = 1e-6
    ref = (O.step(W + h * dW, B + h * dB, dt, p, bc) - O.step(W - h * dW, B - h * dB, dt, p, bc)) / (2 * h)
    assert rel(t, ref) < FD_TOL


def test_observables_closed_forms():
    """P_z of a Fermi-Dirac state in the sigma_3 basis is dv^2 sum (n_up - n_dn); Phi_E of a state
    even in v_x vanishes on the symmetric part of the grid."""
    p = O.Params(N=16, J=4, M=2)
    Nx = 3
    beta, mu_up, mu_dn = 1.0, 0.4, -0.2
    wfd = O.fermi_dirac_pauli(beta, mu_up, mu_dn, np.eye(2), p)
    W = np.repeat(wfd[None], Nx, axis=0)
    vx, vy = O.velocity_nodes(p)
    e = 0.5 * (vx**2 + vy**2)
    n_up = 1.0 / (np.exp(beta * (e - mu_up)) + 1.0)
    n_dn = 1.0 / (np.exp(beta * (e - mu_dn)) + 1.0)
    obs = T.observables(W, p)
    dv2 = O.delta_v(p) ** 2
    assert abs(obs[0] - dv2 * np.sum(n_up - n_dn)) < 1e-14
    # only the unpaired v_x = -L column contributes to the energy flux of an even state
    col = vx[0] * 0.5 * (vx[0] ** 2 + vy[0] ** 2) * 2.0 * wfd[0][0]
    scale = dv2 * np.sum(np.abs(vx * 0.5 * (vx**2 + vy**2) * 2.0 * wfd[0]))   # size of the cancelling terms
    assert abs(obs[1] - dv2 * np.sum(col)) < 1e-14 * scale
