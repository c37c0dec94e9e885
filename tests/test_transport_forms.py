"""The transport kernels evaluate eq. slopeLimiterStep in an upwind form and transpose that form;
these CPU tests check both reformulations, restated here in numpy, against the oracle's update and
its forward-mode derivative.

Upwind form (s = sgn v_x, q_d = W(j + s (d - 2)), d = 0..3, k = tau / (2 dx), nu = tau v_x / dx):
    W_out = q2 - c_g (q2 - q1) + c_l (minmod(q2 - q1, q1 - q0) - minmod(q3 - q2, q2 - q1)),
    c_g = 2 k |v_x|,  c_l = k (1 - |nu|) |v_x|.
Transpose at frozen branches (lam = 0 outside the domain, mu(m) = c_l (lam(m + s) - lam(m))):
    lam_in(i) = (1 - c_g) lam(i) + c_g lam(i + s) + sum over the slopes sig(i - s), sig(i), sig(i + s)
    of mu times their derivative in W(i); a tie |a| = |b| takes the x-forward difference.
"""
import numpy as np
import pytest

from oracle import qbe_oracle as O
from oracle import tangent as T
from paper_1408_1782_gb300 import inputs


def _minmod(a, b):
    return np.where(a * b > 0.0, np.where(np.abs(a) <= np.abs(b), a, b), 0.0)


def upwind_update(ext, tau, dx, p):
    """ext: [Nx + 4][4][N][N] with two ghost cells per side."""
    vx, _ = O.velocity_nodes(p)
    n = ext.shape[0] - 4
    N = p.N
    out = np.empty((n,) + ext.shape[1:])
    k = tau / (2.0 * dx)
    for ix in range(N):
        v = vx[ix, 0]
        s = -1 if ix < N // 2 else 1
        av = abs(v)
        cg, cl = 2.0 * k * av, k * (1.0 - tau * av / dx) * av
        col = ext[:, :, ix, :]
        q = [col[2 + s * (d - 2) + np.arange(n)] for d in range(4)]
        b = q[2] - q[1]
        out[:, :, ix, :] = q[2] - cg * b + cl * (_minmod(b, q[1] - q[0]) - _minmod(q[3] - q[2], b))
    return out


@pytest.mark.parametrize("nu_max", [0.9, 2.5])
@pytest.mark.parametrize("N", [8, 16])
def test_upwind_form_equals_the_limiter_update(N, nu_max):
    """For every velocity (both signs of v_x and v_x = 0) and any |nu| (the identity is algebraic)."""
    p = O.Params(N=N)
    Nx = 7
    rng = np.random.default_rng(N)
    ext = inputs.synthetic_w(N, Nx + 4, seed=3) + 0.05 * rng.normal(size=(Nx + 4, 4, N, N))
    dx = 1.0 / Nx
    tau = nu_max * dx / p.L
    ref = O.limiter_update(ext, tau, dx, p)
    got = upwind_update(ext, tau, dx, p)
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()


def upwind_transpose(ext, lam, tau, dx, p):
    """Cotangent of every cell of ext (interior and ghosts) for the output cotangent lam [Nx]."""
    vx, _ = O.velocity_nodes(p)
    n = ext.shape[0] - 4
    N = p.N
    out = np.zeros_like(ext)
    k = tau / (2.0 * dx)

    def branch(a, b, tie_a):
        if not a * b > 0.0:
            return 0
        return 1 if (abs(a) < abs(b) or (tie_a and abs(a) == abs(b))) else 2

    for ix in range(N):
        v = vx[ix, 0]
        s = -1 if ix < N // 2 else 1
        av = abs(v)
        cg, cl = 2.0 * k * av, k * (1.0 - tau * av / dx) * av
        for c in range(4):
            for iy in range(N):
                W = lambda m: ext[m + 2, c, ix, iy] if -2 <= m < n + 2 else 0.0
                L = lambda m: lam[m, c, ix, iy] if 0 <= m < n else 0.0
                for i in range(-2, n + 2):
                    w = [W(i + s * (e - 2)) for e in range(5)]
                    l = [L(i + s * (e - 1)) for e in range(4)]
                    acc = l[1] + cg * (l[2] - l[1])
                    if branch(w[2] - w[1], w[1] - w[0], s > 0) == 1:
                        acc += cl * (l[1] - l[0])
                    b0 = branch(w[3] - w[2], w[2] - w[1], s > 0)
                    if b0:
                        acc += (-cl if b0 == 1 else cl) * (l[2] - l[1])
                    if branch(w[4] - w[3], w[3] - w[2], s > 0) == 2:
                        acc -= cl * (l[3] - l[2])
                    out[i + 2, c, ix, iy] = acc
    return out


@pytest.mark.parametrize("ties", [False, True])
def test_transposed_upwind_form_against_the_oracle_tangent(ties):
    """<lam, J dext> = <J^T lam, dext> with J the oracle's derivative of the limiter update at ext;
    with ties (x-differences exactly 0 or 1/64) the tie rule decides the frozen branches."""
    N, Nx = 8, 5
    p = O.Params(N=N)
    if ties:
        ext = inputs.minmod_tie_w(N, Nx + 4, seed=50)
    else:
        rng = np.random.default_rng(5)
        ext = inputs.synthetic_w(N, Nx + 4, seed=4) + 0.05 * rng.normal(size=(Nx + 4, 4, N, N))
    dx = 1.0 / Nx
    tau = 0.9 * dx / p.L
    rng = np.random.default_rng(6)
    lam = rng.normal(size=(Nx, 4, N, N))
    dext = rng.normal(size=ext.shape)
    jd = T.limiter_update_tangent(ext, dext, tau, dx, p)
    a = np.sum(lam * jd)
    b = np.sum(upwind_transpose(ext, lam, tau, dx, p) * dext)
    assert abs(a - b) <= 1e-12 * (np.sum(np.abs(lam * jd)) + np.abs(b))
