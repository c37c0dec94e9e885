"""Independent pins for the Fourier oracle (TEST INFRASTRUCTURE, tests only).

Two checks that do not go through the oracle's convolution machinery:

1. ``collision_direct``: C[W](v) from the paper's *matrix* form of the
   integrand -- the effective Hamiltonian of eq. Heff inside -i[H_eff, W]
   (eq. Cc) and A + A^* of eq. Cd -- after the Carleman change of variables
   v1 -> v, v3 -> v+u, v4 -> v+u', v2 = v+u+u' (Sec. 3.2), integrated by
   quadrature directly in real space:
     * principal-value part: u = r theta, u' = r' theta' over full circles with
       the staggered trapezoidal angles of eq. theta_grid (2J points each) and
       Gauss-Legendre in r, r' on [0, R];
     * delta(u.u') part: u = r theta, u' = s theta^perp, theta on the half
       circle (J trapezoidal points, weight pi/J), Gauss-Legendre in r, s on
       [-R, R].
   W is evaluated off-grid by its trigonometric interpolant.  For band-limited
   W (all triple products still inside Xi) the Fourier method is exact up to
   the same angular quadrature, so the two must agree to round-off when the
   radial rules are converged (large M in the Hu-Ying form).

2. ``integral_bruteforce``: hat I_k(xi) as the literal triple sum over
   chi + eta + zeta = xi in Xi with the kernels G_J, H_J, H_JM of eqs. approxG,
   approxH-J and approxH-JM evaluated per triple; phi_R and psi_R are computed
   here by numerical quadrature of their defining integrals, not from their
   closed forms.
"""
from __future__ import annotations

import numpy as np

from .qbe_oracle import Params, xi_axis, velocity_nodes, coarse_to_xi

SIGMA = np.array(
    [[[1, 0], [0, 1]], [[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]],
    dtype=np.complex128,
)


def _gl(n, a, b):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def trig_eval(fh: np.ndarray, p: Params, pts: np.ndarray) -> np.ndarray:
    """f(v) = sum_{xi in Xi} fhat(xi) exp(i pi xi.v/L) at points pts [P, 2]; fh [..., N, N]."""
    k = xi_axis(p)
    Ex = np.exp(1j * np.pi * pts[:, 0:1] * k[None, :] / p.L)
    Ey = np.exp(1j * np.pi * pts[:, 1:2] * k[None, :] / p.L)
    return np.einsum("pa,...ab,pb->...p", Ex, fh, Ey)


def _mat(wh, p, pts):
    """Matrices W(pts) [P, 2, 2] from Pauli coefficients wh [4, N, N]."""
    comps = trig_eval(wh, p, pts)                       # [4, P]
    return np.einsum("cp,cij->pij", comps, SIGMA)


def _tr(A):
    return np.trace(A, axis1=-2, axis2=-1)


def collision_direct(w: np.ndarray, p: Params, n_radial: int = 24, points=None):
    """C[W] at grid points by direct quadrature of the matrix-form integrand; returns Pauli [4, P].

    w: one cell, [4, N, N] real, band-limited.  points: optional list of (ix, iy) grid indices.
    """
    wh = coarse_to_xi(w.astype(np.complex128), Params(p.N, p.L, p.R, p.J, p.M, "keep"))
    vx, vy = velocity_nodes(p)
    if points is None:
        points = [(ix, iy) for ix in range(p.N) for iy in range(p.N)]
    V = np.array([[vx[i, j], vy[i, j]] for (i, j) in points])      # [P, 2]
    P = V.shape[0]
    eye = np.eye(2, dtype=np.complex128)
    W1 = _mat(wh, p, V)                                               # [P,2,2]
    J = p.J

    # ---- conservative part: C_c = -i [H_eff, W1] (eq. Cc, eq. Heff) ----
    rr, wr = _gl(n_radial, 0.0, p.R)
    Heff = np.zeros((P, 2, 2), dtype=np.complex128)
    ang = np.arange(2 * J) * np.pi / J
    angp = (np.arange(2 * J) + 0.5) * np.pi / J
    for ta in ang:
        th = np.array([np.cos(ta), np.sin(ta)])
        pts3 = (V[:, None, :] + rr[None, :, None] * th).reshape(-1, 2)
        W3 = _mat(wh, p, pts3).reshape(P, n_radial, 1, 2, 2)
        for tb in angp:
            thp = np.array([np.cos(tb), np.sin(tb)])
            pts4 = (V[:, None, :] + rr[None, :, None] * thp).reshape(-1, 2)
            W4 = _mat(wh, p, pts4).reshape(P, 1, n_radial, 2, 2)
            pts2 = (V[:, None, None, :] + rr[None, :, None, None] * th + rr[None, None, :, None] * thp).reshape(-1, 2)
            W2 = _mat(wh, p, pts2).reshape(P, n_radial, n_radial, 2, 2)
            F = (W3 @ W4 - W2 @ W3 - W3 @ W2 - _tr(W4)[..., None, None] * W3
                 + _tr(W2)[..., None, None] * W3 + W2)
            wt = (np.pi / J) ** 2 / float(th @ thp)
            Heff += wt * np.einsum("r,s,prsij->pij", wr, wr, F)
    Cc = -1j * (Heff @ W1 - W1 @ Heff)

    # ---- dissipative part: pi int int delta(u.u') (A + A^*) (eq. Cd) ----
    rs, ws = _gl(n_radial, -p.R, p.R)
    Cd = np.zeros((P, 2, 2), dtype=np.complex128)
    W1b = W1[:, None, None]
    for ta in np.arange(J) * np.pi / J:
        th = np.array([np.cos(ta), np.sin(ta)])
        tp = np.array([-np.sin(ta), np.cos(ta)])
        W3 = _mat(wh, p, (V[:, None, :] + rs[None, :, None] * th).reshape(-1, 2)).reshape(P, n_radial, 1, 2, 2)
        W4 = _mat(wh, p, (V[:, None, :] + rs[None, :, None] * tp).reshape(-1, 2)).reshape(P, 1, n_radial, 2, 2)
        pts2 = (V[:, None, None, :] + rs[None, :, None, None] * th + rs[None, None, :, None] * tp).reshape(-1, 2)
        W2 = _mat(wh, p, pts2).reshape(P, n_radial, n_radial, 2, 2)
        W2t, W4t = eye - W2, eye - W4
        tr = lambda X: _tr(X)[..., None, None]
        A = (-W4 @ W2t @ W3 + W4 * tr(W2t @ W3)
             - (W4t @ W3 - W4t @ W2 - W2t @ W3 + W4t * tr(W2) - W4t * tr(W3) + tr(W3 @ W2t) * eye) @ W1b)
        AA = A + np.conj(np.swapaxes(A, -1, -2))
        Cd += np.pi * (np.pi / J) * np.einsum("r,s,prsij->pij", ws, ws, AA)
    to_pauli = lambda X: (0.5 * np.einsum("pij,cji->cp", X, SIGMA))
    return to_pauli(Cc), to_pauli(Cd)


# ----------------------------------------------------------------------------
# Brute-force triple sums in Fourier space
# ----------------------------------------------------------------------------

def phi_numeric(s, p: Params, n=80):
    r, w = _gl(n, 0.0, p.R)
    return np.einsum("r,...r->...", w, np.sin(np.pi * np.asarray(s)[..., None] * r / p.L))


def psi_numeric(s, p: Params, n=80):
    r, w = _gl(n, -p.R, p.R)
    return np.einsum("r,...r->...", w, np.cos(np.pi * np.asarray(s)[..., None] * r / p.L))


def kernel_G(xi, chi, p: Params):
    """G_J(xi, chi) of eq. approxG; xi, chi [..., 2]."""
    J = p.J
    th = np.stack([np.cos(np.arange(J) * np.pi / J), np.sin(np.arange(J) * np.pi / J)], -1)
    thp = np.stack([np.cos((np.arange(J) + 0.5) * np.pi / J), np.sin((np.arange(J) + 0.5) * np.pi / J)], -1)
    w = -((2 * np.pi / J) ** 2) / (th @ thp.T)
    a = phi_numeric(xi @ th.T, p)          # [..., J]
    b = phi_numeric(chi @ thp.T, p)        # [..., J]
    return np.einsum("...j,jk,...k->...", a, w, b)


def kernel_HJ(xi, chi, p: Params):
    """H_J(xi, chi) of eq. approxH-J."""
    J = p.J
    t = np.arange(J) * np.pi / J
    th = np.stack([np.cos(t), np.sin(t)], -1)
    tp = np.stack([-np.sin(t), np.cos(t)], -1)
    return (np.pi / J) * np.sum(psi_numeric(xi @ th.T, p) * psi_numeric(chi @ tp.T, p), axis=-1)


def kernel_HJM(xi, chi, p: Params):
    """H_JM(xi, chi) of eq. approxH-JM (Gauss-Legendre radial nodes, exponential factor)."""
    J = p.J
    t = np.arange(J) * np.pi / J
    th = np.stack([np.cos(t), np.sin(t)], -1)
    tp = np.stack([-np.sin(t), np.cos(t)], -1)
    rho, wm = _gl(p.M, -p.R, p.R)
    ph = np.exp(1j * np.pi * (xi @ th.T)[..., None] * rho / p.L)      # [..., J, M]
    e = np.einsum("...jm,m->...j", ph, wm)
    return (np.pi / J) * np.sum(e * psi_numeric(chi @ tp.T, p), axis=-1)


def integral_bruteforce(kind: str, fh, gh, hh, p: Params):
    """hat I_kind on Xi by the literal triple sum; fh, gh, hh [N, N] coefficients on Xi."""
    k = xi_axis(p)
    N = p.N
    XI = np.stack(np.meshgrid(k, k, indexing="ij"), -1).reshape(-1, 2).astype(np.float64)   # [N^2, 2]
    fv, gv, hv = fh.reshape(-1), gh.reshape(-1), hh.reshape(-1)
    out = np.zeros(N * N, dtype=np.complex128)
    lo, hi = -N // 2, N // 2 - 1
    for ic in range(N * N):
        chi = XI[ic]
        eta = XI[None, :, :]
        zeta = XI[:, None, :]
        tot = chi[None, None, :] + eta + zeta                       # [zeta, eta, 2]
        ok = np.all((tot >= lo) & (tot <= hi), axis=-1)
        if not ok.any():
            continue
        zi, ei = np.nonzero(ok)
        z, e = XI[zi], XI[ei]
        c = np.broadcast_to(chi, z.shape)
        if kind == "I1":
            K = kernel_G(c + e, e, p)
        elif kind == "I2":
            K = kernel_HJ(c, e, p)
        elif kind == "I3":
            K = kernel_HJM(c + z, e + z, p)
        elif kind == "I4":
            K = kernel_HJ(c + e, e, p)
        else:
            raise ValueError(kind)
        val = fv[ic] * gv[ei] * hv[zi] * K
        tgt = tot[zi, ei]
        idx = (tgt[:, 0] - lo).astype(int) * N + (tgt[:, 1] - lo).astype(int)
        np.add.at(out, idx, val)
    return out.reshape(N, N)
