"""Forward-mode derivatives (tangents) of the oracle's maps.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests, the smoke
check and the benchmark's CPU baseline may import it.  The paper computes no
derivatives; these are the derivatives of the oracle's own discrete maps
(qbe_oracle), written from the chain rule in forward mode and sharing nothing
with the library's reverse-mode (adjoint) kernels, so that the identity
<lam, J dW> = <J^T lam, dW> checks the library's transposed products against
an independent derivation.

* C[W] is a polynomial of degree 3 in W (eq. CcPauli: D is quadratic, times w;
  eq. CdPauli: K2, K3, K4 times (1 - W) or {W, .}), so along a line
  C(W + e dW) is a cubic in e and the five-point difference
  [8 (C(h) - C(-h)) - (C(2h) - C(-2h))] / (12 h) is its exact derivative at
  e = 0 for every h (up to rounding).
* The ghost cells (Sec. 2) are an affine map of W: periodic wrap and copies
  are linear, the Dirichlet states are constant and the Maxwell wall adds
  alpha W_FD Fbar / Z with Fbar linear in W.  Its derivative is
  G(dW) - G(0).
* The minmod limiter (eq. minmod) is differentiated at the branch the forward
  state takes: d minmod(a, b) = da if |a| <= |b| and ab > 0, db if |b| < |a|
  and ab > 0, 0 if ab <= 0.
* Heun's RK2 for dW/dt = C[W] + 2 (B x w).sigma and the split step
  A(dt/2) o RK2(dt) o A(dt/2) of Sec. 4 by the chain rule, the precession
  term being bilinear in (B, W).
"""
from __future__ import annotations

import numpy as np

from . import qbe_oracle as O


def collision_jvp(w: np.ndarray, dw: np.ndarray, p: O.Params, mapper=map) -> np.ndarray:
    """dC/dW at w applied to dw (exact: five-point difference of a cubic)."""
    scale_w = max(float(np.abs(w).max()), 1e-300)
    scale_d = float(np.abs(dw).max())
    if scale_d == 0.0:
        return np.zeros_like(w)
    h = 0.25 * scale_w / scale_d
    c = {k: O.collision(w + k * h * dw, p, mapper=mapper) for k in (-2, -1, 1, 2)}
    return (8.0 * (c[1] - c[-1]) - (c[2] - c[-2])) / (12.0 * h)


def collision_vjp_brute(w: np.ndarray, lam: np.ndarray, p: O.Params, mapper=map) -> np.ndarray:
    """(dC/dW)^T lam by one exact directional derivative per input value (tiny grids only).

    All 4 N^2 unit directions of one cell are evaluated as a batch of cells
    (the cells of C are independent)."""
    ncells = w.shape[0]
    N = p.N
    K = 4 * N * N
    out = np.zeros_like(w)
    for c in range(ncells):
        base = np.repeat(w[c:c + 1], K, axis=0)
        units = np.eye(K).reshape(K, 4, N, N)
        jv = collision_jvp(base, units, p, mapper)           # [K, 4, N, N]: column k of the Jacobian
        out[c] = np.einsum("kaij,aij->k", jv, lam[c]).reshape(4, N, N)
    return out


def precession_jvp(w, B, dw, dB):
    """d[2 (B x w).sigma] = 2 (dB x w + B x dw).sigma."""
    return O.precession(dw, B) + O.precession(w, dB)


def ghosts_tangent(dW, p: O.Params, bc: O.Boundary):
    """Derivative of the ghost-cell extension (an affine map): G(dW) - G(0)."""
    return O._ghosts(dW, p, bc) - O._ghosts(np.zeros_like(dW), p, bc)


def minmod_tangent(a, b, da, db):
    return np.where(a * b > 0.0, np.where(np.abs(a) <= np.abs(b), da, db), 0.0)


def limiter_update_tangent(ext, dext, tau, dx, p: O.Params):
    """Derivative of eq. slopeLimiterStep at the extended state ext, applied to dext."""
    vx, _ = O.velocity_nodes(p)
    n = ext.shape[0] - 4
    a = ext[2:n + 4] - ext[1:n + 3]
    b = ext[1:n + 3] - ext[0:n + 2]
    da = dext[2:n + 4] - dext[1:n + 3]
    db = dext[1:n + 3] - dext[0:n + 2]
    dS = np.zeros_like(ext)
    dS[1:n + 3] = minmod_tangent(a, b, da, db)
    nu = tau * vx / dx
    lim = 0.5 * (np.sign(nu) - nu)
    dWm1, dW0, dWp1 = dext[1:n + 1], dext[2:n + 2], dext[3:n + 3]
    dSm1, dS0, dSp1 = dS[1:n + 1], dS[2:n + 2], dS[3:n + 3]
    godunov = -vx * (dWp1 - dWm1) + np.abs(vx) * (dWp1 - 2.0 * dW0 + dWm1)
    limiter = lim * (-vx * (dSp1 - dSm1) + np.abs(vx) * (dSp1 - 2.0 * dS0 + dSm1))
    return dW0 + (tau / (2.0 * dx)) * (godunov + limiter)


def advect_jvp(W, dW, tau, p: O.Params, bc: O.Boundary):
    """(A(tau) W, dA(tau) dW) with the same sub-cycling as the oracle's advect."""
    Nx = W.shape[0]
    dx = 1.0 / Nx
    s = O.transport_substeps(tau, dx, p)
    for _ in range(s):
        ext = O._ghosts(W, p, bc)
        dext = ghosts_tangent(dW, p, bc)
        W, dW = O.limiter_update(ext, tau / s, dx, p), limiter_update_tangent(ext, dext, tau / s, dx, p)
    return W, dW


def collide_rk2_jvp(W, B, dt, p: O.Params, dW, dB, mapper=map):
    """Heun's RK2 for C + precession and its derivative in (W, B)."""
    F0 = O.rhs(W, B, p)
    dF0 = collision_jvp(W, dW, p, mapper) + precession_jvp(W, B, dW, dB)
    W1 = W + dt * F0
    dW1 = dW + dt * dF0
    F1 = O.rhs(W1, B, p)
    dF1 = collision_jvp(W1, dW1, p, mapper) + precession_jvp(W1, B, dW1, dB)
    return W + 0.5 * dt * (F0 + F1), dW + 0.5 * dt * (dF0 + dF1)


def step_jvp(W, B, dt, p: O.Params, bc: O.Boundary, dW, dB, mapper=map):
    """One split step A(dt/2) o RK2(dt) o A(dt/2) and its derivative in (W, B)."""
    W, dW = advect_jvp(W, dW, 0.5 * dt, p, bc)
    W, dW = collide_rk2_jvp(W, B, dt, p, dW, dB, mapper)
    W, dW = advect_jvp(W, dW, 0.5 * dt, p, bc)
    return W, dW


def evolve_jvp(W, B, dt, nsteps, p: O.Params, bc: O.Boundary, dW, dB, mapper=map):
    for _ in range(nsteps):
        W, dW = step_jvp(W, B, dt, p, bc, dW, dB, mapper)
    return W, dW


def observables(W, p: O.Params):
    """[P_z, Phi_E]: dx dv^2 sum 2 w3 and dx dv^2 sum v_x |v|^2/2 2 w0 over all cells and velocities."""
    vx, vy = O.velocity_nodes(p)
    Nx = W.shape[0]
    w = (1.0 / Nx) * O.delta_v(p) ** 2
    pz = w * np.sum(2.0 * W[:, 3])
    phie = w * np.sum(vx * 0.5 * (vx**2 + vy**2) * 2.0 * W[:, 0])
    return np.array([pz, phie])
