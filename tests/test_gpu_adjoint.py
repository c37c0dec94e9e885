"""Adjoint (transposed-derivative) products of the library against the oracle.

* (dC/dW)^T lam element by element against the oracle's column-by-column
  transpose (tests/golden/collision_vjp_n8.npz), and through the identity
  <lam, J dW> = <J^T lam, dW> with J dW the oracle's exact directional
  derivative (oracle/tangent.py: C is cubic, the five-point difference is
  exact) at N = 16, 32 and, for one cell, at the paper's N = 64, J = M = 32.
  Both sides are FP64 sums of O(10^4) products of O(1) terms: the identity is
  held to 1e-11 of the sum of the absolute products.
* The split step's reverse sweep (qbe_step_checkpointed + qbe_step_vjp)
  against the oracle's forward-mode derivative of the same steps, in W and B
  together, for every boundary condition, over several checkpoint segments.
* FP64 central differences (h = 1e-6) of the final-time observables (spin
  polarisation P_z and energy flux Phi_E) computed by the library's own
  forward steps, along relative directions dW = r W (an absolute perturbation
  would flip the minmod branches of the Fermi-Dirac tails, where slopes are
  ~0) and along random field directions dB.
* The FP32-split form of the product against the FP64 form (same tolerances
  as the forward FP32-split form: 5e-6 of the maximum).
"""
import os

import numpy as np
import pytest

from oracle import qbe_oracle as O
from oracle import tangent as T
from paper_1408_1782_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL_ID = 1e-11


@pytest.fixture(scope="module")
def qbe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    from paper_1408_1782_gb300 import qbe as q

    return q


@pytest.fixture(scope="module")
def pool():
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as p:
        yield lambda f, it: p.map(f, list(it), chunksize=1)


def vjp(q, w, lam, N, J, M, precision=0):
    s = q.Solver(N, w.shape[0], J=J, M=M, precision=precision)
    g = s.collide_vjp(np.ascontiguousarray(w), np.ascontiguousarray(lam))
    s.close()
    return g


def identity_gap(lam, jv, g, dw):
    """|<lam, J dw> - <g, dw>| relative to the sum of absolute products."""
    a, b = np.sum(lam * jv), np.sum(g * dw)
    scale = np.sum(np.abs(lam * jv)) + np.sum(np.abs(g * dw))
    return abs(a - b) / scale


def test_collide_vjp_matches_oracle_columns_n8(qbe):
    d = np.load(os.path.join(GOLDEN, "collision_vjp_n8.npz"))
    g = vjp(qbe, d["W"], d["lam"], 8, 4, 2)
    err = np.abs(g - d["grad"]).max() / np.abs(d["grad"]).max()
    assert err < 1e-12, err


def test_collide_vjp_fp32_split_n8(qbe):
    d = np.load(os.path.join(GOLDEN, "collision_vjp_n8.npz"))
    g = vjp(qbe, d["W"], d["lam"], 8, 4, 2, precision=1)
    err = np.abs(g - d["grad"]).max() / np.abs(d["grad"]).max()
    assert err < 5e-6, err


@pytest.mark.parametrize("N,J,M,ncells,lam_kind", [
    (16, 8, 8, 3, "random"), (16, 8, 8, 2, "density"), (16, 8, 8, 2, "energy"), (32, 8, 4, 2, "random"),
    (48, 4, 4, 1, "random"),
])
def test_collide_vjp_transpose_identity(qbe, pool, N, J, M, ncells, lam_kind):
    """lam = 1 on w0 (density) and |v|^2/2 on w0 (energy) are conserved quantities of C: the products
    then measure the conservation defect of the discrete operator, on both sides alike."""
    p = O.Params(N=N, J=J, M=M)
    w = inputs.synthetic_w(N, ncells, seed=40 + N, perturb=0.05)
    dw = inputs.random_field(w.shape, seed=41 + N, scale=0.05)
    if lam_kind == "random":
        lam = inputs.random_field(w.shape, seed=42 + N)
    else:
        vx, vy = O.velocity_nodes(p)
        lam = np.zeros_like(w)
        lam[:, 0] = 1.0 if lam_kind == "density" else 0.5 * (vx**2 + vy**2)
    jv = T.collision_jvp(w, dw, p, mapper=pool)
    g = vjp(qbe, w, lam, N, J, M)
    assert identity_gap(lam, jv, g, dw) < TOL_ID


def test_collide_vjp_transpose_identity_paper_grid(qbe, pool):
    """One cell of the N = 64 Dirichlet workload at J = M = 32 (the paper's quadrature)."""
    wl = inputs.WORKLOADS["plain_fp64_n64"]
    N = wl["N"]
    p = O.Params(N=N, J=32, M=32)
    w = inputs.synthetic_w(N, wl["Nx"], L=wl["L"], seed=0, perturb=wl["perturb"])[77:78].copy()
    dw = inputs.random_field(w.shape, seed=3, scale=0.05)
    lam = inputs.random_field(w.shape, seed=4)
    jv = T.collision_jvp(w, dw, p, mapper=pool)
    g = vjp(qbe, w, lam, N, 32, 32)
    assert identity_gap(lam, jv, g, dw) < TOL_ID


def test_collide_vjp_fp32_split_matches_fp64_n64(qbe):
    wl = inputs.WORKLOADS["plain_fp64_n64"]
    W = inputs.synthetic_w(wl["N"], 16, L=wl["L"], seed=0, perturb=wl["perturb"])
    lam = inputs.random_field(W.shape, seed=5)
    g64 = vjp(qbe, W, lam, 64, 32, 32, 0)
    g32 = vjp(qbe, W, lam, 64, 32, 32, 1)
    err = np.abs(g32 - g64).max() / np.abs(g64).max()
    assert err < 5e-6, err


@pytest.mark.parametrize("ncells,J,M", [(3, 8, 6), (20, 8, 7)])
def test_collide_vjp_i3_variants_agree(qbe, ncells, J, M):
    """FP32-split, N = 64: the warp-local I3 transpose (variant 0, the default) and the element-pass
    kernel (variant 1) against the FP64 product.  (3, 8, 6): one m per work unit; (20, 8, 7): m-chunks
    of two with a ragged last chunk, so the partials accumulate over m inside a unit."""
    import torch

    N = 64
    W = inputs.synthetic_w(N, ncells, seed=33, perturb=0.05)
    lam = inputs.random_field(W.shape, seed=34)
    g64 = vjp(qbe, W, lam, N, J, M, 0)
    s = qbe.Solver(N, ncells, J=J, M=M, precision=1)
    assert s.vjp_i3_variant() == (0, 2)
    w, l = torch.from_numpy(W).cuda(), torch.from_numpy(lam).cuda()
    out = []
    for v in (0, 1):
        s.set_vjp_i3_variant(v)
        assert s.vjp_i3_variant()[0] == v
        out.append(s.collide_vjp(w, l).cpu().numpy())
        err = np.abs(out[-1] - g64).max() / np.abs(g64).max()
        assert err < 5e-6, (v, err)
    with pytest.raises(qbe.QbeError):
        s.set_vjp_i3_variant(2)
    s.set_vjp_i3_variant(-1)
    assert s.vjp_i3_variant()[0] == 0
    assert np.array_equal(s.collide_vjp(w, l).cpu().numpy(), out[0])
    s.close()
    s64 = qbe.Solver(N, 1, J=4, M=2, precision=0)
    assert s64.vjp_i3_variant() == (0, 1)
    s64.close()


def test_collide_vjp_fp32_split_matches_fp64_largest_grid(qbe):
    """N = 128 (the staged FP32 transpose on the 256-point grid), two cotangents in one product
    against the FP64 form's single products."""
    import torch

    N, J, M, ncells = 128, 4, 4, 2
    W = inputs.synthetic_w(N, ncells, seed=31, perturb=0.05)
    lams = np.stack([inputs.random_field(W.shape, seed=32 + k) for k in range(2)])
    s = qbe.Solver(N, ncells, J=J, M=M, precision=1)
    g32 = s.collide_vjp_many(torch.from_numpy(W).cuda(), torch.from_numpy(lams).cuda()).cpu().numpy()
    s.close()
    for k in range(2):
        g64 = vjp(qbe, W, lams[k], N, J, M, 0)
        err = np.abs(g32[k] - g64).max() / np.abs(g64).max()
        assert err < 5e-6, (k, err)


@pytest.mark.parametrize("precision,N", [(0, 8), (1, 16), (1, 48), (1, 96)])
def test_collide_vjp_many_equals_single_products(qbe, precision, N):
    """qbe_collide_vjp_n: five cotangents at one state give exactly the single products.  The staged
    transpose kernels (FP64 at N = 8, FP32 at N = 96) carry them as a group of four sharing the state's
    transforms and a group of one; the FP32 shared-memory kernel (N = 16, 48) one at a time."""
    import torch

    J, M, ncells, ncot = 4, 3, 3, 5
    w = inputs.synthetic_w(N, ncells, seed=71, perturb=0.05)
    lams = np.stack([inputs.random_field(w.shape, seed=72 + k) for k in range(ncot)])
    s = qbe.Solver(N, ncells, J=J, M=M, precision=precision)
    wd = torch.from_numpy(w).cuda()
    got = s.collide_vjp_many(wd, torch.from_numpy(lams).cuda()).cpu().numpy()
    for k in range(ncot):
        one = s.collide_vjp(w, lams[k])
        assert np.array_equal(got[k], one), k
    # argument errors: null pointers, host memory
    assert qbe.lib().qbe_collide_vjp_n(s._h, 2, None, None, None, ncells, 1) == qbe.QBE_ERR_ARG
    assert qbe.lib().qbe_collide_vjp_n(s._h, 1, w.ctypes.data, lams.ctypes.data, lams.ctypes.data, ncells,
                                       0) == qbe.QBE_ERR_ARG
    s.close()


def test_collide_vjp_batches_and_device_memory(qbe):
    """More cells than one batch of the handle, device pointers, grad aliasing lam."""
    import torch

    N, J, M = 16, 8, 8
    w = inputs.synthetic_w(N, 5, seed=8, perturb=0.05)
    lam = inputs.random_field(w.shape, seed=9)
    ref = vjp(qbe, w, lam, N, J, M)
    s = qbe.Solver(N, 2, J=J, M=M)                       # batch of 2 cells: 3 batches
    wd = torch.from_numpy(w).cuda()
    ld = torch.from_numpy(lam).cuda()
    s.collide_vjp(wd, ld, out=ld)
    torch.cuda.synchronize()
    assert np.abs(ld.cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max()
    s.close()


def boundary(kind):
    fdL = (1.0, 0.2, -0.3, np.eye(2))
    fdR = (0.8, 0.0, 0.1, np.eye(2))
    return fdL, fdR, O.Boundary(kind, fdL, fdR, alpha=0.6)


def gpu_solver(q, N, Nx, J, M, kind, precision=0, R=7.5):
    fdL, fdR, _ = boundary(kind)
    s = q.Solver(N, Nx, J=J, M=M, R=R, precision=precision)
    s.set_boundary(kind, q.fd_state(*fdL), q.fd_state(*fdR), alpha=0.6)
    return s


@pytest.mark.parametrize("N,Nx,J,M,nsteps,ties", [(8, 5, 4, 2, 3, False), (8, 5, 4, 2, 3, True),
                                                   (8, 1, 4, 2, 2, False), (64, 4, 2, 1, 1, True)])
@pytest.mark.parametrize("kind", ["periodic", "dirichlet", "maxwell"])
def test_step_vjp_transpose_identity(qbe, pool, kind, N, Nx, J, M, nsteps, ties):
    """Split steps with checkpoint segments of two steps, B != 0.  R = 2 keeps the explicit RK2
    stable on the coarse N = 8 grid (at R = 7.5, |C| ~ 26 and dt = 0.01 diverges).  At N = 8 a warp
    spans velocity rows of both signs of v_x; at N = 64 every warp is within one row.  With ties
    the state's x-differences are exactly 0 or 1/64 (inputs.minmod_tie_w), so that every minmod
    pair with ab > 0 away from the walls is a tie |a| = |b| in the first transport sub-step and the
    tie convention of eq. minmod (a's branch) decides the derivative."""
    R = 2.0
    dt = 0.01
    p = O.Params(N=N, J=J, M=M, R=R)
    _, _, bc = boundary(kind)
    W = inputs.minmod_tie_w(N, Nx, seed=50) if ties else inputs.synthetic_w(N, Nx, seed=50, perturb=0.05)
    B = inputs.uniform_b(Nx, (0.3, -0.2, 0.5)) + inputs.random_field((Nx, 3), seed=51, scale=0.2)
    dW = inputs.random_field(W.shape, seed=52, scale=0.05)
    dB = inputs.random_field(B.shape, seed=53, scale=0.5)
    lam = inputs.random_field(W.shape, seed=54)
    Wn, jv = T.evolve_jvp(W, B, dt, nsteps, p, bc, dW, dB, mapper=pool)
    s = gpu_solver(qbe, N, Nx, J, M, kind, R=R)
    s.set_state(W)
    s.set_bfield(B)
    s.step_checkpointed(dt, nsteps, 2)
    assert np.abs(s.get_state() - Wn).max() < 1e-13
    lam0, gB = s.step_vjp(lam)
    a = np.sum(lam * jv)
    b = np.sum(lam0 * dW) + np.sum(gB * dB)
    scale = np.sum(np.abs(lam * jv)) + np.sum(np.abs(lam0 * dW)) + np.sum(np.abs(gB * dB))
    assert abs(a - b) / scale < TOL_ID
    # the state is W_n again and the tape can be swept a second time
    assert np.abs(s.get_state() - Wn).max() < 1e-13
    lam0b, gBb = s.step_vjp(lam)
    assert np.array_equal(lam0b, lam0) and np.array_equal(gBb, gB)
    s.close()


def test_step_vjp_segment_length_does_not_matter(qbe):
    N, Nx, J, M = 8, 4, 4, 2
    W = inputs.synthetic_w(N, Nx, seed=60, perturb=0.05)
    B = inputs.uniform_b(Nx, (0.1, 0.2, 0.3))
    lam = inputs.random_field(W.shape, seed=61)
    out = []
    for every in (1, 3, 5, 9):
        s = gpu_solver(qbe, N, Nx, J, M, "maxwell", R=2.0)
        s.set_state(W)
        s.set_bfield(B)
        s.step_checkpointed(0.01, 5, every)
        out.append(s.step_vjp(lam))
        s.close()
    for l0, gb in out[1:]:
        assert np.array_equal(l0, out[0][0]) and np.array_equal(gb, out[0][1])


@pytest.mark.parametrize("precision", [0, 1])
def test_full_tape_equals_checkpointed_tape(qbe, precision):
    """qbe_step_taped keeps every intermediate state of the forward; its reverse sweep (no
    recomputation) equals the checkpointed sweep bit for bit, for one and for several cotangents,
    and the forward itself equals plain stepping."""
    N, Nx, J, M = 16, 4, 4, 3
    W = inputs.synthetic_w(N, Nx, seed=62, perturb=0.05)
    B = inputs.uniform_b(Nx, (0.1, 0.2, 0.3))
    lams = np.stack([inputs.random_field(W.shape, seed=63 + k) for k in range(2)])
    dt, nsteps = 0.01, 4
    s = gpu_solver(qbe, N, Nx, J, M, "maxwell", precision=precision, R=2.0)
    s.set_state(W)
    s.set_bfield(B)
    s.step(dt, nsteps)
    Wn = s.get_state()
    s.set_state(W)
    s.step_checkpointed(dt, nsteps, 3)
    ref = [s.step_vjp(lams[k].copy()) for k in range(2)]
    ref_many = s.step_vjp_many(lams)
    s.set_state(W)
    s.step_taped(dt, nsteps)
    assert np.array_equal(s.get_state(), Wn)
    got = [s.step_vjp(lams[k].copy()) for k in range(2)]
    got_many = s.step_vjp_many(lams)
    assert np.array_equal(s.get_state(), Wn)
    for k in range(2):
        assert np.array_equal(got[k][0], ref[k][0]) and np.array_equal(got[k][1], ref[k][1]), k
    assert np.array_equal(got_many[0], ref_many[0]) and np.array_equal(got_many[1], ref_many[1])
    s.step_checkpointed(dt, 2, 1)       # a checkpointed forward after a full tape sweeps its own tape
    a = s.step_vjp(lams[0].copy())
    s.set_state(Wn)
    s.step_checkpointed(dt, 2, 2)
    b = s.step_vjp(lams[0].copy())
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    s.close()


def test_full_tape_that_does_not_fit_fails_cleanly(qbe):
    """A full tape larger than the device memory: QBE_ERR_ALLOC before any step, the state unchanged,
    no valid tape afterwards; a checkpointed tape still works on the same handle."""
    N, Nx = 16, 4
    W = inputs.synthetic_w(N, Nx, seed=64, perturb=0.05)
    s = qbe.Solver(N, Nx, J=4, M=2)
    s.set_state(W)
    with pytest.raises(qbe.QbeError):
        s.step_taped(0.01, 2_000_000_000)        # about 2.6e14 bytes of intermediate states
    assert np.array_equal(s.get_state(), W)
    with pytest.raises(qbe.QbeError):
        s.step_vjp(np.zeros_like(W))
    s.step_checkpointed(0.01, 2, 1)
    lam0, _ = s.step_vjp(inputs.random_field(W.shape, seed=65))
    assert np.isfinite(lam0).all()
    s.close()


def observables_grad(s, W, B, dt, nsteps, every):
    s.set_state(W)
    s.set_bfield(B)
    s.step_checkpointed(dt, nsteps, every)
    out = []
    for k in range(2):
        gbar = np.zeros(2)
        gbar[k] = 1.0
        lam = s.observables_vjp(gbar)
        out.append(s.step_vjp(lam))
    return out


def observables_after(s, W, B, dt, nsteps):
    s.set_state(W)
    s.set_bfield(B)
    s.step(dt, nsteps)
    return s.observables()


@pytest.mark.parametrize("kind,h", [("periodic", 1e-6), ("dirichlet", 1e-6), ("maxwell", 1e-7)])
def test_observable_gradients_against_central_differences(qbe, kind, h):
    """The transport is piecewise linear (minmod), so a central difference is only a derivative when no
    branch switch lies within +-h along the direction.  For this Maxwell state one lies between 1e-7 and
    1e-6 (the oracle's own forward-mode derivative against the oracle's own differences: relative gap
    1.7e-5 at h = 1e-5, 5.1e-6 at 1e-6, 1.1e-9 at 1e-7); the library's adjoint agrees with the oracle's
    derivative to 1e-11 (test_step_vjp_transpose_identity), so the Maxwell case is checked at h = 1e-7."""
    N, Nx, J, M = 16, 6, 8, 8
    dt, nsteps = 0.005, 4
    W = inputs.synthetic_w(N, Nx, seed=70, perturb=0.05)
    B = inputs.uniform_b(Nx, (0.3, -0.2, 0.5)) + inputs.random_field((Nx, 3), seed=71, scale=0.2)
    dW = inputs.random_field(W.shape, seed=72) * W
    dB = inputs.random_field(B.shape, seed=73)
    s = gpu_solver(qbe, N, Nx, J, M, kind)
    grads = observables_grad(s, W, B, dt, nsteps, 3)
    fp = observables_after(s, W + h * dW, B + h * dB, dt, nsteps)
    fm = observables_after(s, W - h * dW, B - h * dB, dt, nsteps)
    fd = (fp - fm) / (2 * h)
    for k in range(2):
        lam0, gB = grads[k]
        ad = np.sum(lam0 * dW) + np.sum(gB * dB)
        assert abs(ad - fd[k]) <= 1e-7 * max(abs(fd[k]), np.sum(np.abs(lam0 * dW)) + np.sum(np.abs(gB * dB))), \
            (k, ad, fd[k])
    s.close()


def test_spin_polarisation_gradient_without_field_is_conserved(qbe):
    """With B = 0 and periodic walls the total spin is conserved by transport and collision, so
    dP_z(W_n)/dW_0 = dP_z/dW (2 dx dv^2 on w3) up to the operator's conservation defect.  J = M = 32:
    at N = 16 the quadratures then conserve to round-off (oracle: |sum_v C_a| / sum_v |C_a| ~ 1e-15;
    at J = M = 8 the defect is 1e-2 for w0 and 1e-4 for the spin components)."""
    N, Nx, J, M = 16, 6, 32, 32
    W = inputs.synthetic_w(N, Nx, seed=80, perturb=0.05)
    s = gpu_solver(qbe, N, Nx, J, M, "periodic")
    (lam0, gB), _ = observables_grad(s, W, np.zeros((Nx, 3)), 0.005, 3, 2)
    direct = s.observables_vjp(np.array([1.0, 0.0]))
    assert np.abs(lam0 - direct).max() < 1e-6 * np.abs(direct).max()
    s.close()


def test_observables_match_oracle(qbe):
    N, Nx = 16, 5
    W = inputs.synthetic_w(N, Nx, seed=90, perturb=0.05)
    s = qbe.Solver(N, Nx, J=4, M=2)
    s.set_state(W)
    ref = T.observables(W, O.Params(N=N, J=4, M=2))
    assert np.abs(s.observables() - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(s.observables(W) - ref).max() < 1e-13 * np.abs(ref).max()
    s.close()


def test_step_vjp_needs_a_valid_tape(qbe):
    N, Nx = 8, 3
    W = inputs.synthetic_w(N, Nx, seed=91)
    s = qbe.Solver(N, Nx, J=4, M=2)
    s.set_state(W)
    with pytest.raises(qbe.QbeError):
        s.step_vjp(np.zeros_like(W))
    s.step_checkpointed(0.01, 2, 1)
    s.set_state(W)                      # invalidates the tape
    with pytest.raises(qbe.QbeError):
        s.step_vjp(np.zeros_like(W))
    s.close()


def test_autograd_functions(qbe):
    """torch.autograd: evolve + observables backward equals the direct products, and a second forward
    on the same solver before backward re-records the tape."""
    import torch

    from paper_1408_1782_gb300 import autograd as A

    N, Nx, J, M = 8, 4, 4, 2
    dt, nsteps = 0.01, 3
    W = inputs.synthetic_w(N, Nx, seed=95, perturb=0.05)
    B = inputs.uniform_b(Nx, (0.2, 0.1, -0.3))
    s = gpu_solver(qbe, N, Nx, J, M, "maxwell", R=2.0)
    (ref_l, ref_b), (ref_l2, ref_b2) = observables_grad(s, W, B, dt, nsteps, 2)
    W0 = torch.from_numpy(W).cuda().requires_grad_(True)
    B0 = torch.from_numpy(B).cuda().requires_grad_(True)
    Wn = A.evolve(s, W0, B0, dt, nsteps, 2)
    other = A.evolve(s, W0.detach() * 0.5, B0.detach(), dt, 1, 1)   # overwrites the solver's tape
    obs = A.observables(s, Wn)
    obs[0].backward()
    assert np.abs(W0.grad.cpu().numpy() - ref_l).max() <= 1e-14 * np.abs(ref_l).max()
    assert np.abs(B0.grad.cpu().numpy() - ref_b).max() <= 1e-14 * np.abs(ref_b).max()
    # the collision operator's autograd node
    w = torch.from_numpy(W[:2]).cuda().requires_grad_(True)
    c = A.collide(s, w)
    lam = torch.from_numpy(inputs.random_field(c.shape, seed=96)).cuda()
    (c * lam).sum().backward()
    ref = s.collide_vjp(W[:2].copy(), lam.cpu().numpy())
    assert np.abs(w.grad.cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max()
    del other
    # checkpoint_every = 0: the full tape, the same gradients
    W1 = torch.from_numpy(W).cuda().requires_grad_(True)
    B1 = torch.from_numpy(B).cuda().requires_grad_(True)
    A.observables(s, A.evolve(s, W1, B1, dt, nsteps, 0))[0].backward()
    assert torch.equal(W1.grad, W0.grad) and torch.equal(B1.grad, B0.grad)
    s.close()


@pytest.mark.parametrize("precision,N,ncot", [(0, 8, 2), (1, 16, 5)])
def test_step_vjp_for_several_cotangents_in_one_sweep(qbe, precision, N, ncot):
    """One reverse sweep for several cotangents equals one sweep per cotangent, bitwise: the
    cotangents of a group share the state's transforms of each collision product but none of their
    own arithmetic.  Precision 0 (staged FP64 transpose) carries the two cotangents as one group;
    precision 1 at N = 16 (shared-memory FP32 transpose) sweeps five cotangents one at a time."""
    Nx, J, M = 4, 4, 2
    W = inputs.synthetic_w(N, Nx, seed=97, perturb=0.05)
    B = inputs.uniform_b(Nx, (0.1, -0.3, 0.2))
    s = gpu_solver(qbe, N, Nx, J, M, "maxwell", precision=precision, R=2.0)
    s.set_state(W)
    s.set_bfield(B)
    s.step_checkpointed(0.01, 5, 2)
    lams = [s.observables_vjp(np.array([1.0, 0.0])), s.observables_vjp(np.array([0.0, 1.0]))]
    lams += [inputs.random_field(W.shape, seed=98 + k) for k in range(ncot - 2)]
    lams = np.stack(lams)
    l0, gb = s.step_vjp_many(lams)
    for k in range(ncot):
        a, b = s.step_vjp(lams[k].copy())
        assert np.array_equal(a, l0[k]) and np.array_equal(b, gb[k]), k
    s.close()


def test_step_vjp_fp32_split_matches_fp64(qbe):
    """The reverse sweep of the FP32-split form against the FP64 form (N = 16, J = M = 8, four steps with
    a field and Maxwell walls): the FP32 collision products carry the FP32-split tolerance."""
    N, Nx, J, M = 16, 5, 8, 8
    W = inputs.synthetic_w(N, Nx, seed=98, perturb=0.05)
    B = inputs.uniform_b(Nx, (0.2, -0.1, 0.4))
    out = []
    for prec in (0, 1):
        s = gpu_solver(qbe, N, Nx, J, M, "maxwell", precision=prec)
        s.set_state(W)
        s.set_bfield(B)
        s.step_checkpointed(0.005, 4, 2)
        lam = s.observables_vjp(np.array([1.0, 0.5]))
        out.append(s.step_vjp(lam))
        s.close()
    (l64, b64), (l32, b32) = out
    assert np.abs(l32 - l64).max() < 5e-6 * np.abs(l64).max()
    assert np.abs(b32 - b64).max() < 5e-6 * np.abs(b64).max()
