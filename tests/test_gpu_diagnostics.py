"""Diagnostics kernels (entropy, Fermi-Dirac fit, relative entropy, L1) against
the oracle, and the paper's entropy experiments reproduced qualitatively
(Sec. 5.3, Figs. 5-6: periodic inhomogeneous relaxation, global entropy
increasing, relative entropies decaying, global = local + local-to-global)."""
import numpy as np
import pytest

from oracle import diagnostics as D
from oracle import qbe_oracle as O
from paper_1408_1782_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qbe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    from paper_1408_1782_gb300 import qbe as q

    return q


def to_oracle(fit):
    return D.FDFit(T=fit.T, mu_up=fit.mu_up, mu_dn=fit.mu_dn, U=fit.U(), u=np.array(fit.u[:]), ok=bool(fit.ok))


def test_diagnostics_match_the_oracle(qbe):
    N, Nx = 32, 4
    p = O.Params(N=N)
    W = inputs.synthetic_w(N, Nx, seed=12, perturb=0.05)
    s = qbe.Solver(N, Nx, J=4, M=2)
    s.set_state(W)
    S = s.entropy()
    S_ref = D.entropy(W, p)
    assert np.abs(S - S_ref).max() < 1e-13 * np.abs(S_ref).max()
    loc = s.fd_fit()
    glob = s.fd_fit(global_fit=True)
    loc_ref = D.fit_local(W, p)
    glob_ref = D.fit_global(W, p)
    for a, b in zip(loc + [glob], loc_ref + [glob_ref]):
        assert a.ok == 1 and b.ok
        assert abs(a.T - b.T) < 1e-11 * b.T
        assert abs(a.mu_up - b.mu_up) < 1e-10 and abs(a.mu_dn - b.mu_dn) < 1e-10
    for ref, ref_o in ((loc, loc_ref), (glob, glob_ref)):
        rel, l1 = s.relative_entropy(ref)
        rel_o = D.relative_entropy(W, [to_oracle(f) for f in ref] if isinstance(ref, list) else to_oracle(ref), p)
        l1_o = D.l1_distance(W, [to_oracle(f) for f in ref] if isinstance(ref, list) else to_oracle(ref), p)
        assert np.abs(rel - rel_o).max() < 1e-11 * np.abs(rel_o).max()
        assert np.abs(l1 - l1_o).max() < 1e-12 * np.abs(l1_o).max()
    s.close()


def test_relative_entropy_rejects_unfitted_references(qbe):
    s = qbe.Solver(8, 2, J=4, M=2)
    s.set_state(inputs.synthetic_w(8, 2, seed=1))
    bad = qbe.QbeFermiDirac()
    with pytest.raises(qbe.QbeError):
        s.relative_entropy(bad)
    with pytest.raises(qbe.QbeError):
        s.relative_entropy([s.fd_fit(True)] * 3)         # neither 1 nor Nx references
    s.close()


def test_periodic_relaxation_entropy_experiment(qbe):
    """Sec. 5.3 parameters (N = 32, L = 12, J = M = 32, R = 7.5, dx = 0.1, dt = 0.008), B = 0, periodic,
    an x-dependent Fermi-Dirac-like initial state: the x-integrated entropy increases every step, the
    relative entropy to the global Fermi-Dirac state decreases, and S(W || F_glob) = S(W || F_loc) +
    S(F_loc || F_glob) (the last computed by the oracle from the fits; the identity is linear in W).
    The local relative entropy itself is not checked: the spectral operator does not preserve
    positivity, and W acquires eigenvalues down to about -3e-3 in the Fermi-Dirac tails within a few
    steps (the oracle shows the same), where -<s|W|s> log n_s with log n_s ~ -70 turns it negative."""
    N, Nx, dt, nsteps = 32, 10, 0.008, 12
    p = O.Params(N=N)
    W0 = inputs.synthetic_w(N, Nx, seed=3)
    s = qbe.Solver(N, Nx, J=32, M=32)
    s.set_state(W0)
    glob = s.fd_fit(global_fit=True)
    S_tot, rel_g, rel_l = [], [], []
    for k in range(nsteps + 1):
        if k:
            s.step(dt, 1)
        S_tot.append(s.entropy().mean())
        rel_g.append(s.relative_entropy(glob, with_l1=False)[0].mean())
        rel_l.append(s.relative_entropy(s.fd_fit(), with_l1=False)[0].mean())
    S_tot, rel_g, rel_l = map(np.array, (S_tot, rel_g, rel_l))
    assert np.all(np.diff(S_tot) > 0), np.diff(S_tot)
    assert np.all(np.diff(rel_g) < 0), np.diff(rel_g)
    # the identity on the final state
    W = s.get_state()
    loc = [to_oracle(f) for f in s.fd_fit()]
    F_loc = np.stack([np.moveaxis(0.5 * np.einsum("xyij,aji->xya", D.fd_state(f, p), O.SIGMA).real, -1, 0)
                      for f in loc])
    rhs = rel_l[-1] + D.relative_entropy(F_loc, to_oracle(glob), p).mean()
    assert abs(rel_g[-1] - rhs) < 1e-6 * rel_g[-1]
    # the global Fermi-Dirac state of the final state is the initial one (conserved moments)
    g2 = s.fd_fit(global_fit=True)
    assert abs(g2.T - glob.T) < 1e-4 * glob.T
    s.close()


def test_positivity_loss_of_the_spectral_operator_matches_the_oracle(qbe):
    """The paper's homogeneous example (eq. W0homogeneous, N = 32, J = M = 32, R = 7.5): one Heun step of
    0.008 takes the smallest eigenvalue of W from 0 to about -1.6e-3 (Fourier spectral collision operators do
    not preserve positivity); the library's state after the step equals the oracle's."""
    N, dt = 32, 0.008
    p = O.Params(N=N)
    W0 = inputs.homogeneous_w0(N)[None].copy()
    ref = O.collide_rk2(W0, np.zeros((1, 3)), dt, p)
    s = qbe.Solver(N, 1, J=32, M=32)
    s.set_state(W0)
    s.collide_rk2(dt)
    W = s.get_state()
    assert np.abs(W - ref).max() < 1e-13
    lam = np.linalg.eigvalsh(D.pauli_to_matrix(np.moveaxis(W, 1, -1)))
    lam_ref = np.linalg.eigvalsh(D.pauli_to_matrix(np.moveaxis(ref, 1, -1)))
    assert -2e-3 < lam.min() < -1e-3 and abs(lam.min() - lam_ref.min()) < 1e-13
    s.close()
