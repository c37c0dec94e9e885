"""Momentum and energy conservation of the oracle's discrete collision operator (Sec. 2: the
continuous operator conserves density, momentum and energy; Sec. 5.2, Fig. 2).  CPU only.

The continuous operator conserves momentum and energy because its integrand is symmetric under
the exchanges of the four collision velocities.  The discrete operator keeps that symmetry only
up to its quadrature (J, M) and the resolution of the state on the N x N grid, so its momentum
and energy defects must fall toward zero as the state becomes resolved.  A term with a wrong
sign, a dropped eta or a transposed operand in the component-0 equation breaks the symmetry
itself and leaves a defect of order one that does not converge (flipping the sign of the
eta_1 I3 terms gives relative rates of 0.5 at N = 32 and at N = 48).

Findings pinned here (paper's L = 12, R = 7.5, J = M = 32; eq. W0homogeneous):
* at N = 32 the defect is set by the Fermi-Dirac envelope (kT = 5/4 on a grid of spacing 0.75):
  the same state without its v-dependent rotation has nearly the same momentum rate;
* it falls spectrally with N for a smooth state (the kink of |v_y| in X(v) removed);
* the kink itself limits convergence at N = 48 and beyond.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import qbe_oracle as O
from paper_1408_1782_gb300 import inputs


@pytest.fixture(scope="module")
def mapper():
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        yield lambda f, it: pool.map(f, list(it), chunksize=1)


def _rates(w, p, mapper):
    """Relative rates |d mom/dt| / |mom| and |d E/dt| / E and the density defect of C[W] (Sec. 2
    moments eq. density, velocity, internal_energy; tr W = 2 w0)."""
    C = O.collision(w[None], p, mapper=mapper)
    rho, mom, en = O.moments(w[None], p)
    drho, dmom, den = O.moments(C, p)
    return (float(np.abs(dmom).max() / np.linalg.norm(mom)), float(abs(den[0]) / en[0]),
            float(np.abs(drho).max() / np.abs(rho).max()))


def test_momentum_energy_defects_converge_for_a_resolved_state(mapper):
    r32 = _rates(inputs.homogeneous_w0(32, vy_smoothing=0.5), O.Params(N=32), mapper)
    r48 = _rates(inputs.homogeneous_w0(48, vy_smoothing=0.5), O.Params(N=48), mapper)
    # N = 32: 2.6e-2 and 2.5e-3 per unit time; N = 48: 6.9e-5 and 1.5e-6
    assert r32[0] > 1e-2 and r32[1] > 1e-3
    assert r48[0] < 2e-4 and r48[1] < 5e-6
    assert r32[0] / r48[0] > 100 and r32[1] / r48[1] > 500
    assert r32[2] < 1e-9 and r48[2] < 1e-7          # density: quadrature level


def test_defect_at_n32_is_the_fermi_dirac_envelope(mapper):
    """The paper's state and the same state without its rotation (a pure Fermi-Dirac state in the
    basis U0, drifting with v0) have momentum rates within 15 % of each other at N = 32."""
    p = O.Params(N=32)
    paper = _rates(inputs.homogeneous_w0(32), p, mapper)
    fd = _rates(inputs.homogeneous_w0(32, rotation=0.0), p, mapper)
    assert abs(paper[0] - fd[0]) < 0.15 * paper[0]
    assert abs(paper[1] - fd[1]) < 0.15 * paper[1]


def test_kink_limits_convergence_at_n48(mapper):
    """With the |v_y| kink (the paper's X(v)) the N = 48 momentum rate is several times that of the
    smooth variant (4.7e-4 against 6.9e-5)."""
    p = O.Params(N=48)
    paper = _rates(inputs.homogeneous_w0(48), p, mapper)
    smooth = _rates(inputs.homogeneous_w0(48, vy_smoothing=0.5), p, mapper)
    assert paper[0] > 3 * smooth[0] and paper[1] > 5 * smooth[1]
