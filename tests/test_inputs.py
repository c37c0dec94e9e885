"""The seeded input generators (paper_1408_1782_gb300/inputs.py) have the structure the tests that
use them rely on; CPU only."""
import numpy as np
import pytest

from oracle import qbe_oracle as O
from paper_1408_1782_gb300 import inputs


@pytest.mark.parametrize("N,Nx", [(8, 5), (64, 4)])
def test_minmod_tie_state_makes_every_limited_pair_a_tie(N, Nx):
    """minmod_tie_w: the x-differences are exactly 0 or 1/64, so away from the walls every minmod
    argument pair with ab > 0 is an exact tie |a| = |b|, and there are such pairs."""
    W = inputs.minmod_tie_w(N, Nx, seed=50)
    d = np.diff(W, axis=0)
    assert np.all((d == 0.0) | (d == 1.0 / 64.0))
    ext = O._ghosts(W, O.Params(N=N), O.Boundary("periodic"))
    # pair i: a = W(m + 1) - W(m), b = W(m) - W(m - 1) with m = i - 1 (ext holds two ghosts per side);
    # keep m = 1 .. Nx - 2, whose three cells are interior (the periodic wrap breaks the ramp)
    a = ext[2:-1] - ext[1:-2]
    b = ext[1:-2] - ext[:-3]
    inner = slice(2, Nx - 1)
    a, b = a[inner], b[inner]
    limited = a * b > 0.0
    assert limited.sum() > 0
    assert np.all(np.abs(a[limited]) == np.abs(b[limited]))


def test_synthetic_state_is_hermitian_in_range_and_seeded():
    """synthetic_w: eigenvalues of W(x, v) in [0, 1] (a Fermi-Dirac-like state rotated by SU(2)),
    reproducible per seed, different across seeds."""
    W = inputs.synthetic_w(16, 3, seed=7)
    w0, w = W[:, 0], W[:, 1:]
    r = np.sqrt((w ** 2).sum(axis=1))
    assert np.all(w0 - r >= -1e-12) and np.all(w0 + r <= 1.0 + 1e-12)
    assert np.array_equal(W, inputs.synthetic_w(16, 3, seed=7))
    assert not np.array_equal(W, inputs.synthetic_w(16, 3, seed=8))
