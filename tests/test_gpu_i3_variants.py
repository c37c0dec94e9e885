"""Launch variants of the I3 (Hu-Ying term, eq. approxH-JM) kernel and the autotuner that picks among
them: every variant of every size computes C[W] within the form's tolerance of the oracle (FP64) or of
the plain FP64 GPU form (FP32-split), and qbe_autotune leaves a valid shape whose results agree."""
import numpy as np
import pytest

from oracle import qbe_oracle as O
from paper_1408_1782_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-11      # max |dC| / max |C| against the oracle (the parity tests' bound)
TOL_F32 = 5e-6       # the FP32-split form's stated bound


@pytest.fixture(scope="module")
def qbe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    from paper_1408_1782_gb300 import qbe as q

    return q


def _collide_all_variants(q, w, N, J, M, prec):
    import torch

    s = q.Solver(N, w.shape[0], J=J, M=M, stream=torch.cuda.current_stream(), precision=prec)
    wd = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    out = {}
    for v in range(s.i3_shape()["nvariants"]):
        s.set_i3_shape(variant=v)
        assert s.i3_shape()["variant"] == v and s.i3_variant_name(v)
        out[v] = s.collide(wd).cpu().numpy()
    assert s.i3_variant_name(s.i3_shape()["nvariants"]) is None
    s.close()
    return out


@pytest.mark.parametrize("N,J,M,ncells", [(16, 8, 6, 3), (48, 4, 2, 1), (64, 4, 3, 2)])
def test_fp64_variants_match_oracle(qbe, N, J, M, ncells):
    w = inputs.synthetic_w(N, ncells, seed=40 + N, perturb=0.05)
    ref = O.collision(w, O.Params(N=N, J=J, M=M))
    res = _collide_all_variants(qbe, w, N, J, M, 0)
    assert len(res) == 4
    for v, got in res.items():
        assert np.abs(got - ref).max() < TOL_F64 * np.abs(ref).max(), v


@pytest.mark.parametrize("N,J,M,ncells", [(32, 8, 6, 3), (48, 4, 4, 2), (64, 8, 6, 3), (96, 4, 3, 2),
                                           (128, 2, 3, 2)])
def test_fp32_variants_match_fp64(qbe, N, J, M, ncells):
    """The fused kernel in its shapes and the element-pass kernel (N = 32, 48, 64: padded grids of
    64, 96 and 128 points; at 128 also the warp-local kernel), several (cell, j, m-chunk) units per
    block; the cluster kernel in both shapes (N = 96, 128: 192 and 256 points), several units and
    several m per cluster."""
    w = inputs.synthetic_w(N, ncells, seed=50 + N, perturb=0.05)
    ref = _collide_all_variants(qbe, w, N, J, M, 0)[0]
    res = _collide_all_variants(qbe, w, N, J, M, 1)
    assert len(res) == {64: 5, 96: 2, 128: 2}.get(N, 4)
    for v, got in res.items():
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < TOL_F32, (v, err)


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_keeps_a_valid_fast_shape(qbe, prec):
    import torch

    N, Nx, J, M = 64, 6, 8, 8
    w = inputs.synthetic_w(N, Nx, seed=60, perturb=0.05)
    s = qbe.Solver(N, Nx, J=J, M=M, stream=torch.cuda.current_stream(), precision=prec)
    wd = torch.from_numpy(w).cuda()
    before = s.collide(wd).cpu().numpy()
    s.set_state(w)
    ms = s.autotune()
    shape = s.i3_shape()
    assert ms > 0 and 0 <= shape["variant"] < shape["nvariants"] and shape["grid"] >= 1 and shape["m_chunks"] >= 1
    assert np.array_equal(s.get_state(), w)                 # tuning leaves the state alone
    after = s.collide(wd).cpu().numpy()
    tol = 1e-13 if prec == 0 else TOL_F32
    assert np.abs(after - before).max() <= tol * np.abs(before).max()
    with pytest.raises(qbe.QbeError):
        s.set_i3_shape(variant=shape["nvariants"])
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_grid_and_m_chunks_change_only_the_summation_order(qbe, prec):
    """qbe_set_i3_shape: a smaller persistent grid and another m-chunking regroup the per-unit partial
    sums of I3; C[W] agrees with the default shape to rounding, and out-of-range requests fail."""
    import torch

    N, Nx, J, M = 32, 5, 8, 8
    w = torch.from_numpy(inputs.synthetic_w(N, Nx, seed=80, perturb=0.05)).cuda()
    s = qbe.Solver(N, Nx, J=J, M=M, stream=torch.cuda.current_stream(), precision=prec)
    ref = s.collide(w).cpu().numpy()
    base = s.i3_shape()
    tol = 1e-13 if prec == 0 else 1e-6
    for grid, m_chunks in ((7, 0), (0, 1), (19, base["m_chunks"])):
        s.set_i3_shape(grid=grid, m_chunks=m_chunks)
        sh = s.i3_shape()
        if grid:
            assert sh["grid"] == grid
        if m_chunks:
            assert sh["m_chunks"] == m_chunks
        got = s.collide(w).cpu().numpy()
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (grid, m_chunks)
    with pytest.raises(qbe.QbeError):
        s.set_i3_shape(m_chunks=base["m_chunks"] + 1)       # more than the partial sums hold
    with pytest.raises(qbe.QbeError):
        s.set_i3_shape(grid=-1)
    s.close()
