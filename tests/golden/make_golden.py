"""Write the stored expected values used by the GPU parity tests.

Every number written here comes from the FP64 CPU oracle (oracle/qbe_oracle.py)
applied to the seeded synthetic inputs; nothing comes from the CUDA library.

  plain_fp64_n16.npz   N=16, Nx=16, J=M=32, L=12, R=7.5, periodic, B=0:
                       initial state, state after 1 step and after 10 split
                       steps with dt=0.01, and the moments after every step.
  plain_fp64_n64_cells.npz
                       N=64, J=M=32: two cells (0 and 77) of the 128-cell
                       Dirichlet workload's initial state (5% perturbation) and
                       their collision operator C[W].

  precision_n128_cells.npz
                       N=128, J=M=32: two cells (0 and 131) of the 256-cell
                       Maxwell workload's initial state (5% perturbation) and
                       their C[W] (the FP32-split form is checked against it).

  collision_vjp_n8.npz
                       N=8, J=4, M=2: two cells (5% perturbation), a seeded
                       cotangent lam and the transposed derivative
                       (dC/dW)^T lam assembled column by column from exact
                       directional derivatives of the oracle (oracle/tangent.py).

Usage: python tests/golden/make_golden.py [n16|n64|n128|vjp8|all]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import qbe_oracle as O  # noqa: E402
from oracle import tangent as T  # noqa: E402
from paper_1408_1782_gb300 import inputs  # noqa: E402


def make_n16():
    wl = inputs.WORKLOADS["plain_fp64_n16"]
    p = O.Params(N=wl["N"], L=wl["L"], R=wl["R"], J=wl["J"], M=wl["M"])
    W = inputs.synthetic_w(wl["N"], wl["Nx"], L=wl["L"], seed=0)
    B = inputs.uniform_b(wl["Nx"], wl["B"])
    bc = O.Boundary("periodic")
    out = {"W0": W.copy()}
    rho, mom, en = [], [], []
    for k in range(wl["steps"]):
        t = time.time()
        W = O.step(W, B, wl["dt"], p, bc)
        r, m, e = O.moments(W, p)
        rho.append(r); mom.append(m); en.append(e)
        if k == 0:
            out["W1"] = W.copy()
        print(f"n16 step {k + 1}/{wl['steps']} {time.time() - t:.1f}s", flush=True)
    out["W10"] = W
    out["rho"], out["mom"], out["energy"] = np.array(rho), np.array(mom), np.array(en)
    np.savez_compressed(os.path.join(HERE, "plain_fp64_n16.npz"), **out)


def make_n64():
    wl = inputs.WORKLOADS["plain_fp64_n64"]
    p = O.Params(N=wl["N"], L=wl["L"], R=wl["R"], J=wl["J"], M=wl["M"])
    W = inputs.synthetic_w(wl["N"], wl["Nx"], L=wl["L"], seed=0, perturb=wl["perturb"])
    cells = np.array([0, 77])
    t = time.time()
    C = O.collision(W[cells], p)
    print(f"n64 cells {time.time() - t:.1f}s", flush=True)
    np.savez_compressed(os.path.join(HERE, "plain_fp64_n64_cells.npz"), cells=cells, W=W[cells], C=C)


def make_n128():
    import multiprocessing as mp

    wl = inputs.WORKLOADS["precision_n128"]
    p = O.Params(N=wl["N"], L=wl["L"], R=wl["R"], J=wl["J"], M=wl["M"])
    W = inputs.synthetic_w(wl["N"], wl["Nx"], L=wl["L"], seed=0, perturb=wl["perturb"])
    cells = np.array([0, 131])
    t = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        C = O.collision(W[cells], p, mapper=lambda f, it: pool.map(f, list(it), chunksize=1))
    print(f"n128 cells {time.time() - t:.1f}s", flush=True)
    np.savez_compressed(os.path.join(HERE, "precision_n128_cells.npz"), cells=cells, W=W[cells], C=C)


def make_vjp8():
    import multiprocessing as mp

    p = O.Params(N=8, J=4, M=2)
    W = inputs.synthetic_w(8, 2, seed=31, perturb=0.05)
    lam = inputs.random_field(W.shape, seed=32)
    t = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        G = T.collision_vjp_brute(W, lam, p, mapper=lambda f, it: pool.map(f, list(it), chunksize=4))
    print(f"vjp8 {time.time() - t:.1f}s", flush=True)
    np.savez_compressed(os.path.join(HERE, "collision_vjp_n8.npz"), W=W, lam=lam, grad=G, N=8, J=4, M=2)


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "all"
    if which in ("n64", "all"):
        make_n64()
    if which in ("n16", "all"):
        make_n16()
    if which in ("n128", "all"):
        make_n128()
    if which in ("vjp8", "all"):
        make_vjp8()
