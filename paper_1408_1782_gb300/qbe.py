"""Thin Python binding of the C ABI in include/qbe.h (argument marshalling only).

Every computation runs in the sm_103a kernels of ``libqbe.so``; there is no
CPU fallback.  If the library has not been built, importing ``lib()`` raises.

Arrays: numpy float64 arrays are passed as host memory (the library copies
them); CUDA torch tensors (float64, contiguous) are passed as device memory.
State layout: ``w[cell][4][ix][iy]`` Pauli components, v = (2L/N)(ix-N/2, iy-N/2).

Example (ten split steps of the N = 64, Nx = 128 workload with Dirichlet walls)::

    from paper_1408_1782_gb300 import inputs, qbe
    s = qbe.Solver(64, 128, J=32, M=32)                  # precision=1: the FP32-split form
    wall = qbe.fd_state(1.0, 0.0, 0.0)                   # Fermi-Dirac inflow, beta = 1, mu = 0
    s.set_boundary("dirichlet", wall, wall)
    s.set_state(inputs.synthetic_w(64, 128, seed=0, perturb=0.05))
    s.set_bfield(inputs.uniform_b(128, (0.0, 0.0, 0.5)))
    s.step(0.005, 10)
    W = s.get_state()                                    # numpy [128][4][64][64]
    rho, momentum, energy = s.moments()
    s.close()
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqbe.so")

QBE_PERIODIC, QBE_DIRICHLET, QBE_MAXWELL = 0, 1, 2
QBE_OK, QBE_ERR_ARG = 0, -1
_BC = {"periodic": QBE_PERIODIC, "dirichlet": QBE_DIRICHLET, "maxwell": QBE_MAXWELL}

# Every entry point declared in include/qbe.h, with its ctypes signature.
_c_int, _c_double, _c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class QbeGrid(ctypes.Structure):
    _fields_ = [("N", _c_int), ("Nx", _c_int), ("J", _c_int), ("M", _c_int), ("L", _c_double),
                ("R", _c_double), ("precision", _c_int), ("device", _c_int)]


class QbeFD(ctypes.Structure):
    _fields_ = [("beta", _c_double), ("mu_up", _c_double), ("mu_dn", _c_double),
                ("U_re", (_c_double * 2) * 2), ("U_im", (_c_double * 2) * 2)]


class QbeFermiDirac(ctypes.Structure):
    """Mirror of qbe_fermi_dirac (include/qbe.h)."""
    _fields_ = [("T", _c_double), ("mu_up", _c_double), ("mu_dn", _c_double), ("bloch", _c_double * 3),
                ("U_re", (_c_double * 2) * 2), ("U_im", (_c_double * 2) * 2), ("u", _c_double * 2), ("ok", _c_int)]

    def U(self):
        return np.array([[complex(self.U_re[r][c], self.U_im[r][c]) for c in range(2)] for r in range(2)])


SIGNATURES = {
    "qbe_create": (_c_int, [ctypes.POINTER(QbeGrid), ctypes.POINTER(_c_void_p)]),
    "qbe_destroy": (None, [_c_void_p]),
    "qbe_last_error": (ctypes.c_char_p, [_c_void_p]),
    "qbe_set_stream": (_c_int, [_c_void_p, _c_void_p]),
    "qbe_set_boundary": (_c_int, [_c_void_p, _c_int, ctypes.POINTER(QbeFD), ctypes.POINTER(QbeFD), _c_double]),
    "qbe_set_bfield": (_c_int, [_c_void_p, _c_void_p, _c_int]),
    "qbe_set_state": (_c_int, [_c_void_p, _c_void_p, _c_int]),
    "qbe_get_state": (_c_int, [_c_void_p, _c_void_p, _c_int]),
    "qbe_collide": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_int, _c_int]),
    "qbe_advect": (_c_int, [_c_void_p, _c_double]),
    "qbe_collide_rk2": (_c_int, [_c_void_p, _c_double]),
    "qbe_step": (_c_int, [_c_void_p, _c_double, _c_int]),
    "qbe_moments": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_int]),
    "qbe_launch_count": (ctypes.c_longlong, [_c_void_p]),
    "qbe_enable_timing": (_c_int, [_c_void_p, _c_int]),
    "qbe_kernel_time": (_c_int, [_c_void_p, _c_int, ctypes.POINTER(_c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "qbe_collide_vjp": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_int, _c_int]),
    "qbe_collide_vjp_n": (_c_int, [_c_void_p, _c_int, _c_void_p, _c_void_p, _c_void_p, _c_int, _c_int]),
    "qbe_step_checkpointed": (_c_int, [_c_void_p, _c_double, _c_int, _c_int]),
    "qbe_step_taped": (_c_int, [_c_void_p, _c_double, _c_int]),
    "qbe_step_vjp": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_int]),
    "qbe_step_vjp_n": (_c_int, [_c_void_p, _c_int, _c_void_p, _c_void_p, _c_void_p, _c_int]),
    "qbe_observables": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_int]),
    "qbe_observables_vjp": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_int]),
    "qbe_entropy": (_c_int, [_c_void_p, _c_void_p, _c_int]),
    "qbe_fd_fit": (_c_int, [_c_void_p, _c_int, _c_void_p]),
    "qbe_fd_fit_moments": (_c_int, [_c_void_p, _c_void_p, _c_double, _c_void_p]),
    "qbe_dilog": (_c_double, [_c_double]),
    "qbe_relative_entropy": (_c_int, [_c_void_p, _c_void_p, _c_int, _c_void_p, _c_void_p, _c_int]),
    "qbe_collide_noalloc": (_c_int, [ctypes.POINTER(QbeGrid), _c_void_p, _c_void_p, _c_int, _c_void_p]),
    "qbe_i3_shape": (_c_int, [_c_void_p, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                              ctypes.POINTER(_c_int)]),
    "qbe_i3_variant_name": (ctypes.c_char_p, [_c_void_p, _c_int]),
    "qbe_set_i3_shape": (_c_int, [_c_void_p, _c_int, _c_int, _c_int]),
    "qbe_autotune": (_c_int, [_c_void_p, ctypes.POINTER(_c_double)]),
    "qbe_arith_issue_rates": (_c_int, [_c_int, _c_void_p, ctypes.POINTER(_c_double)]),
    "qbe_vjp_i3_variant": (_c_int, [_c_void_p, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "qbe_set_vjp_i3_variant": (_c_int, [_c_void_p, _c_int]),
    "qbe_batch_create": (_c_int, [ctypes.POINTER(_c_void_p), _c_int, ctypes.POINTER(_c_void_p)]),
    "qbe_batch_destroy": (None, [_c_void_p]),
    "qbe_batch_last_error": (ctypes.c_char_p, [_c_void_p]),
    "qbe_batch_set_stream": (_c_int, [_c_void_p, _c_void_p]),
    "qbe_batch_autotune": (_c_int, [_c_void_p]),
    "qbe_batch_tuned_shape": (_c_int, [_c_void_p, _c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                       ctypes.POINTER(_c_double)]),
    "qbe_batch_step": (_c_int, [_c_void_p, _c_double, _c_int]),
}

KERNEL_GROUPS = {"prep": 0, "i1": 1, "i24": 2, "i3": 3, "assemble": 4, "transport": 5, "rk": 6,
                 "vjp": 7, "vjp_i3": 8, "adj_transport": 9}

_lib = None


class QbeError(RuntimeError):
    pass


def lib():
    """Load libqbe.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise QbeError(f"{LIB_PATH} is missing; build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def fd_state(beta, mu_up, mu_dn, U=None) -> QbeFD:
    """Fermi-Dirac wall state; U: 2x2 complex unitary, columns = spin basis (default identity)."""
    U = np.eye(2) if U is None else np.asarray(U, dtype=np.complex128)
    f = QbeFD()
    f.beta, f.mu_up, f.mu_dn = float(beta), float(mu_up), float(mu_dn)
    for r in range(2):
        for c in range(2):
            f.U_re[r][c] = float(U[r, c].real)
            f.U_im[r][c] = float(U[r, c].imag)
    return f


def _arg(x, shape):
    """(pointer, on_device, keepalive) for a numpy array or a CUDA torch tensor of the given shape."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"] or x.shape != tuple(shape):
            raise ValueError(f"expected C-contiguous float64 array of shape {tuple(shape)}, got {x.dtype} {x.shape}")
        return x.ctypes.data, 0, x
    try:
        import torch
    except ImportError as e:  # pragma: no cover
        raise TypeError("expected numpy array") from e
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous() or tuple(x.shape) != tuple(shape):
            raise ValueError(f"expected contiguous float64 tensor of shape {tuple(shape)}")
        return x.data_ptr(), 1 if x.is_cuda else 0, x
    raise TypeError(f"unsupported array type {type(x)}")


class Batch:
    """Independent simulations stepped together, one CUDA graph launch per split step."""

    def __init__(self, solvers, stream=None):
        self.solvers = list(solvers)
        arr = (_c_void_p * len(self.solvers))(*[s._h for s in self.solvers])
        h = _c_void_p()
        rc = lib().qbe_batch_create(arr, len(self.solvers), ctypes.byref(h))
        if rc != 0:
            raise QbeError(f"qbe_batch_create failed with code {rc}")
        self._b = h
        if stream is not None:
            handle = getattr(stream, "cuda_stream", stream)
            self._check(lib().qbe_batch_set_stream(self._b, _c_void_p(int(handle) if handle else 0)), "set_stream")

    def _check(self, rc, what):
        if rc != 0:
            msg = lib().qbe_batch_last_error(self._b)
            raise QbeError(f"{what} failed ({rc}): {msg.decode() if msg else ''}")

    def autotune(self):
        self._check(lib().qbe_batch_autotune(self._b), "qbe_batch_autotune")
        out = []
        for i in range(len(self.solvers)):
            g, m, ms = _c_int(), _c_int(), _c_double()
            self._check(lib().qbe_batch_tuned_shape(self._b, i, ctypes.byref(g), ctypes.byref(m), ctypes.byref(ms)),
                        "qbe_batch_tuned_shape")
            out.append((g.value, m.value, ms.value))
        return out

    def step(self, dt, nsteps=1):
        for sv in self.solvers:
            sv._gen += 1
        self._check(lib().qbe_batch_step(self._b, float(dt), int(nsteps)), "qbe_batch_step")

    def close(self):
        if getattr(self, "_b", None):
            lib().qbe_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def collide_noalloc(w, out, J=32, M=32, L=12.0, R=7.5, stream=None):
    """C[W] through qbe_collide_noalloc (no allocation inside the library): w and out are CUDA float64
    tensors [ncells][4][N][N] on the current device; runs on `stream` (default: legacy stream)."""
    import torch

    ncells, N = w.shape[0], w.shape[-1]
    shape = (ncells, 4, N, N)
    pw, dev, _k1 = _arg(w, shape)
    po, dev2, _k2 = _arg(out, shape)
    if not (dev and dev2):
        raise ValueError("qbe_collide_noalloc takes device memory")
    g = QbeGrid(N, ncells, J, M, L, R, 0, torch.cuda.current_device())
    handle = getattr(stream, "cuda_stream", stream)
    rc = lib().qbe_collide_noalloc(ctypes.byref(g), _c_void_p(pw), _c_void_p(po), ncells,
                                   _c_void_p(int(handle) if handle else 0))
    if rc != 0:
        raise QbeError(f"qbe_collide_noalloc failed with code {rc}")
    return out


class Solver:
    """One simulation on one GPU (see include/qbe.h for the semantics of each call)."""

    def __init__(self, N, Nx, J=32, M=32, L=12.0, R=7.5, device=0, stream=None, precision=0):
        """precision 0: plain FP64; 1: FP32-split (collision transforms in FP32, the rest in FP64)."""
        self.N, self.Nx, self.J, self.M, self.L, self.R = N, Nx, J, M, L, R
        self.precision = precision
        g = QbeGrid(N, Nx, J, M, L, R, precision, device)
        h = _c_void_p()
        rc = lib().qbe_create(ctypes.byref(g), ctypes.byref(h))
        if rc != 0:
            raise QbeError(f"qbe_create failed with code {rc}")
        self._h = h
        self._gen = 0   # bumped by every call that changes the state, the field or the boundary
        if stream is not None:
            self.set_stream(stream)

    # -- plumbing ---------------------------------------------------------
    def _check(self, rc, what):
        if rc != 0:
            msg = lib().qbe_last_error(self._h)
            raise QbeError(f"{what} failed ({rc}): {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            lib().qbe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: an int handle or a torch.cuda.Stream."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(lib().qbe_set_stream(self._h, _c_void_p(int(handle) if handle else 0)), "qbe_set_stream")

    @property
    def state_shape(self):
        return (self.Nx, 4, self.N, self.N)

    # -- configuration ----------------------------------------------------
    def set_boundary(self, kind="periodic", left=None, right=None, alpha=0.0):
        self._gen += 1
        k = _BC[kind] if isinstance(kind, str) else int(kind)
        lp = ctypes.byref(left) if left is not None else None
        rp = ctypes.byref(right) if right is not None else None
        self._check(lib().qbe_set_boundary(self._h, k, lp, rp, float(alpha)), "qbe_set_boundary")

    def set_bfield(self, B):
        self._gen += 1
        p, dev, keep = _arg(B, (self.Nx, 3))
        self._check(lib().qbe_set_bfield(self._h, _c_void_p(p), dev), "qbe_set_bfield")

    def set_state(self, w):
        self._gen += 1
        p, dev, keep = _arg(w, self.state_shape)
        self._check(lib().qbe_set_state(self._h, _c_void_p(p), dev), "qbe_set_state")

    def get_state(self, out=None):
        out = np.empty(self.state_shape) if out is None else out
        p, dev, keep = _arg(out, self.state_shape)
        self._check(lib().qbe_get_state(self._h, _c_void_p(p), dev), "qbe_get_state")
        return out

    # -- the hot path -----------------------------------------------------
    def collide(self, w, out=None):
        """C[W] for w[ncells][4][N][N] (host numpy or CUDA tensor); result in the same memory kind."""
        ncells = w.shape[0]
        shape = (ncells, 4, self.N, self.N)
        pw, dev, keep = _arg(w, shape)
        if out is None:
            if dev:
                import torch
                out = torch.empty(shape, dtype=torch.float64, device=w.device)
            else:
                out = np.empty(shape)
        po, dev2, keep2 = _arg(out, shape)
        if dev2 != dev:
            raise ValueError("input and output must both be host or both be device memory")
        self._check(lib().qbe_collide(self._h, _c_void_p(pw), _c_void_p(po), ncells, dev), "qbe_collide")
        return out

    def advect(self, tau):
        self._gen += 1
        self._check(lib().qbe_advect(self._h, float(tau)), "qbe_advect")

    def collide_rk2(self, dt):
        self._gen += 1
        self._check(lib().qbe_collide_rk2(self._h, float(dt)), "qbe_collide_rk2")

    def step(self, dt, nsteps=1):
        self._gen += 1
        self._check(lib().qbe_step(self._h, float(dt), int(nsteps)), "qbe_step")

    # -- differentiation ---------------------------------------------------
    def _like(self, x, shape, out):
        if out is not None:
            return out
        if isinstance(x, np.ndarray):
            return np.empty(shape)
        import torch
        return torch.empty(shape, dtype=torch.float64, device=x.device)

    def collide_vjp(self, w, lam, out=None):
        """(dC/dW at w)^T lam, cell by cell; w, lam, out of shape [ncells][4][N][N], same memory kind."""
        ncells = w.shape[0]
        shape = (ncells, 4, self.N, self.N)
        pw, dev, k1 = _arg(w, shape)
        pl, dev2, k2 = _arg(lam, shape)
        out = self._like(w, shape, out)
        po, dev3, k3 = _arg(out, shape)
        if not (dev == dev2 == dev3):
            raise ValueError("w, lam and out must all be host or all be device memory")
        self._check(lib().qbe_collide_vjp(self._h, _c_void_p(pw), _c_void_p(pl), _c_void_p(po), ncells, dev),
                    "qbe_collide_vjp")
        return out

    def collide_vjp_many(self, w, lams, out=None):
        """(dC/dW at w)^T lams[k] for a stack of cotangents lams[ncot][ncells][4][N][N] (CUDA tensors;
        the products share the state's transforms in groups of up to four)."""
        ncells, ncot = w.shape[0], lams.shape[0]
        shape = (ncells, 4, self.N, self.N)
        pw, dev, k1 = _arg(w, shape)
        pl, dev2, k2 = _arg(lams, (ncot,) + shape)
        out = self._like(lams, (ncot,) + shape, out)
        po, dev3, k3 = _arg(out, (ncot,) + shape)
        if not (dev and dev2 and dev3):
            raise ValueError("qbe_collide_vjp_n takes device memory")
        self._check(lib().qbe_collide_vjp_n(self._h, ncot, _c_void_p(pw), _c_void_p(pl), _c_void_p(po), ncells, 1),
                    "qbe_collide_vjp_n")
        return out

    def step_checkpointed(self, dt, nsteps, checkpoint_every=20):
        """step(dt, nsteps) recording the tape that step_vjp sweeps backwards."""
        self._gen += 1
        self._check(lib().qbe_step_checkpointed(self._h, float(dt), int(nsteps), int(checkpoint_every)),
                    "qbe_step_checkpointed")
        return self._gen

    def step_taped(self, dt, nsteps):
        """step(dt, nsteps) keeping every intermediate state, so that step_vjp recomputes nothing
        (nsteps x (2 s + 2) states of device memory; QbeError if they do not fit)."""
        self._gen += 1
        self._check(lib().qbe_step_taped(self._h, float(dt), int(nsteps)), "qbe_step_taped")
        return self._gen

    def step_vjp(self, lam_final, out=None, grad_B=None):
        """(lam_init, grad_B) for the tape of the last step_checkpointed or step_taped call."""
        pl, dev, k1 = _arg(lam_final, self.state_shape)
        out = self._like(lam_final, self.state_shape, out)
        grad_B = self._like(lam_final, (self.Nx, 3), grad_B)
        po, dev2, k2 = _arg(out, self.state_shape)
        pb, dev3, k3 = _arg(grad_B, (self.Nx, 3))
        if not (dev == dev2 == dev3):
            raise ValueError("cotangents must all be host or all be device memory")
        self._check(lib().qbe_step_vjp(self._h, _c_void_p(pl), _c_void_p(po), _c_void_p(pb), dev), "qbe_step_vjp")
        return out, grad_B

    def step_vjp_many(self, lams, out=None, grad_B=None):
        """step_vjp for a stack of cotangents lams[ncot][Nx][4][N][N] in one reverse sweep."""
        ncot = lams.shape[0]
        shape = (ncot,) + self.state_shape
        pl, dev, k1 = _arg(lams, shape)
        out = self._like(lams, shape, out)
        grad_B = self._like(lams, (ncot, self.Nx, 3), grad_B)
        po, dev2, k2 = _arg(out, shape)
        pb, dev3, k3 = _arg(grad_B, (ncot, self.Nx, 3))
        if not (dev == dev2 == dev3):
            raise ValueError("cotangents must all be host or all be device memory")
        self._check(lib().qbe_step_vjp_n(self._h, ncot, _c_void_p(pl), _c_void_p(po), _c_void_p(pb), dev),
                    "qbe_step_vjp_n")
        return out, grad_B

    def observables(self, w=None, out=None):
        """[P_z, Phi_E] of w (default: the solver state)."""
        if w is None:
            out = np.empty(2) if out is None else out
            po, dev, k = _arg(out, (2,))
            self._check(lib().qbe_observables(self._h, None, _c_void_p(po), dev), "qbe_observables")
            return out
        pw, dev, k1 = _arg(w, self.state_shape)
        out = self._like(w, (2,), out)
        po, dev2, k2 = _arg(out, (2,))
        if dev != dev2:
            raise ValueError("w and out must both be host or both be device memory")
        self._check(lib().qbe_observables(self._h, _c_void_p(pw), _c_void_p(po), dev), "qbe_observables")
        return out

    def observables_vjp(self, gbar, out=None):
        """gbar[0] dP_z/dW + gbar[1] dPhi_E/dW."""
        pg, dev, k1 = _arg(gbar, (2,))
        out = self._like(gbar, self.state_shape, out)
        po, dev2, k2 = _arg(out, self.state_shape)
        if dev != dev2:
            raise ValueError("gbar and out must both be host or both be device memory")
        self._check(lib().qbe_observables_vjp(self._h, _c_void_p(pg), _c_void_p(po), dev), "qbe_observables_vjp")
        return out

    # -- diagnostics (Sec. 2, Sec. 5) ----------------------------------------
    def entropy(self):
        """Local entropy per cell, [Nx] (host)."""
        out = np.empty(self.Nx)
        self._check(lib().qbe_entropy(self._h, _c_void_p(out.ctypes.data), 0), "qbe_entropy")
        return out

    def fd_fit(self, global_fit=False):
        """Fermi-Dirac states with the moments of each cell (list of Nx QbeFermiDirac) or of the domain (one)."""
        n = 1 if global_fit else self.Nx
        arr = (QbeFermiDirac * n)()
        self._check(lib().qbe_fd_fit(self._h, 1 if global_fit else 0, ctypes.cast(arr, _c_void_p)), "qbe_fd_fit")
        return arr[0] if global_fit else list(arr)

    def relative_entropy(self, ref, with_l1=True):
        """(rel[Nx], l1[Nx] or None) to ref: one QbeFermiDirac (global) or a list of Nx (local)."""
        refs = [ref] if isinstance(ref, QbeFermiDirac) else list(ref)
        arr = (QbeFermiDirac * len(refs))(*refs)
        rel = np.empty(self.Nx)
        l1 = np.empty(self.Nx) if with_l1 else None
        self._check(lib().qbe_relative_entropy(self._h, ctypes.cast(arr, _c_void_p), len(refs),
                                               _c_void_p(rel.ctypes.data),
                                               _c_void_p(l1.ctypes.data) if with_l1 else None, 0),
                    "qbe_relative_entropy")
        return rel, l1

    def moments(self):
        rho = np.empty((self.Nx, 4))
        mom = np.empty((self.Nx, 2))
        en = np.empty(self.Nx)
        self._check(lib().qbe_moments(self._h, _c_void_p(rho.ctypes.data), _c_void_p(mom.ctypes.data),
                                      _c_void_p(en.ctypes.data), 0), "qbe_moments")
        return rho, mom, en

    def launch_count(self):
        return int(lib().qbe_launch_count(self._h))

    def enable_timing(self, on=True):
        self._check(lib().qbe_enable_timing(self._h, 1 if on else 0), "qbe_enable_timing")

    def kernel_time(self, group):
        """(total device ms, launches) of a kernel group since enable_timing()."""
        ms, n = _c_double(), ctypes.c_longlong()
        self._check(lib().qbe_kernel_time(self._h, KERNEL_GROUPS[group], ctypes.byref(ms), ctypes.byref(n)),
                    "qbe_kernel_time")
        return ms.value, n.value

    def i3_shape(self):
        """Current I3 launch shape: dict(variant, nvariants, grid, m_chunks, name)."""
        v, nv, g, m = _c_int(), _c_int(), _c_int(), _c_int()
        self._check(lib().qbe_i3_shape(self._h, ctypes.byref(v), ctypes.byref(nv), ctypes.byref(g), ctypes.byref(m)),
                    "qbe_i3_shape")
        return {"variant": v.value, "nvariants": nv.value, "grid": g.value, "m_chunks": m.value,
                "name": self.i3_variant_name(v.value)}

    def i3_variant_name(self, variant):
        name = lib().qbe_i3_variant_name(self._h, int(variant))
        return name.decode() if name else None

    def set_i3_shape(self, variant=-1, grid=0, m_chunks=0):
        """Set the I3 launch variant / persistent grid / m-chunks (-1, 0, 0 keep the current one)."""
        self._check(lib().qbe_set_i3_shape(self._h, int(variant), int(grid), int(m_chunks)), "qbe_set_i3_shape")

    def autotune(self):
        """Time the I3 launch shapes on the current state and keep the fastest; returns its predicted ms."""
        ms = _c_double()
        self._check(lib().qbe_autotune(self._h, ctypes.byref(ms)), "qbe_autotune")
        return ms.value

    def vjp_i3_variant(self):
        """(variant, count) of the I3 transpose kernel of the collision product."""
        v, nv = _c_int(), _c_int()
        self._check(lib().qbe_vjp_i3_variant(self._h, ctypes.byref(v), ctypes.byref(nv)), "qbe_vjp_i3_variant")
        return v.value, nv.value

    def set_vjp_i3_variant(self, variant=-1):
        self._check(lib().qbe_set_vjp_i3_variant(self._h, int(variant)), "qbe_set_vjp_i3_variant")


def arith_issue_rates(device=0, stream=None):
    """Measured FP64 fma / add / mul and FP32 fma lane-operations per second of the device
    (qbe_arith_issue_rates); `stream` a torch.cuda.Stream or None."""
    out = (_c_double * 4)()
    h = _c_void_p(getattr(stream, "cuda_stream", stream))
    rc = lib().qbe_arith_issue_rates(int(device), h, out)
    if rc != 0:
        raise QbeError(f"qbe_arith_issue_rates failed ({rc})")
    return {"dfma": out[0], "dadd": out[1], "dmul": out[2], "ffma": out[3]}


def fd_fit_moments(rho4, mom, energy) -> QbeFermiDirac:
    """Fermi-Dirac fit for given moments (host only; no GPU needed)."""
    r = np.ascontiguousarray(rho4, dtype=np.float64)
    m = np.ascontiguousarray(mom, dtype=np.float64)
    out = QbeFermiDirac()
    rc = lib().qbe_fd_fit_moments(_c_void_p(r.ctypes.data), _c_void_p(m.ctypes.data), float(energy),
                                  ctypes.cast(ctypes.byref(out), _c_void_p))
    if rc != 0:
        raise QbeError(f"qbe_fd_fit_moments failed with code {rc}")
    return out


def dilog(x: float) -> float:
    """Li2(x), x <= 0 (the library's own implementation)."""
    return float(lib().qbe_dilog(float(x)))
