"""torch.autograd bindings of the library's vector-Jacobian products.

Every forward and backward computation runs in the library's CUDA kernels;
this module only routes tensors between torch's autograd and the C ABI:

    Wn = evolve(solver, W0, B, dt, nsteps, checkpoint_every)   # split steps of Sec. 4
    Pz, PhiE = observables(solver, Wn).unbind()
    Pz.backward()            # W0.grad, B.grad

collide(solver, w) is C[W] (Sec. 3.2) with its transposed derivative.
Tensors are CUDA float64 tensors on the solver's device.
"""
import torch

from . import qbe as _q


def _contig(t):
    return t.detach().contiguous()


class CollideFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, w):
        w = _contig(w)
        ctx.solver = solver
        ctx.save_for_backward(w)
        return solver.collide(w)

    @staticmethod
    def backward(ctx, gc):
        (w,) = ctx.saved_tensors
        return None, ctx.solver.collide_vjp(w, _contig(gc))


def _record(solver, dt, nsteps, checkpoint_every):
    """checkpoint_every = 0: keep every intermediate state (no recomputation in the backward)."""
    if checkpoint_every == 0:
        return solver.step_taped(dt, nsteps)
    return solver.step_checkpointed(dt, nsteps, checkpoint_every)


class EvolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, W0, B, dt, nsteps, checkpoint_every):
        W0, B = _contig(W0), _contig(B)
        solver.set_state(W0)
        solver.set_bfield(B)
        ctx.solver, ctx.args = solver, (float(dt), int(nsteps), int(checkpoint_every))
        ctx.gen = _record(solver, *ctx.args)
        ctx.save_for_backward(W0, B)
        Wn = torch.empty_like(W0)
        solver.get_state(Wn)
        return Wn

    @staticmethod
    def backward(ctx, gWn):
        solver = ctx.solver
        W0, B = ctx.saved_tensors
        if solver._gen != ctx.gen:
            # the solver ran something else since this forward: record the tape again
            solver.set_state(W0)
            solver.set_bfield(B)
            ctx.gen = _record(solver, *ctx.args)
        lam0, gB = solver.step_vjp(_contig(gWn))
        return None, lam0, gB, None, None, None


class ObservablesFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, W):
        ctx.solver = solver
        return solver.observables(_contig(W))

    @staticmethod
    def backward(ctx, g):
        return None, ctx.solver.observables_vjp(_contig(g))


def collide(solver: "_q.Solver", w: torch.Tensor) -> torch.Tensor:
    """C[W] for w[ncells][4][N][N], differentiable in w."""
    return CollideFn.apply(solver, w)


def evolve(solver: "_q.Solver", W0: torch.Tensor, B: torch.Tensor, dt: float, nsteps: int,
           checkpoint_every: int = 20) -> torch.Tensor:
    """W_n after nsteps split steps from W0 with field B, differentiable in W0 and B.  The backward
    recomputes each segment of checkpoint_every steps from its checkpoint; checkpoint_every = 0
    keeps every intermediate state of the forward instead (more device memory, no recomputation)."""
    if checkpoint_every < 0:
        raise ValueError("checkpoint_every must be >= 0")
    return EvolveFn.apply(solver, W0, B, dt, nsteps, checkpoint_every)


def observables(solver: "_q.Solver", W: torch.Tensor) -> torch.Tensor:
    """[P_z, Phi_E] of the state W, differentiable in W."""
    return ObservablesFn.apply(solver, W)
