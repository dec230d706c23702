"""Differentiable multi-step rollout: torch.autograd.Function around the CUDA
step and its hand-written discrete adjoint (af_adjoint_step).

    xN = rollout(x0, grid, gamma, dt, n_steps, checkpoint_every=50)
    J = functional(xN); J.backward()   # x0.grad = dJ/dx0

x0 is a float64 CUDA tensor of shape (16, ny, nx) (the state layout of the
package).  The forward pass keeps a checkpoint every `checkpoint_every` steps;
the backward pass walks the segments in reverse, recomputes the states of a
segment from its checkpoint, and applies the adjoint step to them in reverse.
Memory: one state per checkpoint plus the states of one segment.  The solver
and the checkpoints live until the backward pass, which releases them: a
graph is differentiated once (a second backward raises), and a graph that is
never differentiated holds them until it is garbage-collected.
"""
import torch

from . import Solver


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, grid, gamma, dt, n_steps, every, precision, variant):
        stream = torch.cuda.current_stream()
        solver = Solver(grid, gamma, x0.detach().contiguous(), precision=precision,
                        variant=variant, stream=stream)
        ckpts = []
        done = 0
        while done < n_steps:
            c = torch.empty_like(x0)
            solver.state(c)
            ckpts.append(c)
            k = min(every, n_steps - done)
            solver.step(dt, k)
            done += k
        xn = torch.empty_like(x0)
        solver.state(xn)
        solver.sync()
        ctx.solver = solver
        ctx.ckpts = ckpts
        ctx.meta = (dt, n_steps, every)
        return xn

    @staticmethod
    def backward(ctx, g):
        if ctx.solver is None:
            raise RuntimeError("rollout supports one backward pass: its solver and checkpoints "
                               "are released by the first")
        solver, ckpts = ctx.solver, ctx.ckpts
        dt, n_steps, every = ctx.meta
        lam = g.contiguous()
        for seg in range(len(ckpts) - 1, -1, -1):
            length = min(every, n_steps - seg * every)
            states = [ckpts[seg]]
            solver.set_state(ckpts[seg])
            for _ in range(length - 1):
                solver.step(dt, 1)
                st = torch.empty_like(lam)
                solver.state(st)
                states.append(st)
            for st in reversed(states):
                solver.set_state(st)
                lam = solver.adjoint(dt, lam)
        solver.close()
        ctx.solver = None
        ctx.ckpts = None
        return lam, None, None, None, None, None, None, None


def rollout(x0, grid, gamma, dt, n_steps, checkpoint_every=50, precision="fp64", variant="tai"):
    """State after n_steps steps, differentiable with respect to x0."""
    return _Rollout.apply(x0, grid, gamma, dt, n_steps, checkpoint_every, precision, variant)


def kinetic_energy(x, h):
    """Domain-integrated kinetic energy of the cell averages, h^2 sum |m|^2 / (2 rho)."""
    return 0.5 * h * h * torch.sum((x[1] ** 2 + x[2] ** 2) / x[0])
