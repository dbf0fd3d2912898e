"""Differentiation of the PW stencil with the hand-written adjoint kernels.

``PWAdvect`` maps (u, v, w) to (su, sv, sw); its backward is the adjoint kernel
(pw_advect_adjoint).  ``PWEulerSegment`` runs n forward-Euler steps
x <- x + dt S(x) (advection only; the "step fields" integration of the paper's
dynamics group, section 3) with the fused step kernel (pw_advect_step) and keeps
only its input: the backward recomputes
the segment's states and sweeps them in reverse with the Euler adjoint kernel
(g <- g + dt J(x)^T g), so a long loop split into segments stores one state
per segment (checkpointed recomputation).

Tensors use the library layout (Mesh.shape) with filled halos.  Gradients
returned for such tensors live on the interior (halo entries 0): whatever
reached a halo copy has been folded onto the interior value it copies.
Meshes must be PW_F32 or PW_F64.
"""
import torch

from .api import Mesh


def _grad_in(mesh: Mesh, g, like):
    """Incoming gradient as a fresh tensor with its halo folded onto the interior."""
    if g is None:
        return torch.zeros_like(like)
    g = g.contiguous().clone()
    mesh.halo_fold(g)
    return g


class PWAdvect(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh: Mesh, u, v, w):
        su, sv, sw = mesh.advect(u, v, w)
        ctx.mesh = mesh
        ctx.save_for_backward(u, v, w)
        return su, sv, sw

    @staticmethod
    def backward(ctx, gsu, gsv, gsw):
        mesh = ctx.mesh
        u, v, w = ctx.saved_tensors
        ys = [_grad_in(mesh, g, u) for g in (gsu, gsv, gsw)]
        gu, gv, gw = mesh.adjoint(u, v, w, *ys)
        return None, gu, gv, gw


class PWEulerSegment(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh: Mesh, dt: float, nsteps: int, u, v, w):
        # fused steps (stencil + update + halos in one pass), ping-ponged
        x = [u, v, w]
        bufs = [[mesh.empty() for _ in range(3)] for _ in range(min(nsteps, 2))]
        for n in range(nsteps):
            y = bufs[n % 2]
            mesh.step(*x, *y, dt=dt)
            x = y
        if nsteps == 0:
            x = [t.clone() for t in x]
        ctx.mesh, ctx.dt, ctx.nsteps = mesh, float(dt), int(nsteps)
        ctx.save_for_backward(u, v, w)
        return tuple(x)

    @staticmethod
    def backward(ctx, gu, gv, gw):
        mesh, dt, n = ctx.mesh, ctx.dt, ctx.nsteps
        u, v, w = ctx.saved_tensors
        states = [[u, v, w]]
        for _ in range(n - 1):
            states.append(list(mesh.step(*states[-1], dt=dt)))
        g = [_grad_in(mesh, t, u) for t in (gu, gv, gw)]
        for t in reversed(range(n)):
            g = list(mesh.euler_adjoint(*states[t], *g, dt=dt))
        return None, None, None, g[0], g[1], g[2]


def advect(mesh: Mesh, u, v, w):
    return PWAdvect.apply(mesh, u, v, w)


def euler_loop(mesh: Mesh, u, v, w, dt: float, steps: int, checkpoint_every: int = 2):
    """`steps` Euler steps as ceil(steps / checkpoint_every) recomputed segments."""
    x = (u, v, w)
    done = 0
    while done < steps:
        n = min(checkpoint_every, steps - done)
        x = PWEulerSegment.apply(mesh, dt, n, *x)
        done += n
    return x


def source_energy_loss(mesh: Mesh, u, v, w, dt: float, steps: int, checkpoint_every: int = 2):
    """L = sum(su^2 + sv^2 + sw^2) over interior points of the sources at the
    state reached after `steps` Euler steps (the adjoint-loop workload)."""
    x = euler_loop(mesh, u, v, w, dt, steps, checkpoint_every)
    s = advect(mesh, *x)
    return sum((mesh.interior(t).double() ** 2).sum() for t in s)
