"""torch.autograd over forward-Euler rollouts of the PW advection system.

PWRollout.apply(u, v, w, handle, dt, nsteps, checkpoint_every) runs nsteps
fused Euler steps (pw_step) from the state (u, v, w) (flat allocations of the
handle's FP32 grid; interior values are the state, halos are refreshed) and
returns the final state as new allocations.  Backward runs the reverse sweep
g_n = g_{n+1} + dt * F^T J(q_n)^T g_{n+1} (pw_adjoint with PW_ADJ_PERIODIC |
PW_ADJ_ADD_LAMBDA), recomputing the states of each checkpoint segment from
its stored start state: memory holds one state per checkpoint plus one
segment, not every step.

Gradients flow through interior values: the gradient returned for u, v, w
is zero on halo entries (they are copies of interior values), and the halo
entries of the incoming output gradients are ignored.
"""
import torch

from .pw import PW_ADJ_ADD_LAMBDA, PW_ADJ_PERIODIC


def _interior_mask(grid, device):
    m = torch.zeros(grid.alloc_elems, dtype=torch.bool, device=device)
    grid.view(m)[1:-1, grid.halo:grid.halo + grid.ny, grid.halo:grid.halo + grid.nx] = True
    return m


class PWRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, v, w, handle, dt, nsteps, checkpoint_every=5):
        grid = handle.grid
        if grid.dtype != "f32":
            raise ValueError("PWRollout needs an FP32 grid")
        every = max(1, int(checkpoint_every))
        state = [t.detach().clone() for t in (u, v, w)]
        tmp = [grid.alloc(device=u.device, fill=None) for _ in range(3)]
        ckpts = []
        n = 0
        handle.step(*state, *tmp, dt, 0)           # refresh halos of the start state
        while n < nsteps:
            ckpts.append([t.clone() for t in state])
            m = min(every, nsteps - n)
            handle.step(*state, *tmp, dt, m)
            n += m
        ctx.handle, ctx.dt, ctx.nsteps, ctx.every = handle, float(dt), int(nsteps), every
        ctx.save_for_backward(*[t for c in ckpts for t in c])
        return tuple(state)

    @staticmethod
    def backward(ctx, gu, gv, gw):
        h, dt, nsteps, every = ctx.handle, ctx.dt, ctx.nsteps, ctx.every
        grid = h.grid
        saved = ctx.saved_tensors
        ckpts = [saved[3 * i:3 * i + 3] for i in range(len(saved) // 3)]
        dev = saved[0].device if saved else gu.device
        mask = _interior_mask(grid, dev)
        g = []
        for x in (gu, gv, gw):
            y = torch.zeros(grid.alloc_elems, dtype=torch.float32, device=dev)
            if x is not None:
                y[mask] = x.to(torch.float32)[mask]
            g.append(y)
        g2 = [torch.zeros_like(t) for t in g]
        tmp = [grid.alloc(device=dev, fill=None) for _ in range(3)]
        for s in range(len(ckpts) - 1, -1, -1):
            n0 = s * every
            m = min(every, nsteps - n0)
            # recompute the states q_{n0} .. q_{n0+m-1} of this segment
            states = [[t.clone() for t in ckpts[s]]]
            for _ in range(m - 1):
                nxt = [t.clone() for t in states[-1]]
                h.step(*nxt, *tmp, dt, 1)
                states.append(nxt)
            for q in reversed(states):
                h.adjoint(*q, *g, *g2, alpha=dt, flags=PW_ADJ_PERIODIC | PW_ADJ_ADD_LAMBDA)
                g, g2 = g2, g
            del states
        for t in g:
            t[~mask] = 0.0
        return g[0], g[1], g[2], None, None, None, None


def rollout(u, v, w, handle, dt, nsteps, checkpoint_every=5):
    """Differentiable nsteps forward-Euler rollout (see PWRollout)."""
    return PWRollout.apply(u, v, w, handle, dt, nsteps, checkpoint_every)
