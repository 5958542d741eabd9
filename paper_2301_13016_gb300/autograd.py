"""torch.autograd over forward-Euler rollouts of the PW advection system.

PWRollout.apply(u, v, w, handle, dt, nsteps, checkpoint_every) runs nsteps
forward-Euler steps from the state (u, v, w) (flat allocations of the
handle's FP32 grid; interior values are the state, halos are refreshed) and
returns the final state as new allocations.  Each step is one out-of-place
pass (pw_step_to), so a state, once written, is never modified: the
checkpoints are the states themselves, kept by reference.  Backward runs the
reverse sweep g_n = g_{n+1} + dt * F^T J(q_n)^T g_{n+1} (pw_adjoint with
PW_ADJ_PERIODIC | PW_ADJ_ADD_LAMBDA), recomputing the states of each
checkpoint segment from its start state: memory holds one state per
checkpoint plus one segment, not every step.

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


def _new_state(grid, device, fill=None):
    """Three fields for a state that a step pass writes: levels 1..nz with
    their lateral halos (the z-halo planes and the padding are never read;
    they are left unset inside the sweep and zeroed for a returned state)."""
    return [grid.alloc(device=device, fill=fill) for _ in range(3)]


class PWRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, v, w, handle, dt, nsteps, checkpoint_every=5):
        grid = handle.grid
        if grid.dtype != "f32":
            raise ValueError("PWRollout needs an FP32 grid")
        every = max(1, int(checkpoint_every))
        state = [t.detach().clone() for t in (u, v, w)]
        for t in state:                              # periodic halos of the start state
            handle.fill_halo_periodic(t)
        ckpts = []
        for n in range(int(nsteps)):
            if n % every == 0:
                ckpts.append(state)
            nxt = _new_state(grid, u.device, fill=0.0 if n == nsteps - 1 else None)
            handle.step_to(*state, *nxt, dt)
            state = nxt
        if not ckpts:                                # nsteps = 0: the result is a copy of the start state
            state = [t.clone() for t in state]
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
            g.append(torch.where(mask, x.to(torch.float32), 0.0) if x is not None
                     else torch.zeros(grid.alloc_elems, dtype=torch.float32, device=dev))
        # the adjoint writes every interior cell; the halo starts (and, as the
        # periodic adjoint leaves it, stays) at zero, so the next call's
        # incoming sensitivities have no stale values anywhere
        g2 = [torch.zeros_like(t) for t in g]
        for s in range(len(ckpts) - 1, -1, -1):
            n0 = s * every
            m = min(every, nsteps - n0)
            # recompute the states q_{n0} .. q_{n0+m-1} of this segment
            states = [list(ckpts[s])]
            for _ in range(m - 1):
                nxt = _new_state(grid, dev)
                h.step_to(*states[-1], *nxt, dt)
                states.append(nxt)
            for q in reversed(states):
                h.adjoint(*q, *g, *g2, alpha=dt, flags=PW_ADJ_PERIODIC | PW_ADJ_ADD_LAMBDA)
                g, g2 = g2, g
            del states
        for t in g:
            t.masked_fill_(~mask, 0.0)
        return g[0], g[1], g[2], None, None, None, None


def rollout(u, v, w, handle, dt, nsteps, checkpoint_every=5):
    """Differentiable nsteps forward-Euler rollout (see PWRollout)."""
    return PWRollout.apply(u, v, w, handle, dt, nsteps, checkpoint_every)
