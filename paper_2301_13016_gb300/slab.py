"""One grid split across ranks in y slabs, for the forward-Euler march.

The paper scales its design by giving independent compute units their own
part of the domain (Sec. 5).  A single doubly periodic grid split in y into
slabs, one per rank, needs one exchange per step: every rank's first and
last interior rows become its neighbours' halo rows (a ring, as the domain
is periodic in y).  Each rank advances its slab with the fused step kernel
(`PW.step_to`, which also writes the x images and wraps y within the slab),
then the exchange overwrites the slab's two y-halo rows with the
neighbours' rows, x images and all, so that the next step reads exactly the
cells of the undivided grid.

The exchange is plain point-to-point messages through torch.distributed:
NCCL between GPUs, gloo on the CPU (where the tests run it).  One rank holds
the whole grid and exchanges nothing.
"""
import torch


def slab_rows(ny, world, rank):
    """(j0, nyr): the slab of `rank` holds global interior rows j0+1 .. j0+nyr
    (1-based).  Rows are split as evenly as possible, the first ny % world
    ranks taking one more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    if ny < world:
        raise ValueError("every rank needs at least one row")
    base, extra = divmod(ny, world)
    nyr = base + (1 if rank < extra else 0)
    j0 = rank * base + min(rank, extra)
    return j0, nyr


class HaloExchangeY:
    """The per-step y-halo exchange of a slab: row 1 goes to the rank below
    (its top halo row nyr+1), row nyr to the rank above (its bottom halo row
    0), for each field.  Fields are 3D views (nz+2, nyr+2, row) of the
    rank's slab, on the device the process group serves."""

    TAG_DOWN, TAG_UP = 11, 12

    def __init__(self, world, rank, group=None):
        self.world, self.rank, self.group = world, rank, group
        self.down = (rank - 1) % world
        self.up = (rank + 1) % world

    def exchange(self, fields):
        if self.world == 1:
            return   # the kernel's own periodic images are the neighbours' rows
        import torch.distributed as dist
        ops, land = [], []
        for f in fields:
            nyr = f.shape[1] - 2
            first = f[:, 1, :].contiguous()      # to the rank below
            last = f[:, nyr, :].contiguous()     # to the rank above
            top = torch.empty_like(first)        # from the rank above: its first row
            bottom = torch.empty_like(last)      # from the rank below: its last row
            # the same order on every rank, one tag per direction, so that
            # two messages between the same pair of ranks cannot cross
            ops += [dist.P2POp(dist.isend, first, self.down, self.group, self.TAG_DOWN),
                    dist.P2POp(dist.irecv, top, self.up, self.group, self.TAG_DOWN),
                    dist.P2POp(dist.isend, last, self.up, self.group, self.TAG_UP),
                    dist.P2POp(dist.irecv, bottom, self.down, self.group, self.TAG_UP)]
            land.append((f, nyr, top, bottom))
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        for f, nyr, top, bottom in land:
            f[:, nyr + 1, :] = top
            f[:, 0, :] = bottom


def step_slabs(h, grid, q, nq, dt, nsteps, exchange, scale=None, stream=None):
    """nsteps forward-Euler steps of the rank's slab: the fused step kernel
    out of place (q -> nq), then the y-halo exchange of the new state.  q
    (three fields of `grid`, a one-cell lateral halo: the scheme's reach)
    must hold the slab with its halos filled as the undivided grid's would
    be (`exchange` after a periodic fill does that).  Returns the three
    fields that hold the final state (q or nq)."""
    if grid.halo != 1:
        raise ValueError("the slab exchange moves one halo row: the grid needs halo = 1")
    a, b = list(q), list(nq)
    for _ in range(nsteps):
        h.step_to(*a, *b, dt, scale=scale, stream=stream)
        exchange.exchange([grid.view(t) for t in b])
        a, b = b, a
    return a
