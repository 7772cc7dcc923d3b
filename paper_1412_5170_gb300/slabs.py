"""Y-slab decomposition of one periodic lattice over ranks: the host-side
split, halo exchange and reassembly for lattices larger than one GPU.

A lattice of ny rows splits into contiguous row slabs, one per rank.  One
time step of a node needs the populations of its own row and of the rows
within two of it: the pull (Eq. 1) reads rows y - 1 and y + 1, and the force
there (Eq. 6) reads psi (Eq. 7) of rows y - 2 and y + 2.  Each rank therefore
steps an extended slab -- its rows plus HALO = 2 rows on each side -- as a
lattice periodic in y (the wrap corrupts only the halo rows), and after each
step swaps its two boundary rows with each neighbour: 9 populations x 2 rows
x nx values per side, the one exchange a step needs.  Populations are kept
in the post-streaming form f[a, y, x] (the distribution at time t, as
lbm_read_populations / lbm_write_populations give it), so the stepping
function is any periodic stepper of that form: the library's step on each
rank's device, or, in the CPU test, the oracle.

The exchange uses torch.distributed point-to-point calls (gloo on CPU
tensors; NCCL takes the same calls on device tensors): each rank sends its
top rows to the rank above and its bottom rows to the rank below, and
receives its halos from them.  With one rank the halos are its own
boundary rows (periodic wrap).

exchange_lattice does the same for an extended slab held by the library
(a Lattice of ny_rank + 2 HALO rows): the rows move between the lattice's
stored state (the post-collision populations the next step pulls) and
device buffers by lbm_copy_rows on the lattice's stream, and between
ranks by the same point-to-point calls on that stream.
"""
from __future__ import annotations

import numpy as np

HALO = 2


def split_rows(ny: int, world: int) -> list:
    """[(y0, y1)] of each rank: contiguous, as even as possible, each at
    least HALO rows (so a halo never reaches past the next rank)."""
    if world < 1 or ny < HALO * world:
        raise ValueError("%d rows cannot give %d ranks %d rows each" % (ny, world, HALO))
    return [(ny * r // world, ny * (r + 1) // world) for r in range(world)]


def extended(f: np.ndarray, y0: int, y1: int) -> np.ndarray:
    """The extended slab of rows [y0 - HALO, y1 + HALO) (periodic) of a full
    lattice f[9, ny, nx]."""
    ny = f.shape[1]
    rows = [(y % ny) for y in range(y0 - HALO, y1 + HALO)]
    return np.ascontiguousarray(f[:, rows, :])


def interior(ext: np.ndarray) -> np.ndarray:
    return ext[:, HALO:-HALO, :]


def exchange(ext: np.ndarray, rank: int, world: int) -> None:
    """Refresh the halo rows of this rank's extended slab (in place) from its
    neighbours' boundary rows (collective over the world's ranks)."""
    if world == 1:
        ext[:, :HALO, :] = ext[:, -2 * HALO:-HALO, :]
        ext[:, -HALO:, :] = ext[:, HALO:2 * HALO, :]
        return
    import torch
    import torch.distributed as dist
    up, down = (rank + 1) % world, (rank - 1) % world
    top = torch.from_numpy(np.ascontiguousarray(ext[:, -2 * HALO:-HALO, :]))     # the rank above's lower halo
    bottom = torch.from_numpy(np.ascontiguousarray(ext[:, HALO:2 * HALO, :]))    # the rank below's upper halo
    lower = torch.empty_like(top)
    upper = torch.empty_like(top)
    # tags tell the two directions apart when both neighbours are one rank
    reqs = [dist.isend(top, up, tag=1), dist.isend(bottom, down, tag=2),
            dist.irecv(lower, down, tag=1), dist.irecv(upper, up, tag=2)]
    for r in reqs:
        r.wait()
    ext[:, :HALO, :] = lower.numpy()
    ext[:, -HALO:, :] = upper.numpy()


def run(ext: np.ndarray, step, nsteps: int, rank: int, world: int) -> np.ndarray:
    """nsteps steps of this rank's extended slab: step(ext) -> ext advances
    it by one step as a periodic lattice; the halos are exchanged after each
    step.  Returns the final extended slab (halos valid)."""
    for _ in range(nsteps):
        ext = step(ext)
        exchange(ext, rank, world)
    return ext


def gather(ext: np.ndarray, rank: int, world: int, ny: int) -> np.ndarray:
    """The full lattice f[9, ny, nx] from every rank's interior rows
    (collective; every rank receives it)."""
    own = np.ascontiguousarray(interior(ext))
    if world == 1:
        return own
    import torch
    import torch.distributed as dist
    spans = split_rows(ny, world)
    parts = [torch.empty((own.shape[0], y1 - y0, own.shape[2]), dtype=torch.float64) for y0, y1 in spans]
    # all_gather wants equal shapes: pad every rank's rows to the largest slab
    rows = max(y1 - y0 for y0, y1 in spans)
    mine = torch.zeros((own.shape[0], rows, own.shape[2]), dtype=torch.float64)
    mine[:, :own.shape[1], :] = torch.from_numpy(own)
    got = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(got, mine)
    for r, (y0, y1) in enumerate(spans):
        parts[r] = got[r][:, :y1 - y0, :]
    return torch.cat(parts, dim=1).numpy()


def exchange_lattice(lat, rank: int, world: int, bufs=None):
    """Refresh the halo rows of an extended slab held by a library Lattice
    (2 HALO of its rows are halo, HALO at each end) from its neighbours'
    boundary rows of the stored state, after a step.  bufs: four device
    buffers (9, HALO, nx) of the storage type from an earlier call, or None;
    returns them for the next call.  Collective over the world's ranks; with
    one rank the lattice's own rows (periodic wrap)."""
    import torch
    ny_ext, nx = lat.shape
    if bufs is None:
        dt = torch.float64 if lat.p.precision == 0 else torch.float32
        bufs = [torch.empty((9, HALO, nx), dtype=dt, device="cuda") for _ in range(4)]
    top, bottom, lower, upper = bufs
    lat.copy_rows(ny_ext - 2 * HALO, top)    # the rank above's lower halo
    lat.copy_rows(HALO, bottom)              # the rank below's upper halo
    if world == 1:
        lower, upper = top, bottom
    else:
        import torch.distributed as dist
        up, down = (rank + 1) % world, (rank - 1) % world
        with torch.cuda.stream(lat.stream):   # ordered with the copies on the lattice's stream
            reqs = [dist.isend(top, up, tag=1), dist.isend(bottom, down, tag=2),
                    dist.irecv(lower, down, tag=1), dist.irecv(upper, up, tag=2)]
            for r in reqs:
                r.wait()
    lat.copy_rows(0, lower, to_lattice=True)
    lat.copy_rows(ny_ext - HALO, upper, to_lattice=True)
    return bufs
