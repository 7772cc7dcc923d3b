"""The y-slab decomposition of one lattice over ranks (paper_1412_5170_gb300
/slabs.py): split, two-row halo exchange per step and reassembly, with
gloo ranks on the CPU and the oracle as each rank's stepper.  Every node's
update sees the same inputs as in the undivided lattice, so the gathered
lattice must equal the single-lattice oracle run bit for bit; an uneven
split (25 rows over 3 ranks) and two neighbours that are one rank (2 ranks)
are both covered."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

MRT = dict(s_e=0.8, s_eps=0.8, s_q=1.1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(nx, ny, coll):
    from paper_1412_5170_gb300 import synth
    rho0 = synth.density_field(nx, ny, "droplet", 0.3, 0.02, 6.0, seed=9)
    return rho0, dict(T_over_Tc=0.8, tau=0.9, A=-0.304, K=1.0, collision=coll, forcing="guo", **MRT)


def _worker(rank, ws, port, nx, ny, coll, steps, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=ws)
    import oracle
    from paper_1412_5170_gb300 import slabs
    rho0, kw = _case(nx, ny, coll)
    f0 = oracle.init_rest(rho0)
    y0, y1 = slabs.split_rows(ny, ws)[rank]
    ext = slabs.extended(f0, y0, y1)
    q = oracle.params(nx, ext.shape[1], **kw)

    def step(e):
        g, st = oracle.step(q, e)
        assert st == oracle.OK
        return g

    ext = slabs.run(ext, step, steps, rank, ws)
    full = slabs.gather(ext, rank, ws, ny)
    if rank == 0:
        out["full"] = full
    dist.destroy_process_group()


@pytest.mark.parametrize("ws,nx,ny,coll", [(2, 20, 24, "mrt"), (3, 16, 25, "bgk")])
def test_slabs_reassemble_the_undivided_lattice(ws, nx, ny, coll):
    import oracle
    steps = 25
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(ws, _free_port(), nx, ny, coll, steps, out), nprocs=ws, join=True,
                       start_method="spawn")
    rho0, kw = _case(nx, ny, coll)
    ref, st = oracle.run(oracle.params(nx, ny, **kw), oracle.init_rest(rho0), steps)
    assert st == oracle.OK
    assert np.array_equal(out["full"], ref)


def test_one_rank_wraps_its_own_halos():
    import oracle
    from paper_1412_5170_gb300 import slabs
    nx, ny, steps = 12, 10, 15
    rho0, kw = _case(nx, ny, "bgk")
    f0 = oracle.init_rest(rho0)
    ext = slabs.extended(f0, 0, ny)
    q = oracle.params(nx, ext.shape[1], **kw)
    ext = slabs.run(ext, lambda e: oracle.step(q, e)[0], steps, 0, 1)
    ref, _ = oracle.run(oracle.params(nx, ny, **kw), f0, steps)
    assert np.array_equal(slabs.gather(ext, 0, 1, ny), ref)


def test_split_rows_covers_the_lattice():
    from paper_1412_5170_gb300 import slabs
    for ny, ws in ((25, 3), (8, 4), (1000, 7)):
        spans = slabs.split_rows(ny, ws)
        assert spans[0][0] == 0 and spans[-1][1] == ny
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
        assert all(y1 - y0 >= slabs.HALO for y0, y1 in spans)
    with pytest.raises(ValueError):
        slabs.split_rows(5, 3)
