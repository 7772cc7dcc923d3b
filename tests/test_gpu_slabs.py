"""The y-slab halo exchange on the device (paper_1412_5170_gb300/slabs.py,
exchange_lattice over lbm_copy_rows) on one GPU: an extended slab -- the
lattice's rows plus two halo rows on each side -- whose halos are refreshed
from its own boundary rows after every step is the periodic lattice itself,
so its interior must equal the undivided lattice bit for bit.  (The
multi-rank exchange moves the same buffers by torch.distributed
point-to-point calls; its host logic is tested on CPU ranks in
test_dist_slabs.py.)"""
import numpy as np
import pytest

from paper_1412_5170_gb300 import slabs, synth

pytestmark = pytest.mark.gpu

MRT = dict(s_e=0.8, s_eps=0.8, s_q=1.1)


@pytest.mark.parametrize("precision,coll,config", [("fp64", "mrt", 0), ("fp64", "bgk", 1), ("fp32", "mrt", 0),
                                                   ("fp32", "mrt", 10), ("fp32", "bgk", 5)])
def test_extended_slab_with_its_own_halos_is_the_lattice(lbm, precision, coll, config):
    nx, ny, steps = 64, 48, 80
    rv, rl = lbm.maxwell(0.8)
    rho0 = synth.density_field(nx, ny, "droplet", rl, rv, 12.0, seed=3)
    p = lbm.make_params(nx, ny, 0.8, 0.9, -0.304, 1.0, coll, "guo", precision, **MRT)
    pe = lbm.make_params(nx, ny + 2 * slabs.HALO, 0.8, 0.9, -0.304, 1.0, coll, "guo", precision, **MRT)
    with lbm.Lattice(p) as lat, lbm.Lattice(pe) as ext:
        lat.config = config
        ext.config = config
        lat.init_density(rho0)
        f0 = lat.read_populations()
        lat.write_populations(f0)                      # both from the same doubles
        ext.write_populations(slabs.extended(f0, 0, ny))
        bufs = None
        for _ in range(steps):
            lat.step(1)
            ext.step(1)
            bufs = slabs.exchange_lattice(ext, 0, 1, bufs)
        assert lat.stats()["status"] == 0 and ext.stats()["status"] == 0
        f, fe = lat.read_populations(), ext.read_populations()
    assert np.array_equal(slabs.interior(fe), f)


def test_copy_rows_round_trip_and_bounds(lbm):
    import torch
    nx, ny = 32, 20
    p = lbm.make_params(nx, ny, 0.8, 0.9, -0.304, 1.0, "bgk", "guo", "fp64")
    rv, rl = lbm.maxwell(0.8)
    with lbm.Lattice(p) as lat:
        lat.init_density(synth.density_field(nx, ny, "droplet", rl, rv, 6.0, seed=1))
        f = lat.read_populations()
        buf = torch.empty((9, 3, nx), dtype=torch.float64, device="cuda")
        lat.copy_rows(5, buf)
        zero = torch.zeros_like(buf)
        lat.copy_rows(5, zero, to_lattice=True)
        lat.copy_rows(5, buf, to_lattice=True)        # put the rows back
        lat.stream.synchronize()
        assert np.array_equal(lat.read_populations(), f)
        with pytest.raises(lbm.LbmError):
            lat.copy_rows(ny - 2, buf)                 # rows 18..20: past the lattice
