"""FP32-deviation populations against the FP64 oracle where FP32 is hardest.

At low temperature and a small EOS scale K (Sec. 4.1, Eq. 30: K scales the
pressure and widens the interface) the vapour density responds to the
smallest systematic change of the pressure: a change of about 1e-8 rho moves
rho_v by about 1e-4 of itself at T/Tc = 0.5, K = 1/16.  The FP32 step must
therefore apply its constants without bias (see lbm_device.cuh); these
tests hold its steady droplets to the FP32 tolerances against the FP64
oracle run on the same seeded input:

  * coexistence densities -- liquid at the droplet centre, vapour at the
    lattice corner -- within 1e-4 relative;
  * the spurious-velocity magnitude Us_max = max |v| within 5 %.

Droplet of R = 16 on 64 x 64, tau = 0.8, A = -0.84 (eps = 1.68, Sec. 4.3),
MRT rates 0.8 / 0.8 / 1.1, 30 000 steps, T/Tc in {0.5, 0.6}, K in {1, 1/16},
BGK and MRT (Guo forcing).  BGK at T/Tc = 0.5, K = 1 leaves the EOS domain in
the oracle as well and is left out.  The generic kernel, a block-strip and a
warp-strip configuration each run every case.  The oracle runs (about 35 s
each on one core) start on host threads when the module's first test asks
for them and overlap the GPU runs.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1412_5170_gb300 import synth

pytestmark = pytest.mark.gpu

N, R, TAU, A, STEPS = 64, 16.0, 0.8, -0.84, 30000
MRT = dict(s_e=0.8, s_eps=0.8, s_q=1.1)
CASES = [(coll, tr, K) for coll in ("bgk", "mrt") for tr in (0.5, 0.6) for K in (1.0, 1.0 / 16)
         if not (coll == "bgk" and tr == 0.5 and K == 1.0)]


def initial_density(lbm, tr, seed=7):
    rv, rl = lbm.maxwell(tr)
    return synth.density_field(N, N, "droplet", rl, rv, R, seed=seed)


def oracle_probes(case, rho0):
    coll, tr, K = case
    q = oracle.params(N, N, tr, TAU, A, K, coll, "guo", **MRT)
    f, st = oracle.run(q, oracle.init_rest(rho0), STEPS)
    m, mst = oracle.macro(q, f)
    assert st == oracle.OK and mst == oracle.OK, case
    return m["rho"][N // 2, N // 2], m["rho"][0, 0], float(np.hypot(m["vx"], m["vy"]).max())


@pytest.fixture(scope="module")
def reference(lbm):
    """FP64 oracle probes per case, computed on host threads (the C oracle
    releases the GIL) while the GPU tests run."""
    oracle.build()
    pool = ThreadPoolExecutor(len(CASES))
    futures = {c: pool.submit(oracle_probes, c, initial_density(lbm, c[1])) for c in CASES}
    yield futures
    pool.shutdown(wait=True)


def staged_configs(lat):
    """The generic kernel, the first block-strip and the first warp-strip configuration."""
    cfgs = lat.configs()
    block = next(c for c, threads, *_ in cfgs if c >= 1 and threads > 32)
    warp = next(c for c, threads, *_ in cfgs if c >= 1 and threads == 32)
    return [0, block, warp]


@pytest.mark.parametrize("case", CASES, ids=["%s-T%.1f-K%g" % c for c in CASES])
def test_fp32_steady_droplet_matches_fp64_oracle(lbm, reference, case):
    coll, tr, K = case
    rho0 = initial_density(lbm, tr)
    p = lbm.make_params(N, N, tr, TAU, A, K, coll, "guo", "fp32", **MRT)
    got = {}
    with lbm.Lattice(p) as lat:
        for cfg in staged_configs(lat):
            lat.config = cfg
            lat.init_density(rho0)
            lat.step(STEPS)
            st = lat.stats()
            assert st["status"] == 0, (case, cfg)
            got[cfg] = (st["rho_center"], st["rho_corner"], st["max_v"])
    rl, rv, us = reference[case].result()
    for cfg, (gl, gv, gu) in got.items():
        assert abs(gl - rl) / rl < 1e-4, (case, cfg, gl, rl)
        assert abs(gv - rv) / rv < 1e-4, (case, cfg, gv, rv)
        assert abs(gu - us) / us < 0.05, (case, cfg, gu, us)
