"""Flat-interface coexistence curves on the batched engine (FP32 deviations):
the data behind the paper's Figs. 2-6 and Table 6 (Secs. 4.2.2, 4.3 and
4.4.1; Eqs. 18-19).  Each scheme runs as one batch of 8 x 128 periodic slabs
(half-width 32, tau = 1) at three temperatures for 40 000 steps:

  * Kupershtokh's force with Guo's scheme, eps = 1.68 (A = -0.84);
  * Li et al.'s model, sigma = 0.105 (eps = 16 sigma = 1.68, Eq. 32);
  * Kupershtokh's force with the exact-difference scheme, eps = 0.52.

Each slab is held to the same slab run by the FP64 oracle: both coexistence
densities (mid-row and edge-row means, reading 11) within 1e-4 relative, the
FP32 tolerance.  The batched curve is held to the mechanical-stability
solution of its eps (Eq. 18, the library's host solver) where the FP64
curves of the paper's schemes meet it: Guo and Li at T/Tc = 0.9 within 1 %
and at 0.8 within 3 % (the FP64 slabs sit at +0.1 % / -0.2 % and +2.1 % /
-0.8 %); and the exact-difference scheme, which the paper finds farther from
Eq. 18 than Guo's (Sec. 4.2.2), off it by more than Guo's at T/Tc = 0.8.
The oracle runs on host threads while the GPU batches run.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1412_5170_gb300 import synth

pytestmark = pytest.mark.gpu

NX, NY, HALF, TAU, STEPS = 8, 128, 32.0, 1.0, 40000
TEMPS = (0.7, 0.8, 0.9)
SCHEMES = {"guo": dict(A=-0.84, sigma=0.0, eps=1.68), "li": dict(A=0.0, sigma=0.105, eps=1.68),
           "edm": dict(A=-0.26, sigma=0.0, eps=0.52)}


def slab(lbm, tr, seed):
    rv, rl = lbm.maxwell(tr)
    return synth.density_field(NX, NY, "slab", rl, rv, HALF, seed=seed)


def oracle_probes(forc, tr, rho0):
    s = SCHEMES[forc]
    q = oracle.params(NX, NY, tr, TAU, s["A"], 1.0, "bgk", forc, sigma=s["sigma"])
    f, st = oracle.run(q, oracle.init_rest(rho0), STEPS)
    assert st == oracle.OK
    rho = f.sum(0)
    return rho[NY // 2].mean(), rho[0].mean()


@pytest.fixture(scope="module")
def curves(lbm):
    """{scheme: (batched FP32 probes [T][2], oracle futures [T])}."""
    oracle.build()
    pool = ThreadPoolExecutor(len(SCHEMES) * len(TEMPS))
    out = {}
    for forc, s in SCHEMES.items():
        futs = [pool.submit(oracle_probes, forc, tr, slab(lbm, tr, 40 + j)) for j, tr in enumerate(TEMPS)]
        inst = [dict(nx=NX, ny=NY, kind="slab", T_over_Tc=tr, tau=TAU, A=s["A"], K=1.0, size=HALF, seed=40 + j)
                for j, tr in enumerate(TEMPS)]
        with lbm.Batch(inst, collision="bgk", forcing=forc, sigma=s["sigma"]) as b:
            b.init()
            b.step(STEPS)
            b.observe()
            state, code, steps, obs = b.results()
        assert (code == 0).all(), (forc, code)
        out[forc] = (np.stack([obs["rho_row_mid"], obs["rho_row0"]], axis=1), futs)
    yield out
    pool.shutdown(wait=True)


@pytest.mark.parametrize("forc", list(SCHEMES))
def test_batched_slabs_match_fp64_oracle(curves, forc):
    got, futs = curves[forc]
    for j, tr in enumerate(TEMPS):
        rl, rv = futs[j].result()
        assert abs(got[j, 0] - rl) / rl < 1e-4, (forc, tr, got[j, 0], rl)
        assert abs(got[j, 1] - rv) / rv < 1e-4, (forc, tr, got[j, 1], rv)


def test_batched_curves_against_eq18(lbm, curves):
    # (Eq. 18 has no root for eps = 0.52 below T/Tc of about 0.75)
    rel = {}
    for forc, tr in (("guo", 0.8), ("guo", 0.9), ("li", 0.8), ("li", 0.9), ("edm", 0.8)):
        mv, ml = lbm.mechanical(tr, 1.0, SCHEMES[forc]["eps"])
        rel[forc, tr] = curves[forc][0][TEMPS.index(tr), 1] / mv - 1
    for forc in ("guo", "li"):
        assert abs(rel[forc, 0.9]) < 0.01, (forc, rel[forc, 0.9])
        assert abs(rel[forc, 0.8]) < 0.03, (forc, rel[forc, 0.8])
    assert abs(rel["edm", 0.8]) > abs(rel["guo", 0.8])
