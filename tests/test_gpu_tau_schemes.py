"""The relaxation-time dependence of the force schemes on straight
interfaces (Sec. 4.2.1, Table 2, Figs. 2-4), on the batched engine (FP32
deviations): flat slabs of 8 x 127 nodes centred between two rows, 40 000
steps, one batch per scheme over relaxation times and temperatures.

  * Fig. 2: with EDM and Guo's scheme the gas density does not depend on
    tau; with Shan-Chen's it grows with tau, and equals EDM's at tau = 1.
  * Figs. 3 and 4: EDM (A = -0.26) and Guo's scheme (A = -0.5) give the same
    density ratio at tau = 0.7 and 1.5 over the temperatures.

Shan-Chen's gas densities at tau = 0.7 and 1.5 are also held to the FP64
oracle's on the same slabs (run on host threads beside the GPU batches)."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1412_5170_gb300 import synth

pytestmark = pytest.mark.gpu

NX, NY, HALF, STEPS = 8, 127, 32.0, 40000


def slabs(lbm, forcing, A, cases):
    """cases: [(tau, T/Tc)] -> (rho_g, rho_l) arrays from one FP32 batch."""
    inst = [dict(nx=NX, ny=NY, kind="slab", T_over_Tc=T, tau=tau, A=A, K=1.0, size=HALF, seed=11) for tau, T in cases]
    with lbm.Batch(inst, collision="bgk", forcing=forcing) as b:
        b.init()
        b.step(STEPS)
        b.observe()
        state, code, _, obs = b.results()
    assert (code == 0).all(), (forcing, code)
    return np.array(obs["rho_row0"]), np.array(obs["rho_row_mid"])


TAUS = (0.7, 0.8, 1.0, 1.2, 1.5)


def oracle_gas(lbm, forcing, A, tau, T):
    rv, rl = lbm.maxwell(T)
    rho0 = synth.density_field(NX, NY, "slab", rl, rv, HALF, seed=11)
    f, st = oracle.run(oracle.params(NX, NY, T, tau, A, 1.0, "bgk", forcing), oracle.init_rest(rho0), STEPS)
    assert st == oracle.OK
    return f.sum(0)[0].mean()


def test_fig2_gas_density_against_tau(lbm):
    oracle.build()
    pool = ThreadPoolExecutor(2)
    ref = [pool.submit(oracle_gas, lbm, "sc", -0.26, tau, 0.8) for tau in (0.7, 1.5)]
    cases = [(tau, 0.8) for tau in TAUS]
    edm, _ = slabs(lbm, "edm", -0.26, cases)
    guo, _ = slabs(lbm, "guo", -0.26, cases)
    sc, _ = slabs(lbm, "sc", -0.26, cases)
    for g in (edm, guo):
        assert np.abs(g / g[2] - 1).max() < 1e-4
    assert np.all(np.diff(sc) > 0) and sc[-1] > 1.5 * sc[0]
    assert abs(sc[2] / edm[2] - 1) < 1e-5
    assert sc[0] == pytest.approx(ref[0].result(), rel=1e-4) and sc[-1] == pytest.approx(ref[1].result(), rel=1e-4)
    pool.shutdown()


@pytest.mark.parametrize("forcing,A,temps", [("edm", -0.26, (0.6, 0.7, 0.8, 0.9)), ("guo", -0.5, (0.7, 0.8, 0.9))])
def test_figs3_4_density_ratio_does_not_depend_on_tau(lbm, forcing, A, temps):
    cases = [(tau, T) for T in temps for tau in (0.7, 1.5)]
    g, l = slabs(lbm, forcing, A, cases)
    ratio = (l / g).reshape(len(temps), 2)
    assert np.abs(ratio[:, 1] / ratio[:, 0] - 1).max() < 2e-4, ratio
    assert np.all(np.diff(ratio[:, 0]) < 0)    # the ratio falls towards the critical point
