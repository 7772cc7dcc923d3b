"""Laplace's law on static gas bubbles (FP64 GPU path): the pressure jump of
the K-scaled EOS (Eq. 30) across the interface, between the bubble's centre
and the corner of the 128x128 box, falls on a straight line through the
origin in 1/R_eq, for the Table 3 setups (T/Tc = 0.6, K = 0.5; Guo with
A = -0.9, EDM with A = -0.26, reading 16)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("forcing,A", [("guo", -0.9), ("edm", -0.26)])
def test_pressure_jump_follows_laplace_law(lbm, forcing, A):
    K, T = 0.5, 0.6
    Tabs = T * oracle.Tc()
    xs, ys = [], []
    for R in (15.0, 22.0, 30.0):
        p = lbm.make_params(128, 128, T, 1.5, A, K, "bgk", forcing, "fp64")
        with lbm.Lattice(p) as lat:
            lat.init_preset("bubble", R, seed=1)
            lat.autotune(3)
            lat.step(30000)
            st = lat.stats()
            rho = lat.read_moments()[0]
        assert st["status"] == 0
        rg, rl = st["rho_center"], st["rho_corner"]
        r_eq = np.sqrt(np.sum(rl - rho) / (np.pi * (rl - rg)))
        xs.append(1.0 / r_eq)
        ys.append(oracle.pressure(rg, Tabs, K) - oracle.pressure(rl, Tabs, K))
    slope, icpt = np.polyfit(xs, ys, 1)
    fit = slope * np.array(xs) + icpt
    assert slope > 0
    assert np.max(np.abs(fit - ys)) < 0.01 * max(ys)      # a straight line in 1/R
    assert abs(icpt) < 0.05 * max(ys)                     # through the origin
