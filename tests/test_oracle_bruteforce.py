"""The C oracle against an independent 50-digit stepper on tiny lattices."""
import numpy as np
import pytest

from paper_1412_5170_gb300 import synth

SCHEMES = [("bgk", "guo"), ("bgk", "edm"), ("bgk", "sc"), ("mrt", "guo"), ("bgk", "li")]


@pytest.mark.parametrize("nx,ny", [(4, 4), (5, 3)])
@pytest.mark.parametrize("coll,forc", SCHEMES)
def test_oracle_matches_50_digit_stepper(orc, nx, ny, coll, forc):
    pytest.importorskip("mpmath")
    from mpmath import mpf
    from tests import bruteforce_mp as bf
    li = forc == "li"   # Li et al.'s model: the Eq. 4 force (A = 0) and sigma of Eq. 31
    prm = dict(T_over_Tc=0.75, K=0.5, tau=0.8, A=0.0 if li else -0.3, collision=coll, forcing=forc,
               s_e=0.8, s_eps=0.9, s_q=1.1, sigma=0.105 if li else 0.0)
    f0 = synth.random_populations(nx, ny, seed=5, base=0.25, amp=0.2)
    p = orc.params(nx, ny, prm["T_over_Tc"], prm["tau"], prm["A"], prm["K"], coll, forc,
                   s_e=0.8, s_eps=0.9, s_q=1.1, sigma=prm["sigma"])
    steps = 6
    fo, st = orc.run(p, f0, steps)
    assert st == 0
    fm = {(a, x, y): mpf(float(f0[a, y, x])) for a in range(9) for y in range(ny) for x in range(nx)}
    for _ in range(steps):
        fm = bf.step(fm, nx, ny, prm)
    ref = np.array([[[float(fm[(a, x, y)]) for x in range(nx)] for y in range(ny)] for a in range(9)])
    np.testing.assert_allclose(fo, ref, rtol=1e-13, atol=1e-16)
