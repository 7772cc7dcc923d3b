"""The learned warm start end to end on the batched solver: a restart from
converged profiles (a perfect prediction) and a network trained on the
solver's own converged profiles both reach the cold run's steady state in
fewer steps."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CRIT = dict(tol_coex=1e-5, check_every=1000, max_steps=60000)


def narrow(n, seed):
    """Droplets and slabs from a narrow band of the batched sweep (sides 96 to
    160, T/Tc 0.72 to 0.85, K 0.4 to 1), MRT+Guo with A = -0.84: every
    instance is stable and converges within a few ten thousand steps."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(rng.choice([96, 128, 160]))
        kind = "droplet" if i % 2 == 0 else "slab"
        out.append(dict(side=side, kind=kind, T_over_Tc=float(rng.uniform(0.72, 0.85)),
                        tau=float(rng.uniform(0.7, 1.0)), A=-0.84, K=float(rng.uniform(0.4, 1.0)),
                        size=float(rng.uniform(12, side / 4)), seed=int(seed * 1000 + i)))
    return out


def test_restart_from_converged_profiles_at_rest(lbm):
    from paper_1412_5170_gb300 import warmstart as ws
    inst = narrow(6, 1)
    cold = ws.solve(inst, **CRIT)
    assert np.all(cold["state"] == lbm.CONVERGED)
    again = ws.solve(inst, profiles=cold["profiles"], sizes=cold["sizes"], **CRIT)
    assert again["warm"].all() and np.all(again["state"] == lbm.CONVERGED)
    # the mass of the warm field is matched to the preset's, which the dynamics conserve
    np.testing.assert_allclose(again["obs"]["mass"], cold["obs"]["mass"], rtol=1e-5)
    rl_c, rv_c = ws.coexistence(inst, cold["obs"])
    rl_a, rv_a = ws.coexistence(inst, again["obs"])
    np.testing.assert_allclose(rl_a, rl_c, rtol=2e-4)
    np.testing.assert_allclose(rv_a, rv_c, rtol=2e-3)
    assert np.median(again["steps"] / cold["steps"]) <= 0.75
    assert np.all(again["steps"] <= cold["steps"])


def test_trained_network_reduces_steps_to_steady(lbm):
    from paper_1412_5170_gb300 import warmstart as ws
    train, test = narrow(48, 2), narrow(8, 3)
    gen = ws.solve(train, **CRIT)
    net = ws.WarmStart(seed=1)
    losses = net.fit(train, gen["profiles"], gen["sizes"], epochs=1500)
    assert set(losses) == {"droplet", "slab"}
    cold = ws.solve(test, **CRIT)
    warm = ws.solve(test, warm=net, **CRIT)
    net.close()
    assert warm["warm"].all()
    ok = (cold["state"] == lbm.CONVERGED) & (warm["state"] == lbm.CONVERGED)
    assert ok.sum() >= 7
    rl_c, rv_c = ws.coexistence(test, cold["obs"])
    rl_w, rv_w = ws.coexistence(test, warm["obs"])
    np.testing.assert_allclose(rl_w[ok], rl_c[ok], rtol=5e-4)
    np.testing.assert_allclose(rv_w[ok], rv_c[ok], rtol=5e-3)
    assert np.median(warm["steps"][ok] / cold["steps"][ok]) <= 0.8
