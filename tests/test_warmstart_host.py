"""Host-side logic of the learned warm start (no GPU): equivalent sizes,
the profile interpolation, the two-phase test on converged states, the
Maxwell normalisation, and the mass-consistent size iteration."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def ws(lbm):
    from paper_1412_5170_gb300 import warmstart
    return warmstart


def test_equivalent_size_inverts_a_sharp_droplet_and_slab(ws):
    rl, rv = 0.35, 0.01
    d = dict(side=256, kind="droplet", K=0.5)
    R = 37.5
    mass = rv * 256 * 256 + (rl - rv) * math.pi * R * R
    assert ws.equivalent_size(d, mass, rl, rv) == pytest.approx(R, rel=1e-12)
    s = dict(nx=32, ny=200, kind="slab", K=1.0)
    h = 41.0
    mass = rv * 32 * 200 + (rl - rv) * 2 * h * 32
    assert ws.equivalent_size(s, mass, rl, rv) == pytest.approx(h, rel=1e-12)
    # no mass excess: no liquid region
    assert ws.equivalent_size(d, rv * 256 * 256 * 0.9, rl, rv) == 0.0


def test_size_slope_is_the_derivative_of_the_mass(ws):
    rl, rv = 0.3, 0.02
    for d in (dict(side=128, kind="droplet", K=1.0), dict(nx=16, ny=128, kind="slab", K=1.0)):
        def mass(R):
            n = 128 * 128 if d["kind"] == "droplet" else 16 * 128
            area = math.pi * R * R if d["kind"] == "droplet" else 2 * R * 16
            return rv * n + (rl - rv) * area
        R, h = 20.0, 1e-4
        assert ws.size_slope(d, R, rl, rv) == pytest.approx((mass(R + h) - mass(R - h)) / (2 * h), rel=1e-6)


def test_profile_value_is_linear_between_samples_and_flat_beyond(ws):
    p = np.linspace(0.4, 0.01, 64)
    centre, h = 30.0, 0.5
    pos = centre + h * (np.arange(64) - 31.5)
    for k in (0, 10, 31, 62):
        assert ws.profile_value(p, centre, h, pos[k]) == pytest.approx(p[k], abs=1e-15)
        mid = 0.5 * (pos[k] + pos[k + 1])
        assert ws.profile_value(p, centre, h, mid) == pytest.approx(0.5 * (p[k] + p[k + 1]), abs=1e-15)
    assert ws.profile_value(p, centre, h, pos[0] - 5) == p[0]
    assert ws.profile_value(p, centre, h, pos[-1] + 5) == p[-1]


def test_converged_geometry_keeps_two_phase_states_only(ws, lbm):
    inst = [dict(side=64, kind="droplet", K=1.0, size=10.0), dict(side=64, kind="droplet", K=0.25, size=12.0),
            dict(nx=16, ny=64, kind="slab", K=1.0, size=8.0)]
    rl, rv = 0.3, 0.02
    R = 15.0
    obs = {"mass": np.array([rv * 4096 + (rl - rv) * math.pi * R * R, 0.05 * 4096, rv * 1024 + (rl - rv) * 2 * 9 * 16]),
           "rho_center": np.array([rl, 0.0501, 0.0]), "rho_corner": np.array([rv, 0.05, 0.0]),
           "rho_row_mid": np.array([0.0, 0.0, rl]), "rho_row0": np.array([0.0, 0.0, rv])}
    state = np.array([lbm.CONVERGED, lbm.CONVERGED, lbm.CONVERGED])
    size, geom = ws.converged_geometry(inst, state, obs)
    assert size[0] == pytest.approx(R)
    assert np.isnan(size[1])                  # uniform vapour: no interface to learn
    assert size[2] == pytest.approx(9.0)
    assert geom[1][1] == inst[1]["size"] and geom[1][2] == pytest.approx(0.5 / math.sqrt(0.25))
    state[0] = lbm.FAILED
    assert np.isnan(ws.converged_geometry(inst, state, obs)[0][0])


def test_maxwell_normalisation_round_trips(ws, lbm):
    inst = [dict(T_over_Tc=0.6), dict(T_over_Tc=0.85)]
    m = ws.maxwell_logs(inst)
    for i, d in enumerate(inst):
        rv, rl = lbm.maxwell(d["T_over_Tc"])
        assert m[i, 0] == pytest.approx(math.log(rv)) and m[i, 1] == pytest.approx(math.log(rl))
        rho = np.array([rv, rl, math.sqrt(rv * rl)])
        y = (np.log(rho) - m[i, 0]) / (m[i, 1] - m[i, 0])
        np.testing.assert_allclose(y, [0.0, 1.0, 0.5], atol=1e-12)


def test_initial_profiles_reach_the_mass_consistent_size(ws, lbm):
    """The size iteration ends at a fixed point: the equivalent size of the
    conserved mass under the predicted plateaus."""
    obj = ws.WarmStart.__new__(ws.WarmStart)     # no networks: a stand-in prediction
    rl, rv = 0.33, 0.012

    def predict(instances, sizes):
        out = np.empty((len(instances), ws.NB))
        for i, (d, R) in enumerate(zip(instances, sizes)):
            r = np.abs(R + ws.spacing(d) * (np.arange(ws.NB) - 31.5))
            lap = 1.0 + 0.02 / max(R, 1.0)      # plateaus that depend weakly on the size
            out[i] = rv * lap + (rl - rv) * 0.5 * (1 - np.tanh((r - R) / 2.0))
        return out
    obj.predict = predict
    inst = [dict(side=256, kind="droplet", K=1.0, size=20.0), dict(nx=16, ny=256, kind="slab", K=0.5, size=30.0)]
    mass0 = np.array([0.02 * 256 * 256 + 0.3 * math.pi * 25 ** 2, 0.02 * 16 * 256 + 0.3 * 2 * 35 * 16])
    prof, size = obj.initial_profiles(inst, mass0, rounds=8)
    for i, d in enumerate(inst):
        p = prof[i]
        r_l = ws.profile_value(p, size[i], ws.spacing(d), 0.0)
        assert size[i] == pytest.approx(ws.equivalent_size(d, mass0[i], r_l, p[-1]), rel=1e-6)
