"""The batched solver (many lattices per launch, graph-captured check
intervals, per-instance convergence and failure) against the single-lattice
path and the oracle."""
import numpy as np
import pytest

import oracle
from paper_1412_5170_gb300 import synth

pytestmark = pytest.mark.gpu


def instances():
    return [dict(side=64, kind="droplet", T_over_Tc=0.8, tau=1.0, A=-0.304, K=1.0, size=14.0, seed=1),
            dict(nx=96, ny=40, kind="slab", T_over_Tc=0.75, tau=0.8, A=-0.304, K=0.5, size=10.0, seed=2),
            dict(side=132, kind="droplet", T_over_Tc=0.85, tau=0.6, A=-0.304, K=0.25, size=30.0, seed=3),
            dict(nx=260, ny=36, kind="bubble", T_over_Tc=0.8, tau=1.2, A=-0.304, K=1.0, size=12.0, seed=4)]


@pytest.mark.parametrize("coll,forc", [("bgk", "guo"), ("mrt", "guo"), ("bgk", "edm"), ("bgk", "sc")])
def test_batch_matches_single_lattice_path(lbm, coll, forc):
    """Every instance of a batch evolves as the same lattice run alone with the
    warp strip kernel.  The per-node arithmetic is the same; the initial fields
    differ in the last bits (the batch evaluates the tanh preset on the device,
    the single-lattice call on the host) and the vapour's early transient
    amplifies that, so the bar is the FP32 element-wise bar."""
    inst = instances()
    with lbm.Batch(inst, collision=coll, forcing=forc) as b:
        b.init()
        b.step(57)
        got = [b.read_density(i) for i in range(len(inst))]
    for i, d in enumerate(inst):
        nx, ny = d.get("nx", d.get("side")), d.get("ny", d.get("side"))
        p = lbm.make_params(nx, ny, d["T_over_Tc"], d["tau"], d["A"], d["K"], coll, forc, "fp32",
                            s_e=0.8, s_eps=0.8, s_q=1.1)
        with lbm.Lattice(p) as lat:
            lat.config = 1
            lat.init_preset(d["kind"], d["size"], seed=d["seed"], noise_amp=1e-6)
            lat.step(57)
            rho, _, _ = lat.read_moments()
        assert (np.abs(got[i] - rho) / rho).max() < 2e-5


def test_batch_initial_field_matches_generator(lbm):
    inst = instances()
    with lbm.Batch(inst) as b:
        b.init()
        for i, d in enumerate(inst):
            nx, ny = d.get("nx", d.get("side")), d.get("ny", d.get("side"))
            rv, rl = lbm.maxwell(d["T_over_Tc"])
            want = synth.density_field(nx, ny, d["kind"], rl, rv, d["size"], seed=d["seed"])
            np.testing.assert_allclose(b.read_density(i), want, rtol=2e-7)


def test_batch_against_oracle(lbm):
    inst = instances()[:2]
    steps = 120
    with lbm.Batch(inst, collision="mrt") as b:
        b.init()
        b.step(steps)
        got = [b.read_density(i) for i in range(len(inst))]
    for i, d in enumerate(inst):
        nx, ny = d.get("nx", d.get("side")), d.get("ny", d.get("side"))
        rv, rl = lbm.maxwell(d["T_over_Tc"])
        rho0 = synth.density_field(nx, ny, d["kind"], rl, rv, d["size"], seed=d["seed"])
        q = oracle.params(nx, ny, d["T_over_Tc"], d["tau"], d["A"], d["K"], "mrt", "guo", s_e=0.8, s_eps=0.8, s_q=1.1)
        f, _ = oracle.run(q, oracle.init_rest(rho0), steps)
        ref = f.sum(0)
        assert (np.abs(got[i] - ref) / ref).max() < 2e-5


# the default one-warp walk, and the block walk of 512-column strips
TUNINGS = [None, (512, 2, 16, True)]


@pytest.mark.parametrize("tuning", TUNINGS)
def test_run_to_steady_isolates_failures_and_converges_the_rest(lbm, tuning):
    """One unstable instance fails on its own; the two slabs converge on the
    coexistence criterion (tail rule).  (The all-node criterion tol_rho is not
    used here: in FP32 the rounding of the collision's momentum lets a slab
    drift along y by ~1e-3 lattice units per 10^4 steps, which keeps the
    densities at its interface nodes changing by 1e-4-1e-3 per check although
    the coexistence densities have settled.)"""
    inst = [dict(nx=8, ny=64, kind="slab", T_over_Tc=0.85, tau=1.0, A=-0.304, K=1.0, size=16.0, seed=5),
            dict(side=48, kind="droplet", T_over_Tc=0.5, tau=0.55, A=-0.152, K=1.0, size=12.0, seed=6),   # unstable
            dict(nx=12, ny=64, kind="slab", T_over_Tc=0.8, tau=0.9, A=-0.304, K=0.5, size=16.0, seed=7)]
    with lbm.Batch(inst) as b:
        if tuning:
            b.set_tuning(*tuning)
        b.init()
        b.set_coex_rule("tail")
        st, done = b.run_to_steady(tol_coex=1e-6, check_every=500, max_steps=100000)
        state, code, steps, obs = b.results()
    assert st == lbm.OK
    assert state[1] == lbm.FAILED and code[1] in (lbm.E_NONFINITE, lbm.E_EOS_DOMAIN)
    assert state[0] == lbm.CONVERGED and state[2] == lbm.CONVERGED
    assert steps[1] < steps[0] or steps[1] < steps[2]
    assert done == max(steps)
    # the converged slabs' coexistence densities against a much longer run
    with lbm.Batch([inst[0], inst[2]]) as r:
        r.init()
        r.step(int(max(steps)) + 20000)
        r.observe()
        _, _, _, ref = r.results()
    for j, i in ((0, 0), (1, 2)):
        assert abs(obs["rho_row_mid"][i] / ref["rho_row_mid"][j] - 1) < 1e-5
        assert abs(obs["rho_row0"][i] / ref["rho_row0"][j] - 1) < 1e-4


def test_observe_marks_flagged_instances_failed(lbm):
    """Plain steps and an observation, no run to steady state: an instance
    whose kernels flagged a non-finite or out-of-domain value is reported
    failed with its code; the others keep running."""
    inst = [dict(nx=8, ny=64, kind="slab", T_over_Tc=0.85, tau=1.0, A=-0.304, K=1.0, size=16.0, seed=5),
            dict(side=48, kind="droplet", T_over_Tc=0.5, tau=0.55, A=-0.152, K=1.0, size=12.0, seed=6)]   # unstable
    with lbm.Batch(inst) as b:
        b.init()
        b.step(20000)
        b.observe()
        state, code, _, obs = b.results()
    assert state[1] == lbm.FAILED and code[1] in (lbm.E_NONFINITE, lbm.E_EOS_DOMAIN)
    assert state[0] == lbm.RUNNING and code[0] == 0 and np.isfinite(obs["rho_row_mid"][0])


def test_coexistence_criterion_stops_when_probes_settle(lbm):
    """tol_coex: both coexistence probes (centre/corner, or mid/edge row) stop
    changing; the final probes match a much longer run."""
    inst = [dict(side=64, kind="droplet", T_over_Tc=0.85, tau=1.0, A=-0.5, K=1.0, size=16.0, seed=11),
            dict(nx=16, ny=96, kind="slab", T_over_Tc=0.8, tau=0.8, A=-0.5, K=0.5, size=24.0, seed=12)]
    with lbm.Batch(inst, collision="mrt") as b:
        b.init()
        st, done = b.run_to_steady(tol_coex=1e-5, check_every=1000, max_steps=100000)
        state, _, steps, obs = b.results()
    assert st == lbm.OK and list(state) == [lbm.CONVERGED, lbm.CONVERGED]
    with lbm.Batch(inst, collision="mrt") as c:
        c.init()
        c.step(int(max(steps)) + 20000)
        c.observe()
        _, _, _, ref = c.results()
    assert obs["rho_center"][0] == pytest.approx(ref["rho_center"][0], rel=1e-4)
    assert obs["rho_corner"][0] == pytest.approx(ref["rho_corner"][0], rel=1e-3)
    assert obs["rho_row_mid"][1] == pytest.approx(ref["rho_row_mid"][1], rel=1e-4)
    assert obs["rho_row0"][1] == pytest.approx(ref["rho_row0"][1], rel=1e-3)


def _bench():
    import importlib
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    return importlib.import_module("bench")


def test_tail_rule_decides_as_the_host_rule(lbm):
    """LBM_COEX_TAIL on the device against the host statement of the same
    rule (bench.coex_measure): stepping one check interval at a time, every
    instance stops exactly at the first check where its probes' relative
    change and the remaining changes estimated from the last two pairs of
    changes are all below tol_coex, and no
    earlier than under the change-only rule; its probes then sit at least as
    close to a much longer run's."""
    bench = _bench()
    inst = [dict(side=64, kind="droplet", T_over_Tc=0.85, tau=1.0, A=-0.5, K=1.0, size=16.0, seed=11),
            dict(nx=16, ny=96, kind="slab", T_over_Tc=0.8, tau=0.8, A=-0.5, K=0.5, size=24.0, seed=12),
            dict(side=96, kind="droplet", T_over_Tc=0.6, tau=0.7, A=-0.84, K=0.25, size=14.0, seed=13)]
    tol, every = 1e-5, 1000
    keys = [("rho_row_mid", "rho_row0") if d["kind"] == "slab" else ("rho_center", "rho_corner") for d in inst]
    with lbm.Batch(inst, collision="mrt") as b:
        b.init()
        b.set_coex_rule("tail")
        prev = [None] * len(inst)
        nan = float("nan")
        hist = [((nan, nan), (nan, nan))] * len(inst)
        expect = [None] * len(inst)
        for k in range(1, 200):
            st, _ = b.run_to_steady(tol_coex=tol, check_every=every, max_steps=every)
            state, _, steps, obs = b.results()
            for i in range(len(inst)):
                if expect[i] is not None:
                    continue
                cur = (obs[keys[i][0]][i], obs[keys[i][1]][i])
                if prev[i] is not None:
                    m, hist[i] = bench.coex_measure(prev[i], cur, hist[i], "tail")
                    if m < tol:
                        expect[i] = k * every
                prev[i] = cur
                assert (state[i] == lbm.CONVERGED) == (expect[i] is not None), (i, k)
            if st == lbm.OK:
                break
        assert all(e is not None for e in expect)
        assert list(steps) == expect
        tail_obs = {key: obs[key].copy() for key in ("rho_center", "rho_corner", "rho_row_mid", "rho_row0")}
    with lbm.Batch(inst, collision="mrt") as c:
        c.init()
        st, _ = c.run_to_steady(tol_coex=tol, check_every=every, max_steps=10 ** 6)
        assert st == lbm.OK
        _, _, steps_change, obs_change = c.results()
    assert all(t >= s for t, s in zip(expect, steps_change))
    with lbm.Batch(inst, collision="mrt") as r:
        r.init()
        r.step(max(expect) + 30000)
        r.observe()
        _, _, _, ref = r.results()
    for i, ks in enumerate(keys):
        for key in ks:
            e_tail = abs(tail_obs[key][i] / ref[key][i] - 1)
            e_change = abs(obs_change[key][i] / ref[key][i] - 1)
            assert e_tail <= e_change + 1e-6, (i, key, e_tail, e_change)


@pytest.mark.parametrize("tuning", TUNINGS)
def test_graph_intervals_equal_plain_steps(lbm, tuning):
    inst = instances()
    with lbm.Batch(inst) as a, lbm.Batch(inst) as c:
        if tuning:
            a.set_tuning(*tuning)
            c.set_tuning(*tuning)
        a.init()
        c.init()
        a.run_to_steady(tol_v=1e-30, check_every=50, max_steps=150)   # 3 graph-captured intervals
        c.step(150)
        for i in range(len(inst)):
            assert np.array_equal(a.read_density(i), c.read_density(i))


def test_profiles_of_initial_fields_and_profile_init(lbm):
    """Radial profile of a fresh tanh droplet / slab on an interface-centred
    grid follows the tanh law; a field built from a profile reproduces it."""
    import torch
    inst = [dict(side=128, kind="droplet", T_over_Tc=0.8, tau=1.0, A=-0.304, K=1.0, size=30.0, seed=8, noise_amp=0.0),
            dict(nx=16, ny=128, kind="slab", T_over_Tc=0.8, tau=1.0, A=-0.304, K=1.0, size=25.0, seed=9, noise_amp=0.0)]
    rv, rl = lbm.maxwell(0.8)
    nb, h = 64, 0.5
    geom = [(1, d["size"], h) for d in inst]
    with lbm.Batch(inst) as b:
        b.init()
        prof = b.profiles(nb, geom)
        for i, d in enumerate(inst):
            r = np.abs(d["size"] + h * (np.arange(nb) - 31.5))
            want = rv + (rl - rv) * 0.5 * (1 - np.tanh(2 * (r - d["size"]) / 4.0))
            assert np.abs(prof[i] - want).max() < 0.02 * (rl - rv)
        dev = torch.tensor(prof, dtype=torch.float64, device="cuda")
        b.init_profiles(dev, geom, rest=False)
        prof2 = b.profiles(nb, geom)
    assert np.abs(prof2 - prof).max() < 0.02 * (rl - rv)


def _profile_field(d, p, centre, h):
    """rho0 of a profile laid on an instance (the library's interpolation)."""
    ny, nx = d.get("ny", d.get("side")), d.get("nx", d.get("side"))
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.abs(y - ny / 2.0) if d["kind"] == "slab" else np.hypot(x - nx / 2.0, y - ny / 2.0)
    u = (r - centre) / h + 0.5 * (len(p) - 1)
    k = np.clip(np.floor(u).astype(int), 0, len(p) - 2)
    t = u - k
    out = p[k] + t * (p[k + 1] - p[k])
    out = np.where(u > 0, out, p[0])
    return np.where(u >= len(p) - 1, p[-1], out)


def test_profile_init_at_rest(lbm):
    """LBM_INIT_REST: the populations carry momentum -F/2, so the observed
    velocity v = u + F/(2 rho) starts at zero up to FP32 rounding, while the
    plain start f = w rho0 has v = F/(2 rho) at the interface; the density
    is the profile's either way."""
    import torch
    inst = [dict(side=96, kind="droplet", T_over_Tc=0.75, tau=0.9, A=-0.5, K=0.7, size=20.0, seed=1),
            dict(nx=32, ny=96, kind="slab", T_over_Tc=0.8, tau=0.8, A=-0.5, K=1.0, size=18.0, seed=2)]
    nb, h = 64, 0.5
    rv, rl = lbm.maxwell(0.75)
    prof = np.empty((2, nb))
    geom = []
    for i, d in enumerate(inst):
        r = np.abs(d["size"] + h * (np.arange(nb) - 31.5))
        prof[i] = rv + (rl - rv) * 0.5 * (1 - np.tanh(2 * (r - d["size"]) / 5.0))
        geom.append((1, d["size"], h))
    dev = torch.tensor(prof, dtype=torch.float64, device="cuda")
    out = {}
    with lbm.Batch(inst, collision="mrt") as b:
        for rest in (False, True):
            b.init_profiles(dev, geom, rest=rest)
            b.observe()
            out[rest] = b.results()[3]["max_v"].copy()
            for i, d in enumerate(inst):
                want = _profile_field(d, prof[i], d["size"], h)
                got = b.read_density(i)
                assert np.abs(got - want).max() < 1e-6 * want.max()
    assert np.all(out[False] > 1e-4)
    assert np.all(out[True] < 1e-6) and np.all(out[True] < 1e-3 * out[False])


def test_batch_autotune_keeps_state(lbm):
    inst = instances()
    with lbm.Batch(inst) as b:
        b.init()
        b.step(5)
        before = [b.read_density(i) for i in range(len(inst))]
        cols, ns, rows, carry, ms = b.autotune(3)
        assert (cols, ns, carry) in {(128, 3, False), (128, 4, False), (128, 2, True), (128, 3, True),
                                     (256, 3, True), (512, 2, True), (512, 3, True)}
        assert rows in (32, 64, 128, 256) and ms > 0
        after = [b.read_density(i) for i in range(len(inst))]
    for x, y in zip(before, after):
        assert np.array_equal(x, y)


def wide_instances():
    """The batch instances plus a slab wider than a 512-column strip: ragged
    last strips for both block walks (260 = 256 + 4, 520 = 512 + 8), and
    instances narrower than a strip (64, 96, 132)."""
    return instances() + [dict(nx=520, ny=24, kind="slab", T_over_Tc=0.8, tau=0.9, A=-0.304, K=0.7, size=6.0,
                               seed=13)]


@pytest.mark.parametrize("columns,stages", [(256, 3), (512, 2), (512, 3)])
@pytest.mark.parametrize("coll,forc", [("mrt", "guo"), ("bgk", "guo"), ("bgk", "edm"), ("bgk", "sc")])
def test_block_walks_match_warp_walk_and_oracle(lbm, columns, stages, coll, forc):
    """The block-wide strip walks (a CTA per 256- or 512-column strip) give
    the one-warp walk's fields, and both the oracle's, on 8-row items that
    alternate their walk direction."""
    inst = wide_instances()
    steps = 60
    out = {}
    for w, s, c in ((128, 3, False), (columns, stages, True)):
        with lbm.Batch(inst, collision=coll, forcing=forc) as b:
            b.set_tuning(w, s, 8, c)
            b.init()
            b.step(steps)
            out[w] = [b.read_density(i) for i in range(len(inst))]
    for i, d in enumerate(inst):
        assert np.abs(out[columns][i] - out[128][i]).max() < 1e-6 * out[128][i].max()
        nx, ny = d.get("nx", d.get("side")), d.get("ny", d.get("side"))
        rv, rl = lbm.maxwell(d["T_over_Tc"])
        rho0 = synth.density_field(nx, ny, d["kind"], rl, rv, d["size"], seed=d["seed"])
        q = oracle.params(nx, ny, d["T_over_Tc"], d["tau"], d["A"], d["K"], coll, forc, s_e=0.8, s_eps=0.8, s_q=1.1)
        f, _ = oracle.run(q, oracle.init_rest(rho0), steps)
        ref = f.sum(0)
        assert (np.abs(out[columns][i] - ref) / ref).max() < 2e-5


def test_batch_tuning_rejects_unknown_shapes(lbm):
    with lbm.Batch(instances()[:1]) as b:
        for bad in ((256, 2, 32, True), (256, 3, 32, False), (512, 4, 32, True), (512, 3, 32, False),
                    (384, 3, 32, True),
                    (128, 2, 32, False), (128, 3, 4, False)):
            with pytest.raises(lbm.LbmError):
                b.set_tuning(*bad)
        b.set_tuning(512, 2, 32, True)
        b.set_tuning(512, 3, 32, True)


@pytest.mark.parametrize("tuning", [(128, 3, 16, False), (512, 2, 16, True)])
def test_batch_li_model_matches_oracle(lbm, tuning):
    """Li et al.'s model (Sec. 4.3, Eq. 31; Eq. 4's force, A = 0) in a batch,
    with sigma shared by the batch, against the oracle: per-node density
    within the FP32 element-wise bar after 80 steps, on the one-warp walk and
    the 512-column block walk."""
    inst = [dict(d, A=0.0) for d in wide_instances()[:2]]
    steps, sigma = 80, 0.105
    with lbm.Batch(inst, collision="bgk", forcing="li", sigma=sigma) as b:
        b.set_tuning(*tuning)
        b.init()
        b.step(steps)
        got = [b.read_density(i) for i in range(len(inst))]
    for i, d in enumerate(inst):
        nx, ny = d.get("nx", d.get("side")), d.get("ny", d.get("side"))
        rv, rl = lbm.maxwell(d["T_over_Tc"])
        rho0 = synth.density_field(nx, ny, d["kind"], rl, rv, d["size"], seed=d["seed"])
        q = oracle.params(nx, ny, d["T_over_Tc"], d["tau"], 0.0, d["K"], "bgk", "li", sigma=sigma)
        f, _ = oracle.run(q, oracle.init_rest(rho0), steps)
        ref = f.sum(0)
        assert (np.abs(got[i] - ref) / ref).max() < 2e-5


def test_batch_li_model_needs_eq4_force(lbm):
    """Li et al.'s model takes Eq. 4's force (A = 0 in Eq. 6); a batch whose
    instance has another A is rejected, as a single lattice would be."""
    with pytest.raises(lbm.LbmError):
        lbm.Batch(instances()[:1], collision="bgk", forcing="li", sigma=0.105)


def test_coex_rule_rejects_unknown_values(lbm):
    with lbm.Batch(instances()[:1]) as b:
        assert lbm.lbm_batch_set_coex_rule(b.h, 2) == lbm.E_INVALID
        assert lbm.lbm_batch_set_coex_rule(b.h, -1) == lbm.E_INVALID
        b.set_coex_rule("change")
        b.set_coex_rule("tail")
