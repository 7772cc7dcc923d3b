"""Runtime behaviour of the CUDA path through the C ABI: conservation and
determinism of the FP64 reductions, population I/O, checkpoints, presets,
run-to-steady, and failure detection (host-side fault injection only)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1412_5170_gb300 import synth

pytestmark = pytest.mark.gpu
MRT = dict(s_e=0.8, s_eps=0.8, s_q=1.1)


def lattice(lbm, nx=64, ny=48, precision="fp64", coll="mrt", tr=0.8, tau=0.9, A=-0.304, K=1.0, **kw):
    p = lbm.make_params(nx, ny, tr, tau, A, K, coll, "guo", precision, **MRT, **kw)
    return lbm.Lattice(p)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_mass_is_conserved(lbm, precision, tol):
    """FP32: the rest population is closed on the mass, so the FP64 mass sum
    of the deviations drifts only by rounding.  FP64: each population keeps
    its own formula, as in the oracle, whose weights (4/9, 1/9, 1/36) are
    inexact in binary; the mass then drifts by a few 1e-14 per 1000 steps,
    and the bar is 1e-13 or twice the oracle's own drift on the same run."""
    with lattice(lbm, precision=precision) as lat:
        lat.init_preset("droplet", 12.0, seed=1)
        m0 = lat.stats()["mass"]
        lat.step(1000)
        st = lat.stats()
    assert st["status"] == 0
    if precision == "fp64":
        rv, rl = lbm.maxwell(0.8)
        rho0 = synth.density_field(64, 48, "droplet", rl, rv, 12.0, seed=1)
        q = oracle.params(64, 48, 0.8, 0.9, -0.304, 1.0, "mrt", "guo", **MRT)
        f, ost = oracle.run(q, oracle.init_rest(rho0), 1000)
        assert ost == oracle.OK
        tol = max(tol, 2 * abs(f.sum() - rho0.sum()) / rho0.sum())
    assert abs(st["mass"] - m0) / m0 < tol


def test_runs_are_bitwise_deterministic(lbm):
    out = []
    for _ in range(2):
        with lattice(lbm, 96, 64, "fp32") as lat:
            lat.init_preset("droplet", 20.0, seed=5)
            lat.stats(snapshot=True)
            lat.step(300)
            out.append((lat.read_populations(), lat.stats()))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("nx", [80, 81])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stats_match_host_reductions(lbm, nx, precision):
    """The FP64 reductions of lbm_stats against the host's reductions of the
    moment fields, on a lattice the strip observation covers (nx % 4 == 0,
    one launch with its last-CTA reduction) and on one it does not (the
    generic tiles and the one-CTA final reduce); three calls in a row, so the
    last-CTA counter must be ready again after each."""
    with lattice(lbm, nx, 60, precision) as lat:
        lat.init_preset("slab", 15.0, seed=2)
        for k in range(3):
            lat.step(50)
            st = lat.stats()
            rho, vx, vy = lat.read_moments()
            assert st["mass"] == pytest.approx(rho.sum(), rel=1e-14)
            assert st["max_v"] == pytest.approx(np.hypot(vx, vy).max(), rel=1e-14 if precision == "fp64" else 1e-6)
            assert st["rho_min"] == rho.min() and st["rho_max"] == rho.max()
            assert st["rho_center"] == rho[30, nx // 2] and st["rho_corner"] == rho[0, 0]
            assert st["rho_row_mid"] == pytest.approx(rho[30].mean(), rel=1e-14)
            assert st["rho_row0"] == pytest.approx(rho[0].mean(), rel=1e-14)
            assert st["steps"] == 50 * (k + 1) and st["max_dv"] == -1.0 and st["status"] == 0


@pytest.mark.parametrize("nx", [64, 66])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_snapshot_difference(lbm, nx, precision):
    with lattice(lbm, nx, 64, precision) as lat:
        lat.init_preset("droplet", 16.0, seed=3)
        lat.step(10)
        _, vx0, vy0 = lat.read_moments()
        lat.stats(snapshot=True)
        lat.step(25)
        _, vx1, vy1 = lat.read_moments()
        st = lat.stats()
    # FP32: v is computed (and snapshotted) in float, the fields are its exact doubles
    assert st["max_dv"] == pytest.approx(np.hypot(vx1 - vx0, vy1 - vy0).max(), rel=1e-13 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_population_roundtrip(lbm, precision):
    f = synth.random_populations(36, 20, seed=8)
    with lattice(lbm, 36, 20, precision) as lat:
        lat.write_populations(f)
        g = lat.read_populations()
    if precision == "fp64":
        assert np.array_equal(f, g)
    else:
        assert np.abs(f - g).max() < 1e-7 * np.abs(f).max()


def test_write_populations_then_step_matches_oracle(lbm):
    f = synth.random_populations(24, 20, seed=12, base=0.25, amp=0.1)
    with lattice(lbm, 24, 20, tr=0.75, A=-0.3, K=0.5) as lat:
        lat.write_populations(f)
        lat.step(5)
        g = lat.read_populations()
    q = oracle.params(24, 20, 0.75, 0.9, -0.3, 0.5, "mrt", "guo", **MRT)
    ref, _ = oracle.run(q, f, 5)
    assert np.abs(g - ref).max() / np.abs(ref).max() < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume_is_bitwise(lbm, tmp_path, precision):
    path = tmp_path / "ck.lbm"
    with lattice(lbm, 68, 44, precision) as a:
        a.init_preset("droplet", 11.0, seed=4)
        a.step(40)
        a.save(path)
        a.step(40)
        fa = a.read_populations()
    with lattice(lbm, 68, 44, precision) as b:
        b.load(path)
        assert b.stats()["steps"] == 40
        b.step(40)
        fb = b.read_populations()
    assert np.array_equal(fa, fb)


def test_corrupt_or_mismatched_checkpoint_is_rejected(lbm, tmp_path):
    path = tmp_path / "ck.lbm"
    with lattice(lbm, 32, 32) as a:
        a.init_preset("droplet", 8.0)
        a.save(path)
    raw = bytearray(path.read_bytes())
    raw[-5] ^= 0xFF
    bad = tmp_path / "bad.lbm"
    bad.write_bytes(bytes(raw))
    with lattice(lbm, 32, 32) as b:
        with pytest.raises(lbm.LbmError) as e:
            b.load(bad)
        assert e.value.status == lbm.E_IO
    with lattice(lbm, 32, 36) as c:
        with pytest.raises(lbm.LbmError):
            c.load(path)
    (tmp_path / "short.lbm").write_bytes(bytes(raw[:100]))
    with lattice(lbm, 32, 32) as d:
        with pytest.raises(lbm.LbmError):
            d.load(tmp_path / "short.lbm")


@pytest.mark.parametrize("kind", ["slab", "droplet", "bubble", "droplet_array"])
def test_preset_matches_synthetic_generator(lbm, kind):
    nx, ny = 96, 80
    rv, rl = lbm.maxwell(0.8)
    want = synth.density_field(nx, ny, kind, rl, rv, 13.0, width=5.0, seed=77, noise_amp=1e-5, cell=48)
    with lattice(lbm, nx, ny) as lat:
        lat.init_preset(kind, 13.0, width=5.0, seed=77, noise_amp=1e-5, cell=48)
        rho, _, _ = lat.read_moments()
    np.testing.assert_allclose(rho, want, rtol=1e-14, atol=0)   # rho = sum_a w_a rho0: 9 roundings


def test_run_to_steady_converges_on_flat_interface(lbm):
    with lattice(lbm, 8, 64, coll="bgk", tr=0.85, tau=1.0) as lat:
        lat.init_preset("slab", 16.0)
        st, done = lat.run_to_steady(1e-10, check_every=500, max_steps=200000)
        s = lat.stats()
    assert st == lbm.OK, lbm.lbm_strerror(st)
    assert 0 < done < 200000 and s["max_dv"] < 1e-10


def test_run_to_steady_reports_not_converged(lbm):
    with lattice(lbm, 32, 32) as lat:
        lat.init_preset("droplet", 8.0)
        st, done = lat.run_to_steady(1e-30, check_every=10, max_steps=50)
    assert st == lbm.E_NOT_CONVERGED and done == 50


def test_nonfinite_input_is_detected(lbm):
    """Fault injection on the host: a NaN in the initial density."""
    rho0 = np.full((16, 16), 0.2)
    rho0[3, 5] = np.nan
    with lattice(lbm, 16, 16, "fp32") as lat:
        lat.init_density(rho0)
        lat.step(3)
        st = lat.stats()
        assert st["status"] in (lbm.E_NONFINITE, lbm.E_EOS_DOMAIN)
        code, _ = lat.run_to_steady(1e-9, 10, 100)
        assert code in (lbm.E_NONFINITE, lbm.E_EOS_DOMAIN)


def test_eos_domain_violation_is_detected(lbm):
    """rho >= 1 is outside the Carnahan-Starling domain (eta = rho < 1)."""
    rho0 = np.full((12, 12), 0.3)
    rho0[6, 6] = 1.2
    with lattice(lbm, 12, 12) as lat:
        lat.init_density(rho0)
        lat.step(1)
        assert lat.stats()["status"] == lbm.E_EOS_DOMAIN


def test_unstable_run_fails_cleanly_then_context_is_reusable(lbm):
    """BGK at tau = 0.55, T/Tc = 0.5 with the small-eps weight blows up; the
    library reports it, and re-initialising the same context works."""
    with lattice(lbm, 48, 48, "fp64", coll="bgk", tr=0.5, tau=0.55, A=-0.152) as lat:
        lat.init_preset("droplet", 12.0)
        code, _ = lat.run_to_steady(1e-9, 200, 4000)
        assert code in (lbm.E_NONFINITE, lbm.E_EOS_DOMAIN)
        rv, rl = lbm.maxwell(0.5)
        lat.init_density(np.full((48, 48), rv))
        lat.step(10)
        assert lat.stats()["status"] == 0


def test_workspace_from_library_allocation(lbm):
    p = lbm.make_params(32, 32, 0.8, 0.9, -0.304, collision="mrt", **MRT)
    a = lbm.Lattice(p, torch_workspace=False)
    b = lbm.Lattice(p, torch_workspace=True)
    for lat in (a, b):
        lat.init_preset("droplet", 8.0, seed=1)
        lat.step(20)
    assert np.array_equal(a.read_populations(), b.read_populations())
    a.close()
    b.close()


def test_variant_selection(lbm):
    with lattice(lbm, 30, 30) as lat:
        assert lat.variant == 0                  # nx % 4 != 0: the generic kernel only
        with pytest.raises(lbm.LbmError):
            lat.variant = 1
    with lattice(lbm, 64, 30) as lat:
        assert lat.variant == 0                  # too few strips x chunks to give every SM a CTA
        lat.variant = 1
        assert lat.variant == 1
        lat.variant = -1
        assert lat.variant == 0
    with lattice(lbm, 1024, 2560) as lat:        # 4 strips x 160 chunks: the strip kernel
        assert lat.variant == 1


def test_every_kernel_configuration_matches_oracle(lbm):
    """Each strip-kernel tile configuration the autotuner can pick (FP64)."""
    nx, ny, steps = 136, 44, 12
    rv, rl = lbm.maxwell(0.8)
    rho0 = synth.density_field(nx, ny, "droplet", rl, rv, 10.0, seed=21)
    q = oracle.params(nx, ny, 0.8, 0.9, -0.304, 1.0, "mrt", "guo", **MRT)
    ref, _ = oracle.run(q, oracle.init_rest(rho0), steps)
    p = lbm.make_params(nx, ny, 0.8, 0.9, -0.304, 1.0, "mrt", "guo", "fp64", **MRT)
    with lbm.Lattice(p) as lat:
        cfgs = lat.configs()
        assert len(cfgs) >= 3 and cfgs[0][0] == 0
        for cid, *_ in cfgs:
            lat.config = cid
            lat.init_density(rho0)
            lat.step(steps)
            f = lat.read_populations()
            assert np.abs(f - ref).max() / np.abs(ref).max() < 1e-12, cid


@pytest.mark.parametrize("coll,forc,nx,ny,steps", [("mrt", "guo", 260, 40, 150), ("bgk", "guo", 1028, 24, 60),
                                                     ("bgk", "li", 2056, 20, 40), ("bgk", "edm", 260, 40, 60),
                                                     ("bgk", "sc", 1028, 24, 60)])
def test_every_fp32_configuration_matches_oracle(lbm, coll, forc, nx, ny, steps):
    """Each FP32-deviation kernel configuration (generic, warp-per-strip and
    block-strip tile shapes) against the FP64 oracle: per-node relative
    density error below 2e-5.  Widths give ragged last strips for every strip
    width: 260 = 2 x 128 + 4 (one partial strip for 256 and 512 threads),
    1028 = 1024 + 4, 2056 = 2048 + 8."""
    rv, rl = lbm.maxwell(0.8)
    rho0 = synth.density_field(nx, ny, "droplet", rl, rv, min(11.0, ny / 3), seed=23)
    A, sigma = (0.0, 0.105) if forc == "li" else (-0.304, 0.0)
    q = oracle.params(nx, ny, 0.8, 0.9, A, 1.0, coll, forc, sigma=sigma, **MRT)
    ref, _ = oracle.run(q, oracle.init_rest(rho0), steps)
    rho_ref = ref.sum(0)
    p = lbm.make_params(nx, ny, 0.8, 0.9, A, 1.0, coll, forc, "fp32", sigma=sigma, **MRT)
    with lbm.Lattice(p) as lat:
        for cid, *_ in lat.configs():
            lat.config = cid
            lat.init_density(rho0)
            lat.step(steps)
            assert lat.stats()["status"] == 0
            rho = lat.read_populations().sum(0)
            assert (np.abs(rho - rho_ref) / rho_ref).max() < 2e-5, cid


def test_fp32_configurations_agree(lbm):
    nx, ny = 520, 36
    p = lbm.make_params(nx, ny, 0.75, 0.8, -0.304, 0.5, "mrt", "guo", "fp32", **MRT)
    outs = []
    with lbm.Lattice(p) as lat:
        for cid, *_ in lat.configs():
            lat.config = cid
            lat.init_preset("droplet", 12.0, seed=2)
            lat.step(25)
            outs.append(lat.read_populations())
    for o in outs[1:]:
        assert np.abs(o - outs[0]).max() < 1e-6 * np.abs(outs[0]).max()


def test_autotune_picks_a_configuration_without_advancing_the_state(lbm):
    with lattice(lbm, 512, 256, "fp32") as lat:
        lat.init_preset("droplet", 60.0, seed=6)
        lat.step(3)
        before = lat.read_populations()
        cfg, ms = lat.autotune(5)
        after = lat.read_populations()
        assert np.array_equal(before, after)
        assert 0 <= cfg < len(lat.configs()) and ms > 0
        assert lat.config == cfg
        assert lat.stats()["steps"] == 3


def _pinned(shape):
    import torch
    return torch.empty(shape, dtype=torch.float64).pin_memory().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_async_io_matches_synchronous_calls(lbm, precision):
    """Asynchronous init and moment reads give the synchronous calls' fields
    bit for bit, with three reads in flight over the two device slots (the
    third reuses the first read's slot) and two asynchronous inits in a row
    (the second reuses the staging array)."""
    nx, ny = 264, 72
    rv, rl = lbm.maxwell(0.8)
    rho_a = synth.density_field(nx, ny, "droplet", rl, rv, 20.0, seed=31)
    rho_b = synth.density_field(nx, ny, "slab", rl, rv, 15.0, seed=32)
    want = []
    with lattice(lbm, nx, ny, precision) as lat:
        lat.init_density(rho_a)
        lat.init_density(rho_b)
        want.append(lat.read_moments())
        lat.step(25)
        want.append(lat.read_moments())
        lat.step(25)
        want.append(lat.read_moments())
    h_a, h_b = _pinned((ny, nx)), _pinned((ny, nx))
    h_a[:], h_b[:] = rho_a, rho_b
    outs = [tuple(_pinned((ny, nx)) for _ in range(3)) for _ in range(3)]
    with lattice(lbm, nx, ny, precision) as lat:
        lat.init_density_async(h_a)
        lat.init_density_async(h_b)
        lat.read_moments_async(outs[0])
        lat.step(25)
        lat.read_moments_async(outs[1])
        lat.step(25)
        lat.read_moments_async(outs[2])
        lat.wait_io()
        assert lat.stats()["steps"] == 50
    for got, ref in zip(outs, want):
        for g, r in zip(got, ref):
            assert np.array_equal(g, r)


def test_async_reads_into_pageable_memory(lbm):
    """Pageable host arrays work too (the copies then do not overlap)."""
    with lattice(lbm, 64, 48, "fp32") as lat:
        lat.init_preset("droplet", 12.0, seed=3)
        lat.step(10)
        ref = lat.read_moments()
        out = tuple(np.empty((48, 64)) for _ in range(3))
        lat.read_moments_async(out)
        lat.wait_io()
    for g, r in zip(out, ref):
        assert np.array_equal(g, r)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stage_wait_timeout_is_reported_and_the_context_recovers(lbm, precision):
    """Failure detection of the staged kernels, without a stuck copy: in one
    step every CTA's first shared-memory stage wait gives up at once (as a
    copy that never lands would make it, after its poll limit).  Each
    configuration of the block-strip and warp kernels must then flag the
    timeout, drain the copies it issued and return: lbm_stats reports
    LBM_E_TIMEOUT, and after re-initialisation the same context steps exactly
    as a context that never timed out (and, in FP64, as the oracle)."""
    nx, ny, steps = 136, 40, 12
    p = lbm.make_params(nx, ny, 0.8, 0.9, -0.304, 1.0, "mrt", "guo", precision, **MRT)
    rv, rl = lbm.maxwell(0.8)
    rho0 = synth.density_field(nx, ny, "droplet", rl, rv, 10.0, seed=4)
    with lbm.Lattice(p) as lat:
        staged = [cid for cid, *_ in lat.configs() if cid >= 1]
        assert staged
        for cid in staged:
            lat.config = cid
            lat.init_density(rho0)
            lat.step(2)
            lat.inject_stage_timeout()
            lat.step(1)
            assert lat.stats()["status"] == lbm.E_TIMEOUT, cid
            lat.init_density(rho0)
            lat.step(steps)
            st = lat.stats()
            assert st["status"] == 0, cid
            f = lat.read_populations()
            with lbm.Lattice(p) as clean:
                clean.config = cid
                clean.init_density(rho0)
                clean.step(steps)
                assert np.array_equal(f, clean.read_populations()), cid
        lat.config = 0
        with pytest.raises(lbm.LbmError):
            lat.inject_stage_timeout()          # the generic kernel stages nothing
    if precision == "fp64":
        q = oracle.params(nx, ny, 0.8, 0.9, -0.304, 1.0, "mrt", "guo", **MRT)
        ref, ost = oracle.run(q, oracle.init_rest(rho0), steps)
        assert ost == oracle.OK
        assert np.abs(f - ref).max() / np.abs(ref).max() < 1e-12


def test_fma_peak_measures_both_precisions(lbm):
    """lbm_fma_peak, the FP64 step's roofline: the FP64 FMA rate is a small
    fraction of the FP32 one on this GPU, both positive and below what the
    clock and SM count allow (152 SMs x 2.1 GHz x 128 FP32 lanes x 2 flops =
    82 TFLOP/s)."""
    p64, p32 = lbm.fma_peak("fp64"), lbm.fma_peak("fp32")
    assert 0.1 < p64 < p32 / 8
    assert 10.0 < p32 < 90.0
