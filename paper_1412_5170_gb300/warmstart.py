"""Learned warm start for batched runs to steady state.

Training data come from the batched solver itself: instances drawn from the
workload distribution are run to steady state, and each converged density
field is summarised by its equivalent size (the radius of a droplet, or the
half-width of a slab, that holds the mass excess over the vapour) and 64
samples of its radial density profile on a grid centred on the interface,
r_k = R_eq + h (k - 31.5) with h = 0.5 / sqrt(K) lattice units (the
interface widens as 1/sqrt(K) under the EOS rescaling of Eq. 30).  A network
per geometry, trained by liblbm's own FP32 kernels, maps (T/Tc, tau, A, K,
R_eq) to those samples as log rho normalised by the Maxwell densities of the
temperature (Eq. 19, liblbm's host solver): y = (log rho - log rho_v^M) /
(log rho_l^M - log rho_v^M), about 0 in the vapour and 1 in the liquid, so the
network learns the departure from the equal-area construction rather than
the decades over which the vapour density ranges with T/Tc.

A warm start for a new instance:
  1. its preset is initialised and its mass M0 read: the dynamics conserve
     mass, so the warm field must hold M0 to reach the same steady state;
  2. R_eq is found by iterating R_eq -> network -> plateau densities ->
     R_eq from M0 (a few rounds; the profile depends on R_eq only through the
     Laplace pressure);
  3. the profile is laid on the lattice with the populations at rest
     (lbm_batch_init_profiles with LBM_INIT_REST: v = u + F/(2 rho) = 0), and
     its centre is corrected twice by Newton steps on the lattice mass;
  4. the batched solver runs to the same convergence criterion as the cold
     run, so it judges the prediction; an instance whose warm start fails is
     rerun cold by the caller.

Orchestration only: every lattice update, reduction, profile extraction and
network evaluation runs in liblbm's CUDA kernels.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import lbm

NB = 64
KINDS = ("droplet", "slab")


def spacing(inst) -> float:
    return 0.5 / math.sqrt(inst["K"])


def shape(inst):
    return int(inst.get("ny", inst.get("side"))), int(inst.get("nx", inst.get("side")))


def equivalent_size(inst, mass, rho_l, rho_v) -> float:
    """Radius (droplet) or half-width (slab) of a sharp liquid region that
    holds the mass excess over a uniform vapour of density rho_v."""
    ny, nx = shape(inst)
    area = (mass - rho_v * nx * ny) / (rho_l - rho_v)
    if inst["kind"] == "slab":
        return area / (2.0 * nx)
    return math.sqrt(max(area, 0.0) / math.pi)


def size_slope(inst, size, rho_l, rho_v) -> float:
    """d(mass)/d(size) of a sharp liquid region."""
    ny, nx = shape(inst)
    if inst["kind"] == "slab":
        return 2.0 * nx * (rho_l - rho_v)
    return 2.0 * math.pi * size * (rho_l - rho_v)


def features(inst, size) -> list:
    return [inst["T_over_Tc"], inst["tau"], inst["A"], inst["K"], size]


_MAXWELL: dict = {}


def maxwell_logs(instances):
    """(log rho_v^M, log rho_l^M) per instance from liblbm's Eq. 19 solver."""
    out = np.empty((len(instances), 2))
    for i, d in enumerate(instances):
        T = float(d["T_over_Tc"])
        if T not in _MAXWELL:
            rv, rl = lbm.maxwell(T)
            _MAXWELL[T] = (math.log(rv), math.log(rl))
        out[i] = _MAXWELL[T]
    return out


def coexistence(instances, obs):
    """(rho_liquid, rho_vapour) per instance: droplet centre / corner, slab mid / edge row."""
    slab = np.array([i["kind"] == "slab" for i in instances])
    rl = np.where(slab, obs["rho_row_mid"], obs["rho_center"])
    rv = np.where(slab, obs["rho_row0"], obs["rho_corner"])
    return rl, rv


def profile_value(p, centre, h, r):
    """The library's profile interpolation (linear in r, end values beyond)."""
    u = (r - centre) / h + 0.5 * (len(p) - 1)
    if not u > 0:
        return p[0]
    if u >= len(p) - 1:
        return p[-1]
    k = int(u)
    return p[k] + (u - k) * (p[k + 1] - p[k])


def converged_geometry(instances, state, obs):
    """Equivalent size per converged two-phase instance (NaN elsewhere: a
    uniform final state has no interface to learn) and the sample grids
    centred on it."""
    rl, rv = coexistence(instances, obs)
    size = np.full(len(instances), np.nan)
    for i, d in enumerate(instances):
        if state[i] == lbm.CONVERGED and rl[i] > 1.5 * rv[i] and rv[i] > 0:   # two phases
            size[i] = equivalent_size(d, obs["mass"][i], rl[i], rv[i])
    geom = [(1, s if np.isfinite(s) else d["size"], spacing(d)) for d, s in zip(instances, size)]
    return size, geom


def _rest_init(b, instances, prof, size, use, mass0, keep=None, newton=2):
    """Lay the profiles on the lattice with the populations at rest, the
    centre corrected by Newton steps on the lattice mass; `keep` instances
    are laid down as given (flat profiles) without correction."""
    import torch
    dev = torch.tensor(np.nan_to_num(prof, nan=1.0), dtype=torch.float64, device="cuda")
    keep = np.zeros(len(instances), dtype=bool) if keep is None else keep
    lay = use | keep
    centre = np.where(lay, size, [d["size"] for d in instances]).astype(np.float64)
    h = [spacing(d) for d in instances]
    for it in range(newton + 1):
        b.init_profiles(dev, [(u, c, hh) for u, c, hh in zip(lay, centre, h)], rest=True)
        if it == newton:
            break
        b.observe()
        m = b.results()[3]["mass"]
        for i, d in enumerate(instances):
            if use[i]:
                rl = profile_value(prof[i], centre[i], h[i], 0.0)
                slope = size_slope(d, centre[i], rl, prof[i][-1])
                if slope > 0 and np.isfinite(m[i]):
                    centre[i] += (mass0[i] - m[i]) / slope
    return centre


def solve(instances, collision="mrt", tol_v=0.0, tol_rho=0.0, tol_coex=1e-5, check_every=1000, max_steps=100000,
          warm=None, profiles=None, sizes=None, fallback="failed", tune=True, trace=False, coex_rule="change"):
    """Run a batch to steady state.

    warm: a trained WarmStart (predicts every instance it has a network for);
    or profiles / sizes: given profiles [n, NB] and equivalent sizes (rows
    with a NaN size start from the preset), e.g. the converged profiles of a
    cold run, to measure what a perfect prediction would give.

    When the predicted plateaus leave no mass for a liquid region (equivalent
    size below one lattice unit) the predicted steady state is a uniform
    vapour: the instance starts at rest at its mean density.

    The solver judges every warm start: an instance that fails, or converges
    to a different steady state than the one laid down (one phase where two
    were predicted -- liquid probe below 1.5 x the vapour one, e.g. a droplet
    that evaporated --, a liquid region whose equivalent size is off by more
    than half, or two phases where a uniform vapour was predicted), is rerun
    cold when fallback is "failed" or "all", and its cold result replaces the
    warm one; with "all" so is an instance still running at max_steps.  A
    prediction without two phases (liquid plateau below 1.5 x the vapour) is
    not used at all.

    Returns a dict with per-instance state, failure code, steps of the run
    whose result is kept, steps_total (warm plus fallback steps: the work
    spent), observables, the converged equivalent sizes and profiles (on
    grids centred on them), which instances were warm-started and which fell
    back, the warm run's own outcome before any fallback (`first`), and the
    wall time of everything (initialisation, prediction, mass matching and
    fallback runs included).  trace: also step the batch one check interval
    per call and return, per interval, the instances and nodes still running
    and its wall time (`trace`; the first run only).  coex_rule: how tol_coex
    is judged ("change" per check, or "tail": also the estimated change still
    to come; Batch.set_coex_rule)."""
    import torch
    n = len(instances)
    with lbm.Batch(instances, collision=collision) as b:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.init()
        use = np.zeros(n, dtype=bool)
        uniform = np.zeros(n, dtype=bool)
        centre_used = np.full(n, np.nan)
        if warm is not None or profiles is not None:
            b.observe()
            mass0 = b.results()[3]["mass"].copy()
            if warm is not None:
                prof, size = warm.initial_profiles(instances, mass0)
            else:
                prof, size = np.asarray(profiles, dtype=np.float64), np.asarray(sizes, dtype=np.float64)
            use = np.isfinite(size) & np.all(np.isfinite(prof), axis=1) & np.all(prof > 0, axis=1)
            # a liquid region smaller than one lattice unit holds no mass: the
            # predicted steady state is a uniform vapour at the mean density
            uniform = use & (size < 1.0)
            for i in np.nonzero(uniform)[0]:
                ny, nx = shape(instances[i])
                prof[i] = mass0[i] / (nx * ny)
                size[i] = instances[i]["size"]
            # a two-phase prediction whose liquid plateau is below 1.5 x the vapour is not used
            for i in np.nonzero(use & ~uniform)[0]:
                if not profile_value(prof[i], size[i], spacing(instances[i]), 0.0) > 1.5 * prof[i][-1]:
                    use[i] = False
            if use.any():
                centre_used = _rest_init(b, instances, prof, size, use & ~uniform, mass0, keep=uniform)
        if tune:
            b.autotune(3)
        b.set_coex_rule(coex_rule)
        intervals = []
        if trace:
            sides = np.array([shape(d)[0] * shape(d)[1] for d in instances], dtype=np.float64)
            done = 0
            st = lbm.E_NOT_CONVERGED
            while done < max_steps and st == lbm.E_NOT_CONVERGED:
                running = b.results()[0] == lbm.RUNNING
                torch.cuda.synchronize()
                ti = time.perf_counter()
                st, d = b.run_to_steady(tol_v=tol_v, tol_rho=tol_rho, tol_coex=tol_coex, check_every=check_every,
                                        max_steps=min(check_every, max_steps - done))
                intervals.append((int(running.sum()), float(sides[running].sum()), time.perf_counter() - ti))
                done += d
        else:
            st, done = b.run_to_steady(tol_v=tol_v, tol_rho=tol_rho, tol_coex=tol_coex, check_every=check_every,
                                       max_steps=max_steps)
        state, code, steps, obs = b.results()
        eq_size, geom = converged_geometry(instances, state, obs)
        prof_out = b.profiles(NB, geom)
        nodes = b.nodes
    wall = time.perf_counter() - t0
    steps_total = steps.copy()
    rl, rv = coexistence(instances, obs)
    with np.errstate(invalid="ignore", divide="ignore"):
        # a different steady state than the one laid down: one phase left, or a
        # liquid region of another size (two phases predicted); two phases
        # (uniform vapour predicted)
        two = rl > 1.5 * rv
        off = np.where(uniform, two, ~two | ~(np.abs(eq_size / centre_used - 1) < 0.5))
    first = dict(state=state.copy(), code=code.copy(), steps=steps.copy(), off=off & (state == lbm.CONVERGED),
                 uniform=uniform.copy(),
                 rho_l=rl.copy(), rho_v=rv.copy(), size=eq_size.copy(), centre=centre_used.copy())
    redo = use & ((state == lbm.FAILED) | ((state == lbm.CONVERGED) & off) |
                  ((state == lbm.RUNNING) & (fallback == "all")))
    if fallback not in ("failed", "all"):
        redo[:] = False
    if redo.any():
        idx = np.nonzero(redo)[0]
        r2 = solve([instances[i] for i in idx], collision, tol_v, tol_rho, tol_coex, check_every, max_steps,
                   tune=tune, coex_rule=coex_rule)
        wall += r2["wall_s"]
        state, code, steps = state.copy(), code.copy(), steps.copy()
        obs = {k: v.copy() for k, v in obs.items()}
        for j, i in enumerate(idx):
            state[i], code[i], steps[i] = r2["state"][j], r2["code"][j], r2["steps"][j]
            steps_total[i] += r2["steps"][j]
            for k in obs:
                obs[k][i] = r2["obs"][k][j]
            eq_size[i] = r2["sizes"][j]
            prof_out[i] = r2["profiles"][j]
    return dict(status=st, steps_done=done, state=state, code=code, steps=steps, steps_total=steps_total, obs=obs,
                sizes=eq_size, profiles=prof_out, warm=use, fallback=redo, first=first,
                wall_s=wall, nodes=nodes, trace=intervals)


class WarmStart:
    """One network per geometry: (T/Tc, tau, A, K, R_eq) -> the 64
    interface-centred samples of the Maxwell-normalised log density."""

    def __init__(self, hidden=128, layers=3, seed=0):
        self.nets = {k: lbm.WarmStartNet(5, hidden, layers, NB, seed=seed + i) for i, k in enumerate(KINDS)}
        self.trained = set()

    def fit(self, instances, profiles, sizes, epochs=3000, batch=64, lr=2e-3, seed=0, chunks=30):
        """Train on converged profiles [n, NB] with their equivalent sizes
        (rows with a NaN size are skipped): Adam on minibatches with the step
        size decayed along a cosine over `chunks` stages.  Returns the final
        loss per geometry."""
        ok = np.isfinite(sizes) & np.all(np.asarray(profiles) > 0, axis=1)
        X = np.array([features(d, s) for d, s in zip(instances, sizes)], dtype=np.float32)
        m = maxwell_logs(instances)
        Y = ((np.log(np.where(ok[:, None], profiles, 1.0)) - m[:, :1]) / (m[:, 1:] - m[:, :1])).astype(np.float32)
        losses = {}
        per = max(1, epochs // chunks)
        for k, net in self.nets.items():
            sel = ok & np.array([d["kind"] == k for d in instances])
            if sel.sum() < 2:
                continue
            xs, ys = X[sel].std(0), Y[sel].std(0)
            xs[xs == 0] = 1.0
            ys[ys == 0] = 1.0
            net.set_scaling(X[sel].mean(0), xs, Y[sel].mean(0), ys)
            for c in range(chunks):
                step = lr * (0.5 * (1.0 + math.cos(math.pi * c / chunks)) + 1e-3)
                losses[k] = net.train(X[sel], Y[sel], epochs=per, batch=batch, lr=step, seed=seed + c)
            self.trained.add(k)
        return losses

    def predict(self, instances, sizes) -> np.ndarray:
        """Predicted density profiles [n, NB] (NaN rows for untrained geometries)."""
        X = np.array([features(d, s) for d, s in zip(instances, sizes)], dtype=np.float32)
        m = maxwell_logs(instances)
        out = np.full((len(instances), NB), np.nan)
        for k in self.trained:
            sel = np.array([d["kind"] == k for d in instances])
            if sel.any():
                y = self.nets[k].predict(X[sel]).astype(np.float64)
                out[sel] = np.exp(m[sel, :1] + y * (m[sel, 1:] - m[sel, :1]))
        return out

    def initial_profiles(self, instances, mass0, rounds=3):
        """Profiles and equivalent sizes consistent with the conserved masses
        mass0: R_eq -> prediction -> plateaus -> R_eq, starting from the
        nominal sizes."""
        size = np.array([d["size"] for d in instances], dtype=np.float64)
        prof = self.predict(instances, size)
        for _ in range(rounds):
            for i, d in enumerate(instances):
                p = prof[i]
                if not np.all(np.isfinite(p)):
                    continue
                rl = profile_value(p, size[i], spacing(d), 0.0)
                rv = p[-1]
                if rl > rv > 0:
                    size[i] = equivalent_size(d, mass0[i], rl, rv)
            prof = self.predict(instances, size)
        bad = ~np.all(np.isfinite(prof), axis=1)
        size[bad] = np.nan
        return prof, size

    def close(self):
        for n in self.nets.values():
            n.close()
