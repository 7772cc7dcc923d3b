"""Learned warm start for batched runs to steady state.

Training data come from the batched solver itself: instances drawn from the
workload distribution are run to steady state and their converged density
profiles are sampled at s_k = (k + 1/2) * 2/64, s = r/R (droplet) or
|y - ny/2|/h (slab).  A network per geometry (inputs T/Tc, tau, A, K, radius
or half-width; outputs log rho at the 64 samples), trained by liblbm's own
FP32 kernels, predicts the profile of a new instance; the batched solver then
starts from that profile instead of the tanh preset and runs to the same
convergence criterion, so the solver itself judges the prediction (an
instance whose warm start fails is simply rerun cold).

Orchestration only: every lattice update, reduction, profile extraction and
network evaluation runs in liblbm's CUDA kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import lbm

NB, SMAX = 64, 2.0
KINDS = ("droplet", "slab")


def features(inst) -> list:
    return [inst["T_over_Tc"], inst["tau"], inst["A"], inst["K"], inst["size"]]


def solve(instances, collision="mrt", tol_v=0.0, tol_rho=0.0, tol_coex=1e-5, check_every=1000, max_steps=100000,
          profiles=None, tune=True):
    """Run a batch to steady state.  profiles: optional (n, NB) densities for
    a warm start (rows of NaN start from the preset).  Returns a dict with
    per-instance state, failure code, steps, observables, converged profiles,
    and the wall time of the run (initialisation included)."""
    import torch
    with lbm.Batch(instances, collision=collision) as b:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if profiles is None:
            b.init()
        else:
            use = [int(np.all(np.isfinite(p))) for p in profiles]
            dev = torch.tensor(np.nan_to_num(np.asarray(profiles, dtype=np.float64), nan=0.0), device="cuda")
            b.init(dev, use, SMAX)
        if tune:
            b.autotune(3)
        st, done = b.run_to_steady(tol_v=tol_v, tol_rho=tol_rho, tol_coex=tol_coex, check_every=check_every,
                                   max_steps=max_steps)
        wall = time.perf_counter() - t0
        state, code, steps, obs = b.results()
        prof = b.profiles(NB, SMAX)
        nodes = b.nodes
    return dict(status=st, steps_done=done, state=state, code=code, steps=steps, obs=obs, profiles=prof,
                wall_s=wall, nodes=nodes)


def coexistence(instances, obs):
    """(rho_liquid, rho_vapour) per instance: droplet centre / corner, slab mid / edge row."""
    rl = np.where([i["kind"] == "slab" for i in instances], obs["rho_row_mid"], obs["rho_center"])
    rv = np.where([i["kind"] == "slab" for i in instances], obs["rho_row0"], obs["rho_corner"])
    return rl, rv


class WarmStart:
    """One network per geometry, trained on converged profiles."""

    def __init__(self, hidden=128, layers=3, seed=0):
        self.nets = {k: lbm.WarmStartNet(5, hidden, layers, NB, seed=seed + i) for i, k in enumerate(KINDS)}

    def fit(self, instances, profiles, epochs=2000, batch=256, lr=1e-3, seed=0):
        """Train on converged profiles (n, NB); returns the final loss per geometry."""
        X = np.array([features(i) for i in instances], dtype=np.float32)
        Y = np.log(np.asarray(profiles, dtype=np.float64)).astype(np.float32)
        losses = {}
        for k, net in self.nets.items():
            sel = np.array([i["kind"] == k for i in instances])
            if sel.sum() < 2:
                continue
            xs, ys = X[sel].std(0), Y[sel].std(0)
            xs[xs == 0] = 1.0
            ys[ys == 0] = 1.0
            net.set_scaling(X[sel].mean(0), xs, Y[sel].mean(0), ys)
            losses[k] = net.train(X[sel], Y[sel], epochs=epochs, batch=batch, lr=lr, seed=seed)
        return losses

    def predict(self, instances) -> np.ndarray:
        """Predicted density profiles (n, NB)."""
        X = np.array([features(i) for i in instances], dtype=np.float32)
        out = np.full((len(instances), NB), np.nan)
        for k, net in self.nets.items():
            sel = np.array([i["kind"] == k for i in instances])
            if sel.any():
                out[sel] = np.exp(net.predict(X[sel]).astype(np.float64))
        return out

    def close(self):
        for n in self.nets.values():
            n.close()
