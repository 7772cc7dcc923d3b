"""Throughput benchmark of the fused D2Q9 pseudo-potential step on GB300.

Workload (the paper's method at the throughput configuration): a 4096 x 4096
periodic lattice holding a 16 x 16 array of droplets of radius 80 (one per
256 x 256 cell), T/Tc = 0.7, tau = 0.8, MRT (s_e = s_eps = 0.8, s_q = 1.1)
with Guo forcing, Kupershtokh weight A = -0.304 (A_K = -0.152 in
Kupershtokh's own convention), K = 1; populations held in FP32 as deviations
from w_a rho_v, FP64 reductions.  A "step" is one fused time step over the
whole lattice; the timed region ends with the FP64 mass / max|v| reduction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 runs independent replicas, one per GPU
(launched with torch.distributed.run); the value is the sum over replicas
divided by the slowest replica's time.  --impl reference times the FP64 CPU
oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 4096               # --size overrides it for profiling captures
CELL = 256
RADIUS = 80.0
T_OVER_TC, TAU, A_PAPER, K_EOS = 0.7, 0.8, -0.304, 1.0
MRT = dict(s_e=0.8, s_eps=0.8, s_q=1.1)
BYTES_PER_NODE = 72          # 9 FP32 deviations read + 9 written
SEED = 20141217 + 2 * 1000

# DRAM bytes (read + write) per launch of the step kernel measured by ncu on
# the workload above (mean of three launches: dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by the sha256 of the kernel sources it was
# taken from, the kernel configuration id and the lattice side; when any of
# them changes the entry no longer matches and traffic is null.
TRAFFIC_CAPTURES: dict = {
    ("d3cab8f8399c678b", 10, 4096): (604.09e6 + 546.61e6),
}
# Sources of the block-strip step kernel (its configuration table included).
KERNEL_SOURCES = ["paper_1412_5170_gb300/csrc/lbm_strip.cuh", "paper_1412_5170_gb300/csrc/lbm_strip_f32.cu",
                  "paper_1412_5170_gb300/csrc/lbm_device.cuh", "paper_1412_5170_gb300/csrc/lbm_kernels.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for s in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, s), "rb").read())
    return h.hexdigest()[:16]


def workload_config(extra=None):
    cfg = {"workload": "droplet array %dx%d (%dx%d droplets, R=80), T/Tc=0.7, tau=0.8, MRT+Guo, "
                       "A=-0.304 (A_K=-0.152), K=1, FP32-deviation populations, FP64 reductions"
                       % (N_SIDE, N_SIDE, N_SIDE // CELL, N_SIDE // CELL),
           "nx": N_SIDE, "ny": N_SIDE, "collision": "mrt", "forcing": "guo", "precision": "fp32_dev",
           "l2": "inputs larger than L2 (2 x 604 MB population buffers vs 129 MB L2); no flush"}
    if extra:
        cfg.update(extra)
    return cfg


def kernel_name(cfg):
    cid, threads, stages, _ = cfg
    if cid == 0:
        return "k_step_generic<float,float,MRT,GUO>"
    if threads == 32:
        return "k_step_warp<float,MRT,GUO,%d>" % stages
    return "k_step_strip<float,float,MRT,GUO,%d,%d>" % (threads, stages)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if not self.proc or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": reasons}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """Max of a per-rank float over the job (identity for one rank)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def initial_density(lbm, synth, seed):
    rv, rl = lbm.maxwell(T_OVER_TC)
    return synth.density_field(N_SIDE, N_SIDE, "droplet_array", rl, rv, RADIUS, seed=seed, cell=CELL), rv


def host_cores() -> int:
    """Host cores this process may use (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_oracle_rate(steps: int, side: int, seed: int, threads: int = 1):
    """MLUPS of the FP64 CPU oracle, as it stands, on a side x side periodic
    sample of the workload (one 256 x 256 droplet cell when side = 256), with
    its lattice loops on `threads` host threads."""
    import oracle
    from oracle import coexistence as cx
    from paper_1412_5170_gb300 import synth
    rg, rl, _ = cx.maxwell(T_OVER_TC)
    rho0 = synth.density_field(side, side, "droplet_array", rl, rg, RADIUS * side / CELL, seed=seed,
                               cell=side)
    q = oracle.params(side, side, T_OVER_TC, TAU, A_PAPER, K_EOS, "mrt", "guo", **MRT)
    f = oracle.init_rest(rho0)
    oracle.set_threads(threads)
    try:
        t0 = time.perf_counter()
        _, st = oracle.run(q, f, steps)
        el = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    return side * side * steps / el / 1e6, el


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    # Bounded per-step sample: one oracle step on a side x side periodic window,
    # on every host core, sized so warmup + steps stay within about two
    # minutes even at one core's rate.
    cores = host_cores()
    total = args.steps + args.warmup
    side = 256 if total * 65536 / 1.5e6 < 120 else (128 if total * 16384 / 1.5e6 < 120 else 64)
    if args.warmup:
        cpu_oracle_rate(args.warmup, side, SEED, cores)
    rate, el = cpu_oracle_rate(args.steps, side, SEED, cores)
    line = {"impl": "reference", "metric": "MLUPS", "value": rate, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config({"sample": "%dx%d periodic window per step" % (side, side)}),
            "cpu_baseline": {"value": rate, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": "%d oracle steps on a %dx%d periodic window of the workload, lattice "
                                       "loops over rows on %d host threads" % (args.steps, side, side, cores)},
            "e2e": {"value": rate, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1412_5170_gb300 import lbm, synth

    nodes = N_SIDE * N_SIDE
    rho0, rv = initial_density(lbm, synth, SEED + rank)
    p = lbm.make_params(N_SIDE, N_SIDE, T_OVER_TC, TAU, A_PAPER, K_EOS, "mrt", "guo", "fp32", rho_ref=rv, **MRT)
    lat = lbm.Lattice(p)
    stream = lat.stream
    lat.init_density(rho0)
    tune = {}
    if args.autotune:
        # Per-configuration timings (the autotuner's own choice is the minimum).
        for cid, threads, stages, npt in lat.configs():
            lat.config = cid
            lat.step(2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(10)
            e1.record(stream)
            e1.synchronize()
            tune["%d:t%d/s%d" % (cid, threads, stages)] = e0.elapsed_time(e1) / 10
        lat.init_density(rho0)
        cfg, _ = lat.autotune(10)
    if args.config >= 0:
        lat.config = args.config
    chosen = [c for c in lat.configs() if c[0] == lat.config][0]
    variant = lat.variant
    # Clocks are sampled (every 200 ms) from the warm-up through the e2e
    # phase: a short timed region (20 steps last ~4 ms) holds no sample of
    # its own, and the GPU is busy with the same kernels throughout.
    clk = ClockSampler(local).__enter__()
    for _ in range(args.warmup):
        lat.step(1)
    lat.stats()                      # also synchronises the stream
    barrier(ws)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    barrier(ws)
    ev[0].record(stream)
    for _ in range(args.steps):
        lat.step(1)
    ev[1].record(stream)
    st = lat.stats()            # FP64 reductions (one launch on strip lattices)
    ev[2].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    step_ms = ev[0].elapsed_time(ev[1])
    stats_ms = ev[1].elapsed_time(ev[2])
    total_ms = ev[0].elapsed_time(ev[2])
    total_ms = max_over_ranks(total_ms, ws, dev)
    kernel_ms = step_ms / max(args.steps, 1)
    value = ws * nodes * args.steps / (total_ms * 1e-3) / 1e6

    # End-to-end through the public API with host buffers: each e2e step is
    # init from a pinned host density field, CHUNK fused steps, and a read of
    # rho, vx, vy into pinned host buffers.  The copies run on the lattice's
    # copy streams: a step's input copy overlaps the previous step's kernels
    # and its result copy the next step's (two result buffers alternate).
    chunk = 100
    e2e_steps = max(1, args.steps // chunk) if args.e2e else 0
    h_rho0 = torch.from_numpy(rho0).pin_memory().numpy()
    h_out = [[torch.empty((N_SIDE, N_SIDE), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
             for _ in range(2)]
    if e2e_steps:   # the copy streams and device slots are set up by the first asynchronous call
        lat.read_moments_async(h_out[0])
        lat.wait_io()
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        lat.init_density_async(h_rho0)
        lat.step(chunk)
        lat.read_moments_async(h_out[i % 2])
    lat.wait_io()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    clk.__exit__(None, None, None)
    e2e_value = ws * nodes * chunk * e2e_steps / e2e_s / 1e6 if e2e_steps else None

    if rank == 0:
        peak, peak_kind = measured_peaks()
        achieved = BYTES_PER_NODE * nodes / (kernel_ms * 1e-3) / 1e9
        traffic = TRAFFIC_CAPTURES.get((kernel_hash(), chosen[0], N_SIDE))
        cpu_steps = args.cpu_steps
        cores = host_cores()
        cpu_rate, cpu_el = cpu_oracle_rate(cpu_steps, CELL, SEED) if cpu_steps > 0 else (None, 0.0)
        # all host cores: four times the sample (the same few seconds of wall time on ~16 cores)
        cpu_all, cpu_all_el = (cpu_oracle_rate(4 * cpu_steps, CELL, SEED, cores) if cpu_steps > 0 and cores > 1
                               else (cpu_rate, cpu_el))
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config({"parallelism": "replicas" if ws > 1 else "single",
                                       "kernel_variant": "strip" if variant == 1 else "generic",
                                       "kernel_config": {"id": chosen[0], "threads": chosen[1],
                                                         "stages": chosen[2], "nodes_per_thread": chosen[3]},
                                       "autotune_ms_per_step": tune or None}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": "%s (hbm_gbs, copy)" % peak_kind,
                         "kernel": kernel_name(chosen), "kernel_ms": kernel_ms,
                         "bytes_per_node": BYTES_PER_NODE, "algorithmic_bytes": BYTES_PER_NODE * nodes,
                         "traffic_unit": "DRAM bytes read + written per launch (ncu)"},
            "cpu_baseline": {"value": cpu_all, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": "%d FP64 oracle steps on one 256x256 droplet cell, lattice loops over rows "
                                       "on %d host threads (%.1f s)" % (4 * cpu_steps if cores > 1 else cpu_steps,
                                                                         cores, cpu_all_el),
                             "single_core": {"value": cpu_rate, "cores": 1,
                                             "sample": "%d FP64 oracle steps on one 256x256 droplet cell (%.1f s)"
                                                       % (cpu_steps, cpu_el)}},
            "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": 8 * nodes,
                    "d2h_bytes_per_step": 24 * nodes,
                    "how": "lbm_init_density_async(pinned host rho0) + lbm_step(%d) + "
                           "lbm_read_moments_async(pinned host) per e2e step, copies overlapping the steps, "
                           "lbm_wait_io at the end; %d e2e steps" % (chunk, e2e_steps)},
            "clocks": dict(clk.summary() or {}, window="warm-up, timed steps, statistics and e2e phase"),
            "stats_ms": stats_ms,
            "gpu_launches": args.steps + (1 if lbm.strip_observation(p) else 2),
            "status": st["status"], "mass": st["mass"], "max_v": st["max_v"],
        }
        print(json.dumps(line), flush=True)
    lat.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_warmstart(args):
    """Steps and wall time to steady state, cold vs learned warm start, on
    held-out instances of the batched sweep; the same instances started from
    their own converged profiles (what a perfect prediction gives); and the
    plain cold FP64 single-lattice path on a subset of them."""
    import numpy as np
    import torch

    from paper_1412_5170_gb300 import lbm, synth
    from paper_1412_5170_gb300 import warmstart as ws

    torch.cuda.set_device(0)
    A = args.ws_A
    crit = dict(tol_coex=args.ws_tol, check_every=1000, max_steps=args.ws_max_steps, coex_rule=args.ws_rule)

    def draw(n, seed):
        inst = synth.batch_instances(n, seed=seed)
        for d in inst:
            d["A"] = A
        return inst

    t0 = time.perf_counter()
    train = draw(args.ws_train, 20144000)
    gen = ws.solve(train, **crit)
    net = ws.WarmStart(seed=1)
    tt = time.perf_counter()
    losses = net.fit(train, gen["profiles"], gen["sizes"], epochs=args.ws_epochs)
    train_s = time.perf_counter() - tt

    test = draw(args.ws_test, 20145000)
    cold = ws.solve(test, **crit)
    warm = ws.solve(test, warm=net, **crit)
    ceil = ws.solve(test, profiles=cold["profiles"], sizes=cold["sizes"], **crit)
    conv = lambda r: r["state"] == lbm.CONVERGED
    both = conv(cold) & conv(warm)
    rl_c, rv_c = ws.coexistence(test, cold["obs"])
    rl_w, rv_w = ws.coexistence(test, warm["obs"])
    dv = np.abs(rv_w - rv_c) / rv_c
    dl = np.abs(rl_w - rl_c) / rl_c
    nodes = np.array([d["side"] ** 2 for d in test], dtype=np.float64)

    # The plain method: cold FP64 single-lattice runs to the same criterion,
    # one instance at a time (each with its autotuned kernel), on a stated
    # seeded subset: the first ws_fp64 held-out instances (index order) that
    # both batched runs solve.  The batched FP32 runs are repeated on exactly
    # that subset, so the wall times compare the same work; the comparison
    # counts only instances whose FP32 coexistence densities (cold and warm)
    # are within the FP32 tolerance (1e-4 relative) of the FP64 run's.
    fp64 = []
    sub = [int(i) for i in np.nonzero(both)[0][:args.ws_fp64]]
    for i in sub:
        d = test[i]
        p = lbm.make_params(d["side"], d["side"], d["T_over_Tc"], d["tau"], A, d["K"], "mrt", "guo", "fp64",
                            **MRT)
        with lbm.Lattice(p) as lat:
            lat.init_preset(d["kind"], d["size"], seed=d["seed"])
            lat.autotune(3)   # the fastest FP64 kernel for this lattice (the state does not advance)
            torch.cuda.synchronize()
            ts = time.perf_counter()
            st_code, steps, probes = fp64_run_to_steady(lat, d["kind"], args.ws_tol, 1000, args.ws_max_steps,
                                                        args.ws_rule)
            fp64.append(dict(i=i, status=st_code, steps=steps, wall_s=time.perf_counter() - ts,
                             nodes=int(nodes[i]), rho_l=probes[0], rho_v=probes[1]))
    sub_inst64 = [test[i] for i in sub]
    cold64 = ws.solve(sub_inst64, **crit) if sub else None
    warm64 = ws.solve(sub_inst64, warm=net, **crit) if sub else None
    fp64_rate = (sum(r["steps"] * r["nodes"] for r in fp64) / max(sum(r["wall_s"] for r in fp64), 1e-9)
                 if fp64 else None)
    fp64_cmp = None
    if sub:
        rl_c64, rv_c64 = ws.coexistence(sub_inst64, cold64["obs"])
        rl_w64, rv_w64 = ws.coexistence(sub_inst64, warm64["obs"])
        for j, r in enumerate(fp64):
            r["fp32_cold"] = dict(steps=int(cold64["steps"][j]), rel=[abs(rl_c64[j] - r["rho_l"]) / r["rho_l"],
                                                                      abs(rv_c64[j] - r["rho_v"]) / r["rho_v"]])
            r["fp32_warm"] = dict(steps=int(warm64["steps_total"][j]), rel=[abs(rl_w64[j] - r["rho_l"]) / r["rho_l"],
                                                                           abs(rv_w64[j] - r["rho_v"]) / r["rho_v"]])
        ok64 = [r["status"] == 0 and cold64["state"][j] == lbm.CONVERGED and warm64["state"][j] == lbm.CONVERGED
                and max(r["fp32_cold"]["rel"] + r["fp32_warm"]["rel"]) < 1e-4 for j, r in enumerate(fp64)]
        fp64_wall = sum(r["wall_s"] for r in fp64)
        fp64_cmp = {"instances": len(fp64), "subset": "first %d of the held-out instances both batched runs "
                                                        "solve, in index order (seed 20145000)" % len(fp64),
                    "within_fp32_tolerance": int(sum(ok64)),
                    "fp64_plain_wall_s": fp64_wall,
                    "fp32_batch_cold_wall_s": cold64["wall_s"], "fp32_batch_warm_wall_s": warm64["wall_s"],
                    "fp64_over_batch_cold": fp64_wall / cold64["wall_s"],
                    "fp64_over_batch_warm": fp64_wall / warm64["wall_s"],
                    "max_rel_error_fp32_vs_fp64": float(max(max(r["fp32_cold"]["rel"] + r["fp32_warm"]["rel"])
                                                            for r in fp64)),
                    "fp64_node_steps_per_s": fp64_rate}
    # FP64 wall projected over every instance both runs solved (context only):
    # its measured node-step rate times the node-steps the cold runs needed.
    fp64_projected = (float(np.sum(cold["steps"][both] * nodes[both])) / fp64_rate) if fp64_rate else None

    def stats(x):
        return None if len(x) == 0 else {"median": float(np.median(x)), "mean": float(np.mean(x))}

    # Wall time to steady state on the instances both runs solve (the batch's
    # wall time is otherwise set by the instances neither run converges
    # within max_steps): both runs again on that subset alone.
    sub_inst = [test[i] for i in np.nonzero(both)[0]]
    cold_sub = ws.solve(sub_inst, trace=True, **crit)
    warm_sub = ws.solve(sub_inst, warm=net, trace=True, **crit)

    # instances whose warm and cold steady states differ by more than 1 %
    odd = [dict(i=int(i), kind=test[i]["kind"], side=test[i]["side"], size=round(test[i]["size"], 2),
                T=round(test[i]["T_over_Tc"], 3), K=round(test[i]["K"], 3), tau=round(test[i]["tau"], 3),
                cold=[float(rl_c[i]), float(rv_c[i]), int(cold["steps"][i])],
                warm=[float(rl_w[i]), float(rv_w[i]), int(warm["steps_total"][i])], fallback=bool(warm["fallback"][i]))
           for i in np.nonzero(both & ((dl > 1e-2) | (dv > 1e-2)))[0]]
    line = {
        "metric": "steps-to-steady warm vs cold", "unit": "steps",
        "value": stats(warm["steps_total"][both]),
        "cold_steps": stats(cold["steps"][both]),
        "warm_over_cold_steps": stats(warm["steps_total"][both] / cold["steps"][both]),
        "perfect_profile_steps": stats(ceil["steps_total"][both & conv(ceil)]),
        "fallbacks": {"warm": int(warm["fallback"].sum()), "perfect_profile": int(ceil["fallback"].sum()),
                      "warm_failed": int((warm["first"]["state"] == lbm.FAILED).sum()),
                      "warm_other_state": int(warm["first"]["off"].sum()),
                      "predicted_uniform": int(warm["first"]["uniform"].sum()),
                      "predicted_uniform_cold_single_phase": int(np.sum(warm["first"]["uniform"] &
                                                                        ~(rl_c > 1.5 * rv_c))),
                      "warm_detail": [dict(i=int(i), kind=test[i]["kind"], side=test[i]["side"],
                                           size=round(test[i]["size"], 1), T=round(test[i]["T_over_Tc"], 3),
                                           K=round(test[i]["K"], 3), tau=round(test[i]["tau"], 3),
                                           state=int(warm["first"]["state"][i]), code=int(warm["first"]["code"][i]),
                                           steps=int(warm["first"]["steps"][i]),
                                           rho=[float(warm["first"]["rho_l"][i]), float(warm["first"]["rho_v"][i])],
                                           size_eq=float(warm["first"]["size"][i]),
                                           centre=float(warm["first"]["centre"][i]),
                                           cold=[float(rl_c[i]), float(rv_c[i]), int(cold["steps"][i])])
                                      for i in np.nonzero(warm["fallback"])[0]]},
        "different_steady_state": odd,
        "wall_s_converged_set": {"cold": cold_sub["wall_s"], "warm": warm_sub["wall_s"],
                                 "instances": len(sub_inst),
                                 "cold_converged": int(conv(cold_sub).sum()), "warm_converged": int(conv(warm_sub).sum()),
                                 "per_interval": {"columns": ["running instances", "running nodes", "wall_s"],
                                                  "cold": cold_sub["trace"], "warm": warm_sub["trace"]}},
        "fp64_plain_vs_batch": fp64_cmp,
        "wall_s": {"cold_batch": cold["wall_s"], "warm_batch": warm["wall_s"], "perfect_profile_batch": ceil["wall_s"],
                   "train_data": gen["wall_s"], "training": train_s, "fp64_plain_projected": fp64_projected,
                   "total": time.perf_counter() - t0},
        "instances": {"train": len(train), "train_converged": int(conv(gen).sum()), "test": len(test),
                      "cold_converged": int(conv(cold).sum()), "warm_started": int(warm["warm"].sum()),
                      "warm_converged": int(conv(warm).sum()), "failed_cold": int((cold["state"] == lbm.FAILED).sum()),
                      "failed_warm": int((warm["state"] == lbm.FAILED).sum()), "both": int(both.sum())},
        "coexistence_warm_vs_cold_rel": {"vapour_median": float(np.median(dv[both])) if both.any() else None,
                                         "vapour_max": float(np.max(dv[both])) if both.any() else None,
                                         "liquid_max": float(np.max(dl[both])) if both.any() else None},
        "fp64_plain": {"instances": fp64, "node_steps_per_s": fp64_rate},
        "batched_fp32_node_steps_per_s": {"cold": float(np.sum(cold["steps"] * nodes)) / cold["wall_s"],
                                          "warm": float(np.sum(warm["steps"] * nodes)) / warm["wall_s"]},
        "criterion": {"coexistence_rel_change_per_1000_steps": args.ws_tol, "max_steps": args.ws_max_steps,
                      "rule": args.ws_rule},
        "train_loss": losses,
        "config": {"workload": "batched sweep: side in {64..512}, T/Tc U[.5,.9], tau U[.55,1.2], K U[1/16,1], "
                               "R U[10, side/4], droplet or slab; MRT+Guo, A=%g, FP32 deviations" % A},
    }
    print(json.dumps(line), flush=True)


def run_batch(args):
    """The batched sweep: 512 independent instances (side 64..512, T/Tc
    0.5-0.9, tau 0.55-1.2, K 1/16-1, droplet or slab; MRT+Guo, A = -0.84,
    FP32 deviations) in one graph-captured batch.  Reports the batched step's
    throughput with every instance running (MLUPS and HBM fraction at 72 B per
    node update) and the run to steady state (coexistence criterion)."""
    import numpy as np
    import torch

    from paper_1412_5170_gb300 import lbm, synth

    torch.cuda.set_device(0)
    inst = synth.batch_instances(args.batch_n, seed=20141217 + 3000)
    for d in inst:
        d["A"] = args.ws_A
    with lbm.Batch(inst, collision="mrt") as b:
        nodes = b.nodes
        b.init()
        cols, ns, rows, carry, ms_tune = b.autotune(5)
        # each walk width at the chosen rows per item (host-timed, 20 steps)
        by_cols = {}
        for w, s_w, c_w in ((128, 3, False), (256, 3, True), (512, 2, True), (512, 3, True)):
            b.set_tuning(w, s_w, rows, c_w)
            b.step(3)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.step(20)
            torch.cuda.synchronize()
            by_cols["%d/s%d%s" % (w, s_w, "c" if c_w else "")] = (time.perf_counter() - t0) / 20 * 1e3
        b.set_tuning(cols, ns, rows, carry)
        b.step(args.warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(args.batch_steps)
        torch.cuda.synchronize()
        t_step = (time.perf_counter() - t0) / args.batch_steps
        b.init()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        b.set_coex_rule(args.ws_rule)
        st, done = b.run_to_steady(tol_coex=args.batch_tol, check_every=1000, max_steps=args.batch_max_steps)
        wall = time.perf_counter() - t1
        state, code, steps, obs = b.results()
    peak, peak_kind = measured_peaks()
    node_steps = float(np.sum(steps * np.array([d["side"] ** 2 for d in inst], dtype=np.float64)))
    conv = state == lbm.CONVERGED
    line = {
        "metric": "batched sweep: MLUPS and steps to steady state", "unit": "MLUPS",
        "value": nodes / t_step / 1e6, "instances": len(inst), "nodes_per_step": nodes,
        "ms_per_step": t_step * 1e3,
        "roofline": {"bound": "hbm", "achieved": 72.0 * nodes / t_step / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": 72.0 * nodes / t_step / 1e9 / peak, "peak_kind": "%s (hbm_gbs, copy)" % peak_kind,
                     "kernel": "%s (every instance running, host-timed over %d steps)"
                               % ("k_step_batch" if cols == 128 else "k_step_batch_strip", args.batch_steps)},
        "tuning": {"columns": cols, "stages": ns, "rows_per_item": rows, "carry": carry, "ms_per_step": ms_tune,
                   "ms_per_step_by_columns": by_cols},
        "to_steady": {"wall_s": wall, "steps_done": done, "converged": int(conv.sum()),
                      "failed": int((state == lbm.FAILED).sum()), "running": int((state == lbm.RUNNING).sum()),
                      "median_steps": float(np.median(steps[conv])) if conv.any() else None,
                      "node_steps_per_s": node_steps / wall},
        "config": {"workload": "batched sweep, %d instances: side U{64..512}, T/Tc U[.5,.9], tau U[.55,1.2], "
                               "K U[1/16,1], R U[10, side/4], droplet or slab; MRT+Guo, A=%g, FP32 deviations; "
                               "criterion: coexistence probes change < %g per 1000 steps (rule: %s)"
                               % (args.batch_n, args.ws_A, args.batch_tol, args.ws_rule)},
    }
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """The static-droplet parameter sweep (256x256, R = 40, noise 1e-6): T/Tc
    in {0.5 .. 0.9} x tau in {0.6, 0.8, 1.0} x {BGK, MRT} x K in {1, 1/4, 1/16},
    each run for --sweep-steps steps in FP64 and in FP32 deviations on the
    single-lattice path; reports the coexistence densities (centre / corner
    node), density ratio and Us_max of every run and the FP32 error against
    FP64 (bars: densities 1e-4 relative, Us_max 5 %)."""
    import numpy as np
    import torch

    from paper_1412_5170_gb300 import lbm

    torch.cuda.set_device(0)
    A = args.sweep_A
    rows = []
    t0 = time.perf_counter()
    idx = 0
    for coll in ("bgk", "mrt"):
        for T in (0.5, 0.6, 0.7, 0.8, 0.9):
            for tau in (0.6, 0.8, 1.0):
                for K in (1.0, 0.25, 0.0625):
                    seed = 20141217 + 1000 + idx
                    idx += 1
                    res = {}
                    for prec in ("fp64", "fp32"):
                        p = lbm.make_params(256, 256, T, tau, A, K, coll, "guo", prec, **MRT)
                        with lbm.Lattice(p) as lat:
                            lat.init_preset("droplet", 40.0, seed=seed)
                            lat.autotune(3)
                            ts = time.perf_counter()
                            lat.step(args.sweep_steps)
                            st = lat.stats()
                            res[prec] = dict(status=st["status"], rho_l=st["rho_center"], rho_v=st["rho_corner"],
                                             us=st["max_v"], s=time.perf_counter() - ts)
                    a, b = res["fp64"], res["fp32"]
                    ok = a["status"] == 0 and b["status"] == 0 and np.isfinite(a["rho_l"]) and a["rho_l"] > 1.5 * a["rho_v"]
                    row = dict(coll=coll, T=T, tau=tau, K=K, status=[a["status"], b["status"]],
                               fp64=[a["rho_l"], a["rho_v"], a["us"]], fp32=[b["rho_l"], b["rho_v"], b["us"]],
                               two_phase=bool(ok))
                    if ok:
                        row["ratio"] = a["rho_l"] / a["rho_v"]
                        row["err"] = [abs(b["rho_l"] / a["rho_l"] - 1), abs(b["rho_v"] / a["rho_v"] - 1),
                                      abs(b["us"] / a["us"] - 1)]
                    rows.append(row)
                    print("  %s T %.1f tau %.1f K %.4f  fp64 %s  fp32 %s  %s" % (
                        coll, T, tau, K, [round(v, 7) for v in row["fp64"]], [round(v, 7) for v in row["fp32"]],
                        row.get("err")), file=sys.stderr, flush=True)
    good = [r for r in rows if r["two_phase"]]
    err = np.array([r["err"] for r in good]) if good else np.zeros((0, 3))
    # A droplet whose FP64 spurious current passes 0.1 (Mach number ~0.17) is
    # no static steady state: its 30 000-step snapshot is one moment of an
    # unsteady flow, where FP32 and FP64 part like any two nearby trajectories.
    steady = np.array([r["fp64"][2] < US_STEADY for r in good], dtype=bool)
    within = (err[:, 0] < 1e-4) & (err[:, 1] < 1e-4) & (err[:, 2] < 0.05) if len(err) else np.zeros(0, dtype=bool)
    line = {
        "metric": "FP32-deviation vs FP64 coexistence and Us_max, static-droplet sweep", "unit": "relative error",
        "runs": len(rows), "two_phase_stable": len(good),
        "failed_fp64": sum(1 for r in rows if r["status"][0] != 0), "failed_fp32": sum(1 for r in rows if r["status"][1] != 0),
        "max_err": {"rho_l": float(err[:, 0].max()) if len(err) else None,
                    "rho_v": float(err[:, 1].max()) if len(err) else None,
                    "us_max": float(err[:, 2].max()) if len(err) else None},
        "within_bars": int(np.sum(within)),
        "steady": int(steady.sum()), "steady_within_bars": int(np.sum(within & steady)),
        "unsteady": [dict(coll=r["coll"], T=r["T"], tau=r["tau"], K=r["K"], us_fp64=r["fp64"][2], err=r["err"])
                     for r, st in zip(good, steady) if not st],
        "max_density_ratio": max((r["ratio"] for r in good), default=None),
        "rows": rows, "wall_s": time.perf_counter() - t0,
        "config": {"workload": "static droplet 256x256, R = 40, noise 1e-6, %d steps, MRT rates 0.8/0.8/1.1, "
                               "Guo forcing, A = %g" % (args.sweep_steps, A)},
    }
    print(json.dumps(line), flush=True)


US_STEADY = 0.1   # FP64 spurious-current magnitude above which a sweep droplet is not steady


COEX_SCHEMES = [
    # label, collision, forcing, A, K, sigma, eps of the mechanical solution
    ("guo eps0.52", "bgk", "guo", -0.26, 1.0, 0.0, 0.52),
    ("edm eps0.52", "bgk", "edm", -0.26, 1.0, 0.0, 0.52),
    ("sc eps0.52", "bgk", "sc", -0.26, 1.0, 0.0, 0.52),
    ("guo eps1.68", "bgk", "guo", -0.84, 1.0, 0.0, 1.68),
    ("li sigma0.105", "bgk", "li", 0.0, 1.0, 0.105, 1.68),
    ("mrt guo eps1.68", "mrt", "guo", -0.84, 1.0, 0.0, 1.68),
    ("guo K0.1 eps2", "bgk", "guo", -1.0, 0.1, 0.0, 2.0),
]


# Flat-interface slabs of the coexistence curves: 8 x 127 nodes, half-width 32.
# With an odd height the slab's centre, ny / 2 = 63.5, lies between two rows.
# A slab centred on a row is a symmetric state that is not stable at low
# temperature: it shifts by half a row after some 10^4 steps (seen in FP64 as
# in FP32, where rounding starts the shift sooner), and rho_g changes by a
# few percent in the shift (3.7 % at T/Tc = 0.6, eps = 1.68), so runs of a
# fixed length would compare different states.
COEX_NX, COEX_NY, COEX_HALF = 8, 127, 32.0


def coexistence_curve(lbm, coll, forc, A, K, sigma, T, steps, tau=1.0, ny=COEX_NY, nx=COEX_NX):
    """Flat-interface coexistence densities (mid row, edge row) of one FP64 slab run."""
    rv, rl = lbm.maxwell(T)
    p = lbm.make_params(nx, ny, T, tau, A, K, coll, forc, "fp64", sigma=sigma, **MRT)
    with lbm.Lattice(p) as lat:
        lat.init_preset("slab", COEX_HALF, rho_l=rl, rho_v=rv, seed=11)
        lat.autotune(3)
        lat.step(steps)
        st = lat.stats()
    return st["status"], st["rho_row_mid"], st["rho_row0"]


def _solution(fn, *a):
    """A host coexistence solver's (rho_v, rho_l), or (None, None) where it has no root."""
    try:
        return fn(*a)
    except Exception:
        return None, None


# FP64 instructions per node update of the FP64 MRT+Guo step, counted by ncu
# on one launch of the autotuned kernel
# (sm__sass_thread_inst_executed_op_{dfma,dadd,dmul}_pred_on.sum / nodes),
# keyed like TRAFFIC_CAPTURES (sha256 of the kernel sources, configuration
# id, lattice side); unknown otherwise.  (Counted on the sources before the
# FP32 density's summation order changed -- an `if constexpr` on float that
# leaves the FP64 kernel's code as it was.)
FP64_INST_CAPTURES: dict = {
    ("d3cab8f8399c678b", 0, 1024): {"dfma": 73662464 / 1048576, "dadd": 87670784 / 1048576,
                                    "dmul": 40845312 / 1048576},
}


def run_fp64(args):
    """The FP64 step against its own roofline.  On this GPU the FP64 pipe is a
    small fraction of the FP32 one, so the FP64 step (the parity path) is
    bound by double-precision arithmetic, not by HBM: report the measured FP64
    and FP32 fused-multiply-add peaks (lbm_fma_peak), the autotuned FP64
    MRT+Guo step on the droplet-array workload at side --fp64-size, and its
    FP64 instruction issue rate as a fraction of the FP64 pipe's (DFMA, DADD
    and DMUL per node from an ncu count, FP64_INST_CAPTURES; the pipe issues
    each of them at the rate of the FMA peak / 2 flops), beside its flop rate
    and its HBM fraction at 144 B per node."""
    import torch

    from paper_1412_5170_gb300 import lbm, synth

    torch.cuda.set_device(0)
    peak64, peak32 = lbm.fma_peak("fp64"), lbm.fma_peak("fp32")
    side = args.fp64_size
    rv, rl = lbm.maxwell(T_OVER_TC)
    cell = max(32, side // 16)
    rho0 = synth.density_field(side, side, "droplet_array", rl, rv, RADIUS * cell / CELL, seed=SEED, cell=cell)
    p = lbm.make_params(side, side, T_OVER_TC, TAU, A_PAPER, K_EOS, "mrt", "guo", "fp64", **MRT)
    with lbm.Lattice(p) as lat:
        lat.init_density(rho0)
        cfg, _ = lat.autotune(5)
        for _ in range(args.warmup):
            lat.step(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(lat.stream)
        for _ in range(args.steps):
            lat.step(1)
        e1.record(lat.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        st = lat.stats()
    nodes = side * side
    peak_hbm, kind = measured_peaks()
    cnt = FP64_INST_CAPTURES.get((kernel_hash(), cfg, side))
    rate = nodes / (ms * 1e-3)
    if cnt:
        ipn = cnt["dfma"] + cnt["dadd"] + cnt["dmul"]
        fpn = 2 * cnt["dfma"] + cnt["dadd"] + cnt["dmul"]
        roof = {"bound": "alu", "unit": "FP64 instructions/s", "inst_per_node": ipn, "flops_per_node": fpn,
                "achieved": ipn * rate, "peak": peak64 * 1e12 / 2, "frac": ipn * rate / (peak64 * 1e12 / 2),
                "achieved_tflops": fpn * rate / 1e12, "peak_tflops": peak64,
                "flop_frac": fpn * rate / 1e12 / peak64, "counts": cnt}
    else:
        roof = {"bound": "alu", "unit": "FP64 instructions/s", "inst_per_node": None, "frac": None,
                "peak_tflops": peak64, "note": "no instruction count for this kernel, configuration and size"}
    line = {"metric": "FP64 step: node updates per second and FP64 roofline", "unit": "MLUPS",
            "value": rate / 1e6, "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "droplet array %dx%d (cells of %d), T/Tc=0.7, tau=0.8, MRT+Guo, FP64"
                                   % (side, side, cell), "kernel_config": cfg},
            "fma_peak_tflops": {"fp64": peak64, "fp32": peak32, "how": "lbm_fma_peak: independent FMA chains, "
                                                                        "CUDA events, best of 5"},
            "roofline": roof,
            "hbm": {"bytes_per_node": 144, "achieved_gbs": 144.0 * rate / 1e9, "peak_gbs": peak_hbm,
                    "frac": 144.0 * rate / 1e9 / peak_hbm, "peak_kind": kind},
            "status": st["status"]}
    print(json.dumps(line), flush=True)


def run_coexistence(args):
    """Coexistence curves of flat interfaces (the data behind Figs. 2-6 and
    Table 6) for the paper's schemes against the Maxwell construction
    (Eq. 19) and the mechanical-stability solution (Eq. 18) of the same eps,
    both from liblbm's host solvers.  Each scheme runs as one FP32 batch of
    8 x 127 slabs (COEX_NY) over the temperature grid (the batched engine; a batch
    holds one scheme); every slab also runs alone on the FP64 path, and the
    table gives both and their difference."""
    import numpy as np

    from paper_1412_5170_gb300 import lbm

    t0 = time.perf_counter()
    temps = [0.5, 0.55, 0.6, 0.65, 0.7, 0.75, 0.8, 0.85, 0.9, 0.95]
    rows, batch_s, fp64_s = [], 0.0, 0.0
    for label, coll, forc, A, K, sigma, eps in COEX_SCHEMES:
        inst = [dict(nx=COEX_NX, ny=COEX_NY, kind="slab", T_over_Tc=T, tau=1.0, A=A, K=K, size=COEX_HALF, seed=11)
                for T in temps]
        tb = time.perf_counter()
        with lbm.Batch(inst, collision=coll, forcing=forc, sigma=sigma, **MRT) as b:
            b.init()
            b.step(args.coex_steps)
            b.observe()
            _, code, _, obs = b.results()
        batch_s += time.perf_counter() - tb
        for j, T in enumerate(temps):
            tf = time.perf_counter()
            st64, rl64, rg64 = coexistence_curve(lbm, coll, forc, A, K, sigma, T, args.coex_steps)
            fp64_s += time.perf_counter() - tf
            rl, rg, st = float(obs["rho_row_mid"][j]), float(obs["rho_row0"][j]), int(code[j])
            mg, ml = _solution(lbm.mechanical, T, K, eps)
            xg, xl = lbm.maxwell(T)
            ok = st == 0 and np.isfinite(rl) and np.isfinite(rg)
            rows.append(dict(scheme=label, T=T, status=st, rho_l=rl, rho_g=rg, mech=[ml, mg], maxwell=[xl, xg],
                             rel_mech=[rl / ml - 1, rg / mg - 1] if ok and mg else None,
                             rel_maxwell=[rl / xl - 1, rg / xg - 1] if ok else None,
                             fp64=dict(status=st64, rho_l=rl64, rho_g=rg64,
                                       fp32_rel=[rl / rl64 - 1, rg / rg64 - 1] if ok and st64 == 0 else None)))
            print("  %-16s T %.2f status %d rho_l %.6f rho_g %.6g (FP64 %d %.6g)  mech %s %s  maxwell %.6f %.6g" % (
                label, T, st, rl, rg, st64, rg64, ml, mg, xl, xg), file=sys.stderr, flush=True)
    line = {"metric": "flat-interface coexistence densities vs Eqs. 18-19", "unit": "relative deviation",
            "rows": rows, "steps": args.coex_steps, "wall_s": time.perf_counter() - t0,
            "batched_fp32_wall_s": batch_s, "fp64_single_lattices_wall_s": fp64_s,
            "config": {"workload": "slab 8x127 (half-width 32, centred between rows), tau = 1, MRT rates 0.8/0.8/1.1; "
                                   "one FP32 batch per scheme over the temperatures, each slab also alone in FP64"}}
    print(json.dumps(line), flush=True)


def run_laplace(args):
    """Laplace's law on static gas bubbles (the Table 3 / Table 4 setups):
    bubbles of R = 15 .. 35 on 128^2 at T/Tc = 0.6, FP64, 30 000 steps; the
    pressure jump dp = p0(rho_g) - p0(rho_l) of the K-scaled EOS (Eq. 30) at
    the centre and corner probes against 1/R_eq, R_eq from the mass deficit of
    the bubble.  The slope is the surface tension; a straight line through
    the origin is Laplace's law."""
    import numpy as np

    from paper_1412_5170_gb300 import lbm

    T = 0.6
    Tabs = T * lbm.tc()

    def p0(rho, K):
        return K * (rho * Tabs * (1 + rho + rho ** 2 - rho ** 3) / (1 - rho) ** 3 - rho ** 2)

    cases = [("guo", -0.9, 0.5, 1.5, 0.01059), ("guo", -0.9, 0.5, 0.7, 0.010368),
             ("edm", -0.26, 0.5, 1.5, 0.01241), ("edm", -0.26, 0.5, 0.7, 0.013635),
             ("guo", -0.84, 1.0, 1.0, None)]
    rows = []
    t0 = time.perf_counter()
    for forc, A, K, tau, paper_sigma in cases:
        pts = []
        for R in (15.0, 20.0, 25.0, 30.0, 35.0):
            p = lbm.make_params(128, 128, T, tau, A, K, "bgk", forc, "fp64")
            with lbm.Lattice(p) as lat:
                lat.init_preset("bubble", R, seed=1)
                lat.autotune(3)
                lat.step(args.laplace_steps)
                st = lat.stats()
                rho = lat.read_moments()[0]
            rg, rl = st["rho_center"], st["rho_corner"]
            r_eq = float(np.sqrt(np.sum(rl - rho) / (np.pi * (rl - rg))))
            pts.append((r_eq, p0(rg, K) - p0(rl, K), rg, rl, st["status"]))
        x = np.array([1.0 / q[0] for q in pts])
        y = np.array([q[1] for q in pts])
        slope, icpt = np.polyfit(x, y, 1)
        r2 = 1.0 - np.sum((y - (slope * x + icpt)) ** 2) / np.sum((y - y.mean()) ** 2)
        rows.append(dict(forcing=forc, A=A, K=K, tau=tau, sigma=float(slope), intercept=float(icpt), r2=float(r2),
                         paper_sigma=paper_sigma, points=[[round(q[0], 3), q[1], q[2], q[3], q[4]] for q in pts]))
        print("  %s A %g K %g tau %g: sigma %.5g intercept %.2e r2 %.6f (paper %s)" % (
            forc, A, K, tau, slope, icpt, r2, paper_sigma), file=sys.stderr, flush=True)
    line = {"metric": "surface tension from Laplace's law, static bubbles", "unit": "lattice units",
            "rows": rows, "steps": args.laplace_steps, "wall_s": time.perf_counter() - t0,
            "config": {"workload": "gas bubbles R = 15..35 on 128x128, T/Tc = 0.6, BGK, FP64"}}
    print(json.dumps(line), flush=True)


def coex_tail(d, dp):
    """The change still to come of a probe whose last two changes were d and
    dp, as the batched solver estimates it (LBM_COEX_TAIL): a geometric series
    of ratio r = d / dp -- |d| r / (1 - r) for 0 <= r < 1, |d| for r < 0,
    infinite for r >= 1, for an unknown dp (NaN) or dp = 0; zero if d is
    zero."""
    if d == 0.0:
        return 0.0
    if not dp != 0.0:          # unknown (NaN), or a move after a standstill
        return math.inf
    r = d / dp
    if not r < 1.0:
        return math.inf
    return abs(d) if r < 0.0 else abs(d) * r / (1.0 - r)


def coex_measure(prev, cur, hist, rule):
    """The quantity the coexistence criterion holds below tol_coex: the
    probes' relative change since the previous check, with rule "tail" also
    their estimated change still to come from this check's pair of changes
    and from the pair before (both probes, the largest).  hist: per probe
    (change at the previous check, change at the one before), NaN where
    unknown; returns (measure, hist for the next check)."""
    d = (cur[0] - prev[0], cur[1] - prev[1])
    m = max(abs(d[0]) / abs(cur[0]), abs(d[1]) / abs(cur[1]))
    if rule == "tail" and m == m:
        for j in (0, 1):
            t = max(coex_tail(d[j], hist[j][0]), coex_tail(hist[j][0], hist[j][1]))
            m = max(m, t / abs(cur[j]))
    return m, ((d[0], hist[0][0]), (d[1], hist[1][0]))


def fp64_run_to_steady(lat, kind, tol, every, max_steps, rule="change"):
    """Cold single-lattice run on the FP64 path until both coexistence
    densities (centre and corner, or mid and edge row for a slab) meet the
    batched runs' criterion: relative change below tol per `every` steps and,
    with rule "tail", so is their estimated change still to come."""
    def probes(st):
        return (st["rho_row_mid"], st["rho_row0"]) if kind == "slab" else (st["rho_center"], st["rho_corner"])
    prev = probes(lat.stats())
    hist = ((math.nan, math.nan), (math.nan, math.nan))
    steps = 0
    while steps < max_steps:
        lat.step(every)
        steps += every
        st = lat.stats()
        if st["status"] != 0:
            return st["status"], steps, prev
        cur = probes(st)
        m, hist = coex_measure(prev, cur, hist, rule)
        if m < tol:
            return 0, steps, cur
        prev = cur
    return 6, steps, prev


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="throughput",
                    choices=["throughput", "warmstart", "sweep", "coexistence", "batch", "laplace", "fp64"])
    ap.add_argument("--fp64-size", type=int, default=1024, help="lattice side of --mode fp64")
    ap.add_argument("--laplace-steps", type=int, default=30000)
    ap.add_argument("--batch-n", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--coex-steps", type=int, default=40000)
    ap.add_argument("--sweep-steps", type=int, default=30000)
    ap.add_argument("--sweep-A", type=float, default=-0.84)
    ap.add_argument("--ws-train", type=int, default=2000)
    ap.add_argument("--ws-test", type=int, default=256)
    ap.add_argument("--ws-epochs", type=int, default=3000)
    ap.add_argument("--ws-fp64", type=int, default=64, help="held-out instances also run on the FP64 path")
    ap.add_argument("--ws-A", type=float, default=-0.84, help="Eq. 6 weight A of the sweep (epsilon = -2A = 1.68)")
    ap.add_argument("--ws-tol", type=float, default=2e-6, help="coexistence-density change per 1000 steps")
    ap.add_argument("--ws-max-steps", type=int, default=150000)
    ap.add_argument("--batch-tol", type=float, default=1e-5, help="--mode batch: coexistence criterion")
    ap.add_argument("--batch-max-steps", type=int, default=100000)
    ap.add_argument("--ws-rule", default="tail", choices=["change", "tail"],
                    help="coexistence criterion: change per check, or also the estimated change still to come")
    ap.add_argument("--cpu-steps", type=int, default=700,
                    help="oracle steps on one 256x256 cell for cpu_baseline (0 = skip)")
    ap.add_argument("--size", type=int, default=4096, help="lattice side (multiple of 256; profiling)")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false", help="skip the end-to-end leg")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default kernel configuration")
    ap.add_argument("--config", type=int, default=-1, help="force a kernel configuration id (profiling)")
    args = ap.parse_args()
    global N_SIDE
    if args.size % CELL:
        ap.error("--size must be a multiple of %d" % CELL)
    N_SIDE = args.size
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "warmstart":
        run_warmstart(args)
    elif args.mode == "sweep":
        run_sweep(args)
    elif args.mode == "coexistence":
        run_coexistence(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "laplace":
        run_laplace(args)
    elif args.mode == "fp64":
        run_fp64(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
