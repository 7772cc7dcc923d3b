"""Thin ctypes binding of liblbm (include/lbm.h), same names as the C ABI.

Only argument marshalling happens here: every step of the lattice update runs
in the CUDA kernels of ``liblbm.so``.  PyTorch supplies device memory (the
context workspace) and the CUDA stream.  Importing this module fails if the
library has not been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("liblbm.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)

OK, E_INVALID, E_CUDA, E_NONFINITE, E_EOS_DOMAIN, E_TIMEOUT, E_NOT_CONVERGED, E_IO, E_UNSUPPORTED = range(9)
BGK, MRT = 0, 1
GUO, EDM, SC, LI = 0, 1, 2, 3
FP64, FP32_DEV = 0, 1
SLAB, DROPLET, BUBBLE, DROPLET_ARRAY = 0, 1, 2, 3
COLLISION = {"bgk": BGK, "mrt": MRT}
FORCING = {"guo": GUO, "edm": EDM, "sc": SC, "li": LI}
PRECISION = {"fp64": FP64, "fp32": FP32_DEV}
PRESET = {"slab": SLAB, "droplet": DROPLET, "bubble": BUBBLE, "droplet_array": DROPLET_ARRAY}


class lbm_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("collision", ctypes.c_int32),
                ("forcing", ctypes.c_int32), ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("T_over_Tc", ctypes.c_double), ("tau", ctypes.c_double), ("A", ctypes.c_double),
                ("K", ctypes.c_double), ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double),
                ("s_q", ctypes.c_double), ("rho_ref", ctypes.c_double), ("sigma", ctypes.c_double)]


class lbm_stats_t(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("max_v", ctypes.c_double), ("max_dv", ctypes.c_double),
                ("rho_min", ctypes.c_double), ("rho_max", ctypes.c_double), ("rho_center", ctypes.c_double),
                ("rho_corner", ctypes.c_double), ("rho_row_mid", ctypes.c_double),
                ("rho_row0", ctypes.c_double), ("steps", ctypes.c_int64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class lbm_batch_params(ctypes.Structure):
    _fields_ = [("collision", ctypes.c_int32), ("forcing", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double),
                ("s_q", ctypes.c_double), ("sigma", ctypes.c_double)]


class lbm_profile_geom(ctypes.Structure):
    _fields_ = [("use", ctypes.c_int32), ("reserved", ctypes.c_int32), ("centre", ctypes.c_double),
                ("spacing", ctypes.c_double)]


class lbm_instance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("kind", ctypes.c_int32), ("cell", ctypes.c_int32),
                ("T_over_Tc", ctypes.c_double), ("tau", ctypes.c_double), ("A", ctypes.c_double),
                ("K", ctypes.c_double), ("size", ctypes.c_double), ("width", ctypes.c_double),
                ("rho_l", ctypes.c_double), ("rho_v", ctypes.c_double), ("noise_amp", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class lbm_ws_cfg(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("n_hidden", ctypes.c_int32), ("hidden_layers", ctypes.c_int32),
                ("n_out", ctypes.c_int32), ("seed", ctypes.c_uint64)]


BATCH_NOBS = 10
BATCH_OBS = ("mass", "max_v", "max_dv", "max_drho", "rho_min", "rho_max", "rho_center", "rho_corner",
             "rho_row_mid", "rho_row0")
RUNNING, CONVERGED, FAILED = 0, 1, 2
LBM_INIT_REST = 1
COEX_RULES = {"change": 0, "tail": 1}   # LBM_COEX_CHANGE, LBM_COEX_TAIL

_vp, _dp, _i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
_PROTOS = {
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_version": (ctypes.c_int, []),
    "lbm_tc": (ctypes.c_double, []),
    "lbm_mechanical": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]),
    "lbm_fma_peak": (ctypes.c_int, [ctypes.c_int, _dp]),
    "lbm_maxwell": (ctypes.c_int, [ctypes.c_double, _dp, _dp]),
    "lbm_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(lbm_params), ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(lbm_params), _vp, _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "lbm_destroy": (None, [_vp]),
    "lbm_init_density": (ctypes.c_int, [_vp, _vp]),
    "lbm_init_density_dev": (ctypes.c_int, [_vp, _vp]),
    "lbm_init_preset": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double]),
    "lbm_step": (ctypes.c_int, [_vp, _i64]),
    "lbm_stats": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(lbm_stats_t)]),
    "lbm_run_to_steady": (ctypes.c_int, [_vp, ctypes.c_double, _i64, _i64, ctypes.POINTER(_i64)]),
    "lbm_read_moments": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_init_density_async": (ctypes.c_int, [_vp, _vp]),
    "lbm_read_moments_async": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_wait_io": (ctypes.c_int, [_vp]),
    "lbm_read_populations": (ctypes.c_int, [_vp, _vp]),
    "lbm_write_populations": (ctypes.c_int, [_vp, _vp]),
    "lbm_copy_rows": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int]),
    "lbm_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "lbm_load": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "lbm_inject_stage_timeout": (ctypes.c_int, [_vp]),
    "lbm_get_variant": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "lbm_set_variant": (ctypes.c_int, [_vp, ctypes.c_int]),
    "lbm_config_count": (ctypes.c_int, [ctypes.POINTER(lbm_params), ctypes.POINTER(ctypes.c_int)]),
    "lbm_config_describe": (ctypes.c_int, [ctypes.POINTER(lbm_params), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lbm_get_config": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "lbm_set_config": (ctypes.c_int, [_vp, ctypes.c_int]),
    "lbm_autotune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.POINTER(lbm_batch_params), ctypes.POINTER(lbm_instance), ctypes.c_int,
                                        ctypes.POINTER(_vp)]),
    "lbm_batch_destroy": (None, [_vp]),
    "lbm_batch_init": (ctypes.c_int, [_vp]),
    "lbm_batch_init_profiles": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int]),
    "lbm_batch_step": (ctypes.c_int, [_vp, _i64]),
    "lbm_batch_run_to_steady": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _i64, _i64,
                                               ctypes.POINTER(_i64)]),
    "lbm_batch_observe": (ctypes.c_int, [_vp]),
    "lbm_batch_results": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lbm_batch_read_density": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "lbm_batch_profiles": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "lbm_batch_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lbm_batch_set_coex_rule": (ctypes.c_int, [_vp, ctypes.c_int]),
    "lbm_batch_autotune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp]),
    "lbm_batch_nodes": (ctypes.c_int64, [_vp]),
    "lbm_ws_create": (ctypes.c_int, [ctypes.POINTER(lbm_ws_cfg), ctypes.POINTER(_vp)]),
    "lbm_ws_destroy": (None, [_vp]),
    "lbm_ws_num_params": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "lbm_ws_set_scaling": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lbm_ws_get_params": (ctypes.c_int, [_vp, _vp]),
    "lbm_ws_set_params": (ctypes.c_int, [_vp, _vp]),
    "lbm_ws_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float), _vp]),
    "lbm_ws_train": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                    ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)]),
    "lbm_ws_predict": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "lbm_stats_noalloc": (ctypes.c_int, [ctypes.POINTER(lbm_params), _vp, _vp, ctypes.POINTER(lbm_stats_t)]),
}
for _name, (_res, _args) in _PROTOS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class LbmError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, lbm_strerror(status).decode(), status))


def check(status, what=""):
    if status != OK:
        raise LbmError(status, what)
    return status


def strip_observation(p: lbm_params) -> bool:
    """Whether lbm_stats observes p's lattice with the strip walk (one launch,
    reduction included): the lattices the strip kernel takes, nx % 4 == 0."""
    return p.nx >= 4 and p.nx % 4 == 0


def fma_peak(precision: str = "fp64") -> float:
    """Measured FMA throughput of the current GPU (TFLOP/s) in FP64 or FP32."""
    t = ctypes.c_double()
    check(lbm_fma_peak(PRECISION[precision], ctypes.byref(t)), "lbm_fma_peak")
    return t.value


def tc() -> float:
    return lbm_tc()


def maxwell(T_over_Tc: float):
    """(rho_v, rho_l) of the Maxwell construction (Eq. 19), host FP64."""
    rv, rl = ctypes.c_double(), ctypes.c_double()
    check(lbm_maxwell(float(T_over_Tc), ctypes.byref(rv), ctypes.byref(rl)), "lbm_maxwell")
    return rv.value, rl.value


def mechanical(T_over_Tc: float, K: float, eps: float):
    """(rho_v, rho_l) of the mechanical-stability condition (Eq. 18)."""
    rv, rl = ctypes.c_double(), ctypes.c_double()
    check(lbm_mechanical(float(T_over_Tc), float(K), float(eps), ctypes.byref(rv), ctypes.byref(rl)), "lbm_mechanical")
    return rv.value, rl.value


def make_params(nx, ny, T_over_Tc, tau, A, K=1.0, collision="bgk", forcing="guo", precision="fp64",
                s_e=1.0, s_eps=1.0, s_q=1.0, rho_ref=None, sigma=0.0) -> lbm_params:
    if rho_ref is None:
        rho_ref = maxwell(T_over_Tc)[0] if precision == "fp32" else 0.0
    return lbm_params(int(nx), int(ny), COLLISION[collision], FORCING[forcing], PRECISION[precision], 0,
                      float(T_over_Tc), float(tau), float(A), float(K), float(s_e), float(s_eps), float(s_q),
                      float(rho_ref), float(sigma))


def _host_ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_vp)


class Lattice:
    """One periodic lattice on the current CUDA device.

    The device workspace is a torch uint8 tensor and work runs on a torch
    stream (its handle is passed to lbm_create); all arithmetic is in liblbm."""

    def __init__(self, params: lbm_params, stream=None, torch_workspace: bool = True):
        import torch
        self.p = params
        self.stream = stream if stream is not None else torch.cuda.Stream()
        nbytes = ctypes.c_size_t()
        check(lbm_workspace_bytes(ctypes.byref(params), ctypes.byref(nbytes)), "lbm_workspace_bytes")
        self.workspace_bytes = nbytes.value
        self._ws = None
        ws_ptr = None
        if torch_workspace:
            self._ws = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
            ws_ptr = self._ws.data_ptr()
        ctx = _vp()
        check(lbm_create(ctypes.byref(params), _vp(self.stream.cuda_stream), _vp(ws_ptr) if ws_ptr else None,
                         nbytes.value, ctypes.byref(ctx)), "lbm_create")
        self.ctx = ctx
        self._io_refs = []   # host arrays of asynchronous copies in flight

    @property
    def shape(self):
        return (self.p.ny, self.p.nx)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init_density(self, rho0: np.ndarray):
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
        assert rho0.shape == self.shape
        check(lbm_init_density(self.ctx, _host_ptr(rho0)), "lbm_init_density")
        self.stream.synchronize()   # rho0 is pageable host memory owned by this call

    def init_density_async(self, rho0: np.ndarray):
        """As init_density, with the host-to-device copy on the context's copy
        stream (no synchronisation).  rho0: C-contiguous float64 of the
        lattice shape, page-locked for the copy to overlap; it is held until
        wait_io and must not change before then."""
        assert rho0.shape == self.shape
        ptr = _host_ptr(rho0)
        self._io_refs.append(rho0)
        check(lbm_init_density_async(self.ctx, ptr), "lbm_init_density_async")

    def read_moments_async(self, out):
        """Queue a read of (rho, vx, vy) at the state reached by the work
        queued so far into out (three C-contiguous float64 arrays of the
        lattice shape, page-locked for overlap); they are filled once wait_io
        returns."""
        rho, vx, vy = out
        assert rho.shape == vx.shape == vy.shape == self.shape
        ptrs = [_host_ptr(a) for a in (rho, vx, vy)]
        self._io_refs.append(out)
        check(lbm_read_moments_async(self.ctx, *ptrs), "lbm_read_moments_async")

    def wait_io(self):
        """Wait for every asynchronous copy of this lattice."""
        check(lbm_wait_io(self.ctx), "lbm_wait_io")
        self._io_refs.clear()

    def init_density_dev(self, rho0_dev):
        check(lbm_init_density_dev(self.ctx, _vp(rho0_dev.data_ptr())), "lbm_init_density_dev")

    def init_preset(self, kind, size, width=4.0, rho_l=0.0, rho_v=0.0, cell=256, seed=0, noise_amp=1e-6):
        check(lbm_init_preset(self.ctx, PRESET[kind] if isinstance(kind, str) else int(kind), float(size),
                              float(width), float(rho_l), float(rho_v), int(cell), int(seed) & (2 ** 64 - 1),
                              float(noise_amp)), "lbm_init_preset")

    def step(self, n: int = 1):
        check(lbm_step(self.ctx, int(n)), "lbm_step")

    def stats(self, snapshot: bool = False) -> dict:
        s = lbm_stats_t()
        check(lbm_stats(self.ctx, int(bool(snapshot)), ctypes.byref(s)), "lbm_stats")
        return s.as_dict()

    def run_to_steady(self, tol, check_every=1000, max_steps=10 ** 6):
        done = _i64()
        st = lbm_run_to_steady(self.ctx, float(tol), int(check_every), int(max_steps), ctypes.byref(done))
        return st, done.value

    def read_moments(self, out=None):
        """(rho, vx, vy) at the current time; out: three C-contiguous float64
        arrays of the lattice shape to fill (e.g. pinned host memory)."""
        rho, vx, vy = out if out is not None else (np.empty(self.shape) for _ in range(3))
        check(lbm_read_moments(self.ctx, _host_ptr(rho), _host_ptr(vx), _host_ptr(vy)), "lbm_read_moments")
        return rho, vx, vy

    def read_populations(self) -> np.ndarray:
        f = np.empty((9,) + self.shape)
        check(lbm_read_populations(self.ctx, _host_ptr(f)), "lbm_read_populations")
        return f

    def write_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9,) + self.shape
        check(lbm_write_populations(self.ctx, _host_ptr(f)), "lbm_write_populations")

    def copy_rows(self, y0: int, buf, to_lattice: bool = False):
        """Stored rows [y0, y0 + buf.shape[1]) to (to_lattice False) or from
        (True) a contiguous CUDA tensor buf of shape (9, nrows, nx) in the
        storage type (float64 for FP64, float32 deviations for FP32), queued
        on the lattice's stream."""
        assert buf.is_cuda and buf.is_contiguous() and buf.dim() == 3 and buf.shape[0] == 9
        assert buf.shape[2] == self.shape[1]
        check(lbm_copy_rows(self.ctx, int(y0), int(buf.shape[1]), _vp(buf.data_ptr()), int(bool(to_lattice))),
              "lbm_copy_rows")

    def save(self, path):
        check(lbm_save(self.ctx, str(path).encode()), "lbm_save")

    def load(self, path):
        check(lbm_load(self.ctx, str(path).encode()), "lbm_load")

    @property
    def config(self) -> int:
        v = ctypes.c_int()
        check(lbm_get_config(self.ctx, ctypes.byref(v)), "lbm_get_config")
        return v.value

    @config.setter
    def config(self, v: int):
        check(lbm_set_config(self.ctx, int(v)), "lbm_set_config")

    def configs(self):
        """[(id, threads, stages, nodes_per_thread)] of every kernel configuration."""
        n = ctypes.c_int()
        check(lbm_config_count(ctypes.byref(self.p), ctypes.byref(n)), "lbm_config_count")
        out = []
        for i in range(n.value):
            t, s_, v = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            check(lbm_config_describe(ctypes.byref(self.p), i, ctypes.byref(t), ctypes.byref(s_), ctypes.byref(v)),
                  "lbm_config_describe")
            out.append((i, t.value, s_.value, v.value))
        return out

    def inject_stage_timeout(self):
        """The next step's staged kernels give up their first stage wait at
        once (the timeout path, for failure-detection tests)."""
        check(lbm_inject_stage_timeout(self.ctx), "lbm_inject_stage_timeout")

    def autotune(self, trial_steps: int = 20):
        """Time every kernel configuration on this lattice and keep the fastest;
        returns (config, ms_per_step).  The lattice state is not advanced."""
        cfg, ms = ctypes.c_int(), ctypes.c_double()
        check(lbm_autotune(self.ctx, int(trial_steps), ctypes.byref(cfg), ctypes.byref(ms)), "lbm_autotune")
        return cfg.value, ms.value

    @property
    def variant(self) -> int:
        v = ctypes.c_int()
        check(lbm_get_variant(self.ctx, ctypes.byref(v)), "lbm_get_variant")
        return v.value

    @variant.setter
    def variant(self, v: int):
        check(lbm_set_variant(self.ctx, int(v)), "lbm_set_variant")


class Batch:
    """Many independent lattices advanced together (FP32 deviations).

    instances: list of dicts with keys nx, ny (or side), kind, T_over_Tc, tau,
    A, K, size and optional width (4), rho_l / rho_v (0: Maxwell), cell, seed,
    noise_amp (1e-6)."""

    def __init__(self, instances, collision="bgk", forcing="guo", s_e=0.8, s_eps=0.8, s_q=1.1, sigma=0.0):
        bp = lbm_batch_params(COLLISION[collision], FORCING[forcing], FP32_DEV, 0, float(s_e), float(s_eps),
                              float(s_q), float(sigma))
        arr = (lbm_instance * len(instances))()
        for i, d in enumerate(instances):
            nx = int(d.get("nx", d.get("side")))
            ny = int(d.get("ny", d.get("side")))
            kind = d.get("kind", "droplet")
            arr[i] = lbm_instance(nx, ny, PRESET[kind] if isinstance(kind, str) else int(kind), int(d.get("cell", 256)),
                                  float(d["T_over_Tc"]), float(d["tau"]), float(d["A"]), float(d.get("K", 1.0)),
                                  float(d["size"]), float(d.get("width", 4.0)), float(d.get("rho_l", 0.0)),
                                  float(d.get("rho_v", 0.0)), float(d.get("noise_amp", 1e-6)),
                                  int(d.get("seed", 0)) & (2 ** 64 - 1))
        self.n = len(instances)
        self.shapes = [(arr[i].ny, arr[i].nx) for i in range(self.n)]
        h = _vp()
        check(lbm_batch_create(ctypes.byref(bp), arr, self.n, ctypes.byref(h)), "lbm_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def nodes(self) -> int:
        return int(lbm_batch_nodes(self.h))

    def init(self):
        """Every instance from its preset (f = w rho0)."""
        check(lbm_batch_init(self.h), "lbm_batch_init")

    def _geom(self, geom):
        """geom: n entries of (use, centre, spacing)."""
        arr = (lbm_profile_geom * self.n)()
        for i, (use, centre, spacing) in enumerate(geom):
            arr[i] = lbm_profile_geom(int(bool(use)), 0, float(centre), float(spacing))
        return arr

    def init_profiles(self, profiles, geom, rest=True):
        """Instances with use != 0 from radial density profiles: profiles is a
        torch CUDA float64 tensor [n, nb], geom n tuples (use, centre, spacing)
        placing sample k at |centre + spacing (k - (nb-1)/2)|; rest: start the
        populations at rest (v = 0) instead of f = w rho0."""
        assert profiles.is_cuda and profiles.dtype.itemsize == 8 and profiles.is_contiguous()
        check(lbm_batch_init_profiles(self.h, _vp(profiles.data_ptr()), int(profiles.shape[1]), self._geom(geom),
                                      LBM_INIT_REST if rest else 0), "lbm_batch_init_profiles")

    def step(self, n: int):
        check(lbm_batch_step(self.h, int(n)), "lbm_batch_step")

    def set_coex_rule(self, rule: str):
        """How tol_coex is judged: "change" (the probes' change per check) or
        "tail" (also their estimated change still to come)."""
        check(lbm_batch_set_coex_rule(self.h, COEX_RULES[rule]), "lbm_batch_set_coex_rule")

    def run_to_steady(self, tol_v=0.0, tol_rho=0.0, tol_coex=0.0, check_every=1000, max_steps=10 ** 6):
        done = _i64()
        st = lbm_batch_run_to_steady(self.h, float(tol_v), float(tol_rho), float(tol_coex), int(check_every),
                                     int(max_steps), ctypes.byref(done))
        return st, done.value

    def observe(self):
        check(lbm_batch_observe(self.h), "lbm_batch_observe")

    def results(self):
        state = np.zeros(self.n, dtype=np.int32)
        code = np.zeros(self.n, dtype=np.int32)
        steps = np.zeros(self.n, dtype=np.int64)
        obs = np.zeros((self.n, BATCH_NOBS))
        check(lbm_batch_results(self.h, state.ctypes.data_as(_vp), code.ctypes.data_as(_vp),
                                steps.ctypes.data_as(_vp), obs.ctypes.data_as(_vp)), "lbm_batch_results")
        return state, code, steps, {k: obs[:, i] for i, k in enumerate(BATCH_OBS)}

    def read_density(self, i: int) -> np.ndarray:
        rho = np.empty(self.shapes[i])
        check(lbm_batch_read_density(self.h, int(i), rho.ctypes.data_as(_vp)), "lbm_batch_read_density")
        return rho

    def profiles(self, nb, geom) -> np.ndarray:
        """Radial density profiles [n, nb] on the grids geom (n tuples
        (use, centre, spacing); use is ignored)."""
        out = np.empty((self.n, nb))
        check(lbm_batch_profiles(self.h, int(nb), self._geom(geom), out.ctypes.data_as(_vp)), "lbm_batch_profiles")
        return out

    def set_tuning(self, columns, stages, rows, carry=False):
        """Strip width of a work item (128: one warp; 256, 512: a CTA), row
        stages, rows per item, rows carried in registers."""
        check(lbm_batch_set_tuning(self.h, int(columns), int(stages), int(rows), int(bool(carry))),
              "lbm_batch_set_tuning")

    def autotune(self, trial_steps=10):
        """Time the tile shapes; returns (columns, stages, rows per item, carry, ms per step)."""
        w, a, b, c, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        check(lbm_batch_autotune(self.h, int(trial_steps), ctypes.byref(w), ctypes.byref(a), ctypes.byref(b),
                                 ctypes.byref(c), ctypes.byref(ms)), "lbm_batch_autotune")
        return w.value, a.value, b.value, bool(c.value), ms.value


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        assert a.shape == shape, (a.shape, shape)
    return a


class WarmStartNet:
    """The warm-start MLP (FP32, trained by liblbm's own kernels)."""

    def __init__(self, n_in=5, n_hidden=128, hidden_layers=3, n_out=64, seed=0):
        self.n_in, self.n_out = n_in, n_out
        self.sizes = [n_in] + [n_hidden] * hidden_layers + [n_out]
        h = _vp()
        check(lbm_ws_create(ctypes.byref(lbm_ws_cfg(n_in, n_hidden, hidden_layers, n_out, int(seed))),
                            ctypes.byref(h)), "lbm_ws_create")
        self.h = h
        n = _i64()
        check(lbm_ws_num_params(h, ctypes.byref(n)), "lbm_ws_num_params")
        self.n_params = n.value

    def close(self):
        if getattr(self, "h", None):
            lbm_ws_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scaling(self, x_mean, x_std, y_mean, y_std):
        args = [_f32(x_mean), _f32(x_std), _f32(y_mean), _f32(y_std)]
        check(lbm_ws_set_scaling(self.h, *[a.ctypes.data_as(_vp) for a in args]), "lbm_ws_set_scaling")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        check(lbm_ws_get_params(self.h, out.ctypes.data_as(_vp)), "lbm_ws_get_params")
        return out

    def set_params(self, theta):
        theta = _f32(theta, (self.n_params,))
        check(lbm_ws_set_params(self.h, theta.ctypes.data_as(_vp)), "lbm_ws_set_params")

    def loss_grad(self, X, Y):
        X, Y = _f32(X), _f32(Y)
        loss = ctypes.c_float()
        g = np.empty(self.n_params, dtype=np.float32)
        check(lbm_ws_loss_grad(self.h, X.ctypes.data_as(_vp), Y.ctypes.data_as(_vp), X.shape[0], ctypes.byref(loss),
                               g.ctypes.data_as(_vp)), "lbm_ws_loss_grad")
        return loss.value, g

    def train(self, X, Y, epochs, batch=256, lr=1e-3, seed=0):
        X, Y = _f32(X), _f32(Y)
        loss = ctypes.c_float()
        check(lbm_ws_train(self.h, X.ctypes.data_as(_vp), Y.ctypes.data_as(_vp), X.shape[0], int(epochs),
                           int(batch), float(lr), int(seed), ctypes.byref(loss)), "lbm_ws_train")
        return loss.value

    def predict(self, X) -> np.ndarray:
        X = _f32(X)
        out = np.empty((X.shape[0], self.n_out), dtype=np.float32)
        check(lbm_ws_predict(self.h, X.ctypes.data_as(_vp), X.shape[0], out.ctypes.data_as(_vp)), "lbm_ws_predict")
        return out
