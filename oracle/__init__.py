"""FP64 CPU oracle for the pseudo-potential D2Q9 LBM of arXiv:1412.5170.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The product library (``paper_1412_5170_gb300``) never imports it, and the
two share no code: the oracle is a plain C file (``lbm_oracle.c``) compiled
with gcc, plus the coexistence solvers in ``coexistence.py``.

The C file follows the paper's equations node by node (Eqs. 1-7, 20-23,
29-30, 34-36); see its header for the readings taken where the paper is
silent or garbled.  This module only marshals numpy arrays through ctypes.

Array layout: populations ``f[a, y, x]`` (shape ``(9, ny, nx)``, float64),
fields ``rho[y, x]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

BGK, MRT = 0, 1
GUO, EDM, SC, LI = 0, 1, 2, 3
_COLL = {"bgk": BGK, "mrt": MRT}
_FORC = {"guo": GUO, "edm": EDM, "sc": SC, "li": LI}

OK, E_INVALID, E_NONFINITE, E_EOS_DOMAIN = 0, 1, 3, 4


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into liboracle.so (plain gcc, no FMA contraction).

    If ORACLE_SO is set, that prebuilt library is used instead (the mutation
    test points it at deliberately broken copies of the oracle)."""
    if os.environ.get("ORACLE_SO"):
        return os.environ["ORACLE_SO"]
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:   # OpenMP over rows for the multi-core CPU baseline; plain if the compiler lacks it
            subprocess.check_call(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("collision", ctypes.c_int32), ("forcing", ctypes.c_int32),
                ("T_over_Tc", ctypes.c_double), ("tau", ctypes.c_double),
                ("A", ctypes.c_double), ("K", ctypes.c_double),
                ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
                ("sigma", ctypes.c_double)]


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(Params)
        lib.orc_Tc.restype = ctypes.c_double
        lib.orc_pressure.restype = ctypes.c_double
        lib.orc_pressure.argtypes = [ctypes.c_double] * 3
        lib.orc_psi2.restype = ctypes.c_double
        lib.orc_psi2.argtypes = [ctypes.c_double] * 3
        lib.orc_feq.argtypes = [ctypes.c_double] * 3 + [dp]
        lib.orc_guo_source.argtypes = [ctypes.c_double] * 5 + [dp]
        lib.orc_force.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, dp, dp]
        lib.orc_mrt_matrix.argtypes = [dp]
        lib.orc_invert9.argtypes = [dp, dp]
        lib.orc_collide_node.argtypes = [pp, dp] + [ctypes.c_double] * 6 + [dp]
        lib.orc_macro.argtypes = [pp, dp] + [dp] * 8
        lib.orc_step.argtypes = [pp, dp, dp]
        lib.orc_run.argtypes = [pp, dp, ctypes.c_int64]
        lib.orc_init_rest.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_get_threads.restype = ctypes.c_int
        _lib_handle = lib
    return _lib_handle


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params(nx, ny, T_over_Tc, tau, A, K=1.0, collision="bgk", forcing="guo",
           s_e=1.0, s_eps=1.0, s_q=1.0, sigma=0.0) -> Params:
    return Params(int(nx), int(ny), _COLL[collision], _FORC[forcing], float(T_over_Tc),
                  float(tau), float(A), float(K), float(s_e), float(s_eps), float(s_q), float(sigma))


def set_threads(n: int) -> None:
    """Host threads of the lattice loops (1 by default; results are the same
    bit for bit for any count)."""
    _lib().orc_set_threads(int(n))


def get_threads() -> int:
    return _lib().orc_get_threads()


# ---- thermodynamics (Sec. 4.1, Eqs. 7, 29, 30) ----

def Tc() -> float:
    return _lib().orc_Tc()


def pressure(rho: float, T: float, K: float = 1.0) -> float:
    return _lib().orc_pressure(float(rho), float(T), float(K))


def psi2(rho: float, T: float, K: float = 1.0) -> float:
    return _lib().orc_psi2(float(rho), float(T), float(K))


# ---- node-level pieces ----

def feq(rho, ux, uy) -> np.ndarray:
    out = np.zeros(9)
    _lib().orc_feq(float(rho), float(ux), float(uy), _ptr(out))
    return out


def guo_source(prefactor, Fx, Fy, vx, vy) -> np.ndarray:
    out = np.zeros(9)
    _lib().orc_guo_source(float(prefactor), float(Fx), float(Fy), float(vx), float(vy), _ptr(out))
    return out


def mrt_matrix() -> np.ndarray:
    M = np.zeros(81)
    _lib().orc_mrt_matrix(_ptr(M))
    return M.reshape(9, 9)


def invert9(M: np.ndarray) -> np.ndarray:
    Min = np.ascontiguousarray(M, dtype=np.float64).reshape(81)
    out = np.zeros(81)
    if _lib().orc_invert9(_ptr(Min), _ptr(out)) != 0:
        raise ValueError("singular matrix")
    return out.reshape(9, 9)


def collide_node(p: Params, f9, rho, ux, uy, Fx, Fy, psi=0.0) -> np.ndarray:
    f9 = np.ascontiguousarray(f9, dtype=np.float64)
    out = np.zeros(9)
    _lib().orc_collide_node(ctypes.byref(p), _ptr(f9), float(rho), float(ux), float(uy),
                            float(Fx), float(Fy), float(psi), _ptr(out))
    return out


def force(psi: np.ndarray, A: float):
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    ny, nx = psi.shape
    Fx = np.zeros_like(psi)
    Fy = np.zeros_like(psi)
    _lib().orc_force(nx, ny, _ptr(psi), float(A), _ptr(Fx), _ptr(Fy))
    return Fx, Fy


# ---- lattice-level ----

def init_rest(rho0: np.ndarray) -> np.ndarray:
    """f_a = w_a rho0 (equilibrium at rest)."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    ny, nx = rho0.shape
    f = np.zeros((9, ny, nx))
    _lib().orc_init_rest(nx, ny, _ptr(rho0), _ptr(f))
    return f


def macro(p: Params, f: np.ndarray):
    """Fields at time t from the post-streaming populations: returns (dict, status)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    shape = (p.ny, p.nx)
    names = ("rho", "ux", "uy", "psi", "Fx", "Fy", "vx", "vy")
    out = {k: np.zeros(shape) for k in names}
    st = _lib().orc_macro(ctypes.byref(p), _ptr(f), *[_ptr(out[k]) for k in names])
    return out, st


def step(p: Params, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    st = _lib().orc_step(ctypes.byref(p), _ptr(f), _ptr(out))
    return out, st


def run(p: Params, f: np.ndarray, nsteps: int):
    """nsteps steps; returns (f, status).  The input array is not modified."""
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    st = _lib().orc_run(ctypes.byref(p), _ptr(g), int(nsteps))
    return g, st
