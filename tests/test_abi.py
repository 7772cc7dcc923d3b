"""The C-ABI library loads and exports every function include/lbm.h declares,
and its host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(lbm_[a-z_0-9]+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1412_5170_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def declared_prototypes():
    """{name: number of parameters} of every function include/*.h declares."""
    out = {}
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for name, args in re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(lbm_[a-z_0-9]+)\s*\(([^;]*?)\)\s*;",
                                         text, flags=re.M | re.S):
                args = args.strip()
                out[name] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_declares_every_function_with_its_arity(lbm):
    """The Python binding carries the same names as the C ABI, each with as
    many ctypes argument types as the header's prototype has parameters."""
    protos = declared_prototypes()
    assert set(protos) == set(declared_functions())
    assert set(lbm._PROTOS) == set(protos)
    wrong = {n: (k, len(lbm._PROTOS[n][1])) for n, k in protos.items() if len(lbm._PROTOS[n][1]) != k}
    assert not wrong, wrong


def test_strerror_and_version(lbm):
    assert lbm.lbm_strerror(0) == b"ok"
    assert b"converged" in lbm.lbm_strerror(lbm.E_NOT_CONVERGED)
    assert lbm.lbm_version() >> 16 == 1


def test_library_maxwell_matches_oracle(lbm, orc):
    """The library's own host Maxwell solver (equal pressure and chemical
    potential) against the oracle's equal-area quadrature (Eq. 19)."""
    from oracle import coexistence as cx
    for tr in (0.5, 0.6, 0.7, 0.8, 0.9):
        rv, rl = lbm.maxwell(tr)
        g, l, _ = cx.maxwell(tr)
        assert rv == pytest.approx(g, rel=1e-9)
        assert rl == pytest.approx(l, rel=1e-9)
    assert lbm.tc() == orc.Tc()


def test_invalid_parameters_are_rejected(lbm):
    base = dict(nx=16, ny=16, T_over_Tc=0.7, tau=0.8, A=-0.3)
    bad = [dict(tau=0.5), dict(T_over_Tc=1.0), dict(T_over_Tc=0.0), dict(K=0.0), dict(nx=0)]
    for b in bad:
        kw = dict(base, **b)
        p = lbm.make_params(kw.pop("nx"), kw.pop("ny"), **kw)
        n = ctypes.c_size_t()
        assert lbm.lbm_workspace_bytes(ctypes.byref(p), ctypes.byref(n)) == lbm.E_INVALID, b
    p = lbm.make_params(16, 16, 0.7, 0.8, -0.3, collision="mrt", forcing="edm")
    n = ctypes.c_size_t()
    assert lbm.lbm_workspace_bytes(ctypes.byref(p), ctypes.byref(n)) == lbm.E_UNSUPPORTED
    p = lbm.make_params(16, 16, 0.7, 0.8, -0.3, collision="mrt", s_e=2.5)
    assert lbm.lbm_workspace_bytes(ctypes.byref(p), ctypes.byref(n)) == lbm.E_INVALID
    assert lbm.lbm_maxwell(1.2, None, None) == lbm.E_INVALID


@pytest.mark.parametrize("tr,K,eps", [(0.8, 1.0, 0.52), (0.6, 1.0, 1.68), (0.6, 0.1, 2.0), (0.7, 0.5, 1.68),
                                      (0.9, 1.0, 1.0), (0.55, 0.25, 1.68)])
def test_library_mechanical_solution_matches_oracle(lbm, orc, tr, K, eps):
    """The library's Eq. 18 solver (bisection + Gauss-Legendre in log rho)
    against the oracle's (scipy brentq + adaptive quad, finite-difference
    psi'): independent codes, same densities."""
    from oracle import coexistence as cx
    rv, rl = lbm.mechanical(tr, K, eps)
    g, l, _ = cx.mechanical(tr, K, eps)
    assert rv == pytest.approx(g, rel=1e-6)
    assert rl == pytest.approx(l, rel=1e-8)
